"""Named single-decode cases for kernel profiling (ncu captures) and quick timing.

    python -m paper_2508_15743_gb300.cases <case> [--shots B]

runs one warm-up decode of 64 shots, then one decode of the case's batch, and prints one JSON line
with the device counters (shots, BP sweeps, LSD shots, rescans) and the kernel times.

    python -m paper_2508_15743_gb300.cases <case> --precisions [--shots B]

decodes the same shots with FP32 and FP16 message storage and reports both throughputs, logical
error rates with 2-sigma binomial intervals and the fraction of differing corrections.

    python -m paper_2508_15743_gb300.cases <image-engine case> --ensembles [--shots B]

decodes the same shots (FP32) with the serial ensemble, with its first members on the parallel
(flooding) schedule, with members differing in the scaling factor, and with both, reporting the
same figures against the serial ensemble. Inputs are seeded and synthetic; the bench workload's
numbers come from bench.py.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import circuit as C
from . import dem as D

# name -> (DEM builder, K, T, M, msg_fp16, engine, default shots, sampling seed)
CASES = {
    # the bench workload (d=9 phenomenological, K=16) on a batch small enough for a full ncu capture
    "image_pheno_d9": (lambda: D.build_workload("cc666_d9_pheno"), 16, 30, 5, False, 1, 20_000, 2),
    "image_pheno_d9_fp16": (lambda: D.build_workload("cc666_d9_pheno"), 16, 30, 5, True, 1, 20_000, 2),
    # circuit-level d=9 colour code on the summary engine, short ensemble
    "summary_circuit_d9": (lambda: C.circuit_dem(9, 9, 0.001, noise="si1000", basis="X"), 8, 10, 3, False, 2,
                           1216, 5),
    # circuit-level d=9 at p = 3e-3 with the config-4 ensemble (K=32, T=50): enough logical failures
    # in 2e4 shots to compare precisions
    "summary_circuit_d9_p3": (lambda: C.circuit_dem(9, 9, 0.003, noise="si1000", basis="X"), 32, 50, 5, False,
                              2, 20_000, 4),
    # XYZ colour-code circuit (X, Y and Z plaquette measurements in turn), d=7, 7 rounds, K=16
    "summary_circuit_xyz_d7": (lambda: C.circuit_dem(7, 7, 0.001, noise="si1000", basis="X", schedule="xyz"), 16, 30,
                               5, False, 2, 4000, 6),
    # circuit-level d=11, the full ensemble (K=64, T=50)
    "summary_circuit_d11": (lambda: C.circuit_dem(11, 11, 0.001, noise="si1000", basis="X"), 64, 50, 5, False, 2,
                            2432, 3),
}


def run_case(name: str, shots: int = 0) -> dict:
    import torch

    from . import vibe as V

    build, K, T, M, fp16, engine, default_shots, seed = CASES[name]
    dm = build()
    B = shots or default_shots
    dec = V.Decoder(dm, K, D.schedules(dm.n, K, seed), T=T, M=M, msg_fp16=fp16, engine=engine)
    syn, obs = D.sample(dm, B, seed)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    dec.decode(syn_t[:64])
    torch.cuda.synchronize()
    cnt = torch.zeros(V.VIBE_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    dec.profile(True)
    dec.decode(syn_t, counters=cnt)
    torch.cuda.synchronize()
    prof = dec.profile_read()
    c = cnt.cpu().numpy()
    dec.close()
    return dict(case=name, shots=int(c[V.CNT_SHOTS]), sweeps=int(c[V.CNT_PAIR_ITERS]), lsd=int(c[V.CNT_LSD]),
                rescans=int(c[V.CNT_RESCANS]), bp_ms=prof["bp_ms"], lsd_ms=prof["lsd_ms"], n=dm.n, m=dm.m,
                E=int(len(dm.H.colidx)))


def _ler(fails: int, shots: int) -> dict:
    p = fails / shots
    half = 2.0 * np.sqrt(max(p * (1.0 - p), 1.0 / shots) / shots)
    return dict(ler=p, two_sigma=[max(p - half, 0.0), p + half], failures=int(fails), shots=int(shots))


def compare_precisions(name: str, shots: int = 0) -> dict:
    """Decodes the same shots with FP32 and with FP16 message storage: throughput of each, logical
    error rates with 2-sigma binomial intervals, and the fraction of shots whose correction differs."""
    import time

    import torch

    from . import vibe as V

    build, K, T, M, _, engine, default_shots, seed = CASES[name]
    dm = build()
    B = shots or default_shots
    syn, obs = D.sample(dm, B, seed)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    obs_t = torch.from_numpy(obs.view(np.int32)).cuda()
    out, res = {}, {}
    for fp16 in (False, True):
        dec = V.Decoder(dm, K, D.schedules(dm.n, K, seed), T=T, M=M, msg_fp16=fp16, engine=engine)
        dec.decode(syn_t[:64])
        torch.cuda.synchronize()
        cnt = torch.zeros(V.VIBE_NUM_COUNTERS, dtype=torch.int64, device="cuda")
        t0 = time.perf_counter()
        o = dec.decode(syn_t, observables=obs_t, counters=cnt)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c = cnt.cpu().numpy()
        key = "fp16" if fp16 else "fp32"
        out[key] = o["corrections"].cpu().numpy()
        res[key] = dict(shots_per_s=B / dt, ler=_ler(int(c[V.CNT_FAILURES]), B), lsd_fraction=float(c[V.CNT_LSD]) / B,
                        sweeps_per_shot=float(c[V.CNT_PAIR_ITERS]) / B)
        dec.close()
    res["corrections_differ"] = float((out["fp32"] != out["fp16"]).any(axis=1).mean())
    res["fp16_ler_inside_fp32_interval"] = bool(
        res["fp32"]["ler"]["two_sigma"][0] <= res["fp16"]["ler"]["ler"] <= res["fp32"]["ler"]["two_sigma"][1])
    res.update(case=name, shots=B, n=dm.n, m=dm.m, K=K, T=T, M=M)
    return res


# scaling factors of a mixed-heuristic ensemble of 16 members (member i takes entry i)
ALPHA_MIX16 = [0.5, 0.625, 0.75, 1.0, 0.875, 0.5625, 0.6875, 0.8125] * 2

# name -> (members on the flooding schedule, per-member factors or None)
ENSEMBLES = {
    "serial": (0, None),
    "flood4": (4, None),
    "alpha_mix": (0, ALPHA_MIX16),
    "flood4_alpha_mix": (4, ALPHA_MIX16),
    "flood_all": (-1, None),
}


def compare_ensembles(name: str, shots: int = 0) -> dict:
    """Decodes the same shots (FP32 messages) with each ensemble of ENSEMBLES: throughput, logical
    error rate with its 2-sigma binomial interval, LSD fraction, sweeps per shot and the fraction of
    corrections that differ from the serial ensemble's."""
    import time

    import torch

    from . import vibe as V

    build, K, T, M, _, engine, default_shots, seed = CASES[name]
    if engine != 1 or K != len(ALPHA_MIX16):
        raise ValueError("ensemble comparisons run on the 16-member image-engine cases")
    dm = build()
    B = shots or default_shots
    syn, obs = D.sample(dm, B, seed)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    obs_t = torch.from_numpy(obs.view(np.int32)).cuda()
    perms = D.schedules(dm.n, K, seed)
    res, base = {}, None
    for label, (n_flood, alphas) in ENSEMBLES.items():
        dec = V.Decoder(dm, K, perms, T=T, M=M, engine=engine, n_flood=K if n_flood < 0 else n_flood,
                        member_alpha=alphas)
        dec.decode(syn_t[:64])
        torch.cuda.synchronize()
        cnt = torch.zeros(V.VIBE_NUM_COUNTERS, dtype=torch.int64, device="cuda")
        t0 = time.perf_counter()
        o = dec.decode(syn_t, observables=obs_t, counters=cnt)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c = cnt.cpu().numpy()
        corr = o["corrections"].cpu().numpy()
        if base is None:
            base = corr
        res[label] = dict(shots_per_s=B / dt, ler=_ler(int(c[V.CNT_FAILURES]), B),
                          lsd_fraction=float(c[V.CNT_LSD]) / B, sweeps_per_shot=float(c[V.CNT_PAIR_ITERS]) / B,
                          corrections_differ_from_serial=float((corr != base).any(axis=1).mean()))
        dec.close()
    res.update(case=name, shots=B, n=dm.n, m=dm.m, K=K, T=T, M=M)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--shots", type=int, default=0)
    ap.add_argument("--precisions", action="store_true", help="compare FP32 and FP16 message storage")
    ap.add_argument("--ensembles", action="store_true", help="compare serial, flooding and mixed-alpha ensembles")
    args = ap.parse_args()
    if args.ensembles:
        print(json.dumps(compare_ensembles(args.case, args.shots)))
    elif args.precisions:
        print(json.dumps(compare_precisions(args.case, args.shots)))
    else:
        print(json.dumps(run_case(args.case, args.shots)))


if __name__ == "__main__":
    main()
