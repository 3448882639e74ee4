"""Named single-decode cases for kernel profiling (ncu captures) and quick timing.

    python -m paper_2508_15743_gb300.cases <case> [--shots B]

runs one warm-up decode of 64 shots, then one decode of the case's batch, and prints one JSON line
with the device counters (shots, BP sweeps, LSD shots, rescans) and the kernel times. Inputs are
seeded and synthetic; nothing here is timed for reporting (bench.py does that).
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--shots", type=int, default=0)
    args = ap.parse_args()
    print(json.dumps(run_case(args.case, args.shots)))


if __name__ == "__main__":
    main()
