"""Writes the stored oracle outputs of the circuit-level parity tests (tests/test_gpu_golden.py).

The oracle needs minutes per LSD-bound shot at these sizes (one member sweep of the d=11 problem scans
~2e7 row entries, and an LSD-bound shot runs K x T of them), so the expected values are computed once
here and stored as JSON beside this script. Only the CPU oracle (`oracle/`) and the seeded input
generators (`paper_2508_15743_gb300.dem`, `.circuit`, which hold none of the decoder's arithmetic)
are called; nothing here touches the CUDA library.

Cases (each a JSON file named after it):

* circuit_d11_k64_t50_fp32_lsd0 -- config 3's problem and decoder: colour code d=11, 11 rounds,
  Si1000 noise at p = 1e-3 (X memory), K=64 seeded serial schedules, T=50, M=5, alpha=0.625,
  LSD-0, FP32 messages; 128 seeded shots.
* circuit_d11_k64_t50_fp16_lsd0 -- the same shots with FP16 message storage.
* circuit_d11_k64_t50_fp32_lsd5 -- the same decoder with LSD order 5, on the shots of the FP32 run
  that reached LSD.
* circuit_d13_k32_t50_fp16_lsd0 -- the d=13 member of the mixed-distance family (p = 1e-3, the
  problem the streaming workload also serves): K=32, T=50, M=7 (the larger correction limit at
  higher distance, Sec. III.D.2 step 3), FP16 messages, LSD-0; 128 seeded shots.
* circuit_d15_k32_t20_fp16_lsd0 -- the largest problem of the mixed-distance family with its decoder
  (d=15, p = 2e-3, K=32, T=20, M=7, FP16 messages, LSD-0); 128 seeded shots.

Each file records the problem, the decoder parameters, the seeds, a SHA-256 of the syndromes (so the
GPU test can confirm it regenerated the same inputs), and per shot: the correction as its set-bit
indices, the logical words, every per-shot record field, and a SHA-256 of the float32 soft output
(the chosen member's posterior, or the averaged vector handed to LSD), which the GPU test compares
with the digest of its own soft output -- equal digests mean every element is equal.

Usage: python tests/golden/make_circuit_golden.py [case ...]   (all cases by default)
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2508_15743_gb300 import circuit as C  # noqa: E402
from paper_2508_15743_gb300 import dem as D  # noqa: E402

CASES = {
    "circuit_d11_k64_t50_fp32_lsd0": dict(d=11, p=1e-3, K=64, T=50, M=5, lsd_order=0, mode="fp32",
                                          shots=128, shot_seed=3, sched_seed=3),
    "circuit_d11_k64_t50_fp16_lsd0": dict(d=11, p=1e-3, K=64, T=50, M=5, lsd_order=0, mode="fp16",
                                          shots=128, shot_seed=3, sched_seed=3),
    "circuit_d11_k64_t50_fp32_lsd5": dict(d=11, p=1e-3, K=64, T=50, M=5, lsd_order=5, mode="fp32",
                                          shots=128, shot_seed=3, sched_seed=3,
                                          rows_from="circuit_d11_k64_t50_fp32_lsd0"),
    "circuit_d13_k32_t50_fp16_lsd0": dict(d=13, p=1e-3, K=32, T=50, M=7, lsd_order=0, mode="fp16",
                                          shots=128, shot_seed=13, sched_seed=113),
    "circuit_d15_k32_t20_fp16_lsd0": dict(d=15, p=2e-3, K=32, T=20, M=7, lsd_order=0, mode="fp16",
                                          shots=128, shot_seed=15, sched_seed=115),
}
MODES = {"fp32": oracle.FP32, "fp16": oracle.FP16MSG}
ALPHA = 0.625


def problem(cfg):
    return C.circuit_dem(cfg["d"], cfg["d"], cfg["p"], noise="si1000", basis="X")


def inputs(cfg, dm):
    syn, obs = D.sample(dm, cfg["shots"], cfg["shot_seed"])
    perms = D.schedules(dm.n, cfg["K"], cfg["sched_seed"])
    return syn, obs, perms


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make(name, nthreads):
    cfg = CASES[name]
    dm = problem(cfg)
    syn, obs, perms = inputs(cfg, dm)
    if "rows_from" in cfg:
        with open(os.path.join(HERE, cfg["rows_from"] + ".json")) as f:
            base = json.load(f)
        rows = [r for r, lsd in zip(base["rows"], base["stats"]["lsd_invoked"]) if lsd]
    else:
        rows = list(range(cfg["shots"]))
    t0 = time.time()
    r = oracle.decode(dm, perms, syn[rows], cfg["T"], ALPHA, cfg["M"], lsd_order=cfg["lsd_order"],
                      mode=MODES[cfg["mode"]], nthreads=nthreads, want_soft=True)
    secs = time.time() - t0
    e = D.unpack_bits(r["corrections"], dm.n)
    st = r["stats"]
    out = dict(
        case=name,
        generator="tests/golden/make_circuit_golden.py (CPU oracle only)",
        problem=dict(kind="circuit_dem", d=cfg["d"], rounds=cfg["d"], p=cfg["p"], noise="si1000", basis="X",
                     m=int(dm.m), n=int(dm.n), E=int(len(dm.H.colidx)), k=int(dm.k)),
        decoder=dict(K=cfg["K"], T=cfg["T"], M=cfg["M"], alpha=ALPHA, lsd_order=cfg["lsd_order"],
                     mode=cfg["mode"], schedules="dem.schedules(n, K, %d)" % cfg["sched_seed"]),
        shots=dict(count=cfg["shots"], seed=cfg["shot_seed"], sampler="dem.sample(dm, count, seed)",
                   syndrome_sha256=digest(syn), schedule_sha256=digest(perms)),
        oracle_seconds=round(secs, 1), oracle_threads=nthreads,
        rows=rows,
        corrections=[np.nonzero(e[i])[0].tolist() for i in range(len(rows))],
        logical=r["logical"].tolist(),
        stats={f: st[f].tolist() for f in st.dtype.names},
        soft_sha256=[digest(r["soft"][i].astype(np.float32)) for i in range(len(rows))],
    )
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    lsd = int(np.sum(st["lsd_invoked"]))
    print(f"{name}: {len(rows)} shots ({lsd} on the LSD path) in {secs:.0f} s", flush=True)


def main(argv):
    names = argv or list(CASES)
    nthreads = os.cpu_count() or 1
    for name in names:
        make(name, nthreads)


if __name__ == "__main__":
    main(sys.argv[1:])
