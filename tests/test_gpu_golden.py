"""Circuit-level parity at the full decoder settings, against stored oracle outputs.

The oracle needs minutes per LSD-bound shot at these sizes, so `tests/golden/make_circuit_golden.py`
(CPU oracle only) decoded the shots once and stored the results beside itself. Here the GPU decodes
the same seeded shots -- the test first checks that it regenerated the same syndromes and schedules
(SHA-256) -- and every shot must match the stored values element by element: the correction (as its
set-bit indices), the logical words, every per-shot record field, and the float32 soft output (the
chosen member's posterior, or the averaged LLR vector handed to LSD), compared through a SHA-256 of
its bytes: equal digests mean every one of the n floats is equal.

Cases: config 3's problem and decoder (d=11 colour code, 11 rounds, Si1000 p = 1e-3, K=64, T=50, M=5)
with FP32 messages and LSD-0, FP16 messages and LSD-0, and FP32 messages with LSD order 5 on the
shots that reach LSD; the d=13 problem of the mixed-distance family (K=32, T=50, M=7, FP16); and its
d=15 problem with its decoder (p = 2e-3, K=32, T=20, M=7, FP16).
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2508_15743_gb300 import circuit as C
from paper_2508_15743_gb300 import dem as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = ["circuit_d11_k64_t50_fp32_lsd0", "circuit_d11_k64_t50_fp16_lsd0", "circuit_d11_k64_t50_fp32_lsd5",
         "circuit_d13_k32_t50_fp16_lsd0", "circuit_d15_k32_t20_fp16_lsd0"]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_15743_gb300 import build
    build.build_library()
    from paper_2508_15743_gb300 import vibe
    return vibe


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("case", CASES)
def test_matches_stored_oracle_outputs(V, case):
    path = os.path.join(GOLDEN, case + ".json")
    if not os.path.exists(path):
        pytest.skip(f"{case}.json not generated")
    with open(path) as f:
        g = json.load(f)
    pr, dc, sh = g["problem"], g["decoder"], g["shots"]
    dm = C.circuit_dem(pr["d"], pr["rounds"], pr["p"], noise=pr["noise"], basis=pr["basis"])
    assert (dm.m, dm.n, len(dm.H.colidx)) == (pr["m"], pr["n"], pr["E"])
    syn, _ = D.sample(dm, sh["count"], sh["seed"])
    sched_seed = int(dc["schedules"].split(",")[-1].strip(" )"))
    perms = D.schedules(dm.n, dc["K"], sched_seed)
    assert digest(syn) == sh["syndrome_sha256"], "regenerated syndromes differ from the stored inputs"
    assert digest(perms) == sh["schedule_sha256"], "regenerated schedules differ from the stored inputs"
    rows = np.asarray(g["rows"], dtype=np.int64)
    dec = V.Decoder(dm, dc["K"], perms, T=dc["T"], alpha=dc["alpha"], M=dc["M"], lsd_order=dc["lsd_order"],
                    msg_fp16=dc["mode"] == "fp16")
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn[rows]).view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    corr = D.unpack_bits(out["corrections"].cpu().numpy().view(np.uint32), dm.n)
    logical = out["logical"].cpu().numpy().view(np.uint32)
    st = V.stats_to_numpy(out["stats"])
    soft = out["soft"].cpu().numpy()
    dec.close()
    lsd = int(np.sum(g["stats"]["lsd_invoked"]))
    assert len(rows) >= 60 and (dc["lsd_order"] > 0 or lsd >= 30)
    for i in range(len(rows)):
        assert np.nonzero(corr[i])[0].tolist() == g["corrections"][i], f"shot {rows[i]}: correction"
        assert logical[i].tolist() == g["logical"][i], f"shot {rows[i]}: logical"
        for f in st.dtype.names:
            assert int(st[f][i]) == g["stats"][f][i], f"shot {rows[i]}: stats.{f}"
        assert digest(soft[i].astype(np.float32)) == g["soft_sha256"][i], f"shot {rows[i]}: soft output"
