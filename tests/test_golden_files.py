"""The stored circuit-level oracle outputs (tests/golden/*.json, written by make_circuit_golden.py)
reproduce from the oracle: a few cheap shots of each file (BP-resolved ones, which stop after a few
members) are decoded again here and must equal the stored values, and the stored inputs' digests
match a fresh run of the seeded generators."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import circuit as C
from paper_2508_15743_gb300 import dem as D

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = sorted(f for f in os.listdir(GOLDEN) if f.startswith("circuit_") and f.endswith(".json"))


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def test_generator_lists_every_file():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(GOLDEN, "make_circuit_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert {f[:-5] for f in FILES} <= set(mk.CASES)


@pytest.mark.parametrize("name", FILES)
def test_stored_values_reproduce(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    pr, dc, sh = g["problem"], g["decoder"], g["shots"]
    dm = C.circuit_dem(pr["d"], pr["rounds"], pr["p"], noise=pr["noise"], basis=pr["basis"])
    syn, _ = D.sample(dm, sh["count"], sh["seed"])
    perms = D.schedules(dm.n, dc["K"], int(dc["schedules"].split(",")[-1].strip(" )")))
    assert digest(syn) == sh["syndrome_sha256"]
    assert digest(perms) == sh["schedule_sha256"]
    st = g["stats"]
    # the two BP-resolved shots that stopped earliest
    cand = [i for i in range(len(g["rows"])) if not st["lsd_invoked"][i]]
    if not cand:
        pytest.skip("no BP-resolved shot in this file")
    pick = sorted(cand, key=lambda i: st["iters"][i])[:2]
    rows = [g["rows"][i] for i in pick]
    mode = {"fp32": oracle.FP32, "fp16": oracle.FP16MSG}[dc["mode"]]
    r = oracle.decode(dm, perms, syn[rows], dc["T"], dc["alpha"], dc["M"], lsd_order=dc["lsd_order"], mode=mode,
                      nthreads=2, want_soft=True)
    e = D.unpack_bits(r["corrections"], dm.n)
    for j, i in enumerate(pick):
        assert np.nonzero(e[j])[0].tolist() == g["corrections"][i]
        assert r["logical"][j].tolist() == g["logical"][i]
        for f in r["stats"].dtype.names:
            assert int(r["stats"][f][j]) == st[f][i]
        assert digest(r["soft"][j].astype(np.float32)) == g["soft_sha256"][i]
