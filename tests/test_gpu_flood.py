"""GPU parity of flooding members (Algorithm 1's parallel schedule, reading R8) in the image engine.

An ensemble whose first n_flood members run the parallel schedule and the rest serial schedules
must match the oracle bit for bit: corrections, logical flips, per-shot records, posteriors.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_15743_gb300 import build
    build.build_library()
    from paper_2508_15743_gb300 import vibe
    return vibe


@pytest.mark.parametrize("name,shots,K,M,n_flood", [("cc666_d5_codecap", 3000, 1, 1, 1),
                                                    ("cc666_d9_pheno", 1500, 16, 5, 4)])
def test_flooding_members_match_oracle(V, name, shots, K, M, n_flood):
    w = D.WORKLOADS[name]
    dm = D.build_workload(name)
    syn, obs = D.sample(dm, shots, 31)
    perms = D.schedules(dm.n, K, 5, natural=(K == 1))
    dec = V.Decoder(dm, K, perms, T=w["T"], alpha=w["alpha"], M=M, n_flood=n_flood)
    out = dec.decode(torch.from_numpy(syn.view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], M, nthreads=8, n_flood=n_flood)
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    assert np.array_equal(out["logical"].cpu().numpy().view(np.uint32), r["logical"])
    st = V.stats_to_numpy(out["stats"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    if n_flood < K:   # the instance must pick flooding and serial members both
        chosen = st["chosen_member"][st["lsd_invoked"] == 0]
        assert (chosen < n_flood).any() and (chosen >= n_flood).any()
    dec.close()
