"""GPU parity of ensembles whose members differ in the min-sum scaling factor (reading R9).

Member i scales its check-to-variable messages by its own factor; both BP engines, FP32 and FP16
storage, and flooding members on the image engine must match the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import circuit as C
from paper_2508_15743_gb300 import dem as D

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHAS16 = np.array([0.5, 0.625, 0.75, 1.0, 0.875, 0.5625, 0.6875, 0.8125] * 2, np.float32)


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_15743_gb300 import build
    build.build_library()
    from paper_2508_15743_gb300 import vibe
    return vibe


def _check(V, dm, perms, syn, T, M, engine, fp16, n_flood, alphas):
    dec = V.Decoder(dm, perms.shape[0], perms, T=T, alpha=0.625, M=M, msg_fp16=fp16, engine=engine,
                    n_flood=n_flood, member_alpha=alphas)
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    mode = oracle.FP16MSG if fp16 else oracle.FP32
    r = oracle.decode(dm, perms, syn, T, 0.625, M, mode=mode, nthreads=8, n_flood=n_flood, member_alpha=alphas)
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    st = V.stats_to_numpy(out["stats"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    dec.close()
    return st


@pytest.mark.parametrize("engine,fp16,n_flood", [(1, False, 0), (1, True, 0), (1, False, 4), (2, False, 0),
                                                 (2, True, 0)])
def test_member_alphas_match_oracle_pheno_d9(V, engine, fp16, n_flood):
    dm = D.build_workload("cc666_d9_pheno")
    syn, _ = D.sample(dm, 1000, 41)
    perms = D.schedules(dm.n, 16, 6)
    st = _check(V, dm, perms, syn, 30, 5, engine, fp16, n_flood, ALPHAS16)
    chosen = st["chosen_member"][st["lsd_invoked"] == 0]
    assert len(np.unique(ALPHAS16[chosen])) >= 4   # members with several factors were kept


def test_member_alphas_match_oracle_circuit_d5(V):
    dm = C.circuit_dem(5, 5, 0.004, noise="si1000", basis="X")
    syn, _ = D.sample(dm, 200, 42)
    perms = D.schedules(dm.n, 6, 7)
    _check(V, dm, perms, syn, 12, 3, 2, False, 0, np.array([1.0, 0.5, 0.625, 0.75, 0.9, 0.55], np.float32))
