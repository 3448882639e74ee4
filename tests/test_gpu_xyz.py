"""GPU parity on the XYZ colour-code workload (circuit-level DEMs whose detectors span X, Y and Z
outcomes of three rounds): both BP engines, FP32 and FP16 storage, bit-exact with the oracle,
including the LSD-decided shots."""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import circuit as C
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


@pytest.mark.parametrize("d,rounds,engine,fp16", [(3, 4, 1, False), (3, 4, 2, False), (5, 5, 2, False),
                                                  (5, 5, 2, True), (5, 5, 1, False)])
def test_xyz_matches_oracle(V, d, rounds, engine, fp16):
    dm = C.circuit_dem(d, rounds, 0.004, noise="si1000", basis="X", schedule="xyz")
    syn, obs = D.sample(dm, 300, 50 + d)
    K, T, M = 8, 12, 3
    perms = D.schedules(dm.n, K, d)
    dec = V.Decoder(dm, K, perms, T=T, alpha=0.625, M=M, msg_fp16=fp16, engine=engine)
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda(),
                     observables=torch.from_numpy(np.ascontiguousarray(obs).view(np.int32)).cuda(),
                     want_soft=True, counters=cnt)
    torch.cuda.synchronize()
    r = oracle.decode(dm, perms, syn, T, 0.625, M, mode=oracle.FP16MSG if fp16 else oracle.FP32, nthreads=8)
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    assert np.array_equal(out["logical"].cpu().numpy().view(np.uint32), r["logical"])
    st = V.stats_to_numpy(out["stats"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    assert r["stats"]["lsd_invoked"].sum() > 0
    c = cnt.cpu().numpy()
    assert c[V.CNT_SHOTS] == len(syn)
    assert c[V.CNT_FAILURES] == int((r["logical"] != obs).any(axis=1).sum())
    dec.close()
