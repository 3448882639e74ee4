"""GPU parity on the square-octagon (4.8.8) colour code: code-capacity and phenomenological problems,
both BP engines, FP32 and FP16 message storage, against the oracle bit for bit (corrections, logical
flips, per-shot records, posteriors or the averaged LLR vectors handed to LSD)."""
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


CASES = [
    # name, DEM builder, K, M, T, natural order, shots, seed
    ("codecap_d5", lambda: D.code_capacity_dem(5, 0.05, "488"), 1, 1, 20, True, 4000, 11),
    ("codecap_d7", lambda: D.code_capacity_dem(7, 0.06, "488"), 8, 3, 20, False, 3000, 12),
    ("pheno_d5", lambda: D.phenomenological_dem(5, 5, 0.015, 0.015, "488"), 8, 3, 20, False, 2000, 13),
    ("pheno_d9", lambda: D.build_workload("cc488_d9_pheno"), 16, 5, 30, False, 1500, 14),
]


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("engine", ["image", "summary"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_square_octagon_matches_oracle(V, case, engine, fp16):
    name, build, K, M, T, natural, shots, seed = case
    dm = build()
    syn, obs = D.sample(dm, shots, seed)
    perms = D.schedules(dm.n, K, seed, natural=natural)
    eng = V.ENGINE_IMAGE if engine == "image" else V.ENGINE_SUMMARY
    dec = V.Decoder(dm, K, perms, T=T, alpha=0.625, M=M, msg_fp16=fp16, engine=eng)
    out = dec.decode(torch.from_numpy(syn.view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    r = oracle.decode(dm, perms, syn, T, 0.625, M, nthreads=8, mode=oracle.FP16MSG if fp16 else oracle.FP32)
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    assert np.array_equal(out["logical"].cpu().numpy().view(np.uint32), r["logical"])
    st = V.stats_to_numpy(out["stats"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    assert st["lsd_invoked"].sum() > 0 and (st["n_converged"] > 0).sum() > 0   # both paths exercised
    dec.close()


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("engine", ["image", "summary"])
def test_square_octagon_circuit_level_matches_oracle(V, engine, fp16):
    """The 4.8.8 d=5 memory circuit (5 rounds, Si1000 p = 3e-3; eight edge-coloured CNOT layers)."""
    from paper_2508_15743_gb300 import circuit as C
    dm = C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X", tiling="488")
    syn, _ = D.sample(dm, 200, 15)
    perms = D.schedules(dm.n, 8, 15)
    eng = V.ENGINE_IMAGE if engine == "image" else V.ENGINE_SUMMARY
    dec = V.Decoder(dm, 8, perms, T=20, alpha=0.625, M=3, msg_fp16=fp16, engine=eng)
    out = dec.decode(torch.from_numpy(syn.view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    r = oracle.decode(dm, perms, syn, 20, 0.625, 3, nthreads=8, mode=oracle.FP16MSG if fp16 else oracle.FP32)
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    assert np.array_equal(out["logical"].cpu().numpy().view(np.uint32), r["logical"])
    st = V.stats_to_numpy(out["stats"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    dec.close()
