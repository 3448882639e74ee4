"""GPU parity of layered members (the oracle's reading R10: row-layered min-sum over greedy check
layers) and of flooding members with FP16 message storage (reading R8), both in the image engine.

The device's check layers must equal the oracle's; ensembles mixing flooding, layered and serial
members must match the oracle bit for bit: corrections, logical flips, per-shot records, posteriors
(or the averaged LLR vectors handed to LSD), in shot mode and in pair mode.
"""
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


def problems():
    return {
        "codecap_d5": D.build_workload("cc666_d5_codecap"),
        "pheno_d9": D.build_workload("cc666_d9_pheno"),
        "pheno_d5": D.phenomenological_dem(5, 5, 0.02, 0.02),
        "circuit_d5": C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X"),
        "circuit_d3": C.circuit_dem(3, 3, 0.004, noise="si1000", basis="X"),
    }


@pytest.mark.parametrize("name", ["codecap_d5", "pheno_d9", "circuit_d5"])
def test_device_layers_equal_the_oracle(V, name):
    dm = problems()[name]
    # FP16 storage: the d=5 circuit's rows of up to ~170 entries need it for the image to fit
    dec = V.Decoder(dm, 2, D.schedules(dm.n, 2, 1), T=5, M=1, n_layered=1, engine=V.ENGINE_IMAGE, msg_fp16=True)
    got, nl = dec.layers()
    ref, rnl = oracle.check_layers(dm)
    assert nl == rnl
    assert np.array_equal(got, ref)
    dec.close()


def run_both(V, dm, K, M, T, n_flood, n_layered, fp16, shots, seed, pair=False, lsd_order=0):
    syn, _ = D.sample(dm, shots, seed)
    perms = D.schedules(dm.n, K, seed + 1, natural=(K == 1))
    dec = V.Decoder(dm, K, perms, T=T, M=M, msg_fp16=fp16, n_flood=n_flood, n_layered=n_layered,
                    engine=V.ENGINE_IMAGE, pair_mode=pair, lsd_order=lsd_order)
    out = dec.decode(torch.from_numpy(syn.view(np.int32)).cuda(), want_soft=True)
    torch.cuda.synchronize()
    r = oracle.decode(dm, perms, syn, T, 0.625, M, lsd_order=lsd_order, nthreads=8, n_flood=n_flood,
                      n_layered=n_layered, mode=oracle.FP16MSG if fp16 else oracle.FP32)
    st = V.stats_to_numpy(out["stats"])
    assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
    assert np.array_equal(out["logical"].cpu().numpy().view(np.uint32), r["logical"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(st[f], r["stats"][f]), f
    soft = out["soft"].cpu().numpy()
    assert np.array_equal(soft.view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))
    dec.close()
    return st


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("name,shots,K,M,T,n_flood,n_layered", [
    ("codecap_d5", 3000, 1, 1, 20, 0, 1),
    ("pheno_d9", 1200, 8, 3, 30, 2, 3),
    ("pheno_d5", 2000, 6, 3, 15, 0, 6),
    ("circuit_d3", 900, 6, 2, 20, 1, 3),
])
def test_layered_members_match_oracle(V, fp16, name, shots, K, M, T, n_flood, n_layered):
    st = run_both(V, problems()[name], K, M, T, n_flood, n_layered, fp16, shots, 40)
    if name == "pheno_d9":   # the instance picks members of each schedule type
        chosen = st["chosen_member"][st["lsd_invoked"] == 0]
        assert (chosen < n_flood).any()
        assert ((chosen >= n_flood) & (chosen < n_flood + n_layered)).any()
        assert (chosen >= n_flood + n_layered).any()


@pytest.mark.parametrize("name,shots,K,M,T", [("pheno_d9", 1500, 16, 5, 30), ("codecap_d5", 3000, 1, 1, 20)])
def test_flooding_members_with_fp16_storage_match_oracle(V, name, shots, K, M, T):
    run_both(V, problems()[name], K, M, T, min(4, K), 0, True, shots, 50)


def test_layered_members_in_pair_mode_match_oracle(V):
    run_both(V, problems()["pheno_d9"], 8, 3, 30, 1, 4, False, 1000, 60, pair=True)
    run_both(V, problems()["pheno_d9"], 8, 3, 30, 1, 4, True, 1000, 61, pair=True, lsd_order=3)
