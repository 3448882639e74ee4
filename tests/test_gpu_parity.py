"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

FP32 and FP16-storage messages are both compared bit for bit (same corrections, logical flips,
per-shot records and posterior floats) because both sides use the same per-node operation order.
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


def run_gpu(V, dm, perms, syn, T, alpha, M, fp16=False, want_soft=True, obs=None, K=None, seed=0, order=0):
    K = perms.shape[0] if perms is not None else K
    dec = V.Decoder(dm, K, perms, T=T, alpha=alpha, M=M, msg_fp16=fp16, seed=seed, lsd_order=order)
    syn_t = torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda()
    obs_t = None if obs is None else torch.from_numpy(np.ascontiguousarray(obs).view(np.int32)).cuda()
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    out = dec.decode(syn_t, observables=obs_t, want_soft=want_soft, counters=cnt)
    torch.cuda.synchronize()
    res = dict(corrections=out["corrections"].cpu().numpy().view(np.uint32),
               logical=out["logical"].cpu().numpy().view(np.uint32),
               stats=V.stats_to_numpy(out["stats"]),
               soft=None if out["soft"] is None else out["soft"].cpu().numpy(),
               counters=cnt.cpu().numpy())
    dec.close()
    return res


def assert_same(g, r, soft=True, what=""):
    assert np.array_equal(g["corrections"], r["corrections"]), what + ": corrections"
    assert np.array_equal(g["logical"], r["logical"]), what + ": logical"
    for f in r["stats"].dtype.names:
        assert np.array_equal(g["stats"][f], r["stats"][f]), what + f": stats.{f}"
    if soft:
        a = g["soft"].view(np.uint32)
        b = r["soft"].astype(np.float32).view(np.uint32)
        bad = np.nonzero((a != b).any(axis=1))[0]
        assert len(bad) == 0, f"{what}: posteriors differ on shots {bad[:10]}"


def workload(name, shots=None, seed=None):
    w = D.WORKLOADS[name]
    dm = D.build_workload(name)
    syn, obs = D.sample(dm, shots or w["shots"], w["seed"] if seed is None else seed)
    perms = D.schedules(dm.n, w["K"], w["seed"], natural=w["natural"])
    return w, dm, syn, obs, perms


def test_codecap_d5_full_workload(V):
    w, dm, syn, obs, perms = workload("cc666_d5_codecap")
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"], obs=obs)
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], nthreads=8)
    assert_same(g, r, what="d5 code capacity")
    fails = (r["logical"] != obs).any(axis=1).sum()
    assert g["counters"][0] == len(syn) and g["counters"][1] == fails
    assert g["counters"][2] == r["stats"]["lsd_invoked"].sum()


@pytest.mark.parametrize("seed", [2, 7])
def test_pheno_d9_subset_fp32(V, seed):
    w, dm, syn, obs, perms = workload("cc666_d9_pheno", shots=2000, seed=seed)
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"], obs=obs)
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], nthreads=8)
    assert_same(g, r, what=f"d9 pheno seed {seed}")
    assert r["stats"]["lsd_invoked"].sum() > 100, "subset must exercise LSD"


def test_pheno_d9_subset_fp16_messages(V):
    w, dm, syn, obs, perms = workload("cc666_d9_pheno", shots=1500, seed=5)
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"], fp16=True)
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], mode=oracle.FP16MSG, nthreads=8)
    assert_same(g, r, what="d9 pheno FP16 messages")


@pytest.mark.parametrize("B", [1, 3, 31, 33, 129, 1001])
def test_ragged_batches(V, B):
    w, dm, syn, obs, perms = workload("cc666_d9_pheno", shots=B, seed=100 + B)
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"])
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], nthreads=4)
    assert_same(g, r, what=f"B={B}")


def test_empty_batch_is_noop(V):
    dm = D.build_workload("cc666_d5_codecap")
    dec = V.Decoder(dm, 1, D.schedules(dm.n, 1, 0, natural=True), T=20, M=1)
    V.vibe_decode(dec.handle, 0, 0, 0)
    dec.close()


@pytest.mark.parametrize("want_soft", [False, True])
def test_zero_syndromes(V, want_soft):
    w, dm, syn, obs, perms = workload("cc666_d9_pheno", shots=64, seed=3)
    syn[::2] = 0
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"], want_soft=want_soft)
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], nthreads=4)
    assert_same(g, r, soft=want_soft, what="zero syndromes")


@pytest.mark.parametrize("d,R,p,K,M,T", [(5, 5, 0.02, 8, 3, 15), (7, 3, 0.015, 4, 4, 10), (3, 2, 0.05, 2, 1, 25)])
def test_other_pheno_shapes(V, d, R, p, K, M, T):
    dm = D.phenomenological_dem(d, R, p, p)
    syn, obs = D.sample(dm, 700, d * 100 + R)
    perms = D.schedules(dm.n, K, d)
    g = run_gpu(V, dm, perms, syn, T, 0.625, M, obs=obs)
    r = oracle.decode(dm, perms, syn, T, 0.625, M, nthreads=8)
    assert_same(g, r, what=f"pheno d{d} R{R}")


def test_alpha_one_and_codecap_d7(V):
    dm = D.code_capacity_dem(7, 0.07)
    syn, obs = D.sample(dm, 3000, 12)
    perms = D.schedules(dm.n, 6, 1)
    g = run_gpu(V, dm, perms, syn, 12, 1.0, 2)
    r = oracle.decode(dm, perms, syn, 12, 1.0, 2, nthreads=8)
    assert_same(g, r, what="d7 alpha 1")


@pytest.mark.parametrize("order", [1, 3, 5, 10])
def test_lsd_higher_order(V, order):
    dm = D.phenomenological_dem(7, 5, 0.02, 0.02)
    syn, obs = D.sample(dm, 1200, 40 + order)
    perms = D.schedules(dm.n, 8, 3)
    g = run_gpu(V, dm, perms, syn, 10, 0.625, 3, order=order)
    r = oracle.decode(dm, perms, syn, 10, 0.625, 3, lsd_order=order, nthreads=8)
    assert_same(g, r, what=f"LSD order {order}")
    r0 = oracle.decode(dm, perms, syn, 10, 0.625, 3, lsd_order=0, nthreads=8)
    assert (r0["corrections"] != r["corrections"]).any(axis=1).sum() > 0, "the search must change some shots"


def test_seeded_schedules_match_definition(V):
    dm = D.build_workload("cc666_d9_pheno")
    syn, _ = D.sample(dm, 400, 9)
    seed = 0xC0FFEE
    perms = oracle.seeded_schedules(dm.n, 16, seed)
    g = run_gpu(V, dm, None, syn, 30, 0.625, 5, K=16, seed=seed)
    r = oracle.decode(dm, perms, syn, 30, 0.625, 5, nthreads=8)
    assert_same(g, r, what="device-drawn schedules")


def test_unsolvable_shot_is_flagged(V):
    A = np.array([[1, 1, 0, 0], [1, 1, 0, 0], [0, 1, 1, 1]], np.uint8)
    dm = D.DEM(D.CSR.from_dense(A), D.CSR.from_rows([[0]], 4), np.full(4, 0.1))
    syn = D.pack_bits(np.array([[1, 0, 0], [1, 1, 0], [0, 0, 1]], np.uint8))
    perms = np.arange(4, dtype=np.uint32)[None]
    g = run_gpu(V, dm, perms, syn, 5, 0.625, 1)
    r = oracle.decode(dm, perms, syn, 5, 0.625, 1)
    assert_same(g, r, what="unsolvable")
    assert g["stats"]["status"][0] == 1 and g["counters"][4] == 1


def test_host_buffer_path_matches_device_path(V):
    w, dm, syn, obs, perms = workload("cc666_d9_pheno", shots=3000, seed=21)
    dec = V.Decoder(dm, w["K"], perms, T=w["T"], alpha=w["alpha"], M=w["M"])
    h = dec.decode_host(syn, obs)
    dec.close()
    r = oracle.decode(dm, perms, syn, w["T"], w["alpha"], w["M"], nthreads=8)
    assert np.array_equal(h["corrections"], r["corrections"])
    assert np.array_equal(h["logical"], r["logical"])
    assert np.array_equal(h["stats"], r["stats"])
    assert h["counters"][0] == len(syn)
    assert h["counters"][1] == (r["logical"] != obs).any(axis=1).sum()


def _levels_by_definition(dm, perm):
    Ht = dm.H.transpose()
    last = np.full(dm.m, -1)
    lev = np.zeros(dm.n, np.int64)
    for v in perm:
        cs = Ht.row(int(v))
        lv = 1 + max([last[c] for c in cs], default=-1)
        lev[v] = lv
        for c in cs:
            last[c] = lv
    return lev


@pytest.mark.parametrize("name", ["cc666_d5_codecap", "cc666_d9_pheno"])
def test_wavefronts_match_definition(V, name):
    w = D.WORKLOADS[name]
    dm = D.build_workload(name)
    perms = D.schedules(dm.n, w["K"], w["seed"], natural=w["natural"])
    dec = V.Decoder(dm, w["K"], perms, T=w["T"], alpha=w["alpha"], M=w["M"])
    Ht = dm.H.transpose()
    for i in range(w["K"]):
        order, offs, nl = dec.wavefronts(i)
        assert np.array_equal(np.sort(order), np.arange(dm.n))
        lev = _levels_by_definition(dm, perms[i])
        assert nl == lev.max() + 1
        for l in range(nl):
            cols = order[offs[l]:offs[l + 1]]
            assert (lev[cols] == l).all()
            checks = np.concatenate([Ht.row(int(v)) for v in cols])
            assert len(checks) == len(np.unique(checks)), "a level's columns must not share a check"
    dec.close()


def test_full_size_pheno_sampled(V):
    """The full 10^6-shot workload in one call: sampled shots against the oracle, H e = s on all."""
    w, dm, syn, obs, perms = workload("cc666_d9_pheno")
    g = run_gpu(V, dm, perms, syn, w["T"], w["alpha"], w["M"], want_soft=False, obs=obs)
    e = D.unpack_bits(g["corrections"], dm.n)
    s2, o2 = D.syndromes_of(dm, e)
    unsolv = g["stats"]["status"] != 0
    assert not unsolv.any()
    assert np.array_equal(s2, syn), "every correction satisfies its syndrome"
    assert np.array_equal(o2, g["logical"])
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(syn), 1500, replace=False))
    r = oracle.decode(dm, perms, syn[idx], w["T"], w["alpha"], w["M"], nthreads=8, want_soft=False)
    sub = dict(corrections=g["corrections"][idx], logical=g["logical"][idx], stats=g["stats"][idx])
    assert_same(sub, r, soft=False, what="full-size sample")
    assert g["counters"][0] == len(syn)
    assert g["counters"][1] == (g["logical"] != obs).any(axis=1).sum()
    assert g["counters"][2] == g["stats"]["lsd_invoked"].sum()
