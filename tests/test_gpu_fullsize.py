"""Full-size configurations on sampled shots (the oracle cannot decode whole circuit-level batches:
one LSD-bound shot of the d=11 problem with K=64, T=50 costs it minutes).

Config 3 (d=11 circuit level, K=64, T=50, M=5): the GPU decodes a batch in the launch configuration
the library picks; every shot's correction must satisfy H e = s with consistent records, and sampled
shots that BP resolved are compared with the oracle bit for bit. The LSD path at that size is compared
on sampled shots of the same batch decoded with T=3 (so that most shots reach LSD), for LSD orders 0
and 5.

Config 4 (colour codes d = 5..15 under circuit-level noise at p = 1, 2, 3, 5 per mille, K=32, FP16,
one mixed launch): every shot equals the decode of its own handle, and shots of the smaller problems
match the oracle. T is reduced to 10 to bound the run time (an LSD-bound d=15 shot at T=50 runs
32 x 50 sweeps of ~1300 levels each).
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


@pytest.fixture(scope="module")
def d11():
    dm = C.circuit_dem(11, 11, 0.001, noise="si1000", basis="X")
    syn, obs = D.sample(dm, 2432, 3)
    return dm, syn, obs


def decode(V, dm, perms, syn, T, M, order=0, fp16=False):
    dec = V.Decoder(dm, perms.shape[0], perms, T=T, M=M, lsd_order=order, msg_fp16=fp16)
    out = dec.decode(torch.from_numpy(syn.view(np.int32)).cuda())
    torch.cuda.synchronize()
    res = dict(corrections=out["corrections"].cpu().numpy().view(np.uint32),
               logical=out["logical"].cpu().numpy().view(np.uint32), stats=V.stats_to_numpy(out["stats"]))
    dec.close()
    return res


def check_valid(V, dm, syn, g, T):
    e = D.unpack_bits(g["corrections"], dm.n)
    s2, l2 = D.syndromes_of(dm, e)
    st = g["stats"]
    ok = st["status"] == V.VIBE_STATUS_OK
    assert np.array_equal(s2[ok], syn[ok]), "H e != s on a solved shot"
    assert np.array_equal(l2, g["logical"]), "logical flips differ from L e"
    assert np.all(st["n_converged"][st["lsd_invoked"] == 1] == 0)
    assert np.all(st["iters"] <= T)
    assert not np.any(st["status"] == V.VIBE_STATUS_CLUSTER_LIMIT)


def compare(g, r, rows, what):
    assert np.array_equal(g["corrections"][rows], r["corrections"]), what + ": corrections"
    assert np.array_equal(g["logical"][rows], r["logical"]), what + ": logical"
    for f in r["stats"].dtype.names:
        assert np.array_equal(g["stats"][rows][f], r["stats"][f]), f"{what}: stats.{f}"


def test_config3_d11_bp_resolved_shots_match_oracle(V, d11):
    dm, syn, obs = d11
    K, T, M = 64, 50, 5
    perms = D.schedules(dm.n, K, 3)
    g = decode(V, dm, perms, syn, T, M)
    check_valid(V, dm, syn, g, T)
    st = g["stats"]
    rows = np.nonzero((st["lsd_invoked"] == 0) & (st["n_converged"] == M))[0][:6]
    assert len(rows) == 6
    r = oracle.decode(dm, perms, syn[rows], T, 0.625, M, nthreads=6, want_soft=False)
    compare(g, r, rows, "d11 K64 T50")


@pytest.mark.parametrize("order", [0, 5])
def test_config3_d11_lsd_shots_match_oracle(V, d11, order):
    dm, syn, obs = d11
    K, T, M = 64, 3, 5
    perms = D.schedules(dm.n, K, 3)
    g = decode(V, dm, perms, syn, T, M, order=order)
    check_valid(V, dm, syn, g, T)
    rows = np.nonzero(g["stats"]["lsd_invoked"] == 1)[0][:6]
    assert len(rows) == 6
    r = oracle.decode(dm, perms, syn[rows], T, 0.625, M, lsd_order=order, nthreads=6, want_soft=False)
    compare(g, r, rows, f"d11 K64 T3 LSD order {order}")


def test_config4_mixed_circuit_family(V):
    ds, ps = (5, 7, 9, 11, 13, 15), (1e-3, 2e-3, 3e-3, 5e-3)
    K, T, M = 32, 10, 5
    dems, decs, perms = [], [], []
    for d in ds:
        base = None
        for p in ps:
            dm = C.circuit_dem(d, d, p, noise="si1000", basis="X")
            if base is None:
                base = dm
            else:   # one graph structure per distance: the same matrix, other priors
                assert np.array_equal(dm.H.colidx, base.H.colidx) and np.array_equal(dm.H.rowptr, base.H.rowptr)
            pm = D.schedules(dm.n, K, 100 + d)
            dems.append(dm)
            perms.append(pm)
            decs.append(V.Decoder(dm, K, pm, T=T, M=M, msg_fp16=True))
    mb = V.MixedBatch(decs)
    rng = np.random.default_rng(4)
    B = 24 * 24
    pid = rng.permutation(np.repeat(np.arange(24, dtype=np.int32), 24))
    mw = max(dc.mw for dc in decs)
    syn = np.zeros((B, mw), np.uint32)
    for i, dm in enumerate(dems):
        rows = np.nonzero(pid == i)[0]
        s, _ = D.sample(dm, len(rows), 400 + i)
        syn[rows, :s.shape[1]] = s
    out = mb.decode(torch.from_numpy(pid).cuda(), torch.from_numpy(syn.view(np.int32)).cuda())
    torch.cuda.synchronize()
    corr = out["corrections"].cpu().numpy().view(np.uint32)
    st = V.stats_to_numpy(out["stats"])
    for i, (dm, dc) in enumerate(zip(dems, decs)):
        rows = np.nonzero(pid == i)[0]
        one = dc.decode(torch.from_numpy(np.ascontiguousarray(syn[rows][:, :dc.mw]).view(np.int32)).cuda())
        assert np.array_equal(corr[rows][:, :dc.nw], one["corrections"].cpu().numpy().view(np.uint32)), i
        assert np.array_equal(st[rows], V.stats_to_numpy(one["stats"])), i
        if dm.n < 10_000:   # d = 5 and 7: the oracle decodes these quickly
            r = oracle.decode(dm, perms[i], syn[rows][:, :D.words(dm.m)], T, 0.625, M, mode=oracle.FP16MSG,
                              nthreads=16, want_soft=False)
            assert np.array_equal(corr[rows][:, :dc.nw], r["corrections"]), i
    mb.close()
    for dc in decs:
        dc.close()
