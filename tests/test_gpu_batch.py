"""GPU parity of the batching layer: mixed-problem launches, CUDA-graph replay and the launch tuner.

Every shot of a mixed batch must decode exactly as the oracle decodes it with its own problem's
matrix, schedules and limits (Sec. III.D.2 per shot); batching only changes which launch carries it.
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
    """(name, dem, K, M, T, lsd_order, schedule seed): code-capacity, phenomenological and circuit-level
    problems of different sizes, ensemble shapes and LSD orders."""
    return [
        ("codecap_d5", D.build_workload("cc666_d5_codecap"), 1, 1, 20, 0, 1),
        ("pheno_d5", D.phenomenological_dem(5, 5, 0.02, 0.02), 8, 3, 15, 0, 5),
        ("pheno_d9", D.build_workload("cc666_d9_pheno"), 16, 5, 30, 0, 2),
        ("pheno_d3_order3", D.phenomenological_dem(3, 3, 0.04, 0.04), 4, 2, 12, 3, 3),
        ("circuit_d3_si1000", C.circuit_dem(3, 3, 0.004, noise="si1000", basis="X"), 6, 2, 20, 0, 4),
    ]


def pad_words(a, width):
    out = np.zeros((a.shape[0], width), np.uint32)
    out[:, :a.shape[1]] = a
    return out


@pytest.mark.parametrize("fp16", [False, True])
def test_mixed_batch_matches_per_problem_oracle(V, fp16):
    probs = problems()
    rng = np.random.default_rng(11 + fp16)
    B = 3000
    pid = rng.integers(0, len(probs), B).astype(np.int32)
    pid[[5, 77, 1234]] = [-1, len(probs), 1 << 20]   # out-of-range ids: not decoded
    mw = max(D.words(p[1].m) for p in probs)
    nw = max(D.words(p[1].n) for p in probs)
    kw = max(D.words(p[1].k) for p in probs)
    syn = np.zeros((B, mw), np.uint32)
    obs = np.zeros((B, kw), np.uint32)
    perms, decs = [], []
    for i, (name, dm, K, M, T, order, s) in enumerate(probs):
        rows = np.nonzero(pid == i)[0]
        si, oi = D.sample(dm, len(rows), 1000 + i)
        syn[rows] = pad_words(si, mw)
        obs[rows] = pad_words(oi, kw)
        pm = D.schedules(dm.n, K, s, natural=(K == 1))
        perms.append(pm)
        decs.append(V.Decoder(dm, K, pm, T=T, alpha=0.625, M=M, lsd_order=order, msg_fp16=fp16))
    mb = V.MixedBatch(decs)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    obs_t = torch.from_numpy(obs.view(np.int32)).cuda()
    pid_t = torch.from_numpy(pid).cuda()
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    # pre-fill outputs with a pattern: words past a problem's own are left as they are
    corr_t = torch.full((B, nw), -1, dtype=torch.int32, device="cuda")
    log_t = torch.full((B, kw), -1, dtype=torch.int32, device="cuda")
    st_t = torch.empty((B, 12), dtype=torch.uint8, device="cuda")
    mb.decode(pid_t, syn_t, observables=obs_t, counters=cnt, out=dict(corrections=corr_t, logical=log_t, stats=st_t))
    torch.cuda.synchronize()
    corr = corr_t.cpu().numpy().view(np.uint32)
    logi = log_t.cpu().numpy().view(np.uint32)
    stats = V.stats_to_numpy(st_t)
    counters = cnt.cpu().numpy()
    mode = oracle.FP16MSG if fp16 else oracle.FP32
    fails = 0
    for i, (name, dm, K, M, T, order, s) in enumerate(probs):
        rows = np.nonzero(pid == i)[0]
        r = oracle.decode(dm, perms[i], syn[rows][:, :D.words(dm.m)], T, 0.625, M, lsd_order=order, mode=mode,
                          nthreads=8)
        nwi, kwi = D.words(dm.n), D.words(dm.k)
        assert np.array_equal(corr[rows][:, :nwi], r["corrections"]), name
        assert np.all(corr[rows][:, nwi:] == 0xFFFFFFFF), name + ": words past the problem's were written"
        assert np.array_equal(logi[rows][:, :kwi], r["logical"]), name
        for f in r["stats"].dtype.names:
            assert np.array_equal(stats[rows][f], r["stats"][f]), f"{name}: stats.{f}"
        fails += int((r["logical"] != obs[rows][:, :kwi]).any(axis=1).sum())
    bad = np.nonzero((pid < 0) | (pid >= len(probs)))[0]
    assert np.all(stats[bad]["status"] == V.VIBE_STATUS_BAD_PROBLEM)
    assert np.all(corr[bad] == 0) and np.all(logi[bad] == 0)
    assert counters[V.CNT_BAD_PROBLEM] == len(bad)
    assert counters[V.CNT_SHOTS] == B - len(bad)
    assert counters[V.CNT_FAILURES] == fails
    assert counters[V.CNT_LSD] == int(stats["lsd_invoked"].sum())
    mb.close()
    for d in decs:
        d.close()


def test_mixed_batch_equals_separate_decodes(V):
    """The same shots through vibe_batch_decode and through each handle's vibe_decode."""
    probs = problems()[:3]
    decs = [V.Decoder(dm, K, D.schedules(dm.n, K, s, natural=(K == 1)), T=T, M=M, lsd_order=o)
            for (_, dm, K, M, T, o, s) in probs]
    mb = V.MixedBatch(decs)
    rng = np.random.default_rng(5)
    B = 1200
    pid = rng.integers(0, len(probs), B).astype(np.int32)
    mw = max(d.mw for d in decs)
    syn = np.zeros((B, mw), np.uint32)
    for i, (_, dm, *_rest) in enumerate(probs):
        rows = np.nonzero(pid == i)[0]
        syn[rows] = pad_words(D.sample(dm, len(rows), 70 + i)[0], mw)
    out = mb.decode(torch.from_numpy(pid).cuda(), torch.from_numpy(syn.view(np.int32)).cuda())
    corr = out["corrections"].cpu().numpy()
    st = V.stats_to_numpy(out["stats"])
    for i, d in enumerate(decs):
        rows = np.nonzero(pid == i)[0]
        one = d.decode(torch.from_numpy(np.ascontiguousarray(syn[rows][:, :d.mw]).view(np.int32)).cuda())
        assert np.array_equal(corr[rows][:, :d.nw], one["corrections"].cpu().numpy())
        assert np.array_equal(st[rows], V.stats_to_numpy(one["stats"]))
    mb.close()
    for d in decs:
        d.close()


def test_mixed_batch_rejects_mixed_precision_and_small_strides(V):
    dm = D.build_workload("cc666_d5_codecap")
    pm = D.schedules(dm.n, 1, 0, natural=True)
    a = V.Decoder(dm, 1, pm, T=10, M=1)
    b = V.Decoder(dm, 1, pm, T=10, M=1, msg_fp16=True)
    with pytest.raises(V.VibeError) as e:
        V.vibe_batch_create([a.handle, b.handle])
    assert e.value.code == V.VIBE_ERR_INVALID
    mb = V.MixedBatch([a])
    syn = torch.zeros((4, 1), dtype=torch.int32, device="cuda")
    pid = torch.zeros(4, dtype=torch.int32, device="cuda")
    corr = torch.zeros((4, 1), dtype=torch.int32, device="cuda")
    with pytest.raises(V.VibeError):
        V.vibe_batch_decode(mb.handle, pid, syn, 0, 4, corr, a.nw)
    mb.close()
    a.close()
    b.close()


def test_cuda_graph_replay_matches_oracle(V):
    """A decode captured once into a CUDA graph and replayed on fresh syndromes."""
    w = D.WORKLOADS["cc666_d9_pheno"]
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, w["K"], w["seed"])
    dec = V.Decoder(dm, w["K"], perms, T=w["T"], M=w["M"])
    B = 700
    s0, _ = D.sample(dm, B, 41)
    static_syn = torch.from_numpy(s0.view(np.int32)).cuda()
    out = dec.decode(static_syn)            # warm-up: sizes the workspace and kernel attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dec.decode(static_syn, out=out)
    for seed in (42, 43):
        s, _ = D.sample(dm, B, seed)
        static_syn.copy_(torch.from_numpy(s.view(np.int32)))
        g.replay()
        torch.cuda.synchronize()
        r = oracle.decode(dm, perms, s, w["T"], w["alpha"], w["M"], nthreads=8)
        assert np.array_equal(out["corrections"].cpu().numpy().view(np.uint32), r["corrections"])
        st = V.stats_to_numpy(out["stats"])
        for f in r["stats"].dtype.names:
            assert np.array_equal(st[f], r["stats"][f]), f
    del g
    dec.close()


def test_autotune_keeps_results(V):
    w = D.WORKLOADS["cc666_d9_pheno"]
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, w["K"], w["seed"])
    dec = V.Decoder(dm, w["K"], perms, T=w["T"], M=w["M"])
    s, _ = D.sample(dm, 4000, 9)
    syn_t = torch.from_numpy(s.view(np.int32)).cuda()
    before = dec.decode(syn_t)["corrections"].cpu().numpy()
    eng, bp, lsd, nt = dec.autotune(syn_t)
    assert eng in (V.ENGINE_IMAGE, V.ENGINE_SUMMARY) and bp >= 1 and lsd >= 1 and nt in (64, 128, 256)
    after = dec.decode(syn_t)["corrections"].cpu().numpy()
    assert np.array_equal(before, after)
    dec.close()


def test_autotune_may_switch_engine_and_keeps_results(V):
    dm = C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X")
    perms = D.schedules(dm.n, 8, 2)
    dec = V.Decoder(dm, 8, perms, T=15, M=3, msg_fp16=True)
    s, _ = D.sample(dm, 3000, 6)
    syn_t = torch.from_numpy(s.view(np.int32)).cuda()
    before = dec.decode(syn_t)
    b_corr, b_st = before["corrections"].cpu().numpy(), V.stats_to_numpy(before["stats"])
    eng, bp, lsd, nt = dec.autotune(syn_t)
    assert eng in (V.ENGINE_IMAGE, V.ENGINE_SUMMARY) and nt in (64, 128, 256)
    after = dec.decode(syn_t)
    assert np.array_equal(b_corr, after["corrections"].cpu().numpy())
    assert np.array_equal(b_st, V.stats_to_numpy(after["stats"]))
    dec.close()


def test_batch_autotune_keeps_results(V):
    """The batch tuner's launch search (shot/pair mode, BP grids, LSD CTA size and grid) changes the
    time only: stats, corrections and logical flips are the same before and after it."""
    probs = [(C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X"), 8, 3, 20, V.ENGINE_SUMMARY),
             (D.phenomenological_dem(5, 5, 0.02, 0.02), 8, 3, 15, V.ENGINE_IMAGE),
             (C.circuit_dem(7, 7, 0.002, noise="si1000", basis="X"), 8, 3, 20, V.ENGINE_SUMMARY)]
    decs = [V.Decoder(dm, K, D.schedules(dm.n, K, 80 + i), T=T, M=M, msg_fp16=True, engine=eng)
            for i, (dm, K, M, T, eng) in enumerate(probs)]
    mb = V.MixedBatch(decs)
    rng = np.random.default_rng(12)
    B = 2000
    pid = rng.integers(0, len(probs), B).astype(np.int32)
    mw = max(d.mw for d in decs)
    syn = np.zeros((B, mw), np.uint32)
    for i, (dm, *_r) in enumerate(probs):
        rows = np.nonzero(pid == i)[0]
        syn[rows] = pad_words(D.sample(dm, len(rows), 90 + i)[0], mw)
    pid_t = torch.from_numpy(pid).cuda()
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    before = mb.decode(pid_t, syn_t)
    b = {k: v.cpu().numpy() for k, v in before.items()}
    start = mb.launch()
    assert start["engines"] == 3 and start["lsd_threads"] == 128
    got = mb.autotune(pid_t, syn_t)
    assert got == mb.launch()
    assert got["pair_mode"] in (0, 1) and got["lsd_threads"] in (64, 128, 256)
    assert 1 <= got["bp_blocks_per_sm"] <= start["bp_blocks_per_sm"]
    assert 1 <= got["bpx_blocks_per_sm"] <= start["bpx_blocks_per_sm"]
    after = mb.decode(pid_t, syn_t)
    for k in ("corrections", "logical", "stats"):
        assert np.array_equal(b[k], after[k].cpu().numpy()), k
    mb.close()
    for d in decs:
        d.close()


def test_mixed_batch_in_a_cuda_graph(V):
    """A mixed decode captured once and replayed on new problem ids and syndromes. A shot writes only
    its own problem's correction words, so the outputs are cleared before each replay to compare
    whole rows with a fresh decode."""
    probs = problems()[:3]
    decs = [V.Decoder(dm, K, D.schedules(dm.n, K, s, natural=(K == 1)), T=T, M=M, lsd_order=o)
            for (_, dm, K, M, T, o, s) in probs]
    mb = V.MixedBatch(decs)
    rng = np.random.default_rng(9)
    B = 800
    mw = max(d.mw for d in decs)

    def draw(seed):
        pid = rng.integers(0, len(probs), B).astype(np.int32)
        syn = np.zeros((B, mw), np.uint32)
        for i, (_, dm, *_r) in enumerate(probs):
            rows = np.nonzero(pid == i)[0]
            syn[rows] = pad_words(D.sample(dm, len(rows), seed + i)[0], mw)
        return pid, syn

    pid0, syn0 = draw(10)
    pid_t = torch.from_numpy(pid0).cuda()
    syn_t = torch.from_numpy(syn0.view(np.int32)).cuda()
    out = mb.decode(pid_t, syn_t)          # warm-up: workspace and kernel attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mb.decode(pid_t, syn_t, out=out)
    for seed in (20, 30):
        pid, syn = draw(seed)
        pid_t.copy_(torch.from_numpy(pid))
        syn_t.copy_(torch.from_numpy(syn.view(np.int32)))
        out["corrections"].zero_()
        out["logical"].zero_()
        g.replay()
        torch.cuda.synchronize()
        ref = mb.decode(pid_t, syn_t)
        assert np.array_equal(out["corrections"].cpu().numpy(), ref["corrections"].cpu().numpy())
        assert np.array_equal(out["logical"].cpu().numpy(), ref["logical"].cpu().numpy())
        assert np.array_equal(out["stats"].cpu().numpy(), ref["stats"].cpu().numpy())
    del g
    mb.close()
    for d in decs:
        d.close()
