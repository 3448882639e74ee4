"""GPU parity of pair mode (one warp per (shot, member) pair) with shot mode and with the oracle.

Pair mode runs a shot's members at the same time on different warps; a member stops once M members
with a smaller (iteration, member) key have converged, and the last member to finish applies the
correction-limit rule (Sec. III.D.2 steps 3-5) to the members' records. Its outputs must equal shot
mode's bit for bit -- corrections, logical flips, every per-shot record field and the soft output --
on both BP engines, both message precisions, LSD-bound and BP-resolved shots, and mixed batches.
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


def decode(V, dm, perms, syn, T, M, pair, engine, fp16=False, soft=True, order=0, obs=None):
    dec = V.Decoder(dm, perms.shape[0], perms, T=T, M=M, msg_fp16=fp16, engine=engine, lsd_order=order,
                    pair_mode=pair)
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    obs_t = None if obs is None else torch.from_numpy(np.ascontiguousarray(obs).view(np.int32)).cuda()
    out = dec.decode(torch.from_numpy(np.ascontiguousarray(syn).view(np.int32)).cuda(), want_soft=soft,
                     observables=obs_t, counters=cnt)
    torch.cuda.synchronize()
    r = dict(corrections=out["corrections"].cpu().numpy().view(np.uint32),
             logical=out["logical"].cpu().numpy().view(np.uint32),
             stats=V.stats_to_numpy(out["stats"]), soft=None if out["soft"] is None else out["soft"].cpu().numpy(),
             counters=cnt.cpu().numpy())
    dec.close()
    return r


def same(a, b, what):
    assert np.array_equal(a["corrections"], b["corrections"]), what + ": corrections"
    assert np.array_equal(a["logical"], b["logical"]), what + ": logical"
    for f in a["stats"].dtype.names:
        assert np.array_equal(a["stats"][f], b["stats"][f]), f"{what}: stats.{f}"
    if a["soft"] is not None:
        assert np.array_equal(a["soft"].view(np.uint32), b["soft"].view(np.uint32)), what + ": soft output"


CASES = [
    # (name, DEM builder, K, M, T, engine, shots, seed)
    ("pheno_d9_image", lambda: D.build_workload("cc666_d9_pheno"), 16, 5, 30, 1, 1500, 31),
    ("pheno_d5_summary", lambda: D.phenomenological_dem(5, 5, 0.02, 0.02), 8, 3, 15, 2, 1200, 32),
    ("circuit_d5_summary", lambda: C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X"), 16, 5, 20, 2, 700, 33),
    ("circuit_d3_image", lambda: C.circuit_dem(3, 3, 0.004, noise="si1000", basis="X"), 6, 2, 20, 1, 900, 34),
]


@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pair_mode_equals_shot_mode(V, case, fp16):
    name, build, K, M, T, engine, B, seed = case
    dm = build()
    syn, obs = D.sample(dm, B, seed)
    perms = D.schedules(dm.n, K, seed)
    a = decode(V, dm, perms, syn, T, M, False, engine, fp16=fp16, obs=obs)
    b = decode(V, dm, perms, syn, T, M, True, engine, fp16=fp16, obs=obs)
    same(a, b, f"{name} fp16={fp16}")
    st = a["stats"]
    assert st["lsd_invoked"].sum() > 20 and (st["n_converged"] > 0).sum() > 20   # both paths exercised
    for c in (0, 1, 2):   # shots, failures, LSD shots (sweep counts differ: pair mode runs more)
        assert a["counters"][c] == b["counters"][c]


def test_pair_mode_matches_oracle_with_lsd_order(V):
    dm = C.circuit_dem(3, 3, 0.006, noise="si1000", basis="X")
    syn, _ = D.sample(dm, 400, 35)
    perms = D.schedules(dm.n, 8, 35)
    g = decode(V, dm, perms, syn, 12, 3, True, 2, order=3)
    r = oracle.decode(dm, perms, syn, 12, 0.625, 3, lsd_order=3, nthreads=8)
    assert np.array_equal(g["corrections"], r["corrections"])
    assert np.array_equal(g["logical"], r["logical"])
    for f in r["stats"].dtype.names:
        assert np.array_equal(g["stats"][f], r["stats"][f]), f
    assert np.array_equal(g["soft"].view(np.uint32), r["soft"].astype(np.float32).view(np.uint32))


def test_pair_mode_mixed_batch(V):
    probs = [(D.build_workload("cc666_d9_pheno"), 16, 5, 30), (D.phenomenological_dem(5, 5, 0.02, 0.02), 8, 3, 15),
             (C.circuit_dem(5, 5, 0.003, noise="si1000", basis="X"), 8, 3, 20)]
    outs = []
    rng = np.random.default_rng(36)
    B = 1500
    pid = rng.integers(0, len(probs), B).astype(np.int32)
    mw = max(D.words(p[0].m) for p in probs)
    syn = np.zeros((B, mw), np.uint32)
    for i, (dm, K, M, T) in enumerate(probs):
        rows = np.nonzero(pid == i)[0]
        s, _ = D.sample(dm, len(rows), 600 + i)
        syn[rows, :s.shape[1]] = s
    for pair in (False, True):
        decs = [V.Decoder(dm, K, D.schedules(dm.n, K, 700 + i), T=T, M=M, pair_mode=pair)
                for i, (dm, K, M, T) in enumerate(probs)]
        mb = V.MixedBatch(decs)
        out = mb.decode(torch.from_numpy(pid).cuda(), torch.from_numpy(syn.view(np.int32)).cuda())
        torch.cuda.synchronize()
        outs.append((out["corrections"].cpu().numpy(), out["logical"].cpu().numpy(), out["stats"].cpu().numpy()))
        mb.close()
        for dc in decs:
            dc.close()
    for x, y in zip(outs[0], outs[1]):
        assert np.array_equal(x, y)
