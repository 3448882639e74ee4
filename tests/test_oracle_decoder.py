"""Pins for the oracle's full decoder (Sec. III.D: ensemble, correction limit, ranking, LLR average, LSD).

Independent facts used:
  * every output satisfies H e = s (LSD guarantees a syndrome-consistent answer, Sec. III.C);
  * no decoder beats the minimum-weight solution of the coset (brute force on tiny DEMs);
  * a single fault of a distance >= 3 problem is decoded to the right logical class (exhaustive);
  * s = 0 gives e = 0 after one iteration without LSD;
  * the M-of-K rule and the ranking recomputed from independent single-member runs;
  * the normalised average recomputed in numpy (FP64) and in an explicit float32 replay.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from tests.helpers import coset_min_weight, f32_fold


def _check_valid(dm, syn, corr):
    e = D.unpack_bits(corr, dm.n)
    s2, _ = D.syndromes_of(dm, e)
    return np.array_equal(s2, syn)


@pytest.mark.parametrize("name,K,M", [("codecap", 1, 1), ("codecap", 8, 3), ("pheno3", 1, 1), ("pheno3", 8, 5)])
def test_never_beats_minimum_weight(name, K, M):
    if name == "codecap":
        dm = D.code_capacity_dem(5, 0.08)
    else:
        dm = D.phenomenological_dem(3, 2, 0.06, 0.04)
    assert dm.n <= 20
    A = dm.H.to_dense()
    lam = np.log((1 - dm.priors) / dm.priors)
    syn, obs, err = D.sample(dm, 60, 9, return_errors=True)
    perms = D.schedules(dm.n, K, 4, natural=(K == 1))
    out = oracle.decode(dm, perms, syn, 20, 0.625, M, mode=oracle.FP64)
    assert _check_valid(dm, syn, out["corrections"])
    e_hat = D.unpack_bits(out["corrections"], dm.n)
    hits = 0
    for b in range(len(syn)):
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        wmin = coset_min_weight(A, lam, s)
        w = float(np.dot(lam, e_hat[b]))
        assert w >= wmin - 1e-9
        hits += abs(w - wmin) < 1e-9
    assert hits >= 0.8 * len(syn)


@pytest.mark.parametrize("kind", ["codecap", "pheno"])
@pytest.mark.parametrize("K,M", [(1, 1), (16, 5)])
def test_single_faults_decode_to_their_logical_class(kind, K, M):
    dm = D.code_capacity_dem(5, 0.05) if kind == "codecap" else D.phenomenological_dem(5, 3, 0.01, 0.01)
    errs = np.eye(dm.n, dtype=np.uint8)
    syn, obs = D.syndromes_of(dm, errs)
    perms = D.schedules(dm.n, K, 7, natural=(K == 1))
    for mode in [oracle.FP32, oracle.FP16MSG, oracle.FP64]:
        out = oracle.decode(dm, perms, syn, 20, 0.625, M, mode=mode)
        assert _check_valid(dm, syn, out["corrections"])
        assert np.array_equal(out["logical"], obs), mode


@pytest.mark.parametrize("kind", ["codecap", "pheno"])
def test_square_octagon_single_faults_decode_to_their_logical_class(kind):
    """The same fact on the 4.8.8 colour code (distance 5): every single fault, exhaustively."""
    dm = D.code_capacity_dem(5, 0.05, "488") if kind == "codecap" else D.phenomenological_dem(5, 3, 0.01, 0.01, "488")
    errs = np.eye(dm.n, dtype=np.uint8)
    syn, obs = D.syndromes_of(dm, errs)
    for K, M in [(1, 1), (8, 3)]:
        perms = D.schedules(dm.n, K, 8, natural=(K == 1))
        out = oracle.decode(dm, perms, syn, 20, 0.625, M, mode=oracle.FP32)
        assert _check_valid(dm, syn, out["corrections"])
        assert np.array_equal(out["logical"], obs)


def test_zero_syndrome():
    dm = D.build_workload("cc666_d9_pheno")
    syn = np.zeros((3, D.words(dm.m)), np.uint32)
    perms = D.schedules(dm.n, 16, 2)
    out = oracle.decode(dm, perms, syn, 30, 0.625, 5)
    st = out["stats"]
    assert not out["corrections"].any()
    assert (st["iters"] == 1).all() and (st["n_converged"] == 5).all()
    assert (st["chosen_member"] == 0).all() and (st["lsd_invoked"] == 0).all()


def _members(dm, perms, s, T, mode, n_flood=0, alphas=None, n_layered=0):
    al = [0.625] * len(perms) if alphas is None else [float(np.float32(a)) for a in alphas]

    def one(i, p):
        if i < n_flood:
            return oracle.bp_member_flood(dm, s, T, al[i], mode)
        if i < n_flood + n_layered:
            return oracle.bp_member_layered(dm, s, T, al[i], mode)
        return oracle.bp_member(dm, s, p, T, al[i], mode)
    runs = [one(i, p) for i, p in enumerate(perms)]
    return [r[0] for r in runs], [r[1] for r in runs], [r[2] for r in runs]


# members differing in the scaling factor (reading R9), 16 members
MEMBER_ALPHA = np.array([0.5, 0.625, 0.75, 1.0, 0.875, 0.5625, 0.6875, 0.8125] * 2, np.float32)


@pytest.mark.parametrize("mode,n_flood,alphas,n_layered", [
    (oracle.FP32, 0, None, 0), (oracle.FP16MSG, 0, None, 0), (oracle.FP32, 4, None, 0),
    (oracle.FP32, 0, MEMBER_ALPHA, 0), (oracle.FP32, 4, MEMBER_ALPHA, 0), (oracle.FP16MSG, 0, MEMBER_ALPHA, 0),
    (oracle.FP32, 0, None, 6), (oracle.FP32, 3, MEMBER_ALPHA, 5), (oracle.FP16MSG, 2, None, 4)])
def test_correction_limit_and_ranking_from_independent_members(mode, n_flood, alphas, n_layered):
    """n_flood > 0: a mixed ensemble whose first members run the parallel schedule (reading R8);
    alphas: member i scales its check messages by alphas[i] (reading R9); n_layered: the next
    members run the layered schedule (reading R10)."""
    dm = D.build_workload("cc666_d9_pheno")
    K, M, T = 16, 5, 30
    perms = D.schedules(dm.n, K, 2)
    syn, _ = D.sample(dm, 40, 21)
    out = oracle.decode(dm, perms, syn, T, 0.625, M, mode=mode, n_flood=n_flood, member_alpha=alphas,
                        n_layered=n_layered)
    l32, _ = oracle.prior_llr(dm.priors)
    st = out["stats"]
    seen_bp = 0
    for b in range(len(syn)):
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        tconv, posts, ebits = _members(dm, perms, s, T, mode, n_flood, alphas, n_layered)
        conv = sorted((t, i) for i, t in enumerate(tconv) if t > 0)
        cand = conv[:M]
        if not cand:
            assert st["lsd_invoked"][b] == 1 and st["chosen_member"][b] == 255
            assert st["iters"][b] == T
            continue
        seen_bp += 1
        weights = [f32_fold(l32[np.nonzero(ebits[i])[0]]) for _, i in cand]
        best = int(np.argmin(weights))          # first minimum = earliest (t, member)
        chosen = cand[best][1]
        assert st["chosen_member"][b] == chosen
        assert st["n_converged"][b] == len(cand)
        assert st["iters"][b] == (cand[-1][0] if len(cand) == M else T)
        assert np.array_equal(D.unpack_bits(out["corrections"][b:b + 1], dm.n)[0], ebits[chosen])
        assert np.array_equal(out["soft"][b], posts[chosen])
    assert seen_bp > 10


def test_ranking_picks_lightest_candidate_when_candidates_differ():
    """A noisy small DEM where members converge to different corrections: the lightest wins."""
    dm = D.phenomenological_dem(3, 3, 0.08, 0.08)
    K, M, T = 16, 16, 30
    perms = D.schedules(dm.n, K, 2)
    syn, _ = D.sample(dm, 2000, 21)
    out = oracle.decode(dm, perms, syn, T, 0.625, M)
    l32, _ = oracle.prior_llr(dm.priors)
    not_first = 0
    for b in range(len(syn)):
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        tconv, posts, ebits = _members(dm, perms, s, T, oracle.FP32)
        cand = sorted((t, i) for i, t in enumerate(tconv) if t > 0)[:M]
        if not cand:
            continue
        weights = [f32_fold(l32[np.nonzero(ebits[i])[0]]) for _, i in cand]
        best = int(np.argmin(weights))
        assert out["stats"]["chosen_member"][b] == cand[best][1]
        not_first += best != 0
    assert not_first >= 2, "the instance must exercise the ranking"


def _canonical_norm_f32(x):
    part = np.zeros(32, np.float32)
    for l in range(32):
        acc = np.float32(0)
        for j in range(l, len(x), 32):
            v = np.float32(x[j])
            sq = np.float32(v * v) if np.isfinite(v) else np.float32(0)
            acc = np.float32(acc + sq)
        part[l] = acc
    for off in [16, 8, 4, 2, 1]:
        part = np.array([np.float32(part[l] + part[l ^ off]) for l in range(32)], np.float32)
    return np.float32(np.sqrt(part[0]))


@pytest.mark.parametrize("alphas", [None, np.array([1.0, 0.5, 0.625, 0.75], np.float32)])
def test_llr_average_matches_numpy_and_float32_replay(alphas):
    dm = D.build_workload("cc666_d9_pheno")
    K, M, T = 4, 2, 6
    perms = D.schedules(dm.n, K, 8)
    syn, _ = D.sample(dm, 60, 33)
    out32 = oracle.decode(dm, perms, syn, T, 0.625, M, mode=oracle.FP32, member_alpha=alphas)
    out64 = oracle.decode(dm, perms, syn, T, 0.625, M, mode=oracle.FP64, member_alpha=alphas)
    checked = 0
    for b in range(len(syn)):
        if out32["stats"]["lsd_invoked"][b] != 1:
            continue
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        # FP32: replay the documented order in float32
        _, posts, _ = _members(dm, perms, s, T, oracle.FP32, alphas=alphas)
        acc = np.zeros(dm.n, np.float32)
        for p in posts:
            p = p.astype(np.float32)
            nrm = _canonical_norm_f32(p)
            fin = np.isfinite(p)
            term = np.where(fin, (p / nrm) if nrm != 0 else np.float32(0), p).astype(np.float32)
            acc = (acc + term).astype(np.float32)
        ref = (acc / np.float32(K)).astype(np.float32)
        assert np.array_equal(out32["soft"][b].astype(np.float32), ref)
        # FP64 mode: the displayed formula in numpy (finite entries normalised)
        if out64["stats"]["lsd_invoked"][b] == 1:
            _, posts64, _ = _members(dm, perms, s, T, oracle.FP64, alphas=alphas)
            tot = np.zeros(dm.n)
            for p in posts64:
                fin = np.isfinite(p)
                tot += np.where(fin, p / np.linalg.norm(p[fin]), p)
            assert np.allclose(out64["soft"][b], tot / K, rtol=1e-12, atol=1e-15)
        checked += 1
    assert checked >= 3


def test_identical_members_average_is_normalised_llr():
    dm = D.build_workload("cc666_d9_pheno")
    perm = D.schedules(dm.n, 1, 5)
    perms = np.repeat(perm, 8, axis=0)
    syn, _ = D.sample(dm, 40, 44)
    out = oracle.decode(dm, perms, syn, 4, 0.625, 8, mode=oracle.FP32)
    for b in np.nonzero(out["stats"]["lsd_invoked"])[0][:5]:
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        _, post, _ = oracle.bp_member(dm, s, perm[0], 4, 0.625, oracle.FP32)
        fin = np.isfinite(post)
        ref = np.where(fin, post / np.linalg.norm(post[fin]), post)
        assert np.allclose(out["soft"][b][fin], ref[fin], rtol=1e-5, atol=1e-7)


def test_single_member_equals_bp_then_lsd():
    dm = D.build_workload("cc666_d5_codecap")
    perms = D.schedules(dm.n, 1, 0, natural=True)
    syn, _ = D.sample(dm, 400, 3)
    out = oracle.decode(dm, perms, syn, 20, 0.625, 1, mode=oracle.FP32)
    for b in range(len(syn)):
        s = D.unpack_bits(syn[b:b + 1], dm.m)[0]
        t, post, eb = oracle.bp_member(dm, s, perms[0], 20, 0.625, oracle.FP32)
        got = D.unpack_bits(out["corrections"][b:b + 1], dm.n)[0]
        if t:
            assert np.array_equal(got, eb)
        else:
            soft = out["soft"][b]
            st, eb2, _, _, _ = oracle.lsd(dm, soft, s, 0)
            assert np.array_equal(got, eb2)
            p32 = post.astype(np.float32)
            assert np.array_equal(soft.astype(np.float32),
                                  ((p32 / _canonical_norm_f32(p32)) / np.float32(1)).astype(np.float32))


def test_threads_do_not_change_results():
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, 16, 2)
    syn, _ = D.sample(dm, 64, 5)
    a = oracle.decode(dm, perms, syn, 30, 0.625, 5, nthreads=1)
    b = oracle.decode(dm, perms, syn, 30, 0.625, 5, nthreads=4)
    for k in ["corrections", "logical", "soft"]:
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["stats"], b["stats"])


def test_logical_output_is_L_times_correction():
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, 4, 2)
    syn, _ = D.sample(dm, 100, 6)
    out = oracle.decode(dm, perms, syn, 10, 0.625, 2)
    _, o = D.syndromes_of(dm, D.unpack_bits(out["corrections"], dm.n))
    assert np.array_equal(o, out["logical"])


def test_equal_member_alphas_equal_the_shared_alpha():
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, 8, 3)
    syn, _ = D.sample(dm, 80, 4)
    a = oracle.decode(dm, perms, syn, 20, 0.75, 3, n_flood=2)
    b = oracle.decode(dm, perms, syn, 20, 0.625, 3, n_flood=2, member_alpha=np.full(8, 0.75, np.float32))
    for k in ["corrections", "logical", "soft"]:
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["stats"], b["stats"])
    with pytest.raises(ValueError):
        oracle.decode(dm, perms, syn, 20, 0.625, 3, member_alpha=np.ones(7, np.float32))
    with pytest.raises(ValueError):   # more flooding and layered members than members
        oracle.decode(dm, perms, syn, 20, 0.625, 3, n_flood=5, n_layered=4)
