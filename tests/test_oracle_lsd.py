"""Pins for the oracle's LSD post-processor (Sec. III.C) and its order-lambda search.

Independent facts used:
  * LSD returns a syndrome-consistent answer: H e = s for every solvable syndrome;
  * each final cluster is valid and its answer equals OSD-0 (dense GF(2) elimination with columns
    in reliability order, free columns zero) on the cluster's submatrix, computed here in numpy;
  * clusters are disjoint, hold every flipped check, and hold all checks of their columns;
  * the order-lambda answer of a cluster is the minimum-weight one among the 2^q settings of its
    first q free columns (enumerated here), never heavier than order 0;
  * a syndrome outside the column span is reported unsolvable.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from tests.helpers import f32_fold, gf2_solve_one, osd0


def _rank_order(soft, cols):
    return sorted(cols, key=lambda j: (soft[j], j))


def _clusters(cl):
    out = {}
    for j, r in enumerate(cl):
        if r >= 0:
            out.setdefault(int(r), []).append(j)
    return out


def _random_case(dm, rng, density=0.04):
    e = (rng.random(dm.n) < density).astype(np.uint8)
    s = dm.H.to_dense().astype(np.int64).dot(e) % 2
    soft = rng.normal(size=dm.n)
    soft[e == 1] -= 1.5       # make the true error look likely, as BP soft output would
    return s.astype(np.uint8), soft


@pytest.mark.parametrize("seed", range(8))
def test_lsd_valid_and_clusterwise_osd0(seed):
    dm = D.phenomenological_dem(5, 3, 0.01, 0.01)
    A = dm.H.to_dense()
    Ht = dm.H.transpose()
    rng = np.random.default_rng(seed)
    for _ in range(15):
        s, soft = _random_case(dm, rng)
        st, eb, cl, ncl, big = oracle.lsd(dm, soft, s, 0)
        assert st == 0
        assert np.array_equal(A.astype(np.int64).dot(eb) % 2, s)
        clusters = _clusters(cl)
        assert ncl == len(clusters), "every final (valid) cluster holds a column"
        assert big == max([len(v) for v in clusters.values()] + [0])
        # every column's checks, and the checks' cluster, are consistent; collect checks per cluster
        chk_owner = {}
        for r, cols in clusters.items():
            for j in cols:
                for c in Ht.row(j):
                    assert chk_owner.setdefault(int(c), r) == r, "clusters must be disjoint in checks"
        for c in np.nonzero(s)[0]:
            if int(c) not in chk_owner:
                # a flipped check whose cluster holds no column cannot be valid
                pytest.fail("flipped check left outside every column-holding cluster")
        for r, cols in clusters.items():
            checks = sorted(c for c, o in chk_owner.items() if o == r)
            sub = A[np.ix_(checks, cols)]
            order = sorted(range(len(cols)), key=lambda t: (soft[cols[t]], cols[t]))
            x = osd0(sub, s[checks], order)
            assert x is not None, "final clusters are valid"
            assert np.array_equal(eb[cols], x)
        outside = np.ones(dm.n, bool)
        for cols in clusters.values():
            outside[cols] = False
        assert not eb[outside].any()


def test_lsd_single_cluster_equals_full_osd0():
    """When one cluster takes every column of a connected H, LSD is OSD-0 on the whole of H.

    Construction: each column owns a private check and shared checks join all columns; flipping
    every private check puts every column into the first round's growth, and the shared checks
    merge the clusters into one that covers H."""
    rng = np.random.default_rng(0)
    seen = 0
    for trial in range(30):
        n = int(rng.integers(3, 9))
        shared = (rng.random((3, n)) < 0.6).astype(np.uint8)
        shared[0, :] = 1                       # connects every column
        A = np.vstack([np.eye(n, dtype=np.uint8), shared])
        e = np.ones(n, np.uint8)
        s = (A.astype(np.int64).dot(e) % 2).astype(np.uint8)
        dm = D.DEM(D.CSR.from_dense(A), D.CSR.from_rows([[0]], n), np.full(n, 0.1))
        soft = rng.normal(size=n)
        st, eb, cl, ncl, big = oracle.lsd(dm, soft, s, 0)
        assert st == 0 and ncl == 1 and big == n
        x = osd0(A, s, _rank_order(soft, range(n)))
        assert np.array_equal(eb, x)
        seen += 1
    assert seen == 30


@pytest.mark.parametrize("order", [1, 3, 5])
def test_lsd_order_search_is_min_weight_over_settings(order):
    dm = D.phenomenological_dem(5, 3, 0.02, 0.01)
    A = dm.H.to_dense()
    Ht = dm.H.transpose()
    l32, _ = oracle.prior_llr(dm.priors)
    rng = np.random.default_rng(order)
    improved = 0
    for _ in range(25):
        s, soft = _random_case(dm, rng, density=0.08)
        st0, eb0, cl0, _, _ = oracle.lsd(dm, soft, s, 0)
        st, eb, cl, _, _ = oracle.lsd(dm, soft, s, order)
        assert st == 0 and st0 == 0
        assert np.array_equal(cl, cl0), "the search does not change the clusters"
        assert np.array_equal(A.astype(np.int64).dot(eb) % 2, s)
        for r, cols in _clusters(cl).items():
            checks = sorted({int(c) for j in cols for c in Ht.row(j)})
            sub = A[np.ix_(checks, cols)].astype(np.uint8)
            rank_pos = sorted(range(len(cols)), key=lambda t: (soft[cols[t]], cols[t]))
            # free columns in rank order: those that are not pivots of OSD-0
            piv, basis = [], np.zeros((0, len(checks)), np.uint8)
            from tests.helpers import gf2_rank
            for t in rank_pos:
                trial = np.vstack([basis, sub[:, t]])
                if gf2_rank(trial) > len(basis):
                    basis = trial
                    piv.append(t)
            free = [t for t in rank_pos if t not in piv][:order]
            best = None
            for a in range(1 << len(free)):
                x = np.zeros(len(cols), np.uint8)
                for b, t in enumerate(free):
                    x[t] = (a >> b) & 1
                rhs = (s[checks].astype(np.int64) + sub.astype(np.int64).dot(x)) % 2
                xp = gf2_solve_one(sub[:, piv], rhs)
                x[piv] = xp
                idx = sorted(cols[t] for t in range(len(cols)) if x[t])
                w = f32_fold(l32[idx])
                if best is None or w < best[0]:
                    best = (w, x.copy())
            assert np.array_equal(eb[cols], best[1])
            w0 = f32_fold(l32[sorted(j for j in cols if eb0[j])])
            assert best[0] <= w0
            improved += best[0] < w0
    assert improved >= 1


def test_unsolvable_syndrome_is_reported():
    # two identical rows: any syndrome with s_0 != s_1 is outside the column span
    A = np.array([[1, 1, 0, 0], [1, 1, 0, 0], [0, 1, 1, 1]], np.uint8)
    H = D.CSR.from_dense(A)
    dm = D.DEM(H, D.CSR.from_rows([[0]], 4), np.full(4, 0.1))
    st, eb, cl, ncl, big = oracle.lsd(dm, np.zeros(4), np.array([1, 0, 0], np.uint8), 0)
    assert st == 1 and not eb.any()
    # the full decoder marks the shot and returns a zero correction
    syn = D.pack_bits(np.array([[1, 0, 0]], np.uint8))
    out = oracle.decode(dm, np.arange(4, dtype=np.uint32)[None], syn, 5, 0.625, 1)
    assert out["stats"]["status"][0] == 1 and not out["corrections"].any()


def test_lsd_prefers_reliable_columns():
    """A flipped check with two private columns: the column ranked more reliable is the answer."""
    A = np.array([[1, 1, 0, 0], [0, 0, 1, 1]], np.uint8)
    dm = D.DEM(D.CSR.from_dense(A), D.CSR.from_rows([[0]], 4), np.full(4, 0.1))
    s = np.array([1, 0], np.uint8)
    for favoured, other in [(0, 1), (1, 0)]:
        soft = np.ones(4)
        soft[favoured] = -1.0
        st, eb, cl, ncl, big = oracle.lsd(dm, soft, s, 0)
        assert eb[favoured] == 1 and eb[other] == 0 and big == 1 and ncl == 1
    # equal soft values: ties go to the lower column index
    st, eb, cl, ncl, big = oracle.lsd(dm, np.zeros(4), s, 0)
    assert list(eb) == [1, 0, 0, 0]
