"""Pins for the oracle's serial min-sum BP member (Appendix A, Algorithm 1).

What fixes the answer independently of the oracle:
  * a single parity check on two variables has a closed form;
  * on a tree-shaped Tanner graph, min-sum (alpha = 1) reaches the exact min-marginals
    L_v = C_1(v) - C_0(v), C_b(v) = min{sum_j lambda_j e_j : H e = s, e_v = b} (brute force);
  * variables that share no check commute, so any order that respects the dependency levels of a
    permutation gives bit-identical results (the wavefront claim the GPU path relies on);
  * s = 0 converges in the first iteration to e = 0;
  * a degree-1 check forces its variable (hard constraint).
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from tests.helpers import brute_force_costs


def _dem_from_dense(A, priors, L=None):
    H = D.CSR.from_dense(np.asarray(A, np.uint8))
    if L is None:
        L = D.CSR.from_rows([[0]], H.ncols)
    return D.DEM(H, L, np.asarray(priors, np.float64))


def _lam64(priors):
    return np.log((1 - np.asarray(priors)) / np.asarray(priors))


@pytest.mark.parametrize("s", [0, 1])
def test_single_check_two_variables_closed_form(s):
    priors = [0.1, 0.02]
    dm = _dem_from_dense([[1, 1]], priors)
    l32, l64 = oracle.prior_llr(priors)
    # alpha = 1, natural order: v0 sees lambda_1 through the check, then v1 sees v0's fresh message
    t, post, eb = oracle.bp_member(dm, np.array([s], np.uint8), np.array([0, 1]), 1, 1.0, oracle.FP64,
                                   early_stop=False)
    sign = -1.0 if s else 1.0
    assert post[0] == pytest.approx(l64[0] + sign * l64[1], abs=1e-12)
    assert post[1] == pytest.approx(l64[1] + sign * l64[0], abs=1e-12)
    # FP32: one multiply (alpha * min, exact for alpha = 1) and one add, each rounded once
    t, post32, _ = oracle.bp_member(dm, np.array([s], np.uint8), np.array([0, 1]), 1, 1.0, oracle.FP32,
                                    early_stop=False)
    assert np.float32(post32[0]) == np.float32(l32[0] + np.float32(sign) * l32[1])
    # with s = 1 the likelier single flip (larger p, smaller lambda) is chosen: e = (1, 0)
    if s:
        assert list(eb) == [1, 0]


def _random_tree(rng, nvar, max_check_deg=4):
    """Random bipartite tree in which every check has degree >= 2."""
    checks = []
    var_count = 1
    while var_count < nvar:
        anchor = int(rng.integers(0, var_count))
        k = int(min(rng.integers(1, max_check_deg), nvar - var_count))
        new = list(range(var_count, var_count + k))
        var_count += k
        checks.append([anchor] + new)
    A = np.zeros((len(checks), nvar), np.uint8)
    for r, c in enumerate(checks):
        A[r, c] = 1
    return A


@pytest.mark.parametrize("seed", range(12))
def test_tree_exact_min_marginals(seed):
    rng = np.random.default_rng(seed)
    nvar = int(rng.integers(4, 14))
    A = _random_tree(rng, nvar)
    priors = rng.uniform(0.01, 0.3, size=nvar)
    dm = _dem_from_dense(A, priors)
    lam = _lam64(priors)
    e = (rng.random(nvar) < 0.3).astype(np.uint8)
    s = A.dot(e) % 2
    sols = brute_force_costs(A, lam, s)
    exact = np.zeros(nvar)
    for v in range(nvar):
        c1 = min(c for c, x in sols if x[v] == 1)
        c0 = min(c for c, x in sols if x[v] == 0)
        exact[v] = c1 - c0
    perm = rng.permutation(nvar)
    for mode, tol in [(oracle.FP64, 1e-9), (oracle.FP32, 2e-5)]:
        _, post, _ = oracle.bp_member(dm, s.astype(np.uint8), perm, 2 * nvar + 2, 1.0, mode, early_stop=False)
        scale = np.abs(lam).sum()
        assert np.max(np.abs(post - exact)) <= tol * scale, (mode, post, exact)


def test_path_graph_min_marginals_any_order():
    """A repetition-code chain: variables 0..n-1, checks on neighbours."""
    n = 9
    A = np.zeros((n - 1, n), np.uint8)
    for i in range(n - 1):
        A[i, i] = A[i, i + 1] = 1
    priors = np.linspace(0.02, 0.2, n)
    dm = _dem_from_dense(A, priors)
    lam = _lam64(priors)
    s = np.zeros(n - 1, np.uint8)
    s[2] = 1
    s[6] = 1
    sols = brute_force_costs(A, lam, s)
    exact = np.array([min(c for c, x in sols if x[v]) - min(c for c, x in sols if not x[v]) for v in range(n)])
    for order in [np.arange(n), np.arange(n)[::-1], np.random.default_rng(1).permutation(n)]:
        _, post, _ = oracle.bp_member(dm, s, order, 2 * n, 1.0, oracle.FP64, early_stop=False)
        assert np.allclose(post, exact, atol=1e-9)


def _levels(dm, perm):
    """Dependency level of each variable: 1 + max level of earlier variables sharing a check."""
    last = np.full(dm.m, -1)
    Ht = dm.H.transpose()
    lev = np.zeros(dm.n, np.int64)
    for v in perm:
        cs = Ht.row(int(v))
        lv = 1 + (max(last[c] for c in cs) if len(cs) else -1)
        lev[v] = lv
        for c in cs:
            last[c] = lv
    return lev


@pytest.mark.parametrize("mode", [oracle.FP32, oracle.FP16MSG])
def test_wavefront_order_is_bit_identical(mode):
    dm = D.build_workload("cc666_d9_pheno")
    rng = np.random.default_rng(3)
    syn, _ = D.sample(dm, 6, 17)
    sb = D.unpack_bits(syn, dm.m)
    for trial in range(3):
        perm = rng.permutation(dm.n)
        lev = _levels(dm, perm)
        # re-order: by level, random order inside each level
        keys = lev * dm.n + rng.permutation(dm.n)
        wave = np.argsort(keys, kind="stable")
        assert not np.array_equal(wave, perm)
        for s in sb:
            a = oracle.bp_member(dm, s, perm, 7, 0.625, mode, early_stop=False)
            b = oracle.bp_member(dm, s, wave, 7, 0.625, mode, early_stop=False)
            assert a[0] == b[0]
            assert np.array_equal(a[1].view(np.uint64), b[1].view(np.uint64))


def test_level_violating_order_differs():
    """Control for the test above: an order that breaks the levels changes the floats."""
    dm = D.build_workload("cc666_d9_pheno")
    syn, _ = D.sample(dm, 20, 17)
    sb = D.unpack_bits(syn, dm.m)
    perm = np.random.default_rng(4).permutation(dm.n)
    other = np.random.default_rng(5).permutation(dm.n)
    diff = 0
    for s in sb:
        a = oracle.bp_member(dm, s, perm, 5, 0.625, oracle.FP32, early_stop=False)
        b = oracle.bp_member(dm, s, other, 5, 0.625, oracle.FP32, early_stop=False)
        diff += not np.array_equal(a[1], b[1])
    assert diff > 0


def test_zero_syndrome_converges_immediately():
    dm = D.build_workload("cc666_d9_pheno")
    for mode in [oracle.FP32, oracle.FP16MSG, oracle.FP64]:
        t, post, eb = oracle.bp_member(dm, np.zeros(dm.m, np.uint8), np.arange(dm.n), 30, 0.625, mode)
        assert t == 1 and not eb.any() and (post > 0).all()


def test_degree_one_check_is_hard_constraint():
    # v0 alone in check 1: its posterior must be -inf when s_1 = 1 and +inf when s_1 = 0
    A = [[1, 1, 0], [1, 0, 0], [0, 1, 1]]
    dm = _dem_from_dense(A, [0.1, 0.1, 0.1])
    for s1 in [0, 1]:
        s = np.array([s1, s1, 0], np.uint8)
        t, post, eb = oracle.bp_member(dm, s, np.arange(3), 5, 0.625, oracle.FP32)
        assert post[0] == (-np.inf if s1 else np.inf)
        assert eb[0] == s1 and t >= 1


def test_scaling_factor_matters():
    """alpha = 0.625 and alpha = 1 give different posteriors (the factor is applied)."""
    dm = D.build_workload("cc666_d5_codecap")
    s = np.zeros(dm.m, np.uint8)
    s[[0, 3]] = 1
    a = oracle.bp_member(dm, s, np.arange(dm.n), 3, 0.625, oracle.FP32, early_stop=False)[1]
    b = oracle.bp_member(dm, s, np.arange(dm.n), 3, 1.0, oracle.FP32, early_stop=False)[1]
    assert not np.array_equal(a, b)
