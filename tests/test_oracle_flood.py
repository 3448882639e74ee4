"""Pins for the oracle's parallel-schedule (flooding) member, Algorithm 1's other branch (reading R8).

What fixes the answer independently of the oracle:
  * a single parity check on two variables: after one iteration each posterior is its prior plus the
    other variable's prior, signed by the syndrome and scaled by alpha (one message exchange);
  * on a tree-shaped Tanner graph, flooding min-sum (alpha = 1) reaches the exact min-marginals
    C_1(v) - C_0(v) after enough iterations (brute force), like the serial schedule;
  * locality: after t flooding iterations a variable's posterior depends only on the priors and
    syndrome bits within 2t hops of it in the Tanner graph (messages move one check and one variable
    per iteration). A serial sweep can carry information along a whole path in one iteration, so this
    pin separates the two schedules;
  * the flooding result does not depend on any processing order.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from tests.helpers import brute_force_costs


def _dem_from_dense(A, priors):
    H = D.CSR.from_dense(np.asarray(A, np.uint8))
    return D.DEM(H, D.CSR.from_rows([[0]], H.ncols), np.asarray(priors, np.float64))


def _lam64(priors):
    p = np.asarray(priors)
    return np.log((1 - p) / p)


@pytest.mark.parametrize("s", [0, 1])
@pytest.mark.parametrize("alpha", [1.0, 0.625])
def test_single_check_two_variables_one_iteration(s, alpha):
    """One exchange: each variable receives (-1)^s * alpha * (the other's prior)."""
    priors = [0.1, 0.02]
    dm = _dem_from_dense([[1, 1]], priors)
    lam = _lam64(priors)
    _, post, _ = oracle.bp_member_flood(dm, np.array([s], np.uint8), 1, alpha, oracle.FP64, early_stop=False)
    sign = -1.0 if s else 1.0
    assert post[0] == pytest.approx(lam[0] + sign * alpha * lam[1], abs=1e-12)
    assert post[1] == pytest.approx(lam[1] + sign * alpha * lam[0], abs=1e-12)
    # FP32: one multiply (alpha * min) and one add, each rounded once
    l32, _ = oracle.prior_llr(priors)
    _, p32, _ = oracle.bp_member_flood(dm, np.array([s], np.uint8), 1, alpha, oracle.FP32, early_stop=False)
    mag = np.float32(alpha) * np.float32(l32[1])
    assert np.float32(p32[0]) == np.float32(l32[0]) + (-mag if s else mag)


def _random_tree(rng, nvar, max_check_deg=4):
    checks, var_count = [], 1
    while var_count < nvar:
        anchor = int(rng.integers(0, var_count))
        k = int(min(rng.integers(1, max_check_deg), nvar - var_count))
        checks.append([anchor] + list(range(var_count, var_count + k)))
        var_count += k
    A = np.zeros((len(checks), nvar), np.uint8)
    for r, c in enumerate(checks):
        A[r, c] = 1
    return A


@pytest.mark.parametrize("seed", range(10))
def test_tree_exact_min_marginals(seed):
    rng = np.random.default_rng(100 + seed)
    nvar = int(rng.integers(4, 14))
    A = _random_tree(rng, nvar)
    priors = rng.uniform(0.01, 0.3, size=nvar)
    dm = _dem_from_dense(A, priors)
    lam = _lam64(priors)
    e = (rng.random(nvar) < 0.3).astype(np.uint8)
    s = (A.dot(e) % 2).astype(np.uint8)
    sols = brute_force_costs(A, lam, s)
    exact = np.array([min(c for c, x in sols if x[v] == 1) - min(c for c, x in sols if x[v] == 0)
                      for v in range(nvar)])
    for mode, tol in [(oracle.FP64, 1e-9), (oracle.FP32, 2e-5)]:
        _, post, _ = oracle.bp_member_flood(dm, s, 2 * nvar + 2, 1.0, mode, early_stop=False)
        assert np.max(np.abs(post - exact)) <= tol * np.abs(lam).sum(), (mode, post, exact)


def _chain(n):
    A = np.zeros((n - 1, n), np.uint8)
    for i in range(n - 1):
        A[i, i] = A[i, i + 1] = 1
    return A


@pytest.mark.parametrize("t", [1, 2, 3])
def test_locality_after_t_iterations(t):
    """Variable 0 of a chain: after t iterations only variables 0..t and checks 0..t-1 can matter."""
    n = 12
    A = _chain(n)
    rng = np.random.default_rng(t)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    base = rng.uniform(0.02, 0.3, n)
    _, p0, _ = oracle.bp_member_flood(_dem_from_dense(A, base), s, t, 0.625, oracle.FP64, early_stop=False)
    far = base.copy()
    far[t + 1:] = rng.uniform(0.02, 0.3, n - t - 1)      # change every prior beyond distance t
    s2 = s.copy()
    s2[t:] ^= 1                                         # and every syndrome bit beyond check t-1
    _, p1, _ = oracle.bp_member_flood(_dem_from_dense(A, far), s2, t, 0.625, oracle.FP64, early_stop=False)
    assert p0[0] == p1[0]
    # the serial schedule in natural order is not local: the same change moves variable 0's posterior
    # within one iteration when the order runs from the far end
    order = np.arange(n)[::-1]
    _, q0, _ = oracle.bp_member(_dem_from_dense(A, base), s, order, 1, 0.625, oracle.FP64, early_stop=False)
    _, q1, _ = oracle.bp_member(_dem_from_dense(A, far), s2, order, 1, 0.625, oracle.FP64, early_stop=False)
    assert q0[0] != q1[0]


def test_flooding_differs_from_serial_and_converges_on_colour_code():
    dm = D.build_workload("cc666_d5_codecap")
    syn, _ = D.sample(dm, 200, 9)
    bits = D.unpack_bits(syn, dm.m).astype(np.uint8)
    differ = 0
    for b in bits:
        t_f, pf, ef = oracle.bp_member_flood(dm, b, 20, 0.625, oracle.FP32)
        t_s, ps, es = oracle.bp_member(dm, b, np.arange(dm.n), 20, 0.625, oracle.FP32)
        if t_f:   # a converged decision satisfies the syndrome
            assert np.array_equal(dm.H.to_dense().dot(ef) % 2, b)
        differ += int(t_f != t_s or not np.array_equal(pf, ps))
    assert differ > 0


def test_zero_syndrome_converges_in_one_iteration():
    dm = D.build_workload("cc666_d5_codecap")
    t, post, eb = oracle.bp_member_flood(dm, np.zeros(dm.m, np.uint8), 10, 0.625, oracle.FP32)
    assert t == 1 and not eb.any()


def test_fp16_storage_rounds_only_the_stored_messages():
    """With priors whose LLRs are exact in binary16 and alpha = 1 on a short chain, every stored
    message is a sum of a few of them and stays exact: FP16 storage then equals FP32."""
    n = 6
    A = _chain(n)
    lam = np.array([1.0, 2.0, 1.5, 3.0, 2.5, 1.25])
    priors = 1.0 / (1.0 + np.exp(lam))
    dm = _dem_from_dense(A, priors)
    s = np.array([1, 0, 0, 1, 0], np.uint8)
    l32, _ = oracle.prior_llr(priors)
    if not np.all(np.float16(l32) == l32):
        pytest.skip("prior LLRs not exact in binary16 on this platform's log")
    _, a, _ = oracle.bp_member_flood(dm, s, 6, 1.0, oracle.FP32, early_stop=False)
    _, b, _ = oracle.bp_member_flood(dm, s, 6, 1.0, oracle.FP16MSG, early_stop=False)
    assert np.array_equal(a, b)
