"""Pins for the oracle's layered-schedule member (reading R10: row-layered min-sum with greedy check
layers; the paper names layered schedules as a middle ground between serial and parallel updates).

What fixes the answer independently of the oracle:
  * the layers, recomputed here from their definition: no two checks of a layer share a variable,
    and a check sits in layer l only if every lower layer holds an earlier check sharing a variable
    with it (greedy colouring in ascending check order);
  * a single parity check on two variables: one iteration is one exchange (closed form);
  * trees (alpha = 1): exact min-marginals C_1(v) - C_0(v) after enough iterations (brute force);
  * a dependency horizon on a chain, whose greedy layers alternate: after t iterations the first
    variable's posterior depends on exactly the first 2t variables and 2t - 1 checks -- twice the
    flooding horizon, because the second layer already sees the first layer's update;
  * when no two checks share a variable there is one layer and the schedule is the flooding one.
"""
import numpy as np
import pytest

import oracle
from paper_2508_15743_gb300 import dem as D
from tests.helpers import brute_force_costs


def _dem_from_dense(A, priors):
    H = D.CSR.from_dense(np.asarray(A, np.uint8))
    return D.DEM(H, D.CSR.from_rows([[0]], H.ncols), np.asarray(priors, np.float64))


def _chain(n):
    A = np.zeros((n - 1, n), np.uint8)
    for i in range(n - 1):
        A[i, i] = A[i, i + 1] = 1
    return A


@pytest.mark.parametrize("name", ["cc666_d5_codecap", "cc666_d9_pheno"])
def test_layers_follow_their_definition(name):
    dm = D.build_workload(name)
    A = dm.H.to_dense().astype(bool)
    lay, nl = oracle.check_layers(dm)
    assert nl == lay.max() + 1
    share = (A.astype(np.int32) @ A.T.astype(np.int32)) > 0
    for c in range(dm.m):
        same = np.nonzero(lay == lay[c])[0]
        assert not any(share[c, o] for o in same if o != c)              # a layer shares no variable
        for l in range(lay[c]):                                          # greedy: every lower layer is blocked
            assert any(share[c, o] and lay[o] == l for o in range(c))


def test_colour_code_plaquettes_form_three_layers():
    """Plaquettes of one colour are disjoint; the greedy layers of the d=5 code-capacity code are the colours."""
    dm = D.build_workload("cc666_d5_codecap")
    lay, nl = oracle.check_layers(dm)
    assert nl == 3


@pytest.mark.parametrize("s", [0, 1])
def test_single_check_two_variables_one_iteration(s):
    priors = [0.1, 0.02]
    dm = _dem_from_dense([[1, 1]], priors)
    lam = np.log((1 - np.array(priors)) / np.array(priors))
    _, post, _ = oracle.bp_member_layered(dm, np.array([s], np.uint8), 1, 0.625, oracle.FP64, early_stop=False)
    sign = -1.0 if s else 1.0
    assert post[0] == pytest.approx(lam[0] + sign * 0.625 * lam[1], abs=1e-12)
    assert post[1] == pytest.approx(lam[1] + sign * 0.625 * lam[0], abs=1e-12)


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
    rng = np.random.default_rng(300 + seed)
    nvar = int(rng.integers(4, 14))
    A = _random_tree(rng, nvar)
    priors = rng.uniform(0.01, 0.3, size=nvar)
    dm = _dem_from_dense(A, priors)
    lam = np.log((1 - priors) / priors)
    e = (rng.random(nvar) < 0.3).astype(np.uint8)
    s = (A.dot(e) % 2).astype(np.uint8)
    sols = brute_force_costs(A, lam, s)
    exact = np.array([min(c for c, x in sols if x[v] == 1) - min(c for c, x in sols if x[v] == 0)
                      for v in range(nvar)])
    for mode, tol in [(oracle.FP64, 1e-9), (oracle.FP32, 2e-5)]:
        _, post, _ = oracle.bp_member_layered(dm, s, 2 * nvar + 2, 1.0, mode, early_stop=False)
        assert np.max(np.abs(post - exact)) <= tol * np.abs(lam).sum(), (mode, post, exact)


@pytest.mark.parametrize("mode", [oracle.FP64, oracle.FP32])
@pytest.mark.parametrize("t", [1, 2, 3])
def test_chain_horizon_is_twice_the_iterations(t, mode):
    n = 14
    A = _chain(n)
    lay, nl = oracle.check_layers(_dem_from_dense(A, np.full(n, 0.1)))
    assert nl == 2 and np.array_equal(lay, np.arange(n - 1) % 2)
    rng = np.random.default_rng(10 + t)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    base = rng.uniform(0.02, 0.3, n)
    h = 2 * t          # variables 0 .. h-1 and checks 0 .. h-2 can matter
    _, p0, _ = oracle.bp_member_layered(_dem_from_dense(A, base), s, t, 0.625, mode, early_stop=False)
    far = base.copy()
    far[h:] = rng.uniform(0.02, 0.3, n - h)
    s2 = s.copy()
    s2[h - 1:] ^= 1
    _, p1, _ = oracle.bp_member_layered(_dem_from_dense(A, far), s2, t, 0.625, mode, early_stop=False)
    assert p0[0] == p1[0]
    # and the last variable inside the horizon does matter: with s = 0 every message is positive and
    # each check passes on its other variable's message scaled by alpha
    z = np.zeros(n - 1, np.uint8)
    pr = np.linspace(0.05, 0.2, n)
    moved = pr.copy()
    moved[h - 1] = 0.01
    _, q0, _ = oracle.bp_member_layered(_dem_from_dense(A, pr), z, t, 0.625, mode, early_stop=False)
    _, q1, _ = oracle.bp_member_layered(_dem_from_dense(A, moved), z, t, 0.625, mode, early_stop=False)
    assert q0[0] != q1[0]
    # flooding reaches only variables 0 .. t in t iterations, short of variable 2t - 1 once t >= 2
    if t >= 2:
        _, f0, _ = oracle.bp_member_flood(_dem_from_dense(A, pr), z, t, 0.625, mode, early_stop=False)
        _, f1, _ = oracle.bp_member_flood(_dem_from_dense(A, moved), z, t, 0.625, mode, early_stop=False)
        assert f0[0] == f1[0]


@pytest.mark.parametrize("mode", [oracle.FP32, oracle.FP64, oracle.FP16MSG])
def test_disjoint_checks_reduce_to_flooding(mode):
    """No variable in two checks: one layer, and the layered iteration is the flooding one."""
    rng = np.random.default_rng(5)
    A = np.zeros((4, 13), np.uint8)
    cols = rng.permutation(13)
    for r, chunk in enumerate(np.array_split(cols[:12], 4)):
        A[r, chunk] = 1
    A[0, cols[12]] = 1
    priors = rng.uniform(0.02, 0.3, 13)
    dm = _dem_from_dense(A, priors)
    assert oracle.check_layers(dm)[1] == 1
    for trial in range(8):
        s = rng.integers(0, 2, 4).astype(np.uint8)
        a = oracle.bp_member_layered(dm, s, 5, 0.625, mode, early_stop=False)
        b = oracle.bp_member_flood(dm, s, 5, 0.625, mode, early_stop=False)
        assert np.array_equal(a[1], b[1])


def test_zero_syndrome_converges_in_one_iteration():
    dm = D.build_workload("cc666_d5_codecap")
    t, post, eb = oracle.bp_member_layered(dm, np.zeros(dm.m, np.uint8), 10, 0.625, oracle.FP32)
    assert t == 1 and not eb.any()


def test_layered_converges_validly_and_differs_from_other_schedules():
    dm = D.build_workload("cc666_d9_pheno")
    syn, _ = D.sample(dm, 150, 19)
    bits = D.unpack_bits(syn, dm.m).astype(np.uint8)
    Hd = dm.H.to_dense()
    differ_f = differ_s = conv = 0
    for b in bits:
        t_l, pl, el = oracle.bp_member_layered(dm, b, 30, 0.625, oracle.FP32)
        t_f, pf, _ = oracle.bp_member_flood(dm, b, 30, 0.625, oracle.FP32)
        t_s, ps, _ = oracle.bp_member(dm, b, np.arange(dm.n), 30, 0.625, oracle.FP32)
        if t_l:
            conv += 1
            assert np.array_equal(Hd.dot(el) % 2, b)
        differ_f += int(t_l != t_f or not np.array_equal(pl, pf))
        differ_s += int(t_l != t_s or not np.array_equal(pl, ps))
    assert conv > 50 and differ_f > 0 and differ_s > 0


def test_fp16_storage_rounds_only_the_stored_messages():
    n = 6
    A = _chain(n)
    lam = np.array([1.0, 2.0, 1.5, 3.0, 2.5, 1.25])
    priors = 1.0 / (1.0 + np.exp(lam))
    dm = _dem_from_dense(A, priors)
    s = np.array([1, 0, 0, 1, 0], np.uint8)
    l32, _ = oracle.prior_llr(priors)
    if not np.all(np.float16(l32) == l32):
        pytest.skip("prior LLRs not exact in binary16 on this platform's log")
    _, a, _ = oracle.bp_member_layered(dm, s, 6, 1.0, oracle.FP32, early_stop=False)
    _, b, _ = oracle.bp_member_layered(dm, s, 6, 1.0, oracle.FP16MSG, early_stop=False)
    assert np.array_equal(a, b)
