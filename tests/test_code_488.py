"""Pins for the square-octagon (4.8.8) triangular colour code generator (dem.color_code_488).

Facts from Sec. II.A: a triangular colour code has n qubits, (n-1)/2 plaquettes, each an even-weight
X and Z generator; the generators commute, n-1 of them are independent (k = 1), and the tiling is
three-colourable. On the 4.8.8 tiling the plaquettes are squares and octagons in the bulk and
quadrilaterals on the boundary. The distance-d family has n = (d^2 + 2d - 1)/2 (7, 17, 31, 49, ...;
d = 3 is the 7-qubit Steane code). Nothing here re-derives the construction: the checks are the code's
parameters, the tiling's local structure and a brute-force distance.
"""
import itertools
from collections import defaultdict

import numpy as np
import pytest

from paper_2508_15743_gb300 import dem as D
from tests.helpers import gf2_nullspace, gf2_rank

DS = [3, 5, 7, 9, 11, 13, 15]


def dense(d):
    H, logical, coords, colours = D.color_code_488(d)
    return H.to_dense().astype(np.int64), logical, coords, colours


@pytest.mark.parametrize("d", DS)
def test_counts_and_membership(d):
    A, logical, _, colours = dense(d)
    n = A.shape[1]
    assert n == (d * d + 2 * d - 1) // 2
    assert A.shape[0] == (n - 1) // 2
    w = A.sum(axis=1)
    assert set(w.tolist()) <= {4, 8}
    assert (w[colours == 2] == 4).all(), "squares"
    # triangular colour code: 3 corner qubits in one plaquette, d-2 more per side in two, bulk in three
    per_qubit = A.sum(axis=0)
    assert (per_qubit == 1).sum() == 3
    assert (per_qubit == 2).sum() == 3 * (d - 2)
    assert (per_qubit == 3).sum() == n - 3 * (d - 1)
    assert len(logical) == d


@pytest.mark.parametrize("d", DS)
def test_three_colouring(d):
    A, _, _, colours = dense(d)
    for q in range(A.shape[1]):
        cs = colours[np.nonzero(A[:, q])[0]]
        assert len(set(cs.tolist())) == len(cs), "plaquettes sharing a qubit have different colours"


@pytest.mark.parametrize("d", [5, 7, 9, 11])
def test_bulk_is_the_square_octagon_tiling(d):
    """Two qubits are neighbours in the tiling when they share two plaquettes. Every bulk qubit has
    three neighbours (the tiling is 3-regular), and the qubits of a plaquette made only of bulk
    qubits form one cycle of its length: a square (4) or an octagon (8)."""
    A, _, _, _ = dense(d)
    n = A.shape[1]
    shared = A.T @ A
    nb = [set(np.nonzero((shared[q] >= 2) & (np.arange(n) != q))[0].tolist()) for q in range(n)]
    bulk = A.sum(axis=0) == 3
    assert all(len(nb[q]) == 3 for q in range(n) if bulk[q])
    cycles = 0
    for r in range(A.shape[0]):
        qs = np.nonzero(A[r])[0].tolist()
        if not all(bulk[q] for q in qs):
            continue
        inside = {q: nb[q] & set(qs) for q in qs}
        assert all(len(v) == 2 for v in inside.values())
        seen, cur, prev = {qs[0]}, qs[0], None
        while True:   # walk the cycle
            nxt = [x for x in inside[cur] if x != prev][0]
            if nxt == qs[0]:
                break
            seen.add(nxt)
            prev, cur = cur, nxt
        assert len(seen) == len(qs)
        cycles += 1
    if d >= 7:
        assert cycles > 0


@pytest.mark.parametrize("d", [3, 5, 7, 9, 11])
def test_algebra(d):
    A, logical, _, _ = dense(d)
    n = A.shape[1]
    assert not ((A @ A.T) % 2).any(), "plaquettes overlap evenly (X and Z generators commute)"
    r = gf2_rank(A)
    assert r == (n - 1) // 2 and n - 2 * r == 1
    Lv = np.zeros(n, np.uint8)
    Lv[logical] = 1
    assert not (A @ Lv % 2).any(), "logical commutes with every plaquette"
    assert gf2_rank(np.vstack([A, Lv])) == r + 1, "logical is not a product of plaquettes"


def test_d3_is_the_steane_code():
    A, _, _, _ = dense(3)
    assert A.shape == (3, 7)
    ov = A @ A.T
    assert (np.diag(ov) == 4).all() and (ov[~np.eye(3, dtype=bool)] == 2).all()
    assert (A.prod(axis=0) == 1).sum() == 1, "one qubit in all three plaquettes"


@pytest.mark.parametrize("d", [3, 5, 7])
def test_distance_by_enumeration(d):
    """Minimum weight of x in ker(H) with odd overlap with the logical equals d."""
    A, logical, _, _ = dense(d)
    N = gf2_nullspace(A.astype(np.uint8))
    Lv = np.zeros(A.shape[1], np.uint8)
    Lv[logical] = 1
    k = N.shape[0]
    best = 10 ** 9
    for start in range(0, 1 << k, 1 << 14):
        idx = np.arange(start, min(1 << k, start + (1 << 14)), dtype=np.int64)
        coeff = ((idx[:, None] >> np.arange(k)) & 1).astype(np.int64)
        X = (coeff @ N.astype(np.int64)) % 2
        odd = (X @ Lv) % 2 == 1
        if odd.any():
            best = min(best, int(X[odd].sum(axis=1).min()))
    assert best == d


def test_distance_9_meet_in_the_middle():
    """d = 9: no odd-weight x in ker(H) of weight 1, 3, 5 or 7 (with k = 1 the all-ones vector is the
    other logical, so exactly the odd-weight kernel vectors are logical operators), and the weight-9
    boundary logical exists."""
    A, logical, _, _ = dense(9)
    n = A.shape[1]
    ones = np.ones(n, np.uint8)
    assert not (A @ ones % 2).any() and gf2_rank(np.vstack([A, ones])) == gf2_rank(A) + 1
    cols = [int("".join(str(int(b)) for b in A[:, j]), 2) for j in range(n)]
    for w in (1, 3, 5, 7):
        a = w // 2
        table = defaultdict(list)
        for S in itertools.combinations(range(n), a):
            x = 0
            for j in S:
                x ^= cols[j]
            table[x].append(frozenset(S))
        for S in itertools.combinations(range(n), w - a):
            x = 0
            for j in S:
                x ^= cols[j]
            for T in table.get(x, ()):
                assert T & set(S), f"logical operator of weight {w} < 9"
    assert len(logical) == 9


def test_phenomenological_and_code_capacity_workloads():
    dm = D.build_workload("cc488_d9_pheno")
    n488 = (81 + 18 - 1) // 2
    mp = (n488 - 1) // 2
    assert dm.m == mp * 10 and dm.n == 9 * n488 + 9 * mp
    assert dm.k == 1 and len(dm.L.row(0)) == 9 * 9
    cc = D.build_workload("cc488_d5_codecap")
    assert cc.n == 17 and cc.m == 8
    assert np.array_equal(np.diff(cc.H.rowptr), D.color_code_488(5)[0].to_dense().sum(axis=1))
