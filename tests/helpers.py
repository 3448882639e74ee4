"""Small independent helpers for the tests: GF(2) algebra and brute force, in plain numpy/Python."""
import itertools

import numpy as np


def gf2_rank(A):
    A = (np.array(A, dtype=np.uint8) % 2).copy()
    rows, cols = A.shape
    r = 0
    for c in range(cols):
        piv = [i for i in range(r, rows) if A[i, c]]
        if not piv:
            continue
        p = piv[0]
        A[[r, p]] = A[[p, r]]
        for i in range(rows):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        r += 1
        if r == rows:
            break
    return r


def gf2_nullspace(A):
    """Basis (rows) of {x : A x = 0 mod 2}."""
    A = (np.array(A, dtype=np.uint8) % 2).copy()
    rows, cols = A.shape
    pivcols = []
    r = 0
    for c in range(cols):
        piv = [i for i in range(r, rows) if A[i, c]]
        if not piv:
            continue
        p = piv[0]
        A[[r, p]] = A[[p, r]]
        for i in range(rows):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        pivcols.append(c)
        r += 1
        if r == rows:
            break
    free = [c for c in range(cols) if c not in pivcols]
    basis = []
    for f in free:
        x = np.zeros(cols, np.uint8)
        x[f] = 1
        for i, pc in enumerate(pivcols):
            x[pc] = A[i, f]
        basis.append(x)
    return np.array(basis, dtype=np.uint8).reshape(len(basis), cols)


def gf2_solve_one(A, s):
    """Some x with A x = s (mod 2), or None."""
    A = np.array(A, dtype=np.uint8) % 2
    aug = np.concatenate([A, np.array(s, dtype=np.uint8).reshape(-1, 1)], axis=1)
    rows, cols = A.shape
    r = 0
    pivcols = []
    for c in range(cols):
        piv = [i for i in range(r, rows) if aug[i, c]]
        if not piv:
            continue
        p = piv[0]
        aug[[r, p]] = aug[[p, r]]
        for i in range(rows):
            if i != r and aug[i, c]:
                aug[i] ^= aug[r]
        pivcols.append(c)
        r += 1
        if r == rows:
            break
    if aug[r:, cols].any():
        return None
    x = np.zeros(cols, np.uint8)
    for i, pc in enumerate(pivcols):
        x[pc] = aug[i, cols]
    return x


def osd0(A, s, col_order):
    """OSD-0: eliminate columns of A in col_order, pivots = first independent, free columns = 0.

    Returns x (over the original column indices) or None if s is not in the column span."""
    A = np.array(A, dtype=np.uint8) % 2
    order = list(col_order)
    B = A[:, order]
    aug = np.concatenate([B, np.array(s, dtype=np.uint8).reshape(-1, 1)], axis=1)
    rows, cols = B.shape
    r = 0
    piv = {}
    for c in range(cols):
        if r == rows:
            break
        cand = [i for i in range(r, rows) if aug[i, c]]
        if not cand:
            continue
        p = cand[0]
        aug[[r, p]] = aug[[p, r]]
        for i in range(rows):
            if i != r and aug[i, c]:
                aug[i] ^= aug[r]
        piv[c] = r
        r += 1
    if aug[r:, cols].any():
        return None
    x = np.zeros(A.shape[1], np.uint8)
    for c, row in piv.items():
        x[order[c]] = aug[row, cols]
    return x


def f32_fold(values):
    """Left fold of float32 additions starting from +0.0, in the given order."""
    acc = np.float32(0.0)
    for v in values:
        acc = np.float32(acc + np.float32(v))
    return acc


def brute_force_costs(H, lam, s):
    """All solutions e of H e = s by enumeration (n <= ~20), with costs sum lam_j e_j (float64)."""
    H = np.array(H, dtype=np.uint8)
    n = H.shape[1]
    sols = []
    for bits in itertools.product((0, 1), repeat=n):
        e = np.array(bits, np.uint8)
        if np.array_equal(H.dot(e) % 2, np.asarray(s) % 2):
            sols.append((float(np.dot(lam, e)), e))
    return sols


def coset_min_weight(A, lam, s):
    """Minimum of sum lam_j e_j over the coset {e : A e = s}, by enumerating e0 + ker(A)."""
    e0 = gf2_solve_one(A, s)
    assert e0 is not None
    N = gf2_nullspace(A)
    k = N.shape[0]
    best = float(np.dot(lam, e0))
    chunk = 1 << 12
    for start in range(0, 1 << k, chunk):
        idx = np.arange(start, min(1 << k, start + chunk), dtype=np.int64)
        coeff = ((idx[:, None] >> np.arange(k)) & 1).astype(np.int64)
        X = (coeff @ N.astype(np.int64) + e0) % 2
        best = min(best, float((X @ lam).min()))
    return best
