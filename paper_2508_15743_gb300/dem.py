"""Seeded synthetic inputs: colour codes, detector error models, syndrome samples, schedules.

This module is the one piece shared by the CUDA path, its tests and the CPU oracle. It holds
none of the decoder's arithmetic: it builds check matrices H, logical matrices L and priors p_j
(the decoding problem of Sec. II.B, Eq. 1), draws errors e ~ Bernoulli(p_j) and returns
s = H e mod 2 and obs = L e mod 2, and draws the K random variable permutations of the offline
setup (Sec. III.D.1, step 3). Log-likelihood ratios, BP and LSD live on each side separately.

Matrices are returned as CSR with int32 index arrays, columns ascending within each row.
Bit-packed vectors use little-endian bit order inside uint32 words (bit b of word w is entry
32*w + b) and zero padding bits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Neighbour offsets of a point of the triangular lattice, in (i, j) lattice coordinates where the
# point sits at i*(1, 0) + j*(1/2, sqrt(3)/2).
_TRI_NEIGHBOURS = ((1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1))


@dataclass
class CSR:
    """Sparse binary matrix in CSR form (int32 indices, columns ascending per row)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    colidx: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @staticmethod
    def from_rows(rows, ncols: int) -> "CSR":
        rowptr = np.zeros(len(rows) + 1, dtype=np.int32)
        for r, cols in enumerate(rows):
            rowptr[r + 1] = rowptr[r] + len(cols)
        colidx = np.zeros(int(rowptr[-1]), dtype=np.int32)
        for r, cols in enumerate(rows):
            colidx[rowptr[r]:rowptr[r + 1]] = np.sort(np.asarray(cols, dtype=np.int32))
        return CSR(len(rows), ncols, rowptr, colidx)

    @staticmethod
    def from_dense(a: np.ndarray) -> "CSR":
        a = np.asarray(a) % 2
        return CSR.from_rows([np.nonzero(r)[0] for r in a], a.shape[1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols), dtype=np.uint8)
        for r in range(self.nrows):
            out[r, self.colidx[self.rowptr[r]:self.rowptr[r + 1]]] = 1
        return out

    def row(self, r: int) -> np.ndarray:
        return self.colidx[self.rowptr[r]:self.rowptr[r + 1]]

    def transpose(self) -> "CSR":
        cols = [[] for _ in range(self.ncols)]
        for r in range(self.nrows):
            for c in self.row(r):
                cols[c].append(r)
        return CSR.from_rows(cols, self.nrows)


@dataclass
class DEM:
    """A decoding problem: check matrix H (m detectors x n mechanisms), logicals L (k x n), priors p."""

    H: CSR
    L: CSR
    priors: np.ndarray  # float64[n], each in (0, 0.5)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.H.nrows

    @property
    def n(self) -> int:
        return self.H.ncols

    @property
    def k(self) -> int:
        return self.L.nrows


# --------------------------------------------------------------------------------------------
# Triangular 6.6.6 colour code (Sec. II.A)
# --------------------------------------------------------------------------------------------

def color_code_layout(d: int):
    """Lattice layout of the distance-d triangular 6.6.6 colour code.

    Plaquette centres are the points (i, j) of the triangular lattice with (i - j) = 0 mod 3; every
    other lattice point is a qubit (together they form the honeycomb's vertices). The code occupies
    the closed lattice triangle i >= 0, j >= -1, i + j <= 3(d-1)/2 - 1, whose three corners are
    qubits. A plaquette acts on its lattice neighbours inside the triangle: six in the bulk, four on
    the boundary. This gives n = (3d^2 + 1)/4 qubits and (n - 1)/2 plaquettes (Sec. II.A).

    Returns (qubits, plaquettes): lists of (i, j) coordinates, in the index order used everywhere.
    """
    if d < 3 or d % 2 == 0:
        raise ValueError("distance must be odd and >= 3")
    side = 3 * (d - 1) // 2
    a, b = 0, -1
    c = side + a + b
    pts = [(i, j) for j in range(b, c - a + 1) for i in range(a, c - j + 1)]
    qubits = [p for p in pts if (p[0] - p[1]) % 3 != 0]
    plaqs = [p for p in pts if (p[0] - p[1]) % 3 == 0]
    return qubits, plaqs


def color_code_666(d: int):
    """Triangular hexagonal-tiling colour code of odd distance d (layout in color_code_layout).

    Returns (H, L_support, coords): H the plaquette/qubit incidence as a CSR, L_support the sorted
    qubit indices of the weight-d logical on the j = -1 boundary, coords the (i, j) of each qubit.
    """
    qubits, plaq_pts = color_code_layout(d)
    qidx = {q: k for k, q in enumerate(qubits)}
    plaqs = []
    for (i, j) in plaq_pts:
        sup = sorted(qidx[(i + di, j + dj)] for di, dj in _TRI_NEIGHBOURS if (i + di, j + dj) in qidx)
        plaqs.append(sup)
    H = CSR.from_rows(plaqs, len(qubits))
    logical = sorted(qidx[q] for q in qubits if q[1] == -1)
    return H, np.asarray(logical, dtype=np.int32), qubits


# --------------------------------------------------------------------------------------------
# Triangular 4.8.8 (square-octagon) colour code (Sec. II.A)
# --------------------------------------------------------------------------------------------
#
# Built on the dual lattice, where the construction is a closed lattice path. The dual of the
# square-octagon tiling is the square lattice with both diagonals of every cell drawn: an octagon is a
# lattice point, a square is a cell centre, and each cell splits into four triangles, one per vertex
# of the tiling (a qubit). Coordinates are doubled so that all of them are integers: octagons at
# (2a, 2b), squares at (2a+1, 2b+1). Octagons are red when a + b is even and blue otherwise, squares
# green; the three colours are those of the plaquettes.
#
# A colour code with three boundaries is such a triangulated region with one extra "boundary vertex"
# per boundary, joined to every lattice point along its stretch of the region's boundary: a boundary
# stretch whose points carry two of the colours belongs to the third colour's boundary vertex. The
# qubits are the region's triangles (bulk qubits, in three plaquettes), one triangle per boundary edge
# (boundary qubits, in two) and one triangle at each of the three points where two stretches meet
# (corner qubits, in one). A plaquette is every qubit around its lattice point.
#
# The region of the distance-d code is bounded by a counterclockwise cycle of 3(d-2) lattice edges
# starting at the square centre (1, 1):
#   1. d-2 half-diagonal steps eastward in a zigzag through blue octagons at heights 0 and 2 (turning
#      north-east at height 0 and south-east at height 2, straight on through squares);
#   2. d-2 axis steps of a staircase through octagons, alternately west and north (west first when
#      the zigzag ended at height 2 mod 4, north first otherwise);
#   3. d-2 half-diagonal steps southward in a zigzag through red octagons at x = 0 and 2 (turning
#      south-east at x = 0 and south-west at x = 2) back to (1, 1).
# The region is made of the triangles the cycle winds around once; where the staircase touches a
# zigzag the region is pinched to a single point. Every octagon the cycle turns at holds either 90
# degrees of region (a weight-4 half octagon on the boundary) or 270 degrees (a whole octagon), and
# every square it passes straight through holds 180 degrees (a weight-4 square), so the plaquettes
# are quadrilaterals on the boundary and squares or octagons in the bulk. The result has
# n = (d^2 + 2d - 1)/2 qubits and (n - 1)/2 plaquettes of weight 4 or 8; tests/test_inputs.py pins
# the code parameters and the distance.

def _dual_cycle_488(d: int):
    steps = d - 2
    cyc = [(1, 1)]
    x, y = 1, 1
    dx, dy = 1, -1
    for _ in range(steps):                       # 1. zigzag east
        if x % 2 == 0:
            dx, dy = (1, 1) if y == 0 else (1, -1)
        x, y = x + dx, y + dy
        cyc.append((x, y))
    west = (y % 4) == 2
    for _ in range(steps):                       # 2. staircase
        x, y = (x - 2, y) if west else (x, y + 2)
        west = not west
        cyc.append((x, y))
    for _ in range(steps):                       # 3. zigzag south
        if x % 2 == 0:
            dx, dy = (1, -1) if x == 0 else (-1, -1)
        x, y = x + dx, y + dy
        cyc.append((x, y))
    if cyc[-1] != (1, 1):
        raise AssertionError("boundary cycle does not close")
    return cyc[:-1]


def _dual_colour(pt) -> int:
    """0 red octagon, 1 blue octagon, 2 green square."""
    if pt[0] % 2:
        return 2
    return (pt[0] // 2 + pt[1] // 2) % 2


def _winding(cyc, px: float, py: float) -> int:
    w = 0
    for k in range(len(cyc)):
        (x1, y1), (x2, y2) = cyc[k], cyc[(k + 1) % len(cyc)]
        if (y1 <= py < y2) or (y2 <= py < y1):
            if x1 + (py - y1) * (x2 - x1) / (y2 - y1) > px:
                w += 1 if y2 > y1 else -1
    return w


def color_code_488(d: int):
    """Triangular square-octagon colour code of odd distance d (construction in the comment above).

    Returns (H, L_support, coords, colours): H the plaquette/qubit incidence as a CSR, L_support the
    sorted qubit indices of a weight-d boundary logical (the qubits along the eastward zigzag, corners
    included), coords the dual-lattice position of each qubit (its triangle's centroid; a boundary
    qubit sits on its boundary edge, a corner qubit on its corner point), colours the plaquettes'
    colours (0 red, 1 blue, 2 green).
    """
    if d < 3 or d % 2 == 0:
        raise ValueError("distance must be odd and >= 3")
    cyc = _dual_cycle_488(d)
    F = len(cyc)
    xs = [p[0] for p in cyc]
    ys = [p[1] for p in cyc]
    qubit_pos, qubit_pts = [], []                 # position, lattice points the qubit touches
    for a in range(min(xs) // 2 - 1, max(xs) // 2 + 1):
        for b in range(min(ys) // 2 - 1, max(ys) // 2 + 1):
            c = (2 * a + 1, 2 * b + 1)
            corners = [(2 * a, 2 * b), (2 * a + 2, 2 * b), (2 * a + 2, 2 * b + 2), (2 * a, 2 * b + 2)]
            for i in range(4):
                tri = (c, corners[i], corners[(i + 1) % 4])
                cx = sum(t[0] for t in tri) / 3.0
                cy = sum(t[1] for t in tri) / 3.0
                w = _winding(cyc, cx, cy)
                if w == 1:
                    qubit_pos.append((cx, cy))
                    qubit_pts.append(tri)
                elif w != 0:
                    raise AssertionError("boundary cycle winds twice")
    # a boundary stretch is named by the colour its edges lack
    lack = [3 - _dual_colour(cyc[k]) - _dual_colour(cyc[(k + 1) % F]) for k in range(F)]
    edge_qubit = []
    for k in range(F):
        u, v = cyc[k], cyc[(k + 1) % F]
        edge_qubit.append(len(qubit_pos))
        qubit_pos.append(((u[0] + v[0]) / 2.0, (u[1] + v[1]) / 2.0))
        qubit_pts.append((u, v))
    corner_qubit = {}
    for k in range(F):
        if lack[k] != lack[(k + 1) % F]:
            v = cyc[(k + 1) % F]
            corner_qubit[k] = len(qubit_pos)
            qubit_pos.append((float(v[0]), float(v[1])))
            qubit_pts.append((v,))
    if len(corner_qubit) != 3:
        raise AssertionError("expected three boundary stretches")
    # qubits in (y, x) order, plaquettes in (y, x) order of their lattice points
    order = sorted(range(len(qubit_pos)), key=lambda q: (qubit_pos[q][1], qubit_pos[q][0]))
    new = {q: i for i, q in enumerate(order)}
    members = {}
    for q, pts in enumerate(qubit_pts):
        for pt in pts:
            members.setdefault(pt, []).append(new[q])
    plaq_pts = sorted(members, key=lambda pt: (pt[1], pt[0]))
    H = CSR.from_rows([members[pt] for pt in plaq_pts], len(order))
    steps = d - 2
    logical = [new[edge_qubit[k]] for k in range(steps)]          # the eastward zigzag's edges
    logical += [new[corner_qubit[F - 1]], new[corner_qubit[steps - 1]]]   # its two corners
    coords = [qubit_pos[q] for q in order]
    colours = np.asarray([_dual_colour(pt) for pt in plaq_pts], dtype=np.int8)
    return H, np.asarray(sorted(logical), dtype=np.int32), coords, colours


def _color_code(d: int, tiling: str):
    if tiling == "666":
        H, logical, _ = color_code_666(d)
    elif tiling == "488":
        H, logical, _, _ = color_code_488(d)
    else:
        raise ValueError("tiling must be '666' or '488'")
    return H, logical


def code_capacity_dem(d: int, p: float, tiling: str = "666") -> DEM:
    """Code-capacity bit-flip model on the d colour code (hexagonal '666' or square-octagon '488'
    tiling): H = plaquette incidence, L = boundary logical."""
    H, logical = _color_code(d, tiling)
    L = CSR.from_rows([logical], H.ncols)
    priors = np.full(H.ncols, float(p), dtype=np.float64)
    return DEM(H, L, priors, name=f"cc{tiling}_d{d}_codecap_p{p}", meta={"d": d, "p": p, "tiling": tiling})


def phenomenological_dem(d: int, noisy_rounds: int, p: float, q: float, tiling: str = "666") -> DEM:
    """Phenomenological noise over `noisy_rounds` noisy rounds plus one perfect round.

    Rounds r = 0..R-1 with R = noisy_rounds + 1; the last one is perfect. Detector (P, r) is the XOR of
    plaquette P's outcomes in rounds r and r-1 (round -1 reads 0). Before each noisy round every data
    qubit flips with probability p: column (q, r) hits detectors (P, r) for P containing q. Each noisy
    round's outcome of P flips with probability q: column (P, r) hits detectors (P, r) and (P, r+1).
    The observable is the boundary logical, flipped by data flips on its support in any round.
    Column order: all data columns (round-major, qubit-minor), then all measurement columns.
    tiling: '666' (hexagonal) or '488' (square-octagon) colour code.
    """
    Hc, logical = _color_code(d, tiling)
    nq, mp = Hc.ncols, Hc.nrows
    R = noisy_rounds + 1
    qubit_plaqs = [[] for _ in range(nq)]
    for P in range(mp):
        for qq in Hc.row(P):
            qubit_plaqs[qq].append(P)
    cols = []
    for r in range(noisy_rounds):
        for qq in range(nq):
            cols.append([r * mp + P for P in qubit_plaqs[qq]])
    for r in range(noisy_rounds):
        for P in range(mp):
            cols.append([r * mp + P, (r + 1) * mp + P])
    n = len(cols)
    rows = [[] for _ in range(mp * R)]
    for v, cc in enumerate(cols):
        for c in cc:
            rows[c].append(v)
    H = CSR.from_rows(rows, n)
    lset = set(int(x) for x in logical)
    lcols = [r * nq + qq for r in range(noisy_rounds) for qq in range(nq) if qq in lset]
    L = CSR.from_rows([lcols], n)
    priors = np.concatenate([np.full(noisy_rounds * nq, float(p)), np.full(noisy_rounds * mp, float(q))])
    return DEM(H, L, priors.astype(np.float64), name=f"cc{tiling}_d{d}_pheno_r{noisy_rounds}_p{p}_q{q}",
               meta={"d": d, "rounds": noisy_rounds, "p": p, "q": q, "tiling": tiling})


# --------------------------------------------------------------------------------------------
# Sampling and packing
# --------------------------------------------------------------------------------------------

def words(nbits: int) -> int:
    return (nbits + 31) // 32


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8/bool [B, nbits] -> uint32 [B, ceil(nbits/32)], little-endian bit order, zero padding."""
    bits = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    B, nb = bits.shape
    w = words(nb)
    padded = np.zeros((B, w * 32), dtype=np.uint8)
    padded[:, :nb] = bits
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u4").astype(np.uint32).reshape(B, w)


def unpack_bits(packed: np.ndarray, nbits: int) -> np.ndarray:
    packed = np.ascontiguousarray(np.asarray(packed, dtype=np.uint32))
    by = packed.astype("<u4").view(np.uint8).reshape(packed.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :nbits]


def _apply_sparse(M: CSR, err_rows: np.ndarray, err_cols: np.ndarray, B: int) -> np.ndarray:
    """Parity M e for a batch given the nonzero (shot, column) positions of e; returns uint8 [B, M.nrows]."""
    Mt = M.transpose()
    out = np.zeros((B, M.nrows), dtype=np.uint8)
    if len(err_cols) == 0:
        return out
    deg = np.diff(Mt.rowptr)[err_cols]
    shots = np.repeat(err_rows, deg)
    starts = Mt.rowptr[err_cols]
    offs = np.arange(int(deg.sum())) - np.repeat(np.cumsum(deg) - deg, deg)
    checks = Mt.colidx[np.repeat(starts, deg) + offs]
    np.bitwise_xor.at(out, (shots, checks), 1)
    return out


def sample(dem: DEM, shots: int, seed: int, chunk: int = 1 << 16, return_errors: bool = False):
    """Draw `shots` errors e_j ~ Bernoulli(p_j) from a PCG64 stream seeded with `seed`.

    Returns (syndromes uint32 [shots, ceil(m/32)], observables uint32 [shots, ceil(k/32)]) and, if
    requested, the errors as uint8 [shots, n].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    syn = np.zeros((shots, words(dem.m)), dtype=np.uint32)
    obs = np.zeros((shots, words(dem.k)), dtype=np.uint32)
    errs = np.zeros((shots, dem.n), dtype=np.uint8) if return_errors else None
    p = dem.priors
    for s0 in range(0, shots, chunk):
        b = min(chunk, shots - s0)
        e = rng.random((b, dem.n)) < p
        r, c = np.nonzero(e)
        syn[s0:s0 + b] = pack_bits(_apply_sparse(dem.H, r, c, b))
        obs[s0:s0 + b] = pack_bits(_apply_sparse(dem.L, r, c, b))
        if return_errors:
            errs[s0:s0 + b] = e
    if return_errors:
        return syn, obs, errs
    return syn, obs


def syndromes_of(dem: DEM, errors: np.ndarray):
    """Exact s = H e and obs = L e for given error vectors (uint8 [B, n]), packed."""
    errors = np.asarray(errors, dtype=np.uint8)
    r, c = np.nonzero(errors)
    B = errors.shape[0]
    return pack_bits(_apply_sparse(dem.H, r, c, B)), pack_bits(_apply_sparse(dem.L, r, c, B))


def schedules(n: int, K: int, seed: int, natural: bool = False) -> np.ndarray:
    """K serial schedules (permutations of the n columns) as uint32 [K, n] (Sec. III.D.1, step 3).

    natural=True gives the identity order for every member (the plain serial decoder).
    """
    if natural:
        return np.tile(np.arange(n, dtype=np.uint32), (K, 1))
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.permutation(n).astype(np.uint32) for _ in range(K)])


# --------------------------------------------------------------------------------------------
# Named workloads (the shapes of the paper's decoding problems)
# --------------------------------------------------------------------------------------------

WORKLOADS = {
    # d=5 colour code, code capacity p=0.05, plain decoder K=1, natural order.
    "cc666_d5_codecap": dict(kind="codecap", d=5, p=0.05, K=1, M=1, T=20, alpha=0.625,
                             natural=True, shots=10_000, seed=1),
    # d=9 colour code, 9 noisy + 1 perfect phenomenological rounds, p=q=0.01, K=16 random schedules.
    "cc666_d9_pheno": dict(kind="pheno", d=9, rounds=9, p=0.01, q=0.01, K=16, M=5, T=30, alpha=0.625,
                           natural=False, shots=1_000_000, seed=2),
    # the same decoder and noise on the square-octagon colour code of the same distance
    "cc488_d9_pheno": dict(kind="pheno", d=9, rounds=9, p=0.01, q=0.01, K=16, M=5, T=30, alpha=0.625,
                           natural=False, shots=100_000, seed=2, tiling="488"),
    "cc488_d5_codecap": dict(kind="codecap", d=5, p=0.05, K=1, M=1, T=20, alpha=0.625,
                             natural=True, shots=10_000, seed=1, tiling="488"),
}


def build_workload(name: str) -> DEM:
    w = WORKLOADS[name]
    tiling = w.get("tiling", "666")
    if w["kind"] == "codecap":
        return code_capacity_dem(w["d"], w["p"], tiling)
    if w["kind"] == "pheno":
        return phenomenological_dem(w["d"], w["rounds"], w["p"], w["q"], tiling)
    raise KeyError(name)
