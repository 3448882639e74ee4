"""Pins for the seeded input generators (colour codes, DEMs, sampler, schedules).

Facts from Sec. II.A: the triangular colour code has n qubits, (n-1)/2 plaquettes, even-weight
commuting plaquettes, n-1 independent generators and k = 1; for odd distance d it has
n = (3d^2+1)/4 qubits. Eq. 1 gives s = H e mod 2.
"""
import numpy as np
import pytest

from paper_2508_15743_gb300 import dem as D
from tests.helpers import gf2_nullspace, gf2_rank


@pytest.mark.parametrize("d", [3, 5, 7, 9, 11, 13, 15])
def test_colour_code_counts(d):
    H, logical, coords = D.color_code_666(d)
    n = H.ncols
    assert n == (3 * d * d + 1) // 4
    assert H.nrows == (n - 1) // 2
    w = np.diff(H.rowptr)
    assert set(w.tolist()) <= {4, 6}
    assert (w == 4).sum() == 3 * (d - 1) // 2, "boundary squares"
    assert (w == 6).sum() == H.nrows - 3 * (d - 1) // 2, "bulk hexagons"
    col = np.bincount(H.colidx, minlength=n)
    assert col.max() <= 3 and col.min() >= 1
    assert len(logical) == d


@pytest.mark.parametrize("d", [3, 5, 7, 9, 11])
def test_colour_code_algebra(d):
    H, logical, _ = D.color_code_666(d)
    A = H.to_dense().astype(np.int64)
    n = A.shape[1]
    assert not ((A @ A.T) % 2).any(), "plaquettes must overlap evenly (X and Z generators commute)"
    r = gf2_rank(A)
    assert r == (n - 1) // 2
    assert n - 2 * r == 1, "k = 1 logical qubit"
    Lv = np.zeros(n, np.uint8)
    Lv[logical] = 1
    assert not (A @ Lv % 2).any(), "logical commutes with every plaquette"
    assert gf2_rank(np.vstack([A, Lv])) == r + 1, "logical is not a product of plaquettes"


@pytest.mark.parametrize("d", [3, 5, 7])
def test_colour_code_distance(d):
    """Minimum weight of x in ker(H) with odd overlap with the logical equals d."""
    H, logical, _ = D.color_code_666(d)
    A = H.to_dense()
    N = gf2_nullspace(A)
    Lv = np.zeros(A.shape[1], np.uint8)
    Lv[logical] = 1
    k = N.shape[0]
    best = 10 ** 9
    chunk = 1 << 14
    for start in range(0, 1 << k, chunk):
        idx = np.arange(start, min(1 << k, start + chunk), dtype=np.int64)
        coeff = ((idx[:, None] >> np.arange(k)) & 1).astype(np.uint8)
        X = (coeff.astype(np.int64) @ N.astype(np.int64)) % 2
        odd = (X @ Lv) % 2 == 1
        if odd.any():
            best = min(best, int(X[odd].sum(axis=1).min()))
    assert best == d


def test_code_capacity_workload_shape():
    dm = D.build_workload("cc666_d5_codecap")
    assert (dm.m, dm.n, dm.H.nnz) == (9, 19, 42)
    assert dm.L.nnz == 5
    assert np.allclose(dm.priors, 0.05)


def test_phenomenological_shape():
    dm = D.build_workload("cc666_d9_pheno")
    assert dm.m == 30 * 10 and dm.n == 61 * 9 + 30 * 9
    assert dm.H.nnz == 1944
    rowdeg = np.diff(dm.H.rowptr)
    coldeg = np.bincount(dm.H.colidx, minlength=dm.n)
    assert rowdeg.max() <= 8
    # the final (perfect) layer's detectors see only the last noisy round's measurement error
    assert (rowdeg[:30 * 9] >= 5).all() and (rowdeg[30 * 9:] == 1).all()
    assert coldeg.max() == 3
    assert (coldeg[61 * 9:] == 2).all()


def test_phenomenological_matches_measurement_record():
    """Simulate the noisy plaquette outcomes round by round and XOR consecutive rounds."""
    d, R = 5, 4
    dm = D.phenomenological_dem(d, R, 0.02, 0.03)
    Hc, logical, _ = D.color_code_666(d)
    A = Hc.to_dense().astype(np.int64)
    nq, mp = A.shape[1], A.shape[0]
    rng = np.random.default_rng(5)
    for _ in range(50):
        data = rng.random((R, nq)) < 0.1
        meas = rng.random((R, mp)) < 0.1
        frame = np.zeros(nq, np.int64)
        prev = np.zeros(mp, np.int64)
        det = []
        for r in range(R + 1):
            if r < R:
                frame = (frame + data[r]) % 2
            out = (A @ frame) % 2
            if r < R:
                out = (out + meas[r]) % 2
            det.append((out + prev) % 2)
            prev = out
        det = np.concatenate(det)
        e = np.concatenate([data.reshape(-1), meas.reshape(-1)]).astype(np.uint8)[None, :]
        s, o = D.syndromes_of(dm, e)
        assert np.array_equal(D.unpack_bits(s, dm.m)[0], det)
        obs = int(frame[logical].sum() % 2)
        assert int(D.unpack_bits(o, 1)[0, 0]) == obs


def test_sampler_parity_and_rate():
    dm = D.build_workload("cc666_d9_pheno")
    syn, obs, err = D.sample(dm, 3000, 11, return_errors=True, chunk=1000)
    A = dm.H.to_dense().astype(np.int64)
    Lm = dm.L.to_dense().astype(np.int64)
    s_ref = (err.astype(np.int64) @ A.T) % 2
    o_ref = (err.astype(np.int64) @ Lm.T) % 2
    assert np.array_equal(D.unpack_bits(syn, dm.m), s_ref)
    assert np.array_equal(D.unpack_bits(obs, dm.k), o_ref)
    rate = err.mean()
    assert abs(rate - 0.01) < 5 * np.sqrt(0.01 * 0.99 / err.size)
    # same seed, same stream
    syn2, obs2 = D.sample(dm, 3000, 11, chunk=1000)
    assert np.array_equal(syn, syn2) and np.array_equal(obs, obs2)


def test_pack_roundtrip_and_padding():
    rng = np.random.default_rng(0)
    for nb in [1, 31, 32, 33, 300, 819]:
        bits = (rng.random((7, nb)) < 0.5).astype(np.uint8)
        p = D.pack_bits(bits)
        assert p.shape == (7, (nb + 31) // 32)
        assert np.array_equal(D.unpack_bits(p, nb), bits)
        if nb % 32:
            assert (p[:, -1] >> (nb % 32) == 0).all()


def test_schedules_are_permutations():
    P = D.schedules(819, 16, 3)
    assert P.shape == (16, 819)
    for row in P:
        assert np.array_equal(np.sort(row), np.arange(819))
    assert len({tuple(r) for r in P}) == 16
    nat = D.schedules(19, 1, 0, natural=True)
    assert np.array_equal(nat[0], np.arange(19))


# ------------------------------------------------------------------------------------------------
# Circuit-level detector error models (circuit.py)
# ------------------------------------------------------------------------------------------------

from paper_2508_15743_gb300 import circuit as C  # noqa: E402


@pytest.mark.parametrize("d,R,tiling", [(3, 2, "666"), (5, 4, "666"), (9, 9, "666"), (3, 2, "488"), (5, 4, "488"),
                                         (7, 3, "488")])
def test_circuit_builder_reproduces_phenomenological_dem(d, R, tiling):
    """Z memory with only data bit flips and Z-measurement flips is the phenomenological model:
    the Pauli-frame builder must give the closed-form matrix, priors and logical, column for column."""
    dm = C.circuit_dem(d, R, 0.0, noise="custom", basis="Z", custom=dict(data_x=0.01, meas_z=0.02), tiling=tiling)
    ph = D.phenomenological_dem(d, R, 0.01, 0.02, tiling)
    rows = [i for i, t in enumerate(dm.meta["det_type"]) if t == "Z"]
    A = dm.H.to_dense()
    assert not np.delete(A, rows, axis=0).any(), "X-type detectors see no X errors"
    A = A[rows]
    B = ph.H.to_dense()
    assert A.shape == B.shape
    la, lb = set(dm.L.row(0).tolist()), set(ph.L.row(0).tolist())
    ka = sorted((tuple(A[:, j]), round(float(dm.priors[j]), 15), j in la) for j in range(dm.n))
    kb = sorted((tuple(B[:, j]), round(float(ph.priors[j]), 15), j in lb) for j in range(ph.n))
    assert ka == kb


@pytest.mark.parametrize("basis", ["X", "Z"])
@pytest.mark.parametrize("tiling", ["666", "488"])
def test_circuit_dem_invariants(basis, tiling):
    dm = C.circuit_dem(5, 5, 1e-3, noise="si1000", basis=basis, tiling=tiling)
    mp = 9 if tiling == "666" else 8
    assert dm.m == mp * 2 * 5, "B-type: 5 rounds + final; other type: rounds 2..5"
    coldeg = np.bincount(dm.H.colidx, minlength=dm.n)
    assert coldeg.min() >= 1, "every column flips a detector"
    assert np.diff(dm.H.rowptr).min() >= 1
    assert ((dm.priors > 0) & (dm.priors < 0.5)).all()
    assert dm.meta["undetectable_logical_prob"] == 0.0, "no single fault flips the logical unseen"
    # columns are distinct signatures
    A = dm.H.to_dense()
    lcols = set(dm.L.row(0).tolist())
    sig = {(tuple(A[:, j]), j in lcols) for j in range(dm.n)}
    assert len(sig) == dm.n
    # merged priors never exceed the sum of their parts: the total probability mass is at most the
    # fault list's, and each column is a probability of an odd number of its faults
    assert dm.priors.sum() < 5 * 1e-3 * dm.meta["faults"]


@pytest.mark.parametrize("schedule,tiling,d", [("xz", "666", 3), ("xyz", "666", 3), ("xz", "488", 3),
                                               ("xyz", "488", 3), ("xz", "488", 5)])
def test_circuit_single_faults_get_valid_corrections(schedule, tiling, d):
    """Every single fault of a small circuit DEM gets a correction with H e = s (oracle, exhaustive).

    The logical class is not pinned: the schedule's hook errors give pairs of single faults with the
    same syndrome and different logical effect (circuit distance 2 at d = 3), and Si1000's unequal
    priors let lighter multi-fault explanations win."""
    import oracle
    dm = C.circuit_dem(d, 3 if schedule == "xz" else 4, 1e-3, noise="si1000", basis="X", schedule=schedule,
                       tiling=tiling)
    errs = np.eye(dm.n, dtype=np.uint8)
    syn, obs = D.syndromes_of(dm, errs)
    perms = D.schedules(dm.n, 8, 1)
    out = oracle.decode(dm, perms, syn, 20, 0.625, 3, nthreads=8)
    e = D.unpack_bits(out["corrections"], dm.n)
    s2, _ = D.syndromes_of(dm, e)
    assert np.array_equal(s2, syn)
    A = dm.H.to_dense()
    groups = {}
    for j in range(dm.n):
        groups.setdefault(tuple(A[:, j]), set()).add(j in set(dm.L.row(0).tolist()))
    if tiling == "666":
        assert any(len(v) == 2 for v in groups.values()), "hook errors of this schedule (documented)"


def _logical_pairs_and_triples(dm, triples):
    """Whether two (or, with triples, three) DEM columns with zero total syndrome flip the logical."""
    A = dm.H.to_dense()
    lset = set(dm.L.row(0).tolist())
    sy = [int.from_bytes(np.packbits(A[:, j]).tobytes(), "big") for j in range(dm.n)]
    lg = [int(j in lset) for j in range(dm.n)]
    by = {}
    for j in range(dm.n):
        by.setdefault(sy[j], []).append(j)
    two = any(len({lg[j] for j in js}) == 2 for js in by.values())
    three = False
    if triples:
        for i in range(dm.n):
            for j in range(i + 1, dm.n):
                if any(k not in (i, j) and lg[k] ^ lg[i] ^ lg[j] for k in by.get(sy[i] ^ sy[j], ())):
                    three = True
                    break
            if three:
                break
    return two, three


@pytest.mark.parametrize("tiling", ["666", "488"])
def test_circuit_distance_is_not_cut_to_two(tiling):
    """Hook errors of the CNOT order: at d = 5 and 7 no two single faults have the same detectors and
    different logical effect (circuit distance >= 3), and at d = 7 no three do (>= 4), for both
    tilings' circuits in both memory bases."""
    for basis in ("X", "Z"):
        two, _ = _logical_pairs_and_triples(C.circuit_dem(5, 5, 1e-3, noise="si1000", basis=basis, tiling=tiling),
                                            False)
        assert not two
    two, three = _logical_pairs_and_triples(C.circuit_dem(7, 7, 1e-3, noise="si1000", basis="X", tiling=tiling), True)
    assert not two and not three


def test_merged_columns_take_the_odd_number_probability():
    """Faults with one signature merge into one column whose prior is the probability that an odd
    number of them occur (brute-force enumeration over the mechanisms); a fault flipping only the
    observable is reported as undetectable."""
    import itertools
    p1, p2, p3, p4, p5 = 0.01, 0.03, 0.2, 0.05, 0.004
    B = C._Builder(3)
    B.moment()
    B.gate("R", [0, 1, 2])
    B.fault("X", [0], p1)
    B.fault("X", [0], p2)
    B.fault("X", [2], p5)
    B.moment()
    ks = B.gate("M", [0, 1, 2], None)
    B.moments[-1][0][-1] = ("M", ([0, 1, 2], ks))
    B.fault("MFLIP", [ks[0]], p3)
    B.fault("MFLIP", [ks[1]], p4)
    circ = dict(builder=B, det_meas=[[ks[0]], [ks[1]]], obs_meas=[ks[1], ks[2]])
    H, L, pri, F, undetectable = C.dem_from_circuit(circ)
    assert F == 5 and H.ncols == 2
    assert H.to_dense().tolist() == [[1, 0], [0, 1]]
    assert L.to_dense().tolist() == [[0, 1]]
    ps = [p1, p2, p3]
    odd = sum(np.prod([p if b else 1 - p for p, b in zip(ps, bits)])
              for bits in itertools.product([0, 1], repeat=3) if sum(bits) % 2 == 1)
    assert pri[0] == pytest.approx(odd, rel=1e-12)
    assert pri[1] == pytest.approx(p4, rel=1e-12)
    assert undetectable == pytest.approx(p5, rel=1e-12)
