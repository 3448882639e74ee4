"""Circuit-level detector error models for the 6.6.6 and 4.8.8 colour codes (seeded-input side).

The decoding problem of circuit-level noise (Sec. II.B): columns are independent fault mechanisms of
a syndrome-extraction circuit, rows are detectors (parities of measurement outcomes that are fixed
without noise). This module builds the circuit, propagates every single fault through it as a Pauli
frame, and merges faults with identical detector and observable signatures. It holds none of the
decoder's arithmetic.

Circuit (our own schedule; the paper's circuits are third-party). Qubits: the n data qubits, then one
ancilla per plaquette. Memory in basis B in {X, Z}: data prepared in the +1 eigenstate of B, then
`rounds` rounds, each measuring all Z-type plaquettes and then all X-type plaquettes with the
plaquette's ancilla:
    Z block: reset ancillas | 6 CNOT layers data -> ancilla | measure ancillas (Z basis)
    X block: reset ancillas | H ancillas | 6 CNOT layers ancilla -> data | H ancillas | measure
CNOT layer k couples every plaquette with its neighbour in lattice direction k (the six neighbour
offsets in counter-clockwise order), so no qubit takes part in two gates of one layer. On the 4.8.8
code (dem.color_code_488) the blocks have eight CNOT layers, a proper edge colouring of the
plaquette/qubit graph. Finally every data qubit is measured in basis B.

Detectors: B-type plaquettes are deterministic from the first round (detector = outcome), the other
type from the second (detector = XOR of consecutive outcomes); B-type plaquettes get a final detector
comparing the data measurement's plaquette parity with the last round. The observable is the B-type
logical (the weight-d boundary) read from the final data measurement.

Noise, Si1000-style (Table I, with CNOT as the two-qubit gate): two-qubit depolarising p after each
CNOT; one-qubit depolarising p/10 after each H and on every qubit idle during a gate layer; bit-flip
2p after each reset (phase-flip for the |+> data preparation); outcome flip 5p on each measurement;
one-qubit depolarising 2p on qubits idle during a measurement or reset layer. The Uniform model
(Table II) uses p everywhere.
"""
from __future__ import annotations

import numpy as np

from .dem import CSR, DEM, color_code_488, color_code_layout

# counter-clockwise lattice directions around a plaquette centre
_DIRS = ((1, 0), (0, 1), (-1, 1), (-1, 0), (0, -1), (1, -1))

SI1000 = dict(cx=1.0, h=0.1, idle_gate=0.1, reset=2.0, meas=5.0, idle_mr=2.0)
UNIFORM = dict(cx=1.0, h=1.0, idle_gate=0.0, reset=1.0, meas=1.0, idle_mr=0.0)

# two-qubit Paulis (x1, z1, x2, z2) except the identity, for depolarising channels
_P2 = [(a & 1, (a >> 1) & 1, b & 1, (b >> 1) & 1) for a in range(4) for b in range(4) if a or b]
_P1 = [(1, 0), (1, 1), (0, 1)]   # X, Y, Z as (x, z)


class _Builder:
    """Layered circuit with a fault list; faults are simulated in parallel as packed Pauli frames."""

    def __init__(self, nq):
        self.nq = nq
        self.moments = []   # list of (gates, faults); gates: list of (kind, args)
        self.nmeas = 0

    def moment(self):
        self.moments.append(([], []))
        return self.moments[-1]

    def gate(self, kind, *args):
        self.moments[-1][0].append((kind, args))
        if kind == "M":
            idx = list(range(self.nmeas, self.nmeas + len(args[0])))
            self.nmeas += len(args[0])
            return idx
        return None

    def fault(self, kind, args, p):
        if p > 0:
            self.moments[-1][1].append((kind, args, p))

    def fault_list(self):
        """Every single fault: (moment, "P", ((qubit, x, z), ...), p) for a Pauli applied after the moment's
        gates, or (moment, "M", measurement index, p) for an outcome flip."""
        faults = []
        for mi, (_, fl) in enumerate(self.moments):
            for kind, args, p in fl:
                if kind == "DEP1":
                    for q in args:
                        for (x, z) in _P1:
                            faults.append((mi, "P", ((q, x, z),), p / 3.0))
                elif kind == "DEP2":
                    for (a, b) in args:
                        for (x1, z1, x2, z2) in _P2:
                            faults.append((mi, "P", ((a, x1, z1), (b, x2, z2)), p / 15.0))
                elif kind == "X":
                    for q in args:
                        faults.append((mi, "P", ((q, 1, 0),), p))
                elif kind == "Z":
                    for q in args:
                        faults.append((mi, "P", ((q, 0, 1),), p))
                elif kind == "MFLIP":
                    for k in args:
                        faults.append((mi, "M", k, p))
        return faults

    def simulate(self):
        """Measurement-flip record of every single fault of fault_list(): uint64 [nmeas, words] (fault f
        is bit f % 64 of word f // 64), and the fault probabilities."""
        faults = self.fault_list()
        F = len(faults)
        W = (F + 63) // 64
        X = np.zeros((self.nq, W), np.uint64)
        Z = np.zeros((self.nq, W), np.uint64)
        rec = np.zeros((self.nmeas, W), np.uint64)
        by_moment = [[] for _ in self.moments]
        for f, (mi, kind, args, p) in enumerate(faults):
            by_moment[mi].append((f, kind, args))
        for mi, (gates, _) in enumerate(self.moments):
            for kind, args in gates:
                if kind == "CX":
                    for c, t in args[0]:
                        X[t] ^= X[c]
                        Z[c] ^= Z[t]
                elif kind == "CY":
                    # controlled-Y: X_c -> X_c Y_t, X_t -> Z_c X_t, Z_t -> Z_c Z_t, Z_c fixed
                    for c, t in args[0]:
                        Z[c] ^= X[t] ^ Z[t]
                        X[t] ^= X[c]
                        Z[t] ^= X[c]
                elif kind == "H":
                    for q in args[0]:
                        X[q], Z[q] = Z[q].copy(), X[q].copy()
                elif kind == "R":
                    for q in args[0]:
                        X[q] = 0
                        Z[q] = 0
                elif kind == "M":
                    qs, ks = args[0], args[1]
                    for q, k in zip(qs, ks):
                        rec[k] = X[q]
            for f, kind, args in by_moment[mi]:
                w, bit = f >> 6, np.uint64(1) << np.uint64(f & 63)
                if kind == "P":
                    for (q, x, z) in args:
                        if x:
                            X[q, w] ^= bit
                        if z:
                            Z[q, w] ^= bit
                else:
                    rec[args, w] ^= bit
        probs = np.array([p for (_, _, _, p) in faults], np.float64)
        return rec, probs


def _edge_colour_layers(sup, n, seed=0):
    """CNOT layers for plaquettes with supports `sup` over n data qubits: a proper edge colouring of
    the bipartite plaquette/qubit graph with as many colours as the largest degree (Konig's theorem;
    alternating-path recolouring), so that no qubit takes part in two gates of one layer. The edges
    are coloured in a seeded random order, each taking a random colour free at its plaquette: the
    order of a plaquette's CNOTs decides which data qubits a mid-block ancilla fault reaches (its
    hook), and the index order gave hooks that let two single faults share detectors with different
    logical effect at d = 5; seed 0 gives none at d = 5 and 7 (tests/test_inputs.py). Returns one
    list of (data qubit, plaquette) pairs per colour."""
    rng = np.random.default_rng(seed)
    deg = max(max(len(x) for x in sup), max(np.bincount([q for x in sup for q in x], minlength=n)))
    at_p = [dict() for _ in sup]       # plaquette -> {colour: qubit}
    at_q = [dict() for _ in range(n)]  # qubit -> {colour: plaquette}
    edges = [(P, q) for P, qs in enumerate(sup) for q in qs]
    for e in rng.permutation(len(edges)):
        P, q = edges[e]
        free_p = [c for c in range(deg) if c not in at_p[P]]
        a = free_p[rng.integers(len(free_p))]
        b = next(c for c in range(deg) if c not in at_q[q])
        if a in at_q[q]:
            # swap a and b along the path q -a- P1 -b- q2 -a- ... (it cannot reach P)
            path, node, side, col = [], q, "q", a
            while True:
                nxt = (at_q[node] if side == "q" else at_p[node]).get(col)
                if nxt is None:
                    break
                path.append((node, nxt, col) if side == "q" else (nxt, node, col))
                node, side, col = nxt, ("p" if side == "q" else "q"), (b if col == a else a)
            for (qq, PP, c) in path:
                del at_q[qq][c]
                del at_p[PP][c]
            for (qq, PP, c) in path:
                c2 = b if c == a else a
                at_q[qq][c2] = PP
                at_p[PP][c2] = qq
        at_p[P][a] = q
        at_q[q][a] = P
    return [sorted((q, P) for P in range(len(sup)) for c, q in at_p[P].items() if c == col) for col in range(deg)]


def _code_geometry(d, tiling):
    """(n, plaquette supports, CNOT layers of (data, plaquette) pairs, logical support) of a tiling."""
    if tiling == "666":
        qubits, plaqs = color_code_layout(d)
        qidx = {q: k for k, q in enumerate(qubits)}
        layers = []
        for (di, dj) in _DIRS:
            layers.append([(qidx[(i + di, j + dj)], P) for P, (i, j) in enumerate(plaqs) if (i + di, j + dj) in qidx])
        sup = [[qidx[(i + di, j + dj)] for (di, dj) in _DIRS if (i + di, j + dj) in qidx] for (i, j) in plaqs]
        logical = sorted(qidx[q] for q in qubits if q[1] == -1)
        return len(qubits), sup, layers, logical
    if tiling == "488":
        H, logical, _, _ = color_code_488(d)
        sup = [H.row(P).tolist() for P in range(H.nrows)]
        return H.ncols, sup, _edge_colour_layers(sup, H.ncols), logical.tolist()
    raise ValueError("tiling must be '666' or '488'")


def _unpack_rows(packed, F):
    """uint64 [r, W] -> uint8 [r, F] bits (fault f is bit f % 64 of word f // 64)."""
    by = packed.astype("<u8").view(np.uint8).reshape(packed.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :F]


def memory_circuit(d: int, rounds: int, p: float, noise="si1000", basis="X", custom=None, schedule="xz",
                   tiling="666") -> dict:
    """The colour-code memory circuit as a _Builder plus its detectors and observable.

    schedule "xz": every round measures all Z-type then all X-type plaquettes (module docstring).
    schedule "xyz": round r measures every plaquette in one basis, cycling (B, Y, other) with B the
    memory basis; a Y measurement is an ancilla in |+>, six layers of controlled-Y ancilla -> data
    and H before the measurement. On an even-weight plaquette X_P Y_P Z_P is a constant, so the
    outcomes of three consecutive rounds have a fixed parity: that is the detector of round r >= 2;
    round 0 (basis B) is deterministic on its own, round 1 (Y) is random, and the final data
    measurement is compared with the last round that measured B.

    tiling: "666" (six CNOT layers in lattice directions) or "488" (the square-octagon code of
    dem.color_code_488; its eight CNOT layers are a proper edge colouring of the plaquette/qubit
    graph, in no geometric order).

    Returns dict(builder, det_meas: lists of measurement indices, det_type, obs_meas).
    """
    if schedule not in ("xz", "xyz"):
        raise ValueError(schedule)
    n, sup, play, logical = _code_geometry(d, tiling)
    mp = len(sup)
    anc = [n + P for P in range(mp)]
    nq = n + mp
    layers = [[(q, n + P) for (q, P) in L] for L in play]
    if noise == "si1000":
        w = SI1000
    elif noise == "uniform":
        w = UNIFORM
    elif noise == "custom":
        w = None
        custom = dict(custom or {})
    else:
        raise ValueError(noise)

    B = _Builder(nq)
    allq = list(range(nq))

    def idle(busy, factor):
        if w is None:
            return
        rest = [q for q in allq if q not in busy]
        B.fault("DEP1", rest, factor * p)

    def block(kind):
        """Reset the ancillas, measure every plaquette in basis kind ("X", "Y" or "Z"); returns the
        measurement indices, one per plaquette."""
        B.moment()
        B.gate("R", anc)
        if w is not None:
            B.fault("X", anc, w["reset"] * p)
            idle(set(anc), w["idle_mr"])
        if kind != "Z":
            B.moment()
            B.gate("H", anc)
            if w is not None:
                B.fault("DEP1", anc, w["h"] * p)
                idle(set(anc), w["idle_gate"])
        gate = {"X": "CX", "Y": "CY", "Z": "CX"}[kind]
        for L in layers:
            pairs = L if kind == "Z" else [(a, q) for (q, a) in L]
            B.moment()
            B.gate(gate, pairs)
            if w is not None:
                B.fault("DEP2", pairs, w["cx"] * p)
                idle({q for pr in pairs for q in pr}, w["idle_gate"])
        if kind != "Z":
            B.moment()
            B.gate("H", anc)
            if w is not None:
                B.fault("DEP1", anc, w["h"] * p)
                idle(set(anc), w["idle_gate"])
        B.moment()
        ks = B.gate("M", anc, None)
        B.moments[-1][0][-1] = ("M", (anc, ks))
        if w is not None:
            B.fault("MFLIP", ks, w["meas"] * p)
            idle(set(anc), w["idle_mr"])
        else:
            B.fault("MFLIP", ks, custom.get("meas_" + kind.lower(), 0.0))
        return ks

    # data preparation in the +1 eigenstate of the memory basis
    B.moment()
    B.gate("R", list(range(n)))
    if basis == "X":
        B.gate("H", list(range(n)))
    if w is not None:
        B.fault("Z" if basis == "X" else "X", list(range(n)), w["reset"] * p)
        idle(set(range(n)), w["idle_mr"])
    obasis = "Z" if basis == "X" else "X"
    cycle = (basis, "Y", obasis)
    meas = {"X": [], "Y": [], "Z": []}   # xz schedule: per-round indices of each type
    seq = []                             # xyz schedule: (basis, indices) per round
    for r in range(rounds):
        if w is None:
            B.moment()
            B.fault("X", list(range(n)), custom.get("data_x", 0.0))
            B.fault("Z", list(range(n)), custom.get("data_z", 0.0))
        if schedule == "xz":
            meas["Z"].append(block("Z"))
            meas["X"].append(block("X"))
        else:
            kind = cycle[r % 3]
            seq.append((kind, block(kind)))
    # final data measurement in the memory basis
    B.moment()
    if basis == "X":
        B.gate("H", list(range(n)))
    B.moment()
    kd = B.gate("M", list(range(n)), None)
    B.moments[-1][0][-1] = ("M", (list(range(n)), kd))
    if w is not None:
        B.fault("MFLIP", kd, w["meas"] * p)
    else:
        B.fault("MFLIP", kd, custom.get("final_meas", 0.0))

    det_meas, det_type = [], []
    if schedule == "xz":
        same, other = meas[basis], meas[obasis]
        for r in range(rounds):
            for P in range(mp):
                det_meas.append([same[r][P]] if r == 0 else [same[r][P], same[r - 1][P]])
                det_type.append(basis)
            if r > 0:
                for P in range(mp):
                    det_meas.append([other[r][P], other[r - 1][P]])
                    det_type.append(obasis)
        last = same[rounds - 1] if rounds > 0 else None
    else:
        for r in range(rounds):
            if r == 0:
                for P in range(mp):
                    det_meas.append([seq[0][1][P]])
                    det_type.append(basis)
            elif r >= 2:
                for P in range(mp):
                    det_meas.append([seq[r - 2][1][P], seq[r - 1][1][P], seq[r][1][P]])
                    det_type.append("XYZ")
        mine = [ks for kind, ks in seq if kind == basis]
        last = mine[-1] if mine else None
    for P in range(mp):
        det_meas.append([kd[q] for q in sup[P]] + ([last[P]] if last is not None else []))
        det_type.append(basis)
    return dict(builder=B, det_meas=det_meas, det_type=det_type, obs_meas=[kd[q] for q in logical])


def circuit_dem(d: int, rounds: int, p: float, noise="si1000", basis="X", custom=None, schedule="xz",
                tiling="666") -> DEM:
    """Detector error model of `rounds` rounds of the colour-code memory circuit in basis X or Z.

    noise: "si1000", "uniform", or "custom" with `custom` a dict of per-location probabilities
    (keys data_x / data_z: flips on data before each round, meas_z / meas_x / meas_y: outcome flips
    of the plaquette measurements, final_meas: flips of the data measurement) for testing.
    schedule: "xz" (X and Z plaquettes every round) or "xyz" (one basis per round, cycling; see
    memory_circuit). tiling: "666" or "488" (memory_circuit).
    """
    circ = memory_circuit(d, rounds, p, noise, basis, custom, schedule, tiling)
    H, L, pcol, F, undetectable = dem_from_circuit(circ)
    tag = "" if schedule == "xz" else "_xyz"
    return DEM(H, L, pcol, name=f"cc{tiling}_d{d}_circuit{tag}_{noise}_{basis}_r{rounds}_p{p}",
               meta={"d": d, "rounds": rounds, "p": p, "noise": noise, "basis": basis, "faults": F,
                     "tiling": tiling,
                     "schedule": schedule, "undetectable_logical_prob": undetectable,
                     "det_type": circ["det_type"]})


def dem_from_circuit(circ: dict):
    """Detector error model of a circuit from memory_circuit (or any dict with builder, det_meas and
    obs_meas): every single fault is propagated, faults that flip no detector are dropped, and faults
    with the same detector and observable signature merge into one column whose probability is that
    of an odd number of them, (1 - prod(1 - 2 p_i)) / 2. Columns are ordered by first appearance.

    Returns (H, L, priors, number of faults, total probability of faults that flip the observable
    and no detector)."""
    rec, probs = circ["builder"].simulate()
    det_meas, obs_meas = circ["det_meas"], circ["obs_meas"]
    F = len(probs)
    Wd = rec.shape[1]
    D = np.zeros((len(det_meas) + 1, Wd), np.uint64)
    for i, ms in enumerate(det_meas):
        for k in ms:
            D[i] ^= rec[k]
    for k in obs_meas:
        D[-1] ^= rec[k]
    bits = _unpack_rows(D, F)                     # [ndet + 1, F]
    keys = np.packbits(bits, axis=0, bitorder="little").T.copy()   # [F, bytes]
    flips_det = bits[:-1].any(axis=0)
    keep = np.nonzero(flips_det)[0]
    void = np.ascontiguousarray(keys[keep]).view(np.dtype((np.void, keys.shape[1]))).ravel()
    uniq, first, inv = np.unique(void, return_index=True, return_inverse=True)
    order = np.argsort(first)                     # columns in order of first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    col_of_fault = rank[inv]
    ncol = len(uniq)
    # combine independent mechanisms with the same signature: P(odd number) = (1 - prod(1 - 2 p_i)) / 2
    logs = np.zeros(ncol)
    np.add.at(logs, col_of_fault, np.log1p(-2.0 * probs[keep]))
    pcol = 0.5 * (1.0 - np.exp(logs))
    rep = keep[first[order]]                      # representative fault of each column
    rows = [[] for _ in range(len(det_meas))]
    lcols = []
    for c, f in enumerate(rep):
        for r in np.nonzero(bits[:-1, f])[0]:
            rows[r].append(c)
        if bits[-1, f]:
            lcols.append(c)
    H = CSR.from_rows(rows, ncol)
    L = CSR.from_rows([lcols], ncol)
    undetectable = float(probs[(~flips_det) & (bits[-1] == 1)].sum())
    return H, L, pcol.astype(np.float64), F, undetectable
