"""The circuit builder's noise against the paper's noise-model tables (Sec. IV.A, Tables I and II),
stored as a text fixture in tests/golden/noise_models.txt.

Every fault location of the built circuits is classified by what happens in its moment (a two-qubit
gate layer, single-qubit Cliffords, a reset, a measurement) and its probability must be the table's
multiple of p; every gate, reset and measurement must carry its fault. The data's |+> preparation
(reset and H in one moment) and X-basis readout count as one reset and one measurement, as the
Uniform table treats X-basis resets and measurements.
"""
import os

import numpy as np
import pytest

from paper_2508_15743_gb300 import circuit as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "noise_models.txt")


def _table():
    t = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                model, op, _channel, mult = line
                t[(model, op)] = float(mult)
    return t


@pytest.mark.parametrize("noise", ["si1000", "uniform"])
@pytest.mark.parametrize("schedule,basis,rounds,tiling", [("xz", "X", 2, "666"), ("xz", "Z", 2, "666"),
                                                          ("xyz", "X", 4, "666"), ("xz", "X", 2, "488"),
                                                          ("xyz", "Z", 4, "488")])
def test_fault_probabilities_follow_the_tables(noise, schedule, basis, rounds, tiling):
    tab = _table()
    p = 1e-3
    circ = C.memory_circuit(3, rounds, p, noise, basis, schedule=schedule, tiling=tiling)
    B = circ["builder"]
    mult = {op: tab[(noise, op)] for (model, op) in tab if model == noise}
    seen = set()
    for gates, faults in B.moments:
        two = [pr for k, a in gates if k in ("CX", "CY") for pr in a[0]]
        h = [q for k, a in gates if k == "H" for q in a[0]]
        resets = [q for k, a in gates if k == "R" for q in a[0]]
        meas = [k for kk, a in gates if kk == "M" for k in a[1]]
        # a moment with a reset or a measurement idles the others at the measure/reset rate
        gate_layer = (bool(two) or bool(h)) and not resets and not meas
        for kind, args, prob in faults:
            if kind == "DEP2":
                op = "two_qubit_gate"
                assert sorted(args) == sorted(two)
            elif kind == "DEP1":
                if h and sorted(args) == sorted(h) and not two:
                    op = "one_qubit_clifford"
                else:
                    op = "idle_gate" if gate_layer else "idle_measure_reset"
                    busy = {q for pr in two for q in pr} | set(h) | set(resets) | \
                        {q for k, a in gates if k == "M" for q in a[0]}
                    assert not (set(args) & busy), "idle noise only on idle qubits"
            elif kind in ("X", "Z"):
                op = "reset"
                assert sorted(args) == sorted(resets)
                # a reset followed by H in its moment prepares |+> and takes a phase flip; others a bit flip
                prepared_in_x = bool(h) and set(h) == set(resets)
                assert kind == ("Z" if prepared_in_x else "X")
            elif kind == "MFLIP":
                op = "measure"
                assert sorted(args) == sorted(meas)
            else:
                raise AssertionError(kind)
            assert prob == pytest.approx(mult[op] * p, rel=1e-12), (op, prob)
            seen.add(op)
        # every operation carries its fault (where the table gives it a non-zero probability)
        if two and mult["two_qubit_gate"] > 0:
            assert any(k == "DEP2" for k, _, _ in faults)
        if meas and mult["measure"] > 0:
            assert any(k == "MFLIP" for k, _, _ in faults)
        if resets and mult["reset"] > 0:
            assert any(k in ("X", "Z") for k, _, _ in faults)
    expected = {op for op, m in mult.items() if m > 0}
    assert seen == expected
