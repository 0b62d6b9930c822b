"""Seeded circuit generator: determinism, coupler classes, the stated gate counts."""
import math

import numpy as np
import pytest

from paper_2512_07311_gb300 import circuits as C


def test_deterministic():
    a = C.config_circuit("30q_5x6_14cyc")
    b = C.config_circuit("30q_5x6_14cyc")
    assert a.gates.tobytes() == b.gates.tobytes()
    c = C.generate(C.Grid(5, 6), 14, "EFGH", seed=2, jitter=0.05)
    assert a.gates.tobytes() != c.gates.tobytes()


@pytest.mark.parametrize("grid", [C.Grid(3, 4), C.Grid(5, 6), C.Grid(5, 7, (34,)), C.Grid(4, 8), C.grid_for_n(23)])
def test_coupler_classes_partition(grid):
    cls = C.coupler_classes(grid)
    allc = C.all_couplers(grid)
    union = [cp for v in cls.values() for cp in v]
    assert sorted(union) == sorted(allc)
    assert len(set(union)) == len(union)
    for name, cps in cls.items():  # each class is a matching: no qubit twice
        qs = [q for cp in cps for q in cp]
        assert len(qs) == len(set(qs)), name
    qof = grid.qubit_of()
    cell = {q: rc for rc, q in qof.items()}
    for a, b in allc:  # nearest neighbours only
        (r0, c0), (r1, c1) = cell[a], cell[b]
        assert abs(r0 - r1) + abs(c0 - c1) == 1


@pytest.mark.parametrize("name,fsim,one", [("12q_3x4_8cyc", 34, 96 + 12), ("30q_5x6_14cyc", 174, 420 + 30),
                                          ("34q_5x7m1_20cyc", 280, 680 + 34), ("32q_4x8_20cyc", 260, 640 + 32)])
def test_gate_counts(name, fsim, one):
    c = C.config_circuit(name)
    assert c.counts() == {"fsim": fsim, "one_qubit": one}


def test_cycle_structure_and_no_repeat():
    c = C.config_circuit("34q_5x7m1_20cyc")
    n = c.n_qubits
    g = c.gates
    prev = {}
    pos = 0
    for cyc in range(c.cycles + 1):
        layer = g[pos:pos + n]
        assert list(layer["q0"]) == list(range(n))
        assert (layer["kind"] < C.FSIM).all()
        for rec in layer:
            q = int(rec["q0"])
            assert prev.get(q) != int(rec["kind"])
            prev[q] = int(rec["kind"])
        pos += n
        while pos < len(g) and g[pos]["kind"] == C.FSIM:
            pos += 1
    assert pos == len(g)


def test_patterns_map_classes():
    grid = C.Grid(4, 4)
    cls = C.coupler_classes(grid)
    ab = C.generate(grid, 8, "ABCDCDAB", seed=0)
    ef = C.generate(grid, 4, "EFGH", seed=0)

    def layers(circ):
        out, cur = [], []
        for rec in circ.gates:
            if rec["kind"] == C.FSIM:
                cur.append((int(rec["q0"]), int(rec["q1"])))
            elif cur:
                out.append(cur)
                cur = []
        return out

    assert layers(ab) == [cls[x] for x in "ABCDCDAB"]
    assert layers(ef) == [cls[x] for x in "CADB"]


def test_jitter_once_per_coupler():
    c = C.config_circuit("32q_4x8_20cyc")
    fs = c.gates[c.gates["kind"] == C.FSIM]
    seen = {}
    for rec in fs:
        key = (int(rec["q0"]), int(rec["q1"]))
        val = (float(rec["theta"]), float(rec["phi"]))
        assert abs(val[0] - math.pi / 2) <= 0.05 and abs(val[1] - math.pi / 6) <= 0.05
        assert seen.setdefault(key, val) == val
    thetas = np.array([v[0] for v in seen.values()])
    assert thetas.std() > 0.01
    plain = C.config_circuit("34q_5x7m1_20cyc")
    pf = plain.gates[plain.gates["kind"] == C.FSIM]
    assert (pf["theta"] == math.pi / 2).all() and (pf["phi"] == math.pi / 6).all()


def test_batch_workload_ranges():
    b = C.batch_workload(64, 1000)
    assert len(b) == 64
    assert all(16 <= c.n_qubits <= 26 and 10 <= c.cycles <= 20 and c.pattern in C.PATTERNS for c in b)
    assert len({c.n_qubits for c in b}) > 5 and {c.pattern for c in b} == set(C.PATTERNS)
    for c in b:
        assert c.grid.n_qubits == c.n_qubits


def test_inverse_gates():
    c = C.config_circuit("12q_3x4_8cyc")
    inv = C.inverse_gates(c.gates)
    assert len(inv) == len(c.gates)
    assert (inv["flags"] == C.ADJOINT).all()
    np.testing.assert_array_equal(inv["q0"], c.gates["q0"][::-1])
    assert (C.inverse_gates(inv)["flags"] == 0).all()
