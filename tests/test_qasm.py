"""QASM ingestion (no GPU): exact round trips of generated circuits, the standard gates pinned
to closed-form states (Bell and GHZ states, basis-state moves, rotation phases), register
broadcast, expressions, and the rejected inputs with their line numbers. States come from
the oracle applying the parsed gate list."""
import math

import numpy as np
import pytest

from paper_2512_07311_gb300 import circuits as C
from paper_2512_07311_gb300 import qasm

HDR = 'OPENQASM 2.0;\ninclude "qelib1.inc";\n'


def state(text):
    from oracle import oracle
    n, gates, umats = qasm.parse_qasm(text)
    return oracle.simulate(n, gates, umats)


@pytest.mark.parametrize("name", ["12q_3x4_8cyc", "30q_5x6_14cyc", "34q_5x7m1_20cyc"])
def test_generated_circuits_round_trip_exactly(name):
    c = C.config_circuit(name)
    n, g, u = qasm.parse_qasm(qasm.to_qasm(c.n_qubits, c.gates))
    assert n == c.n_qubits and u == {}
    np.testing.assert_array_equal(g, c.gates)  # kinds, qubits, flags and angles bit for bit


def test_adjoint_and_general_gates_round_trip():
    from oracle import oracle
    rng = np.random.default_rng(4)

    def unitary(d):
        q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        return q * (np.diag(r) / abs(np.diag(r)))

    n = 5
    recs = [(C.SQRT_X, 1, C.ADJOINT, 0, -1, 0, 0, 0), (C.FSIM, 2, C.ADJOINT, 1, 3, 0.3, -1.1, 0),
            (C.U1, 1, 0, 2, -1, 0, 0, 0), (C.U2, 2, 0, 4, 1, 0, 0, 0), (C.U2, 2, C.ADJOINT, 0, 2, 0, 0, 0),
            (C.SQRT_W, 1, 0, 3, -1, 0, 0, 0), (C.U1, 1, C.ADJOINT, 4, -1, 0, 0, 0)]
    gates = C.gate_array(recs)
    umats = {2: unitary(2), 3: unitary(4), 4: unitary(4), 6: unitary(2)}
    text = qasm.to_qasm(n, gates, umats)
    n2, g2, u2 = qasm.parse_qasm(text)
    assert n2 == n and len(g2) == len(gates)
    np.testing.assert_array_equal(g2["kind"], gates["kind"])
    np.testing.assert_array_equal(g2["q0"], gates["q0"])
    np.testing.assert_array_equal(g2["q1"], gates["q1"])
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    want = oracle.run(psi0.copy(), gates, umats)
    got = oracle.run(psi0.copy(), g2, u2)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_bell_and_ghz_states():
    r = 1 / math.sqrt(2)
    psi = state(HDR + "qreg q[2];\nh q[0];\ncx q[0], q[1];\n")
    np.testing.assert_allclose(psi, [r, 0, 0, r], atol=1e-15)
    text = HDR + "qreg q[5];\nh q[0];\n" + "".join(f"cx q[{i}],q[{i + 1}];\n" for i in range(4))
    psi = state(text)
    want = np.zeros(32, dtype=complex)
    want[0] = want[31] = r
    np.testing.assert_allclose(psi, want, atol=1e-15)


@pytest.mark.parametrize("body,index,amp", [
    ("x q[2];", 4, 1.0),                           # basis state |100>
    ("rx(pi) q[0];", 1, -1j),                     # exp(-i pi X / 2) = -i X
    ("x q[0];\nswap q[0], q[1];", 2, 1.0),
    ("x q[1];\ncx q[0], q[1];", 2, 1.0),          # control (first argument) is 0: unchanged
    ("x q[0];\ncx q[0], q[1];", 3, 1.0),          # control 1: the target (second) flips
    ("x q[0];\nx q[1];\ncz q[0], q[1];", 3, -1.0),
    ("x q[0];\niswap q[0], q[1];", 2, 1j),
    ("rzz(pi) q[0], q[1];", 0, -1j),              # exp(-i pi/2 Z(x)Z) on |00>
    ("x q[0];\ncu1(pi/2) q[0], q[2];\nx q[2];\ncu1(pi/2) q[0], q[2];", 5, 1j),
    ("u3(pi, 0, 0) q[1];", 2, 1.0),               # u3(pi,0,0) = [[0,-1],[1,0]]: |0> -> |1>
    ("x q[0];\nt q[0];\nt q[0];", 1, 1j),         # T^2 = S
    ("x q[0];\nsdg q[0];", 1, -1j),
])
def test_standard_gates_move_basis_states(body, index, amp):
    psi = state(HDR + "qreg q[3];\n" + body + "\n")
    want = np.zeros(8, dtype=complex)
    want[index] = amp
    np.testing.assert_allclose(psi, want, atol=1e-15)


def test_rotations_and_superpositions():
    r = 1 / math.sqrt(2)
    np.testing.assert_allclose(state(HDR + "qreg q[1];\nry(pi/2) q[0];\n"), [r, r], atol=1e-15)
    np.testing.assert_allclose(state(HDR + "qreg q[1];\nh q[0];\ns q[0];\n"), [r, 1j * r], atol=1e-15)
    np.testing.assert_allclose(state(HDR + "qreg q[1];\nu2(0, pi) q[0];\n"), [r, r], atol=1e-15)  # u2(0,pi) = H
    np.testing.assert_allclose(state(HDR + "qreg q[1];\nsx q[0];\nsx q[0];\n"), [0, 1], atol=1e-15)  # sx^2 = X
    # rz(t) = diag(e^{-it/2}, e^{it/2}) on H|0>: relative phase e^{it}
    psi = state(HDR + "qreg q[1];\nh q[0];\nrz(2*pi/3) q[0];\n")
    assert abs(psi[1] / psi[0] - np.exp(2j * math.pi / 3)) < 1e-14
    # the paper's family through QASM equals the same gates from the generator
    from oracle import oracle
    text = HDR + "qreg q[2];\nsqrt_x q[0];\nsqrt_y q[1];\nfsim(pi/2, pi/6) q[0], q[1];\nsqrt_w_dg q[0];\n"
    gates = C.gate_array([(C.SQRT_X, 1, 0, 0, -1, 0, 0, 0), (C.SQRT_Y, 1, 0, 1, -1, 0, 0, 0),
                          (C.FSIM, 2, 0, 0, 1, math.pi / 2, math.pi / 6, 0),
                          (C.SQRT_W, 1, C.ADJOINT, 0, -1, 0, 0, 0)])
    np.testing.assert_array_equal(state(text), oracle.simulate(2, gates))


def test_registers_broadcast_and_skipped_statements():
    text = (HDR + "qreg a[2];\nqreg b[3];\ncreg c[5];\n"
            "gate mine(x) p, r { rz(x) p; cx p, r; }\n"   # a declaration: skipped
            "opaque other a;\n"
            "h b;   // every qubit of b\n"
            "barrier a, b;\n"
            "x a[1];\n"
            "measure b -> c;\n")
    n, gates, umats = qasm.parse_qasm(text)
    assert n == 5 and len(gates) == 4 and list(gates["q0"]) == [2, 3, 4, 1]
    psi = state(text)
    nz = np.flatnonzero(abs(psi) > 1e-12)
    # qubit 1 set, qubits 2..4 in uniform superposition, qubit 0 clear
    assert sorted(nz.tolist()) == [2 + 4 * k for k in range(8)]
    np.testing.assert_allclose(abs(psi[nz]), 1 / math.sqrt(8), atol=1e-15)
    # two registers of one size: pairwise
    n, gates, _ = qasm.parse_qasm(HDR + "qreg a[3];\nqreg b[3];\ncx a, b;\n")
    assert list(zip(gates["q0"], gates["q1"])) == [(0, 3), (1, 4), (2, 5)]


def test_parameter_expressions():
    ev = qasm.eval_param
    assert ev("pi/2") == math.pi / 2 and ev("-pi") == -math.pi and ev("2*pi/3") == 2 * math.pi / 3
    assert ev("sin(pi/2)") == 1.0 and ev("2^3") == 8.0 and abs(ev("ln(exp(1.5))") - 1.5) < 1e-15
    assert ev("sqrt(4) + (1 - 3) * 0.5") == 1.0
    for bad in ["__import__('os')", "pi.real", "foo", "1/0", "", "[1]", "abs(-1)"]:
        with pytest.raises((ValueError, ZeroDivisionError, SyntaxError)):
            ev(bad)


@pytest.mark.parametrize("body,line,word", [
    ("qreg q[2];\nfoo q[0];", 4, "unknown gate"),
    ("qreg q[2];\nh q[2];", 4, "outside the register"),
    ("qreg q[3];\nccx q[0], q[1], q[2];", 4, "unknown gate"),
    ("qreg q[2];\ncx q[0];", 4, "qubit argument"),
    ("qreg q[2];\ncx q[1], q[1];", 4, "twice"),
    ("qreg q[2];\nreset q[0];", 4, "not a unitary"),
    ("qreg q[2];\nrx(__import__('os')) q[0];", 4, "rx"),
    ("qreg q[2];\nrx q[0];", 4, "parameter"),
    ("qreg q[2];\nfsim(1.0) q[0], q[1];", 4, "two parameters"),
    ("qreg q[2];\nh r[0];", 4, "unknown quantum register"),
    ("qreg q[2];\nqreg q[3];", 4, "twice"),
    ("qreg q[2];\nh q[0]", 4, "not terminated"),
])
def test_rejected_programs_name_their_line(body, line, word):
    with pytest.raises(qasm.QasmError) as e:
        qasm.parse_qasm(HDR + body + "\n")
    assert e.value.line == line and word in str(e.value), str(e.value)


def test_header_and_register_are_required():
    with pytest.raises(qasm.QasmError):
        qasm.parse_qasm("qreg q[2];\nh q[0];\n")
    with pytest.raises(qasm.QasmError):
        qasm.parse_qasm("OPENQASM 3.0;\nqreg q[2];\n")
    with pytest.raises(qasm.QasmError):
        qasm.parse_qasm(HDR)


def test_file_helpers(tmp_path):
    c = C.config_circuit("12q_3x4_8cyc")
    p = tmp_path / "c.qasm"
    qasm.write_qasm(str(p), c.n_qubits, c.gates)
    n, g, _ = qasm.read_qasm(str(p))
    assert n == 12
    np.testing.assert_array_equal(g, c.gates)
