"""Circuits read from QASM text, run through the C ABI (needs a GB300) against the oracle
on the same parsed gate list: a generated Sycamore-class circuit written out and read back
(the tensor-core path), and a circuit of standard gates (general 1- and 2-qubit matrices,
through the plain, fused FP32 and tensor-core paths). Tolerances of the parity tests:
infidelity <= 1e-5, max amplitude error <= 1e-6."""
import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C
from paper_2512_07311_gb300 import qasm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def infidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def run(n, gates, umats, precision):
    ctx = capi.rcs_create(C.grid_for_n(n), precision)
    try:
        capi.rcs_apply_circuit(ctx, gates, umats)
        return capi.rcs_state_read(ctx).astype(np.complex128)
    finally:
        capi.rcs_destroy(ctx)


def test_generated_circuit_through_qasm(lib, oracle):
    c = C.generate(C.grid_for_n(20), 12, "EFGH", seed=31, jitter=0.05)
    n, gates, umats = qasm.parse_qasm(qasm.to_qasm(c.n_qubits, c.gates))
    want = oracle.simulate(n, gates, umats)
    got = run(n, gates, umats, capi.RCS_PREC_BF16X3)
    assert infidelity(got, want) <= 1e-5
    assert np.abs(got - want).max() <= 1e-6


def standard_gate_program(n, layers, seed):
    rng = np.random.default_rng(seed)
    one = ["h", "x", "s", "t", "sx", "sdg"]
    lines = ['OPENQASM 2.0;', 'include "qelib1.inc";', f"qreg q[{n}];", "creg m[%d];" % n]
    for _ in range(layers):
        for q in range(n):
            r = rng.integers(0, 3)
            if r == 0:
                lines.append(f"{one[rng.integers(0, len(one))]} q[{q}];")
            elif r == 1:
                lines.append(f"u3({rng.uniform(-3, 3)!r}, {rng.uniform(-3, 3)!r}, {rng.uniform(-3, 3)!r}) q[{q}];")
            else:
                lines.append(f"rz({rng.uniform(-3, 3)!r}) q[{q}];")
        perm = rng.permutation(n)
        for a, b in zip(perm[0::2], perm[1::2]):
            two = ["cx", "cz", "swap", "iswap", f"crz({rng.uniform(-3, 3)!r})", f"rzz({rng.uniform(-3, 3)!r})"]
            lines.append(f"{two[rng.integers(0, len(two))]} q[{a}], q[{b}];")
    lines.append("measure q -> m;")
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("precision", [capi.RCS_PREC_FP32_PLAIN, capi.RCS_PREC_FP32_FUSED, capi.RCS_PREC_BF16X3])
def test_standard_gate_circuit_through_qasm(lib, oracle, precision):
    n, gates, umats = qasm.parse_qasm(standard_gate_program(16, 10, seed=5))
    assert n == 16 and len(umats) == len(gates)  # every standard gate is a general matrix
    want = oracle.simulate(n, gates, umats)
    got = run(n, gates, umats, precision)
    assert infidelity(got, want) <= 1e-5
    assert np.abs(got - want).max() <= 1e-6
