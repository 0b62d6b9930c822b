"""The two-unitary tensor-core kernel (two consecutive 6-qubit passes per round trip of
the state) against the complex128 oracle and against the single-pass kernel, through
the C ABI (needs a GB300).

Tolerances:
  * against the oracle: each output within 3 x 4e-5 x |union slice|_2, where the union
    slice is the 2^|T1 u T2| amplitudes both unitaries mix (its norm bounds every slice
    norm either unitary sees; 4e-5 is the single-pass BF16x3 bound), and infidelity
    <= 2e-8 (twice the single-pass bound);
  * against two single passes on the same input: each output within 4e-6 x |union
    slice|_2. Both paths split the same FP32 values into the same bf16 hi/lo words
    and form the same products; only the FP32 accumulation order differs (complex
    block form here, realified form there), so they agree far more closely than
    either agrees with the oracle.
Cases cover disjoint, overlapping and identical target sets, the lowest U2 target
on index bit 0 and 1 (16-byte store paths), every target set that puts index bits
0..4 in the tile, one tile (13 qubits) and many tiles per CTA (22, 24 qubits).
"""
import math

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi

pytestmark = pytest.mark.gpu

AMP_REL = 4e-5
INFID = 2e-8
VS_SINGLE = 4e-6


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def rand_unitary(d, rng):
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def infidelity(a, b):
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def union_slice_max_norm(psi, targets):
    mask = sum(1 << t for t in set(targets))
    base = np.arange(psi.size) & ~mask
    s = np.zeros(psi.size)
    np.add.at(s, base, np.abs(psi) ** 2)
    return math.sqrt(s.max())


CASES = [(13, [0, 1, 2, 3, 4, 5], [6, 7, 8, 9, 10, 11]),
         (13, [7, 8, 9, 10, 11, 12], [12, 11, 10, 9, 8, 7]),
         (14, [1, 6, 8, 9, 12, 13], [1, 3, 5, 7, 10, 12]),
         (15, [0, 5, 7, 8, 9, 12], [2, 5, 8, 9, 10, 14]),
         (14, [2, 3, 4, 5, 6, 13], [0, 1, 9, 10, 11, 12]),
         (16, [3, 9, 10, 11, 14, 15], [0, 4, 9, 12, 13, 15]),
         (22, [21, 0, 10, 4, 17, 6], [3, 8, 13, 16, 20, 21]),
         (24, [9, 10, 11, 12, 13, 14], [12, 13, 14, 15, 16, 17]),
         (22, [5, 9, 14, 17, 20, 21], [1, 6, 12, 13, 19, 20])]


@pytest.mark.parametrize("n,t1,t2", CASES)
def test_pair_vs_oracle_and_single_passes(lib, oracle, n, t1, t2):
    rng = np.random.default_rng(1000 * n + t1[0] + 7 * t2[0])
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    pair = capi.rcs_create(n, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
    single = capi.rcs_create(n, capi.RCS_PREC_BF16X3)
    try:
        capi.rcs_state_write(pair, psi0)
        want = psi0.astype(np.complex128)
        for rep in range(2):
            U1, U2 = rand_unitary(64, rng), rand_unitary(64, rng)
            start = capi.rcs_state_read(pair)
            capi.rcs_state_write(single, start)
            capi.rcs_apply_unitaries(pair, [(t1, U1), (t2, U2)])
            capi.rcs_apply_unitaries(single, [(t1, U1), (t2, U2)])
            capi.rcs_sync(pair)
            capi.rcs_sync(single)
            got = capi.rcs_state_read(pair).astype(np.complex128)
            ref = capi.rcs_state_read(single).astype(np.complex128)
            want = start.astype(np.complex128)
            scale = union_slice_max_norm(want, t1 + t2)
            oracle.apply_matrix(want, t1, U1)
            oracle.apply_matrix(want, t2, U2)
            err = np.abs(got - want).max()
            assert err <= 3 * AMP_REL * scale, (rep, err, scale)
            assert infidelity(got, want) <= INFID
            d = np.abs(got - ref).max()
            assert d <= VS_SINGLE * scale, (rep, d, scale)
    finally:
        capi.rcs_destroy(pair)
        capi.rcs_destroy(single)


def test_pair_lists_of_three_and_four(lib, oracle):
    """Odd lists: a pair then a single pass; even lists: two pairs."""
    n = 18
    rng = np.random.default_rng(5)
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    targets = [[0, 4, 8, 12, 16, 17], [1, 2, 3, 9, 10, 11], [5, 6, 7, 13, 14, 15], [2, 6, 10, 14, 15, 16]]
    for count in (3, 4):
        Us = [rand_unitary(64, rng) for _ in range(count)]
        ctx = capi.rcs_create(n, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
        try:
            capi.rcs_state_write(ctx, psi0)
            capi.rcs_apply_unitaries(ctx, list(zip(targets[:count], Us)))
            capi.rcs_sync(ctx)
            got = capi.rcs_state_read(ctx).astype(np.complex128)
        finally:
            capi.rcs_destroy(ctx)
        want = psi0.astype(np.complex128)
        for t, U in zip(targets[:count], Us):
            oracle.apply_matrix(want, t, U)
        assert infidelity(got, want) <= 2 * INFID
        assert np.abs(got - want).max() <= 2 * 3 * AMP_REL


def test_pair_rejects_a_bad_list_without_touching_the_state(lib):
    n = 14
    rng = np.random.default_rng(9)
    ctx = capi.rcs_create(n, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
    try:
        psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
        capi.rcs_state_write(ctx, psi0)
        U = rand_unitary(64, rng)
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_apply_unitaries(ctx, [([0, 1, 2, 3, 4, 5], U), ([6, 7, 8, 9, 10, 10], U)])
        assert e.value.code == capi.RCS_ERR_QUBIT
        np.testing.assert_array_equal(capi.rcs_state_read(ctx), psi0)
    finally:
        capi.rcs_destroy(ctx)


def test_pair_circuit_from_zero_vs_oracle(lib, oracle):
    """A whole circuit with RCS_OPT_PAIR_PASSES from |0...0>: pairs run inside the sub-state
    stages and on the full state; the result meets the circuit tolerances of the parity
    tests (infidelity 1e-5, max amplitude error 1e-6)."""
    from paper_2512_07311_gb300 import circuits as C

    n = 22
    circ = C.generate(C.grid_for_n(n), cycles=10, pattern="ABCDCDAB", seed=91, jitter=0.05)
    plan = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
    info = capi.rcs_plan_info(plan)
    capi.rcs_plan_destroy(plan)
    assert info["pair_passes"] >= 2 and info["prefix_passes"] >= 2
    ctx = capi.rcs_create(n, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        got = capi.rcs_state_read(ctx).astype(np.complex128)
    finally:
        capi.rcs_destroy(ctx)
    want = oracle.simulate(n, circ.gates)
    assert infidelity(got, want) <= 1e-5
    assert np.abs(got - want).max() <= 1e-6
