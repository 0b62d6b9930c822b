"""GPU path vs the complex128 CPU oracle, through the C ABI (needs a GB300).

Tolerances (stated once, used throughout):
  * final-state infidelity 1 - |<a|b>|^2 / (|a|^2 |b|^2) <= 1e-5, both in FP64;
  * max amplitude error |psi_gpu - psi_oracle|_inf <= 1e-6 absolute (same gate
    convention on both sides, so no global phase is removed);
  * |XEB_gpu - XEB_oracle| <= 0.005 on the same shots (observed: ~1e-7);
  * samples: inverse-CDF draws on the GPU's own state agree with the oracle's
    draws on that same state (promoted exactly to complex128) in >= 99.99% of
    shots (a flip needs a uniform within ~1e-16 of a CDF boundary); against the
    oracle's own state at 12 qubits >= 99.9%.
  * one tensor-core pass: each output within 4e-5 * |slice|_2 for BF16x3, from the
    BF16 split residuals (2^-17 relative on each operand, lo*lo dropped) plus FP32
    accumulation over 128 terms; within 4e-6 * |slice|_2 for TF32x3 (split
    residuals 2^-21 relative, so the FP32 accumulation dominates);
  * norm drift of the tensor-core path <= 2e-6 per pass: its FP32 accumulation
    loses about 8e-7 of the norm per pass, always downward (measured; a scale
    factor only -- the sampler and XEB divide by the computed norm and the
    infidelity above is taken between normalised vectors). FP32 SIMT paths keep
    |norm - 1| <= 1e-5.
"""
import math

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

pytestmark = pytest.mark.gpu

INFID_TOL = 1e-5
AMP_TOL = 1e-6
XEB_TOL = 0.005
PRECS = [capi.RCS_PREC_FP32_PLAIN, capi.RCS_PREC_FP32_FUSED, capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3]
TC_PRECS = (capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def infidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    return 1.0 - (abs(ov) ** 2) / (np.vdot(a, a).real * np.vdot(b, b).real)


def run_gpu(n_or_grid, gates, precision, k_max=0):
    ctx = capi.rcs_create(n_or_grid, precision, k_max)
    capi.rcs_apply_circuit(ctx, gates)
    capi.rcs_sync(ctx)
    return ctx


def rand_unitary(d, rng):
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


# ------------------------------------------------------------------ whole circuits

@pytest.mark.parametrize("precision", PRECS)
def test_config_12q_vs_oracle(lib, oracle, precision):
    circ = C.config_circuit("12q_3x4_8cyc")
    n = circ.n_qubits
    want = oracle.simulate(n, circ.gates)
    ctx = run_gpu(circ.grid, circ.gates, precision)
    try:
        got = capi.rcs_state_read(ctx)
        assert infidelity(got, want) <= INFID_TOL
        assert np.abs(got - want).max() <= AMP_TOL
        assert abs(capi.rcs_norm(ctx) - 1.0) <= 1e-5  # 12 qubits: every path is FP32 SIMT
        # samples on the same uniforms against the oracle's own state
        shots, seed = 10_000, 2024
        xs = capi.rcs_sample(ctx, shots, seed)
        xo = oracle.sample(want, shots, seed)
        assert np.mean(xs == xo) >= 0.999
        F_gpu = capi.rcs_xeb(ctx, xs)
        F_or = oracle.xeb(want, xs)
        assert abs(F_gpu - F_or) <= XEB_TOL
        assert abs(F_gpu - F_or) <= 1e-4
        assert abs(oracle.xeb(want, xo) - F_gpu) <= 0.05  # same shots up to boundary flips
    finally:
        capi.rcs_destroy(ctx)


@pytest.fixture(scope="module")
def circ20(oracle):
    circ = C.generate(C.Grid(4, 5), cycles=10, pattern="EFGH", seed=7, jitter=0.05)
    return circ, oracle.simulate(circ.n_qubits, circ.gates)


@pytest.mark.parametrize("precision", PRECS)
def test_circuit_20q_vs_oracle(lib, oracle, circ20, precision):
    circ, want = circ20
    ctx = run_gpu(circ.grid, circ.gates, precision)
    try:
        got = capi.rcs_state_read(ctx)
        inf = infidelity(got, want)
        err = np.abs(got - want).max()
        assert inf <= INFID_TOL, inf
        assert err <= AMP_TOL, err
        # sampler on the GPU's own state vs the oracle sampler on the same state
        shots, seed = 200_000, 99
        xs = capi.rcs_sample(ctx, shots, seed)
        xo = oracle.sample(got.astype(np.complex128), shots, seed)
        assert np.mean(xs == xo) >= 0.9999
        p = np.abs(got.astype(np.complex128)) ** 2
        assert (p[xs.astype(np.int64)] > 0).all()
        F_gpu = capi.rcs_xeb(ctx, xs)
        assert abs(F_gpu - oracle.xeb(want, xs)) <= XEB_TOL
        assert abs(F_gpu - oracle.xeb(got.astype(np.complex128), xs)) <= 1e-9
    finally:
        capi.rcs_destroy(ctx)


@pytest.mark.parametrize("k_max", [2, 3, 5, 6, 7])
def test_fused_widths_vs_oracle(lib, oracle, circ20, k_max):
    circ, want = circ20
    ctx = run_gpu(circ.grid, circ.gates, capi.RCS_PREC_FP32_FUSED, k_max)
    try:
        got = capi.rcs_state_read(ctx)
        assert infidelity(got, want) <= INFID_TOL
        assert np.abs(got - want).max() <= AMP_TOL
    finally:
        capi.rcs_destroy(ctx)


def test_autotuned_fused_path(lib, oracle):
    """autotune = 1 picks k_max by timed trial passes on the live state; the trials
    must leave that state bit-identical, so the result equals a fixed-k run."""
    n = 18
    circ = C.generate(C.grid_for_n(n), cycles=8, pattern="EFGH", seed=77, jitter=0.05)
    rng = np.random.default_rng(5)
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    results = []
    for autotune, k in ((1, 0), (0, None)):
        if k is None:  # the width the autotuner chose
            k = chosen
        ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED, k_max=k, autotune=autotune)
        try:
            capi.rcs_state_write(ctx, psi0)
            capi.rcs_apply_circuit(ctx, circ.gates)
            results.append(capi.rcs_state_read(ctx))
        finally:
            capi.rcs_destroy(ctx)
        if autotune:
            # recover the chosen width: the plan with that width has the same pass count as the run
            chosen = next(kk for kk in (2, 3, 4, 5) if np.array_equal(
                _fixed_k_state(n, circ, psi0, kk), results[0]))
    np.testing.assert_array_equal(results[0], results[1])
    want = oracle.run(psi0.astype(np.complex128), circ.gates)
    assert infidelity(results[0], want) <= INFID_TOL
    assert np.abs(results[0] - want).max() <= AMP_TOL


def test_substate_prefix_is_exact(lib):
    """From a fresh |0...0> the leading passes run on a compact sub-state and one
    expansion pass writes the whole state. Every slice computes exactly what it
    computes in the full state, so the result equals the same plan run on an
    explicitly written |0...0> (which is not fresh: no prefix) bit for bit. At 11
    qubits the plan carries no layout, so it runs on either state."""
    n = 11
    circ = C.generate(C.grid_for_n(n), cycles=8, pattern="EFGH", seed=93, jitter=0.05)
    plan = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_FP32_FUSED, 4)
    info = capi.rcs_plan_info(plan)
    assert info["prefix_passes"] >= 2
    assert (capi.rcs_plan_layout(plan, n) == np.arange(n)).all()
    zero = np.zeros(1 << n, dtype=np.complex64)
    zero[0] = 1
    out = []
    try:
        for fresh in (True, False):
            ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED, k_max=4)
            try:
                if not fresh:
                    capi.rcs_state_write(ctx, zero)
                capi.rcs_plan_upload(ctx, plan)
                capi.rcs_plan_run(ctx, plan)
                ms, full = capi.rcs_last_pass_timing(ctx)
                assert full == info["n_passes"] - (info["prefix_passes"] if fresh else 0)
                out.append(capi.rcs_state_read(ctx))
            finally:
                capi.rcs_destroy(ctx)
    finally:
        capi.rcs_plan_destroy(plan)
    np.testing.assert_array_equal(out[0], out[1])


_PREFIX_WANT = {}  # oracle states of the nested-stage circuits, shared by the precisions


@pytest.mark.parametrize("n,cycles,stages", [(22, 8, 2), (25, 10, 3)])
@pytest.mark.parametrize("precision", [capi.RCS_PREC_FP32_FUSED, capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3])
def test_substate_prefix_vs_oracle(lib, oracle, precision, n, cycles, stages):
    circ = C.generate(C.grid_for_n(n), cycles=cycles, pattern="ABCDCDAB", seed=91, jitter=0.05)
    plan = capi.rcs_plan_build(n, circ.gates, precision)
    info = capi.rcs_plan_info(plan)
    assert info["prefix_passes"] >= 2 and info["prefix_qubits"] <= n - 1
    assert info["prefix_stages"] == stages  # nested sub-states, each expanded into the next
    # a tensor-core pass after the sub-states reads the last sub-state itself (expansion and
    # pass in one launch) unless it needs the memory-order kernel (4+ targets below bit 5)
    t_next, _ = capi.rcs_plan_pass(plan, info["prefix_passes"])
    fuses = precision != capi.RCS_PREC_FP32_FUSED and sum(int(x) < 5 for x in t_next) < 4
    assert fuses == (precision != capi.RCS_PREC_FP32_FUSED)
    ctx = capi.rcs_create(n, precision)
    try:
        capi.rcs_plan_upload(ctx, plan)
        capi.rcs_plan_run(ctx, plan)
        ms, full = capi.rcs_last_pass_timing(ctx)
        assert full == info["n_passes"] - info["prefix_passes"] - int(fuses) and ms > 0
        got = capi.rcs_state_read(ctx)
    finally:
        capi.rcs_destroy(ctx)
        capi.rcs_plan_destroy(plan)
    if (n, cycles) not in _PREFIX_WANT:
        _PREFIX_WANT[(n, cycles)] = oracle.simulate(n, circ.gates)
    want = _PREFIX_WANT[(n, cycles)]
    assert infidelity(got, want) <= INFID_TOL
    assert np.abs(got - want).max() <= AMP_TOL


def _fixed_k_state(n, circ, psi0, k):
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED, k_max=k)
    try:
        capi.rcs_state_write(ctx, psi0)
        capi.rcs_apply_circuit(ctx, circ.gates)
        return capi.rcs_state_read(ctx)
    finally:
        capi.rcs_destroy(ctx)


# ------------------------------------------------------------------ tensor-core pass alone

# targets with four or more below qubit 5 run the memory-order (staged) kernel variant,
# the others the slice-order variant, whose stores depend on the lowest target (bit 0,
# bit 1 and higher each take another path); n >= 22 gives every CTA several tiles
# One FP32 pass of width k (5, 6 or 7: U in shared memory): each real output sums 2 * 2^k
# FP32 products of U (rounded to FP32, 2^-24 relative) and the FP32 state by fused
# multiply-adds, so |error| <= (2 * 2^k + 1) 2^-24 * sum |U_jl| |x_l|
# <= (2 * 2^k + 1) 2^-24 * |slice|_2 (a row of U has unit norm).
@pytest.mark.parametrize("precision", [capi.RCS_PREC_FP32_FUSED, capi.RCS_PREC_BF16X3])
@pytest.mark.parametrize("n,targets", [(5, [4, 3, 2, 1, 0]), (9, [0, 2, 4, 6, 8]), (21, [1, 2, 3, 4, 20]),
                                       (6, [0, 1, 2, 3, 4, 5]), (7, [6, 0, 5, 1, 4, 2, 3]), (8, [1, 2, 3, 5, 6, 7]),
                                       (10, [9, 0, 4, 7, 2, 5, 8]), (13, [0, 1, 2, 3, 4, 5]),
                                       (13, [6, 7, 8, 9, 10, 11, 12]), (16, [2, 5, 1, 15, 8, 11]),
                                       (17, [3, 16, 9, 0, 12, 6, 14]), (20, [5, 6, 7, 8, 9, 10, 11])])
def test_wide_simt_pass_vs_oracle(lib, oracle, n, targets, precision):
    """5- to 7-qubit unitaries on the tiled FP32 SIMT kernel (from 5 to 21 qubits, so from
    one ragged tile of 1 slice to 2^16 slices), element by element against the oracle. On a
    BF16X3 context a 5- or 7-qubit unitary, and a 6-qubit one below 13 qubits, take the
    same FP32 kernel."""
    if precision == capi.RCS_PREC_BF16X3 and len(targets) == 6 and n >= 13:
        pytest.skip("the tensor-core kernel takes this case (test_tc_pass_vs_oracle)")
    k = len(targets)
    rng = np.random.default_rng(n * 1000 + k * 10 + targets[0])
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    ctx = capi.rcs_create(n, precision)
    try:
        capi.rcs_state_write(ctx, psi0)
        want = psi0.astype(np.complex128)
        for rep in range(2):
            U = rand_unitary(1 << k, rng)
            capi.rcs_apply_unitary(ctx, targets, U)
            capi.rcs_sync(ctx)
            got = capi.rcs_state_read(ctx).astype(np.complex128)
            prev = want.copy()
            oracle.apply_matrix(want, targets, U)
            mask = sum(1 << t for t in targets)
            base = np.arange(1 << n) & ~mask
            slice_norm2 = np.zeros(1 << n)
            np.add.at(slice_norm2, base, np.abs(prev) ** 2)
            bound = (2 * 2**k + 1) * 2.0**-24 * math.sqrt(slice_norm2.max())
            err = np.abs(got - want).max()
            assert err <= bound, (rep, err, bound)
            assert infidelity(got, want) <= 1e-10
            want = got
    finally:
        capi.rcs_destroy(ctx)


TC_PASS_BOUND = {capi.RCS_PREC_BF16X3: (4e-5, 1e-8), capi.RCS_PREC_TF32X3: (4e-6, 1e-10)}


@pytest.mark.parametrize("precision", TC_PRECS)
@pytest.mark.parametrize("n,targets", [(13, [0, 1, 2, 3, 4, 5]), (13, [7, 8, 9, 10, 11, 12]),
                                       (14, [0, 3, 6, 9, 12, 13]), (16, [2, 5, 1, 15, 8, 11]),
                                       (22, [21, 0, 10, 4, 17, 6]), (24, [9, 10, 11, 12, 13, 14]),
                                       (24, [1, 2, 3, 4, 5, 6]), (22, [5, 9, 14, 17, 20, 21]),
                                       (23, [0, 1, 2, 7, 14, 22]), (20, [1, 7, 9, 12, 15, 18]),
                                       (20, [2, 6, 8, 10, 14, 19]), (21, [3, 5, 9, 11, 13, 20]),
                                       (21, [4, 6, 9, 11, 13, 20])])
def test_tc_pass_vs_oracle(lib, oracle, n, targets, precision):
    rng = np.random.default_rng(n * 100 + targets[0])
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    amp_rel, infid = TC_PASS_BOUND[precision]
    ctx = capi.rcs_create(n, precision)
    try:
        capi.rcs_state_write(ctx, psi0)
        want = psi0.astype(np.complex128)
        for rep in range(3):
            U = rand_unitary(64, rng)
            capi.rcs_apply_unitary(ctx, targets, U)
            capi.rcs_sync(ctx)
            got = capi.rcs_state_read(ctx).astype(np.complex128)
            prev = want.copy()
            oracle.apply_matrix(want, targets, U)
            # per-output bound: amp_rel * |slice|_2 <= amp_rel * max slice norm
            mask = sum(1 << t for t in targets)
            idx = np.arange(1 << n)
            base = idx & ~mask
            slice_norm2 = np.zeros(1 << n)
            np.add.at(slice_norm2, base, np.abs(prev) ** 2)
            bound = amp_rel * math.sqrt(slice_norm2.max())
            err = np.abs(got - want).max()
            assert err <= bound, (rep, err, bound)
            assert infidelity(got, want) <= infid
            want = got  # continue from the GPU's state
    finally:
        capi.rcs_destroy(ctx)


NORM_DRIFT_PER_TC_PASS = 2e-6


@pytest.mark.parametrize("precision", PRECS)
def test_echo_24q(lib, precision):
    """C followed by C^dagger returns |0...0>: no oracle needed, any size."""
    circ = C.generate(C.grid_for_n(24), cycles=14, pattern="ABCDCDAB", seed=31, jitter=0.05)
    plan = capi.rcs_plan_build(24, circ.gates, precision)
    passes = 2 * capi.rcs_plan_info(plan)["n_passes"]
    capi.rcs_plan_destroy(plan)
    ctx = capi.rcs_create(24, precision)
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        capi.rcs_apply_circuit(ctx, C.inverse_gates(circ.gates))
        a0 = capi.rcs_amplitudes(ctx, [0])[0]
        norm = capi.rcs_norm(ctx)
        assert abs(a0) ** 2 / norm >= 1 - INFID_TOL
        drift = NORM_DRIFT_PER_TC_PASS * passes if precision in TC_PRECS else 1e-5
        assert abs(norm - 1) <= drift, (norm, drift)
    finally:
        capi.rcs_destroy(ctx)


# ------------------------------------------------------------------ sampler and readout

def test_planted_state_sampler_exact(lib, oracle):
    n = 18
    psi = np.zeros(1 << n, dtype=np.complex64)
    support = {5: 0.5, 77_777: 0.25, 77_778: 0.125, (1 << n) - 1: 0.0625, 1 << 17: 0.0625}
    for i, pr in support.items():
        psi[i] = np.complex64(math.sqrt(pr) * np.exp(0.3j * i))
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED)
    try:
        capi.rcs_state_write(ctx, psi)
        shots = 100_000
        xs = capi.rcs_sample(ctx, shots, seed=12)
        xo = oracle.sample(psi.astype(np.complex128), shots, seed=12)
        assert set(np.unique(xs).tolist()) <= set(support)
        assert np.mean(xs == xo) >= 0.9999
        assert abs(capi.rcs_norm(ctx) - float(np.sum(np.abs(psi.astype(np.complex128)) ** 2))) <= 1e-12
        one = capi.rcs_sample(ctx, 1, seed=12)
        assert one[0] == xs[0]
    finally:
        capi.rcs_destroy(ctx)


def _floor_sq_2p62(x) -> int:
    """floor(x^2 * 2^62) of a float32, exactly, from its integer significand and exponent."""
    m, e = math.frexp(float(x))  # x = m 2^e, 0.5 <= |m| < 1 (exact for float32)
    mi = int(abs(m) * 2**24)  # 24-bit integer significand: x = mi 2^(e - 24)
    sh = 2 * (e - 24) + 62
    return (mi * mi) << sh if sh >= 0 else (mi * mi) >> -sh


def test_fixed_point_norm_is_exact(lib):
    """The norm is the exact sum of floor(x^2 2^62) over every float component: a state of
    small amplitudes (every exponent from subnormal to 2^-16, random significands) whose sum
    stays below 2^53 in those units reads back from rcs_norm without rounding; and single
    amplitudes of 1, 0.75 and 1.5 give their exact squares."""
    n = 16
    rng = np.random.default_rng(5)
    re = (rng.uniform(1, 2, 1 << n) * 2.0 ** rng.integers(-40, -22, 1 << n)).astype(np.float32)
    im = (rng.uniform(1, 2, 1 << n) * 2.0 ** rng.integers(-40, -22, 1 << n)).astype(np.float32)
    re[:8] = np.array([0.0, 1e-45, 2.0**-126, 2.0**-31, 2.0**-31 * 1.5, 2.0**-30, 2.0**-16, 2.0**-16 * 1.75],
                      dtype=np.float32)
    im[:4] = -re[4:8]
    psi = re + 1j * im
    want = sum(_floor_sq_2p62(v) for v in re) + sum(_floor_sq_2p62(v) for v in im)
    assert want < 2**53
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED)
    try:
        capi.rcs_state_write(ctx, psi.astype(np.complex64))
        assert capi.rcs_norm(ctx) * 2.0**62 == float(want)
        for a in (1.0, 0.75, 1.5):
            one = np.zeros(1 << n, dtype=np.complex64)
            one[12345] = a
            capi.rcs_state_write(ctx, one)
            assert capi.rcs_norm(ctx) == a * a
            assert np.all(capi.rcs_sample(ctx, 1000, seed=3) == 12345)
    finally:
        capi.rcs_destroy(ctx)


def test_zero_state_sampler(lib):
    """A state of norm 0 has no distribution to draw from: every shot reads 2^64 - 1."""
    n = 14
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED)
    try:
        capi.rcs_state_write(ctx, np.zeros(1 << n, dtype=np.complex64))
        assert capi.rcs_norm(ctx) == 0.0
        xs = capi.rcs_sample(ctx, 5000, seed=1)
        assert np.all(xs == np.uint64(2**64 - 1))
    finally:
        capi.rcs_destroy(ctx)


@pytest.mark.parametrize("n", [1, 2, 3, 9, 10, 11])
def test_small_and_ragged_states(lib, oracle, n):
    circ = C.generate(C.grid_for_n(n), cycles=3, seed=n)
    want = oracle.simulate(n, circ.gates)
    for prec in PRECS:
        ctx = run_gpu(n, circ.gates, prec)
        try:
            got = capi.rcs_state_read(ctx)
            assert np.abs(got - want).max() <= AMP_TOL
            xs = capi.rcs_sample(ctx, 3000, seed=4)
            xo = oracle.sample(got.astype(np.complex128), 3000, seed=4)
            assert np.mean(xs == xo) >= 0.999
            assert abs(capi.rcs_xeb(ctx, xs) - oracle.xeb(got.astype(np.complex128), xs)) <= 1e-9
        finally:
            capi.rcs_destroy(ctx)


def test_amplitudes_and_errors(lib):
    n = 16
    circ = C.generate(C.grid_for_n(n), cycles=4, seed=3)
    ctx = run_gpu(n, circ.gates, capi.RCS_PREC_FP32_FUSED)
    try:
        full = capi.rcs_state_read(ctx)
        idx = np.random.default_rng(0).integers(0, 1 << n, size=5000, dtype=np.uint64)
        amps = capi.rcs_amplitudes(ctx, idx)
        np.testing.assert_array_equal(amps, full[idx.astype(np.int64)].astype(np.complex128))
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_amplitudes(ctx, [1 << n])
        assert e.value.code == capi.RCS_ERR_ARG
        with pytest.raises(capi.RcsError):
            capi.rcs_xeb(ctx, [0, 1 << n])
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_apply_circuit(ctx, np.array([C.make_gate(C.SQRT_X, n)]))
        assert e.value.code == capi.RCS_ERR_QUBIT
        # dense unitaries take 1..7 targets; a list with a bad entry is rejected before any runs
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_apply_unitary(ctx, list(range(8)), np.eye(256))
        assert e.value.code == capi.RCS_ERR_ARG and "1..7" in str(e.value)
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_apply_unitaries(ctx, [(list(range(7)), np.eye(128)), (list(range(8)), np.eye(256))])
        assert e.value.code == capi.RCS_ERR_ARG
        # the state is unchanged by the rejected calls
        np.testing.assert_array_equal(capi.rcs_state_read(ctx), full)
    finally:
        capi.rcs_destroy(ctx)


def test_device_pointer_calls(lib, oracle):
    torch = pytest.importorskip("torch")
    n = 20
    circ = C.generate(C.grid_for_n(n), cycles=6, seed=8)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = capi.rcs_create(n, capi.RCS_PREC_BF16X3, stream=stream)
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        shots = 50_000
        d_bits = torch.empty(shots, dtype=torch.int64, device="cuda")
        d_xeb = torch.empty(1, dtype=torch.float64, device="cuda")
        capi.rcs_sample_device(ctx, shots, 5, d_bits.data_ptr())
        capi.rcs_xeb_device(ctx, d_bits.data_ptr(), shots, d_xeb.data_ptr())
        torch.cuda.current_stream().synchronize()
        xs = d_bits.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(xs, capi.rcs_sample(ctx, shots, 5))
        assert abs(float(d_xeb.item()) - capi.rcs_xeb(ctx, xs)) <= 1e-12
        bad = torch.tensor([1 << n], dtype=torch.int64, device="cuda")
        capi.rcs_xeb_device(ctx, bad.data_ptr(), 1, d_xeb.data_ptr())
        torch.cuda.current_stream().synchronize()
        assert math.isnan(float(d_xeb.item()))
    finally:
        capi.rcs_destroy(ctx)


@pytest.mark.parametrize("n,precision", [(20, capi.RCS_PREC_BF16X3), (24, capi.RCS_PREC_FP32_FUSED)])
def test_sampler_follows_caller_order_in_any_layout(lib, oracle, n, precision):
    """With the state stored in a permuted qubit layout, the sampler still draws
    x = min{i : C_i > u T} with C in the circuit's own index order: the same shots as
    the oracle sampler on the same state, drawn before anything restores the layout."""
    circ = C.generate(C.grid_for_n(n), cycles=8, pattern="EFGH", seed=123)
    ctx = capi.rcs_create(circ.grid, precision)
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        phys = capi.rcs_qubit_layout(ctx)
        assert any(int(p) != q for q, p in enumerate(phys)), "the test needs a non-identity layout"
        shots, seed = 100_000, 77
        xs = capi.rcs_sample(ctx, shots, seed)
        norm = capi.rcs_norm(ctx)
        F = capi.rcs_xeb(ctx, xs)
        got = capi.rcs_state_read(ctx).astype(np.complex128)  # restores the identity layout
        assert abs(np.vdot(got, got).real - norm) <= 1e-9
        xo = oracle.sample(got, shots, seed)
        assert np.mean(xs == xo) >= 0.9999
        assert abs(F - oracle.xeb(got, xs)) <= 1e-9
        assert np.array_equal(capi.rcs_sample(ctx, shots, seed), xs)  # identity layout now: same draws
    finally:
        capi.rcs_destroy(ctx)
