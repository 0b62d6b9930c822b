"""Batched mode (one persistent launch in one captured graph) vs the CPU oracle.

Same tolerances as the single-circuit tests: infidelity <= 1e-5, max amplitude
error <= 1e-6, sampler agreement with the oracle sampler on the same state
>= 99.99%, XEB equal to the oracle's on the same samples to 1e-9."""
import math
import time

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def infidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def small_batch():
    out = []
    for i, (n, cyc, pat) in enumerate([(12, 6, "ABCDCDAB"), (14, 9, "EFGH"), (16, 12, "ABCDCDAB"),
                                       (17, 10, "EFGH"), (19, 8, "ABCDCDAB"), (20, 11, "EFGH")]):
        out.append(C.generate(C.grid_for_n(n), cyc, pat, seed=500 + i, jitter=0.05 * (i % 2)))
    return out


@pytest.mark.parametrize("k_max", [0, 3, 5])
def test_batch_vs_oracle(lib, oracle, k_max):
    circs = small_batch()
    shots = 20_000
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, shots, 40 + i) for i, c in enumerate(circs)], k_max=k_max,
                              autotune=int(k_max == 0))
    try:
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        assert capi.rcs_batch_size(b) == len(circs)
        with pytest.raises(capi.RcsError) as e:  # the FP32 engine has no persistent tensor-core kernel
            capi.rcs_batch_tuning(b)
        assert e.value.code == capi.RCS_ERR_UNSUPPORTED
        for i, c in enumerate(circs):
            info = capi.rcs_batch_info(b, i)
            assert info["n_qubits"] == c.n_qubits and 2 <= info["k"] <= 5
            if k_max:
                assert info["k"] == min(k_max, c.n_qubits)
            want = oracle.simulate(c.n_qubits, c.gates)
            got = capi.rcs_batch_state_read(b, i)
            assert infidelity(got, want) <= 1e-5
            assert np.abs(got - want).max() <= 1e-6
            xs, F = capi.rcs_batch_result(b, i, shots)
            g128 = got.astype(np.complex128)
            xo = oracle.sample(g128, shots, 40 + i)
            assert np.mean(xs == xo) >= 0.9999
            assert abs(F - oracle.xeb(g128, xs)) <= 1e-9
    finally:
        capi.rcs_batch_destroy(b)


def test_batch_replay_is_deterministic(lib):
    circs = small_batch()[:4]
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, 5000, 7) for c in circs], k_max=4, autotune=0)
    try:
        runs = []
        for _ in range(2):
            capi.rcs_batch_launch(b)
            capi.rcs_batch_wait(b)
            runs.append([capi.rcs_batch_result(b, i, 5000) for i in range(len(circs))])
        for (x0, f0), (x1, f1) in zip(*runs):
            np.testing.assert_array_equal(x0, x1)
            assert f0 == f1
    finally:
        capi.rcs_batch_destroy(b)


def test_batch_wait_limit_reports_timeout(lib, oracle):
    """A work item that never publishes its completion makes the next pass of its
    circuit wait past the limit: the launch ends with RCS_ERR_TIMEOUT, the device
    stays usable, and a normal launch afterwards gives correct states."""
    circs = small_batch()[:3]
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, 1000, 3) for c in circs], k_max=4, autotune=0)
    try:
        capi.rcs_batch_set_fault(b, 0, 0.1)  # item 0 = first item of the first pass
        capi.rcs_batch_launch(b)
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_batch_wait(b)
        assert e.value.code == capi.RCS_ERR_TIMEOUT
        capi.rcs_batch_set_fault(b, -1)
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        for i, c in enumerate(circs):
            got = capi.rcs_batch_state_read(b, i)
            assert infidelity(got, oracle.simulate(c.n_qubits, c.gates)) <= 1e-5
    finally:
        capi.rcs_batch_destroy(b)


@pytest.mark.parametrize("precision", [capi.RCS_PREC_FP32_FUSED, capi.RCS_PREC_BF16X3])
def test_batch_run_one_call(lib, oracle, precision):
    """rcs_batch_run (grids, gate lists, shots and seeds in, samples and XEB out, in one
    call) gives the draws and scores of the same batch built and launched step by step,
    and samples that follow each circuit's oracle distribution."""
    circs = small_batch()[:4]
    items = [(c.n_qubits, c.gates, 3000 + 1000 * i, 40 + i) for i, c in enumerate(circs)]
    res = capi.rcs_batch_run([(c.grid, c.gates, sh, sd) for c, (_, _, sh, sd) in zip(circs, items)],
                             precision=precision, k_max=4 if precision == capi.RCS_PREC_FP32_FUSED else 0,
                             autotune=0)
    b = capi.rcs_batch_create(items, k_max=4 if precision == capi.RCS_PREC_FP32_FUSED else 0, autotune=0,
                              precision=precision)
    try:
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        for i, (c, (_, _, sh, _)) in enumerate(zip(circs, items)):
            xs, F = capi.rcs_batch_result(b, i, sh)
            np.testing.assert_array_equal(res[i][0], xs)
            assert res[i][1] == F
            want = oracle.simulate(c.n_qubits, c.gates)
            assert abs(F - oracle.xeb(want, xs)) <= 5e-3
    finally:
        capi.rcs_batch_destroy(b)
    with pytest.raises(capi.RcsError) as e:
        capi.rcs_batch_run([], precision=precision)
    assert e.value.code == capi.RCS_ERR_ARG


def test_batch_rejects_bad_input(lib):
    c = small_batch()[0]
    with pytest.raises(capi.RcsError):
        capi.rcs_batch_create([(c.n_qubits, c.gates, 10, 1), (40, c.gates, 10, 1)])
    bad = c.gates.copy()
    bad["q0"][3] = 99
    with pytest.raises(capi.RcsError) as e:
        capi.rcs_batch_create([(c.n_qubits, bad, 10, 1)])
    assert e.value.code == capi.RCS_ERR_QUBIT


def test_batched_workload_64(lib, oracle):
    """The batched workload: 64 circuits, 16-26 qubits, 10-20 cycles, 10^5 shots each."""
    circs = C.batch_workload(64, 1000)
    shots = 100_000
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, shots, c.seed) for c in circs])
    try:
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        checked = 0
        for i, c in enumerate(circs):
            got = capi.rcs_batch_state_read(b, i).astype(np.complex128)
            p = np.abs(got) ** 2
            T = p.sum()
            assert abs(T - 1) <= 1e-5
            xs, F = capi.rcs_batch_result(b, i, shots)
            assert (p[xs.astype(np.int64)] > 0).all()
            # ideal sampling: E[F] = 2^n sum (p/T)^2 - 1, sd = 2^n sd(p(x)/T) / sqrt(N)
            q = p / T
            mean = (1 << c.n_qubits) * float(np.sum(q * q)) - 1
            sd = (1 << c.n_qubits) * math.sqrt(max(float(np.sum(q ** 3)) - float(np.sum(q * q)) ** 2, 0)) / math.sqrt(shots)
            assert abs(F - mean) <= 6 * sd + 1e-9, (i, F, mean, sd)
            if c.n_qubits <= 20 and checked < 6:
                assert infidelity(got, oracle.simulate(c.n_qubits, c.gates)) <= 1e-5
                checked += 1
        assert checked >= 3
    finally:
        capi.rcs_batch_destroy(b)


# ------------------------------------------------------------------ tensor-core engine

@pytest.mark.parametrize("precision", [capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3])
def test_batch_tensor_core_vs_oracle(lib, oracle, precision):
    """The tensor-core engine: each circuit planned with its own layout and sub-state
    prefix, the passes of every circuit of 13 or more qubits in the persistent kernel
    (12 qubits: FP32 fused passes in a launch chain of its own), states, samples and XEB
    in the circuit's own qubit numbering."""
    circs = small_batch()
    shots = 20_000
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, shots, 40 + i) for i, c in enumerate(circs)],
                              precision=precision)
    try:
        for _ in range(2):  # the graph replays
            capi.rcs_batch_launch(b)
            capi.rcs_batch_wait(b)
        for i, c in enumerate(circs):
            info = capi.rcs_batch_info(b, i)
            assert info["k"] == (6 if c.n_qubits >= 13 else 5)
            want = oracle.simulate(c.n_qubits, c.gates)
            got = capi.rcs_batch_state_read(b, i)
            assert infidelity(got, want) <= 1e-5
            assert np.abs(got - want).max() <= 1e-6
            xs, F = capi.rcs_batch_result(b, i, shots)
            g128 = got.astype(np.complex128)
            assert np.mean(xs == oracle.sample(g128, shots, 40 + i)) >= 0.9999
            assert abs(F - oracle.xeb(g128, xs)) <= 1e-9
    finally:
        capi.rcs_batch_destroy(b)


@pytest.mark.parametrize("precision", [capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3])
def test_batch_tensor_core_wait_limit_reports_timeout(lib, oracle, precision):
    """The persistent tensor-core kernel's bounded waits: a work item that never publishes
    its completion (everything it issued still completes) makes the next pass of its
    circuit wait past a short limit; the launch ends with RCS_ERR_TIMEOUT, every CTA stops,
    and after the hook is cleared a normal launch gives the oracle's states."""
    circs = small_batch()[1:4]  # 14, 16, 17 qubits: all in the persistent kernel
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, 1000, 3) for c in circs], precision=precision)
    try:
        capi.rcs_batch_set_fault(b, 0, 0.05)
        t0 = time.perf_counter()
        capi.rcs_batch_launch(b)
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_batch_wait(b)
        assert e.value.code == capi.RCS_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 1.0  # one short limit, not the default
        capi.rcs_batch_set_fault(b, -1)
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        for i, c in enumerate(circs):
            got = capi.rcs_batch_state_read(b, i)
            assert infidelity(got, oracle.simulate(c.n_qubits, c.gates)) <= 1e-5
    finally:
        capi.rcs_batch_destroy(b)


def test_batched_workload_64_tensor_core(lib, oracle):
    circs = C.batch_workload(64, 1000)
    shots = 100_000
    b = capi.rcs_batch_create([(c.n_qubits, c.gates, shots, c.seed) for c in circs], precision=capi.RCS_PREC_BF16X3)
    try:
        capi.rcs_batch_launch(b)
        capi.rcs_batch_wait(b)
        checked = 0
        for i, c in enumerate(circs):
            got = capi.rcs_batch_state_read(b, i).astype(np.complex128)
            p = np.abs(got) ** 2
            T = p.sum()
            assert abs(T - 1) <= 2e-6 * capi.rcs_batch_info(b, i)["n_passes"]
            xs, F = capi.rcs_batch_result(b, i, shots)
            assert (p[xs.astype(np.int64)] > 0).all()
            q = p / T
            mean = (1 << c.n_qubits) * float(np.sum(q * q)) - 1
            sd = (1 << c.n_qubits) * math.sqrt(max(float(np.sum(q ** 3)) - float(np.sum(q * q)) ** 2, 0)) / math.sqrt(shots)
            assert abs(F - mean) <= 6 * sd + 1e-9, (i, F, mean, sd)
            if c.n_qubits <= 20 and checked < 6:
                assert infidelity(got, oracle.simulate(c.n_qubits, c.gates)) <= 1e-5
                checked += 1
        assert checked >= 3
    finally:
        capi.rcs_batch_destroy(b)


def test_batch_tensor_core_edge_cases(lib, oracle):
    """Persistent tensor-core engine at its edges, in one batch: a 13-qubit circuit (one tile,
    items of one tile), a circuit with no gates (|0...0>: not a persistent-kernel circuit, it
    runs as its own chain), circuits without shots next to ones with shots, and a 14-qubit
    circuit whose first pass reads |0...0> directly (a sub-state would have under 13 qubits)."""
    circs = [C.generate(C.grid_for_n(13), 8, "ABCDCDAB", seed=71),
             C.generate(C.grid_for_n(14), 9, "EFGH", seed=72, jitter=0.05),
             C.generate(C.grid_for_n(18), 10, "ABCDCDAB", seed=73)]
    items = [(circs[0].n_qubits, circs[0].gates, 0, 1), (circs[1].n_qubits, circs[1].gates, 4000, 2),
             (14, np.zeros(0, dtype=C.GATE_DTYPE), 500, 3), (circs[2].n_qubits, circs[2].gates, 0, 4)]
    b = capi.rcs_batch_create(items, precision=capi.RCS_PREC_BF16X3)
    try:
        tuning = capi.rcs_batch_tuning(b)
        assert tuning["tiles_per_item"] in (2, 4, 8, 16, 32)
        for _ in range(2):
            capi.rcs_batch_launch(b)
            capi.rcs_batch_wait(b)
        for i, c in [(0, circs[0]), (1, circs[1]), (3, circs[2])]:
            got = capi.rcs_batch_state_read(b, i)
            want = oracle.simulate(c.n_qubits, c.gates)
            assert infidelity(got, want) <= 1e-5
            assert np.abs(got - want).max() <= 1e-6
        zero = capi.rcs_batch_state_read(b, 2)
        assert zero[0] == 1 and np.count_nonzero(zero) == 1
        xs, F = capi.rcs_batch_result(b, 2, 500)
        assert (xs == 0).all() and abs(F - ((1 << 14) - 1)) <= 1e-9  # XEB of a basis state: 2^n - 1
        xs, F = capi.rcs_batch_result(b, 1, 4000)
        g128 = capi.rcs_batch_state_read(b, 1).astype(np.complex128)
        assert np.mean(xs == oracle.sample(g128, 4000, 2)) >= 0.9999
    finally:
        capi.rcs_batch_destroy(b)
