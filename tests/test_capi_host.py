"""C-ABI library on the CPU: it loads, exports every declared symbol, and its host
logic (gate validation, the fusion planner) is right. No GPU call is made here."""
import os
import re

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(rcs_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    bound = {n for n, _, _ in capi.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_error_messages_without_gpu(lib):
    with pytest.raises(capi.RcsError) as e:
        capi.rcs_plan_build(4, np.array([C.make_gate(C.SQRT_X, 7)]))
    assert e.value.code == capi.RCS_ERR_QUBIT
    assert "out of range" in str(e.value)
    with pytest.raises(capi.RcsError) as e:
        capi.rcs_plan_build(4, np.array([C.make_gate(C.FSIM, 1, 1)]))
    assert e.value.code == capi.RCS_ERR_QUBIT
    bad = np.array([C.make_gate(C.U1, 0)])
    with pytest.raises(capi.RcsError) as e:
        capi.rcs_plan_build(4, bad, umats={0: np.array([[1, 1], [0, 1]])})
    assert e.value.code == capi.RCS_ERR_ARG
    with pytest.raises(capi.RcsError):
        capi.rcs_plan_build(4, np.array([C.make_gate(9, 0)]))
    with pytest.raises(capi.RcsError):
        capi.rcs_plan_build(40, np.zeros(0, dtype=C.GATE_DTYPE))
    # FP32 fused widths are 2..7
    gates = C.generate(C.grid_for_n(10), cycles=2, pattern="EFGH", seed=1).gates
    for k in (1, 8):
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_plan_build(10, gates, capi.RCS_PREC_FP32_FUSED, k)
        assert e.value.code == capi.RCS_ERR_ARG and "2..7" in str(e.value)


def _plan_passes(plan):
    info = capi.rcs_plan_info(plan)
    return info, [capi.rcs_plan_pass(plan, i) for i in range(info["n_passes"])]


@pytest.mark.parametrize("precision,kmax,n", [(capi.RCS_PREC_FP32_FUSED, 2, 10), (capi.RCS_PREC_FP32_FUSED, 4, 10),
                                              (capi.RCS_PREC_FP32_FUSED, 5, 9), (capi.RCS_PREC_BF16X3, 0, 13),
                                              (capi.RCS_PREC_FP32_FUSED, 4, 14), (capi.RCS_PREC_FP32_PLAIN, 0, 9),
                                              (capi.RCS_PREC_TF32X3, 0, 14), (capi.RCS_PREC_BF16X3, 0, 20),
                                              (capi.RCS_PREC_FP32_FUSED, 6, 12), (capi.RCS_PREC_FP32_FUSED, 7, 13)])
def test_fused_plan_reproduces_circuit(oracle, lib, precision, kmax, n):
    """Applying the planned passes (FP64 matrices) with the oracle equals applying
    the circuit gate by gate with the oracle."""
    grid = C.grid_for_n(n)
    circ = C.generate(grid, cycles=6, pattern="EFGH", seed=17, jitter=0.05)
    plan = capi.rcs_plan_build(n, circ.gates, precision, kmax)
    try:
        info, passes = _plan_passes(plan)
        phys = capi.rcs_plan_layout(plan, n)
    finally:
        capi.rcs_plan_destroy(plan)
    want = oracle.simulate(n, circ.gates)
    psi = oracle.zero_state(n)
    for targets, U in passes:
        assert list(targets) == sorted(targets)
        np.testing.assert_allclose(U @ U.conj().T, np.eye(len(U)), atol=1e-12)
        oracle.apply_matrix(psi, targets, U)
    # the passes act on the stored layout: circuit qubit q sits at bit phys[q]
    assert sorted(phys.tolist()) == list(range(n))
    idx = np.arange(1 << n)
    stored = np.zeros(1 << n, dtype=np.int64)
    for q in range(n):
        stored |= ((idx >> q) & 1) << int(phys[q])
    np.testing.assert_allclose(psi[stored], want, atol=1e-12)
    assert info["n_gates"] == len(circ.gates)
    if precision == capi.RCS_PREC_FP32_PLAIN:
        assert info["n_passes"] == len(circ.gates)
    elif precision in (capi.RCS_PREC_BF16X3, capi.RCS_PREC_TF32X3):
        assert all(len(t) == 6 for t, _ in passes)
    else:
        assert max(len(t) for t, _ in passes) <= kmax
        assert info["n_passes"] < len(circ.gates)


def test_fusion_counts_34q():
    circ = C.config_circuit("34q_5x7m1_20cyc")
    counts = {}
    for prec, k in [(capi.RCS_PREC_FP32_PLAIN, 0), (capi.RCS_PREC_FP32_FUSED, 4), (capi.RCS_PREC_BF16X3, 0)]:
        plan = capi.rcs_plan_build(34, circ.gates, prec, k)
        info = capi.rcs_plan_info(plan)
        capi.rcs_plan_destroy(plan)
        counts[prec] = info["n_passes"]
        assert info["hbm_bytes"] == 16.0 * 2**34 * info["n_passes"]
    assert counts[capi.RCS_PREC_FP32_PLAIN] == 994
    assert counts[capi.RCS_PREC_FP32_FUSED] < 100
    assert counts[capi.RCS_PREC_BF16X3] < 60


def test_plan_pass_targets_and_adjoint(oracle, lib):
    # a U2 gate with reversed qubit order and the adjoint flag
    rng = np.random.default_rng(3)
    A = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    Q, _ = np.linalg.qr(A)
    g = C.make_gate(C.U2, 5, 2, flags=C.ADJOINT)
    plan = capi.rcs_plan_build(6, np.array([g]), capi.RCS_PREC_FP32_PLAIN, 0, umats={0: Q})
    t, U = capi.rcs_plan_pass(plan, 0)
    capi.rcs_plan_destroy(plan)
    assert list(t) == [2, 5]
    psi0 = rng.normal(size=64) + 1j * rng.normal(size=64)
    want = oracle.apply_matrix(psi0.copy(), [5, 2], Q.conj().T)
    got = oracle.apply_matrix(psi0.copy(), list(t), U)
    np.testing.assert_allclose(got, want, atol=1e-12)


def test_layout_keeps_low_bits_apart():
    """On the 34-qubit workload the chosen layout puts circuit qubits that never share
    a pass on bits 0..4: no tensor-core pass targets two of them."""
    circ = C.config_circuit("34q_5x7m1_20cyc")
    plan = capi.rcs_plan_build(34, circ.gates, capi.RCS_PREC_BF16X3)
    try:
        info, passes = _plan_passes(plan)
        phys = capi.rcs_plan_layout(plan, 34)
    finally:
        capi.rcs_plan_destroy(plan)
    assert sorted(phys.tolist()) == list(range(34))
    assert sum(int(p != q) for q, p in enumerate(phys)) <= 10  # at most five transpositions
    for targets, _ in passes:
        assert sum(1 for t in targets if t < 5) <= 1, targets


def test_zero_state_plan_uses_a_substate_prefix():
    """A plan for a fresh state is chosen by cost with the sub-state prefix counted: on
    the 34-qubit workload most of the early passes run on a sub-state of at most n - 2
    qubits, leaving at most 30 full-state passes (greedy fewest-blocks planning: 37)."""
    circ = C.config_circuit("34q_5x7m1_20cyc")
    plan = capi.rcs_plan_build(34, circ.gates, capi.RCS_PREC_BF16X3)
    try:
        info, passes = _plan_passes(plan)
    finally:
        capi.rcs_plan_destroy(plan)
    pre, m = info["prefix_passes"], info["prefix_qubits"]
    assert pre >= 8 and 13 <= m <= 32
    assert info["n_passes"] - pre <= 30
    union = set()
    for t, _ in passes[:pre]:
        union |= set(int(x) for x in t)
    assert len(union) <= m


def test_zero_state_byte_count():
    """rcs_plan_stats.zero_hbm_bytes, the algorithmic bytes of a run from |0...0>: with no
    sub-state prefix it is exactly the zero fill plus 16 x 2^n per pass. With one, each stage's
    passes count at that stage's size, plus the zero fill of the first sub-state, the expansions,
    and the first full pass reading the last sub-state (8 x 2^m in, 8 x 2^n out): it lies between
    the bounds that the passes' growing target union and the widest sub-state give."""
    circ = C.config_circuit("34q_5x7m1_20cyc")
    n = 34
    plain = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_FP32_PLAIN)
    try:
        info = capi.rcs_plan_info(plain)
        assert info["prefix_passes"] == 0
        assert info["zero_hbm_bytes"] == 8.0 * 2**n + 16.0 * 2**n * info["n_passes"]
    finally:
        capi.rcs_plan_destroy(plain)
    plan = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_BF16X3)
    try:
        info, passes = _plan_passes(plan)
    finally:
        capi.rcs_plan_destroy(plan)
    assert info["pair_passes"] == 0
    pre = info["prefix_passes"]
    assert pre > 0 and info["prefix_stages"] >= 1
    # the union of targets after each prefix pass: no stage is narrower than the union of the
    # targets so far (nor than 13 qubits, one tensor-core tile), none wider than the last
    unions = []
    u = set()
    for t, _ in passes[:pre]:
        u |= set(int(x) for x in t)
        unions.append(len(u))
    m_last = info["prefix_qubits"]
    assert unions[-1] <= m_last
    # every pass of the prefix runs on a state of at most m_last qubits and at least 13
    lo = 8.0 * 2**13 + sum(16.0 * 2**max(13, s) for s in unions) + 8.0 * 2**m_last + 8.0 * 2**n
    hi = 8.0 * 2**m_last + 16.0 * 2**m_last * pre + 8.0 * 2**m_last * 2 * info["prefix_stages"] + 8.0 * 2**n
    full = 16.0 * 2**n * (info["n_passes"] - pre - 1)  # the first full pass reads the sub-state
    assert lo + full <= info["zero_hbm_bytes"] <= hi + full
    assert info["zero_hbm_bytes"] < info["hbm_bytes"]
    # the same plan with two-unitary round trips (opt-in): the same passes; every pair saves
    # one round trip of the state it runs on, and the full-state passes after the first pair
    # up in order
    plan = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_BF16X3, flags=capi.RCS_OPT_PAIR_PASSES)
    try:
        info2, passes2 = _plan_passes(plan)
    finally:
        capi.rcs_plan_destroy(plan)
    assert [tuple(t) for t, _ in passes2] == [tuple(t) for t, _ in passes]
    n_full = info["n_passes"] - pre - 1
    saved = info["zero_hbm_bytes"] - info2["zero_hbm_bytes"]
    assert n_full // 2 <= info2["pair_passes"] <= info["n_passes"] // 2
    assert 16.0 * 2**n * (n_full // 2) <= saved <= 16.0 * 2**n * info2["pair_passes"]


@pytest.mark.parametrize("name,full_max,stages", [("34q_5x7m1_20cyc", 26, 3), ("30q_5x6_14cyc", 17, 3),
                                                  ("32q_4x8_20cyc", 28, 2)])
def test_closure_search_pass_counts(name, full_max, stages):
    """The closure search and the three-stage candidates: at k = 6 the plans from |0...0> keep
    at most this many full-state passes (the grown-block beams and two-stage candidates alone
    gave 27, 18 and 29), and their cost in full-pass units is below the previous plans'."""
    circ = C.config_circuit(name)
    n = circ.n_qubits
    plan = capi.rcs_plan_build(n, circ.gates, capi.RCS_PREC_BF16X3)
    try:
        info = capi.rcs_plan_info(plan)
    finally:
        capi.rcs_plan_destroy(plan)
    assert info["n_passes"] - info["prefix_passes"] <= full_max
    assert info["prefix_stages"] == stages
    previous = {"34q_5x7m1_20cyc": 7.585e12, "30q_5x6_14cyc": 0.325e12, "32q_4x8_20cyc": 1.976e12}[name]
    assert info["zero_hbm_bytes"] < previous


def test_plans_are_deterministic():
    """The searches run on host threads; every step is merged in index order, so two builds of
    the same circuit give the same passes, bit for bit."""
    circ = C.config_circuit("30q_5x6_14cyc")
    out = []
    for _ in range(2):
        plan = capi.rcs_plan_build(30, circ.gates, capi.RCS_PREC_BF16X3)
        try:
            info, passes = _plan_passes(plan)
            out.append((info, passes, capi.rcs_plan_layout(plan, 30)))
        finally:
            capi.rcs_plan_destroy(plan)
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][2], out[1][2])
    for (t0, u0), (t1, u1) in zip(out[0][1], out[1][1]):
        np.testing.assert_array_equal(t0, t1)
        np.testing.assert_array_equal(u0, u1)


@pytest.mark.parametrize("n,layers", [(12, 6), (20, 10)])
def test_densely_coupled_plan_reproduces_circuit(oracle, lib, n, layers):
    """fSim gates on random qubit pairs, a fresh pairing per layer: at 12 qubits (32 coupled pairs)
    the closure search runs over the 829 connected 6-sets of the coupling graph; at 20 qubits (77
    pairs) there are 25 092, more than the 20 000 it takes, so the planner keeps the grown-block
    searches alone. Either way the planned passes, applied with the oracle, equal the circuit."""
    rng = np.random.default_rng(n)
    gates = []
    for layer in range(layers):
        for q in range(n):
            gates.append(C.make_gate(int(rng.integers(0, 3)), q))
        perm = rng.permutation(n)
        for i in range(0, n - 1, 2):
            gates.append(C.make_gate(C.FSIM, int(perm[i]), int(perm[i + 1]), theta=float(rng.uniform(0, np.pi)),
                                     phi=float(rng.uniform(0, np.pi))))
    gates = np.array(gates)
    want = oracle.simulate(n, gates)
    for prec in (capi.RCS_PREC_BF16X3, capi.RCS_PREC_FP32_FUSED):
        plan = capi.rcs_plan_build(n, gates, prec)
        try:
            info, passes = _plan_passes(plan)
            phys = capi.rcs_plan_layout(plan, n)
        finally:
            capi.rcs_plan_destroy(plan)
        psi = oracle.zero_state(n)
        for targets, U in passes:
            oracle.apply_matrix(psi, targets, U)
        idx = np.arange(1 << n)
        stored = np.zeros(1 << n, dtype=np.int64)
        for q in range(n):
            stored |= ((idx >> q) & 1) << int(phys[q])
        np.testing.assert_allclose(psi[stored], want, atol=1e-12)
        assert info["n_passes"] < len(gates)


@pytest.mark.parametrize("kmax,n,extra", [(2, 16, 0), (3, 16, 0), (5, 17, 0), (7, 16, 0), (6, 17, 2)])
def test_staged_closure_plans_reproduce_circuit(oracle, lib, kmax, n, extra):
    """Plans from |0...0> at 16-19 qubits have staged candidates, so the closure search blocks
    their stages and their rest, at every fusion width. `extra` qubits carry single-qubit gates
    only (no coupler), which only the search's grown-block moves can place. The planned passes,
    applied with the oracle, equal the circuit."""
    circ = C.generate(C.grid_for_n(n), cycles=8, pattern="ABCDCDAB", seed=23, jitter=0.05)
    gates = list(circ.gates)
    rng = np.random.default_rng(kmax)
    for q in range(n, n + extra):
        for _ in range(5):
            gates.insert(int(rng.integers(0, len(gates) + 1)), C.make_gate(int(rng.integers(0, 3)), q))
    gates = np.array(gates)
    m = n + extra
    prec = capi.RCS_PREC_BF16X3 if kmax == 6 else capi.RCS_PREC_FP32_FUSED
    plan = capi.rcs_plan_build(m, gates, prec, 0 if kmax == 6 else kmax)
    try:
        info, passes = _plan_passes(plan)
        phys = capi.rcs_plan_layout(plan, m)
    finally:
        capi.rcs_plan_destroy(plan)
    assert info["prefix_passes"] > 0
    want = oracle.simulate(m, gates)
    psi = oracle.zero_state(m)
    for targets, U in passes:
        assert len(targets) <= max(kmax, 6 if prec == capi.RCS_PREC_BF16X3 else kmax)
        oracle.apply_matrix(psi, targets, U)
    idx = np.arange(1 << m)
    stored = np.zeros(1 << m, dtype=np.int64)
    for q in range(m):
        stored |= ((idx >> q) & 1) << int(phys[q])
    np.testing.assert_allclose(psi[stored], want, atol=1e-12)
