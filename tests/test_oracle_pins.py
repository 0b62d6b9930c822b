"""Pins of the CPU oracle against facts fixed by mathematics, not by the oracle.

Each check is chosen so a plausible mistake in the oracle (a wrong sign in a
gate, a transposed matrix, a wrong bit in the index arithmetic, an off-by-one in
the inverse CDF, a dropped 2^n in XEB) fails at least one of them:

* gate matrices: algebraic identities ((sqrtP)^2 = P, principal branch,
  matrix exponentials from scipy, fSim special cases CZ / iSWAP / identity);
* state update: the full 2^n x 2^n operator built from Kronecker products of
  per-qubit 2x2 factors (numpy), and an independent einsum tensor contraction;
* invariants: norm conservation, echo (C then C^dagger gives |0>),
  Porter-Thomas statistics of a random circuit;
* sampling: numpy's own Philox4x64-10 stream plus numpy.searchsorted on a
  cumulative sum; exact frequencies on a planted sparse state; chi-squared on
  the uniform state made by a sqrtY layer;
* XEB: E[F] = 2^n sum p^2 - 1 under ideal sampling, E[F] = 0 for uniformly
  random bitstrings, F = 2^n - 1 on a basis state.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from paper_2512_07311_gb300 import circuits as C

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
W = (X + Y) / math.sqrt(2)
I2 = np.eye(2, dtype=complex)


# ------------------------------------------------------------------ gate matrices

@pytest.mark.parametrize("kind,P", [(C.SQRT_X, X), (C.SQRT_Y, Y), (C.SQRT_W, W)])
def test_sqrt_gates_square_to_pauli(oracle, kind, P):
    m = oracle.gate_matrix(kind)
    np.testing.assert_allclose(m @ m, P, atol=1e-15)
    np.testing.assert_allclose(m @ m.conj().T, I2, atol=1e-15)


@pytest.mark.parametrize("kind,P", [(C.SQRT_X, X), (C.SQRT_Y, Y), (C.SQRT_W, W)])
def test_sqrt_gates_principal_branch(oracle, kind, P):
    # principal root of an involution: eigenvalues {1, i}; equals e^{i pi/4} exp(-i pi P / 4)
    m = oracle.gate_matrix(kind)
    ev = np.sort_complex(np.linalg.eigvals(m))
    np.testing.assert_allclose(ev, np.sort_complex(np.array([1, 1j])), atol=1e-14)
    np.testing.assert_allclose(m, np.exp(1j * math.pi / 4) * scipy.linalg.expm(-1j * math.pi / 4 * P), atol=1e-14)
    np.testing.assert_allclose(m, scipy.linalg.sqrtm(P), atol=1e-12)


def test_sqrt_w_matches_config_definition(oracle):
    # sqrtW = sqrt((X+Y)/sqrt2): W = [[0, e^{-i pi/4}], [e^{i pi/4}, 0]]
    m = oracle.gate_matrix(C.SQRT_W)
    Wexp = np.array([[0, np.exp(-1j * math.pi / 4)], [np.exp(1j * math.pi / 4), 0]])
    np.testing.assert_allclose(m @ m, Wexp, atol=1e-15)


def _kron_all(*ops):
    out = np.eye(1, dtype=complex)
    for o in ops:
        out = np.kron(out, o)
    return out


def test_fsim_special_cases(oracle):
    f = lambda t, p: oracle.gate_matrix(C.FSIM, theta=t, phi=p)
    np.testing.assert_allclose(f(0, 0), np.eye(4), atol=1e-15)
    np.testing.assert_allclose(f(0, math.pi), np.diag([1, 1, 1, -1]), atol=1e-15)  # CZ
    iswap_m = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    np.testing.assert_allclose(f(math.pi / 2, 0), iswap_m, atol=1e-15)
    for t, p in [(0.3, 0.7), (math.pi / 2, math.pi / 6), (1.62, 0.49)]:
        np.testing.assert_allclose(f(t, p) @ f(-t, -p), np.eye(4), atol=1e-14)
        np.testing.assert_allclose(f(t, p) @ f(t, p).conj().T, np.eye(4), atol=1e-14)
        # fSim is symmetric under exchanging its two qubits
        swap = np.eye(4)[[0, 2, 1, 3]]
        np.testing.assert_allclose(swap @ f(t, p) @ swap, f(t, p), atol=1e-15)


def test_fsim_generators(oracle):
    # fSim(theta, 0) = exp(-i theta (XX + YY)/2); fSim(0, phi) = exp(-i phi |11><11|)
    t, p = 0.91, 0.37
    XX, YY = np.kron(X, X), np.kron(Y, Y)
    np.testing.assert_allclose(oracle.gate_matrix(C.FSIM, theta=t, phi=0.0),
                               scipy.linalg.expm(-1j * t * (XX + YY) / 2), atol=1e-14)
    P11 = np.diag([0, 0, 0, 1]).astype(complex)
    np.testing.assert_allclose(oracle.gate_matrix(C.FSIM, theta=0.0, phi=p),
                               scipy.linalg.expm(-1j * p * P11), atol=1e-14)
    # the two parts commute, so fSim(t, p) is their product
    np.testing.assert_allclose(oracle.gate_matrix(C.FSIM, theta=t, phi=p),
                               scipy.linalg.expm(-1j * t * (XX + YY) / 2) @ scipy.linalg.expm(-1j * p * P11),
                               atol=1e-14)


def test_adjoint_flag(oracle):
    for kind in (C.SQRT_X, C.SQRT_Y, C.SQRT_W):
        m, md = oracle.gate_matrix(kind), oracle.gate_matrix(kind, flags=C.ADJOINT)
        np.testing.assert_allclose(m @ md, I2, atol=1e-15)
    m = oracle.gate_matrix(C.FSIM, theta=1.1, phi=0.4)
    md = oracle.gate_matrix(C.FSIM, flags=C.ADJOINT, theta=1.1, phi=0.4)
    np.testing.assert_allclose(md, m.conj().T, atol=1e-15)


# ------------------------------------------------------------------ state update vs brute force

def _full_operator(n, targets, m):
    """2^n x 2^n operator of matrix m on `targets` (local index j = sum bit(t_i) 2^i):
    m = sum_{r,c} m[r,c] |r><c|, and |r><c| factors into per-qubit |r_i><c_i| on
    each target with identity elsewhere; numpy's kron puts qubit n-1 first."""
    k = len(targets)
    full = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(1 << k):
        for c in range(1 << k):
            if m[r, c] == 0:
                continue
            ops = []
            for q in range(n - 1, -1, -1):
                if q in targets:
                    i = targets.index(q)
                    e = np.zeros((2, 2), dtype=complex)
                    e[(r >> i) & 1, (c >> i) & 1] = 1
                    ops.append(e)
                else:
                    ops.append(I2)
            full += m[r, c] * _kron_all(*ops)
    return full


def _einsum_apply(psi, n, targets, m):
    """Tensor contraction: psi as an n-axis tensor (axis a = qubit n-1-a)."""
    k = len(targets)
    T = psi.reshape((2,) * n)
    G = m.reshape((2,) * (2 * k))  # row bits (t_{k-1}..t_0), then column bits
    axes_in = [n - 1 - targets[i] for i in range(k - 1, -1, -1)]
    out = np.tensordot(G, T, axes=(list(range(k, 2 * k)), axes_in))
    # out axes: k output axes (t_{k-1}..t_0) then the remaining axes of T in order
    rest = [a for a in range(n) if a not in axes_in]
    perm_src = axes_in + rest
    inv = np.argsort(perm_src)
    return np.transpose(out, inv).reshape(-1)


def _gate_targets(g):
    return [int(g["q0"])] if g["nq"] == 1 else [int(g["q0"]), int(g["q1"])]


@pytest.mark.parametrize("seed", [0, 5])
def test_circuit_matches_kronecker_unitary(oracle, seed):
    circ = C.generate(C.Grid(2, 3), cycles=4, pattern="ABCDCDAB", seed=seed, jitter=0.05)
    n = circ.n_qubits
    psi_ref = np.zeros(1 << n, dtype=complex)
    psi_ref[0] = 1
    U = np.eye(1 << n, dtype=complex)
    for g in circ.gates:
        m = oracle.gate_matrix(int(g["kind"]), int(g["flags"]), float(g["theta"]), float(g["phi"]))
        U = _full_operator(n, _gate_targets(g), m) @ U
    psi_ref = U[:, 0]
    psi = oracle.simulate(n, circ.gates)
    np.testing.assert_allclose(psi, psi_ref, atol=1e-12)


def test_circuit_matches_einsum_10q(oracle):
    circ = C.generate(C.Grid(2, 5), cycles=6, pattern="EFGH", seed=3, jitter=0.05)
    n = circ.n_qubits
    psi_ref = np.zeros(1 << n, dtype=complex)
    psi_ref[0] = 1
    for g in circ.gates:
        m = oracle.gate_matrix(int(g["kind"]), int(g["flags"]), float(g["theta"]), float(g["phi"]))
        psi_ref = _einsum_apply(psi_ref, n, _gate_targets(g), m)
    psi = oracle.simulate(n, circ.gates)
    np.testing.assert_allclose(psi, psi_ref, atol=1e-12)


def test_general_k_qubit_matrix_vs_kron(oracle):
    rng = np.random.default_rng(7)
    n = 7
    for targets in ([0, 3, 5], [6, 1], [2, 4, 0, 6], [5]):
        k = len(targets)
        A = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
        Q, _ = np.linalg.qr(A)
        psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        want = _full_operator(n, targets, Q) @ psi0
        got = oracle.apply_matrix(psi0.copy(), targets, Q)
        np.testing.assert_allclose(got, want, atol=1e-12)
        np.testing.assert_allclose(_einsum_apply(psi0, n, targets, Q), want, atol=1e-12)


def test_fused_product_equals_sequence(oracle):
    # a 3-qubit product of gates applied as one matrix equals the gates one by one
    rng = np.random.default_rng(1)
    n = 6
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    seq = [(C.SQRT_X, [1]), (C.FSIM, [1, 4]), (C.SQRT_W, [4]), (C.FSIM, [4, 2]), (C.SQRT_Y, [2])]
    tg = [1, 2, 4]
    M = np.eye(8, dtype=complex)
    psi_seq = psi0.copy()
    for kind, t in seq:
        m = oracle.gate_matrix(kind, theta=1.3, phi=0.5)
        psi_seq = oracle.apply_matrix(psi_seq, t, m)
        loc = [tg.index(q) for q in t]
        M = _full_operator(3, loc, m) @ M
    got = oracle.apply_matrix(psi0.copy(), tg, M)
    np.testing.assert_allclose(got, psi_seq, atol=1e-12)


# ------------------------------------------------------------------ invariants

def test_norm_conserved_and_echo(oracle):
    circ = C.config_circuit("12q_3x4_8cyc")
    n = circ.n_qubits
    psi = oracle.simulate(n, circ.gates)
    assert abs(oracle.norm2(psi) - 1.0) <= 1e-12
    oracle.run(psi, C.inverse_gates(circ.gates))
    assert abs(psi[0] - 1.0) <= 1e-12
    assert np.abs(psi[1:]).max() <= 1e-12


def test_porter_thomas_12q(oracle):
    circ = C.config_circuit("12q_3x4_8cyc")
    n = circ.n_qubits
    psi = oracle.simulate(n, circ.gates)
    p = np.abs(psi) ** 2
    collision = (1 << n) * float(np.sum(p * p))
    assert 1.8 <= collision <= 2.2, collision
    ks = scipy.stats.kstest((1 << n) * p, "expon").statistic
    assert ks < 0.05, ks


def test_product_state_closed_form(oracle):
    # one sqrtX on every qubit: each qubit is ((1+i)|0> + (1-i)|1>)/2
    n = 5
    gates = np.array([C.make_gate(C.SQRT_X, q) for q in range(n)])
    psi = oracle.simulate(n, gates)
    one = np.array([(1 + 1j) / 2, (1 - 1j) / 2])
    want = _kron_all(*([one] * n)).reshape(-1)
    np.testing.assert_allclose(psi, want, atol=1e-15)
    # two sqrtX per qubit = X: |1...1>
    psi2 = oracle.simulate(n, np.concatenate([gates, gates]))
    assert abs(abs(psi2[(1 << n) - 1]) - 1) < 1e-15


# ------------------------------------------------------------------ RNG

@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 11])
def test_philox_matches_numpy(oracle, seed):
    # numpy's Philox is Philox4x64-10 and increments its counter before each block,
    # so numpy(counter = c - 1) yields block c.
    key = np.array([seed, 0], dtype=np.uint64)
    raw = np.random.Philox(key=key, counter=0).random_raw(4 * 6)
    for c in range(1, 7):
        got = oracle.philox4x64_10([c, 0, 0, 0], [seed, 0])
        np.testing.assert_array_equal(got, raw[4 * (c - 1): 4 * c])
    raw0 = np.random.Philox(key=key, counter=2**256 - 1).random_raw(4)  # wraps to block 0
    np.testing.assert_array_equal(oracle.philox4x64_10([0, 0, 0, 0], [seed, 0]), raw0)
    # multi-word counter carry: numpy counter 2^64 - 1 -> block (0, 1, 0, 0)
    raw_c = np.random.Philox(key=key, counter=2**64 - 1).random_raw(4)
    np.testing.assert_array_equal(oracle.philox4x64_10([0, 1, 0, 0], [seed, 0]), raw_c)


def _numpy_uniforms(seed, count):
    raw = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=2**256 - 1).random_raw(count)
    return (raw >> np.uint64(11)).astype(np.float64) * 2.0**-53


def test_uniforms_match_numpy(oracle):
    u = _numpy_uniforms(99, 40)
    got = np.array([oracle.uniform(99, s) for s in range(40)])
    np.testing.assert_array_equal(got, u)


# ------------------------------------------------------------------ sampling

def test_sample_matches_searchsorted(oracle):
    circ = C.generate(C.Grid(2, 4), cycles=5, seed=11)
    n = circ.n_qubits
    psi = oracle.simulate(n, circ.gates)
    shots, seed = 5000, 42
    got = oracle.sample(psi, shots, seed)
    p = np.abs(psi) ** 2
    cdf = np.cumsum(p)
    want = np.searchsorted(cdf, _numpy_uniforms(seed, shots) * cdf[-1], side="right")
    mismatch = np.count_nonzero(got != want)
    assert mismatch <= 1, mismatch  # only a float tie at a CDF boundary may differ
    # sample windows compose: shots [1000, 1500) equal the slice of the full run
    np.testing.assert_array_equal(oracle.sample(psi, 500, seed, first=1000), got[1000:1500])


def test_sample_planted_sparse_state(oracle):
    n = 10
    psi = np.zeros(1 << n, dtype=complex)
    support = {3: 0.5, 700: 0.25, 701: 0.125, 1023: 0.125}
    for i, pr in support.items():
        psi[i] = math.sqrt(pr) * np.exp(1j * i)
    shots = 40000
    x = oracle.sample(psi, shots, seed=5)
    assert set(np.unique(x).tolist()) <= set(support)  # zero-probability cells never chosen
    obs = np.array([np.count_nonzero(x == i) for i in support])
    exp = np.array(list(support.values())) * shots
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < scipy.stats.chi2.ppf(0.9999, len(support) - 1), chi2


def test_sample_uniform_state_chi2(oracle):
    n = 6
    gates = np.array([C.make_gate(C.SQRT_Y, q) for q in range(n)])
    psi = oracle.simulate(n, gates)
    np.testing.assert_allclose(np.abs(psi) ** 2, np.full(1 << n, 2.0**-n), atol=1e-15)
    shots = 64000
    x = oracle.sample(psi, shots, seed=8)
    obs = np.bincount(x.astype(np.int64), minlength=1 << n)
    exp = shots / (1 << n)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < scipy.stats.chi2.ppf(0.9999, (1 << n) - 1), chi2


# ------------------------------------------------------------------ XEB

def test_xeb_basis_state_and_definition(oracle):
    n = 8
    psi = np.zeros(1 << n, dtype=complex)
    psi[17] = 1j
    assert oracle.xeb(psi, np.array([17, 17, 17], dtype=np.uint64)) == pytest.approx((1 << n) - 1)
    assert oracle.xeb(psi, np.array([16], dtype=np.uint64)) == pytest.approx(-1.0)
    # an unnormalised state is renormalised
    assert oracle.xeb(3 * psi, np.array([17], dtype=np.uint64)) == pytest.approx((1 << n) - 1)


def test_xeb_ideal_and_uniform_sampling(oracle):
    circ = C.config_circuit("12q_3x4_8cyc")
    n = circ.n_qubits
    psi = oracle.simulate(n, circ.gates)
    p = np.abs(psi) ** 2
    N = 10_000
    expected = (1 << n) * float(np.sum(p * p)) - 1.0
    # std of F under ideal sampling: 2^n * std(p(x)) / sqrt(N)
    sd_ideal = (1 << n) * math.sqrt(float(np.sum(p * p * p)) - float(np.sum(p * p)) ** 2) / math.sqrt(N)
    F = oracle.xeb(psi, oracle.sample(psi, N, seed=3))
    assert abs(F - expected) < 5 * sd_ideal, (F, expected, sd_ideal)
    assert 0.8 < F < 1.2
    rnd = C.random_bitstrings(n, N, seed=4)
    sd_unif = (1 << n) * math.sqrt(float(np.mean(p * p)) - float(np.mean(p)) ** 2) / math.sqrt(N)
    F0 = oracle.xeb(psi, rnd)
    assert abs(F0) < 5 * sd_unif, (F0, sd_unif)
