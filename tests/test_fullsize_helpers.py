"""CPU checks of the chunked full-size comparison helpers (oracle/fullsize.py) that
the 30- and 32-qubit oracle comparisons rely on: each must agree with the plain
whole-array computation, and the draw-window check must flag a draw that is not
an inverse-CDF draw for its uniform."""
import numpy as np

from oracle import fullsize as F


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return psi / np.linalg.norm(psi)


def test_cdf_at_matches_cumsum_across_chunks():
    psi = rand_state(12, 1)
    idx = np.random.default_rng(2).integers(0, 1 << 12, size=500)
    idx[:3] = [0, (1 << 12) - 1, 777]
    C = np.cumsum(np.abs(psi) ** 2)
    C /= C[-1]
    for chunk in (1000, 1 << 12, 1 << 20):
        np.testing.assert_allclose(F.cdf_at(psi, idx, chunk=chunk), C[idx], rtol=0, atol=1e-14)


def test_compare_states_against_direct_formula():
    a = rand_state(11, 3)
    b = a.copy()
    b[5] *= -1  # a real, known infidelity
    b[100] += 1e-3
    got = F.compare_states(a, lambda f, c: b[f:f + c], chunk=300)
    want = 1 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
    assert abs(got["infidelity"] - want) <= 1e-14
    assert abs(got["max_abs_diff"] - np.abs(a - b).max()) <= 1e-15


def test_draw_window_accepts_exact_draws_and_flags_wrong_ones(oracle):
    psi = rand_state(12, 4)
    seed, shots = 9, 4000
    xs = oracle.sample(psi, shots, seed)
    u = F.uniforms(seed, 0, shots)
    assert F.draw_window_violations(psi, xs, u, 1e-12) == 0
    bad = xs.copy()
    bad[17] = (int(bad[17]) + 40) % (1 << 12)
    bad[1000] = (int(bad[1000]) + 1) % (1 << 12)
    assert F.draw_window_violations(psi, bad, u, 1e-12) == 2
    # a draw from a nearby distribution stays inside the window widened by sqrt(infidelity)
    psi2 = psi * np.exp(1j * 1e-3 * np.random.default_rng(5).normal(size=psi.size))
    psi2 = psi2 + 1e-4 * rand_state(12, 6)
    inf = F.compare_states(psi, lambda f, c: psi2[f:f + c])["infidelity"]
    assert F.draw_window_violations(psi, oracle.sample(psi2, shots, seed), u, F.window_eps(inf)) == 0
