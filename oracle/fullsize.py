"""Full-size comparisons of a state held elsewhere (read in chunks) with an oracle state.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the GPU tests and the
benchmark's oracle-check leg use it; the product library never does. It imports
nothing from the CUDA package: the other state arrives through a callable
read_chunk(first, count) -> complex array of amplitudes first .. first+count-1.

What is compared follows the definitions the oracle implements (Section 3.2:
the built state, its inverse-CDF samples, their linear XEB):
  * fidelity |<a|b>|^2 / (|a|^2 |b|^2) over the whole state, and the largest
    amplitude difference max_i |a_i - b_i| (no phase removed: both sides use
    the same gate convention);
  * the normalised cumulative distribution C_i / T of the oracle state at given
    indices, so that a draw x made for uniform u under the other state can be
    checked against the oracle's distribution: an exact inverse-CDF draw under
    a distribution q satisfies Q_{x-1} <= u < Q_x, and |Q_i - C_i / T| is at most
    the total-variation distance of the two distributions, which for pure states
    is at most sqrt(1 - fidelity). So every draw must satisfy
    C_{x-1}/T - eps <= u < C_x/T + eps with eps = sqrt(1 - fidelity) (plus the
    rounding of the sums here).
"""
from __future__ import annotations

import math

import numpy as np

CHUNK = 1 << 26


def compare_states(psi_or: np.ndarray, read_chunk, chunk: int = CHUNK) -> dict:
    """Whole-state overlap of the chunked state b with the oracle state a."""
    N = psi_or.size
    ab = 0j
    aa = 0.0
    bb = 0.0
    max_diff = 0.0
    for first in range(0, N, chunk):
        cnt = min(chunk, N - first)
        b = np.asarray(read_chunk(first, cnt), dtype=np.complex128)
        a = psi_or[first:first + cnt]
        ab += np.vdot(a, b)
        aa += float(np.vdot(a, a).real)
        bb += float(np.vdot(b, b).real)
        max_diff = max(max_diff, float(np.abs(a - b).max()))
    fid = abs(ab) ** 2 / (aa * bb)
    return {"infidelity": float(1.0 - fid), "max_abs_diff": max_diff, "norm_or": aa, "norm_other": bb}


def cdf_at(psi: np.ndarray, idx: np.ndarray, chunk: int = CHUNK) -> np.ndarray:
    """C_i / T for every index in idx (any order): C_i = sum_{j<=i} |psi_j|^2, T = C_{N-1}."""
    idx = np.asarray(idx, dtype=np.int64)
    order = np.argsort(idx, kind="stable")
    srt = idx[order]
    out = np.empty(srt.size, dtype=np.float64)
    N = psi.size
    carry = 0.0
    pos = 0
    for first in range(0, N, chunk):
        cnt = min(chunk, N - first)
        p = psi[first:first + cnt]
        c = np.cumsum(p.real * p.real + p.imag * p.imag)
        end = int(np.searchsorted(srt, first + cnt, side="left"))
        if end > pos:
            out[pos:end] = carry + c[srt[pos:end] - first]
            pos = end
        carry += float(c[-1])
    res = np.empty_like(out)
    res[order] = out / carry
    return res


def draw_window_violations(psi_or: np.ndarray, draws: np.ndarray, uniforms: np.ndarray, eps: float) -> int:
    """How many draws x (made for uniforms u) fall outside the oracle's inverse-CDF
    window [C_{x-1}/T - eps, C_x/T + eps)."""
    x = np.asarray(draws, dtype=np.int64)
    u = np.asarray(uniforms, dtype=np.float64)
    hi = cdf_at(psi_or, x)
    lo = np.where(x > 0, cdf_at(psi_or, np.maximum(x - 1, 0)), 0.0)
    bad = (u < lo - eps) | (u >= hi + eps)
    return int(bad.sum())


def window_eps(infidelity: float) -> float:
    """sqrt(1 - fidelity) bounds the total-variation distance; 1e-8 covers the rounding
    of the plain float64 cumulative sums here (at most 2^26 terms per chunk, each
    within 2^-53 of the running total)."""
    return math.sqrt(max(infidelity, 0.0)) + 1e-8


def uniforms(seed: int, first: int, count: int) -> np.ndarray:
    """The oracle's uniforms u_s for shots first .. first+count-1."""
    from . import oracle as O

    f = O.lib().orc_uniform
    return np.fromiter((f(seed, first + s) for s in range(count)), dtype=np.float64, count=count)
