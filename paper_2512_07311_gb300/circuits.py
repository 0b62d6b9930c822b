"""Seeded synthetic Sycamore-class random circuits (the shared input generator).

This module only decides *which* gate goes *where*: gate kinds, qubit indices
and the fSim angles theta/phi. It holds no gate matrix, no state arithmetic and
nothing of the simulation method; the CUDA path and the CPU oracle each build
their own matrices from the (kind, theta, phi) records written here.

The paper names the circuit family (53-qubit Sycamore random circuits, coupler
patterns EFGH and ABCDCDAB, Section 3.1) but defines neither the gate set nor
the coupler classes. The readings used here:

* qubit q is bit q of the basis index; grid cell (r, c) maps to q by row-major
  order over the cells that are kept;
* coupler classes on an R x C grid: A = horizontal (r,c)-(r,c+1) with c even,
  B = horizontal with c odd, C = vertical (r,c)-(r+1,c) with r even,
  D = vertical with r odd; the EFGH pattern relabels them E=C, F=A, G=D, H=B;
  couplers touching a removed cell are dropped;
* cycle c (1-based) = one single-qubit layer on every qubit, then every coupler
  of class pattern[(c-1) mod len(pattern)]; an extra single-qubit layer follows
  the last cycle unless ``final_layer=False``;
* single-qubit gates: cycle 1 draws uniformly from {sqrtX, sqrtY, sqrtW}; later
  cycles draw uniformly from the two gates that differ from the previous gate
  on that qubit; draw order is (cycle, qubit);
* fSim angles: theta = pi/2, phi = pi/6, or with ``jitter`` each coupler draws
  theta and phi once, uniformly within +-jitter of those values, before any
  gate choice, in canonical coupler order, and keeps them for the whole circuit;
* the random source is ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Gate kinds (same numbering as the C ABI's RCS_GATE_* constants).
SQRT_X, SQRT_Y, SQRT_W, FSIM, U1, U2 = 0, 1, 2, 3, 4, 5
KIND_NAMES = {SQRT_X: "sqrtX", SQRT_Y: "sqrtY", SQRT_W: "sqrtW", FSIM: "fSim", U1: "U1", U2: "U2"}

THETA0 = math.pi / 2
PHI0 = math.pi / 6

# Gate flags: bit 0 = apply the adjoint (conjugate transpose) of the gate.
ADJOINT = 1

# One record per gate. Field layout mirrors `rcs_gate` in include/rcs.h
# (kind u8, nq u8, flags u8, 1 pad byte, q int32[2], theta f64, phi f64, u pointer).
GATE_DTYPE = np.dtype(
    {
        "names": ["kind", "nq", "flags", "q0", "q1", "theta", "phi", "u"],
        "formats": [np.uint8, np.uint8, np.uint8, np.int32, np.int32, np.float64, np.float64, np.uint64],
        "offsets": [0, 1, 2, 4, 8, 16, 24, 32],
        "itemsize": 40,
    }
)

PATTERNS = ("ABCDCDAB", "EFGH")
_EFGH_TO_ABCD = {"E": "C", "F": "A", "G": "D", "H": "B"}


@dataclass(frozen=True)
class Grid:
    rows: int
    cols: int
    removed: tuple[int, ...] = ()  # row-major cell ids

    def cells(self) -> list[tuple[int, int]]:
        rm = set(self.removed)
        return [(r, c) for r in range(self.rows) for c in range(self.cols) if r * self.cols + c not in rm]

    @property
    def n_qubits(self) -> int:
        return self.rows * self.cols - len(set(self.removed))

    def qubit_of(self) -> dict[tuple[int, int], int]:
        return {rc: q for q, rc in enumerate(self.cells())}


def grid_for_n(n: int) -> Grid:
    """Grid used for an arbitrary qubit count: rows = floor(sqrt(n)),
    cols = ceil(n / rows), trailing cells of the last row removed."""
    rows = max(1, math.isqrt(n))
    cols = -(-n // rows)
    extra = rows * cols - n
    removed = tuple(rows * cols - 1 - i for i in range(extra))
    return Grid(rows, cols, tuple(sorted(removed)))


def coupler_classes(grid: Grid) -> dict[str, list[tuple[int, int]]]:
    """Couplers of each class A, B, C, D as (q_low, q_high) pairs in canonical
    (row-major) order."""
    qof = grid.qubit_of()
    out = {"A": [], "B": [], "C": [], "D": []}
    for r in range(grid.rows):
        for c in range(grid.cols - 1):
            a, b = (r, c), (r, c + 1)
            if a in qof and b in qof:
                out["A" if c % 2 == 0 else "B"].append((qof[a], qof[b]))
    for r in range(grid.rows - 1):
        for c in range(grid.cols):
            a, b = (r, c), (r + 1, c)
            if a in qof and b in qof:
                out["C" if r % 2 == 0 else "D"].append((qof[a], qof[b]))
    return out


def all_couplers(grid: Grid) -> list[tuple[int, int]]:
    """Canonical coupler order: horizontal row-major, then vertical row-major."""
    qof = grid.qubit_of()
    hs, vs = [], []
    for r in range(grid.rows):
        for c in range(grid.cols - 1):
            if (r, c) in qof and (r, c + 1) in qof:
                hs.append((qof[(r, c)], qof[(r, c + 1)]))
    for r in range(grid.rows - 1):
        for c in range(grid.cols):
            if (r, c) in qof and (r + 1, c) in qof:
                vs.append((qof[(r, c)], qof[(r + 1, c)]))
    return hs + vs


@dataclass
class Circuit:
    grid: Grid
    cycles: int
    pattern: str
    seed: int
    jitter: float
    final_layer: bool
    gates: np.ndarray = field(repr=False)  # GATE_DTYPE records

    @property
    def n_qubits(self) -> int:
        return self.grid.n_qubits

    def __len__(self) -> int:
        return len(self.gates)

    def counts(self) -> dict[str, int]:
        k = self.gates["kind"]
        return {"fsim": int((k == FSIM).sum()), "one_qubit": int((k < FSIM).sum())}


def make_gate(kind: int, q0: int, q1: int = -1, theta: float = 0.0, phi: float = 0.0,
              flags: int = 0) -> np.ndarray:
    g = np.zeros((), dtype=GATE_DTYPE)
    g["kind"] = kind
    g["flags"] = flags
    g["nq"] = 2 if kind in (FSIM, U2) else 1
    g["q0"] = q0
    g["q1"] = q1
    g["theta"] = theta
    g["phi"] = phi
    return g


def generate(grid: Grid, cycles: int, pattern: str = "ABCDCDAB", seed: int = 0,
             jitter: float = 0.0, final_layer: bool = True) -> Circuit:
    """Seeded Sycamore-class circuit on `grid` (see module docstring for the rules)."""
    if pattern not in PATTERNS and not set(pattern) <= set("ABCD"):
        raise ValueError(f"unknown coupler pattern {pattern!r}")
    rng = np.random.default_rng(seed)
    n = grid.n_qubits
    classes = coupler_classes(grid)
    angles = {}
    for cp in all_couplers(grid):
        if jitter > 0.0:
            dt = rng.uniform(-jitter, jitter)
            dp = rng.uniform(-jitter, jitter)
        else:
            dt = dp = 0.0
        angles[cp] = (THETA0 + dt, PHI0 + dp)

    recs = []
    prev = [-1] * n

    def one_qubit_layer():
        for q in range(n):
            if prev[q] < 0:
                g = int(rng.integers(0, 3))
            else:
                others = [x for x in (SQRT_X, SQRT_Y, SQRT_W) if x != prev[q]]
                g = others[int(rng.integers(0, 2))]
            prev[q] = g
            recs.append((g, 1, 0, q, -1, 0.0, 0.0, 0))

    for c in range(1, cycles + 1):
        one_qubit_layer()
        letter = pattern[(c - 1) % len(pattern)]
        cls = _EFGH_TO_ABCD.get(letter, letter)
        for (a, b) in classes[cls]:
            th, ph = angles[(a, b)]
            recs.append((FSIM, 2, 0, a, b, th, ph, 0))
    if final_layer:
        one_qubit_layer()
    return Circuit(grid, cycles, pattern, seed, jitter, final_layer, gate_array(recs))


def gate_array(recs) -> np.ndarray:
    """GATE_DTYPE array from (kind, nq, flags, q0, q1, theta, phi, u) tuples,
    with the padding bytes zeroed so equal gate lists are equal byte for byte."""
    gates = np.zeros(len(recs), dtype=GATE_DTYPE)
    for name, col in zip(GATE_DTYPE.names, zip(*recs) if recs else [()] * len(GATE_DTYPE.names)):
        gates[name] = col
    return gates


def inverse_gates(gates: np.ndarray) -> np.ndarray:
    """Gate records of the inverse circuit, for the echo check: reversed order
    with the ADJOINT flag toggled on every gate."""
    inv = gates[::-1].copy()
    inv["flags"] ^= ADJOINT
    return inv


# --- the benchmark workloads --------------------------------------------------------

CONFIGS = {
    # 12-qubit 3x4 grid, 8 cycles, ABCDCDAB, no jitter, 10^4 shots
    "12q_3x4_8cyc": dict(grid=Grid(3, 4), cycles=8, pattern="ABCDCDAB", seed=0, jitter=0.0, shots=10_000),
    # 30-qubit 5x6 grid, 14 cycles, EFGH, jittered fSim, 10^6 shots
    "30q_5x6_14cyc": dict(grid=Grid(5, 6), cycles=14, pattern="EFGH", seed=1, jitter=0.05, shots=1_000_000),
    # 34-qubit 5x7 grid minus corner (4,6), 20 cycles, ABCDCDAB, 10^6 shots
    "34q_5x7m1_20cyc": dict(grid=Grid(5, 7, (34,)), cycles=20, pattern="ABCDCDAB", seed=2, jitter=0.0,
                            shots=1_000_000),
    # 32-qubit 4x8 grid, 20 cycles, EFGH, jittered fSim, 2.5*10^6 shots
    "32q_4x8_20cyc": dict(grid=Grid(4, 8), cycles=20, pattern="EFGH", seed=4, jitter=0.05, shots=2_500_000),
}


def config_circuit(name: str) -> Circuit:
    c = CONFIGS[name]
    return generate(c["grid"], c["cycles"], c["pattern"], c["seed"], c["jitter"])


def batch_instance(seed: int) -> Circuit:
    """One instance of the batched workload: qubit count uniform in 16..26,
    depth uniform in 10..20 cycles, pattern ABCDCDAB or EFGH, all drawn from
    default_rng(seed); the circuit itself then uses the same seed."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(16, 27))
    cycles = int(rng.integers(10, 21))
    pattern = PATTERNS[int(rng.integers(0, 2))]
    return generate(grid_for_n(n), cycles, pattern, seed=seed)


def batch_workload(count: int = 64, first_seed: int = 1000) -> list[Circuit]:
    return [batch_instance(first_seed + i) for i in range(count)]


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """Uniformly random n-bit basis indices (uint64), for XEB null checks."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << n, size=count, dtype=np.uint64) if n < 64 else \
        rng.integers(0, 2**63, size=count, dtype=np.uint64)
