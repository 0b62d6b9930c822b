"""Writes tests/golden/oracle_12q_3x4_8cyc.txt from the CPU oracle alone.

The paper prints no worked example that a small program can reproduce (its
XEB scores are for Google's 53-qubit circuits, whose gate lists and reference
amplitudes are not available), so the stored values come from the oracle: the
12-qubit 3x4-grid, 8-cycle ABCDCDAB circuit (seed 0) of the synthetic
workloads. The file freezes the oracle's output, so a later change to the
oracle's arithmetic shows up as a failing test and has to be justified.
Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2512_07311_gb300 import circuits as C  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_12q_3x4_8cyc.txt")
AMPS = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377, 610, 987, 1597, 2584, 4095]
SHOTS, SEED = 64, 7


def main():
    circ = C.config_circuit("12q_3x4_8cyc")
    psi = O.simulate(circ.n_qubits, circ.gates)
    xs = O.sample(psi, SHOTS, SEED)
    lines = [
        "# Oracle output for the 12-qubit 3x4-grid, 8-cycle ABCDCDAB circuit (seed 0), written by",
        "# tests/golden/make_golden.py from oracle/ only (complex128 gate-by-gate state, Section 3.2",
        "# item 1; inverse-CDF sampling with Philox4x64-10 uniforms, item 3; linear XEB, item 4).",
        f"gates {len(circ.gates)}",
        f"norm {O.norm2(psi):.17g}",
    ]
    for i in AMPS:
        lines.append(f"amp {i} {psi[i].real:.17g} {psi[i].imag:.17g}")
    lines.append(f"samples seed={SEED} " + " ".join(str(int(x)) for x in xs))
    lines.append(f"xeb {O.xeb(psi, xs):.17g}")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
