"""Stored oracle output (tests/golden/oracle_12q_3x4_8cyc.txt, written by
tests/golden/make_golden.py from oracle/ only) against the oracle as it stands (CPU)
and against the CUDA path (GPU).

The CPU test freezes the oracle: a change to its arithmetic fails here and has to be
justified. The GPU test checks the library's FP32 state, samples and XEB against the
same stored values."""
import os

import numpy as np
import pytest

from paper_2512_07311_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_12q_3x4_8cyc.txt")


def load_golden():
    g = {"amps": {}}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == "gates":
                g["gates"] = int(f[1])
            elif f[0] == "norm":
                g["norm"] = float(f[1])
            elif f[0] == "amp":
                g["amps"][int(f[1])] = complex(float(f[2]), float(f[3]))
            elif f[0] == "samples":
                g["seed"] = int(f[1].split("=")[1])
                g["samples"] = np.array([int(x) for x in f[2:]], dtype=np.uint64)
            elif f[0] == "xeb":
                g["xeb"] = float(f[1])
    return g


def test_oracle_reproduces_golden(oracle):
    g = load_golden()
    circ = C.config_circuit("12q_3x4_8cyc")
    assert len(circ.gates) == g["gates"]
    psi = oracle.simulate(circ.n_qubits, circ.gates)
    # the x86 and Arm builds may contract multiply-adds differently: last-bit tolerances
    assert abs(oracle.norm2(psi) - g["norm"]) <= 1e-13
    for i, a in g["amps"].items():
        assert abs(psi[i] - a) <= 1e-13, i
    xs = oracle.sample(psi, len(g["samples"]), g["seed"])
    np.testing.assert_array_equal(xs, g["samples"])
    assert abs(oracle.xeb(psi, xs) - g["xeb"]) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("precision_name", ["RCS_PREC_FP32_PLAIN", "RCS_PREC_FP32_FUSED", "RCS_PREC_BF16X3"])
def test_library_reproduces_golden(precision_name, oracle):
    from paper_2512_07311_gb300 import build as B
    from paper_2512_07311_gb300 import capi

    B.build()
    capi.load()
    g = load_golden()
    circ = C.config_circuit("12q_3x4_8cyc")
    ctx = capi.rcs_create(circ.grid, getattr(capi, precision_name))
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        idx = np.array(sorted(g["amps"]), dtype=np.uint64)
        got = capi.rcs_amplitudes(ctx, idx)
        for i, a in zip(idx, got):
            assert abs(a - g["amps"][int(i)]) <= 1e-6, int(i)
        assert abs(capi.rcs_norm(ctx) - g["norm"]) <= 1e-5
        xs = capi.rcs_sample(ctx, len(g["samples"]), g["seed"])
        assert np.mean(xs == g["samples"]) >= 63 / 64
        # the stored shots scored by the library's state give the stored XEB
        assert abs(capi.rcs_xeb(ctx, g["samples"]) - g["xeb"]) <= 1e-3
        # and the library's own shots score as the oracle scores them
        psi = oracle.simulate(circ.n_qubits, circ.gates)
        assert abs(capi.rcs_xeb(ctx, xs) - oracle.xeb(psi, xs)) <= 1e-3
    finally:
        capi.rcs_destroy(ctx)
