"""Error of every numerical path against the FP64 (complex128) oracle on one circuit
of the benchmark's family, at a size the oracle finishes in seconds: 24 qubits,
20 cycles, ABCDCDAB. Each path must stay within the stated tolerances (infidelity
<= 1e-5, max amplitude error <= 1e-6); the measured errors are printed (pytest -s)
and written to $RCS_PRECISION_REPORT when that variable names a file."""
import json
import os

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

pytestmark = pytest.mark.gpu

PATHS = [("fp32_plain", capi.RCS_PREC_FP32_PLAIN, 0), ("fp32_fused_k4", capi.RCS_PREC_FP32_FUSED, 4),
         ("fp32_fused_k5", capi.RCS_PREC_FP32_FUSED, 5), ("fp32_fused_k6", capi.RCS_PREC_FP32_FUSED, 6),
         ("fp32_fused_k7", capi.RCS_PREC_FP32_FUSED, 7), ("bf16x3_tensor_core", capi.RCS_PREC_BF16X3, 0),
         ("tf32x3_tensor_core", capi.RCS_PREC_TF32X3, 0)]


def test_precision_error_report(oracle):
    B.build()
    capi.load()
    n = 24
    circ = C.generate(C.grid_for_n(n), 20, "ABCDCDAB", seed=2)
    want = oracle.simulate(n, circ.gates)
    wn = want / np.linalg.norm(want)
    report = {"qubits": n, "cycles": 20, "gates": len(circ.gates)}
    for name, prec, k in PATHS:
        ctx = capi.rcs_create(circ.grid, prec, k_max=k)
        try:
            capi.rcs_apply_circuit(ctx, circ.gates)
            norm = capi.rcs_norm(ctx)
            got = capi.rcs_state_read(ctx).astype(np.complex128)
            plan = capi.rcs_plan_build(n, circ.gates, prec, k)
            passes = capi.rcs_plan_info(plan)["n_passes"]
            capi.rcs_plan_destroy(plan)
        finally:
            capi.rcs_destroy(ctx)
        gn = got / np.linalg.norm(got)
        inf = 1.0 - abs(np.vdot(gn, wn)) ** 2
        err = float(np.abs(got - want).max())
        rel = err * 2 ** (n / 2)
        report[name] = {"passes": passes, "infidelity": inf, "max_abs_amp_error": err,
                        "max_amp_error_x_2^(n/2)": rel, "norm_minus_1": norm - 1.0}
        assert inf <= 1e-5, (name, inf)
        assert err <= 1e-6, (name, err)
    print(json.dumps(report, indent=1))
    path = os.environ.get("RCS_PRECISION_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(report, fh, indent=1)
