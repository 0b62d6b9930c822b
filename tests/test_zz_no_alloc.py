"""rcs_xeb_static: the allocation-free XEB entry point, for callers that cannot
call cudaMalloc (for example when all device memory comes from the caller's own
arena). It must give the
same score as rcs_xeb_device on the same state and samples, call after call,
although its scratch is one fixed device array shared by every call.

Collected last on purpose (file name), so a run that stops at the first failure
has run every other test before this one."""
import math

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

pytestmark = pytest.mark.gpu

XEB_MATCH = 1e-9  # the two paths reduce in the same order; observed equal to the last bit


def test_static_scratch_xeb_matches_context_xeb():
    torch = pytest.importorskip("torch")
    B.build()
    capi.load()
    n = 20
    circ = C.generate(C.grid_for_n(n), cycles=8, pattern="EFGH", seed=21, jitter=0.05)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED, stream=stream)
    try:
        capi.rcs_apply_circuit(ctx, circ.gates)
        d_state = capi.rcs_state_device(ctx)
        # larger call first, then a smaller one: the second must not pick up the
        # first call's leftovers in the shared scratch array
        for call, (shots, seed) in enumerate([(90_000, 3), (20_000, 4)]):
            d_bits = torch.empty(shots, dtype=torch.int64, device="cuda")
            capi.rcs_sample_device(ctx, shots, seed, d_bits.data_ptr())
            d_ref = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            capi.rcs_xeb_device(ctx, d_bits.data_ptr(), shots, d_ref.data_ptr())
            d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            capi.rcs_xeb_static(d_state, n, d_bits.data_ptr(), shots, d_out.data_ptr(), stream)
            torch.cuda.current_stream().synchronize()
            ref, got = float(d_ref.item()), float(d_out.item())
            assert math.isfinite(ref) and 0.5 < ref < 1.5, (call, ref)
            assert abs(got - ref) <= XEB_MATCH, (call, got, ref)
        # sizes beyond the fixed scratch are refused before any launch
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_xeb_static(d_state, n, d_bits.data_ptr(), (1 << 26) + 1, d_out.data_ptr(), stream)
        assert e.value.code == capi.RCS_ERR_ARG
        # so are misaligned views (checked on the host: nothing is launched)
        for args in ((d_state + 8, d_bits.data_ptr(), d_out.data_ptr()),
                     (d_state, d_bits.data_ptr() + 4, d_out.data_ptr()),
                     (d_state, d_bits.data_ptr(), d_out.data_ptr() + 4)):
            with pytest.raises(capi.RcsError) as e:
                capi.rcs_xeb_static(args[0], n, args[1], 1000, args[2], stream)
            assert e.value.code == capi.RCS_ERR_ARG
    finally:
        capi.rcs_destroy(ctx)
    # a third call on a much smaller state: its norm uses fewer partial slots than the
    # calls before it left behind in the shared array
    n2 = 10
    circ2 = C.generate(C.grid_for_n(n2), cycles=8, pattern="ABCDCDAB", seed=22)
    ctx2 = capi.rcs_create(n2, capi.RCS_PREC_FP32_FUSED, stream=stream)
    try:
        capi.rcs_apply_circuit(ctx2, circ2.gates)
        d_state2 = capi.rcs_state_device(ctx2)
        shots = 5000
        d_bits = torch.empty(shots, dtype=torch.int64, device="cuda")
        capi.rcs_sample_device(ctx2, shots, 5, d_bits.data_ptr())
        d_ref = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        capi.rcs_xeb_device(ctx2, d_bits.data_ptr(), shots, d_ref.data_ptr())
        d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        capi.rcs_xeb_static(d_state2, n2, d_bits.data_ptr(), shots, d_out.data_ptr(), stream)
        torch.cuda.current_stream().synchronize()
        ref, got = float(d_ref.item()), float(d_out.item())
        assert math.isfinite(ref), ref
        assert abs(got - ref) <= XEB_MATCH, (got, ref)
    finally:
        capi.rcs_destroy(ctx2)
