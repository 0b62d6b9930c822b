"""The bounded waits of the tensor-core kernels, exercised without a GPU fault: a host-set
hook (rcs_tc_test_fault) makes the first CTA skip the MMAs of one of its tiles, so nothing
asynchronous is ever issued for it and every wait on that tile runs out after a short
limit. The launch must then end on its own with the error rcs_sync reports as
RCS_ERR_TIMEOUT, and the context must stay usable: with the hook cleared, the next launch
allocates the tensor memory again (so the failed one released it) and gives the oracle's
state. Covers the single-pass kernel (both splits) and the pair kernel."""
import time

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi

pytestmark = pytest.mark.gpu

N = 22  # 512 tiles: the first CTA has several, so a middle one can be skipped


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


def rand_unitary(d, rng):
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    Q, R = np.linalg.qr(A)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def infidelity(a, b):
    return 1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


@pytest.mark.parametrize("precision,flags", [(capi.RCS_PREC_BF16X3, 0), (capi.RCS_PREC_TF32X3, 0),
                                             (capi.RCS_PREC_BF16X3, capi.RCS_OPT_PAIR_PASSES)])
def test_skipped_tile_times_out_and_the_context_recovers(lib, oracle, precision, flags):
    rng = np.random.default_rng(77 + precision + 10 * flags)
    psi0 = (rng.normal(size=1 << N) + 1j * rng.normal(size=1 << N)).astype(np.complex64)
    psi0 /= np.linalg.norm(psi0)
    items = [([2, 5, 9, 13, 17, 21], rand_unitary(64, rng))]
    if flags:
        items.append(([5, 6, 10, 14, 18, 21], rand_unitary(64, rng)))
    ctx = capi.rcs_create(N, precision, flags=flags)
    try:
        capi.rcs_state_write(ctx, psi0)
        try:
            capi.rcs_tc_test_fault(1, 0.002)
            t0 = time.perf_counter()
            capi.rcs_apply_unitaries(ctx, items)
            with pytest.raises(capi.RcsError) as e:
                capi.rcs_sync(ctx)
            waited = time.perf_counter() - t0
        finally:
            capi.rcs_tc_test_fault(-1, 0.0)
        assert e.value.code == capi.RCS_ERR_TIMEOUT
        assert waited < 0.5, waited  # a few 2 ms waits, not the default one-second limit
        # the context is usable again: the same launch, from the same input, now completes
        capi.rcs_state_write(ctx, psi0)
        capi.rcs_apply_unitaries(ctx, items)
        capi.rcs_sync(ctx)
        got = capi.rcs_state_read(ctx).astype(np.complex128)
    finally:
        capi.rcs_destroy(ctx)
    want = psi0.astype(np.complex128)
    for t, U in items:
        oracle.apply_matrix(want, t, U)
    assert infidelity(got, want) <= 2e-8
