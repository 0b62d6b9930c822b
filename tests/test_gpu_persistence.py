"""State persistence and sharded sampling (the hand-off between the paper's state
construction and its many sampling jobs, Section 3.2 items 2-3): a state saved by one
context and loaded by another gives the same amplitudes, norm and draws; shots drawn in
ranges, by one process or by several that loaded the same file, equal one rcs_sample
call; bad files and qubit counts are rejected without touching the state."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2512_07311_gb300 import build as B
from paper_2512_07311_gb300 import capi
from paper_2512_07311_gb300 import circuits as C

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return capi.load()


@pytest.fixture(scope="module")
def saved(lib, tmp_path_factory):
    """A 20-qubit circuit state (tensor-core path, stored in a permuted layout) on disk."""
    n = 20
    circ = C.generate(C.grid_for_n(n), cycles=10, pattern="EFGH", seed=61, jitter=0.05)
    path = str(tmp_path_factory.mktemp("state") / "psi20.rcs")
    ctx = capi.rcs_create(circ.grid, capi.RCS_PREC_BF16X3)
    capi.rcs_apply_circuit(ctx, circ.gates)
    layout = capi.rcs_qubit_layout(ctx)
    assert any(int(p) != q for q, p in enumerate(layout))
    capi.rcs_state_save(ctx, path)
    yield n, circ, ctx, path, layout
    capi.rcs_destroy(ctx)


def test_file_format(saved):
    n, _, _, path, _ = saved
    assert os.path.getsize(path) == 280 + 8 * (1 << n)
    with open(path, "rb") as fh:
        head = fh.read(280)
    assert head[:8] == b"RCSSTATE"
    assert int.from_bytes(head[8:12], "little") == 1 and int.from_bytes(head[12:16], "little") == n
    assert int.from_bytes(head[272:280], "little") == 1 << n


def test_load_reproduces_state_and_draws(saved):
    n, circ, src, path, layout = saved
    dst = capi.rcs_create(circ.grid, capi.RCS_PREC_BF16X3)
    try:
        capi.rcs_state_load(dst, path)
        np.testing.assert_array_equal(capi.rcs_qubit_layout(dst), layout)
        idx = np.random.default_rng(4).integers(0, 1 << n, 5000).astype(np.uint64)
        np.testing.assert_array_equal(capi.rcs_amplitudes(dst, idx), capi.rcs_amplitudes(src, idx))
        assert capi.rcs_norm(dst) == capi.rcs_norm(src)
        shots, seed = 60_000, 123
        xs = capi.rcs_sample(src, shots, seed)
        np.testing.assert_array_equal(capi.rcs_sample(dst, shots, seed), xs)
        # the same draws in ranges
        parts = [capi.rcs_sample_range(dst, a, b - a, seed) for a, b in ((0, 1), (1, 20_001), (20_001, shots))]
        np.testing.assert_array_equal(np.concatenate(parts), xs)
        assert capi.rcs_xeb(dst, xs) == capi.rcs_xeb(src, xs)
    finally:
        capi.rcs_destroy(dst)


def test_sharded_sampling_across_processes(saved, tmp_path):
    """Two child processes load the saved state and draw disjoint shot ranges; together
    they reproduce one process's rcs_sample."""
    n, circ, src, path, _ = saved
    shots, seed = 40_000, 7
    want = capi.rcs_sample(src, shots, seed)
    code = textwrap.dedent("""
        import sys
        import numpy as np
        sys.path.insert(0, sys.argv[1])
        from paper_2512_07311_gb300 import capi
        capi.load()
        n, path, first, count, seed, out = int(sys.argv[2]), sys.argv[3], int(sys.argv[4]), int(sys.argv[5]), int(sys.argv[6]), sys.argv[7]
        ctx = capi.rcs_create(n, capi.RCS_PREC_BF16X3)
        capi.rcs_state_load(ctx, path)
        np.save(out, capi.rcs_sample_range(ctx, first, count, seed))
        capi.rcs_destroy(ctx)
    """)
    half = shots // 2
    outs = [str(tmp_path / f"part{i}.npy") for i in range(2)]
    procs = [subprocess.Popen([sys.executable, "-c", code, ROOT, str(n), path, str(a), str(cnt), str(seed), o])
             for (a, cnt), o in zip(((0, half), (half, shots - half)), outs)]
    for p in procs:
        assert p.wait(timeout=300) == 0
    got = np.concatenate([np.load(o) for o in outs])
    np.testing.assert_array_equal(got, want)


def test_rejected_loads_leave_the_state(saved, tmp_path):
    n, circ, src, path, _ = saved
    other = capi.rcs_create(n - 1, capi.RCS_PREC_FP32_FUSED)
    try:
        capi.rcs_apply_circuit(other, np.array([C.make_gate(C.SQRT_X, 0)]))
        before = capi.rcs_state_read(other)
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_state_load(other, path)  # 20-qubit file, 19-qubit context
        assert e.value.code == capi.RCS_ERR_ARG and "qubits" in str(e.value)
        bad = tmp_path / "junk.rcs"
        bad.write_bytes(b"not a state" * 40)
        with pytest.raises(capi.RcsError):
            capi.rcs_state_load(other, str(bad))
        with pytest.raises(capi.RcsError):
            capi.rcs_state_load(other, str(tmp_path / "missing.rcs"))
        np.testing.assert_array_equal(capi.rcs_state_read(other), before)
    finally:
        capi.rcs_destroy(other)
    truncated = tmp_path / "short.rcs"
    with open(path, "rb") as fh:
        truncated.write_bytes(fh.read(280 + 1000))
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED)
    try:
        with pytest.raises(capi.RcsError) as e:
            capi.rcs_state_load(ctx, str(truncated))
        assert "truncated" in str(e.value)
    finally:
        capi.rcs_destroy(ctx)
