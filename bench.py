"""Benchmark of the random-circuit-sampling hot path on GB300.

One step = the whole path on one circuit: reset the state to |0...0>, apply the
fused circuit (tensor-core BF16x3 passes), draw the shots, score them with
linear XEB. Default workload: 34 qubits on a 5x7 grid minus one corner,
20 cycles, coupler pattern ABCDCDAB, 10^6 shots (128 GiB complex64 state).

Prints one JSON line (rank 0). `value` is seconds per circuit (lower is better),
device-resident inputs; `e2e` times the same step through the public host-buffer
calls (gate list uploaded, samples copied back and re-uploaded for XEB).
`--impl reference` times the CPU oracle instead (bounded sample, see below).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2512_07311_gb300 import circuits as C  # noqa: E402

METRIC = "34q 20-cycle circuit time (s), shots/s; fused-TC vs plain FP32 at 1e-5 infid"
# DRAM bytes (read + write) per amplitude per tensor-core pass, from ncu captures of the first seven
# full passes on a 2^27-amplitude state (mean per launch: BF16x3 2.0854 GB, TF32x3 2.0852 GB); the
# traffic of a pass is proportional to the state size, so a launch at n qubits moves this x 2^n.
TC_DRAM_BYTES_PER_AMP = {"bf16x3": 2.0854e9 / 2**27, "tf32x3": 2.0852e9 / 2**27}
PAIR_DRAM_BYTES_PER_AMP = (1.074e9 + 1.012e9) / 2**27  # the two-unitary kernel, captured at 27 qubits
# the persistent batch kernel on the 64-circuit workload: DRAM bytes of one launch (ncu)
BATCH64_TC_DRAM_BYTES = 86.469e9 + 92.177e9
WORKLOAD = "34q_5x7m1_20cyc"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(C.CONFIGS) + ["batch64"],
                    help="batch64: the 64-circuit batched workload (its own JSON line, not the headline)")
    ap.add_argument("--shots", type=int, default=None)
    ap.add_argument("--qubits", type=int, default=None,
                    help="profiling size: a circuit of the same family (20 cycles, ABCDCDAB) on a grid of this "
                         "many qubits instead of the named workload")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3"],
                    help="split precision of the tensor-core passes (bf16x3: the headline path)")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 plain/fused comparison runs")
    ap.add_argument("--pair-passes", action="store_true",
                    help="time the opt-in two-unitary kernel (RCS_OPT_PAIR_PASSES) as the headline path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--fp32-wide-pass", type=int, default=0, metavar="N",
                    help="only time one full-state pass of each fused FP32 width 4..7 on an N-qubit state "
                         "(20..30) and print it as one JSON line")
    ap.add_argument("--oracle-check", action="store_true",
                    help="also build the workload's whole state with the CPU oracle (timed: apply, sample, XEB) and "
                         "compare every GPU path with it at full size; needs host memory for the complex128 state "
                         "(30 q: 16 GiB, 32 q: 64 GiB) and its CDF")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.proc = None
        self.gpu = gpu  # nvidia-smi -i accepts an index or a UUID

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks

def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The maximum of a per-rank value over all ranks (the slowest replica sets the
    job's step time); the value itself when running alone."""
    if dist is None:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_circuit_seconds(ms_step_max: float, world: int) -> float:
    """Whole-job seconds per circuit: every rank runs one circuit per step, so the job
    finishes `world` circuits in the slowest rank's step time."""
    return ms_step_max / 1e3 / max(1, world)


# ------------------------------------------------------------------ peaks

def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# ------------------------------------------------------------------ CPU oracle baseline

def cpu_baseline(circ: C.Circuit, shots: int, budget_s: float = 20.0) -> dict:
    """Times the CPU oracle (as it stands) on a bounded sample of the workload:
    the workload's own gate sequence applied, in order, to a 2^n_s-amplitude
    complex128 state (qubit q acts as q mod n_s; gates that collapse onto one
    qubit are skipped), then the oracle's inverse-CDF sampler and XEB. Times are
    scaled to the full workload by 2^(n - n_s) and by gates applied."""
    from oracle import oracle as O

    O.build()
    n = circ.n_qubits
    n_s = min(n, 26)
    g = circ.gates.copy()
    g["q0"] %= n_s
    two = g["nq"] == 2
    g["q1"][two] %= n_s
    keep = ~(two & (g["q0"] == g["q1"]))
    g = g[keep]
    psi = O.zero_state(n_s)
    t0 = time.perf_counter()
    done = 0
    step = 8
    while done < len(g) and time.perf_counter() - t0 < budget_s * 0.7:
        O.run(psi, g[done:done + step])
        done += min(step, len(g) - done)
    t_apply = time.perf_counter() - t0
    s_shots = min(shots, 100_000)
    t1 = time.perf_counter()
    xs = O.sample(psi, s_shots, seed=1)
    t_sample = time.perf_counter() - t1
    t2 = time.perf_counter()
    O.xeb(psi, xs)
    t_xeb = time.perf_counter() - t2
    scale = 2.0 ** (n - n_s)
    # sampling = one 2^n CDF pass (dominant) + shots * log2(2^n) searches; scale the pass by 2^(n-n_s)
    est = t_apply * scale * len(circ.gates) / max(done, 1) + t_sample * scale + t_xeb * shots / s_shots
    whole = n_s == n and done == len(g) and s_shots == shots  # the whole workload ran: no scaling
    return {"value": est, "unit": "s", "cores": O.threads(), "kind": "oracle", "measured": bool(whole),
            "sample": (f"oracle on a 2^{n_s}-amplitude complex128 state: first {done} of {len(circ.gates)} "
                       f"workload gates (qubit q -> q mod {n_s}), {s_shots} shots + XEB; "
                       f"scaled x2^{n - n_s} per amplitude pass and by gate count"),
            "measured_s": {"apply": t_apply, "sample": t_sample, "xeb": t_xeb}}


def host_memory_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def oracle_check(circ: C.Circuit, shots: int, ctx, plans: dict, headline: str, capi) -> tuple[dict, dict]:
    """The workload's whole complex128 oracle state, built and timed on the host cores,
    against each GPU path in `plans` (name -> uploaded plan) run from |0...0> on ctx.
    Returns (cpu_baseline measured on the full workload, comparison figures)."""
    from oracle import fullsize as F
    from oracle import oracle as O

    O.build()
    n = circ.n_qubits
    need = 16 * 2**n * 2.5
    if host_memory_bytes() < need:
        return None, {"skipped": f"host memory {host_memory_bytes() / 2**30:.0f} GiB < {need / 2**30:.0f} GiB"}
    seed = 31
    t0 = time.perf_counter()
    psi = O.simulate(n, circ.gates)
    t_apply = time.perf_counter() - t0
    rng = np.random.default_rng(2**20)
    S = np.unique(rng.integers(0, 1 << n, size=1 << 20, dtype=np.uint64))
    out = {"seed": seed, "shots": shots, "paths": {}}
    xs = None
    for name, plan in plans.items():
        capi.rcs_reset(ctx)
        capi.rcs_plan_run(ctx, plan)
        capi.rcs_sync(ctx)
        if name == headline:
            xs = capi.rcs_sample(ctx, shots, seed)
            F_gpu = capi.rcs_xeb(ctx, xs)
        a = capi.rcs_amplitudes(ctx, S)
        b = psi[S.astype(np.int64)]
        sub = float(1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
        cmp = F.compare_states(psi, lambda f, c: capi.rcs_state_read(ctx, f, c))
        out["paths"][name] = {"infidelity": cmp["infidelity"], "subset_infidelity": sub,
                              "max_abs_amp_err": cmp["max_abs_diff"],
                              "norm": cmp["norm_other"]}
    t1 = time.perf_counter()
    x_or = O.sample(psi, shots, seed)
    t_sample = time.perf_counter() - t1
    t2 = time.perf_counter()
    F_or_own = O.xeb(psi, x_or)
    t_xeb = time.perf_counter() - t2
    F_or = O.xeb(psi, xs)
    eps = F.window_eps(out["paths"][headline]["infidelity"])
    u = F.uniforms(seed, 0, shots)
    out[headline] = {"xeb_gpu": F_gpu, "xeb_oracle_same_shots": F_or, "xeb_diff": abs(F_gpu - F_or),
                     "xeb_oracle_own_shots": F_or_own,
                     "draws_equal_oracle_own_state": float(np.mean(xs == x_or)),
                     "draw_window_eps": eps,
                     "draws_outside_oracle_window": F.draw_window_violations(psi, xs, u, eps)}
    del psi, x_or
    # the oracle's sampler on the headline path's own state (read back, promoted exactly)
    capi.rcs_reset(ctx)
    capi.rcs_plan_run(ctx, plans[headline])
    capi.rcs_sync(ctx)
    mine = np.empty(1 << n, dtype=np.complex128)
    for f in range(0, 1 << n, F.CHUNK):
        c = min(F.CHUNK, (1 << n) - f)
        mine[f:f + c] = capi.rcs_state_read(ctx, f, c)
    out[headline]["draws_equal_oracle_on_same_state"] = float(np.mean(O.sample(mine, shots, seed) == xs))
    del mine
    cpu = {"value": t_apply + t_sample + t_xeb, "unit": "s", "cores": O.threads(), "kind": "oracle",
           "measured": True, "sample": f"the whole workload: {len(circ.gates)} gates on the 2^{n}-amplitude "
                                       f"complex128 state, {shots} shots + XEB",
           "measured_s": {"apply": t_apply, "sample": t_sample, "xeb": t_xeb}}
    return cpu, out


# ------------------------------------------------------------------ reference arm (the CPU oracle)

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    cfg = C.CONFIGS[args.workload]
    circ = C.config_circuit(args.workload)
    shots = args.shots or cfg["shots"]
    for _ in range(args.warmup):
        cpu_baseline(circ, shots, budget_s=3.0)
    vals = [cpu_baseline(circ, shots, budget_s=10.0) for _ in range(args.steps)]
    v = statistics.median(x["value"] for x in vals)
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "qubits": circ.n_qubits, "cycles": circ.cycles,
                       "pattern": circ.pattern, "shots": shots},
            "cpu_baseline": {k: vals[-1][k] for k in ("kind", "cores", "sample")} | {"value": v, "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def batch64_measure(args, torch, capi, precision: str):
    """64 seeded circuits (16-26 qubits, 10-20 cycles, 10^5 shots each) in one graph launch,
    through the tensor-core engine (every pass of every circuit in one persistent tensor-core
    launch, tiles per work item autotuned; then sampling and XEB) and the persistent FP32 engine (every
    pass of every circuit as items of one cooperative launch, fusion width and item size
    autotuned). Returns both timings with their byte counts."""
    circs = C.batch_workload(64, 1000)
    shots = args.shots or 100_000
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()

    def timed(precision, shots=shots):
        b = capi.rcs_batch_create([(c.n_qubits, c.gates, shots, c.seed) for c in circs], precision=precision)
        infos = [capi.rcs_batch_info(b, i) for i in range(len(circs))]
        tuning = capi.rcs_batch_tuning(b) if precision != capi.RCS_PREC_FP32_FUSED else None
        for _ in range(args.warmup):
            capi.rcs_batch_launch(b, stream.cuda_stream)
        capi.rcs_batch_wait(b, stream.cuda_stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            capi.rcs_batch_launch(b, stream.cuda_stream)
        e1.record(stream)
        capi.rcs_batch_wait(b, stream.cuda_stream)
        ms = e0.elapsed_time(e1) / args.steps
        xebs = [capi.rcs_batch_result(b, i, 0)[1] for i in range(len(circs))]
        capi.rcs_batch_destroy(b)
        return ms, infos, xebs, tuning

    def state_bytes(precision, infos):
        """HBM bytes of state construction: passes (the sub-state prefix at its own size), reset/expansion."""
        total = 0.0
        for c, inf in zip(circs, infos):
            n = c.n_qubits
            if precision == capi.RCS_PREC_FP32_FUSED:
                total += 16.0 * 2**n * inf["n_passes"] + 8.0 * 2**n
                continue
            plan = capi.rcs_plan_build(n, c.gates, precision)
            pi = capi.rcs_plan_info(plan)
            capi.rcs_plan_destroy(plan)
            # each pass at the size of the state it runs on, the zero fill and the expansions
            total += pi["zero_hbm_bytes"]
        return total

    prec = capi.PRECISIONS[precision]
    ms, infos, xebs, tuning = timed(prec)
    # the same batch without shots: its graph is the persistent tensor-core kernel alone
    # (plus the clear of its counters), so this times state construction by itself
    ms_apply = timed(prec, shots=0)[0]
    apply_bytes = state_bytes(prec, infos)
    sample_bytes = sum(16.0 * 2**c.n_qubits for c in circs)  # block sums + the sampled blocks, about two reads
    ms_f, infos_f, xebs_f, _ = timed(capi.RCS_PREC_FP32_FUSED)
    bytes_f = state_bytes(capi.RCS_PREC_FP32_FUSED, infos_f)
    return {"circs": circs, "shots": shots, "ms": ms, "infos": infos, "xebs": xebs, "apply_bytes": apply_bytes,
            "sample_bytes": sample_bytes, "ms_f": ms_f, "infos_f": infos_f, "xebs_f": xebs_f, "bytes_f": bytes_f,
            "ms_apply": ms_apply, "tuning": tuning, "peak": peaks["hbm_gbs"]}


def config_measure(args, torch, capi, name: str):
    """One of the other single-circuit workloads, timed in the default run: the BF16x3 step
    (reset, passes, shots, XEB) over the run's warm-up and timed steps, and one apply of each
    other path (TF32x3, fused FP32 k = 4, plain FP32 per gate) from |0...0>, with their subset
    infidelities against the fused FP32 state (seeded 2^20 amplitudes, as for the headline),
    and the CPU oracle on the same workload (whole when it fits the sample, else a bounded
    sample scaled up)."""
    circ = C.config_circuit(name)
    n = circ.n_qubits
    shots = C.CONFIGS[name]["shots"]
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    ctx = capi.rcs_create(circ.grid, capi.RCS_PREC_BF16X3, stream=stream.cuda_stream)
    out = {"qubits": n, "shots": shots, "gates": len(circ.gates)}
    try:
        d_bits = torch.empty(shots, dtype=torch.int64, device="cuda")
        d_xeb = torch.empty(1, dtype=torch.float64, device="cuda")
        rng = np.random.default_rng(2**20)
        subset = np.unique(rng.integers(0, 1 << n, size=min(1 << 20, 1 << n), dtype=np.uint64))
        amps = {}
        arms = [("bf16x3", capi.RCS_PREC_BF16X3, 0), ("tf32x3", capi.RCS_PREC_TF32X3, 0),
                ("fp32_fused_k4", capi.RCS_PREC_FP32_FUSED, 4), ("fp32_plain", capi.RCS_PREC_FP32_PLAIN, 0)]
        if n <= 30:  # the fused FP32 widths 5..7 (6 and 7 bound by the FMA pipe) up to the 30-qubit workload
            arms[3:3] = [(f"fp32_fused_k{k}", capi.RCS_PREC_FP32_FUSED, k) for k in (5, 6, 7)]
        for arm, prec, kmax in arms:
            plan = capi.rcs_plan_build(n, circ.gates, prec, kmax)
            info = capi.rcs_plan_info(plan)
            capi.rcs_plan_upload(ctx, plan)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

            def run(seed, sample):
                ev[0].record(stream)
                capi.rcs_reset(ctx)
                capi.rcs_plan_run(ctx, plan)
                ev[1].record(stream)
                if sample:
                    capi.rcs_sample_device(ctx, shots, seed, d_bits.data_ptr())
                    capi.rcs_xeb_device(ctx, d_bits.data_ptr(), shots, d_xeb.data_ptr())
                ev[2].record(stream)
                stream.synchronize()
                return ev[0].elapsed_time(ev[1]), ev[0].elapsed_time(ev[2])

            reps = args.steps if arm == "bf16x3" else 1
            warm = args.warmup if arm in ("bf16x3", "tf32x3", "fp32_fused_k4") else (1 if arm != "fp32_plain" else 0)
            for w in range(warm):
                run(1000 + w, arm == "bf16x3")
            times = [run(s, arm == "bf16x3") for s in range(reps)]
            capi.rcs_sync(ctx)
            apply_s = statistics.median(t[0] for t in times) / 1e3
            rec = {"apply_s": apply_s, "passes": int(info["n_passes"]),
                   "hbm_frac": info["zero_hbm_bytes"] / apply_s / 1e9 / peaks["hbm_gbs"]}
            if arm == "bf16x3":
                rec["step_s"] = statistics.median(t[1] for t in times) / 1e3
                rec["xeb"] = float(d_xeb.item())
                rec["prefix_passes_on_substate"] = int(info["prefix_passes"])
            amps[arm] = capi.rcs_amplitudes(ctx, subset)
            out[arm] = rec
            capi.rcs_plan_destroy(plan)
        ref = amps["fp32_fused_k4"]
        out["subset_infidelity_vs_fp32_fused_k4"] = {
            k: float(1.0 - abs(np.vdot(amps[k], ref)) ** 2 / (np.vdot(amps[k], amps[k]).real * np.vdot(ref, ref).real))
            for k in amps if k != "fp32_fused_k4"}
        out["speedup_bf16x3_vs_fp32_plain"] = out["fp32_plain"]["apply_s"] / out["bf16x3"]["apply_s"]
        if n <= 30 and n >= 20:
            out["fp32_wide_pass"] = wide_pass_measure(torch, capi, n, stream)
    finally:
        capi.rcs_destroy(ctx)
    if not args.no_cpu:
        # the CPU oracle on the same workload: whole at 12 qubits, a bounded sample above
        out["cpu_baseline"] = cpu_baseline(circ, shots, budget_s=8.0)
    return out


# FP32 FMA peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop at the 2070 MHz
# maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def wide_pass_measure(torch, capi, n, stream):
    """One full-state pass of each FP32 fused width 4..7 on its own FP32 context (width 4
    carries U in the kernel parameters, 5..7 multiply tiles by U in shared memory): one
    untimed pass, then three passes applied in one call and timed by the library's CUDA
    events around their launches (rcs_last_pass_timing; the host's validation and upload of
    the matrices fall outside). Against the FP32 FMA peak (8 * 2^k real flop per amplitude)
    and against HBM (16 bytes per amplitude)."""
    rng = np.random.default_rng(7)
    res = {}
    ctx = capi.rcs_create(n, capi.RCS_PREC_FP32_FUSED, stream=stream.cuda_stream)
    for k in (4, 5, 6, 7):
        targets = list(range(5, 5 + k))  # above the 32 slices a warp stores side by side
        mats = []
        for _ in range(4):
            a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
            q, r = np.linalg.qr(a)
            mats.append(q * (np.diag(r) / abs(np.diag(r))))
        capi.rcs_apply_unitary(ctx, targets, mats[0])
        capi.rcs_apply_unitaries(ctx, [(targets, u) for u in mats[1:]])
        total_ms, launches = capi.rcs_last_pass_timing(ctx)
        ms = total_ms / launches
        flops = 8.0 * 2**k * 2**n
        res[f"k{k}"] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12,
                        "alu_frac": flops / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                        "hbm_frac": 16.0 * 2**n / (ms / 1e3) / 1e9 / measured_peaks()["hbm_gbs"]}
    capi.rcs_destroy(ctx)
    res["peak_tflops"] = FP32_PEAK_TFLOPS
    res["peak_source"] = "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (unit counts and maximum clock)"
    return res


def run_batch(args, torch, capi):
    """The 64-circuit batched workload as its own JSON line: the tensor-core engine is the
    line's value, the persistent FP32 engine is in `compare`."""
    m = batch64_measure(args, torch, capi, args.precision)
    circs, shots, ms, infos, xebs = m["circs"], m["shots"], m["ms"], m["infos"], m["xebs"]
    apply_bytes, sample_bytes, ms_f, infos_f, xebs_f, bytes_f = (m["apply_bytes"], m["sample_bytes"], m["ms_f"],
                                                                 m["infos_f"], m["xebs_f"], m["bytes_f"])
    peaks = {"hbm_gbs": m["peak"]}
    line = {"metric": "64-circuit batched workload time (s)", "value": ms / 1e3, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "data": "synthetic", "dtype": f"{args.precision} (fp32 accumulate); fp32 state",
            "config": {"workload": "batch64", "circuits": len(circs), "engine": "persistent tensor-core kernel",
                       "qubits": [c.n_qubits for c in circs], "shots_per_circuit": shots,
                       "k": [inf["k"] for inf in infos], "passes": [inf["n_passes"] for inf in infos],
                       "l2": "states of 16-26 qubits: the largest (512 MiB) exceed L2; no flush between steps"},
            "state_hbm_bytes": apply_bytes,
            "state_plus_sampling_GBps": (apply_bytes + sample_bytes) / (ms / 1e3) / 1e9,
            "frac_of_hbm": (apply_bytes + sample_bytes) / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "xeb_mean": float(np.mean(xebs)), "xeb_min": float(np.min(xebs)), "xeb_max": float(np.max(xebs)),
            "roofline": {"bound": "hbm", "kernel": "k_batch_tc (all passes of all circuits, one launch)",
                         "achieved": apply_bytes / (m["ms_apply"] / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": apply_bytes / (m["ms_apply"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "traffic": BATCH64_TC_DRAM_BYTES,
                         "traffic_src": "ncu capture of one launch on this workload (dram read + write)",
                         "duration_ms": m["ms_apply"]},
            "apply_only_s": m["ms_apply"] / 1e3, "sampling_and_xeb_s": (ms - m["ms_apply"]) / 1e3,
            "tuning": m["tuning"],
            "compare": {"fp32_persistent": {
                "value": ms_f / 1e3, "k_chosen": [inf["k"] for inf in infos_f],
                "passes_total": int(sum(inf["n_passes"] for inf in infos_f)), "state_hbm_bytes": bytes_f,
                "frac_of_hbm": (bytes_f + sample_bytes) / (ms_f / 1e3) / 1e9 / peaks["hbm_gbs"],
                "xeb_mean": float(np.mean(xebs_f))},
                "speedup_vs_fp32_persistent": ms_f / ms}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    from paper_2512_07311_gb300 import build as B
    from paper_2512_07311_gb300 import capi

    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    capi.load()
    if args.workload == "batch64":
        return run_batch(args, torch, capi)
    if args.fp32_wide_pass:
        if not 20 <= args.fp32_wide_pass <= 30:
            raise SystemExit("--fp32-wide-pass takes 20..30 qubits")
        res = wide_pass_measure(torch, capi, args.fp32_wide_pass, torch.cuda.current_stream())
        print(json.dumps({"fp32_wide_pass": res, "qubits": args.fp32_wide_pass}))
        return 0
    cfg = C.CONFIGS[args.workload]
    if args.qubits:
        circ = C.generate(C.grid_for_n(args.qubits), 20, "ABCDCDAB", seed=2)
        args.workload = f"{args.qubits}q_profile_20cyc"
    else:
        circ = C.config_circuit(args.workload)
    n = circ.n_qubits
    shots = args.shots or cfg["shots"]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prec = capi.PRECISIONS[args.precision]
    other = "tf32x3" if args.precision == "bf16x3" else "bf16x3"
    flags = capi.RCS_OPT_PAIR_PASSES if args.pair_passes else 0
    ctx = capi.rcs_create(circ.grid, prec, stream=sh, flags=flags)
    plan = capi.rcs_plan_build(n, circ.gates, prec, flags=flags)
    info = capi.rcs_plan_info(plan)
    pairs = int(info["pair_passes"])
    # operand images uploaded per tensor-core pass: the single-pass image, plus the pair
    # kernel's complex-form image when the plan pairs passes
    ops_bytes = (65536 if args.precision == "bf16x3" else 98304) + (32768 if pairs else 0)
    capi.rcs_plan_upload(ctx, plan)
    d_bits = torch.empty(shots, dtype=torch.int64, device="cuda")
    d_xeb = torch.empty(1, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    apply_ms, sample_ms, xeb_ms = [], [], []

    def step(seed, timed):
        ev[0].record(stream)
        capi.rcs_reset(ctx)
        capi.rcs_plan_run(ctx, plan)
        ev[1].record(stream)
        capi.rcs_sample_device(ctx, shots, seed, d_bits.data_ptr())
        ev[2].record(stream)
        capi.rcs_xeb_device(ctx, d_bits.data_ptr(), shots, d_xeb.data_ptr())
        ev[3].record(stream)
        if timed:
            stream.synchronize()
            apply_ms.append(ev[0].elapsed_time(ev[1]))
            sample_ms.append(ev[1].elapsed_time(ev[2]))
            xeb_ms.append(ev[2].elapsed_time(ev[3]))

    for w in range(args.warmup):
        step(1000 + w, False)
    capi.rcs_sync(ctx)
    barrier()
    pass_ms = []  # device time of the full-state tensor-core passes of each timed step
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        barrier()
        t_start.record(stream)
        for s in range(args.steps):
            step(s, False)
            # the library's events around this step's full-state passes; reading them
            # waits for those passes only (the sampler of this step keeps running)
            ms_p, full = capi.rcs_last_pass_timing(ctx)
            pass_ms.append(ms_p)
            timed_full = full
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    capi.rcs_sync(ctx)
    # per-phase breakdown from a separate, identical set of steps
    for s in range(min(args.steps, 3)):
        step(s, True)
    ms_step = max_over_ranks(total_ms / args.steps, dist, "cuda")
    F = float(d_xeb.item())

    # roofline of the dominant kernel (the tensor-core pass): algorithmic bytes per launch / mean launch time,
    # from the CUDA events the library records around the full-state passes of every timed step
    peaks = measured_peaks()
    passes = int(info["n_passes"])
    prefix = int(info["prefix_passes"])
    # the library times the full-state passes; the first full pass may run fused with the
    # expansion of the last sub-state, before the timed region of the passes
    full_passes = timed_full
    t_pass_s = statistics.median(pass_ms) / 1e3 / full_passes
    # launches per step: sub-state reset, expansions between sub-states, the final expansion
    # unless the first full pass reads the last sub-state, every pass, block sums, the 3-phase
    # scan, the sampler (locate, 3-phase scan of its per-block counts, order, resolve) and the
    # 2-phase XEB
    stages = int(info["prefix_stages"])
    fused = prefix > 0 and full_passes == passes - prefix - 1
    setup = 1 + max(stages - 1, 0) + (0 if (prefix == 0 or fused) else 1)
    gpu_launches = (passes - pairs) + setup + 1 + 3 + 6 + 2
    bytes_per_launch = 16.0 * 2.0**n
    achieved = bytes_per_launch / t_pass_s / 1e9
    # traffic: DRAM bytes per launch from an ncu capture of the same kernel (None for a kernel
    # not captured since it last changed)
    traffic = PAIR_DRAM_BYTES_PER_AMP if pairs else TC_DRAM_BYTES_PER_AMP[args.precision]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic * 2.0**n if traffic else None,
                "traffic_src": "ncu capture at 27 qubits scaled by 2^(n-27)" if traffic else None,
                "kernel": "k_pair_tc (two unitaries per launch)" if pairs else "k_fused_tc", "peak_src": peaks["src"],
                "algorithmic_bytes_per_launch": bytes_per_launch, "launches_per_step": full_passes,
                "mean_launch_ms": t_pass_s * 1e3}

    # end to end through the host-buffer API: gate list in, samples out, samples in, XEB out
    e2e_ms = []
    for s in range(max(1, min(args.steps, 3))):
        barrier()
        t0 = time.perf_counter()
        capi.rcs_reset(ctx)
        capi.rcs_apply_circuit(ctx, circ.gates)
        xs = capi.rcs_sample(ctx, shots, 77 + s)
        F_e2e = capi.rcs_xeb(ctx, xs)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = circ.gates.nbytes + passes * ops_bytes + shots * 8
    d2h = shots * 8 + 8

    compare = {}
    if not args.no_compare:
        # same circuit through the plain FP32 per-gate path, the fused FP32 path and the other
        # tensor-core split (one run each), and the subset infidelity of each state against the
        # fused FP32 state on a seeded 2^20-amplitude subset
        rng = np.random.default_rng(2**20)
        subset = np.unique(rng.integers(0, 1 << n, size=1 << 20, dtype=np.uint64))
        capi.rcs_reset(ctx)
        capi.rcs_plan_run(ctx, plan)
        amps = {args.precision: capi.rcs_amplitudes(ctx, subset)}
        arms = [("fp32_plain", capi.RCS_PREC_FP32_PLAIN, 0, 0), ("fp32_fused_k4", capi.RCS_PREC_FP32_FUSED, 4, 0),
                (other, capi.PRECISIONS[other], 0, 0)]
        if args.precision == "bf16x3":
            # the opt-in two-unitary round trips, timed beside the default single passes
            arms.append(("bf16x3_pair_passes", prec, 0, 0 if pairs else capi.RCS_OPT_PAIR_PASSES))
        for name, p2prec, kmax, flags in arms:
            p2 = capi.rcs_plan_build(n, circ.gates, p2prec, kmax, flags=flags)
            i2 = capi.rcs_plan_info(p2)
            capi.rcs_plan_upload(ctx, p2)
            capi.rcs_reset(ctx)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            capi.rcs_plan_run(ctx, p2)
            e1.record(stream)
            capi.rcs_sync(ctx)
            t = e0.elapsed_time(e1) / 1e3
            amps[name] = capi.rcs_amplitudes(ctx, subset)
            # algorithmic bytes of the run from |0...0> (sub-state passes at their own size)
            compare[name] = {"apply_s": t, "passes": int(i2["n_passes"]),
                             "hbm_frac": i2["zero_hbm_bytes"] / t / 1e9 / peaks["hbm_gbs"]}
            capi.rcs_plan_destroy(p2)

        def subset_infidelity(a, b):
            return float(1.0 - abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))

        ref = amps["fp32_fused_k4"]
        compare["subset_infidelity_vs_fp32_fused_k4"] = {k: subset_infidelity(amps[k], ref)
                                                         for k in amps if k != "fp32_fused_k4"}
        compare[f"{args.precision}_apply_s"] = statistics.median(apply_ms) / 1e3
        compare["speedup_vs_fp32_plain"] = compare["fp32_plain"]["apply_s"] / compare[f"{args.precision}_apply_s"]

    cpu = None
    check = None
    if args.oracle_check and rank == 0 and world == 1:
        plans = {args.precision: plan}
        extra = []
        for name, p2prec in ((other, capi.PRECISIONS[other]), ("fp32_plain", capi.RCS_PREC_FP32_PLAIN)):
            p2 = capi.rcs_plan_build(n, circ.gates, p2prec)
            capi.rcs_plan_upload(ctx, p2)
            plans[name] = p2
            extra.append(p2)
        cpu, check = oracle_check(circ, shots, ctx, plans, args.precision, capi)
        for p2 in extra:
            capi.rcs_plan_destroy(p2)
    if cpu is None and rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(circ, shots)

    capi.rcs_plan_destroy(plan)
    capi.rcs_destroy(ctx)
    clocks = clk.summary()
    if not args.no_compare and world == 1 and args.precision == "bf16x3":
        # the batched workload (64 circuits of 16-26 qubits), timed in the same run
        m = batch64_measure(args, torch, capi, "bf16x3")
        both = m["apply_bytes"] + m["sample_bytes"]
        compare["batch64"] = {
            "tensor_core_s": m["ms"] / 1e3, "fp32_persistent_s": m["ms_f"] / 1e3,
            "tensor_core_frac_of_hbm": both / (m["ms"] / 1e3) / 1e9 / m["peak"],
            "tensor_core_apply_only_s": m["ms_apply"] / 1e3,
            "tensor_core_apply_frac_of_hbm": m["apply_bytes"] / (m["ms_apply"] / 1e3) / 1e9 / m["peak"],
            "tiles_per_item": m["tuning"]["tiles_per_item"] if m["tuning"] else None,
            "fp32_frac_of_hbm": (m["bytes_f"] + m["sample_bytes"]) / (m["ms_f"] / 1e3) / 1e9 / m["peak"],
            "xeb_mean_tensor_core": float(np.mean(m["xebs"])), "steps": args.steps}
        # the other single-circuit workloads (12, 30 and 32 qubits), timed in the same run
        compare["configs"] = {name: config_measure(args, torch, capi, name)
                              for name in ("12q_3x4_8cyc", "30q_5x6_14cyc", "32q_4x8_20cyc")}
    if rank == 0:
        line = {
            "metric": METRIC, "value": per_circuit_seconds(ms_step, world), "unit": "s", "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": f"{args.precision} (fp32 accumulate); fp32 state; exact fixed-point/f64 reductions",
            "data": "synthetic",
            "config": {"workload": args.workload, "qubits": n, "cycles": circ.cycles, "pattern": circ.pattern,
                       "grid": f"{circ.grid.rows}x{circ.grid.cols}-{len(circ.grid.removed)}", "shots": shots,
                       "gates": len(circ.gates), "passes": passes, "prefix_passes_on_substate": prefix,
                       "prefix_qubits": int(info["prefix_qubits"]), "precision": args.precision,
                       "state_bytes": 8 * 2**n, "l2": (f"inputs larger than L2 (state {8 * 2**n / 2**30:.0f} GiB > 129 MB)" if 8 * 2**n > 129e6
                              else "state fits in L2: no flush between steps"),
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "shots_per_s": shots / (statistics.median(sample_ms) / 1e3),
            "phases_ms": {"reset+apply": statistics.median(apply_ms), "sample": statistics.median(sample_ms),
                          "xeb": statistics.median(xeb_ms)},
            "xeb": F, "xeb_e2e": F_e2e,
            "roofline": roofline,
            "e2e": {"value": statistics.median(e2e_ms) / 1e3, "unit": "s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "compare": compare,
            "cpu_baseline": cpu,
        }
        if check is not None:
            line["oracle_check"] = check
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
