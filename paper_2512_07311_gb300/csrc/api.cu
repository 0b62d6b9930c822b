// C ABI of the library (include/rcs.h): context and device memory, validation,
// planning, pass launches, sampling and scoring calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"

using namespace rcs;

struct rcs_ctx {
    int n = 0;
    int dev = 0;
    cudaStream_t stream = nullptr;
    rcs_opts opts{};
    float2 *psi = nullptr;
    uint64_t *bsum = nullptr, *bpre = nullptr, *chunk = nullptr, *total = nullptr;
    int *d_err = nullptr;
    bool sums_valid = false;  // bsum/bpre/total describe the current state
    // growable scratch for host-provided arrays and results
    uint64_t *d_u64 = nullptr;
    size_t u64_cap = 0;
    double *d_f64 = nullptr;
    size_t f64_cap = 0;
    uint64_t *d_order = nullptr;  // the sampler's shots grouped by block
    size_t order_cap = 0;
    uint8_t *d_ops = nullptr;  // tensor-core operand images of rcs_apply_circuit plans
    size_t ops_cap = 0;
    // Qubit layout: circuit qubit q is stored at index bit phys_of[q]. A fresh state
    // (|0...0>, after create or reset) looks the same in every layout, so the first
    // circuit on it may choose one; later circuits follow it.
    int phys_of[64] = {};
    bool fresh = true;
    // The state is |0...0> but not written yet (create/reset are lazy): the first
    // fused run from it writes the whole state itself, anything else fills it first.
    bool zero_pending = false;
    float2 *d_sub = nullptr;  // compact sub-state for the first passes of a run from |0...0>
    size_t sub_cap = 0;
    cudaEvent_t ev_full[2] = {nullptr, nullptr};  // around the full-state passes of the last run
    int64_t timed_passes = -1;
    std::string err;
};

struct rcs_plan {
    Plan p;
    uint8_t *d_ops = nullptr;
    int d_ops_dev = -1;
};

namespace {

thread_local std::string g_err;

int fail(rcs_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_err = msg;
    return code;
}

int cuda_fail(rcs_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? RCS_ERR_OOM : RCS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define RCS_CUDA(ctx, call, what)                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

int dev_sms[64] = {};

int ensure_u64(rcs_ctx *c, size_t count) {
    if (count <= c->u64_cap) return RCS_OK;
    RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (c->d_u64) cudaFree(c->d_u64);
    c->d_u64 = nullptr;
    c->u64_cap = 0;
    size_t cap = std::max<size_t>(count, 1024);
    RCS_CUDA(c, cudaMalloc(&c->d_u64, cap * sizeof(uint64_t)), "cudaMalloc scratch");
    c->u64_cap = cap;
    return RCS_OK;
}

int ensure_order(rcs_ctx *c, size_t count) {
    if (count <= c->order_cap) return RCS_OK;
    RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (c->d_order) cudaFree(c->d_order);
    c->d_order = nullptr;
    c->order_cap = 0;
    size_t cap = std::max<size_t>(count, 1024);
    RCS_CUDA(c, cudaMalloc(&c->d_order, cap * sizeof(uint64_t)), "cudaMalloc sampler scratch");
    c->order_cap = cap;
    return RCS_OK;
}

int ensure_f64(rcs_ctx *c, size_t count) {
    if (count <= c->f64_cap) return RCS_OK;
    RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
    if (c->d_f64) cudaFree(c->d_f64);
    c->d_f64 = nullptr;
    c->f64_cap = 0;
    size_t cap = std::max<size_t>(count, 1024);
    RCS_CUDA(c, cudaMalloc(&c->d_f64, cap * sizeof(double)), "cudaMalloc scratch");
    c->f64_cap = cap;
    return RCS_OK;
}

// Synchronises the stream and turns the device error word into a status (and clears it).
int drain_errors(rcs_ctx *c) {
    RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
    int h = 0;
    RCS_CUDA(c, cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (h == 0) return RCS_OK;
    RCS_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)), "clear error word");
    if (h & kErrTimeout) return fail(c, RCS_ERR_TIMEOUT, "a bounded wait inside a tensor-core pass ran out");
    if (h & kErrBadIndex) return fail(c, RCS_ERR_ARG, "bitstring index >= 2^n");
    if (h & kErrBadAmplitude) return fail(c, RCS_ERR_ARG, "state holds an amplitude component >= 2 or not finite");
    return fail(c, RCS_ERR_ARG, "state norm too large for the fixed-point reduction (>= 4)");
}

int valid_gates(rcs_ctx *ctx, int n, const rcs_gate *gates, size_t count, std::vector<HostGate> *out) {
    if (count && !gates) return fail(ctx, RCS_ERR_ARG, "null gate array");
    out->resize(count);
    for (size_t i = 0; i < count; ++i) {
        std::string why;
        int rc = gate_to_host(gates[i], n, &(*out)[i], &why);
        if (rc != RCS_OK) return fail(ctx, rc, "gate " + std::to_string(i) + ": " + why);
    }
    return RCS_OK;
}


// ---- autotuner for the fused FP32 path: k_max in 2..5 minimising
// (passes of the circuit at width k) x (measured time of one width-k pass on this
// state), cached per (device, qubit count). Widths 6 and 7 are not tried: at 32 and
// 64 flop per byte their passes are bound by the FP32 FMA pipe, several times longer
// than a round trip through HBM, while they cut the passes by far less. The trial passes are phase permutations
// (entries 0 and i): FP32 multiply-adds apply them exactly, and applying their
// inverses afterwards restores the caller's state bit for bit.
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned_k;

int autotune_fused_k(rcs_ctx *c, const std::vector<HostGate> &hg, int *k_out) {
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned_k.find({c->dev, c->n});
        if (it != g_tuned_k.end()) {
            *k_out = it->second;
            return RCS_OK;
        }
    }
    cudaEvent_t e0, e1;
    RCS_CUDA(c, cudaEventCreate(&e0), "event");
    RCS_CUDA(c, cudaEventCreate(&e1), "event");
    double best = 1e300;
    int best_k = std::min(4, c->n);
    const int reps = 3;
    for (int k = 2; k <= std::min(5, c->n); ++k) {
        Pass fwd, inv;
        fwd.kind = inv.kind = PASS_SIMT;
        fwd.k = inv.k = k;
        for (int i = 0; i < 8; ++i) fwd.t[i] = inv.t[i] = i < k ? i * (c->n / k) : -1;
        const int d = 1 << k;
        fwd.U.assign(size_t(d) * d, cd(0.0));
        inv.U.assign(size_t(d) * d, cd(0.0));
        for (int j = 0; j < d; ++j) {
            fwd.U[size_t(j) * d + (j + 1) % d] = cd(0.0, 1.0);  // i * cyclic shift
            inv.U[size_t((j + 1) % d) * d + j] = cd(0.0, -1.0);
        }
        // widths above the parameter-space kernel read U from a device image
        const size_t ib = simt_ops_bytes(k);
        uint8_t *d_img = nullptr;
        int rc = RCS_OK;
        if (ib > 0) {
            std::vector<uint8_t> img(2 * ib);
            simt_build_ops(fwd, img.data());
            simt_build_ops(inv, img.data() + ib);
            if (cudaMalloc(&d_img, 2 * ib) != cudaSuccess ||
                cudaMemcpy(d_img, img.data(), 2 * ib, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = RCS_ERR_CUDA;
        }
        const uint8_t *ops_f = d_img, *ops_i = d_img ? d_img + ib : nullptr;
        if (rc == RCS_OK) rc = launch_pass_simt(c->psi, c->n, fwd, ops_f, c->stream);  // warm-up
        if (rc == RCS_OK) rc = launch_pass_simt(c->psi, c->n, inv, ops_i, c->stream);
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && rc == RCS_OK; ++r) rc = launch_pass_simt(c->psi, c->n, fwd, ops_f, c->stream);
        cudaEventRecord(e1, c->stream);
        for (int r = 0; r < reps && rc == RCS_OK; ++r) rc = launch_pass_simt(c->psi, c->n, inv, ops_i, c->stream);
        if (d_img) {
            cudaStreamSynchronize(c->stream);
            cudaFree(d_img);
        }
        if (rc != RCS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(c, rc, "autotune trial: " + take_launch_error());
        }
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        std::vector<Pass> passes;
        plan_fuse(c->n, hg, k, 0, &passes);
        const double est = double(ms) / reps * double(passes.size());
        if (est < best) {
            best = est;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned_k[{c->dev, c->n}] = best_k;
    *k_out = best_k;
    return RCS_OK;
}

// Fused plans built with allow_layout may store the circuit in a permuted qubit
// layout (choose_layout) when that keeps two of the lowest bits out of every pass;
// plan->phys_of then records it.
int build_plan(rcs_ctx *ctx, int n, const std::vector<HostGate> &hg, const rcs_opts &o, Plan *plan,
               bool allow_layout) {
    plan->n = n;
    plan->precision = o.precision;
    plan->pairs = o.precision == RCS_PREC_BF16X3 && (o.flags & RCS_OPT_PAIR_PASSES);
    plan->n_gates = int64_t(hg.size());
    plan->phys_of.clear();
    plan->stage_spans.clear();
    // allow_layout: the plan is for a fresh state, so it may choose a layout and is
    // planned for a run from |0...0> (sub-state prefix counted)
    auto fused = [&](int k, int pad) {
        Blocking bl = plan_blocks(n, hg, k, allow_layout);
        plan->stage_spans = bl.spans;
        int phys[64];
        if (allow_layout && choose_layout(n, hg, bl, phys)) {
            std::vector<HostGate> moved = hg;
            for (HostGate &g : moved)
                for (int a = 0; a < g.nq; ++a) g.q[a] = phys[g.q[a]];
            for (uint64_t &av : bl.avoid) {
                uint64_t moved_av = 0;
                for (int q = 0; q < n; ++q)
                    if ((av >> q) & 1) moved_av |= 1ull << phys[q];
                av = moved_av;
            }
            make_passes(n, moved, bl, pad, &plan->passes);
            plan->phys_of.assign(phys, phys + n);
        } else {
            make_passes(n, hg, bl, pad, &plan->passes);
        }
    };
    switch (o.precision) {
        case RCS_PREC_FP32_PLAIN:
            plan->k_max = 2;
            plan_plain(n, hg, &plan->passes);
            break;
        case RCS_PREC_FP32_FUSED: {
            int k = o.k_max > 0 ? o.k_max : 4;
            if (k < 2 || k > kSimtKMax) return fail(ctx, RCS_ERR_ARG, "FP32_FUSED k_max must be 2..7");
            plan->k_max = std::min(k, n);
            if (n == 1) plan_plain(n, hg, &plan->passes);
            else fused(plan->k_max, 0);
            break;
        }
        case RCS_PREC_BF16X3:
        case RCS_PREC_TF32X3:
            if (o.k_max > 0 && o.k_max != kTcK) return fail(ctx, RCS_ERR_ARG, "the tensor-core paths use k_max = 6");
            if (n >= kTcK + 7) {
                plan->k_max = kTcK;
                fused(kTcK, kTcK);
            } else {  // fewer than one 128-slice tile: the FP32 fused path serves small states
                plan->k_max = std::min(5, n);
                if (n == 1) plan_plain(n, hg, &plan->passes);
                else fused(plan->k_max, 0);
            }
            break;
        default:
            return fail(ctx, RCS_ERR_ARG, "unknown precision");
    }
    return RCS_OK;
}

bool layout_identity(const rcs_ctx *c) {
    for (int q = 0; q < c->n; ++q)
        if (c->phys_of[q] != q) return false;
    return true;
}

void set_identity_layout(rcs_ctx *c) {
    for (int q = 0; q < 64; ++q) c->phys_of[q] = q;
}

// caller's basis index -> stored index
BitMap to_stored(const rcs_ctx *c) {
    BitMap m = identity_map(c->n);
    if (layout_identity(c)) return m;
    m.identity = 0;
    for (int q = 0; q < c->n; ++q) m.to[q] = uint8_t(c->phys_of[q]);
    return m;
}

// Brings the stored state back to the identity layout with exact swap passes
// (entries 0 and 1, so FP32 moves the amplitudes unchanged).
int restore_layout(rcs_ctx *c) {
    if (c->zero_pending) {  // |0...0> in any layout
        set_identity_layout(c);
        return RCS_OK;
    }
    int log_of[64];
    for (int q = 0; q < c->n; ++q) log_of[c->phys_of[q]] = q;
    for (int p = 0; p < c->n; ++p) {
        while (log_of[p] != p) {
            const int l = log_of[p];
            const int q = c->phys_of[p];  // where circuit qubit p sits now
            Pass sw;
            sw.kind = PASS_2Q;
            sw.k = 2;
            for (int i = 0; i < 8; ++i) sw.t[i] = -1;
            sw.t[0] = std::min(p, q);
            sw.t[1] = std::max(p, q);
            sw.U.assign(16, cd(0.0));
            sw.U[0] = sw.U[6] = sw.U[9] = sw.U[15] = 1.0;
            if (launch_pass_plain(c->psi, c->n, sw, c->stream) != RCS_OK)
                return fail(c, RCS_ERR_CUDA, "layout swap: " + take_launch_error());
            c->phys_of[p] = p;
            c->phys_of[l] = q;
            log_of[p] = p;
            log_of[q] = l;
        }
    }
    c->sums_valid = false;
    return RCS_OK;
}

bool plan_tf32(const Plan &plan) { return plan.precision == RCS_PREC_TF32X3; }

// Builds the device images of a plan into one host buffer: the split operand images of
// every tensor-core pass, the pair kernel's images, and the FP32 U of every SIMT pass
// wider than the kernel parameters hold.
void build_ops_images(Plan &plan, std::vector<uint8_t> *img) {
    const bool tf32 = plan_tf32(plan);
    const size_t per = tc_ops_bytes(tf32);
    plan.tc_offset.assign(plan.passes.size(), -1);
    size_t count = 0;
    for (size_t i = 0; i < plan.passes.size(); ++i)
        if (plan.passes[i].kind == PASS_TC) plan.tc_offset[i] = int64_t(per * count++);
    // the pair kernel's images (complex block form) follow the single-pass ones
    plan.pair_offset.assign(plan.passes.size(), -1);
    size_t total = per * count;
    if (plan.pairs)
        for (size_t i = 0; i < plan.passes.size(); ++i)
            if (plan.passes[i].kind == PASS_TC) {
                plan.pair_offset[i] = int64_t(total);
                total += pair_ops_bytes();
            }
    // FP32 images of the wide SIMT passes (16-byte multiples, so every offset stays aligned)
    for (size_t i = 0; i < plan.passes.size(); ++i)
        if (plan.passes[i].kind == PASS_SIMT && simt_ops_bytes(plan.passes[i].k) > 0) {
            plan.tc_offset[i] = int64_t(total);
            total += simt_ops_bytes(plan.passes[i].k);
        }
    img->assign(total, 0);
    // independent images in disjoint slices of the buffer
    host_parallel_for(plan.passes.size(), [&](size_t i) {
        if (plan.tc_offset[i] >= 0 && plan.passes[i].kind == PASS_SIMT)
            simt_build_ops(plan.passes[i], img->data() + plan.tc_offset[i]);
        else if (plan.tc_offset[i] >= 0) tc_build_ops(plan.passes[i], img->data() + plan.tc_offset[i], tf32);
        if (plan.pair_offset[i] >= 0) pair_build_ops(plan.passes[i], img->data() + plan.pair_offset[i]);
    });
}

int materialize(rcs_ctx *c) {
    if (!c->zero_pending) return RCS_OK;
    if (launch_init_zero(c->psi, c->n, c->stream) != RCS_OK) return fail(c, RCS_ERR_CUDA, "reset: " + take_launch_error());
    c->zero_pending = false;
    return RCS_OK;
}

Pass compact_pass(const Pass &p, uint64_t T) {
    Pass q = p;
    for (int i = 0; i < p.k; ++i) q.t[i] = std::popcount(T & ((1ull << p.t[i]) - 1ull));
    return q;
}

// Launches the plan's passes. from_zero: the state is |0...0> (it may not be written
// yet); the leading passes that touch few qubits then run on a compact sub-state
// that one expansion pass writes out as the whole state.
int run_passes(rcs_ctx *c, const Plan &plan, const uint8_t *d_ops, bool from_zero) {
    size_t first = 0;
    std::vector<SubStage> stages;
    const int pre = from_zero ? plan_stages(plan, &stages) : 0;
    if (pre > 0) {
        const size_t bytes = substage_bytes(stages);
        if (bytes > c->sub_cap) {
            RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
            cudaFree(c->d_sub);
            c->d_sub = nullptr;
            c->sub_cap = 0;
            RCS_CUDA(c, cudaMalloc(&c->d_sub, bytes), "cudaMalloc sub-state");
            c->sub_cap = bytes;
        }
        int fused = 0;
        if (run_substages(plan, stages, c->psi, c->d_sub, d_ops, c->d_err, c->stream, &fused) != RCS_OK)
            return fail(c, RCS_ERR_CUDA, "sub-state stages: " + take_launch_error());
        c->zero_pending = false;
        first = size_t(pre + fused);
    } else if (int rc = materialize(c); rc != RCS_OK) {
        return rc;
    }
    cudaEventRecord(c->ev_full[0], c->stream);
    int64_t launches = 0;
    if (launch_pass_range(plan, c->psi, c->n, first, plan.passes.size(), 0, d_ops, c->d_err, c->stream, &launches) !=
        RCS_OK)
        return fail(c, RCS_ERR_CUDA, "launch of a full-state pass failed: " + take_launch_error());
    cudaEventRecord(c->ev_full[1], c->stream);
    c->timed_passes = launches;
    c->sums_valid = false;
    return RCS_OK;
}

int ensure_sums(rcs_ctx *c) {
    if (c->sums_valid) return RCS_OK;
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    int rc = launch_block_sums(c->psi, c->n, c->bsum, c->d_err, to_stored(c), c->stream);
    if (rc == RCS_OK) rc = launch_block_scan(c->bsum, c->bpre, c->chunk, c->total, c->n, c->d_err, c->stream);
    if (rc != RCS_OK) return fail(c, rc, "reduction launch failed: " + take_launch_error());
    c->sums_valid = true;
    return RCS_OK;
}

}  // namespace

namespace rcs {
thread_local std::string g_launch_err;

int note_launch_error(const char *what, cudaError_t e) {
    g_launch_err = std::string(what) + ": " + cudaGetErrorString(e);
    return RCS_ERR_CUDA;
}

int note_launch_refusal(int code, const char *msg) {
    g_launch_err = msg;
    return code;
}

int launch_status(const char *what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RCS_OK : note_launch_error(what, e);
}

std::string take_launch_error() {
    std::string s;
    s.swap(g_launch_err);
    return s.empty() ? std::string("unknown launch failure") : s;
}

int set_thread_error(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int plan_fresh_circuit(int n, const std::vector<HostGate> &gates, const rcs_opts &o, Plan *plan,
                       std::vector<uint8_t> *images) {
    const int rc = build_plan(nullptr, n, gates, o, plan, true);
    if (rc == RCS_OK) build_ops_images(*plan, images);
    return rc;
}

Pass substate_pass(const Pass &p, uint64_t T) { return compact_pass(p, T); }

int launch_plan_pass(void *psi, int n, const Pass &p, const uint8_t *ops, int *d_err, void *stream, bool tf32) {
    switch (p.kind) {
        case PASS_1Q:
        case PASS_2Q: return launch_pass_plain(psi, n, p, stream);
        case PASS_SIMT: return launch_pass_simt(psi, n, p, ops, stream);
        case PASS_TC: return launch_pass_tc(psi, n, p, ops, d_err, stream, tf32);
        default: return RCS_ERR_ARG;
    }
}

int run_substages(const Plan &plan, const std::vector<SubStage> &stages, void *psi, void *sub, const uint8_t *d_ops,
                  int *d_err, void *stream, int *fused) {
    const bool tf32 = plan_tf32(plan);
    *fused = 0;
    uint8_t *buf = static_cast<uint8_t *>(sub);
    uint8_t *cur = nullptr;
    uint64_t cur_mask = 0;
    for (size_t si = 0; si < stages.size(); ++si) {
        const SubStage &st = stages[si];
        const int m = std::popcount(st.tmask);
        uint8_t *next = buf;
        buf += size_t(8) << m;
        if (cur == nullptr) {
            if (launch_init_zero(next, m, stream) != RCS_OK) return RCS_ERR_CUDA;
        } else {  // the previous sub-state's qubits, numbered inside this one
            uint64_t inner = 0;
            for (int q = 0, k = 0; q < plan.n; ++q)
                if ((st.tmask >> q) & 1) {
                    if ((cur_mask >> q) & 1) inner |= 1ull << k;
                    ++k;
                }
            if (launch_expand(next, m, cur, inner, stream) != RCS_OK) return RCS_ERR_CUDA;
        }
        int64_t launches = 0;
        if (launch_pass_range(plan, next, m, size_t(st.first), size_t(st.first + st.count), st.tmask, d_ops, d_err,
                              stream, &launches) != RCS_OK)
            return RCS_ERR_CUDA;
        cur = next;
        cur_mask = st.tmask;
    }
    const size_t after = size_t(stages.back().first + stages.back().count);
    if (after < plan.passes.size() && tc_pass_takes_substate(plan.passes[after], plan.n)) {
        const int rc = launch_pass_tc_from_sub(psi, plan.n, plan.passes[after], d_ops + plan.tc_offset[after], d_err,
                                               stream, tf32, cur, cur_mask);
        if (rc == RCS_OK) *fused = 1;
        return rc;
    }
    return launch_expand(psi, plan.n, cur, cur_mask, stream);
}

bool plan_pairs_at(const Plan &plan, size_t i, size_t end, int n) {
    return plan.pairs && i + 1 < end && pair_fits(plan.passes[i], plan.passes[i + 1], n);
}

int launch_pass_range(const Plan &plan, void *psi, int n, size_t first, size_t end, uint64_t T, const uint8_t *d_ops,
                      int *d_err, void *stream, int64_t *launches) {
    const bool tf32 = plan_tf32(plan);
    Pass c0, c1;  // targets renumbered into the sub-state
    auto at = [&](size_t i, Pass &tmp) -> const Pass & {
        if (!T) return plan.passes[i];
        tmp = compact_pass(plan.passes[i], T);
        return tmp;
    };
    for (size_t i = first; i < end;) {
        const Pass &p = at(i, c0);
        if (plan_pairs_at(plan, i, end, n) && plan.pair_offset.size() == plan.passes.size() &&
            plan.pair_offset[i] >= 0 && plan.pair_offset[i + 1] >= 0) {
            const Pass &p2 = at(i + 1, c1);
            if (launch_pair_tc(psi, n, p, p2, d_ops + plan.pair_offset[i], d_ops + plan.pair_offset[i + 1], d_err,
                               stream) != RCS_OK)
                return RCS_ERR_CUDA;
            ++*launches;
            i += 2;
            continue;
        }
        const uint8_t *ops = plan.tc_offset.size() == plan.passes.size() && plan.tc_offset[i] >= 0
                                 ? d_ops + plan.tc_offset[i]
                                 : nullptr;
        if (launch_plan_pass(psi, n, p, ops, d_err, stream, tf32) != RCS_OK) return RCS_ERR_CUDA;
        ++*launches;
        ++i;
    }
    return RCS_OK;
}

BitMap plan_to_stored(const Plan &plan) {
    BitMap m = identity_map(plan.n);
    if (plan.phys_of.empty()) return m;
    m.identity = 0;
    for (int q = 0; q < plan.n; ++q) m.to[q] = uint8_t(plan.phys_of[q]);
    return m;
}

int device_sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!dev_sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        dev_sms[dev] = v > 0 ? v : 148;
    }
    return dev_sms[dev];
}
}  // namespace rcs

#define RCS_TRY(ctx) try {
#define RCS_CATCH(ctx)                                                         \
    }                                                                          \
    catch (const std::bad_alloc &) {                                           \
        return fail(ctx, RCS_ERR_OOM, "host allocation failed");                \
    }                                                                          \
    catch (const std::exception &ex) {                                         \
        return fail(ctx, RCS_ERR_ARG, std::string("internal error: ") + ex.what()); \
    }

extern "C" {

const char *rcs_last_error(const rcs_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int rcs_num_qubits(const rcs_ctx *ctx) { return ctx ? ctx->n : -1; }

void rcs_destroy(rcs_ctx *c) {
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->psi);
    cudaFree(c->bsum);
    cudaFree(c->bpre);
    cudaFree(c->chunk);
    cudaFree(c->total);
    cudaFree(c->d_err);
    cudaFree(c->d_u64);
    cudaFree(c->d_f64);
    cudaFree(c->d_order);
    cudaFree(c->d_ops);
    cudaFree(c->d_sub);
    if (c->ev_full[0]) cudaEventDestroy(c->ev_full[0]);
    if (c->ev_full[1]) cudaEventDestroy(c->ev_full[1]);
    cudaSetDevice(prev);
    delete c;
}

int rcs_create(const rcs_grid *grid, const rcs_opts *opts, rcs_ctx **out) {
    RCS_TRY(nullptr)
    if (!grid || !out) return fail(nullptr, RCS_ERR_ARG, "null argument");
    *out = nullptr;
    if (grid->rows <= 0 || grid->cols <= 0 || grid->n_removed < 0 || (grid->n_removed && !grid->removed))
        return fail(nullptr, RCS_ERR_ARG, "bad grid");
    const int64_t cells = int64_t(grid->rows) * grid->cols;
    std::vector<char> gone(size_t(std::min<int64_t>(cells, 1 << 20)), 0);
    if (cells > (1 << 20)) return fail(nullptr, RCS_ERR_ARG, "grid too large");
    for (int i = 0; i < grid->n_removed; ++i) {
        int id = grid->removed[i];
        if (id < 0 || id >= cells || gone[id]) return fail(nullptr, RCS_ERR_ARG, "bad removed cell id");
        gone[id] = 1;
    }
    const int64_t n = cells - grid->n_removed;
    if (n < 1 || n > kMaxQubits) return fail(nullptr, RCS_ERR_ARG, "qubit count must be 1..34");
    rcs_opts o{};
    o.precision = RCS_PREC_FP32_FUSED;
    o.k_max = 4;
    if (opts) o = *opts;
    if (o.precision < RCS_PREC_FP32_PLAIN || o.precision > RCS_PREC_TF32X3)
        return fail(nullptr, RCS_ERR_ARG, "unknown precision");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, RCS_ERR_UNSUPPORTED, std::string("no CUDA device: ") + cudaGetErrorString(e));
    auto *c = new rcs_ctx;
    c->n = int(n);
    c->opts = o;
    c->stream = reinterpret_cast<cudaStream_t>(o.stream);
    cudaGetDevice(&c->dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->dev) == cudaSuccess && prop.major < 10) {
        delete c;
        return fail(nullptr, RCS_ERR_UNSUPPORTED, "device is not a Blackwell (sm_10x) GPU");
    }
    const size_t amps = size_t(1) << n;
    const int bl = std::min(c->n, kSampleBlockLog2);
    const size_t nblocks = size_t(1) << (n - bl);
    auto alloc = [&](void **p, size_t bytes, const char *what) -> int {
        cudaError_t ee = cudaMalloc(p, bytes);
        if (ee != cudaSuccess) {
            cudaGetLastError();
            std::string msg = std::string(what) + ": " + cudaGetErrorString(ee);
            rcs_destroy(c);
            return fail(nullptr, ee == cudaErrorMemoryAllocation ? RCS_ERR_OOM : RCS_ERR_CUDA, msg);
        }
        return RCS_OK;
    };
    int rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->psi), amps * sizeof(float2), "state allocation")) != RCS_OK) return rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->bsum), nblocks * 8, "block sums")) != RCS_OK) return rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->bpre), nblocks * 8, "block prefix")) != RCS_OK) return rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->chunk), (scan_chunks(c->n) + 1) * 8, "scan chunks")) != RCS_OK)
        return rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->total), 8, "total")) != RCS_OK) return rc;
    if ((rc = alloc(reinterpret_cast<void **>(&c->d_err), sizeof(int), "error word")) != RCS_OK) return rc;
    if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess || cudaEventCreate(&c->ev_full[0]) != cudaSuccess ||
        cudaEventCreate(&c->ev_full[1]) != cudaSuccess) {
        std::string msg = std::string("initialisation: ") + cudaGetErrorString(cudaGetLastError());
        rcs_destroy(c);
        return fail(nullptr, RCS_ERR_CUDA, msg);
    }
    c->zero_pending = true;  // |0...0>, written on first use
    set_identity_layout(c);
    c->fresh = true;
    *out = c;
    return RCS_OK;
    RCS_CATCH(nullptr)
}

int rcs_set_stream(rcs_ctx *c, uint64_t stream) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->opts.stream = stream;
    return RCS_OK;
}

int rcs_reset(rcs_ctx *c) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    c->sums_valid = false;
    c->zero_pending = true;  // written by the next run from |0...0>, or on first other use
    set_identity_layout(c);  // |0...0> is the same in every layout
    c->fresh = true;
    return RCS_OK;
}

int rcs_sync(rcs_ctx *c) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    return drain_errors(c);
}

int rcs_apply_circuit(rcs_ctx *c, const rcs_gate *gates, size_t n_gates) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    RCS_TRY(c)
    std::vector<HostGate> hg;
    int rc = valid_gates(c, c->n, gates, n_gates, &hg);
    if (rc != RCS_OK) return rc;
    Plan plan;
    rcs_opts o = c->opts;
    if (o.precision == RCS_PREC_FP32_FUSED && o.autotune && c->n >= 2) {
        int k = 4;
        if ((rc = materialize(c)) != RCS_OK) return rc;
        if ((rc = autotune_fused_k(c, hg, &k)) != RCS_OK) return rc;
        o.k_max = k;
    }
    // a fresh state may take a new layout; otherwise the circuit follows the current one
    const bool fresh = c->fresh;
    if (!fresh && !layout_identity(c))
        for (HostGate &g : hg)
            for (int a = 0; a < g.nq; ++a) g.q[a] = c->phys_of[g.q[a]];
    if ((rc = build_plan(c, c->n, hg, o, &plan, fresh)) != RCS_OK) return rc;
    std::vector<uint8_t> img;
    build_ops_images(plan, &img);
    if (!img.empty()) {
        if (img.size() > c->ops_cap) {
            RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
            cudaFree(c->d_ops);
            c->d_ops = nullptr;
            c->ops_cap = 0;
            RCS_CUDA(c, cudaMalloc(&c->d_ops, img.size()), "cudaMalloc operand images");
            c->ops_cap = img.size();
        }
        // pageable source: the call returns once the bytes are staged, ordered on the stream
        RCS_CUDA(c, cudaMemcpyAsync(c->d_ops, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream),
                 "upload operand images");
    }
    if (fresh) {
        set_identity_layout(c);
        for (size_t q = 0; q < plan.phys_of.size(); ++q) c->phys_of[q] = plan.phys_of[q];
    }
    c->fresh = false;
    return run_passes(c, plan, c->d_ops, fresh);
    RCS_CATCH(c)
}

namespace {
// One caller unitary as a pass on the context's stored qubits: validated (targets,
// unitarity to 1e-6), reordered to ascending targets, and given the kernel kind.
int unitary_pass(rcs_ctx *c, int k, const int32_t *targets, const double *u_re_im, Pass *out) {
    if (k < 1 || k > kSimtKMax || !targets || !u_re_im) return fail(c, RCS_ERR_ARG, "k must be 1..7 with targets and u");
    if (k > c->n) return fail(c, RCS_ERR_QUBIT, "more targets than qubits");
    uint64_t seen = 0;
    for (int i = 0; i < k; ++i) {
        if (targets[i] < 0 || targets[i] >= c->n || ((seen >> targets[i]) & 1))
            return fail(c, RCS_ERR_QUBIT, "bad or repeated target");
        seen |= 1ull << targets[i];
    }
    int tg[8];
    for (int i = 0; i < k; ++i) tg[i] = c->phys_of[targets[i]];  // stored positions
    const int d = 1 << k;
    std::vector<cd> U(size_t(d) * d);
    for (size_t e = 0; e < U.size(); ++e) U[e] = cd(u_re_im[2 * e], u_re_im[2 * e + 1]);
    double worst = 0.0;
    for (int r = 0; r < d; ++r)
        for (int cc = 0; cc < d; ++cc) {
            cd s = 0.0;
            for (int l = 0; l < d; ++l) s += U[size_t(r) * d + l] * std::conj(U[size_t(cc) * d + l]);
            worst = std::max(worst, std::abs(s - (r == cc ? 1.0 : 0.0)));
        }
    if (!(worst <= 1e-6)) return fail(c, RCS_ERR_ARG, "matrix is not unitary to 1e-6");
    // reorder to ascending targets: local bit i (tg[i]) moves to its rank
    int order[8], rank[8];
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order, order + k, [&](int x, int y) { return tg[x] < tg[y]; });
    for (int p = 0; p < k; ++p) rank[order[p]] = p;
    auto remap = [&](int j) {
        int r = 0;
        for (int i = 0; i < k; ++i)
            if ((j >> i) & 1) r |= 1 << rank[i];
        return r;
    };
    Pass &p = *out;
    p.k = k;
    for (int i = 0; i < 8; ++i) p.t[i] = i < k ? tg[order[i]] : -1;
    p.U.assign(U.size(), cd(0.0));
    for (int j = 0; j < d; ++j)
        for (int l = 0; l < d; ++l) p.U[size_t(remap(j)) * d + remap(l)] = U[size_t(j) * d + l];
    const bool tc_prec = c->opts.precision == RCS_PREC_BF16X3 || c->opts.precision == RCS_PREC_TF32X3;
    p.kind = k == kTcK && tc_prec && c->n >= kTcK + 7 ? PASS_TC : PASS_SIMT;
    return RCS_OK;
}
}  // namespace

int rcs_tc_test_fault(int64_t skip_tile, double wait_limit_s) {
    if (skip_tile > (int64_t(1) << 30)) return fail(nullptr, RCS_ERR_ARG, "skip_tile out of range");
    long long cycles = 0;
    if (wait_limit_s > 0) {
        if (!(wait_limit_s <= 100.0)) return fail(nullptr, RCS_ERR_ARG, "wait limit must be at most 100 s");
        int dev = 0, khz = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
            khz <= 0)
            khz = 2070000;  // the GB300 maximum SM clock
        cycles = std::max(1000ll, (long long)(wait_limit_s * double(khz) * 1e3));
    }
    tc_set_test_fault(skip_tile < 0 ? -1 : int(skip_tile), cycles);
    return RCS_OK;
}

int rcs_apply_unitary(rcs_ctx *c, int k, const int32_t *targets, const double *u_re_im) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    const double *u[1] = {u_re_im};
    return rcs_apply_unitaries(c, 1, &k, targets, u);
}

int rcs_apply_unitaries(rcs_ctx *c, size_t count, const int32_t *k, const int32_t *targets,
                        const double *const *u_re_im) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    RCS_TRY(c)
    if (count == 0) return RCS_OK;
    if (!k || !targets || !u_re_im) return fail(c, RCS_ERR_ARG, "null argument");
    if (c->fresh) set_identity_layout(c);
    Plan plan;
    plan.n = c->n;
    plan.precision = c->opts.precision;
    plan.pairs = c->opts.precision == RCS_PREC_BF16X3 && (c->opts.flags & RCS_OPT_PAIR_PASSES);
    plan.n_gates = int64_t(count);
    plan.passes.resize(count);
    size_t off = 0;
    for (size_t i = 0; i < count; ++i) {
        if (k[i] < 1 || k[i] > kSimtKMax) return fail(c, RCS_ERR_ARG, "k must be 1..7 with targets and u");
        if (int rc = unitary_pass(c, k[i], targets + off, u_re_im[i], &plan.passes[i]); rc != RCS_OK) return rc;
        off += size_t(k[i]);
    }
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    std::vector<uint8_t> img;
    build_ops_images(plan, &img);
    if (!img.empty()) {
        if (img.size() > c->ops_cap) {
            RCS_CUDA(c, cudaStreamSynchronize(c->stream), "stream sync");
            cudaFree(c->d_ops);
            c->d_ops = nullptr;
            c->ops_cap = 0;
            RCS_CUDA(c, cudaMalloc(&c->d_ops, img.size()), "cudaMalloc operand images");
            c->ops_cap = img.size();
        }
        RCS_CUDA(c, cudaMemcpyAsync(c->d_ops, img.data(), img.size(), cudaMemcpyHostToDevice, c->stream),
                 "upload operand images");
    }
    c->fresh = false;
    return run_passes(c, plan, c->d_ops, false);
    RCS_CATCH(c)
}

int rcs_plan_build(int n, const rcs_gate *gates, size_t n_gates, const rcs_opts *opts, rcs_plan **out) {
    RCS_TRY(nullptr)
    if (!out) return fail(nullptr, RCS_ERR_ARG, "null output");
    *out = nullptr;
    if (n < 1 || n > kMaxQubits) return fail(nullptr, RCS_ERR_ARG, "qubit count must be 1..34");
    rcs_opts o{};
    o.precision = RCS_PREC_FP32_FUSED;
    o.k_max = 4;
    if (opts) o = *opts;
    std::vector<HostGate> hg;
    int rc = valid_gates(nullptr, n, gates, n_gates, &hg);
    if (rc != RCS_OK) return rc;
    auto *p = new rcs_plan;
    rc = build_plan(nullptr, n, hg, o, &p->p, true);
    if (rc != RCS_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return RCS_OK;
    RCS_CATCH(nullptr)
}

int rcs_plan_info(const rcs_plan *plan, rcs_plan_stats *out) {
    if (!plan || !out) return fail(nullptr, RCS_ERR_ARG, "null argument");
    const Plan &p = plan->p;
    std::memset(out, 0, sizeof(*out));
    out->n_qubits = p.n;
    out->precision = p.precision;
    out->n_gates = p.n_gates;
    out->n_passes = int64_t(p.passes.size());
    const double amps = double(uint64_t(1) << p.n);
    int kmax = 0;
    for (const Pass &q : p.passes) {
        kmax = std::max(kmax, q.k);
        const double mult = q.kind == PASS_TC ? 3.0 : 1.0;
        out->flops += mult * 8.0 * double(1 << q.k) * amps;
    }
    out->k_max = kmax;
    out->hbm_bytes = 16.0 * amps * double(p.passes.size());
    std::vector<SubStage> stages;
    out->prefix_passes = plan_stages(p, &stages);
    out->prefix_qubits = stages.empty() ? 0 : std::popcount(stages.back().tmask);
    out->prefix_stages = int32_t(stages.size());
    // round trips of passes [first, end) on a 2^m state, counting the two-unitary ones
    int32_t pairs = 0;
    auto trips = [&](size_t first, size_t end, int m) {
        double t = 0;
        for (size_t i = first; i < end; ++t) {
            if (plan_pairs_at(p, i, end, m)) {
                ++pairs;
                i += 2;
            } else {
                ++i;
            }
        }
        return t;
    };
    // what run_substages and the passes after it move, from |0...0>
    if (stages.empty()) {
        // zero fill, then every round trip on the full state
        out->zero_hbm_bytes = 8.0 * amps + 16.0 * amps * trips(0, p.passes.size(), p.n);
    } else {
        double z = 8.0 * std::ldexp(1.0, std::popcount(stages.front().tmask));  // first sub-state's zero fill
        for (size_t si = 0; si < stages.size(); ++si) {
            const int mb = std::popcount(stages[si].tmask);
            const double m = std::ldexp(1.0, mb);
            z += 16.0 * m * trips(size_t(stages[si].first), size_t(stages[si].first + stages[si].count), mb);
            if (si + 1 < stages.size()) z += 8.0 * m + 8.0 * std::ldexp(1.0, std::popcount(stages[si + 1].tmask));
        }
        // the last sub-state is read once into the full state: by the first full pass itself or by an
        // expansion before it; either way 8 * 2^m in and 8 * 2^n out, plus 16 * 2^n per other round trip
        const size_t after = size_t(out->prefix_passes);
        const double mlast = std::ldexp(1.0, std::popcount(stages.back().tmask));
        const bool fused = after < p.passes.size() && tc_pass_takes_substate(p.passes[after], p.n);
        z += 8.0 * mlast + 8.0 * amps;
        z += 16.0 * amps * trips(after + (fused ? 1 : 0), p.passes.size(), p.n);
        out->zero_hbm_bytes = z;
    }
    out->pair_passes = pairs;
    return RCS_OK;
}

int rcs_last_pass_timing(rcs_ctx *c, float *ms, int64_t *full_passes) {
    if (!c || !ms || !full_passes) return fail(c, RCS_ERR_ARG, "null argument");
    if (c->timed_passes < 0) return fail(c, RCS_ERR_ARG, "no circuit has run on this context");
    RCS_CUDA(c, cudaEventSynchronize(c->ev_full[1]), "event sync");
    RCS_CUDA(c, cudaEventElapsedTime(ms, c->ev_full[0], c->ev_full[1]), "event time");
    *full_passes = c->timed_passes;
    return RCS_OK;
}

int rcs_plan_pass(const rcs_plan *plan, size_t i, int32_t *k, int32_t *targets, double *u_re_im) {
    if (!plan || !k || !targets) return fail(nullptr, RCS_ERR_ARG, "null argument");
    if (i >= plan->p.passes.size()) return fail(nullptr, RCS_ERR_ARG, "pass index out of range");
    const Pass &p = plan->p.passes[i];
    *k = p.k;
    for (int j = 0; j < 8; ++j) targets[j] = j < p.k ? p.t[j] : -1;
    if (u_re_im)
        for (size_t e = 0; e < p.U.size(); ++e) {
            u_re_im[2 * e] = p.U[e].real();
            u_re_im[2 * e + 1] = p.U[e].imag();
        }
    return RCS_OK;
}

int rcs_plan_upload(rcs_ctx *c, rcs_plan *plan) {
    if (!c || !plan) return fail(c, RCS_ERR_ARG, "null argument");
    RCS_TRY(c)
    if (plan->p.n != c->n) return fail(c, RCS_ERR_ARG, "plan was built for another qubit count");
    if (plan->d_ops_dev == c->dev) return RCS_OK;
    std::vector<uint8_t> img;
    build_ops_images(plan->p, &img);
    if (plan->d_ops) cudaFree(plan->d_ops);
    plan->d_ops = nullptr;
    if (!img.empty()) {
        RCS_CUDA(c, cudaMalloc(&plan->d_ops, img.size()), "cudaMalloc plan operands");
        RCS_CUDA(c, cudaMemcpy(plan->d_ops, img.data(), img.size(), cudaMemcpyHostToDevice), "upload plan operands");
    }
    plan->d_ops_dev = c->dev;
    return RCS_OK;
    RCS_CATCH(c)
}

int rcs_plan_run(rcs_ctx *c, rcs_plan *plan) {
    if (!c || !plan) return fail(c, RCS_ERR_ARG, "null argument");
    if (plan->p.n != c->n) return fail(c, RCS_ERR_ARG, "plan was built for another qubit count");
    if (plan->d_ops_dev != c->dev) {
        int rc = rcs_plan_upload(c, plan);
        if (rc != RCS_OK) return rc;
    }
    // a plan is built for a fresh state in its own layout
    if (!plan->p.phys_of.empty()) {
        if (!c->fresh)
            return fail(c, RCS_ERR_ARG, "this plan stores the circuit in its own qubit layout and needs a fresh "
                                        "state (rcs_create or rcs_reset first)");
        set_identity_layout(c);
        for (size_t q = 0; q < plan->p.phys_of.size(); ++q) c->phys_of[q] = plan->p.phys_of[q];
    } else if (!layout_identity(c)) {
        if (c->fresh) set_identity_layout(c);
        else if (int rc = restore_layout(c); rc != RCS_OK) return rc;
    }
    const bool fresh = c->fresh;
    c->fresh = false;
    return run_passes(c, plan->p, plan->d_ops, fresh);
}

void rcs_plan_destroy(rcs_plan *plan) {
    if (!plan) return;
    if (plan->d_ops) cudaFree(plan->d_ops);
    delete plan;
}

int rcs_qubit_layout(const rcs_ctx *c, int32_t *phys_of) {
    if (!c || !phys_of) return fail(nullptr, RCS_ERR_ARG, "null argument");
    for (int q = 0; q < c->n; ++q) phys_of[q] = c->phys_of[q];
    return RCS_OK;
}

int rcs_plan_layout(const rcs_plan *plan, int32_t *phys_of) {
    if (!plan || !phys_of) return fail(nullptr, RCS_ERR_ARG, "null argument");
    for (int q = 0; q < plan->p.n; ++q)
        phys_of[q] = plan->p.phys_of.empty() ? q : plan->p.phys_of[size_t(q)];
    return RCS_OK;
}

int rcs_amplitudes(rcs_ctx *c, const uint64_t *bits, size_t n, double *out_re_im) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (n == 0) return RCS_OK;
    if (!bits || !out_re_im) return fail(c, RCS_ERR_ARG, "null argument");
    const uint64_t lim = uint64_t(1) << c->n;
    for (size_t i = 0; i < n; ++i)
        if (bits[i] >= lim) return fail(c, RCS_ERR_ARG, "bitstring index >= 2^n");
    int rc;
    if ((rc = materialize(c)) != RCS_OK) return rc;
    if ((rc = ensure_u64(c, n)) != RCS_OK || (rc = ensure_f64(c, 2 * n)) != RCS_OK) return rc;
    RCS_CUDA(c, cudaMemcpyAsync(c->d_u64, bits, n * 8, cudaMemcpyHostToDevice, c->stream), "upload bitstrings");
    if (launch_gather(c->psi, c->n, c->d_u64, n, c->d_f64, c->d_err, to_stored(c), c->stream) != RCS_OK)
        return fail(c, RCS_ERR_CUDA, "gather launch: " + take_launch_error());
    RCS_CUDA(c, cudaMemcpyAsync(out_re_im, c->d_f64, n * 16, cudaMemcpyDeviceToHost, c->stream), "download");
    return drain_errors(c);
}

int rcs_state_read(rcs_ctx *c, uint64_t first, uint64_t count, float *out_re_im) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    const uint64_t lim = uint64_t(1) << c->n;
    if (first > lim || count > lim - first || (count && !out_re_im)) return fail(c, RCS_ERR_ARG, "bad range");
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    if (!layout_identity(c)) {
        if (int rc = restore_layout(c); rc != RCS_OK) return rc;
    }
    if (count)
        RCS_CUDA(c, cudaMemcpyAsync(out_re_im, c->psi + first, count * 8, cudaMemcpyDeviceToHost, c->stream),
                 "read state");
    return drain_errors(c);
}

int rcs_state_write(rcs_ctx *c, uint64_t first, uint64_t count, const float *in_re_im) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    const uint64_t lim = uint64_t(1) << c->n;
    if (first > lim || count > lim - first || (count && !in_re_im)) return fail(c, RCS_ERR_ARG, "bad range");
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    if (!layout_identity(c)) {
        if (int rc = restore_layout(c); rc != RCS_OK) return rc;
    }
    c->fresh = false;
    if (count)
        RCS_CUDA(c, cudaMemcpyAsync(c->psi + first, in_re_im, count * 8, cudaMemcpyHostToDevice, c->stream),
                 "write state");
    c->sums_valid = false;
    return drain_errors(c);
}

namespace {
// File form of a saved state: this header, then the 2^n stored amplitudes (complex64,
// interleaved, little-endian) in stored order.
struct StateFileHeader {
    char magic[8];       // "RCSSTATE"
    uint32_t version;    // 1
    int32_t n;
    int32_t phys_of[64];  // stored bit of each circuit qubit (the layout)
    uint64_t amplitudes;  // 2^n
};
static_assert(sizeof(StateFileHeader) == 280, "state file header layout");
constexpr size_t kIoChunk = size_t(64) << 20;  // bytes per copy through the pinned buffer

struct PinnedBuffer {
    void *p = nullptr;
    ~PinnedBuffer() {
        if (p) cudaFreeHost(p);
    }
};
}  // namespace

int rcs_state_save(rcs_ctx *c, const char *path) {
    if (!c || !path) return fail(c, RCS_ERR_ARG, "null argument");
    RCS_TRY(c)
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    StateFileHeader h{};
    std::memcpy(h.magic, "RCSSTATE", 8);
    h.version = 1;
    h.n = c->n;
    for (int q = 0; q < 64; ++q) h.phys_of[q] = q < c->n ? c->phys_of[q] : q;
    h.amplitudes = uint64_t(1) << c->n;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, RCS_ERR_ARG, std::string("cannot open for writing: ") + path);
    PinnedBuffer buf;
    const size_t total = size_t(8) << c->n;
    const size_t chunk = std::min(total, kIoChunk);
    int rc = RCS_OK;
    if (std::fwrite(&h, sizeof(h), 1, f) != 1) rc = fail(c, RCS_ERR_ARG, "short write of the state header");
    if (rc == RCS_OK && cudaHostAlloc(&buf.p, chunk, cudaHostAllocDefault) != cudaSuccess)
        rc = fail(c, RCS_ERR_OOM, "pinned staging buffer");
    for (size_t off = 0; rc == RCS_OK && off < total; off += chunk) {
        const size_t len = std::min(chunk, total - off);
        if (cudaMemcpyAsync(buf.p, reinterpret_cast<const uint8_t *>(c->psi) + off, len, cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = fail(c, RCS_ERR_CUDA, "state download");
        else if (std::fwrite(buf.p, 1, len, f) != len)
            rc = fail(c, RCS_ERR_ARG, std::string("short write: ") + path);
    }
    if (std::fclose(f) != 0 && rc == RCS_OK) rc = fail(c, RCS_ERR_ARG, std::string("close failed: ") + path);
    if (rc != RCS_OK) return rc;
    return drain_errors(c);
    RCS_CATCH(c)
}

int rcs_state_load(rcs_ctx *c, const char *path) {
    if (!c || !path) return fail(c, RCS_ERR_ARG, "null argument");
    RCS_TRY(c)
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, RCS_ERR_ARG, std::string("cannot open: ") + path);
    StateFileHeader h{};
    int rc = RCS_OK;
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "RCSSTATE", 8) != 0 || h.version != 1)
        rc = fail(c, RCS_ERR_ARG, std::string("not a saved state (version 1): ") + path);
    else if (h.n != c->n || h.amplitudes != (uint64_t(1) << c->n))
        rc = fail(c, RCS_ERR_ARG, "the saved state has " + std::to_string(h.n) + " qubits, the context " +
                                      std::to_string(c->n));
    if (rc == RCS_OK) {  // the layout must be a permutation of 0..n-1
        uint64_t seen = 0;
        for (int q = 0; q < c->n; ++q) {
            const int p = h.phys_of[q];
            if (p < 0 || p >= c->n || ((seen >> p) & 1)) {
                rc = fail(c, RCS_ERR_ARG, "corrupt layout in the state header");
                break;
            }
            seen |= 1ull << p;
        }
    }
    PinnedBuffer buf;
    const size_t total = size_t(8) << c->n;
    const size_t chunk = std::min(total, kIoChunk);
    if (rc == RCS_OK && cudaHostAlloc(&buf.p, chunk, cudaHostAllocDefault) != cudaSuccess)
        rc = fail(c, RCS_ERR_OOM, "pinned staging buffer");
    if (rc == RCS_OK) {  // the state is being replaced: anything pending on it is dropped
        c->zero_pending = false;
        c->fresh = false;
        c->sums_valid = false;
    }
    for (size_t off = 0; rc == RCS_OK && off < total; off += chunk) {
        const size_t len = std::min(chunk, total - off);
        if (std::fread(buf.p, 1, len, f) != len) {
            rc = fail(c, RCS_ERR_ARG, std::string("truncated state file: ") + path);
        } else if (cudaMemcpyAsync(reinterpret_cast<uint8_t *>(c->psi) + off, buf.p, len, cudaMemcpyHostToDevice,
                                   c->stream) != cudaSuccess ||
                   cudaStreamSynchronize(c->stream) != cudaSuccess) {
            rc = fail(c, RCS_ERR_CUDA, "state upload");
        }
    }
    std::fclose(f);
    if (rc != RCS_OK) return rc;
    for (int q = 0; q < c->n; ++q) c->phys_of[q] = h.phys_of[q];
    return drain_errors(c);
    RCS_CATCH(c)
}

int rcs_state_device(rcs_ctx *c, void **d_state) {
    if (!c || !d_state) return fail(c, RCS_ERR_ARG, "null argument");
    if (int rc = materialize(c); rc != RCS_OK) return rc;
    if (!layout_identity(c)) {
        if (int rc = restore_layout(c); rc != RCS_OK) return rc;
    }
    *d_state = c->psi;
    c->fresh = false;
    c->sums_valid = false;  // the caller may write through the pointer
    return RCS_OK;
}

int rcs_norm(rcs_ctx *c, double *out) {
    if (!c || !out) return fail(c, RCS_ERR_ARG, "null argument");
    int rc = ensure_sums(c);
    if (rc != RCS_OK) return rc;
    uint64_t t = 0;
    RCS_CUDA(c, cudaMemcpyAsync(&t, c->total, 8, cudaMemcpyDeviceToHost, c->stream), "download total");
    if ((rc = drain_errors(c)) != RCS_OK) {
        c->sums_valid = false;
        return rc;
    }
    *out = std::ldexp(double(t), -62);
    return RCS_OK;
}

int rcs_sample_device(rcs_ctx *c, uint64_t shots, uint64_t seed, uint64_t *d_out_bits) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (shots == 0) return RCS_OK;
    if (!d_out_bits) return fail(c, RCS_ERR_ARG, "null output");
    int rc = ensure_sums(c);
    if (rc != RCS_OK) return rc;
    if ((rc = ensure_order(c, size_t(shots))) != RCS_OK) return rc;
    // the block sums are spent as the sampler's per-block counts (the prefix and T stay)
    if (launch_sample(c->psi, c->n, c->bsum, c->bpre, c->total, c->chunk, 0, shots, seed, d_out_bits, c->d_order,
                      c->d_err, to_stored(c), c->stream) != RCS_OK)
        return fail(c, RCS_ERR_CUDA, "sampler launch: " + take_launch_error());
    return RCS_OK;
}

int rcs_sample_range(rcs_ctx *c, uint64_t first_shot, uint64_t shots, uint64_t seed, uint64_t *out_bits) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (shots == 0) return RCS_OK;
    if (!out_bits) return fail(c, RCS_ERR_ARG, "null output");
    if (first_shot > ~0ull - shots) return fail(c, RCS_ERR_ARG, "shot range overflows");
    int rc = ensure_sums(c);
    if (rc != RCS_OK) return rc;
    if ((rc = ensure_u64(c, size_t(shots))) != RCS_OK || (rc = ensure_order(c, size_t(shots))) != RCS_OK) return rc;
    if (launch_sample(c->psi, c->n, c->bsum, c->bpre, c->total, c->chunk, first_shot, shots, seed, c->d_u64,
                      c->d_order, c->d_err, to_stored(c), c->stream) != RCS_OK)
        return fail(c, RCS_ERR_CUDA, "sampler launch: " + take_launch_error());
    RCS_CUDA(c, cudaMemcpyAsync(out_bits, c->d_u64, shots * 8, cudaMemcpyDeviceToHost, c->stream), "download samples");
    if ((rc = drain_errors(c)) != RCS_OK) {
        c->sums_valid = false;
        return rc;
    }
    return RCS_OK;
}

int rcs_sample(rcs_ctx *c, uint64_t shots, uint64_t seed, uint64_t *out_bits) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (shots == 0) return RCS_OK;
    if (!out_bits) return fail(c, RCS_ERR_ARG, "null output");
    int rc = ensure_u64(c, size_t(shots));
    if (rc != RCS_OK) return rc;
    if ((rc = rcs_sample_device(c, shots, seed, c->d_u64)) != RCS_OK) return rc;
    RCS_CUDA(c, cudaMemcpyAsync(out_bits, c->d_u64, shots * 8, cudaMemcpyDeviceToHost, c->stream), "download samples");
    if ((rc = drain_errors(c)) != RCS_OK) {
        c->sums_valid = false;
        return rc;
    }
    return RCS_OK;
}

int rcs_xeb_device(rcs_ctx *c, const uint64_t *d_samples, size_t n, double *d_out_xeb) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (n == 0 || !d_samples || !d_out_xeb) return fail(c, RCS_ERR_ARG, "need samples and an output");
    int rc = ensure_sums(c);
    if (rc != RCS_OK) return rc;
    if ((rc = ensure_f64(c, xeb_partials_count(n) + 2)) != RCS_OK) return rc;
    if (launch_xeb(c->psi, c->n, d_samples, n, c->total, c->d_f64, d_out_xeb, to_stored(c), c->stream) != RCS_OK)
        return fail(c, RCS_ERR_CUDA, "xeb launch: " + take_launch_error());
    return RCS_OK;
}

int rcs_xeb(rcs_ctx *c, const uint64_t *samples, size_t n, double *out_xeb) {
    if (!c) return fail(nullptr, RCS_ERR_ARG, "null context");
    if (n == 0 || !samples || !out_xeb) return fail(c, RCS_ERR_ARG, "need samples and an output");
    const uint64_t lim = uint64_t(1) << c->n;
    for (size_t i = 0; i < n; ++i)
        if (samples[i] >= lim) return fail(c, RCS_ERR_ARG, "sample index >= 2^n");
    int rc = ensure_u64(c, n + 1);
    if (rc != RCS_OK) return rc;
    if ((rc = ensure_f64(c, xeb_partials_count(n) + 2)) != RCS_OK) return rc;
    RCS_CUDA(c, cudaMemcpyAsync(c->d_u64, samples, n * 8, cudaMemcpyHostToDevice, c->stream), "upload samples");
    if ((rc = ensure_sums(c)) != RCS_OK) return rc;
    double *d_res = c->d_f64 + xeb_partials_count(n);
    if (launch_xeb(c->psi, c->n, c->d_u64, n, c->total, c->d_f64, d_res, to_stored(c), c->stream) != RCS_OK)
        return fail(c, RCS_ERR_CUDA, "xeb launch: " + take_launch_error());
    RCS_CUDA(c, cudaMemcpyAsync(out_xeb, d_res, 8, cudaMemcpyDeviceToHost, c->stream), "download xeb");
    return drain_errors(c);
}

}  // extern "C"
