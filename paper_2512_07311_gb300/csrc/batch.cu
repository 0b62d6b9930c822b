// Batched mode: many independent circuits, of different qubit counts and depths,
// in one persistent kernel launch inside one captured CUDA graph, with the fusion
// width and work-item size chosen by timed trials.
//
// Work items. Each circuit i is planned (FP32 fused, k <= 5) into passes; each pass
// is cut into items of a few thousand slices. The host lays the items out in rounds
// -- round r holds pass r of every circuit that has one -- so every item of pass p
// of circuit i is handed out before any item of its pass p+1. A CTA takes the next
// item from a global counter, waits until circuit i has finished all items of its
// earlier passes (a per-circuit completion counter), applies the pass to its slices
// and adds one to the counter. Items of other circuits fill the gaps, and a wait can
// only be on items already handed to running CTAs, which never wait on later
// items: with every CTA resident (a cooperative launch) the schedule cannot
// deadlock. Waits are bounded: past the limit the kernel raises an error bit, sets
// an abort flag that makes every CTA stop taking work, and returns.
//
// Memory coherence: the state is read with ld.global.cg and written with
// st.global.cg (L2, never a stale L1 line from an earlier pass); a CTA publishes
// its stores with a fence before its counter increment, and a waiting CTA fences
// after seeing the count.
//
// Tensor-core engine (precision BF16X3 or TF32X3). Each circuit is planned like a
// single one (fused 6-qubit passes, its own qubit layout and sub-state prefix). Every
// pass of every circuit of 13 or more qubits is then a work item of one cooperative
// launch of the persistent tensor-core kernel (k_batch_tc.cu: tile ranges of one pass,
// ordered by per-circuit completion counters; the sub-state stages' zero fill and
// expansions folded into passes that read a sub-state). The tiles per item are chosen
// at creation by timed launches of that kernel on the batch itself. Circuits it cannot
// run (under 13 qubits, or with no gates) go first as launch chains of their own; after
// the kernel, every circuit's sampler and XEB run on parallel branches of the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <bit>
#include <chrono>
#include <cmath>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"

using namespace rcs;

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kSlicesPerItem = 2048;  // default item: 8 slices per thread
// item sizes the autotuner tries (slices; a multiple of the CTA's threads)
constexpr uint32_t kItemSizes[] = {1024, 2048, 4096, 8192};
constexpr int kMaxK = 5;

struct BInst {
    float2 *psi;
    uint32_t n;
    uint32_t items_per_pass;
    uint32_t slices_per_item;
    uint32_t reserved;
};
struct BPass {
    int32_t k;
    int32_t t[kMaxK];
    uint32_t u_off;  // index of the first float4 entry (re, im, -im, 0) of U, row-major
};
struct BSeg {
    uint64_t first_item;
    uint32_t inst;
    uint32_t pass;  // global index into the pass table
    uint32_t pass_in_inst;
};

struct BArgs {
    const BInst *inst;
    const BPass *pass;
    const float4 *U;
    const BSeg *seg;
    uint32_t nseg;
    const uint32_t *item_seg;  // segment of each item
    uint64_t nitems;
    unsigned long long *next_item;
    unsigned int *done;  // per instance: items completed
    int *err;
    int *abort_flag;
    long long wait_cycles;
    long long skip_item;  // an item whose completion is never published (fault test), or -1
};

// offs: the 2^K target offsets in shared memory, read back through a volatile
// pointer at each use so they are not held in registers across the mat-vec.
template <int K>
__device__ __forceinline__ void apply_items(float2 *__restrict__ psi, const int *t, const float4 *sU,
                                            const volatile uint64_t *offs, uint64_t s_begin, uint64_t s_end) {
    constexpr int D = 1 << K;
#pragma unroll 1
    for (uint64_t s = s_begin + threadIdx.x; s < s_end; s += kThreads) {
        uint64_t base = s;
#pragma unroll
        for (int i = 0; i < K; ++i) base = insert_zero(base, t[i]);
        float2 v[D];
#pragma unroll
        for (int j = 0; j < D; ++j) v[j] = __ldcg(psi + base + offs[j]);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const float4 u = sU[j * D + l];
                acc.x = fmaf(u.x, v[l].x, acc.x);
                acc.x = fmaf(u.z, v[l].y, acc.x);
                acc.y = fmaf(u.x, v[l].y, acc.y);
                acc.y = fmaf(u.y, v[l].x, acc.y);
            }
            __stcg(psi + base + offs[j], acc);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_batch_apply(const __grid_constant__ BArgs a) {
    __shared__ float4 sU[32 * 32];
    __shared__ uint64_t sOff[32];
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_seg;
    __shared__ int s_go, s_reload;
    // thread 0 claims the CTA's next item while the CTA works on the current one: the
    // atomic, the item's segment and a first poll of its circuit's counter are in flight
    // during the work. Items are still taken in claim order, so a wait is only ever on
    // items claimed earlier, which no CTA holds back.
    unsigned long long nxt = 0;
    uint32_t nxt_seg = 0, cur_pass = ~0u;
    bool nxt_ready = false;
    auto claim = [&]() {
        nxt = *(volatile int *)a.abort_flag ? a.nitems : atomicAdd(a.next_item, 1ull);
        nxt_ready = false;
        if (nxt < a.nitems) {
            nxt_seg = a.item_seg[nxt];
            const BSeg sg = a.seg[nxt_seg];
            const unsigned int need = sg.pass_in_inst * a.inst[sg.inst].items_per_pass;
            nxt_ready = *(const volatile unsigned int *)(a.done + sg.inst) >= need;
        }
    };
    if (threadIdx.x == 0) claim();
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = nxt;
            s_go = 0;
            if (nxt < a.nitems) {
                s_seg = nxt_seg;
                const BSeg sg = a.seg[nxt_seg];
                const unsigned int need = sg.pass_in_inst * a.inst[sg.inst].items_per_pass;
                const volatile unsigned int *done = a.done + sg.inst;
                const long long t0 = clock64();
                s_go = 1;
                if (!nxt_ready)
                    while (*done < need) {
                        if (*(volatile int *)a.abort_flag) {
                            s_go = 0;
                            break;
                        }
                        if (clock64() - t0 > a.wait_cycles) {
                            atomicOr(a.err, kErrTimeout);
                            atomicExch(a.abort_flag, 1);
                            s_go = 0;
                            break;
                        }
                        __nanosleep(200);
                    }
                __threadfence();
                s_reload = sg.pass != cur_pass;
                cur_pass = sg.pass;
            }
        }
        __syncthreads();
        if (s_item >= a.nitems) break;
        if (!s_go) {
            if (threadIdx.x == 0) claim();  // sees the abort flag: the loop ends
            __syncthreads();
            continue;
        }
        const BSeg sg = a.seg[s_seg];
        const BInst in = a.inst[sg.inst];
        const BPass ps = a.pass[sg.pass];
        const int D = 1 << ps.k;
        if (s_reload) {  // a new pass: its unitary and target offsets
            for (int e = threadIdx.x; e < D * D; e += kThreads) sU[e] = __ldg(a.U + ps.u_off + e);
            if (threadIdx.x < D) {
                uint64_t o = 0;
                for (int i = 0; i < ps.k; ++i)
                    if ((threadIdx.x >> i) & 1) o |= 1ull << ps.t[i];
                sOff[threadIdx.x] = o;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) claim();
        const uint64_t item_in_pass = s_item - sg.first_item;
        const uint64_t nslices = 1ull << (in.n - ps.k);
        const uint64_t s0 = item_in_pass * in.slices_per_item;
        const uint64_t s1 = s0 + in.slices_per_item < nslices ? s0 + in.slices_per_item : nslices;
        int t[kMaxK];
#pragma unroll
        for (int i = 0; i < kMaxK; ++i) t[i] = ps.t[i];
        switch (ps.k) {
            case 1: apply_items<1>(in.psi, t, sU, sOff, s0, s1); break;
            case 2: apply_items<2>(in.psi, t, sU, sOff, s0, s1); break;
            case 3: apply_items<3>(in.psi, t, sU, sOff, s0, s1); break;
            case 4: apply_items<4>(in.psi, t, sU, sOff, s0, s1); break;
            default: apply_items<5>(in.psi, t, sU, sOff, s0, s1); break;
        }
        __syncthreads();
        if (threadIdx.x == 0 && (long long)s_item != a.skip_item) {
            __threadfence();
            atomicAdd(a.done + sg.inst, 1u);
        }
    }
}

__global__ void k_batch_reset(const BInst *inst, int n_inst) {
    for (int i = blockIdx.y; i < n_inst; i += gridDim.y) {
        float4 *p = reinterpret_cast<float4 *>(inst[i].psi);
        const uint64_t n4 = (1ull << inst[i].n) / 2;
        for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n4; j += uint64_t(gridDim.x) * blockDim.x)
            p[j] = make_float4(j == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
}

struct InstHost {
    int n = 0;
    uint64_t shots = 0, seed = 0;
    int k = 0;
    Plan plan;
    // tensor-core engine: operand images, sub-state prefix, layout maps
    uint8_t *d_ops = nullptr;
    void *d_sub = nullptr;
    int prefix = 0;
    std::vector<SubStage> stages;
    bool persistent = false;  // tensor-core engine: its passes run in the persistent kernel
    float2 *psi = nullptr;
    uint64_t *bsum = nullptr, *bpre = nullptr, *chunk = nullptr, *total = nullptr;
    uint64_t *d_bits = nullptr;  // shots
    uint64_t *d_order = nullptr;  // shots: the sampler's scratch
    double *d_xeb = nullptr;     // result + partials
    uint64_t items_per_pass = 0;
    uint32_t slices_per_item = kSlicesPerItem;  // FP32 engine: the work-item size
};

// ---- autotuner: chosen fusion width per qubit count, by timed trials (cached per device)
std::mutex g_tune_mu;
struct Tuned {
    int k;
    uint32_t slices_per_item;
};
std::map<std::pair<int, int>, Tuned> g_tuned;  // (device, n) -> fusion width and item size

}  // namespace

struct rcs_batch {
    int dev = 0;
    bool tc = false;  // tensor-core engine
    BtcPlan *btc = nullptr;        // tensor-core engine: the persistent kernel's tables
    uint32_t tiles_per_item = 0;   // ... and their chosen item size
    double trial_ms[5] = {0, 0, 0, 0, 0};  // the trials (candidates kTilesPerItem)
    std::vector<InstHost> inst;
    BInst *d_inst = nullptr;
    BPass *d_pass = nullptr;
    float4 *d_U = nullptr;
    BSeg *d_seg = nullptr;
    uint32_t nseg = 0;
    uint32_t *d_item_seg = nullptr;
    uint64_t nitems = 0;
    unsigned long long *d_next = nullptr;
    unsigned int *d_done = nullptr;
    int *d_err = nullptr;  // [0] error bits, [1] abort flag
    long long wait_cycles = 0;
    long long skip_item = -1;
    int grid = 0;
    bool cooperative = true;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    std::string err;
};

namespace {

int bfail(rcs_batch *b, int code, const std::string &m) {
    if (b) b->err = m;
    return set_thread_error(code, m);
}

#define BCUDA(b, call, what)                                                                             \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? RCS_ERR_OOM : RCS_ERR_CUDA,                \
                         std::string(what) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

// Pass table, U entries and segments for the current plans.
void build_tables(const std::vector<InstHost> &inst, std::vector<BPass> *passes, std::vector<float4> *U,
                  std::vector<BSeg> *segs, std::vector<uint32_t> *pass0, uint64_t *nitems) {
    passes->clear();
    U->clear();
    segs->clear();
    pass0->clear();
    for (const InstHost &h : inst) {
        pass0->push_back(uint32_t(passes->size()));
        for (const Pass &p : h.plan.passes) {
            BPass bp{};
            bp.k = p.k;
            for (int i = 0; i < kMaxK; ++i) bp.t[i] = i < p.k ? p.t[i] : 0;
            bp.u_off = uint32_t(U->size());
            for (const cd &u : p.U) U->push_back(make_float4(float(u.real()), float(u.imag()), -float(u.imag()), 0.f));
            passes->push_back(bp);
        }
    }
    size_t maxp = 0;
    for (const InstHost &h : inst) maxp = std::max(maxp, h.plan.passes.size());
    uint64_t item = 0;
    for (size_t r = 0; r < maxp; ++r)
        for (size_t i = 0; i < inst.size(); ++i) {
            if (r >= inst[i].plan.passes.size()) continue;
            BSeg s;
            s.first_item = item;
            s.inst = uint32_t(i);
            s.pass = (*pass0)[i] + uint32_t(r);
            s.pass_in_inst = uint32_t(r);
            segs->push_back(s);
            item += inst[i].items_per_pass;
        }
    *nitems = item;
}

// Segment of every item (items of a segment are consecutive), so the kernel finds an
// item's pass with one load.
std::vector<uint32_t> item_segments(const std::vector<BSeg> &segs, uint64_t nitems) {
    std::vector<uint32_t> out(static_cast<size_t>(nitems));
    for (size_t i = 0; i < segs.size(); ++i) {
        const uint64_t end = i + 1 < segs.size() ? segs[i + 1].first_item : nitems;
        for (uint64_t it = segs[i].first_item; it < end; ++it) out[size_t(it)] = uint32_t(i);
    }
    return out;
}

uint64_t items_per_pass(int n, int k, uint32_t slices_per_item) {
    const uint64_t slices = 1ull << (n - k);
    return (slices + slices_per_item - 1) / slices_per_item;
}

int launch_apply(rcs_batch *b, cudaStream_t st, uint64_t nitems) {
    BArgs a;
    a.inst = b->d_inst;
    a.pass = b->d_pass;
    a.U = b->d_U;
    a.seg = b->d_seg;
    a.nseg = b->nseg;
    a.item_seg = b->d_item_seg;
    a.nitems = nitems;
    a.next_item = b->d_next;
    a.done = b->d_done;
    a.err = b->d_err;
    a.abort_flag = b->d_err + 1;
    a.wait_cycles = b->wait_cycles;
    a.skip_item = b->skip_item;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(b->grid));
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = b->cooperative ? attr : nullptr;
    cfg.numAttrs = b->cooperative ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch_apply, a);
    return e == cudaSuccess ? RCS_OK : note_launch_error("batched apply", e);
}

// Resident CTAs of the persistent kernel: all of them must fit at once.
int persistent_grid() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_apply, kThreads, 0);
    return std::max(1, per_sm) * device_sm_count();
}

// Times `reps` passes of width k on an n-qubit scratch state through the persistent
// kernel (the same code path the batch runs) and returns ms per pass.
double time_trial(int n, int k, uint32_t spi, float2 *scratch, rcs_batch *tmpl) {
    InstHost h;
    h.n = n;
    h.psi = scratch;
    h.plan.n = n;
    const int reps = 3;
    for (int r = 0; r < reps; ++r) {
        Pass p;
        p.kind = PASS_SIMT;
        p.k = k;
        for (int i = 0; i < 8; ++i) p.t[i] = i < k ? (r + i * (n / k)) % n : -1;  // distinct, spread out
        std::sort(p.t, p.t + k);
        const int d = 1 << k;
        p.U.assign(size_t(d) * d, cd(0.0));
        for (int j = 0; j < d; ++j) p.U[size_t(j) * d + ((j + 1) % d)] = cd(0.0, 1.0);  // a permutation: unitary
        h.plan.passes.push_back(p);
    }
    h.items_per_pass = items_per_pass(n, k, spi);
    rcs_batch t;
    t.dev = tmpl->dev;
    t.grid = tmpl->grid;
    t.cooperative = tmpl->cooperative;
    t.wait_cycles = tmpl->wait_cycles;
    std::vector<InstHost> one{h};
    std::vector<BPass> passes;
    std::vector<float4> U;
    std::vector<BSeg> segs;
    std::vector<uint32_t> pass0;
    build_tables(one, &passes, &U, &segs, &pass0, &t.nitems);
    const std::vector<uint32_t> iseg = item_segments(segs, t.nitems);
    BInst bi{scratch, uint32_t(n), uint32_t(h.items_per_pass), spi, 0};
    double ms = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&t.d_inst, sizeof(BInst)) == cudaSuccess && cudaMalloc(&t.d_pass, passes.size() * sizeof(BPass)) == cudaSuccess &&
        cudaMalloc(&t.d_U, U.size() * sizeof(float4)) == cudaSuccess && cudaMalloc(&t.d_seg, segs.size() * sizeof(BSeg)) == cudaSuccess &&
        cudaMalloc(&t.d_item_seg, std::max<size_t>(iseg.size(), 1) * 4) == cudaSuccess &&
        cudaMalloc(&t.d_next, 8) == cudaSuccess && cudaMalloc(&t.d_done, 4) == cudaSuccess && cudaMalloc(&t.d_err, 8) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        t.nseg = uint32_t(segs.size());
        cudaMemcpy(t.d_inst, &bi, sizeof(BInst), cudaMemcpyHostToDevice);
        cudaMemcpy(t.d_pass, passes.data(), passes.size() * sizeof(BPass), cudaMemcpyHostToDevice);
        cudaMemcpy(t.d_U, U.data(), U.size() * sizeof(float4), cudaMemcpyHostToDevice);
        cudaMemcpy(t.d_seg, segs.data(), segs.size() * sizeof(BSeg), cudaMemcpyHostToDevice);
        if (!iseg.empty()) cudaMemcpy(t.d_item_seg, iseg.data(), iseg.size() * 4, cudaMemcpyHostToDevice);
        for (int rep = 0; rep < 2; ++rep) {  // first run warms up
            cudaMemset(t.d_next, 0, 8);
            cudaMemset(t.d_done, 0, 4);
            cudaMemset(t.d_err, 0, 8);
            cudaEventRecord(e0, 0);
            launch_apply(&t, 0, t.nitems);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
        }
        float f = 0.f;
        int herr[2] = {0, 0};
        cudaMemcpy(herr, t.d_err, 8, cudaMemcpyDeviceToHost);
        if (cudaEventElapsedTime(&f, e0, e1) == cudaSuccess && herr[0] == 0) ms = double(f) / reps;
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(t.d_inst);
    cudaFree(t.d_pass);
    cudaFree(t.d_U);
    cudaFree(t.d_seg);
    cudaFree(t.d_item_seg);
    cudaFree(t.d_next);
    cudaFree(t.d_done);
    cudaFree(t.d_err);
    t.d_inst = nullptr;
    t.d_pass = nullptr;
    t.d_U = nullptr;
    t.d_seg = nullptr;
    t.d_item_seg = nullptr;
    t.d_next = nullptr;
    t.d_done = nullptr;
    t.d_err = nullptr;
    return ms;
}

// Chooses the fusion width k in [2, 5] and the work-item size (slices per item, the
// tile each CTA takes from the queue) minimising (passes of the circuit at width k) x
// (measured ms per pass of width k in items of that size at this qubit count); cached
// per (device, n).
Tuned autotune(rcs_batch *b, int n, const std::vector<HostGate> &hg, float2 *scratch) {
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find({b->dev, n});
        if (it != g_tuned.end()) return it->second;
    }
    Tuned best{std::min(4, n), kSlicesPerItem};
    double best_ms = 1e300;
    for (int k = 2; k <= std::min(kMaxK, n); ++k) {
        std::vector<Pass> passes;
        plan_fuse(n, hg, k, 0, &passes);
        for (uint32_t spi : kItemSizes) {
            if (spi > 2 * kSlicesPerItem && (1ull << (n - k)) < uint64_t(spi) * 64) continue;  // too few items
            const double ms = time_trial(n, k, spi, scratch, b);
            if (ms <= 0) continue;
            const double est = ms * double(passes.size());
            if (est < best_ms) {
                best_ms = est;
                best = Tuned{k, spi};
            }
        }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[{b->dev, n}] = best;
    return best;
}

void free_batch(rcs_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (InstHost &h : b->inst) {
        cudaFree(h.psi);
        cudaFree(h.bsum);
        cudaFree(h.bpre);
        cudaFree(h.chunk);
        cudaFree(h.total);
        cudaFree(h.d_bits);
        cudaFree(h.d_order);
        cudaFree(h.d_xeb);
        cudaFree(h.d_ops);
        cudaFree(h.d_sub);
    }
    cudaFree(b->d_inst);
    cudaFree(b->d_pass);
    cudaFree(b->d_U);
    cudaFree(b->d_seg);
    cudaFree(b->d_item_seg);
    cudaFree(b->d_next);
    cudaFree(b->d_done);
    cudaFree(b->d_err);
    btc_destroy(b->btc);
    delete b;
}

int launch_sampling(rcs_batch *b, InstHost &h, cudaStream_t st) {
    if (h.shots == 0) return RCS_OK;
    int rc;
    if ((rc = launch_block_sums(h.psi, h.n, h.bsum, b->d_err, plan_to_stored(h.plan), st)) != RCS_OK ||
        (rc = launch_block_scan(h.bsum, h.bpre, h.chunk, h.total, h.n, b->d_err, st)) != RCS_OK ||
        (rc = launch_sample(h.psi, h.n, h.bsum, h.bpre, h.total, h.chunk, 0, h.shots, h.seed, h.d_bits, h.d_order,
                            b->d_err, plan_to_stored(h.plan), st)) != RCS_OK ||
        (rc = launch_xeb(h.psi, h.n, h.d_bits, h.shots, h.total, h.d_xeb + 1, h.d_xeb, plan_to_stored(h.plan), st)) !=
            RCS_OK)
        return bfail(b, rc, "sampling launch: " + take_launch_error());
    return RCS_OK;
}

// One circuit of the tensor-core engine: |0...0> (through the sub-state stages when the
// plan has them), every pass, then the sampler and XEB.
int record_chain(rcs_batch *b, InstHost &h, cudaStream_t st) {
    size_t first = 0;
    int rc = RCS_OK;
    if (h.prefix > 0) {
        int fused = 0;
        if ((rc = run_substages(h.plan, h.stages, h.psi, h.d_sub, h.d_ops, b->d_err, st, &fused)) != RCS_OK)
            return bfail(b, rc, "sub-state stages: " + take_launch_error());
        first = size_t(h.prefix + fused);
    } else if ((rc = launch_init_zero(h.psi, h.n, st)) != RCS_OK) {
        return bfail(b, rc, "reset: " + take_launch_error());
    }
    int64_t launches = 0;
    if ((rc = launch_pass_range(h.plan, h.psi, h.n, first, h.plan.passes.size(), 0, h.d_ops, b->d_err, st,
                                &launches)) != RCS_OK)
        return bfail(b, rc, "pass launch: " + take_launch_error());
    return launch_sampling(b, h, st);
}

// The circuit's passes as steps of the persistent tensor-core kernel: the stages' passes on
// their sub-states, then the full-state passes; the first pass of each stage and the first
// full pass read the state before them as a sub-state (the very first reads |0...0>), so no
// zero fill or expansion is left. False if a pass cannot run there (not a 6-qubit
// tensor-core pass, a state under 13 qubits) or no full pass follows the last stage.
bool persistent_steps(const InstHost &h, std::vector<BtcStep> *out) {
    out->clear();
    const Plan &plan = h.plan;
    if (h.n < kTcK + 7 || plan.passes.empty() || plan.tc_offset.size() != plan.passes.size() || !h.d_ops) return false;
    for (size_t i = 0; i < plan.passes.size(); ++i)
        if (plan.passes[i].kind != PASS_TC || plan.passes[i].k != kTcK || plan.tc_offset[i] < 0) return false;
    const void *cur = nullptr;  // input of the next stage's first pass (null: |0...0>)
    uint64_t cur_mask = 0;      // its qubits, in the circuit's stored numbering
    size_t first = 0;
    auto step = [&](void *dst, int m, size_t i, const Pass &p, bool stage_first, uint64_t tmask) {
        BtcStep s;
        s.dst = dst;
        s.m = m;
        s.ops = h.d_ops + plan.tc_offset[i];
        s.p = p;
        if (stage_first) {
            s.from_zero = cur == nullptr;
            s.src = cur;
            s.src_m = std::popcount(cur_mask);
            s.tmask = tmask;
        }
        out->push_back(s);
    };
    if (h.prefix > 0) {
        uint8_t *buf = static_cast<uint8_t *>(h.d_sub);
        for (const SubStage &st : h.stages) {
            const int m = std::popcount(st.tmask);
            void *next = buf;
            buf += size_t(8) << m;
            if (st.count == 0) continue;
            if (m < kTcK + 7) return false;
            uint64_t inner = 0;  // the previous sub-state's qubits, numbered inside this one
            for (int q = 0, k = 0; q < plan.n; ++q)
                if ((st.tmask >> q) & 1) {
                    if ((cur_mask >> q) & 1) inner |= 1ull << k;
                    ++k;
                }
            for (int i = st.first; i < st.first + st.count; ++i)
                step(next, m, size_t(i), substate_pass(plan.passes[size_t(i)], st.tmask), i == st.first, inner);
            cur = next;
            cur_mask = st.tmask;
        }
        first = size_t(h.stages.back().first + h.stages.back().count);
        if (first >= plan.passes.size()) return false;
    }
    for (size_t i = first; i < plan.passes.size(); ++i) step(h.psi, h.n, i, plan.passes[i], i == first, cur_mask);
    return true;
}

// Tensor-core engine: the circuits the persistent kernel cannot run go first, one launch
// chain each (with their sampling); then the persistent kernel applies every pass of all
// the others in one launch, and their samplers and XEB run on parallel branches.
int record_tc(rcs_batch *b) {
    cudaStream_t s0 = b->cap;
    std::vector<size_t> chains, rest;
    for (size_t i = 0; i < b->inst.size(); ++i) (b->inst[i].persistent ? rest : chains).push_back(i);
    auto fork = [&]() -> int {
        BCUDA(b, cudaEventRecord(b->ev[0], s0), "fork event");
        for (size_t j = 0; j < b->side.size(); ++j) BCUDA(b, cudaStreamWaitEvent(b->side[j], b->ev[0], 0), "fork");
        return RCS_OK;
    };
    auto join = [&]() -> int {
        for (size_t j = 0; j < b->side.size(); ++j) {
            BCUDA(b, cudaEventRecord(b->ev[1 + j], b->side[j]), "join event");
            BCUDA(b, cudaStreamWaitEvent(s0, b->ev[1 + j], 0), "join");
        }
        return RCS_OK;
    };
    int rc = RCS_OK;
    if (!chains.empty()) {
        if ((rc = fork()) != RCS_OK) return rc;
        for (size_t r = 0; r < chains.size(); ++r)
            if ((rc = record_chain(b, b->inst[chains[r]], b->side[r % b->side.size()])) != RCS_OK) return rc;
        if ((rc = join()) != RCS_OK) return rc;
    }
    if (rest.empty()) return RCS_OK;
    if ((rc = btc_launch(b->btc, b->d_err, b->wait_cycles, b->skip_item, s0)) != RCS_OK)
        return bfail(b, rc, "persistent tensor-core launch: " + take_launch_error());
    if ((rc = fork()) != RCS_OK) return rc;
    for (size_t r = 0; r < rest.size(); ++r)
        if ((rc = launch_sampling(b, b->inst[rest[r]], b->side[r % b->side.size()])) != RCS_OK) return rc;
    return join();
}

// Tiles per work item of the persistent tensor-core kernel: each candidate builds its
// tables and times three launches (after one untimed) on the batch's own states; the
// fastest is kept. Every candidate must finish without a device error.
constexpr uint32_t kTilesPerItem[] = {2, 4, 8, 16, 32};

int tune_persistent(rcs_batch *b, const std::vector<std::vector<BtcStep>> &steps) {
    const bool tf32 = b->inst.front().plan.precision == RCS_PREC_TF32X3;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCUDA(b, cudaEventCreate(&e0), "event");
    BCUDA(b, cudaEventCreate(&e1), "event");
    float best_ms = 0.f;
    int rc = RCS_OK;
    for (size_t gi = 0; gi < std::size(kTilesPerItem); ++gi) {
        const uint32_t g = kTilesPerItem[gi];
        BtcPlan *pl = nullptr;
        if ((rc = btc_create(steps, tf32, g, &pl)) != RCS_OK) break;
        float ms = 0.f;
        rc = btc_launch(pl, b->d_err, b->wait_cycles, -1, b->cap);
        if (rc == RCS_OK && cudaEventRecord(e0, b->cap) != cudaSuccess) rc = RCS_ERR_CUDA;
        for (int r = 0; r < 3 && rc == RCS_OK; ++r) rc = btc_launch(pl, b->d_err, b->wait_cycles, -1, b->cap);
        if (rc == RCS_OK && (cudaEventRecord(e1, b->cap) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = RCS_ERR_CUDA;
        int h[2] = {0, 0};
        if (rc == RCS_OK && cudaMemcpy(h, b->d_err, 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = RCS_ERR_CUDA;
        if (rc == RCS_OK && h[0] != 0) rc = (h[0] & kErrTimeout) ? RCS_ERR_TIMEOUT : RCS_ERR_CUDA;
        if (rc != RCS_OK) {
            btc_destroy(pl);
            break;
        }
        b->trial_ms[gi] = double(ms) / 3.0;
        if (!b->btc || ms < best_ms) {
            btc_destroy(b->btc);
            b->btc = pl;
            b->tiles_per_item = g;
            best_ms = ms;
        } else {
            btc_destroy(pl);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != RCS_OK) {
        cudaMemset(b->d_err, 0, 8);
        return bfail(b, rc, "persistent tensor-core trial: " + take_launch_error());
    }
    return RCS_OK;
}

// Records the whole batch on b->cap: reset, persistent apply, then per circuit the
// sampler and XEB kernels spread over side streams.
int record(rcs_batch *b) {
    if (b->tc) return record_tc(b);
    cudaStream_t s0 = b->cap;
    BCUDA(b, cudaMemsetAsync(b->d_next, 0, 8, s0), "clear work counter");
    BCUDA(b, cudaMemsetAsync(b->d_done, 0, b->inst.size() * sizeof(unsigned int), s0), "clear completion counters");
    BCUDA(b, cudaMemsetAsync(b->d_err + 1, 0, sizeof(int), s0), "clear abort flag");
    k_batch_reset<<<dim3(unsigned(2 * device_sm_count()), unsigned(std::min<size_t>(b->inst.size(), 64))), 256, 0, s0>>>(
        b->d_inst, int(b->inst.size()));
    BCUDA(b, cudaGetLastError(), "batched reset launch");
    int rc = launch_apply(b, s0, b->nitems);
    if (rc != RCS_OK) return bfail(b, rc, take_launch_error());
    BCUDA(b, cudaEventRecord(b->ev[0], s0), "fork event");
    for (size_t j = 0; j < b->side.size(); ++j) BCUDA(b, cudaStreamWaitEvent(b->side[j], b->ev[0], 0), "fork");
    for (size_t i = 0; i < b->inst.size(); ++i)
        if ((rc = launch_sampling(b, b->inst[i], b->side[i % b->side.size()])) != RCS_OK) return rc;
    for (size_t j = 0; j < b->side.size(); ++j) {
        BCUDA(b, cudaEventRecord(b->ev[1 + j], b->side[j]), "join event");
        BCUDA(b, cudaStreamWaitEvent(s0, b->ev[1 + j], 0), "join");
    }
    return RCS_OK;
}

int capture(rcs_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = record(b);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (rc != RCS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    BCUDA(b, e, "end capture");
    b->graph = g;
    BCUDA(b, cudaGraphInstantiate(&b->exec, g, 0), "instantiate graph");
    return RCS_OK;
}

}  // namespace

extern "C" {

int rcs_batch_create(const rcs_batch_item *items, size_t n_items, const rcs_opts *opts, rcs_batch **out) {
    if (!out || (!items && n_items)) return set_thread_error(RCS_ERR_ARG, "null argument");
    *out = nullptr;
    if (n_items == 0) return set_thread_error(RCS_ERR_ARG, "empty batch");
    rcs_batch *b = nullptr;
    try {
        b = new rcs_batch;
        cudaGetDevice(&b->dev);
        b->tc = opts && (opts->precision == RCS_PREC_BF16X3 || opts->precision == RCS_PREC_TF32X3);
        if (opts && (opts->precision < RCS_PREC_FP32_PLAIN || opts->precision > RCS_PREC_TF32X3)) {
            free_batch(b);
            return set_thread_error(RCS_ERR_ARG, "unknown precision");
        }
        int k_fixed = opts && !b->tc ? opts->k_max : 0;
        const bool tune = !b->tc && (!opts || opts->autotune != 0 || k_fixed == 0);
        if (b->tc && opts->k_max != 0 && opts->k_max != kTcK) {
            free_batch(b);
            return set_thread_error(RCS_ERR_ARG, "the tensor-core batch uses k_max = 6 (or 0)");
        }
        if (k_fixed != 0 && (k_fixed < 2 || k_fixed > kMaxK)) {
            free_batch(b);
            return set_thread_error(RCS_ERR_ARG, "batched k_max must be 2..5 (0 = autotune)");
        }
        b->grid = persistent_grid();
        int clk_khz = 0;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, b->dev);
        b->wait_cycles = (long long)(std::max(clk_khz, 1000000)) * 1000ll * 2;  // ~2 s of SM clock
        b->inst.resize(n_items);
        // validate and allocate
        size_t max_amps = 0;
        std::vector<std::vector<HostGate>> hg(n_items);
        for (size_t i = 0; i < n_items; ++i) {
            const rcs_batch_item &it = items[i];
            if (it.n_qubits < 2 || it.n_qubits > 30) {
                free_batch(b);
                return set_thread_error(RCS_ERR_ARG, "batched circuits need 2..30 qubits");
            }
            hg[i].resize(it.n_gates);
            for (size_t g = 0; g < it.n_gates; ++g) {
                std::string why;
                int rc = gate_to_host(it.gates[g], it.n_qubits, &hg[i][g], &why);
                if (rc != RCS_OK) {
                    free_batch(b);
                    return set_thread_error(rc, "circuit " + std::to_string(i) + " gate " + std::to_string(g) + ": " + why);
                }
            }
            if (it.shots > (1ull << 26)) {
                free_batch(b);
                return set_thread_error(RCS_ERR_ARG, "at most 2^26 shots per circuit");
            }
            InstHost &h = b->inst[i];
            h.n = it.n_qubits;
            h.shots = it.shots;
            h.seed = it.seed;
            max_amps = std::max(max_amps, size_t(1) << h.n);
            const size_t nb = size_t(1) << (h.n - std::min(h.n, kSampleBlockLog2));
            BCUDA(b, cudaMalloc(&h.psi, (size_t(8) << h.n)), "state allocation");
            BCUDA(b, cudaMalloc(&h.bsum, nb * 8), "block sums");
            BCUDA(b, cudaMalloc(&h.bpre, nb * 8), "block prefix");
            BCUDA(b, cudaMalloc(&h.chunk, (scan_chunks(h.n) + 1) * 8), "scan chunks");
            BCUDA(b, cudaMalloc(&h.total, 8), "total");
            BCUDA(b, cudaMalloc(&h.d_bits, std::max<uint64_t>(h.shots, 1) * 8), "samples");
            BCUDA(b, cudaMalloc(&h.d_order, std::max<uint64_t>(h.shots, 1) * 8), "sampler scratch");
            BCUDA(b, cudaMalloc(&h.d_xeb, (1 + xeb_partials_count(std::max<uint64_t>(h.shots, 1))) * 8), "xeb");
        }
        BCUDA(b, cudaMalloc(&b->d_err, 8), "error word");
        BCUDA(b, cudaMemset(b->d_err, 0, 8), "error word");
        if (b->tc) {
            rcs_opts o{};
            o.precision = opts->precision;
            o.flags = opts->flags;
            for (size_t i = 0; i < n_items; ++i) {
                InstHost &h = b->inst[i];
                std::vector<uint8_t> img;
                int rc = plan_fresh_circuit(h.n, hg[i], o, &h.plan, &img);
                if (rc != RCS_OK) {
                    std::string m = "circuit " + std::to_string(i) + ": " + rcs_last_error(nullptr);
                    free_batch(b);
                    return set_thread_error(rc, m);
                }
                h.k = h.plan.k_max;
                if (!img.empty()) {
                    BCUDA(b, cudaMalloc(&h.d_ops, img.size()), "operand images");
                    BCUDA(b, cudaMemcpy(h.d_ops, img.data(), img.size(), cudaMemcpyHostToDevice), "operand images");
                }
                h.prefix = plan_stages(h.plan, &h.stages);
                if (h.prefix > 0) BCUDA(b, cudaMalloc(&h.d_sub, substage_bytes(h.stages)), "sub-state");
            }
            int prc = tc_prepare_device();
            if (prc == RCS_OK) prc = simt_prepare_device();
            if (prc != RCS_OK) {
                std::string m = take_launch_error();
                free_batch(b);
                return set_thread_error(prc, m);
            }
            BCUDA(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream");
            std::vector<std::vector<BtcStep>> steps;
            for (InstHost &h : b->inst) {
                std::vector<BtcStep> st;
                h.persistent = persistent_steps(h, &st);
                if (h.persistent) steps.push_back(std::move(st));
            }
            if (!steps.empty()) {
                if (int rc = tune_persistent(b, steps); rc != RCS_OK) {
                    std::string m = b->err;
                    free_batch(b);
                    return set_thread_error(rc, m);
                }
            }
            const size_t nside = std::min<size_t>(64, n_items);
            b->side.resize(nside, nullptr);
            for (auto &s : b->side) BCUDA(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
            b->ev.resize(1 + nside, nullptr);
            for (auto &e : b->ev) BCUDA(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            if (int rc = capture(b); rc != RCS_OK) {
                std::string m = b->err;
                free_batch(b);
                return set_thread_error(rc, m);
            }
            *out = b;
            return RCS_OK;
        }
        // fusion width per circuit: fixed, or by timed trials on a scratch state of the largest size
        float2 *scratch = nullptr;
        if (tune) {
            BCUDA(b, cudaMalloc(&scratch, max_amps * 8), "autotune scratch");
            BCUDA(b, cudaMemset(scratch, 0, max_amps * 8), "autotune scratch");
        }
        for (size_t i = 0; i < n_items; ++i) {
            InstHost &h = b->inst[i];
            const Tuned tu = tune ? autotune(b, h.n, hg[i], scratch) : Tuned{std::min(k_fixed, h.n), kSlicesPerItem};
            h.k = tu.k;
            h.slices_per_item = tu.slices_per_item;
            h.plan.n = h.n;
            h.plan.precision = RCS_PREC_FP32_FUSED;
            h.plan.k_max = h.k;
            h.plan.n_gates = int64_t(hg[i].size());
            plan_fuse(h.n, hg[i], h.k, 0, &h.plan.passes);
        }
        if (scratch) cudaFree(scratch);
        // one item count for every pass of a circuit (the dependency test counts items):
        // that of its narrowest pass, which has the most slices; wider passes leave the
        // surplus items empty
        for (InstHost &h : b->inst) {
            int kmin = 8;
            for (const Pass &p : h.plan.passes) kmin = std::min(kmin, p.k);
            h.items_per_pass = h.plan.passes.empty() ? 0 : items_per_pass(h.n, kmin, h.slices_per_item);
        }
        std::vector<BPass> passes;
        std::vector<float4> U;
        std::vector<BSeg> segs;
        std::vector<uint32_t> pass0;
        build_tables(b->inst, &passes, &U, &segs, &pass0, &b->nitems);
        std::vector<BInst> binst(n_items);
        for (size_t i = 0; i < n_items; ++i)
            binst[i] = BInst{b->inst[i].psi, uint32_t(b->inst[i].n), uint32_t(b->inst[i].items_per_pass),
                             b->inst[i].slices_per_item, 0};
        b->nseg = uint32_t(segs.size());
        BCUDA(b, cudaMalloc(&b->d_inst, binst.size() * sizeof(BInst)), "tables");
        BCUDA(b, cudaMalloc(&b->d_pass, std::max<size_t>(passes.size(), 1) * sizeof(BPass)), "tables");
        BCUDA(b, cudaMalloc(&b->d_U, std::max<size_t>(U.size(), 1) * sizeof(float4)), "tables");
        BCUDA(b, cudaMalloc(&b->d_seg, std::max<size_t>(segs.size(), 1) * sizeof(BSeg)), "tables");
        BCUDA(b, cudaMalloc(&b->d_next, 8), "tables");
        BCUDA(b, cudaMalloc(&b->d_done, n_items * sizeof(unsigned int)), "tables");
        BCUDA(b, cudaMemcpy(b->d_inst, binst.data(), binst.size() * sizeof(BInst), cudaMemcpyHostToDevice), "upload");
        if (!passes.empty())
            BCUDA(b, cudaMemcpy(b->d_pass, passes.data(), passes.size() * sizeof(BPass), cudaMemcpyHostToDevice), "upload");
        if (!U.empty()) BCUDA(b, cudaMemcpy(b->d_U, U.data(), U.size() * sizeof(float4), cudaMemcpyHostToDevice), "upload");
        if (!segs.empty())
            BCUDA(b, cudaMemcpy(b->d_seg, segs.data(), segs.size() * sizeof(BSeg), cudaMemcpyHostToDevice), "upload");
        {
            const std::vector<uint32_t> iseg = item_segments(segs, b->nitems);
            BCUDA(b, cudaMalloc(&b->d_item_seg, std::max<size_t>(iseg.size(), 1) * 4), "tables");
            if (!iseg.empty())
                BCUDA(b, cudaMemcpy(b->d_item_seg, iseg.data(), iseg.size() * 4, cudaMemcpyHostToDevice), "upload");
        }
        BCUDA(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream");
        const size_t nside = std::min<size_t>(8, n_items);
        b->side.resize(nside, nullptr);
        for (auto &s : b->side) BCUDA(b, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
        b->ev.resize(1 + nside, nullptr);
        for (auto &e : b->ev) BCUDA(b, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        int rc = capture(b);
        if (rc != RCS_OK && b->cooperative) {
            // capture of a cooperative launch refused: all CTAs still fit at once (grid sized by occupancy)
            cudaGetLastError();
            b->cooperative = false;
            rc = capture(b);
        }
        if (rc != RCS_OK) {
            std::string m = b->err;
            free_batch(b);
            return set_thread_error(rc, m);
        }
        *out = b;
        return RCS_OK;
    } catch (const std::bad_alloc &) {
        free_batch(b);
        return set_thread_error(RCS_ERR_OOM, "host allocation failed");
    }
}

int rcs_batch_launch(rcs_batch *b, uint64_t stream) {
    if (!b) return set_thread_error(RCS_ERR_ARG, "null batch");
    BCUDA(b, cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)), "graph launch");
    return RCS_OK;
}

int rcs_batch_wait(rcs_batch *b, uint64_t stream) {
    if (!b) return set_thread_error(RCS_ERR_ARG, "null batch");
    BCUDA(b, cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream sync");
    int h[2] = {0, 0};
    BCUDA(b, cudaMemcpy(h, b->d_err, 8, cudaMemcpyDeviceToHost), "read error word");
    if (h[0] == 0) return RCS_OK;
    BCUDA(b, cudaMemset(b->d_err, 0, 8), "clear error word");
    if (h[0] & kErrTimeout) return bfail(b, RCS_ERR_TIMEOUT, "a pass of the batched kernel waited past its limit");
    return bfail(b, RCS_ERR_ARG, "a batched state could not be sampled (error bits " + std::to_string(h[0]) + ")");
}

int rcs_batch_size(const rcs_batch *b) { return b ? int(b->inst.size()) : -1; }

int rcs_batch_info(const rcs_batch *b, size_t i, int32_t *n_qubits, int32_t *k, int64_t *n_passes) {
    if (!b || i >= b->inst.size()) return set_thread_error(RCS_ERR_ARG, "bad batch index");
    if (n_qubits) *n_qubits = b->inst[i].n;
    if (k) *k = b->inst[i].k;
    if (n_passes) *n_passes = int64_t(b->inst[i].plan.passes.size());
    return RCS_OK;
}

int rcs_batch_tuning(const rcs_batch *b, uint32_t *tiles_per_item, double *trial_ms) {
    if (!b) return set_thread_error(RCS_ERR_ARG, "null batch");
    if (!b->btc) return set_thread_error(RCS_ERR_UNSUPPORTED, "no circuit of this batch runs in the persistent kernel");
    if (tiles_per_item) *tiles_per_item = b->tiles_per_item;
    if (trial_ms)
        for (int i = 0; i < 5; ++i) trial_ms[i] = b->trial_ms[i];
    return RCS_OK;
}

int rcs_batch_result(rcs_batch *b, size_t i, uint64_t *out_bits, double *out_xeb) {
    if (!b || i >= b->inst.size()) return set_thread_error(RCS_ERR_ARG, "bad batch index");
    const InstHost &h = b->inst[i];
    if (out_bits && h.shots) BCUDA(b, cudaMemcpy(out_bits, h.d_bits, h.shots * 8, cudaMemcpyDeviceToHost), "download samples");
    if (out_xeb) BCUDA(b, cudaMemcpy(out_xeb, h.d_xeb, 8, cudaMemcpyDeviceToHost), "download xeb");
    return RCS_OK;
}

int rcs_batch_state_read(rcs_batch *b, size_t i, uint64_t first, uint64_t count, float *out_re_im) {
    if (!b || i >= b->inst.size()) return set_thread_error(RCS_ERR_ARG, "bad batch index");
    const InstHost &h = b->inst[i];
    const uint64_t lim = uint64_t(1) << h.n;
    if (first > lim || count > lim - first || (count && !out_re_im)) return set_thread_error(RCS_ERR_ARG, "bad range");
    if (!count) return RCS_OK;
    if (h.plan.phys_of.empty()) {
        BCUDA(b, cudaMemcpy(out_re_im, h.psi + first, count * 8, cudaMemcpyDeviceToHost), "read state");
        return RCS_OK;
    }
    // stored in the plan's qubit layout: read it all and put caller index c at position c
    try {
        std::vector<float2> all(static_cast<size_t>(lim));
        BCUDA(b, cudaMemcpy(all.data(), h.psi, lim * 8, cudaMemcpyDeviceToHost), "read state");
        const BitMap m = plan_to_stored(h.plan);
        float2 *out = reinterpret_cast<float2 *>(out_re_im);
        for (uint64_t c = first; c < first + count; ++c) {
            uint64_t s = 0;
            for (int q = 0; q < h.n; ++q) s |= ((c >> q) & 1ull) << m.to[q];
            out[c - first] = all[size_t(s)];
        }
    } catch (const std::bad_alloc &) {
        return set_thread_error(RCS_ERR_OOM, "host allocation failed");
    }
    return RCS_OK;
}

int rcs_batch_set_fault(rcs_batch *b, int64_t skip_item, double wait_limit_s) {
    if (!b) return set_thread_error(RCS_ERR_ARG, "null batch");
    if (b->tc && !b->btc) return bfail(b, RCS_ERR_UNSUPPORTED, "no circuit of this batch runs in the persistent kernel");
    int clk_khz = 0;
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, b->dev);
    b->skip_item = skip_item;
    b->wait_cycles = (long long)(double(std::max(clk_khz, 1000000)) * 1000.0 * (wait_limit_s > 0 ? wait_limit_s : 2.0));
    return capture(b);
}

const char *rcs_batch_last_error(const rcs_batch *b) { return b ? b->err.c_str() : ""; }

void rcs_batch_destroy(rcs_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
}

}  // extern "C"
