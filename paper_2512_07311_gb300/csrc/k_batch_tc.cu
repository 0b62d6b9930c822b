// Persistent tensor-core kernel of the batched engine: every 6-qubit pass of many
// independent circuits (Section 3.2 items 1 and 4, run as many jobs) in one launch.
//
// Each CTA owns one SM for the whole launch (17 warps, the roles and tensor-memory
// plan of the single-pass kernel in k_tc.cu: 8 loader warps, 8 epilogue warps, one
// MMA warp, two stages of one tile in shared memory, two tiles in flight in tensor
// memory). It allocates tensor memory and initialises its barriers once, then works
// through a fixed list of work items: an item is a range of tiles (128 slices of 64
// amplitudes each) of one pass of one circuit. CTA b takes items b, b + G, b + 2G, ...
// (G = the grid), and all of its roles walk that list in the same order.
//
// Order between passes. The host lists the items in rounds (round r holds step r of
// every circuit), so every item of a pass comes before every item of the same
// circuit's next pass. When an epilogue warp has stored its part of an item's last
// tile it publishes one completion on the circuit's counter (a release: fence, then
// atomic add); a loader warp that starts the first tile of an item waits until the
// counter holds the completions of all earlier passes of that circuit (an acquire:
// each lane's own ld.acquire, then a fence), so its copies see the earlier passes'
// stores. The loaders never block on that wait while a tile of their CTA is still
// unconverted: the look-ahead copy of the next tile is issued only if its pass is
// already free to start; otherwise it is issued once the current tile is converted.
// A wait is therefore only on items that come earlier in the list, which CTAs that
// are all resident (a cooperative launch) finish without waiting on later ones: the
// schedule cannot deadlock.
//
// Operand images. The MMA warp keeps the B image of the current pass in shared
// memory. At an item of another pass it waits until the MMAs of the previous tile
// have completed (so no MMA still reads the old image), loads the new one with bulk
// async copies (cp.async.bulk, completion counted on an mbarrier) and goes on.
//
// Sub-state inputs. Every circuit starts from |0...0>: its first pass reads a one-
// amplitude "sub-state" (the constant 1) with no qubits, and the first pass of every
// later stage reads the previous stage's state as a sub-state (the qubits outside it
// at 0), exactly as the single-pass kernel's sub-state variant does. So no zero fill
// or expansion runs between passes: the whole state construction is this one launch.
// All loads and stores go in slice order (each lane one slice of the tile); the
// memory-order variant of the single-pass kernel is not used here.
//
// Every wait is bounded. When a wait runs out the kernel raises kErrTimeout, sets the
// launch-wide abort word (every other CTA's waits then end at once), drains its own
// MMAs and copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <bit>
#include <cstring>
#include <new>
#include <vector>

#include "dev_common.cuh"
#include "internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rcs {

// One pass of one circuit as the kernel reads it (built on the host, read-only).
struct BtcPass {
    float2 *dst;          // the state the pass writes (2^m amplitudes, m <= 30)
    const float2 *src;    // sub-state input, or null: the pass reads dst in place
    const uint4 *ops;     // B operand image in its shared-memory layout (16-byte aligned)
    uint32_t tiles;       // 2^(m - 13)
    uint32_t circuit;     // completion counter of the circuit
    uint32_t need;        // completions of the circuit's earlier passes (8 per item)
    int32_t t[tc::K];     // ascending targets, in dst's numbering
    uint32_t off[tc::D];  // offset in dst of local amplitude j (j's bits on the targets)
    // sub-state input: offset in src of off[j] (its bits at their ranks among the
    // sub-state's qubits), or ~0u if off[j] sets a qubit outside the sub-state
    uint32_t soff[tc::D];
    // sub-state input: rank in the sub-state of the i-th lowest non-target qubit of dst,
    // or -1 if it lies outside (a slice with that bit set is all zeros)
    int8_t sbit[32];
};

struct BtcItem {
    uint32_t pass;    // index into the pass table
    uint32_t tile0;   // first tile of the item within the pass
    uint32_t ntiles;  // tiles in the item (>= 1)
    uint32_t reserved;
};

struct BtcArgs {
    const BtcPass *pass;
    const BtcItem *items;
    uint32_t nitems;
    unsigned int *done;  // per circuit: completions published
    int *err;            // error bits (kErrTimeout)
    int *abort;          // launch-wide abort word
    long long wait_cycles;
    long long skip_item;  // test hook: an item whose completion is never published (-1: none)
};

namespace btc {
// Shared-memory map (offsets from a 1024-aligned base): the B image, two stages of
// one tile, then the barriers and the tensor-memory slot.
template <bool kTf32>
struct Layout {
    static constexpr int kBBytes = tc::Layout<kTf32>::kBBytes;
    static constexpr int kStage0 = kBBytes;
    static constexpr int kBar = kStage0 + 2 * tc::kStageBytes;  // 24 mbarriers
    static constexpr int kMisc = kBar + 24 * 8;                  // tmem slot, abort flag
    static constexpr int kAlloc = kMisc + 16 + 1024;             // slack for 1024-byte alignment
    static_assert(kAlloc <= 227 * 1024, "shared memory");
};
constexpr int kBulkChunk = 16384;  // bytes per bulk copy of the B image
}  // namespace btc

// The constant amplitude 1: the "sub-state" with no qubits that every circuit's
// first pass reads (its state is |0...0>).
__device__ float2 g_btc_one = {1.0f, 0.0f};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Warp-wide wait for done >= need. block = false: one poll. Returns 1 when met (every
// lane has made its own acquiring load that saw it, then fenced), 0 when not met on a
// poll, -1 when the CTA or the launch aborted or the wait ran out (which aborts both).
__device__ __forceinline__ int dep_wait(const unsigned int *done, unsigned int need, bool block, const BtcArgs &a,
                                        volatile int *abort_flag, long long lim) {
    if (need == 0) return 1;
    const long long t0 = clock64();
    for (;;) {
        const unsigned int v = ld_acquire_gpu(done);
        if (__all_sync(0xffffffffu, v >= need)) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            return 1;
        }
        if (!block) return 0;
        int stop = 0;
        if ((threadIdx.x & 31) == 0) {
            if (*abort_flag || *reinterpret_cast<volatile int *>(a.abort)) {
                *abort_flag = 1;  // the CTA's other roles stop waiting too
                stop = 1;
            } else if (clock64() - t0 > lim) {
                *abort_flag = 1;
                atomicOr(a.err, kErrTimeout);
                atomicExch(a.abort, 1);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return -1;
        __nanosleep(128);
    }
}

template <bool kTf32>
__global__ void __launch_bounds__(tc::kThreads, 1) k_batch_tc(const __grid_constant__ BtcArgs a) {
    using namespace tc;
    using L = btc::Layout<kTf32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t bar0 = smem_u32(sm + L::kBar);
    auto bar_full = [&](int b) { return bar0 + 8u * uint32_t(b); };
    auto bar_done = [&](int b) { return bar0 + 16u + 8u * uint32_t(b); };
    auto bar_free = [&](int b) { return bar0 + 32u + 8u * uint32_t(b); };
    // TF32 (as in the single-pass kernel): A is filled and consumed in two K halves;
    // bar_full(b) counts the first half's loader warps, bar_full1(b) the second's, and
    // bar_done_a(b) completes once the MMAs that read the first half are done.
    auto bar_full1 = [&](int b) { return bar0 + 48u + 8u * uint32_t(b); };
    auto bar_done_a = [&](int b) { return bar0 + 64u + 8u * uint32_t(b); };
    auto bar_full_h = [&](int b, int h) { return (kTf32 && h) ? bar_full1(b) : bar_full(b); };
    const uint32_t bar_b = bar0 + 80u;  // the B image's bulk copies have landed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + L::kMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + L::kMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim = a.wait_cycles;
    const uint32_t G = gridDim.x;

    // ---- set-up: barriers, tensor memory (once for the whole launch)
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_full(b), kTf32 ? kLoaderWarps / 2 : kLoaderWarps);
            mbar_init(bar_full1(b), kLoaderWarps / 2);
            mbar_init(bar_done_a(b), 1);
            mbar_init(bar_done(b), 1);
            mbar_init(bar_free(b), kEpiWarps);
        }
        mbar_init(bar_b, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kLoaderWarps + kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // tiles of this CTA, over all its items
    uint32_t my_tiles = 0;
    for (uint32_t j = blockIdx.x; j < a.nitems; j += G) my_tiles += a.items[j].ntiles;

    // Tensor-memory plan, as in the single-pass kernel. BF16: two buffers of {D: 128
    // cols, A_hi: 64, A_lo: 64} at column 256 b. TF32: D double-buffered at column 128 b
    // and one A region at 256 holding, per K half h, Re_hi, Re_lo, Im_hi, Im_lo (32
    // columns each) at 256 + 128 h.
    auto dcol_of = [&](int b) { return tmem + uint32_t(b) * (kTf32 ? 128u : 256u); };
    auto acol_of = [&](int b) { return kTf32 ? tmem + 256u : tmem + uint32_t(b) * 256u + 128u; };
    auto wait_a_free = [&](uint32_t i, int h) {
        if constexpr (kTf32) {
            if (i < 1) return true;
            const uint32_t j = i - 1;
            return warp_wait<!kTf32>(h ? bar_done(int(j & 1)) : bar_done_a(int(j & 1)), (j >> 1) & 1, abort_flag, lim);
        } else {
            if (i < 2) return true;
            const uint32_t j = i - 2;
            return warp_wait<!kTf32>(bar_done(int(j & 1)), (j >> 1) & 1, abort_flag, lim);
        }
    };
    auto abase_of = [&](int b, int h) { return kTf32 ? acol_of(b) + 128u * uint32_t(h) : acol_of(b); };
    auto acol_in = [&](int h, int ch) { return kTf32 ? 16 * ch : 32 * h + 16 * ch; };
    auto put16 = [&](uint32_t abase, int col, const float2 (&v)[16]) {
        if constexpr (kTf32) {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) split_tf32(v[jj].x, hi[jj], lo[jj]);
            tmem_st16(abase + uint32_t(col), hi);
            tmem_st16(abase + 32u + uint32_t(col), lo);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) split_tf32(v[jj].y, hi[jj], lo[jj]);
            tmem_st16(abase + 64u + uint32_t(col), hi);
            tmem_st16(abase + 96u + uint32_t(col), lo);
        } else {
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) split_bf16x2(v[jj], hi[jj], lo[jj]);
            tmem_st16(abase + uint32_t(col), hi);
            tmem_st16(abase + 64u + uint32_t(col), lo);
        }
    };
    auto get16 = [&](uint32_t dbase, int j0, float2 (&v)[16]) {
        if constexpr (kTf32) {
            uint32_t re[16], im[16];
            tmem_ld16(dbase + uint32_t(j0), re);
            tmem_ld16(dbase + 64u + uint32_t(j0), im);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj]));
        } else {
            uint32_t x[32];
            tmem_ld32(dbase + uint32_t(2 * j0), x);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] = make_float2(__uint_as_float(x[2 * jj]), __uint_as_float(x[2 * jj + 1]));
        }
    };

    const uint32_t stage0_u32 = smem_u32(sm + L::kStage0);
    if (warp < kLoaderWarps) {
        // ---------------------------------------------------------------- loaders
        const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, amplitude half
        const int srow = 32 * q + lane;          // slice within the tile = TMEM lane
        // the next tile to issue: item ij, tile ik of it
        uint32_t ij = blockIdx.x, ik = 0, issued = 0;
        bool have = false, ready = false;  // item ij's fields loaded / its earlier passes done
        uint32_t tile0 = 0, ntiles = 0, need = 0, circuit = 0;
        float2 *dst = nullptr;
        const float2 *src = nullptr;
        int t[K];
        uint32_t myoff = 0, mysoff = 0;  // lane l: off[32 h + l], soff[32 h + l]
        uint64_t row_cb = 0;             // sub-state input: compact bits of this lane's slice row
        bool row_z = false;              // ... or the row sets a qubit outside the sub-state
        int lane_c = -1;                 // rank in the sub-state of tile bit `lane`, or -1
        auto load_item = [&]() {
            const BtcItem it = a.items[ij];
            const BtcPass *P = a.pass + it.pass;
            tile0 = it.tile0;
            ntiles = it.ntiles;
            need = P->need;
            circuit = P->circuit;
            dst = P->dst;
            src = P->src;
#pragma unroll
            for (int i = 0; i < K; ++i) t[i] = P->t[i];
            myoff = P->off[32 * h + lane];
            if (src) {
                mysoff = P->soff[32 * h + lane];
                row_cb = 0;
                row_z = false;
#pragma unroll
                for (int i = 0; i < 7; ++i)
                    if ((srow >> i) & 1) {
                        const int c = P->sbit[i];
                        if (c < 0) row_z = true;
                        else row_cb |= 1ull << c;
                    }
                lane_c = 7 + lane < 32 ? int(P->sbit[7 + lane]) : -1;
            }
            have = true;
        };
        // Issues the copies of the next tile into stage `issued & 1`. block = false: only if
        // its pass may start now. Returns 1 (issued), 0 (not yet) or -1 (abort).
        auto issue_next = [&](bool block) -> int {
            if (!have) load_item();
            if (!ready) {
                const int r = dep_wait(a.done + circuit, need, block, a, abort_flag, lim);
                if (r <= 0) return r;
                ready = true;
            }
            const int b = int(issued & 1);
            const uint64_t tile = uint64_t(tile0) + ik;
            if (src == nullptr) {
                const uint64_t base = slice_base(tile * M + uint64_t(srow), t);
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const uint32_t o = __shfl_sync(0xffffffffu, myoff, jj);
                    const float2 *p = dst + (base | o);
                    const uint32_t d = stage0_u32 + uint32_t(b * kStageBytes + ((32 * h + jj) * M + srow) * 8);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(p) : "memory");
                }
            } else {
                // a slice with a qubit outside the sub-state is all zeros; otherwise amplitude
                // j sits at compact index (row and tile bits of the slice) | soff[j], unless
                // off[j] leaves the sub-state. Zeros are copies of 0 source bytes (no read).
                const bool tbit = (tile >> lane) & 1ull;
                uint64_t cb = (tbit && lane_c >= 0) ? (1ull << lane_c) : 0ull;
                uint32_t zt = (tbit && lane_c < 0) ? 1u : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    cb |= __shfl_xor_sync(0xffffffffu, cb, o);
                    zt |= __shfl_xor_sync(0xffffffffu, zt, o);
                }
                cb |= row_cb;
                const bool zslice = row_z || zt != 0;
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const uint32_t so = __shfl_sync(0xffffffffu, mysoff, jj);
                    const bool zero = zslice || so == ~0u;
                    const float2 *p = zero ? src : src + (cb | so);
                    const uint32_t nbytes = zero ? 0u : 8u;
                    const uint32_t d = stage0_u32 + uint32_t(b * kStageBytes + ((32 * h + jj) * M + srow) * 8);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(p), "r"(nbytes)
                                 : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            ++issued;
            if (++ik == ntiles) {
                ij += G;
                ik = 0;
                have = ready = false;
            }
            return 1;
        };
        for (uint32_t i = 0; i < my_tiles; ++i) {
            // tile i must be in flight; every earlier tile of this CTA is converted, so a
            // blocking wait here cannot hold up work that the awaited passes need
            bool ok = true;
            while (ok && issued <= i) ok = issue_next(true) > 0;
            // look ahead by one tile, without waiting on another CTA
            if (ok && issued == i + 1 && issued < my_tiles) ok = issue_next(false) >= 0;
            if (!ok) break;
            if (issued > i + 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (!wait_a_free(i, h)) break;
            tc_fence_after();
            const int b = int(i & 1);
            const float2 *stage = reinterpret_cast<const float2 *>(sm + L::kStage0 + b * kStageBytes);
            const uint32_t abase = abase_of(b, h) + (uint32_t(32 * q) << 16);
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                float2 v[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] = stage[(32 * h + 16 * ch + jj) * M + srow];
                put16(abase, acol_in(h, ch), v);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full_h(b, h));
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < kLoaderWarps + kEpiWarps) {
        // ---------------------------------------------------------------- epilogue
        const int e = warp - kLoaderWarps;
        const int q = e & 3, h = e >> 2;
        const int srow = 32 * q + lane;
        const bool odd = lane & 1;
        auto st16 = [](float2 *p, float2 x, float2 y) {
            asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y)
                         : "memory");
        };
        uint32_t i = 0;
        bool stop = false;
        for (uint32_t j = blockIdx.x; j < a.nitems && !stop; j += G) {
            const BtcItem it = a.items[j];
            const BtcPass *P = a.pass + it.pass;
            float2 *dst = P->dst;
            int t[K];
#pragma unroll
            for (int x = 0; x < K; ++x) t[x] = P->t[x];
            const uint32_t myoff = P->off[32 * h + lane];
            // 16-byte stores, as in the single-pass kernel: lowest target on bit 0, a slice's
            // amplitudes j, j+1 are adjacent; on bit 1, lane pairs swap one amplitude so
            // that each lane writes two adjacent slices of one j
            const int smode = t[0] == 0 ? 1 : (t[0] == 1 ? 2 : 0);
            for (uint32_t k = 0; k < it.ntiles; ++k, ++i) {
                const int b = int(i & 1);
                if (!warp_wait<!kTf32>(bar_done(b), (i >> 1) & 1, abort_flag, lim)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint64_t base = slice_base((uint64_t(it.tile0) + k) * M + uint64_t(srow), t);
                const uint32_t dbase = dcol_of(b) + (uint32_t(32 * q) << 16);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    float2 v[16];
                    get16(dbase, 32 * h + 16 * c, v);
                    if (smode == 1) {
#pragma unroll
                        for (int jj = 0; jj < 16; jj += 2) {
                            const uint32_t o = __shfl_sync(0xffffffffu, myoff, 16 * c + jj);
                            st16(dst + (base | o), v[jj], v[jj + 1]);
                        }
                    } else if (smode == 2) {
                        const uint64_t pbase = base & ~1ull;
#pragma unroll
                        for (int jj = 0; jj < 16; jj += 2) {
                            const float2 send = odd ? v[jj] : v[jj + 1];
                            const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                                            __shfl_xor_sync(0xffffffffu, send.y, 1));
                            const float2 x = odd ? recv : v[jj], y = odd ? v[jj + 1] : recv;
                            const uint32_t o = __shfl_sync(0xffffffffu, myoff, 16 * c + jj + (odd ? 1 : 0));
                            st16(dst + (pbase | o), x, y);
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const uint32_t o = __shfl_sync(0xffffffffu, myoff, 16 * c + jj);
                            dst[base | o] = v[jj];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_free(b));
            }
            if (stop) break;
            // publish: this warp's stores of item j are done (release)
            __syncwarp();
            if (lane == 0 && (long long)j != a.skip_item) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                atomicAdd(a.done + P->circuit, 1u);
            }
        }
    } else {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t bimg = smem_u32(sm);
            uint32_t last_bar = 0, last_par = 0;
            bool committed = false, stop = false;
            auto commit = [&](uint32_t bar, uint32_t par) {
                mma_commit(bar);
                last_bar = bar;
                last_par = par;
                committed = true;
            };
            const uint4 *cur_ops = nullptr;
            uint32_t bphase = 0, i = 0;
            bool bulk_pending = false;  // a B image copy was issued and not yet seen complete
            for (uint32_t j = blockIdx.x; j < a.nitems && !stop; j += G) {
                const BtcItem it = a.items[j];
                const uint4 *ops = a.pass[it.pass].ops;
                if (ops != cur_ops) {
                    // no MMA may still read the old image: wait for the previous tile's MMAs
                    if (i > 0 && !mbar_wait<!kTf32>(bar_done(int((i - 1) & 1)), ((i - 1) >> 1) & 1, abort_flag, lim))
                        break;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_b),
                                 "r"(uint32_t(L::kBBytes))
                                 : "memory");
                    for (int c = 0; c < L::kBBytes; c += btc::kBulkChunk)
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                bimg + uint32_t(c)),
                            "l"(reinterpret_cast<const uint8_t *>(ops) + c), "r"(uint32_t(btc::kBulkChunk)), "r"(bar_b)
                            : "memory");
                    bulk_pending = true;
                    if (!mbar_wait<false>(bar_b, bphase, abort_flag, lim)) break;
                    bulk_pending = false;
                    bphase ^= 1u;
                    cur_ops = ops;
                }
                for (uint32_t k = 0; k < it.ntiles; ++k, ++i) {
                    const int b = int(i & 1);
                    const uint32_t par = (i >> 1) & 1;
                    if (!mbar_wait<!kTf32>(bar_full(b), par, abort_flag, lim) ||
                        (i >= 2 && !mbar_wait<!kTf32>(bar_free(b), ((i >> 1) - 1) & 1, abort_flag, lim))) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dcol = dcol_of(b), acol = acol_of(b);
                    if constexpr (kTf32) {
                        auto half = [&](int hh) {
#pragma unroll
                            for (int k4 = 0; k4 < 4; ++k4) {
                                const int kk = 4 * hh + k4;
                                const uint32_t kof = uint32_t(hh) * uint32_t(kTf32Atom) + uint32_t(k4) * 32u;
                                const uint32_t hi = bimg + kof, lo = bimg + uint32_t(kTf32Split) + kof;
                                const uint64_t b1h = sw128_desc(hi + 64u * 128u), b1l = sw128_desc(lo + 64u * 128u);
                                const uint64_t b2h = sw128_desc(hi), b2l = sw128_desc(lo);
                                const uint32_t ac = acol + 128u * uint32_t(hh) + uint32_t(k4) * 8u;
                                mma_tf32_tmemA(dcol, ac, b1h, kIdescTf32, kk > 0 ? 1u : 0u);
                                mma_tf32_tmemA(dcol, ac + 32u, b1h, kIdescTf32, 1u);
                                mma_tf32_tmemA(dcol, ac, b1l, kIdescTf32, 1u);
                                mma_tf32_tmemA(dcol, ac + 64u, b2h, kIdescTf32, 1u);
                                mma_tf32_tmemA(dcol, ac + 96u, b2h, kIdescTf32, 1u);
                                mma_tf32_tmemA(dcol, ac + 64u, b2l, kIdescTf32, 1u);
                            }
                        };
                        half(0);
                        commit(bar_done_a(b), par);
                        if (!mbar_wait<!kTf32>(bar_full1(b), par, abort_flag, lim)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        half(1);
                    } else {
                        const uint32_t bhi = bimg + uint32_t(kSmBhi), blo = bimg + uint32_t(kSmBlo);
#pragma unroll
                        for (int kk = 0; kk < KR / 16; ++kk) {
                            const uint32_t boff = uint32_t(kk >> 2) * uint32_t(NR * 128) + uint32_t(kk & 3) * 32u;
                            const uint64_t dhi = sw128_desc(bhi + boff), dlo = sw128_desc(blo + boff);
                            const uint32_t ac = acol + uint32_t(kk) * 8u;
                            mma_bf16_tmemA(dcol, ac, dhi, kk > 0 ? 1u : 0u);
                            mma_bf16_tmemA(dcol, ac + 64u, dhi, 1u);
                            mma_bf16_tmemA(dcol, ac, dlo, 1u);
                        }
                    }
                    commit(bar_done(b), par);
                }
            }
            if (*abort_flag) {
                // drain: the last committed MMAs and any bulk copy in flight must finish
                // before tensor memory is freed and the CTA exits
                const long long t0 = clock64();
                if (committed)
                    while (!mbar_try_wait(last_bar, last_par) && clock64() - t0 < lim) {
                    }
                if (bulk_pending)
                    while (!mbar_try_wait(bar_b, bphase) && clock64() - t0 < lim) {
                    }
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        atomicOr(a.err, kErrTimeout);
        atomicExch(a.abort, 1);
    }
    if (warp == kLoaderWarps + kEpiWarps) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- host side

struct BtcPlan {
    BtcPass *d_pass = nullptr;
    BtcItem *d_items = nullptr;
    unsigned int *d_done = nullptr;
    uint32_t nitems = 0, ncircuits = 0, grid = 0;
    bool tf32 = false;
};

namespace {

template <bool kTf32>
int btc_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_batch_tc<kTf32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         btc::Layout<kTf32>::kAlloc);
    return e == cudaSuccess ? RCS_OK : note_launch_error("tensor-core batch attribute", e);
}

// rank of qubit qb among the set bits of mask, or -1 if qb is not in it
int rank_in(uint64_t mask, int qb) {
    if (!((mask >> qb) & 1ull)) return -1;
    return std::popcount(mask & ((1ull << qb) - 1ull));
}

}  // namespace

// The pass and item tables of a batch (host side of btc_create): `one` is the device
// address of the constant amplitude 1 that from_zero passes read.
int btc_build_tables(const std::vector<std::vector<BtcStep>> &circuits, uint32_t tiles_per_item, const void *one,
                     std::vector<BtcPass> *passes_out, std::vector<BtcItem> *items_out) {
    using namespace tc;
    if (tiles_per_item == 0) return RCS_ERR_ARG;
    std::vector<BtcPass> &passes = *passes_out;
    std::vector<BtcItem> &items = *items_out;
    passes.clear();
    items.clear();
    std::vector<std::vector<uint32_t>> pass_of(circuits.size());  // circuit -> its pass indices, in order
    for (size_t c = 0; c < circuits.size(); ++c) {
        uint32_t done_before = 0;
        for (const BtcStep &s : circuits[c]) {
            const Pass &p = s.p;
            if (p.kind != PASS_TC || p.k != K || s.m < K + 7 || s.m > 30) return RCS_ERR_UNSUPPORTED;
            if ((reinterpret_cast<uintptr_t>(s.ops) & 15u) || (reinterpret_cast<uintptr_t>(s.dst) & 15u) ||
                (reinterpret_cast<uintptr_t>(s.src) & 7u) || !s.dst || !s.ops)
                return RCS_ERR_ARG;
            const uint64_t tmask = s.from_zero ? 0ull : s.tmask;
            // a sub-state input holds exactly the amplitudes of its qubits: 2^popcount(tmask)
            if ((s.from_zero || s.src) && (std::popcount(tmask) != (s.from_zero ? 0 : s.src_m) ||
                                          (s.m < 64 && (tmask >> s.m) != 0)))
                return RCS_ERR_ARG;
            BtcPass bp;
            std::memset(&bp, 0, sizeof(bp));
            bp.dst = static_cast<float2 *>(s.dst);
            bp.src = s.from_zero ? static_cast<const float2 *>(one) : static_cast<const float2 *>(s.src);
            bp.ops = static_cast<const uint4 *>(s.ops);
            bp.tiles = uint32_t(1u << (s.m - K - 7));
            bp.circuit = uint32_t(c);
            bp.need = done_before;
            for (int i = 0; i < K; ++i) {
                if (p.t[i] < 0 || p.t[i] >= s.m || (i > 0 && p.t[i] <= p.t[i - 1])) return RCS_ERR_ARG;
                bp.t[i] = p.t[i];
            }
            for (int j = 0; j < D; ++j) {
                uint32_t o = 0;
                for (int i = 0; i < K; ++i)
                    if ((j >> i) & 1) o |= 1u << p.t[i];
                bp.off[j] = o;
                uint32_t so = 0;
                for (int i = 0; i < K && so != ~0u; ++i)
                    if ((j >> i) & 1) {
                        const int r = rank_in(tmask, p.t[i]);
                        so = r < 0 ? ~0u : (so | (1u << r));
                    }
                bp.soff[j] = so;
            }
            for (int i = 0; i < 32; ++i) bp.sbit[i] = -1;
            for (int qb = 0, i = 0; qb < s.m && i < 32; ++qb) {
                if (std::find(p.t, p.t + K, qb) != p.t + K) continue;
                bp.sbit[i++] = int8_t(rank_in(tmask, qb));
            }
            const uint32_t nit = (bp.tiles + tiles_per_item - 1) / tiles_per_item;
            done_before += uint32_t(kEpiWarps) * nit;
            pass_of[c].push_back(uint32_t(passes.size()));
            passes.push_back(bp);
        }
    }
    // items in rounds: round r holds pass r of every circuit, the largest passes first
    size_t rounds = 0;
    for (const auto &v : pass_of) rounds = std::max(rounds, v.size());
    for (size_t r = 0; r < rounds; ++r) {
        std::vector<size_t> here;
        for (size_t c = 0; c < circuits.size(); ++c)
            if (r < pass_of[c].size()) here.push_back(c);
        std::stable_sort(here.begin(), here.end(), [&](size_t x, size_t y) {
            return passes[pass_of[x][r]].tiles > passes[pass_of[y][r]].tiles;
        });
        for (size_t c : here) {
            const uint32_t pi = pass_of[c][r];
            const uint32_t T = passes[pi].tiles;
            for (uint32_t t0 = 0; t0 < T; t0 += tiles_per_item)
                items.push_back(BtcItem{pi, t0, std::min(tiles_per_item, T - t0), 0});
        }
    }
    return RCS_OK;
}

int btc_create(const std::vector<std::vector<BtcStep>> &circuits, bool tf32, uint32_t tiles_per_item,
               BtcPlan **out) {
    *out = nullptr;
    void *one = nullptr;
    if (cudaError_t e = cudaGetSymbolAddress(&one, g_btc_one); e != cudaSuccess)
        return note_launch_error("tensor-core batch constant", e);
    std::vector<BtcPass> passes;
    std::vector<BtcItem> items;
    if (int rc = btc_build_tables(circuits, tiles_per_item, one, &passes, &items); rc != RCS_OK) return rc;
    BtcPlan *pl = new (std::nothrow) BtcPlan;
    if (!pl) return RCS_ERR_OOM;
    pl->tf32 = tf32;
    pl->nitems = uint32_t(items.size());
    pl->ncircuits = uint32_t(circuits.size());
    pl->grid = uint32_t(std::min<size_t>(items.size(), size_t(device_sm_count())));
    int rc = tf32 ? btc_smem_attr<true>() : btc_smem_attr<false>();
    auto fail = [&](int code) {
        btc_destroy(pl);
        return code;
    };
    if (rc != RCS_OK) return fail(rc);
    if (!passes.empty()) {
        if (cudaMalloc(&pl->d_pass, passes.size() * sizeof(BtcPass)) != cudaSuccess ||
            cudaMalloc(&pl->d_items, items.size() * sizeof(BtcItem)) != cudaSuccess ||
            cudaMalloc(&pl->d_done, std::max<size_t>(circuits.size(), 1) * sizeof(unsigned int)) != cudaSuccess)
            return fail(RCS_ERR_OOM);
        if (cudaMemcpy(pl->d_pass, passes.data(), passes.size() * sizeof(BtcPass), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(pl->d_items, items.data(), items.size() * sizeof(BtcItem), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(RCS_ERR_CUDA);
    }
    *out = pl;
    return RCS_OK;
}

uint32_t btc_items(const BtcPlan *p) { return p ? p->nitems : 0; }

int btc_launch(const BtcPlan *p, int *d_err, long long wait_cycles, long long skip_item, void *stream) {
    if (!p) return RCS_ERR_ARG;
    if (p->nitems == 0) return RCS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(p->d_done, 0, p->ncircuits * sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return note_launch_error("tensor-core batch counters", e);
    BtcArgs a;
    a.pass = p->d_pass;
    a.items = p->d_items;
    a.nitems = p->nitems;
    a.done = p->d_done;
    a.err = d_err;
    a.abort = d_err + 1;
    a.wait_cycles = wait_cycles > 0 ? wait_cycles : kTcWaitCycles;
    a.skip_item = skip_item;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->grid);
    cfg.blockDim = dim3(tc::kThreads);
    cfg.dynamicSmemBytes = p->tf32 ? btc::Layout<true>::kAlloc : btc::Layout<false>::kAlloc;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = p->tf32 ? cudaLaunchKernelEx(&cfg, k_batch_tc<true>, a) : cudaLaunchKernelEx(&cfg, k_batch_tc<false>, a);
    return e == cudaSuccess ? RCS_OK : note_launch_error("tensor-core batch", e);
}

void btc_destroy(BtcPlan *p) {
    if (!p) return;
    cudaFree(p->d_pass);
    cudaFree(p->d_items);
    cudaFree(p->d_done);
    delete p;
}

}  // namespace rcs
