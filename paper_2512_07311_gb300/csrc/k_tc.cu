// Fused 6-qubit state update on the 5th-generation tensor cores (tcgen05), with a
// BF16 hi/lo split of both operands and three products accumulated in FP32.
//
// One pass applies a 64x64 complex unitary U to every slice of the state: slice s
// is the 64 amplitudes that differ only in the 6 target bits. Written as a real
// GEMM on interleaved (re, im) data, each slice x (128 reals) maps to R x with the
// realified R (128 x 128): R[2a][2b] = Re U[a][b], R[2a][2b+1] = -Im U[a][b],
// R[2a+1][2b] = Im U[a][b], R[2a+1][2b+1] = Re U[a][b]. A tile of 128 slices is
//     D (128 slices x 128 outputs) = X (128 x 128) * R^T (128 x 128),
// one tcgen05 MMA chain with M = N = 128 and K = 128 (8 steps of K = 16).
// Split precision: x = x_hi + x_lo, R = R_hi + R_lo with hi = bf16(v), lo =
// bf16(v - hi); D = X_hi R_hi^T + X_lo R_hi^T + X_hi R_lo^T (the lo*lo term, about
// 2^-17 relative, is dropped), accumulated in FP32 in tensor memory.
//
// Data flow per CTA (persistent, one CTA per SM, 17 warps):
//   warps 0-7  (loaders):  cp.async 8-byte copies of a tile's amplitudes into a
//              shared-memory stage (two tiles in flight), then split each amplitude
//              into bf16x2 hi and lo words and write them to tensor memory with
//              tcgen05.st: the slice's 64 amplitudes become row s of the A operand
//              (A is read by the MMA straight from TMEM, lane = slice).
//   warp 16    (MMA):      one thread issues the 24 MMAs of a tile (B = R^T from
//              shared memory, 128-byte swizzled, K-major) and commits to an mbarrier.
//   warps 8-15 (epilogue): tcgen05.ld of the FP32 accumulator rows (lane = slice)
//              and coalesced 8-byte stores of the new amplitudes, in place.
// Tensor memory holds two buffers of {D: 128 cols, A_hi: 64 cols, A_lo: 64 cols},
// so loading tile i+1, the MMAs of tile i and the stores of tile i-1 overlap.
// Lanes of a warp always take 32 consecutive slices, so every global load and store
// instruction walks consecutive addresses along the lowest non-target qubits; with
// the lowest target on bit 0 or 1 the stores are 16 bytes wide (see the epilogue).
//
// Variants (template parameters):
//   kStaged: loads and stores walk the tile in memory order through a swizzled stage
//            (for passes with 4 or more targets below bit 5);
//   kTf32:   a TF32 hi/lo split in the complex block form, Re y = Xr Ur^T - Xi Ui^T and
//            Im y = Xr Ui^T + Xi Ur^T: 48 MMAs of M = N = 128, K = 8 per tile, B images
//            [Ur; Ui] and [-Ui; Ur] as windows of one [-Ui; Ur; Ui] image per split;
//   kSub:    the input comes from a compact sub-state (the state is |0> on the qubits
//            outside it), so the pass also expands that sub-state into the full state.
//
// Every wait is bounded (about one second of SM clock); on expiry the kernel raises
// an error bit, drains its own MMAs and copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "dev_common.cuh"
#include "internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rcs {

struct TcArgs {
    float2 *psi;
    const uint4 *ops;  // B operand images in their shared-memory layout (BF16: 64 KB, TF32: 96 KB)
    int *err;
    uint32_t tiles;
    int t[tc::K];      // ascending targets
    uint64_t vmask;    // qubits varying inside a tile: the targets and the 7 lowest other qubits
    int r;             // qubits 0 .. r-1 all lie in vmask (r >= 7): contiguous runs of 2^r amplitudes
    // Input from a sub-state (kSub): the state is |0> on the qubits outside `tmask`, and
    // its amplitudes with those qubits at 0 sit in `sub` at their compact index (the
    // index bits in tmask, in order). The pass writes the whole state to psi.
    const float2 *sub;
    uint64_t tmask;
    long long wait_cycles;  // limit of every wait (SM clock cycles)
    int skip_tile;          // test hook: CTA 0 issues no MMAs for its tile skip_tile (-1: none)
};

// Position of compact tile index c in the memory-order stage: XOR-swizzles bits
// 6..9 into bits 0..3 so that both consecutive c (global-side copies) and c that
// differ only in slice bits (TMEM-side rows) spread over the shared-memory banks.
__device__ __forceinline__ uint32_t swz(uint32_t c) { return c ^ ((c >> 6) & 15u); }

// kStaged = false: lanes of a loader or epilogue warp take 32 consecutive slices
// and move 8 bytes each straight between global memory and the stage / registers;
// coalesced when no target is below qubit 5 (the slices then sit side by side).
// kStaged = true: for passes with low targets, loads and stores walk the tile in
// memory order (32 consecutive amplitudes per warp instruction) through the
// swizzled shared-memory stage, which also carries the outputs back out.
// kTf32 = false: BF16 split of the realified operands (24 MMAs of K = 16 per tile).
// kTf32 = true: TF32 split of the complex block form (48 MMAs of K = 8 per tile).
// kSub (slice order only): the loads come from the sub-state a.sub instead of psi (see
// TcArgs), so the pass both expands the sub-state and applies its unitary.
template <bool kStaged, bool kTf32, bool kSub>
__global__ void __launch_bounds__(tc::kThreads, 1) k_fused_tc(const __grid_constant__ TcArgs a) {
    static_assert(!(kStaged && kSub), "the sub-state input has a slice-order loader only");
    using namespace tc;
    using L = Layout<kTf32>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *off = reinterpret_cast<uint64_t *>(sm + L::kOff);
    const uint32_t bar0 = smem_u32(sm + L::kBar);
    auto bar_full = [&](int b) { return bar0 + 8u * uint32_t(b); };
    auto bar_done = [&](int b) { return bar0 + 16u + 8u * uint32_t(b); };
    auto bar_free = [&](int b) { return bar0 + 32u + 8u * uint32_t(b); };
    auto bar_loaded = [&](int b) { return bar0 + 48u + 8u * uint32_t(b); };    // stage b holds the tile's inputs
    auto bar_outready = [&](int b) { return bar0 + 64u + 8u * uint32_t(b); };  // stage b holds the tile's outputs
    auto bar_sfree = [&](int b) { return bar0 + 80u + 8u * uint32_t(b); };     // stage b read out by the stores
    // TF32: A is filled and consumed in two K halves (inputs 0..31 by loader warps 0-3,
    // 32..63 by warps 4-7). bar_full(b) then counts the first half's warps and
    // bar_full1(b) the second's; bar_done_a(b) completes once the MMAs that read the
    // first half are done, bar_done(b) once all of the tile's MMAs are.
    auto bar_full1 = [&](int b) { return bar0 + 96u + 8u * uint32_t(b); };
    auto bar_done_a = [&](int b) { return bar0 + 112u + 8u * uint32_t(b); };
    auto bar_full_h = [&](int b, int h) { return (kTf32 && h) ? bar_full1(b) : bar_full(b); };
    uint64_t *hi_off = reinterpret_cast<uint64_t *>(sm + L::kHiOff);
    uint16_t *cj = reinterpret_cast<uint16_t *>(sm + L::kCj);
    uint16_t *cs = reinterpret_cast<uint16_t *>(sm + L::kCs);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + L::kMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + L::kMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim = a.wait_cycles;
    int t[K];
#pragma unroll
    for (int i = 0; i < K; ++i) t[i] = a.t[i];

    // ---- set-up: operand image, offset table, barriers, tensor memory
    {
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        for (int i = threadIdx.x; i < L::kBBytes / 16; i += kThreads) dst[i] = a.ops[i];
        const uint64_t V = a.vmask;
        auto cpos = [&](int qb) { return __popcll(V & ((1ull << qb) - 1ull)); };  // compact position of qubit qb
        if (threadIdx.x < D) {
            uint64_t o = 0;
            uint32_t c = 0;
#pragma unroll
            for (int i = 0; i < K; ++i)
                if ((threadIdx.x >> i) & 1) {
                    o |= 1ull << t[i];
                    c |= 1u << cpos(t[i]);
                }
            off[threadIdx.x] = o;
            cj[threadIdx.x] = uint16_t(c);
            // high compact bits r..12 of c sit on the qubits of V above r, in order
            uint64_t ho = 0;
            int bit = 0;
            for (int qb = a.r; qb < 64 && bit < 13 - a.r; ++qb)
                if ((V >> qb) & 1) {
                    if ((threadIdx.x >> bit) & 1) ho |= 1ull << qb;
                    ++bit;
                }
            hi_off[threadIdx.x] = ho;
            if constexpr (kSub) {  // per j: compact offset of off[j] in the sub-state, or ~0 if it leaves it
                uint64_t cpos_sub = 0;
                if (o & ~a.tmask) {
                    cpos_sub = ~0ull;
                } else {
                    int k = 0;
                    for (int qb = 0; qb < 64; ++qb)
                        if ((a.tmask >> qb) & 1) {
                            cpos_sub |= ((o >> qb) & 1ull) << k;
                            ++k;
                        }
                }
                hi_off[threadIdx.x] = cpos_sub;  // hi_off serves the memory-order variant only
            }
        }
        if (threadIdx.x < M) {
            // slice bit k sits on the k-th lowest qubit that is not a target
            uint32_t c = 0;
            int k = 0;
            for (int qb = 0; qb < 64 && k < 7; ++qb) {
                bool tgt = false;
#pragma unroll
                for (int i = 0; i < K; ++i) tgt |= (t[i] == qb);
                if (tgt) continue;
                if ((threadIdx.x >> k) & 1) c |= 1u << cpos(qb);
                ++k;
            }
            cs[threadIdx.x] = uint16_t(c);
        }
        if (threadIdx.x == 0) {
            for (int b = 0; b < 2; ++b) {
                mbar_init(bar_full(b), kTf32 ? kLoaderWarps / 2 : kLoaderWarps);
                mbar_init(bar_full1(b), kLoaderWarps / 2);
                mbar_init(bar_done_a(b), 1);
                mbar_init(bar_done(b), 1);
                mbar_init(bar_free(b), kEpiWarps);
                mbar_init(bar_loaded(b), kLoaderWarps * 32);
                mbar_init(bar_outready(b), kEpiWarps);
                mbar_init(bar_sfree(b), kEpiWarps);
            }
            *abort_flag = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (warp == kLoaderWarps + kEpiWarps) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                         "r"(kTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    const uint32_t tmem = *tmem_slot;
    const uint32_t ntile = a.tiles;
    const uint32_t my_tiles = blockIdx.x < ntile ? (ntile - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // Tensor-memory plan. BF16: two buffers of {D: 128 cols, A_hi: 64, A_lo: 64} at
    // column 256 b. TF32: D double-buffered at column 128 b (Re outputs in its first 64
    // columns, Im in the last 64) and one A region at 256 holding, per K half h, the
    // 32 columns each of Re_hi, Re_lo, Im_hi, Im_lo at 256 + 128 h. A K half of tile i
    // is converted once the MMAs of tile i - 1 that read it are done, so converting
    // one half overlaps the MMAs on the other.
    auto dcol_of = [&](int b) { return tmem + uint32_t(b) * (kTf32 ? 128u : 256u); };
    auto acol_of = [&](int b) { return kTf32 ? tmem + 256u : tmem + uint32_t(b) * 256u + 128u; };
    // The loader warps of K half h may overwrite their part of A for tile i once the
    // MMAs that read it for the previous tile in that buffer completed.
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
    // TMEM column of the A region for K half h (TF32) or the A_hi image (BF16).
    auto abase_of = [&](int b, int h) { return kTf32 ? acol_of(b) + 128u * uint32_t(h) : acol_of(b); };
    auto acol_in = [&](int h, int ch) { return kTf32 ? 16 * ch : 32 * h + 16 * ch; };
    // Splits 16 amplitudes (TMEM columns) of one slice and writes them to A.
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
    // Reads 16 output amplitudes (j = j0 .. j0 + 15) of one slice from D.
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

    const uint32_t rmask = (1u << a.r) - 1u;
    const uint32_t stage0_u32 = smem_u32(sm + L::kStage0);
    if (warp < kLoaderWarps && !kStaged) {
        // ---------------------------------------------------------------- loaders (slice order)
        const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, amplitude half
        const int srow = 32 * q + lane;          // slice within the tile = TMEM lane
        // kSub: bit i of the slice index s sits on the i-th lowest non-target qubit p_i; its
        // place in the sub-state is c(p_i) = the rank of p_i in tmask, or none (the slice is
        // then all zeros). The 7 row bits of this thread's slice are folded once here; tile
        // bit L is this lane's job for lane L, combined over the warp per tile.
        uint64_t row_cb = 0;
        bool row_z = false;
        int lane_c = -1;
        if constexpr (kSub) {
            auto place = [&](int pos) {
                return ((a.tmask >> pos) & 1ull) ? __popcll(a.tmask & ((1ull << pos) - 1ull)) : -1;
            };
            for (int qb = 0, i = 0; qb < 64 && i < 7 + 32; ++qb) {
                bool tgt = false;
#pragma unroll
                for (int x = 0; x < K; ++x) tgt |= (t[x] == qb);
                if (tgt) continue;
                const int c = place(qb);
                if (i < 7) {
                    if ((srow >> i) & 1) {
                        if (c < 0) row_z = true;
                        else row_cb |= 1ull << c;
                    }
                } else if (i - 7 == lane) {
                    lane_c = c;
                }
                ++i;
            }
        }
        // kSub: bit j of jnz = amplitude j of a slice can be nonzero (its target bits keep it in
        // the sub-state). The others are 0 in every tile, so their stage entries and tensor-memory
        // columns are written with zeros once here and never copied or converted again: a pass that
        // admits x qubits copies and converts 2^-x of a normal pass's amplitudes.
        uint64_t jnz = ~0ull;
        if constexpr (kSub) {
            jnz = 0;
            for (int j = 0; j < D; ++j)
                if (hi_off[j] != ~0ull) jnz |= 1ull << j;
            float2 *stz = reinterpret_cast<float2 *>(sm + L::kStage0);
            for (int b = 0; b < 2; ++b)
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = 32 * h + jj;
                    if (!((jnz >> j) & 1ull)) stz[b * (kStageBytes / 8) + j * M + srow] = make_float2(0.f, 0.f);
                }
            float2 zero16[16];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) zero16[jj] = make_float2(0.f, 0.f);
            for (int b = 0; b < 2; ++b)
                for (int ch = 0; ch < 2; ++ch)
                    if (((jnz >> (32 * h + 16 * ch)) & 0xffffull) == 0)
                        put16(abase_of(b, h) + (uint32_t(32 * q) << 16), acol_in(h, ch), zero16);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        auto issue = [&](uint32_t i, int b) {
            const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(i) * gridDim.x;
            const uint64_t base = slice_base(tile * M + srow, t);
            if constexpr (kSub) {
                // a slice with a qubit outside the sub-state set is all zeros; otherwise amplitude
                // j is at compact index (row and tile parts of the slice) | pext(off[j]) unless
                // off[j] leaves the sub-state. Zeros come from copies of 0 source bytes (no read):
                // this keeps the loader paced like a normal pass (skipping them measured slower)
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
                    const int j = 32 * h + jj;
                    if (!((jnz >> j) & 1ull)) continue;  // zero in every tile, already in the stage
                    const uint64_t cj_sub = hi_off[j];
                    const bool zero = zslice || cj_sub == ~0ull;
                    const float2 *src = zero ? a.sub : a.sub + (cb | cj_sub);
                    const uint32_t nbytes = zero ? 0u : 8u;
                    const uint32_t dst = stage0_u32 + uint32_t(b * kStageBytes + (j * M + srow) * 8);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(nbytes)
                                 : "memory");
                }
            } else {
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = 32 * h + jj;
                    const float2 *src = a.psi + (base | off[j]);
                    const uint32_t dst = stage0_u32 + uint32_t(b * kStageBytes + (j * M + srow) * 8);
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if (my_tiles > 0) issue(0, 0);
        if (my_tiles > 1) issue(1, 1);
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (i + 1 < my_tiles) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (!wait_a_free(i, h)) break;
            tc_fence_after();
            const float2 *stage = reinterpret_cast<const float2 *>(sm + L::kStage0 + b * kStageBytes);
            const uint32_t abase = abase_of(b, h) + (uint32_t(32 * q) << 16);
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {  // 16 amplitudes (TMEM columns) at a time
                if (((jnz >> (32 * h + 16 * ch)) & 0xffffull) == 0) continue;  // kSub: zero columns
                float2 v[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] = stage[(32 * h + 16 * ch + jj) * M + srow];
                put16(abase, acol_in(h, ch), v);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full_h(b, h));
            if (i + 2 < my_tiles) issue(i + 2, b);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < kLoaderWarps) {
        // ---------------------------------------------------------------- loaders (memory order)
        const int q = warp & 3, h = warp >> 2;
        const int srow = 32 * q + lane;
        auto issue = [&](uint32_t i, int b) {
            const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(i) * gridDim.x;
            const uint64_t tbase = slice_base(tile * M, t);
#pragma unroll 8
            for (int it = 0; it < 32; ++it) {
                const uint32_t c = uint32_t((it * kLoaderWarps + warp) * 32 + lane);
                const float2 *src = a.psi + (tbase | (c & rmask) | hi_off[c >> a.r]);
                const uint32_t dst = stage0_u32 + uint32_t(b * kStageBytes) + swz(c) * 8u;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
            }
            // arrives on the stage's barrier once this thread's copies have landed
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar_loaded(b)) : "memory");
        };
        if (my_tiles > 0) issue(0, 0);
        if (my_tiles > 1) issue(1, 1);
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<!kTf32>(bar_loaded(b), (i >> 1) & 1, abort_flag, lim)) break;
            if (!wait_a_free(i, h)) break;
            tc_fence_after();
            const float2 *stage = reinterpret_cast<const float2 *>(sm + L::kStage0 + b * kStageBytes);
            const uint32_t csr = cs[srow];
            const uint32_t abase = abase_of(b, h) + (uint32_t(32 * q) << 16);
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                float2 v[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] = stage[swz(uint32_t(cj[32 * h + 16 * ch + jj]) | csr)];
                put16(abase, acol_in(h, ch), v);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_full_h(b, h));
            // the other stage takes tile i+1 once tile i-1's outputs have been stored from
            // it (tiles 0 and 1 were issued up front); converting tile i first keeps its
            // MMA and epilogue running while tile i+1 is in flight
            if (i >= 1 && i + 1 < my_tiles) {
                if (!warp_wait<!kTf32>(bar_sfree(b ^ 1), ((i - 1) >> 1) & 1, abort_flag, lim)) break;
                issue(i + 1, b ^ 1);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < kLoaderWarps + kEpiWarps && !kStaged) {
        // ---------------------------------------------------------------- epilogue (slice order)
        const int e = warp - kLoaderWarps;
        const int q = e & 3, h = e >> 2;
        const int srow = 32 * q + lane;
        // Lowest target on index bit 0: the thread writes amplitudes j and j+1 of its slice
        // (adjacent) as one 16-byte store. On bit 1: index bit 0 is the lowest slice bit, and
        // lane pairs swap one amplitude so that each lane writes two adjacent slices of one j
        // (the even lane j, the odd lane j+1). Either way a store instruction covers 512
        // contiguous bytes; otherwise 8-byte stores already fill whole 32-byte sectors.
        const int smode = t[0] == 0 ? 1 : (t[0] == 1 ? 2 : 0);
        const bool odd = lane & 1;
        auto st16 = [](float2 *p, float2 x, float2 y) {
            asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y)
                         : "memory");
        };
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<!kTf32>(bar_done(b), (i >> 1) & 1, abort_flag, lim)) break;
            tc_fence_after();
            const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(i) * gridDim.x;
            const uint64_t base = slice_base(tile * M + srow, t);
            const uint32_t dbase = dcol_of(b) + (uint32_t(32 * q) << 16);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float2 v[16];
                get16(dbase, 32 * h + 16 * c, v);
                const int j0 = 32 * h + 16 * c;
                if (smode == 1) {
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 2) st16(a.psi + (base | off[j0 + jj]), v[jj], v[jj + 1]);
                } else if (smode == 2) {
                    const uint64_t pbase = base & ~1ull;  // the even slice of the lane pair
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 2) {
                        // selects, not branches: one 16-byte store instruction for the whole warp
                        const float2 send = odd ? v[jj] : v[jj + 1];
                        const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                                        __shfl_xor_sync(0xffffffffu, send.y, 1));
                        const float2 x = odd ? recv : v[jj], y = odd ? v[jj + 1] : recv;
                        st16(a.psi + (pbase | off[j0 + jj + (odd ? 1 : 0)]), x, y);
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) a.psi[base | off[j0 + jj]] = v[jj];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_free(b));
        }
    } else if (warp < kLoaderWarps + kEpiWarps) {
        // ---------------------------------------------------------------- epilogue (memory order)
        const int e = warp - kLoaderWarps;
        const int q = e & 3, h = e >> 2;
        const int srow = 32 * q + lane;
        const uint32_t csr = cs[srow];
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<!kTf32>(bar_done(b), (i >> 1) & 1, abort_flag, lim)) break;
            tc_fence_after();
            float2 *stage = reinterpret_cast<float2 *>(sm + L::kStage0 + b * kStageBytes);
            const uint32_t dbase = dcol_of(b) + (uint32_t(32 * q) << 16);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float2 v[16];
                get16(dbase, 32 * h + 16 * c, v);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) stage[swz(uint32_t(cj[32 * h + 16 * c + jj]) | csr)] = v[jj];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar_free(b));
                mbar_arrive(bar_outready(b));
            }
            if (!warp_wait<!kTf32>(bar_outready(b), (i >> 1) & 1, abort_flag, lim)) break;
            const uint64_t tile = uint64_t(blockIdx.x) + uint64_t(i) * gridDim.x;
            const uint64_t tbase = slice_base(tile * M, t);
#pragma unroll 8
            for (int it = 0; it < 32; ++it) {
                const uint32_t c = uint32_t((it * kEpiWarps + e) * 32 + lane);
                a.psi[tbase | (c & rmask) | hi_off[c >> a.r]] = stage[swz(c)];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_sfree(b));
        }
    } else {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t bimg = smem_u32(sm);
            uint32_t last_bar = 0, last_par = 0;  // the most recent commit, for the drain
            bool committed = false;
            auto commit = [&](uint32_t bar, uint32_t par) {
                mma_commit(bar);
                last_bar = bar;
                last_par = par;
                committed = true;
            };
            for (uint32_t i = 0; i < my_tiles; ++i) {
                const int b = i & 1;
                const uint32_t par = (i >> 1) & 1;
                if (!mbar_wait<!kTf32>(bar_full(b), par, abort_flag, lim)) break;
                if (i >= 2 && !mbar_wait<!kTf32>(bar_free(b), ((i >> 1) - 1) & 1, abort_flag, lim)) break;
                // test hook: nothing issued or committed for this tile, so every wait on it runs out
                if (blockIdx.x == 0 && int(i) == a.skip_tile) continue;
                tc_fence_after();
                const uint32_t dcol = dcol_of(b), acol = acol_of(b);
                if constexpr (kTf32) {
                    // D[:, 0:64] += X_re Ur^T - X_im Ui^T and D[:, 64:128] += X_re Ui^T + X_im Ur^T:
                    // B1 = [Ur; Ui] for the Re inputs, B2 = [-Ui; Ur] for the Im inputs, both
                    // 128-row windows of one [-Ui; Ur; Ui] image per split.
                    auto half = [&](int hh) {
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            const int kk = 4 * hh + k4;
                            // K step kk covers inputs [8 kk, 8 kk + 8): atom column kk / 4, 32-byte step kk % 4
                            const uint32_t kof = uint32_t(hh) * uint32_t(kTf32Atom) + uint32_t(k4) * 32u;
                            const uint32_t hi = bimg + kof, lo = bimg + uint32_t(kTf32Split) + kof;
                            const uint64_t b1h = sw128_desc(hi + 64u * 128u), b1l = sw128_desc(lo + 64u * 128u);
                            const uint64_t b2h = sw128_desc(hi), b2l = sw128_desc(lo);
                            // A columns of this K step: Re_hi, Re_lo (+32), Im_hi (+64), Im_lo (+96)
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
                    if (!mbar_wait<!kTf32>(bar_full1(b), par, abort_flag, lim)) break;
                    tc_fence_after();
                    half(1);
                } else {
                    const uint32_t bhi = bimg + uint32_t(kSmBhi), blo = bimg + uint32_t(kSmBlo);
#pragma unroll
                    for (int kk = 0; kk < KR / 16; ++kk) {
                        // K step kk covers reals [16 kk, 16 kk + 16): atom column kk / 4, 32-byte step kk % 4
                        const uint32_t boff = uint32_t(kk >> 2) * uint32_t(NR * 128) + uint32_t(kk & 3) * 32u;
                        const uint64_t dhi = sw128_desc(bhi + boff), dlo = sw128_desc(blo + boff);
                        const uint32_t ac = acol + uint32_t(kk) * 8u;  // 16 bf16 = 8 TMEM columns
                        mma_bf16_tmemA(dcol, ac, dhi, kk > 0 ? 1u : 0u);
                        mma_bf16_tmemA(dcol, ac + 64u, dhi, 1u);
                        mma_bf16_tmemA(dcol, ac, dlo, 1u);
                    }
                }
                commit(bar_done(b), par);
            }
            if (*abort_flag && committed) {
                // drain: the last committed MMAs must finish before tensor memory is freed
                const long long t0 = clock64();
                while (!mbar_try_wait(last_bar, last_par) && clock64() - t0 < lim) {
                }
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicOr(a.err, 8);
    if (warp == kLoaderWarps + kEpiWarps) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- host side

namespace {
std::atomic<long long> g_tc_wait_cycles{kTcWaitCycles};
std::atomic<int> g_tc_skip_tile{-1};
}  // namespace

void tc_test_fault(long long *wait_cycles, int *skip_tile) {
    *wait_cycles = g_tc_wait_cycles.load();
    *skip_tile = g_tc_skip_tile.load();
}

void tc_set_test_fault(int skip_tile, long long wait_cycles) {
    g_tc_skip_tile.store(skip_tile < 0 ? -1 : skip_tile);
    g_tc_wait_cycles.store(wait_cycles > 0 ? wait_cycles : kTcWaitCycles);
}

static uint16_t bf16_rn_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return uint16_t((u >> 16) | 0x40);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}
static float bf16_to_float(uint16_t b) {
    uint32_t u = uint32_t(b) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

size_t tc_ops_bytes(bool tf32) {
    return size_t(tf32 ? tc::Layout<true>::kBBytes : tc::Layout<false>::kBBytes);
}

// Byte offset of element (row n, k) in the K-major, 128-byte-swizzled image of a
// 128 x 128 bf16 operand: two 64-element atom columns of 128 rows x 128 bytes;
// within a row the 16-byte chunk c sits at chunk c ^ (n mod 8).
static size_t sw128_offset(int n, int k) {
    const int kc = k >> 6, within = (k & 63) * 2;
    const int chunk = within >> 4, byte = within & 15;
    return size_t(kc) * (tc::NR * 128) + size_t(n) * 128 + size_t(((chunk ^ (n & 7)) << 4) + byte);
}

// The same for the 192 x 64 tf32 image: two 32-element atom columns of 192 rows.
static size_t sw128_offset_tf32(int n, int k) {
    const int kc = k >> 5, within = (k & 31) * 4;
    const int chunk = within >> 4, byte = within & 15;
    return size_t(kc) * tc::kTf32Atom + size_t(n) * 128 + size_t(((chunk ^ (n & 7)) << 4) + byte);
}

// Round to nearest (ties away from zero) at 10 stored mantissa bits, kept as an fp32
// bit pattern with the low 13 bits clear: the tf32 value the tensor cores read.
static uint32_t tf32_rna_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u & 0xffffe000u;  // Inf / NaN: truncate
    return (u + 0x1000u) & 0xffffe000u;
}
static float bits_to_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static void build_ops_bf16(const Pass &p, uint8_t *img) {
    using namespace tc;
    for (int oa = 0; oa < D; ++oa)
        for (int ib = 0; ib < D; ++ib) {
            const cd u = p.U[size_t(oa) * D + ib];
            // R rows 2oa (re out), 2oa+1 (im out); columns 2ib (re in), 2ib+1 (im in)
            const double r[2][2] = {{u.real(), -u.imag()}, {u.imag(), u.real()}};
            for (int ro = 0; ro < 2; ++ro)
                for (int ci = 0; ci < 2; ++ci) {
                    const double v = r[ro][ci];
                    const uint16_t h = bf16_rn_bits(float(v));
                    const uint16_t l = bf16_rn_bits(float(v - double(bf16_to_float(h))));
                    const size_t o = sw128_offset(2 * oa + ro, 2 * ib + ci);
                    std::memcpy(img + kSmBhi + o, &h, 2);
                    std::memcpy(img + kSmBlo + o, &l, 2);
                }
        }
}

static void build_ops_tf32(const Pass &p, uint8_t *img) {
    using namespace tc;
    for (int oa = 0; oa < D; ++oa)
        for (int ib = 0; ib < D; ++ib) {
            const cd u = p.U[size_t(oa) * D + ib];
            // rows 0..63: -Im U, rows 64..127: Re U, rows 128..191: Im U
            const double v[3] = {-u.imag(), u.real(), u.imag()};
            for (int blk = 0; blk < 3; ++blk) {
                const uint32_t h = tf32_rna_bits(float(v[blk]));
                const uint32_t l = tf32_rna_bits(float(v[blk] - double(bits_to_float(h))));
                const size_t o = sw128_offset_tf32(blk * D + oa, ib);
                std::memcpy(img + o, &h, 4);
                std::memcpy(img + kTf32Split + o, &l, 4);
            }
        }
}

void tc_build_ops(const Pass &p, void *host_image, bool tf32) {
    uint8_t *img = static_cast<uint8_t *>(host_image);
    std::memset(img, 0, tc_ops_bytes(tf32));
    if (tf32) build_ops_tf32(p, img);
    else build_ops_bf16(p, img);
}

template <bool kStaged, bool kTf32, bool kSub = false>
static int set_smem_attr() {
    const cudaError_t e = cudaFuncSetAttribute(k_fused_tc<kStaged, kTf32, kSub>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Layout<kTf32>::kAlloc);
    return e == cudaSuccess ? RCS_OK : note_launch_error("tensor-core kernel shared-memory attribute", e);
}

int tc_prepare_device() {
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && attr_done[dev]) return RCS_OK;
    int rc = set_smem_attr<false, false>();
    if (rc == RCS_OK) rc = set_smem_attr<true, false>();
    if (rc == RCS_OK) rc = set_smem_attr<false, true>();
    if (rc == RCS_OK) rc = set_smem_attr<true, true>();
    if (rc == RCS_OK) rc = set_smem_attr<false, false, true>();
    if (rc == RCS_OK) rc = set_smem_attr<false, true, true>();
    if (rc == RCS_OK && dev >= 0 && dev < 64) attr_done[dev] = true;
    return rc;
}

static int launch_tc(void *psi, int n, const Pass &p, const void *d_ops, int *d_err, void *stream, bool tf32,
                     const void *sub, uint64_t tmask) {
    using namespace tc;
    if (p.k != K || n < K + 7) return RCS_ERR_UNSUPPORTED;
    if (int rc = tc_prepare_device(); rc != RCS_OK) return rc;
    TcArgs a;
    a.psi = static_cast<float2 *>(psi);
    a.sub = static_cast<const float2 *>(sub);
    a.tmask = tmask;
    a.ops = static_cast<const uint4 *>(d_ops);
    a.err = d_err;
    tc_test_fault(&a.wait_cycles, &a.skip_tile);
    a.tiles = uint32_t((1ull << (n - K)) / M);
    for (int i = 0; i < K; ++i) a.t[i] = p.t[i];
    // qubits varying inside a tile: the targets plus the 7 lowest other qubits
    uint64_t V = 0;
    for (int i = 0; i < K; ++i) V |= 1ull << p.t[i];
    for (int qb = 0, k = 0; qb < n && k < 7; ++qb)
        if (!((V >> qb) & 1) && !(std::find(p.t, p.t + K, qb) != p.t + K)) {
            V |= 1ull << qb;
            ++k;
        }
    a.vmask = V;
    a.r = 0;
    while (a.r < 64 && ((V >> a.r) & 1)) ++a.r;
    const unsigned grid = unsigned(std::min<uint64_t>(a.tiles, uint64_t(device_sm_count())));
    // With no target below qubit 5 the 32 slices of a warp sit side by side in memory and the
    // slice-order variant streams at full rate. With 4 or more targets below qubit 5 every slice is
    // a short contiguous run and the memory-order variant is faster (158 -> 79 ms for targets 0..5
    // at 34 qubits); for fewer low targets the slice-order variant measured faster.
    int low = 0;
    for (int i = 0; i < K; ++i) low += p.t[i] < 5;
    const bool staged = low >= 4;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (sub) {
        if (staged) return RCS_ERR_UNSUPPORTED;  // the sub-state input has a slice-order loader only
        if (tf32) k_fused_tc<false, true, true><<<grid, kThreads, Layout<true>::kAlloc, st>>>(a);
        else k_fused_tc<false, false, true><<<grid, kThreads, Layout<false>::kAlloc, st>>>(a);
    } else if (tf32) {
        if (staged) k_fused_tc<true, true, false><<<grid, kThreads, Layout<true>::kAlloc, st>>>(a);
        else k_fused_tc<false, true, false><<<grid, kThreads, Layout<true>::kAlloc, st>>>(a);
    } else {
        if (staged) k_fused_tc<true, false, false><<<grid, kThreads, Layout<false>::kAlloc, st>>>(a);
        else k_fused_tc<false, false, false><<<grid, kThreads, Layout<false>::kAlloc, st>>>(a);
    }
    return launch_status("tensor-core pass");
}

int launch_pass_tc(void *psi, int n, const Pass &p, const void *d_ops, int *d_err, void *stream, bool tf32) {
    return launch_tc(psi, n, p, d_ops, d_err, stream, tf32, nullptr, 0);
}

bool tc_pass_takes_substate(const Pass &p, int n) {
    int low = 0;
    for (int i = 0; i < tc::K; ++i) low += p.t[i] < 5;
    return p.kind == PASS_TC && p.k == tc::K && n >= tc::K + 7 && low < 4;
}

int launch_pass_tc_from_sub(void *psi, int n, const Pass &p, const void *d_ops, int *d_err, void *stream, bool tf32,
                            const void *sub, uint64_t tmask) {
    if (!sub) return RCS_ERR_ARG;
    return launch_tc(psi, n, p, d_ops, d_err, stream, tf32, sub, tmask);
}

}  // namespace rcs
