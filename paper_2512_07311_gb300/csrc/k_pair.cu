// Two consecutive fused 6-qubit unitaries in one HBM round trip, on the tcgen05 tensor
// cores (BF16 hi/lo split of both operands, three products, FP32 accumulate).
//
// Every full-state pass of the tensor-core path already streams the state at about the
// HBM copy rate, so the time of a circuit is set by how many times the state crosses
// HBM. This kernel applies U2 U1 for two consecutive passes of a plan (targets T1, T2,
// 6 each) per crossing. It works on tiles of 2^13 amplitudes: the index bits of a tile
// are V = T1 u T2 plus the lowest other bits (|V| = 13; index bit 0 is always in V), so
// both unitaries act inside it. For U1 a tile is 128 slices of 64 amplitudes (slice bits
// V \ T1, local index over T1, both in ascending bit order); for U2 the same amplitudes
// regroup into 128 slices over V \ T2.
//
// Each GEMM uses the complex block form with the state as the A operand in tensor
// memory: D_re = Xr Ur^T - Xi Ui^T and D_im = Xr Ui^T + Xi Ur^T (128 slices x 64 outputs
// each), where Xr, Xi hold the real and imaginary parts of the inputs. The four B images
// Ur, Ui (hi and lo splits, 64 x 64 bf16 each, 32 KB per unitary) serve every term: the
// -Ui terms set the MMA's negate-B bit. Split precision as in the single-pass kernel:
// X_hi B_hi + X_lo B_hi + X_hi B_lo per product, 48 MMAs of M = 128, N = 64, K = 16 per
// GEMM.
//
// Data flow per CTA (persistent, one CTA per SM, 17 warps):
//   warps 0-3   (loaders): 16-byte cp.async copies of a tile in memory order into a
//               swizzled stage (two 64 KB stages); then each thread converts its U1
//               slice row (bf16 hi/lo) into the four A planes Xr_hi, Xr_lo, Xi_hi, Xi_lo in
//               tensor memory. The stage is free again right after the conversion, so
//               the copies of tile i+2 start while tile i is still in the tensor memory.
//   warp 16     (MMA): GEMM 1 of the oldest tile whose U1 operand is ready and whose D
//               buffer is free, or GEMM 2 of the oldest tile whose U2 operand is ready,
//               whichever is ready first.
//   warps 4-11  (middle): after GEMM 1, regroup the tile for U2 through a 32 KB buffer
//               in two halves (split on the tile's highest bit): read D1 (FP32) from
//               tensor memory, split into (hi, lo) bf16x2 words at U2 positions, then read
//               them back in U2 order into the A planes of the tile's tensor-memory buffer.
//   warps 12-15 (epilogue): after GEMM 2, D2 -> global memory in U2 slice order (16-byte
//               stores where the lowest index bit allows).
// Tensor memory: two buffers of {D: 128 columns, A: 128 columns}.
//
// Numerically each unitary sees what a single pass gives it: the input split into bf16
// hi/lo from FP32 values, the same products, FP32 accumulation; only the order of the
// FP32 accumulation differs from the single-pass kernel's realified form.
//
// Every wait is bounded; on expiry the kernel raises an error bit, drains its MMAs and
// copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <bit>
#include <cstring>

#include "dev_common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace rcs {

namespace pr {
constexpr int K = kTcK;                    // 6 targets per unitary
constexpr int D = 1 << K;                  // 64 amplitudes per slice
constexpr int M = 128;                     // slices per GEMM (tensor-memory lanes)
constexpr int kBits = 13;                  // a tile is 2^13 amplitudes
constexpr int kAmps = 1 << kBits;
constexpr int kLoaderWarps = 4;            // one per tensor-memory lane quarter
constexpr int kMidWarps = 8;               // lane quarter x half of the local indices
constexpr int kEpiWarps = 4;               // one per lane quarter
constexpr int kMmaWarp = kLoaderWarps + kMidWarps + kEpiWarps;
constexpr int kThreads = (kMmaWarp + 1) * 32;  // 544
constexpr int kCopyIters = kAmps / 2 / (kLoaderWarps * 32);  // 32 copies of 16 bytes per loader thread and tile
constexpr int kMatBytes = D * 128;         // one 64 x 64 bf16 image, 128-byte rows: 8 KB
constexpr int kOpBytes = 4 * kMatBytes;    // Ur_hi, Ui_hi, Ur_lo, Ui_lo: 32 KB per unitary
constexpr int kStageBytes = kAmps * 8;     // one tile of complex64: 64 KB
constexpr int kHalfBytes = kStageBytes / 2;  // the regrouping buffer: half a tile of (hi, lo) words
// shared-memory map (offsets from a 1024-aligned base)
constexpr int kStage0 = 2 * kOpBytes;            // U1 image, U2 image, then two stages
constexpr int kMid = kStage0 + 2 * kStageBytes;  // the regrouping buffer
constexpr int kHiP = kMid + kHalfBytes;          // 32 u64: global offset of compact bits 8..12 (copy iteration)
constexpr int kOff2 = kHiP + 32 * 8;             // 64 u64: global offset of U2 local index j
constexpr int kAj = kOff2 + 64 * 8;              // 64 u16: raw-stage position part of U1 local index j
constexpr int kQj = kAj + D * 2;                 // 64 u16: regrouping position part of U1 local index j
constexpr int kBar = kQj + D * 2;                // 16 mbarriers
constexpr int kMisc = kBar + 16 * 8;             // tensor-memory slot, abort flag
constexpr int kAlloc = kMisc + 16 + 1024;        // slack for the 1024-byte alignment
static_assert(kAlloc <= 227 * 1024, "shared memory");
static_assert(kBar % 8 == 0, "mbarrier alignment");
constexpr uint32_t kTmemCols = 512;
// instruction descriptor: D f32, A bf16, B bf16, both K-major, N = 64, M = 128; bit 14 negates B
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(64 >> 3) << 17) | (uint32_t(M >> 4) << 24);
constexpr uint32_t kIdescNegB = kIdesc | (1u << 14);
}  // namespace pr

struct PairArgs {
    float2 *psi;
    const uint4 *ops1;  // image of U1 (32 KB, shared-memory layout)
    const uint4 *ops2;  // image of U2
    int *err;
    uint32_t tiles;     // 2^(n - 13)
    int n;
    int t1[pr::K];      // ascending targets of U1
    int t2[pr::K];      // ascending targets of U2
    uint64_t vmask;     // the 13 index bits of a tile
    long long wait_cycles;  // limit of every wait (SM clock cycles)
    int skip_tile;          // test hook: CTA 0 runs no GEMM 1 for its tile skip_tile (-1: none)
};

namespace {

// Position (8-byte units) of compact tile index c in the stage while it holds the raw
// tile: XOR-swizzles bits 6..8 into bits 1..3, which keeps the two amplitudes of a
// 16-byte copy (c, c ^ 1) together. Linear over GF(2): the position of c = a | b
// (disjoint bits) is swz_raw(a) ^ swz_raw(b).
__device__ __forceinline__ uint32_t swz_raw(uint32_t c) { return c ^ (((c >> 6) & 7u) << 1); }

// Compact position of index bit b inside mask V.
__device__ __forceinline__ int cpos_of(uint64_t V, int b) { return __popcll(V & ((1ull << b) - 1ull)); }

// Scatters the low bits of x onto the set bits of mask, lowest first.
__device__ __forceinline__ uint64_t pdep64(uint64_t x, uint64_t mask) {
    uint64_t r = 0;
    for (int k = 0; mask; ++k) {
        const uint64_t bit = mask & (~mask + 1ull);
        if ((x >> k) & 1ull) r |= bit;
        mask ^= bit;
    }
    return r;
}
// Gathers the bits of x at the set bits of mask into the low bits, lowest first.
__device__ __forceinline__ uint32_t pext32(uint32_t x, uint32_t mask) {
    uint32_t r = 0;
    for (int k = 0; mask; ++k) {
        const uint32_t bit = mask & (~mask + 1u);
        if (x & bit) r |= 1u << k;
        mask ^= bit;
    }
    return r;
}

// Position in the regrouping buffer of the amplitude with compact index c: its U2 slice
// s2 and local index j2 with the split bit (the tile's highest bit) left out, then an
// XOR fold of the j2 part into the low bits. The split bit is local-index bit 5 of U2
// when it is a U2 target (form 1), else slice bit 6 (form 2). Linear in c.
__device__ __forceinline__ uint32_t mid_pos(uint32_t c, uint32_t s2c, uint32_t t2c, bool form1) {
    const uint32_t s2 = pext32(c, s2c), j2 = pext32(c, t2c);
    if (form1) {
        const uint32_t p = ((j2 & 31u) << 7) | s2;
        return p ^ (p >> 7);
    }
    const uint32_t p = (j2 << 6) | (s2 & 63u);
    return p ^ (p >> 6);
}
// The same for U2 slice row s2 and local index j2 directly (the split bit already fixed).
__device__ __forceinline__ uint32_t mid_pos_rj(uint32_t s2, uint32_t j2, bool form1) {
    if (form1) {
        const uint32_t p = ((j2 & 31u) << 7) | s2;
        return p ^ (p >> 7);
    }
    const uint32_t p = (j2 << 6) | (s2 & 63u);
    return p ^ (p >> 6);
}

// (re, im) hi and lo words of two neighbouring amplitudes -> one column of the Xr and
// Xi planes (bf16x2: the even local index in the low half).
__device__ __forceinline__ uint32_t lo_halves(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5410); }
__device__ __forceinline__ uint32_t hi_halves(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x7632); }

// Writes 16 amplitudes' (re, im) hi and lo words, local indices j0 .. j0+15 (j0 even),
// into the four A planes of one slice row: Xr_hi at column 0, Xr_lo at 32, Xi_hi at 64,
// Xi_lo at 96 (plus j0 / 2).
__device__ __forceinline__ void put_planes(uint32_t arow, int j0, const uint32_t (&hi)[16], const uint32_t (&lo)[16]) {
    uint32_t xr[8], xi[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        xr[m] = lo_halves(hi[2 * m], hi[2 * m + 1]);
        xi[m] = hi_halves(hi[2 * m], hi[2 * m + 1]);
    }
    tmem_st8(arow + uint32_t(j0 / 2), xr);
    tmem_st8(arow + 64u + uint32_t(j0 / 2), xi);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        xr[m] = lo_halves(lo[2 * m], lo[2 * m + 1]);
        xi[m] = hi_halves(lo[2 * m], lo[2 * m + 1]);
    }
    tmem_st8(arow + 32u + uint32_t(j0 / 2), xr);
    tmem_st8(arow + 96u + uint32_t(j0 / 2), xi);
}

// The 48 MMAs of one GEMM: D_re = Xr Ur^T - Xi Ui^T, D_im = Xr Ui^T + Xi Ur^T, three split
// products each. img: Ur_hi, Ui_hi, Ur_lo, Ui_lo images, 8 KB apart.
__device__ __forceinline__ void gemm_cx(uint32_t img, uint32_t dcol, uint32_t acol) {
    using namespace pr;
    const uint32_t dre = dcol, dim = dcol + 64u;
#pragma unroll 1
    for (int kk = 0; kk < D / 16; ++kk) {
        // K step kk covers inputs [16 kk, 16 kk + 16): 32 bytes into each 128-byte image row
        const uint32_t ko = uint32_t(kk) * 32u;
        const uint64_t ur_h = sw128_desc(img + ko), ui_h = sw128_desc(img + uint32_t(kMatBytes) + ko);
        const uint64_t ur_l = sw128_desc(img + 2u * kMatBytes + ko), ui_l = sw128_desc(img + 3u * kMatBytes + ko);
        const uint32_t xr_hi = acol + uint32_t(kk) * 8u, xr_lo = xr_hi + 32u, xi_hi = xr_hi + 64u, xi_lo = xr_hi + 96u;
        const uint32_t acc = kk > 0 ? 1u : 0u;
        mma_f16_tmemA(dre, xr_hi, ur_h, kIdesc, acc);
        mma_f16_tmemA(dre, xr_lo, ur_h, kIdesc, 1u);
        mma_f16_tmemA(dre, xr_hi, ur_l, kIdesc, 1u);
        mma_f16_tmemA(dre, xi_hi, ui_h, kIdescNegB, 1u);
        mma_f16_tmemA(dre, xi_lo, ui_h, kIdescNegB, 1u);
        mma_f16_tmemA(dre, xi_hi, ui_l, kIdescNegB, 1u);
        mma_f16_tmemA(dim, xr_hi, ui_h, kIdesc, acc);
        mma_f16_tmemA(dim, xr_lo, ui_h, kIdesc, 1u);
        mma_f16_tmemA(dim, xr_hi, ui_l, kIdesc, 1u);
        mma_f16_tmemA(dim, xi_hi, ur_h, kIdesc, 1u);
        mma_f16_tmemA(dim, xi_lo, ur_h, kIdesc, 1u);
        mma_f16_tmemA(dim, xi_hi, ur_l, kIdesc, 1u);
    }
}

}  // namespace

// Roles (17 warps): 0-3 loaders, 4-11 middle, 12-15 epilogue, 16 MMA issuer.
__global__ void __launch_bounds__(pr::kThreads, 1) k_pair_tc(const __grid_constant__ PairArgs a) {
    using namespace pr;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint64_t *hip = reinterpret_cast<const uint64_t *>(sm + kHiP);
    const uint64_t *off2 = reinterpret_cast<const uint64_t *>(sm + kOff2);
    const uint16_t *aj = reinterpret_cast<const uint16_t *>(sm + kAj);
    const uint16_t *qj = reinterpret_cast<const uint16_t *>(sm + kQj);
    uint2 *mid = reinterpret_cast<uint2 *>(sm + kMid);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kMisc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + kMisc + 4);
    const uint32_t bar0 = smem_u32(sm + kBar);
    // per TMEM buffer b (tiles i with i % 2 = b); each completes once per such tile
    auto bar_loaded = [&](int b) { return bar0 + 8u * uint32_t(b); };         // stage b holds the raw tile
    auto bar_a1 = [&](int b) { return bar0 + 16u + 8u * uint32_t(b); };       // A holds the U1 operand; stage b free
    auto bar_done1 = [&](int b) { return bar0 + 32u + 8u * uint32_t(b); };    // GEMM 1 complete
    auto bar_a2 = [&](int b) { return bar0 + 48u + 8u * uint32_t(b); };       // A holds the U2 operand
    auto bar_done2 = [&](int b) { return bar0 + 64u + 8u * uint32_t(b); };    // GEMM 2 complete
    auto bar_dfree = [&](int b) { return bar0 + 80u + 8u * uint32_t(b); };    // D2 stored, D free
    // the regrouping buffer, twice per tile (half h): written, then read back
    const uint32_t bar_mw = bar0 + 96u, bar_mr = bar0 + 104u;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long lim = a.wait_cycles;
    const uint64_t V = a.vmask;
    // compact masks (tile bit positions) of the target and slice bits of each unitary
    uint32_t t1c = 0, t2c = 0;
    uint64_t t2m = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        t1c |= 1u << cpos_of(V, a.t1[i]);
        t2c |= 1u << cpos_of(V, a.t2[i]);
        t2m |= 1ull << a.t2[i];
    }
    const uint32_t all = (1u << kBits) - 1u;
    const uint32_t s1c = all & ~t1c, s2c = all & ~t2c;
    // the split bit is the tile's highest bit (compact bit 12): local-index bit 5 of a
    // unitary that targets it, else slice bit 6
    const bool split_t1 = (t1c >> 12) & 1u, split_t2 = (t2c >> 12) & 1u;

    // ---- set-up: operand images, tables, barriers, tensor memory
    {
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        for (int i = threadIdx.x; i < kOpBytes / 16; i += kThreads) {
            dst[i] = a.ops1[i];
            dst[kOpBytes / 16 + i] = a.ops2[i];
        }
        const int t = threadIdx.x;
        if (t < 32) {  // copy iteration t: compact bits 8..12 = t
            reinterpret_cast<uint64_t *>(sm + kHiP)[t] = pdep64(uint64_t(t) << 8, V);
        } else if (t >= 64 && t < 128) {
            reinterpret_cast<uint64_t *>(sm + kOff2)[t - 64] = pdep64(uint64_t(t - 64), t2m);
        } else if (t >= 128 && t < 128 + D) {
            const uint32_t j = t - 128;
            const uint32_t c = uint32_t(pdep64(j, t1c));  // compact index of U1 local index j
            reinterpret_cast<uint16_t *>(sm + kAj)[j] = uint16_t(swz_raw(c));
            reinterpret_cast<uint16_t *>(sm + kQj)[j] = uint16_t(mid_pos(c, s2c, t2c, split_t2));
        }
        if (threadIdx.x == 0) {
            for (int b = 0; b < 2; ++b) {
                mbar_init(bar_loaded(b), kLoaderWarps * 32);
                mbar_init(bar_a1(b), kLoaderWarps);
                mbar_init(bar_done1(b), 1);
                mbar_init(bar_a2(b), kMidWarps);
                mbar_init(bar_done2(b), 1);
                mbar_init(bar_dfree(b), kEpiWarps);
            }
            mbar_init(bar_mw, kMidWarps);
            mbar_init(bar_mr, kMidWarps);
            *abort_flag = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (warp == kMmaWarp) {
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
    auto dcol_of = [&](int b) { return tmem + uint32_t(b) * 256u; };
    auto acol_of = [&](int b) { return tmem + uint32_t(b) * 256u + 128u; };
    const uint32_t stage0 = smem_u32(sm + kStage0);
    auto tile_base = [&](uint32_t i) {  // the tile's index bits scattered onto the bits outside V
        uint64_t x = uint64_t(blockIdx.x) + uint64_t(i) * gridDim.x;
        uint64_t m = V;
        while (m) {
            const int b = __ffsll(static_cast<long long>(m)) - 1;
            x = insert_zero(x, b);
            m &= m - 1ull;
        }
        return x;
    };

    if (warp < kLoaderWarps) {
        // ---------------------------------------------------------------- loaders
        const int q = warp;
        const int srow = 32 * q + lane;  // U1 slice = tensor-memory lane
        const uint32_t pos_s = swz_raw(uint32_t(pdep64(uint64_t(srow), s1c)));  // raw-stage part of this slice
        // copies: thread t = 32 q + lane takes the amplitude pairs c = 256 it + 2 t, c + 1
        const uint32_t ct = uint32_t(2 * (32 * q + lane));
        const uint64_t cofs = pdep64(ct, V);  // global offset of compact bits 1..7
        const uint32_t cpos = swz_raw(ct);
        auto issue = [&](uint32_t i, int b) {
            const float2 *src0 = a.psi + (tile_base(i) | cofs);
            const uint32_t dst0 = stage0 + uint32_t(b * kStageBytes);
#pragma unroll 8
            for (int it = 0; it < kCopyIters; ++it) {
                // swz_raw(256 it) = 256 it ^ (((4 it) & 7) << 1)
                const uint32_t pos = cpos ^ ((uint32_t(it) * 256u) ^ (((uint32_t(it) * 4u) & 7u) << 1));
                const float2 *src = src0 + hip[it];
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + pos * 8u), "l"(src) : "memory");
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar_loaded(b)) : "memory");
        };
        if (my_tiles > 0) issue(0, 0);
        if (my_tiles > 1) issue(1, 1);
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<true>(bar_loaded(b), (i >> 1) & 1, abort_flag, lim)) break;
            if (i >= 2 && !warp_wait<true>(bar_done2(b), ((i - 2) >> 1) & 1, abort_flag, lim)) break;
            tc_fence_after();
            const float2 *stage = reinterpret_cast<const float2 *>(sm + kStage0 + b * kStageBytes);
            const uint32_t arow = acol_of(b) + (uint32_t(32 * q) << 16);
#pragma unroll 1
            for (int ch = 0; ch < 4; ++ch) {  // 16 inputs (local index 16 ch ..) at a time
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const float2 v = stage[pos_s ^ aj[16 * ch + jj]];
                    split_bf16x2(v, hi[jj], lo[jj]);
                }
                put_planes(arow, 16 * ch, hi, lo);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_a1(b));
            // this warp has read its part of stage b: once every loader warp has (bar_a1), the
            // stage takes tile i+2
            if (i + 2 < my_tiles) {
                if (!warp_wait<true>(bar_a1(b), (i >> 1) & 1, abort_flag, lim)) break;
                issue(i + 2, b);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp < kLoaderWarps + kMidWarps) {
        // ---------------------------------------------------------------- middle: U1 result -> U2 operand
        const int e = warp - kLoaderWarps;
        const int q = e & 3, hh = e >> 2;
        const int srow = 32 * q + lane;
        const uint32_t cs1 = uint32_t(pdep64(uint64_t(srow), s1c));
        const uint32_t pos_s1 = mid_pos(cs1, s2c, t2c, split_t2);  // this U1 slice's part of its positions
        const int rowhalf = srow >> 6;                             // slice bit 6 of this row (warp-uniform)
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<true>(bar_done1(b), (i >> 1) & 1, abort_flag, lim)) break;
            tc_fence_after();
            const uint32_t drow = dcol_of(b) + (uint32_t(32 * q) << 16);
            const uint32_t arow = acol_of(b) + (uint32_t(32 * q) << 16);
            bool ok = true;
            for (int h = 0; h < 2 && ok; ++h) {
                // write half h: the amplitudes whose split bit is h
                if (split_t1) {  // local-index bit 5 of U1: every thread, 16 of its inputs
                    const int j0 = 32 * h + 16 * hh;
                    uint32_t re[16], im[16];
                    tmem_ld16(drow + uint32_t(j0), re);
                    tmem_ld16(drow + 64u + uint32_t(j0), im);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        uint32_t whi, wlo;
                        split_bf16x2(make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj])), whi, wlo);
                        mid[pos_s1 ^ qj[j0 + jj]] = make_uint2(whi, wlo);
                    }
                } else if (rowhalf == h) {  // slice bit 6 of U1: the rows of half h, 32 inputs each
#pragma unroll 1
                    for (int ch = 0; ch < 2; ++ch) {
                        const int j0 = 32 * hh + 16 * ch;
                        uint32_t re[16], im[16];
                        tmem_ld16(drow + uint32_t(j0), re);
                        tmem_ld16(drow + 64u + uint32_t(j0), im);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            uint32_t whi, wlo;
                            split_bf16x2(make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj])), whi, wlo);
                            mid[pos_s1 ^ qj[j0 + jj]] = make_uint2(whi, wlo);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_mw);
                if (!warp_wait<true>(bar_mw, uint32_t(h), abort_flag, lim)) {
                    ok = false;
                    break;
                }
                // read half h back in U2 order
                if (split_t2) {  // local-index bit 5 of U2: every thread, 16 of its outputs' inputs
                    const int j0 = 32 * h + 16 * hh;
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const uint2 w = mid[mid_pos_rj(uint32_t(srow), uint32_t(j0 + jj), true)];
                        hi[jj] = w.x;
                        lo[jj] = w.y;
                    }
                    put_planes(arow, j0, hi, lo);
                } else if (rowhalf == h) {  // slice bit 6 of U2: the rows of half h, 32 each
#pragma unroll 1
                    for (int ch = 0; ch < 2; ++ch) {
                        const int j0 = 32 * hh + 16 * ch;
                        uint32_t hi[16], lo[16];
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) {
                            const uint2 w = mid[mid_pos_rj(uint32_t(srow), uint32_t(j0 + jj), false)];
                            hi[jj] = w.x;
                            lo[jj] = w.y;
                        }
                        put_planes(arow, j0, hi, lo);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_mr);
                if (!warp_wait<true>(bar_mr, uint32_t(h), abort_flag, lim)) {
                    ok = false;
                    break;
                }
            }
            if (!ok) break;
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_a2(b));
        }
    } else if (warp < kMmaWarp) {
        // ---------------------------------------------------------------- epilogue: D2 -> global memory
        const int q = warp - kLoaderWarps - kMidWarps;
        const int srow = 32 * q + lane;
        const uint64_t sb2 = pdep64(uint64_t(srow), V & ~t2m);  // this U2 slice's global offset
        // Lowest U2 target on index bit 0: amplitudes j, j+1 of a slice are adjacent (one
        // 16-byte store). On bit 1: index bit 0 is the lowest U2 slice bit, so lane pairs swap
        // one amplitude and each lane stores two adjacent slices of one j.
        const int smode = a.t2[0] == 0 ? 1 : (a.t2[0] == 1 ? 2 : 0);
        const bool odd = lane & 1;
        auto st16 = [](float2 *p, float2 x, float2 y) {
            asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x.x), "f"(x.y), "f"(y.x), "f"(y.y)
                         : "memory");
        };
        for (uint32_t i = 0; i < my_tiles; ++i) {
            const int b = i & 1;
            if (!warp_wait<true>(bar_done2(b), (i >> 1) & 1, abort_flag, lim)) break;
            tc_fence_after();
            float2 *const base = a.psi + (tile_base(i) | sb2);
            const uint32_t drow = dcol_of(b) + (uint32_t(32 * q) << 16);
#pragma unroll 1
            for (int ch = 0; ch < 2; ++ch) {  // 32 outputs (local index 32 ch ..) per tensor-memory round trip
                const int j0 = 32 * ch;
                uint32_t re[32], im[32];
                tmem_ld32(drow + uint32_t(j0), re);
                tmem_ld32(drow + 64u + uint32_t(j0), im);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (smode == 1) {
#pragma unroll
                    for (int jj = 0; jj < 32; jj += 2)
                        st16(base + off2[j0 + jj], make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj])),
                             make_float2(__uint_as_float(re[jj + 1]), __uint_as_float(im[jj + 1])));
                } else if (smode == 2) {
                    float2 *const pbase = reinterpret_cast<float2 *>(reinterpret_cast<uintptr_t>(base) & ~uintptr_t(15));
#pragma unroll
                    for (int jj = 0; jj < 32; jj += 2) {
                        const float2 v0 = make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj]));
                        const float2 v1 = make_float2(__uint_as_float(re[jj + 1]), __uint_as_float(im[jj + 1]));
                        const float2 send = odd ? v0 : v1;
                        const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 1),
                                                        __shfl_xor_sync(0xffffffffu, send.y, 1));
                        const float2 x = odd ? recv : v0, y = odd ? v1 : recv;
                        st16(pbase + off2[j0 + jj + (odd ? 1 : 0)], x, y);
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj)
                        base[off2[j0 + jj]] = make_float2(__uint_as_float(re[jj]), __uint_as_float(im[jj]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_dfree(b));
        }
    } else {
        // ---------------------------------------------------------------- MMA issuer
        // Two queues: GEMM 1 of tile n1 (needs its U1 operand and, two tiles back in the same
        // buffer, D stored) and GEMM 2 of tile n2 < n1 (needs its U2 operand). The issuer polls
        // both without blocking and issues whichever is ready, so neither waits behind the
        // other's hand-off. It gives up after the wait limit without progress.
        if (lane == 0) {
            const uint32_t img1 = smem_u32(sm), img2 = img1 + uint32_t(kOpBytes);
            uint32_t last_bar = 0, last_par = 0;
            bool committed = false;
            uint32_t n1 = 0, n2 = 0;
            long long t0 = clock64();
            while (n2 < my_tiles) {
                bool progress = false;
                if (n1 < my_tiles) {
                    const int b = n1 & 1;
                    const uint32_t par = (n1 >> 1) & 1;
                    if (blockIdx.x == 0 && int(n1) == a.skip_tile) {
                        // test hook: nothing issued or committed for this tile, so every wait on it
                        // runs out
                    } else if (mbar_test_wait(bar_a1(b), par) &&
                               (n1 < 2 || mbar_test_wait(bar_dfree(b), ((n1 - 2) >> 1) & 1))) {
                        tc_fence_after();
                        gemm_cx(img1, dcol_of(b), acol_of(b));
                        mma_commit(bar_done1(b));
                        last_bar = bar_done1(b);
                        last_par = par;
                        committed = true;
                        ++n1;
                        progress = true;
                    }
                }
                if (n2 < n1) {
                    const int b = n2 & 1;
                    const uint32_t par = (n2 >> 1) & 1;
                    if (mbar_test_wait(bar_a2(b), par)) {
                        tc_fence_after();
                        gemm_cx(img2, dcol_of(b), acol_of(b));
                        mma_commit(bar_done2(b));
                        last_bar = bar_done2(b);
                        last_par = par;
                        committed = true;
                        ++n2;
                        progress = true;
                    }
                }
                if (progress) {
                    t0 = clock64();
                } else {
                    if (*abort_flag) break;
                    if (clock64() - t0 > lim) {
                        *abort_flag = 1;
                        break;
                    }
                }
            }
            if (*abort_flag && committed) {
                // drain: the last committed MMAs must finish before tensor memory is freed
                const long long t1 = clock64();
                while (!mbar_try_wait(last_bar, last_par) && clock64() - t1 < lim) {
                }
            }
        }
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicOr(a.err, 8);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------- host side

namespace {

uint16_t bf16_rn_bits_host(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return uint16_t((u >> 16) | 0x40);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}
float bf16_value_host(uint16_t b) {
    const uint32_t u = uint32_t(b) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

size_t pair_ops_bytes() { return size_t(pr::kOpBytes); }

// Image of one unitary for k_pair_tc: four 64 x 64 bf16 matrices, 8 KB apart: Re U hi,
// Im U hi, Re U lo, Im U lo (row = output, K = input), each K-major with 128-byte swizzle:
// row r at byte 128 r, element k in 16-byte chunk (k / 8) XOR (r mod 8).
void pair_build_ops(const Pass &p, void *host_image) {
    using namespace pr;
    uint8_t *img = static_cast<uint8_t *>(host_image);
    std::memset(img, 0, kOpBytes);
    for (int o = 0; o < D; ++o)
        for (int b = 0; b < D; ++b) {
            const cd u = p.U[size_t(o) * D + b];
            const double v[2] = {u.real(), u.imag()};
            const size_t off = size_t(o) * 128 + size_t((((2 * b) >> 4) ^ (o & 7)) << 4) + size_t((2 * b) & 15);
            for (int part = 0; part < 2; ++part) {
                const uint16_t h = bf16_rn_bits_host(float(v[part]));
                const uint16_t l = bf16_rn_bits_host(float(v[part] - double(bf16_value_host(h))));
                std::memcpy(img + size_t(part) * kMatBytes + off, &h, 2);
                std::memcpy(img + size_t(2 + part) * kMatBytes + off, &l, 2);
            }
        }
}

bool pair_fits(const Pass &p1, const Pass &p2, int n) {
    return p1.kind == PASS_TC && p2.kind == PASS_TC && p1.k == pr::K && p2.k == pr::K && n >= pr::kBits;
}

int launch_pair_tc(void *psi, int n, const Pass &p1, const Pass &p2, const void *d_ops1, const void *d_ops2, int *d_err,
                   void *stream) {
    using namespace pr;
    if (!pair_fits(p1, p2, n)) return RCS_ERR_UNSUPPORTED;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(k_pair_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kAlloc);
        if (e != cudaSuccess) return note_launch_error("pair kernel shared-memory attribute", e);
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    PairArgs a;
    a.psi = static_cast<float2 *>(psi);
    a.ops1 = static_cast<const uint4 *>(d_ops1);
    a.ops2 = static_cast<const uint4 *>(d_ops2);
    a.err = d_err;
    a.n = n;
    a.tiles = uint32_t((1ull << n) >> kBits);
    uint64_t T = 0;
    for (int i = 0; i < K; ++i) {
        a.t1[i] = p1.t[i];
        a.t2[i] = p2.t[i];
        T |= (1ull << p1.t[i]) | (1ull << p2.t[i]);
    }
    // the tile: both target sets plus the lowest other bits
    uint64_t V = T;
    for (int b = 0; b < n && std::popcount(V) < kBits; ++b) V |= 1ull << b;
    a.vmask = V;
    tc_test_fault(&a.wait_cycles, &a.skip_tile);
    const unsigned grid = unsigned(std::min<uint64_t>(a.tiles, uint64_t(device_sm_count())));
    k_pair_tc<<<grid, kThreads, kAlloc, static_cast<cudaStream_t>(stream)>>>(a);
    return launch_status("tensor-core pair pass");
}

}  // namespace rcs
