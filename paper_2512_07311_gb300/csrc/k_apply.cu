// State-update kernels on FP32 SIMT cores.
//
//  * k_plain_1q / k_plain_2q: one launch per gate (the "plain FP32 per-gate"
//    baseline). Each thread moves 128-bit vectors: for a target above qubit 0,
//    two neighbouring pairs (quads) share one float4 per operand row; for a
//    target at qubit 0 the pair itself is one float4. HBM-bound: 16 * 2^n bytes
//    per gate against 8 (1q) or 16 (2q) real flop per amplitude, i.e. 0.5 or 1
//    flop per byte, far below the FP32 ridge.
//  * k_fused_simt<K>: one launch per fused K-qubit unitary (K <= 4). Thread =
//    one slice of 2^K amplitudes (the amplitudes that differ only in the target
//    bits); lanes of a warp take consecutive slices, so each load instruction
//    covers consecutive addresses along the lowest non-target qubits. The
//    unitary travels in the kernel's parameter space (constant bank) and the
//    fully unrolled complex mat-vec reads it as immediate constant operands.
//    8 * 2^K real flop per amplitude: HBM-bound up to K = 4 on GB300.
//  * k_fused_wide<K>: fused K = 5, 6 or 7 qubit unitaries, a CTA per tile of 128
//    (K = 5) or 64 slices, U from a device image in shared memory (see below).
//    Bound by the FP32 FMA pipe.
#include "dev_common.cuh"
#include "internal.h"

namespace rcs {

struct Mat2 {
    float2 m[4];
};
struct Mat4 {
    float2 m[16];
};

constexpr int kUnroll = 4;

template <bool T0>
__global__ void __launch_bounds__(256) k_plain_1q(float2 *__restrict__ psi, uint64_t items, int t, Mat2 M) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t hstep = 1ull << t;
    for (uint64_t it0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; it0 < items; it0 += stride * kUnroll) {
        float4 lo[kUnroll], hi[kUnroll];
        uint64_t idx[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t it = it0 + u * stride;
            if (it < items) {
                if (T0) {
                    idx[u] = it * 2;
                    lo[u] = *reinterpret_cast<const float4 *>(psi + idx[u]);
                } else {
                    idx[u] = insert_zero(it * 2, t);
                    lo[u] = *reinterpret_cast<const float4 *>(psi + idx[u]);
                    hi[u] = *reinterpret_cast<const float4 *>(psi + idx[u] + hstep);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t it = it0 + u * stride;
            if (it >= items) continue;
            if (T0) {
                float2 a0 = make_float2(lo[u].x, lo[u].y), a1 = make_float2(lo[u].z, lo[u].w);
                float2 b0 = cmac(cmac(make_float2(0.f, 0.f), M.m[0], a0), M.m[1], a1);
                float2 b1 = cmac(cmac(make_float2(0.f, 0.f), M.m[2], a0), M.m[3], a1);
                *reinterpret_cast<float4 *>(psi + idx[u]) = make_float4(b0.x, b0.y, b1.x, b1.y);
            } else {
                float2 a0 = make_float2(lo[u].x, lo[u].y), a1 = make_float2(hi[u].x, hi[u].y);
                float2 c0 = make_float2(lo[u].z, lo[u].w), c1 = make_float2(hi[u].z, hi[u].w);
                float2 b0 = cmac(cmac(make_float2(0.f, 0.f), M.m[0], a0), M.m[1], a1);
                float2 b1 = cmac(cmac(make_float2(0.f, 0.f), M.m[2], a0), M.m[3], a1);
                float2 d0 = cmac(cmac(make_float2(0.f, 0.f), M.m[0], c0), M.m[1], c1);
                float2 d1 = cmac(cmac(make_float2(0.f, 0.f), M.m[2], c0), M.m[3], c1);
                *reinterpret_cast<float4 *>(psi + idx[u]) = make_float4(b0.x, b0.y, d0.x, d0.y);
                *reinterpret_cast<float4 *>(psi + idx[u] + hstep) = make_float4(b1.x, b1.y, d1.x, d1.y);
            }
        }
    }
}

__device__ __forceinline__ void mv4(const Mat4 &M, const float2 a[4], float2 b[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 4; ++l) s = cmac(s, M.m[j * 4 + l], a[l]);
        b[j] = s;
    }
}

// Two-qubit gate on qubits lo < hi, local index j = bit(lo) + 2 bit(hi).
template <bool LO0>
__global__ void __launch_bounds__(256) k_plain_2q(float2 *__restrict__ psi, uint64_t items, int lo, int hi,
                                                   Mat4 M) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t sl = 1ull << lo, sh = 1ull << hi;
    for (uint64_t it0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; it0 < items; it0 += stride * 2) {
        float4 v[2][4];
        uint64_t base[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t it = it0 + u * stride;
            if (it >= items) continue;
            if (LO0) {
                base[u] = insert_zero(insert_zero(it, 0), hi);
                v[u][0] = *reinterpret_cast<const float4 *>(psi + base[u]);       // j = 0, 1
                v[u][1] = *reinterpret_cast<const float4 *>(psi + base[u] + sh);  // j = 2, 3
            } else {
                base[u] = insert_zero(insert_zero(it * 2, lo), hi);
                v[u][0] = *reinterpret_cast<const float4 *>(psi + base[u]);
                v[u][1] = *reinterpret_cast<const float4 *>(psi + base[u] + sl);
                v[u][2] = *reinterpret_cast<const float4 *>(psi + base[u] + sh);
                v[u][3] = *reinterpret_cast<const float4 *>(psi + base[u] + sl + sh);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const uint64_t it = it0 + u * stride;
            if (it >= items) continue;
            if (LO0) {
                float2 a[4] = {make_float2(v[u][0].x, v[u][0].y), make_float2(v[u][0].z, v[u][0].w),
                               make_float2(v[u][1].x, v[u][1].y), make_float2(v[u][1].z, v[u][1].w)};
                float2 b[4];
                mv4(M, a, b);
                *reinterpret_cast<float4 *>(psi + base[u]) = make_float4(b[0].x, b[0].y, b[1].x, b[1].y);
                *reinterpret_cast<float4 *>(psi + base[u] + sh) = make_float4(b[2].x, b[2].y, b[3].x, b[3].y);
            } else {
                // float4 e holds quads q (x,y) and q+1 (z,w) of operand row e
                float2 a[4], c[4], b[4], d[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    a[e] = make_float2(v[u][e].x, v[u][e].y);
                    c[e] = make_float2(v[u][e].z, v[u][e].w);
                }
                mv4(M, a, b);
                mv4(M, c, d);
                const uint64_t off[4] = {0, sl, sh, sl + sh};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    *reinterpret_cast<float4 *>(psi + base[u] + off[e]) = make_float4(b[e].x, b[e].y, d[e].x, d[e].y);
            }
        }
    }
}

// Complex matrix entry as the two packed operands of its multiply-adds, precomputed on
// the host: rr = (re, re) and ni = (-im, im). With (x, y) an input amplitude, the packed
// FP32x2 fused multiply-adds acc += rr * (x, y) and acc += ni * (y, x) form
// (acc.x + re x - im y, acc.y + re y + im x): per component the same two fused
// multiply-adds, in the same order, as four scalar ones, in half the instructions.
struct CEnt {
    float2 rr, ni;
};

template <int K>
struct SimtArgs {
    CEnt U[1 << K][1 << K];
    int t[K];  // ascending
    uint64_t slices;
};

// Resident CTAs per SM for width K, set by the registers the mat-vec needs without
// spilling (the two stages of 256 slices x 2^K amplitudes fit in shared memory).
template <int K>
constexpr int simt_blocks_per_sm() {
    return K == 4 ? 2 : 3;
}

// One thread per 2^K-amplitude slice, persistent over the slices (grid-stride). Each
// thread double-buffers its own slice through shared memory with cp.async: the copies of
// its next slice are in flight while it multiplies the current one, so the loads of a
// slice never wait behind the previous slice's mat-vec and stores. The stage slots are
// private to the thread (slot [b][j][thread]), so no block barrier is needed; lanes of a
// warp take neighbouring slices, and with no target below qubit 5 every copy and store
// instruction of a warp covers 256 contiguous bytes.
template <int K>
__global__ void __launch_bounds__(256, simt_blocks_per_sm<K>()) k_fused_simt(float2 *__restrict__ psi, const SimtArgs<K> a) {
    constexpr int D = 1 << K;
    extern __shared__ float2 stage[];  // [2][D][256]
    // target offsets of local index j, warp-uniform; read back through a volatile
    // pointer at every use so they are not held in registers across the mat-vec
    __shared__ uint64_t offs_s[D];
    if (threadIdx.x < D) {
        uint64_t o = 0;
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((threadIdx.x >> i) & 1) o |= 1ull << a.t[i];
        offs_s[threadIdx.x] = o;
    }
    __syncthreads();
    const volatile uint64_t *offs = offs_s;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint32_t slot0 = uint32_t(__cvta_generic_to_shared(stage)) + threadIdx.x * 8u;
    auto base_of = [&](uint64_t sl) {
        uint64_t b = sl;
#pragma unroll
        for (int i = 0; i < K; ++i) b = insert_zero(b, a.t[i]);
        return b;
    };
    auto issue = [&](uint64_t sl, int buf) {
        if (sl < a.slices) {
            const float2 *p = psi + base_of(sl);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const uint32_t dst = slot0 + uint32_t((buf * D + j) * 256) * 8u;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(p + offs[j]) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    issue(s, 0);
    int buf = 0;
#pragma unroll 1
    for (; s < a.slices; s += stride, buf ^= 1) {
        issue(s + stride, buf ^ 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // this slice's copies have landed
        float2 v[D], w[D];  // each input and its swapped form (y, x)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            v[j] = stage[(buf * D + j) * 256 + threadIdx.x];
            w[j] = make_float2(v[j].y, v[j].x);
        }
        float2 *p = psi + base_of(s);
#pragma unroll
        for (int j = 0; j < D; ++j) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const CEnt &u = a.U[j][l];
                acc = __ffma2_rn(u.rr, v[l], acc);
                acc = __ffma2_rn(u.ni, w[l], acc);
            }
            p[offs[j]] = acc;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- k_fused_wide<K>: fused 5- to 7-qubit unitaries on FP32 SIMT cores.
//
// From K = 5 a 2^K x 2^K complex matrix no longer fits the constant cache (as packed
// operands it is 16 KB at K = 5), and from K = 6 not the parameter space or a thread's
// registers, so a CTA applies it to a tile of T consecutive slices as a small complex
// GEMM in shared memory: out[s][j] = sum_l U[j][l] in[s][l], FP32 fused multiply-adds
// over l in increasing order. U comes from a device image laid out [l][j] (float2 re, im) and is
// copied into shared memory once per CTA. Each tile is copied in with cp.async into a
// [j][s] buffer (rows padded by one amplitude), multiplied, written back into the same
// buffer and stored with the same coalesced [j][s] walk. 8 * 2^K real flop per amplitude
// (16 to 64 flop/B): past the FP32 ridge, so these passes are bound by the FMA pipe.
constexpr int kWideThreads = 256;

// Per width: each thread computes RS slices x RJ outputs (slices sg + SG r, outputs
// jg + JG c; JG x SG = 256 threads), so a tile holds T = SG x RS slices: 4 x 4 on 128
// slices at K = 5, 4 x 4 and 4 x 8 on 64 slices at K = 6 and 7. Up to K = 6 two tile
// buffers let the next tile's copies run under the current tile's multiply-adds (the
// CTAs of an SM otherwise stay in step: all copying, then all multiplying); at K = 7 only
// one fits beside U. Resident CTAs per SM, by shared memory: three at K = 5 (74 KB), two
// at K = 6 (99 KB), one at K = 7 (194 KB).
template <int K>
struct WideShape {
    static constexpr int D = 1 << K;
    static constexpr int RS = 4;
    static constexpr int RJ = K == 7 ? 8 : 4;
    static constexpr int JG = D / RJ;
    static constexpr int SG = kWideThreads / JG;
    static constexpr int T = SG * RS;
    static constexpr int Row = T + 1;  // buffer row, padded by one amplitude
    static constexpr bool Dbl = K <= 6;  // two tile buffers: the next tile's copies run under the multiply-adds
    static constexpr int Blocks = K == 5 ? 3 : (K == 6 ? 2 : 1);
    static constexpr size_t Smem = size_t(D) * D * 8 + (Dbl ? 2 : 1) * size_t(D) * Row * 8 + size_t(D) * 8;
    static_assert(JG * SG == kWideThreads && T <= kWideThreads && kWideThreads % T == 0, "tile shape");
};

template <int K>
constexpr int wide_blocks_per_sm() {
    return WideShape<K>::Blocks;
}

template <int K>
constexpr size_t wide_smem_bytes() {
    return WideShape<K>::Smem;
}

struct WideArgs {
    int t[8];  // ascending targets (K used)
    uint64_t slices;
};

template <int K>
__global__ void __launch_bounds__(kWideThreads, wide_blocks_per_sm<K>())
    k_fused_wide(float2 *__restrict__ psi, const float2 *__restrict__ ut, const __grid_constant__ WideArgs a) {
    using S = WideShape<K>;
    constexpr int D = S::D, RS = S::RS, RJ = S::RJ, JG = S::JG, SG = S::SG, T = S::T, Row = S::Row;
    extern __shared__ __align__(16) unsigned char wide_smem[];
    float2 *U = reinterpret_cast<float2 *>(wide_smem);  // [l][j]
    float2 *buf = U + D * D;                             // [j][Row], twice when double-buffered
    uint64_t *offs = reinterpret_cast<uint64_t *>(buf + (S::Dbl ? 2 : 1) * D * Row);
    const int tid = threadIdx.x;
    const uint64_t slices = a.slices;
    for (int j = tid; j < D; j += kWideThreads) {
        uint64_t o = 0;
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((j >> i) & 1) o |= 1ull << a.t[i];
        offs[j] = o;
    }
    {  // U image: D * D * 8 bytes in 16-byte copies
        const uint32_t dst0 = uint32_t(__cvta_generic_to_shared(U));
        for (int c = tid; c < D * D / 2; c += kWideThreads)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + uint32_t(c) * 16u), "l"(ut + 2 * c)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    __syncthreads();  // offs
    const uint64_t ntiles = (slices + T - 1) / T;
    // copy / store walk: slice s = tid % T, rows j = tid / T + (256 / T) i
    const int ws = tid % T, wj = tid / T;
    // compute: slices sg + SG r, outputs jg + JG c
    const int jg = tid % JG, sg = tid / JG;
    const uint32_t buf0 = uint32_t(__cvta_generic_to_shared(buf));
    auto base_of = [&](uint64_t sl) {
        uint64_t b = sl;
#pragma unroll
        for (int i = 0; i < K; ++i) b = insert_zero(b, a.t[i]);
        return b;
    };
    // copies of tile `tile` into buffer `which` (one commit group per call, possibly empty)
    auto issue = [&](uint64_t tile, int which) {
        const uint64_t sl = tile * T + uint64_t(ws);
        if (tile < ntiles && sl < slices) {
            const uint64_t b = base_of(sl);
            const uint32_t dst0 = buf0 + uint32_t(which * D * Row) * 8u;
#pragma unroll 4
            for (int j = wj; j < D; j += kWideThreads / T) {
                const uint32_t dst = dst0 + uint32_t(j * Row + ws) * 8u;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(psi + (b | offs[j])) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int cur = 0;
    if (S::Dbl) issue(blockIdx.x, 0);
#pragma unroll 1
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t s = tile * T + uint64_t(ws);
        const bool live = s < slices;
        const uint64_t base = base_of(s);
        if (S::Dbl) {
            issue(tile + gridDim.x, cur ^ 1);  // that buffer's last stores ended before the last barrier
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            issue(tile, 0);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        float2 *bt = buf + cur * D * Row;
        __syncthreads();
        float2 acc[RS][RJ];
#pragma unroll
        for (int r = 0; r < RS; ++r)
#pragma unroll
            for (int c = 0; c < RJ; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int l = 0; l < D; ++l) {
            float2 x[RS], u[RJ];
#pragma unroll
            for (int r = 0; r < RS; ++r) x[r] = bt[l * Row + sg + SG * r];
#pragma unroll
            for (int c = 0; c < RJ; ++c) u[c] = U[l * D + jg + JG * c];
#pragma unroll
            for (int r = 0; r < RS; ++r)
#pragma unroll
                for (int c = 0; c < RJ; ++c) {
                    acc[r][c].x = fmaf(u[c].x, x[r].x, acc[r][c].x);
                    acc[r][c].x = fmaf(-u[c].y, x[r].y, acc[r][c].x);
                    acc[r][c].y = fmaf(u[c].x, x[r].y, acc[r][c].y);
                    acc[r][c].y = fmaf(u[c].y, x[r].x, acc[r][c].y);
                }
        }
        __syncthreads();  // every input read before the buffer takes the outputs
#pragma unroll
        for (int r = 0; r < RS; ++r)
#pragma unroll
            for (int c = 0; c < RJ; ++c) bt[(jg + JG * c) * Row + sg + SG * r] = acc[r][c];
        __syncthreads();
        if (live) {
#pragma unroll 4
            for (int j = wj; j < D; j += kWideThreads / T) psi[base | offs[j]] = bt[j * Row + ws];
        }
        __syncthreads();  // the stores have read the buffer before copies into it are issued
        if (S::Dbl) cur ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__global__ void k_init_zero(float4 *__restrict__ psi4, uint64_t n4) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride)
        psi4[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
}

static int check_launch() { return launch_status("state-update kernel"); }

// Full state from a compact sub-state: psi[i] = sub[c(i)] when every bit of i outside
// tmask is 0 (c(i) gathers the bits of i at the positions of tmask, in order), else 0.
// A circuit started from |0...0> leaves every qubit its first passes do not touch in
// |0>, so those passes can run on the 2^popcount(tmask) sub-state and this one write
// pass replaces the reset and them. c(i) is assembled from the runs of consecutive
// bits of tmask: run r moves the bits (i & mask[r]) down by shift[r] to its place in
// c, so a few shifts replace a loop over every bit of tmask (which made the kernel
// issue-bound: 22 ms from a 30- to a 32-qubit sub-state, 1.8 TB/s).
constexpr int kExpandRuns = 32;  // a 64-bit mask holds at most 32 runs of ones
struct ExpandArgs {
    uint64_t tmask;
    uint64_t mask[kExpandRuns];
    int runs;
    uint8_t shift[kExpandRuns];
};

// One thread per output float4 (amplitudes 2f and 2f + 1). With bit 0 in tmask both
// come from sub[c], sub[c + 1] (c even: one 16-byte load); without it 2f + 1 is 0.
__global__ void k_expand(float4 *__restrict__ psi4, uint64_t n4, const float2 *__restrict__ sub,
                         const __grid_constant__ ExpandArgs a) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const bool pair = a.tmask & 1ull;
    for (uint64_t f = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; f < n4; f += stride) {
        const uint64_t i0 = 2 * f;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(i0 & ~a.tmask)) {
            uint64_t c = 0;
            for (int r = 0; r < a.runs; ++r) c |= (i0 & a.mask[r]) >> a.shift[r];
            if (pair) {
                out = __ldg(reinterpret_cast<const float4 *>(sub) + (c >> 1));
            } else {
                const float2 v = __ldg(sub + c);
                out = make_float4(v.x, v.y, 0.f, 0.f);
            }
        }
        psi4[f] = out;
    }
}

int launch_expand(void *psi, int n, const void *sub, uint64_t tmask, void *stream) {
    if (n < 1 || (reinterpret_cast<uintptr_t>(sub) & 15u))
        return note_launch_refusal(RCS_ERR_ARG, "state expansion: bad size or a sub-state not 16-byte aligned");
    ExpandArgs a{};
    a.tmask = tmask;
    int placed = 0;  // bits of tmask below the current run
    for (int q = 0; q < 64;) {
        if (!((tmask >> q) & 1)) {
            ++q;
            continue;
        }
        int len = 0;
        while (q + len < 64 && ((tmask >> (q + len)) & 1)) ++len;
        a.mask[a.runs] = (len == 64 ? ~0ull : ((1ull << len) - 1ull)) << q;
        a.shift[a.runs] = uint8_t(q - placed);
        ++a.runs;
        placed += len;
        q += len;
    }
    const uint64_t n4 = (1ull << n) / 2;
    k_expand<<<grid_for(n4, 256, device_sm_count(), 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<float4 *>(psi), n4, static_cast<const float2 *>(sub), a);
    return launch_status("state expansion");
}

int launch_init_zero(void *psi, int n, void *stream) {
    auto st = static_cast<cudaStream_t>(stream);
    if (n == 0) return RCS_ERR_ARG;
    const uint64_t n4 = (1ull << n) / 2;  // n >= 1: whole float4s
    k_init_zero<<<grid_for(n4, 256, device_sm_count(), 8), 256, 0, st>>>(static_cast<float4 *>(psi), n4);
    return check_launch();
}

int launch_pass_plain(void *psi, int n, const Pass &p, void *stream) {
    auto st = static_cast<cudaStream_t>(stream);
    auto *s = static_cast<float2 *>(psi);
    const int sms = device_sm_count();
    if (p.kind == PASS_1Q) {
        Mat2 M;
        for (int e = 0; e < 4; ++e) M.m[e] = make_float2(float(p.U[e].real()), float(p.U[e].imag()));
        const int t = p.t[0];
        if (t == 0) {
            const uint64_t items = 1ull << (n - 1);
            k_plain_1q<true><<<grid_for(items, 256, sms, 8), 256, 0, st>>>(s, items, t, M);
        } else {
            const uint64_t items = 1ull << (n - 2);
            k_plain_1q<false><<<grid_for(items, 256, sms, 8), 256, 0, st>>>(s, items, t, M);
        }
    } else if (p.kind == PASS_2Q) {
        Mat4 M;
        for (int e = 0; e < 16; ++e) M.m[e] = make_float2(float(p.U[e].real()), float(p.U[e].imag()));
        const int lo = p.t[0], hi = p.t[1];
        if (lo == 0) {
            const uint64_t items = 1ull << (n - 2);
            k_plain_2q<true><<<grid_for(items, 256, sms, 8), 256, 0, st>>>(s, items, lo, hi, M);
        } else {
            const uint64_t items = 1ull << (n - 3);
            k_plain_2q<false><<<grid_for(items, 256, sms, 8), 256, 0, st>>>(s, items, lo, hi, M);
        }
    } else {
        return RCS_ERR_ARG;
    }
    return check_launch();
}

// Shared-memory attribute of k_fused_simt<K> on the current device (once).
template <int K>
static int simt_attr() {
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && attr_done[dev]) return RCS_OK;
    const int smem = 2 * (1 << K) * 256 * int(sizeof(float2));
    const cudaError_t e = cudaFuncSetAttribute(k_fused_simt<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return note_launch_error("fused kernel shared-memory attribute", e);
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
    return RCS_OK;
}

// Shared-memory attribute of k_fused_wide<K> on the current device (once).
template <int K>
static int wide_attr() {
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && attr_done[dev]) return RCS_OK;
    const cudaError_t e =
        cudaFuncSetAttribute(k_fused_wide<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(wide_smem_bytes<K>()));
    if (e != cudaSuccess) return note_launch_error("wide fused kernel shared-memory attribute", e);
    if (dev >= 0 && dev < 64) attr_done[dev] = true;
    return RCS_OK;
}

int simt_prepare_device() {
    int rc = simt_attr<1>();
    if (rc == RCS_OK) rc = simt_attr<2>();
    if (rc == RCS_OK) rc = simt_attr<3>();
    if (rc == RCS_OK) rc = simt_attr<4>();
    if (rc == RCS_OK) rc = wide_attr<5>();
    if (rc == RCS_OK) rc = wide_attr<6>();
    if (rc == RCS_OK) rc = wide_attr<7>();
    return rc;
}

size_t simt_ops_bytes(int k) { return k > kSimtParamK ? size_t(8) << (2 * k) : 0; }

// FP32 image of a wide pass: entry (l, j) = U[j][l] as (re, im), l-major.
void simt_build_ops(const Pass &p, uint8_t *out) {
    const int D = 1 << p.k;
    auto *f = reinterpret_cast<float *>(out);
    for (int l = 0; l < D; ++l)
        for (int j = 0; j < D; ++j) {
            const cd &u = p.U[size_t(j) * D + l];
            f[2 * (size_t(l) * D + j)] = float(u.real());
            f[2 * (size_t(l) * D + j) + 1] = float(u.imag());
        }
}

template <int K>
static int launch_simt_k(float2 *psi, int n, const Pass &p, cudaStream_t st) {
    SimtArgs<K> a;
    const int D = 1 << K;
    for (int j = 0; j < D; ++j)
        for (int l = 0; l < D; ++l) {
            const cd &u = p.U[size_t(j) * D + l];
            a.U[j][l] = CEnt{make_float2(float(u.real()), float(u.real())), make_float2(-float(u.imag()), float(u.imag()))};
        }
    for (int i = 0; i < K; ++i) a.t[i] = p.t[i];
    a.slices = 1ull << (n - K);
    const int threads = 256;
    const int smem = 2 * (1 << K) * threads * int(sizeof(float2));
    if (int rc = simt_attr<K>(); rc != RCS_OK) return rc;
    // persistent: the resident CTAs, never more than the slices need
    const unsigned grid = grid_for(a.slices, threads, device_sm_count(), simt_blocks_per_sm<K>());
    k_fused_simt<K><<<grid, threads, smem, st>>>(psi, a);
    return check_launch();
}

template <int K>
static int launch_wide_k(float2 *psi, int n, const Pass &p, const uint8_t *ops, cudaStream_t st) {
    if (!ops || (reinterpret_cast<uintptr_t>(ops) & 15u))
        return note_launch_refusal(RCS_ERR_ARG, "fused pass of width 5..7 without a 16-byte aligned U image");
    WideArgs a{};
    for (int i = 0; i < K; ++i) a.t[i] = p.t[i];
    a.slices = 1ull << (n - K);
    if (int rc = wide_attr<K>(); rc != RCS_OK) return rc;
    const uint64_t tiles = (a.slices + WideShape<K>::T - 1) / WideShape<K>::T;
    const uint64_t resident = uint64_t(device_sm_count()) * wide_blocks_per_sm<K>();
    const unsigned grid = unsigned(tiles < resident ? tiles : resident);
    k_fused_wide<K><<<grid, kWideThreads, wide_smem_bytes<K>(), st>>>(psi, reinterpret_cast<const float2 *>(ops), a);
    return check_launch();
}

int launch_pass_simt(void *psi, int n, const Pass &p, const uint8_t *ops, void *stream) {
    auto st = static_cast<cudaStream_t>(stream);
    auto *s = static_cast<float2 *>(psi);
    if (p.k > n) return RCS_ERR_ARG;
    switch (p.k) {
        case 1: return launch_simt_k<1>(s, n, p, st);
        case 2: return launch_simt_k<2>(s, n, p, st);
        case 3: return launch_simt_k<3>(s, n, p, st);
        case 4: return launch_simt_k<4>(s, n, p, st);
        case 5: return launch_wide_k<5>(s, n, p, ops, st);
        case 6: return launch_wide_k<6>(s, n, p, ops, st);
        case 7: return launch_wide_k<7>(s, n, p, ops, st);
        default: return RCS_ERR_UNSUPPORTED;
    }
}

}  // namespace rcs
