// Device helpers shared by the library's kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rcs {

// Inserts a 0 bit at position t of x (bits >= t move up by one).
__device__ __forceinline__ uint64_t insert_zero(uint64_t x, int t) {
    const uint64_t low = x & ((1ull << t) - 1ull);
    return ((x >> t) << (t + 1)) | low;
}

// acc + m * a over complex64.
__device__ __forceinline__ float2 cmac(float2 acc, float2 m, float2 a) {
    acc.x = fmaf(m.x, a.x, acc.x);
    acc.x = fmaf(-m.y, a.y, acc.x);
    acc.y = fmaf(m.x, a.y, acc.y);
    acc.y = fmaf(m.y, a.x, acc.y);
    return acc;
}

// floor(x^2 * 2^62) for finite |x| < 2, exactly, in integer arithmetic only.
// With the float's biased exponent e and 24-bit significand m (implicit bit set),
// x = m * 2^(e - 150); with a = m * 2^8 (a 32-bit word whose top bit is the implicit
// bit), x^2 * 2^62 = a^2 * 2^-(254 - 2e), so the value is a^2 (< 2^64) shifted right
// by 254 - 2e. The shift clamps at 64 (PTX shr), which gives the exact 0 for zero
// and subnormals (e = 0: shift 254) and for every |x| < 2^-31.
// `seen` collects the raw bits: bit 30 of it is set once any input had |x| >= 2,
// Inf or NaN (e >= 128), for which the value returned is 0.
// Branch-free and 32-bit except one wide multiply and one 64-bit shift: on GB300 the
// reduction over a 2^34-amplitude state stays bound by HBM, not by the integer pipe
// (a two-path form that rounded to nearest ran the ALU pipe at 75% and HBM at 36%).
__device__ __forceinline__ uint64_t fx_sq(float x, uint32_t &seen) {
    const uint32_t u = __float_as_uint(x);
    seen |= u;
    const uint32_t a = (u << 8) | 0x80000000u;
    const uint32_t k = 254u - ((u >> 22) & 0x1feu);  // 254 - 2e; wraps to a huge shift for e >= 128
    const uint64_t t = uint64_t(a) * uint64_t(a);
    uint64_t q;
    asm("shr.b64 %0, %1, %2;" : "=l"(q) : "l"(t), "r"(k));
    return q;
}

// True once fx_sq has seen an input it cannot represent (|x| >= 2, Inf, NaN).
__device__ __forceinline__ bool fx_overflow(uint32_t seen) { return (seen & 0x40000000u) != 0; }

// Applies a bit permutation of basis indices (see BitMap).
template <class Map>
__device__ __forceinline__ uint64_t map_bits(const Map &m, uint64_t x) {
    if (m.identity) return x;
    uint64_t y = 0;
    for (int b = 0; b < m.n; ++b) y |= ((x >> b) & 1ull) << m.to[b];
    return y;
}

// Grid size for a grid-stride kernel: enough CTAs to fill every SM `per_sm`
// times, never more than the work needs.
inline unsigned grid_for(uint64_t items, unsigned threads, int sms, int per_sm) {
    uint64_t need = (items + threads - 1) / threads;
    uint64_t cap = uint64_t(sms) * uint64_t(per_sm);
    if (need < 1) need = 1;
    return unsigned(need < cap ? need : cap);
}

int device_sm_count();

// Launch bookkeeping: the launchers return RCS_ERR_CUDA on failure and leave the
// CUDA error text for the caller (consumed with take_launch_error()).
int note_launch_error(const char *what, cudaError_t e);
// Records msg as the launch error text (for a launch refused before it reached CUDA); returns code.
int note_launch_refusal(int code, const char *msg);
int launch_status(const char *what);  // RCS_OK, or notes cudaGetLastError()

}  // namespace rcs
