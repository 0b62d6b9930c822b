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

// round(x^2 * 2^62) for finite |x| < 2, exactly (from the float's exponent and
// 24-bit mantissa, one 32x32->64 multiply); sets bad for |x| >= 2, Inf or NaN.
// Integer-only on purpose: on GB300 the 64-bit float-to-integer conversions of an
// FP32 error-free split run at the FP64 rate and made the reduction 2.6x slower.
__device__ __forceinline__ uint64_t fx_sq(float x, int &bad) {
    const uint32_t b = __float_as_uint(x) & 0x7fffffffu;
    uint32_t e = b >> 23;
    uint32_t m = b & 0x7fffffu;
    if (e) m |= 0x800000u;
    else e = 1;
    if (e >= 128u) bad = 1;
    const int sh = 2 * int(e) - 238;  // x^2 * 2^62 = m^2 * 2^sh, m^2 < 2^48
    if (sh <= -18) {
        // r = -sh >= 18 (|x| < 2^-8, the usual case): the result is below 2^31, so
        // floor(m^2 / 2^(r-1)) = floor(floor(m^2 / 2^16) / 2^(r-17)) in 32-bit integers,
        // with floor(m^2 / 2^16) the high word of (m * 2^8)^2
        const int r = -sh;
        if (r > 48) return 0ull;
        const uint32_t a = m << 8;
        return uint64_t(((__umulhi(a, a) >> (r - 17)) + 1u) >> 1);  // round half up
    }
    const uint64_t m2 = uint64_t(m) * uint64_t(m);
    if (sh >= 0) return sh <= 16 ? (m2 << sh) : 0ull;
    const int r = -sh;
    return ((m2 >> (r - 1)) + 1ull) >> 1;  // round half up
}

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
int launch_status(const char *what);  // RCS_OK, or notes cudaGetLastError()

}  // namespace rcs
