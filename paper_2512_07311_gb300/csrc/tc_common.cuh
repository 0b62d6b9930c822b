// Shapes, shared-memory layout constants and MMA wrappers shared by the tensor-core
// kernels that apply one 64 x 64 unitary per pass (the single-pass kernel and the
// persistent batch kernel): M = 128 slices per tile, K = N = 128 reals, the BF16
// realified and TF32 complex-block operand images, and the instruction descriptors.
#pragma once

#include <cstdint>

#include "dev_common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace rcs {

namespace tc {
constexpr int K = kTcK;         // 6 target qubits
constexpr int D = 1 << K;       // 64 amplitudes per slice
constexpr int KR = 2 * D;       // 128 reals per slice (GEMM K)
constexpr int NR = 2 * D;       // 128 real outputs (GEMM N)
constexpr int M = 128;          // slices per tile (GEMM M, TMEM lanes)
constexpr int kLoaderWarps = 8;
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kLoaderWarps + kEpiWarps + 1) * 32;  // 544
constexpr int kOpBytes = NR * KR * 2;                          // one bf16 operand image: 32 KB
constexpr int kStageBytes = D * M * 8;                         // one tile of complex64: 64 KB
constexpr int kSmBhi = 0;                                      // BF16: B_hi image, then B_lo
constexpr int kSmBlo = kOpBytes;
// TF32: per split (hi, lo) one K-major image of the 192 x 64 matrix [-Ui; Ur; Ui]
// (rows = outputs, K = inputs), in two 128-byte swizzle atom columns of 32 inputs.
constexpr int kTf32Rows = 3 * D;
constexpr int kTf32Atom = kTf32Rows * 128;   // 24 KB
constexpr int kTf32Split = 2 * kTf32Atom;    // 48 KB
// Shared-memory map (offsets from a 1024-aligned base): the B images, two stages of
// one tile each, then the small tables.
template <bool kTf32>
struct Layout {
    static constexpr int kBBytes = kTf32 ? 2 * kTf32Split : 2 * kOpBytes;
    static constexpr int kStage0 = kBBytes;
    static constexpr int kOff = kStage0 + 2 * kStageBytes;  // 64 x u64 target offsets
    static constexpr int kHiOff = kOff + D * 8;             // 64 x u64 offsets of the high compact bits
    static constexpr int kCj = kHiOff + 64 * 8;             // 64 x u16 compact index of local amplitude j
    static constexpr int kCs = kCj + D * 2;                 // 128 x u16 compact index of slice s within the tile
    static constexpr int kBar = kCs + M * 2;                // 16 mbarriers
    static constexpr int kMisc = kBar + 16 * 8;             // tmem slot, abort flag
    static constexpr int kAlloc = kMisc + 16 + 1024;        // slack for 1024-byte alignment
    static_assert(kAlloc <= 227 * 1024, "shared memory");
};
constexpr uint32_t kTmemCols = 512;
// instruction descriptor: D f32, A bf16, B bf16, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NR >> 3) << 17) | (uint32_t(M >> 4) << 24);
// TF32 variant: D f32, A tf32, B tf32, both K-major, N = 128 (Re outputs, then Im), M = 128
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(128 >> 3) << 17) | (uint32_t(M >> 4) << 24);
}  // namespace tc

__device__ __forceinline__ void mma_bf16_tmemA(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(tc::kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_tf32_tmemA(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                               uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ uint64_t slice_base(uint64_t s, const int (&t)[tc::K]) {
#pragma unroll
    for (int i = 0; i < tc::K; ++i) s = insert_zero(s, t[i]);
    return s;
}

}  // namespace rcs
