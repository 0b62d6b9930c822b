// Linear XEB for callers that cannot allocate device memory.
//
// rcs_xeb_device() keeps its partial sums and the norm's block sums in buffers the
// context allocates with cudaMalloc. Some callers cannot do that: code whose
// memory is handed out by a host framework's own allocator or a fixed arena, and
// hosts that forbid device allocations after start-up. rcs_xeb_static() computes the same quantity from caller-owned device
// buffers only: its scratch is one file-scope __device__ array, fixed in size and
// held by every GPU that loads this library until the process exits.
//
// Scratch layout (192 KiB): kNormParts uint64 fixed-point norm partials (one per
// CTA of the norm kernel), then kXebParts double XEB partials (one per 4096
// samples). Every slot a call reads is written earlier in the same call, so no
// slot has to start at zero; nothing is cleared between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "dev_common.cuh"
#include "internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kNormParts = 8192;
constexpr int kXebParts = 16384;
constexpr uint64_t kPerCta = 4096;  // samples per XEB partial (the same split as rcs_xeb_device)
constexpr size_t kScratchBytes = size_t(kNormParts) * 8 + size_t(kXebParts) * 8;

}  // namespace

static __device__ __align__(256) unsigned char g_xeb_scratch[kScratchBytes];

namespace {

// Sum over the CTA in the same order as the context path: xor-shuffle within each
// warp, then thread 0 adds the 8 warp sums in order.
__device__ double cta_sum_f64_static(double v) {
    __shared__ double ws[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) r += ws[i];
    __syncthreads();
    return r;
}

__device__ uint64_t cta_sum_u64_static(uint64_t v) {
    __shared__ uint64_t ws[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    uint64_t r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kThreads / 32; ++i) r += ws[i];
    __syncthreads();
    return r;
}

// Exact fixed-point |psi|^2 partial sums, one per CTA (grid-stride over float4 pairs).
__global__ void __launch_bounds__(kThreads) k_static_norm(const float4 *__restrict__ psi4, uint64_t n4,
                                                           uint64_t *__restrict__ parts) {
    uint32_t seen = 0;
    uint64_t s = 0;
    const uint64_t stride = uint64_t(gridDim.x) * kThreads;
    for (uint64_t i = uint64_t(blockIdx.x) * kThreads + threadIdx.x; i < n4; i += stride) {
        const float4 v = __ldg(psi4 + i);
        s += rcs::fx_sq(v.x, seen) + rcs::fx_sq(v.y, seen) + rcs::fx_sq(v.z, seen) + rcs::fx_sq(v.w, seen);
    }
    const uint64_t r = cta_sum_u64_static(s);
    const int anybad = __syncthreads_or(rcs::fx_overflow(seen));
    if (threadIdx.x == 0) parts[blockIdx.x] = anybad ? ~0ull : r;
}

// |psi_x|^2 summed in FP64 over 4096 samples per CTA; NaN marks an index >= 2^n.
__global__ void __launch_bounds__(kThreads) k_static_xeb(const float2 *__restrict__ psi, uint64_t namps,
                                                          const uint64_t *__restrict__ x, uint64_t count,
                                                          double *__restrict__ parts) {
    const uint64_t beg = uint64_t(blockIdx.x) * kPerCta;
    const uint64_t end = beg + kPerCta < count ? beg + kPerCta : count;
    double s = 0.0;
    bool bad = false;
    for (uint64_t i = beg + threadIdx.x; i < end; i += kThreads) {
        const uint64_t xi = x[i];
        if (xi >= namps) {
            bad = true;
            continue;
        }
        const float2 a = psi[xi];
        s += double(a.x) * double(a.x) + double(a.y) * double(a.y);
    }
    const int anybad = __syncthreads_or(bad);
    const double r = cta_sum_f64_static(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000ll) : r;
}

__global__ void __launch_bounds__(kThreads) k_static_final(const uint64_t *__restrict__ norm_parts, int nnorm,
                                                            const double *__restrict__ xeb_parts, int nxeb,
                                                            uint64_t count, int n, double *__restrict__ out) {
    uint64_t t = 0;
    bool bad = false;
    for (int i = threadIdx.x; i < nnorm; i += kThreads) {
        const uint64_t v = norm_parts[i];
        if (v == ~0ull) bad = true;
        else t += v;
    }
    const int anybad = __syncthreads_or(bad);
    const uint64_t T = cta_sum_u64_static(t);
    double s = 0.0;
    for (int i = threadIdx.x; i < nxeb; i += kThreads) s += xeb_parts[i];
    const double r = cta_sum_f64_static(s);
    if (threadIdx.x == 0) {
        const double Td = ldexp(double(T), -62);
        *out = anybad || T == 0 ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(r / double(count), n) / Td - 1.0;
    }
}

std::mutex g_setup_mu;
// Device address of g_xeb_scratch, per device ordinal, looked up once. It stays valid for
// the life of the device's primary context; a cudaDeviceReset() unloads the module, so a
// process that resets a device does not call this entry point on it again.
void *g_scratch_addr[64] = {};

}  // namespace

extern "C" int rcs_xeb_static(const void *d_state, int n_qubits, const uint64_t *d_samples, size_t count,
                              double *d_out_xeb, uint64_t stream) {
    using namespace rcs;
    if (!d_state || !d_samples || !d_out_xeb)
        return set_thread_error(RCS_ERR_ARG, "rcs_xeb_static: null device pointer");
    if (n_qubits < 1 || n_qubits > kMaxQubits) return set_thread_error(RCS_ERR_ARG, "rcs_xeb_static: n must be 1..34");
    if (count == 0 || count > uint64_t(kXebParts) * kPerCta)
        return set_thread_error(RCS_ERR_ARG, "rcs_xeb_static: sample count must be 1.." +
                                                 std::to_string(uint64_t(kXebParts) * kPerCta));
    // the norm kernel reads the state as float4 pairs, the XEB kernels 8-byte words: a
    // misaligned view (an offset slice of someone else's buffer) is refused here, on the host
    if (reinterpret_cast<uintptr_t>(d_state) % 16 != 0)
        return set_thread_error(RCS_ERR_ARG, "rcs_xeb_static: d_state must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(d_samples) % 8 != 0 || reinterpret_cast<uintptr_t>(d_out_xeb) % 8 != 0)
        return set_thread_error(RCS_ERR_ARG, "rcs_xeb_static: d_samples and d_out_xeb must be 8-byte aligned");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_thread_error(RCS_ERR_CUDA, std::string("rcs_xeb_static: cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64)
        return set_thread_error(RCS_ERR_UNSUPPORTED,
                                "rcs_xeb_static: device ordinal " + std::to_string(dev) + " is beyond the 64 this call serves");
    void *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            // host code only sees a stand-in for the array: ask the runtime for its address on this device
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_xeb_scratch);
            if (e != cudaSuccess || !p)
                return set_thread_error(RCS_ERR_CUDA,
                                        std::string("rcs_xeb_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    auto *norm_parts = static_cast<uint64_t *>(scratch);
    auto *xeb_parts = reinterpret_cast<double *>(static_cast<unsigned char *>(scratch) + size_t(kNormParts) * 8);
    auto st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t namps = uint64_t(1) << n_qubits;
    const uint64_t n4 = namps / 2;
    const int nnorm = int(grid_for(n4, kThreads, device_sm_count(), 8) < unsigned(kNormParts)
                              ? grid_for(n4, kThreads, device_sm_count(), 8)
                              : unsigned(kNormParts));
    const int nxeb = int((count + kPerCta - 1) / kPerCta);
    k_static_norm<<<nnorm, kThreads, 0, st>>>(static_cast<const float4 *>(d_state), n4, norm_parts);
    k_static_xeb<<<nxeb, kThreads, 0, st>>>(static_cast<const float2 *>(d_state), namps, d_samples, count, xeb_parts);
    k_static_final<<<1, kThreads, 0, st>>>(norm_parts, nnorm, xeb_parts, nxeb, count, n_qubits, d_out_xeb);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_thread_error(RCS_ERR_CUDA, std::string("rcs_xeb_static: launch: ") + cudaGetErrorString(e));
    return RCS_OK;
}
