// Measurement sampling and scoring kernels (Section 3.2 items 3 and 4 of the paper:
// draw shots from |psi|^2, then score them with linear XEB).
//
// Probabilities enter every 2^n-term reduction as exact fixed-point integers:
// q(x) = floor(x^2 * 2^62) for each FP32 component x, computed from the float's
// exponent and 24-bit mantissa with one 32x32->64 integer multiply and one shift.
// Sums of q are exact (no rounding, any order), so the block sums, the block prefix
// scan, the norm T and every cumulative probability C_i are exact multiples of 2^-62
// that do not depend on the summation order. GB300 runs FP64 at a small fraction of
// its FP32/INT32 rate, so this keeps the reduction pass bound by HBM instead of by
// the FP64 pipe, with an error below 2^-62 per term (far below FP64's rounding of a
// 2^34-term sum).
//
// Sampling (inverse CDF): x_s = smallest i with C_i > u_s * T. The comparison
// C_i * 2^53 > m_s * T, with u_s = m_s * 2^-53, is done exactly in 128-bit integers.
//   1. k_block_sums: S_b = sum of q over block b (1024 amplitudes), one warp per block.
//   2. k_scan_*:     exclusive prefix P_b of S_b, and T = sum_b S_b.
//   3. the sampler (below): the block of each shot by binary search of P, the shots
//      grouped by block in stored order, then each block gathered and walked.
//
// Blocks, prefixes and the walk follow the caller's basis order also when the state is
// stored in a permuted qubit layout (caller bit q at stored bit to[q]): then block b is
// the 1024 caller indices [1024 b, 1024 b + 1024), whose stored positions vary in the
// bits P = {to[0..9]}. k_block_sums_map reads tiles that vary in the stored bits
// P u {0..5} (coalesced: lane = stored bits 1..5, a float4 = stored bit 0); each
// lane's amplitudes then lie in one or two caller blocks, and lanes of the same block
// are combined by shuffles. The sampler gathers the chosen block in caller order. So
// x_s is the same index, for the same uniform, whatever the layout.
// XEB: k_xeb_partial / k_xeb_final gather |psi_x|^2 in FP64 and reduce in a fixed
// tree order, F = 2^n * mean / T - 1.
#include <bit>

#include "dev_common.cuh"
#include "internal.h"

namespace rcs {

__device__ __forceinline__ uint64_t fx_amp(float2 a, uint32_t &seen) { return fx_sq(a.x, seen) + fx_sq(a.y, seen); }

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

static inline int block_log2(int n) { return n < kSampleBlockLog2 ? n : kSampleBlockLog2; }

// ---------------------------------------------------------------- block sums

__global__ void __launch_bounds__(256) k_block_sums(const float2 *__restrict__ psi, int blog2, uint64_t nblocks,
                                                     uint64_t *__restrict__ bsum, int *__restrict__ d_err) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
    const uint32_t nf4 = (1u << blog2) >> 1;  // float4 per block (blog2 >= 1)
    uint32_t seen = 0;
    for (uint64_t b = uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nblocks; b += warps) {
        const float4 *p4 = reinterpret_cast<const float4 *>(psi + (b << blog2));
        uint64_t s = 0;
#pragma unroll 4
        for (uint32_t c = lane; c < nf4; c += 32) {
            float4 v = __ldg(p4 + c);
            s += fx_sq(v.x, seen) + fx_sq(v.y, seen) + fx_sq(v.z, seen) + fx_sq(v.w, seen);
        }
        s = warp_sum_u64(s);
        if (lane == 0) bsum[b] = s;
    }
    if (fx_overflow(seen)) atomicOr(d_err, 1);
}

// Layout form: tile t = all amplitudes whose stored bits outside `tsmask` = P u {0..5}
// equal t's bits (deposited in order). Lane = stored bits 1..5 and a float4 carries the
// two amplitudes of stored bit 0, so a load instruction reads 512 contiguous bytes;
// `inner` = tsmask minus bits 0..5 is walked by the loop. Every amplitude of a lane
// with the same stored bit 0 lies in one caller block; `plane` = the lane bits in P
// (lanes that differ only there share a block), `b0p` = stored bit 0 is in P.
__global__ void __launch_bounds__(256) k_block_sums_map(const float2 *__restrict__ psi, int n, uint64_t tsmask,
                                                         uint64_t inner, uint32_t plane, int b0p, uint64_t ntiles,
                                                         int blog2, const BitMap to_caller,
                                                         uint64_t *__restrict__ bsum, int *__restrict__ d_err) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
    uint32_t seen = 0;
    for (uint64_t t = uint64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles; t += warps) {
        uint64_t base = 0;
        for (int bit = 0, k = 0; bit < n; ++bit)
            if (!((tsmask >> bit) & 1ull)) base |= ((t >> k++) & 1ull) << bit;
        base |= uint64_t(lane) << 1;
        uint64_t s0 = 0, s1 = 0, off = 0;
        auto next = [&](uint64_t o) { return ((o | ~inner) + 1ull) & inner; };  // masked increment
        do {  // every value of the inner bits in increasing order, eight loads in flight
            // (the count 2^popcount(inner) is a power of two >= 16: P has 10 bits, at most 6 of
            // them among bits 0..5)
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = __ldg(reinterpret_cast<const float4 *>(psi + (base | off)));
                off = next(off);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s0 += fx_sq(v[u].x, seen) + fx_sq(v[u].y, seen);
                s1 += fx_sq(v[u].z, seen) + fx_sq(v[u].w, seen);
            }
        } while (off != 0);
        if (b0p) s0 += s1;
#pragma unroll
        for (int bit = 0; bit < 5; ++bit)
            if ((plane >> bit) & 1u) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, 1 << bit);
                s1 += __shfl_xor_sync(0xffffffffu, s1, 1 << bit);
            }
        if ((uint32_t(lane) & plane) == 0) {
            bsum[map_bits(to_caller, base) >> blog2] = s0;
            if (!b0p) bsum[map_bits(to_caller, base | 1ull) >> blog2] = s1;
        }
    }
    if (fx_overflow(seen)) atomicOr(d_err, 1);
}

int launch_block_sums(const void *psi, int n, uint64_t *bsum, int *d_err, const BitMap &to_stored, void *stream) {
    const int bl = block_log2(n);
    const uint64_t nblocks = 1ull << (n - bl);
    if (to_stored.identity) {
        const unsigned grid = grid_for(nblocks * 32, 256, device_sm_count(), 8);
        k_block_sums<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<const float2 *>(psi), bl,
                                                                          nblocks, bsum, d_err);
        return launch_status(__func__);
    }
    // the tile bits P u {0..5} lie below n (layouts are only chosen for n >= 12)
    uint64_t pmask = 0;
    for (int q = 0; q < bl; ++q) pmask |= 1ull << to_stored.to[q];
    const uint64_t tsmask = pmask | 63ull;
    const uint64_t ntiles = 1ull << (n - std::popcount(tsmask));
    BitMap to_caller = identity_map(n);
    to_caller.identity = 0;
    for (int q = 0; q < n; ++q) to_caller.to[to_stored.to[q]] = uint8_t(q);
    const unsigned grid = grid_for(ntiles * 32, 256, device_sm_count(), 8);
    k_block_sums_map<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2 *>(psi), n, tsmask, tsmask & ~63ull, uint32_t((pmask >> 1) & 31ull), int(pmask & 1ull),
        ntiles, bl, to_caller, bsum, d_err);
    return launch_status(__func__);
}

// ---------------------------------------------------------------- scan

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanChunk = kScanThreads * kScanPer;  // 2048 entries per CTA

// Exclusive scan over the CTA of one value per thread; returns the CTA total in *tot.
__device__ uint64_t cta_excl_scan_u64(uint64_t v, uint64_t *tot) {
    __shared__ uint64_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t incl = warp_incl_scan_u64(v, lane);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint64_t x = lane < kScanThreads / 32 ? wsum[lane] : 0ull;
        uint64_t xi = warp_incl_scan_u64(x, lane);
        if (lane < kScanThreads / 32) wsum[lane] = xi - x;  // exclusive offsets of the warps
        if (lane == kScanThreads / 32 - 1) *tot = xi;
    }
    __syncthreads();
    const uint64_t r = wsum[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const uint64_t *__restrict__ x, uint64_t count,
                                                               uint64_t *__restrict__ chunk_tot) {
    const uint64_t base = uint64_t(blockIdx.x) * kScanChunk + uint64_t(threadIdx.x) * kScanPer;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i)
        if (base + i < count) s += x[base + i];
    __shared__ uint64_t tot;
    cta_excl_scan_u64(s, &tot);
    if (threadIdx.x == 0) chunk_tot[blockIdx.x] = tot;
}

// One CTA: exclusive scan of the chunk totals in place, grand total to *total.
__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint64_t *__restrict__ chunk_tot, uint64_t nchunks,
                                                            uint64_t *__restrict__ total, int *__restrict__ d_err) {
    __shared__ uint64_t tot;
    uint64_t carry = 0;
    int overflow = 0;
    for (uint64_t off = 0; off < nchunks; off += kScanChunk) {
        const uint64_t base = off + uint64_t(threadIdx.x) * kScanPer;
        uint64_t v[kScanPer], s = 0;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            v[i] = base + i < nchunks ? chunk_tot[base + i] : 0ull;
            if (s + v[i] < s) overflow = 1;
            s += v[i];
        }
        uint64_t e = cta_excl_scan_u64(s, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanPer; ++i) {
            if (base + i < nchunks) chunk_tot[base + i] = e;
            e += v[i];
        }
        if (carry + tot < carry) overflow = 1;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
    if (overflow) atomicOr(d_err, 2);
}

// x and out may be the same array (each thread reads its entries before writing them).
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint64_t *x, uint64_t count,
                                                              const uint64_t *__restrict__ chunk_off,
                                                              uint64_t *out) {
    const uint64_t base = uint64_t(blockIdx.x) * kScanChunk + uint64_t(threadIdx.x) * kScanPer;
    uint64_t v[kScanPer], s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = base + i < count ? x[base + i] : 0ull;
        s += v[i];
    }
    __shared__ uint64_t tot;
    uint64_t e = cta_excl_scan_u64(s, &tot) + chunk_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < count) out[base + i] = e;
        e += v[i];
    }
}

size_t scan_chunks(int n) {
    const uint64_t nb = 1ull << (n - block_log2(n));
    return size_t((nb + kScanChunk - 1) / kScanChunk);
}

int launch_block_scan(const uint64_t *bsum, uint64_t *bpre, uint64_t *chunk_tot, uint64_t *total, int n, int *d_err,
                      void *stream) {
    auto st = static_cast<cudaStream_t>(stream);
    const uint64_t nb = 1ull << (n - block_log2(n));
    const unsigned nch = unsigned(scan_chunks(n));
    k_scan_chunks<<<nch, kScanThreads, 0, st>>>(bsum, nb, chunk_tot);
    k_scan_top<<<1, kScanThreads, 0, st>>>(chunk_tot, nch, total, d_err);
    k_scan_apply<<<nch, kScanThreads, 0, st>>>(bsum, nb, chunk_tot, bpre);
    return launch_status(__func__);
}

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// 10 rounds; round: (hi0,lo0) = M0*x0, (hi1,lo1) = M1*x2,
// x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); key += (W0, W1) between rounds.

__device__ __forceinline__ uint64_t philox_word(uint64_t ctr0, uint64_t key0, int word) {
    uint64_t x0 = ctr0, x1 = 0, x2 = 0, x3 = 0, k0 = key0, k1 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * x0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, x0);
        const uint64_t lo1 = 0xCA5A826395121157ull * x2, hi1 = __umul64hi(0xCA5A826395121157ull, x2);
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    return word == 0 ? x0 : word == 1 ? x1 : word == 2 ? x2 : x3;
}

// a * 2^53 > (rhi, rlo) as 128-bit unsigned integers
__device__ __forceinline__ bool above(uint64_t a, uint64_t rhi, uint64_t rlo) {
    const uint64_t hi = a >> 11, lo = a << 53;
    return hi > rhi || (hi == rhi && lo > rlo);
}

// ---------------------------------------------------------------- sampler
//
// A call runs four kernels and the scan:
//   k_sample_locate  one thread per shot: the target u_s T, the binary search of the block
//                    prefix for the block b that holds it (out[s] = b), and a count of the
//                    shot under key(b) in hist.
//   scan             hist -> the first position of each key's shots (in place).
//   k_sample_order   one thread per shot: order[position] = (b, s), shots grouped by key.
//   k_sample_resolve one warp per position: the shot's block is gathered in caller order and
//                    walked (warp prefix over the 32 lanes' ranges, then over the crossing
//                    lane's 32 amplitudes), and the index replaces out[s].
// key(b) is b's rank in the stored order of blocks: the block-index bits read from the
// stored positions of caller bits 10.., low stored bits first (identity layout: key = b).
// Blocks whose amplitudes share cache lines (they differ only in stored bits 0..3) then
// have adjacent keys, and their shots are resolved by neighbouring warps while the lines
// are in L2. In a permuted layout a block's 1024 amplitudes lie in up to 1024 lines, each
// shared with up to 15 other blocks; resolved in shot order, every shot fetched all of its
// lines from DRAM (about 115 KB per shot at 30 qubits).

// smallest block b with inclusive prefix (bpre[b + 1], or T for the last) above the target
__device__ __forceinline__ uint64_t find_block(const uint64_t *__restrict__ bpre, uint64_t nblocks, uint64_t rhi,
                                               uint64_t rlo) {
    uint64_t lo = 0, hi = nblocks - 1;
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);  // mid + 1 <= hi < nblocks
        if (above(bpre[mid + 1], rhi, rlo)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// u_s T as a 128-bit integer (rhi, rlo), u_s = m 2^-53
__device__ __forceinline__ void shot_target(uint64_t g, uint64_t seed, uint64_t T, uint64_t &rhi, uint64_t &rlo) {
    const uint64_t m = philox_word(g >> 2, seed, int(g & 3)) >> 11;
    rlo = m * T;
    rhi = __umul64hi(m, T);
}

__global__ void __launch_bounds__(256) k_sample_locate(const uint64_t *__restrict__ bpre, uint64_t nblocks,
                                                        const uint64_t *__restrict__ total, uint64_t first,
                                                        uint64_t shots, uint64_t seed, const BitMap key_map,
                                                        uint64_t *__restrict__ out,
                                                        unsigned long long *__restrict__ hist) {
    const uint64_t T = *total;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    // warp-uniform trip count: the per-key counts below are combined across the warp
    for (uint64_t s0 = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); s0 < shots; s0 += stride) {
        const uint64_t s = s0 + uint64_t(lane);
        uint64_t key = ~0ull;
        if (s < shots) {
            if (T == 0) {
                out[s] = ~0ull;
            } else {
                uint64_t rhi, rlo;
                shot_target(first + s, seed, T, rhi, rlo);
                const uint64_t b = find_block(bpre, nblocks, rhi, rlo);
                out[s] = b;
                key = map_bits(key_map, b);
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key != ~0ull && lane == __ffs(peers) - 1) atomicAdd(hist + key, (unsigned long long)__popc(peers));
    }
}

// hist holds each key's first position; it is advanced as positions are taken.
// order[position] = (b << 32) | s: the shot and its block (s < 2^31 per launch, b < 2^24).
__global__ void __launch_bounds__(256) k_sample_order(const uint64_t *__restrict__ total, uint64_t shots,
                                                       const BitMap key_map, const uint64_t *__restrict__ out,
                                                       unsigned long long *__restrict__ hist,
                                                       uint64_t *__restrict__ order) {
    if (*total == 0) return;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t s0 = uint64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); s0 < shots; s0 += stride) {
        const uint64_t s = s0 + uint64_t(lane);
        const uint64_t b = s < shots ? out[s] : 0ull;
        const uint64_t key = s < shots ? map_bits(key_map, b) : ~0ull;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        unsigned long long base = 0;
        if (key != ~0ull && lane == leader) base = atomicAdd(hist + key, (unsigned long long)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (key != ~0ull) order[base + __popc(peers & ((1u << lane) - 1u))] = (b << 32) | s;
    }
}

// smap: caller index -> stored index (identity: the plain contiguous block reads).
// Each CTA takes one contiguous range of positions, in one of two schedules:
//   interleaved (the other cases): the CTA's warps step through the range
//     together (warp w: positions start + w, start + w + 8, ..., a barrier per round), so the
//     blocks in flight on an SM at any moment are neighbours in stored order and share
//     their cache lines while these are in L1/L2. In a permuted layout a block spans up to
//     1024 sectors, shared with its neighbours: a grid-stride assignment, or one warp walking
//     a group of neighbours by itself, fetched them again and again (the sample phase of 10^6
//     shots at 30 qubits took 6.0 ms interleaved, 11.5-13.2 ms so);
//   contiguous (at least 4 shots per block on average, or a state of at most 2^26
//     amplitudes, whose re-read sectors mostly come from L2): warp w takes the w-th eighth of
//     the range, so a warp's consecutive shots mostly fall in one block.
// Per block: lane l sums its 32 caller offsets 32 l .. 32 l + 31 of the block (exact
// fixed-point terms) and the warp scans the 32 sums. Per shot: a ballot on that scan
// finds the lane L whose range crosses the target, then the 32 lanes load one amplitude
// each of L's range and a second scan finds the index. A warp keeps the lane sums of its
// last block, so a block that holds many shots is summed once per warp and not once per
// shot (the sums are exact: the same index either way). Each warp fetches the records and
// targets of its next 32 positions at once, one per lane.
__global__ void __launch_bounds__(256) k_sample_resolve(const float2 *__restrict__ psi, int blog2,
                                                         const uint64_t *__restrict__ bpre,
                                                         const uint64_t *__restrict__ total, uint64_t first,
                                                         uint64_t shots, uint64_t seed,
                                                         const uint64_t *__restrict__ order, uint64_t *out,
                                                         const BitMap smap, int contiguous) {
    const uint64_t T = *total;
    if (T == 0) return;  // every out[s] is already ~0
    const int lane = threadIdx.x & 31;
    const uint32_t nw = blockDim.x >> 5;
    const uint32_t bamps = 1u << blog2;
    uint32_t seen = 0;
    // layout: stored offset of caller offset 32 lane + a = lmap | emap[a] (disjoint bits), and
    // the stored base of block b = OR over its four 6-bit chunks c of btab[c][chunk value]
    __shared__ uint64_t emap[32];
    __shared__ uint64_t btab[4][64];
    uint64_t lmap = 0;
    if (!smap.identity) {
        if (threadIdx.x < 32) {
            uint64_t e = 0;
            for (int q = 0; q < 5; ++q)
                if ((threadIdx.x >> q) & 1) e |= 1ull << smap.to[q];
            emap[threadIdx.x] = e;
        }
        {
            const int c = int(threadIdx.x >> 6), v = int(threadIdx.x & 63u);  // 256 threads: one entry each
            uint64_t e = 0;
            for (int k = 0; k < 6; ++k) {
                const int q = blog2 + 6 * c + k;
                if (q < smap.n && ((v >> k) & 1)) e |= 1ull << smap.to[q];
            }
            btab[c][v] = e;
        }
        for (int q = 5; q < blog2; ++q)
            if (((32u * uint32_t(lane)) >> q) & 1u) lmap |= 1ull << smap.to[q];
        __syncthreads();
    }
    const uint64_t per = (shots + gridDim.x - 1) / gridDim.x;
    const uint64_t beg = uint64_t(blockIdx.x) * per;
    if (beg >= shots) return;  // the whole CTA: past the last position (before any count below)
    const uint64_t end = beg + per < shots ? beg + per : shots;
    const uint32_t w = threadIdx.x >> 5;
    const int Lmax = int((bamps - 1u) >> 5);  // last lane that owns offsets (blocks hold <= 1024)
    const uint32_t a0 = uint32_t(lane) * 32u;
    uint64_t cur_b = ~0ull;       // block whose lane sums this warp holds
    uint64_t base = 0, ls = 0, incl = 0;
    const float2 *lb = psi;       // layout: the block's stored base; identity: the block itself
    // the warp's positions: wbeg, wbeg + step, ... below wend, in `trips` steps (the same
    // number in every warp of the CTA); 32 at a time, lane l holding the record and target of
    // the l-th
    const uint64_t pw = contiguous ? (end - beg + nw - 1) / nw : 0;
    const uint64_t wbeg = contiguous ? beg + uint64_t(w) * pw : beg + w;
    const uint64_t wend = contiguous ? (wbeg + pw < end ? wbeg + pw : end) : end;
    const uint64_t step = contiguous ? 1 : nw;
    const uint64_t trips = contiguous ? pw : (end - beg + nw - 1) / nw;
    for (uint64_t t0 = 0; t0 < trips; t0 += 32) {
        uint64_t my_sb = 0, my_rhi = 0, my_rlo = 0, my_out = 0;
        const uint64_t mine = wbeg + (t0 + uint64_t(lane)) * step;
        const bool have = t0 + uint64_t(lane) < trips && mine < wend;
        if (have) {
            my_sb = order[mine];
            shot_target(first + (my_sb & 0xffffffffull), seed, T, my_rhi, my_rlo);
        }
        const uint32_t nk = trips - t0 < 32 ? uint32_t(trips - t0) : 32u;
        for (uint32_t k = 0; k < nk; ++k) {  // same trip count in every warp: the barrier below
            const uint64_t i = wbeg + (t0 + k) * step;
            if (i < wend) {
                const uint64_t sb = __shfl_sync(0xffffffffu, my_sb, int(k));
                const uint64_t b = sb >> 32;
                const uint64_t rhi = __shfl_sync(0xffffffffu, my_rhi, int(k));
                const uint64_t rlo = __shfl_sync(0xffffffffu, my_rlo, int(k));
                if (b != cur_b) {
                    cur_b = b;
                    base = bpre[b];
                    ls = 0;
                    if (!smap.identity) {  // blog2 = 10: every lane owns 32 caller offsets
                        lb = psi + (btab[0][b & 63u] | btab[1][(b >> 6) & 63u] | btab[2][(b >> 12) & 63u] |
                                    btab[3][(b >> 18) & 63u]);
                        const float2 *ll = lb + lmap;
#pragma unroll 16
                        for (int a = 0; a < 32; ++a) ls += fx_amp(__ldg(ll + emap[a]), seen);
                    } else {
                        lb = psi + (b << blog2);
                        const uint32_t cnt = a0 < bamps ? (bamps - a0 < 32u ? bamps - a0 : 32u) : 0u;
                        for (uint32_t a = 0; a < cnt; a += 2) {
                            const float4 v = __ldg(reinterpret_cast<const float4 *>(lb + a0 + a));
                            ls += fx_sq(v.x, seen) + fx_sq(v.y, seen) + fx_sq(v.z, seen) + fx_sq(v.w, seen);
                        }
                    }
                    incl = warp_incl_scan_u64(ls, lane);
                }
                const unsigned hit = __ballot_sync(0xffffffffu, above(base + incl, rhi, rlo));
                const int L = hit ? __ffs(hit) - 1 : Lmax;  // hit != 0: lane 31's prefix is the block's inclusive prefix
                const uint64_t run0 = __shfl_sync(0xffffffffu, base + incl - ls, L);  // prefix before L's range
                // lane j takes caller offset 32 L + j
                const uint32_t aL = uint32_t(L) * 32u;
                uint64_t v = 0;
                if (!smap.identity) {
                    const uint64_t lmL = __shfl_sync(0xffffffffu, lmap, L);
                    v = fx_amp(__ldg(lb + (lmL | emap[lane])), seen);
                } else if (aL + uint32_t(lane) < bamps) {
                    v = fx_amp(__ldg(lb + aL + uint32_t(lane)), seen);
                }
                const uint64_t incl2 = warp_incl_scan_u64(v, lane);
                const unsigned hit2 = __ballot_sync(0xffffffffu, above(run0 + incl2, rhi, rlo));
                const uint32_t cntL = bamps - aL < 32u ? bamps - aL : 32u;
                const uint32_t j = hit2 ? uint32_t(__ffs(hit2) - 1) : cntL - 1;
                if (uint32_t(lane) == k) my_out = (b << blog2) + aL + j;
            }
            if (!contiguous) __syncthreads();  // keeps the CTA's warps on neighbouring positions
        }
        if (have) out[my_sb & 0xffffffffull] = my_out;
    }
}

BitMap identity_map(int n) {
    BitMap m;
    for (int i = 0; i < 64; ++i) m.to[i] = uint8_t(i);
    m.n = n;
    m.identity = 1;
    return m;
}

// Block b -> its rank among blocks in stored order: block bit j is caller bit bl + j,
// stored at bit to[bl + j]; its key bit is the number of those stored bits below it.
static BitMap block_key_map(int n, int bl, const BitMap &to_stored) {
    BitMap k = identity_map(n - bl);
    if (to_stored.identity) return k;
    k.identity = 1;
    for (int j = 0; j < n - bl; ++j) {
        int rank = 0;
        for (int i = 0; i < n - bl; ++i) rank += to_stored.to[bl + i] < to_stored.to[bl + j];
        k.to[j] = uint8_t(rank);
        if (rank != j) k.identity = 0;
    }
    return k;
}

int launch_sample(const void *psi, int n, uint64_t *hist, const uint64_t *bpre, const uint64_t *total,
                  uint64_t *chunk, uint64_t first, uint64_t shots, uint64_t seed, uint64_t *d_out, uint64_t *order,
                  int *d_err, const BitMap &to_stored, void *stream) {
    if (shots == 0) return RCS_OK;
    const int bl = block_log2(n);
    if (!to_stored.identity && bl < 10) return RCS_ERR_UNSUPPORTED;
    auto st = static_cast<cudaStream_t>(stream);
    const uint64_t nblocks = 1ull << (n - bl);
    const BitMap key_map = block_key_map(n, bl, to_stored);
    const int sms = device_sm_count();
    auto *h = reinterpret_cast<unsigned long long *>(hist);
    const size_t nch = scan_chunks(n);
    // at most 2^31 shots per round, so that a position's record packs the shot and its block
    // (the block index has at most 24 bits for n <= 34)
    constexpr uint64_t kRound = 1ull << 31;
    for (uint64_t off = 0; off < shots; off += kRound) {
        const uint64_t cnt = shots - off < kRound ? shots - off : kRound;
        uint64_t *out = d_out + off;
        cudaError_t e = cudaMemsetAsync(hist, 0, nblocks * sizeof(uint64_t), st);
        if (e != cudaSuccess) return note_launch_error(__func__, e);
        const unsigned g1 = grid_for(cnt, 256, sms, 8);
        k_sample_locate<<<g1, 256, 0, st>>>(bpre, nblocks, total, first + off, cnt, seed, key_map, out, h);
        // in place: the counts become each key's first position (the scan's total, the shot
        // count, goes to the spare slot after the chunk totals)
        int rc = launch_block_scan(hist, hist, chunk, chunk + nch, n, d_err, stream);
        if (rc != RCS_OK) return rc;
        k_sample_order<<<g1, 256, 0, st>>>(total, cnt, key_map, out, h, order);
        const unsigned g2 = grid_for(cnt * 32, 256, sms, 8);
        // contiguous ranges per warp (which keep a block's lane sums) for many shots per block,
        // or for states of at most 2^26 amplitudes, whose sectors a warp re-reads mostly from
        // L2; the interleaved rounds for the larger states, where those re-reads go to DRAM
        // (measured: 64 circuits of 16-26 qubits, 10^5 shots each: 7.0 against 7.8 ms for their
        // sampling; 30 qubits, 10^6 shots: 5.2 against 11.5 ms)
        const int contiguous = (cnt >= 4 * nblocks || n <= 26) ? 1 : 0;
        k_sample_resolve<<<g2, 256, 0, st>>>(static_cast<const float2 *>(psi), bl, bpre, total, first + off, cnt, seed,
                                              order, out, to_stored, contiguous);
    }
    return launch_status(__func__);
}

// ---------------------------------------------------------------- gather

__global__ void k_gather(const float2 *__restrict__ psi, uint64_t namps, const uint64_t *__restrict__ bits,
                         uint64_t count, double *__restrict__ out, int *__restrict__ d_err, const BitMap in_map) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint64_t x = bits[i];
        if (x >= namps) {
            out[2 * i] = out[2 * i + 1] = __longlong_as_double(0x7ff8000000000000ll);
            atomicOr(d_err, 4);
            continue;
        }
        const float2 a = psi[map_bits(in_map, x)];
        out[2 * i] = double(a.x);
        out[2 * i + 1] = double(a.y);
    }
}

int launch_gather(const void *psi, int n, const uint64_t *d_bits, size_t count, double *d_out_re_im, int *d_err,
                  const BitMap &in_map, void *stream) {
    if (count == 0) return RCS_OK;
    k_gather<<<grid_for(count, 256, device_sm_count(), 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2 *>(psi), 1ull << n, d_bits, count, d_out_re_im, d_err, in_map);
    return launch_status(__func__);
}

// ---------------------------------------------------------------- XEB

constexpr int kXebThreads = 256;
constexpr uint64_t kXebPerCta = 4096;

size_t xeb_partials_count(size_t count) { return size_t((count + kXebPerCta - 1) / kXebPerCta); }

__device__ double cta_sum_f64(double v) {
    __shared__ double ws[kXebThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kXebThreads / 32; ++i) r += ws[i];
    __syncthreads();
    return r;  // valid in thread 0
}

__global__ void __launch_bounds__(kXebThreads) k_xeb_partial(const float2 *__restrict__ psi, uint64_t namps,
                                                              const uint64_t *__restrict__ x, uint64_t count,
                                                              double *__restrict__ partials, const BitMap in_map) {
    const uint64_t beg = uint64_t(blockIdx.x) * kXebPerCta;
    const uint64_t end = beg + kXebPerCta < count ? beg + kXebPerCta : count;
    double s = 0.0;
    bool bad = false;
    for (uint64_t i = beg + threadIdx.x; i < end; i += kXebThreads) {
        const uint64_t xi = x[i];
        if (xi >= namps) {
            bad = true;
            continue;
        }
        const float2 a = psi[map_bits(in_map, xi)];
        s += double(a.x) * double(a.x) + double(a.y) * double(a.y);
    }
    const int anybad = __syncthreads_or(bad);
    const double r = cta_sum_f64(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000ll) : r;
}

__global__ void __launch_bounds__(kXebThreads) k_xeb_final(const double *__restrict__ partials, uint64_t nparts,
                                                            uint64_t count, int n, const uint64_t *__restrict__ total,
                                                            double *__restrict__ out) {
    double s = 0.0;
    for (uint64_t i = threadIdx.x; i < nparts; i += kXebThreads) s += partials[i];
    const double r = cta_sum_f64(s);
    if (threadIdx.x == 0) {
        const double T = ldexp(double(*total), -62);
        *out = ldexp(r / double(count), n) / T - 1.0;
    }
}

int launch_xeb(const void *psi, int n, const uint64_t *d_samples, size_t count, const uint64_t *total,
               double *d_partials, double *d_out, const BitMap &in_map, void *stream) {
    auto st = static_cast<cudaStream_t>(stream);
    if (count == 0) return RCS_ERR_ARG;
    const size_t np = xeb_partials_count(count);
    k_xeb_partial<<<unsigned(np), kXebThreads, 0, st>>>(static_cast<const float2 *>(psi), 1ull << n, d_samples, count,
                                                        d_partials, in_map);
    k_xeb_final<<<1, kXebThreads, 0, st>>>(d_partials, np, count, n, total, d_out);
    return launch_status(__func__);
}

}  // namespace rcs
