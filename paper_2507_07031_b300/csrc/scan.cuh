// scan.cuh -- exclusive prefix sums of uint32 counts (bucket offsets of the
// MSM's counting sort).  Three launches: per-tile sums, a single-block scan of
// the tile sums, and per-tile scans with their offsets.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace zk {

void count_launches(unsigned k);

namespace scan_detail {

constexpr int kThreads = 256;
constexpr int kPer = 8;
constexpr int kTile = kThreads * kPer;

// Element b of the scanned sequence: in[b] when K = 0; for bucket offsets
// `in`, the number of K-item slices of bucket b, ceil((in[b+1] - in[b]) / K),
// when K > 0 (0 for buckets of at most `thr` items); and the number of fixed
// chunks of -K consecutive entries that bucket b's entries meet, when K < 0.
__device__ __forceinline__ uint32_t elem(const uint32_t *in, uint32_t b, uint32_t n, int K, uint32_t thr) {
    if (b >= n) return 0;
    if (K == 0) return in[b];
    const uint32_t lo = in[b], hi = in[b + 1];
    if (K > 0) return hi - lo > thr ? (hi - lo + (uint32_t)K - 1) / (uint32_t)K : 0u;
    const uint32_t c = (uint32_t)(-K);
    return hi > lo ? (hi - 1) / c - lo / c + 1 : 0u;
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[kThreads / 32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kThreads / 32 ? ws[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= (uint32_t)d) w += y;
        }
        if (lane < kThreads / 32) ws[lane] = w;
    }
    __syncthreads();
    uint32_t before = warp ? ws[warp - 1] : 0;
    *total = ws[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void k_tile_sums(const uint32_t *__restrict__ in, uint32_t n, int K,
                            uint32_t *__restrict__ sums, const uint32_t *gate, const int *Kp,
                            const uint32_t *const *in_p, uint32_t thr, const uint32_t *thr_p) {
    if (gate && !*gate) return;
    if (Kp) K = *Kp;
    if (thr_p) thr = *thr_p;
    if (in_p) in = *in_p;
    uint32_t base = blockIdx.x * kTile + threadIdx.x * kPer;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kPer; i++) s += elem(in, base + i, n, K, thr);
    uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint32_t *__restrict__ sums, uint32_t tiles, const uint32_t *gate) {
    if (gate && !*gate) return;
    const uint32_t per = (tiles + kThreads - 1) / kThreads;
    const uint32_t lo = threadIdx.x * per;
    uint32_t s = 0;
    for (uint32_t i = lo; i < lo + per && i < tiles; i++) s += sums[i];
    uint32_t tot;
    uint32_t before = block_excl_scan(s, &tot);
    for (uint32_t i = lo; i < lo + per && i < tiles; i++) {
        uint32_t v = sums[i];
        sums[i] = before;
        before += v;
    }
    if (threadIdx.x == 0) sums[tiles] = tot;
}

__global__ void k_tile_scan(const uint32_t *__restrict__ in, uint32_t n, int K,
                            const uint32_t *__restrict__ sums, uint32_t tiles,
                            uint32_t *__restrict__ out, const uint32_t *gate, const int *Kp,
                            const uint32_t *const *in_p, uint32_t thr, const uint32_t *thr_p) {
    if (gate && !*gate) return;
    if (Kp) K = *Kp;
    if (thr_p) thr = *thr_p;
    if (in_p) in = *in_p;
    uint32_t base = blockIdx.x * kTile + threadIdx.x * kPer;
    uint32_t v[kPer];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        v[i] = elem(in, base + i, n, K, thr);
        s += v[i];
    }
    uint32_t tot;
    uint32_t before = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kPer; i++) {
        if (base + i < n) out[base + i] = before;
        before += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = sums[tiles];
}

}  // namespace scan_detail

inline size_t scan_temp_bytes(uint32_t n) {
    return ((size_t)n / scan_detail::kTile + 2) * sizeof(uint32_t);
}

// out[b] = sum_{b' < b} elem(b'), out[n] = total.  `in` may equal neither
// `out` nor `tmp`.  With a `gate` (device word), the scan does nothing when
// the word is zero at execution time.  With `Kp` (device word), K is read
// from it at execution time instead, and with `in_p` (a device word holding
// a pointer), the input array.  `thr`: see elem(); with `thr_p` (device
// word) it is read from there at execution time.
inline int scan_exclusive(const uint32_t *in, uint32_t *out, uint32_t n, int K, void *tmp,
                          cudaStream_t s, const uint32_t *gate = nullptr, const int *Kp = nullptr,
                          const uint32_t *const *in_p = nullptr, uint32_t thr = 0,
                          const uint32_t *thr_p = nullptr) {
    using namespace scan_detail;
    uint32_t tiles = (n + kTile - 1) / kTile;
    if (tiles == 0) tiles = 1;
    uint32_t *sums = (uint32_t *)tmp;
    k_tile_sums<<<tiles, kThreads, 0, s>>>(in, n, K, sums, gate, Kp, in_p, thr, thr_p);
    k_scan_sums<<<1, kThreads, 0, s>>>(sums, tiles, gate);
    k_tile_scan<<<tiles, kThreads, 0, s>>>(in, n, K, sums, tiles, out, gate, Kp, in_p, thr, thr_p);
    count_launches(3);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // namespace zk
