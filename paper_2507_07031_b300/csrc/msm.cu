// msm.cu -- KZG commitment as a multi-scalar multiplication over the SRS
// (paper Sec. 2.1: com = [f(tau)]_1 = sum_i c_i [tau^i]_1), batched.
//
// Pippenger's bucket method with signed windows of c bits, in five phases:
//   1. recode: every scalar is recentred (s > (r-1)/2 becomes r - s with the
//      point negated) and split into W = ceil(254/c) signed digits in
//      [-2^(c-1), 2^(c-1)]; digit d of window w of scalar i contributes
//      sign(d) * 2^(c w) SRS[i], a point read from the precomputed window
//      table, to bucket |d| - 1 of its MSM.  A warp-aggregated counting pass
//      builds the bucket histogram;
//   2. sort: an exclusive scan gives bucket offsets and a warp-aggregated
//      scatter writes the (table index, sign) words bucket by bucket;
//   3. accumulate: the sorted entries are cut into equal chunks, one thread
//      per chunk adds its entries in XYZZ coordinates (mixed additions) and
//      emits a partial sum per bucket it meets; the partial sums are combined
//      in further rounds, which a plan made on the device from the largest
//      bucket skips when the buckets do not need them, so skewed buckets
//      (quantised ML values put 2^20 points into 128 buckets) keep the whole
//      GPU busy and uniform ones pay for no extra round;
//   4. reduce: sum_b (b + 1) S_b per MSM by segment-level suffix scans in up
//      to three levels, each point addition spread over the four warps of a
//      block (team.cuh) because this phase is latency bound;
//   5. normalise the result to canonical affine coordinates.
// Every MSM of a batch (uneven lengths) goes through the same launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "check.cuh"
#include "ctx.cuh"
#include "curve.cuh"
#include "scan.cuh"
#include "team.cuh"

namespace zk {

ZK_CHECK_UNIT()

namespace {

constexpr uint32_t kInvalid = 0xffffffffu;
constexpr int kMaxLevels = 4;  // bucket-reduction levels (phase 4)
constexpr size_t kStatsMin = 4096;  // scalars below which the width scan is skipped

// One MSM of a batch.  Jobs are ordered by window width so that each width's
// scalars form one contiguous range for its recode launch.  The host writes
// the full-width shape (window width c, ceil(254 / c) windows over the
// width's window table); when the scalars' widths are measured, a plan
// kernel rewrites shift, wins, logB and table on the device before the
// recode runs (small-scalar path).
struct JobDesc {
    const uint32_t *scalars;  // n canonical scalars (device)
    void *out;                // canonical affine result (device)
    const AffineS *table;     // entries the sorted entries index (a window table, or its window 0)
    const AffineS *wtable;    // window table of width c over the base points (SRS, or the
                              // Lagrange basis of H); window 0 is the base points
    const AffineS *t16;       // window table of width 16 over the base points, or null
    uint32_t t16n;            // its points per window
    uint32_t n;
    uint32_t logB;            // buckets in use: 2^logB (2^(c - 1), or fewer for short scalars)
    uint32_t shift;           // every scalar of the job is a multiple of 2^shift
    uint32_t wins;            // windows that can hold nonzero digits (after the shift)
    uint32_t c;               // window width of the job's recode launch
    uint32_t dbl;             // doublings of the reduced sum (the shifted-out factor 2^dbl)
    uint32_t lbase[kMaxLevels - 1];  // first item of the job in reduction levels 1, 2, 3
};

struct DevJobs {
    const JobDesc *jobs;     // count entries
    const uint32_t *sbase;   // scalar prefix over jobs, count + 1
    const uint32_t *bbase;   // first global bucket of each job, count + 1
    const uint32_t *cbase;   // prefix of the jobs' wide-recode chunks (0 for the others), count + 1
    uint32_t count;
};

// Largest i in [lo, hi) with off[i] <= x (off nondecreasing, off[lo] <= x < off[hi]).
__device__ __forceinline__ uint32_t search(const uint32_t *off, uint32_t lo, uint32_t hi, uint32_t x) {
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t upper_index(const uint32_t *off, uint32_t nb, uint32_t x) {
    return search(off, 0, nb, x);
}

template <int C>
__device__ __forceinline__ uint32_t window_bits(const uint32_t (&s)[8], int w) {
    const int pos = w * C;
    const int word = pos >> 5;
    const int off = pos & 31;
    uint32_t lo = word < 8 ? (s[word] >> off) : 0u;
    uint32_t hi = (off + C > 32 && word + 1 < 8) ? (s[word + 1] << (32 - off)) : 0u;
    return (lo | hi) & ((1u << C) - 1u);
}

// s >> k for a 256-bit s held in registers (k < 256), by static word moves
// selected on the bits of k, so that s never needs dynamic indexing.
__device__ __forceinline__ void shr256(uint32_t (&s)[8], uint32_t k) {
#pragma unroll
    for (int step = 4; step >= 1; step >>= 1) {
        if ((k >> 5) & step) {
#pragma unroll
            for (int j = 0; j < 8; j++) s[j] = j + step < 8 ? s[j + step] : 0u;
        }
    }
    const uint32_t b = k & 31;
    if (b) {
#pragma unroll
        for (int j = 0; j < 8; j++) s[j] = __funnelshift_r(s[j], j + 1 < 8 ? s[j + 1] : 0u, b);
    }
}

// Loads a scalar, recentres it, and returns the negation flag.
__device__ __forceinline__ bool load_recentred(const uint32_t *p, uint32_t (&s)[8]) {
    Fr x = fe_load<FrP>(p);
    if (ZK_FAILED(!fe_ge_modulus<FrP>(x), kCheckScalar)) x = fe_zero<FrP>();
    bool neg = fe_gt_half<FrP>(x);
    if (neg) x = fe_neg<FrP>(x);
#pragma unroll
    for (int j = 0; j < 8; j++) s[j] = x.v[j];
    return neg;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Phases 1 and 2 for the jobs [g0, g1) of window width C: with SCATTER false,
// the bucket histogram; with SCATTER true, the (table index << 1 | sign)
// words written bucket by bucket.  The scalars are cut into chunks of
// kRecPer.  A chunk whose scalars all belong to one job that uses a single
// window over at most kSmemBuckets buckets (short scalars) is counted in
// shared memory by one block (k_recode_short), which touches each global
// counter (or cursor) once: quantised values put 2^20 scalars into about a
// hundred buckets, and same-address global atomics serialise.  Every other
// chunk goes through k_recode, one scalar per thread, where lanes with equal
// keys are aggregated into one atomic per warp.  The order of entries within
// a bucket is unspecified (bucket sums do not depend on it).
constexpr uint32_t kRecThreads = 256;
constexpr uint32_t kRecPer = 2048;
constexpr uint32_t kRecEach = kRecPer / kRecThreads;
constexpr uint32_t kSmemBucketsLog = 12;
constexpr uint32_t kSmemBuckets = 1u << kSmemBucketsLog;
constexpr uint32_t kAggLogB = 11;  // bucket sets up to 2^11: warp-aggregated atomics in k_recode

struct Chunk {
    uint32_t first, last, job;
    bool smem;
};

// Chunk k of the scalars of jobs [g0, g1): its range and whether it takes
// the shared-memory path.
__device__ __forceinline__ Chunk rec_chunk(const DevJobs &dj, uint32_t g0, uint32_t g1, uint32_t k) {
    Chunk c;
    c.first = dj.sbase[g0] + k * kRecPer;
    c.last = min(c.first + kRecPer, dj.sbase[g1]) - 1;
    c.job = search(dj.sbase, g0, g1, c.first);
    const JobDesc &J = dj.jobs[c.job];
    c.smem = search(dj.sbase, g0, g1, c.last) == c.job && J.wins == 1 && J.logB <= kSmemBucketsLog;
    return c;
}

template <bool SCATTER>
__global__ void __launch_bounds__(kRecThreads)
    k_recode_short(DevJobs dj, uint32_t g0, uint32_t g1, uint32_t *__restrict__ counts,
                   uint32_t *__restrict__ cursor, uint32_t *__restrict__ sorted, const uint32_t *off0) {
    __shared__ uint32_t hist[kSmemBuckets];
    const Chunk ch = rec_chunk(dj, g0, g1, blockIdx.x);
    if (!ch.smem) return;  // block-uniform
    const JobDesc &J = dj.jobs[ch.job];
    const uint32_t nbj = 1u << J.logB, bb = dj.bbase[ch.job], sb = dj.sbase[ch.job];
    for (uint32_t b = threadIdx.x; b < nbj; b += kRecThreads) hist[b] = 0;
    __syncthreads();
    uint32_t key[kRecEach], word[kRecEach];
#pragma unroll
    for (uint32_t e = 0; e < kRecEach; e++) {
        const uint32_t gid = ch.first + threadIdx.x + e * kRecThreads;
        key[e] = kInvalid;
        if (gid <= ch.last) {
            uint32_t sc[8];
            const bool neg = load_recentred(J.scalars + 8 * (size_t)(gid - sb), sc);
            shr256(sc, J.shift);
            // One window: the shifted scalar is its own digit (below 2^(c' - 1)).
            const uint32_t d = sc[0];
            if (d && ZK_FAILED(d <= nbj, kCheckBucket)) continue;
            if (d) {
                key[e] = d - 1u;
                word[e] = ((gid - sb) << 1) | (neg ? 1u : 0u);
                atomicAdd(&hist[d - 1u], 1u);
            }
        }
    }
    __syncthreads();
    if constexpr (!SCATTER) {
        for (uint32_t b = threadIdx.x; b < nbj; b += kRecThreads)
            if (hist[b]) atomicAdd(&counts[bb + b], hist[b]);
    } else {
        for (uint32_t b = threadIdx.x; b < nbj; b += kRecThreads)
            if (hist[b]) hist[b] = atomicAdd(&cursor[bb + b], hist[b]);
        __syncthreads();
#pragma unroll
        for (uint32_t e = 0; e < kRecEach; e++) {
            if (key[e] == kInvalid) continue;
            const uint32_t pos = atomicAdd(&hist[key[e]], 1u);
            if (ZK_FAILED(!off0 || pos < off0[bb + key[e] + 1], kCheckEntry)) continue;
            sorted[pos] = word[e];
        }
    }
}

template <int C, bool SCATTER>
__global__ void __launch_bounds__(kRecThreads)
    k_recode(DevJobs dj, uint32_t g0, uint32_t g1, uint32_t table_n, uint32_t *__restrict__ counts,
             uint32_t *__restrict__ cursor, uint32_t *__restrict__ sorted, const uint32_t *off0) {
    constexpr int W = (kScalarBits + C - 1) / C;
    static_assert(kRecPer % kRecThreads == 0, "a block lies in one chunk");
    if (rec_chunk(dj, g0, g1, blockIdx.x / kRecEach).smem) return;  // block-uniform
    const uint32_t gid = dj.sbase[g0] + blockIdx.x * kRecThreads + threadIdx.x;
    const bool live = gid < dj.sbase[g1];
    uint32_t sc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t job = g0, i = 0, bb = 0;
    bool neg = false;
    if (live) {
        job = search(dj.sbase, g0, g1, gid);
        i = gid - dj.sbase[job];
        bb = dj.bbase[job];
        neg = load_recentred(dj.jobs[job].scalars + 8 * (size_t)i, sc);
        shr256(sc, dj.jobs[job].shift);
    }
    const uint32_t wins = live ? dj.jobs[job].wins : 0;
    // Windows past every lane's last one hold no digits: stop before them.
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, wins);
    const uint32_t lt_mask = (1u << lane_id()) - 1u;
    // Lanes with equal keys share one atomic only where keys do collide:
    // when the warp holds a job of at most 2^kAggLogB buckets, and in the
    // warp's last window, which may hold only a few bits (254 = 14 x 18 + 2:
    // at width 18 every scalar's top digit lands in three buckets).  Elsewhere
    // 32 lanes among 2^16 buckets almost never meet, and the match costs
    // every window.
    const bool agg_all = __any_sync(0xffffffffu, live && dj.jobs[job].logB <= kAggLogB);
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        if ((uint32_t)w >= wmax) break;
        uint32_t d = ((uint32_t)w < wins ? window_bits<C>(sc, w) : 0u) + carry;
        carry = d > (1u << (C - 1)) ? 1u : 0u;
        int sd = carry ? (int)d - (1 << C) : (int)d;
        uint32_t key = (live && sd != 0) ? bb + (uint32_t)(sd < 0 ? -sd : sd) - 1u : kInvalid;
        if (key != kInvalid && ZK_FAILED(key < dj.bbase[job + 1], kCheckBucket)) key = kInvalid;
        const bool agg = agg_all || (uint32_t)w + 1 == wmax;
        if (!agg) {  // warp-uniform
            if (key == kInvalid) continue;
            if (!SCATTER) {
                atomicAdd(&counts[key], 1u);
            } else {
                const uint32_t pos = atomicAdd(&cursor[key], 1u);
                const uint32_t sign = ((sd < 0) ? 1u : 0u) ^ (neg ? 1u : 0u);
                if (!ZK_FAILED(!off0 || pos < off0[key + 1], kCheckEntry))
                    sorted[pos] = (((uint32_t)w * table_n + i) << 1) | sign;
            }
            continue;
        }
        uint32_t group = __match_any_sync(0xffffffffu, key);
        uint32_t leader = (uint32_t)(__ffs(group) - 1);
        if (!SCATTER) {
            if (key != kInvalid && lane_id() == leader) atomicAdd(&counts[key], (uint32_t)__popc(group));
        } else {
            uint32_t base = 0;
            if (key != kInvalid && lane_id() == leader)
                base = atomicAdd(&cursor[key], (uint32_t)__popc(group));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (key != kInvalid) {
                uint32_t sign = ((sd < 0) ? 1u : 0u) ^ (neg ? 1u : 0u);
                const uint32_t pos = base + __popc(group & lt_mask);
                if (!ZK_FAILED(!off0 || pos < off0[key + 1], kCheckEntry))
                    sorted[pos] = (((uint32_t)w * table_n + i) << 1) | sign;
            }
        }
    }
}

// Phases 1 and 2 for the large jobs of a big batch (a fold-tree level: 512
// jobs of 2^16 scalars): one block per chunk of kWidePer scalars of one job,
// counting the chunk's digits in a shared-memory histogram of the job's
// 2^logB buckets (c <= 16: at most 128 KB), so that one global atomic per
// bucket stands for the chunk's ~kWidePer W / 2^logB digits of that bucket
// instead of one per digit.  With SCATTER the block counts again, reserves
// each bucket's range with one atomic on its cursor, and places the entries
// through shared-memory atomics.  The digits (signed windows) are those of
// k_recode.  Chunk k of jobs [g0, g1) is k - cbase[job] of that job.
constexpr uint32_t kWidePer = 8192;
constexpr uint32_t kWideThreads = 1024;
constexpr uint32_t kWideMaxLogB = 15;
// Shared memory every block requests (at least its histogram): more than half
// of an SM's, so that one block runs per SM.  With three blocks per SM the
// chunks in flight (their scalars, which the scatter pass reads twice, and
// their entries' write ranges) overflowed L2 and the sort of a 512 x 2^16
// batch at width 15 took three times as long (16.7 against 5.4 ms, B300).
constexpr int kWideSmemMin = 128 << 10;
constexpr uint32_t kWideMinN = 1u << 14;  // shorter jobs stay on k_recode / k_recode_short

template <int C>
__device__ __forceinline__ void wide_digits(const JobDesc &J, uint32_t i, uint32_t table_n, uint32_t nbj,
                                            uint32_t *hist, bool place, uint32_t *sorted, const uint32_t *end) {
    constexpr int W = (kScalarBits + C - 1) / C;
    uint32_t sc[8];
    const bool neg = load_recentred(J.scalars + 8 * (size_t)i, sc);
    shr256(sc, J.shift);
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        if ((uint32_t)w >= J.wins) break;
        const uint32_t d = window_bits<C>(sc, w) + carry;
        carry = d > (1u << (C - 1)) ? 1u : 0u;
        const int sd = carry ? (int)d - (1 << C) : (int)d;
        if (sd == 0) continue;
        const uint32_t key = (uint32_t)(sd < 0 ? -sd : sd) - 1u;
        if (ZK_FAILED(key < nbj, kCheckBucket)) continue;
        const uint32_t pos = atomicAdd(&hist[key], 1u);
        if (place && !ZK_FAILED(!end || pos < end[key + 1], kCheckEntry)) {
            const uint32_t sign = ((sd < 0) ? 1u : 0u) ^ (neg ? 1u : 0u);
            sorted[pos] = (((uint32_t)w * table_n + i) << 1) | sign;
        }
    }
}

template <int C, bool SCATTER>
__global__ void __launch_bounds__(kWideThreads)
    k_recode_wide(DevJobs dj, uint32_t g0, uint32_t g1, uint32_t table_n, uint32_t *__restrict__ counts,
                  uint32_t *__restrict__ cursor, uint32_t *__restrict__ sorted, const uint32_t *off0) {
    extern __shared__ uint32_t hist[];
    const uint32_t k = dj.cbase[g0] + blockIdx.x;
    const uint32_t job = search(dj.cbase, g0, g1, k);
    const JobDesc &J = dj.jobs[job];
    const uint32_t first = (k - dj.cbase[job]) * kWidePer, last = min(first + kWidePer, J.n);
    const uint32_t nbj = 1u << J.logB, bb = dj.bbase[job];
    for (uint32_t b = threadIdx.x; b < nbj; b += kWideThreads) hist[b] = 0;
    __syncthreads();
    for (uint32_t i = first + threadIdx.x; i < last; i += kWideThreads)
        wide_digits<C>(J, i, table_n, nbj, hist, false, nullptr, nullptr);
    __syncthreads();
    if constexpr (!SCATTER) {
        for (uint32_t b = threadIdx.x; b < nbj; b += kWideThreads)
            if (hist[b]) atomicAdd(&counts[bb + b], hist[b]);
    } else {
        for (uint32_t b = threadIdx.x; b < nbj; b += kWideThreads)
            if (hist[b]) hist[b] = atomicAdd(&cursor[bb + b], hist[b]);
        __syncthreads();
        for (uint32_t i = first + threadIdx.x; i < last; i += kWideThreads)
            wide_digits<C>(J, i, table_n, nbj, hist, true, sorted, off0 ? off0 + bb : nullptr);
    }
}

// Per job: the largest bit length (st_len[j], initialised to 0) and the
// fewest trailing zeros (st_tz[j], initialised to 0xffffffff) of the
// recentred nonzero scalars.  A block takes kRecPer consecutive scalars;
// when they all belong to one job the block reduces them and makes one
// atomic per statistic, else one per warp and job.
__global__ void __launch_bounds__(kRecThreads)
    k_scalar_stats(DevJobs dj, uint32_t total, uint32_t *__restrict__ st_len, uint32_t *__restrict__ st_tz) {
    __shared__ uint32_t red[2][kRecThreads / 32];
    const uint32_t first = blockIdx.x * kRecPer;
    const uint32_t last = min(first + kRecPer, total) - 1;
    const uint32_t jf = search(dj.sbase, 0, dj.count, first);
    const uint32_t jl = search(dj.sbase, 0, dj.count, last);
    const bool one_job = jf == jl;  // block-uniform
    uint32_t blen = 0, btz = 0xffffffffu;
    for (uint32_t e = 0; e < kRecEach; e++) {
        const uint32_t gid = first + threadIdx.x + e * kRecThreads;
        uint32_t len = 0, tz = 0xffffffffu, job = jf;
        if (gid <= last) {
            if (!one_job) job = search(dj.sbase, jf, jl + 1, gid);
            uint32_t sc[8];
            load_recentred(dj.jobs[job].scalars + 8 * (size_t)(gid - dj.sbase[job]), sc);
#pragma unroll
            for (int j = 7; j >= 0; j--)
                if (!len && sc[j]) len = 32 * j + 32 - __clz(sc[j]);
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (tz == 0xffffffffu && sc[j]) tz = 32 * j + __ffs(sc[j]) - 1;
        }
        if (one_job) {
            blen = max(blen, len);
            btz = min(btz, tz);
            continue;
        }
        // one atomic per warp and job
        const uint32_t key = gid <= last ? job : 0xffffffffu;
        const uint32_t group = __match_any_sync(0xffffffffu, key);
        const uint32_t gl = __reduce_max_sync(group, len);
        const uint32_t gt = __reduce_min_sync(group, tz);
        if (key != 0xffffffffu && lane_id() == (uint32_t)(__ffs(group) - 1)) {
            if (gl) atomicMax(&st_len[key], gl);
            if (gt != 0xffffffffu) atomicMin(&st_tz[key], gt);
        }
    }
    if (!one_job) return;
    blen = __reduce_max_sync(0xffffffffu, blen);
    btz = __reduce_min_sync(0xffffffffu, btz);
    if (lane_id() == 0) {
        red[0][threadIdx.x >> 5] = blen;
        red[1][threadIdx.x >> 5] = btz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < kRecThreads / 32; w++) {
            blen = max(blen, red[0][w]);
            btz = min(btz, red[1][w]);
        }
        if (blen) atomicMax(&st_len[jf], blen);
        if (btz != 0xffffffffu) atomicMin(&st_tz[jf], btz);
    }
}

// Small-scalar plan, one thread per job, from the width statistics: the
// common trailing zeros are shifted out (the result is doubled back at the
// end) and only the windows that can hold digits are used; when the rest
// fits one window (c' = bits + 1 <= c) the digits index the base points
// directly, with 2^(c' - 1) buckets.  When at least 16 trailing zeros are
// shifted out and the base's width-16 window table exists, the single window
// indexes window k = tz / 16 of that table (points 2^(16 k) P_i) instead, so
// the factor 2^(16 k) needs no doublings at the end (quantised values times
// 2^16 have exactly 16).  Jobs whose scalars are all zero get no windows.
// Scalars that are full width keep the host's shape.
__global__ void k_msm_plan(JobDesc *__restrict__ jobs, uint32_t count, const uint32_t *__restrict__ st_len,
                           const uint32_t *__restrict__ st_tz) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    JobDesc &d = jobs[k];
    const uint32_t len = min(st_len[k], (uint32_t)kScalarBits - 1);
    const uint32_t tz = st_tz[k];
    const uint32_t c = d.c;
    if (len == 0) {  // all scalars zero
        d.wins = 0;
        d.shift = 0;
        d.dbl = 0;
        d.logB = kMinWindow - 1;
        d.table = d.wtable;
    } else if (len < (uint32_t)kScalarBits - 1 || tz > 0) {
        const uint32_t sh = min(tz, len - 1);
        const uint32_t eff = len - sh;  // bits left after the shift
        d.shift = sh;
        d.dbl = sh;
        if (eff + 1 <= c) {
            d.wins = 1;
            d.logB = max(eff + 1, (uint32_t)kMinWindow) - 1;
            d.table = d.wtable;  // window 0: the base points
            const uint32_t k16 = min(sh / 16, 15u);
            if (d.t16 && k16 && (sh & 15) <= 1 && eff + (sh & 15) + 1 <= c) {
                d.shift = 16 * k16;
                d.dbl = 0;
                d.logB = max(eff + (sh & 15) + 1, (uint32_t)kMinWindow) - 1;
                d.table = d.t16 + (size_t)k16 * d.t16n;
            }
        } else {
            d.wins = (eff + 1 + c - 1) / c;
        }
    }
}

// Phase 3: bucket sums.  Round 0 cuts the sorted entries into fixed chunks
// of p0 consecutive entries (whatever the bucket boundaries, so every thread
// does the same work) and emits one partial sum (piece) per bucket a chunk
// meets; bucket b's pieces are off1[b] .. off1[b + 1] - 1, in chunk order.
// What completes a bucket depends on its piece count m:
//   m = 1:                the piece is the bucket sum, stored as such;
//   2 <= m <= kThreadMax: one thread per bucket (k_buckets_final);
//   m > kThreadMax:       teams (k_tail_slices, k_tail_buckets): small bucket
//                         sets with many entries each (quantised scalars put
//                         2^20 entries in about a hundred buckets), or a
//                         skewed bucket.
// Empty buckets are set to infinity by k_buckets_final.  The thread path's
// limit is kThreadMax when many buckets hold several pieces (a throughput
// matter), but only kThreadMaxFew when the buckets of more than that many
// pieces fit one wave of tail teams: a small MSM of quantised values has a
// few buckets of 20-30 pieces, whose one-thread chains of full additions set
// its latency (190 us at 2^12 x 4) while a team sums them in a few steps.
// (Completing buckets
// of a few pieces inside round 0 instead -- the last thread to finish one,
// found by a per-bucket counter, adding the others -- made a 2^20 MSM of
// uniform scalars 2 % slower on B300: the fences, atomics and extra registers
// cost the loop more than the separate pass.)
constexpr uint32_t kP0Min = 8;              // smallest round-0 chunk
constexpr uint32_t kThreadMax = 32;
constexpr uint32_t kThreadMaxFew = 4;
constexpr uint32_t kTailBuckets = 4096;     // bucket sets that take longer round-0 chunks (chunk_log)

struct RoundPlan {
    uint32_t p0;   // round-0 chunk (entries per thread)
    int p0neg;     // -p0 (the scan's chunk-count mode)
    uint32_t thr;  // buckets of more pieces take the team tail
};

// Round-0 chunk before the few-bucket multiplier.
__device__ __forceinline__ uint32_t p0_base(uint32_t entries, uint32_t resident) {
    return max(kP0Min, (uint32_t)(((uint64_t)entries + resident - 1) / resident));
}

// Into stat (three words, zeroed by the caller): the largest bucket, the
// number of nonempty buckets, and the number of buckets with more than
// kThreadMaxFew - 1 chunks' worth of entries (about kThreadMaxFew pieces or
// more; the few-bucket multiplier only makes pieces fewer).
__global__ void k_count_max(const uint32_t *__restrict__ counts, uint32_t nb, const uint32_t *total,
                            uint32_t resident, uint32_t *stat) {
    const uint32_t big = (kThreadMaxFew - 1) * p0_base(*total, resident);
    uint32_t m = 0, used = 0, many = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        m = max(m, counts[i]);
        used += counts[i] != 0;
        many += counts[i] > big;
    }
    m = __reduce_max_sync(0xffffffffu, m);
    used = __reduce_add_sync(0xffffffffu, used);
    many = __reduce_add_sync(0xffffffffu, many);
    if (lane_id() == 0 && m) atomicMax(&stat[0], m);
    if (lane_id() == 0 && used) atomicAdd(&stat[1], used);
    if (lane_id() == 0 && many) atomicAdd(&stat[2], many);
}

// Round-0 chunk from the actual entries (their count at off0[nb]): every
// resident thread gets one chunk of p0 = ceil(entries / resident) entries (at
// least kP0Min), so round 0 runs as one wave; 2^chunk_log times more when few
// buckets are in use (fewer pieces for the team tail).
__global__ void k_round_plan(const uint32_t *stat, const uint32_t *total, uint32_t resident, uint32_t chunk_log,
                             uint32_t tail_teams, RoundPlan *plan) {
    if (threadIdx.x || blockIdx.x) return;
    const bool few = stat[1] <= kTailBuckets;
    const uint32_t p0 = p0_base(*total, resident) << (few ? chunk_log : 0u);
    plan->p0 = p0;
    plan->p0neg = -(int)p0;
    plan->thr = stat[2] <= tail_teams ? kThreadMaxFew : kThreadMax;
}

// Stores piece j of bucket b (of m pieces): the bucket sum itself when it is
// the only one.
__device__ __forceinline__ void piece_out(const Xyzz &acc, uint32_t b, uint32_t j, uint32_t m, Xyzz *pieces,
                                          Xyzz *buckets) {
    if (m == 1) buckets[b] = acc;
    else pieces[j] = acc;
}

// Round 0.  Thread c adds entries [c p0, (c + 1) p0).
__global__ void k_pieces_first(const uint32_t *__restrict__ sorted, const uint32_t *__restrict__ off0,
                               const uint32_t *__restrict__ off1, uint32_t nb, DevJobs dj,
                               const RoundPlan *__restrict__ plan, Xyzz *__restrict__ pieces,
                               Xyzz *__restrict__ buckets) {
    const uint32_t p0 = plan->p0;
    const uint32_t total = off0[nb];  // entries (zero digits have none)
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if ((uint64_t)c * p0 >= total) return;
    const uint32_t lo = c * p0, hi = min(lo + p0, total);
    uint32_t b = upper_index(off0, nb, lo);  // bucket holding entry lo
    uint32_t end = off0[b + 1];
    uint32_t job = search(dj.bbase, 0, dj.count, b);
    const AffineS *table = dj.jobs[job].table;
    uint32_t jend = dj.bbase[job + 1];
    Xyzz acc = xyzz_inf();
    for (uint32_t j = lo; j < hi; j++) {
        if (j >= end) {  // bucket b ends inside the chunk
            const uint32_t plo = off1[b];
            piece_out(acc, b, plo + c - off0[b] / p0, off1[b + 1] - plo, pieces, buckets);
            acc = xyzz_inf();
            // The next nonempty bucket: usually b + 1; past a run of empty
            // ones (a short-scalar job uses 2^8 of its 2^(c-1) buckets, so a
            // chunk entering the next job would walk the rest), a search.
            b++;
            if (off0[b + 1] <= j) b = search(off0, b, nb, j);
            end = off0[b + 1];
            if (b >= jend) {
                job = search(dj.bbase, 0, dj.count, b);
                table = dj.jobs[job].table;
                jend = dj.bbase[job + 1];
            }
        }
        const uint32_t v = sorted[j];
        acc = xyzz_add_entry(acc, affines_ldg(table + (v >> 1)), v & 1);
    }
    const uint32_t plo = off1[b];
    piece_out(acc, b, plo + c - off0[b] / p0, off1[b + 1] - plo, pieces, buckets);
}

// Empty buckets (infinity) and buckets of 2 <= m <= kThreadMax pieces, one
// thread per bucket.  Buckets past a job's 2^logB (short scalars) are never
// read and are left alone.
__global__ void k_buckets_final(const Xyzz *__restrict__ pieces, const uint32_t *__restrict__ off1, uint32_t nb,
                                DevJobs dj, const RoundPlan *__restrict__ plan, Xyzz *__restrict__ buckets) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint32_t job = search(dj.bbase, 0, dj.count, b);
    if (b - dj.bbase[job] >= (1u << dj.jobs[job].logB)) return;
    const uint32_t lo = off1[b], m = off1[b + 1] - lo;
    if (m == 0) {
        buckets[b] = xyzz_inf();
        return;
    }
    if (m == 1 || m > plan->thr) return;
    Xyzz acc = pieces[lo];
    for (uint32_t j = lo + 1; j < lo + m; j++) acc = xyzz_add(acc, pieces[j]);
    buckets[b] = acc;
}

// Buckets of more than kThreadMax pieces, on teams, in two levels.  Level A:
// team g sums slice g of a bucket's pieces, at most 32 L of them (lane l adds
// pieces l, l + 32, ..., then a tree over the lanes; L = 2^tail_log);
// bucket b's slices are off_s[b] .. off_s[b + 1] - 1 (a scan of
// ceil(m / 32 L) over those buckets, 0 for the others), and slice k covers
// its pieces 32 L k .. 32 L (k + 1) - 1.  Level B: a team per bucket adds its
// slice sums the same way.  Every team operation spreads one point addition
// over the block's four warps (team.cuh).
constexpr int kBtAcc = 0, kBtIn = 4, kBtTmp = 8, kBtT = 12;

// Team sum of the points src[0 .. cnt - 1] into slots kBtAcc of lane 0
// (block-uniform cnt >= 1; the next point is fetched during each addition).
__device__ __forceinline__ void team_sum(uint32_t *f, const Xyzz *src, uint32_t cnt) {
    const uint32_t l = team_lane();
    tf_store(f, kBtAcc + team_warp(), team_fetch(src + l, l < cnt));
    Fq nx = team_fetch(src + 32 + l, 32 + l < cnt);
    for (uint32_t j = 32; j < cnt; j += 32) {
        tf_store(f, kBtIn + team_warp(), nx);
        nx = team_fetch(src + j + 32 + l, j + 32 + l < cnt);
        __syncthreads();
        team_add(f, kBtAcc, kBtIn, kBtAcc, kBtT);
    }
    __syncthreads();
    for (uint32_t d = 16; d >= 1; d >>= 1) {
        if (d >= cnt) continue;  // lanes d.. hold infinity
        team_shift(f, kBtAcc, kBtTmp, (int)d);
        team_add(f, kBtAcc, kBtTmp, kBtAcc, kBtT);
    }
}

__global__ void __launch_bounds__(kTeamThreads)
    k_tail_slices(const Xyzz *__restrict__ pieces, const uint32_t *__restrict__ off1, uint32_t nb,
                  uint32_t tail_log, const uint32_t *__restrict__ off_s, Xyzz *__restrict__ parts) {
    __shared__ uint32_t f[(kBtT + kTeamTemps) * 8 * 32];
    const uint32_t slice = 32u << tail_log;
    const uint32_t nslices = off_s[nb];
    for (uint32_t g = blockIdx.x; g < nslices; g += gridDim.x) {  // block-uniform
        const uint32_t b = upper_index(off_s, nb, g);
        const uint32_t lo = off1[b] + (g - off_s[b]) * slice;
        const uint32_t hi = min(lo + slice, off1[b + 1]);
        team_sum(f, pieces + lo, hi - lo);
        if (team_lane() == 0) team_put(f, kBtAcc, parts + g);
        __syncthreads();  // the slots are reused by the next slice
    }
}

__global__ void __launch_bounds__(kTeamThreads)
    k_tail_buckets(uint32_t nb, const uint32_t *__restrict__ off_s, const Xyzz *__restrict__ parts,
                   Xyzz *__restrict__ buckets) {
    __shared__ uint32_t f[(kBtT + kTeamTemps) * 8 * 32];
    __shared__ uint32_t multi[kTeamThreads], nmulti;
    // Block k takes buckets k, k + G, k + 2G, ... (G blocks), 128 at a time:
    // one thread per bucket copies a single slice sum, and the buckets with
    // several (a few per block) are summed by the team one by one.  Buckets
    // without slices are complete already.
    const uint32_t mine = blockIdx.x < nb ? (nb - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    for (uint32_t j0 = 0; j0 < mine; j0 += kTeamThreads) {  // block-uniform
        if (threadIdx.x == 0) nmulti = 0;
        __syncthreads();
        const uint32_t j = j0 + threadIdx.x;
        if (j < mine) {
            const uint32_t b = blockIdx.x + j * gridDim.x;
            const uint32_t lo = off_s[b], cnt = off_s[b + 1] - lo;
            if (cnt == 1) buckets[b] = parts[lo];
            else if (cnt > 1) multi[atomicAdd(&nmulti, 1u)] = b;
        }
        __syncthreads();
        const uint32_t nm = nmulti;
        for (uint32_t i = 0; i < nm; i++) {  // block-uniform
            const uint32_t b = multi[i];
            const uint32_t lo = off_s[b];
            team_sum(f, parts + lo, off_s[b + 1] - lo);
            if (team_lane() == 0) team_put(f, kBtAcc, buckets + b);
            __syncthreads();
        }
    }
}

// Host bounds of phase 3 for at most `total` entries in `nb` buckets; the
// actual chunk is decided on the device (k_round_plan).
struct AccumShape {
    size_t cap0;       // pieces of round 0 (bound); also the team tail's slice sums
    uint32_t resident; // threads of one wave of k_pieces_first
    uint32_t blocks;   // its grid
    MsmLayout layout;  // bucket layout (chunk multiplier, tail slices)
};

AccumShape accum_shape(size_t total, uint32_t nb, int sms, const MsmLayout &layout) {
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pieces_first, 128, 0) != cudaSuccess || b < 1) {
            cudaGetLastError();
            b = 1;
        }
        return b;
    }();
    AccumShape a;
    a.layout = layout;
    a.blocks = (uint32_t)std::max(sms, 1) * (uint32_t)per_sm;
    a.resident = a.blocks * 128;
    // p0 >= entries / resident and p0 >= kP0Min bound the chunks, and every
    // chunk emits one piece per bucket it meets.
    const size_t chunks = std::min<size_t>(a.resident, (total + kP0Min - 1) / kP0Min);
    // The team tail's slice sums (at most pieces / 32 + nb) go to a second
    // buffer of the same size.
    a.cap0 = chunks + nb + 1;
    return a;
}

struct AccumBufs {
    uint32_t *off1;   // nb + 1 words: piece offsets
    Xyzz *pieces, *parts;
    uint32_t *stat;   // three words (k_count_max)
    RoundPlan *plan;
    void *scan_tmp;
    uint32_t *offs;   // nb + 1 words: slice offsets of the team tail
};

// Phase 3 launches: sorted entries (offsets off0, histogram counts) -> one
// point per bucket.
int launch_accumulate(const uint32_t *sorted, const uint32_t *counts, const uint32_t *off0, uint32_t nb,
                      const AccumShape &a, const DevJobs &dj, const AccumBufs &w, Xyzz *buckets, int sms,
                      cudaStream_t s) {
    ZK_CUDA_TRY(cudaMemsetAsync(w.stat, 0, 3 * sizeof(uint32_t), s));
    const unsigned mb = (unsigned)std::min<size_t>((nb + 255) / 256, (size_t)sms * 4);
    const unsigned tb = (unsigned)std::min<size_t>(std::max<uint32_t>(nb, 1), (size_t)sms * 8);  // tail teams
    k_count_max<<<std::max(mb, 1u), 256, 0, s>>>(counts, nb, off0 + nb, a.resident, w.stat);
    ZK_LAUNCHED();
    k_round_plan<<<1, 32, 0, s>>>(w.stat, off0 + nb, a.resident, a.layout.chunk_log, tb, w.plan);
    ZK_LAUNCHED();
    ZK_TRY(scan_exclusive(off0, w.off1, nb, -(int)kP0Min, w.scan_tmp, s, nullptr, &w.plan->p0neg));
    k_pieces_first<<<a.blocks, 128, 0, s>>>(sorted, off0, w.off1, nb, dj, w.plan, w.pieces, buckets);
    ZK_LAUNCHED();
    k_buckets_final<<<(nb + 127) / 128, 128, 0, s>>>(w.pieces, w.off1, nb, dj, w.plan, buckets);
    ZK_LAUNCHED();
    // Buckets of more than plan->thr pieces: slices of 32 L pieces.
    ZK_TRY(scan_exclusive(w.off1, w.offs, nb, (int)(32u << a.layout.tail_log), w.scan_tmp, s, nullptr, nullptr,
                          nullptr, kThreadMax, &w.plan->thr));
    k_tail_slices<<<tb, kTeamThreads, 0, s>>>(w.pieces, w.off1, nb, a.layout.tail_log, w.offs, w.parts);
    ZK_LAUNCHED();
    k_tail_buckets<<<tb, kTeamThreads, 0, s>>>(nb, w.offs, w.parts, buckets);
    ZK_LAUNCHED();
    return ZK_OK;
}

// Phase 4: bucket reduction, sum_b (b + 1) S_b per MSM, on teams (team.cuh):
// its scans and trees have few additions in flight, so the latency of one
// addition, not the SM's throughput, sets their time.
//
// Level 0 reads the buckets.  Every level cuts its m items into segments of
// 2^g, and one team reduces one segment: with items k carrying points X_k
// and Y_k (Y = X at level 0),
//     V = sum_k Y_k + 2^f sum_k k X_k,   S = sum_k X_k,
// f the sum of the earlier levels' g.  Segment h of a level becomes item h
// of the next one (X = S, Y = V); for k = 2^g h + j,
//     sum_k Y_k + 2^f sum_k k X_k = sum_h (V_h + 2^(f + g) h S_h),
// so the sum is invariant across levels, and at level 0 it is
// sum_b S_b + sum_b b S_b = sum_b (b + 1) S_b.  The level whose items fit one
// team (at most 32) is final: its V, doubled `dbl` times, is the MSM.
//
// Segments are 2^8 items while a level holds at least 2^13 (many teams, each
// with a serial part), else 2^5 (one item per lane, no serial part), so a
// small bucket set (quantised scalars: 2^8 buckets) spreads over several
// teams instead of one team walking all of them.  The schedule depends only
// on log2 of the bucket count, which the device may lower (short scalars),
// so every kernel derives it from the job's logB.
//
// Within a segment, lane l owns the q = seg / 32 consecutive items
// k = l q + t and runs the suffix form  w_l = sum_t t X_{lq+t}  (adding the
// running sum r of the later items before each new item), r_l = sum_t X;
// then sum_k k X_k = sum_l (w_l + q l r_l) and sum_l l r_l = sum_{l >= 1}
// R_l with R the suffix scan of r over the lanes.
struct RedSched {
    uint32_t levels;
    uint32_t mlog[kMaxLevels];  // log2 of the items at each level
    uint32_t glog[kMaxLevels];  // log2 of the segment (the final level: all items)
};

// With gseq > 0 (large batches), level 0 instead cuts the buckets into
// segments of 2^gseq that one thread each reduces by running sums (k_reduce_seq:
// two additions per bucket, none of the teams' scans and trees); the team
// levels follow.  gseq < kMinWindow - 1 <= logB, so level 0 is never final.
__host__ __device__ constexpr RedSched red_sched(uint32_t logB, uint32_t gbig = 8, uint32_t gsmall = 5,
                                                 uint32_t gseq = 0) {
    RedSched r{};
    uint32_t m = logB;
    uint32_t L0 = 0;
    if (gseq) {
        r.mlog[0] = m;
        r.glog[0] = gseq;
        m -= gseq;
        L0 = 1;
    }
    for (uint32_t L = L0; L < (uint32_t)kMaxLevels; L++) {
        r.mlog[L] = m;
        const uint32_t g = m >= 13 ? gbig : gsmall;
        // A level whose items fit one team, or one segment, is final; so is
        // the last level, which takes what is left.
        if (m <= 5 || g >= m || L + 1 == (uint32_t)kMaxLevels) {
            r.glog[L] = m;
            r.levels = L + 1;
            break;
        }
        r.glog[L] = g;
        m -= g;
    }
    return r;
}

// k_reduce_seq: threads resident per SM (its occupancy at 128 threads per
// block, rounded down) and the longest segment (log2; below kMinWindow - 1).
constexpr uint32_t kSeqThreadsPerSm = 512;
constexpr uint32_t kMaxSeqLog = 5;
static_assert(kMaxSeqLog < (uint32_t)kMinWindow - 1, "level 0 of the sequential schedule is never final");

// Item buffers of levels 1 .. kMaxLevels - 1 (V and S); job j's items of
// level L start at jobs[j].lbase[L - 1].
struct RedBufs {
    Xyzz *v[kMaxLevels];
    Xyzz *s[kMaxLevels];
};

// Shared-memory slots of the reduction team (points take four slots).
constexpr int kSlR = 0, kSlW = 4, kSlYA = 8, kSlIn = 12, kSlYIn = 16, kSlTmp = 20, kSlT = 24;
constexpr int kSlots = kSlT + kTeamTemps;

__global__ void __launch_bounds__(kTeamThreads)
    k_reduce_team(const Xyzz *__restrict__ buckets, RedBufs rb, DevJobs dj, uint32_t level, uint32_t gbig,
                  uint32_t gsmall, uint32_t gseq) {
    __shared__ uint32_t f[kSlots * 8 * 32];
    const uint32_t job = blockIdx.y;
    const JobDesc &J = dj.jobs[job];
    const RedSched r = red_sched(J.logB, gbig, gsmall, gseq);
    if (level >= r.levels) return;  // final at an earlier level
    const bool final_level = level + 1 == r.levels;
    const uint32_t seg = 1u << r.glog[level];
    if (blockIdx.x >= (1u << (r.mlog[level] - r.glog[level]))) return;
    uint32_t fl = 0;  // f: doublings of this level's weights
    for (uint32_t L = 0; L < level; L++) fl += r.glog[L];
    const Xyzz *X, *Y;
    if (level == 0) {
        X = buckets + dj.bbase[job];
        Y = nullptr;
    } else {
        X = rb.s[level] + J.lbase[level - 1];
        Y = rb.v[level] + J.lbase[level - 1];
    }
    X += (size_t)blockIdx.x * seg;
    if (Y) Y += (size_t)blockIdx.x * seg;
    const uint32_t l = team_lane(), w = team_warp();
    const uint32_t q = seg >= 32 ? seg / 32 : 1;

    // Serial part, items t = q - 1 .. 0 of this lane; the next item's
    // coordinate is fetched while the current one is added.  The first item
    // starts the running sums (w stays infinity).
    team_set_inf_nosync(f, kSlW);
    uint32_t k = l * q + (q - 1);
    tf_store(f, kSlR + w, team_fetch(X + k, k < seg));
    if (Y) tf_store(f, kSlYA + w, team_fetch(Y + k, k < seg));
    if (!Y) team_set_inf_nosync(f, kSlYA);
    Fq nx = fe_zero<FqP>(), ny = fe_zero<FqP>();
    if (q > 1) {
        k = l * q + (q - 2);
        nx = team_fetch(X + k, k < seg);
        if (Y) ny = team_fetch(Y + k, k < seg);
    }
    __syncthreads();
    for (uint32_t t = q - 1; t-- > 0;) {
        tf_store(f, kSlIn + w, nx);
        if (Y) tf_store(f, kSlYIn + w, ny);
        if (t > 0) {
            k = l * q + (t - 1);
            nx = team_fetch(X + k, k < seg);
            if (Y) ny = team_fetch(Y + k, k < seg);
        }
        __syncthreads();
        team_add(f, kSlW, kSlR, kSlW, kSlT);  // w += (sum of the later items)
        team_add(f, kSlR, kSlIn, kSlR, kSlT);
        if (Y) team_add(f, kSlYA, kSlYIn, kSlYA, kSlT);
    }
    // Inclusive suffix scan of r over the lanes: R_l = sum_{l' >= l} r_l'
    // (lanes past the segment hold infinity).
    for (uint32_t d = 1; d < 32; d <<= 1) {
        if (d >= seg) break;
        team_shift(f, kSlR, kSlTmp, (int)d);
        team_add(f, kSlR, kSlTmp, kSlR, kSlT);
    }
    // term_l = w_l + q R_l (l >= 1), then u_l = y_l + 2^f term_l.
    team_copy(f, kSlR, kSlTmp, l >= 1);
    for (uint32_t e = q; e > 1; e >>= 1) team_dbl(f, kSlTmp, kSlTmp, kSlT);
    team_add(f, kSlW, kSlTmp, kSlW, kSlT);
    for (uint32_t e = 0; e < fl; e++) team_dbl(f, kSlW, kSlW, kSlT);
    if (Y) team_add(f, kSlW, kSlYA, kSlW, kSlT);
    // Sum over the lanes (lane 0), then sum_k Y_k = R_0 at level 0.
    for (uint32_t d = 16; d >= 1; d >>= 1) {
        if (d >= seg) continue;
        team_shift(f, kSlW, kSlTmp, (int)d);
        team_add(f, kSlW, kSlTmp, kSlW, kSlT);
    }
    if (!Y) team_add(f, kSlW, kSlR, kSlW, kSlT);
    if (final_level) {
        const uint32_t sh = min(J.dbl, (uint32_t)kScalarBits);
        for (uint32_t e = 0; e < sh; e++) team_dbl(f, kSlW, kSlW, kSlT);  // x 2^dbl
        if (threadIdx.x == 0) xyzz_store_canonical(J.out, team_point(f, kSlW));
    } else if (l == 0) {
        const size_t o = J.lbase[level] + blockIdx.x;
        team_put(f, kSlW, rb.v[level + 1] + o);
        team_put(f, kSlR, rb.s[level + 1] + o);
    }
}

// Level 0 of a large batch's reduction (red_sched with gseq > 0): thread t
// takes buckets q t .. q t + q - 1 (q = 2^gseq, in the bucket array's
// layout, jobs at dj.bbase) and, from the top, keeps the running sum r and
// the sum w of the running sums:
//     r = sum_k X_k,   w = sum_j sum_{k >= j} X_k = sum_k (k + 1) X_k,
// i.e. S and V of the segment for f = 0 (Y = X), in 2q - 2 additions.  The
// threads of a job's buckets beyond its device-side 2^logB exit.
__global__ void __launch_bounds__(128, 4)
    k_reduce_seq(const Xyzz *__restrict__ buckets, RedBufs rb, DevJobs dj, uint32_t gseq, uint32_t segs) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= segs) return;
    const uint32_t q = 1u << gseq, b = t << gseq;
    const uint32_t job = search(dj.bbase, 0, dj.count, b);
    const JobDesc &J = dj.jobs[job];
    const uint32_t local = b - dj.bbase[job];
    if (local >= (1u << J.logB)) return;
    // w waits in shared memory while r takes the next bucket, so that one
    // point is live across each addition (the register budget of four
    // blocks per SM).
    __shared__ Xyzz ws[128];
    const Xyzz *X = buckets + b;
    Xyzz r = X[q - 1];
    ws[threadIdx.x] = r;
    for (uint32_t k = q - 1; k-- > 0;) {
        r = xyzz_add(r, X[k]);
        ws[threadIdx.x] = xyzz_add(ws[threadIdx.x], r);
    }
    const size_t o = J.lbase[0] + (local >> gseq);
    rb.v[1][o] = ws[threadIdx.x];
    rb.s[1][o] = r;
}

// Item capacity of reduction level L (1 .. kMaxLevels - 1) and the teams of
// level L (0 ..) for a job whose bucket count may be any 2^logB with
// logB in [lo, hi] (the device lowers logB for short scalars).
constexpr uint32_t red_cap(uint32_t lo, uint32_t hi, uint32_t L, uint32_t gbig = 8, uint32_t gsmall = 5,
                           uint32_t gseq = 0) {
    uint32_t c = 0;
    for (uint32_t b = lo; b <= hi; b++) {
        const RedSched r = red_sched(b, gbig, gsmall, gseq);
        if (L < r.levels) c = std::max(c, 1u << r.mlog[L]);
    }
    return c;
}
constexpr uint32_t red_teams(uint32_t lo, uint32_t hi, uint32_t L, uint32_t gbig = 8, uint32_t gsmall = 5,
                             uint32_t gseq = 0) {
    uint32_t t = 0;
    for (uint32_t b = lo; b <= hi; b++) {
        const RedSched r = red_sched(b, gbig, gsmall, gseq);
        if (L < r.levels) t = std::max(t, 1u << (r.mlog[L] - r.glog[L]));
    }
    return t;
}

// Launches the reduction levels for jobs whose bucket counts are 2^logB with
// logB in [lo[k], hi[k]] (nb buckets in all, in the bucket array's layout).
int launch_reduce(const Xyzz *buckets, const RedBufs &rb, const DevJobs &dj, const uint32_t *lo,
                  const uint32_t *hi, size_t count, uint32_t nb, const MsmLayout &ly, cudaStream_t s) {
    uint32_t level = 0;
    if (ly.seq_log) {
        const uint32_t segs = nb >> ly.seq_log;
        k_reduce_seq<<<(segs + 127) / 128, 128, 0, s>>>(buckets, rb, dj, ly.seq_log, segs);
        ZK_LAUNCHED();
        level = 1;
    }
    for (; level < (uint32_t)kMaxLevels; level++) {
        uint32_t gx = 0;
        for (size_t k = 0; k < count; k++)
            gx = std::max(gx, red_teams(lo[k], hi[k], level, ly.seg_big, ly.seg_small, ly.seq_log));
        if (!gx) break;
        k_reduce_team<<<dim3(gx, (unsigned)count), kTeamThreads, 0, s>>>(buckets, rb, dj, level, ly.seg_big,
                                                                          ly.seg_small, ly.seq_log);
        ZK_LAUNCHED();
    }
    return ZK_OK;
}

// off0: the bucket offsets (scatter pass; the checked build bounds each
// sorted-entry position by its bucket's end).
template <int C, bool SCATTER>
int launch_recode_c(const DevJobs &dj, uint32_t g0, uint32_t g1, uint32_t nscalars,
                    uint32_t table_n, uint32_t *counts, uint32_t *cursor, uint32_t *sorted,
                    const uint32_t *off0, cudaStream_t s) {
    if (nscalars == 0) return ZK_OK;
    k_recode_short<SCATTER><<<(nscalars + kRecPer - 1) / kRecPer, kRecThreads, 0, s>>>(dj, g0, g1, counts,
                                                                                      cursor, sorted, off0);
    ZK_LAUNCHED();
    k_recode<C, SCATTER><<<(nscalars + kRecThreads - 1) / kRecThreads, kRecThreads, 0, s>>>(dj, g0, g1, table_n,
                                                                                          counts, cursor, sorted,
                                                                                          off0);
    ZK_LAUNCHED();
    return ZK_OK;
}

// Jobs [g0, g1) of width C, all on the wide path: `chunks` chunks of
// kWidePer scalars (C <= kWideMaxLogB + 1).
template <int C, bool SCATTER>
int launch_recode_wide_c(const DevJobs &dj, uint32_t g0, uint32_t g1, uint32_t chunks, uint32_t table_n,
                         uint32_t *counts, uint32_t *cursor, uint32_t *sorted, const uint32_t *off0,
                         cudaStream_t s) {
    if constexpr (C - 1 > (int)kWideMaxLogB) {
        return ZK_EINVAL;
    } else {
        if (chunks == 0) return ZK_OK;
        constexpr int kSmem = std::max((1 << (C - 1)) * 4, kWideSmemMin);
        ZK_TRY(set_max_dynamic_smem((const void *)k_recode_wide<C, SCATTER>, kSmem));
        k_recode_wide<C, SCATTER><<<chunks, kWideThreads, kSmem, s>>>(dj, g0, g1, table_n, counts, cursor, sorted,
                                                                     off0);
        ZK_LAUNCHED();
        return ZK_OK;
    }
}

template <bool SCATTER>
int recode_wide(int c, const DevJobs &dj, uint32_t g0, uint32_t g1, uint32_t chunks, uint32_t table_n,
                uint32_t *counts, uint32_t *cursor, uint32_t *sorted, const uint32_t *off0, cudaStream_t s) {
    if (chunks == 0) return ZK_OK;
#define ZK_RECODE_WIDE_CASE(C) \
    case C: return launch_recode_wide_c<C, SCATTER>(dj, g0, g1, chunks, table_n, counts, cursor, sorted, off0, s);
    switch (c) {
        ZK_RECODE_WIDE_CASE(9) ZK_RECODE_WIDE_CASE(10) ZK_RECODE_WIDE_CASE(11) ZK_RECODE_WIDE_CASE(12)
        ZK_RECODE_WIDE_CASE(13) ZK_RECODE_WIDE_CASE(14) ZK_RECODE_WIDE_CASE(15) ZK_RECODE_WIDE_CASE(16)
        default: return ZK_EINVAL;
    }
#undef ZK_RECODE_WIDE_CASE
}

template <bool SCATTER>
int recode(int c, const DevJobs &dj, uint32_t g0, uint32_t g1, uint32_t nscalars, uint32_t table_n,
           uint32_t *counts, uint32_t *cursor, uint32_t *sorted, const uint32_t *off0, cudaStream_t s) {
#define ZK_RECODE_CASE(C) \
    case C: return launch_recode_c<C, SCATTER>(dj, g0, g1, nscalars, table_n, counts, cursor, sorted, off0, s);
    switch (c) {
        ZK_RECODE_CASE(9) ZK_RECODE_CASE(10) ZK_RECODE_CASE(11) ZK_RECODE_CASE(12)
        ZK_RECODE_CASE(13) ZK_RECODE_CASE(14) ZK_RECODE_CASE(15) ZK_RECODE_CASE(16)
        ZK_RECODE_CASE(17) ZK_RECODE_CASE(18) ZK_RECODE_CASE(19) ZK_RECODE_CASE(20)
        default: return ZK_EINVAL;
    }
#undef ZK_RECODE_CASE
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Built-in window width per log2 length when no tuned value is recorded:
// the fastest widths of an autotuner sweep on B300 (single MSMs of uniform
// scalars, 2^10 .. 2^22).  Wider windows cut mixed additions (n ceil(254/c))
// but the bucket reduction's serial depth grows with the bucket count.
int default_window(size_t n) {
    int lg = 0;
    while (((size_t)1 << lg) < n) lg++;
    if (lg <= 10) return 10;
    if (lg <= 11) return 12;
    if (lg <= 13) return 13;
    if (lg <= 18) return 15;
    if (lg <= 19) return 16;
    return 17;
}

}  // namespace

// Built-in bucket layout, the winners of a tuning sweep on B300 (int8 x 2^16
// and uniform scalars, 2^16 .. 2^20; leaf commitments of 2^12): chunk
// multiplier 1, eight items per lane in a tail slice, reduction segments of
// 2^4 (2^5 up to 2^13 points, one team level fewer) and 2^6 (2^8 above 2^18
// points).
MsmLayout msm_layout(const Shared &sh, int lg) {
    MsmLayout m{0, 3, lg <= 13 ? 5u : 4u, lg <= 18 ? 6u : 8u};
    if (lg < 0 || lg > kMaxLogN) return m;
    if (sh.tuned_layout[0][lg]) m.chunk_log = (uint32_t)sh.tuned_layout[0][lg] - 1;
    if (sh.tuned_layout[1][lg]) m.tail_log = (uint32_t)sh.tuned_layout[1][lg] - 1;
    if (sh.tuned_layout[2][lg]) m.seg_small = (uint32_t)sh.tuned_layout[2][lg];
    if (sh.tuned_layout[3][lg]) m.seg_big = (uint32_t)sh.tuned_layout[3][lg];
    return m;
}

// Reads and clears this translation unit's check flags (always 0 in the
// normal build).
int msm_check_read(uint32_t *flags) {
    *flags = 0;
#ifdef ZK_CHECK
    ZK_CUDA_TRY(cudaMemcpyFromSymbol(flags, g_zk_check_flags, sizeof(uint32_t)));
    const uint32_t zero = 0;
    ZK_CUDA_TRY(cudaMemcpyToSymbol(g_zk_check_flags, &zero, sizeof(uint32_t)));
#endif
    return ZK_OK;
}

// Window width of one job of a call of `count` jobs: the tuned width of its
// length, else the built-in one.  The built-in widths suit single MSMs, whose
// bucket reduction is latency bound; in a batch of many jobs it is throughput
// bound (and its first level runs on threads), so a wider window pays
// earlier: 2^17 and 2^18 points take width 16 instead of 15 in calls of at
// least kBatchWindowJobs jobs (256-polynomial CNN batch: 86.7 -> 84.1 ms on
// B300; 2^16 at width 16 and 2^18 at 17 were slower).
constexpr size_t kBatchWindowJobs = 64;

int msm_pick_window(zk_ctx *ctx, size_t n, size_t count) {
    int lg = 0;
    while (((size_t)1 << lg) < n) lg++;
    const Shared &sh = *ctx->sh;
    if (lg <= kMaxLogN && sh.tuned_window[lg]) return sh.tuned_window[lg];
    if (count >= kBatchWindowJobs && (lg == 17 || lg == 18)) return 16;
    return default_window(n);
}

int msm_batch_impl(zk_ctx *ctx, const MsmJob *jobs_in, size_t count, int c_fixed, cudaStream_t s) {
    if (count == 0) return ZK_OK;
    Shared &sh = *ctx->sh;
    size_t total_in = 0;
    for (size_t k = 0; k < count; k++) {
        const MsmJob &m = jobs_in[k];
        if (!m.out || (m.n && !m.scalars)) return ZK_EINVAL;
        if (m.n > sh.srs_n) return ZK_ESRS;
        total_in += m.n;
    }
    if (total_in >= (1ull << 32)) return ZK_EINVAL;
    // Small-scalar path: when the recentred scalars of a job are short (e.g.
    // quantised int8 values times 2^16), its common trailing zeros are
    // shifted out and only the windows that can hold digits are used -- one
    // window when the rest fits, read straight from the base points.  A
    // statistics pass and a plan kernel decide this on the device (k_msm_plan),
    // so the host lays out every job for its full-width shape and nothing is
    // read back; the same launches serve graph capture.  Skipped for tuning
    // runs (fixed c) and for calls too small to pay for the pass.
    const bool stats = c_fixed == 0 && total_in >= kStatsMin;
    struct J {
        MsmJob job;
        int c;
        bool big;  // may take the wide recode path (long enough, histogram fits)
    };
    std::vector<J> jv(count);
    size_t total64 = 0, entries64 = 0, nb64 = 0;
    for (size_t k = 0; k < count; k++) {
        const MsmJob &m = jobs_in[k];
        int c = c_fixed > 0 ? c_fixed : msm_pick_window(ctx, std::max<uint32_t>(m.n, 1), count);
        if (c < kMinWindow || c > kMaxWindow) return ZK_EINVAL;
        jv[k] = {m, c, m.n >= kWideMinN && (uint32_t)c - 1 <= kWideMaxLogB};
        total64 += m.n;
        entries64 += (size_t)m.n * windows_for(c);
        nb64 += (size_t)1 << (c - 1);
    }
    if (nb64 >= (1ull << 31) || entries64 >= (1ull << 32)) return ZK_EINVAL;
    std::stable_sort(jv.begin(), jv.end(), [](const J &a, const J &b) {
        if (a.c != b.c) return a.c < b.c;
        if (a.job.basis != b.job.basis) return a.job.basis < b.job.basis;
        return a.big < b.big;
    });
    // Point tables: the base points (SRS, or the Lagrange basis of H for
    // evaluation-form jobs) and the width's window table of that basis
    // (built on first use, outside timed loops).
    // (The jobs are sorted by width and basis, so each pair's jobs are
    // contiguous: one table lookup per group, sized for its longest job.)
    std::vector<const AffineS *> tabs(count);
    std::vector<uint32_t> tabn(count);
    for (size_t g0 = 0; g0 < count;) {
        const int basis = jv[g0].job.basis;
        size_t g1 = g0, need = 1;
        for (; g1 < count && jv[g1].c == jv[g0].c && jv[g1].job.basis == basis; g1++) {
            if (basis && (!sh.lag[basis].p || jv[g1].job.n != (1u << basis))) return ZK_EINVAL;
            need = std::max(need, (size_t)jv[g1].job.n);
        }
        const WindowTable *t;
        ZK_TRY(table_get(ctx, jv[g0].c, need, basis, &t, s));
        for (size_t k = g0; k < g1; k++) {
            tabs[k] = (const AffineS *)t->buf.p;
            tabn[k] = (uint32_t)t->n;
        }
        g0 = g1;
    }
    // Width-16 tables that already exist (SRS loading builds the SRS's),
    // for the single-window path of scalars with 16 or more trailing zeros.
    std::vector<const AffineS *> t16s(count, nullptr);
    std::vector<uint32_t> t16n(count, 0);
    if (stats) {
        std::lock_guard<std::mutex> g(sh.mu);
        for (size_t k = 0; k < count; k++)
            for (auto &t : sh.tables)
                if (t.c == 16 && t.basis == jv[k].job.basis && t.n >= jv[k].job.n) {
                    t16s[k] = (const AffineS *)t.buf.p;
                    t16n[k] = (uint32_t)t.n;
                    break;
                }
    }
    const uint32_t nb = (uint32_t)nb64;
    const size_t entries_max = entries64;

    // Bucket layout of the call: tuned for the longest job.
    uint32_t maxn = 1;
    for (size_t k = 0; k < count; k++) maxn = std::max(maxn, jv[k].job.n);
    int lgmax = 0;
    while (((size_t)1 << lgmax) < maxn) lgmax++;
    MsmLayout ly = msm_layout(sh, lgmax);
    // The tuned segments suit one MSM, whose reduction is latency bound.  A
    // batch of many MSMs (a fold-tree level: 512 of them; a model's tiny
    // commitments: thousands) keeps every SM busy instead, and there the
    // work of the teams' scans and trees (several additions per bucket)
    // dominates.  When the buckets give every resident thread at least two
    // segments of 2^g (g <= kMaxSeqLog), level 0 runs one thread per segment
    // (two additions per bucket, k_reduce_seq) with the largest such g.
    ly.seq_log = 0;
    {
        const size_t threads = (size_t)std::max(sh.sms, 1) * kSeqThreadsPerSm;
        for (uint32_t g = kMaxSeqLog; g >= 1; g--)
            if ((nb64 >> g) >= 2 * threads) {
                ly.seq_log = g;
                break;
            }
    }
    // Then the team levels' segments grow (the small one first, if any job
    // uses it) while their first level would still hold far more teams than
    // the GPU keeps resident (about six per SM): larger segments amortise
    // each team's scans.
    {
        auto teams0 = [&](uint32_t gb, uint32_t gs) {
            size_t t = 0;
            for (size_t k = 0; k < count; k++) {
                const uint32_t lb = (uint32_t)jv[k].c - 1 - ly.seq_log, g = lb >= 13 ? gb : gs;
                t += lb > g ? (size_t)1 << (lb - g) : 1;
            }
            return t;
        };
        bool small_used = false;
        for (size_t k = 0; k < count; k++) small_used |= jv[k].c - 1 - (int)ly.seq_log < 13;
        const size_t resident = (size_t)std::max(sh.sms, 1) * 6;
        while (teams0(ly.seg_big, ly.seg_small) > 4 * resident) {
            if (small_used && ly.seg_small < 8) ly.seg_small++;
            else if (ly.seg_big < 8) ly.seg_big++;
            else break;
        }
    }
    const AccumShape shape = accum_shape(entries_max, nb, sh.sms, ly);
    const size_t piece_cap = shape.cap0;
    // Reduction levels: a job's bucket count is 2^logB with logB between
    // kMinWindow - 1 (short scalars, decided on the device) and c - 1.
    std::vector<uint32_t> lo(count), hi(count);
    size_t lvl_items[kMaxLevels] = {0, 0, 0, 0};
    for (size_t k = 0; k < count; k++) {
        hi[k] = (uint32_t)(jv[k].c - 1);
        lo[k] = stats ? (uint32_t)(kMinWindow - 1) : hi[k];
        for (uint32_t L = 1; L < (uint32_t)kMaxLevels; L++)
            lvl_items[L] += red_cap(lo[k], hi[k], L, ly.seg_big, ly.seg_small, ly.seq_log);
    }

    // Workspace.
    int err = ZK_OK;
    const size_t jd_bytes = align_up(count * sizeof(JobDesc), 256);
    const size_t pre_bytes = align_up((count + 1) * 4, 256);
    char *jt = (char *)scratch(ctx, "msm.jobs", jd_bytes + 3 * pre_bytes, &err);
    uint32_t *counts = (uint32_t *)scratch(ctx, "msm.counts", (nb + 1) * 4, &err);
    uint32_t *off0 = (uint32_t *)scratch(ctx, "msm.off0", (nb + 1) * 4, &err);
    uint32_t *off1 = (uint32_t *)scratch(ctx, "msm.off1", (nb + 1) * 4, &err);
    uint32_t *cursor = (uint32_t *)scratch(ctx, "msm.cursor", (nb + 1) * 4, &err);
    uint32_t *offs = (uint32_t *)scratch(ctx, "msm.offs", (nb + 1) * 4, &err);
    uint32_t *sorted = (uint32_t *)scratch(ctx, "msm.sorted", std::max<size_t>(entries_max, 1) * 4, &err);
    Xyzz *pa = (Xyzz *)scratch(ctx, "msm.piecea", piece_cap * sizeof(Xyzz), &err);
    Xyzz *pb = (Xyzz *)scratch(ctx, "msm.pieceb", piece_cap * sizeof(Xyzz), &err);
    Xyzz *buckets = (Xyzz *)scratch(ctx, "msm.buckets", nb64 * sizeof(Xyzz), &err);
    static const char *const kRedNames[kMaxLevels][2] = {
        {"", ""}, {"msm.rv1", "msm.rs1"}, {"msm.rv2", "msm.rs2"}, {"msm.rv3", "msm.rs3"}};
    RedBufs rb{};
    bool red_ok = true;
    for (uint32_t L = 1; L < (uint32_t)kMaxLevels; L++) {
        const size_t bytes = std::max<size_t>(lvl_items[L], 1) * sizeof(Xyzz);
        rb.v[L] = (Xyzz *)scratch(ctx, kRedNames[L][0], bytes, &err);
        rb.s[L] = (Xyzz *)scratch(ctx, kRedNames[L][1], bytes, &err);
        red_ok = red_ok && rb.v[L] && rb.s[L];
    }
    void *scan_tmp = scratch(ctx, "msm.scantmp", scan_temp_bytes(nb), &err);
    char *plan = (char *)scratch(ctx, "msm.plan", 256 + sizeof(RoundPlan), &err);
    uint32_t *st = (uint32_t *)scratch(ctx, "msm.stats", 2 * align_up(count * 4, 256), &err);
    if (!jt || !counts || !off0 || !off1 || !cursor || !offs || !sorted || !pa || !pb || !buckets ||
        !red_ok || !scan_tmp || !plan || !st)
        return err;

    // Job table: descriptors and the two prefix arrays.
    std::vector<char> h(jd_bytes + 3 * pre_bytes, 0);
    JobDesc *hd = (JobDesc *)h.data();
    uint32_t *hs = (uint32_t *)(h.data() + jd_bytes);
    uint32_t *hb = (uint32_t *)(h.data() + jd_bytes + pre_bytes);
    uint32_t *hc = (uint32_t *)(h.data() + jd_bytes + 2 * pre_bytes);
    // Wide recode path: per group of one width and table, its big jobs (at
    // the group's end) when their chunks give every SM at least two.
    std::vector<bool> wide(count, false);
    for (size_t g0 = 0; g0 < count;) {
        size_t g1 = g0;
        while (g1 < count && jv[g1].c == jv[g0].c && tabs[g1] == tabs[g0]) g1++;
        size_t chunks = 0;
        for (size_t k = g0; k < g1; k++)
            if (jv[k].big) chunks += (jv[k].job.n + kWidePer - 1) / kWidePer;
        if (chunks >= 2 * (size_t)std::max(sh.sms, 1))
            for (size_t k = g0; k < g1; k++) wide[k] = jv[k].big;
        g0 = g1;
    }
    uint32_t lb[kMaxLevels] = {0, 0, 0, 0};
    for (size_t k = 0; k < count; k++) {
        hd[k].scalars = jv[k].job.scalars;
        hd[k].out = jv[k].job.out;
        hd[k].table = tabs[k];
        hd[k].wtable = tabs[k];
        hd[k].n = jv[k].job.n;
        hd[k].logB = (uint32_t)(jv[k].c - 1);
        hd[k].shift = 0;
        hd[k].wins = (uint32_t)windows_for(jv[k].c);
        hd[k].c = (uint32_t)jv[k].c;
        hd[k].dbl = 0;
        hd[k].t16 = t16s[k];
        hd[k].t16n = t16n[k];
        for (uint32_t L = 1; L < (uint32_t)kMaxLevels; L++) {
            hd[k].lbase[L - 1] = lb[L];
            lb[L] += red_cap(lo[k], hi[k], L, ly.seg_big, ly.seg_small, ly.seq_log);
        }
        hs[k + 1] = hs[k] + jv[k].job.n;
        hb[k + 1] = hb[k] + (1u << (jv[k].c - 1));
        hc[k + 1] = hc[k] + (wide[k] ? (jv[k].job.n + kWidePer - 1) / kWidePer : 0u);
    }
    ZK_TRY(upload(ctx, jt, h.data(), h.size(), s));
    DevJobs dj;
    dj.jobs = (const JobDesc *)jt;
    dj.sbase = (const uint32_t *)(jt + jd_bytes);
    dj.bbase = (const uint32_t *)(jt + jd_bytes + pre_bytes);
    dj.cbase = (const uint32_t *)(jt + jd_bytes + 2 * pre_bytes);
    dj.count = (uint32_t)count;

    // 1-2: width statistics and plan, histogram, offsets, scatter (one
    // recode launch per window width and table).
    PhaseScope ph_sort(ctx, ZK_PHASE_MSM_SORT, s);
    if (stats) {
        uint32_t *st_len = st, *st_tz = st + align_up(count * 4, 256) / 4;
        ZK_CUDA_TRY(cudaMemsetAsync(st_len, 0, count * 4, s));
        ZK_CUDA_TRY(cudaMemsetAsync(st_tz, 0xff, count * 4, s));
        const uint32_t tot = hs[count];
        k_scalar_stats<<<(tot + kRecPer - 1) / kRecPer, kRecThreads, 0, s>>>(dj, tot, st_len, st_tz);
        ZK_LAUNCHED();
        k_msm_plan<<<(unsigned)((count + 127) / 128), 128, 0, s>>>((JobDesc *)jt, (uint32_t)count, st_len, st_tz);
        ZK_LAUNCHED();
    }
    ZK_CUDA_TRY(cudaMemsetAsync(counts, 0, (nb + 1) * 4, s));
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            ZK_TRY(scan_exclusive(counts, off0, nb, 0, scan_tmp, s));
            ZK_CUDA_TRY(cudaMemcpyAsync(cursor, off0, (nb + 1) * 4, cudaMemcpyDeviceToDevice, s));
        }
        for (size_t g0 = 0; g0 < count;) {
            size_t g1 = g0;
            while (g1 < count && jv[g1].c == jv[g0].c && tabs[g1] == tabs[g0]) g1++;
            size_t gw = g0;  // the group's wide jobs are [gw, g1)
            while (gw < g1 && !wide[gw]) gw++;
            const uint32_t ns = hs[gw] - hs[g0], nc = hc[g1] - hc[gw];
            const uint32_t tn = tabn[g0];
            const uint32_t a = (uint32_t)g0, m = (uint32_t)gw, b = (uint32_t)g1;
            if (pass == 0) {
                ZK_TRY(recode<false>(jv[g0].c, dj, a, m, ns, tn, counts, nullptr, nullptr, nullptr, s));
                ZK_TRY(recode_wide<false>(jv[g0].c, dj, m, b, nc, tn, counts, nullptr, nullptr, nullptr, s));
            } else {
                ZK_TRY(recode<true>(jv[g0].c, dj, a, m, ns, tn, nullptr, cursor, sorted, off0, s));
                ZK_TRY(recode_wide<true>(jv[g0].c, dj, m, b, nc, tn, nullptr, cursor, sorted, off0, s));
            }
            g0 = g1;
        }
    }
    ph_sort.end();

    // 3: bucket sums.
    PhaseScope ph_accum(ctx, ZK_PHASE_MSM_ACCUM, s);
    const AccumBufs ab{off1, pa, pb, (uint32_t *)plan, (RoundPlan *)(plan + 256), scan_tmp, offs};
    ZK_TRY(launch_accumulate(sorted, counts, off0, nb, shape, dj, ab, buckets, sh.sms, s));
    ph_accum.end();

    // 4-5: bucket reduction and output.
    PhaseScope ph_reduce(ctx, ZK_PHASE_MSM_REDUCE, s);
    return launch_reduce(buckets, rb, dj, lo.data(), hi.data(), count, nb, ly, s);
}

}  // namespace zk

// ---------------------------------------------------------------------------
// Allocation-free commitment (zk_commit_noalloc).
//
// Some callers cannot call cudaMalloc: a host thread that must never block on
// the device-wide synchronisation cudaFree implies, or a process whose device
// memory is all owned by another allocator (a framework's caching allocator
// that reserved the HBM up front).  For them the MSM below runs the same
// kernels as msm_batch_impl with its whole workspace in one fixed device
// array compiled into this library, sized for one MSM of at most
// kNoAllocMaxN points at window width 16.  Every GPU that loads the library
// holds the array until the process exits.
// ---------------------------------------------------------------------------

namespace zk {

namespace {

constexpr uint32_t kNoAllocMaxN = 1u << 12;
constexpr int kNoAllocC = 16;
constexpr uint32_t kNoAllocB = 1u << (kNoAllocC - 1);
constexpr uint32_t kNoAllocW = (kScalarBits + kNoAllocC - 1) / kNoAllocC;
constexpr size_t kNoAllocEntries = (size_t)kNoAllocMaxN * kNoAllocW;
constexpr size_t kNoAllocPieces = kNoAllocEntries / kP0Min + kNoAllocB + 1;
// Reduction items of levels 1 and 2 (2^15 buckets: levels of 2^15, 2^7 and 2^2 items).
constexpr size_t kNoAllocL1 = red_cap(kNoAllocC - 1, kNoAllocC - 1, 1);
constexpr size_t kNoAllocL2 = red_cap(kNoAllocC - 1, kNoAllocC - 1, 2);
static_assert(red_cap(kNoAllocC - 1, kNoAllocC - 1, 3) == 0, "no-alloc reduction levels");
constexpr size_t kNoAllocPre = 256;  // one prefix array of the job table

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
// Workspace layout (byte offsets).
constexpr size_t kNaJobs = 0;                                          // JobDesc + 2 prefixes
constexpr size_t kNaCounts = kNaJobs + 256 + 2 * kNoAllocPre;
constexpr size_t kNaOff0 = kNaCounts + na_align((kNoAllocB + 1) * 4);
constexpr size_t kNaOff1 = kNaOff0 + na_align((kNoAllocB + 1) * 4);
constexpr size_t kNaCursor = kNaOff1 + na_align((kNoAllocB + 1) * 4);
constexpr size_t kNaOffS = kNaCursor + na_align((kNoAllocB + 1) * 4);
constexpr size_t kNaSorted = kNaOffS + na_align((kNoAllocB + 1) * 4);
constexpr size_t kNaPieceA = kNaSorted + na_align(kNoAllocEntries * 4);
constexpr size_t kNaPieceB = kNaPieceA + na_align(kNoAllocPieces * sizeof(Xyzz));
constexpr size_t kNaBuckets = kNaPieceB + na_align(kNoAllocPieces * sizeof(Xyzz));
constexpr size_t kNaV1 = kNaBuckets + na_align(kNoAllocB * sizeof(Xyzz));
constexpr size_t kNaS1 = kNaV1 + na_align(kNoAllocL1 * sizeof(Xyzz));
constexpr size_t kNaV2 = kNaS1 + na_align(kNoAllocL1 * sizeof(Xyzz));
constexpr size_t kNaS2 = kNaV2 + na_align(kNoAllocL2 * sizeof(Xyzz));
constexpr size_t kNaScan = kNaS2 + na_align(kNoAllocL2 * sizeof(Xyzz));
constexpr size_t kNaPlan = kNaScan + na_align(((size_t)kNoAllocB / 2048 + 2) * 4);
constexpr size_t kNoAllocBytes = kNaPlan + 256 + na_align(sizeof(RoundPlan));

// The workspace.  Host code must not use this name as an address: it is a
// host-side stand-in.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_ws[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices];

// Device address of g_noalloc_ws on the current device (looked up once per
// device, with that device current).
int noalloc_workspace(int device, unsigned char **out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return ZK_EINVAL;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) {
            cudaGetLastError();
            return ZK_ECUDA;
        }
        g_noalloc_addr[device] = p;
    }
    *out = (unsigned char *)g_noalloc_addr[device];
    return ZK_OK;
}

// Writes the one-job table (descriptor and prefix arrays) that the MSM
// kernels read, without a host-to-device copy.
__global__ void k_noalloc_jobs(unsigned char *ws, const uint32_t *scalars, uint32_t n, void *out,
                               const AffineS *table) {
    if (threadIdx.x || blockIdx.x) return;
    JobDesc *d = reinterpret_cast<JobDesc *>(ws + kNaJobs);
    d->scalars = scalars;
    d->out = out;
    d->table = table;  // no plan kernel runs: always the full-width shape
    d->wtable = table;
    d->t16 = nullptr;
    d->t16n = 0;
    d->n = n;
    d->logB = kNoAllocC - 1;
    d->shift = 0;
    d->wins = kNoAllocW;
    d->c = kNoAllocC;
    d->dbl = 0;
    for (int L = 0; L < kMaxLevels - 1; L++) d->lbase[L] = 0;
    uint32_t *sb = reinterpret_cast<uint32_t *>(ws + kNaJobs + 256);
    uint32_t *bb = sb + kNoAllocPre / 4;
    sb[0] = 0;
    sb[1] = n;
    bb[0] = 0;
    bb[1] = kNoAllocB;
}

}  // namespace

}  // namespace zk

extern "C" int zk_commit_noalloc(zk_ctx *ctx, const zk_fr *coeffs, size_t n, zk_g1 *out,
                                 zk_stream stream) {
    ZK_NVTX("zk_commit_noalloc");
    using namespace zk;
    if (!ctx || !coeffs || !out || n == 0) return ZK_EINVAL;
    if (n > kNoAllocMaxN) return ZK_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    const int device = ctx->sh->device;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    struct Restore {
        int prev, dev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, device};
    if (!is_device_ptr(coeffs) || !is_device_ptr(out)) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    if (sh.srs_n == 0 || n > sh.srs_n) return ZK_ESRS;
    const WindowTable *tab = nullptr;
    {
        std::lock_guard<std::mutex> g(sh.mu);
        for (auto &t : sh.tables)
            if (t.c == kNoAllocC && t.basis == 0 && t.n >= n) tab = &t;
    }
    if (!tab) return ZK_ESRS;  // the c = 16 table is built when the SRS is loaded
    unsigned char *ws = nullptr;
    ZK_TRY(noalloc_workspace(device, &ws));
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t nb = kNoAllocB;
    uint32_t *counts = (uint32_t *)(ws + kNaCounts);
    uint32_t *off0 = (uint32_t *)(ws + kNaOff0);
    uint32_t *off1 = (uint32_t *)(ws + kNaOff1);
    uint32_t *cursor = (uint32_t *)(ws + kNaCursor);
    uint32_t *sorted = (uint32_t *)(ws + kNaSorted);
    Xyzz *pa = (Xyzz *)(ws + kNaPieceA);
    Xyzz *pb = (Xyzz *)(ws + kNaPieceB);
    Xyzz *buckets = (Xyzz *)(ws + kNaBuckets);
    RedBufs rb{};
    rb.v[1] = (Xyzz *)(ws + kNaV1);
    rb.s[1] = (Xyzz *)(ws + kNaS1);
    rb.v[2] = (Xyzz *)(ws + kNaV2);
    rb.s[2] = (Xyzz *)(ws + kNaS2);  // level 3 never runs (2^15 buckets)
    void *scan_tmp = ws + kNaScan;

    k_noalloc_jobs<<<1, 1, 0, s>>>(ws, (const uint32_t *)coeffs, (uint32_t)n, out,
                                   (const AffineS *)tab->buf.p);
    ZK_LAUNCHED();
    DevJobs dj;
    dj.jobs = (const JobDesc *)(ws + kNaJobs);
    dj.sbase = (const uint32_t *)(ws + kNaJobs + 256);
    dj.bbase = dj.sbase + kNoAllocPre / 4;
    dj.cbase = nullptr;  // no wide recode chunks
    dj.count = 1;
    const uint32_t total = (uint32_t)n;
    // The workspace keeps the previous call's contents: the histogram must
    // start at zero; every other region is fully written before it is read.
    ZK_CUDA_TRY(cudaMemsetAsync(counts, 0, (nb + 1) * 4, s));
    ZK_TRY((launch_recode_c<kNoAllocC, false>(dj, 0, 1, total, (uint32_t)tab->n, counts, nullptr,
                                               nullptr, nullptr, s)));
    ZK_TRY(scan_exclusive(counts, off0, nb, 0, scan_tmp, s));
    ZK_CUDA_TRY(cudaMemcpyAsync(cursor, off0, (nb + 1) * 4, cudaMemcpyDeviceToDevice, s));
    ZK_TRY((launch_recode_c<kNoAllocC, true>(dj, 0, 1, total, (uint32_t)tab->n, nullptr, cursor,
                                              sorted, off0, s)));
    // The built-in layout (the workspace is sized for it).
    const MsmLayout ly{0, 1, 5, 8};
    const AccumShape shape = accum_shape((size_t)n * kNoAllocW, nb, sh.sms, ly);
    if (shape.cap0 > kNoAllocPieces) return ZK_EINVAL;  // cannot happen: p0 >= kP0Min
    const AccumBufs ab{off1, pa, pb, (uint32_t *)(ws + kNaPlan), (RoundPlan *)(ws + kNaPlan + 256),
                       scan_tmp, (uint32_t *)(ws + kNaOffS)};
    ZK_TRY(launch_accumulate(sorted, counts, off0, nb, shape, dj, ab, buckets, sh.sms, s));
    const uint32_t logB = kNoAllocC - 1;
    return launch_reduce(buckets, rb, dj, &logB, &logB, 1, kNoAllocB, ly, s);
}
