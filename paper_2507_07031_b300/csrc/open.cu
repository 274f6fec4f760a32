// open.cu -- KZG opening proofs (paper Sec. 2.1): for f = sum_k c_k X^k and a
// point x, y = f(x) and the proof [q(tau)]_1 with q(X) = (f(X) - y) / (X - x);
// batched at one point, y_i = f_i(x) and the proof of
// h(X) = sum_i gamma^i (f_i(X) - f_i(x)) / (X - x), the quotient of
// F = sum_i gamma^i f_i.
//
// Synthetic division by (X - x) is the suffix recurrence
//     Q_n = 0,   Q_k = c_k + x Q_{k+1},   y = Q_0,   q_{k-1} = Q_k,
// a first-order linear recurrence, evaluated as a scan:
//   1. k_open_local: each thread runs the recurrence over one chunk of
//      kOpenL coefficients from 0, giving the chunk's map
//      Q_start = B + x^kOpenL Q_after;
//   2. k_open_scan: one block per polynomial; each thread folds a run of
//      chunk maps, the threads' maps (a, b) are combined by a suffix scan
//      under (a1, b1) o (a2, b2) = (a1 a2, b1 + a1 b2), and each thread
//      re-runs its chunks from its true incoming value, leaving the value that
//      enters every chunk (and y = Q_0);
//   3. k_open_quot: each chunk re-runs its recurrence from its incoming value
//      and writes its quotient coefficients.
// That is 2 products per coefficient plus a logarithmic scan, against the n
// dependent products of a sequential division; the proof is then one MSM.
// Values stay canonical: the multipliers x, x^kOpenL and gamma are kept in
// Montgomery form, so mont(v, x R) = v x.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "curve.cuh"

namespace zk {

namespace {

constexpr int kOpenLog = 5;
constexpr uint32_t kOpenL = 1u << kOpenLog;  // coefficients per chunk
constexpr int kOpenT = 256;                  // threads of the scan block

struct OpenJob {
    const uint32_t *c;  // n canonical coefficients
    uint32_t n;
    uint32_t *y;        // where f(x) goes (canonical), or null
};

struct OpenJobs {
    const OpenJob *jobs;
    const uint32_t *cpre;  // first chunk of each job, count + 1
    uint32_t count;
    const uint32_t *x;     // canonical
};

ZK_DEV uint32_t open_search(const uint32_t *pre, uint32_t count, uint32_t g) {
    uint32_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

ZK_DEV Fr fr_ld(const uint32_t *p) { return fe_load<FrP>(p); }

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// (a R)^e in Montgomery form by square-and-multiply.
ZK_DEV Fr mont_pow(const Fr &aR, uint32_t e) {
    Fr r = fe_mont_one<FrP>(), b = aR;
    while (e) {
        if (e & 1) r = fe_mul<FrP>(r, b);
        b = fe_mul<FrP>(b, b);
        e >>= 1;
    }
    return r;
}

__global__ void k_open_local(OpenJobs oj, uint32_t chunks, uint32_t *__restrict__ B) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= chunks) return;
    const uint32_t job = open_search(oj.cpre, oj.count, g);
    const OpenJob J = oj.jobs[job];
    const uint32_t lo = (g - oj.cpre[job]) * kOpenL, hi = min(lo + kOpenL, J.n);
    const Fr xR = fe_to_mont<FrP>(fr_ld(oj.x));
    Fr v = fe_zero<FrP>();
    for (uint32_t k = hi; k-- > lo;) v = fe_add<FrP>(fr_ld(J.c + 8 * (size_t)k), fe_mul<FrP>(v, xR));
    fe_store<FrP>(B + 8 * (size_t)g, v);
}

__global__ void __launch_bounds__(kOpenT)
    k_open_scan(OpenJobs oj, const uint32_t *__restrict__ B, uint32_t *__restrict__ Qin) {
    __shared__ uint32_t sa[2][8][kOpenT], sb[2][8][kOpenT];
    const uint32_t job = blockIdx.x, t = threadIdx.x;
    const OpenJob J = oj.jobs[job];
    const uint32_t base = oj.cpre[job], m = oj.cpre[job + 1] - base;
    const uint32_t C = (m + kOpenT - 1) / kOpenT;
    const uint32_t lo = min(t * C, m), hi = min(lo + C, m);
    const Fr xR = fe_to_mont<FrP>(fr_ld(oj.x));
    Fr XR = xR;
    for (int i = 0; i < kOpenLog; i++) XR = fe_mul<FrP>(XR, XR);  // x^kOpenL R
    // this thread's chunks folded from 0: map Q_start = v + a Q_after
    Fr v = fe_zero<FrP>();
    for (uint32_t g = hi; g-- > lo;) v = fe_add<FrP>(fr_ld(B + 8 * (size_t)(base + g)), fe_mul<FrP>(v, XR));
    Fr a = mont_pow(XR, hi - lo);
    // suffix scan of the maps over the threads
    int cur = 0;
    for (int w = 0; w < 8; w++) {
        sa[cur][w][t] = a.v[w];
        sb[cur][w][t] = v.v[w];
    }
    __syncthreads();
    for (uint32_t d = 1; d < (uint32_t)kOpenT; d <<= 1) {
        if (t + d < (uint32_t)kOpenT) {
            Fr a2, b2;
            for (int w = 0; w < 8; w++) {
                a2.v[w] = sa[cur][w][t + d];
                b2.v[w] = sb[cur][w][t + d];
            }
            v = fe_add<FrP>(v, fe_mul<FrP>(b2, a));
            a = fe_mul<FrP>(a, a2);
        }
        for (int w = 0; w < 8; w++) {
            sa[cur ^ 1][w][t] = a.v[w];
            sb[cur ^ 1][w][t] = v.v[w];
        }
        cur ^= 1;
        __syncthreads();
    }
    // value entering this thread's chunks: Q at the start of the next thread's
    Fr q = fe_zero<FrP>();
    if (t + 1 < (uint32_t)kOpenT)
        for (int w = 0; w < 8; w++) q.v[w] = sb[cur][w][t + 1];
    for (uint32_t g = hi; g-- > lo;) {
        fe_store<FrP>(Qin + 8 * (size_t)(base + g), q);
        q = fe_add<FrP>(fr_ld(B + 8 * (size_t)(base + g)), fe_mul<FrP>(q, XR));
    }
    if (t == 0 && J.y) fe_store<FrP>(J.y, q);  // Q_0 = f(x)
}

// Quotient coefficients of job `job`: q_{k-1} = Q_k for k >= 1.
__global__ void k_open_quot(OpenJobs oj, uint32_t job, const uint32_t *__restrict__ Qin,
                            uint32_t *__restrict__ q) {
    const OpenJob J = oj.jobs[job];
    const uint32_t base = oj.cpre[job], m = oj.cpre[job + 1] - base;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= m) return;
    const uint32_t lo = g * kOpenL, hi = min(lo + kOpenL, J.n);
    const Fr xR = fe_to_mont<FrP>(fr_ld(oj.x));
    Fr v = fr_ld(Qin + 8 * (size_t)(base + g));
    for (uint32_t k = hi; k-- > lo;) {
        v = fe_add<FrP>(fr_ld(J.c + 8 * (size_t)k), fe_mul<FrP>(v, xR));
        if (k >= 1) fe_store<FrP>(q + 8 * (size_t)(k - 1), v);
    }
}

// F_j = sum_i gamma^i f_i[j] (zero past a polynomial's length), by Horner
// over i.
__global__ void k_open_rlc(const uint32_t *const *__restrict__ polys, const uint32_t *__restrict__ lens,
                           uint32_t count, const uint32_t *__restrict__ gamma, uint32_t nmax,
                           uint32_t *__restrict__ F) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nmax) return;
    const Fr gR = fe_to_mont<FrP>(fr_ld(gamma));
    Fr acc = fe_zero<FrP>();
    for (uint32_t i = count; i-- > 0;) {
        acc = fe_mul<FrP>(acc, gR);
        if (j < lens[i]) acc = fe_add<FrP>(acc, fr_ld(polys[i] + 8 * (size_t)j));
    }
    fe_store<FrP>(F + 8 * (size_t)j, acc);
}

}  // namespace

int open_impl(zk_ctx *ctx, const uint32_t *const *polys, const size_t *lens, size_t count, const uint32_t *x,
              const uint32_t *gamma, uint32_t *ys, uint32_t *quotient, uint32_t *proof, cudaStream_t s) {
    if (count == 0 || !x || !proof || (count > 1 && !gamma)) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    size_t nmax = 0;
    for (size_t i = 0; i < count; i++) {
        if (!polys[i] || lens[i] == 0 || lens[i] > ((size_t)1 << 31)) return ZK_EINVAL;
        nmax = std::max(nmax, lens[i]);
    }
    if (nmax - 1 > sh.srs_n) return ZK_ESRS;
    const bool batch = gamma != nullptr;
    // Jobs: with gamma, one evaluation per polynomial and the quotient of the
    // combination F; without, the polynomial itself (evaluated and divided).
    int err = ZK_OK;
    const uint32_t *F = polys[0];
    if (batch) {
        uint32_t *Fw = (uint32_t *)scratch(ctx, "open.F", nmax * 32, &err);
        const size_t tb = align_up(count * sizeof(void *), 256);
        char *tab = (char *)scratch(ctx, "open.polys", tb + count * 4, &err);
        if (!Fw || !tab) return err;
        std::vector<char> h(tb + count * 4, 0);
        for (size_t i = 0; i < count; i++) {
            ((const uint32_t **)h.data())[i] = polys[i];
            ((uint32_t *)(h.data() + tb))[i] = (uint32_t)lens[i];
        }
        ZK_TRY(upload(ctx, tab, h.data(), h.size(), s));
        k_open_rlc<<<(unsigned)((nmax + 127) / 128), 128, 0, s>>>((const uint32_t *const *)tab,
                                                                 (const uint32_t *)(tab + tb), (uint32_t)count,
                                                                 gamma, (uint32_t)nmax, Fw);
        ZK_LAUNCHED();
        F = Fw;
    }
    const size_t njobs = batch ? count + 1 : 1;
    std::vector<OpenJob> jobs(njobs);
    if (batch)
        for (size_t i = 0; i < count; i++) jobs[i] = {polys[i], (uint32_t)lens[i], ys ? ys + 8 * i : nullptr};
    jobs[njobs - 1] = {F, (uint32_t)nmax, batch ? nullptr : ys};
    std::vector<uint32_t> cpre(njobs + 1, 0);
    for (size_t i = 0; i < njobs; i++) cpre[i + 1] = cpre[i] + (jobs[i].n + kOpenL - 1) / kOpenL;
    const uint32_t chunks = cpre[njobs];
    const size_t jb = align_up(njobs * sizeof(OpenJob), 256);
    char *jt = (char *)scratch(ctx, "open.jobs", jb + (njobs + 1) * 4, &err);
    uint32_t *B = (uint32_t *)scratch(ctx, "open.B", (size_t)chunks * 32, &err);
    uint32_t *Qin = (uint32_t *)scratch(ctx, "open.Qin", (size_t)chunks * 32, &err);
    uint32_t *q = quotient;
    if (!q) q = (uint32_t *)scratch(ctx, "open.q", std::max<size_t>(nmax - 1, 1) * 32, &err);
    if (!jt || !B || !Qin || !q) return err;
    std::vector<char> h(jb + (njobs + 1) * 4, 0);
    memcpy(h.data(), jobs.data(), njobs * sizeof(OpenJob));
    memcpy(h.data() + jb, cpre.data(), (njobs + 1) * 4);
    ZK_TRY(upload(ctx, jt, h.data(), h.size(), s));
    const OpenJobs oj{(const OpenJob *)jt, (const uint32_t *)(jt + jb), (uint32_t)njobs, x};
    k_open_local<<<(chunks + 127) / 128, 128, 0, s>>>(oj, chunks, B);
    ZK_LAUNCHED();
    k_open_scan<<<(unsigned)njobs, kOpenT, 0, s>>>(oj, B, Qin);
    ZK_LAUNCHED();
    const uint32_t qchunks = cpre[njobs] - cpre[njobs - 1];
    k_open_quot<<<(qchunks + 127) / 128, 128, 0, s>>>(oj, (uint32_t)(njobs - 1), Qin, q);
    ZK_LAUNCHED();
    if (nmax == 1) {  // constant polynomial: the quotient is 0, the proof infinity
        ZK_CUDA_TRY(cudaMemsetAsync(proof, 0, 64, s));
        return ZK_OK;
    }
    MsmJob mj;
    mj.scalars = q;
    mj.n = (uint32_t)(nmax - 1);
    mj.out = proof;
    return msm_batch_impl(ctx, &mj, 1, 0, s);
}

}  // namespace zk
