// lagrange.cu -- the Lagrange basis [L_k(tau)]_1 of H = <omega_n>, derived
// from the SRS, so that a vector of evaluations over H is committed without
// interpolating it first.
//
// The commitment of the interpolant f of v over H (paper Sec. 2.1 and
// Sec. 4.4.1: com = [f(tau)]_1, f|_H = v) equals sum_k v_k [L_k(tau)]_1 with
// L_k(X) = n^{-1} sum_j omega^{-jk} X^j.  Hence the basis points are the
// inverse DFT over G1 of the first n SRS points:
//   [L_k(tau)]_1 = n^{-1} sum_j omega^{-jk} [tau^j]_1.
// It is computed once per size with radix-2 Stockham stages (natural order
// in and out), one kernel per stage; each butterfly multiplies one point by
// its twiddle (a full scalar multiplication), then a final pass multiplies by
// n^{-1} and normalises to affine.  The MSM then reads evaluation vectors
// directly: quantised witness values keep their short scalars (one window)
// instead of becoming full-width coefficients after an INTT.
#include <cuda_runtime.h>

#include "ctx.cuh"
#include "curve.cuh"

namespace zk {

namespace {

__global__ void k_lag_load(const Affine *__restrict__ srs, Xyzz *__restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = xyzz_from_affine(srs[i]);
}

// One inverse radix-2 Stockham stage: for j < n/2, with m = j mod Ns,
//   v1 = x[j + n/2] * omega_{2 Ns}^{-m},  y[(j / Ns) 2 Ns + m] = x[j] + v1,
//   y[(j / Ns) 2 Ns + m + Ns] = x[j] - v1.
__global__ void k_lag_stage(const Xyzz *__restrict__ in, Xyzz *__restrict__ out, uint32_t lg,
                            uint32_t logNs, const Fr *__restrict__ tw) {
    const size_t n = (size_t)1 << lg;
    const size_t half = n >> 1;
    size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (j >= half) return;
    const size_t Ns = (size_t)1 << logNs;
    const size_t m = j & (Ns - 1);
    Xyzz a = in[j];
    Xyzz b = in[j + half];
    const size_t e = m << (lg - 1 - logNs);  // omega_{2 Ns}^m = omega_n^{m n / (2 Ns)}
    if (e) {
        Fr w = fe_from_mont<FrP>(tw[n - e]);  // omega_n^{-e}
        b = xyzz_mul(b, w.v);
    }
    const size_t dst = ((j >> logNs) << (logNs + 1)) + m;
    out[dst] = xyzz_add(a, b);
    out[dst + Ns] = xyzz_add(a, xyzz_neg(b));
}

__global__ void k_lag_scale(Xyzz *__restrict__ p, size_t n, const Fr *__restrict__ ninv) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Fr k = fe_from_mont<FrP>(*ninv);
    p[i] = xyzz_mul(p[i], k.v);
}

}  // namespace

int lagrange_get(zk_ctx *ctx, int lg, const Affine **out, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    if (lg < 1 || lg > kMaxSrsLog) return ZK_EINVAL;
    const size_t n = (size_t)1 << lg;
    if (sh.srs_n < n) return ZK_ESRS;
    const uint32_t *tw;
    ZK_TRY(twiddles(ctx, lg, &tw, s));  // takes the shared lock itself
    std::lock_guard<std::mutex> g(sh.mu);
    if (!sh.lag[lg].p) {
        if (ctx->capturing) return ZK_EINVAL;
        int err = ZK_OK;
        Xyzz *a = (Xyzz *)scratch(ctx, "lag.a", n * sizeof(Xyzz), &err);
        Xyzz *b = (Xyzz *)scratch(ctx, "lag.b", n * sizeof(Xyzz), &err);
        if (!a || !b) return err;
        DevBuf buf;
        ZK_TRY(dev_alloc(sh, buf, n * sizeof(Affine)));
        const unsigned blocks = (unsigned)((n + 127) / 128);
        k_lag_load<<<blocks, 128, 0, s>>>((const Affine *)sh.srs.p, a, n);
        ZK_LAUNCHED();
        for (int st = 0; st < lg; st++) {
            k_lag_stage<<<(unsigned)((n / 2 + 127) / 128), 128, 0, s>>>(a, b, (uint32_t)lg, (uint32_t)st,
                                                                       (const Fr *)tw);
            ZK_LAUNCHED();
            std::swap(a, b);
        }
        k_lag_scale<<<blocks, 128, 0, s>>>(a, n, (const Fr *)tw + n);
        ZK_LAUNCHED();
        int rc = normalize_points(ctx, a, (Affine *)buf.p, n, s);
        if (rc == ZK_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = ZK_ECUDA;
        if (rc != ZK_OK) {
            dev_free(sh, buf);
            return rc;
        }
        sh.lag[lg] = buf;
    }
    *out = (const Affine *)sh.lag[lg].p;
    return ZK_OK;
}

}  // namespace zk
