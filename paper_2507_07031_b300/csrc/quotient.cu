// quotient.cu -- the quotient polynomial of the Mul basic block (paper
// Sec. 4.4.1), which is also MatMul's Q_l: for evaluation vectors a, b over
// H = <omega_n> with interpolants A, B, and L the interpolant of a o b,
//     t(X) = (A(X) B(X) - L(X)) / (X^n - 1),
// and its commitment [t(tau)]_1.
//
// Write A B = P_lo + X^n P_hi with deg P_lo, P_hi < n.  On H, X^n = 1, so
// (A B)|_H = (P_lo + P_hi)|_H = a o b: L = P_lo + P_hi and t = P_hi, an exact
// division for every a, b.  On the coset zeta H with zeta = omega_{2n}
// (zeta^n = -1), (A B)|_{zeta H} = (P_lo - P_hi)|_{zeta H}.  Hence with
//     U = INTT(a o b) = P_lo + P_hi,
//     V = the interpolant over zeta H of A' o B' = P_lo - P_hi,
//         (A' = A on zeta H = NTT(A_i zeta^i); V_i = INTT(A' o B')_i zeta^-i)
// the quotient is t = (U - V) / 2: six transforms of length n and three
// pointwise passes, with no transform of length 2n.
#include <cuda_runtime.h>

#include <algorithm>

#include "ctx.cuh"
#include "field.cuh"

namespace zk {

namespace {

// A_i zeta^i, B_i zeta^i (canonical values times Montgomery twiddles).
__global__ void k_mq_shift(uint32_t *__restrict__ A, uint32_t *__restrict__ B, const uint32_t *__restrict__ tw2,
                           size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Fr z = fe_load<FrP>(tw2 + 8 * i);
    fe_store<FrP>(A + 8 * i, fe_mul<FrP>(fe_load<FrP>(A + 8 * i), z));
    fe_store<FrP>(B + 8 * i, fe_mul<FrP>(fe_load<FrP>(B + 8 * i), z));
}

// A <- A' o B' and B <- a o b.
__global__ void k_mq_products(uint32_t *__restrict__ A, uint32_t *__restrict__ B, const uint32_t *__restrict__ a,
                              const uint32_t *__restrict__ b, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Fr w = fe_mul<FrP>(fe_load<FrP>(A + 8 * i), fe_to_mont<FrP>(fe_load<FrP>(B + 8 * i)));
    const Fr p = fe_mul<FrP>(fe_load<FrP>(a + 8 * i), fe_to_mont<FrP>(fe_load<FrP>(b + 8 * i)));
    fe_store<FrP>(A + 8 * i, w);
    fe_store<FrP>(B + 8 * i, p);
}

// t_i = (U_i - V0_i zeta^-i) / 2 for i < n - 1 (t_{n-1} = 0 by the degree
// bound).  zeta^-i = tw2[2n - i].
__global__ void k_mq_combine(const uint32_t *__restrict__ V0, const uint32_t *__restrict__ U,
                             const uint32_t *__restrict__ tw2, size_t n, uint32_t *__restrict__ t) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i + 1 >= n) return;
    Fr v = fe_load<FrP>(V0 + 8 * i);
    if (i) v = fe_mul<FrP>(v, fe_load<FrP>(tw2 + 8 * (2 * n - i)));
    Fr half = fe_zero<FrP>();  // (r + 1) / 2
#pragma unroll
    for (int w = 0; w < 8; w++) half.v[w] = (FrP::p(w) >> 1) | (w < 7 ? (FrP::p(w + 1) << 31) : 0u);
    half.v[0] += 1;  // p odd: (p >> 1) + 1 = (p + 1) / 2, no carry out of word 0
    fe_store<FrP>(t + 8 * i, fe_mul<FrP>(fe_sub<FrP>(fe_load<FrP>(U + 8 * i), v), fe_to_mont<FrP>(half)));
}

}  // namespace

int mul_quotient_impl(zk_ctx *ctx, const uint32_t *a, const uint32_t *b, size_t n, uint32_t *t, uint32_t *com,
                      cudaStream_t s) {
    if (!a || !b || !com || n == 0 || (n & (n - 1)) || n > ((size_t)1 << (kMaxLogN - 1))) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    if (n - 1 > sh.srs_n) return ZK_ESRS;
    if (n == 1) {  // A B - L = 0: t = 0, commitment infinity
        ZK_CUDA_TRY(cudaMemsetAsync(com, 0, 64, s));
        return ZK_OK;
    }
    int lg = 0;
    while (((size_t)1 << lg) < n) lg++;
    const uint32_t *tw2;
    ZK_TRY(twiddles(ctx, lg + 1, &tw2, s));
    int err = ZK_OK;
    uint32_t *A = (uint32_t *)scratch(ctx, "mq.A", n * 32, &err);
    uint32_t *B = (uint32_t *)scratch(ctx, "mq.B", n * 32, &err);
    uint32_t *tt = t ? t : (uint32_t *)scratch(ctx, "mq.t", (n - 1) * 32, &err);
    if (!A || !B || !tt) return err;
    ZK_CUDA_TRY(cudaMemcpyAsync(A, a, n * 32, cudaMemcpyDeviceToDevice, s));
    ZK_CUDA_TRY(cudaMemcpyAsync(B, b, n * 32, cudaMemcpyDeviceToDevice, s));
    uint32_t *const v[2] = {A, B};
    const size_t lens[2] = {n, n};
    const unsigned blocks = (unsigned)((n + 127) / 128);
    ZK_TRY(ntt_batch_impl(ctx, v, lens, 2, true, s));  // coefficients of A, B
    k_mq_shift<<<blocks, 128, 0, s>>>(A, B, tw2, n);
    ZK_LAUNCHED();
    ZK_TRY(ntt_batch_impl(ctx, v, lens, 2, false, s));  // A, B on zeta H
    k_mq_products<<<blocks, 128, 0, s>>>(A, B, a, b, n);
    ZK_LAUNCHED();
    ZK_TRY(ntt_batch_impl(ctx, v, lens, 2, true, s));  // V0 = INTT(A' o B'), U = INTT(a o b)
    k_mq_combine<<<blocks, 128, 0, s>>>(A, B, tw2, n, tt);
    ZK_LAUNCHED();
    MsmJob mj;
    mj.scalars = tt;
    mj.n = (uint32_t)(n - 1);
    mj.out = com;
    return msm_batch_impl(ctx, &mj, 1, 0, s);
}

}  // namespace zk
