// hiding.cu -- hiding KZG commitments: com = [f(tau)]_1 + s H for a random
// scalar s and a group element H (the blinding of the paper's
// zero-knowledge argument for the accumulation scheme, Sec. 4.2).
//
// s H is a fixed-base product: with s split into 32 signed 8-bit digits
// d_w in [-128, 128] (s < 2^254, so no carry leaves the top window),
// s H = sum_w sign(d_w) |d_w| 2^(8w) H, and a table of the 32 x 128 points
// d 2^(8w) H (256 KB, built once per H) turns it into a sum of 32 table
// points.  One team (team.cuh) adds them in a 5-level tree, adds the MSM
// result and normalises: a few team additions on top of the MSM, instead of
// a 254-step double-and-add.
#include <cuda_runtime.h>

#include "ctx.cuh"
#include "curve.cuh"
#include "team.cuh"

namespace zk {

namespace {

constexpr int kHideWin = 32;
constexpr int kHideMul = 128;

// Table entry (w, d): (d + 1) 2^(8w) H; thread 0 also validates H.
__global__ void k_hide_table(const uint32_t *__restrict__ Hc, Affine *__restrict__ tab, uint32_t *__restrict__ bad) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (uint32_t)(kHideWin * kHideMul)) return;
    Affine h;
    h.x = fe_load<FqP>(Hc);
    h.y = fe_load<FqP>(Hc + 8);
    const bool canon = !fe_ge_modulus<FqP>(h.x) && !fe_ge_modulus<FqP>(h.y);
    h.x = fe_to_mont<FqP>(h.x);
    h.y = fe_to_mont<FqP>(h.y);
    if (idx == 0) *bad = (canon && affine_on_curve(h)) ? 0u : 1u;  // (0, 0) fails: 0 != 3
    const uint32_t w = idx / kHideMul, d = idx % kHideMul + 1;
    uint32_t k[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // d 2^(8w) < 2^256
    const uint32_t bit = 8 * w;
    k[bit >> 5] |= d << (bit & 31);
    if ((bit & 31) > 24 && (bit >> 5) + 1 < 8) k[(bit >> 5) + 1] |= d >> (32 - (bit & 31));
    tab[idx] = xyzz_to_affine(xyzz_mul(xyzz_from_affine(h), k));
}

constexpr int kHdAcc = 0, kHdIn = 4, kHdTmp = 8, kHdT = 12;

// out = canonical affine of (msm + s H); msm is the canonical affine MSM.
__global__ void __launch_bounds__(kTeamThreads)
    k_hide_add(const uint32_t *__restrict__ msm, const uint32_t *__restrict__ sc, const Affine *__restrict__ tab,
               uint32_t *__restrict__ out) {
    __shared__ uint32_t f[(kHdT + kTeamTemps) * 8 * 32];
    __shared__ int digit[kHideWin];
    const uint32_t l = team_lane(), w = team_warp();
    if (threadIdx.x == 0) {
        const Fr s = fe_load<FrP>(sc);
        uint32_t carry = 0;
        for (int i = 0; i < kHideWin; i++) {
            const uint32_t v = ((s.v[i >> 2] >> (8 * (i & 3))) & 0xffu) + carry;
            carry = v > 128u ? 1u : 0u;
            digit[i] = carry ? (int)v - 256 : (int)v;
        }
    }
    __syncthreads();
    // lane l: sign(d_l) |d_l| 2^(8l) H; warp w supplies coordinate w
    const int d = digit[l];
    Fq c = fe_zero<FqP>();
    if (d != 0) {
        const Affine &p = tab[l * kHideMul + (d < 0 ? -d : d) - 1];
        if (w == 0) c = p.x;
        else if (w == 1) c = d < 0 ? fe_neg<FqP>(p.y) : p.y;
        else c = fe_mont_one<FqP>();
    }
    tf_store(f, kHdAcc + w, c);
    __syncthreads();
    for (int dd = 16; dd >= 1; dd >>= 1) {
        team_shift(f, kHdAcc, kHdTmp, dd);
        team_add(f, kHdAcc, kHdTmp, kHdAcc, kHdT);
    }
    // + the MSM (lane 0 only; the other lanes add infinity)
    Fq m = fe_zero<FqP>();
    if (l == 0) {
        const Xyzz p = xyzz_load_canonical(msm);
        m = w == 0 ? p.X : (w == 1 ? p.Y : (w == 2 ? p.ZZ : p.ZZZ));
    }
    tf_store(f, kHdIn + w, m);
    __syncthreads();
    team_add(f, kHdAcc, kHdIn, kHdAcc, kHdT);
    if (threadIdx.x == 0) xyzz_store_canonical(out, team_point(f, kHdAcc));
}

}  // namespace

int hiding_base_impl(zk_ctx *ctx, const uint32_t *H, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    int err = ZK_OK;
    uint32_t *bad = (uint32_t *)scratch(ctx, "hide.bad", 4, &err);
    if (!bad) return err;
    std::lock_guard<std::mutex> g(sh.mu);
    if (!sh.hide_tab.p) ZK_TRY(dev_alloc(sh, sh.hide_tab, (size_t)kHideWin * kHideMul * sizeof(Affine)));
    k_hide_table<<<(kHideWin * kHideMul + 127) / 128, 128, 0, s>>>(H, (Affine *)sh.hide_tab.p, bad);
    ZK_LAUNCHED();
    uint32_t hbad = 1;
    ZK_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) {
        dev_free(sh, sh.hide_tab);
        return ZK_EINVAL;
    }
    return ZK_OK;
}

int commit_hiding_impl(zk_ctx *ctx, const uint32_t *coeffs, size_t n, const uint32_t *sc, uint32_t *out,
                       cudaStream_t s) {
    Shared &sh = *ctx->sh;
    if (!sh.hide_tab.p) return ZK_EINVAL;  // no hiding base set
    int err = ZK_OK;
    uint32_t *m = (uint32_t *)scratch(ctx, "hide.msm", 64, &err);
    if (!m) return err;
    MsmJob mj;
    mj.scalars = coeffs;
    mj.n = (uint32_t)n;
    mj.out = m;
    ZK_TRY(msm_batch_impl(ctx, &mj, 1, 0, s));
    k_hide_add<<<1, kTeamThreads, 0, s>>>(m, sc, (const Affine *)sh.hide_tab.p, out);
    ZK_LAUNCHED();
    return ZK_OK;
}

}  // namespace zk
