// srs.cu -- SRS [tau^i]_1 (paper Sec. 2.1) resident on the device, and the
// window tables 2^(c w) * SRS[i] that the MSM reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ctx.cuh"
#include "curve.cuh"

namespace zk {

namespace {

constexpr int kNormChunk = 32;  // points per thread in a batch normalisation

// ---------------------------------------------------------------------------
// Batch conversion XYZZ -> affine with one inversion per kNormChunk points
// (Montgomery's simultaneous-inversion trick).  `pref` is scratch of n Fq.
// ---------------------------------------------------------------------------
__global__ void k_normalize(const Xyzz *__restrict__ in, Affine *__restrict__ out,
                           Fq *__restrict__ pref, size_t n) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t lo = t * kNormChunk;
    if (lo >= n) return;
    size_t hi = lo + kNormChunk < n ? lo + kNormChunk : n;
    Fq acc = fe_mont_one<FqP>();
    for (size_t j = lo; j < hi; j++) {
        pref[j] = acc;
        Fq z = in[j].ZZZ;
        if (!fe_is_zero<FqP>(z)) acc = fe_mul<FqP>(acc, z);
    }
    Fq inv = fe_inv<FqP>(acc);
    for (size_t j = hi; j-- > lo;) {
        Xyzz p = in[j];
        Affine a;
        if (fe_is_zero<FqP>(p.ZZZ)) {
            a.x = fe_zero<FqP>();
            a.y = fe_zero<FqP>();
        } else {
            Fq izzz = fe_mul<FqP>(inv, pref[j]);
            inv = fe_mul<FqP>(inv, p.ZZZ);
            Fq iz = fe_mul<FqP>(p.ZZ, izzz);
            Fq izz = fe_sqr<FqP>(iz);
            a.x = fe_mul<FqP>(p.X, izz);
            a.y = fe_mul<FqP>(p.Y, izzz);
        }
        out[j] = a;
    }
}

int normalize(zk_ctx *ctx, const Xyzz *in, Affine *out, size_t n, cudaStream_t s) {
    int err = ZK_OK;
    Fq *pref = (Fq *)scratch(ctx, "srs.pref", n * sizeof(Fq), &err);
    if (!pref) return err;
    size_t threads = (n + kNormChunk - 1) / kNormChunk;
    unsigned blocks = (unsigned)((threads + 127) / 128);
    k_normalize<<<blocks, 128, 0, s>>>(in, out, pref, n);
    ZK_LAUNCHED();
    return ZK_OK;
}

// ---------------------------------------------------------------------------
// Loading: canonical affine -> validated Montgomery affine.
// ---------------------------------------------------------------------------
__global__ void k_srs_import(const uint32_t *__restrict__ in, Affine *__restrict__ out, size_t n,
                             unsigned long long *bad) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Fq x = fe_load<FqP>(in + 16 * i);
    Fq y = fe_load<FqP>(in + 16 * i + 8);
    bool ok = !fe_ge_modulus<FqP>(x) && !fe_ge_modulus<FqP>(y);
    Affine a;
    a.x = fe_to_mont<FqP>(x);
    a.y = fe_to_mont<FqP>(y);
    ok = ok && affine_on_curve(a);  // (0, 0) fails: 0 != 3
    if (!ok) atomicAdd(bad, 1ull);
    out[i] = a;
}

__global__ void k_srs_export(const Affine *__restrict__ in, uint32_t *__restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Affine a = in[i];
    fe_store<FqP>(out + 16 * i, fe_from_mont<FqP>(a.x));
    fe_store<FqP>(out + 16 * i + 8, fe_from_mont<FqP>(a.y));
}

// ---------------------------------------------------------------------------
// Generation from a known tau.
// ---------------------------------------------------------------------------

// gk[k] = 2^k G (XYZZ), k < 254, by one thread.
__global__ void k_gen_base_powers(Xyzz *gk) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    Affine g;
    g.x = fe_zero<FqP>();
    g.x.v[0] = 1;
    g.y = fe_zero<FqP>();
    g.y.v[0] = 2;
    g.x = fe_to_mont<FqP>(g.x);
    g.y = fe_to_mont<FqP>(g.y);
    Xyzz p = xyzz_from_affine(g);
    for (int k = 0; k < 254; k++) {
        gk[k] = p;
        p = xyzz_dbl(p);
    }
}

// powers[i] = tau^i (canonical), `chunk` consecutive powers per thread.
__global__ void k_tau_powers(const uint32_t *__restrict__ tau_can, uint32_t *__restrict__ powers,
                             size_t n, size_t chunk) {
    size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t lo = t * chunk;
    if (lo >= n) return;
    size_t hi = lo + chunk < n ? lo + chunk : n;
    Fr tau = fe_to_mont<FrP>(fe_load<FrP>(tau_can));
    uint32_t e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    e[0] = (uint32_t)lo;
    e[1] = (uint32_t)((uint64_t)lo >> 32);
    Fr acc = fe_pow<FrP>(tau, e);
    for (size_t i = lo; i < hi; i++) {
        fe_store<FrP>(powers + 8 * i, fe_from_mont<FrP>(acc));
        acc = fe_mul<FrP>(acc, tau);
    }
}

// out[i] = powers[i] * G by adding 2^k G for every set bit k.
__global__ void k_fixed_base(const uint32_t *__restrict__ powers, const Affine *__restrict__ gk,
                             Xyzz *__restrict__ out, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k[8];
#pragma unroll
    for (int j = 0; j < 8; j++) k[j] = powers[8 * i + j];
    Xyzz acc = xyzz_inf();
    for (int b = 0; b < 254; b++) {
        if ((k[b >> 5] >> (b & 31)) & 1) acc = xyzz_add_affine(acc, gk[b]);
    }
    out[i] = acc;
}

// ---------------------------------------------------------------------------
// Window tables: dst[i] = 2^c * src[i]; entries (AffineS) of a window.
// ---------------------------------------------------------------------------
__global__ void k_table_entries(const Affine *__restrict__ src, AffineS *__restrict__ dst, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    affines_store(dst + i, affines_from_affine(affine_ldg(src + i)));
}

__global__ void k_shift_window(const Affine *__restrict__ src, Xyzz *__restrict__ dst, size_t n,
                               int c) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Xyzz p = xyzz_dbl_affine(src[i]);
    for (int k = 1; k < c; k++) p = xyzz_dbl(p);
    dst[i] = p;
}

int build_table(zk_ctx *ctx, WindowTable &t, int c, size_t n, int basis, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    const Affine *base = (const Affine *)sh.srs.p;
    if (basis) base = (const Affine *)sh.lag[basis].p;
    const int W = windows_for(c);
    ZK_TRY(dev_alloc(sh, t.buf, (size_t)W * n * sizeof(AffineS)));
    t.c = c;
    t.W = W;
    t.n = n;
    t.basis = basis;
    AffineS *tab = (AffineS *)t.buf.p;
    int err = ZK_OK;
    Xyzz *tmp = (Xyzz *)scratch(ctx, "srs.xyzz", n * sizeof(Xyzz), &err);
    Affine *win = (Affine *)scratch(ctx, "srs.window", n * sizeof(Affine), &err);  // window w, Montgomery
    if (!tmp || !win) return err;
    unsigned blocks = (unsigned)((n + 127) / 128);
    k_table_entries<<<blocks, 128, 0, s>>>(base, tab, n);
    ZK_LAUNCHED();
    for (int w = 1; w < W; w++) {
        k_shift_window<<<blocks, 128, 0, s>>>(w == 1 ? base : win, tmp, n, c);
        ZK_LAUNCHED();
        ZK_TRY(normalize(ctx, tmp, win, n, s));
        k_table_entries<<<blocks, 128, 0, s>>>(win, tab + (size_t)w * n, n);
        ZK_LAUNCHED();
    }
    // Tables are shared read-only by lanes on other streams: finish now.
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

void drop_srs(Shared &sh) {
    for (auto &t : sh.tables) dev_free(sh, t.buf);
    sh.tables.clear();
    for (auto &l : sh.lag) dev_free(sh, l);
    dev_free(sh, sh.srs);
    sh.srs_n = 0;
}

}  // namespace

int normalize_points(zk_ctx *ctx, const Xyzz *in, Affine *out, size_t n, cudaStream_t s) {
    return normalize(ctx, in, out, n, s);
}

int table_get(zk_ctx *ctx, int c, size_t n, int basis, const WindowTable **out, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    if (sh.srs_n == 0 || n > sh.srs_n) return ZK_ESRS;
    if (basis && (n > ((size_t)1 << basis) || !sh.lag[basis].p)) return ZK_EINVAL;
    std::lock_guard<std::mutex> g(sh.mu);
    for (auto &t : sh.tables) {
        if (t.c == c && t.basis == basis && t.n >= n) {
            *out = &t;
            return ZK_OK;
        }
    }
    // A table covers the next power of two of the request (at most the SRS);
    // a smaller table of the same width stays alive for work still queued.
    size_t tn = 1;
    while (tn < n) tn <<= 1;
    tn = std::min(tn, basis ? ((size_t)1 << basis) : sh.srs_n);
    if ((size_t)windows_for(c) * tn >= ((size_t)1 << 31)) return ZK_EINVAL;
    sh.tables.emplace_back();
    int r = build_table(ctx, sh.tables.back(), c, tn, basis, s);
    if (r != ZK_OK) {
        dev_free(sh, sh.tables.back().buf);
        sh.tables.pop_back();
        return r;
    }
    *out = &sh.tables.back();
    return ZK_OK;
}

int srs_load_impl(zk_ctx *ctx, const zk_g1 *pts, size_t n, cudaStream_t s) {
    if (!pts || n == 0 || n > ((size_t)1 << kMaxSrsLog)) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    {
        std::lock_guard<std::mutex> g(sh.mu);
        drop_srs(sh);
        ZK_TRY(dev_alloc(sh, sh.srs, n * sizeof(Affine)));
    }
    int err = ZK_OK;
    const uint32_t *src = (const uint32_t *)pts;
    if (!is_device_ptr(pts)) {
        void *stage = scratch(ctx, "srs.stage", n * sizeof(zk_g1), &err);
        if (!stage) return err;
        ZK_CUDA_TRY(cudaMemcpyAsync(stage, pts, n * sizeof(zk_g1), cudaMemcpyHostToDevice, s));
        src = (const uint32_t *)stage;
    }
    unsigned long long *bad =
        (unsigned long long *)scratch(ctx, "srs.bad", sizeof(unsigned long long), &err);
    if (!bad) return err;
    ZK_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof *bad, s));
    k_srs_import<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, (Affine *)sh.srs.p, n, bad);
    ZK_LAUNCHED();
    unsigned long long nbad = 0;
    ZK_CUDA_TRY(cudaMemcpyAsync(&nbad, bad, sizeof nbad, cudaMemcpyDeviceToHost, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    if (nbad) {
        std::lock_guard<std::mutex> g(sh.mu);
        drop_srs(sh);
        return ZK_EINVAL;
    }
    sh.srs_n = n;
    const WindowTable *t;
    ZK_TRY(table_get(ctx, 16, n, 0, &t, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int srs_generate_impl(zk_ctx *ctx, const zk_fr *tau, size_t n, cudaStream_t s) {
    if (!tau || n == 0 || n > ((size_t)1 << kMaxSrsLog)) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    {
        std::lock_guard<std::mutex> g(sh.mu);
        drop_srs(sh);
        ZK_TRY(dev_alloc(sh, sh.srs, n * sizeof(Affine)));
    }
    int err = ZK_OK;
    uint32_t *tau_d = (uint32_t *)scratch(ctx, "srs.tau", 32, &err);
    Xyzz *gk_x = (Xyzz *)scratch(ctx, "srs.gkx", 254 * sizeof(Xyzz), &err);
    Affine *gk = (Affine *)scratch(ctx, "srs.gk", 254 * sizeof(Affine), &err);
    uint32_t *powers = (uint32_t *)scratch(ctx, "srs.powers", n * 32, &err);
    Xyzz *tmp = (Xyzz *)scratch(ctx, "srs.xyzz", n * sizeof(Xyzz), &err);
    if (!tau_d || !gk_x || !gk || !powers || !tmp) return err;
    zk_fr tau_h;
    memcpy(&tau_h, tau, sizeof tau_h);  // tau is a host pointer
    ZK_CUDA_TRY(cudaMemcpyAsync(tau_d, &tau_h, 32, cudaMemcpyHostToDevice, s));
    k_gen_base_powers<<<1, 1, 0, s>>>(gk_x);
    ZK_LAUNCHED();
    ZK_TRY(normalize(ctx, gk_x, gk, 254, s));
    const size_t chunk = 64;
    size_t threads = (n + chunk - 1) / chunk;
    k_tau_powers<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(tau_d, powers, n, chunk);
    ZK_LAUNCHED();
    k_fixed_base<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(powers, gk, tmp, n);
    ZK_LAUNCHED();
    ZK_TRY(normalize(ctx, tmp, (Affine *)sh.srs.p, n, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    sh.srs_n = n;
    const WindowTable *t;
    ZK_TRY(table_get(ctx, 16, n, 0, &t, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int srs_export_impl(zk_ctx *ctx, zk_g1 *out, size_t first, size_t count, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    if (!out) return ZK_EINVAL;
    if (sh.srs_n == 0 || first + count > sh.srs_n) return ZK_ESRS;
    if (count == 0) return ZK_OK;
    int err = ZK_OK;
    bool dev = is_device_ptr(out);
    uint32_t *dst = (uint32_t *)out;
    if (!dev) {
        dst = (uint32_t *)scratch(ctx, "srs.export", count * sizeof(zk_g1), &err);
        if (!dst) return err;
    }
    k_srs_export<<<(unsigned)((count + 255) / 256), 256, 0, s>>>((const Affine *)sh.srs.p + first,
                                                                  dst, count);
    ZK_LAUNCHED();
    if (!dev) {
        ZK_CUDA_TRY(cudaMemcpyAsync(out, dst, count * sizeof(zk_g1), cudaMemcpyDeviceToHost, s));
        ZK_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return ZK_OK;
}

}  // namespace zk
