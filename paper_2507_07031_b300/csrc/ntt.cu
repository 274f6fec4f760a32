// ntt.cu -- natural-order NTT / inverse NTT over F_r (the interpolation of a
// witness vector of evaluations over H = <omega_n> into coefficients, paper
// Sec. 3 and Sec. 4.4), n = 2^L <= 2^28.
//
// Stockham autosort formulation in P = ceil(L / m) passes of radix R_p = 2^s_p
// (s_p <= m; m is tuned per length, at most 11): pass p computes, for each of the n / R sub-transforms j,
//   v_r = x[j + r n/R] * omega_{Ns R}^{r (j mod Ns)},  r < R,
//   V   = R-point DFT of v,
//   y[(j / Ns) Ns R + (j mod Ns) + r Ns] = V_r,
// with Ns = prod_{p' < p} R_p'.  A CTA stages J = min(4, n/R, 4096/R) consecutive
// sub-transforms (J R elements, up to 128 KiB) in shared memory in a
// limb-planar, sub-transform-interleaved layout (word l of element r of
// sub-transform jj at l J R + r J + jj, so consecutive threads touch
// consecutive banks), runs the R-point DFT as log2 R
// radix-2 decimation-in-frequency stages, and writes the bit-reversed
// positions back in natural order.  Global loads and stores move runs of J
// consecutive 32-byte elements (J R contiguous ones in the first pass).
//
// Data are canonical in memory.  The inter-pass twiddles are stored in
// Montgomery form, so mont(x, w R) = x w is already canonical.  Inside a
// pass the butterflies keep values in [0, 2r) (4r < 2^256): their stage
// twiddles come from a table of (w, floor(w 2^256 / r)) pairs and use the
// precomputed-quotient product (fe_mul_shoup_2p, 22 % fewer multiply-pipe
// cycles than a Montgomery product) on the lazy difference x - y + 2r; the
// store reduces to canonical.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <vector>

#include "check.cuh"
#include "ctx.cuh"
#include "field.cuh"

namespace zk {

ZK_CHECK_UNIT()

namespace {

constexpr int kMaxRadixLog = 11;
constexpr int kMaxJ = 4;
constexpr size_t kMaxSmem = (size_t)128 << 10;  // J R 32 bytes per CTA
constexpr uint32_t kMaxRegJR = 1u << kMaxRadixLog;  // largest J R of the register-tiled pass (R alone can reach it)
constexpr uint32_t kRegJR = 1024;               // its J R where the length allows
constexpr int kRegMinLog = 9;                   // smallest radix (log2) on the register-tiled pass

// w = 5^((r - 1) / 2^lg), the primitive 2^lg-th root of unity (5 generates
// the 2-Sylow subgroup of F_r^*: it is a quadratic non-residue).
__global__ void k_root(uint32_t lg, Fr *out) {
    if (threadIdx.x || blockIdx.x) return;
    uint32_t e[8];
#pragma unroll
    for (int i = 0; i < 8; i++) e[i] = FrP::p(i);
    e[0] -= 1;  // r - 1 (r is odd)
    for (uint32_t k = 0; k < lg; k++) {
#pragma unroll
        for (int i = 0; i < 7; i++) e[i] = (e[i] >> 1) | (e[i + 1] << 31);
        e[7] >>= 1;
    }
    Fr five = fe_zero<FrP>();
    five.v[0] = 5;
    *out = fe_pow<FrP>(fe_to_mont<FrP>(five), e);
}

// tw[k] = w^k for k < n (chunks of 64 per thread); tw[n] = n^{-1} (Montgomery
// form), tw[n + 1] = n^{-1} and tw[n + 2] = floor(n^{-1} 2^256 / r) (canonical:
// the inverse transform's final scaling by a precomputed-quotient product).
__global__ void k_twiddles(const Fr *__restrict__ root, uint32_t lg, Fr *__restrict__ tw) {
    const uint64_t n = 1ull << lg;
    uint64_t lo = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) * 64;
    if (lo == 0 && threadIdx.x == 0 && blockIdx.x == 0) {
        Fr nn = fe_zero<FrP>();
        nn.v[0] = (uint32_t)n;
        nn.v[1] = (uint32_t)(n >> 32);
        const Fr ninv = fe_inv_canonical<FrP>(nn);
        tw[n] = fe_to_mont<FrP>(ninv);
        tw[n + 1] = ninv;
        tw[n + 2] = fe_shoup_quotient<FrP>(ninv);
    }
    if (lo >= n) return;
    uint64_t hi = lo + 64 < n ? lo + 64 : n;
    uint32_t e[8] = {(uint32_t)lo, (uint32_t)(lo >> 32), 0, 0, 0, 0, 0, 0};
    Fr w = *root;
    Fr acc = fe_pow<FrP>(w, e);
    for (uint64_t k = lo; k < hi; k++) {
        tw[k] = acc;
        acc = fe_mul<FrP>(acc, w);
    }
}

// Stage-twiddle table: tws[k] = (w^k, floor(w^k 2^256 / r)), both canonical,
// 16 words per entry, from the Montgomery table tw (one thread per entry).
__global__ void k_stage_twiddles(const Fr *__restrict__ tw, uint32_t n, uint32_t *__restrict__ tws) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const Fr w = fe_from_mont<FrP>(tw[k]);
    fe_store<FrP>(tws + 16 * (size_t)k, w);
    fe_store<FrP>(tws + 16 * (size_t)k + 8, fe_shoup_quotient<FrP>(w));
}

// Butterfly difference (x - y) w_pos in [0, 2r) for x, y in [0, 2r) and a
// stage twiddle entry (w, wq).
__device__ __forceinline__ Fr stage_diff(const Fr &x, const Fr &y, const uint32_t *e) {
    return fe_mul_shoup_2p<FrP>(fe_sub_2p_lazy<FrP>(x, y), fe_ldg<FrP>(e), fe_ldg<FrP>(e + 8));
}

struct PassArgs {
    const uint32_t *const *in_tab;  // per vector (blockIdx.y)
    uint32_t *const *out_tab;
    uint32_t logn, logR, logNs, J, logJ;  // J = 2^logJ sub-transforms per CTA
    const Fr *tw_n;  // size-n table (+ n^{-1} and its quotient at n + 1, n + 2)
    const uint32_t *tw_S;  // size-R stage table (w, wq), 16 words per entry
    int inverse;
    int scale;  // multiply outputs by n^{-1}
};

// One instance per staged size J R = 2^LJR (2 .. 4096): limb l of staged
// element i is at sm[l JR + i], so with JR a compile-time constant every
// limb's offset is an immediate of the shared-memory access.
template <int LJR>
__global__ void __launch_bounds__(512) k_ntt_pass(PassArgs a) {
    extern __shared__ uint32_t sm[];
    const uint32_t R = 1u << a.logR;
    const uint32_t J = a.J;
    constexpr uint32_t JR = 1u << LJR;
    const uint64_t n = 1ull << a.logn;
    const uint32_t Ns = 1u << a.logNs;
    const uint64_t stride = n >> a.logR;  // n / R
    const uint32_t *in = a.in_tab[blockIdx.y];
    uint32_t *out = a.out_tab[blockIdx.y];
    const uint64_t j0 = (uint64_t)blockIdx.x * J;
    const uint32_t tshift = a.logn - a.logNs - a.logR;

    // Load, apply the inter-pass twiddle omega_{Ns R}^{r (j mod Ns)}.
    for (uint32_t e = threadIdx.x; e < JR; e += blockDim.x) {
        uint32_t r = e >> a.logJ, jj = e & (J - 1);
        uint64_t j = j0 + jj;
        if (ZK_FAILED(j + (uint64_t)r * stride < n, kCheckNttIdx)) continue;
        Fr x = fe_load<FrP>(in + 8 * (j + (uint64_t)r * stride));
        uint64_t m = j & (Ns - 1);
        uint64_t ex = ((uint64_t)r * m) << tshift;
        if (ex) {
            uint64_t idx = a.inverse ? n - ex : ex;
            x = fe_mul<FrP>(x, fe_ldg<FrP>(a.tw_n + idx));
        }
#pragma unroll
        for (int l = 0; l < 8; l++) sm[l * JR + r * J + jj] = x.v[l];
    }
    __syncthreads();

    // R-point DIF radix-2: (a, b) -> (a + b, (a - b) omega_{2h}^pos).
    const uint32_t half = R >> 1;
    (void)half;
    for (uint32_t lh = a.logR; lh >= 1; lh--) {
        const uint32_t h = 1u << (lh - 1);
        for (uint32_t bf = threadIdx.x; bf < J * half; bf += blockDim.x) {
            uint32_t jj = bf & (J - 1), k = bf >> a.logJ;
            uint32_t pos = k & (h - 1);
            uint32_t i0 = ((((k >> (lh - 1)) << lh) + pos) * J) + jj;
            uint32_t i1 = i0 + h * J;
            Fr x, y;
#pragma unroll
            for (int l = 0; l < 8; l++) {
                x.v[l] = sm[l * JR + i0];
                y.v[l] = sm[l * JR + i1];
            }
            Fr s = fe_add_2p<FrP>(x, y);
            Fr d;
            if (pos) {
                uint32_t idx = pos << (a.logR - lh);
                if (a.inverse) idx = R - idx;
                d = stage_diff(x, y, a.tw_S + 16 * idx);
            } else {
                d = fe_sub_2p<FrP>(x, y);
            }
#pragma unroll
            for (int l = 0; l < 8; l++) {
                sm[l * JR + i0] = s.v[l];
                sm[l * JR + i1] = d.v[l];
            }
        }
        __syncthreads();
    }

    // Store V_r (at bit-reversed position r) to its natural-order place.
    Fr sc, scq;
    if (a.scale) {
        sc = fe_ldg<FrP>(a.tw_n + n + 1);
        scq = fe_ldg<FrP>(a.tw_n + n + 2);
    }
    for (uint32_t e = threadIdx.x; e < JR; e += blockDim.x) {
        uint32_t r, jj;
        if (Ns >= J) {
            r = e >> a.logJ;
            jj = e & (J - 1);
        } else {
            uint32_t q = e >> (a.logNs + a.logR);
            uint32_t rem = e & ((Ns << a.logR) - 1);
            r = rem >> a.logNs;
            jj = q * Ns + (rem & (Ns - 1));
        }
        uint64_t j = j0 + jj;
        uint32_t src = a.logR ? (__brev(r) >> (32 - a.logR)) : 0;
        Fr x;
#pragma unroll
        for (int l = 0; l < 8; l++) x.v[l] = sm[l * JR + src * J + jj];
        x = a.scale ? fe_mul_shoup<FrP>(x, sc, scq) : fe_canon_2p<FrP>(x);  // [0, 2r) -> canonical
        uint64_t dst = ((j >> a.logNs) << (a.logNs + a.logR)) + (j & (Ns - 1)) + ((uint64_t)r << a.logNs);
        if (ZK_FAILED(dst < n, kCheckNttIdx)) continue;
        fe_store<FrP>(out + 8 * dst, x);
    }
}

// Register-tiled pass for sub-transforms of R = 2^LR >= 8 points, J = 2^logJ
// of them per CTA (the host picks J R = 1024 where it can), T = J R / 4
// threads.  Each thread holds E = 4 elements of one sub-transform in
// registers and runs the radix-2 DIF stages two at a time: for stages
// s0 .. s0 + ne - 1 (half-sizes h = R / 2^(s + 1)) the
// pairs (r, r + h) of a thread are its own elements when it holds
//     r = blk 2^ne S + kk S + b,   kk < 2^ne,  S = R / 2^(s0 + ne)
// (b < S, blk < 2^s0), so one shared-memory exchange per group of two
// stages (instead of one per stage) re-deals the elements between groups.
// Four elements per thread measured faster than eight (more resident warps)
// at 2^20 and 2^22.
// Shared memory is limb-planar with one padding word per 32 (word of
// element i of sub-transform jj at l P + pad(i J + jj)), which keeps the
// strided exchanges free of bank conflicts.  Inter-pass twiddles, the
// output permutation and the final n^-1 scaling are as in k_ntt_pass.
constexpr int kRegLE = 2;  // log2 elements per thread

__device__ __forceinline__ uint32_t pad32(uint32_t i) { return i + (i >> 5); }

template <int LR>
__global__ void __launch_bounds__(512, 2) k_ntt_reg(PassArgs a) {
    extern __shared__ uint32_t sm[];
    constexpr uint32_t R = 1u << LR, E = 1u << kRegLE;
    const uint32_t LJ = a.logJ, J = 1u << LJ, JR = J * R;
    const uint32_t T = JR / E;            // threads doing work
    const uint32_t P = JR + JR / 32;      // padded words per limb plane
    constexpr int G = (LR + kRegLE - 1) / kRegLE;  // stage groups
    const uint64_t n = 1ull << a.logn;
    const uint32_t Ns = 1u << a.logNs;
    const uint64_t stride = n >> LR;  // n / R
    const uint32_t *in = a.in_tab[blockIdx.y];
    uint32_t *out = a.out_tab[blockIdx.y];
    const uint64_t j0 = (uint64_t)blockIdx.x * J;
    const uint32_t tshift = a.logn - a.logNs - LR;
    const uint32_t t = threadIdx.x;
    const bool worker = t < T;
    const uint32_t jj = t & (J - 1), rest = t >> LJ;
    Fr x[E];

    // Element k of this thread in stage group g (ne stages starting at s0).
    auto elem_r = [&](int g, uint32_t k) -> uint32_t {
        const int s0 = g * kRegLE;
        const int ne = LR - s0 < kRegLE ? LR - s0 : kRegLE;
        const int lS = LR - s0 - ne;
        const uint32_t gi = (rest << (kRegLE - ne)) + (k >> ne);
        const uint32_t blk = gi >> lS, b = gi & ((1u << lS) - 1);
        return (blk << (ne + lS)) + ((k & ((1u << ne) - 1)) << lS) + b;
    };

    // Load group 0's elements with the inter-pass twiddle omega_{Ns R}^{r (j mod Ns)}.
    if (worker) {
        const uint64_t j = j0 + jj;
        const uint64_t m = j & (Ns - 1);
#pragma unroll
        for (uint32_t k = 0; k < E; k++) {
            const uint32_t r = elem_r(0, k);
            if (ZK_FAILED(j + (uint64_t)r * stride < n, kCheckNttIdx)) {
                x[k] = fe_zero<FrP>();
                continue;
            }
            Fr v = fe_load<FrP>(in + 8 * (j + (uint64_t)r * stride));
            const uint64_t ex = ((uint64_t)r * m) << tshift;
            if (ex) v = fe_mul<FrP>(v, fe_ldg<FrP>(a.tw_n + (a.inverse ? n - ex : ex)));
            x[k] = v;
        }
    }
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int s0 = g * kRegLE;
        const int ne = LR - s0 < kRegLE ? LR - s0 : kRegLE;
        if (g > 0) {  // re-deal: write by group g-1's layout, read by group g's
            if (worker) {
#pragma unroll
                for (uint32_t k = 0; k < E; k++) {
                    const uint32_t w = pad32(elem_r(g - 1, k) * J + jj);
#pragma unroll
                    for (int l = 0; l < 8; l++) sm[l * P + w] = x[k].v[l];
                }
            }
            __syncthreads();
            if (worker) {
#pragma unroll
                for (uint32_t k = 0; k < E; k++) {
                    const uint32_t w = pad32(elem_r(g, k) * J + jj);
#pragma unroll
                    for (int l = 0; l < 8; l++) x[k].v[l] = sm[l * P + w];
                }
            }
            __syncthreads();
        }
        if (!worker) continue;
#pragma unroll
        for (int ls = 0; ls < ne; ls++) {
            const int s = s0 + ls;
            const uint32_t hk = 1u << (ne - 1 - ls);  // pair distance in k
#pragma unroll
            for (uint32_t k = 0; k < E; k++) {
                if (k & hk) continue;
                const uint32_t k2 = k + hk;
                const Fr u = x[k], v = x[k2];
                x[k] = fe_add_2p<FrP>(u, v);
                // pos = r mod h with h = S 2^(ne - 1 - ls)
                const uint32_t pos = elem_r(g, k) & ((R >> (s + 1)) - 1);
                if (pos) {
                    uint32_t idx = pos << s;
                    if (a.inverse) idx = R - idx;
                    x[k2] = stage_diff(u, v, a.tw_S + 16 * idx);
                } else {
                    x[k2] = fe_sub_2p<FrP>(u, v);
                }
            }
        }
    }
    // Natural-order output: element at position i holds V_{bitrev(i)}.
    if (worker) {
#pragma unroll
        for (uint32_t k = 0; k < E; k++) {
            const uint32_t w = pad32(elem_r(G - 1, k) * J + jj);
#pragma unroll
            for (int l = 0; l < 8; l++) sm[l * P + w] = x[k].v[l];
        }
    }
    __syncthreads();
    Fr sc, scq;
    if (a.scale) {
        sc = fe_ldg<FrP>(a.tw_n + n + 1);
        scq = fe_ldg<FrP>(a.tw_n + n + 2);
    }
    for (uint32_t e = threadIdx.x; e < JR; e += blockDim.x) {
        uint32_t r, jx;
        if (Ns >= J) {
            r = e >> LJ;
            jx = e & (J - 1);
        } else {
            uint32_t q = e >> (a.logNs + LR);
            uint32_t rem = e & ((Ns << LR) - 1);
            r = rem >> a.logNs;
            jx = q * Ns + (rem & (Ns - 1));
        }
        const uint64_t j = j0 + jx;
        const uint32_t src = __brev(r) >> (32 - LR);
        const uint32_t w = pad32(src * J + jx);
        Fr v;
#pragma unroll
        for (int l = 0; l < 8; l++) v.v[l] = sm[l * P + w];
        v = a.scale ? fe_mul_shoup<FrP>(v, sc, scq) : fe_canon_2p<FrP>(v);  // [0, 2r) -> canonical
        const uint64_t dst = ((j >> a.logNs) << (a.logNs + LR)) + (j & (Ns - 1)) + ((uint64_t)r << a.logNs);
        if (ZK_FAILED(dst < n, kCheckNttIdx)) continue;
        fe_store<FrP>(out + 8 * dst, v);
    }
}

template <int LR>
int launch_reg_t(dim3 grid, cudaStream_t s, const PassArgs &a) {
    const uint32_t JR = 1u << (LR + a.logJ);
    const uint32_t threads = std::max<uint32_t>(32, JR >> kRegLE);
    const size_t smem = (size_t)8 * (JR + JR / 32) * 4;
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    ZK_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = dev < 64 ? 1ull << dev : 0;
    if (!bit || !(attr_set.load() & bit)) {
        ZK_CUDA_TRY(cudaFuncSetAttribute(k_ntt_reg<LR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)8 * (kMaxRegJR + kMaxRegJR / 32) * 4)));
        attr_set.fetch_or(bit);
    }
    k_ntt_reg<LR><<<grid, threads, smem, s>>>(a);
    ZK_LAUNCHED();
    return ZK_OK;
}

// Register-tiled pass for kRegMinLog <= logR <= 11.
int launch_reg(uint32_t logR, dim3 grid, cudaStream_t s, const PassArgs &a) {
    static_assert(kRegMinLog == 9, "instances below");
    switch (logR) {
        case 9: return launch_reg_t<9>(grid, s, a);
        case 10: return launch_reg_t<10>(grid, s, a);
        case 11: return launch_reg_t<11>(grid, s, a);
        default: return ZK_EINVAL;
    }
}

template <int LJR>
int launch_pass_t(dim3 grid, uint32_t threads, size_t smem, cudaStream_t s, const PassArgs &a) {
    // The shared-memory limit is a per-device attribute of the kernel: set it
    // once on each device this instance runs on (the context's device is
    // current here).
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    ZK_CUDA_TRY(cudaGetDevice(&dev));
    const uint64_t bit = dev < 64 ? 1ull << dev : 0;
    if (!bit || !(attr_set.load() & bit)) {
        ZK_CUDA_TRY(cudaFuncSetAttribute(k_ntt_pass<LJR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSmem));
        attr_set.fetch_or(bit);
    }
    k_ntt_pass<LJR><<<grid, threads, smem, s>>>(a);
    ZK_LAUNCHED();
    return ZK_OK;
}

// J R = 2^ljr with 1 <= ljr <= 12 (J <= 4, J R 32 bytes <= 128 KiB).
int launch_pass(uint32_t ljr, dim3 grid, uint32_t threads, size_t smem, cudaStream_t s, const PassArgs &a) {
    switch (ljr) {
        case 1: return launch_pass_t<1>(grid, threads, smem, s, a);
        case 2: return launch_pass_t<2>(grid, threads, smem, s, a);
        case 3: return launch_pass_t<3>(grid, threads, smem, s, a);
        case 4: return launch_pass_t<4>(grid, threads, smem, s, a);
        case 5: return launch_pass_t<5>(grid, threads, smem, s, a);
        case 6: return launch_pass_t<6>(grid, threads, smem, s, a);
        case 7: return launch_pass_t<7>(grid, threads, smem, s, a);
        case 8: return launch_pass_t<8>(grid, threads, smem, s, a);
        case 9: return launch_pass_t<9>(grid, threads, smem, s, a);
        case 10: return launch_pass_t<10>(grid, threads, smem, s, a);
        case 11: return launch_pass_t<11>(grid, threads, smem, s, a);
        case 12: return launch_pass_t<12>(grid, threads, smem, s, a);
        default: return ZK_EINVAL;
    }
}

// Radix split of L into the fewest passes of at most maxlog, as even as possible.
std::vector<int> plan_passes(int L, int maxlog) {
    std::vector<int> s;
    if (L == 0) return s;
    int P = (L + maxlog - 1) / maxlog;
    for (int p = 0; p < P; p++) s.push_back(L / P + (p < L % P ? 1 : 0));
    return s;
}

int ilog2(size_t n) {
    int l = 0;
    while (((size_t)1 << l) < n) l++;
    return l;
}

bool is_pow2(size_t n) { return n && !(n & (n - 1)); }

}  // namespace

// Reads and clears this translation unit's check flags (always 0 in the
// normal build).
int ntt_check_read(uint32_t *flags) {
    *flags = 0;
#ifdef ZK_CHECK
    ZK_CUDA_TRY(cudaMemcpyFromSymbol(flags, g_zk_check_flags, sizeof(uint32_t)));
    const uint32_t zero = 0;
    ZK_CUDA_TRY(cudaMemcpyToSymbol(g_zk_check_flags, &zero, sizeof(uint32_t)));
#endif
    return ZK_OK;
}

int twiddles(zk_ctx *ctx, int lg, const uint32_t **out, cudaStream_t s) {
    Shared &sh = *ctx->sh;
    std::lock_guard<std::mutex> g(sh.mu);
    DevBuf &b = sh.tw[lg];
    if (!b.p) {
        const size_t n = (size_t)1 << lg;
        ZK_TRY(dev_alloc(sh, b, (n + 3) * sizeof(Fr)));
        int err = ZK_OK;
        Fr *root = (Fr *)scratch(ctx, "ntt.root", sizeof(Fr), &err);
        if (!root) return err;
        k_root<<<1, 1, 0, s>>>((uint32_t)lg, root);
        count_launches(1);
        size_t threads = (n + 63) / 64;
        k_twiddles<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(root, (uint32_t)lg, (Fr *)b.p);
        ZK_LAUNCHED();
        // Shared read-only with lanes on other streams: finish before use.
        ZK_CUDA_TRY(cudaStreamSynchronize(s));
    }
    *out = (const uint32_t *)b.p;
    return ZK_OK;
}

// The stage-twiddle table of 2^lg points (lg <= kMaxRadixLog), built once.
static int stage_twiddles(zk_ctx *ctx, int lg, const uint32_t **out, cudaStream_t s) {
    if (lg < 0 || lg > kMaxRadixLog) return ZK_EINVAL;
    const uint32_t *tw;
    ZK_TRY(twiddles(ctx, lg, &tw, s));  // takes the shared lock itself
    Shared &sh = *ctx->sh;
    std::lock_guard<std::mutex> g(sh.mu);
    DevBuf &b = sh.tws[lg];
    if (!b.p) {
        const uint32_t n = 1u << lg;
        ZK_TRY(dev_alloc(sh, b, (size_t)n * 64));
        k_stage_twiddles<<<(n + 127) / 128, 128, 0, s>>>((const Fr *)tw, n, (uint32_t *)b.p);
        ZK_LAUNCHED();
        // Shared read-only with lanes on other streams: finish before use.
        ZK_CUDA_TRY(cudaStreamSynchronize(s));
    }
    *out = (const uint32_t *)b.p;
    return ZK_OK;
}

// Built-in largest pass radix (log2) when none is tuned: the fastest choices
// of an autotuner sweep on B300.  Up to 2^18 the shared-memory pass with
// radices 2^6 .. 2^8 wins (small CTAs, many resident per SM); from 2^19 on,
// two register-tiled passes (2^10 + 2^9 .. 2^11 + 2^11), half the DRAM
// passes of four and two stages per shared-memory exchange.
static int default_radix(int L) {
    if (L <= 9) return L ? L : 1;
    if (L <= 16) return 6;
    if (L <= 18) return 8;
    if (L <= 20) return 10;
    return 11;  // 2^21 .. : two register-tiled passes
}

static int radix_for(const Shared &sh, int L) {
    int r = sh.tuned_radix[L];
    return (r >= 1 && r <= kMaxRadixLog) ? r : default_radix(L);
}

int ntt_pass_radix(const Shared &sh, int L) { return radix_for(sh, L); }

// Workspace of one group: ping-pong buffers and per-pass pointer tables.
static size_t group_buf_bytes(const Shared &sh, size_t count, size_t n) {
    int L = ilog2(n);
    int P = (int)plan_passes(L, radix_for(sh, L)).size();
    return P > 1 ? (size_t)(P > 2 ? 2 : 1) * count * n * 32 : 0;
}
static size_t group_tab_words(const Shared &sh, size_t count, size_t n) {
    int L = ilog2(n);
    return plan_passes(L, radix_for(sh, L)).size() * 2 * count;
}

// Runs every pass for `count` vectors of the same length n.  `buf` and
// `tabs` are this group's workspace (sizes from the two functions above).
static int ntt_group(zk_ctx *ctx, uint32_t *const *data_h, size_t count, size_t n, bool inverse,
                     uint32_t *buf, uint64_t *tabs, cudaStream_t s) {
    const int L = ilog2(n);
    if (L == 0) return ZK_OK;  // a length-1 transform is the identity
    std::vector<int> passes = plan_passes(L, radix_for(*ctx->sh, L));
    const int P = (int)passes.size();
    const size_t tab_words = 2 * count;
    std::vector<uint64_t> h((size_t)P * tab_words);
    for (int p = 0; p < P; p++) {
        for (size_t v = 0; v < count; v++) {
            uint64_t src = p == 0 ? (uint64_t)data_h[v]
                                  : (uint64_t)(buf + (((p - 1) % 2) * count + v) * n * 8);
            uint64_t dst = p == P - 1 ? (uint64_t)data_h[v]
                                      : (uint64_t)(buf + ((p % 2) * count + v) * n * 8);
            h[p * tab_words + v] = src;
            h[p * tab_words + count + v] = dst;
        }
    }
    ZK_TRY(upload(ctx, tabs, h.data(), h.size() * 8, s));
    const uint32_t *tw_n;
    ZK_TRY(twiddles(ctx, L, &tw_n, s));
    int logNs = 0;
    PhaseScope ph(ctx, ZK_PHASE_NTT, s);
    for (int p = 0; p < P; p++) {
        const int logR = passes[p];
        const uint32_t *tw_S;
        ZK_TRY(stage_twiddles(ctx, logR, &tw_S, s));
        PassArgs a;
        a.in_tab = (const uint32_t *const *)(tabs + p * tab_words);
        a.out_tab = (uint32_t *const *)(tabs + p * tab_words + count);
        a.logn = (uint32_t)L;
        a.logR = (uint32_t)logR;
        a.logNs = (uint32_t)logNs;
        const uint64_t subs = (uint64_t)n >> logR;
        // Radices of 2^9 and more: register-tiled pass (J R = 1024 elements
        // per CTA where the length allows); smaller ones: shared-memory pass
        // (J <= 4, J R 32 bytes <= 128 KiB), which measured faster there.
        const bool reg = logR >= kRegMinLog;
        a.J = reg ? (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, kRegJR >> logR), subs)
                  : (uint32_t)std::min<uint64_t>(std::min<uint64_t>(kMaxJ, subs),
                                                 kMaxSmem / ((size_t)32 << logR));
        a.logJ = 0;
        while ((1u << a.logJ) < a.J) a.logJ++;
        a.tw_n = (const Fr *)tw_n;
        a.tw_S = tw_S;
        a.inverse = inverse ? 1 : 0;
        a.scale = (inverse && p == P - 1) ? 1 : 0;
        const uint32_t JR = a.J << logR;
        dim3 grid((unsigned)(subs / a.J), (unsigned)count);
        if (reg) {
            ZK_TRY(launch_reg((uint32_t)logR, grid, s, a));
        } else {
            const uint32_t threads = std::min<uint32_t>(512, std::max<uint32_t>(32, JR / 2));
            const size_t smem = (size_t)JR * 32;
            ZK_TRY(launch_pass(a.logJ + (uint32_t)logR, grid, threads, smem, s, a));
        }
        logNs += logR;
    }
    return ZK_OK;
}

int ntt_impl(zk_ctx *ctx, uint32_t *data, size_t n, bool inverse, cudaStream_t s) {
    if (!data || !is_pow2(n) || n > ((size_t)1 << kMaxLogN)) return ZK_EINVAL;
    size_t lens[1] = {n};
    uint32_t *const v[1] = {data};
    return ntt_batch_impl(ctx, v, lens, 1, inverse, s);
}

int ntt_batch_impl(zk_ctx *ctx, uint32_t *const *data, const size_t *lens, size_t count,
                   bool inverse, cudaStream_t s) {
    if (count == 0) return ZK_OK;
    if (!data || !lens) return ZK_EINVAL;
    std::map<size_t, std::vector<uint32_t *>> groups;
    for (size_t k = 0; k < count; k++) {
        if (!data[k] || !is_pow2(lens[k]) || lens[k] > ((size_t)1 << kMaxLogN)) return ZK_EINVAL;
        groups[lens[k]].push_back(data[k]);
    }
    // Size the whole batch's workspace first so that no buffer is reallocated
    // while an earlier group's passes are still queued.
    size_t buf_bytes = 0, tab_words = 0;
    for (auto &g : groups) {
        buf_bytes += group_buf_bytes(*ctx->sh, g.second.size(), g.first);
        tab_words += group_tab_words(*ctx->sh, g.second.size(), g.first);
    }
    int err = ZK_OK;
    uint32_t *buf = nullptr;
    if (buf_bytes) {
        buf = (uint32_t *)scratch(ctx, "ntt.buf", buf_bytes, &err);
        if (!buf) return err;
    }
    uint64_t *tabs = (uint64_t *)scratch(ctx, "ntt.tabs", std::max<size_t>(tab_words, 1) * 8, &err);
    if (!tabs) return err;
    for (auto &g : groups) {
        ZK_TRY(ntt_group(ctx, g.second.data(), g.second.size(), g.first, inverse, buf, tabs, s));
        buf += group_buf_bytes(*ctx->sh, g.second.size(), g.first) / 4;
        tabs += group_tab_words(*ctx->sh, g.second.size(), g.first);
    }
    return ZK_OK;
}

}  // namespace zk
