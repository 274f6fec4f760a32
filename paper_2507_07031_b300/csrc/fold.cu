// fold.cu -- generalised Mira accumulation (paper Sec. 4.2, prover steps 2-7)
// for the degree-2 relation m1 o m2 - mu m3 = e over H (or, selected per
// context, the degree-3 relation m1 o m2 o m3 - mu^2 m4 = e), batched over all
// folds of a tree level.
//
// For fold(L, R, gamma) (L plays acc, scaled by gamma; R plays acc'):
//   K4  per element k (one pass over both accumulators, in place on R allowed):
//         e1  = m1 m2' + m1' m2 - mu m3' - mu' m3            (step 2)
//         m_i'' = gamma m_i + m_i'  (i = 1..4),  e'' = e' + gamma e1 + gamma^2 e
//   INTT of every e1, then one batched MSM: E1 = Commit(e1)  (step 3)
//   K5  per fold: C_i'' = gamma C_i + C_i', E'' = E' + gamma E1 + gamma^2 E,
//       mu'' = gamma mu + mu'                                (step 5)
// Degree 3 has two cross terms (the gamma^1 and gamma^2 coefficients of
// R(gamma L + R)), e1 and e2, committed as E1, E2, and
//   e'' = e' + gamma e1 + gamma^2 e2 + gamma^3 e,  E'' = E' + gamma E1 + gamma^2 E2 + gamma^3 E.
// Field vectors are canonical.  The per-fold constants (gamma and its powers
// in Montgomery form, so that mont(x, gamma R) = gamma x stays canonical;
// gamma's precomputed quotient for the witness RLC; the mu coefficients of
// the cross terms) are computed once per fold by K4c, not by every thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctx.cuh"
#include "curve.cuh"
#include "team.cuh"

namespace zk {

namespace {

// Per-fold constants of the witness pass (device workspace, written by
// k_fold_consts).  Montgomery form where marked, canonical otherwise.
struct FoldConsts {
    Fr g, g2, g3;  // gamma, gamma^2, gamma^3 (Montgomery)
    Fr gc, gq;     // gamma and floor(gamma 2^256 / r): the RLC product m'' = gamma m + m'
    Fr kc, kq;     // the cross terms' conversion factor (R mod r for degree 2, R^2 mod r
                   // for degree 3) and its quotient
    Fr c0, c1, c2;  // degree 2: r - mu, r - mu'; degree 3: -mu^2 R^-1, -mu'^2 R^-1,
                    // -2 mu mu' R^-1
};

struct FoldDesc {
    const uint32_t *Lm[4];
    const uint32_t *Le;
    const uint32_t *Lx;  // zk_acc_inst
    const uint32_t *Rm[4];
    const uint32_t *Re;
    const uint32_t *Rx;
    uint32_t *Om[4];
    uint32_t *Oe;
    uint32_t *Ox;
    const uint32_t *gamma;  // canonical F_r, device
    uint32_t *e1;           // n elements (workspace)
    uint32_t *E1;           // one canonical affine point (workspace or caller)
    uint32_t *e2;           // degree 3: second cross term (workspace)
    uint32_t *E2;           // degree 3: its commitment
    uint32_t deg;           // 2 or 3
    FoldConsts *fc;         // this fold's constants (device workspace)
};

constexpr int kInstMu = 40 * 2;  // word offset of mu in zk_acc_inst (5 points x 16 words)

// K4c: the per-fold constants, one thread per fold.
__global__ void k_fold_consts(const FoldDesc *__restrict__ descs, uint32_t F) {
    const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    const FoldDesc &d = descs[f];
    FoldConsts &c = *d.fc;
    const Fr gc = fe_load<FrP>(d.gamma);
    const Fr g = fe_to_mont<FrP>(gc);
    const Fr g2 = fe_mul<FrP>(g, g);
    fe_store<FrP>(c.g.v, g);
    fe_store<FrP>(c.g2.v, g2);
    fe_store<FrP>(c.g3.v, fe_mul<FrP>(g2, g));
    fe_store<FrP>(c.gc.v, gc);
    fe_store<FrP>(c.gq.v, fe_shoup_quotient_mont<FrP>(g));
    const Fr uL = fe_load<FrP>(d.Lx + kInstMu), uR = fe_load<FrP>(d.Rx + kInstMu);
    Fr kc;
    if (d.deg == 3) {
#pragma unroll
        for (int i = 0; i < 8; i++) kc.v[i] = FrP::r2(i);  // R^2 mod r as a plain residue
        fe_store<FrP>(c.c0.v, fe_neg<FrP>(fe_mul<FrP>(uL, uL)));
        fe_store<FrP>(c.c1.v, fe_neg<FrP>(fe_mul<FrP>(uR, uR)));
        fe_store<FrP>(c.c2.v, fe_neg<FrP>(fe_dbl<FrP>(fe_mul<FrP>(uL, uR))));
    } else {
#pragma unroll
        for (int i = 0; i < 8; i++) kc.v[i] = FrP::one(i);  // R mod r as a plain residue
        fe_store<FrP>(c.c0.v, fe_neg<FrP>(uL));
        fe_store<FrP>(c.c1.v, fe_neg<FrP>(uR));
        fe_store<FrP>(c.c2.v, fe_zero<FrP>());
    }
    fe_store<FrP>(c.kc.v, kc);
    fe_store<FrP>(c.kq.v, fe_shoup_quotient<FrP>(kc));
}

// K4: cross terms and witness RLC, grid (elements, folds); one instance per
// relation degree.  Both fit two blocks per SM (at most 128 registers, no
// spill), twice the warps that one block at ~190-240 registers gave, which
// the pass needs to keep its product chains issuing.  The RLC products by
// gamma and the cross terms' conversion factor are products by a per-fold
// constant, taken with its precomputed quotient (fe_mul_shoup).
template <int DEG>
__global__ void __launch_bounds__(256, 2)
    k_fold_witness(const FoldDesc *__restrict__ descs, uint32_t n) {
    const FoldDesc &d = descs[blockIdx.y];
    const FoldConsts &c = *d.fc;
    const Fr g = fe_ldg<FrP>(c.g.v), g2 = fe_ldg<FrP>(c.g2.v);
    // gamma m + m' for one witness column (precomputed-quotient product)
    auto rlc = [&](const Fr &a, const Fr &b) {
        return fe_add<FrP>(fe_mul_shoup<FrP>(a, fe_ldg<FrP>(c.gc.v), fe_ldg<FrP>(c.gq.v)), b);
    };
    // the canonical cross term from its reduced lazy sum
    auto convert = [&](const Fr &x) { return fe_mul_shoup<FrP>(x, fe_ldg<FrP>(c.kc.v), fe_ldg<FrP>(c.kq.v)); };
    if constexpr (DEG == 3) {
        // Sums of products share one Montgomery reduction (see the degree-2
        // branch).  The pair products enter as x R^-1 (a Montgomery product
        // of canonical values), so each cross term is a sum of four products
        // of values below r whose reduction is e R^-2; a product with R^2
        // (convert) gives the canonical e.  The mu coefficients are prepared
        // the same way: -mu_L^2 R^-1, -mu_R^2 R^-1, -2 mu_L mu_R R^-1.
        using namespace detail;
        const Fr cLL = fe_ldg<FrP>(c.c0.v), cRR = fe_ldg<FrP>(c.c1.v), cLR = fe_ldg<FrP>(c.c2.v);
        const Fr g3 = fe_ldg<FrP>(c.g3.v);
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const size_t o = 8 * (size_t)k;
            // Consumed in three groups, each finished (its RLC outputs
            // stored) before the next is loaded, to keep the live set small.
            Fr sx, paa, pbb;  // (a1 b2 + b1 a2, a1 a2, b1 b2) R^-1
            {
                const Fr a1 = fe_load<FrP>(d.Lm[0] + o), a2 = fe_load<FrP>(d.Lm[1] + o);
                const Fr b1 = fe_load<FrP>(d.Rm[0] + o), b2 = fe_load<FrP>(d.Rm[1] + o);
                paa = fe_mul<FrP>(a1, a2);
                pbb = fe_mul<FrP>(b1, b2);
                sx = redc_wide<FrP>(wide_add<FrP>(wide_mul<FrP>(a1, b2), wide_mul<FrP>(b1, a2)));
                fe_store<FrP>(d.Om[0] + o, rlc(a1, b1));
                fe_store<FrP>(d.Om[1] + o, rlc(a2, b2));
            }
            Wide w2, w1;
            {
                const Fr a3 = fe_load<FrP>(d.Lm[2] + o), b3 = fe_load<FrP>(d.Rm[2] + o);
                // gamma^2: a1 a2 b3 + (a1 b2 + b1 a2) a3;  gamma^1: (a1 b2 + b1 a2) b3 + b1 b2 a3
                w2 = wide_add<FrP>(wide_mul<FrP>(paa, b3), wide_mul<FrP>(sx, a3));
                w1 = wide_add<FrP>(wide_mul<FrP>(sx, b3), wide_mul<FrP>(pbb, a3));
                fe_store<FrP>(d.Om[2] + o, rlc(a3, b3));
            }
            Fr e1, e2;
            {
                const Fr a4 = fe_load<FrP>(d.Lm[3] + o), b4 = fe_load<FrP>(d.Rm[3] + o);
                // - mu_L^2 b4 - 2 mu_L mu_R a4 (gamma^2), - 2 mu_L mu_R b4 - mu_R^2 a4 (gamma^1)
                w2 = wide_add<FrP>(w2, wide_add<FrP>(wide_mul<FrP>(b4, cLL), wide_mul<FrP>(a4, cLR)));
                w1 = wide_add<FrP>(w1, wide_add<FrP>(wide_mul<FrP>(b4, cLR), wide_mul<FrP>(a4, cRR)));
                e2 = convert(redc_wide<FrP>(w2));
                e1 = convert(redc_wide<FrP>(w1));
                fe_store<FrP>(d.Om[3] + o, rlc(a4, b4));
            }
            fe_store<FrP>(d.e1 + o, e1);
            fe_store<FrP>(d.e2 + o, e2);
            const Fr eL = fe_load<FrP>(d.Le + o), eR = fe_load<FrP>(d.Re + o);
            // e'' = e' + gamma e1 + gamma^2 e2 + gamma^3 e (three products, one reduction)
            const Fr t = redc_wide<FrP>(wide_add<FrP>(wide_add<FrP>(wide_mul<FrP>(e1, g), wide_mul<FrP>(e2, g2)),
                                                      wide_mul<FrP>(eL, g3)));
            fe_store<FrP>(d.Oe + o, fe_add<FrP>(eR, t));
        }
    } else {
        // Sums of products share one Montgomery reduction (lazy reduction):
        // a sum of at most four products of values below r is below
        // 4 r^2 < r 2^256, the reduction's bound.  The mu terms enter with
        // the canonical negations r - mu, so every term is a plain product.
        using namespace detail;
        const Fr nmuL = fe_ldg<FrP>(c.c0.v), nmuR = fe_ldg<FrP>(c.c1.v);
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
            const size_t o = 8 * (size_t)k;
            Fr a1 = fe_load<FrP>(d.Lm[0] + o), a2 = fe_load<FrP>(d.Lm[1] + o);
            Fr a3 = fe_load<FrP>(d.Lm[2] + o), a4 = fe_load<FrP>(d.Lm[3] + o);
            Fr b1 = fe_load<FrP>(d.Rm[0] + o), b2 = fe_load<FrP>(d.Rm[1] + o);
            Fr b3 = fe_load<FrP>(d.Rm[2] + o), b4 = fe_load<FrP>(d.Rm[3] + o);
            Fr eL = fe_load<FrP>(d.Le + o), eR = fe_load<FrP>(d.Re + o);
            // e1 = m1 m2' + m1' m2 - mu m3' - mu' m3: one reduction gives
            // e1 R^-1, a product with R (convert) the canonical value.
            const Wide w = wide_add<FrP>(wide_add<FrP>(wide_mul<FrP>(a1, b2), wide_mul<FrP>(b1, a2)),
                                         wide_add<FrP>(wide_mul<FrP>(b3, nmuL), wide_mul<FrP>(a3, nmuR)));
            const Fr e1 = convert(redc_wide<FrP>(w));
            fe_store<FrP>(d.e1 + o, e1);
            fe_store<FrP>(d.Om[0] + o, rlc(a1, b1));
            fe_store<FrP>(d.Om[1] + o, rlc(a2, b2));
            fe_store<FrP>(d.Om[2] + o, rlc(a3, b3));
            fe_store<FrP>(d.Om[3] + o, rlc(a4, b4));
            // e'' = e' + gamma e1 + gamma^2 e (g, g2 in Montgomery form)
            const Fr t = redc_wide<FrP>(wide_add<FrP>(wide_mul<FrP>(e1, g), wide_mul<FrP>(eL, g2)));
            fe_store<FrP>(d.Oe + o, fe_add<FrP>(eR, t));
        }
    }
}

// mu'' = gamma mu + mu' (one thread per fold).  Runs after the witness pass,
// which reads both mu (the output may alias R).
__global__ void k_fold_mu(const FoldDesc *__restrict__ descs, uint32_t folds) {
    uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= folds) return;
    const FoldDesc &d = descs[f];
    Fr gm = fe_to_mont<FrP>(fe_load<FrP>(d.gamma));
    Fr mu = fe_add<FrP>(fe_mul<FrP>(fe_load<FrP>(d.Lx + kInstMu), gm), fe_load<FrP>(d.Rx + kInstMu));
    fe_store<FrP>(d.Ox + kInstMu, mu);
}

// K5: instance RLC, C_i'' = gamma C_i + C_i' and E'' = E' + gamma E1 +
// gamma^2 E (degree 3: E' + gamma E1 + gamma^2 E2 + gamma^3 E).  It touches
// only the points of the instances, so it may run on a side stream while the
// next tree level's witness work (which reads only vectors and mu) proceeds.
//
// Every product of a scalar and a point is its own lane of a team (four warps
// sharing each point operation): per fold, lanes C_1..C_4 (gamma), gamma E1,
// then gamma^2 E (degree 2) or gamma^2 E2, gamma^3 E (degree 3).  A lane runs
// its scalar k as k1 P1 + k2 P2 with the GLV split k = k1 + k2 lambda
// (curve.cuh; |k1|, |k2| < 2^130, P1 = sign(k1) P, P2 = sign(k2) phi(P)): a
// table of d1 P1 + d2 P2 for d1, d2 < 4 (each lane its own, in shared
// memory), then per 2-bit digit pair from the top two doublings and one
// addition of its table entry.  About 130 doublings and 65 additions instead
// of 254 of each for plain double-and-add (a team addition costs four
// product latencies, a doubling three); a 4-bit window without the split took
// 252 and 64, and 1.0 ms against 1.7 per fold.  The lanes of one fold then
// meet in one thread per output point, which adds the primed point and
// normalises.
constexpr int kInstAcc = 0, kInstTmp = 4, kInstT = 8, kInstTab = kInstT + kTeamTemps;
constexpr int kInstSlots = kInstTab + 4 * 16;
constexpr size_t kInstSmem = (size_t)kInstSlots * 8 * 32 * sizeof(uint32_t);

template <int DEG>
__global__ void __launch_bounds__(kTeamThreads) k_fold_instance(const FoldDesc *__restrict__ descs,
                                                                uint32_t folds) {
    constexpr int kOps = DEG == 3 ? 7 : 6;  // scalar-point products per fold
    constexpr int kFolds = 32 / kOps;       // folds per team
    constexpr int kAcc = kInstAcc, kTmp = kInstTmp, kT = kInstT, kTab = kInstTab;
    extern __shared__ uint32_t f[];  // kInstSlots slots
    const uint32_t l = team_lane(), w = team_warp();
    const uint32_t fl = blockIdx.x * kFolds + l / kOps, op = l % kOps;
    const bool valid = l < kFolds * kOps && fl < folds;
    uint32_t k[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    Xyzz base = xyzz_inf();
    if (valid) {
        const FoldDesc &d = descs[fl];
        const Fr gm = fe_to_mont<FrP>(fe_load<FrP>(d.gamma));
        const int pw = op < 5 ? 1 : (int)op - 3;  // power of gamma
        Fr sm = gm;
        for (int j = 1; j < pw; j++) sm = fe_mul<FrP>(sm, gm);
        const Fr sc = fe_from_mont<FrP>(sm);
#pragma unroll
        for (int i = 0; i < 8; i++) k[i] = sc.v[i];
        const uint32_t *src = op < 4 ? d.Lx + 16 * op : op == 4 ? d.E1 : (DEG == 3 && op == 5) ? d.E2 : d.Lx + 64;
        base = xyzz_load_canonical(src);
    }
    uint32_t k1[kGlvWords], k2[kGlvWords];
    bool n1, n2;
    glv_split(k, k1, n1, k2, n2);
    const Xyzz p1 = n1 ? xyzz_neg(base) : base;
    Xyzz p2 = xyzz_phi(base);
    if (n2) p2 = xyzz_neg(p2);
    // Table T[d1 + 4 d2] = d1 P1 + d2 P2 (T[0] = infinity).
    team_set_inf_nosync(f, kTab);
    tf_store(f, kTab + 4 + w, w == 0 ? p1.X : w == 1 ? p1.Y : w == 2 ? p1.ZZ : p1.ZZZ);
    tf_store(f, kTab + 16 + w, w == 0 ? p2.X : w == 1 ? p2.Y : w == 2 ? p2.ZZ : p2.ZZZ);
    __syncthreads();
    team_dbl(f, kTab + 4, kTab + 8, kT);               // 2 P1
    team_add(f, kTab + 8, kTab + 4, kTab + 12, kT);    // 3 P1
    team_dbl(f, kTab + 16, kTab + 32, kT);             // 2 P2
    team_add(f, kTab + 32, kTab + 16, kTab + 48, kT);  // 3 P2
    for (int d2 = 1; d2 < 4; d2++)
        for (int d1 = 1; d1 < 4; d1++) team_add(f, kTab + 4 * d1, kTab + 16 * d2, kTab + 4 * (d1 + 4 * d2), kT);
    team_set_inf_nosync(f, kAcc);
    __syncthreads();
    // 2-bit digit pairs from bit 129 down; leading windows where no lane has
    // a digit are skipped (block-uniform).
    bool started = false;
    for (int i = 16 * kGlvWords - 1; i >= 0; i--) {
        const int bit = 2 * i;  // digits do not cross words
        const uint32_t e = ((k1[bit >> 5] >> (bit & 31)) & 3u) + 4u * ((k2[bit >> 5] >> (bit & 31)) & 3u);
        if (started) {
            team_dbl(f, kAcc, kAcc, kT);
            team_dbl(f, kAcc, kAcc, kT);
        }
        if (!__syncthreads_or(e != 0)) continue;
        started = true;
        tf_store(f, kTmp + w, tf_load(f, kTab + 4 * (int)e + w));  // this lane's entry
        __syncthreads();
        team_add(f, kAcc, kTmp, kAcc, kT);
    }
    // One thread per output point: C_1..C_4 and E of each fold.
    const uint32_t t = threadIdx.x;
    const uint32_t fo = blockIdx.x * kFolds + t / 5, out = t % 5;
    if (t >= 5 * kFolds || fo >= folds) return;
    const FoldDesc &d = descs[fo];
    const uint32_t lane0 = (t / 5) * kOps;
    Xyzz r = xyzz_load_canonical(d.Rx + 16 * out);
    const uint32_t first = out < 4 ? out : 4, last = out < 4 ? out : kOps - 1;
    for (uint32_t j = first; j <= last; j++) r = xyzz_add(r, team_point_of(f, kAcc, lane0 + j));
    xyzz_store_canonical(d.Ox + 16 * out, r);
}

// Leaves: out = m1 o m2 (degree 2: out = m3) or m1 o m2 o m3 (degree 3, m3
// given: out = m4), e = 0, mu = 1, E = infinity (C_i are written by the MSM).
// A group of leaves in one launch (blockIdx.y = leaf): the k_leaf work, and
// on the INTT route a copy of the four witness vectors (the derived one as
// just computed) into the workspace the batched INTT transforms in place.
struct LeafDesc {
    const uint32_t *m[4];
    uint32_t *out;  // the derived vector: m[2] (degree 2) or m[3] (degree 3)
    uint32_t *e, *x;
    uint32_t *ws;   // 4 n elements, or null (Lagrange route: commit in place)
};

__global__ void k_leaf_batch(const LeafDesc *__restrict__ descs, uint32_t n, int degree) {
    const LeafDesc &L = descs[blockIdx.y];
    const int derived = degree == 3 ? 3 : 2;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t o = 8 * (size_t)k;
        Fr p = fe_mul<FrP>(fe_to_mont<FrP>(fe_load<FrP>(L.m[0] + o)), fe_load<FrP>(L.m[1] + o));  // canonical m1 m2
        if (degree == 3) p = fe_mul<FrP>(fe_to_mont<FrP>(p), fe_load<FrP>(L.m[2] + o));
        fe_store<FrP>(L.out + o, p);
        fe_store<FrP>(L.e + o, fe_zero<FrP>());
        if (L.ws) {
#pragma unroll
            for (int i = 0; i < 4; i++)
                fe_store<FrP>(L.ws + (size_t)i * n * 8 + o, i == derived ? p : fe_load<FrP>(L.m[i] + o));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 16) {
        L.x[64 + threadIdx.x] = 0;                        // E = infinity
        if (threadIdx.x < 8) L.x[kInstMu + threadIdx.x] = threadIdx.x == 0 ? 1u : 0u;  // mu = 1
    }
}

bool pow2(size_t n) { return n && !(n & (n - 1)); }

int ilog2_size(size_t n) {
    int l = 0;
    while (((size_t)1 << l) < n) l++;
    return l;
}

bool acc_ok(const zk_acc *a, size_t n) {
    if (!a || a->n != n || !a->e || !a->x) return false;
    for (int i = 0; i < 4; i++)
        if (!a->m[i]) return false;
    return true;
}

unsigned elem_blocks(uint32_t n) { return std::min<unsigned>((n + 255) / 256, 1024u); }

// Runs a batch of folds that share the length n.  dd: device descriptor
// slots (F), fc: device constant slots (F), E1: device points (F); the
// instance pass runs on s_inst after the batch's E1 commitments exist
// (s_inst may equal s).
int fold_batch(zk_ctx *ctx, std::vector<FoldDesc> &descs, uint32_t n, FoldDesc *dd, FoldConsts *fc,
               uint32_t *E1, cudaStream_t s, cudaStream_t s_inst, cudaEvent_t ev) {
    const size_t F = descs.size();
    if (F == 0) return ZK_OK;
    int err = ZK_OK;
    const bool three = descs[0].deg == 3;
    const size_t nx = three ? 2 : 1;  // cross terms per fold
    uint32_t *e1 = (uint32_t *)scratch(ctx, "fold.e1", nx * F * (size_t)n * 32, &err);
    if (!e1) return err;
    // E1 = Commit(e1): INTT then the SRS, or the Lagrange basis directly.
    const int lg = ilog2_size(n);
    const bool lagrange = ctx->sh->commit_route == ZK_ROUTE_LAGRANGE;
    if (lagrange) {
        const Affine *lb;
        ZK_TRY(lagrange_get(ctx, lg, &lb, s));
    }
    // E1 points of the batch at E1[16 f], E2 points (degree 3) at E1[16 (F + f)].
    std::vector<uint32_t *> vecs(nx * F);
    std::vector<size_t> lens(nx * F, n);
    std::vector<MsmJob> jobs(nx * F);
    for (size_t f = 0; f < F; f++) {
        descs[f].fc = fc + f;
        descs[f].e1 = e1 + f * (size_t)n * 8;
        if (!descs[f].E1) descs[f].E1 = E1 + 16 * f;
        vecs[f] = descs[f].e1;
        jobs[f].scalars = descs[f].e1;
        jobs[f].n = n;
        jobs[f].out = descs[f].E1;
        jobs[f].basis = lagrange ? lg : 0;
        if (three) {
            descs[f].e2 = e1 + (F + f) * (size_t)n * 8;
            if (!descs[f].E2) descs[f].E2 = E1 + 16 * (F + f);
            vecs[F + f] = descs[f].e2;
            jobs[F + f].scalars = descs[f].e2;
            jobs[F + f].n = n;
            jobs[F + f].out = descs[f].E2;
            jobs[F + f].basis = lagrange ? lg : 0;
        }
    }
    ZK_TRY(upload(ctx, dd, descs.data(), F * sizeof(FoldDesc), s));
    dim3 g(elem_blocks(n), (unsigned)F);
    {
        PhaseScope ph(ctx, ZK_PHASE_FOLD_WITNESS, s);
        k_fold_consts<<<(unsigned)((F + 63) / 64), 64, 0, s>>>(dd, (uint32_t)F);
        ZK_LAUNCHED();
        if (three) k_fold_witness<3><<<g, 256, 0, s>>>(dd, n);
        else k_fold_witness<2><<<g, 256, 0, s>>>(dd, n);
        ZK_LAUNCHED();
        k_fold_mu<<<(unsigned)((F + 63) / 64), 64, 0, s>>>(dd, (uint32_t)F);
        ZK_LAUNCHED();
    }
    if (!lagrange) ZK_TRY(ntt_batch_impl(ctx, vecs.data(), lens.data(), nx * F, true, s));
    ZK_TRY(msm_batch_impl(ctx, jobs.data(), nx * F, 0, s));
    if (s_inst != s) {
        ZK_CUDA_TRY(cudaEventRecord(ev, s));
        ZK_CUDA_TRY(cudaStreamWaitEvent(s_inst, ev, 0));
    }
    {
        PhaseScope ph(ctx, ZK_PHASE_FOLD_INSTANCE, s_inst);
        ZK_TRY(set_max_dynamic_smem(three ? (const void *)k_fold_instance<3> : (const void *)k_fold_instance<2>,
                                    (int)kInstSmem));
        if (three) k_fold_instance<3><<<(unsigned)((F + 3) / 4), kTeamThreads, kInstSmem, s_inst>>>(dd, (uint32_t)F);
        else k_fold_instance<2><<<(unsigned)((F + 4) / 5), kTeamThreads, kInstSmem, s_inst>>>(dd, (uint32_t)F);
        ZK_LAUNCHED();
    }
    return ZK_OK;
}

FoldDesc make_desc(const zk_acc *L, const zk_acc *R, const zk_acc *O, const uint32_t *gamma, uint32_t deg) {
    FoldDesc d;
    for (int i = 0; i < 4; i++) {
        d.Lm[i] = (const uint32_t *)L->m[i];
        d.Rm[i] = (const uint32_t *)R->m[i];
        d.Om[i] = (uint32_t *)O->m[i];
    }
    d.Le = (const uint32_t *)L->e;
    d.Re = (const uint32_t *)R->e;
    d.Oe = (uint32_t *)O->e;
    d.Lx = (const uint32_t *)L->x;
    d.Rx = (const uint32_t *)R->x;
    d.Ox = (uint32_t *)O->x;
    d.gamma = gamma;
    d.e1 = nullptr;
    d.E1 = nullptr;
    d.e2 = nullptr;
    d.E2 = nullptr;
    d.deg = deg;
    d.fc = nullptr;
    return d;
}

}  // namespace

int fold_impl(zk_ctx *ctx, const zk_acc *L, const zk_acc *R, const zk_fr *gamma, zk_acc *out,
              zk_g1 *E1_out, cudaStream_t s) {
    if (!L || !R || !out || !gamma) return ZK_EINVAL;
    const size_t n = L->n;
    if (!pow2(n) || n < 2 || n > ((size_t)1 << kMaxSrsLog)) return ZK_EINVAL;
    if (!acc_ok(L, n) || !acc_ok(R, n) || !acc_ok(out, n)) return ZK_EINVAL;
    if (out->x == L->x || out->e == L->e) return ZK_EINVAL;
    if (n > ctx->sh->srs_n) return ZK_ESRS;
    int err = ZK_OK;
    const uint32_t *g = (const uint32_t *)gamma;
    if (!is_device_ptr(gamma)) {
        uint32_t *gd = (uint32_t *)scratch(ctx, "fold.gamma", 32, &err);
        if (!gd) return err;
        ZK_TRY(upload(ctx, gd, gamma, 32, s));
        g = gd;
    }
    const uint32_t deg = (uint32_t)ctx->sh->fold_degree;
    std::vector<FoldDesc> d(1, make_desc(L, R, out, g, deg));
    uint32_t *E1 = (uint32_t *)scratch(ctx, "fold.E1", 128, &err);
    FoldDesc *dd = (FoldDesc *)scratch(ctx, "fold.descs", sizeof(FoldDesc), &err);
    FoldConsts *fc = (FoldConsts *)scratch(ctx, "fold.consts", sizeof(FoldConsts), &err);
    if (!E1 || !dd || !fc) return err;
    ZK_TRY(fold_batch(ctx, d, (uint32_t)n, dd, fc, E1, s, s, nullptr));
    if (E1_out) {  // E1, then E2 for degree 3 (contiguous in the workspace)
        const size_t bytes = 64 * (deg - 1);
        if (is_device_ptr(E1_out)) {
            ZK_CUDA_TRY(cudaMemcpyAsync(E1_out, d[0].E1, bytes, cudaMemcpyDeviceToDevice, s));
        } else {
            ZK_CUDA_TRY(cudaMemcpyAsync(E1_out, d[0].E1, bytes, cudaMemcpyDeviceToHost, s));
            ZK_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    return ZK_OK;
}

int fold_tree_impl(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, zk_acc *root,
                   cudaStream_t s, size_t levels) {
    if (!leaves || !gammas || !pow2(count) || count < 2) return ZK_EINVAL;
    size_t all = 0;
    while (((size_t)1 << all) < count) all++;
    if (levels == 0) levels = all;
    if (levels > all || (levels == all && !root)) return ZK_EINVAL;
    const size_t n = leaves[0].n;
    if (!pow2(n) || n < 2 || n > ((size_t)1 << kMaxSrsLog)) return ZK_EINVAL;
    for (size_t i = 0; i < count; i++)
        if (!acc_ok(&leaves[i], n)) return ZK_EINVAL;
    if (root && !acc_ok(root, n)) return ZK_EINVAL;
    if (n > ctx->sh->srs_n) return ZK_ESRS;
    int err = ZK_OK;
    // The challenges of the levels that run: a prefix of the level-major array.
    const size_t used = count - (count >> levels);
    const uint32_t *g = (const uint32_t *)gammas;
    if (!is_device_ptr(gammas)) {
        uint32_t *gd = (uint32_t *)scratch(ctx, "fold.gammas", used * 32, &err);
        if (!gd) return err;
        ZK_TRY(upload(ctx, gd, gammas, used * 32, s));
        g = gd;
    }
    // Per-fold descriptor slots and E1 points for the whole tree, so that a
    // level's instance pass (side stream) can still read its own while the
    // next level's witness work (main stream) runs.
    FoldDesc *dd = (FoldDesc *)scratch(ctx, "fold.treedescs", (count - 1) * sizeof(FoldDesc), &err);
    uint32_t *E1 = (uint32_t *)scratch(ctx, "fold.treeE1", (count - 1) * 128, &err);
    FoldConsts *fc = (FoldConsts *)scratch(ctx, "fold.treeconsts", (count - 1) * sizeof(FoldConsts), &err);
    if (!dd || !E1 || !fc) return err;
    if (!ctx->side) {
        // Highest priority: the instance pass's few blocks are dispatched
        // ahead of the next level's queued MSM blocks instead of after them.
        int least = 0, greatest = 0;
        ZK_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        ZK_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest));
        ZK_CUDA_TRY(cudaEventCreateWithFlags(&ctx->side_ev[0], cudaEventDisableTiming));
        ZK_CUDA_TRY(cudaEventCreateWithFlags(&ctx->side_ev[1], cudaEventDisableTiming));
    }
    // The side stream starts after everything queued on s so far.
    ZK_CUDA_TRY(cudaEventRecord(ctx->side_ev[1], s));
    ZK_CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->side_ev[1], 0));
    // Level l accumulator j lives in leaf slot j 2^l + 2^l - 1 (the fold
    // output overwrites its R operand).
    size_t width = count, goff = 0;
    for (size_t span = 2; span <= ((size_t)1 << levels); span <<= 1) {
        std::vector<FoldDesc> d;
        d.reserve(width / 2);
        for (size_t j = 0; j < width / 2; j++) {
            const zk_acc *Lp = &leaves[j * span + span / 2 - 1];
            zk_acc *Rp = &leaves[j * span + span - 1];
            d.push_back(make_desc(Lp, Rp, Rp, g + 8 * (goff + j), (uint32_t)ctx->sh->fold_degree));
        }
        // the level's E1 points at 2 goff (E1 then E2 for degree 3): disjoint per level
        ZK_TRY(fold_batch(ctx, d, (uint32_t)n, dd + goff, fc + goff, E1 + 32 * goff, s, ctx->side,
                          ctx->side_ev[0]));
        goff += width / 2;
        width /= 2;
    }
    // Join the side stream before the root's instance is copied (or, after
    // a partial tree, before the caller reads the level's accumulators).
    ZK_CUDA_TRY(cudaEventRecord(ctx->side_ev[1], ctx->side));
    ZK_CUDA_TRY(cudaStreamWaitEvent(s, ctx->side_ev[1], 0));
    if (levels < all) return ZK_OK;
    const zk_acc &top = leaves[count - 1];
    for (int i = 0; i < 4; i++)
        ZK_CUDA_TRY(cudaMemcpyAsync(root->m[i], top.m[i], n * 32, cudaMemcpyDeviceToDevice, s));
    ZK_CUDA_TRY(cudaMemcpyAsync(root->e, top.e, n * 32, cudaMemcpyDeviceToDevice, s));
    ZK_CUDA_TRY(cudaMemcpyAsync(root->x, top.x, sizeof(zk_acc_inst), cudaMemcpyDeviceToDevice, s));
    return ZK_OK;
}

int leaf_init_impl(zk_ctx *ctx, const zk_acc *accs, size_t count, cudaStream_t s) {
    if (!accs || count == 0) return ZK_EINVAL;
    const size_t n = accs[0].n;
    if (!pow2(n) || n < 2 || n > ((size_t)1 << kMaxSrsLog)) return ZK_EINVAL;
    for (size_t i = 0; i < count; i++)
        if (!acc_ok(&accs[i], n)) return ZK_EINVAL;
    if (n > ctx->sh->srs_n) return ZK_ESRS;
    // Commit in groups so the INTT and MSM workspace stays near 2^24 elements.
    const size_t group = std::max<size_t>(1, ((size_t)1 << 24) / (4 * n));
    int err = ZK_OK;
    const int lg = ilog2_size(n);
    const bool lagrange = ctx->sh->commit_route == ZK_ROUTE_LAGRANGE;
    if (lagrange) {
        const Affine *lb;
        ZK_TRY(lagrange_get(ctx, lg, &lb, s));
    }
    for (size_t a0 = 0; a0 < count; a0 += group) {
        const size_t a1 = std::min(count, a0 + group);
        const size_t G = a1 - a0;
        uint32_t *ws = nullptr;
        if (!lagrange) {
            ws = (uint32_t *)scratch(ctx, "leaf.ws", 4 * G * n * 32, &err);
            if (!ws) return err;
        }
        std::vector<uint32_t *> vecs;
        std::vector<size_t> lens;
        std::vector<MsmJob> jobs;
        std::vector<LeafDesc> hd(G);
        const int degree = ctx->sh->fold_degree;
        for (size_t a = a0; a < a1; a++) {
            const zk_acc &A = accs[a];
            LeafDesc &d = hd[a - a0];
            for (int i = 0; i < 4; i++) d.m[i] = (const uint32_t *)A.m[i];
            d.out = (uint32_t *)(degree == 3 ? A.m[3] : A.m[2]);
            d.e = (uint32_t *)A.e;
            d.x = (uint32_t *)A.x;
            d.ws = lagrange ? nullptr : ws + (a - a0) * 4 * n * 8;
            for (int i = 0; i < 4; i++) {
                MsmJob j;
                j.n = (uint32_t)n;
                j.out = (char *)A.x + 64 * i;
                if (lagrange) {  // commit the evaluations in place
                    j.scalars = (const uint32_t *)A.m[i];
                    j.basis = lg;
                } else {         // interpolate the workspace copy, then commit over the SRS
                    uint32_t *dst = d.ws + (size_t)i * n * 8;
                    vecs.push_back(dst);
                    lens.push_back(n);
                    j.scalars = dst;
                }
                jobs.push_back(j);
            }
        }
        LeafDesc *dd = (LeafDesc *)scratch(ctx, "leaf.descs", G * sizeof(LeafDesc), &err);
        if (!dd) return err;
        ZK_TRY(upload(ctx, dd, hd.data(), G * sizeof(LeafDesc), s));
        const unsigned bx = std::max(1u, std::min(elem_blocks((uint32_t)n), (unsigned)(4 * ctx->sh->sms / G + 1)));
        k_leaf_batch<<<dim3(bx, (unsigned)G), 256, 0, s>>>(dd, (uint32_t)n, degree);
        ZK_LAUNCHED();
        if (!lagrange) ZK_TRY(ntt_batch_impl(ctx, vecs.data(), lens.data(), vecs.size(), true, s));
        ZK_TRY(msm_batch_impl(ctx, jobs.data(), jobs.size(), 0, s));
    }
    return ZK_OK;
}

}  // namespace zk
