// curve.cuh -- BN254 G1 (y^2 = x^3 + 3 over F_q) on sm_103a.
//
// Points are kept in extended Jacobian "XYZZ" coordinates (x = X/ZZ,
// y = Y/ZZZ, ZZ^3 = ZZZ^2), whose mixed addition with an affine point costs
// 8 multiplications and 2 squarings.  Formulas: Explicit-Formulas Database,
// short Weierstrass a = 0, xyzz coordinates (madd-2008-s, mdbl-2008-s-1,
// dbl-2008-s-1, add-2008-s; D. Sutherland 2008).  The point at infinity is
// ZZ = ZZZ = 0.  The exceptional cases of addition (P = Q, P = -Q, either
// operand infinite) are handled explicitly, so every sum is exact.
//
// All coordinates are in Montgomery form on the device; affine points that
// cross the library boundary are canonical (x || y, 32 + 32 bytes, little
// endian) with infinity as 64 zero bytes.
#pragma once
#include "field.cuh"

namespace zk {

struct Affine {
    Fq x, y;
};

struct Xyzz {
    Fq X, Y, ZZ, ZZZ;
};

ZK_DEV Xyzz xyzz_inf() {
    Xyzz r;
    r.X = fe_zero<FqP>();
    r.Y = fe_zero<FqP>();
    r.ZZ = fe_zero<FqP>();
    r.ZZZ = fe_zero<FqP>();
    return r;
}

ZK_DEV bool xyzz_is_inf(const Xyzz &p) { return fe_is_zero<FqP>(p.ZZ); }

ZK_DEV Xyzz xyzz_from_affine(const Affine &a) {
    Xyzz r;
    r.X = a.x;
    r.Y = a.y;
    r.ZZ = fe_mont_one<FqP>();
    r.ZZZ = fe_mont_one<FqP>();
    return r;
}

ZK_DEV Affine affine_neg(const Affine &a) {
    Affine r;
    r.x = a.x;
    r.y = fe_neg<FqP>(a.y);
    return r;
}

ZK_DEV Xyzz xyzz_neg(const Xyzz &a) {
    Xyzz r = a;
    r.Y = fe_neg<FqP>(a.Y);
    return r;
}

// 2 * (x, y) for an affine point (mdbl-2008-s-1).
ZK_DEV Xyzz xyzz_dbl_affine(const Affine &a) {
    Fq U = fe_dbl<FqP>(a.y);
    Fq V = fe_sqr<FqP>(U);
    Fq W = fe_mul<FqP>(U, V);
    Fq S = fe_mul<FqP>(a.x, V);
    Fq M = fe_mul3<FqP>(fe_sqr<FqP>(a.x));
    Xyzz r;
    r.X = fe_sub<FqP>(fe_sqr<FqP>(M), fe_dbl<FqP>(S));
    r.Y = fe_mul_sub_mul<FqP>(M, fe_sub<FqP>(S, r.X), W, a.y);
    r.ZZ = V;
    r.ZZZ = W;
    return r;
}

// 2 P (dbl-2008-s-1, a = 0).  Infinity and points with Y = 0 map to infinity
// because V = (2Y)^2 becomes 0.
ZK_DEV Xyzz xyzz_dbl(const Xyzz &p) {
    Fq U = fe_dbl<FqP>(p.Y);
    Fq V = fe_sqr<FqP>(U);
    Fq W = fe_mul<FqP>(U, V);
    Fq S = fe_mul<FqP>(p.X, V);
    Fq M = fe_mul3<FqP>(fe_sqr<FqP>(p.X));
    Xyzz r;
    r.X = fe_sub<FqP>(fe_sqr<FqP>(M), fe_dbl<FqP>(S));
    r.Y = fe_mul_sub_mul<FqP>(M, fe_sub<FqP>(S, r.X), W, p.Y);
    r.ZZ = fe_mul<FqP>(V, p.ZZ);
    r.ZZZ = fe_mul<FqP>(W, p.ZZZ);
    return r;
}

// The mixed addition after U2 = x2 ZZ1 and S2 = y2 ZZZ1 (madd-2008-s), with
// P = U2 - X1 != 0 and R = S2 - Y1.
ZK_DEV Xyzz madd_finish(const Xyzz &p, const Fq &P, const Fq &R) {
    Fq PP = fe_sqr<FqP>(P);
    Fq PPP = fe_mul<FqP>(P, PP);
    Fq Q = fe_mul<FqP>(p.X, PP);
    Xyzz r;
    r.X = fe_sub<FqP>(fe_sub<FqP>(fe_sqr<FqP>(R), PPP), fe_dbl<FqP>(Q));
    r.Y = fe_mul_sub_mul<FqP>(R, fe_sub<FqP>(Q, r.X), p.Y, PPP);
    r.ZZ = fe_mul<FqP>(p.ZZ, PP);
    r.ZZZ = fe_mul<FqP>(p.ZZZ, PPP);
    return r;
}

// P + Q with Q affine (madd-2008-s), all exceptional cases handled.
ZK_DEV Xyzz xyzz_add_affine(const Xyzz &p, const Affine &q) {
    if (xyzz_is_inf(p)) return xyzz_from_affine(q);
    Fq U2 = fe_mul<FqP>(q.x, p.ZZ);
    Fq S2 = fe_mul<FqP>(q.y, p.ZZZ);
    Fq P = fe_sub<FqP>(U2, p.X);
    Fq R = fe_sub<FqP>(S2, p.Y);
    if (fe_is_zero<FqP>(P)) {
        if (fe_is_zero<FqP>(R)) return xyzz_dbl_affine(q);  // P = Q
        return xyzz_inf();                                   // P = -Q
    }
    return madd_finish(p, P, R);
}

// ---------------------------------------------------------------------------
// Window-table entries.  The bucket accumulation's mixed additions multiply
// two accumulator coordinates by the table point's x and y, which are fixed
// when the table is built.  An entry therefore holds them canonical with
// their precomputed quotients (fe_mul_shoup): x ZZ1 with ZZ1 in Montgomery
// form (ZZ1 R) is x ZZ1 R, the Montgomery form of U2, in 207 word products
// instead of a Montgomery product's 264 (S2 likewise).  128 bytes, one
// aligned line per entry; a 64-byte affine point cost the same 128-byte
// fetch from DRAM.
// ---------------------------------------------------------------------------

struct AffineS {
    Fq x, y;    // canonical coordinates
    Fq xq, yq;  // floor(x 2^256 / q), floor(y 2^256 / q)
};

// The entry of an affine point in Montgomery form; the quotients come from
// the Montgomery forms directly (fe_shoup_quotient_mont).
ZK_DEV AffineS affines_from_affine(const Affine &a) {
    AffineS e;
    e.x = fe_from_mont<FqP>(a.x);
    e.y = fe_from_mont<FqP>(a.y);
    e.xq = fe_shoup_quotient_mont<FqP>(a.x);
    e.yq = fe_shoup_quotient_mont<FqP>(a.y);
    return e;
}

// One out-of-line copy of the product (the accumulation kernel's code stays
// within the instruction cache, as for the F_q Montgomery product).
static __device__ __noinline__ Fq fq_mul_shoup_call(const Fq a, const Fq w, const Fq wq) {
    return fe_mul_shoup<FqP>(a, w, wq);
}

// The entry's point, negated when neg, in affine Montgomery form: the
// product of the constant R mod q with x is x R.
ZK_DEV Affine affines_point(const AffineS &e, bool neg) {
    Fq one;
#pragma unroll
    for (int i = 0; i < 8; i++) one.v[i] = FqP::one(i);  // R mod q as a plain residue
    Affine a;
    a.x = fq_mul_shoup_call(one, e.x, e.xq);
    a.y = fq_mul_shoup_call(one, e.y, e.yq);
    if (neg) a.y = fe_neg<FqP>(a.y);
    return a;
}

// The entry's point (negated when neg) as an XYZZ point without a full
// product: any lambda != 0 gives the same point (lambda^2 x, lambda^3 y,
// lambda^2, lambda^3), and lambda = 2^-128 makes the Montgomery words of
// X and ZZ the stored x and the integer 1, ZZZ's the constant 2^-128 mod q,
// and Y's y 2^-128 (four word reduction rounds).  An accumulator that starts
// a bucket takes this, so the lanes of a warp that start one hold the others
// up by 68 word products, not two full products.
ZK_DEV Xyzz xyzz_from_entry(const AffineS &e, bool neg) {
    Xyzz r;
    r.X = e.x;
    r.Y = fe_mul_2m128<FqP>(e.y);
    if (neg) r.Y = fe_neg<FqP>(r.Y);
    r.ZZ = fe_zero<FqP>();
    r.ZZ.v[0] = 1;
#pragma unroll
    for (int i = 0; i < 8; i++) r.ZZZ.v[i] = FqP::rinvh(i);
    return r;
}

// P + Q, Q = +-(the entry's point) (neg selects -), madd-2008-s with every
// exceptional case: -Q has S2 = -(y ZZZ1).
ZK_DEV Xyzz xyzz_add_entry(const Xyzz &p, const AffineS &q, bool neg) {
    if (xyzz_is_inf(p)) return xyzz_from_entry(q, neg);
    Fq U2 = fq_mul_shoup_call(p.ZZ, q.x, q.xq);
    Fq S2 = fq_mul_shoup_call(p.ZZZ, q.y, q.yq);
    if (neg) S2 = fe_neg<FqP>(S2);
    Fq P = fe_sub<FqP>(U2, p.X);
    Fq R = fe_sub<FqP>(S2, p.Y);
    if (fe_is_zero<FqP>(P)) {
        if (fe_is_zero<FqP>(R)) return xyzz_dbl_affine(affines_point(q, neg));  // P = Q
        return xyzz_inf();                                                     // P = -Q
    }
    return madd_finish(p, P, R);
}

// P + Q, both XYZZ (add-2008-s), all exceptional cases handled.
ZK_DEV Xyzz xyzz_add(const Xyzz &p, const Xyzz &q) {
    if (xyzz_is_inf(p)) return q;
    if (xyzz_is_inf(q)) return p;
    Fq U1 = fe_mul<FqP>(p.X, q.ZZ);
    Fq U2 = fe_mul<FqP>(q.X, p.ZZ);
    Fq S1 = fe_mul<FqP>(p.Y, q.ZZZ);
    Fq S2 = fe_mul<FqP>(q.Y, p.ZZZ);
    Fq P = fe_sub<FqP>(U2, U1);
    Fq R = fe_sub<FqP>(S2, S1);
    if (fe_is_zero<FqP>(P)) {
        if (fe_is_zero<FqP>(R)) return xyzz_dbl(p);
        return xyzz_inf();
    }
    Fq PP = fe_sqr<FqP>(P);
    Fq PPP = fe_mul<FqP>(P, PP);
    Fq Q = fe_mul<FqP>(U1, PP);
    Xyzz r;
    r.X = fe_sub<FqP>(fe_sub<FqP>(fe_sqr<FqP>(R), PPP), fe_dbl<FqP>(Q));
    r.Y = fe_mul_sub_mul<FqP>(R, fe_sub<FqP>(Q, r.X), S1, PPP);
    r.ZZ = fe_mul<FqP>(fe_mul<FqP>(p.ZZ, q.ZZ), PP);
    r.ZZZ = fe_mul<FqP>(fe_mul<FqP>(p.ZZZ, q.ZZZ), PPP);
    return r;
}

// XYZZ -> affine (Montgomery form).  Infinity maps to (0, 0).
ZK_DEV Affine xyzz_to_affine(const Xyzz &p) {
    Affine a;
    if (xyzz_is_inf(p)) {
        a.x = fe_zero<FqP>();
        a.y = fe_zero<FqP>();
        return a;
    }
    Fq izzz = fe_inv<FqP>(p.ZZZ);          // Z^-3
    Fq iz = fe_mul<FqP>(p.ZZ, izzz);       // Z^-1
    Fq izz = fe_sqr<FqP>(iz);              // Z^-2
    a.x = fe_mul<FqP>(p.X, izz);
    a.y = fe_mul<FqP>(p.Y, izzz);
    return a;
}

// Curve equation for a Montgomery-form affine point.
ZK_DEV bool affine_on_curve(const Affine &a) {
    Fq y2 = fe_sqr<FqP>(a.y);
    Fq x3 = fe_mul<FqP>(fe_sqr<FqP>(a.x), a.x);
    Fq three = fe_zero<FqP>();
    three.v[0] = 3;
    three = fe_to_mont<FqP>(three);
    return fe_eq<FqP>(y2, fe_add<FqP>(x3, three));
}

// ---------------------------------------------------------------------------
// Memory forms.
//   * device base points (SRS, Lagrange basis): affine Montgomery, 64 bytes
//     (x then y);
//   * window-table entry: AffineS, 128 bytes (x, y, xq, yq, canonical);
//   * boundary form: canonical affine, 64 bytes; infinity = zeros.
// ---------------------------------------------------------------------------

ZK_DEV Affine affine_ldg(const void *p) {
    const char *c = reinterpret_cast<const char *>(p);
    Affine a;
    a.x = fe_ldg<FqP>(c);
    a.y = fe_ldg<FqP>(c + 32);
    return a;
}

ZK_DEV AffineS affines_ldg(const void *p) {
    const char *c = reinterpret_cast<const char *>(p);
    AffineS a;
    a.x = fe_ldg<FqP>(c);
    a.y = fe_ldg<FqP>(c + 32);
    a.xq = fe_ldg<FqP>(c + 64);
    a.yq = fe_ldg<FqP>(c + 96);
    return a;
}

ZK_DEV void affines_store(void *p, const AffineS &a) {
    char *c = reinterpret_cast<char *>(p);
    fe_store<FqP>(c, a.x);
    fe_store<FqP>(c + 32, a.y);
    fe_store<FqP>(c + 64, a.xq);
    fe_store<FqP>(c + 96, a.yq);
}

ZK_DEV void affine_store(void *p, const Affine &a) {
    char *c = reinterpret_cast<char *>(p);
    fe_store<FqP>(c, a.x);
    fe_store<FqP>(c + 32, a.y);
}

ZK_DEV Xyzz xyzz_load(const void *p) {
    const char *c = reinterpret_cast<const char *>(p);
    Xyzz r;
    r.X = fe_load<FqP>(c);
    r.Y = fe_load<FqP>(c + 32);
    r.ZZ = fe_load<FqP>(c + 64);
    r.ZZZ = fe_load<FqP>(c + 96);
    return r;
}

ZK_DEV void xyzz_store(void *p, const Xyzz &a) {
    char *c = reinterpret_cast<char *>(p);
    fe_store<FqP>(c, a.X);
    fe_store<FqP>(c + 32, a.Y);
    fe_store<FqP>(c + 64, a.ZZ);
    fe_store<FqP>(c + 96, a.ZZZ);
}

// XYZZ (Montgomery) -> canonical affine bytes at the boundary.
ZK_DEV void xyzz_store_canonical(void *p, const Xyzz &a) {
    Affine af = xyzz_to_affine(a);
    if (xyzz_is_inf(a)) {
        affine_store(p, af);
        return;
    }
    af.x = fe_from_mont<FqP>(af.x);
    af.y = fe_from_mont<FqP>(af.y);
    affine_store(p, af);
}

// Canonical affine bytes -> XYZZ (Montgomery); zero bytes mean infinity.
ZK_DEV Xyzz xyzz_load_canonical(const void *p) {
    const char *c = reinterpret_cast<const char *>(p);
    Affine a;
    a.x = fe_load<FqP>(c);
    a.y = fe_load<FqP>(c + 32);
    if (fe_is_zero<FqP>(a.x) && fe_is_zero<FqP>(a.y)) return xyzz_inf();
    a.x = fe_to_mont<FqP>(a.x);
    a.y = fe_to_mont<FqP>(a.y);
    return xyzz_from_affine(a);
}

// k * P for a canonical 256-bit k, MSB-first double-and-add on XYZZ.
ZK_DEV Xyzz xyzz_mul(const Xyzz &p, const uint32_t (&k)[8]) {
    Xyzz acc = xyzz_inf();
    int top = 255;
    while (top >= 0 && !((k[top >> 5] >> (top & 31)) & 1)) top--;
    for (int i = top; i >= 0; i--) {
        acc = xyzz_dbl(acc);
        if ((k[i >> 5] >> (i & 31)) & 1) acc = xyzz_add(acc, p);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// GLV (Gallant, Lambert, Vanstone, CRYPTO 2001) on BN254 G1.  The map
// phi(x, y) = (beta x, y), beta a primitive cube root of unity in F_q, is an
// endomorphism of the curve that acts as multiplication by lambda, a primitive
// cube root of unity in F_r (the pair with phi(G) = lambda G).  A scalar k
// splits as k = k1 + k2 lambda (mod r) with |k1|, |k2| < 2^130 using the short
// basis (a1, b1), (a2, b2) of the lattice {(x, y): x + y lambda = 0 (mod r)}
// (extended Euclid on r and lambda, stopped at sqrt(r)):
//   c1 = floor(k G1 / 2^256), c2 = floor(k G2 / 2^256), with
//   G1 = floor(b2 2^256 / r) and G2 = floor(-b1 2^256 / r) (each c within 2 of
//   the rounded k b2 / r and -k b1 / r),
//   k1 = k - c1 a1 - c2 a2,  k2 = -c1 b1 - c2 b2 = c1 |b1| - c2 b2  (b1 < 0).
// Then k P = k1 P + k2 phi(P): two half-length scalars share one chain of
// doublings.  (k1, k2) = e1 (a1, b1) + e2 (a2, b2) with 0 <= e1, e2 < 2 bounds
// |k1| <= 2 (|a1| + |a2|) < 2^129 and |k2| <= 2 (|b1| + |b2|) < 2^129.
// ---------------------------------------------------------------------------
struct Glv {
    static ZK_HD constexpr uint32_t beta_mont(int i) {  // beta R mod q
        constexpr uint32_t v[8] = {0xd782e155u, 0x71930c11u, 0xffbe3323u, 0xa6bb947cu,
                                   0xd4741444u, 0xaa303344u, 0x26594943u, 0x2c3b3f0du};
        return v[i];
    }
    static ZK_HD constexpr uint32_t a1(int i) {
        constexpr uint32_t v[8] = {0x94d213e3u, 0x89d32568u, 0, 0, 0, 0, 0, 0};
        return v[i];
    }
    static ZK_HD constexpr uint32_t b1_abs(int i) {  // -b1
        constexpr uint32_t v[8] = {0x7d4f1128u, 0x8211bbebu, 0xeeb859fcu, 0x6f4d8248u, 0, 0, 0, 0};
        return v[i];
    }
    static ZK_HD constexpr uint32_t a2(int i) {
        constexpr uint32_t v[8] = {0x1221250bu, 0x0be4e154u, 0xeeb859fdu, 0x6f4d8248u, 0, 0, 0, 0};
        return v[i];
    }
    static ZK_HD constexpr uint32_t b2(int i) {
        constexpr uint32_t v[8] = {0x94d213e3u, 0x89d32568u, 0, 0, 0, 0, 0, 0};
        return v[i];
    }
    static ZK_HD constexpr uint32_t g1(int i) {
        constexpr uint32_t v[8] = {0xc7e0b3d7u, 0xd91d232eu, 0x00000002u, 0, 0, 0, 0, 0};
        return v[i];
    }
    static ZK_HD constexpr uint32_t g2(int i) {
        constexpr uint32_t v[8] = {0x391eb18du, 0x7a7bd9d4u, 0xa773d2cfu, 0x4ccef014u, 0x00000002u, 0, 0, 0};
        return v[i];
    }
};

constexpr int kGlvWords = 5;  // |k1|, |k2| < 2^130 fit 160 bits

namespace detail {
// x y for 8-word operands, low 9 words (both small enough that the product
// fits: the callers' products stay below 2^288).
ZK_DEV void glv_mul9(const uint32_t (&x)[8], const uint32_t (&y)[8], uint32_t (&out)[9]) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (i + j >= 9) break;
            const uint64_t p = (uint64_t)x[i] * y[j] + t[i + j] + carry;
            t[i + j] = (uint32_t)p;
            carry = p >> 32;
        }
        if (i + 8 < 9) t[i + 8] = (uint32_t)carry;
    }
#pragma unroll
    for (int i = 0; i < 9; i++) out[i] = t[i];
}
// floor(x y / 2^256) for an 8-word x and constant y, 8 words.
ZK_DEV void glv_mulhi(const uint32_t (&x)[8], const uint32_t (&y)[8], uint32_t (&out)[8]) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint64_t p = (uint64_t)x[i] * y[j] + t[i + j] + carry;
            t[i + j] = (uint32_t)p;
            carry = p >> 32;
        }
        t[i + 8] = (uint32_t)carry;
    }
#pragma unroll
    for (int i = 0; i < 8; i++) out[i] = t[8 + i];
}
// a - b over 9 words (two's complement).
ZK_DEV void glv_sub9(uint32_t (&a)[9], const uint32_t (&b)[9]) {
    uint64_t borrow = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const uint64_t d = (uint64_t)a[i] - b[i] - borrow;
        a[i] = (uint32_t)d;
        borrow = (d >> 32) & 1;
    }
}
// Sign and magnitude (kGlvWords words) of a 9-word two's complement value.
ZK_DEV bool glv_abs(const uint32_t (&a)[9], uint32_t (&m)[kGlvWords]) {
    const bool neg = (a[8] >> 31) != 0;
    uint64_t c = 1;
#pragma unroll
    for (int i = 0; i < kGlvWords; i++) {
        if (neg) {
            const uint64_t v = (uint64_t)(~a[i]) + c;
            m[i] = (uint32_t)v;
            c = v >> 32;
        } else {
            m[i] = a[i];
        }
    }
    return neg;
}
}  // namespace detail

// k (canonical, < r) -> |k1|, |k2| (kGlvWords words each) and their signs,
// with k = k1 + k2 lambda (mod r).
ZK_DEV void glv_split(const uint32_t (&k)[8], uint32_t (&k1)[kGlvWords], bool &neg1, uint32_t (&k2)[kGlvWords],
                      bool &neg2) {
    using namespace detail;
    uint32_t g1[8], g2[8], a1[8], a2[8], b1[8], b2[8], c1[8], c2[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        g1[i] = Glv::g1(i);
        g2[i] = Glv::g2(i);
        a1[i] = Glv::a1(i);
        a2[i] = Glv::a2(i);
        b1[i] = Glv::b1_abs(i);
        b2[i] = Glv::b2(i);
    }
    glv_mulhi(k, g1, c1);  // < 2^66
    glv_mulhi(k, g2, c2);  // < 2^130
    uint32_t x[9], t[9];
    // k1 = k - c1 a1 - c2 a2
#pragma unroll
    for (int i = 0; i < 9; i++) x[i] = i < 8 ? k[i] : 0u;
    glv_mul9(c1, a1, t);
    glv_sub9(x, t);
    glv_mul9(c2, a2, t);
    glv_sub9(x, t);
    neg1 = glv_abs(x, k1);
    // k2 = c1 |b1| - c2 b2
    glv_mul9(c1, b1, x);
    glv_mul9(c2, b2, t);
    glv_sub9(x, t);
    neg2 = glv_abs(x, k2);
}

// phi(P) = (beta x, y) in XYZZ: (beta X, Y, ZZ, ZZZ).
ZK_DEV Xyzz xyzz_phi(const Xyzz &p) {
    Fq b;
#pragma unroll
    for (int i = 0; i < 8; i++) b.v[i] = Glv::beta_mont(i);
    Xyzz r = p;
    r.X = fe_mul<FqP>(p.X, b);
    return r;
}

}  // namespace zk
