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
//   * device table entry: affine Montgomery, 64 bytes (x then y);
//   * boundary form: canonical affine, 64 bytes; infinity = zeros.
// ---------------------------------------------------------------------------

ZK_DEV Affine affine_ldg(const void *p) {
    const char *c = reinterpret_cast<const char *>(p);
    Affine a;
    a.x = fe_ldg<FqP>(c);
    a.y = fe_ldg<FqP>(c + 32);
    return a;
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

}  // namespace zk
