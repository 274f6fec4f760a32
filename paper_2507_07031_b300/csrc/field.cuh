// field.cuh -- 254-bit prime-field arithmetic for BN254 on sm_103a.
//
// Elements are eight 32-bit little-endian limbs.  Multiplication is
// Montgomery's method (R = 2^256) in the coarsely integrated operand scanning
// order, written as PTX carry chains (mad.lo.cc / madc.hi.cc) so that every
// partial product is one IMAD on the integer pipe and carries never leave the
// carry flag.  Both moduli are below 2^254, so the running sum fits in nine
// limbs and needs no extra carry word; a final conditional subtraction returns
// a canonical value in [0, p).
//
// Moduli: q (base field of G1) and r (the group order, scalar field), the
// standard BN254 parameters (the paper's Sec. 6 fixes BN254).
#pragma once
#include <cstdint>

#define ZK_DEV __device__ __forceinline__
#define ZK_HD __host__ __device__ __forceinline__

namespace zk {

// Compile-time limb tables.  `p` is the modulus, `one` = R mod p, `r2` =
// R^2 mod p, `r3` = R^3 mod p, `half` = (p - 1) / 2, `n0` = -p^{-1} mod 2^32.
struct FqP {
    static ZK_HD constexpr uint32_t p(int i) {
        constexpr uint32_t v[8] = {0xd87cfd47u, 0x3c208c16u, 0x6871ca8du, 0x97816a91u,
                                   0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t one(int i) {
        constexpr uint32_t v[8] = {0xc58f0d9du, 0xd35d438du, 0xf5c70b3du, 0x0a78eb28u,
                                   0x7879462cu, 0x666ea36fu, 0x9a07df2fu, 0x0e0a77c1u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t r2(int i) {
        constexpr uint32_t v[8] = {0x538afa89u, 0xf32cfc5bu, 0xd44501fbu, 0xb5e71911u,
                                   0x0a417ff6u, 0x47ab1effu, 0xcab8351fu, 0x06d89f71u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t r3(int i) {
        constexpr uint32_t v[8] = {0xda1530dfu, 0xb1cd6dafu, 0xa7283db6u, 0x62f210e6u,
                                   0x0ada0afbu, 0xef7f0b0cu, 0x2d592544u, 0x20fd6e90u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t half(int i) {
        constexpr uint32_t v[8] = {0x6c3e7ea3u, 0x9e10460bu, 0xb438e546u, 0xcbc0b548u,
                                   0x40c0ac2eu, 0xdc2822dbu, 0x7098d014u, 0x18322739u};
        return v[i];
    }
    static constexpr uint32_t n0 = 0xe4866389u;
};

struct FrP {
    static ZK_HD constexpr uint32_t p(int i) {
        constexpr uint32_t v[8] = {0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u,
                                   0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t one(int i) {
        constexpr uint32_t v[8] = {0x4ffffffbu, 0xac96341cu, 0x9f60cd29u, 0x36fc7695u,
                                   0x7879462eu, 0x666ea36fu, 0x9a07df2fu, 0x0e0a77c1u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t r2(int i) {
        constexpr uint32_t v[8] = {0xae216da7u, 0x1bb8e645u, 0xe35c59e3u, 0x53fe3ab1u,
                                   0x53bb8085u, 0x8c49833du, 0x7f4e44a5u, 0x0216d0b1u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t r3(int i) {
        constexpr uint32_t v[8] = {0xb4bf0040u, 0x5e94d8e1u, 0x1cfbb6b8u, 0x2a489cbeu,
                                   0xa19fcfedu, 0x893cc664u, 0x7fcc657cu, 0x0cf8594bu};
        return v[i];
    }
    static ZK_HD constexpr uint32_t half(int i) {
        constexpr uint32_t v[8] = {0xf8000000u, 0xa1f0fac9u, 0x3cdcb848u, 0x9419f424u,
                                   0x40c0ac2eu, 0xdc2822dbu, 0x7098d014u, 0x18322739u};
        return v[i];
    }
    static constexpr uint32_t n0 = 0xefffffffu;
};

template <class P>
struct Fe {
    uint32_t v[8];
};

using Fq = Fe<FqP>;
using Fr = Fe<FrP>;

// ---------------------------------------------------------------------------
// Constants and predicates
// ---------------------------------------------------------------------------

template <class P> ZK_DEV Fe<P> fe_zero() {
    Fe<P> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = 0;
    return r;
}

template <class P> ZK_DEV Fe<P> fe_mont_one() {
    Fe<P> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = P::one(i);
    return r;
}

template <class P> ZK_DEV Fe<P> fe_r2() {
    Fe<P> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = P::r2(i);
    return r;
}

template <class P> ZK_DEV bool fe_is_zero(const Fe<P> &a) {
    uint32_t x = a.v[0];
#pragma unroll
    for (int i = 1; i < 8; i++) x |= a.v[i];
    return x == 0;
}

template <class P> ZK_DEV bool fe_eq(const Fe<P> &a, const Fe<P> &b) {
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) x |= a.v[i] ^ b.v[i];
    return x == 0;
}

// a >= p (non-canonical) test for validation of inputs.
template <class P> ZK_DEV bool fe_ge_modulus(const Fe<P> &a) {
#pragma unroll
    for (int i = 7; i >= 0; i--) {
        if (a.v[i] > P::p(i)) return true;
        if (a.v[i] < P::p(i)) return false;
    }
    return true;
}

// a > (p - 1) / 2
template <class P> ZK_DEV bool fe_gt_half(const Fe<P> &a) {
#pragma unroll
    for (int i = 7; i >= 0; i--) {
        if (a.v[i] > P::half(i)) return true;
        if (a.v[i] < P::half(i)) return false;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Addition, subtraction, negation (inputs and outputs canonical)
// ---------------------------------------------------------------------------

template <class P> ZK_DEV Fe<P> fe_add(const Fe<P> &a, const Fe<P> &b) {
    Fe<P> s, t;
    asm("add.cc.u32 %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32 %7, %15, %23;"
        : "=r"(s.v[0]), "=r"(s.v[1]), "=r"(s.v[2]), "=r"(s.v[3]), "=r"(s.v[4]), "=r"(s.v[5]),
          "=r"(s.v[6]), "=r"(s.v[7])
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
          "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
    uint32_t borrow;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;"
        : "=r"(t.v[0]), "=r"(t.v[1]), "=r"(t.v[2]), "=r"(t.v[3]), "=r"(t.v[4]), "=r"(t.v[5]),
          "=r"(t.v[6]), "=r"(t.v[7]), "=r"(borrow)
        : "r"(s.v[0]), "r"(s.v[1]), "r"(s.v[2]), "r"(s.v[3]), "r"(s.v[4]), "r"(s.v[5]),
          "r"(s.v[6]), "r"(s.v[7]), "r"(P::p(0)), "r"(P::p(1)), "r"(P::p(2)), "r"(P::p(3)),
          "r"(P::p(4)), "r"(P::p(5)), "r"(P::p(6)), "r"(P::p(7)));
    // borrow = 0xffffffff when s < p: keep s.
#pragma unroll
    for (int i = 0; i < 8; i++) t.v[i] = (s.v[i] & borrow) | (t.v[i] & ~borrow);
    return t;
}

template <class P> ZK_DEV Fe<P> fe_sub(const Fe<P> &a, const Fe<P> &b) {
    Fe<P> d, t;
    uint32_t borrow;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;"
        : "=r"(d.v[0]), "=r"(d.v[1]), "=r"(d.v[2]), "=r"(d.v[3]), "=r"(d.v[4]), "=r"(d.v[5]),
          "=r"(d.v[6]), "=r"(d.v[7]), "=r"(borrow)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
          "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
    // Add back p masked by the borrow.
    asm("add.cc.u32 %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32 %7, %15, %23;"
        : "=r"(t.v[0]), "=r"(t.v[1]), "=r"(t.v[2]), "=r"(t.v[3]), "=r"(t.v[4]), "=r"(t.v[5]),
          "=r"(t.v[6]), "=r"(t.v[7])
        : "r"(d.v[0]), "r"(d.v[1]), "r"(d.v[2]), "r"(d.v[3]), "r"(d.v[4]), "r"(d.v[5]),
          "r"(d.v[6]), "r"(d.v[7]), "r"(P::p(0) & borrow), "r"(P::p(1) & borrow),
          "r"(P::p(2) & borrow), "r"(P::p(3) & borrow), "r"(P::p(4) & borrow),
          "r"(P::p(5) & borrow), "r"(P::p(6) & borrow), "r"(P::p(7) & borrow));
    return t;
}

template <class P> ZK_DEV Fe<P> fe_neg(const Fe<P> &a) {
    return fe_sub<P>(fe_zero<P>(), a);
}

template <class P> ZK_DEV Fe<P> fe_dbl(const Fe<P> &a) { return fe_add<P>(a, a); }

// ---------------------------------------------------------------------------
// Montgomery multiplication: returns a * b * 2^-256 mod p.
// ---------------------------------------------------------------------------
//
// The accumulator is a window t[I .. I+8] of a 17-word array that slides up
// one word per outer iteration, so the "shift right by one word" of the
// textbook loop is a renaming of registers.

namespace detail {

// t[I .. I+8] += x[0..7] * y   (x < p, so the sum stays below 2^(32*9)).
template <int I>
ZK_DEV void mac_row(uint32_t (&t)[17], const uint32_t (&x)[8], uint32_t y) {
    asm("mad.lo.cc.u32  %0, %9,  %17, %0;\n\t"
        "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
        "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
        "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
        "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
        "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
        "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
        "addc.u32       %8, %8, 0;\n\t"
        "mad.hi.cc.u32  %1, %9,  %17, %1;\n\t"
        "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
        "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
        "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
        "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
        "madc.hi.u32    %8, %16, %17, %8;"
        : "+r"(t[I + 0]), "+r"(t[I + 1]), "+r"(t[I + 2]), "+r"(t[I + 3]), "+r"(t[I + 4]),
          "+r"(t[I + 5]), "+r"(t[I + 6]), "+r"(t[I + 7]), "+r"(t[I + 8])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]),
          "r"(x[7]), "r"(y));
}

template <class P, int I>
ZK_DEV void mont_row(uint32_t (&t)[17], const uint32_t (&a)[8], uint32_t bi) {
    mac_row<I>(t, a, bi);
    const uint32_t m = t[I] * P::n0;
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3),
                            P::p(4), P::p(5), P::p(6), P::p(7)};
    mac_row<I>(t, pm, m);  // t[I] becomes 0
}

}  // namespace detail

template <class P> ZK_DEV Fe<P> fe_mul_inline(const Fe<P> &a, const Fe<P> &b) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
    detail::mont_row<P, 0>(t, a.v, b.v[0]);
    detail::mont_row<P, 1>(t, a.v, b.v[1]);
    detail::mont_row<P, 2>(t, a.v, b.v[2]);
    detail::mont_row<P, 3>(t, a.v, b.v[3]);
    detail::mont_row<P, 4>(t, a.v, b.v[4]);
    detail::mont_row<P, 5>(t, a.v, b.v[5]);
    detail::mont_row<P, 6>(t, a.v, b.v[6]);
    detail::mont_row<P, 7>(t, a.v, b.v[7]);
    // t[8..15] < 2p; reduce once.
    Fe<P> s, r;
#pragma unroll
    for (int i = 0; i < 8; i++) s.v[i] = t[8 + i];
    uint32_t borrow;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]),
          "=r"(r.v[6]), "=r"(r.v[7]), "=r"(borrow)
        : "r"(s.v[0]), "r"(s.v[1]), "r"(s.v[2]), "r"(s.v[3]), "r"(s.v[4]), "r"(s.v[5]),
          "r"(s.v[6]), "r"(s.v[7]), "r"(P::p(0)), "r"(P::p(1)), "r"(P::p(2)), "r"(P::p(3)),
          "r"(P::p(4)), "r"(P::p(5)), "r"(P::p(6)), "r"(P::p(7)));
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = (s.v[i] & borrow) | (r.v[i] & ~borrow);
    return r;
}

// One out-of-line copy of the product per field: the curve formulas call it
// ten to fourteen times per point operation, and inlining every call makes
// the kernels' hot code larger than the instruction cache.
template <class P>
__device__ __noinline__ Fe<P> fe_mul_call(const Fe<P> a, const Fe<P> b) {
    return fe_mul_inline<P>(a, b);
}

template <class P> ZK_DEV Fe<P> fe_mul(const Fe<P> &a, const Fe<P> &b);

template <> ZK_DEV Fe<FqP> fe_mul<FqP>(const Fe<FqP> &a, const Fe<FqP> &b) {
#ifdef ZK_INLINE_MUL_FQ
    return fe_mul_inline<FqP>(a, b);
#else
    return fe_mul_call<FqP>(a, b);
#endif
}

template <> ZK_DEV Fe<FrP> fe_mul<FrP>(const Fe<FrP> &a, const Fe<FrP> &b) {
#ifdef ZK_NOINLINE_MUL_FR
    return fe_mul_call<FrP>(a, b);
#else
    return fe_mul_inline<FrP>(a, b);
#endif
}

template <class P> ZK_DEV Fe<P> fe_sqr(const Fe<P> &a) { return fe_mul<P>(a, a); }

// Montgomery form conversions: x -> x R and x R -> x.
template <class P> ZK_DEV Fe<P> fe_to_mont(const Fe<P> &a) { return fe_mul<P>(a, fe_r2<P>()); }

template <class P> ZK_DEV Fe<P> fe_from_mont(const Fe<P> &a) {
    Fe<P> one = fe_zero<P>();
    one.v[0] = 1;
    return fe_mul<P>(a, one);
}

// Small-constant multiples used by the curve formulas.
template <class P> ZK_DEV Fe<P> fe_mul3(const Fe<P> &a) { return fe_add<P>(fe_add<P>(a, a), a); }

// ---------------------------------------------------------------------------
// Inversion of a canonical (non-Montgomery) value by the binary extended
// Euclidean algorithm (Menezes et al., Handbook of Applied Cryptography,
// Alg. 14.61, with halving modulo p).  Variable time; the values inverted in
// this library are public (commitments, twiddle set-up).  Returns 0 for 0.
// ---------------------------------------------------------------------------

namespace detail {

ZK_DEV bool u256_is_one(const uint32_t (&a)[8]) {
    uint32_t x = a[0] ^ 1u;
#pragma unroll
    for (int i = 1; i < 8; i++) x |= a[i];
    return x == 0;
}

ZK_DEV void u256_shr1(uint32_t (&a)[8], uint32_t top) {
#pragma unroll
    for (int i = 0; i < 7; i++) a[i] = __funnelshift_r(a[i], a[i + 1], 1);
    a[7] = (a[7] >> 1) | (top << 31);
}

ZK_DEV bool u256_ge(const uint32_t (&a)[8], const uint32_t (&b)[8]) {
#pragma unroll
    for (int i = 7; i >= 0; i--) {
        if (a[i] != b[i]) return a[i] > b[i];
    }
    return true;
}

ZK_DEV uint32_t u256_add(uint32_t (&r)[8], const uint32_t (&a)[8], const uint32_t (&b)[8]) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        c += (uint64_t)a[i] + b[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    return (uint32_t)c;
}

ZK_DEV void u256_sub(uint32_t (&r)[8], const uint32_t (&a)[8], const uint32_t (&b)[8]) {
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        int64_t d = (int64_t)a[i] - b[i] - br;
        r[i] = (uint32_t)d;
        br = d < 0;
    }
}

template <class P> ZK_DEV void half_mod(uint32_t (&x)[8]) {
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
    uint32_t c = 0;
    if (x[0] & 1) c = u256_add(x, x, pm);
    u256_shr1(x, c);
}

}  // namespace detail

template <class P> ZK_DEV Fe<P> fe_inv_canonical(const Fe<P> &a) {
    using namespace detail;
    if (fe_is_zero<P>(a)) return a;
    uint32_t u[8], v[8], x1[8], x2[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        u[i] = a.v[i];
        v[i] = P::p(i);
        x1[i] = 0;
        x2[i] = 0;
    }
    x1[0] = 1;
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
    while (!u256_is_one(u) && !u256_is_one(v)) {
        while (!(u[0] & 1)) { u256_shr1(u, 0); half_mod<P>(x1); }
        while (!(v[0] & 1)) { u256_shr1(v, 0); half_mod<P>(x2); }
        if (u256_ge(u, v)) {
            u256_sub(u, u, v);
            if (!u256_ge(x1, x2)) u256_add(x1, x1, pm);
            u256_sub(x1, x1, x2);
        } else {
            u256_sub(v, v, u);
            if (!u256_ge(x2, x1)) u256_add(x2, x2, pm);
            u256_sub(x2, x2, x1);
        }
    }
    Fe<P> r;
    const bool uo = u256_is_one(u);
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = uo ? x1[i] : x2[i];
    return r;
}

// Inverse in Montgomery form: (a R)^{-1} R^3 R^{-1} = a^{-1} R.
template <class P> ZK_DEV Fe<P> fe_inv(const Fe<P> &a) {
    Fe<P> x = fe_inv_canonical<P>(a);
    Fe<P> r3;
#pragma unroll
    for (int i = 0; i < 8; i++) r3.v[i] = P::r3(i);
    return fe_mul<P>(x, r3);
}

// Exponentiation by a canonical 256-bit exponent (square-and-multiply).
template <class P> ZK_DEV Fe<P> fe_pow(const Fe<P> &a, const uint32_t (&e)[8]) {
    Fe<P> acc = fe_mont_one<P>();
    for (int i = 255; i >= 0; i--) {
        acc = fe_sqr<P>(acc);
        if ((e[i >> 5] >> (i & 31)) & 1) acc = fe_mul<P>(acc, a);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Memory helpers: 32-byte loads and stores as two 16-byte vectors.
// ---------------------------------------------------------------------------

template <class P> ZK_DEV Fe<P> fe_load(const void *p) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    uint4 a = q[0], b = q[1];
    Fe<P> r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
    r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
    return r;
}

template <class P> ZK_DEV Fe<P> fe_ldg(const void *p) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    uint4 a = __ldg(q), b = __ldg(q + 1);
    Fe<P> r;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
    r.v[4] = b.x; r.v[5] = b.y; r.v[6] = b.z; r.v[7] = b.w;
    return r;
}

template <class P> ZK_DEV void fe_store(void *p, const Fe<P> &a) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    q[0] = make_uint4(a.v[0], a.v[1], a.v[2], a.v[3]);
    q[1] = make_uint4(a.v[4], a.v[5], a.v[6], a.v[7]);
}

}  // namespace zk
