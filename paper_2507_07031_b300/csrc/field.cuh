// field.cuh -- 254-bit prime-field arithmetic for BN254 on sm_103a.
//
// Elements are eight 32-bit little-endian limbs.  Multiplication is
// Montgomery's method (R = 2^256), written as PTX carry chains (mad.lo.cc /
// madc.hi.cc) so that every partial product is one IMAD on the integer pipe
// and carries never leave the carry flag.  F_r products (NTT, folds) use the
// coarsely integrated operand scanning order, inline; both moduli are below
// 2^254, so its running sum fits in nine limbs and needs no extra carry word.
// F_q products (curve arithmetic) use the separated form -- a 512-bit product
// or square, then the reduction rows -- from shared out-of-line pieces, which
// also give a b - c d with one reduction.  A final conditional subtraction
// returns a canonical value in [0, p).
//
// Moduli: q (base field of G1) and r (the group order, scalar field), the
// standard BN254 parameters (the paper's Sec. 6 fixes BN254).
#pragma once
#include <cstdint>

#define ZK_DEV __device__ __forceinline__
#define ZK_HD __host__ __device__ __forceinline__

namespace zk {

// Compile-time limb tables.  `p` is the modulus, `one` = R mod p, `r2` =
// R^2 mod p, `r3` = R^3 mod p, `half` = (p - 1) / 2, `ninv` = -p^{-1} mod
// 2^256, `n0` = -p^{-1} mod 2^32 (its low word), `rinvh` = 2^-128 mod p.
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
    static ZK_HD constexpr uint32_t ninv(int i) {
        constexpr uint32_t v[8] = {0xe4866389u, 0x87d20782u, 0x1eca6ac9u, 0x9ede7d65u,
                                   0x1833da80u, 0xd8afcbd0u, 0x91888c6bu, 0xf57a22b7u};
        return v[i];
    }
    static ZK_HD constexpr uint32_t rinvh(int i) {
        constexpr uint32_t v[8] = {0x34ade680u, 0x1da790e4u, 0xf9905883u, 0x27a2f342u,
                                   0x0dfa3d61u, 0xb5ab3489u, 0x064ef9b1u, 0x1e07f71bu};
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
    static ZK_HD constexpr uint32_t ninv(int i) {
        constexpr uint32_t v[8] = {0xefffffffu, 0xc2e1f593u, 0x4c6911b3u, 0x6586864bu,
                                   0x99062391u, 0xe39a9828u, 0x0d8341b2u, 0x73f82f1du};
        return v[i];
    }
    static ZK_HD constexpr uint32_t rinvh(int i) {
        constexpr uint32_t v[8] = {0x76f9dc6fu, 0x18ee753cu, 0xa329e70fu, 0x54ad7e14u,
                                   0x4f7684dfu, 0x2b16366fu, 0x1fdf3579u, 0x133100d7u};
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

// Montgomery squaring in separated form: the 28 cross products a_i a_j
// (i < j) once, doubled, plus the 8 squares a_i^2 (72 IMADs instead of 128),
// then the 8 reduction rows t += m p 2^(32 i).  Cross-product row i adds
// a_i (a_{i+1} .. a_7) at word 2i + 1; after it the partial sum is below
// 2^(32 (i + 9)), so its chain ends at word i + 8 without a carry out.  A
// reduction row's carry out of word i + 8 is carried into the next row.
namespace detail {

template <int K>
ZK_DEV void sqr_row1(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %2, %3, %0;\n\t"
        "addc.u32       %1, %1, 0;\n\t"
        "mad.hi.u32     %1, %2, %3, %1;"
        : "+r"(t[K + 0]), "+r"(t[K + 1])
        : "r"(x[0]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row2(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %3, %5, %0;\n\t"
        "madc.lo.cc.u32 %1, %4, %5, %1;\n\t"
        "addc.u32       %2, %2, 0;\n\t"
        "mad.hi.cc.u32  %1, %3, %5, %1;\n\t"
        "madc.hi.u32    %2, %4, %5, %2;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2])
        : "r"(x[0]), "r"(x[1]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row3(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %4, %7, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %7, %2;\n\t"
        "addc.u32       %3, %3, 0;\n\t"
        "mad.hi.cc.u32  %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32    %3, %6, %7, %3;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2]), "+r"(t[K + 3])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row4(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %5, %9, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %9, %2;\n\t"
        "madc.lo.cc.u32 %3, %8, %9, %3;\n\t"
        "addc.u32       %4, %4, 0;\n\t"
        "mad.hi.cc.u32  %1, %5, %9, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %9, %3;\n\t"
        "madc.hi.u32    %4, %8, %9, %4;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2]), "+r"(t[K + 3]), "+r"(t[K + 4])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row5(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %6, %11, %0;\n\t"
        "madc.lo.cc.u32 %1, %7, %11, %1;\n\t"
        "madc.lo.cc.u32 %2, %8, %11, %2;\n\t"
        "madc.lo.cc.u32 %3, %9, %11, %3;\n\t"
        "madc.lo.cc.u32 %4, %10, %11, %4;\n\t"
        "addc.u32       %5, %5, 0;\n\t"
        "mad.hi.cc.u32  %1, %6, %11, %1;\n\t"
        "madc.hi.cc.u32 %2, %7, %11, %2;\n\t"
        "madc.hi.cc.u32 %3, %8, %11, %3;\n\t"
        "madc.hi.cc.u32 %4, %9, %11, %4;\n\t"
        "madc.hi.u32    %5, %10, %11, %5;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2]), "+r"(t[K + 3]), "+r"(t[K + 4]), "+r"(t[K + 5])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row6(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %7, %13, %0;\n\t"
        "madc.lo.cc.u32 %1, %8, %13, %1;\n\t"
        "madc.lo.cc.u32 %2, %9, %13, %2;\n\t"
        "madc.lo.cc.u32 %3, %10, %13, %3;\n\t"
        "madc.lo.cc.u32 %4, %11, %13, %4;\n\t"
        "madc.lo.cc.u32 %5, %12, %13, %5;\n\t"
        "addc.u32       %6, %6, 0;\n\t"
        "mad.hi.cc.u32  %1, %7, %13, %1;\n\t"
        "madc.hi.cc.u32 %2, %8, %13, %2;\n\t"
        "madc.hi.cc.u32 %3, %9, %13, %3;\n\t"
        "madc.hi.cc.u32 %4, %10, %13, %4;\n\t"
        "madc.hi.cc.u32 %5, %11, %13, %5;\n\t"
        "madc.hi.u32    %6, %12, %13, %6;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2]), "+r"(t[K + 3]), "+r"(t[K + 4]), "+r"(t[K + 5]), "+r"(t[K + 6])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(y));
}

template <int K>
ZK_DEV void sqr_row7(uint32_t (&t)[17], const uint32_t *x, uint32_t y) {
    asm("mad.lo.cc.u32  %0, %8, %15, %0;\n\t"
        "madc.lo.cc.u32 %1, %9, %15, %1;\n\t"
        "madc.lo.cc.u32 %2, %10, %15, %2;\n\t"
        "madc.lo.cc.u32 %3, %11, %15, %3;\n\t"
        "madc.lo.cc.u32 %4, %12, %15, %4;\n\t"
        "madc.lo.cc.u32 %5, %13, %15, %5;\n\t"
        "madc.lo.cc.u32 %6, %14, %15, %6;\n\t"
        "addc.u32       %7, %7, 0;\n\t"
        "mad.hi.cc.u32  %1, %8, %15, %1;\n\t"
        "madc.hi.cc.u32 %2, %9, %15, %2;\n\t"
        "madc.hi.cc.u32 %3, %10, %15, %3;\n\t"
        "madc.hi.cc.u32 %4, %11, %15, %4;\n\t"
        "madc.hi.cc.u32 %5, %12, %15, %5;\n\t"
        "madc.hi.cc.u32 %6, %13, %15, %6;\n\t"
        "madc.hi.u32    %7, %14, %15, %7;"
        : "+r"(t[K + 0]), "+r"(t[K + 1]), "+r"(t[K + 2]), "+r"(t[K + 3]), "+r"(t[K + 4]), "+r"(t[K + 5]), "+r"(t[K + 6]), "+r"(t[K + 7])
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(y));
}

ZK_DEV void sqr_diag(uint32_t (&t)[17], const uint32_t (&a)[8]) {
    asm("mad.lo.cc.u32  %0, %16, %16, %0;\n\t"
        "madc.hi.cc.u32 %1, %16, %16, %1;\n\t"
        "madc.lo.cc.u32 %2, %17, %17, %2;\n\t"
        "madc.hi.cc.u32 %3, %17, %17, %3;\n\t"
        "madc.lo.cc.u32 %4, %18, %18, %4;\n\t"
        "madc.hi.cc.u32 %5, %18, %18, %5;\n\t"
        "madc.lo.cc.u32 %6, %19, %19, %6;\n\t"
        "madc.hi.cc.u32 %7, %19, %19, %7;\n\t"
        "madc.lo.cc.u32 %8, %20, %20, %8;\n\t"
        "madc.hi.cc.u32 %9, %20, %20, %9;\n\t"
        "madc.lo.cc.u32 %10, %21, %21, %10;\n\t"
        "madc.hi.cc.u32 %11, %21, %21, %11;\n\t"
        "madc.lo.cc.u32 %12, %22, %22, %12;\n\t"
        "madc.hi.cc.u32 %13, %22, %22, %13;\n\t"
        "madc.lo.cc.u32 %14, %23, %23, %14;\n\t"
        "madc.hi.u32    %15, %23, %23, %15;"
        : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "+r"(t[15])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]));
}

template <int I>
ZK_DEV void sqr_red_row(uint32_t (&t)[17], uint32_t &c, const uint32_t (&pm)[8], uint32_t m) {
    asm("mad.lo.cc.u32  %0, %10, %18, %0;\n\t"
        "madc.lo.cc.u32 %1, %11, %18, %1;\n\t"
        "madc.lo.cc.u32 %2, %12, %18, %2;\n\t"
        "madc.lo.cc.u32 %3, %13, %18, %3;\n\t"
        "madc.lo.cc.u32 %4, %14, %18, %4;\n\t"
        "madc.lo.cc.u32 %5, %15, %18, %5;\n\t"
        "madc.lo.cc.u32 %6, %16, %18, %6;\n\t"
        "madc.lo.cc.u32 %7, %17, %18, %7;\n\t"
        "addc.cc.u32    %8, %8, %9;\n\t"
        "addc.u32       %9, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %10, %18, %1;\n\t"
        "madc.hi.cc.u32 %2, %11, %18, %2;\n\t"
        "madc.hi.cc.u32 %3, %12, %18, %3;\n\t"
        "madc.hi.cc.u32 %4, %13, %18, %4;\n\t"
        "madc.hi.cc.u32 %5, %14, %18, %5;\n\t"
        "madc.hi.cc.u32 %6, %15, %18, %6;\n\t"
        "madc.hi.cc.u32 %7, %16, %18, %7;\n\t"
        "madc.hi.cc.u32 %8, %17, %18, %8;\n\t"
        "addc.u32       %9, %9, 0;"
        : "+r"(t[I + 0]), "+r"(t[I + 1]), "+r"(t[I + 2]), "+r"(t[I + 3]), "+r"(t[I + 4]), "+r"(t[I + 5]), "+r"(t[I + 6]), "+r"(t[I + 7]), "+r"(t[I + 8]), "+r"(c)
        : "r"(pm[0]), "r"(pm[1]), "r"(pm[2]), "r"(pm[3]), "r"(pm[4]), "r"(pm[5]), "r"(pm[6]), "r"(pm[7]), "r"(m));
}


}  // namespace detail

// Separated Montgomery arithmetic: a 512-bit product or square, then one
// reduction.  These pieces also let the F_q routines share code (below).
namespace detail {

struct Wide {
    uint32_t w[16];
};

// a b in full (product rows only; a, b < p < 2^254).
template <class P> ZK_DEV Wide wide_mul(const Fe<P> &a, const Fe<P> &b) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
    mac_row<0>(t, a.v, b.v[0]);
    mac_row<1>(t, a.v, b.v[1]);
    mac_row<2>(t, a.v, b.v[2]);
    mac_row<3>(t, a.v, b.v[3]);
    mac_row<4>(t, a.v, b.v[4]);
    mac_row<5>(t, a.v, b.v[5]);
    mac_row<6>(t, a.v, b.v[6]);
    mac_row<7>(t, a.v, b.v[7]);
    Wide r;
#pragma unroll
    for (int i = 0; i < 16; i++) r.w[i] = t[i];
    return r;
}

// a^2 in full, separated form (cross products once, doubled, plus squares).
template <class P> ZK_DEV Wide wide_sqr(const Fe<P> &a) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
    sqr_row7<1>(t, &a.v[1], a.v[0]);
    sqr_row6<3>(t, &a.v[2], a.v[1]);
    sqr_row5<5>(t, &a.v[3], a.v[2]);
    sqr_row4<7>(t, &a.v[4], a.v[3]);
    sqr_row3<9>(t, &a.v[5], a.v[4]);
    sqr_row2<11>(t, &a.v[6], a.v[5]);
    sqr_row1<13>(t, &a.v[7], a.v[6]);
#pragma unroll
    for (int k = 15; k >= 1; k--) t[k] = __funnelshift_l(t[k - 1], t[k], 1);
    sqr_diag(t, a.v);
    Wide r;
#pragma unroll
    for (int i = 0; i < 16; i++) r.w[i] = t[i];
    return r;
}

// x - y over 512 bits, plus p 2^256 when that borrowed out (x, y < p^2):
// the same value modulo p, in [0, p 2^256).  The borrow out of the
// subtraction cancels the carry out of the addition.
template <class P> ZK_DEV Wide wide_sub_lift(const Wide &x, const Wide &y) {
    Wide t = x;
    uint32_t bw, neg;
    asm("sub.cc.u32  %0, %0, %9;\n\t"
        "subc.cc.u32 %1, %1, %10;\n\t"
        "subc.cc.u32 %2, %2, %11;\n\t"
        "subc.cc.u32 %3, %3, %12;\n\t"
        "subc.cc.u32 %4, %4, %13;\n\t"
        "subc.cc.u32 %5, %5, %14;\n\t"
        "subc.cc.u32 %6, %6, %15;\n\t"
        "subc.cc.u32 %7, %7, %16;\n\t"
        "subc.u32    %8, 0, 0;"
        : "+r"(t.w[0]), "+r"(t.w[1]), "+r"(t.w[2]), "+r"(t.w[3]), "+r"(t.w[4]), "+r"(t.w[5]), "+r"(t.w[6]),
          "+r"(t.w[7]), "=r"(bw)
        : "r"(y.w[0]), "r"(y.w[1]), "r"(y.w[2]), "r"(y.w[3]), "r"(y.w[4]), "r"(y.w[5]), "r"(y.w[6]), "r"(y.w[7]));
    asm("{\n\t.reg .u32 z;\n\t"
        "sub.cc.u32  z, 0, %17;\n\t"  // borrow flag <- (bw != 0)
        "subc.cc.u32 %0, %0, %9;\n\t"
        "subc.cc.u32 %1, %1, %10;\n\t"
        "subc.cc.u32 %2, %2, %11;\n\t"
        "subc.cc.u32 %3, %3, %12;\n\t"
        "subc.cc.u32 %4, %4, %13;\n\t"
        "subc.cc.u32 %5, %5, %14;\n\t"
        "subc.cc.u32 %6, %6, %15;\n\t"
        "subc.cc.u32 %7, %7, %16;\n\t"
        "subc.u32    %8, 0, 0;\n\t}"
        : "+r"(t.w[8]), "+r"(t.w[9]), "+r"(t.w[10]), "+r"(t.w[11]), "+r"(t.w[12]), "+r"(t.w[13]),
          "+r"(t.w[14]), "+r"(t.w[15]), "=r"(neg)
        : "r"(y.w[8]), "r"(y.w[9]), "r"(y.w[10]), "r"(y.w[11]), "r"(y.w[12]), "r"(y.w[13]), "r"(y.w[14]),
          "r"(y.w[15]), "r"(bw));
    asm("add.cc.u32  %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32    %7, %7, %15;"
        : "+r"(t.w[8]), "+r"(t.w[9]), "+r"(t.w[10]), "+r"(t.w[11]), "+r"(t.w[12]), "+r"(t.w[13]),
          "+r"(t.w[14]), "+r"(t.w[15])
        : "r"(P::p(0) & neg), "r"(P::p(1) & neg), "r"(P::p(2) & neg), "r"(P::p(3) & neg), "r"(P::p(4) & neg),
          "r"(P::p(5) & neg), "r"(P::p(6) & neg), "r"(P::p(7) & neg));
    return t;
}

// x + y over 512 bits (the caller keeps the sum below 2^512: a few products
// of values below p < 2^254).
template <class P> ZK_DEV Wide wide_add(const Wide &x, const Wide &y) {
    Wide t;
    uint32_t c;
    asm("add.cc.u32  %0, %9, %17;\n\t"
        "addc.cc.u32 %1, %10, %18;\n\t"
        "addc.cc.u32 %2, %11, %19;\n\t"
        "addc.cc.u32 %3, %12, %20;\n\t"
        "addc.cc.u32 %4, %13, %21;\n\t"
        "addc.cc.u32 %5, %14, %22;\n\t"
        "addc.cc.u32 %6, %15, %23;\n\t"
        "addc.cc.u32 %7, %16, %24;\n\t"
        "addc.u32    %8, 0, 0;"
        : "=r"(t.w[0]), "=r"(t.w[1]), "=r"(t.w[2]), "=r"(t.w[3]), "=r"(t.w[4]), "=r"(t.w[5]), "=r"(t.w[6]),
          "=r"(t.w[7]), "=r"(c)
        : "r"(x.w[0]), "r"(x.w[1]), "r"(x.w[2]), "r"(x.w[3]), "r"(x.w[4]), "r"(x.w[5]), "r"(x.w[6]), "r"(x.w[7]),
          "r"(y.w[0]), "r"(y.w[1]), "r"(y.w[2]), "r"(y.w[3]), "r"(y.w[4]), "r"(y.w[5]), "r"(y.w[6]), "r"(y.w[7]));
#pragma unroll
    for (int i = 8; i < 16; i++) t.w[i] = x.w[i];
    asm("{\n\t.reg .u32 z;\n\t"
        "add.cc.u32  z, %16, 0xffffffff;\n\t"  // carry flag <- (c != 0)
        "addc.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32    %7, %7, %15;\n\t}"
        : "+r"(t.w[8]), "+r"(t.w[9]), "+r"(t.w[10]), "+r"(t.w[11]), "+r"(t.w[12]), "+r"(t.w[13]),
          "+r"(t.w[14]), "+r"(t.w[15])
        : "r"(y.w[8]), "r"(y.w[9]), "r"(y.w[10]), "r"(y.w[11]), "r"(y.w[12]), "r"(y.w[13]), "r"(y.w[14]),
          "r"(y.w[15]), "r"(c));
    return t;
}

// Montgomery reduction of x < p 2^256: the 8 rows t += m p 2^(32 i), then
// (x + M p) / 2^256 < 2p (p < 2^254, so no carry leaves word 15) and one
// conditional subtraction.
template <class P> ZK_DEV Fe<P> redc_wide(const Wide &x) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 16; i++) t[i] = x.w[i];
    t[16] = 0;
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
    uint32_t c = 0;
    sqr_red_row<0>(t, c, pm, t[0] * P::n0);
    sqr_red_row<1>(t, c, pm, t[1] * P::n0);
    sqr_red_row<2>(t, c, pm, t[2] * P::n0);
    sqr_red_row<3>(t, c, pm, t[3] * P::n0);
    sqr_red_row<4>(t, c, pm, t[4] * P::n0);
    sqr_red_row<5>(t, c, pm, t[5] * P::n0);
    sqr_red_row<6>(t, c, pm, t[6] * P::n0);
    sqr_red_row<7>(t, c, pm, t[7] * P::n0);
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

}  // namespace detail

template <class P> ZK_DEV Fe<P> fe_sqr_inline(const Fe<P> &a) { return detail::redc_wide<P>(detail::wide_sqr<P>(a)); }

// (a b - c d) 2^-256 mod p with a single Montgomery reduction (lazy
// reduction): both products in full, their difference lifted by p 2^256
// when negative (|a b - c d| < p^2), one reduction.  Against two products
// and a subtraction this drops 8 + 64 mad.lo and 64 mad.hi.
template <class P>
ZK_DEV Fe<P> fe_mul_sub_mul_inline(const Fe<P> &a, const Fe<P> &b, const Fe<P> &c, const Fe<P> &d) {
    using namespace detail;
    return redc_wide<P>(wide_sub_lift<P>(wide_mul<P>(a, b), wide_mul<P>(c, d)));
}

// Out-of-line F_q code.  The curve formulas make ten to fourteen products
// per point operation; inlining them makes the kernels' hot code larger than
// the instruction cache.  The three F_q routines (product, squaring, product
// difference) are built from three shared out-of-line pieces: the 512-bit
// product, the 512-bit square and the reduction.
template <class P>
__device__ __noinline__ Fe<P> fe_mul_call(const Fe<P> a, const Fe<P> b) {
    return fe_mul_inline<P>(a, b);
}
static __device__ __noinline__ detail::Wide fq_wide_mul_call(const Fe<FqP> a, const Fe<FqP> b) {
    return detail::wide_mul<FqP>(a, b);
}
static __device__ __noinline__ detail::Wide fq_wide_sqr_call(const Fe<FqP> a) { return detail::wide_sqr<FqP>(a); }
static __device__ __noinline__ Fe<FqP> fq_redc_call(const detail::Wide x) { return detail::redc_wide<FqP>(x); }

template <class P> ZK_DEV Fe<P> fe_mul(const Fe<P> &a, const Fe<P> &b);

template <> ZK_DEV Fe<FqP> fe_mul<FqP>(const Fe<FqP> &a, const Fe<FqP> &b) {
#ifdef ZK_INLINE_MUL_FQ
    return fe_mul_inline<FqP>(a, b);
#else
    return fq_redc_call(fq_wide_mul_call(a, b));
#endif
}

template <> ZK_DEV Fe<FrP> fe_mul<FrP>(const Fe<FrP> &a, const Fe<FrP> &b) {
#ifdef ZK_NOINLINE_MUL_FR
    return fe_mul_call<FrP>(a, b);
#else
    return fe_mul_inline<FrP>(a, b);
#endif
}

// F_q squarings (two of the ten products of a mixed addition) take the
// separated form; F_r keeps the product (the NTT never squares).
template <class P> ZK_DEV Fe<P> fe_sqr(const Fe<P> &a) { return fe_mul<P>(a, a); }
template <> ZK_DEV Fe<FqP> fe_sqr<FqP>(const Fe<FqP> &a) { return fq_redc_call(fq_wide_sqr_call(a)); }

// a b - c d (Montgomery form in, Montgomery form out).  F_q reduces once (the
// Y coordinate of every point addition and doubling); other fields use two
// products.
template <class P> ZK_DEV Fe<P> fe_mul_sub_mul(const Fe<P> &a, const Fe<P> &b, const Fe<P> &c, const Fe<P> &d) {
    return fe_sub<P>(fe_mul<P>(a, b), fe_mul<P>(c, d));
}
template <>
ZK_DEV Fe<FqP> fe_mul_sub_mul<FqP>(const Fe<FqP> &a, const Fe<FqP> &b, const Fe<FqP> &c, const Fe<FqP> &d) {
    return fq_redc_call(detail::wide_sub_lift<FqP>(fq_wide_mul_call(a, b), fq_wide_mul_call(c, d)));
}

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
// Products by a constant with a precomputed quotient (V. Shoup's method, as
// used for NTT twiddles by D. Harvey, "Faster arithmetic for number-theoretic
// transforms", J. Symb. Comp. 2014), on 256-bit words for a modulus p with
// 3p < 2^256.  For a constant w < p and wq = floor(w 2^256 / p):
//   a w mod p = a w - q p  with  q = floor(a wq / 2^256) in {Q - 1, Q},
// Q = floor(a w / p), for every a < 2^256.  The quotient here is taken from
// the columns >= 7 of a wq only (the dropped partial products sum to below
// 2^228, so q loses at most one more unit): q in {Q - 2, Q - 1, Q}, and
// a w - q p in [0, 3p) is exact in 256 bits, so a w mod 2^256 and q p mod
// 2^256 (the lower triangles of their products) suffice.  Two conditional
// subtractions give the canonical result.  207 word products (99 of them
// high halves) against the Montgomery product's 264 (128).
// ---------------------------------------------------------------------------

namespace detail {

// Runs of partial products into a word window, each one carry chain:
//   lo_run: t[C .. C+K-1] += lo(x[XO .. XO+K-1] y); CARRY adds the carry out
//           into t[C+K], otherwise it is dropped;
//   hi_run: t[C .. C+K-1] += hi(x[XO .. XO+K-1] y), carry out dropped.
// Callers drop a carry only where it leaves the window they keep or where
// the window's bound rules it out.
template <int C, int XO, int K, bool CARRY, int N>
ZK_DEV void lo_run(uint32_t (&t)[N], const uint32_t (&x)[8], uint32_t y) {
    static_assert(K >= 1 && K <= 8 && XO + K <= 8 && C + K + (CARRY ? 1 : 0) <= N, "run out of range");
    if constexpr (K == 1 && !CARRY)
        asm("mad.lo.u32 %0, %1, %2, %0;"
            : "+r"(t[C + 0])
            : "r"(x[XO + 0]), "r"(y));
    else if constexpr (K == 1 && CARRY)
        asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\taddc.u32 %1, %1, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1])
            : "r"(x[XO + 0]), "r"(y));
    else if constexpr (K == 2 && !CARRY)
        asm("mad.lo.cc.u32 %0, %2, %4, %0;\n\tmadc.lo.u32 %1, %3, %4, %1;"
            : "+r"(t[C + 0]), "+r"(t[C + 1])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(y));
    else if constexpr (K == 2 && CARRY)
        asm("mad.lo.cc.u32 %0, %3, %5, %0;\n\tmadc.lo.cc.u32 %1, %4, %5, %1;\n\taddc.u32 %2, %2, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(y));
    else if constexpr (K == 3 && !CARRY)
        asm("mad.lo.cc.u32 %0, %3, %6, %0;\n\tmadc.lo.cc.u32 %1, %4, %6, %1;\n\tmadc.lo.u32 %2, %5, %6, %2;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(y));
    else if constexpr (K == 3 && CARRY)
        asm("mad.lo.cc.u32 %0, %4, %7, %0;\n\tmadc.lo.cc.u32 %1, %5, %7, %1;\n\tmadc.lo.cc.u32 %2, %6, %7, %2;\n\taddc.u32 %3, %3, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(y));
    else if constexpr (K == 4 && !CARRY)
        asm("mad.lo.cc.u32 %0, %4, %8, %0;\n\tmadc.lo.cc.u32 %1, %5, %8, %1;\n\tmadc.lo.cc.u32 %2, %6, %8, %2;\n\tmadc.lo.u32 %3, %7, %8, %3;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(y));
    else if constexpr (K == 4 && CARRY)
        asm("mad.lo.cc.u32 %0, %5, %9, %0;\n\tmadc.lo.cc.u32 %1, %6, %9, %1;\n\tmadc.lo.cc.u32 %2, %7, %9, %2;\n\tmadc.lo.cc.u32 %3, %8, %9, %3;\n\taddc.u32 %4, %4, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(y));
    else if constexpr (K == 5 && !CARRY)
        asm("mad.lo.cc.u32 %0, %5, %10, %0;\n\tmadc.lo.cc.u32 %1, %6, %10, %1;\n\tmadc.lo.cc.u32 %2, %7, %10, %2;\n\tmadc.lo.cc.u32 %3, %8, %10, %3;\n\tmadc.lo.u32 %4, %9, %10, %4;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(y));
    else if constexpr (K == 5 && CARRY)
        asm("mad.lo.cc.u32 %0, %6, %11, %0;\n\tmadc.lo.cc.u32 %1, %7, %11, %1;\n\tmadc.lo.cc.u32 %2, %8, %11, %2;\n\tmadc.lo.cc.u32 %3, %9, %11, %3;\n\tmadc.lo.cc.u32 %4, %10, %11, %4;\n\taddc.u32 %5, %5, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(y));
    else if constexpr (K == 6 && !CARRY)
        asm("mad.lo.cc.u32 %0, %6, %12, %0;\n\tmadc.lo.cc.u32 %1, %7, %12, %1;\n\tmadc.lo.cc.u32 %2, %8, %12, %2;\n\tmadc.lo.cc.u32 %3, %9, %12, %3;\n\tmadc.lo.cc.u32 %4, %10, %12, %4;\n\tmadc.lo.u32 %5, %11, %12, %5;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(y));
    else if constexpr (K == 6 && CARRY)
        asm("mad.lo.cc.u32 %0, %7, %13, %0;\n\tmadc.lo.cc.u32 %1, %8, %13, %1;\n\tmadc.lo.cc.u32 %2, %9, %13, %2;\n\tmadc.lo.cc.u32 %3, %10, %13, %3;\n\tmadc.lo.cc.u32 %4, %11, %13, %4;\n\tmadc.lo.cc.u32 %5, %12, %13, %5;\n\taddc.u32 %6, %6, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(y));
    else if constexpr (K == 7 && !CARRY)
        asm("mad.lo.cc.u32 %0, %7, %14, %0;\n\tmadc.lo.cc.u32 %1, %8, %14, %1;\n\tmadc.lo.cc.u32 %2, %9, %14, %2;\n\tmadc.lo.cc.u32 %3, %10, %14, %3;\n\tmadc.lo.cc.u32 %4, %11, %14, %4;\n\tmadc.lo.cc.u32 %5, %12, %14, %5;\n\tmadc.lo.u32 %6, %13, %14, %6;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(y));
    else if constexpr (K == 7 && CARRY)
        asm("mad.lo.cc.u32 %0, %8, %15, %0;\n\tmadc.lo.cc.u32 %1, %9, %15, %1;\n\tmadc.lo.cc.u32 %2, %10, %15, %2;\n\tmadc.lo.cc.u32 %3, %11, %15, %3;\n\tmadc.lo.cc.u32 %4, %12, %15, %4;\n\tmadc.lo.cc.u32 %5, %13, %15, %5;\n\tmadc.lo.cc.u32 %6, %14, %15, %6;\n\taddc.u32 %7, %7, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6]), "+r"(t[C + 7])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(y));
    else if constexpr (K == 8 && !CARRY)
        asm("mad.lo.cc.u32 %0, %8, %16, %0;\n\tmadc.lo.cc.u32 %1, %9, %16, %1;\n\tmadc.lo.cc.u32 %2, %10, %16, %2;\n\tmadc.lo.cc.u32 %3, %11, %16, %3;\n\tmadc.lo.cc.u32 %4, %12, %16, %4;\n\tmadc.lo.cc.u32 %5, %13, %16, %5;\n\tmadc.lo.cc.u32 %6, %14, %16, %6;\n\tmadc.lo.u32 %7, %15, %16, %7;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6]), "+r"(t[C + 7])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(x[XO + 7]), "r"(y));
    else if constexpr (K == 8 && CARRY)
        asm("mad.lo.cc.u32 %0, %9, %17, %0;\n\tmadc.lo.cc.u32 %1, %10, %17, %1;\n\tmadc.lo.cc.u32 %2, %11, %17, %2;\n\tmadc.lo.cc.u32 %3, %12, %17, %3;\n\tmadc.lo.cc.u32 %4, %13, %17, %4;\n\tmadc.lo.cc.u32 %5, %14, %17, %5;\n\tmadc.lo.cc.u32 %6, %15, %17, %6;\n\tmadc.lo.cc.u32 %7, %16, %17, %7;\n\taddc.u32 %8, %8, 0;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6]), "+r"(t[C + 7]), "+r"(t[C + 8])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(x[XO + 7]), "r"(y));
}

template <int C, int XO, int K, int N>
ZK_DEV void hi_run(uint32_t (&t)[N], const uint32_t (&x)[8], uint32_t y) {
    static_assert(K >= 1 && K <= 8 && XO + K <= 8 && C + K <= N, "run out of range");
    if constexpr (K == 1)
        asm("mad.hi.u32 %0, %1, %2, %0;"
            : "+r"(t[C + 0])
            : "r"(x[XO + 0]), "r"(y));
    else if constexpr (K == 2)
        asm("mad.hi.cc.u32 %0, %2, %4, %0;\n\tmadc.hi.u32 %1, %3, %4, %1;"
            : "+r"(t[C + 0]), "+r"(t[C + 1])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(y));
    else if constexpr (K == 3)
        asm("mad.hi.cc.u32 %0, %3, %6, %0;\n\tmadc.hi.cc.u32 %1, %4, %6, %1;\n\tmadc.hi.u32 %2, %5, %6, %2;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(y));
    else if constexpr (K == 4)
        asm("mad.hi.cc.u32 %0, %4, %8, %0;\n\tmadc.hi.cc.u32 %1, %5, %8, %1;\n\tmadc.hi.cc.u32 %2, %6, %8, %2;\n\tmadc.hi.u32 %3, %7, %8, %3;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(y));
    else if constexpr (K == 5)
        asm("mad.hi.cc.u32 %0, %5, %10, %0;\n\tmadc.hi.cc.u32 %1, %6, %10, %1;\n\tmadc.hi.cc.u32 %2, %7, %10, %2;\n\tmadc.hi.cc.u32 %3, %8, %10, %3;\n\tmadc.hi.u32 %4, %9, %10, %4;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(y));
    else if constexpr (K == 6)
        asm("mad.hi.cc.u32 %0, %6, %12, %0;\n\tmadc.hi.cc.u32 %1, %7, %12, %1;\n\tmadc.hi.cc.u32 %2, %8, %12, %2;\n\tmadc.hi.cc.u32 %3, %9, %12, %3;\n\tmadc.hi.cc.u32 %4, %10, %12, %4;\n\tmadc.hi.u32 %5, %11, %12, %5;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(y));
    else if constexpr (K == 7)
        asm("mad.hi.cc.u32 %0, %7, %14, %0;\n\tmadc.hi.cc.u32 %1, %8, %14, %1;\n\tmadc.hi.cc.u32 %2, %9, %14, %2;\n\tmadc.hi.cc.u32 %3, %10, %14, %3;\n\tmadc.hi.cc.u32 %4, %11, %14, %4;\n\tmadc.hi.cc.u32 %5, %12, %14, %5;\n\tmadc.hi.u32 %6, %13, %14, %6;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(y));
    else if constexpr (K == 8)
        asm("mad.hi.cc.u32 %0, %8, %16, %0;\n\tmadc.hi.cc.u32 %1, %9, %16, %1;\n\tmadc.hi.cc.u32 %2, %10, %16, %2;\n\tmadc.hi.cc.u32 %3, %11, %16, %3;\n\tmadc.hi.cc.u32 %4, %12, %16, %4;\n\tmadc.hi.cc.u32 %5, %13, %16, %5;\n\tmadc.hi.cc.u32 %6, %14, %16, %6;\n\tmadc.hi.u32 %7, %15, %16, %7;"
            : "+r"(t[C + 0]), "+r"(t[C + 1]), "+r"(t[C + 2]), "+r"(t[C + 3]), "+r"(t[C + 4]), "+r"(t[C + 5]), "+r"(t[C + 6]), "+r"(t[C + 7])
            : "r"(x[XO + 0]), "r"(x[XO + 1]), "r"(x[XO + 2]), "r"(x[XO + 3]), "r"(x[XO + 4]), "r"(x[XO + 5]), "r"(x[XO + 6]), "r"(x[XO + 7]), "r"(y));
}

// x - k (k a multiple of p) when x >= k; returns whether it subtracted.
ZK_DEV bool cond_sub_words(uint32_t (&x)[8], const uint32_t (&k)[8]) {
    uint32_t d[8], borrow;
    asm("sub.cc.u32 %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32 %8, 0, 0;"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
          "=r"(d[7]), "=r"(borrow)
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]),
          "r"(x[7]), "r"(k[0]), "r"(k[1]), "r"(k[2]), "r"(k[3]), "r"(k[4]), "r"(k[5]),
          "r"(k[6]), "r"(k[7]));
    // borrow = 0xffffffff when x < k: keep x.
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = (x[i] & borrow) | (d[i] & ~borrow);
    return borrow == 0;
}

// t[0..7] += x y mod 2^256 for row multipliers y_i = Y(i): the lower
// triangle (lo(x_j y_i) for i + j <= 7, hi(x_j y_i) for i + j <= 6).
template <int I, class Y> ZK_DEV void low_row(uint32_t (&t)[8], const uint32_t (&x)[8], Y y) {
    lo_run<I, 0, 8 - I, false>(t, x, y(I));
    if constexpr (I < 7) hi_run<I + 1, 0, 7 - I>(t, x, y(I));
}
template <class Y> ZK_DEV void low_product_add(uint32_t (&t)[8], const uint32_t (&x)[8], Y y) {
    low_row<0>(t, x, y);
    low_row<1>(t, x, y);
    low_row<2>(t, x, y);
    low_row<3>(t, x, y);
    low_row<4>(t, x, y);
    low_row<5>(t, x, y);
    low_row<6>(t, x, y);
    low_row<7>(t, x, y);
}

// Word i of 2^256 - p (p odd, so only word 0 takes the +1).
template <class P> constexpr uint32_t neg_p(int i) { return i == 0 ? 0u - P::p(0) : ~P::p(i); }

// Row i of the quotient: columns >= 7 of a_i wq, into t[7 .. i+8] (each
// partial sum a[0..i] wq / 2^224 fits in those i + 2 words).
template <int I> ZK_DEV void quot_row(uint32_t (&t)[17], const uint32_t (&wq)[8], uint32_t ai) {
    lo_run<7, 7 - I, I + 1, true>(t, wq, ai);
    if constexpr (I < 7) hi_run<7, 6 - I, I + 2>(t, wq, ai);
    else hi_run<8, 0, 8>(t, wq, ai);
}


// Words of p and 2p, and conditional subtractions of them.
template <class P> struct Multiples {
    static constexpr uint32_t p1(int i) { return P::p(i); }
    static constexpr uint32_t p2(int i) { return (P::p(i) << 1) | (i ? P::p(i - 1) >> 31 : 0u); }
};
template <class P> ZK_DEV void cond_sub_p(uint32_t (&x)[8]) {
    const uint32_t k[8] = {Multiples<P>::p1(0), Multiples<P>::p1(1), Multiples<P>::p1(2), Multiples<P>::p1(3),
                           Multiples<P>::p1(4), Multiples<P>::p1(5), Multiples<P>::p1(6), Multiples<P>::p1(7)};
    cond_sub_words(x, k);
}
template <class P> ZK_DEV void cond_sub_2p(uint32_t (&x)[8]) {
    const uint32_t k[8] = {Multiples<P>::p2(0), Multiples<P>::p2(1), Multiples<P>::p2(2), Multiples<P>::p2(3),
                           Multiples<P>::p2(4), Multiples<P>::p2(5), Multiples<P>::p2(6), Multiples<P>::p2(7)};
    cond_sub_words(x, k);
}
// x += y, carry out dropped (callers keep the sum below 2^256).
ZK_DEV void add_words(uint32_t (&x)[8], const uint32_t (&y)[8]) {
    asm("add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32 %7, %7, %15;"
        : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(x[7])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(y[7]));
}
}  // namespace detail

// a w mod p in [0, 2p) for any a < 2^256, w < p canonical and
// wq = floor(w 2^256 / p) (requires 3p < 2^256).  Plain residues (no
// Montgomery factor).
template <class P> ZK_DEV Fe<P> fe_mul_shoup_2p(const Fe<P> &a, const Fe<P> &w, const Fe<P> &wq) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = 0;
    detail::quot_row<0>(t, wq.v, a.v[0]);
    detail::quot_row<1>(t, wq.v, a.v[1]);
    detail::quot_row<2>(t, wq.v, a.v[2]);
    detail::quot_row<3>(t, wq.v, a.v[3]);
    detail::quot_row<4>(t, wq.v, a.v[4]);
    detail::quot_row<5>(t, wq.v, a.v[5]);
    detail::quot_row<6>(t, wq.v, a.v[6]);
    detail::quot_row<7>(t, wq.v, a.v[7]);
    uint32_t q[8];
#pragma unroll
    for (int i = 0; i < 8; i++) q[i] = t[8 + i];
    // a w - q p = a w + q (2^256 - p) mod 2^256, in one accumulator: the
    // quotient's product first (q dies), then a w.
    Fe<P> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = 0;
    detail::low_product_add(r.v, q, [](int i) { return detail::neg_p<P>(i); });
    detail::low_product_add(r.v, w.v, [&](int i) { return a.v[i]; });
    detail::cond_sub_2p<P>(r.v);  // [0, 3p) -> [0, 2p)
    return r;
}

// The same, canonical.
template <class P> ZK_DEV Fe<P> fe_mul_shoup(const Fe<P> &a, const Fe<P> &w, const Fe<P> &wq) {
    Fe<P> r = fe_mul_shoup_2p<P>(a, w, wq);
    detail::cond_sub_p<P>(r.v);
    return r;
}

// Values kept in [0, 2p) (requires 4p < 2^256):
//   fe_add_2p:      a + b reduced to [0, 2p);
//   fe_sub_2p_lazy: a - b + 2p in (0, 4p), a valid first operand of fe_mul_shoup_2p;
//   fe_sub_2p:      the same reduced to [0, 2p);
//   fe_canon_2p:    [0, 2p) -> canonical.
template <class P> ZK_DEV Fe<P> fe_add_2p(const Fe<P> &a, const Fe<P> &b) {
    Fe<P> s = a;
    detail::add_words(s.v, b.v);
    detail::cond_sub_2p<P>(s.v);
    return s;
}
template <class P> ZK_DEV Fe<P> fe_sub_2p_lazy(const Fe<P> &a, const Fe<P> &b) {
    Fe<P> d;
    asm("sub.cc.u32 %0, %8, %16;\n\t"
        "subc.cc.u32 %1, %9, %17;\n\t"
        "subc.cc.u32 %2, %10, %18;\n\t"
        "subc.cc.u32 %3, %11, %19;\n\t"
        "subc.cc.u32 %4, %12, %20;\n\t"
        "subc.cc.u32 %5, %13, %21;\n\t"
        "subc.cc.u32 %6, %14, %22;\n\t"
        "subc.u32 %7, %15, %23;"
        : "=r"(d.v[0]), "=r"(d.v[1]), "=r"(d.v[2]), "=r"(d.v[3]), "=r"(d.v[4]), "=r"(d.v[5]),
          "=r"(d.v[6]), "=r"(d.v[7])
        : "r"(detail::Multiples<P>::p2(0)), "r"(detail::Multiples<P>::p2(1)), "r"(detail::Multiples<P>::p2(2)),
          "r"(detail::Multiples<P>::p2(3)), "r"(detail::Multiples<P>::p2(4)), "r"(detail::Multiples<P>::p2(5)),
          "r"(detail::Multiples<P>::p2(6)), "r"(detail::Multiples<P>::p2(7)), "r"(b.v[0]), "r"(b.v[1]),
          "r"(b.v[2]), "r"(b.v[3]), "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));  // 2p - b
    detail::add_words(d.v, a.v);
    return d;
}
template <class P> ZK_DEV Fe<P> fe_sub_2p(const Fe<P> &a, const Fe<P> &b) {
    Fe<P> d = fe_sub_2p_lazy<P>(a, b);
    detail::cond_sub_2p<P>(d.v);
    return d;
}
template <class P> ZK_DEV Fe<P> fe_canon_2p(const Fe<P> &a) {
    Fe<P> r = a;
    detail::cond_sub_p<P>(r.v);
    return r;
}

// a 2^-128 mod p for a < 2^256: four word-level Montgomery reduction rounds
// (68 word products) give t = (a + m p) / 2^128 < 2p, then one conditional
// subtraction.
template <class P> ZK_DEV Fe<P> fe_mul_2m128(const Fe<P> &a) {
    uint32_t t[17];
#pragma unroll
    for (int i = 0; i < 17; i++) t[i] = i < 8 ? a.v[i] : 0u;
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
    detail::mac_row<0>(t, pm, t[0] * P::n0);  // t[0] becomes 0
    detail::mac_row<1>(t, pm, t[1] * P::n0);
    detail::mac_row<2>(t, pm, t[2] * P::n0);
    detail::mac_row<3>(t, pm, t[3] * P::n0);
    Fe<P> r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = t[4 + i];
    detail::cond_sub_p<P>(r.v);
    return r;
}

// floor(w 2^256 / p) from w's Montgomery form m = w 2^256 mod p (w < p):
// w 2^256 - m is an exact multiple of p, so the quotient is
// (w 2^256 - m) p^-1 = -m p^-1 mod 2^256 (it is below 2^256 as w < p), one
// lower-triangle product with the constant -p^-1 mod 2^256.
template <class P> ZK_DEV Fe<P> fe_shoup_quotient_mont(const Fe<P> &m) {
    Fe<P> q;
#pragma unroll
    for (int i = 0; i < 8; i++) q.v[i] = 0;
    detail::low_product_add(q.v, m.v, [](int i) { return P::ninv(i); });
    return q;
}

// The same from the canonical w.
template <class P> ZK_DEV Fe<P> fe_shoup_quotient(const Fe<P> &w) {
    return fe_shoup_quotient_mont<P>(fe_to_mont<P>(w));
}

// ---------------------------------------------------------------------------
// Inversion of a canonical (non-Montgomery) value by Bernstein-Yang divsteps
// (D. J. Bernstein, B.-Y. Yang, "Fast constant-time gcd computation and
// modular inversion", TCHES 2019), run in variable time: the values inverted
// in this library are public (commitments, twiddle set-up).  Returns 0 for 0.
//
// With f = p, g = x, a divstep maps (delta, f, g), f odd, to
//     (1 - delta, g, (g - f) / 2)   if delta > 0 and g is odd,
//     (1 + delta, f, (g + f) / 2)   if delta <= 0 and g is odd,
//     (1 + delta, f, g / 2)         if g is even,
// and g reaches 0 with f = +-gcd = +-1 after ~526 steps for 254-bit p
// (at most 742 by the paper's bound).  The choices of 30 consecutive steps
// depend only on the low 30 bits of f and g, so they are made on one word
// and gathered into a matrix T with 2^30 [f', g'] = T [f, g] (entries of
// absolute row sum <= 2^30), which is then applied once to the full values
// and to d, e with f = d x, g = e x (mod p): [d', e'] = T [d, e] / 2^30 mod p.
// At the end x^-1 = +-d.  A batch costs ~30 word operations plus four short
// multi-word products, so one inversion is ~18 batches instead of ~750
// multi-word shift/subtract steps of the binary extended Euclid.
// ---------------------------------------------------------------------------

namespace detail {

constexpr int kDivBatch = 30;
constexpr int kDivMaxBatches = 26;  // 780 > 742 divsteps

// 288-bit two's complement integer, little-endian words.
struct S288 {
    uint32_t w[9];
};

// Thirty divsteps on the low words of f and g; returns the new delta and T.
// Branch-free (masks and selects), so the lanes of a warp never diverge:
// with odd = g mod 2 and swap = odd and delta > 0,
//   f' = swap ? g : f,   g' = (g + (odd ? (swap ? -f : f) : 0)) / 2,
//   delta' = 1 + (swap ? -delta : delta),
//   (u, v) <- 2 (swap ? (q, r) : (u, v)),
//   (q, r) <- (q, r) + (odd ? (swap ? -(u, v) : (u, v)) : 0).
ZK_HD int divsteps30(int delta, uint32_t f, uint32_t g, int32_t &u, int32_t &v, int32_t &q, int32_t &r) {
    uint32_t uu = 1, vv = 0, qq = 0, rr = 1;  // two's complement
    uint32_t d = (uint32_t)delta;
    for (int i = 0; i < kDivBatch; i++) {
        const uint32_t odd = g & 1u;
        const uint32_t m_odd = 0u - odd;
        const uint32_t m_sw = 0u - (odd & (uint32_t)((int32_t)d > 0));
        const uint32_t nf = f ^ ((f ^ g) & m_sw);
        g = (g + (((f ^ m_sw) - m_sw) & m_odd)) >> 1;
        f = nf;
        d = 1u + ((d ^ m_sw) - m_sw);
        const uint32_t nu = uu ^ ((uu ^ qq) & m_sw);
        const uint32_t nv = vv ^ ((vv ^ rr) & m_sw);
        qq += ((uu ^ m_sw) - m_sw) & m_odd;
        rr += ((vv ^ m_sw) - m_sw) & m_odd;
        uu = nu << 1;
        vv = nv << 1;
    }
    u = (int32_t)uu;
    v = (int32_t)vv;
    q = (int32_t)qq;
    r = (int32_t)rr;
    return (int)d;
}

// (ca a + cb b) / 2^30 for |ca| + |cb| <= 2^30 (exact division).
ZK_HD S288 lin_shr30(const S288 &a, const S288 &b, int32_t ca, int32_t cb) {
    uint32_t t[9];
    int64_t acc = 0;
    for (int i = 0; i < 9; i++) {
        const int64_t ai = i == 8 ? (int64_t)(int32_t)a.w[i] : (int64_t)a.w[i];
        const int64_t bi = i == 8 ? (int64_t)(int32_t)b.w[i] : (int64_t)b.w[i];
        acc += ai * ca + bi * cb;  // |.| < 2^62 + 2^32
        t[i] = (uint32_t)acc;
        acc >>= 32;  // arithmetic
    }
    S288 r;
    for (int i = 0; i < 8; i++) r.w[i] = (t[i] >> kDivBatch) | (t[i + 1] << (32 - kDivBatch));
    r.w[8] = (uint32_t)((int32_t)t[8] >> kDivBatch);
    return r;
}

// (ca d + cb e) / 2^30 mod p for d, e in [0, p), result in [0, p).
// n0 = -p^-1 mod 2^32 makes the numerator divisible by 2^30.
ZK_HD void lin_mod_shr30(const uint32_t *d, const uint32_t *e, int32_t ca, int32_t cb, const uint32_t *pm,
                         uint32_t n0, uint32_t *out) {
    uint32_t t[9];
    int64_t acc = 0;
    for (int i = 0; i < 8; i++) {
        acc += (int64_t)d[i] * ca + (int64_t)e[i] * cb;
        t[i] = (uint32_t)acc;
        acc >>= 32;
    }
    t[8] = (uint32_t)acc;  // sign word: |ca d + cb e| < 2^30 p < 2^284
    const uint32_t m = (t[0] * n0) & ((1u << kDivBatch) - 1u);
    acc = 0;
    for (int i = 0; i < 9; i++) {
        acc += (int64_t)(i == 8 ? (int64_t)(int32_t)t[i] : (int64_t)t[i]) + (i < 8 ? (int64_t)m * pm[i] : 0);
        t[i] = (uint32_t)acc;
        acc >>= 32;
    }
    // t = (ca d + cb e + m p), divisible by 2^30, in (-2^30 p, 2^31 p): the
    // quotient lies in (-p, 2p).
    uint32_t x[9];
    for (int i = 0; i < 8; i++) x[i] = (t[i] >> kDivBatch) | (t[i + 1] << (32 - kDivBatch));
    x[8] = (uint32_t)((int32_t)t[8] >> kDivBatch);
    if ((int32_t)x[8] < 0) {  // add p
        uint64_t c = 0;
        for (int i = 0; i < 8; i++) {
            c += (uint64_t)x[i] + pm[i];
            x[i] = (uint32_t)c;
            c >>= 32;
        }
        x[8] += (uint32_t)c;
    }
    // subtract p while x >= p (at most once)
    bool ge = x[8] != 0;
    if (!ge) {
        ge = true;
        for (int i = 7; i >= 0; i--)
            if (x[i] != pm[i]) {
                ge = x[i] > pm[i];
                break;
            }
    }
    if (ge) {
        int64_t br = 0;
        for (int i = 0; i < 8; i++) {
            const int64_t dd = (int64_t)x[i] - pm[i] - br;
            x[i] = (uint32_t)dd;
            br = dd < 0;
        }
    }
    for (int i = 0; i < 8; i++) out[i] = x[i];
}

// x^-1 mod p for canonical x (0 for 0); pm = p (odd), n0 = -p^-1 mod 2^32.
ZK_HD void inv_divsteps(const uint32_t *x, const uint32_t *pm, uint32_t n0, uint32_t *out) {
    S288 f, g;
    uint32_t d[8], e[8];
    bool zero = true;
    for (int i = 0; i < 8; i++) {
        f.w[i] = pm[i];
        g.w[i] = x[i];
        zero = zero && x[i] == 0;
        d[i] = 0;
        e[i] = 0;
    }
    f.w[8] = g.w[8] = 0;
    e[0] = 1;
    int delta = 1;
    for (int it = 0; it < kDivMaxBatches && !zero; it++) {
        bool gz = true;
        for (int i = 0; i < 9; i++) gz = gz && g.w[i] == 0;
        if (gz) break;
        int32_t u, v, q, r;
        delta = divsteps30(delta, f.w[0], g.w[0], u, v, q, r);
        const S288 nf = lin_shr30(f, g, u, v);
        const S288 ng = lin_shr30(f, g, q, r);
        f = nf;
        g = ng;
        uint32_t nd[8], ne[8];
        lin_mod_shr30(d, e, u, v, pm, n0, nd);
        lin_mod_shr30(d, e, q, r, pm, n0, ne);
        for (int i = 0; i < 8; i++) {
            d[i] = nd[i];
            e[i] = ne[i];
        }
    }
    // f = -1: x^-1 = p - d
    const bool neg = (int32_t)f.w[8] < 0;
    bool dz = true;
    for (int i = 0; i < 8; i++) dz = dz && d[i] == 0;
    if (neg && !dz) {
        int64_t br = 0;
        for (int i = 0; i < 8; i++) {
            const int64_t dd = (int64_t)pm[i] - d[i] - br;
            d[i] = (uint32_t)dd;
            br = dd < 0;
        }
    }
    for (int i = 0; i < 8; i++) out[i] = zero ? 0u : d[i];
}

}  // namespace detail

template <class P> ZK_DEV Fe<P> fe_inv_canonical(const Fe<P> &a) {
    const uint32_t pm[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
    Fe<P> r;
    detail::inv_divsteps(a.v, pm, P::n0, r.v);
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
