/*
 * zk_oracle.c -- plain, slow CPU oracle for the BN254 prover hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, each written as its plain definition:
 *   - F_q / F_r arithmetic on 256-bit integers held as eight 32-bit words:
 *     schoolbook 512-bit products reduced by long division (Knuth, TAOCP
 *     vol. 2, Sec. 4.3.1, Algorithm D); inverses by the binary extended
 *     Euclidean algorithm (Menezes et al., Handbook of Applied Cryptography,
 *     Alg. 14.61, in its modular-halving form).
 *   - BN254 G1 (y^2 = x^3 + 3 over F_q, generator (1, 2); the paper's Sec. 6
 *     names only "BN254", the constants are the standard ones of EIP-196) in
 *     affine coordinates with explicit infinity / P = Q / P = -Q branches;
 *     scalar multiplication by MSB-first double-and-add.
 *   - KZG commitment com = [f(tau)]_1 (Sec. 2.1): as the multi-scalar
 *     multiplication sum_i c_i [tau^i]_1 over the SRS, and as the closed form
 *     (sum_i c_i tau^i) G when tau is known.  For a vector of evaluations over
 *     H = <omega> (Sec. 4.4, "f|_H"), the polynomial is its interpolant and
 *     f(tau) = sum_k v_k L_k(tau), L_k(tau) = omega^k (tau^n - 1) / (n (tau - omega^k)).
 *   - The NTT over F_r as the O(n^2) DFT  NTT(c)_k = sum_j c_j omega^{jk},
 *     INTT(v)_j = n^{-1} sum_k v_k omega^{-jk},  omega_n = 5^{(r-1)/n}; and, for
 *     checks at sizes where the DFT is out of reach, the geometric-series
 *     fingerprint sum_k z^k NTT(c)_k = sum_j c_j (z^n - 1)/(z omega^j - 1)
 *     beside Horner evaluation.
 *   - KZG opening (Sec. 2.1): y = f(x) and the quotient (f - y) / (X - x) by
 *     synthetic division; batch opening at one point with the gamma-weighted
 *     combination sum_i gamma^i f_i.
 *   - The hiding commitment [f(tau)]_1 + s H (Sec. 4.2).
 *   - The Mul / MatMul quotient (Sec. 4.4.1) t = (A B - L) / (X^n - 1) by
 *     schoolbook multiplication and long division.
 *   - One generalised-Mira fold (Sec. 4.2, prover steps 2-7, degree d = 2) for
 *     the relation m1 o m2 - mu m3 = e over H, and the binary fold tree
 *     ("Merkle tree reduction", Sec. 4.2) as sequential loops.
 *
 * Layouts: a field element is 4 little-endian uint64 limbs (32 bytes,
 * canonical); a G1 point is x limbs then y limbs (64 bytes, canonical affine);
 * infinity is 64 zero bytes (never on the curve since 0 != 3).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { uint32_t w[8]; } u256;

/* q: BN254 base field modulus; r: BN254 group order (scalar field). */
static const u256 MODQ = {{0xd87cfd47u, 0x3c208c16u, 0x6871ca8du, 0x97816a91u,
                           0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u}};
static const u256 MODR = {{0xf0000001u, 0x43e1f593u, 0x79b97091u, 0x2833e848u,
                           0x8181585du, 0xb85045b6u, 0xe131a029u, 0x30644e72u}};

static const u256 *modulus(int f) { return f == 0 ? &MODQ : &MODR; }

/* ------------------------------------------------------------------ */
/* 256-bit integers                                                    */
/* ------------------------------------------------------------------ */

static void load(u256 *a, const uint64_t *src) {
    for (int i = 0; i < 4; i++) {
        a->w[2 * i] = (uint32_t)src[i];
        a->w[2 * i + 1] = (uint32_t)(src[i] >> 32);
    }
}

static void store(uint64_t *dst, const u256 *a) {
    for (int i = 0; i < 4; i++)
        dst[i] = (uint64_t)a->w[2 * i] | ((uint64_t)a->w[2 * i + 1] << 32);
}

static void set_small(u256 *a, uint32_t v) {
    memset(a, 0, sizeof *a);
    a->w[0] = v;
}

static int is_zero(const u256 *a) {
    for (int i = 0; i < 8; i++)
        if (a->w[i]) return 0;
    return 1;
}

static int cmp(const u256 *a, const u256 *b) {
    for (int i = 7; i >= 0; i--) {
        if (a->w[i] < b->w[i]) return -1;
        if (a->w[i] > b->w[i]) return 1;
    }
    return 0;
}

static uint32_t add_raw(u256 *r, const u256 *a, const u256 *b) {
    uint64_t c = 0;
    for (int i = 0; i < 8; i++) {
        c += (uint64_t)a->w[i] + b->w[i];
        r->w[i] = (uint32_t)c;
        c >>= 32;
    }
    return (uint32_t)c;
}

static uint32_t sub_raw(u256 *r, const u256 *a, const u256 *b) {
    int64_t br = 0;
    for (int i = 0; i < 8; i++) {
        int64_t t = (int64_t)a->w[i] - b->w[i] - br;
        br = t < 0;
        r->w[i] = (uint32_t)t;
    }
    return (uint32_t)br;
}

static void shr1(u256 *a, uint32_t top) {
    for (int i = 0; i < 7; i++) a->w[i] = (a->w[i] >> 1) | (a->w[i + 1] << 31);
    a->w[7] = (a->w[7] >> 1) | (top << 31);
}

static int bit(const u256 *a, int i) { return (a->w[i >> 5] >> (i & 31)) & 1; }

/* ------------------------------------------------------------------ */
/* Modular arithmetic (operands canonical: 0 <= a, b < m)              */
/* ------------------------------------------------------------------ */

static void fadd(u256 *r, const u256 *a, const u256 *b, const u256 *m) {
    uint32_t c = add_raw(r, a, b);
    if (c || cmp(r, m) >= 0) sub_raw(r, r, m);
}

static void fsub(u256 *r, const u256 *a, const u256 *b, const u256 *m) {
    if (sub_raw(r, a, b)) add_raw(r, r, m);
}

static void fneg(u256 *r, const u256 *a, const u256 *m) {
    if (is_zero(a)) set_small(r, 0);
    else sub_raw(r, m, a);
}

/* Remainder of the 512-bit u (16 words, little endian) modulo the 8-word m,
 * by long division in base 2^32 (Knuth's Algorithm D; the quotient digits are
 * computed and discarded). */
static void mod512(u256 *rem, const uint32_t u[16], const u256 *m) {
    enum { N = 8, M = 8 };
    int s = __builtin_clz(m->w[N - 1]);
    uint32_t vn[N], un[M + N + 1];
    for (int i = N - 1; i > 0; i--)
        vn[i] = (m->w[i] << s) | (s ? m->w[i - 1] >> (32 - s) : 0);
    vn[0] = m->w[0] << s;
    un[M + N] = s ? u[M + N - 1] >> (32 - s) : 0;
    for (int i = M + N - 1; i > 0; i--)
        un[i] = (u[i] << s) | (s ? u[i - 1] >> (32 - s) : 0);
    un[0] = u[0] << s;

    for (int j = M; j >= 0; j--) {
        uint64_t num = ((uint64_t)un[j + N] << 32) | un[j + N - 1];
        uint64_t qhat = num / vn[N - 1];
        uint64_t rhat = num % vn[N - 1];
        while (qhat > 0xFFFFFFFFull ||
               qhat * vn[N - 2] > ((rhat << 32) | un[j + N - 2])) {
            qhat--;
            rhat += vn[N - 1];
            if (rhat > 0xFFFFFFFFull) break;
        }
        /* un[j .. j+N] -= qhat * vn */
        int64_t k = 0, t;
        for (int i = 0; i < N; i++) {
            uint64_t p = qhat * vn[i];
            t = (int64_t)un[i + j] - k - (int64_t)(p & 0xFFFFFFFFull);
            un[i + j] = (uint32_t)t;
            k = (int64_t)(p >> 32) - (t >> 32);
        }
        t = (int64_t)un[j + N] - k;
        un[j + N] = (uint32_t)t;
        if (t < 0) { /* qhat was one too large: add the divisor back */
            uint64_t c = 0;
            for (int i = 0; i < N; i++) {
                c += (uint64_t)un[i + j] + vn[i];
                un[i + j] = (uint32_t)c;
                c >>= 32;
            }
            un[j + N] += (uint32_t)c;
        }
    }
    /* remainder = un[0 .. N-1] >> s */
    for (int i = 0; i < N - 1; i++)
        rem->w[i] = (un[i] >> s) | (s ? un[i + 1] << (32 - s) : 0);
    rem->w[N - 1] = (un[N - 1] >> s) | (s ? un[N] << (32 - s) : 0);
}

static void fmul(u256 *r, const u256 *a, const u256 *b, const u256 *m) {
    uint32_t prod[16] = {0};
    for (int i = 0; i < 8; i++) {
        uint64_t c = 0;
        for (int j = 0; j < 8; j++) {
            c += (uint64_t)a->w[i] * b->w[j] + prod[i + j];
            prod[i + j] = (uint32_t)c;
            c >>= 32;
        }
        prod[i + 8] = (uint32_t)c;
    }
    mod512(r, prod, m);
}

/* Halve modulo an odd m: x/2 if x is even, else (x + m)/2. */
static void fhalf(u256 *x, const u256 *m) {
    if (x->w[0] & 1) {
        uint32_t c = add_raw(x, x, m);
        shr1(x, c);
    } else {
        shr1(x, 0);
    }
}

/* Inverse of a != 0 modulo the odd prime m by the binary extended Euclidean
 * algorithm.  Invariants: x1 * a = u and x2 * a = v (mod m).  a = 0 has no
 * inverse and returns 0 (the loop would never end on it). */
static void finv(u256 *r, const u256 *a, const u256 *m) {
    u256 u = *a, v = *m, x1, x2, one;
    if (is_zero(&u)) { *r = u; return; }  /* 0 has no inverse: 0 by convention */
    set_small(&x1, 1);
    set_small(&x2, 0);
    set_small(&one, 1);
    while (cmp(&u, &one) != 0 && cmp(&v, &one) != 0) {
        while (!(u.w[0] & 1)) { shr1(&u, 0); fhalf(&x1, m); }
        while (!(v.w[0] & 1)) { shr1(&v, 0); fhalf(&x2, m); }
        if (cmp(&u, &v) >= 0) { sub_raw(&u, &u, &v); fsub(&x1, &x1, &x2, m); }
        else                  { sub_raw(&v, &v, &u); fsub(&x2, &x2, &x1, m); }
    }
    *r = cmp(&u, &one) == 0 ? x1 : x2;
}

/* a^e mod m, square-and-multiply over the 256 bits of e, MSB first. */
static void fpow(u256 *r, const u256 *a, const u256 *e, const u256 *m) {
    u256 acc;
    set_small(&acc, 1);
    for (int i = 255; i >= 0; i--) {
        fmul(&acc, &acc, &acc, m);
        if (bit(e, i)) fmul(&acc, &acc, a, m);
    }
    *r = acc;
}

/* ------------------------------------------------------------------ */
/* G1: y^2 = x^3 + 3 over F_q, affine coordinates                      */
/* ------------------------------------------------------------------ */

typedef struct { u256 x, y; int inf; } pt;

static void pt_load(pt *p, const uint64_t *src) {
    load(&p->x, src);
    load(&p->y, src + 4);
    p->inf = is_zero(&p->x) && is_zero(&p->y);
}

static void pt_store(uint64_t *dst, const pt *p) {
    if (p->inf) { memset(dst, 0, 64); return; }
    store(dst, &p->x);
    store(dst + 4, &p->y);
}

static void pt_set_inf(pt *p) { memset(p, 0, sizeof *p); p->inf = 1; }

static void pt_generator(pt *p) {
    set_small(&p->x, 1);
    set_small(&p->y, 2);
    p->inf = 0;
}

static int pt_on_curve(const pt *p) {
    if (p->inf) return 1;
    if (cmp(&p->x, &MODQ) >= 0 || cmp(&p->y, &MODQ) >= 0) return 0;
    u256 lhs, rhs, three;
    fmul(&lhs, &p->y, &p->y, &MODQ);
    fmul(&rhs, &p->x, &p->x, &MODQ);
    fmul(&rhs, &rhs, &p->x, &MODQ);
    set_small(&three, 3);
    fadd(&rhs, &rhs, &three, &MODQ);
    return cmp(&lhs, &rhs) == 0;
}

static void pt_neg(pt *r, const pt *p) {
    *r = *p;
    if (!p->inf) fneg(&r->y, &p->y, &MODQ);
}

static void pt_dbl(pt *r, const pt *p) {
    if (p->inf || is_zero(&p->y)) { pt_set_inf(r); return; }
    /* lambda = 3 x^2 / (2 y); x3 = lambda^2 - 2x; y3 = lambda (x - x3) - y */
    u256 num, den, lam, t, x3, y3, three;
    set_small(&three, 3);
    fmul(&num, &p->x, &p->x, &MODQ);
    fmul(&num, &num, &three, &MODQ);
    fadd(&den, &p->y, &p->y, &MODQ);
    finv(&den, &den, &MODQ);
    fmul(&lam, &num, &den, &MODQ);
    fmul(&x3, &lam, &lam, &MODQ);
    fsub(&x3, &x3, &p->x, &MODQ);
    fsub(&x3, &x3, &p->x, &MODQ);
    fsub(&t, &p->x, &x3, &MODQ);
    fmul(&y3, &lam, &t, &MODQ);
    fsub(&y3, &y3, &p->y, &MODQ);
    r->x = x3; r->y = y3; r->inf = 0;
}

static void pt_add(pt *r, const pt *p, const pt *q) {
    if (p->inf) { *r = *q; return; }
    if (q->inf) { *r = *p; return; }
    if (cmp(&p->x, &q->x) == 0) {
        if (cmp(&p->y, &q->y) == 0) pt_dbl(r, p);  /* P = Q */
        else pt_set_inf(r);                         /* P = -Q */
        return;
    }
    /* lambda = (y2 - y1) / (x2 - x1); x3 = lambda^2 - x1 - x2; y3 = lambda (x1 - x3) - y1 */
    u256 num, den, lam, t, x3, y3;
    fsub(&num, &q->y, &p->y, &MODQ);
    fsub(&den, &q->x, &p->x, &MODQ);
    finv(&den, &den, &MODQ);
    fmul(&lam, &num, &den, &MODQ);
    fmul(&x3, &lam, &lam, &MODQ);
    fsub(&x3, &x3, &p->x, &MODQ);
    fsub(&x3, &x3, &q->x, &MODQ);
    fsub(&t, &p->x, &x3, &MODQ);
    fmul(&y3, &lam, &t, &MODQ);
    fsub(&y3, &y3, &p->y, &MODQ);
    r->x = x3; r->y = y3; r->inf = 0;
}

/* k * P by double-and-add over the 256 bits of k, most significant first. */
static void pt_mul(pt *r, const pt *p, const u256 *k) {
    pt acc;
    pt_set_inf(&acc);
    for (int i = 255; i >= 0; i--) {
        pt_dbl(&acc, &acc);
        if (bit(k, i)) pt_add(&acc, &acc, p);
    }
    *r = acc;
}

/* ------------------------------------------------------------------ */
/* Exported: field and group primitives (f = 0: F_q, f = 1: F_r)        */
/* ------------------------------------------------------------------ */

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t > 0 ? t : 1; }

/* Degree d of the folded relation: 2 (m1 o m2 - mu m3 = e) or 3
 * (m1 o m2 o m3 - mu^2 m4 = e, the homogeneous degree-3 analogue, whose fold
 * has the two cross terms E_1, E_2 of Sec. 4.2's general-d expansion). */
static int g_degree = 2;
void orc_set_degree(int d) { g_degree = d == 3 ? 3 : 2; }
int orc_get_degree(void) { return g_degree; }
int orc_get_threads(void) { return g_threads; }
int orc_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

void orc_fadd(int f, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    u256 x, y, z; load(&x, a); load(&y, b); fadd(&z, &x, &y, modulus(f)); store(out, &z);
}
void orc_fsub(int f, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    u256 x, y, z; load(&x, a); load(&y, b); fsub(&z, &x, &y, modulus(f)); store(out, &z);
}
void orc_fmul(int f, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    u256 x, y, z; load(&x, a); load(&y, b); fmul(&z, &x, &y, modulus(f)); store(out, &z);
}
void orc_finv(int f, const uint64_t *a, uint64_t *out) {
    u256 x, z; load(&x, a); finv(&z, &x, modulus(f)); store(out, &z);
}
void orc_fpow(int f, const uint64_t *a, const uint64_t *e, uint64_t *out) {
    u256 x, y, z; load(&x, a); load(&y, e); fpow(&z, &x, &y, modulus(f)); store(out, &z);
}
/* 512-bit value (8 limbs) reduced modulo the field modulus. */
void orc_freduce512(int f, const uint64_t *a8, uint64_t *out) {
    uint32_t u[16];
    for (int i = 0; i < 8; i++) { u[2 * i] = (uint32_t)a8[i]; u[2 * i + 1] = (uint32_t)(a8[i] >> 32); }
    u256 z; mod512(&z, u, modulus(f)); store(out, &z);
}

int orc_on_curve(const uint64_t *p64) { pt p; pt_load(&p, p64); return pt_on_curve(&p); }

void orc_g1_add(const uint64_t *a, const uint64_t *b, uint64_t *out) {
    pt p, q, r; pt_load(&p, a); pt_load(&q, b); pt_add(&r, &p, &q); pt_store(out, &r);
}
void orc_g1_dbl(const uint64_t *a, uint64_t *out) {
    pt p, r; pt_load(&p, a); pt_dbl(&r, &p); pt_store(out, &r);
}
void orc_g1_neg(const uint64_t *a, uint64_t *out) {
    pt p, r; pt_load(&p, a); pt_neg(&r, &p); pt_store(out, &r);
}
void orc_g1_mul(const uint64_t *a, const uint64_t *k, uint64_t *out) {
    pt p, r; u256 kk; pt_load(&p, a); load(&kk, k); pt_mul(&r, &p, &kk); pt_store(out, &r);
}
void orc_g1_generator(uint64_t *out) { pt g; pt_generator(&g); pt_store(out, &g); }

/* Count of points that fail the curve equation or are non-canonical. */
size_t orc_count_off_curve(const uint64_t *pts, size_t n) {
    size_t bad = 0;
#pragma omp parallel for reduction(+ : bad) num_threads(g_threads) schedule(static)
    for (size_t i = 0; i < n; i++) {
        pt p; pt_load(&p, pts + 8 * i);
        if (!pt_on_curve(&p)) bad++;
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* SRS and KZG commitments (Sec. 2.1)                                  */
/* ------------------------------------------------------------------ */

/* srs[i] = [tau^i]_1 for i < n, each by its own scalar multiplication. */
void orc_srs_gen(const uint64_t *tau64, size_t n, uint64_t *out) {
    u256 tau; load(&tau, tau64);
    u256 *pw = (u256 *)malloc(sizeof(u256) * (n ? n : 1));
    set_small(&pw[0], 1);
    for (size_t i = 1; i < n; i++) fmul(&pw[i], &pw[i - 1], &tau, &MODR);
    pt g; pt_generator(&g);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 16)
    for (size_t i = 0; i < n; i++) {
        pt r; pt_mul(&r, &g, &pw[i]); pt_store(out + 8 * i, &r);
    }
    free(pw);
}

/* sum_i s_i * P_i: every term by double-and-add, terms summed in affine. */
void orc_msm(const uint64_t *pts, const uint64_t *scalars, size_t n, uint64_t *out) {
    int nt = g_threads;
    pt *part = (pt *)malloc(sizeof(pt) * nt);
    for (int t = 0; t < nt; t++) pt_set_inf(&part[t]);
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        pt acc; pt_set_inf(&acc);
#pragma omp for schedule(static)
        for (size_t i = 0; i < n; i++) {
            pt p, term; u256 s;
            pt_load(&p, pts + 8 * i);
            load(&s, scalars + 4 * i);
            pt_mul(&term, &p, &s);
            pt_add(&acc, &acc, &term);
        }
        part[t] = acc;
    }
    pt sum; pt_set_inf(&sum);
    for (int t = 0; t < nt; t++) pt_add(&sum, &sum, &part[t]);
    pt_store(out, &sum);
    free(part);
}

/* [sum_i c_i tau^i]_1: the commitment's closed form when tau is known. */
void orc_commit_coeffs_tau(const uint64_t *coeffs, size_t n, const uint64_t *tau64, uint64_t *out) {
    u256 tau, acc, c;
    load(&tau, tau64);
    set_small(&acc, 0);
    for (size_t i = n; i-- > 0;) { /* Horner */
        load(&c, coeffs + 4 * i);
        fmul(&acc, &acc, &tau, &MODR);
        fadd(&acc, &acc, &c, &MODR);
    }
    pt g, r; pt_generator(&g); pt_mul(&r, &g, &acc); pt_store(out, &r);
}

void orc_dft(const uint64_t *in, size_t n, int inverse, uint64_t *out);
void orc_msm(const uint64_t *pts, const uint64_t *scalars, size_t n, uint64_t *out);

/* KZG opening (Sec. 2.1): for f = sum_i c_i X^i (n >= 1 coefficients) and a
 * point x, y = f(x) and the quotient q(X) = (f(X) - y) / (X - x), whose n - 1
 * coefficients come from synthetic division by (X - x), highest first:
 * q_{n-2} = c_{n-1},  q_{k-1} = c_k + x q_k,  and y = c_0 + x q_0.
 * The proof is the commitment [q(tau)]_1. */
void orc_open(const uint64_t *coeffs, size_t n, const uint64_t *x64, uint64_t *y_out, uint64_t *q_out) {
    u256 x, carry, c;
    load(&x, x64);
    set_small(&carry, 0); /* the running value: q_k, then y */
    for (size_t k = n; k-- > 0;) {
        load(&c, coeffs + 4 * k);
        u256 t;
        fmul(&t, &carry, &x, &MODR);
        fadd(&carry, &t, &c, &MODR);
        if (k >= 1) store(q_out + 4 * (k - 1), &carry); /* q_{k-1} */
    }
    store(y_out, &carry);
}

/* Batch opening at one point (Sec. 2.1): y_i = f_i(x) for each polynomial and
 * h(X) = sum_i gamma^i (f_i(X) - f_i(x)) / (X - x), the quotient of the
 * combination F = sum_i gamma^i f_i (whose value at x is sum_i gamma^i y_i).
 * polys holds the coefficient vectors back to back, lens their lengths; h has
 * max(lens) - 1 coefficients. */
void orc_open_batch(const uint64_t *polys, const size_t *lens, size_t count, const uint64_t *x64,
                    const uint64_t *gamma64, uint64_t *ys_out, uint64_t *h_out) {
    size_t nmax = 0, off = 0;
    for (size_t i = 0; i < count; i++) if (lens[i] > nmax) nmax = lens[i];
    uint64_t *F = (uint64_t *)calloc(4 * (nmax ? nmax : 1), sizeof(uint64_t));
    uint64_t *qtmp = (uint64_t *)calloc(4 * (nmax ? nmax : 1), sizeof(uint64_t));
    u256 gamma, gpow;
    load(&gamma, gamma64);
    set_small(&gpow, 1); /* gamma^i */
    for (size_t i = 0; i < count; i++) {
        const uint64_t *f = polys + 4 * off;
        orc_open(f, lens[i], x64, ys_out + 4 * i, qtmp); /* y_i */
        for (size_t j = 0; j < lens[i]; j++) {            /* F += gamma^i f_i */
            u256 a, b, t;
            load(&a, F + 4 * j);
            load(&b, f + 4 * j);
            fmul(&t, &b, &gpow, &MODR);
            fadd(&a, &a, &t, &MODR);
            store(F + 4 * j, &a);
        }
        fmul(&gpow, &gpow, &gamma, &MODR);
        off += lens[i];
    }
    uint64_t yF[4];
    if (nmax) orc_open(F, nmax, x64, yF, h_out);
    free(F);
    free(qtmp);
}

/* Quotient of the Mul relation (Sec. 4.4.1; also MatMul's Q_l with l = a o b):
 * for evaluation vectors a, b over H (n = 2^k) with interpolants A, B, and L
 * the interpolant of l_i = a_i b_i, the product A B - L vanishes on H, and
 * t(X) = (A(X) B(X) - L(X)) / (X^n - 1)
 * has n - 1 coefficients.  Steps as defined: A, B, L by the inverse DFT,
 * A B by schoolbook multiplication, then long division by X^n - 1 from the
 * top coefficient down.  Returns 0, or 1 if the remainder is not zero. */
int orc_mul_quotient(const uint64_t *a, const uint64_t *b, size_t n, uint64_t *t_out) {
    uint64_t *A = (uint64_t *)malloc(32 * n), *B = (uint64_t *)malloc(32 * n), *L = (uint64_t *)malloc(32 * n);
    uint64_t *l = (uint64_t *)malloc(32 * n);
    for (size_t i = 0; i < n; i++) {
        u256 x, y, z;
        load(&x, a + 4 * i);
        load(&y, b + 4 * i);
        fmul(&z, &x, &y, &MODR);
        store(l + 4 * i, &z);
    }
    orc_dft(a, n, 1, A);
    orc_dft(b, n, 1, B);
    orc_dft(l, n, 1, L);
    /* D = A B - L, degree <= 2n - 2 */
    u256 *D = (u256 *)calloc(2 * n, sizeof(u256));
    for (size_t i = 0; i < n; i++) {
        u256 ai;
        load(&ai, A + 4 * i);
        for (size_t j = 0; j < n; j++) {
            u256 bj, p;
            load(&bj, B + 4 * j);
            fmul(&p, &ai, &bj, &MODR);
            fadd(&D[i + j], &D[i + j], &p, &MODR);
        }
    }
    for (size_t i = 0; i < n; i++) {
        u256 li;
        load(&li, L + 4 * i);
        fsub(&D[i], &D[i], &li, &MODR);
    }
    /* divide by X^n - 1: for k from the top, q_{k-n} = D_k, D_{k-n} += D_k */
    u256 *q = (u256 *)calloc(n, sizeof(u256));
    for (size_t k = 2 * n; k-- > n;) {
        q[k - n] = D[k];
        fadd(&D[k - n], &D[k - n], &D[k], &MODR);
        memset(&D[k], 0, sizeof(u256));
    }
    int bad = 0;
    for (size_t i = 0; i < n; i++) bad |= !is_zero(&D[i]);
    bad |= n >= 1 && !is_zero(&q[n - 1]);  /* degree <= n - 2 */
    for (size_t i = 0; i + 1 < n; i++) store(t_out + 4 * i, &q[i]);
    free(A); free(B); free(L); free(l); free(D); free(q);
    return bad;
}

/* Hiding commitment (the blinding of the accumulation's zero-knowledge
 * argument, Sec. 4.2): com = [f(tau)]_1 + s H for a random s and a group
 * element H, computed as the MSM over the SRS plus s H by double-and-add. */
void orc_commit_hiding(const uint64_t *srs, const uint64_t *coeffs, size_t n, const uint64_t *H64,
                       const uint64_t *s64, uint64_t *out) {
    uint64_t m[8];
    orc_msm(srs, coeffs, n, m);
    pt a, h, sh, r;
    u256 s;
    pt_load(&a, m);
    pt_load(&h, H64);
    load(&s, s64);
    pt_mul(&sh, &h, &s);
    pt_add(&r, &a, &sh);
    pt_store(out, &r);
}

/* omega_n = 5^{(r-1)/n} for n a power of two dividing 2^28. */
static void root_of_unity(u256 *w, size_t n) {
    u256 e, five, one;
    set_small(&one, 1);
    sub_raw(&e, &MODR, &one);
    size_t k = n;
    while (k > 1) { shr1(&e, 0); k >>= 1; }
    set_small(&five, 5);
    fpow(w, &five, &e, &MODR);
}

void orc_root_of_unity(size_t n, uint64_t *out) { u256 w; root_of_unity(&w, n); store(out, &w); }

/* Lagrange basis of H = <omega_n> at tau (tau not in H):
 * L_k(tau) = omega^k (tau^n - 1) / (n (tau - omega^k)). */
static void lagrange_at(u256 *L, size_t n, const u256 *tau) {
    u256 w, tn, one, nn, num;
    root_of_unity(&w, n);
    set_small(&one, 1);
    set_small(&tn, 1);
    for (size_t i = 0; i < n; i++) fmul(&tn, &tn, tau, &MODR); /* tau^n */
    fsub(&num, &tn, &one, &MODR);
    memset(&nn, 0, sizeof nn);
    nn.w[0] = (uint32_t)n;
    nn.w[1] = (uint32_t)((uint64_t)n >> 32);
    u256 *wk = (u256 *)malloc(sizeof(u256) * (n ? n : 1));
    set_small(&wk[0], 1);
    for (size_t k = 1; k < n; k++) fmul(&wk[k], &wk[k - 1], &w, &MODR);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (size_t k = 0; k < n; k++) {
        u256 den, t;
        fsub(&den, tau, &wk[k], &MODR);
        fmul(&den, &den, &nn, &MODR);
        finv(&den, &den, &MODR);
        fmul(&t, &wk[k], &num, &MODR);
        fmul(&L[k], &t, &den, &MODR);
    }
    free(wk);
}

void orc_lagrange_at(size_t n, const uint64_t *tau64, uint64_t *out) {
    u256 tau; load(&tau, tau64);
    u256 *L = (u256 *)malloc(sizeof(u256) * n);
    lagrange_at(L, n, &tau);
    for (size_t k = 0; k < n; k++) store(out + 4 * k, &L[k]);
    free(L);
}

static void dot_g(pt *r, const uint64_t *v, const u256 *L, size_t n) {
    u256 acc, x, t;
    set_small(&acc, 0);
    for (size_t k = 0; k < n; k++) {
        load(&x, v + 4 * k);
        fmul(&t, &x, &L[k], &MODR);
        fadd(&acc, &acc, &t, &MODR);
    }
    pt g; pt_generator(&g); pt_mul(r, &g, &acc);
}

/* [f(tau)]_1 for the interpolant f of the evaluations v over H. */
void orc_commit_evals_tau(const uint64_t *v, size_t n, const uint64_t *tau64, uint64_t *out) {
    u256 tau; load(&tau, tau64);
    u256 *L = (u256 *)malloc(sizeof(u256) * n);
    lagrange_at(L, n, &tau);
    pt r; dot_g(&r, v, L, n); pt_store(out, &r);
    free(L);
}

/* ------------------------------------------------------------------ */
/* NTT as the O(n^2) DFT over F_r                                      */
/* ------------------------------------------------------------------ */

static void dft_rows(const uint64_t *in, size_t n, int inverse, const int64_t *rows,
                     size_t nrows, uint64_t *out) {
    u256 w, ninv, nn;
    root_of_unity(&w, n);
    if (inverse) finv(&w, &w, &MODR);
    memset(&nn, 0, sizeof nn);
    nn.w[0] = (uint32_t)n;
    nn.w[1] = (uint32_t)((uint64_t)n >> 32);
    finv(&ninv, &nn, &MODR);
    u256 *pw = (u256 *)malloc(sizeof(u256) * (n ? n : 1));
    u256 *x = (u256 *)malloc(sizeof(u256) * (n ? n : 1));
    set_small(&pw[0], 1);
    for (size_t t = 1; t < n; t++) fmul(&pw[t], &pw[t - 1], &w, &MODR);
    for (size_t j = 0; j < n; j++) load(&x[j], in + 4 * j);
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 4)
    for (size_t i = 0; i < nrows; i++) {
        size_t k = (size_t)rows[i];
        u256 acc, t;
        set_small(&acc, 0);
        for (size_t j = 0; j < n; j++) {
            fmul(&t, &x[j], &pw[(j * k) % n], &MODR);
            fadd(&acc, &acc, &t, &MODR);
        }
        if (inverse) fmul(&acc, &acc, &ninv, &MODR);
        store(out + 4 * i, &acc);
    }
    free(pw);
    free(x);
}

/* out[k] = sum_j in[j] omega^{jk}  (inverse: n^{-1} sum_j in[j] omega^{-jk}). */
void orc_dft(const uint64_t *in, size_t n, int inverse, uint64_t *out) {
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * n);
    for (size_t k = 0; k < n; k++) rows[k] = (int64_t)k;
    dft_rows(in, n, inverse, rows, n, out);
    free(rows);
}

/* Only the listed output indices (sampled checks at large n). */
void orc_dft_rows(const uint64_t *in, size_t n, int inverse, const int64_t *rows, size_t nrows,
                  uint64_t *out) {
    dft_rows(in, n, inverse, rows, nrows, out);
}

/* p(z) = sum_k v_k z^k by Horner's rule (values of a transform's output
 * polynomial; the left side of the fingerprint below). */
void orc_poly_eval(const uint64_t *v, size_t n, const uint64_t *z64, uint64_t *out) {
    u256 z, acc, c, t;
    load(&z, z64);
    set_small(&acc, 0);
    for (size_t k = n; k-- > 0;) {
        load(&c, v + 4 * k);
        fmul(&t, &acc, &z, &MODR);
        fadd(&acc, &t, &c, &MODR);
    }
    store(out, &acc);
}

/* Fingerprint of the NTT of c without computing it: for z with z^n != 1 and
 * z omega^j != 1,
 *   sum_k z^k NTT(c)_k = sum_k z^k sum_j c_j omega^{jk}
 *                      = sum_j c_j sum_k (z omega^j)^k
 *                      = sum_j c_j ((z omega^j)^n - 1) / (z omega^j - 1)
 *                      = sum_j c_j (z^n - 1) / (z omega^j - 1)      (omega^n = 1).
 * Every coefficient (z^n - 1)/(z omega^j - 1) is nonzero, so an error in any
 * single output of a transform changes the left side.  O(n) products and n
 * inversions; returns 1, or 0 when z omega^j = 1 for some j (the identity
 * does not apply). */
int orc_ntt_fingerprint(const uint64_t *c, size_t n, const uint64_t *z64, uint64_t *out) {
    u256 z, w, zn, one, num;
    load(&z, z64);
    root_of_unity(&w, n);
    set_small(&one, 1);
    set_small(&zn, 1);
    for (size_t i = 0; i < n; i++) fmul(&zn, &zn, &z, &MODR); /* z^n */
    fsub(&num, &zn, &one, &MODR);
    u256 *zw = (u256 *)malloc(sizeof(u256) * (n ? n : 1)); /* z omega^j */
    zw[0] = z;
    for (size_t j = 1; j < n; j++) fmul(&zw[j], &zw[j - 1], &w, &MODR);
    int ok = 1;
    u256 total;
    set_small(&total, 0);
#pragma omp parallel num_threads(g_threads)
    {
        u256 part;
        set_small(&part, 0);
#pragma omp for schedule(static)
        for (size_t j = 0; j < n; j++) {
            u256 den, x, t;
            fsub(&den, &zw[j], &one, &MODR);
            if (is_zero(&den)) {
#pragma omp atomic write
                ok = 0;
                continue;
            }
            finv(&den, &den, &MODR);
            load(&x, c + 4 * j);
            fmul(&t, &x, &num, &MODR);
            fmul(&t, &t, &den, &MODR);
            fadd(&part, &part, &t, &MODR);
        }
#pragma omp critical
        fadd(&total, &total, &part, &MODR);
    }
    free(zw);
    store(out, &total);
    return ok;
}

/* ------------------------------------------------------------------ */
/* Generalised Mira fold (Sec. 4.2), degree-2 relation m1 o m2 - mu m3 = e */
/* ------------------------------------------------------------------ */
/*
 * An accumulator is held as
 *   m    : 4 n field elements, m_i at offset i n (evaluations over H);
 *   e    : n field elements (error vector);
 *   inst : 44 limbs = C_1..C_4 (4 x 8), E (8), mu (4).
 *
 * fold(L, R, gamma) with L = acc (scaled by gamma) and R = acc' (Sec. 4.2,
 * step 5: v'' = gamma v + v'):
 *   step 2: e1 = m1 o m2' + m1' o m2 - mu m3' - mu' m3, the X^1 coefficient of
 *           (X m1 + m1') o (X m2 + m2') - (X mu + mu')(X m3 + m3');
 *   step 3: E1 = Commit(ck, e1);
 *   step 5: m_i'' = gamma m_i + m_i', C_i'' = gamma C_i + C_i', mu'' = gamma mu + mu',
 *           e'' = e' + gamma e1 + gamma^2 e, E'' = E' + gamma E1 + gamma^2 E.
 *
 * commit_mode: 0 = no commitments (witness side only; instance points left as
 * they are computed with infinity for E1), 1 = MSM over the given SRS of the
 * O(n^2) INTT, 2 = closed form [f(tau)]_1 through the Lagrange basis at tau.
 */
enum { INST_LIMBS = 44 };

typedef struct {
    int mode;
    const uint64_t *srs;
    u256 tau;
    u256 *lag; /* Lagrange basis at tau for the current n (mode 2) */
    size_t n;
} committer;

static void commit_evals(const committer *cm, const uint64_t *v, size_t n, pt *out) {
    if (cm->mode == 0) { pt_set_inf(out); return; }
    if (cm->mode == 2) { dot_g(out, v, cm->lag, n); return; }
    uint64_t *c = (uint64_t *)malloc(32 * n);
    orc_dft(v, n, 1, c);
    uint64_t o[8];
    orc_msm(cm->srs, c, n, o);
    pt_load(out, o);
    free(c);
}

static void inst_get(const uint64_t *inst, pt C[4], pt *E, u256 *mu) {
    for (int i = 0; i < 4; i++) pt_load(&C[i], inst + 8 * i);
    pt_load(E, inst + 32);
    load(mu, inst + 40);
}

static void inst_put(uint64_t *inst, const pt C[4], const pt *E, const u256 *mu) {
    for (int i = 0; i < 4; i++) pt_store(inst + 8 * i, &C[i]);
    pt_store(inst + 32, E);
    store(inst + 40, mu);
}

static void fold_one(const committer *cm, size_t n,
                     const uint64_t *Lm, const uint64_t *Le, const uint64_t *Linst,
                     const uint64_t *Rm, const uint64_t *Re, const uint64_t *Rinst,
                     const uint64_t *gamma64, uint64_t *Om, uint64_t *Oe, uint64_t *Oinst,
                     uint64_t *E1_out) {
    pt CL[4], CR[4], EL, ER;
    u256 muL, muR, g, g2;
    inst_get(Linst, CL, &EL, &muL);
    inst_get(Rinst, CR, &ER, &muR);
    load(&g, gamma64);
    fmul(&g2, &g, &g, &MODR);

    /* step 2: cross terms.  Degree 2: the X^1 coefficient of
     * (X a1 + b1)(X a2 + b2) - (X mu + mu')(X a3 + b3).  Degree 3: the X^1
     * and X^2 coefficients of
     * (X a1 + b1)(X a2 + b2)(X a3 + b3) - (X mu + mu')^2 (X a4 + b4). */
    uint64_t *e1 = (uint64_t *)malloc(32 * n);
    uint64_t *e2 = g_degree == 3 ? (uint64_t *)malloc(32 * n) : NULL;
    u256 muLL, muLR2, muRR;
    fmul(&muLL, &muL, &muL, &MODR);
    fmul(&muLR2, &muL, &muR, &MODR);
    fadd(&muLR2, &muLR2, &muLR2, &MODR);
    fmul(&muRR, &muR, &muR, &MODR);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (size_t k = 0; k < n; k++) {
        u256 a1, a2, a3, a4, b1, b2, b3, b4, t, acc;
        load(&a1, Lm + 4 * (0 * n + k)); load(&a2, Lm + 4 * (1 * n + k)); load(&a3, Lm + 4 * (2 * n + k));
        load(&b1, Rm + 4 * (0 * n + k)); load(&b2, Rm + 4 * (1 * n + k)); load(&b3, Rm + 4 * (2 * n + k));
        load(&a4, Lm + 4 * (3 * n + k)); load(&b4, Rm + 4 * (3 * n + k));
        if (g_degree == 2) {
            fmul(&acc, &a1, &b2, &MODR);
            fmul(&t, &b1, &a2, &MODR);  fadd(&acc, &acc, &t, &MODR);
            fmul(&t, &muL, &b3, &MODR); fsub(&acc, &acc, &t, &MODR);
            fmul(&t, &muR, &a3, &MODR); fsub(&acc, &acc, &t, &MODR);
            store(e1 + 4 * k, &acc);
        } else {
            u256 u;
            /* X^2: a1 a2 b3 + a1 b2 a3 + b1 a2 a3 - mu^2 b4 - 2 mu mu' a4 */
            fmul(&t, &a1, &a2, &MODR); fmul(&acc, &t, &b3, &MODR);
            fmul(&t, &a1, &b2, &MODR); fmul(&u, &t, &a3, &MODR); fadd(&acc, &acc, &u, &MODR);
            fmul(&t, &b1, &a2, &MODR); fmul(&u, &t, &a3, &MODR); fadd(&acc, &acc, &u, &MODR);
            fmul(&u, &muLL, &b4, &MODR); fsub(&acc, &acc, &u, &MODR);
            fmul(&u, &muLR2, &a4, &MODR); fsub(&acc, &acc, &u, &MODR);
            store(e2 + 4 * k, &acc);
            /* X^1: a1 b2 b3 + b1 a2 b3 + b1 b2 a3 - 2 mu mu' b4 - mu'^2 a4 */
            fmul(&t, &a1, &b2, &MODR); fmul(&acc, &t, &b3, &MODR);
            fmul(&t, &b1, &a2, &MODR); fmul(&u, &t, &b3, &MODR); fadd(&acc, &acc, &u, &MODR);
            fmul(&t, &b1, &b2, &MODR); fmul(&u, &t, &a3, &MODR); fadd(&acc, &acc, &u, &MODR);
            fmul(&u, &muLR2, &b4, &MODR); fsub(&acc, &acc, &u, &MODR);
            fmul(&u, &muRR, &a4, &MODR); fsub(&acc, &acc, &u, &MODR);
            store(e1 + 4 * k, &acc);
        }
    }
    /* step 3: E_j = Commit(e_j) */
    pt E1, E2;
    commit_evals(cm, e1, n, &E1);
    if (e2) commit_evals(cm, e2, n, &E2);
    u256 g3;
    fmul(&g3, &g2, &g, &MODR);

    /* step 5: witness RLC; e'' = e' + sum_j gamma^j e_j + gamma^d e */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (size_t k = 0; k < n; k++) {
        u256 a, b, t, c;
        for (int i = 0; i < 4; i++) {
            load(&a, Lm + 4 * (i * n + k));
            load(&b, Rm + 4 * (i * n + k));
            fmul(&t, &g, &a, &MODR);
            fadd(&t, &t, &b, &MODR);
            store(Om + 4 * (i * n + k), &t);
        }
        load(&a, Le + 4 * k);   /* e  */
        load(&b, Re + 4 * k);   /* e' */
        load(&c, e1 + 4 * k);   /* e1 */
        fmul(&t, &g, &c, &MODR);
        fadd(&t, &t, &b, &MODR);
        if (e2) {
            load(&c, e2 + 4 * k);
            fmul(&c, &g2, &c, &MODR);
            fadd(&t, &t, &c, &MODR);
            fmul(&c, &g3, &a, &MODR);
        } else {
            fmul(&c, &g2, &a, &MODR);
        }
        fadd(&t, &t, &c, &MODR);
        store(Oe + 4 * k, &t);
    }
    free(e1);
    free(e2);

    /* step 5: instance RLC */
    pt CO[4], EO, t1, t2;
    u256 muO;
    for (int i = 0; i < 4; i++) {
        pt_mul(&t1, &CL[i], &g);
        pt_add(&CO[i], &t1, &CR[i]);
    }
    pt_mul(&t1, &E1, &g);
    pt_add(&EO, &ER, &t1);
    if (g_degree == 3) {
        pt_mul(&t2, &E2, &g2);
        pt_add(&EO, &EO, &t2);
        pt_mul(&t2, &EL, &g3);
    } else {
        pt_mul(&t2, &EL, &g2);
    }
    pt_add(&EO, &EO, &t2);
    fmul(&muO, &g, &muL, &MODR);
    fadd(&muO, &muO, &muR, &MODR);
    inst_put(Oinst, CO, &EO, &muO);
    if (E1_out) {
        pt_store(E1_out, &E1);
        if (g_degree == 3) pt_store(E1_out + 8, &E2);
    }
}

static void committer_init(committer *cm, int mode, const uint64_t *srs, const uint64_t *tau64, size_t n) {
    memset(cm, 0, sizeof *cm);
    cm->mode = mode;
    cm->srs = srs;
    cm->n = n;
    if (mode == 2) {
        load(&cm->tau, tau64);
        cm->lag = (u256 *)malloc(sizeof(u256) * n);
        lagrange_at(cm->lag, n, &cm->tau);
    }
}

static void committer_free(committer *cm) { free(cm->lag); }

void orc_fold(size_t n,
              const uint64_t *Lm, const uint64_t *Le, const uint64_t *Linst,
              const uint64_t *Rm, const uint64_t *Re, const uint64_t *Rinst,
              const uint64_t *gamma, int commit_mode, const uint64_t *srs, const uint64_t *tau,
              uint64_t *Om, uint64_t *Oe, uint64_t *Oinst, uint64_t *E1_out) {
    committer cm;
    committer_init(&cm, commit_mode, srs, tau, n);
    fold_one(&cm, n, Lm, Le, Linst, Rm, Re, Rinst, gamma, Om, Oe, Oinst, E1_out);
    committer_free(&cm);
}

/* Leaf accumulator from a NARK witness (Sec. 4.2: a NARK proof is the special
 * accumulator with mu = 1 and e = 0): e = 0, E = infinity,
 * mu = 1, C_i = Commit(m_i).  Degree 2: m holds m1, m2, m4 on input and
 * m3 = m1 o m2 is written; degree 3: m holds m1, m2, m3 and m4 = m1 o m2 o m3
 * is written. */
void orc_leaf_init(size_t n, uint64_t *m, uint64_t *e, uint64_t *inst,
                   int commit_mode, const uint64_t *srs, const uint64_t *tau) {
    for (size_t k = 0; k < n; k++) {
        u256 a, b, c;
        load(&a, m + 4 * (0 * n + k));
        load(&b, m + 4 * (1 * n + k));
        fmul(&c, &a, &b, &MODR);
        if (g_degree == 3) { /* m4 = m1 o m2 o m3 */
            load(&a, m + 4 * (2 * n + k));
            fmul(&c, &c, &a, &MODR);
            store(m + 4 * (3 * n + k), &c);
        } else {
            store(m + 4 * (2 * n + k), &c);
        }
    }
    memset(e, 0, 32 * n);
    committer cm;
    committer_init(&cm, commit_mode, srs, tau, n);
    pt C[4], E;
    for (int i = 0; i < 4; i++) commit_evals(&cm, m + 4 * i * n, n, &C[i]);
    pt_set_inf(&E);
    u256 one; set_small(&one, 1);
    inst_put(inst, C, &E, &one);
    committer_free(&cm);
}

/* Binary fold tree over count = 2^L accumulators (Sec. 4.2, "Merkle tree
 * reduction"): at level l = 1..L, fold j of that level combines the two
 * accumulators of the previous level at positions 2j (L, scaled) and 2j + 1
 * (R) with gamma_{l,j}; gammas are level-major (count - 1 of them).  Works in
 * place: accumulator j of level l is written over slot j of the arrays.  The
 * root ends in slot 0. */
void orc_fold_tree(size_t count, size_t n, uint64_t *m, uint64_t *e, uint64_t *inst,
                   const uint64_t *gammas, int commit_mode, const uint64_t *srs,
                   const uint64_t *tau) {
    committer cm;
    committer_init(&cm, commit_mode, srs, tau, n);
    size_t width = count, gi = 0;
    while (width > 1) {
        for (size_t j = 0; j < width / 2; j++) {
            size_t a = 2 * j, b = 2 * j + 1;
            uint64_t *tm = (uint64_t *)malloc(32 * 4 * n);
            uint64_t *te = (uint64_t *)malloc(32 * n);
            uint64_t ti[INST_LIMBS];
            fold_one(&cm, n, m + 16 * n * a, e + 4 * n * a, inst + INST_LIMBS * a,
                     m + 16 * n * b, e + 4 * n * b, inst + INST_LIMBS * b,
                     gammas + 4 * (gi + j), tm, te, ti, NULL);
            memcpy(m + 16 * n * j, tm, 32 * 4 * n);
            memcpy(e + 4 * n * j, te, 32 * n);
            memcpy(inst + INST_LIMBS * j, ti, sizeof ti);
            free(tm);
            free(te);
        }
        gi += width / 2;
        width /= 2;
    }
    committer_free(&cm);
}

/* Decider D (Sec. 4.2): the relaxed test m1 o m2 - mu m3 = e (degree 2) or
 * m1 o m2 o m3 - mu^2 m4 = e (degree 3) holds at every point of H.  Returns
 * the number of failing positions. */
size_t orc_decide_relation(size_t n, const uint64_t *m, const uint64_t *e, const uint64_t *mu64) {
    size_t bad = 0;
    u256 mu; load(&mu, mu64);
#pragma omp parallel for reduction(+ : bad) num_threads(g_threads) schedule(static)
    for (size_t k = 0; k < n; k++) {
        u256 a, b, c, x, t, lhs;
        load(&a, m + 4 * (0 * n + k));
        load(&b, m + 4 * (1 * n + k));
        load(&c, m + 4 * (2 * n + k));
        load(&x, e + 4 * k);
        fmul(&lhs, &a, &b, &MODR);
        if (g_degree == 3) { /* m1 m2 m3 - mu^2 m4 */
            u256 d4;
            load(&d4, m + 4 * (3 * n + k));
            fmul(&lhs, &lhs, &c, &MODR);
            fmul(&t, &mu, &mu, &MODR);
            fmul(&t, &t, &d4, &MODR);
        } else {
            fmul(&t, &mu, &c, &MODR);
        }
        fsub(&lhs, &lhs, &t, &MODR);
        if (cmp(&lhs, &x) != 0) bad++;
    }
    return bad;
}

/* Accumulation verifier V_acc (Sec. 4.2, steps 3-4) on instances only:
 * checks C'' = gamma C + C', mu'' = gamma mu + mu', E'' = E' + gamma E1 + gamma^2 E.
 * Returns 1 when all hold. */
int orc_verify_fold(const uint64_t *Linst, const uint64_t *Rinst, const uint64_t *Oinst,
                    const uint64_t *E1_64, const uint64_t *gamma64) {
    pt CL[4], CR[4], CO[4], EL, ER, EO, E1, t1, t2, want;
    u256 muL, muR, muO, g, g2, m;
    inst_get(Linst, CL, &EL, &muL);
    inst_get(Rinst, CR, &ER, &muR);
    inst_get(Oinst, CO, &EO, &muO);
    pt_load(&E1, E1_64);
    load(&g, gamma64);
    fmul(&g2, &g, &g, &MODR);
    int ok = 1;
    for (int i = 0; i < 4; i++) {
        pt_mul(&t1, &CL[i], &g);
        pt_add(&want, &t1, &CR[i]);
        ok &= want.inf == CO[i].inf && (want.inf || (cmp(&want.x, &CO[i].x) == 0 && cmp(&want.y, &CO[i].y) == 0));
    }
    pt_mul(&t1, &E1, &g);
    pt_add(&want, &ER, &t1);
    if (g_degree == 3) { /* E'' = E' + gamma E1 + gamma^2 E2 + gamma^3 E */
        pt E2;
        u256 g3;
        pt_load(&E2, E1_64 + 8);
        pt_mul(&t2, &E2, &g2);
        pt_add(&want, &want, &t2);
        fmul(&g3, &g2, &g, &MODR);
        pt_mul(&t2, &EL, &g3);
    } else {
        pt_mul(&t2, &EL, &g2);
    }
    pt_add(&want, &want, &t2);
    ok &= want.inf == EO.inf && (want.inf || (cmp(&want.x, &EO.x) == 0 && cmp(&want.y, &EO.y) == 0));
    fmul(&m, &g, &muL, &MODR);
    fadd(&m, &m, &muR, &MODR);
    ok &= cmp(&m, &muO) == 0;
    return ok;
}
