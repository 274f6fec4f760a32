// diag.cu -- measurement helpers for the roofline: the issue rates of the
// integer instruction forms the field products are built from (independent
// chains of mad.lo, mad.hi, mad.wide, lo/hi carry pairs and ALU carry adds)
// and the sustained Montgomery-product rates of this library's F_q and F_r code.
#include <cuda_runtime.h>

#include <algorithm>

#include "ctx.cuh"
#include "field.cuh"

namespace zk {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

// Each iteration issues kChains * kUnroll independent 32-bit IMADs per thread.
__global__ void k_probe_imad(uint32_t *sink, uint32_t iters, uint32_t seed) {
    uint32_t a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = seed + threadIdx.x * 7u + j * 131u;
    const uint32_t b = seed ^ 0x9e3779b9u;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int j = 0; j < kChains; j++)
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(a[(j + 1) % kChains]));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) x ^= a[j];
    if (x == 0x12345678u) sink[0] = x;  // keep the chains alive
}

// The other instruction forms of the product code, each as kChains
// independent chains per thread (kChains * kUnroll instructions, or pairs,
// per iteration):
//   HI   mad.hi.u32                  (the high half of a limb product)
//   WIDE mad.wide.u32 with a 64-bit addend (both halves in one instruction),
//        its multiplicand the accumulator's low word
//   PAIR mad.lo.cc.u32 + madc.hi.u32 (one limb product of a carry chain)
//   ADD  add.cc.u32 + addc.u32        (integer ALU carry chain)
enum ProbeForm { kHi = 0, kWide = 1, kPair = 2, kAdd = 3 };

template <int F>
__global__ void k_probe_form(uint32_t *sink, uint32_t iters, uint32_t seed) {
    uint32_t a[kChains], h[kChains];
    uint64_t w[kChains];
#pragma unroll
    for (int j = 0; j < kChains; j++) {
        a[j] = seed + threadIdx.x * 7u + j * 131u;
        h[j] = a[j] ^ 0x5bd1e995u;
        w[j] = ((uint64_t)h[j] << 32) | a[j];
    }
    const uint32_t b = seed ^ 0x9e3779b9u;
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int j = 0; j < kChains; j++) {
                if (F == kHi)
                    asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(a[(j + 1) % kChains]));
                else if (F == kWide)  // multiplicand from the accumulator: nothing to hoist
                    asm volatile("{\n\t.reg .u32 t;\n\tcvt.u32.u64 t, %0;\n\tmad.wide.u32 %0, t, %1, %0;\n\t}"
                                 : "+l"(w[j]) : "r"(b));
                else if (F == kPair)
                    asm volatile("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
                                 : "+r"(a[j]), "+r"(h[j]) : "r"(a[(j + 1) % kChains]), "r"(b));
                else
                    asm volatile("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;"
                                 : "+r"(a[j]), "+r"(h[j]) : "r"(b), "r"(a[(j + 1) % kChains]));
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < kChains; j++) x ^= a[j] ^ h[j] ^ (uint32_t)w[j] ^ (uint32_t)(w[j] >> 32);
    if (x == 0x12345678u) sink[0] = x;  // keep the chains alive
}

// Each thread runs `iters` rounds of 4 independent Montgomery products of
// the field P (this library's product code).
template <class P>
__global__ void k_probe_mont(uint32_t *sink, uint32_t iters, uint32_t seed) {
    Fe<P> x[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        x[j] = fe_mont_one<P>();
        x[j].v[0] ^= seed + threadIdx.x + 17u * j;
        x[j].v[7] &= 0x0fffffffu;
    }
    Fe<P> y = x[1];
    for (uint32_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) x[j] = fe_mul<P>(x[j], y);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) acc ^= x[j].v[0];
    if (acc == 0x12345678u) sink[0] = acc;
}

template <class K>
double time_kernel(K kern, int blocks, int threads, uint32_t iters, uint32_t *sink) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0);
        kern<<<blocks, threads>>>(sink, iters, 12345u + rep);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best * 1e-3;
}

}  // namespace

}  // namespace zk

using namespace zk;

// Measures every rate of zk_probe_pipes into r[ZK_NPROBES] (or only the
// mad.lo and F_q product rates when `all` is false).
static int probe(int device, bool all, double *r) {
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return ZK_EINVAL;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    uint32_t *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) {
        cudaGetLastError();
        cudaSetDevice(prev);
        return ZK_ENOMEM;
    }
    const int blocks = sms * 8, threads = 256;
    const uint32_t it1 = 2048;
    const double per = (double)blocks * threads * it1 * kChains * kUnroll;  // instructions (pairs)
    r[ZK_PROBE_MAD_LO] = per / time_kernel(k_probe_imad, blocks, threads, it1, sink);
    int launches = 4;
    if (all) {
        r[ZK_PROBE_MAD_HI] = per / time_kernel(k_probe_form<kHi>, blocks, threads, it1, sink);
        r[ZK_PROBE_MAD_WIDE] = per / time_kernel(k_probe_form<kWide>, blocks, threads, it1, sink);
        r[ZK_PROBE_MAD_PAIR] = per / time_kernel(k_probe_form<kPair>, blocks, threads, it1, sink);
        r[ZK_PROBE_ADD_PAIR] = per / time_kernel(k_probe_form<kAdd>, blocks, threads, it1, sink);
        launches += 16;
    }
    const int mblocks = sms * 4, mthreads = 256;
    const uint32_t it2 = 256;
    const double prods = (double)mblocks * mthreads * it2 * 4;
    r[ZK_PROBE_FQ_MUL] = prods / time_kernel(k_probe_mont<FqP>, mblocks, mthreads, it2, sink);
    launches += 4;
    if (all) {
        r[ZK_PROBE_FR_MUL] = prods / time_kernel(k_probe_mont<FrP>, mblocks, mthreads, it2, sink);
        launches += 4;
    }
    count_launches(launches);
    cudaError_t e = cudaGetLastError();
    cudaFree(sink);
    cudaSetDevice(prev);
    return e == cudaSuccess ? ZK_OK : ZK_ECUDA;
}

extern "C" int zk_probe_rates(int device, double *imad_per_s, double *fq_mul_per_s) {
    if (!imad_per_s || !fq_mul_per_s) return ZK_EINVAL;
    double r[ZK_NPROBES] = {0};
    ZK_TRY(probe(device, false, r));
    *imad_per_s = r[ZK_PROBE_MAD_LO];
    *fq_mul_per_s = r[ZK_PROBE_FQ_MUL];
    return ZK_OK;
}

extern "C" int zk_probe_pipes(int device, double *rates) {
    if (!rates) return ZK_EINVAL;
    return probe(device, true, rates);
}

// ---------------------------------------------------------------------------
// zk_field_op: elementwise F_q / F_r arithmetic on canonical vectors, through
// the same device code the prover uses (Montgomery conversions, product,
// squaring, inversion, addition, subtraction, the difference of two
// products that point additions use, and the NTT's product by a constant
// with a precomputed quotient), for tests of that code.
// ---------------------------------------------------------------------------

namespace zk {

namespace {

template <class P>
__global__ void k_field_op(int op, const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                           uint32_t *__restrict__ out, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (op == ZK_FOP_MULC) {  // plain residues: a + (i mod 4) p times the constant b
        Fe<P> x = fe_load<P>(a + 8 * i);
        const Fe<P> w = fe_load<P>(b + 8 * i);
        const uint32_t pw[8] = {P::p(0), P::p(1), P::p(2), P::p(3), P::p(4), P::p(5), P::p(6), P::p(7)};
        for (size_t m = 0; m < (i & 3); m++) detail::add_words(x.v, pw);
        fe_store<P>(out + 8 * i, fe_mul_shoup<P>(x, w, fe_shoup_quotient<P>(w)));
        return;
    }
    const Fe<P> x = fe_to_mont<P>(fe_load<P>(a + 8 * i));
    Fe<P> y = fe_zero<P>();
    if (op != ZK_FOP_SQR && op != ZK_FOP_INV) y = fe_to_mont<P>(fe_load<P>(b + 8 * i));
    Fe<P> r;
    switch (op) {
        case ZK_FOP_MUL: r = fe_mul<P>(x, y); break;
        case ZK_FOP_MULSUB: {
            const size_t m = n - 1 - i;  // mirror element
            r = fe_mul_sub_mul<P>(x, y, fe_to_mont<P>(fe_load<P>(a + 8 * m)), fe_to_mont<P>(fe_load<P>(b + 8 * m)));
            break;
        }
        case ZK_FOP_SQR: r = fe_sqr<P>(x); break;
        case ZK_FOP_INV: r = fe_inv<P>(x); break;
        case ZK_FOP_ADD: r = fe_add<P>(x, y); break;
        default: r = fe_sub<P>(x, y); break;
    }
    fe_store<P>(out + 8 * i, fe_from_mont<P>(r));
}

}  // namespace

}  // namespace zk

extern "C" int zk_field_op(int field, int op, const zk_fr *a, const zk_fr *b, zk_fr *out, size_t n,
                           zk_stream stream) {
    using namespace zk;
    if (field != ZK_FIELD_Q && field != ZK_FIELD_R) return ZK_EINVAL;
    if (op < ZK_FOP_MUL || op > ZK_FOP_MULC) return ZK_EINVAL;
    if (n == 0) return ZK_OK;
    const bool binary = op != ZK_FOP_SQR && op != ZK_FOP_INV;
    if (!a || !out || (binary && !b) || n > ((size_t)1 << 31)) return ZK_EINVAL;
    if (!is_device_ptr(a) || !is_device_ptr(out) || (binary && !is_device_ptr(b))) return ZK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    const uint32_t *pa = (const uint32_t *)a, *pb = (const uint32_t *)b;
    if (field == ZK_FIELD_Q) k_field_op<FqP><<<blocks, 128, 0, s>>>(op, pa, pb, (uint32_t *)out, n);
    else k_field_op<FrP><<<blocks, 128, 0, s>>>(op, pa, pb, (uint32_t *)out, n);
    count_launches(1);
    return cudaGetLastError() == cudaSuccess ? ZK_OK : ZK_ECUDA;
}
