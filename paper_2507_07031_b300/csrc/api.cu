// api.cu -- the extern "C" entry points of zk_b300.h, context management,
// budget-checked allocation and host-buffer staging.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "check.cuh"
#include "ctx.cuh"
#include "field.cuh"

namespace zk {

static std::atomic<unsigned long long> g_launches{0};

void count_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

Shared::~Shared() {
    for (auto &t : tables)
        if (t.buf.p) cudaFree(t.buf.p);
    if (srs.p) cudaFree(srs.p);
    for (auto &b : tw)
        if (b.p) cudaFree(b.p);
    for (auto &b : tws)
        if (b.p) cudaFree(b.p);
    for (auto &b : lag)
        if (b.p) cudaFree(b.p);
    if (hide_tab.p) cudaFree(hide_tab.p);
}

int dev_alloc(Shared &sh, DevBuf &b, size_t bytes) {
    std::lock_guard<std::mutex> g(sh.alloc_mu);
    if (b.p) {
        cudaFree(b.p);
        sh.used -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) return ZK_OK;
    if (sh.budget && sh.used + bytes > sh.budget) return ZK_ENOMEM;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ENOMEM;
    }
    b.p = p;
    b.bytes = bytes;
    sh.used += bytes;
    return ZK_OK;
}

void dev_free(Shared &sh, DevBuf &b) {
    std::lock_guard<std::mutex> g(sh.alloc_mu);
    if (b.p) {
        cudaFree(b.p);
        sh.used -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

void *scratch(zk_ctx *ctx, const char *name, size_t bytes, int *err) {
    DevBuf &b = ctx->scratch[name];
    if (b.p && b.bytes >= bytes) return b.p;
    if (ctx->capturing) {  // a plan's warm-up run sized every buffer already
        *err = ZK_EINVAL;
        return nullptr;
    }
    // Grow by at least 25% so that slowly growing requests do not reallocate
    // (cudaFree waits for the device) on every call.
    size_t want = std::max(bytes, b.bytes + b.bytes / 4);
    want = (want + 255) & ~(size_t)255;
    int r = dev_alloc(*ctx->sh, b, want);
    if (r != ZK_OK) {
        r = dev_alloc(*ctx->sh, b, (bytes + 255) & ~(size_t)255);
        if (r != ZK_OK) {
            *err = r;
            return nullptr;
        }
    }
    return b.p;
}

int set_max_dynamic_smem(const void *func, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    std::lock_guard<std::mutex> g(mu);
    if (done.count({dev, func})) return ZK_OK;
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    done.insert({dev, func});
    return ZK_OK;
}

int upload(zk_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s) {
    Uploader &u = ctx->up;
    const size_t b = (bytes + 255) & ~(size_t)255;
    u.recorded += b;
    if (ctx->capturing) {
        if (!u.arena || u.arena_used + b > u.arena_cap) return ZK_EINVAL;
        char *slot = u.arena + u.arena_used;
        u.arena_used += b;
        memcpy(slot, src, bytes);
        ZK_CUDA_TRY(cudaMemcpyAsync(dst, slot, bytes, cudaMemcpyHostToDevice, s));
        return ZK_OK;
    }
    const size_t kRing = (size_t)8 << 20;
    if (!u.ring) {
        if (cudaHostAlloc((void **)&u.ring, kRing, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            u.ring = nullptr;
        } else {
            u.cap = kRing;
        }
    }
    if (!u.ring || b > u.cap) {  // no ring or oversized: plain (synchronising) copy
        ZK_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return ZK_OK;
    }
    // Retire finished copies; on wrap-around wait for every older copy (the
    // new region may overlap any of them).
    while (!u.inflight.empty() && cudaEventQuery(u.inflight.front().ev) == cudaSuccess) {
        cudaEventDestroy(u.inflight.front().ev);
        u.inflight.pop_front();
    }
    if (u.head + b > u.cap) {
        for (auto &r : u.inflight) {
            cudaEventSynchronize(r.ev);
            cudaEventDestroy(r.ev);
        }
        u.inflight.clear();
        u.head = 0;
    }
    const size_t lo = u.head, hi = u.head + b;
    memcpy(u.ring + lo, src, bytes);
    ZK_CUDA_TRY(cudaMemcpyAsync(dst, u.ring + lo, bytes, cudaMemcpyHostToDevice, s));
    cudaEvent_t ev;
    ZK_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ZK_CUDA_TRY(cudaEventRecord(ev, s));
    u.inflight.push_back({lo, hi, ev});
    u.head = hi;
    return ZK_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(const zk_ctx *ctx) {
        cudaGetDevice(&prev);
        if (ctx && ctx->sh && prev != ctx->sh->device) cudaSetDevice(ctx->sh->device);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Stages `bytes` of a host buffer into the named scratch (or passes a device
// pointer through).
int stage_in(zk_ctx *ctx, const void *src, size_t bytes, const char *name, const void **dev,
             cudaStream_t s) {
    if (is_device_ptr(src)) {
        *dev = src;
        return ZK_OK;
    }
    int err = ZK_OK;
    void *d = scratch(ctx, name, std::max<size_t>(bytes, 32), &err);
    if (!d) return err;
    ZK_CUDA_TRY(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    *dev = d;
    return ZK_OK;
}

__global__ void k_zero_pad(uint4 *dst, size_t from16, size_t to16) {
    for (size_t i = from16 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < to16;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = make_uint4(0, 0, 0, 0);
}

// Workspace copies of many device vectors in one launch (a batch of small
// commitments would otherwise issue a copy and a padding launch per vector):
// vector k (len elements at src) goes to dst, zero-padded to `padded`
// elements.  ebase: prefix of the padded lengths (count + 1 words, elements);
// the grid strides over all 16-byte words.
struct GatherDesc {
    const uint4 *src;
    uint4 *dst;
    uint32_t len, padded;  // elements (32 bytes, two words)
};

__global__ void k_gather_pad(const GatherDesc *__restrict__ d, const uint32_t *__restrict__ ebase, uint32_t count) {
    const size_t words = 2 * (size_t)ebase[count];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t e = (uint32_t)(i >> 1);
        uint32_t lo = 0, hi = count;  // largest k with ebase[k] <= e
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (ebase[mid] <= e) lo = mid;
            else hi = mid;
        }
        const GatherDesc g = d[lo];
        const size_t w = i - 2 * (size_t)ebase[lo];
        g.dst[w] = w < 2 * (size_t)g.len ? g.src[w] : make_uint4(0, 0, 0, 0);
    }
}

// Synthetic canonical F_r elements (253-bit values, so always < r) for
// tuning runs: a SplitMix64-style hash of the index.
__global__ void k_fill_random(uint64_t *out, size_t n, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        for (int l = 0; l < 4; l++) {
            uint64_t z = seed + (4 * i + l + 1) * 0x9E3779B97F4A7C15ull;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            out[4 * i + l] = l == 3 ? (z & ((1ull << 61) - 1)) : z;
        }
    }
}

// Quantised scalars q 2^16 mod r, q a uniform int8 from the same hash (the
// width-tuning data of the MSM's bucket layout).
__global__ void k_fill_quant(uint64_t *out, size_t n, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const int q = (int)(int8_t)(z & 0xff);
        Fr v = fe_zero<FrP>();
        v.v[0] = (uint32_t)((q < 0 ? -q : q) << 16);
        if (q < 0) v = fe_neg<FrP>(v);
        for (int l = 0; l < 4; l++) out[4 * i + l] = ((uint64_t)v.v[2 * l + 1] << 32) | v.v[2 * l];
    }
}

size_t next_pow2(size_t n) {
    size_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

}  // namespace

}  // namespace zk

using namespace zk;

extern "C" {

unsigned long long zk_kernel_launches(void) { return g_launches.load(); }

const char *zk_strerror(int code) {
    switch (code) {
        case ZK_OK: return "ok";
        case ZK_EINVAL: return "invalid argument (null pointer, bad size, non-canonical or off-curve input)";
        case ZK_ESRS: return "no SRS loaded, or request longer than the SRS";
        case ZK_ENOMEM: return "device allocation would exceed the HBM budget";
        case ZK_ECUDA: return "CUDA runtime error";
        case ZK_ETIMEOUT: return "bounded wait expired";
        case ZK_EBUSY: return "queue full";
        default: return "unknown error";
    }
}

int zk_init(zk_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return ZK_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    if (device < 0 || device >= ndev) return ZK_EINVAL;
    zk_ctx *c = new (std::nothrow) zk_ctx();
    if (!c) return ZK_ENOMEM;
    c->sh = std::make_shared<Shared>();
    c->sh->device = device;
    c->sh->budget = hbm_budget_bytes;
    DeviceGuard g(c);
    if (cudaFree(nullptr) != cudaSuccess) {  // create the primary context
        delete c;
        return ZK_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
        c->sh->sms = sms;
    cudaGetLastError();
    *out = c;
    return ZK_OK;
}

static bool layout_value_ok(int op, int value) {
    switch (op) {
        case ZK_TUNE_MSM_CHUNK:
        case ZK_TUNE_MSM_TAIL: return value >= 1 && value <= 4;
        case ZK_TUNE_MSM_SEG: return value >= 3 && value <= 5;
        case ZK_TUNE_MSM_SEGBIG: return value >= 6 && value <= 8;
        default: return false;
    }
}

int zk_check_status(zk_ctx *ctx, unsigned *flags, int *checked) {
    if (!ctx || !flags || !checked) return ZK_EINVAL;
    DeviceGuard g(ctx);
    ZK_CUDA_TRY(cudaDeviceSynchronize());
    uint32_t a = 0, b = 0;
    ZK_TRY(msm_check_read(&a));
    ZK_TRY(ntt_check_read(&b));
    *flags = a | b;
    *checked = kChecked ? 1 : 0;
    return ZK_OK;
}

int zk_tune_set(zk_ctx *ctx, int op, int log2n, int value) {
    if (!ctx || log2n < 0 || log2n > kMaxLogN) return ZK_EINVAL;
    Shared &sh = *ctx->sh;
    std::lock_guard<std::mutex> g(sh.mu);
    if (op == ZK_TUNE_MSM_WINDOW) {
        if (value != 0 && (value < kMinWindow || value > kMaxWindow)) return ZK_EINVAL;
        sh.tuned_window[log2n] = value;
    } else if (op == ZK_TUNE_NTT_RADIX) {
        if (value < 0 || value > 11) return ZK_EINVAL;
        sh.tuned_radix[log2n] = value;
    } else if (op >= ZK_TUNE_MSM_CHUNK && op <= ZK_TUNE_MSM_SEGBIG) {
        if (value != 0 && !layout_value_ok(op, value)) return ZK_EINVAL;
        sh.tuned_layout[op - ZK_TUNE_MSM_CHUNK][log2n] = value;
    } else {
        return ZK_EINVAL;
    }
    return ZK_OK;
}

int zk_tune_get(const zk_ctx *ctx, int op, int log2n, int *value) {
    if (!ctx || !value || log2n < 0 || log2n > kMaxLogN) return ZK_EINVAL;
    if (op == ZK_TUNE_MSM_WINDOW) {
        *value = msm_pick_window(const_cast<zk_ctx *>(ctx), (size_t)1 << log2n, 1);
    } else if (op == ZK_TUNE_NTT_RADIX) {
        *value = ntt_pass_radix(*ctx->sh, log2n);
    } else if (op >= ZK_TUNE_MSM_CHUNK && op <= ZK_TUNE_MSM_SEGBIG) {
        const MsmLayout m = msm_layout(*ctx->sh, log2n);
        const uint32_t v[4] = {m.chunk_log + 1, m.tail_log + 1, m.seg_small, m.seg_big};
        *value = (int)v[op - ZK_TUNE_MSM_CHUNK];
    } else {
        return ZK_EINVAL;
    }
    return ZK_OK;
}

int zk_tune_measure(zk_ctx *ctx, int op, int log2n, int value, int reps, double *ms) {
    ZK_NVTX("zk_tune_measure");
    if (!ctx || !ms || reps < 1 || log2n < 0 || log2n > kMaxLogN) return ZK_EINVAL;
    DeviceGuard g(ctx);
    const size_t n = (size_t)1 << log2n;
    int err = ZK_OK;
    uint64_t *data = (uint64_t *)scratch(ctx, "tune.data", n * 32, &err);
    uint32_t *out = (uint32_t *)scratch(ctx, "tune.out", 64, &err);
    if (!data || !out) return err;
    cudaStream_t s = 0;
    const bool layout = op >= ZK_TUNE_MSM_CHUNK && op <= ZK_TUNE_MSM_SEGBIG;
    if (layout && op != ZK_TUNE_MSM_SEGBIG)
        k_fill_quant<<<1024, 256, 0, s>>>(data, n, 0x5eed0000ull + (uint64_t)log2n);
    else
        k_fill_random<<<1024, 256, 0, s>>>(data, n, 0x5eed0000ull + (uint64_t)log2n);
    ZK_LAUNCHED();
    std::vector<float> t;
    cudaEvent_t e0, e1;
    ZK_CUDA_TRY(cudaEventCreate(&e0));
    ZK_CUDA_TRY(cudaEventCreate(&e1));
    int rc = ZK_OK;
    int saved = 0;
    if (op == ZK_TUNE_NTT_RADIX) {
        if (value < 1 || value > 11) rc = ZK_EINVAL;
        saved = ctx->sh->tuned_radix[log2n];
        ctx->sh->tuned_radix[log2n] = value;
    } else if (layout) {
        if (!layout_value_ok(op, value)) rc = ZK_EINVAL;
        saved = ctx->sh->tuned_layout[op - ZK_TUNE_MSM_CHUNK][log2n];
        ctx->sh->tuned_layout[op - ZK_TUNE_MSM_CHUNK][log2n] = value;
    } else if (op != ZK_TUNE_MSM_WINDOW || value < kMinWindow || value > kMaxWindow) {
        rc = ZK_EINVAL;
    }
    for (int r = 0; rc == ZK_OK && r <= reps; r++) {  // run 0 warms up (tables, twiddles)
        cudaEventRecord(e0, s);
        if (op == ZK_TUNE_MSM_WINDOW || layout) {
            MsmJob j;
            j.scalars = (const uint32_t *)data;
            j.n = (uint32_t)n;
            j.out = out;
            rc = msm_batch_impl(ctx, &j, 1, layout ? 0 : value, s);
        } else {
            rc = ntt_impl(ctx, (uint32_t *)data, n, false, s);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float x = 0;
        cudaEventElapsedTime(&x, e0, e1);
        if (r > 0) t.push_back(x);
    }
    if (op == ZK_TUNE_NTT_RADIX) ctx->sh->tuned_radix[log2n] = saved;
    if (layout && layout_value_ok(op, value)) ctx->sh->tuned_layout[op - ZK_TUNE_MSM_CHUNK][log2n] = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ZK_OK) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return ZK_OK;
}

int zk_set_commit_route(zk_ctx *ctx, int route) {
    if (!ctx || (route != ZK_ROUTE_INTT && route != ZK_ROUTE_LAGRANGE)) return ZK_EINVAL;
    ctx->sh->commit_route = route;
    return ZK_OK;
}

int zk_timing_enable(zk_ctx *ctx, int on) {
    if (!ctx) return ZK_EINVAL;
    ctx->timing = on != 0;
    return ZK_OK;
}

int zk_timing_read(zk_ctx *ctx, double ms[ZK_NPHASES], unsigned long long count[ZK_NPHASES]) {
    if (!ctx || !ms || !count) return ZK_EINVAL;
    DeviceGuard g(ctx);
    for (int i = 0; i < ZK_NPHASES; i++) {
        ms[i] = 0;
        count[i] = 0;
    }
    int rc = ZK_OK;
    for (auto &m : ctx->marks) {
        float t = 0;
        if (cudaEventSynchronize(m.b) != cudaSuccess || cudaEventElapsedTime(&t, m.a, m.b) != cudaSuccess) {
            cudaGetLastError();
            rc = ZK_ECUDA;
        }
        if (m.phase >= 0 && m.phase < ZK_NPHASES) {
            ms[m.phase] += t;
            count[m.phase] += 1;
        }
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    ctx->marks.clear();
    return rc;
}

int zk_lane_create(zk_ctx *parent, zk_ctx **out) {
    if (!parent || !out) return ZK_EINVAL;
    zk_ctx *c = new (std::nothrow) zk_ctx();
    if (!c) return ZK_ENOMEM;
    c->sh = parent->sh;
    c->is_lane = true;
    *out = c;
    return ZK_OK;
}

int zk_destroy(zk_ctx *ctx) {
    if (!ctx) return ZK_EINVAL;
    {
        DeviceGuard g(ctx);
        cudaDeviceSynchronize();
        for (auto &m : ctx->marks) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        ctx->marks.clear();
        if (ctx->side) cudaStreamDestroy(ctx->side);
        for (auto &e : ctx->side_ev)
            if (e) cudaEventDestroy(e);
        for (auto &r : ctx->up.inflight) cudaEventDestroy(r.ev);
        ctx->up.inflight.clear();
        if (ctx->up.ring) cudaFreeHost(ctx->up.ring);
        ctx->up.ring = nullptr;
        for (auto &kv : ctx->scratch) dev_free(*ctx->sh, kv.second);
        ctx->scratch.clear();
        ctx->sh.reset();  // frees SRS and tables with the last owner
    }
    delete ctx;
    return ZK_OK;
}

int zk_srs_load(zk_ctx *ctx, const zk_g1 *pts, size_t n) {
    ZK_NVTX("zk_srs_load");
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return srs_load_impl(ctx, pts, n, 0);
}

int zk_srs_generate(zk_ctx *ctx, const zk_fr *tau, size_t n) {
    ZK_NVTX("zk_srs_generate");
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return srs_generate_impl(ctx, tau, n, 0);
}

int zk_srs_size(const zk_ctx *ctx, size_t *n) {
    if (!ctx || !n) return ZK_EINVAL;
    *n = ctx->sh->srs_n;
    return ZK_OK;
}

int zk_srs_export(zk_ctx *ctx, zk_g1 *out, size_t first, size_t count, zk_stream stream) {
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return srs_export_impl(ctx, out, first, count, (cudaStream_t)stream);
}

// Output buffer of an opening: the caller's device pointer, or workspace
// copied back to the host pointer after the call.
struct OutBuf {
    void *user = nullptr, *dev = nullptr;
    size_t bytes = 0;
    int init(zk_ctx *ctx, void *p, size_t n, const char *name) {
        user = p;
        bytes = n;
        if (!p || is_device_ptr(p)) {
            dev = p;
            return ZK_OK;
        }
        int err = ZK_OK;
        dev = scratch(ctx, name, std::max<size_t>(n, 32), &err);
        return dev ? ZK_OK : err;
    }
    int finish(cudaStream_t s) {
        if (user && dev != user) ZK_CUDA_TRY(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, s));
        return ZK_OK;
    }
    bool host() const { return user && dev != user; }
};

int zk_open(zk_ctx *ctx, const zk_fr *coeffs, size_t n, const zk_fr *x, zk_fr *y, zk_g1 *proof, zk_fr *quotient,
            zk_stream stream) {
    ZK_NVTX("zk_open");
    if (!ctx || !coeffs || !x || !y || !proof || n == 0) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->sh->srs_n == 0) return ZK_ESRS;
    const void *dc = nullptr, *dx = nullptr;
    ZK_TRY(stage_in(ctx, coeffs, n * 32, "open.in0", &dc, s));
    ZK_TRY(stage_in(ctx, x, 32, "open.x", &dx, s));
    OutBuf oy, op, oq;
    ZK_TRY(oy.init(ctx, y, 32, "open.y"));
    ZK_TRY(op.init(ctx, proof, 64, "open.proof"));
    ZK_TRY(oq.init(ctx, quotient, (n - 1) * 32, "open.quot"));
    const uint32_t *pv[1] = {(const uint32_t *)dc};
    const size_t lv[1] = {n};
    ZK_TRY(open_impl(ctx, pv, lv, 1, (const uint32_t *)dx, nullptr, (uint32_t *)oy.dev, (uint32_t *)oq.dev,
                     (uint32_t *)op.dev, s));
    ZK_TRY(oy.finish(s));
    ZK_TRY(op.finish(s));
    ZK_TRY(oq.finish(s));
    if (oy.host() || op.host() || oq.host()) ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int zk_open_batch(zk_ctx *ctx, const zk_fr *const *polys, const size_t *lens, size_t count, const zk_fr *x,
                  const zk_fr *gamma, zk_fr *ys, zk_g1 *proof, zk_stream stream) {
    ZK_NVTX("zk_open_batch");
    if (!ctx || !polys || !lens || !x || !gamma || !ys || !proof || count == 0) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->sh->srs_n == 0) return ZK_ESRS;
    std::vector<const uint32_t *> pv(count);
    std::vector<size_t> lv(count);
    size_t host_bytes = 0;
    for (size_t i = 0; i < count; i++) {
        if (!polys[i] || lens[i] == 0) return ZK_EINVAL;
        lv[i] = lens[i];
        if (!is_device_ptr(polys[i])) host_bytes += lens[i] * 32;
    }
    int err = ZK_OK;
    char *stage = nullptr;
    if (host_bytes) {
        stage = (char *)scratch(ctx, "open.inb", host_bytes, &err);
        if (!stage) return err;
    }
    size_t off = 0;
    for (size_t i = 0; i < count; i++) {
        if (is_device_ptr(polys[i])) {
            pv[i] = (const uint32_t *)polys[i];
        } else {
            ZK_CUDA_TRY(cudaMemcpyAsync(stage + off, polys[i], lens[i] * 32, cudaMemcpyHostToDevice, s));
            pv[i] = (const uint32_t *)(stage + off);
            off += lens[i] * 32;
        }
    }
    const void *dx = nullptr, *dg = nullptr;
    ZK_TRY(stage_in(ctx, x, 32, "open.x", &dx, s));
    ZK_TRY(stage_in(ctx, gamma, 32, "open.gamma", &dg, s));
    OutBuf oy, op;
    ZK_TRY(oy.init(ctx, ys, count * 32, "open.ys"));
    ZK_TRY(op.init(ctx, proof, 64, "open.proof"));
    ZK_TRY(open_impl(ctx, pv.data(), lv.data(), count, (const uint32_t *)dx, (const uint32_t *)dg,
                     (uint32_t *)oy.dev, nullptr, (uint32_t *)op.dev, s));
    ZK_TRY(oy.finish(s));
    ZK_TRY(op.finish(s));
    if (oy.host() || op.host()) ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int zk_mul_quotient(zk_ctx *ctx, const zk_fr *a, const zk_fr *b, size_t n, zk_fr *t, zk_g1 *com,
                    zk_stream stream) {
    ZK_NVTX("zk_mul_quotient");
    if (!ctx || !a || !b || !com || n == 0) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->sh->srs_n == 0) return ZK_ESRS;
    const void *da = nullptr, *db = nullptr;
    ZK_TRY(stage_in(ctx, a, n * 32, "mq.in_a", &da, s));
    ZK_TRY(stage_in(ctx, b, n * 32, "mq.in_b", &db, s));
    OutBuf ot, oc;
    ZK_TRY(ot.init(ctx, t, (n - 1) * 32, "mq.out_t"));
    ZK_TRY(oc.init(ctx, com, 64, "mq.out_com"));
    ZK_TRY(mul_quotient_impl(ctx, (const uint32_t *)da, (const uint32_t *)db, n, (uint32_t *)ot.dev,
                             (uint32_t *)oc.dev, s));
    ZK_TRY(ot.finish(s));
    ZK_TRY(oc.finish(s));
    if (ot.host() || oc.host()) ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int zk_set_fold_degree(zk_ctx *ctx, int degree) {
    if (!ctx || (degree != 2 && degree != 3)) return ZK_EINVAL;
    ctx->sh->fold_degree = degree;
    return ZK_OK;
}

int zk_set_hiding_base(zk_ctx *ctx, const zk_g1 *H) {
    ZK_NVTX("zk_set_hiding_base");
    if (!ctx || !H) return ZK_EINVAL;
    DeviceGuard g(ctx);
    const void *dh = nullptr;
    ZK_TRY(stage_in(ctx, H, 64, "hide.in", &dh, 0));
    return hiding_base_impl(ctx, (const uint32_t *)dh, 0);
}

int zk_commit_hiding(zk_ctx *ctx, const zk_fr *coeffs, size_t n, const zk_fr *s, zk_g1 *out,
                     zk_stream stream) {
    ZK_NVTX("zk_commit_hiding");
    if (!ctx || !coeffs || !s || !out || n == 0) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->sh->srs_n == 0) return ZK_ESRS;
    if (n > ctx->sh->srs_n) return ZK_ESRS;
    const void *dc = nullptr, *ds = nullptr;
    ZK_TRY(stage_in(ctx, coeffs, n * 32, "hide.coeffs", &dc, st));
    ZK_TRY(stage_in(ctx, s, 32, "hide.s", &ds, st));
    OutBuf oo;
    ZK_TRY(oo.init(ctx, out, 64, "hide.out"));
    ZK_TRY(commit_hiding_impl(ctx, (const uint32_t *)dc, n, (const uint32_t *)ds, (uint32_t *)oo.dev, st));
    ZK_TRY(oo.finish(st));
    if (oo.host()) ZK_CUDA_TRY(cudaStreamSynchronize(st));
    return ZK_OK;
}

int zk_commit(zk_ctx *ctx, const zk_fr *coeffs, size_t n, zk_g1 *out, zk_stream stream) {
    ZK_NVTX("zk_commit");
    if (!ctx || !coeffs || !out || n == 0) return ZK_EINVAL;
    const size_t lens[1] = {n};
    const zk_fr *const vecs[1] = {coeffs};
    return zk_commit_batch(ctx, vecs, lens, 1, 0, out, stream);
}

int zk_commit_batch(zk_ctx *ctx, const zk_fr *const *vecs, const size_t *lens, size_t count,
                    unsigned flags, zk_g1 *out, zk_stream stream) {
    ZK_NVTX("zk_commit_batch");
    if (!ctx || !vecs || !lens || !out) return ZK_EINVAL;
    if (count == 0) return ZK_OK;
    if (flags & ~(ZK_EVALS | ZK_LAGRANGE)) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    Shared &sh = *ctx->sh;
    // Evaluation-form vectors go through the INTT and the SRS, or directly
    // through the Lagrange basis of H (ZK_LAGRANGE, or the context's route).
    const bool lagrange = (flags & ZK_LAGRANGE) || ((flags & ZK_EVALS) && sh.commit_route == ZK_ROUTE_LAGRANGE);
    const bool evals = (flags & (ZK_EVALS | ZK_LAGRANGE)) != 0;
    if (sh.srs_n == 0) return ZK_ESRS;
    std::vector<size_t> padded(count);
    size_t total = 0;
    for (size_t k = 0; k < count; k++) {
        if (!vecs[k] && lens[k]) return ZK_EINVAL;
        padded[k] = evals ? next_pow2(std::max<size_t>(lens[k], 1)) : lens[k];
        if (lens[k] == 0) padded[k] = 0;
        if (padded[k] > sh.srs_n) return ZK_ESRS;
        if (evals && padded[k] > ((size_t)1 << kMaxLogN)) return ZK_EINVAL;
        total += padded[k];
    }
    if (total >= ((size_t)1 << 32)) return ZK_EINVAL;  // 32-bit element offsets (workspace, MSM)
    // Inputs: staged (host sources, or a workspace copy for the INTT).
    int err = ZK_OK;
    bool any_host = false;
    std::vector<bool> dev_in(count);
    for (size_t k = 0; k < count; k++) {
        dev_in[k] = !lens[k] || is_device_ptr(vecs[k]);
        any_host |= !dev_in[k];
    }
    bool need_ws = any_host;
    for (size_t k = 0; k < count; k++)
        need_ws |= evals && (!lagrange || padded[k] != lens[k]);
    uint32_t *ws = nullptr;
    if (need_ws) {
        ws = (uint32_t *)scratch(ctx, "commit.ws", std::max<size_t>(total, 1) * 32, &err);
        if (!ws) return err;
    }
    std::vector<MsmJob> jobs(count);
    std::vector<uint32_t *> ntt_vecs;
    std::vector<size_t> ntt_lens;
    std::vector<GatherDesc> gather;  // device sources copied to the workspace
    size_t off = 0;
    for (size_t k = 0; k < count; k++) {
        const uint32_t *src = (const uint32_t *)vecs[k];
        if ((evals && (!lagrange || padded[k] != lens[k])) || !dev_in[k]) {
            uint32_t *dst = ws + off * 8;
            if (dev_in[k] && padded[k]) {
                gather.push_back({(const uint4 *)src, (uint4 *)dst, (uint32_t)lens[k], (uint32_t)padded[k]});
            } else {
                if (lens[k]) ZK_CUDA_TRY(cudaMemcpyAsync(dst, src, lens[k] * 32, cudaMemcpyHostToDevice, s));
                if (padded[k] > lens[k]) {
                    k_zero_pad<<<64, 256, 0, s>>>((uint4 *)dst, lens[k] * 2, padded[k] * 2);
                    ZK_LAUNCHED();
                }
            }
            if (evals && !lagrange && padded[k]) {
                ntt_vecs.push_back(dst);
                ntt_lens.push_back(padded[k]);
            }
            src = dst;
        }
        jobs[k].scalars = src;
        jobs[k].n = (uint32_t)padded[k];
        if (lagrange && padded[k] > 1) {
            int lg = 0;
            while (((size_t)1 << lg) < padded[k]) lg++;
            const Affine *lb;
            ZK_TRY(lagrange_get(ctx, lg, &lb, s));
            jobs[k].basis = lg;
        }
        off += padded[k];
    }
    if (!gather.empty()) {
        const size_t gn = gather.size();
        const size_t dbytes = (gn * sizeof(GatherDesc) + 255) / 256 * 256;
        char *gt = (char *)scratch(ctx, "commit.gather", dbytes + (gn + 1) * 4, &err);
        if (!gt) return err;
        std::vector<char> h(dbytes + (gn + 1) * 4, 0);
        std::memcpy(h.data(), gather.data(), gn * sizeof(GatherDesc));
        uint32_t *eb = (uint32_t *)(h.data() + dbytes);
        for (size_t k = 0; k < gn; k++) eb[k + 1] = eb[k] + gather[k].padded;
        ZK_TRY(upload(ctx, gt, h.data(), h.size(), s));
        const size_t words = 2 * (size_t)eb[gn];
        const unsigned blocks = (unsigned)std::min<size_t>((words + 255) / 256, (size_t)sh.sms * 16);
        k_gather_pad<<<std::max(blocks, 1u), 256, 0, s>>>((const GatherDesc *)gt, (const uint32_t *)(gt + dbytes),
                                                         (uint32_t)gn);
        ZK_LAUNCHED();
    }
    if (!ntt_vecs.empty())
        ZK_TRY(ntt_batch_impl(ctx, ntt_vecs.data(), ntt_lens.data(), ntt_vecs.size(), true, s));
    // Outputs.
    const bool dev_out = is_device_ptr(out);
    uint32_t *obuf = (uint32_t *)out;
    if (!dev_out) {
        obuf = (uint32_t *)scratch(ctx, "commit.out", count * 64, &err);
        if (!obuf) return err;
    }
    size_t maxn = 1;
    for (size_t k = 0; k < count; k++) {
        jobs[k].out = obuf + 16 * k;
        maxn = std::max(maxn, (size_t)jobs[k].n);
    }
    ZK_TRY(msm_batch_impl(ctx, jobs.data(), count, 0, s));
    if (!dev_out) {
        ZK_CUDA_TRY(cudaMemcpyAsync(out, obuf, count * 64, cudaMemcpyDeviceToHost, s));
        ZK_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return ZK_OK;
}

static int ntt_entry(zk_ctx *ctx, zk_fr *data, size_t n, bool inverse, zk_stream stream) {
    ZK_NVTX(inverse ? "zk_intt" : "zk_ntt");
    if (!ctx || !data) return ZK_EINVAL;
    if (!n || (n & (n - 1)) || n > ((size_t)1 << kMaxLogN)) return ZK_EINVAL;
    DeviceGuard g(ctx);
    cudaStream_t s = (cudaStream_t)stream;
    if (is_device_ptr(data)) return ntt_impl(ctx, (uint32_t *)data, n, inverse, s);
    const void *d = nullptr;
    ZK_TRY(stage_in(ctx, data, n * 32, "ntt.stage", &d, s));
    ZK_TRY(ntt_impl(ctx, (uint32_t *)d, n, inverse, s));
    ZK_CUDA_TRY(cudaMemcpyAsync(data, d, n * 32, cudaMemcpyDeviceToHost, s));
    ZK_CUDA_TRY(cudaStreamSynchronize(s));
    return ZK_OK;
}

int zk_ntt(zk_ctx *ctx, zk_fr *data, size_t n, zk_stream stream) {
    return ntt_entry(ctx, data, n, false, stream);
}

int zk_intt(zk_ctx *ctx, zk_fr *data, size_t n, zk_stream stream) {
    return ntt_entry(ctx, data, n, true, stream);
}

int zk_ntt_batch(zk_ctx *ctx, zk_fr *const *data, const size_t *lens, size_t count, int inverse,
                 zk_stream stream) {
    ZK_NVTX("zk_ntt_batch");
    if (!ctx || (count && (!data || !lens))) return ZK_EINVAL;
    DeviceGuard g(ctx);
    for (size_t k = 0; k < count; k++)
        if (!is_device_ptr(data[k])) return ZK_EINVAL;
    return ntt_batch_impl(ctx, (uint32_t *const *)data, lens, count, inverse != 0,
                          (cudaStream_t)stream);
}

int zk_leaf_init(zk_ctx *ctx, const zk_acc *accs, size_t count, zk_stream stream) {
    ZK_NVTX("zk_leaf_init");
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return leaf_init_impl(ctx, accs, count, (cudaStream_t)stream);
}

int zk_fold(zk_ctx *ctx, const zk_acc *L, const zk_acc *R, const zk_fr *gamma, zk_acc *out,
            zk_g1 *E1_out, zk_stream stream) {
    ZK_NVTX("zk_fold");
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return fold_impl(ctx, L, R, gamma, out, E1_out, (cudaStream_t)stream);
}

int zk_fold_tree(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, zk_acc *root,
                 zk_stream stream) {
    ZK_NVTX("zk_fold_tree");
    if (!ctx) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return fold_tree_impl(ctx, leaves, count, gammas, root, (cudaStream_t)stream);
}

int zk_fold_tree_levels(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, size_t levels,
                        zk_stream stream) {
    ZK_NVTX("zk_fold_tree_levels");
    if (!ctx || levels == 0) return ZK_EINVAL;
    DeviceGuard g(ctx);
    return fold_tree_impl(ctx, leaves, count, gammas, nullptr, (cudaStream_t)stream, levels);
}

}  // extern "C"
