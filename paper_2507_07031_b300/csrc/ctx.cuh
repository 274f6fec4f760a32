// ctx.cuh -- library context: device, HBM budget, resident SRS tables,
// twiddle tables and grow-only scratch buffers (host-side C++).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/zk_b300.h"

namespace zk {

struct Affine;
struct Xyzz;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Precomputed window table for window width c: entry (w, i) holds
// 2^(c w) * SRS[i] as a window-table entry (AffineS: canonical x, y and
// their precomputed quotients, 128 bytes), for w < W = ceil(254 / c) and
// i < n; window 0 is the base points themselves.  With one table per c every window of a
// scalar adds into the same bucket set, so the bucket reduction is done once
// per MSM instead of once per window, and no Horner pass over windows is
// needed.
struct WindowTable {
    int c = 0;
    int W = 0;
    int basis = 0;  // 0: the SRS (monomial basis); lg > 0: the Lagrange basis of H, |H| = 2^lg
    size_t n = 0;
    DevBuf buf;
};

// State shared by a context and its lanes: the SRS and the tables derived
// from it never change after loading, so lanes read them concurrently.
struct Shared {
    int device = 0;
    int sms = 148;  // streaming multiprocessors of the device
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;        // SRS / tables / twiddles
    std::mutex alloc_mu;  // budget accounting
    size_t srs_n = 0;
    DevBuf srs;  // affine Montgomery, srs_n points
    std::deque<WindowTable> tables;  // deque: references stay valid as tables are added
    DevBuf tw[29];  // tw[lg][k] = omega_{2^lg}^k in Montgomery form, k < 2^lg; then n^-1 entries
    DevBuf tws[12];  // tws[lg][k] = (omega_{2^lg}^k, floor(omega_{2^lg}^k 2^256 / r)), canonical, k < 2^lg
    DevBuf lag[29];              // lag[lg][k] = [L_k(tau)]_1 over H of size 2^lg (affine Montgomery)
    int commit_route = 0;        // ZK_ROUTE_INTT or ZK_ROUTE_LAGRANGE for evaluation-form commitments
    DevBuf hide_tab;             // hiding base H: d 2^(8w) H, w < 32, d = 1 .. 128 (affine Montgomery)
    int fold_degree = 2;         // folded relation: 2 (m1 o m2 - mu m3 = e) or 3 (m1 o m2 o m3 - mu^2 m4 = e)
    int tuned_window[29] = {};   // MSM window width per log2 length (0 = built-in)
    int tuned_radix[29] = {};    // largest NTT pass radix (log2) per log2 length (0 = built-in)
    int tuned_layout[4][29] = {};  // MSM bucket layout per log2 length (0 = built-in): see MsmLayout
    ~Shared();
};

}  // namespace zk

namespace zk {
// One timed interval of a phase, recorded on the launching stream.
struct PhaseMark {
    int phase;
    cudaEvent_t a, b;
};

// Small host-to-device uploads (job tables, pointer tables, descriptors) go
// through pinned host memory so that they stay asynchronous: a copy from
// pageable memory would first wait for everything queued on the stream.
// Normally a ring of pinned memory, reused once the copies that read a region
// have executed (tracked by events); while a graph is being captured, a
// bump arena owned by the plan, whose contents the graph's copy nodes read at
// every replay.
struct Uploader {
    char *ring = nullptr;
    size_t cap = 0, head = 0;
    struct Region {  // a ring region read by a queued copy
        size_t lo, hi;
        cudaEvent_t ev;
    };
    std::deque<Region> inflight;
    char *arena = nullptr;  // set while capturing
    size_t arena_cap = 0, arena_used = 0;
    size_t recorded = 0;  // bytes uploaded (sizes a plan's arena)
};
}  // namespace zk

struct zk_ctx {
    std::shared_ptr<zk::Shared> sh;
    bool is_lane = false;
    bool timing = false;                  // record phase intervals (zk_timing_enable)
    std::vector<zk::PhaseMark> marks;
    std::map<std::string, zk::DevBuf> scratch;  // per context (per lane)
    zk::Uploader up;
    bool capturing = false;  // inside a plan's graph capture: no allocation allowed
    cudaStream_t side = nullptr;         // fold tree: instance passes overlap the next level
    cudaEvent_t side_ev[2] = {nullptr, nullptr};
    int last_error = 0;
};

namespace zk {

constexpr int kMaxLogN = 28;      // 2-adicity of r - 1
constexpr int kMaxSrsLog = 26;    // window-table index must fit 31 bits at c >= 16
constexpr int kScalarBits = 254;  // |recentred scalar| < r / 2 < 2^253, one spare bit for carries
constexpr int kMinWindow = 9;     // MSM window widths with a recode kernel
constexpr int kMaxWindow = 20;

inline int ceil_div_int(int a, int b) { return (a + b - 1) / b; }
inline int windows_for(int c) { return ceil_div_int(kScalarBits, c); }

// Budget-checked device allocation owned by the shared state.
int dev_alloc(Shared &sh, DevBuf &b, size_t bytes);
void dev_free(Shared &sh, DevBuf &b);
// Grow-only named scratch of a context.
void *scratch(zk_ctx *ctx, const char *name, size_t bytes, int *err);

bool is_device_ptr(const void *p);
// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per (device, kernel) pair (the attribute is per device).
int set_max_dynamic_smem(const void *func, int bytes);
// Asynchronous upload of `bytes` host bytes to `dst` on stream s (see Uploader).
int upload(zk_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s);

#define ZK_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ZK_ECUDA;             \
    } while (0)

// Every kernel launch site counts itself (zk_kernel_launches) and checks the
// launch status.
void count_launches(unsigned k);
#define ZK_LAUNCHED()                                       \
    do {                                                    \
        count_launches(1);                                  \
        ZK_CUDA_TRY(cudaGetLastError());                    \
    } while (0)

#define ZK_TRY(expr)                                        \
    do {                                                    \
        int _r = (expr);                                    \
        if (_r != ZK_OK) return _r;                         \
    } while (0)

// A named NVTX range over one public entry point, so that a profiler's
// timeline shows each call by task type (commit, NTT, fold, ...); with no
// tool attached the push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define ZK_NVTX(name) ::zk::NvtxRange zk_nvtx_range_(name)

// Brackets one phase of a call with CUDA events on its stream when the
// context's timing is on (kernel durations for the roofline report).
struct PhaseScope {
    zk_ctx *ctx;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseScope(zk_ctx *c, int ph, cudaStream_t st) : ctx(c), phase(ph), s(st) {
        if (ctx->timing && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, s);
    }
    void end() {
        if (!a) return;
        cudaEvent_t b;
        if (cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, s);
            ctx->marks.push_back({phase, a, b});
        } else {
            cudaEventDestroy(a);
        }
        a = nullptr;
    }
    ~PhaseScope() { end(); }
};

// --- internal entry points between translation units ----------------------

// Check flags of the ZK_CHECK build (check.cuh), read and cleared per unit.
int msm_check_read(uint32_t *flags);
int ntt_check_read(uint32_t *flags);

// SRS (srs.cu)
int srs_load_impl(zk_ctx *ctx, const zk_g1 *pts, size_t n, cudaStream_t s);
int srs_generate_impl(zk_ctx *ctx, const zk_fr *tau, size_t n, cudaStream_t s);
int srs_export_impl(zk_ctx *ctx, zk_g1 *out, size_t first, size_t count, cudaStream_t s);
int table_get(zk_ctx *ctx, int c, size_t n, int basis, const WindowTable **out, cudaStream_t s);
// Lagrange basis [L_k(tau)]_1 of H (|H| = 2^lg), derived from the SRS by an
// inverse DFT over G1 on first use (lagrange.cu).
int lagrange_get(zk_ctx *ctx, int lg, const Affine **out, cudaStream_t s);
int normalize_points(zk_ctx *ctx, const Xyzz *in, Affine *out, size_t n, cudaStream_t s);

// NTT (ntt.cu)
int ntt_impl(zk_ctx *ctx, uint32_t *data, size_t n, bool inverse, cudaStream_t s);
int ntt_batch_impl(zk_ctx *ctx, uint32_t *const *data, const size_t *lens, size_t count,
                   bool inverse, cudaStream_t s);
int twiddles(zk_ctx *ctx, int lg, const uint32_t **out, cudaStream_t s);
int ntt_pass_radix(const Shared &sh, int L);  // tuned or built-in largest pass radix (log2)

// Bucket layout of the MSM (tuned per log2 length, zk_tune_set ops
// ZK_TUNE_MSM_CHUNK .. ZK_TUNE_MSM_SEGBIG):
//   chunk_log : round-0 chunks are 2^chunk_log times longer when few buckets
//               are in use (fewer partial sums for the tail to combine);
//   tail_log  : a team-tail slice gives each lane 2^tail_log items;
//   seg_small, seg_big : log2 of the bucket-reduction segments (seg_big
//               while a level holds at least 2^13 items);
//   seq_log   : not tuned; set per call for large batches: the reduction's
//               first level runs one thread per 2^seq_log buckets (running
//               sums, two additions per bucket) instead of teams (0 = off).
struct MsmLayout {
    uint32_t chunk_log, tail_log, seg_small, seg_big;
    uint32_t seq_log = 0;
};
MsmLayout msm_layout(const Shared &sh, int log2n);

// MSM (msm.cu).  Each job: scalars (device, canonical, 32 B each), length n,
// output 64-byte canonical affine point (device).  c > 0 fixes the window
// width of every job; c = 0 takes the tuned (or modelled) width per length.

struct MsmJob {
    const uint32_t *scalars;
    uint32_t n;
    void *out;
    int basis = 0;  // 0: scalars are coefficients (SRS); lg: evaluations over H, n = 2^lg (Lagrange basis)
};
int msm_batch_impl(zk_ctx *ctx, const MsmJob *jobs, size_t count, int c, cudaStream_t s);

// KZG opening (open.cu), device pointers only: without gamma, one polynomial
// (count = 1): ys[0] = f(x), quotient = (f - f(x)) / (X - x), proof = its
// commitment; with gamma, ys[i] = f_i(x) and the quotient and proof of
// sum_i gamma^i f_i.  quotient may be null (workspace).
int open_impl(zk_ctx *ctx, const uint32_t *const *polys, const size_t *lens, size_t count, const uint32_t *x,
              const uint32_t *gamma, uint32_t *ys, uint32_t *quotient, uint32_t *proof, cudaStream_t s);

// Mul / MatMul quotient (quotient.cu), device pointers only: t (n - 1
// coefficients, may be null) and its commitment com.
int mul_quotient_impl(zk_ctx *ctx, const uint32_t *a, const uint32_t *b, size_t n, uint32_t *t, uint32_t *com,
                      cudaStream_t s);

// Hiding commitments (hiding.cu), device pointers only.
int hiding_base_impl(zk_ctx *ctx, const uint32_t *H, cudaStream_t s);
int commit_hiding_impl(zk_ctx *ctx, const uint32_t *coeffs, size_t n, const uint32_t *sc, uint32_t *out,
                       cudaStream_t s);
int msm_pick_window(zk_ctx *ctx, size_t max_n, size_t count);

// Fold (fold.cu)
int fold_impl(zk_ctx *ctx, const zk_acc *L, const zk_acc *R, const zk_fr *gamma, zk_acc *out,
              zk_g1 *E1_out, cudaStream_t s);
// levels = 0: the whole tree, root copied to *root; else the first `levels`
// levels only (their accumulators left in the leaves' slots), root may be null.
int fold_tree_impl(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, zk_acc *root,
                   cudaStream_t s, size_t levels = 0);
int leaf_init_impl(zk_ctx *ctx, const zk_acc *accs, size_t count, cudaStream_t s);

}  // namespace zk
