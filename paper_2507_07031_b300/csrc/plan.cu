// plan.cu -- CUDA-graph plans: a whole batched commitment (INTT of every
// vector, then one batched MSM) or a whole fold tree captured once and
// replayed with one cudaGraphLaunch.
//
// The batched kernels already push every uneven task of a batch through one
// fixed sequence of launches (one histogram, sort, accumulation and
// reduction pass over all MSMs; NTT passes grouped by length).  Capturing
// that sequence removes the remaining per-launch host cost, so a batch of
// 256 polynomials, or the ten levels of a 1024-leaf fold tree, is a single
// launch from the host.
//
// A plan owns a lane (private workspace sharing the context's SRS tables and
// twiddles) and a pinned arena for the job tables the graph uploads.  The
// warm-up run sizes every workspace and builds the tables the shapes need, so
// that the capture itself allocates nothing.
#include <cuda_runtime.h>

#include <new>
#include <vector>

#include "ctx.cuh"

struct zk_plan {
    zk_ctx *lane = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    char *arena = nullptr;
    size_t nodes = 0;
};

namespace zk {

namespace {

template <class F>
int make_plan(zk_ctx *ctx, F &&op, zk_plan **out) {
    if (!ctx || !out) return ZK_EINVAL;
    *out = nullptr;
    zk_plan *p = new (std::nothrow) zk_plan();
    if (!p) return ZK_ENOMEM;
    int rc = zk_lane_create(ctx, &p->lane);
    if (rc != ZK_OK) {
        delete p;
        return rc;
    }
    auto fail = [&](int code) {
        zk_plan_destroy(p);
        return code;
    };
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(ZK_ECUDA);
    }
    // The warm-up runs on the plan's own stream: wait for all work already
    // queued (for instance on the caller's stream) on the same buffers.
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(ZK_ECUDA);
    // Warm-up: sizes the lane's workspace, builds tables and twiddles, and
    // measures the bytes the job-table uploads need.
    p->lane->up.recorded = 0;
    rc = op(p->lane, p->stream);
    if (rc != ZK_OK) return fail(rc);
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(ZK_ECUDA);
    const size_t need = p->lane->up.recorded + 4096;
    if (cudaHostAlloc((void **)&p->arena, need, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        p->arena = nullptr;
        return fail(ZK_ENOMEM);
    }
    p->lane->up.arena = p->arena;
    p->lane->up.arena_cap = need;
    p->lane->up.arena_used = 0;
    p->lane->capturing = true;
    if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        p->lane->capturing = false;
        cudaGetLastError();
        return fail(ZK_ECUDA);
    }
    rc = op(p->lane, p->stream);
    cudaError_t e = cudaStreamEndCapture(p->stream, &p->graph);
    p->lane->capturing = false;
    if (rc != ZK_OK) return fail(rc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ZK_ECUDA);
    }
    if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return fail(ZK_ECUDA);
    }
    cudaGraphGetNodes(p->graph, nullptr, &p->nodes);
    *out = p;
    return ZK_OK;
}

bool all_device(const void *const *ptrs, size_t n) {
    for (size_t i = 0; i < n; i++)
        if (ptrs[i] && !is_device_ptr(ptrs[i])) return false;
    return true;
}

}  // namespace

}  // namespace zk

using namespace zk;

extern "C" {

int zk_plan_commit_batch(zk_ctx *ctx, const zk_fr *const *vecs, const size_t *lens, size_t count,
                         unsigned flags, zk_g1 *out, zk_plan **plan) {
    ZK_NVTX("zk_plan_commit_batch");
    if (!ctx || !vecs || !lens || !out || !plan || count == 0) return ZK_EINVAL;
    std::vector<const void *> ptrs(vecs, vecs + count);
    ptrs.push_back(out);
    if (!all_device(ptrs.data(), ptrs.size())) return ZK_EINVAL;
    std::vector<const zk_fr *> v(vecs, vecs + count);
    std::vector<size_t> l(lens, lens + count);
    return make_plan(
        ctx,
        [&](zk_ctx *lane, cudaStream_t s) {
            return zk_commit_batch(lane, v.data(), l.data(), count, flags, out, (zk_stream)s);
        },
        plan);
}

int zk_plan_fold_tree(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, zk_acc *root,
                      zk_plan **plan) {
    ZK_NVTX("zk_plan_fold_tree");
    if (!ctx || !leaves || !gammas || !root || !plan) return ZK_EINVAL;
    if (!is_device_ptr(gammas)) return ZK_EINVAL;
    std::vector<zk_acc> lv(leaves, leaves + count);
    zk_acc r = *root;
    return make_plan(
        ctx,
        [&](zk_ctx *lane, cudaStream_t s) {
            return zk_fold_tree(lane, lv.data(), count, gammas, &r, (zk_stream)s);
        },
        plan);
}

int zk_plan_launch(zk_plan *plan, zk_stream stream) {
    ZK_NVTX("zk_plan_launch");
    if (!plan || !plan->exec) return ZK_EINVAL;
    if (cudaGraphLaunch(plan->exec, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return ZK_ECUDA;
    }
    count_launches(1);
    return ZK_OK;
}

int zk_plan_nodes(const zk_plan *plan, size_t *nodes) {
    if (!plan || !nodes) return ZK_EINVAL;
    *nodes = plan->nodes;
    return ZK_OK;
}

int zk_plan_destroy(zk_plan *plan) {
    if (!plan) return ZK_EINVAL;
    if (plan->stream) cudaStreamSynchronize(plan->stream);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->stream) cudaStreamDestroy(plan->stream);
    if (plan->lane) zk_destroy(plan->lane);
    if (plan->arena) cudaFreeHost(plan->arena);
    delete plan;
    return ZK_OK;
}

}  // extern "C"
