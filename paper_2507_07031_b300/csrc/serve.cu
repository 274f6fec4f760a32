// serve.cu -- serving loop with continuous batching for proof jobs.
//
// A job is the hot-path work of one basic-block instance: commit to its
// witness (INTT + MSM of each vector, as a NARK leaf accumulator: Sec. 4.2
// treats a NARK proof as the accumulator with mu = 1, e = 0) and fold that
// leaf into a resident accumulator (Sec. 4.2, prover steps 2-7).
//
// Jobs queue in arrival order.  A scheduler thread admits the head job as
// soon as a lane (a private workspace and CUDA stream) is free and the job's
// workspace estimate fits in what is left of the HBM budget; admitted jobs of
// different sizes then run concurrently on their lanes' streams.  Completion
// is reported by a host callback on the lane's stream, which also frees the
// lane and the job's memory reservation, so waiting jobs are admitted as soon
// as capacity frees up.  All waits are bounded.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.cuh"

namespace zk {

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t) {
    return std::chrono::duration<double, std::milli>(t - t0).count();
}

struct Ticket {
    zk_job job;
    zk_fr gamma;  // host copy when the caller passed a host pointer
    bool gamma_host = false;
    int status = ZK_JOB_QUEUED;
    int error = ZK_OK;
    size_t reserve = 0;
    int lane = -1;
    Clock::time_point t_submit, t_start, t_end;
};

struct Lane {
    zk_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    uint64_t ticket = 0;
    bool busy = false;
};

}  // namespace

}  // namespace zk

struct zk_server {
    zk_ctx *ctx = nullptr;
    size_t budget = 0;
    size_t reserved = 0, peak_reserved = 0;
    std::vector<zk::Lane> lanes;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, zk::Ticket> tickets;
    uint64_t next = 1;
    uint64_t completed = 0;
    uint64_t cancelled = 0;
    bool stop = false;
    std::thread sched;
    zk::Clock::time_point t0;
};

namespace zk {

namespace {

constexpr size_t kMaxQueue = 1 << 16;

// Device workspace a job needs on its lane (leaf commitments of four
// vectors, then one fold of length n with d - 1 cross terms, d the fold
// degree): INTT copies and ping-pong buffers, MSM entries, piece sums and
// buckets, the fold's cross-term vectors.  The leaf's four MSMs run as one
// batch; a fold's d - 1 cross-term MSMs run as one batch after it, in the
// same workspace, so the larger of the two batches sets the MSM terms.
size_t job_bytes(zk_ctx *ctx, size_t n) {
    const int c = msm_pick_window(ctx, n, 4);
    const size_t W = (size_t)windows_for(c);
    const size_t B = (size_t)1 << (c - 1);
    const size_t cross = (size_t)(ctx->sh->fold_degree - 1);
    const size_t jobs = 4 > cross ? 4 : cross;
    size_t b = 0;
    b += jobs * n * 32;                    // INTT staging
    b += 2 * jobs * n * 32;                // NTT ping-pong
    b += jobs * n * W * 4;                 // sorted MSM entries
    b += 2 * (jobs * n * W / 32 + jobs * B) * 128;  // piece sums
    b += jobs * B * (128 + 5 * 4);         // buckets, counts and offsets
    b += cross * n * 32;                   // fold cross terms
    // The piece-sum term assumes 32 entries per piece.  Round 0 cuts chunks
    // as short as 8 entries when a batch is small, which needs up to
    // 2 x 128 B x (3/4 of the resident accumulation threads) more: 14.5 MB
    // on 148 SMs at 4 blocks of 128 threads, inside the 16 MiB slack below.
    return b + ((size_t)16 << 20);
}

bool pow2(size_t n) { return n && !(n & (n - 1)); }

struct Done {
    zk_server *srv;
    uint64_t ticket;
};

void CUDART_CB on_done(void *p) {
    Done *d = static_cast<Done *>(p);
    zk_server *srv = d->srv;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto it = srv->tickets.find(d->ticket);
        if (it != srv->tickets.end()) {
            Ticket &t = it->second;
            t.t_end = Clock::now();
            t.status = t.error == ZK_OK ? ZK_JOB_DONE : ZK_JOB_FAILED;
            srv->reserved -= t.reserve;
            srv->lanes[t.lane].busy = false;
            srv->completed++;
        }
    }
    srv->cv.notify_all();
    delete d;
}

// Enqueues a job's work on its lane (called by the scheduler thread, lock
// not held).  Returns the first error; the completion callback is queued
// either way so that the lane is released.
int run_job(zk_server *srv, Lane &lane, Ticket &t) {
    const zk_job &j = t.job;
    cudaStream_t s = lane.stream;
    zk_stream zs = (zk_stream)s;
    const size_t n = j.n;
    int rc = ZK_OK;
    // The third witness is m4 for the degree-2 relation (m3 = m1 o m2 is
    // derived) and m3 for the degree-3 one (m4 = m1 o m2 o m3 is derived).
    const int third = lane.ctx->sh->fold_degree == 3 ? 2 : 3;
    const zk_fr *src[3] = {j.w[0], j.w[1], j.w[2]};
    zk_fr *dst[3] = {j.leaf->m[0], j.leaf->m[1], j.leaf->m[third]};
    for (int i = 0; i < 3 && rc == ZK_OK; i++)
        if (src[i] != dst[i] && cudaMemcpyAsync(dst[i], src[i], n * 32, cudaMemcpyDefault, s) != cudaSuccess)
            rc = ZK_ECUDA;
    if (rc == ZK_OK) rc = zk_leaf_init(lane.ctx, j.leaf, 1, zs);
    if (rc == ZK_OK && j.acc_in)
        rc = zk_fold(lane.ctx, j.acc_in, j.leaf, t.gamma_host ? &t.gamma : j.gamma, j.acc_out, nullptr, zs);
    return rc;
}

void scheduler(zk_server *srv) {
    std::unique_lock<std::mutex> g(srv->mu);
    while (!srv->stop) {
        bool launched = false;
        while (!srv->queue.empty()) {
            int free_lane = -1;
            for (size_t i = 0; i < srv->lanes.size(); i++)
                if (!srv->lanes[i].busy) {
                    free_lane = (int)i;
                    break;
                }
            if (free_lane < 0) break;
            const uint64_t id = srv->queue.front();
            Ticket &t = srv->tickets[id];
            if (srv->reserved + t.reserve > srv->budget && srv->reserved > 0) break;  // wait for memory
            srv->queue.pop_front();
            Lane &lane = srv->lanes[free_lane];
            lane.busy = true;
            lane.ticket = id;
            t.lane = free_lane;
            t.status = ZK_JOB_RUNNING;
            t.t_start = Clock::now();
            srv->reserved += t.reserve;
            if (srv->reserved > srv->peak_reserved) srv->peak_reserved = srv->reserved;
            g.unlock();
            int rc = run_job(srv, lane, t);
            g.lock();
            t.error = rc;  // before the callback can run
            g.unlock();
            Done *d = new Done{srv, id};
            cudaError_t e = cudaLaunchHostFunc(lane.stream, on_done, d);
            g.lock();
            if (e != cudaSuccess) {  // could not queue the callback: complete here
                cudaGetLastError();
                t.error = ZK_ECUDA;
                g.unlock();
                cudaStreamSynchronize(lane.stream);
                on_done(d);
                g.lock();
            }
            launched = true;
        }
        if (!launched) srv->cv.wait_for(g, std::chrono::milliseconds(5));
    }
}

}  // namespace

}  // namespace zk

using namespace zk;

extern "C" {

int zk_server_create(zk_ctx *ctx, int lanes, size_t hbm_budget_bytes, zk_server **out) {
    if (!ctx || !out || lanes < 1 || lanes > 64) return ZK_EINVAL;
    *out = nullptr;
    zk_server *srv = new (std::nothrow) zk_server();
    if (!srv) return ZK_ENOMEM;
    srv->ctx = ctx;
    srv->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)-1;
    srv->t0 = Clock::now();
    const int dev = ctx->sh->device;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    // The lanes' streams belong to the context's device.
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return ZK_ECUDA;
    }
    int rc = ZK_OK;
    srv->lanes.resize(lanes);
    for (auto &l : srv->lanes) {
        if (zk_lane_create(ctx, &l.ctx) != ZK_OK ||
            cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = ZK_ECUDA;
            break;
        }
    }
    if (rc == ZK_OK) {
        srv->sched = std::thread([srv, dev] {
            cudaSetDevice(dev);
            scheduler(srv);
        });
        *out = srv;
    } else {
        zk_server_destroy(srv);
    }
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return rc;
}

int zk_submit(zk_server *srv, const zk_job *job, uint64_t *ticket) {
    ZK_NVTX("zk_submit");
    if (!srv || !job || !ticket) return ZK_EINVAL;
    const size_t n = job->n;
    if (!pow2(n) || n < 2 || n > srv->ctx->sh->srs_n) return ZK_EINVAL;
    if (!job->leaf || job->leaf->n != n || !job->w[0] || !job->w[1] || !job->w[2]) return ZK_EINVAL;
    if (job->acc_in && (!job->acc_out || !job->gamma || job->acc_in->n != n || job->acc_out->n != n))
        return ZK_EINVAL;
    Ticket t;
    t.job = *job;
    if (job->gamma && !is_device_ptr(job->gamma)) {
        memcpy(&t.gamma, job->gamma, sizeof t.gamma);
        t.gamma_host = true;
    }
    t.reserve = job_bytes(srv->ctx, n);
    t.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->queue.size() >= kMaxQueue) return ZK_EBUSY;
        if (t.reserve > srv->budget) return ZK_ENOMEM;
        const uint64_t id = srv->next++;
        srv->tickets.emplace(id, t);
        srv->queue.push_back(id);
        *ticket = id;
    }
    srv->cv.notify_all();
    return ZK_OK;
}

int zk_poll(zk_server *srv, uint64_t ticket, zk_ticket_info *info) {
    if (!srv || !info) return ZK_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return ZK_EINVAL;
    const Ticket &t = it->second;
    info->status = t.status;
    info->error = t.error;
    info->submit_ms = ms_since(srv->t0, t.t_submit);
    info->start_ms = t.status >= ZK_JOB_RUNNING ? ms_since(srv->t0, t.t_start) : -1.0;
    info->end_ms = t.status >= ZK_JOB_DONE ? ms_since(srv->t0, t.t_end) : -1.0;
    info->lane = t.lane;
    return ZK_OK;
}

int zk_wait(zk_server *srv, uint64_t ticket, int timeout_ms, zk_ticket_info *info) {
    if (!srv || !info) return ZK_EINVAL;
    std::unique_lock<std::mutex> g(srv->mu);
    auto done = [&] {
        auto it = srv->tickets.find(ticket);
        return it == srv->tickets.end() || it->second.status >= ZK_JOB_DONE;
    };
    if (!srv->cv.wait_for(g, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), done)) {
        g.unlock();
        zk_poll(srv, ticket, info);
        return ZK_ETIMEOUT;
    }
    g.unlock();
    return zk_poll(srv, ticket, info);
}

int zk_cancel(zk_server *srv, uint64_t ticket) {
    if (!srv) return ZK_EINVAL;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto it = srv->tickets.find(ticket);
        if (it == srv->tickets.end()) return ZK_EINVAL;
        Ticket &t = it->second;
        if (t.status != ZK_JOB_QUEUED) return ZK_EBUSY;  // admitted (running) or finished
        for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
            if (*q == ticket) {
                srv->queue.erase(q);
                break;
            }
        t.status = ZK_JOB_CANCELLED;
        t.t_end = Clock::now();
        srv->cancelled++;
    }
    srv->cv.notify_all();
    return ZK_OK;
}

int zk_server_stats(zk_server *srv, zk_server_info *info) {
    if (!srv || !info) return ZK_EINVAL;
    std::lock_guard<std::mutex> g(srv->mu);
    info->completed = srv->completed;
    info->cancelled = srv->cancelled;
    info->queued = srv->queue.size();
    info->reserved_bytes = srv->reserved;
    info->peak_reserved_bytes = srv->peak_reserved;
    int busy = 0;
    for (auto &l : srv->lanes) busy += l.busy;
    info->busy_lanes = busy;
    return ZK_OK;
}

int zk_server_destroy(zk_server *srv) {
    if (!srv) return ZK_EINVAL;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->sched.joinable()) srv->sched.join();
    for (auto &l : srv->lanes) {
        if (l.stream) {
            cudaStreamSynchronize(l.stream);
            cudaStreamDestroy(l.stream);
        }
        if (l.ctx) zk_destroy(l.ctx);
    }
    delete srv;
    return ZK_OK;
}

}  // extern "C"
