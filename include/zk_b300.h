/*
 * zk_b300.h -- C ABI of the B300 (sm_103a) prover hot path for ZKTorch-style
 * proofs of ML inference over BN254 (Chen, Tang, Kang, "ZKTorch: Compiling ML
 * Inference to Zero-Knowledge Proofs via Parallel Proof Accumulation").
 *
 * The library computes, on one GPU:
 *   - KZG commitments com = [f(tau)]_1 = sum_i c_i [tau^i]_1 as multi-scalar
 *     multiplications over a device-resident SRS (paper Sec. 2.1);
 *   - the F_r NTT / inverse NTT that maps a witness vector of evaluations over
 *     H = <omega> to polynomial coefficients (Sec. 3, "witness generation and
 *     encoding"; Sec. 4.4, f|_H);
 *   - generalised-Mira accumulation folds and the parallel fold tree
 *     (Sec. 4.2, accumulation prover steps 2-7, tree reduction).
 *
 * Encodings (all little endian, canonical):
 *   zk_fr  -- an element of F_r (r = BN254 group order) as 4 x uint64, value < r.
 *   zk_g1  -- an affine G1 point (y^2 = x^3 + 3 over F_q), x then y, each
 *             4 x uint64 < q.  The point at infinity is 64 zero bytes.
 *   NTT root of unity: omega_n = 5^((r-1)/n) mod r, n a power of two <= 2^28.
 *
 * Memory: unless stated otherwise a buffer argument may be a device pointer
 * (cudaMalloc / torch) or a host pointer; host buffers are staged through the
 * context's device workspace inside the call, and a call with any host output
 * synchronises the stream before it returns.  Device results are valid once
 * the stream has reached the call.  The caller owns every buffer it passes.
 * A context's workspace is not safe for concurrent calls on different
 * streams: use one lane (zk_lane_create) per concurrent stream.
 *
 * Errors: every function returns ZK_OK (0) or one of the codes below; no
 * function aborts the process.  zk_strerror() gives a static description.
 */
#ifndef ZK_B300_H
#define ZK_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZK_OK 0
#define ZK_EINVAL 1   /* null pointer, bad size, non-canonical or off-curve input */
#define ZK_ESRS 2     /* no SRS loaded, or the request is longer than the SRS */
#define ZK_ENOMEM 3   /* allocation would exceed the context's HBM budget */
#define ZK_ECUDA 4    /* a CUDA runtime call failed */
#define ZK_ETIMEOUT 5 /* a bounded wait on the device or in the job queue expired */
#define ZK_EBUSY 6    /* the serving queue is full */

/* Opaque context: device, HBM budget, SRS and its window tables, NTT twiddle
 * tables and scratch workspace.  A stream handle is a cudaStream_t; NULL is
 * the legacy default stream. */
typedef struct zk_ctx zk_ctx;
typedef struct CUstream_st *zk_stream;

typedef struct { uint64_t l[4]; } zk_fr;
typedef struct { uint64_t x[4]; uint64_t y[4]; } zk_g1;

/* Accumulator instance of the generalised Mira scheme for the degree-2
 * relation m1 o m2 - mu m3 = e over H (Sec. 4.2: acc.x = {C_i, E, mu}; the
 * relation has no public input or verifier challenges, so pi and r_i are
 * absent).  352 bytes; lives in device memory. */
typedef struct {
    zk_g1 C[4]; /* commitments to the interpolants of m_1..m_4 */
    zk_g1 E;    /* commitment to the interpolant of the error vector e */
    zk_fr mu;   /* slack scalar */
} zk_acc_inst;

/* Accumulator (Sec. 4.2: acc.w = {m_i, e} and acc.x).  All pointers are
 * DEVICE pointers: m[i] and e hold n evaluations over H each; x points to one
 * zk_acc_inst.  n is a power of two, 2 <= n <= 2^26. */
typedef struct {
    size_t n;
    zk_fr *m[4];
    zk_fr *e;
    zk_acc_inst *x;
} zk_acc;

/* Create a context on CUDA device `device` that may allocate at most
 * `hbm_budget_bytes` of device memory (0 = no limit).  *out receives the
 * context.  ZK_EINVAL for a null out or a bad device. */
int zk_init(zk_ctx **out, int device, size_t hbm_budget_bytes);

/* Release a context (or a lane) and everything it allocated.  Waits for the
 * device first.  A context must outlive its lanes. */
int zk_destroy(zk_ctx *ctx);

/* A lane shares the parent's SRS, window tables and twiddles (read only) and
 * owns its own scratch workspace, so calls on different lanes may overlap on
 * different streams.  Used by the serving loop. */
int zk_lane_create(zk_ctx *parent, zk_ctx **out);

/* Load the SRS [tau^0]_1 .. [tau^(n-1)]_1 (Sec. 2.1; the powers-of-tau
 * ceremony output).  Every point is checked to be canonical and on the curve
 * (cofactor 1, so on the curve means in the group); infinity is rejected.
 * ZK_EINVAL on a bad point, n == 0 or n > 2^26; the previous SRS is then
 * dropped.  Builds the window tables the MSM uses.  Synchronous. */
int zk_srs_load(zk_ctx *ctx, const zk_g1 *pts, size_t n);

/* Test-and-benchmark set-up: build the SRS [tau^i]_1, i < n, on the device
 * from a known trapdoor tau (host pointer).  A real deployment loads the
 * ceremony output with zk_srs_load instead; this exists because the paper's
 * workloads need SRSs up to 2^22 points and only the commitment, not its
 * setup, is on the prover's hot path.  Synchronous. */
int zk_srs_generate(zk_ctx *ctx, const zk_fr *tau, size_t n);

/* Number of SRS points loaded (0 if none). */
int zk_srs_size(const zk_ctx *ctx, size_t *n);

/* Copy SRS points [first, first + count) out in canonical affine form. */
int zk_srs_export(zk_ctx *ctx, zk_g1 *out, size_t first, size_t count, zk_stream stream);

/* KZG commitment of the polynomial with coefficients coeffs[0..n-1]:
 * *out = sum_i coeffs[i] * SRS[i] = [f(tau)]_1 (Sec. 2.1), by a signed-window
 * Pippenger MSM.  1 <= n <= SRS size (ZK_ESRS otherwise).  Coefficients must
 * be canonical (< r). */
int zk_commit(zk_ctx *ctx, const zk_fr *coeffs, size_t n, zk_g1 *out, zk_stream stream);

/* Allocation-free variant of zk_commit, for callers that cannot call
 * cudaMalloc (a host thread that must never block on the device-wide
 * synchronisation that cudaFree implies, or a process whose device memory is
 * all owned by another allocator).  The paper has no counterpart: this is a
 * deployment variant of the same commitment.
 *   coeffs, out : DEVICE pointers (ZK_EINVAL for host pointers); 1 <= n <= 4096
 *                 (ZK_EINVAL above that), n <= SRS size (ZK_ESRS otherwise).
 *   Workspace   : one fixed 15 MiB device array inside the library, shared by
 *                 every call; each GPU that loads the library holds it until
 *                 the process exits.  The call allocates nothing (no
 *                 cudaMalloc, cudaFree or allocating library routine) and
 *                 uses the window table built by zk_srs_load/zk_srs_generate.
 *   First call  : on each device, the first call looks up the array's device
 *                 address (cudaGetSymbolAddress); make that first call before
 *                 any stream capture.
 *   Concurrency : calls that overlap on the GPU (other streams, other host
 *                 threads) race on the shared array; serialise them.
 * The result equals zk_commit's bit for bit. */
int zk_commit_noalloc(zk_ctx *ctx, const zk_fr *coeffs, size_t n, zk_g1 *out, zk_stream stream);

/* Flags of zk_commit_batch. */
#define ZK_EVALS 1u    /* vectors are evaluations over H: commit to their interpolants, by
                          the context's route (zk_set_commit_route; default: INTT each one
                          on a workspace copy -- the caller's vectors are not modified --
                          then MSM over the SRS) */
#define ZK_LAGRANGE 2u /* vectors are evaluations over H: commit through the Lagrange basis
                          [L_k(tau)]_1 of H, with no INTT (same result as ZK_EVALS) */

/* KZG opening (Sec. 2.1): for f = sum_k coeffs[k] X^k (n >= 1 coefficients,
 * canonical; the quotient's n - 1 coefficients need an SRS of at least n - 1
 * points) and a point x:
 *   y = f(x),  quotient = (f(X) - y) / (X - x)  (n - 1 coefficients),
 *   proof = [quotient(tau)]_1  (the commitment of the quotient),
 * so that the verifier's pairing check e(proof, [tau - x]_2) =
 * e(com - [y]_1, [1]_2) holds.  coeffs and x may be device or host pointers;
 * y (32 bytes), proof (64 bytes, affine canonical) and quotient (optional,
 * NULL to skip) may be device or host pointers (host outputs are written
 * before the call returns; device outputs are stream-ordered).
 * Errors: ZK_EINVAL (null pointer, n = 0 or n > 2^31), ZK_ESRS (no SRS, or
 * n - 1 > SRS size), ZK_ENOMEM, ZK_ECUDA. */
int zk_open(zk_ctx *ctx, const zk_fr *coeffs, size_t n, const zk_fr *x, zk_fr *y, zk_g1 *proof,
            zk_fr *quotient, zk_stream stream);

/* Batch opening at one point (Sec. 2.1): ys[i] = f_i(x) for the count
 * polynomials polys[i] (lens[i] >= 1 coefficients each, device or host
 * pointers; `polys` and `lens` are host arrays), and one proof
 * [h(tau)]_1 with h(X) = sum_i gamma^i (f_i(X) - f_i(x)) / (X - x), the
 * quotient of sum_i gamma^i f_i.  x and gamma: one scalar each (device or
 * host); ys: count scalars; proof: 64 bytes (device or host).  Errors as for
 * zk_open, with max(lens) in place of n. */
int zk_open_batch(zk_ctx *ctx, const zk_fr *const *polys, const size_t *lens, size_t count, const zk_fr *x,
                  const zk_fr *gamma, zk_fr *ys, zk_g1 *proof, zk_stream stream);

/* Quotient of the Mul basic block, also MatMul's Q_l (Sec. 4.4.1): for
 * evaluation vectors a, b over H = <omega_n> (n a power of two, 1 <= n <= 2^27,
 * canonical scalars) with interpolants A, B, and L the interpolant of the
 * elementwise product a o b,
 *   t(X) = (A(X) B(X) - L(X)) / (X^n - 1)   (an exact division; n - 1
 *   coefficients, degree <= n - 2),
 * and com = [t(tau)]_1 (needs an SRS of at least n - 1 points).  a, b: device
 * or host; t (optional, NULL to skip; n - 1 scalars) and com (64 bytes): device
 * or host.  Errors: ZK_EINVAL (null pointer, n not a power of two or too
 * large), ZK_ESRS, ZK_ENOMEM, ZK_ECUDA. */
int zk_mul_quotient(zk_ctx *ctx, const zk_fr *a, const zk_fr *b, size_t n, zk_fr *t, zk_g1 *com,
                    zk_stream stream);

/* Degree of the relation that zk_leaf_init, zk_fold, zk_fold_tree and the
 * fold plans use (Sec. 4.2 folds relations of any degree d with d - 1 cross
 * terms):
 *   2 (default): m1 o m2 - mu m3 = e; leaves get m3 = m1 o m2 (m4 is folded
 *      linearly); one cross term E1.
 *   3: m1 o m2 o m3 - mu^2 m4 = e; leaves get m4 = m1 o m2 o m3 (m1, m2, m3
 *      given); two cross terms E1, E2, and
 *      e'' = e' + gamma e1 + gamma^2 e2 + gamma^3 e,
 *      E'' = E' + gamma E1 + gamma^2 E2 + gamma^3 E.
 * With degree 3, zk_fold's E1_out (when not NULL) receives E1 then E2
 * (128 bytes).  Shared by a context and its lanes; set it before building
 * plans or servers.  Errors: ZK_EINVAL (degree other than 2 or 3). */
int zk_set_fold_degree(zk_ctx *ctx, int degree);

/* Hiding commitments (the blinding in the zero-knowledge argument of the
 * accumulation scheme, Sec. 4.2: every KZG commitment gets an extra s H).
 * zk_set_hiding_base: sets the context's hiding base H (64 bytes, canonical
 * affine, device or host; must be on the curve and not infinity) and builds
 * its fixed-base table (256 KB of device memory); synchronous.  The base is
 * shared with the context's lanes; a failed call leaves no base set.
 * zk_commit_hiding: out = [f(tau)]_1 + s H for n >= 1 canonical coefficients
 * and one scalar s (the caller's random draw), all device or host pointers.
 * The paper draws H and s at random; the caller supplies both.
 * Errors: ZK_EINVAL (null pointer, n = 0, H off the curve, no base set),
 * ZK_ESRS, ZK_ENOMEM, ZK_ECUDA. */
int zk_set_hiding_base(zk_ctx *ctx, const zk_g1 *H);
int zk_commit_hiding(zk_ctx *ctx, const zk_fr *coeffs, size_t n, const zk_fr *s, zk_g1 *out,
                     zk_stream stream);

/* Route of evaluation-form commitments (ZK_EVALS, leaf accumulators, fold
 * cross terms).  ZK_ROUTE_INTT interpolates (INTT) and commits over the SRS,
 * as the paper's encoding describes (Sec. 3).  ZK_ROUTE_LAGRANGE commits the
 * evaluations directly over [L_k(tau)]_1 = n^{-1} sum_j omega^{-jk} [tau^j]_1,
 * a basis the library derives from the SRS once per size (an inverse DFT over
 * G1); the commitment is the same point, and quantised witness values stay
 * short scalars.  The route is shared by a context and its lanes. */
#define ZK_ROUTE_INTT 0
#define ZK_ROUTE_LAGRANGE 1
int zk_set_commit_route(zk_ctx *ctx, int route);

/* Commit `count` vectors in one batched pass: out[k] = commitment of vecs[k]
 * (lens[k] elements).  `vecs` is a host array of pointers (each device or
 * host) and `out` points to count zk_g1.  With ZK_EVALS a vector whose length
 * is not a power of two is zero-padded to the next power of two before the
 * INTT (Sec. 3 encodes each tensor's last axis as one polynomial). */
int zk_commit_batch(zk_ctx *ctx, const zk_fr *const *vecs, const size_t *lens, size_t count,
                    unsigned flags, zk_g1 *out, zk_stream stream);

/* In-place natural-order NTT: data[k] <- sum_j data[j] omega_n^{jk}.  n a power
 * of two, 1 <= n <= 2^28 (ZK_EINVAL otherwise). */
int zk_ntt(zk_ctx *ctx, zk_fr *data, size_t n, zk_stream stream);

/* In-place natural-order inverse NTT: data[j] <- n^{-1} sum_k data[k] omega_n^{-jk}
 * (evaluations over H to coefficients). */
int zk_intt(zk_ctx *ctx, zk_fr *data, size_t n, zk_stream stream);

/* Batched NTT / INTT of `count` device vectors of power-of-two lengths. */
int zk_ntt_batch(zk_ctx *ctx, zk_fr *const *data, const size_t *lens, size_t count, int inverse,
                 zk_stream stream);

/* Leaf accumulators from NARK witnesses (Sec. 4.2: a NARK proof is the
 * accumulator with mu = 1 and e = 0): for each of the `count` accumulators
 * (host array; all of one length n), given m1, m2, m4 in acc->m, writes
 * m3 = m1 o m2, e = 0, and acc->x = {C_i = Commit(INTT(m_i)), E = infinity,
 * mu = 1}.  The commitments of all leaves run as batched INTTs and MSMs. */
int zk_leaf_init(zk_ctx *ctx, const zk_acc *accs, size_t count, zk_stream stream);

/* One fold acc'' = fold(L, R, gamma) (Sec. 4.2, prover steps 2-7, d = 2, L in
 * the role of acc and R of acc'):
 *   e1  = m1 o m2' + m1' o m2 - mu m3' - mu' m3          (step 2)
 *   E1  = Commit(INTT(e1))                                 (step 3)
 *   m_i'' = gamma m_i + m_i',  e'' = e' + gamma e1 + gamma^2 e   (step 5)
 *   C_i'' = gamma C_i + C_i',  E'' = E' + gamma E1 + gamma^2 E,  mu'' = gamma mu + mu'.
 * `gamma` may be a host or device pointer; `out` may alias R (not L).  If
 * E1_out is not NULL it receives E1 (the correction term pf, step 7; with
 * zk_set_fold_degree 3, E1 then E2). */
int zk_fold(zk_ctx *ctx, const zk_acc *L, const zk_acc *R, const zk_fr *gamma, zk_acc *out,
            zk_g1 *E1_out, zk_stream stream);

/* Parallel fold tree (Sec. 4.2, tree reduction): count = 2^levels leaves; at
 * level l = 1..levels fold j combines the two level-(l-1) accumulators 2j (as
 * L) and 2j+1 (as R) with gammas[(count - count/2^(l-1)) + j] (level-major,
 * count - 1 challenges; host or device pointer).  All folds of one level run
 * as one batch.  The leaves' buffers are overwritten (used as the tree's
 * storage); the root is copied into *root (which must not alias a leaf).
 * Each level's instance combination (the G1 part) runs on the context's
 * internal side stream, created at the highest stream priority on first use.
 * It is forked from `stream` by an event and joined back before the root is
 * copied, so the call stays ordered on `stream` like any other. */
int zk_fold_tree(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, zk_acc *root,
                 zk_stream stream);

/* The first `levels` levels of the fold tree above (1 <= levels <= log2
 * count), for checkpointing: the tree's accumulators are the natural
 * checkpoint of the parallel accumulation (Sec. 4.2, tree reduction; each
 * level's accumulators carry everything the rest of the tree needs).  After
 * the call, level-`levels` accumulator j (j < count / 2^levels) is in
 * leaves[j 2^levels + 2^levels - 1]; gammas holds the first count -
 * count/2^levels challenges of the level-major array.  The caller may copy
 * those accumulators (m, e: device vectors; x: the instance) anywhere,
 * and later resume with zk_fold_tree over them and the remaining challenges
 * (gammas + count - count/2^levels), which gives the root of the whole tree.
 * Errors as zk_fold_tree; ZK_EINVAL for levels = 0 or > log2 count. */
int zk_fold_tree_levels(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas, size_t levels,
                        zk_stream stream);

/* Autotuning (the window width and bucket layout of the MSM and the largest
 * NTT pass radix, per length).  op = ZK_TUNE_MSM_WINDOW: value = window width c in [9, 20] for
 * MSMs of length in (2^(log2n-1), 2^log2n]; op = ZK_TUNE_NTT_RADIX: value =
 * log2 of the largest pass radix in [1, 11] for transforms of length 2^log2n.
 * value 0 restores the built-in choice (the winners of a tuning sweep on
 * B300); zk_tune_get returns the value in effect (tuned or built-in).
 * zk_tune_measure times one candidate on synthetic device data (median
 * of `reps` runs, ms) without changing the setting; the first use of a new
 * window width builds its window table (about W x 128 bytes per SRS point).
 * paper_2507_07031_b300/autotune.py sweeps the candidates and stores the
 * winners in a JSON table. */
#define ZK_TUNE_MSM_WINDOW 0
#define ZK_TUNE_NTT_RADIX 1
/* Bucket layout of the MSM, per length (value 0 = built-in):
 *   ZK_TUNE_MSM_CHUNK  : 1 + log2 of the round-0 chunk multiplier used when
 *                        few buckets (<= 4096) are in use, value in [1, 4];
 *   ZK_TUNE_MSM_TAIL   : 1 + log2 of the partial sums each lane adds in a
 *                        slice of the team tail (buckets of many partial
 *                        sums, e.g. quantised scalars), value in [1, 4];
 *   ZK_TUNE_MSM_SEG    : log2 of the bucket-reduction segment of levels with
 *                        fewer than 2^13 items, value in [3, 5];
 *   ZK_TUNE_MSM_SEGBIG : log2 of the segment of larger levels, in [6, 8].
 * zk_tune_measure times these on quantised int8 x 2^16 scalars (CHUNK,
 * TAIL, SEG) or uniform scalars (SEGBIG) through the default MSM path. */
#define ZK_TUNE_MSM_CHUNK 2
#define ZK_TUNE_MSM_TAIL 3
#define ZK_TUNE_MSM_SEG 4
#define ZK_TUNE_MSM_SEGBIG 5
int zk_tune_set(zk_ctx *ctx, int op, int log2n, int value);
int zk_tune_get(const zk_ctx *ctx, int op, int log2n, int *value);
int zk_tune_measure(zk_ctx *ctx, int op, int log2n, int value, int reps, double *ms);

/* Plans: a batched commitment or a fold tree captured once as a CUDA graph
 * and replayed with a single launch.  Every buffer must be a DEVICE pointer
 * (ZK_EINVAL otherwise) and stay valid, with the same shape, for the plan's
 * life; the inputs' contents may change between launches.  Creating a plan
 * synchronises the device, then runs the operation once (a warm-up that sizes
 * the plan's private workspace and builds the tables it needs), so it also
 * produces the result once.  A
 * plan holds a lane of `ctx` (its own workspace, shared SRS tables): it must
 * be destroyed before `ctx`, and reloading the SRS invalidates it.
 * zk_plan_launch enqueues the graph on `stream`; zk_plan_nodes reports the
 * graph's node count (kernels and copies). */
typedef struct zk_plan zk_plan;
int zk_plan_commit_batch(zk_ctx *ctx, const zk_fr *const *vecs, const size_t *lens, size_t count,
                         unsigned flags, zk_g1 *out, zk_plan **plan);
int zk_plan_fold_tree(zk_ctx *ctx, zk_acc *leaves, size_t count, const zk_fr *gammas,
                      zk_acc *root, zk_plan **plan);
int zk_plan_launch(zk_plan *plan, zk_stream stream);
int zk_plan_nodes(const zk_plan *plan, size_t *nodes);
int zk_plan_destroy(zk_plan *plan);

/* Serving loop with continuous batching.  A job commits to one basic-block
 * witness as a NARK leaf accumulator (INTT + MSM of each vector; Sec. 4.2:
 * a NARK proof is the accumulator with mu = 1, e = 0) and, if acc_in is set,
 * folds it into that resident accumulator: *acc_out = fold(*acc_in, *leaf,
 * gamma).  Jobs are admitted in arrival order as soon as one of the server's
 * lanes (private workspace + CUDA stream) is free and the job's workspace
 * estimate fits in the unreserved HBM budget; admitted jobs run concurrently.
 * Pointers in zk_job: w[] are DEVICE pointers; leaf, acc_in and acc_out
 * point to HOST zk_acc structs (the scheduler thread reads them) whose m, e
 * and x buffers are device memory; gamma may be host or device.  All are
 * owned by the caller and left untouched by it until the job is done; acc_in
 * is read only, so many jobs may share it.  The witnesses w[] are m1, m2, m4
 * for the degree-2 relation and m1, m2, m3 under zk_set_fold_degree 3 (the
 * remaining vector is derived by the leaf step); the degree in effect when
 * the scheduler starts a job applies to it, and the job's HBM reservation
 * covers its d - 1 cross terms.  zk_submit returns ZK_EBUSY when 65536 jobs
 * wait, ZK_ENOMEM when one job's estimate exceeds the budget; zk_cancel
 * takes a job out of the queue before it runs.  zk_wait
 * returns ZK_ETIMEOUT after timeout_ms.  Times are ms since server creation.
 * Every ticket stays queryable until zk_server_destroy, so the server keeps
 * a small record (about 200 bytes) per job submitted.  zk_server_create
 * leaves the calling thread's current device as it found it. */
typedef struct zk_server zk_server;
typedef struct {
    size_t n;               /* witness length, power of two <= SRS size */
    const zk_fr *w[3];      /* m1, m2, m4 evaluations (degree 3: m1, m2, m3); device */
    zk_acc *leaf;           /* host struct; receives the leaf accumulator in its device buffers */
    const zk_acc *acc_in;   /* host struct: resident accumulator to fold into, or NULL */
    zk_acc *acc_out;        /* host struct; receives fold(acc_in, leaf, gamma) */
    const zk_fr *gamma;     /* fold challenge */
} zk_job;
#define ZK_JOB_QUEUED 0
#define ZK_JOB_RUNNING 1
#define ZK_JOB_DONE 2
#define ZK_JOB_FAILED 3
#define ZK_JOB_CANCELLED 4
typedef struct {
    int status;       /* ZK_JOB_* */
    int error;        /* ZK_OK or the failing call's code */
    int lane;
    double submit_ms, start_ms, end_ms;
} zk_ticket_info;
typedef struct {
    unsigned long long completed;
    size_t queued;
    size_t reserved_bytes, peak_reserved_bytes;
    int busy_lanes;
    unsigned long long cancelled;
} zk_server_info;
int zk_server_create(zk_ctx *ctx, int lanes, size_t hbm_budget_bytes, zk_server **out);
int zk_submit(zk_server *srv, const zk_job *job, uint64_t *ticket);
int zk_poll(zk_server *srv, uint64_t ticket, zk_ticket_info *info);
int zk_wait(zk_server *srv, uint64_t ticket, int timeout_ms, zk_ticket_info *info);
int zk_server_stats(zk_server *srv, zk_server_info *info);
/* Cancel a job that is still queued: it leaves the queue unrun, its status
 * becomes ZK_JOB_CANCELLED (waiters return at once) and its buffers are
 * never touched.  ZK_EBUSY when the job was already admitted (running) or
 * has finished; ZK_EINVAL for an unknown ticket.  The paper has no serving
 * loop; this is part of the deployment wrapper around its prover steps. */
int zk_cancel(zk_server *srv, uint64_t ticket);
int zk_server_destroy(zk_server *srv);

/* Static description of an error code. */
const char *zk_strerror(int code);

/* Diagnostics (not part of the paper's method).
 * zk_kernel_launches: number of kernels this library has launched in the
 * process so far (every launch site counts itself).
 * zk_probe_rates: measures, on `device`, the issue rate of independent 32-bit
 * integer multiply-adds (IMAD/s, the integer roofline's ceiling) and the
 * throughput of this library's F_q Montgomery multiplication (products/s).
 * Takes a few milliseconds; synchronous. */
unsigned long long zk_kernel_launches(void);
int zk_probe_rates(int device, double *imad_per_s, double *fq_mul_per_s);

/* zk_probe_pipes: the issue rates the roofline of the integer kernels is
 * stated against, measured on `device` (synchronous; tens of milliseconds).
 * rates must hold ZK_NPROBES doubles, indexed by:
 *   ZK_PROBE_MAD_LO   mad.lo.u32 per second (independent chains; the IMAD
 *                     pipe's peak, the denominator of the reported fraction)
 *   ZK_PROBE_MAD_HI   mad.hi.u32 per second
 *   ZK_PROBE_MAD_WIDE mad.wide.u32 (64-bit addend) per second
 *   ZK_PROBE_MAD_PAIR mad.lo.cc.u32 + madc.hi.u32 pairs per second (one limb
 *                     product of a carry chain)
 *   ZK_PROBE_ADD_PAIR add.cc.u32 + addc.u32 pairs per second (integer ALU)
 *   ZK_PROBE_FQ_MUL   this library's F_q Montgomery products per second
 *   ZK_PROBE_FR_MUL   this library's F_r Montgomery products per second
 * Errors: ZK_EINVAL (null rates or bad device), ZK_ENOMEM, ZK_ECUDA. */
#define ZK_PROBE_MAD_LO 0
#define ZK_PROBE_MAD_HI 1
#define ZK_PROBE_MAD_WIDE 2
#define ZK_PROBE_MAD_PAIR 3
#define ZK_PROBE_ADD_PAIR 4
#define ZK_PROBE_FQ_MUL 5
#define ZK_PROBE_FR_MUL 6
#define ZK_NPROBES 7
int zk_probe_pipes(int device, double *rates);

/* Elementwise field arithmetic on canonical vectors (tests of the device
 * field code; the prover does not call it).  The paper has no counterpart:
 * it checks the F_q / F_r arithmetic every step of the hot path is built on
 * (BN254 fields, Sec. 6.1).
 *   field : ZK_FIELD_Q (base field q) or ZK_FIELD_R (scalar field r).
 *   op    : ZK_FOP_MUL out = a b, ZK_FOP_SQR out = a^2, ZK_FOP_INV out = a^-1
 *           (0 for 0), ZK_FOP_ADD out = a + b, ZK_FOP_SUB out = a - b,
 *           ZK_FOP_MULSUB out[i] = a[i] b[i] - a[n-1-i] b[n-1-i] (the
 *           difference of two products that point additions and doublings
 *           take for their Y coordinate; F_q reduces it once), ZK_FOP_MULC
 *           out = a b through the product by a constant with a precomputed
 *           quotient (the NTT's butterfly twiddles): floor(b 2^256 / p) is
 *           computed on the device, and element i's first operand is the
 *           representative a[i] + (i mod 4) p, so the inputs span [0, 4p),
 *           the range the NTT's lazy butterflies pass it; out is canonical.
 *   a, b, out : DEVICE pointers to n canonical 32-byte little-endian elements
 *           (< modulus; not checked); b is ignored by SQR and INV; out may
 *           alias a or b.  Stream-ordered on `stream`.
 * Errors: ZK_EINVAL (bad field/op, null or host pointer, n > 2^31),
 * ZK_ECUDA. */
#define ZK_FIELD_Q 0
#define ZK_FIELD_R 1
#define ZK_FOP_MUL 0
#define ZK_FOP_SQR 1
#define ZK_FOP_INV 2
#define ZK_FOP_ADD 3
#define ZK_FOP_SUB 4
#define ZK_FOP_MULSUB 5
#define ZK_FOP_MULC 6
int zk_field_op(int field, int op, const zk_fr *a, const zk_fr *b, zk_fr *out, size_t n, zk_stream stream);

/* Checked build.  Compiled with -DZK_CHECK (`python
 * paper_2507_07031_b300/build.py --check` writes libzkb300_check.so), the
 * kernels check the invariants their gathers and scatters rely on and, on a
 * failure, set a flag bit and skip the access instead of trapping:
 *   ZK_CHECK_SCALAR  a scalar >= r reached the MSM (a precondition of the API)
 *   ZK_CHECK_BUCKET  a bucket key outside its job's bucket range
 *   ZK_CHECK_ENTRY   a sorted-entry position outside its bucket
 *   ZK_CHECK_NTT_IDX an NTT gather or scatter outside the vector
 * zk_check_status synchronises the device, returns the flags raised since the
 * last call (then clears them) and *checked = 1 in the checked build (in the
 * normal build the checks compile to nothing: flags 0, *checked = 0).
 * The paper has no counterpart; this stands in for a memory sanitizer. */
#define ZK_CHECK_SCALAR 1u
#define ZK_CHECK_BUCKET 2u
#define ZK_CHECK_ENTRY 4u
#define ZK_CHECK_NTT_IDX 8u
int zk_check_status(zk_ctx *ctx, unsigned *flags, int *checked);

/* Phase timing: with timing on, each call brackets its phases with CUDA events
 * on its stream; zk_timing_read waits for them, adds up the device time (ms)
 * and interval count per phase since the last read, and clears the record. */
#define ZK_PHASE_MSM_SORT 0       /* recode + counting sort of bucket entries */
#define ZK_PHASE_MSM_ACCUM 1      /* bucket accumulation (mixed additions) */
#define ZK_PHASE_MSM_REDUCE 2     /* weighted bucket sums and output */
#define ZK_PHASE_NTT 3            /* all NTT / INTT passes */
#define ZK_PHASE_FOLD_WITNESS 4   /* cross term and witness RLC */
#define ZK_PHASE_FOLD_INSTANCE 5  /* instance RLC (G1 scalar multiplications) */
#define ZK_NPHASES 6
int zk_timing_enable(zk_ctx *ctx, int on);
int zk_timing_read(zk_ctx *ctx, double ms[ZK_NPHASES], unsigned long long count[ZK_NPHASES]);

#ifdef __cplusplus
}
#endif

#endif /* ZK_B300_H */
