/*
 * bnedge.h -- C ABI of the GB300 library for exact Bayesian-network edge
 * posteriors (Chen, Tian, Nikolova, Aluru, arXiv 1408.1664; built on
 * Koivisto's forward-backward dynamic program).
 *
 * Given m samples of n discrete variables, an in-degree bound d and the
 * order-modular prior of Eq. 4 (q_i = 1, rho_i(G) = exp(log_rho[|G|])), the
 * library returns P(u->v | D) for all n(n-1) ordered pairs (Eq. 11 divided by
 * P(D) = F(V), Algorithm 1) together with log P(D).  Every step runs in CUDA
 * kernels for sm_103a:
 *   1. BDeu local scores log B_i(G), |G| <= d, from bit-exact contingency
 *      counts (Eq. 6; Algorithm 1, step 1);
 *   2. A_i(S), the truncated upward zeta transform of B_i (Eq. 7,
 *      Definition 1, Algorithm 2);
 *   3. the forward sum F(S) (Eq. 9) and the backward sum R(S) (Eq. 10) over
 *      the subset lattice, level by level in popcount (Section 3.1.1);
 *   4. Gamma_v(G), the truncated downward zeta transform of
 *      F(S) R(V-{v}-S) (Eq. 12, Definition 2, Algorithm 3);
 *   5. the edge reduction of Eq. 11 and the division by P(D).
 *
 * Conventions used by every entry point:
 *   - variable i (0-based) is bit i of a subset mask (the paper's variable
 *     i+1 is bit i, Section 3.1.1);
 *   - data is m x n row-major uint8 with data[s*n + i] < arity[i];
 *   - the families of node i are the parent sets G of V-{i} with |G| <= d,
 *     ordered by |G| and then by increasing mask value; K(n,d) =
 *     sum_{k<=d} C(n-1,k) families per node; per-family arrays are laid out
 *     [i*K + f];
 *   - the parent configuration of a family is a mixed-radix number with the
 *     lowest-numbered parent least significant; cell = config*r_i + x_i;
 *   - post is n x n row-major, post[u*n + v] = P(u->v | D), diagonal 0;
 *   - an in-degree bound d > n-1 is treated as d = n-1;
 *   - limits: 1 <= n <= 32, d >= 0, m >= 0 (m = 0 is valid input),
 *     1 <= arity[i] <= 255, at most 65536 cells (q*r_i) per family.
 *
 * Errors: every function returns BN_OK (0) or a negative BN_E* code and never
 * throws or aborts (a failed host allocation inside the library returns
 * BN_ENOMEM).  bn_strerror() names a code.  On error the output
 * buffers are left unspecified.
 *
 * Ownership: the caller owns every buffer it passes.  The context owns all
 * device memory it allocates (workspace grown on demand and kept for reuse).
 * A context is used by one host thread at a time.
 */
#ifndef BNEDGE_H
#define BNEDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BN_OK = 0,
    BN_EINVAL = -1,          /* invalid argument or input data               */
    BN_ENOMEM = -2,          /* device or host memory budget exceeded        */
    BN_EAGAIN = -3,          /* job not finished yet (bn_poll)               */
    BN_ETIMEOUT = -4,        /* bn_wait timed out                            */
    BN_EDEVICE_TIMEOUT = -5, /* a bounded device-side wait gave up           */
    BN_ECUDA = -6,           /* a CUDA runtime call failed                   */
    BN_ECANCELED = -7,       /* job canceled                                 */
    BN_ENOTFOUND = -8        /* unknown job id                               */
};

enum {
    BN_FP64 = 0,         /* every DP array in FP64, natural-log domain        */
    BN_FP32_SHIFTED = 1  /* DP arrays in FP32 log2 domain, each node's scores
                            shifted by their FP64 maximum; scores, P(D) and the
                            final division stay FP64                          */
};

typedef struct bn_ctx bn_ctx;

typedef struct bn_ctx_opts {
    int32_t device;          /* CUDA device ordinal                           */
    int32_t slots;           /* concurrent jobs for bn_submit (>= 1)          */
    uint64_t mem_budget;     /* device bytes the context may hold; 0 = 90% of
                                the free memory at creation                   */
    int32_t fail_alloc_after;/* test hook: allocations after this many fail
                                with BN_ENOMEM; < 0 disables                  */
    int32_t flags;           /* BN_CTX_* bits, 0 = defaults                   */
} bn_ctx_opts;

/* bn_ctx_opts.flags: BN_CTX_NO_AUTOTUNE, batches keep the default schedule
 * (and a persistent launch keeps clusters of 8 blocks) instead of timing the
 * alternatives; BN_CTX_CLUSTER_STEP3, every FP32 batch group with n >= 5
 * runs step 3 in the persistent cluster kernel whatever the timing says;
 * BN_CTX_GRAPH_BATCH, batches run as a graph of launches instead of one
 * persistent launch (see bn_batch_create; CLUSTER_STEP3 implies it). */
#define BN_CTX_NO_AUTOTUNE 1
#define BN_CTX_CLUSTER_STEP3 2
#define BN_CTX_GRAPH_BATCH 4

typedef struct bn_job_desc {
    int32_t n;               /* number of variables                           */
    int32_t d;               /* in-degree bound                               */
    int32_t m;               /* number of samples                             */
    int32_t precision;       /* BN_FP64 or BN_FP32_SHIFTED                    */
    const uint8_t* data;     /* m*n bytes, host or device (data_on_device)    */
    const uint8_t* arity;    /* n bytes, host                                 */
    double ess;              /* BDeu equivalent sample size (> 0)             */
    const double* log_rho;   /* d+1 host doubles: log prior per parent-set
                                size; NULL = all zero                         */
    int32_t data_on_device;  /* nonzero: data is a device pointer             */
    int32_t reserved;
    const double* log_q;     /* n*n host doubles or NULL: the order prior's
                                log q_i(S) (Eq. 4, entering A_i in Eq. 7 and
                                Gamma_v in Eq. 12) as a function of |S|: row
                                i, column |S| = 0..n-1; NULL = all zero       */
    const double* log_w;     /* n*K host doubles or NULL: a log weight per
                                family (i, G), canonical family order, added
                                to log B_i(G) -- a general rho_i(G) (Eq. 4)
                                beside the per-size log_rho; NULL = all zero  */
} bn_job_desc;
/* log_q and log_w accept -inf (a zero factor; it is held as -1e7 nats,
 * whose exponential, and that of every sum it enters, is exactly 0); NaN or
 * +inf give BN_EINVAL.  Batches and
 * bn_edge_posteriors_static reject a job that sets either (BN_EINVAL).  If
 * every parent set of some node has weight zero, P(D) = 0 and the
 * posteriors are undefined. */

typedef struct bn_stats {
    double ms_scores;        /* device time of each stage, CUDA events on the
                                launching stream                              */
    double ms_upzeta;        /* step 2: all of its launches                   */
    double ms_forward;       /* all F level launches                          */
    double ms_backward;      /* all R' level launches                         */
    double ms_gamma_p1;      /* sum over v of the Gamma phase-1 launches      */
    double ms_gamma_p2;      /* sum over v of the Gamma phase-2 launches      */
    double ms_edges;         /* edge reduction and division                   */
    double ms_total;         /* first kernel to last kernel                   */
    double cells;            /* n * 2^n                                       */
    double alg_bytes;        /* algorithmic HBM bytes of the DP arrays        */
    int32_t kernels;         /* kernel launches of the job                    */
    int32_t precision;
    double ms_upzeta_sums;   /* the part of ms_upzeta spent before the tile
                                butterflies (score reordering and column sums
                                of the 13-dimension tiles; 0 for n < 14)      */
} bn_stats;

/* Context.  bn_ctx_create returns BN_EINVAL for a NULL pointer or bad
 * options, BN_ECUDA when the device cannot be used. */
int bn_ctx_create(bn_ctx** ctx, const bn_ctx_opts* opts /* NULL = defaults */);
int bn_ctx_destroy(bn_ctx* ctx);

/* Number of families per node, K(n, d) = sum_{k<=min(d,n-1)} C(n-1, k);
 * 0 for invalid n or d. */
int64_t bn_num_families(int32_t n, int32_t d);

/* Device bytes one job needs (its DP arrays A, F, R', the Gamma scratch and
 * the score tables; A alone is n * 2^(n-1) values).  bn_submit admits a job
 * only while the sum of the footprints of the jobs it runs stays within the
 * context's budget.  BN_EINVAL for an invalid job. */
int bn_job_footprint(const bn_job_desc* job, uint64_t* bytes);

/* Step 1 only (Eq. 6, Algorithm 1 step 1): parent_mask[i*K+f] and
 * log_B[i*K+f] (FP64, natural log, including log_rho) on the host.  Blocks
 * until done. */
int bn_scores(bn_ctx* ctx, const bn_job_desc* job, uint32_t* parent_mask,
              double* log_B);

/* The posterior of one modular feature f(G) = prod_i f_i(G_i) (Section 2.2,
 * Eqs. 5-9): P(f, D) = F^f(V) from the forward recursion (Eq. 9) over the
 * A^f_i of Eq. 7 with B_i(G) f_i(G) in place of B_i(G), and
 * P(f | D) = P(f, D) / P(D).  log_f: n*K host doubles, log f_i(G) for family
 * f of node i in canonical order (0 for an indicator that is 1, -inf where
 * it is 0; any other log weight is allowed).  Outputs: *p = P(f | D) and
 * *log_PfD = log P(f, D) (natural log; either may be NULL).  Steps 1-3 run
 * twice (F only, no R', Gamma or edges).  Blocks until done.  BN_EINVAL for
 * a NULL ctx, job or log_f, an invalid job or a NaN / +inf in log_f. */
int bn_feature_posterior(bn_ctx* ctx, const bn_job_desc* job, const double* log_f, double* p,
                         double* log_PfD);

/* Steps 1-5 (Algorithm 1).  post: n*n host doubles; log_PD: host double or
 * NULL.  Blocks until the result is in the host buffers.
 *
 * Jobs larger than the device budget (this and bn_edge_posteriors_async):
 * when a job's arrays exceed the context's mem_budget, A (Eq. 7, the
 * n 2^(n-1) values that dominate) moves to one managed allocation: as much
 * of it as the budget leaves beside the other arrays is kept in device
 * memory, the rest in host memory, which the kernels read and write in place
 * over the CPU-GPU link (the same kernels and order: the results equal the
 * in-core run bit for bit, only slower).  BN_ENOMEM when the other arrays
 * alone exceed the budget or the host part exceeds 3/4 of the host memory
 * available.  This is how n = 32 runs on one GB300 (FP32: A is 275 GB). */
int bn_edge_posteriors(bn_ctx* ctx, const bn_job_desc* job, double* post,
                       double* log_PD);

/* Steps 1-5 enqueued on `stream` (a cudaStream_t, NULL = the context's own
 * stream) without host synchronisation.  post_dev: n*n device doubles;
 * log_PD_dev: one device double or NULL.  job->data may be host or device;
 * a host copy is taken before return.  The context's workspace is reused by
 * the next call on the same context: calls on one context are ordered by
 * the caller (same stream, or synchronise in between). */
int bn_edge_posteriors_async(bn_ctx* ctx, const bn_job_desc* job,
                             double* post_dev, double* log_PD_dev,
                             void* stream);

/* No-allocation variant of bn_edge_posteriors_async.  The paper has no
 * counterpart.  It serves callers that cannot let a library allocate device
 * memory: host applications that own and partition all GPU memory
 * themselves (a library may not take memory behind their back), and
 * latency-sensitive loops that cannot pay for cudaMalloc or for the
 * device-wide synchronisation of cudaFree.
 *
 * Needs no context.  Every intermediate array lives in one file-scope device
 * array of BN_STATIC_SCRATCH_BYTES (64 MiB) that every GPU loading this
 * library holds until the process exits.  Jobs whose arrays do not fit it
 * (roughly n > 19 on the FP64 path, n > 20 on the FP32 path) are rejected
 * with BN_ENOMEM before any GPU work; so are jobs whose arities give more
 * than 1024 distinct lgamma-table denominators or more than 1024 distinct
 * (product of parent arities, number of parents) pairs (two fixed host
 * tables; only jobs with many distinct arities come near them).  log_q and
 * log_w are not accepted (BN_EINVAL).  Runs on the current device, enqueued
 * on `stream` (a cudaStream_t, NULL = the legacy default stream).  The first
 * call on a device looks up the array's device address for that device (a
 * one-time set-up; make that first call before any stream capture begins).
 * job->data may be host or device memory (host data and the small tables are
 * copied with cudaMemcpyAsync from pageable memory, which has consumed the
 * host bytes when the call returns); post_dev (n*n doubles) and log_PD_dev
 * (one double, or NULL) are device memory owned by the caller.  Host data is
 * checked on the host (BN_EINVAL).  Device data is checked only on the GPU:
 * since the call never synchronises, a value not below its arity makes every
 * posterior and log P(D) NaN instead of returning an error code.  All calls
 * on a device share the array and it keeps the previous call's contents:
 * calls whose GPU work may overlap (different streams without ordering) race
 * and give undefined results. */
#define BN_STATIC_SCRATCH_BYTES (64u << 20)
int bn_edge_posteriors_static(const bn_job_desc* job, double* post_dev,
                              double* log_PD_dev, void* stream);

/* Batches.  Many independent jobs (typically small n) planned together
 * (Algorithm 1 for each job; the paper has no batch form).
 * bn_batch_create validates every job and copies its host inputs into one
 * device arena.  Jobs with equal n, d, precision and kind of data (every
 * arity 2, or not) form a group: their arrays lie at a fixed stride in a
 * layout padded to the group's largest m, arity and lgamma table, and every
 * launch of steps 1-5 covers the whole group.
 * Unless the context has BN_CTX_NO_AUTOTUNE, the schedule of each group --
 * the kernel of the scores (one lane per 64-sample word or one lane per
 * parent configuration, non-binary data), of the up-zeta (13-dimension
 * tiles or shared-memory tiles), of F and R' (16-subset rows or warp tiles,
 * FP32; then one launch per popcount level or one persistent launch of
 * thread-block clusters, each cluster taking F or R' of one job at a time
 * and running all its levels between cluster barriers) and of the down-zeta
 * phase 1 -- is chosen by timing: the groups run at the same time, so the
 * autotuner times the whole batch on its own data, switching one kernel
 * choice at a time for all groups, the groups with n <= 14 or those with
 * n > 14, and keeps a switch that makes the batch more than 1% faster.  The
 * choices are cached in the context; a later batch whose group shapes are
 * all cached takes them without timing.  Every schedule gives the same
 * values up to rounding (within the stated tolerances, 1e-9 FP64 and 1e-4
 * FP32, of the job run alone; equal bit for bit under the default schedule
 * and with the cluster kernel).  The batch then exists in two forms: the
 * launches of all groups recorded into one CUDA graph, one branch per
 * group; and, unless the context has BN_CTX_GRAPH_BATCH or
 * BN_CTX_CLUSTER_STEP3, one persistent launch per precision that runs the
 * same kernels, in the same order per job, from a device work queue: one
 * item per block of every recorded launch, ordered by stage depth, each
 * item waiting (by bounded polls of a per-launch completion counter) for
 * the launch before it in its job's chain.  With autotuning the faster form
 * on this batch is kept (both are timed; bn_batch_describe reports both
 * times), without it the persistent form.  A wait that exceeds its bound
 * sets an abort flag: every block stops taking items and the batch reports
 * BN_EDEVICE_TIMEOUT from bn_batch_results / bn_batch_download.  bn_batch_run
 * runs the chosen form on `stream` (NULL = the context's stream) without host
 * synchronisation: one graph launch or one kernel launch per precision runs
 * the whole batch.  bn_batch_results
 * waits for the last run and copies job k's posteriors (n*n doubles) and
 * log P(D).  Device data pointers are not accepted (BN_EINVAL).  The arena
 * counts against the context's budget (BN_ENOMEM). */
typedef struct bn_batch bn_batch;
int bn_batch_create(bn_ctx* ctx, const bn_job_desc* jobs, int32_t count, bn_batch** batch);
int bn_batch_run(bn_batch* batch, void* stream);
int bn_batch_results(bn_batch* batch, int32_t k, double* post, double* log_PD);
/* New data for every job of the batch, in job order (count = the batch's
 * job count): the same n, d, m, arities, precision, ess and log_rho as at
 * bn_batch_create (BN_EINVAL otherwise, or for a value not below its arity;
 * host data only).  The data go through one pinned staging buffer and one
 * host-to-device copy into the batch's arena, enqueued on `stream` (NULL =
 * the context's stream) without host synchronisation; the next bn_batch_run
 * on that stream computes on them.  The caller's buffers may be reused when
 * the call returns. */
int bn_batch_upload(bn_batch* batch, const bn_job_desc* jobs, int32_t count, void* stream);
/* Every job's results at once after bn_batch_run: post_all receives the
 * jobs' n*n posteriors one after another in job order (sum of n_k^2
 * doubles), log_PD_all (NULL allowed) one log P(D) per job.  One gather
 * launch and one device-to-host copy; waits for the last run.  BN_EINVAL if
 * some job's device-side input check failed, BN_EDEVICE_TIMEOUT if the
 * persistent launch gave up a wait. */
int bn_batch_download(bn_batch* batch, double* post_all, double* log_PD_all);
/* One line per group into buf (NUL-terminated, truncated to len): its n, d,
 * precision, kind of data, jobs and the schedule it runs, and whether that
 * was timed.
 * BN_EINVAL for NULL arguments. */
int bn_batch_describe(bn_batch* batch, char* buf, size_t len);
int bn_batch_destroy(bn_batch* batch);

/* Shards: one job split over W = 2^k ranks (one GPU each, k <= n - 4 on
 * the FP32 path, n - 3 on the FP64 path; the paper runs everything on one
 * device and has no split).  The split follows Section 3.1.1's level order:
 * the subsets S are grouped into tiles by their top n - 4 (FP32) or n - 3
 * (FP64) variables, and the top k of those fix the rank, so rank r computes
 * the tiles whose top k bits equal r, at every popcount level, and holds the
 * full 2^n arrays of A, F and R'.
 *
 *   bn_shard_create   validates the job (host data or device data of this
 *                     rank's device; no batch restrictions) and allocates
 *                     the rank's arrays (counted in the context's budget);
 *                     BN_EINVAL when W is not a power of two up to 32, rank
 *                     is out of range or W is too large for n.  flags:
 *                     0, or BN_SHARD_DIVIDE_A (below);
 *   bn_shard_prepare  uploads the inputs and runs steps 1-2 (scores and A,
 *                     Eq. 6-7).  Without BN_SHARD_DIVIDE_A every rank
 *                     computes all of A (read by every tile; computing it
 *                     costs less than moving it).  With it, a rank holds
 *                     only the entries its tiles read: for the low
 *                     n - k variables the A_i(S) whose top k variables are
 *                     the rank's bits, for each top variable t its A_t over
 *                     the subsets of the low variables plus the rank's
 *                     other top bits -- about (n + k) 2^(n-1-k) values
 *                     instead of n 2^(n-1).  It computes them with no
 *                     exchange, as truncated zeta transforms over the low
 *                     variables of the score table folded over the rank's
 *                     top bits (every rank holds the small score table).
 *                     It needs n - k >= 14 and no order prior (BN_EINVAL);
 *                     results agree with the whole job to rounding
 *                     (the folded sums add in another order), and the
 *                     down-zeta runs without its relevance cut;
 *   bn_shard_bytes    the device bytes the shard holds;
 *   bn_shard_level    computes level hl (0..H, H = n - 4 FP32 / n - 3 FP64)
 *                     of the forward sum F (sweep 0, Eq. 9; hl = 0..H in
 *                     turn) or of R'(T) = R(V - T) (sweep 1, Eq. 10;
 *                     hl = H..0) for this rank's tiles;
 *   bn_shard_exchange_bytes  the size of one rank's exchange buffer of
 *                     level hl (the same on every rank): a 16-byte header
 *                     and the largest rank's rows;
 *   bn_shard_pack     writes this rank's level-hl rows (and, FP32, the
 *                     level's floored maximum, the per-level base the FP32
 *                     arrays are stored against) into a device buffer;
 *   bn_shard_unpack   stores rank `from`'s packed level-hl rows into this
 *                     rank's arrays and takes the maximum of the level
 *                     words (from == this rank: nothing to do);
 *   bn_shard_finish   runs steps 4-5 (Eq. 11-12) for the endpoints v with
 *                     v mod W = rank (its down-zeta scratch is sized for
 *                     those endpoints only): post_dev (n*n device doubles) gets
 *                     those columns and zeros elsewhere, log_PD_dev (NULL
 *                     allowed) log P(D).  The sum over ranks of post_dev is
 *                     the job's posterior matrix.
 *
 * Every level of a sweep must be packed by every rank and unpacked by every
 * rank before any rank computes the next level of that sweep (an
 * all-gather per level; the two sweeps are independent of each other), and
 * both sweeps must be complete before bn_shard_finish.  The caller moves
 * the buffers (NCCL all-gather, or device copies between contexts); the
 * library does no communication.  Every call is enqueued on `stream` (NULL =
 * the context's stream) without host synchronisation.  Without
 * BN_SHARD_DIVIDE_A the result equals the job run whole, bit for bit: every
 * tile is computed from the same values in the same order. */
typedef struct bn_shard bn_shard;
#define BN_SHARD_DIVIDE_A 1
int bn_shard_create(bn_ctx* ctx, const bn_job_desc* job, int32_t rank, int32_t world,
                    int32_t flags, bn_shard** shard);
int bn_shard_bytes(const bn_shard* shard, uint64_t* bytes);
int bn_shard_prepare(bn_shard* shard, void* stream);
int bn_shard_level(bn_shard* shard, int32_t sweep, int32_t hl, void* stream);
int bn_shard_exchange_bytes(const bn_shard* shard, int32_t hl, uint64_t* bytes);
int bn_shard_pack(bn_shard* shard, int32_t sweep, int32_t hl, void* buf_dev, void* stream);
int bn_shard_unpack(bn_shard* shard, int32_t sweep, int32_t hl, int32_t from,
                    const void* buf_dev, void* stream);
int bn_shard_finish(bn_shard* shard, double* post_dev, double* log_PD_dev, void* stream);
int bn_shard_destroy(bn_shard* shard);

/* Serving.  bn_submit copies the inputs, admits the job when a slot and
 * enough device memory (by its n*2^n footprint) are free -- queuing it
 * otherwise -- and returns at once.  Jobs in different slots run
 * concurrently on separate streams.  BN_ENOMEM if the job can never fit the
 * budget. */
int bn_submit(bn_ctx* ctx, const bn_job_desc* job, uint64_t* job_id);
/* BN_OK with the result copied out and the job retired, BN_EAGAIN while it
 * runs or waits, or the job's error code. */
int bn_poll(bn_ctx* ctx, uint64_t job_id, double* post, double* log_PD);
/* Like bn_poll but blocks up to timeout_s seconds (BN_ETIMEOUT). */
int bn_wait(bn_ctx* ctx, uint64_t job_id, double timeout_s, double* post,
            double* log_PD);
/* Cancels a queued job (BN_OK) or reports that it already runs. */
int bn_cancel(bn_ctx* ctx, uint64_t job_id);
/* Stage timings of a job run by bn_edge_posteriors (job_id 0 = the last
 * such call) or of a retired served job. */
int bn_job_stats(bn_ctx* ctx, uint64_t job_id, bn_stats* stats);
/* Stage timings of the most recent bn_edge_posteriors / _async calls on this
 * context (up to 32 are kept), oldest first: writes min(max, kept) entries
 * and their number to *count.  Waits for those calls to finish. */
int bn_stats_history(bn_ctx* ctx, bn_stats* out, int32_t max, int32_t* count);

const char* bn_strerror(int code);

/* ---- test hooks: stage dumps of the last bn_edge_posteriors call ------- *
 * Declared and exported only in the testing build of the library (compiled
 * with BN_TESTING defined: _build/libbnedge_testing.so); the release build
 * (_build/libbnedge.so) has neither function. */
#ifdef BN_TESTING
enum {
    BN_STAGE_LOGB = 1,   /* n*K doubles, natural log, unshifted               */
    BN_STAGE_MASKS = 2,  /* n*K uint32 parent masks                           */
    BN_STAGE_SHIFT = 3,  /* n doubles: c_i = max_f log_B[i*K+f]               */
    BN_STAGE_A = 4,      /* n*2^(n-1) values: A_i(S) - c_i at index
                            i*2^(n-1) + (S with bit i removed)                */
    BN_STAGE_F = 5,      /* 2^n values: F(S) - sum_{j in S} c_j               */
    BN_STAGE_RC = 6,     /* 2^n values: R(V-T) - sum_{j not in T} c_j at T    */
    BN_STAGE_GAMMA = 7   /* n*K values: Gamma_v(G) - sum_{j != v} c_j         */
};
/* Copies a stage array of the last job into host memory.  DP arrays are
 * doubles (natural log) for BN_FP64 and floats (log2) for BN_FP32_SHIFTED;
 * `bytes` must equal the stage size.  BN_EINVAL otherwise.  For n >= 14 a
 * Gamma_v(G) whose B_v(G) Gamma_v(G) lies more than 64 (FP64) or 24 (FP32)
 * + log2(K 2^(n-14)) bits below F(V) may hold a floor value instead (it moves
 * no posterior by more than 2^-64, resp. 2^-24, in all). */
int bn_debug_stage(bn_ctx* ctx, int32_t stage, void* host_out, size_t bytes);
/* Contingency counts of one family computed by the device counting routine:
 * counts[config*r_i + x_i], q*r_i int64 values on the host. */
int bn_debug_counts(bn_ctx* ctx, const bn_job_desc* job, int32_t i,
                    uint32_t parent_mask, int64_t* counts, int64_t cells);
/* The persistent batch form with a stage missing: every work item of the
 * launches at position `depth` of each group's launch sequence is removed
 * from the queue (their results never come) and every device-side wait gives
 * up after `polls` polls, so the next bn_batch_run ends early and
 * bn_batch_results returns BN_EDEVICE_TIMEOUT.  BN_EINVAL if the batch does
 * not run in the persistent form. */
int bn_debug_batch_drop(bn_batch* batch, int32_t depth, uint64_t polls);
/* The bounded wait of the persistent up-zeta tile kernel (FP32, n >= 14):
 * one block runs with its first bulk copy of column sums withheld, so its
 * mbarrier wait gives up after `polls` polls; *err_word receives the job
 * error word that the kernel leaves (2: a device-side wait gave up, the
 * value that makes a job return BN_EDEVICE_TIMEOUT).  The block returns
 * without a fault and the context stays usable. */
int bn_debug_copy_wait(uint32_t polls, int32_t* err_word);
/* Index checks.  The BN_CHECK_BOUNDS build of the library
 * (_build/libbnedge_checked.so, a debug build with the test hooks) checks
 * the global-memory offsets its kernels form -- rows of A, F and R', the
 * down-zeta gathers and outputs, the column sums, the score and Gamma
 * outputs, the packed levels of a split job -- against their arrays'
 * sizes; a failing access records its source line and goes to offset 0
 * instead (no fault, no trap).  This call waits for the device and returns
 * the first failure since the last call: *unit = 1 (bn_kernels.cu),
 * 2 (bn_tile13.cu), 3 (bn_levels.cu) or 4 (bn_mega.cu) and *line its source
 * line, or both 0 when every check passed.  In the other builds *line = -1
 * (no checks compiled). */
int bn_debug_bounds(int32_t* line, int32_t* unit);
/* The FP64 path's table-driven exp and log (after Tang's method) beside
 * CUDA's own exp and log, evaluated on the current device for `count`
 * host doubles x: out (4 * count host doubles) receives, per x, the
 * library's exp, CUDA's exp, the library's log, CUDA's log. */
int bn_debug_explog(const double* x, int64_t count, double* out);
#endif /* BN_TESTING */

#ifdef __cplusplus
}
#endif

#endif /* BNEDGE_H */
