/*
 * rrs.h - C ABI of the GB300 library for Refined Random Search (RRS)
 * projection depths (arXiv 2506.08262, "Massive parallelization of
 * projection-based depths").
 *
 * The library computes, for every query point z of a batch and a resident
 * data cloud X (n x d), the RRS approximation of a depth that satisfies the
 * projection property (Def. 2): the minimum over r rounds of m = ceil(k/r)
 * directions u of the univariate depth D(u'z | u'X) (Sec. 2), where round 1
 * draws directions uniformly on the sphere and round l >= 2 draws them in a
 * spherical cap of angle (pi/2) alpha^(l-1) around the best direction found
 * so far (Alg. 1, Alg. 4, Alg. S3, Alg. S4).
 *
 * All compute runs on one CUDA device in hand-written sm_103a kernels; there
 * is no CPU fallback.  Pointers are plain host or device addresses as each
 * argument states; no framework types cross this boundary.  Every function
 * returns an rrs_status (0 = success, negative = error) and never throws.
 * rrs_status_string() turns a status into text and rrs_last_error() gives
 * the detail of the last failure on the calling thread.
 *
 * Thread safety: a context may be used from one host thread at a time.
 */
#ifndef RRS_H
#define RRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rrs_ctx rrs_ctx;
typedef int32_t rrs_status;

/* Status codes. */
#define RRS_OK 0
#define RRS_ERR_INVALID_ARG (-1) /* bad size, kind, k < r, alpha outside (0,1], non-finite data */
#define RRS_ERR_NOT_FOUND (-2)   /* unknown dataset id */
#define RRS_ERR_BUDGET (-3)      /* the context's device-memory budget would be exceeded */
#define RRS_ERR_CUDA (-4)        /* a CUDA runtime call failed (see rrs_last_error) */
#define RRS_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define RRS_ERR_INTERNAL (-6)    /* an internal invariant failed */
#define RRS_ERR_UNSUPPORTED (-7) /* valid request the library cannot serve (e.g. d too large) */

/* Element types of X and Z. */
#define RRS_F32 0
#define RRS_F64 1

/* Depth notions (Sec. 2). */
#define RRS_HALFSPACE 0        /* D_H = min(#{y <= y_z}, #{y >= y_z}) / n, closed halfspaces */
#define RRS_PROJECTION 1       /* D_P = 1 / (1 + |y_z - med| / MAD), MAD unscaled */
#define RRS_ASYM_PROJECTION 2  /* D_AP = 1 / (1 + (y_z - med)_+ / MAD_+) */

/* Projection arithmetic. */
#define RRS_PREC_FP32_SIMT 0     /* FP32 dot products on the CUDA cores */
#define RRS_PREC_SPLIT_BF16X3 1  /* halfspace only: tcgen05 tensor cores, x*u as
                                    x_hi u_hi + x_hi u_lo + x_lo u_hi (BF16 parts),
                                    FP32 accumulation */

/*
 * rrs_create - open a context on CUDA device `device`.
 *   hbm_budget_bytes: upper bound on the device memory the context may hold
 *   for datasets and per-call workspace; 0 means no bound.
 *   *out receives the context.  Errors: INVALID_ARG (out NULL, bad device),
 *   CUDA.
 */
rrs_status rrs_create(rrs_ctx** out, int32_t device, uint64_t hbm_budget_bytes);

/* rrs_destroy - free every dataset and workspace of the context, then the
 * context.  NULL is accepted.  Work already queued by the context is
 * synchronised first.  Always returns RRS_OK. */
rrs_status rrs_destroy(rrs_ctx* ctx);

/*
 * rrs_register_dataset - copy a data cloud X into device memory and keep it
 * resident (the paper's X, Sec. 2).
 *   X: n x d row-major array of `dtype` (RRS_F32 or RRS_F64), on the device
 *      if x_on_device != 0, else on the host.  The caller keeps ownership;
 *      the library copies it and never reads X after returning.
 *   n >= 1, 1 <= d <= 1024.  Every entry must be finite and of magnitude
 *   below 2^64 (checked: INVALID_ARG).
 *   *dataset_id_out receives a positive id valid until rrs_free/rrs_destroy.
 * Errors: INVALID_ARG, BUDGET, CUDA.  Synchronous.
 */
rrs_status rrs_register_dataset(rrs_ctx* ctx, const void* X, int64_t n, int32_t d, int32_t dtype,
                                int32_t x_on_device, int64_t* dataset_id_out);

/* rrs_free - release a registered dataset.  Errors: NOT_FOUND. */
rrs_status rrs_free(rrs_ctx* ctx, int64_t dataset_id);

/*
 * rrs_depth - RRS depth of every query of a batch (Alg. 4 run for each row of
 * Z; rows are independent).
 *   Z: n_queries x d row-major array of `dtype` (same d as the dataset), on
 *      the device if z_on_device != 0.  n_queries may be 0 (no work).
 *   kind: RRS_HALFSPACE, RRS_PROJECTION or RRS_ASYM_PROJECTION.
 *   n_dirs (k) >= n_refinements (r) >= 1; m = ceil(k/r) directions per round.
 *   cap_shrink (alpha) in (0, 1]; it is rounded to FP32 before use.
 *   seed keys the Philox4x32-10 direction stream; query row q of this call
 *   uses counter (block, j, l-1, q), so each result depends only on
 *   (X, z, q, kind, k, r, alpha, seed) and not on what else is batched.
 *   precision: RRS_PREC_FP32_SIMT, or RRS_PREC_SPLIT_BF16X3 for halfspace
 *   depth.  Halfspace counts are exact either way: every point whose fast
 *   projection lies in the near-tie band |u'x - u'z| <= b is re-checked
 *   with an exact FP64 sign test.
 *   Projection depths select the points holding the median / MAD / MAD_+ of
 *   the FP32 projections (exact order statistics of the FP32 keys, ties broken
 *   by point index) and form the depth from FP64 projections of those points
 *   and of z.  The keys are held in shared memory while two CTAs of two
 *   directions fit an SM (about n <= 10,000 for d <= 12); beyond that they are
 *   formed once per round in device memory (up to 256 MB of scratch, taken in
 *   chunks) and every selection pass reads them back, with the same
 *   arithmetic, so results do not depend on which form ran.  n is limited to
 *   2^31 - 64 for projection depths.
 * Outputs (each n_queries long, or n_queries*r for round_choice_out):
 *   depth_out[q]   final depth D_min (double).                      required
 *   count_out[q]   halfspace: min(#<=, #>=) at D_min, else -1.        optional
 *   best_out[q]    flat index (l-1)*m + j of the direction that gave
 *                  D_min, or -1 if no direction went below 1.         optional
 *   round_choice_out[q*r + l-1]  index j taken as new pole in round l,
 *                  or -1 if the pole was kept.                        optional
 *   Outputs are device pointers if out_on_device != 0, else host pointers.
 * stream: a cudaStream_t (NULL = the legacy default stream).  With host
 *   outputs the call returns after the results are copied back.  With
 *   device outputs it returns after enqueueing; inputs and outputs must then
 *   stay valid until the stream has run.
 * Errors: INVALID_ARG, NOT_FOUND, BUDGET, UNSUPPORTED, CUDA.
 */
rrs_status rrs_depth(rrs_ctx* ctx, int64_t dataset_id, const void* Z, int64_t n_queries,
                     int32_t dtype, int32_t z_on_device, int32_t kind, int32_t n_dirs,
                     int32_t n_refinements, double cap_shrink, uint64_t seed, int32_t precision,
                     double* depth_out, int64_t* count_out, int32_t* best_out,
                     int32_t* round_choice_out, int32_t out_on_device, void* stream);

/*
 * One request of a batched launch: a dataset, its query batch (device
 * memory, row-major n_queries x d, FP32 or FP64 as `dtype`) and RRS
 * parameters, with device output pointers as in rrs_depth.
 */
typedef struct rrs_request {
    int64_t dataset_id;
    const void* Z;
    int64_t n_queries;
    int32_t dtype;
    int32_t kind;
    int32_t n_dirs;
    int32_t n_refinements;
    double cap_shrink;
    uint64_t seed;
    double* depth_out;
    int64_t* count_out;        /* optional */
    int32_t* best_out;         /* optional */
    int32_t* round_choice_out; /* optional */
    int32_t precision;         /* RRS_PREC_* (halfspace requests; 0 = FP32 CUDA cores) */
    int32_t reserved;          /* set to 0 */
} rrs_request;

/*
 * rrs_depth_batched - run many independent requests (different datasets of
 * uneven n and d, different kinds) together: every refinement round of every
 * request is served by one launch per pipeline stage over all requests
 * (Sec. 4: directions are independent within a round, queries are
 * independent).  Results are identical to calling rrs_depth on each request
 * alone with the request's precision.  Halfspace requests with
 * RRS_PREC_SPLIT_BF16X3 run on the tensor cores, one launch per dataset and
 * round covering all of that dataset's such requests; their counts equal the
 * FP32 path's (both are exact).  Requests may have different r; a request
 * leaves the batch when its rounds are done.
 *   reqs: host array of n_requests descriptors; all pointers inside are
 *   device pointers.  use_graph != 0 captures the launch sequence into a
 *   CUDA graph that is replayed on later calls with identical descriptors.
 * Errors: as rrs_depth.  Stream-ordered on `stream`.
 */
rrs_status rrs_depth_batched(rrs_ctx* ctx, const rrs_request* reqs, int32_t n_requests,
                             int32_t use_graph, void* stream);

/*
 * rrs_autotune - for halfspace depth on the tensor cores, pick the tile width
 * (128 or 256 points per tile; planes of K extent 64 only, other d have one
 * width) and cache it per (n, d); *choice_out receives it (0 when d has no
 * tensor-core path).  For projection / asymmetric projection depth, pick the
 * selection kernel on this dataset with m = ceil(n_dirs / n_refinements)
 * directions per round: 1, 2 or 4 directions per CTA with the keys held in
 * shared memory, RRS_SELECT_STREAM (keys formed once per round in device
 * memory and read at every pass), or RRS_SELECT_WARP (one warp per direction,
 * keys re-formed from X at every pass; d <= 16 and n <= 12,288).  Each
 * feasible choice is
 * timed on one round of probe queries (rows of the dataset, two per SM) and
 * the fastest is cached in the context; later rrs_depth / rrs_depth_batched
 * calls with the same (n, d, m) use it.  Without tuning: two or more
 * directions per CTA with resident keys where that fits two CTAs per SM,
 * else the streamed keys.  Results
 * never depend on the choice.  *choice_out (optional) receives it (0 for
 * halfspace depth, which has nothing to tune, and 0 when no choice keeps the
 * keys in shared memory: they then live in device memory and the kernel runs
 * with a fixed shape).
 * Synchronous.  Errors: INVALID_ARG, NOT_FOUND, CUDA.
 */
#define RRS_SELECT_WARP 64
#define RRS_SELECT_STREAM 32
rrs_status rrs_autotune(rrs_ctx* ctx, int64_t dataset_id, int32_t kind, int32_t n_dirs, int32_t n_refinements,
                        int32_t* choice_out);

/*
 * rrs_select_kernel - fix the selection kernel for (this dataset's n and d,
 * m = ceil(n_dirs / n_refinements)) instead of timing it: choice 1, 2 or 4
 * (directions per CTA, keys in shared memory), RRS_SELECT_WARP,
 * RRS_SELECT_STREAM, or 0 to drop a
 * fixed or tuned choice and return to the default; RRS_SELECT_STREAM keeps the
 * keys outside shared memory (formed once per round by a keys kernel, read
 * at every pass) whatever n.  A choice that does not
 * fit the dataset falls back to the default at launch.  Results never depend
 * on the choice.  Errors: INVALID_ARG (NULL context, unknown choice),
 * NOT_FOUND.
 */
rrs_status rrs_select_kernel(rrs_ctx* ctx, int64_t dataset_id, int32_t n_dirs, int32_t n_refinements,
                             int32_t choice);

/*
 * rrs_select_tc_tile - fix the tensor-core halfspace tile width for this
 * dataset's (n, d): 128 or 256 points per tile (256 exists only for planes of
 * K extent 64, i.e. d + 2 <= 64; a width that does not exist falls back to the
 * one that does), or 0 for the default (256 where it exists).  Counts never
 * depend on the width.  Cached graphs of batched calls are dropped, since they
 * replay the width of their capture; rrs_select_kernel and rrs_autotune do the
 * same.  Errors: INVALID_ARG, NOT_FOUND, UNSUPPORTED (d + 2 > 128).
 */
rrs_status rrs_select_tc_tile(rrs_ctx* ctx, int64_t dataset_id, int32_t tile_points);

/* Text for a status code (static storage). */
const char* rrs_status_string(rrs_status status);

/* Detail of the last failure on the calling thread (static, thread-local). */
const char* rrs_last_error(void);

/*
 * rrs_debug_directions - write the m directions of round `round` (1-based)
 * for query counter q into U (m x d FP32, row-major, device pointer), drawn
 * around `pole` (d FP32, device pointer; ignored for round 1) with the
 * library's generator: Alg. S1 (uniform on the sphere) for round 1, Alg. S4
 * (a cap of angle (pi/2) cap_shrink^(round-1) around the pole) after.  Lets
 * tests compare the device direction stream bit for bit with an independent
 * implementation.  U and pole stay owned by the caller.  Synchronous.
 * Errors: INVALID_ARG (NULL U, m < 0, d < 1, round < 1, q < 0, no pole for
 * round > 1), CUDA.
 */
rrs_status rrs_debug_directions(rrs_ctx* ctx, uint64_t seed, int32_t q, int32_t round, int32_t m,
                                int32_t d, double cap_shrink, const float* pole, float* U);

/*
 * rrs_debug_round_depths - for one dataset, query batch (device, FP32/FP64)
 * and round, the univariate depth of every (query, direction) pair,
 * with the directions supplied by the caller: U (n_queries x m x d FP32,
 * device).  depth_out (n_queries x m, device) receives D(u'z | u'X);
 * count_out (n_queries x m, device, halfspace only, may be NULL) receives
 * min(#<=, #>=); band_out (n_queries x m, device, halfspace only, may be
 * NULL) receives how many points fell in the near-tie band.  The univariate
 * depths are those of Sec. 2 (D_H, D_P, D_AP), computed by the same kernels
 * as rrs_depth.  All buffers stay owned by the caller.  Synchronous.
 * Errors: INVALID_ARG (NULL buffers, n_queries < 1, m < 1), NOT_FOUND,
 * UNSUPPORTED and BUDGET as rrs_depth, CUDA, and INTERNAL / TIMEOUT for
 * failures flagged on the device.
 */
rrs_status rrs_debug_round_depths(rrs_ctx* ctx, int64_t dataset_id, const void* Z,
                                  int64_t n_queries, int32_t dtype, int32_t kind, int32_t m,
                                  const float* U, int32_t precision, double* depth_out,
                                  int64_t* count_out, int64_t* band_out);

/* rrs_check - wait for `stream` (a cudaStream_t, NULL = legacy default) and
 * report device-side failures flagged by earlier stream-ordered calls,
 * clearing the flags.  Use it after rrs_depth with device outputs or
 * rrs_depth_batched.  Errors: INVALID_ARG (NULL context), CUDA, INTERNAL (an
 * invariant failed on the device, e.g. a selection that did not converge),
 * TIMEOUT (a bounded device wait gave up). */
rrs_status rrs_check(rrs_ctx* ctx, void* stream);

/*
 * rrs_debug_wait_timeout - exercise the failure path of the bounded device
 * waits: one thread waits on an mbarrier that nothing completes, gives up after
 * limit_cycles SM clock cycles and flags a timeout.  Returns RRS_ERR_TIMEOUT
 * (the expected outcome) with the context left usable.  Synchronous.
 * Errors besides: INVALID_ARG (NULL context, limit_cycles < 0), CUDA.
 */
rrs_status rrs_debug_wait_timeout(rrs_ctx* ctx, int64_t limit_cycles);

/* Number of kernel launches this context has issued (for accounting). */
uint64_t rrs_launch_count(rrs_ctx* ctx);

/* Pipeline stages timed by the profiler (one slot each in rrs_profile_read). */
#define RRS_STAGE_PREP 0      /* query conversion and state initialisation */
#define RRS_STAGE_GEN 1       /* direction generation (Alg. S1 / S4) and y_z */
#define RRS_STAGE_HD_SIMT 2   /* halfspace counts, FP32 CUDA-core projection */
#define RRS_STAGE_HD_TC 3     /* halfspace counts, tcgen05 split-BF16x3 projection */
#define RRS_STAGE_PDAP 4      /* projection / asymmetric projection depth (selection) */
#define RRS_STAGE_ARGMIN 5    /* round minimum and pole update (Alg. 1 steps 4-6) */
#define RRS_STAGE_KEYS 6      /* selection keys formed once per round (d > 16, or n beyond shared memory) */
#define RRS_NSTAGES 7

/*
 * rrs_profile_enable - turn per-stage timing on (on != 0) or off and reset the
 * accumulated figures.  While on, every launch of rrs_depth /
 * rrs_depth_batched (outside graph capture) is bracketed by two CUDA events
 * recorded on the launching stream.  Errors: INVALID_ARG (NULL context).
 */
rrs_status rrs_profile_enable(rrs_ctx* ctx, int32_t on);

/*
 * rrs_profile_read - wait for the recorded events and return, per stage, the
 * accumulated device milliseconds (ms_out[RRS_NSTAGES], host) and launch
 * counts (launches_out[RRS_NSTAGES], host, may be NULL) since the last
 * rrs_profile_enable.  Errors: INVALID_ARG (NULL context or ms_out), CUDA.
 */
rrs_status rrs_profile_read(rrs_ctx* ctx, double* ms_out, int64_t* launches_out);

/*
 * Serving (continuous batching).  A server keeps a fixed pool of query slots
 * on the device.  Requests queue in arrival order; each rrs_server_step admits
 * the waiting requests that fit in the free slots, runs ONE refinement round
 * (Alg. 4: generate, project + univariate depth, minimum and pole update) for
 * a set of active queries in shared launches -- each query at its own round --
 * and retires the requests whose queries have all run their last round by
 * copying their depths to the caller's host buffer.  The set is bounded by the
 * server's work limit (rrs_server_set_work_limit): every active request, oldest
 * first, takes up to a quarter of the limit (at least one query), then the
 * oldest requests fill the rest.  Requests that arrive while others are on the GPU thus
 * join the next step's launches.  Every query keeps its own direction stream
 * (counter q = its row in its request) and state, so a request's depths do not
 * depend on what else is being served: they equal rrs_depth's results on
 * that request alone (at the server's precision).
 */
typedef struct rrs_server rrs_server;

/*
 * rrs_server_create - a server on ctx with max_slots query slots, each able to
 * hold a request of up to max_dirs_per_round directions per round (m) and
 * dimension max_d.  precision: RRS_PREC_FP32_SIMT, or RRS_PREC_SPLIT_BF16X3 to
 * serve halfspace requests on the tensor cores (datasets with d + 2 <= 128;
 * others stay on the FP32 kernel; counts are exact either way).  Device memory
 * for the pool is taken once (counted against the context's budget).  stream:
 * cudaStream_t every server operation is ordered on (NULL = legacy default
 * stream).  Errors: INVALID_ARG, BUDGET, CUDA.
 */
rrs_status rrs_server_create(rrs_ctx* ctx, int32_t max_slots, int32_t max_dirs_per_round, int32_t max_d,
                             int32_t precision, void* stream, rrs_server** out);

/*
 * rrs_server_submit - queue a request: queries Z (host, n_queries x d, dtype)
 * against a registered dataset with the RRS parameters of rrs_depth (FP32
 * arithmetic).  Z and depth_out (host, n_queries doubles) must stay valid until
 * rrs_server_poll reports the request done; the dataset must stay registered.
 * *request_id_out receives the request's id.  Errors: INVALID_ARG, NOT_FOUND,
 * UNSUPPORTED (request larger than the slot shape or pool).
 */
rrs_status rrs_server_submit(rrs_server* server, int64_t dataset_id, const void* Z, int64_t n_queries,
                             int32_t dtype, int32_t kind, int32_t n_dirs, int32_t n_refinements,
                             double cap_shrink, uint64_t seed, double* depth_out, int64_t* request_id_out);

/*
 * rrs_server_step - admit what fits, run one round for the queries the work
 * limit lets in, retire finished requests (their host copies are enqueued on
 * the stream).  Returns after enqueueing.  *active_queries_out /
 * *pending_requests_out (optional) receive the admitted queries and the
 * requests still waiting.  Each step is one refinement round (Alg. 4) for each
 * chosen query, at that query's own round.  Errors: INVALID_ARG (NULL server),
 * CUDA.
 */
rrs_status rrs_server_step(rrs_server* server, int32_t* active_queries_out, int32_t* pending_requests_out);

/*
 * rrs_server_set_work_limit - bound one step's work: the weighted number of
 * point-direction pairs (n x m per query and round; halfspace pairs on the
 * tensor cores weigh 0.1, all others 1) of the queries that run a round in
 * one step.  A step always runs at least one query, so no request starves.
 * 0 runs every admitted query at every step (the GPU work of a step then grows
 * with the admitted backlog, and so does every request's latency).  The
 * default, RRS_SERVER_DEFAULT_WORK, keeps a step at roughly ten milliseconds
 * of selection work on a GB300.  Errors: INVALID_ARG (NULL server, negative or
 * non-finite limit).
 */
#define RRS_SERVER_DEFAULT_WORK 4e9
rrs_status rrs_server_set_work_limit(rrs_server* server, double max_pairs_per_step);

/* rrs_server_poll - *done_out = 1 once the request's depths are in its host
 * buffer (the request is then forgotten), else 0.  Errors: NOT_FOUND, CUDA. */
rrs_status rrs_server_poll(rrs_server* server, int64_t request_id, int32_t* done_out);

/* rrs_server_destroy - wait for the stream, drop queued requests, free the pool.
 * NULL is accepted.  Always returns RRS_OK. */
rrs_status rrs_server_destroy(rrs_server* server);

/*
 * rrs_depth_noalloc - rrs_depth for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment variant.
 *
 * Callers such as plug-ins living inside another framework's memory pool,
 * processes that forbid allocation once running, or loops that must never
 * wait on the allocator cannot call cudaMalloc.  This call runs the same
 * kernels as rrs_depth with RRS_PREC_FP32_SIMT, but takes the data cloud
 * directly (no rrs_register_dataset, no context) and draws all its working
 * memory from one fixed device array of RRS_NOALLOC_SCRATCH_BYTES that the
 * library holds on every device that loads it, until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   X: n x d row-major, dtype RRS_F32 or RRS_F64, device pointer (read only;
 *      for RRS_F64 the exact recheck reads it during the call).
 *   Z: n_queries x d row-major, same dtype, device pointer.
 *   kind, n_dirs, n_refinements, cap_shrink, seed: as rrs_depth; query row q
 *      uses stream counter q, so results equal rrs_depth's bit for bit.
 *   depth_out (n_queries doubles) and count_out (n_queries int64, halfspace
 *      counts, or -1; may be NULL): device pointers.
 *   stream: cudaStream_t (NULL = legacy default stream).  The call waits for
 *      the stream twice (it reads the input check and the device-side error
 *      flags back to the host) and returns after the stream has finished its
 *      work.
 * Limits: everything the call needs (about 4*(n+1)*(d+4) bytes for X plus
 * about n_queries * m * 4*(d+10) bytes for the rounds, m = ceil(k/r)) must fit
 * in RRS_NOALLOC_SCRATCH_BYTES; a larger request is rejected with
 * RRS_ERR_BUDGET and a message giving both sizes (rrs_last_error).
 * Every call looks up the array's device address (cudaGetSymbolAddress) with
 * the calling device current, so a device reset cannot leave a stale address.
 * The first call on a device also loads the library's device code there;
 * make that first call before any stream capture.  All calls share the one
 * array and it keeps the
 * last call's contents (each call clears what must start at zero); calls
 * whose GPU work overlaps -- other streams or other host threads -- race on
 * it and must be serialised by the caller.
 * Errors: INVALID_ARG, BUDGET, UNSUPPORTED, CUDA, INTERNAL.
 */
#define RRS_NOALLOC_SCRATCH_BYTES (32u << 20)
rrs_status rrs_depth_noalloc(const void* X, int64_t n, int32_t d, int32_t dtype, const void* Z,
                             int64_t n_queries, int32_t kind, int32_t n_dirs, int32_t n_refinements,
                             double cap_shrink, uint64_t seed, double* depth_out, int64_t* count_out,
                             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RRS_H */
