/*
 * sfft.h -- C ABI of libsfft.so, a GB300 (sm_103a) implementation of the sparse Fourier transform of
 * Hassanieh, Indyk, Katabi and Price, "Nearly Optimal Sparse Fourier Transform" (2012).
 *
 * Problem (Sec. 1, Eq. (1); Sec. 2 "Assumptions"): given time-domain access to x in C^n, n a power of
 * two, return a sparse vector zhat approximating the spectrum X = DFT(x).  In the exactly k-sparse case
 * (Sec. 3, Algorithm 1) zhat = X with constant probability; in the general case (Sec. 4, Algorithms 2
 * and 3) ||X - zhat||_2 <= (1 + eps) min_{k-sparse y} ||X - y||_2 + delta ||X||_2.
 *
 * Conventions shared by every entry point:
 *   - X_f = sum_t x_t exp(-2 pi i f t / n) (unnormalised; the paper's unitary spectrum is X / sqrt(n)).
 *   - Indices are 0-based, taken mod n.  n <= 2^30.
 *   - Signals are arrays of interleaved (re, im) pairs: float for SFFT_FP32, double for SFFT_FP64.
 *   - Recovered values are always double (re, im) pairs.
 *   - "d_" pointers are device memory owned by the caller; they must stay valid until the work queued
 *     on the given stream completes.  "h_" pointers are host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every call that
 *     takes a stream only enqueues work: it never synchronises, never allocates, and can be captured
 *     in a CUDA graph.
 *   - Every call returns a status and never throws.  On SFFT_ERR_CUDA the CUDA error string is
 *     available from sfft_last_error().
 *   - Randomness: request r of a call with seed s draws its hashing parameters from Philox4x32-10
 *     keyed by s, counter (round, sub-step, kind, r); the same (x, params, seed, r) gives bit-identical
 *     output on every run.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sfft_status {
    SFFT_OK = 0,
    SFFT_ERR_INVALID_ARG = 1,   /* a null pointer, a size out of range, an inconsistent parameter */
    SFFT_ERR_N_NOT_POW2 = 2,    /* n is not a power of two in [2^6, 2^30] */
    SFFT_ERR_K_RANGE = 3,       /* k == 0 or the schedule needs more bins than supported */
    SFFT_ERR_OOM = 4,           /* device allocation failed (plan creation only) */
    SFFT_ERR_CUDA = 5,          /* a CUDA call failed; see sfft_last_error() */
    SFFT_ERR_TIMEOUT = 6,       /* a wait gave up */
    SFFT_ERR_CAPACITY = 7,      /* a request's zhat outgrew its capacity; the largest-index entries were dropped */
    SFFT_ERR_NOT_CONVERGED = 8, /* warning: the last round saw a bin above thr it could not decode */
    SFFT_ERR_BUSY = 9           /* the plan or queue cannot take more work now */
} sfft_status;

typedef enum sfft_mode { SFFT_EXACT = 0, SFFT_GENERAL = 1 } sfft_mode;
typedef enum sfft_precision { SFFT_FP32 = 0, SFFT_FP64 = 1 } sfft_precision;

/*
 * Parameters.  Fields the paper leaves as Theta(.) constants are explicit; sfft_params_default()
 * fills the values used throughout this library's tests and benchmarks.
 */
typedef struct sfft_params {
    uint64_t n;            /* signal length, a power of two */
    uint32_t k;            /* sparsity */
    uint32_t mode;         /* sfft_mode */
    uint32_t precision;    /* sfft_precision: data path of gather, fold and bin FFT */
    double delta;          /* flat-window tolerance (Sec. 2, Definition of a flat window) */
    double alpha0;         /* alpha of the first round */
    double bins_per_k;     /* B = pow2ceil(bins_per_k k_t) (exact), pow2ceil(bins_per_k k_r / eps) (general) */
    uint32_t B_min;        /* smallest B of any round */
    uint32_t extra_rounds; /* exact: rounds after t = ceil(log2 k) */
    double thr;            /* exact: J = {j : |u_j| > thr} (Algorithm 1's 1/2) */
    double tau_dec;        /* exact: smallest phase tolerance (rad) the location ladder may leave */
    double iso_tol;        /* exact: shifted bins must keep |u_j| to within iso_tol |u_j| */
    double gmin;           /* exact: a decode needs window gain W(-o) >= gmin */
    double prune;          /* exact: after a round drop zhat_i with |zhat_i| < prune thr */
    double ref_lo, ref_hi; /* exact: residual window (times thr) for re-estimating a known value */
    double ref_tol;        /* exact: phase tolerance (rad) of that re-estimate */
    uint32_t z_cap;        /* capacity of zhat per request */
    double eps;            /* general: epsilon of Eq. (1) */
    uint32_t t_regions;    /* general: t of Algorithm 3 (0 -> largest power of two <= log2 n) */
    uint32_t R_loc;        /* general: rounds of LocateInner per level */
    uint32_t R_est;        /* general: hashings of EstimateValues */
    double s;              /* general: vote half-width s pi */
    double est_gmin;       /* general: a hashing joins the median only if W(-o) >= est_gmin */
    uint32_t streams;      /* a batch is split over this many internal streams so that one group's
                              end-of-round work overlaps another group's gather (0 -> 1 in exact
                              mode, whose one launch per group already overlaps its rounds; 4 in
                              general mode) */
    uint32_t gain;         /* the window gain used to subtract recovered coefficients and to divide
                              decoded values: 0 -> the exact response W(o) of the truncated taps
                              (default); 1 -> the paper's closed form Ghat'(o) (Sec. 7: 1 on the pass
                              band, 0 beyond n/2B, a difference of Gaussian cdfs in between) */
    uint32_t chunk_taps;   /* exact mode: window taps gathered per CTA (a power of two in [256, 8192];
                              0 -> 2048); fewer taps spread one request over more CTAs (lower latency),
                              more taps cut partial sums (batch throughput) */
    uint32_t permuted_copy; /* general mode: 0 -> a round whose LocateInner hashings (all under the
                              round's sigma) gather at least 2n samples first writes x_{sigma m} for
                              every m in [n] once per request, and those hashings read it in order
                              instead of at random (the same samples, so the same results; n complex64
                              of device memory per request of max_batch); 1 -> never */
} sfft_params;

/* Fill *p with the library defaults for (n, k, mode); precision SFFT_FP32. */
void sfft_params_default(sfft_params* p, uint64_t n, uint32_t k, uint32_t mode);

/* Human-readable name of a status. */
const char* sfft_status_str(sfft_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* sfft_last_error(void);

/* ---------------------------------------------------------------------------------------------- */
/* Plans                                                                                          */
/* ---------------------------------------------------------------------------------------------- */
typedef struct sfft_plan_s* sfft_plan;

/*
 * Build a plan: the round schedule, the flat-window taps of every round (Sec. 7, Lemma on window
 * construction), the exact window response table W(o), |o| <= n/2B, of every round, and a device
 * workspace for max_batch requests.  The only call that allocates device memory.  Runs on the
 * current CUDA device and synchronises it.
 * Errors: INVALID_ARG (null, max_batch == 0, bad field), N_NOT_POW2, K_RANGE, OOM, CUDA.
 */
sfft_status sfft_plan_create(const sfft_params* p, uint32_t max_batch, sfft_plan* out);

/* Release a plan and its device memory (synchronises the device). NULL is accepted. */
sfft_status sfft_plan_destroy(sfft_plan plan);

/* Number of rounds of the plan's schedule (exact: ceil(log2 k) + 1 + extra_rounds; general: R). */
uint32_t sfft_plan_rounds(sfft_plan plan);

/*
 * Description of exact-mode round t (Algorithm 1, NoiselessSparseFFT loop): B, alpha, the window
 * half-width T (2T+1 taps), the ladder shifts beta_l (finest first), and the hashing parameters
 * (sigma, b) that request `request` of a call with `seed` draws for that round.
 * shifts must hold 4 entries.  Host-only; never touches the device.
 */
sfft_status sfft_plan_round_info(sfft_plan plan, uint32_t t, uint64_t seed, uint32_t request, uint32_t* B,
                                 double* alpha, int64_t* T, uint32_t* nshift, uint64_t* shifts, uint64_t* sigma,
                                 uint64_t* b);

/* Copy round t's window taps g_0..g_T (double, host) into h_taps (T+1 entries). */
sfft_status sfft_plan_taps(sfft_plan plan, uint32_t t, double* h_taps, uint64_t cap);

/* ---------------------------------------------------------------------------------------------- */
/* Whole transforms                                                                               */
/* ---------------------------------------------------------------------------------------------- */
/*
 * Run the sparse FFT on `batch` signals (batch <= max_batch) stored back to back in d_x
 * (batch x n complex values of the plan's precision; device memory, or any memory the device can
 * address, such as page-locked host memory, which is then read in place).  Request r uses seed `seed`, request index r.
 * Outputs, per request r, in caller-owned device arrays:
 *   d_idx[r*cap .. r*cap + count)  recovered frequencies, ascending (uint32)
 *   d_val[...]                    their values X_f as (re, im) doubles
 *   d_count[r]                    number of entries written (<= cap)
 *   d_flag[r]                     sfft_status of the request: OK, NOT_CONVERGED or CAPACITY
 * Exact mode follows Algorithm 1: one kernel launch per stream group covers every round, since the
 * samples of all rounds are known before any is decoded; general mode follows Algorithms 2 and 3 with
 * four launches per round (five in a round that writes the permuted copy; see permuted_copy).
 * Asynchronous on `stream`; the plan may run one call at a time.
 * Errors: INVALID_ARG (null pointer, batch out of range, cap == 0), CUDA (launch failure, including a
 * batch whose chunks would exceed 2^31 - 1 CTAs).
 */
sfft_status sfft_execute(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, void* stream,
                         uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag);

/*
 * Same computation from host memory, outputs copied back into host arrays; synchronises the stream.
 * If h_x (batch x n) is page-locked host memory the device can address (cudaHostAlloc / registered;
 * on Grace-Blackwell reached over NVLink-C2C), the kernels read the samples they need from it in
 * place: a transform moves only its gathered samples across the link, not the whole signal.  Any
 * other host memory is first copied whole to a device staging buffer owned by the plan.  Staging
 * buffers are allocated on the first call with a given batch (the one call besides plan creation
 * that may allocate).
 */
sfft_status sfft_execute_host(sfft_plan plan, const void* h_x, uint32_t batch, uint64_t seed, void* stream,
                              uint32_t* h_idx, double* h_val, uint32_t cap, uint32_t* h_count, int32_t* h_flag);

/*
 * Multi-channel batch with shared hashing (exact mode, SFFT_FP32 plans).  C = `channels` signals
 * sampled at the same times are stored interleaved: d_x holds n rows of C complex64 values, row m
 * holding sample m of every channel (device memory, 16-byte aligned).  Every channel is transformed
 * with the same random hashings, those of request index `id` under `seed` (Algorithm 1's sigma, b of
 * each round are drawn once and shared), so one sigma-strided sample index reads C contiguous values
 * instead of C scattered 32-byte sectors.  Channel c's result equals that of sfft_execute_requests on
 * signal x[.][c] with {seed, id} (up to FP32 rounding of the fold, done in another order); each
 * result on its own is a draw of the algorithm, but the channels' failures are not independent
 * (they share the hashings).  Outputs per channel slot c as for sfft_execute (slot r = channel r).
 * channels: a multiple of 32, at most 256 and at most the plan's max_batch.  The gather stages the
 * sample rows in shared memory with bulk asynchronous copies; should one not land within a bounded
 * wait (never expected), every channel's d_flag reads SFFT_ERR_TIMEOUT and its count 0.
 * Errors: INVALID_ARG (a general-mode or FP64 plan, null pointer, channels out of range, misaligned
 * d_x, cap == 0), CUDA.
 */
sfft_status sfft_execute_channels(sfft_plan plan, const void* d_x, uint32_t channels, uint64_t seed, uint32_t id,
                                  void* stream, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                                  int32_t* d_flag);
/* The same, recording the CUDA events `before` and `after` (cudaEvent_t, either may be NULL) on
 * `stream` right before and right after the gather kernel, so that a caller can time the gather
 * alone. */
sfft_status sfft_execute_channels_timed(sfft_plan plan, const void* d_x, uint32_t channels, uint64_t seed, uint32_t id,
                                        void* stream, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                                        int32_t* d_flag, void* before, void* after);

/*
 * Measurement, no part of the transform: read d_x[r][d_idx[r][i]] (complex64, row r of row_elems
 * values, a power of two <= 2^31; each index taken mod row_elems) for r < rows, i < per_row, in the
 * order given, with nothing else done: 16 reads in flight per thread, each through L2 only (one
 * 32-byte sector per read, as in the transform's gathers), the values folded into d_sink[0..64)
 * (caller-owned device words).  Timed around by the caller, it gives the rate at which this device
 * serves a list of sample reads -- for instance a transform's own sample addresses in its own order,
 * in random order, or sorted by address.
 * Errors: INVALID_ARG (null pointer, zero sizes, row_elems not a power of two), CUDA.
 */
sfft_status sfft_gather_rate(const void* d_x, uint64_t row_elems, uint32_t rows, const uint32_t* d_idx,
                             uint32_t per_row, uint32_t* d_sink, void* stream);

/*
 * One request of sfft_execute_requests: its own signal, seed and request index.  The result depends
 * on (signal, params, seed, id) only, not on the batch or slot the request runs in: request r of
 * sfft_execute with seed s equals a request {row r, s, r}.
 */
typedef struct sfft_request {
    const void* d_x;    /* device signal: n complex values of the plan's precision (or `period` of them),
                           8-byte (FP32) or 16-byte (FP64) aligned; caller-owned, valid until the work
                           completes */
    uint64_t seed;      /* Philox key of the request's draws */
    uint32_t id;        /* request index of the Philox counter */
    uint32_t period;    /* 0: d_x holds the n samples.  Otherwise a power of two dividing n: d_x holds
                           `period` samples and the transform is that of the periodic extension
                           y_i = x_{i mod period}, each sample the algorithm asks for read in place
                           (Sec. 5: with period k, Y is k-sparse on the multiples of n/k and
                           Y_{j n/k} = (n/k) DFT_k(x)_j, so a k-point DFT comes out of the n-point
                           sparse transform; thr should then scale with n/k) */
} sfft_request;

/*
 * sfft_execute over `batch` independent requests (batch <= max_batch) whose signals lie anywhere in
 * device memory.  The table h_reqs (host memory) is copied into page-locked memory owned by the plan
 * before the call returns, so it may be reused or freed at once; the outputs are laid out as for
 * sfft_execute (slot r = h_reqs[r]).
 * A plan serves one stream at a time: the table copy and the kernels go to `stream`.
 * Errors: INVALID_ARG (null pointer, batch out of range, cap == 0, a null or misaligned d_x, a period
 * that is not a power of two dividing n), CUDA.
 */
sfft_status sfft_execute_requests(sfft_plan plan, const sfft_request* h_reqs, uint32_t batch, void* stream,
                                  uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag);

/* ---------------------------------------------------------------------------------------------- */
/* CUDA graphs of a fixed batch                                                                    */
/* ---------------------------------------------------------------------------------------------- */
/*
 * Capture one whole transform of a fixed batch (every round's launches, the internal stream fork and
 * join, the clears) into an instantiated CUDA graph, replayed by sfft_graph_launch with one call.
 * d_x != NULL: the batch is the rows of d_x with `seed` (as sfft_execute).  d_x == NULL: the batch is
 * the plan's request table, refilled between replays with sfft_plan_set_requests (as
 * sfft_execute_requests).  Outputs as for sfft_execute.  The plan must outlive the graph and serve
 * one stream at a time (graph replays included).
 * Errors: INVALID_ARG, CUDA (capture or instantiation failed).
 */
typedef struct sfft_graph_s* sfft_graph;
sfft_status sfft_graph_create(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, uint32_t* d_idx,
                              double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag, sfft_graph* out);
sfft_status sfft_graph_launch(sfft_graph g, void* stream);
sfft_status sfft_graph_destroy(sfft_graph g);

/* Copy `batch` requests (host table) into the plan's request table on `stream` (for graphs captured
 * with d_x == NULL).  Errors: INVALID_ARG (as sfft_execute_requests), CUDA. */
sfft_status sfft_plan_set_requests(sfft_plan plan, const sfft_request* h_reqs, uint32_t batch, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Autotuner                                                                                       */
/* ---------------------------------------------------------------------------------------------- */
/*
 * The paper leaves the bin count B = Theta(k) and the window's transition fraction alpha (hence its
 * width w ~ B log(1/delta) / alpha) as constants; this library also splits a batch over internal
 * streams.  sfft_autotune times candidate settings for base's (n, k, mode, delta, precision):
 * bins_per_k in {2, 4, 8} (exact) or {4, 8, 16} (general), alpha0 in {0.25, 0.5, 0.75}, streams in
 * {1, 2, 4, 8} and, in exact mode, chunk_taps (the gather's taps per CTA) in {1024, 2048}, each on the
 * same `batch` (<= 256) synthetic signals made on the device (exact: k
 * unit-magnitude coefficients; general: k coefficients with |X| = 10^u, u uniform on [0, 1), plus
 * complex Gaussian time noise at snr_db), `reps` timed transforms after one warm-up (CUDA events).
 * Each candidate is scored against the planted coefficients; *best receives the fastest candidate
 * that is at least as accurate as base's own settings (as many exact recoveries with values within
 * 1e-4 in exact mode; a mean relative l2 error ||zhat - X_heavy|| / ||X_heavy|| within 5 % of base's
 * in general mode).  report (may be NULL) receives up to report_cap entries, base's first.
 * Allocates and synchronises the device; not for a latency-critical path.
 */
typedef struct sfft_tune_entry {
    double bins_per_k, alpha0;
    uint32_t streams;
    uint32_t chunk_taps;     /* taps per CTA of the gather (exact mode) */
    int32_t status;          /* plan creation / run status of the candidate */
    double us_per_transform; /* device time per transform */
    uint32_t exact;          /* requests recovered exactly (exact mode) */
    uint32_t chosen;         /* 1 for the candidate copied to *best */
    double rel_err;          /* mean ||zhat - X_heavy|| / ||X_heavy|| */
} sfft_tune_entry;
sfft_status sfft_autotune(const sfft_params* base, uint32_t batch, double snr_db, uint64_t seed, uint32_t reps,
                          sfft_params* best, sfft_tune_entry* report, uint32_t report_cap, uint32_t* n_report);

/* ---------------------------------------------------------------------------------------------- */
/* Mixed batches in one persistent launch                                                          */
/* ---------------------------------------------------------------------------------------------- */
/*
 * A batch plan groups exact-mode plans of any (n, k) (one precision) so that a batch mixing them runs
 * as ONE persistent launch: CTAs take (request, round, chunk) items from a device queue, and the CTA
 * that finishes a request's round (Algorithm 1's loop) queues that request's next round at once, so
 * rounds of different requests overlap with no launch boundary between them.  Results are those of
 * sfft_execute_requests on each request's own plan, bit for bit.  The batch plan owns a workspace for
 * max_requests requests; the plans must outlive it.
 * Errors: INVALID_ARG (null, nplans == 0, a general-mode plan, mixed precisions), OOM, CUDA.
 */
typedef struct sfft_batch_plan_s* sfft_batch_plan;
sfft_status sfft_batch_plan_create(const sfft_plan* plans, uint32_t nplans, uint32_t max_requests,
                                   sfft_batch_plan* out);
sfft_status sfft_batch_plan_destroy(sfft_batch_plan bp);

/*
 * Run nreq (<= max_requests) requests: request r uses plans[h_plan_of[r]] and h_reqs[r] (signal, seed,
 * id, period).  Outputs as for sfft_execute (slot r, capacity cap).  The host tables are staged in
 * page-locked memory owned by the batch plan (two buffers, so consecutive calls on one stream do not
 * wait for each other).  A request whose queue item was not published within about a second (a
 * malfunction, never expected) ends with d_flag = SFFT_ERR_TIMEOUT.
 * Errors: INVALID_ARG (null, nreq out of range, a plan index or request that is out of range), CUDA.
 */
sfft_status sfft_batch_execute(sfft_batch_plan bp, const uint32_t* h_plan_of, const sfft_request* h_reqs,
                               uint32_t nreq, void* stream, uint32_t* d_idx, double* d_val, uint32_t cap,
                               uint32_t* d_count, int32_t* d_flag);

/*
 * Check of the persistent launch's bounded wait: one CTA of the batch kernel takes a queue item that
 * nothing ever publishes.  Its wait gives up after about a second, it sets the launch's error flag and
 * returns; the call synchronises `stream` and returns SFFT_ERR_TIMEOUT when the flag was set (the
 * expected outcome) or SFFT_OK if the wait did not give up.  The device stays usable either way.
 * Errors: OOM, CUDA.
 */
sfft_status sfft_persistent_wait_check(void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Serving: continuous batching of independent transforms                                         */
/* ---------------------------------------------------------------------------------------------- */
/*
 * The paper has no serving layer; this one runs its transforms as a service.  A server owns a
 * dispatcher thread on the device current at creation.  Jobs of any (n, k, mode, ...) are submitted
 * from any thread.  The dispatcher:
 *   - keeps one resident plan set per distinct sfft_params (window taps, W tables and workspace stay
 *     on the device between jobs; the least recently used idle sets beyond max_plans are released);
 *   - admits jobs in submission order: a job whose signal is in host memory is admitted once its
 *     device copy fits in mem_budget (resident plans count against it too), and its copy starts on a
 *     copy stream at once; a job whose signal is already on the device is admitted immediately;
 *   - launches, for each parameter set with admitted jobs and an idle plan instance, one batch of up
 *     to max_batch of them (sfft_execute_requests), so jobs that arrive while earlier batches run on
 *     the GPU are batched into the next launch as instances free up, and batches of different
 *     parameter sets and instances overlap on the device;
 *   - when a batch completes, copies each job's results to its host arrays, frees its staging memory
 *     and marks it done.
 * A job's result equals that of the same request run alone (same params, signal, seed and id),
 * bit for bit.
 */
typedef struct sfft_server_s* sfft_server;

typedef struct sfft_server_config {
    uint64_t mem_budget;  /* device bytes for resident plans and staged signals; 0 -> half of the
                             free device memory at creation */
    uint32_t max_batch;   /* jobs per launch; 0 -> 64 */
    uint32_t instances;   /* plan instances per parameter set (batches of one set in flight at once);
                             0 -> 2 */
    uint32_t max_plans;   /* resident parameter sets; 0 -> 16 */
    uint32_t reserved;    /* 0 */
} sfft_server_config;

typedef struct sfft_job {
    const void* x;        /* the signal: n complex values of the params' precision */
    uint32_t x_on_device; /* 1: device memory, read in place (valid until the job completes);
                             0: host memory, copied on admission (page-locked copies fastest; the
                             array may be reused once the job completes) */
    uint32_t id;          /* request index of the job's draws */
    uint64_t seed;        /* Philox key of the job's draws */
    uint32_t* h_idx;      /* host output: up to cap recovered frequencies, ascending */
    double* h_val;        /* host output: their values as (re, im) doubles */
    uint32_t cap;         /* capacity of h_idx / h_val (entries) */
    uint32_t period;      /* 0, or x holds `period` samples of a periodic signal (as in sfft_request) */
} sfft_job;

typedef struct sfft_job_result {
    uint32_t count;       /* entries written (<= cap) */
    int32_t flag;         /* the transform's status: OK, NOT_CONVERGED or CAPACITY */
    double queued_us;     /* submission to launch */
    double latency_us;    /* submission to completion (host clock) */
} sfft_job_result;

typedef struct sfft_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t launches;    /* batches launched */
    uint64_t plans;       /* resident plan instances */
    uint64_t bytes_in_use, bytes_peak;  /* device bytes held (plans + staged signals) */
    double mean_batch;    /* jobs per launch */
    double p50_us, p99_us;  /* latency of the jobs completed so far */
} sfft_server_stats;

/* Start a server (NULL cfg -> all defaults).  Errors: INVALID_ARG, CUDA (no device), OOM. */
sfft_status sfft_server_create(const sfft_server_config* cfg, sfft_server* out);

/* Finish every submitted job, stop the dispatcher and release all memory.  NULL is accepted. */
sfft_status sfft_server_destroy(sfft_server s);

/*
 * Queue one job; *ticket names it.  The params and the job description are copied.
 * Errors: INVALID_ARG (null, bad params, null outputs, cap == 0), N_NOT_POW2, K_RANGE, OOM (the job's
 * signal and plan can never fit in mem_budget), BUSY (the server is being destroyed).
 */
sfft_status sfft_submit(sfft_server s, const sfft_params* p, const sfft_job* job, uint64_t* ticket);

/*
 * Queue count jobs of one parameter set at once: the same as count calls of sfft_submit in order,
 * under one lock and with one wake-up of the dispatcher (a caller with many requests at hand pays the
 * submission once).  tickets (count entries, caller-owned) receives job i's ticket in tickets[i].
 * Every job is checked before any is queued: on an error status nothing was queued.  Errors: those
 * of sfft_submit; INVALID_ARG also for count == 0 or null arrays.
 */
sfft_status sfft_submit_many(sfft_server s, const sfft_params* p, const sfft_job* jobs, uint32_t count,
                             uint64_t* tickets);

/* OK: done (results written); BUSY: not done yet; INVALID_ARG: unknown ticket; another status: the
 * job failed (e.g. CUDA, OOM at plan creation). */
sfft_status sfft_poll(sfft_server s, uint64_t ticket);

/*
 * Wait up to timeout_us for a job.  On OK the job is done, *res (if not NULL) describes it and the
 * ticket is released; on TIMEOUT it is still pending; on another error status it failed (and is
 * released).  INVALID_ARG: unknown ticket.
 */
sfft_status sfft_wait(sfft_server s, uint64_t ticket, uint64_t timeout_us, sfft_job_result* res);

/*
 * Wait for count jobs, timeout_us in total.  status[i] (count entries, caller-owned) receives what
 * sfft_wait would return for tickets[i], and res[i] (if res is not NULL) describes job i when that is
 * OK; jobs that completed are released, pending ones (TIMEOUT) are kept.  Returns the first failing
 * status in ticket order if a job failed (INVALID_ARG for an unknown ticket), else TIMEOUT if one is
 * still pending, else OK.  INVALID_ARG with status untouched: null arrays or count == 0.
 */
sfft_status sfft_wait_many(sfft_server s, const uint64_t* tickets, uint32_t count, uint64_t timeout_us,
                           sfft_job_result* res, int32_t* status);

/* Counters and latency percentiles since creation. */
sfft_status sfft_server_stats_get(sfft_server s, sfft_server_stats* st);

/* ---------------------------------------------------------------------------------------------- */
/* Single steps (for parity tests and for callers that drive the rounds themselves)               */
/* ---------------------------------------------------------------------------------------------- */
/*
 * One HashToBins (Algorithm 1, procedure HashToBins; the four-step method of Lemma "hashtobins"),
 * with exact-mode round t's window, explicit (sigma odd, a, b), on one signal d_x (n values):
 *   u_j = sum_r (sum_{t' = r mod B} G_t' x_{sigma(t'-a)} w^{sigma b t'}) e^{-2 pi i j r / B}
 *         - sum_{i in zhat} W(-o(i)) zhat_i w^{a sigma i} [h(i) = j]
 * d_zidx / d_zval hold nz entries of zhat (nz may be 0); d_u receives B (re, im) doubles.
 */
sfft_status sfft_hash_to_bins(sfft_plan plan, uint32_t t, const void* d_x, uint64_t sigma, uint64_t a, uint64_t b,
                              const uint32_t* d_zidx, const double* d_zval, uint32_t nz, double* d_u, void* stream);

/*
 * The location and estimation step of exact-mode round t (Algorithm 1, loop over J, with this
 * library's readings: shift-ladder phase decode, value u_j / W(-o), isolation check, and the
 * re-estimation of known values) on caller-supplied bins d_u ((1 + nshift) x B (re, im) doubles: the
 * hashing at a = 0 first, then one per ladder shift of round t).  d_zidx lists the nz indices already
 * in zhat.  Writes up to B entries (d_widx, d_wval) sorted by index, their number in *d_count, |J| in
 * *d_nabove and the number of J decodes kept in *d_nkept.
 */
sfft_status sfft_exact_decode(sfft_plan plan, uint32_t t, uint64_t sigma, uint64_t b, const double* d_u,
                              const uint32_t* d_zidx, uint32_t nz, uint32_t* d_widx, double* d_wval,
                              uint32_t* d_count, uint32_t* d_nabove, uint32_t* d_nkept, void* stream);

/*
 * Description of general-mode round r (Algorithm 2, SparseFFT loop with B_r, k_r): B, the window
 * half-width T, k' = 3 k_r kept by EstimateValues, LocateSignal's level count D_max (Algorithm 3),
 * the number t of regions per level, and per level D (0-based) the integer range of beta
 * ({s n t / 4 w_D, ..., s n t / 2 w_D} rounded inward).  beta_lo/beta_hi hold at least D_max entries.
 * Host-only.  INVALID_ARG for an exact-mode plan.
 */
sfft_status sfft_plan_general_round_info(sfft_plan plan, uint32_t r, uint32_t* B, int64_t* T, uint32_t* kprime,
                                         uint32_t* dmax, uint32_t* t_regions, uint64_t* beta_lo, uint64_t* beta_hi);

/*
 * One LocateInner level (Algorithm 3, procedure LocateInner, after its hashing loop) on caller bins,
 * with general round r's t and the plan's s:  for every bin j with d_valid[j] and each of the nrep
 * rounds q, c_j = phase(u_j / u'_j) (d_u, d_up: nrep x B (re, im) doubles, the hashings at a_q and
 * a_q + beta_q), and region q' in 1..t of [l_j, l_j + w) gets a vote when the circular distance of
 * beta_q theta_{j,q'} and c_j is below s pi.  A bin with no majority region becomes bottom
 * (d_valid[j] = 0); otherwise l_j moves to the start of the four consecutive regions with the most
 * votes.  Region starts d_lfp are fixed point with 16 fraction bits, modulo n 2^16; w_fp is the level's
 * width in the same units.  d_votes receives the B x t vote counts.  B = round r's B.
 */
sfft_status sfft_locate_votes(sfft_plan plan, uint32_t r, uint64_t sigma, uint64_t b, uint64_t w_fp, uint32_t nrep,
                              const uint64_t* d_beta, const double* d_u, const double* d_up, uint64_t* d_lfp,
                              uint8_t* d_valid, uint32_t* d_votes, void* stream);

/*
 * Trace of one general-mode round (Algorithm 2's loop body: LocateSignal, then EstimateValues and
 * zhat += w_J), for checking the pipeline's decisions against a replay of Algorithms 2 and 3 on the
 * pipeline's own bins.  Every pointer is caller-owned device memory of the sizes below, with B, D_max
 * from sfft_plan_general_round_info for `round` and nhash = 2 D_max R_loc + R_est:
 *   d_bins          batch x nhash x B (re, im) doubles: the round's bins after zhat was subtracted
 *                   (HashToBins step 4); rows 2g and 2g + 1 are LocateInner round q of level D + 1
 *                   (g = D R_loc + q, hashings at a_q and a_q + beta_q under the round's sigma, b);
 *                   row 2 D_max R_loc + q is EstimateValues hashing q
 *   d_regions       batch x D_max x B: each bin's region start after each level, fixed point with 16
 *                   fraction bits, modulo n 2^16
 *   d_valid         batch x D_max x B: 1 where the bin still has a region after that level, 0 (bottom)
 *   d_cand          batch x B: each bin's candidate pi^{-1}(tau) after the last level (0xFFFFFFFF for
 *                   bottom), before L is sorted and de-duplicated
 *   d_zidx_before, d_zval_before, d_zcount_before   zhat when the round starts (batch x z_cap
 *                   indices, batch x z_cap (re, im) doubles, batch counts)
 *   d_zidx_after, d_zval_after, d_zcount_after      zhat when the round ends
 */
typedef struct sfft_general_trace {
    uint32_t round;
    uint32_t reserved;         /* 0 */
    double* d_bins;
    uint64_t* d_regions;
    uint8_t* d_valid;
    uint32_t* d_cand;
    uint32_t* d_zidx_before;
    double* d_zval_before;
    uint32_t* d_zcount_before;
    uint32_t* d_zidx_after;
    double* d_zval_after;
    uint32_t* d_zcount_after;
} sfft_general_trace;

/*
 * sfft_execute of a general-mode plan that also records round trace->round into *trace.  The batch
 * runs as one stream group on `stream` (results are those of sfft_execute, bit for bit: requests are
 * independent).  Errors: INVALID_ARG (an exact-mode plan, a null pointer, round out of range), CUDA.
 */
sfft_status sfft_execute_trace(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, void* stream,
                               uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag,
                               const sfft_general_trace* trace);

/*
 * EstimateValues (Algorithm 2, after its hashing loop) on caller bins: for each candidate i of the
 * ascending list d_L (nL <= B), w_i = median_q Re e_q + i median_q Im e_q over the nrep hashings
 * (sigma_q, a_q, b_q) whose window gain W(-o_q(i)) reaches est_gmin, e_q = u^{(q)}_{h_q(i)}
 * w^{-a_q sigma_q i} / W(-o_q(i)) (lower median; 0 when no hashing qualifies); then the kprime
 * largest |w_i| (ties to the smaller index) are written to (d_widx, d_wval) in ascending index order
 * and their number to *d_count.  d_u: nrep x B (re, im) doubles; window of general round r.
 */
sfft_status sfft_estimate_from_bins(sfft_plan plan, uint32_t r, uint32_t nrep, const uint64_t* d_sigma,
                                    const uint64_t* d_b, const uint64_t* d_a, const double* d_u, const uint32_t* d_L,
                                    uint32_t nL, uint32_t kprime, uint32_t* d_widx, double* d_wval, uint32_t* d_count,
                                    void* stream);

/*
 * HashToBins for callers that cannot allocate device memory.  The paper has no counterpart: this is
 * a deployment variant of sfft_hash_to_bins.
 *
 * Who needs it: code that runs where cudaMalloc / cudaFree are not allowed or not wanted -- for
 * example a host that hands out device memory only from its own pool, a latency-critical path where
 * an allocation's implicit synchronisation is unacceptable, or code that is handed fixed buffers and
 * must not touch the allocator at all.  Such a caller cannot create an sfft_plan (plan creation
 * allocates), so this call takes the window itself and keeps its scratch in a fixed array compiled
 * into the library.
 *
 * What it computes: the same bins as sfft_hash_to_bins with explicit (sigma odd, a, b), FP32 data
 * path:  u_j = FFT_B(fold_B(G_t x_{sigma(t-a)} w^{sigma b t}))_j - sum_{i in zhat} W(-o(i)) zhat_i
 * w^{a sigma i} [h(i) = j], written to d_u as B (re, im) doubles.
 *   d_x     n complex64 samples (interleaved float pairs), device
 *   d_taps  T + 1 float taps g_0..g_T of the flat window (g_{-t} = g_t), device
 *   d_wtab  n/(2B) + 1 doubles W(o), o = 0..n/(2B), the window's exact gain; read only when nz > 0
 *           (may be NULL when nz == 0)
 *   d_zidx, d_zval  nz recovered coefficients (uint32 indices, (re, im) doubles); nz <= 4096
 * Every pointer is caller-owned device memory; nothing is allocated or freed.
 *
 * Scratch: partial fold sums and one arrival counter live in a static device array of
 * SFFT_STATIC_SCRATCH_BYTES (4 MiB) that every GPU loading the library holds until the process
 * exits.  A call needs ceil((2T+1) / 2048) * B * 8 + 256 bytes of it; larger requests are rejected
 * with SFFT_ERR_CAPACITY before anything is launched.  n must be a power of two in [2^6, 2^30],
 * B a power of two with 2 <= B <= min(n/2, 4096).
 *
 * All calls share the one array and it keeps the previous call's contents (the counter is cleared
 * on the stream before every launch; the partial sums are overwritten before they are read), so two
 * calls whose work overlaps on the GPU -- on different streams, or from different host threads --
 * race and return wrong bins.  Serialise them.
 *
 * Set-up: the first call on each device (with that device current) looks up the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream capture begins.
 * Errors: INVALID_ARG (null pointer, odd/even sigma, out-of-range a/b/B/T, nz > 4096), CAPACITY
 * (scratch too small), CUDA (set-up or launch failed; see sfft_last_error()).
 */
#define SFFT_STATIC_SCRATCH_BYTES (4u * 1024u * 1024u)
sfft_status sfft_hash_to_bins_static(uint64_t n, uint32_t B, int64_t T, const float* d_taps, const double* d_wtab,
                                     const void* d_x, uint64_t sigma, uint64_t a, uint64_t b, const uint32_t* d_zidx,
                                     const double* d_zval, uint32_t nz, double* d_u, void* stream);

/*
 * Host only (no device needed): the flat-window taps g_0..g_T (g_{-t} = g_t) of bin count B, transition
 * fraction alpha and tolerance delta at length n, as every plan builds them (Sec. 7, with this library's
 * reading: a Gaussian of frequency std alpha / (4 B z), z = sqrt(2 ln(1/delta)), convolved with a
 * box-car of half width (1 - alpha/2) / (2B), times n, cut at T = floor(4 B ln(1/delta) / (pi alpha))).
 * *T receives T; h_taps (cap >= T + 1 entries) may be NULL to query T only.
 */
sfft_status sfft_window_taps(uint64_t n, uint32_t B, double alpha, double delta, int64_t* T, double* h_taps,
                             uint64_t cap);

/*
 * Host only: the exact response of those taps, W(o) = (1/n) (g_0 + 2 sum_{t=1}^{T} g_t cos(2 pi o t / n)),
 * for o = 0..len-1 (len <= n/2 + 1): the gain HashToBins applies to a coefficient at offset o from its
 * bin centre (Lemma "hashtobins").  Plans hold it for |o| <= n/2B; callers of sfft_hash_to_bins_static
 * pass it as d_wtab.  Computed by direct summation or, when that is costlier, as one chirp convolution
 * of length >= len + 4T with a radix-2 FFT (absolute error of order 1e-13).
 */
sfft_status sfft_window_gains(uint64_t n, uint32_t B, double alpha, double delta, uint64_t len, double* h_W);

/*
 * Host only: the twiddle factor tables general-mode plans use for EstimateValues' FP64 terms
 * w^{a sigma i} (Algorithm 2), with w = exp(-2 pi i / n).  For n = 2^L (64 <= n <= 2^30) and
 * sh = ceil(L / 2), h_tw (2^sh + n / 2^sh complex values, (re, im) doubles) receives
 * exp(-2 pi i b / n) for b < 2^sh, then exp(-2 pi i a 2^sh / n) for a < n / 2^sh; then
 * w^e = h_tw[e mod 2^sh] h_tw[2^sh + (e >> sh)].  *len receives the entry count (h_tw may be NULL to
 * query it).  Each entry is within a few ulp of the exact value.
 */
sfft_status sfft_twiddle_tables(uint64_t n, uint64_t* len, double* h_tw, uint64_t cap);

/*
 * Philox4x32-10 as the device computes it (Salmon et al., SC 2011): for i < count, the four output
 * words for key (key0, key1) and counter (ctr[0], ctr[1], ctr[2], ctr[3] + i), written to d_out[4 i..].
 */
sfft_status sfft_philox(uint32_t key0, uint32_t key1, const uint32_t* h_ctr, uint32_t count, uint32_t* d_out,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H */
