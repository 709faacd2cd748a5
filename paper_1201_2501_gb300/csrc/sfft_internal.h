// sfft_internal.h -- plan layout and kernel argument blocks shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sfft.h"

namespace sfft {

constexpr int kThreads = 256;     // threads per CTA of every kernel
constexpr int kChunkTaps = 2048;  // taps per CTA in the gather phase (8 per thread)
constexpr int kMaxHash = 4;       // hashings per exact round: a = 0 plus up to 3 ladder shifts
constexpr uint32_t kCarry = 256;  // zhat entries an exact finisher keeps on chip for the next round
constexpr uint32_t kMaxB = 4096;  // largest B of the fused exact round
constexpr uint32_t kNoIndex = 0xFFFFFFFFu;
constexpr size_t kFinSmemMax = 160 * 1024;  // largest on-chip finisher of the exact round
constexpr uint32_t kMaxRounds = 32;         // rounds of an exact plan (ceil(log2 k) + 1 + extra)

// Per-request descriptor of a launch (device table, optional).  Without a table, request s of a
// launch reads row s of the batch and draws its hashings with the launch's seed and request index s;
// with one, request s reads x, draws with (seed, id), so its result does not depend on which slot of
// which launch it ran in.  period != 0: x holds `period` samples (a power of two dividing n) and the
// transform is that of its periodic extension y_i = x_{i mod period} (Sec. 5), read in place.
struct ReqDesc {
    const void* x;
    uint64_t seed;
    uint32_t id;
    uint32_t period;
};

// One round of the exact schedule (Algorithm 1's loop t = 0..log k, with this library's readings).
struct ExactRound {
    uint32_t B = 0, logB = 0;
    double alpha = 0;
    int64_t T = 0;            // taps t in [-T, T]
    uint32_t nshift = 0;      // ladder length L
    uint64_t shift[4] = {0, 0, 0, 0};
    uint32_t chunks = 0;      // CTAs per request in the gather phase
    uint32_t ctaps = 0;       // taps per CTA (sfft_params.chunk_taps)
    uint32_t stage = 0;       // samples staged per CTA: ctaps + largest shift
    size_t taps_off = 0;      // offset of this round's taps in the tap arrays
    size_t wtab_off = 0;      // offset of this round's W(o), o = 0..n/2B, in the W table (exact rounds:
                              // followed by 1 / W(o) for the same o)
    size_t smem = 0;          // dynamic shared memory of the round kernel
    bool fin_global = false;  // the finisher's arrays do not fit on chip: they live in d_fin
    size_t fin_bytes = 0;     // size of the finisher's arrays of one request
};

// Kernel argument block of the exact round (passed by value).
struct ExactArgs {
    const void* x;             // batch x n complex values (float2 or double2)
    uint64_t n;
    uint32_t nmask;            // n - 1
    uint64_t seed;
    uint32_t round;
    uint32_t req_base;         // request index of blockIdx.y == 0 (a launch may cover part of a batch)
    const ReqDesc* reqs;       // optional per-request table (see ReqDesc)
    uint32_t B, logB;
    int64_t T;
    uint32_t H;                // hashings: hashing h uses offset a_base + a[h]
    uint32_t a_base;           // 0 in the exact rounds; the explicit a of sfft_hash_to_bins
    uint32_t a[kMaxHash];      // a[0] = 0, a[l] = beta_l
    uint64_t shift64[kMaxHash];
    uint32_t chunks, stage, maxshift;
    uint32_t ctaps;            // taps per CTA: chunk c gathers taps [-T + c ctaps, -T + (c + 1) ctaps)
    const float* taps32;
    const double* taps64;
    const double* wtab;
    const double* winv;        // 1 / W(o) for the same o (null: the decode divides by W(o))
    void* part;                // partial fold sums: request s owns [s part_stride, (s + 1) part_stride),
                               // laid out [chunks][H][B] complex R (requests may be in different rounds)
    size_t part_stride;
    uint32_t* counter;         // [batch] arrival counters (zero between launches)
    uint32_t* counter2;        // [batch] the one-launch path's second counters: round t's decode starts
                               // once its bins are ready and round t - 1's decode is done
    uint32_t* zidx;            // [batch][zcap]
    double2* zval;             // [batch][zcap]
    uint32_t* zcount;          // [batch]
    int32_t* zflag;            // [batch] sticky capacity flag
    uint32_t zcap;
    double thr, iso_tol, gmin, prune, ref_lo, ref_hi, ref_tol;
    // the FP32 data path's thresholds, rounded once on the host: thr, iso_tol, ref_lo thr, ref_hi thr,
    // ref_tol, and prune thr rounded up (a float magnitude m is below prune thr iff m < drop_f)
    float thr_f, iso_tol_f, ref_lo_f, ref_hi_f, ref_tol_f, drop_f;
    uint32_t first_round, last_round;
    // outputs written by the last round
    uint32_t* out_idx;
    double2* out_val;
    uint32_t out_cap;
    uint32_t* out_count;
    int32_t* out_flag;
    // the finisher's arrays: in shared memory (fin_scratch null) or, for large B and zcap, in the
    // global region [s fin_stride, (s + 1) fin_stride) of fin_scratch (only one CTA per request uses it)
    unsigned char* fin_scratch;
    size_t fin_stride;
    // single-hashing mode (sfft_hash_to_bins): explicit (sigma, b), bins written to ubins, no decode
    int bins_only;
    uint32_t e_sigma, e_b, e_nz;
    double2* ubins;
};

// One launch of the exact algorithm over a batch: every round's gather chunks at once, grouped by
// round (segment t = chunks_t x batch CTAs, request-major, chunk fastest), since no sample position
// depends on zhat.  A round's finisher comes in two parts.  Its bins (partial sums, B-point FFT) need
// only the round's chunks: the last chunk to arrive computes them (counter) and leaves them in the
// request's partial-fold area.  Its decode (subtraction of zhat, location, estimation, merge) also
// needs round t - 1's zhat: whichever arrives last at counter2 -- the bins part, or round t - 1's
// decode -- runs it, then arrives at round t + 1's counter2.  Nobody waits.  The round
// blocks (tables, workspace and this launch's signal and outputs) travel in the kernel parameters,
// NR of them (8, 16 or 32: the smallest that holds the plan's rounds).
template <int NR>
struct StepParams {
    uint32_t R;
    uint32_t seg[NR + 1];  // first CTA of each round's segment; seg[R] = grid size
    ExactArgs r[NR];
};

// Multi-channel batches with shared hashing (sfft_execute_channels): C signals sampled at the same
// times and stored interleaved, x[m][c], all transformed with the draws of one request (seed, id).
// One CTA gathers the samples s = s0 + i (s0 = -T - maxshift) of round t whose index i falls in
// residue class rho mod B_t, chunk c of kChanRows consecutive rows of that class: the rows (C
// contiguous values each) are staged in shared memory by bulk copies, and thread ch folds channel
// ch.  The ladder's shifts are multiples of B_t, so every hashing of the round puts sample s in bin
// s mod B_t: a channel's H_t sums are one bin each.  The partial folds go to the channel slot's
// partial-fold area laid out as the one-launch path's ([chunk][H][B] per round, round t at
// chan_off[t]); then every (round, slot) forms its bins at once, and one CTA per slot runs the
// decodes in order.
constexpr uint32_t kChanRows = 16;   // rows of a residue class per CTA (one lane of warp 0 each)
static_assert(kChanRows <= 32, "warp 0 issues one row copy per lane");
constexpr uint32_t kChanMaxC = 256;  // channels of one batch (a row of the stage holds them all)
template <int NR>
struct ChanParams {
    uint32_t R;               // rounds
    uint32_t C;               // channels (a multiple of 32, at most kChanMaxC)
    uint32_t cseg[NR + 1];    // first CTA of each round's segment; cseg[R] = CTAs
    uint64_t seed;
    uint32_t id;              // request index of the shared draws
    const void* x;            // n x C complex64, 16-byte aligned
    uint32_t* error;          // set when a bulk copy did not complete within the wait limit
    ExactArgs r[NR];          // round blocks; part at the round's channel layout, chunks = its chunks
};

// The persistent exact path: requests of different plans (n, k, schedule) in one launch, their
// rounds driven by a device work queue.  Item = (request, round, chunk); the CTA that finishes a
// request's round publishes the chunks of its next round.  rdesc holds one argument block per
// (plan, round) with the plan's tables; the per-request fields are pointed at the request's own
// workspace (as slot 0) by the kernel.
struct PersistArgs {
    const ExactArgs* rdesc;         // [sum of the plans' rounds]
    const ReqDesc* reqs;            // [nreq]
    const uint32_t* req_rd0;        // [nreq] index in rdesc of the request's round 0
    const uint32_t* req_rounds;     // [nreq]
    unsigned long long* items;      // [total] (bit 63: published)
    uint32_t* head;                 // items taken
    uint32_t* tail;                 // items reserved
    uint32_t total;
    unsigned char* part;            // [nreq][part_stride] bytes
    size_t part_stride;
    uint32_t* counter;              // [nreq] (zero between rounds)
    uint32_t* zidx;                 // [nreq][z_stride]
    double2* zval;
    size_t z_stride;
    uint32_t* zcount;               // [nreq]
    int32_t* zflag;                 // [nreq]
    unsigned char* fin;             // [nreq][fin_stride] bytes (rounds with fin_global)
    size_t fin_stride;
    uint32_t* out_idx;              // [nreq][out_cap]
    double2* out_val;
    uint32_t out_cap;
    uint32_t* out_count;            // [nreq]
    int32_t* out_flag;              // [nreq]
    int32_t* error;                 // set when a wait for an item ran out
};

struct DecodeArgs {
    uint64_t n;
    uint32_t nmask;
    uint32_t B, logB, H;
    uint64_t shift64[kMaxHash];
    uint32_t sigma, b;
    const double* wtab;
    const double2* u;          // H x B
    const uint32_t* zidx;
    uint32_t nz;
    double thr, iso_tol, gmin, ref_lo, ref_hi, ref_tol;
    uint32_t* widx;
    double2* wval;
    uint32_t* count;
    uint32_t* nabove;
    uint32_t* nkept;
    int fp64;                  // transcendental precision of the decode (that of the plan's data path)
};

// ---- general mode (Algorithms 2 and 3) ----
constexpr int kMaxLevels = 16;   // LocateSignal levels D_max
constexpr int kMaxRloc = 15;     // LocateInner rounds per level
constexpr int kMaxRest = 15;     // EstimateValues hashings
constexpr int kMaxT = 32;        // regions per level t
constexpr int kFracBits = 16;    // fixed-point fraction bits of region positions

struct GeneralRound {
    uint32_t kr = 0, kprime = 0;   // k_r and k' = 3 k_r
    uint32_t B = 0, logB = 0;
    int64_t T = 0;
    uint32_t chunks = 0;           // 2048-tap chunks of the window
    uint32_t cpb = 0;              // chunks per CTA of the gather launch
    uint32_t ctas = 0;             // CTAs per hashing group and request
    uint32_t dmax = 0, t = 0, logtp = 0;
    uint64_t beta_lo[kMaxLevels] = {}, beta_hi[kMaxLevels] = {};
    uint32_t npairs = 0, ngroups = 0, nhash = 0;
    size_t taps_off = 0, wtab_off = 0;
    size_t smem_gather = 0, smem_finish = 0, smem_locate = 0, smem_estimate = 0;
    bool fin_global = false, est_global = false;  // arrays too large for shared memory: in d_gfin / d_gest
    bool perm = false;             // the pairs read the permuted copy x_{sigma m} (written first)
};

// Kernel argument block of the general-mode kernels of one round (passed by value).
struct GenArgs {
    const float2* x;
    float2* xperm;         // [batch][n] x_{sigma m} under the round's LocateInner sigma, or null
    uint64_t n;
    uint32_t nmask, logn;
    uint64_t seed;
    uint32_t round;
    uint32_t req_base;     // request index of the launch's first request
    const ReqDesc* reqs;   // optional per-request table (see ReqDesc)
    uint32_t B, logB;
    int64_t T;
    uint32_t chunks, cpb, ctas;
    uint32_t dmax, t, logtp, R_loc, R_est, npairs, ngroups, nhash, kprime;
    uint64_t beta_lo[kMaxLevels], beta_hi[kMaxLevels];
    double s, est_gmin;
    const float* taps;
    const double* wtab;
    const double2* tw;     // FP64 twiddles w^e = tw[e mod 2^tw_shift] tw[2^tw_shift + (e >> tw_shift)]
    uint32_t tw_shift;
    float2* part;          // [batch][ngroups][ctas][2][B]; after the gather, ctas slot 0 holds the sum
    size_t part_stride;    // elements per request
    uint32_t* gcount;      // [batch][ngroups] arrival counters of the gather CTAs (zero between launches)
    uint32_t* ecount;      // [batch] arrival counters of the estimate CTAs (zero between launches)
    double2* est_w;        // [batch][B] candidates' estimates shared by a request's estimate CTAs
    double* est_mag;       // [batch][B] their squared magnitudes
    unsigned char* fin_scratch;  // k_gen_finish arrays in device memory: [batch][ngroups][fin_stride], or null
    size_t fin_stride;
    unsigned char* est_scratch;  // k_gen_estimate arrays in device memory: [batch][est_stride], or null
    size_t est_stride;
    double2* bins;         // [batch][nhash][B]  (hashing 2g, 2g+1: pair g; 2 npairs + q: estimate q)
    double* phase;         // [batch][npairs][B] phase(u_a conj(u_{a+beta})) / 2 pi
    size_t bins_stride, phase_stride;  // elements per request
    uint32_t* L;           // [batch][B] candidate frequencies
    uint32_t* nL;          // [batch]
    uint32_t* zidx;        // [batch][zcap]
    double2* zval;
    uint32_t* zcount;
    int32_t* zflag;
    uint32_t zcap;
    uint32_t last_round;
    uint32_t* out_idx;
    double2* out_val;
    uint32_t out_cap;
    uint32_t* out_count;
    int32_t* out_flag;
    uint64_t* dbg_lfp;     // trace (or null): [batch][dmax][B] region starts after each LocateInner level
    uint8_t* dbg_valid;    // trace (or null): [batch][dmax][B] 0 where the bin is bottom after that level
};

// One LocateInner level on caller bins (sfft_locate_votes).
struct VoteArgs {
    uint64_t n;
    uint32_t nmask, B, t, nrep;
    uint32_t sigma, b;
    uint64_t w_fp;
    double s;
    const double2* u;      // nrep x B
    const double2* up;     // nrep x B
    const uint64_t* beta;  // nrep
    uint64_t* l_fp;        // B (in/out)
    uint8_t* valid;        // B (in/out)
    uint32_t* votes;       // B x t (out)
};

// EstimateValues on caller bins (sfft_estimate_from_bins).
struct EstArgs {
    uint64_t n;
    uint32_t nmask, B, logB, nrep, nL, kprime;
    const uint64_t* sig;
    const uint64_t* bb;
    const uint64_t* aa;
    const double2* u;      // nrep x B
    const uint32_t* L;     // nL, ascending
    const double* wtab;
    const double2* tw;     // as GenArgs::tw
    uint32_t tw_shift;
    double est_gmin;
    uint32_t* widx;
    double2* wval;
    uint32_t* count;
};

}  // namespace sfft

struct sfft_plan_s {
    sfft_params p{};
    uint32_t max_batch = 0;
    uint32_t max_B = 0, max_groups = 0;  // largest B and number of hashing groups over the rounds
    int device = 0;
    std::vector<sfft::ExactRound> rounds;
    std::vector<sfft::GeneralRound> grounds;  // general mode
    double2* d_bins = nullptr;
    double* d_phase = nullptr;
    uint32_t* d_L = nullptr;  // general mode: per round r, [max_batch][B_r] candidates
    double2* d_tw = nullptr;  // general mode: FP64 twiddle factor tables (2^tw_shift + n / 2^tw_shift)
    uint32_t tw_shift = 0;
    uint32_t* d_nL = nullptr;
    float2* d_xperm = nullptr;  // general mode, rounds with perm: [max_batch][n] permuted signals
    // general mode: per round r, [max_batch][B_r] estimates; then per round [max_batch][B_r] magnitudes
    double2* d_estw = nullptr;
    size_t bins_stride = 0, phase_stride = 0;
    std::vector<double> taps_host;  // every round's taps, FP64
    std::vector<double> wtab_host;  // every round's W(o), o = 0..n/2B
    float* d_taps32 = nullptr;
    double* d_taps64 = nullptr;
    double* d_wtab = nullptr;
    size_t wtab_len = 0;
    void* d_part = nullptr;
    size_t part_bytes = 0;
    size_t part_stride = 0;  // elements of the partial-fold buffer owned by one request
    // arrival counters, zero between launches: exact [2 R][max_batch]; general, per round r,
    // [max_batch][ngroups_r] for the gather, then [max_batch] for the estimate
    uint32_t* d_counter = nullptr;
    std::vector<sfft::ExactArgs> rdesc;  // [R] round blocks of the one-launch exact path
    std::vector<size_t> chan_off;        // exact FP32: round t's partial folds in a channel slot's area
    std::vector<uint32_t> chan_chunks;   // exact FP32: chunks of kChanRows rows per residue class
    size_t step_smem = 0;                // its dynamic shared memory (largest round)
    uint32_t* d_zidx = nullptr;
    double2* d_zval = nullptr;
    uint32_t* d_zcount = nullptr;
    int32_t* d_zflag = nullptr;
    // single-step helpers
    double2* d_ubins = nullptr;
    uint32_t* d_aux = nullptr;
    sfft::ReqDesc* d_reqs = nullptr;  // [max_batch] request table of sfft_execute_requests
    // page-locked copies of the table the caller passes (two, used in turn): the copy to d_reqs reads
    // them asynchronously, so a caller's array (possibly freed at once) is never read by the device
    sfft::ReqDesc* h_reqs[2] = {nullptr, nullptr};
    cudaEvent_t ev_reqs[2] = {nullptr, nullptr};
    int reqs_cur = 0;
    // finisher arrays of the exact rounds with fin_global: per such round, [max_batch][fin_stride]
    unsigned char* d_fin = nullptr;
    size_t fin_stride = 0;
    // general mode, per round r with fin_global: [max_batch][ngroups_r][gfin_stride]
    unsigned char* d_gfin = nullptr;
    size_t gfin_stride = 0, gfin_groups = 0;  // gfin_groups: ngroups summed over those rounds
    unsigned char* d_gest = nullptr;  // general mode: [max_batch][gest_stride]
    size_t gest_stride = 0;
    size_t dev_bytes = 0;          // device memory allocated at plan creation
    uint64_t samples = 0;          // samples one transform gathers (all rounds, all hashings)
    // internal streams: a batch is split into groups whose rounds run on their own streams
    static constexpr int kMaxStreams = 8;
    uint32_t nstreams = 1;
    cudaStream_t aux[kMaxStreams] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kMaxStreams] = {};
    // host-entry staging
    void* d_stage = nullptr;
    size_t stage_bytes = 0;
    uint32_t* d_out_idx = nullptr;
    double* d_out_val = nullptr;
    uint32_t* d_out_count = nullptr;
    int32_t* d_out_flag = nullptr;
    size_t out_cap = 0;
};

namespace sfft {
// sfft_plan_create; with `tables` (a plan of the same parameters) the host schedule and window
// tables are copied from it instead of computed
sfft_status plan_create(const sfft_params* p, uint32_t max_batch, const sfft_plan_s* tables, sfft_plan_s** out);
// the checks sfft_plan_create applies to a parameter set (without allocating anything)
sfft_status validate_params(const sfft_params* p);
// host-side plan construction (sfft_host.cu)
sfft_status build_exact_schedule(sfft_plan_s* pl);
// One batch through every round of the plan's mode: rows of d_x, or the device request table d_reqs
// when it is not null (then d_x and seed are unused).  Arguments are checked by the callers.
sfft_status execute_batch(sfft_plan_s* plan, const void* d_x, const ReqDesc* d_reqs, uint32_t batch, uint64_t seed,
                          cudaStream_t st, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                          int32_t* d_flag);
void window_taps_host(uint64_t n, uint32_t B, double alpha, double delta, int64_t T, double* g);
inline uint32_t ilog2_host(uint64_t v) {  // v a power of two
    uint32_t l = 0;
    while ((uint64_t(1) << l) < v) ++l;
    return l;
}
// FP64 twiddle factor tables for n = 2^L and split sh: out[b] = exp(-2 pi i b / n), b < 2^sh, then
// out[2^sh + a] = exp(-2 pi i a 2^sh / n), a < n / 2^sh
void twiddle_tables_host(uint64_t n, uint32_t sh, std::vector<double2>* out);
void window_table_host(uint64_t n, const double* g, int64_t T, uint64_t len, double* W);
int64_t window_halfwidth(uint32_t B, double alpha, double delta);
void draw_exact_host(uint64_t seed, uint32_t request, uint32_t round, uint64_t n, uint64_t* sigma, uint64_t* b);
void set_last_error(const std::string& s);

// device entry points (sfft_exact.cu)
cudaError_t launch_exact_round(const ExactArgs& a, uint32_t batch, size_t smem, cudaStream_t st, bool fp64);
// rounds[0..R) with this launch's fields filled in; grid = sum over rounds of chunks x batch
cudaError_t launch_exact_step(const ExactArgs* rounds, uint32_t R, uint32_t batch, size_t smem, cudaStream_t st,
                              bool fp64);
// multi-channel batch with shared hashing: the gather (one CTA per round, residue and chunk) between
// two optional events, the bins of every (round, slot), then one CTA per slot for the
// decodes; rounds[t].part and .chunks give each round's channel layout; error: a device word the
// gather sets when a bulk copy times out (cleared here first)
cudaError_t launch_exact_channels(const ExactArgs* rounds, uint32_t R, uint32_t C, const void* x, uint64_t seed,
                                  uint32_t id, size_t smem, uint32_t* error, cudaStream_t st, cudaEvent_t before,
                                  cudaEvent_t after);
// persistent path: CTAs that fit on the device at `smem`, and the launch
int exact_persistent_ctas(size_t smem, bool fp64);
cudaError_t launch_exact_persistent(const PersistArgs& a, uint32_t ctas, size_t smem, cudaStream_t st, bool fp64);
cudaError_t launch_exact_decode(const DecodeArgs& a, cudaStream_t st);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t count, uint32_t* out, cudaStream_t st);
// general mode (sfft_general.cu, sfft_host.cu)
sfft_status build_general_schedule(sfft_plan_s* pl);
size_t general_finish_smem(uint32_t B, uint32_t zcap);
size_t general_locate_smem(uint32_t B);
size_t general_estimate_smem(uint32_t B, uint32_t kprime, uint32_t zcap);
cudaError_t general_set_smem(size_t gather, size_t finish, size_t locate, size_t estimate);
cudaError_t launch_general_round(const GenArgs& a, uint32_t batch, const GeneralRound& r, cudaStream_t st);
cudaError_t launch_locate_votes(const VoteArgs& a, cudaStream_t st);
cudaError_t launch_estimate_from_bins(const EstArgs& a, cudaStream_t st);
size_t exact_finish_smem(uint32_t B, uint32_t H, uint32_t zcap, bool fp64);
size_t exact_gather_smem(uint32_t stage, bool fp64);
cudaError_t set_exact_smem_limit(size_t bytes, bool fp64);
}  // namespace sfft
