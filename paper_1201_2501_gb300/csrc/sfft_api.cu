// sfft_api.cu -- the C ABI of libsfft.so (declared in include/sfft.h): plans, whole transforms and
// single steps.  Everything here is host code that validates arguments and enqueues kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <limits>
#include <new>
#include <string>

#include "philox.cuh"
#include "sfft_internal.h"

using namespace sfft;

namespace {

sfft_status cuda_fail(cudaError_t e, const char* what) {
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return SFFT_ERR_CUDA;
}

#define SFFT_CUDA(call, what)                       \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }

sfft_status validate(const sfft_params* p) {
    if (!p) return SFFT_ERR_INVALID_ARG;
    if (!is_pow2(p->n) || p->n < 64 || p->n > (uint64_t(1) << 30)) return SFFT_ERR_N_NOT_POW2;
    if (p->k == 0 || (uint64_t)p->k > p->n / 4) return SFFT_ERR_K_RANGE;
    if (p->mode != SFFT_EXACT && p->mode != SFFT_GENERAL) return SFFT_ERR_INVALID_ARG;
    if (p->precision != SFFT_FP32 && p->precision != SFFT_FP64) return SFFT_ERR_INVALID_ARG;
    if (!(p->delta > 0 && p->delta < 0.5)) return SFFT_ERR_INVALID_ARG;
    if (!(p->alpha0 > 0 && p->alpha0 < 1)) return SFFT_ERR_INVALID_ARG;
    if (!(p->bins_per_k > 0) || p->B_min < 2 || !is_pow2(p->B_min)) return SFFT_ERR_INVALID_ARG;
    if (!(p->thr > 0) || !(p->tau_dec > 0 && p->tau_dec < 1) || !(p->iso_tol > 0)) return SFFT_ERR_INVALID_ARG;
    if (p->z_cap == 0 || p->z_cap > 4096) return SFFT_ERR_INVALID_ARG;
    if (p->gain > 1) return SFFT_ERR_INVALID_ARG;
    if (p->chunk_taps != 0 && (!is_pow2(p->chunk_taps) || p->chunk_taps < 256 || p->chunk_taps > 8192))
        return SFFT_ERR_INVALID_ARG;
    return SFFT_OK;
}

void free_plan(sfft_plan_s* pl) {
    if (!pl) return;
    cudaFree(pl->d_taps32);
    cudaFree(pl->d_taps64);
    cudaFree(pl->d_wtab);
    cudaFree(pl->d_tw);
    cudaFree(pl->d_part);
    cudaFree(pl->d_counter);
    cudaFree(pl->d_zidx);
    cudaFree(pl->d_zval);
    cudaFree(pl->d_zcount);
    cudaFree(pl->d_zflag);
    cudaFree(pl->d_ubins);
    cudaFree(pl->d_aux);
    cudaFree(pl->d_reqs);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(pl->h_reqs[i]);
        if (pl->ev_reqs[i]) cudaEventDestroy(pl->ev_reqs[i]);
    }
    cudaFree(pl->d_fin);
    cudaFree(pl->d_gfin);
    cudaFree(pl->d_gest);
    cudaFree(pl->d_stage);
    cudaFree(pl->d_out_idx);
    cudaFree(pl->d_out_val);
    cudaFree(pl->d_out_count);
    cudaFree(pl->d_out_flag);
    cudaFree(pl->d_bins);
    cudaFree(pl->d_phase);
    cudaFree(pl->d_L);
    cudaFree(pl->d_nL);
    cudaFree(pl->d_estw);
    cudaFree(pl->d_xperm);
    for (int i = 0; i < sfft_plan_s::kMaxStreams; ++i) {
        if (pl->aux[i]) cudaStreamDestroy(pl->aux[i]);
        if (pl->ev_join[i]) cudaEventDestroy(pl->ev_join[i]);
    }
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    delete pl;
}

ExactArgs base_args(const sfft_plan_s* pl, const ExactRound& r, uint32_t t) {
    ExactArgs a;
    std::memset(&a, 0, sizeof(a));
    const sfft_params& p = pl->p;
    a.n = p.n;
    a.nmask = (uint32_t)(p.n - 1);
    a.round = t;
    a.B = r.B;
    a.logB = r.logB;
    a.T = r.T;
    a.H = 1 + r.nshift;
    a.a_base = 0;
    a.a[0] = 0;
    a.shift64[0] = 0;
    for (uint32_t l = 0; l < r.nshift; ++l) {
        a.a[l + 1] = (uint32_t)r.shift[l];
        a.shift64[l + 1] = r.shift[l];
    }
    a.chunks = r.chunks;
    a.ctaps = r.ctaps;
    a.stage = r.stage;
    a.maxshift = (uint32_t)r.shift[r.nshift - 1];
    a.taps32 = pl->d_taps32 + r.taps_off;
    a.taps64 = pl->d_taps64 + r.taps_off;
    a.wtab = pl->d_wtab + r.wtab_off;
    a.winv = a.wtab + (p.n / r.B) / 2 + 1;  // the exact schedule stores 1 / W(o) after W(o)
    a.part = pl->d_part;
    a.part_stride = pl->part_stride;
    a.fin_scratch = r.fin_global ? pl->d_fin : nullptr;
    a.fin_stride = pl->fin_stride;
    a.counter = pl->d_counter;
    a.zidx = pl->d_zidx;
    a.zval = pl->d_zval;
    a.zcount = pl->d_zcount;
    a.zflag = pl->d_zflag;
    a.zcap = p.z_cap;
    a.thr = p.thr;
    a.iso_tol = p.iso_tol;
    a.gmin = p.gmin;
    a.prune = p.prune;
    a.ref_lo = p.ref_lo;
    a.ref_hi = p.ref_hi;
    a.ref_tol = p.ref_tol;
    a.thr_f = (float)p.thr;
    a.iso_tol_f = (float)p.iso_tol;
    a.ref_lo_f = (float)(p.ref_lo * p.thr);
    a.ref_hi_f = (float)(p.ref_hi * p.thr);
    a.ref_tol_f = (float)p.ref_tol;
    const double drop = p.prune * p.thr;
    a.drop_f = (float)drop;
    if ((double)a.drop_f < drop) a.drop_f = std::nextafter(a.drop_f, std::numeric_limits<float>::infinity());
    return a;
}

}  // namespace

// sfft_execute_requests copies the caller's table byte for byte into the device table
static_assert(sizeof(ReqDesc) == sizeof(sfft_request), "request table layout");
static_assert(offsetof(ReqDesc, x) == offsetof(sfft_request, d_x) && offsetof(ReqDesc, seed) == offsetof(sfft_request, seed) &&
                  offsetof(ReqDesc, id) == offsetof(sfft_request, id) &&
                  offsetof(ReqDesc, period) == offsetof(sfft_request, period),
              "request table layout");

sfft_status sfft::validate_params(const sfft_params* p) {
    const sfft_status st = validate(p);
    if (st != SFFT_OK) return st;
    if (p->mode == SFFT_GENERAL && p->precision != SFFT_FP32) return SFFT_ERR_INVALID_ARG;
    return SFFT_OK;
}

// Plan creation; with `tables` (a plan of the same parameters) its schedule and host window tables
// are copied instead of computed again.
sfft_status sfft::plan_create(const sfft_params* p, uint32_t max_batch, const sfft_plan_s* tables, sfft_plan* out) {
    if (!out) return SFFT_ERR_INVALID_ARG;
    *out = nullptr;
    sfft_status st = validate(p);
    if (st != SFFT_OK) return st;
    if (max_batch == 0) return SFFT_ERR_INVALID_ARG;
    const bool general = p->mode == SFFT_GENERAL;
    if (general && p->precision != SFFT_FP32) return SFFT_ERR_INVALID_ARG;  // general mode: FP32 data path
    sfft_plan_s* pl = new (std::nothrow) sfft_plan_s();
    if (!pl) return SFFT_ERR_OOM;
    pl->p = *p;
    pl->max_batch = max_batch;
    cudaGetDevice(&pl->device);
    if (tables) {
        pl->rounds = tables->rounds;
        pl->grounds = tables->grounds;
        pl->taps_host = tables->taps_host;
        pl->wtab_host = tables->wtab_host;
        pl->wtab_len = tables->wtab_len;
    } else {
        st = general ? build_general_schedule(pl) : build_exact_schedule(pl);
    }
    if (st != SFFT_OK) {
        free_plan(pl);
        return st;
    }
    const bool fp64 = p->precision == SFFT_FP64;
    // taps (FP32 and FP64 copies) and the W tables
    const size_t ntaps = pl->taps_host.size();
    std::vector<float> t32(ntaps);
    for (size_t i = 0; i < ntaps; ++i) t32[i] = (float)pl->taps_host[i];
    size_t part_elems = 0, max_smem = 0, gs_max = 0, fs_max = 0, ls_max = 0, es_max = 0;
    uint32_t maxB = 0, max_groups = 0;
    size_t sum_groups = 0, sum_B = 0;  // general: hashing groups and bins over all rounds
    // exact mode: every round's partial folds live at once (the one-launch path gathers all rounds
    // before their finishers), round t at part_off[t] of a request's region
    std::vector<size_t> part_off;
    if (!general && pl->rounds.size() > kMaxRounds) {
        free_plan(pl);
        return SFFT_ERR_K_RANGE;
    }
    for (const ExactRound& r : pl->rounds) {
        pl->samples += 2 * (uint64_t)r.T + 1 + r.shift[r.nshift - 1];
        part_off.push_back(part_elems);
        part_elems += (size_t)r.chunks * (1 + r.nshift) * r.B;
        if (r.smem > max_smem) max_smem = r.smem;
        if (r.B > maxB) maxB = r.B;
        if (r.fin_global && r.fin_bytes > pl->fin_stride) pl->fin_stride = (r.fin_bytes + 255) & ~size_t(255);
    }
    if (!general && !fp64) {  // the partial folds of a multi-channel batch (sfft_execute_channels)
        size_t chan_elems = 0;
        for (const ExactRound& r : pl->rounds) {
            const uint64_t cnt = 2 * (uint64_t)r.T + 1 + r.shift[r.nshift - 1];
            const uint64_t rows = (cnt + r.B - 1) / r.B;  // rows of the largest residue class
            const uint32_t chunks = (uint32_t)((rows + kChanRows - 1) / kChanRows);
            pl->chan_off.push_back(chan_elems);
            pl->chan_chunks.push_back(chunks);
            chan_elems += (size_t)chunks * (1 + r.nshift) * r.B;
        }
        if (chan_elems > part_elems) part_elems = chan_elems;
    }
    for (const GeneralRound& r : pl->grounds) {
        pl->samples += (uint64_t)r.nhash * (2 * (uint64_t)r.T + 1);
        const size_t e = (size_t)r.ngroups * r.ctas * 2 * r.B;
        if (e > part_elems) part_elems = e;
        if ((size_t)r.nhash * r.B > pl->bins_stride) pl->bins_stride = (size_t)r.nhash * r.B;
        if ((size_t)r.npairs * r.B > pl->phase_stride) pl->phase_stride = (size_t)r.npairs * r.B;
        if (r.B > maxB) maxB = r.B;
        if (r.ngroups > max_groups) max_groups = r.ngroups;
        sum_groups += r.ngroups;
        sum_B += r.B;
        gs_max = r.smem_gather > gs_max ? r.smem_gather : gs_max;
        if (r.fin_global) {
            pl->gfin_stride = std::max(pl->gfin_stride, (r.smem_finish + 255) & ~size_t(255));
            pl->gfin_groups += r.ngroups;  // each such round has its own region
        } else {
            fs_max = r.smem_finish > fs_max ? r.smem_finish : fs_max;
        }
        if (r.est_global) pl->gest_stride = std::max(pl->gest_stride, (r.smem_estimate + 255) & ~size_t(255));
        ls_max = r.smem_locate > ls_max ? r.smem_locate : ls_max;
        if (!r.est_global) es_max = r.smem_estimate > es_max ? r.smem_estimate : es_max;
    }
    pl->part_stride = part_elems;
    pl->max_B = maxB;
    pl->max_groups = max_groups;
    pl->part_bytes = part_elems * (size_t)max_batch * (fp64 ? 16 : 8);
    cudaError_t e = cudaSuccess;
#define SFFT_ALLOC(ptr, bytes)                                        \
    do {                                                              \
        e = cudaMalloc((void**)&(ptr), (bytes));                      \
        pl->dev_bytes += (bytes);                                     \
        if (e != cudaSuccess) {                                       \
            set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e)); \
            free_plan(pl);                                            \
            return SFFT_ERR_OOM;                                      \
        }                                                             \
    } while (0)
    SFFT_ALLOC(pl->d_taps32, ntaps * sizeof(float));
    SFFT_ALLOC(pl->d_taps64, ntaps * sizeof(double));
    SFFT_ALLOC(pl->d_wtab, pl->wtab_len * sizeof(double));
    SFFT_ALLOC(pl->d_part, pl->part_bytes);
    // arrival counters: per (round, request) twice in exact mode; in general mode per (round, request,
    // hashing group), each round in its own region because stream groups may run different rounds at
    // once, then per request
    const size_t ncounters = (size_t)max_batch * (general ? sum_groups + 1 : 2 * pl->rounds.size());
    SFFT_ALLOC(pl->d_counter, ncounters * sizeof(uint32_t));

    SFFT_ALLOC(pl->d_zidx, (size_t)max_batch * p->z_cap * sizeof(uint32_t));
    SFFT_ALLOC(pl->d_zval, (size_t)max_batch * p->z_cap * sizeof(double2));
    SFFT_ALLOC(pl->d_zcount, (size_t)max_batch * sizeof(uint32_t));
    SFFT_ALLOC(pl->d_zflag, (size_t)max_batch * sizeof(int32_t));
    SFFT_ALLOC(pl->d_ubins, (size_t)maxB * kMaxHash * sizeof(double2));
    SFFT_ALLOC(pl->d_aux, 64 * sizeof(uint32_t));
    SFFT_ALLOC(pl->d_reqs, (size_t)max_batch * sizeof(ReqDesc));
    for (int i = 0; i < 2; ++i) {
        if (cudaMallocHost((void**)&pl->h_reqs[i], (size_t)max_batch * sizeof(ReqDesc)) != cudaSuccess ||
            cudaEventCreateWithFlags(&pl->ev_reqs[i], cudaEventDisableTiming) != cudaSuccess) {
            set_last_error("page-locked request table");
            cudaGetLastError();
            free_plan(pl);
            return SFFT_ERR_OOM;
        }
    }
    // one slice per request serves every such round: only the decode part of a finisher uses it (the
    // one-launch path forms a round's bins in the CTA's shared memory), and a request's decodes run one
    // after another (round t + 1's waits for round t's arrival on the request's second counter)
    if (pl->fin_stride) SFFT_ALLOC(pl->d_fin, pl->fin_stride * max_batch);
    if (pl->gfin_stride) SFFT_ALLOC(pl->d_gfin, pl->gfin_stride * pl->gfin_groups * max_batch);
    if (pl->gest_stride) SFFT_ALLOC(pl->d_gest, pl->gest_stride * max_batch);
    if (general) {
        SFFT_ALLOC(pl->d_bins, pl->bins_stride * max_batch * sizeof(double2));
        SFFT_ALLOC(pl->d_phase, pl->phase_stride * max_batch * sizeof(double));
        SFFT_ALLOC(pl->d_L, sum_B * max_batch * sizeof(uint32_t));
        pl->tw_shift = (ilog2_host(p->n) + 1) / 2;
        SFFT_ALLOC(pl->d_tw, ((size_t(1) << pl->tw_shift) + (p->n >> pl->tw_shift)) * sizeof(double2));
        SFFT_ALLOC(pl->d_nL, (size_t)max_batch * sizeof(uint32_t));
        SFFT_ALLOC(pl->d_estw, (size_t)max_batch * sum_B * (sizeof(double2) + sizeof(double)));
        bool perm = false;
        for (const GeneralRound& r : pl->grounds) perm = perm || r.perm;
        if (perm) SFFT_ALLOC(pl->d_xperm, (size_t)max_batch * p->n * sizeof(float2));
    }
#undef SFFT_ALLOC
    auto fail = [&](cudaError_t err, const char* what) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(err));
        free_plan(pl);
        return SFFT_ERR_CUDA;
    };
    if ((e = cudaMemcpy(pl->d_taps32, t32.data(), ntaps * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "upload taps");
    if ((e = cudaMemcpy(pl->d_taps64, pl->taps_host.data(), ntaps * sizeof(double), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return fail(e, "upload taps");
    if (general) {  // twiddle factor tables of the FP64 estimates
        std::vector<double2> tw;
        twiddle_tables_host(p->n, pl->tw_shift, &tw);
        if ((e = cudaMemcpy(pl->d_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e, "upload twiddle tables");
    }
    if ((e = cudaMemcpy(pl->d_wtab, pl->wtab_host.data(), pl->wtab_len * sizeof(double), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return fail(e, "upload window table");
    if ((e = cudaMemset(pl->d_counter, 0, ncounters * sizeof(uint32_t))) != cudaSuccess)
        return fail(e, "clear counters");
    if (!general) {  // the round blocks of the one-launch path (each launch fills in its own fields)
        const size_t csize = fp64 ? 16 : 8;
        for (uint32_t t = 0; t < (uint32_t)pl->rounds.size(); ++t) {
            ExactArgs a = base_args(pl, pl->rounds[t], t);
            a.part = static_cast<unsigned char*>(pl->d_part) + part_off[t] * csize;
            a.counter = pl->d_counter + (size_t)t * max_batch;
            a.counter2 = pl->d_counter + (size_t)(pl->rounds.size() + t) * max_batch;
            a.first_round = t == 0;
            a.last_round = t + 1 == pl->rounds.size();
            pl->rdesc.push_back(a);
        }
        pl->step_smem = max_smem;
    }
    // default stream groups: one for the exact path (its single launch per batch already overlaps
    // rounds; groups only add concurrent tails), four for the general path's per-round kernel chain
    pl->nstreams = p->streams != 0 ? p->streams : (general ? 4 : 1);
    if (pl->nstreams > (uint32_t)sfft_plan_s::kMaxStreams) pl->nstreams = sfft_plan_s::kMaxStreams;
    if ((e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming)) != cudaSuccess)
        return fail(e, "create event");
    for (uint32_t i = 0; i < pl->nstreams; ++i) {
        if ((e = cudaStreamCreateWithFlags(&pl->aux[i], cudaStreamNonBlocking)) != cudaSuccess)
            return fail(e, "create stream");
        if ((e = cudaEventCreateWithFlags(&pl->ev_join[i], cudaEventDisableTiming)) != cudaSuccess)
            return fail(e, "create event");
    }
    if (!general && (e = set_exact_smem_limit(max_smem, fp64)) != cudaSuccess) return fail(e, "shared memory limit");
    if (general && (e = general_set_smem(gs_max, fs_max, ls_max, es_max)) != cudaSuccess)
        return fail(e, "shared memory limit");
    // The gather reads one 8- or 16-byte sample per 32-byte sector at random; ask L2 not to widen
    // its DRAM fetches beyond a sector (a per-context performance hint, ignored where unsupported).
    cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32);
    cudaGetLastError();
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "plan synchronise");
    *out = pl;
    return SFFT_OK;
}

extern "C" {

sfft_status sfft_plan_create(const sfft_params* p, uint32_t max_batch, sfft_plan* out) {
    return plan_create(p, max_batch, nullptr, out);
}

sfft_status sfft_plan_destroy(sfft_plan plan) {
    if (!plan) return SFFT_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return SFFT_OK;
}

uint32_t sfft_plan_rounds(sfft_plan plan) {
    if (!plan) return 0;
    return plan->p.mode == SFFT_GENERAL ? (uint32_t)plan->grounds.size() : (uint32_t)plan->rounds.size();
}

sfft_status sfft_plan_general_round_info(sfft_plan plan, uint32_t r, uint32_t* B, int64_t* T, uint32_t* kprime,
                                         uint32_t* dmax, uint32_t* t_regions, uint64_t* beta_lo, uint64_t* beta_hi) {
    if (!plan || plan->p.mode != SFFT_GENERAL || r >= plan->grounds.size()) return SFFT_ERR_INVALID_ARG;
    const GeneralRound& g = plan->grounds[r];
    if (B) *B = g.B;
    if (T) *T = g.T;
    if (kprime) *kprime = g.kprime;
    if (dmax) *dmax = g.dmax;
    if (t_regions) *t_regions = g.t;
    for (uint32_t D = 0; D < g.dmax; ++D) {
        if (beta_lo) beta_lo[D] = g.beta_lo[D];
        if (beta_hi) beta_hi[D] = g.beta_hi[D];
    }
    return SFFT_OK;
}

sfft_status sfft_plan_round_info(sfft_plan plan, uint32_t t, uint64_t seed, uint32_t request, uint32_t* B,
                                 double* alpha, int64_t* T, uint32_t* nshift, uint64_t* shifts, uint64_t* sigma,
                                 uint64_t* b) {
    if (!plan || t >= plan->rounds.size()) return SFFT_ERR_INVALID_ARG;
    const ExactRound& r = plan->rounds[t];
    if (B) *B = r.B;
    if (alpha) *alpha = r.alpha;
    if (T) *T = r.T;
    if (nshift) *nshift = r.nshift;
    if (shifts)
        for (uint32_t l = 0; l < 4; ++l) shifts[l] = l < r.nshift ? r.shift[l] : 0;
    uint64_t s = 0, bb = 0;
    draw_exact_host(seed, request, t, plan->p.n, &s, &bb);
    if (sigma) *sigma = s;
    if (b) *b = bb;
    return SFFT_OK;
}

sfft_status sfft_plan_taps(sfft_plan plan, uint32_t t, double* h_taps, uint64_t cap) {
    if (!plan || !h_taps || t >= sfft_plan_rounds(plan)) return SFFT_ERR_INVALID_ARG;
    const bool general = plan->p.mode == SFFT_GENERAL;
    const int64_t T = general ? plan->grounds[t].T : plan->rounds[t].T;
    const size_t off = general ? plan->grounds[t].taps_off : plan->rounds[t].taps_off;
    if (cap < (uint64_t)T + 1) return SFFT_ERR_INVALID_ARG;
    std::memcpy(h_taps, plan->taps_host.data() + off, sizeof(double) * ((size_t)T + 1));
    return SFFT_OK;
}

static sfft_status execute_general(sfft_plan plan, const void* d_x, const ReqDesc* d_reqs, uint32_t batch,
                                   uint64_t seed, cudaStream_t st,
                                   uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag,
                                   const sfft_general_trace* tr = nullptr) {
    const sfft_params& p = plan->p;
    SFFT_CUDA(cudaMemsetAsync(plan->d_zcount, 0, batch * sizeof(uint32_t), st), "clear zhat");
    SFFT_CUDA(cudaMemsetAsync(plan->d_zflag, 0, batch * sizeof(int32_t), st), "clear flags");
    const uint32_t R = (uint32_t)plan->grounds.size();
    // stream groups may run different rounds at once, so every round has its own regions: gather
    // counters from max_batch goff[r] (the estimate's counters at max_batch goff[R]), candidates,
    // estimates and magnitudes from max_batch boff[r], device-memory finish arrays from
    // max_batch foff[r] slices
    std::vector<size_t> goff(R + 1, 0), boff(R + 1, 0), foff(R + 1, 0);
    for (uint32_t r = 0; r < R; ++r) {
        goff[r + 1] = goff[r] + plan->grounds[r].ngroups;
        boff[r + 1] = boff[r] + plan->grounds[r].B;
        foff[r + 1] = foff[r] + (plan->grounds[r].fin_global ? plan->grounds[r].ngroups : 0);
    }
    uint32_t groups = plan->nstreams;
    if (groups > batch) groups = batch;
    if (tr) groups = 1;  // a trace records the whole batch's round on the caller's stream
    if (groups > 1) {
        SFFT_CUDA(cudaEventRecord(plan->ev_fork, st), "fork");
        for (uint32_t g = 0; g < groups; ++g) SFFT_CUDA(cudaStreamWaitEvent(plan->aux[g], plan->ev_fork, 0), "fork");
    }
    const size_t zc = p.z_cap;
    for (uint32_t g = 0; g < groups; ++g) {
        const uint32_t r0 = (uint32_t)((uint64_t)batch * g / groups);
        const uint32_t r1 = (uint32_t)((uint64_t)batch * (g + 1) / groups);
        cudaStream_t gs = groups > 1 ? plan->aux[g] : st;
        for (uint32_t r = 0; r < R; ++r) {
            const GeneralRound& gr = plan->grounds[r];
            const bool traced = tr && tr->round == r;
            if (traced) {
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zidx_before, plan->d_zidx, batch * zc * 4, cudaMemcpyDeviceToDevice, gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zval_before, plan->d_zval, batch * zc * 16, cudaMemcpyDeviceToDevice,
                                          gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zcount_before, plan->d_zcount, batch * 4, cudaMemcpyDeviceToDevice, gs),
                          "trace");
            }
            GenArgs a;
            std::memset(&a, 0, sizeof(a));
            a.x = reinterpret_cast<const float2*>(d_x);
            a.xperm = gr.perm ? plan->d_xperm : nullptr;
            a.reqs = d_reqs;
            a.n = p.n;
            a.nmask = (uint32_t)(p.n - 1);
            a.seed = seed;
            a.round = r;
            a.req_base = r0;
            a.B = gr.B;
            a.logB = gr.logB;
            a.T = gr.T;
            a.chunks = gr.chunks;
            a.cpb = gr.cpb;
            a.ctas = gr.ctas;
            a.dmax = gr.dmax;
            a.t = gr.t;
            a.logtp = gr.logtp;
            a.R_loc = p.R_loc;
            a.R_est = p.R_est;
            a.npairs = gr.npairs;
            a.ngroups = gr.ngroups;
            a.nhash = gr.nhash;
            a.kprime = gr.kprime;
            for (uint32_t D = 0; D < gr.dmax; ++D) {
                a.beta_lo[D] = gr.beta_lo[D];
                a.beta_hi[D] = gr.beta_hi[D];
            }
            a.s = p.s;
            a.est_gmin = p.est_gmin;
            a.taps = plan->d_taps32 + gr.taps_off;
            a.wtab = plan->d_wtab + gr.wtab_off;
            a.tw = plan->d_tw;
            a.tw_shift = plan->tw_shift;
            a.part = reinterpret_cast<float2*>(plan->d_part);
            a.part_stride = plan->part_stride;
            a.gcount = plan->d_counter + (size_t)plan->max_batch * goff[r];
            a.ecount = plan->d_counter + (size_t)plan->max_batch * goff[R];
            a.est_w = plan->d_estw + (size_t)plan->max_batch * boff[r];
            a.est_mag = reinterpret_cast<double*>(plan->d_estw + (size_t)plan->max_batch * boff[R]) +
                        (size_t)plan->max_batch * boff[r];
            a.fin_scratch =
                gr.fin_global ? plan->d_gfin + (size_t)plan->max_batch * foff[r] * plan->gfin_stride : nullptr;
            a.fin_stride = plan->gfin_stride;
            a.est_scratch = gr.est_global ? plan->d_gest : nullptr;
            a.est_stride = plan->gest_stride;
            a.bins = plan->d_bins;
            a.phase = plan->d_phase;
            a.bins_stride = plan->bins_stride;
            a.phase_stride = plan->phase_stride;
            a.L = plan->d_L + (size_t)plan->max_batch * boff[r];
            a.nL = plan->d_nL;
            a.zidx = plan->d_zidx;
            a.zval = plan->d_zval;
            a.zcount = plan->d_zcount;
            a.zflag = plan->d_zflag;
            a.zcap = p.z_cap;
            a.last_round = r + 1 == R;
            a.out_idx = d_idx;
            a.out_val = reinterpret_cast<double2*>(d_val);
            a.out_cap = cap;
            a.out_count = d_count;
            a.out_flag = d_flag;
            if (traced) {
                a.dbg_lfp = tr->d_regions;
                a.dbg_valid = tr->d_valid;
            }
            SFFT_CUDA(launch_general_round(a, r1 - r0, gr, gs), "general round");
            if (traced) {
                const size_t row = (size_t)gr.nhash * gr.B * sizeof(double2);
                SFFT_CUDA(cudaMemcpy2DAsync(tr->d_bins, row, plan->d_bins, plan->bins_stride * sizeof(double2), row,
                                            batch, cudaMemcpyDeviceToDevice, gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_cand, a.L, (size_t)batch * gr.B * 4, cudaMemcpyDeviceToDevice, gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zidx_after, plan->d_zidx, batch * zc * 4, cudaMemcpyDeviceToDevice, gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zval_after, plan->d_zval, batch * zc * 16, cudaMemcpyDeviceToDevice, gs),
                          "trace");
                SFFT_CUDA(cudaMemcpyAsync(tr->d_zcount_after, plan->d_zcount, batch * 4, cudaMemcpyDeviceToDevice, gs),
                          "trace");
            }
        }
        if (groups > 1) {
            SFFT_CUDA(cudaEventRecord(plan->ev_join[g], gs), "join");
            SFFT_CUDA(cudaStreamWaitEvent(st, plan->ev_join[g], 0), "join");
        }
    }
    return SFFT_OK;
}

}  // extern "C"

// One batch through every round: rows of d_x (d_reqs == nullptr) or the requests of the device table
// d_reqs.  Arguments are checked by the callers.
sfft_status sfft::execute_batch(sfft_plan plan, const void* d_x, const ReqDesc* d_reqs, uint32_t batch,
                                uint64_t seed, cudaStream_t st, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                          int32_t* d_flag) {
    if (plan->p.mode == SFFT_GENERAL)
        return execute_general(plan, d_x, d_reqs, batch, seed, st, d_idx, d_val, cap, d_count, d_flag);
    const bool fp64 = plan->p.precision == SFFT_FP64;
    SFFT_CUDA(cudaMemsetAsync(plan->d_zcount, 0, batch * sizeof(uint32_t), st), "clear zhat");
    SFFT_CUDA(cudaMemsetAsync(plan->d_zflag, 0, batch * sizeof(int32_t), st), "clear flags");
    const uint32_t R = (uint32_t)plan->rounds.size();
    // One launch per group covers every round (k_exact_step).  Requests are independent, so the batch
    // may be cut into groups on separate streams: one group's last finishers overlap the next group's
    // gathers.  The groups fork from and join back into the caller's stream with events (capturable
    // in a CUDA graph).
    uint32_t groups = plan->nstreams;
    if (groups > batch) groups = batch;
    if (batch < 8) groups = 1;
    if (groups > 1) {
        SFFT_CUDA(cudaEventRecord(plan->ev_fork, st), "fork");
        for (uint32_t g = 0; g < groups; ++g) SFFT_CUDA(cudaStreamWaitEvent(plan->aux[g], plan->ev_fork, 0), "fork");
    }
    for (uint32_t g = 0; g < groups; ++g) {
        const uint32_t r0 = (uint32_t)((uint64_t)batch * g / groups);
        const uint32_t r1 = (uint32_t)((uint64_t)batch * (g + 1) / groups);
        cudaStream_t gs = groups > 1 ? plan->aux[g] : st;
        ExactArgs rounds[kMaxRounds];
        for (uint32_t t = 0; t < R; ++t) {
            ExactArgs& a = rounds[t];
            a = plan->rdesc[t];
            a.x = d_x;
            a.reqs = d_reqs;
            a.seed = seed;
            a.req_base = r0;
            a.out_idx = d_idx;
            a.out_val = reinterpret_cast<double2*>(d_val);
            a.out_cap = cap;
            a.out_count = d_count;
            a.out_flag = d_flag;
        }
        SFFT_CUDA(launch_exact_step(rounds, R, r1 - r0, plan->step_smem, gs, fp64), "exact step");
        if (groups > 1) {
            SFFT_CUDA(cudaEventRecord(plan->ev_join[g], gs), "join");
            SFFT_CUDA(cudaStreamWaitEvent(st, plan->ev_join[g], 0), "join");
        }
    }
    return SFFT_OK;
}

extern "C" {

sfft_status sfft_execute(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, void* stream,
                         uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag) {
    if (!plan || !d_x || !d_idx || !d_val || !d_count || !d_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    if (batch == 0 || batch > plan->max_batch) return SFFT_ERR_INVALID_ARG;
    return execute_batch(plan, d_x, nullptr, batch, seed, (cudaStream_t)stream, d_idx, d_val, cap, d_count, d_flag);
}

static sfft_status execute_channels(sfft_plan plan, const void* d_x, uint32_t channels, uint64_t seed, uint32_t id,
                                   cudaStream_t st, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                                   int32_t* d_flag, cudaEvent_t before, cudaEvent_t after) {
    if (!plan || !d_x || !d_idx || !d_val || !d_count || !d_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    if (plan->p.mode != SFFT_EXACT || plan->p.precision != SFFT_FP32 || plan->chan_off.empty())
        return SFFT_ERR_INVALID_ARG;
    if (channels == 0 || channels % 32 || channels > kChanMaxC || channels > plan->max_batch || ((uintptr_t)d_x & 15))
        return SFFT_ERR_INVALID_ARG;
    SFFT_CUDA(cudaMemsetAsync(plan->d_zcount, 0, channels * sizeof(uint32_t), st), "clear zhat");
    SFFT_CUDA(cudaMemsetAsync(plan->d_zflag, 0, channels * sizeof(int32_t), st), "clear flags");
    const uint32_t R = (uint32_t)plan->rounds.size();
    ExactArgs rounds[kMaxRounds];
    for (uint32_t t = 0; t < R; ++t) {
        ExactArgs& a = rounds[t];
        a = plan->rdesc[t];
        a.x = d_x;
        a.reqs = nullptr;
        a.seed = seed;
        a.req_base = 0;
        a.part = static_cast<unsigned char*>(plan->d_part) + plan->chan_off[t] * sizeof(float2);
        a.chunks = plan->chan_chunks[t];
        a.out_idx = d_idx;
        a.out_val = reinterpret_cast<double2*>(d_val);
        a.out_cap = cap;
        a.out_count = d_count;
        a.out_flag = d_flag;
    }
    SFFT_CUDA(launch_exact_channels(rounds, R, channels, d_x, seed, id, plan->step_smem, plan->d_aux, st, before,
                                    after),
              "channel batch");
    return SFFT_OK;
}

sfft_status sfft_execute_channels(sfft_plan plan, const void* d_x, uint32_t channels, uint64_t seed, uint32_t id,
                                  void* stream, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                                  int32_t* d_flag) {
    return execute_channels(plan, d_x, channels, seed, id, (cudaStream_t)stream, d_idx, d_val, cap, d_count, d_flag,
                            nullptr, nullptr);
}

sfft_status sfft_execute_channels_timed(sfft_plan plan, const void* d_x, uint32_t channels, uint64_t seed, uint32_t id,
                                        void* stream, uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count,
                                        int32_t* d_flag, void* before, void* after) {
    return execute_channels(plan, d_x, channels, seed, id, (cudaStream_t)stream, d_idx, d_val, cap, d_count, d_flag,
                            (cudaEvent_t)before, (cudaEvent_t)after);
}

sfft_status sfft_execute_trace(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, void* stream,
                               uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag,
                               const sfft_general_trace* tr) {
    if (!plan || !d_x || !d_idx || !d_val || !d_count || !d_flag || cap == 0 || !tr) return SFFT_ERR_INVALID_ARG;
    if (batch == 0 || batch > plan->max_batch || plan->p.mode != SFFT_GENERAL) return SFFT_ERR_INVALID_ARG;
    if (tr->round >= plan->grounds.size() || !tr->d_bins || !tr->d_regions || !tr->d_valid || !tr->d_cand ||
        !tr->d_zidx_before || !tr->d_zval_before || !tr->d_zcount_before || !tr->d_zidx_after || !tr->d_zval_after ||
        !tr->d_zcount_after)
        return SFFT_ERR_INVALID_ARG;
    return execute_general(plan, d_x, nullptr, batch, seed, (cudaStream_t)stream, d_idx, d_val, cap, d_count, d_flag,
                           tr);
}

sfft_status sfft_plan_set_requests(sfft_plan plan, const sfft_request* h_reqs, uint32_t batch, void* stream) {
    if (!plan || !h_reqs || batch == 0 || batch > plan->max_batch) return SFFT_ERR_INVALID_ARG;
    const size_t align = plan->p.precision == SFFT_FP64 ? 16 : 8;
    for (uint32_t r = 0; r < batch; ++r) {
        if (!h_reqs[r].d_x || ((uintptr_t)h_reqs[r].d_x % align) != 0) return SFFT_ERR_INVALID_ARG;
        const uint32_t per = h_reqs[r].period;
        if (per != 0 && (!is_pow2(per) || per > plan->p.n)) return SFFT_ERR_INVALID_ARG;
    }
    // The table goes through one of the plan's two page-locked buffers (its previous copy has completed):
    // an asynchronous copy from the caller's array could run after the caller has freed it (on
    // Grace-Blackwell the GPU reads pageable memory directly, without staging it at the call).
    const int cur = plan->reqs_cur;
    plan->reqs_cur ^= 1;
    SFFT_CUDA(cudaEventSynchronize(plan->ev_reqs[cur]), "request table buffer");
    std::memcpy(plan->h_reqs[cur], h_reqs, (size_t)batch * sizeof(ReqDesc));
    cudaStream_t st = (cudaStream_t)stream;
    SFFT_CUDA(cudaMemcpyAsync(plan->d_reqs, plan->h_reqs[cur], (size_t)batch * sizeof(ReqDesc), cudaMemcpyHostToDevice,
                              st),
              "copy request table");
    SFFT_CUDA(cudaEventRecord(plan->ev_reqs[cur], st), "request table event");
    return SFFT_OK;
}

sfft_status sfft_execute_requests(sfft_plan plan, const sfft_request* h_reqs, uint32_t batch, void* stream,
                                  uint32_t* d_idx, double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag) {
    if (!plan || !h_reqs || !d_idx || !d_val || !d_count || !d_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    const sfft_status st = sfft_plan_set_requests(plan, h_reqs, batch, stream);
    if (st != SFFT_OK) return st;
    return execute_batch(plan, nullptr, plan->d_reqs, batch, 0, (cudaStream_t)stream, d_idx, d_val, cap, d_count,
                         d_flag);
}

}  // extern "C"

struct sfft_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

sfft_status sfft_graph_create(sfft_plan plan, const void* d_x, uint32_t batch, uint64_t seed, uint32_t* d_idx,
                              double* d_val, uint32_t cap, uint32_t* d_count, int32_t* d_flag, sfft_graph* out) {
    if (!out) return SFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plan || !d_idx || !d_val || !d_count || !d_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    if (batch == 0 || batch > plan->max_batch) return SFFT_ERR_INVALID_ARG;
    auto* g = new (std::nothrow) sfft_graph_s();
    if (!g) return SFFT_ERR_OOM;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sfft_status st = SFFT_OK;
    if (e == cudaSuccess) {
        st = execute_batch(plan, d_x, d_x ? nullptr : plan->d_reqs, batch, seed, cs, d_idx, d_val, cap, d_count,
                           d_flag);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (st == SFFT_OK && e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && st == SFFT_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess || st != SFFT_OK) {
        if (e != cudaSuccess) set_last_error(std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st != SFFT_OK ? st : SFFT_ERR_CUDA;
    }
    *out = g;
    return SFFT_OK;
}

sfft_status sfft_graph_launch(sfft_graph g, void* stream) {
    if (!g) return SFFT_ERR_INVALID_ARG;
    SFFT_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "graph launch");
    return SFFT_OK;
}

sfft_status sfft_graph_destroy(sfft_graph g) {
    if (!g) return SFFT_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return SFFT_OK;
}

sfft_status sfft_execute_host(sfft_plan plan, const void* h_x, uint32_t batch, uint64_t seed, void* stream,
                              uint32_t* h_idx, double* h_val, uint32_t cap, uint32_t* h_count, int32_t* h_flag) {
    if (!plan || !h_x || !h_idx || !h_val || !h_count || !h_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    if (batch == 0 || batch > plan->max_batch) return SFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elem = plan->p.precision == SFFT_FP64 ? 16 : 8;
    // Page-locked host signals are read in place by the kernels (over NVLink-C2C on Grace-Blackwell)
    // when the gathered samples, at a 64-byte line each, weigh less than the whole signal: only they
    // cross the link.  Otherwise (and for other host memory) the signals are staged whole.
    const void* x_in_place = nullptr;
    if (plan->samples * 64 < plan->p.n * elem) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, h_x) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
            x_in_place = at.devicePointer;
        cudaGetLastError();
    }
    const size_t xbytes = x_in_place ? 0 : (size_t)batch * plan->p.n * elem;
    if (plan->stage_bytes < xbytes || plan->out_cap < (size_t)batch * cap) {
        SFFT_CUDA(cudaStreamSynchronize(st), "sync before staging");
        cudaFree(plan->d_stage);
        cudaFree(plan->d_out_idx);
        cudaFree(plan->d_out_val);
        cudaFree(plan->d_out_count);
        cudaFree(plan->d_out_flag);
        plan->d_stage = nullptr;
        plan->d_out_idx = nullptr;
        plan->d_out_val = nullptr;
        plan->d_out_count = nullptr;
        plan->d_out_flag = nullptr;
        plan->stage_bytes = 0;
        plan->out_cap = 0;
        if (xbytes && cudaMalloc(&plan->d_stage, xbytes) != cudaSuccess) return SFFT_ERR_OOM;
        if (cudaMalloc((void**)&plan->d_out_idx, (size_t)batch * cap * 4) != cudaSuccess) return SFFT_ERR_OOM;
        if (cudaMalloc((void**)&plan->d_out_val, (size_t)batch * cap * 16) != cudaSuccess) return SFFT_ERR_OOM;
        if (cudaMalloc((void**)&plan->d_out_count, (size_t)batch * 4) != cudaSuccess) return SFFT_ERR_OOM;
        if (cudaMalloc((void**)&plan->d_out_flag, (size_t)batch * 4) != cudaSuccess) return SFFT_ERR_OOM;
        plan->stage_bytes = xbytes;
        plan->out_cap = (size_t)batch * cap;
    }
    if (!x_in_place) SFFT_CUDA(cudaMemcpyAsync(plan->d_stage, h_x, xbytes, cudaMemcpyHostToDevice, st), "copy x to device");
    sfft_status s = sfft_execute(plan, x_in_place ? x_in_place : plan->d_stage, batch, seed, stream, plan->d_out_idx,
                                 plan->d_out_val, cap, plan->d_out_count, plan->d_out_flag);
    if (s != SFFT_OK) return s;
    SFFT_CUDA(cudaMemcpyAsync(h_count, plan->d_out_count, (size_t)batch * 4, cudaMemcpyDeviceToHost, st), "copy count");
    SFFT_CUDA(cudaMemcpyAsync(h_flag, plan->d_out_flag, (size_t)batch * 4, cudaMemcpyDeviceToHost, st), "copy flag");
    SFFT_CUDA(cudaMemcpyAsync(h_idx, plan->d_out_idx, (size_t)batch * cap * 4, cudaMemcpyDeviceToHost, st), "copy idx");
    SFFT_CUDA(cudaMemcpyAsync(h_val, plan->d_out_val, (size_t)batch * cap * 16, cudaMemcpyDeviceToHost, st),
              "copy values");
    SFFT_CUDA(cudaStreamSynchronize(st), "synchronise");
    return SFFT_OK;
}

sfft_status sfft_hash_to_bins(sfft_plan plan, uint32_t t, const void* d_x, uint64_t sigma, uint64_t a, uint64_t b,
                              const uint32_t* d_zidx, const double* d_zval, uint32_t nz, double* d_u, void* stream) {
    if (!plan || !d_x || !d_u || t >= plan->rounds.size()) return SFFT_ERR_INVALID_ARG;
    if (nz > 0 && (!d_zidx || !d_zval)) return SFFT_ERR_INVALID_ARG;
    if (!(sigma & 1) || sigma >= plan->p.n || a >= plan->p.n || b >= plan->p.n) return SFFT_ERR_INVALID_ARG;
    if (nz > plan->p.z_cap) return SFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = plan->p.precision == SFFT_FP64;
    ExactRound r = plan->rounds[t];
    ExactArgs args = base_args(plan, r, t);
    args.x = d_x;
    args.H = 1;
    args.a_base = (uint32_t)a;
    args.a[0] = 0;
    args.maxshift = 0;
    args.stage = r.ctaps;
    args.bins_only = 1;
    args.e_sigma = (uint32_t)sigma;
    args.e_b = (uint32_t)b;
    args.ubins = reinterpret_cast<double2*>(d_u);
    args.zidx = const_cast<uint32_t*>(d_zidx);
    args.zval = reinterpret_cast<double2*>(const_cast<double*>(d_zval));
    args.zcap = nz > 0 ? nz : 1;
    args.e_nz = nz;
    const size_t gs = exact_gather_smem(args.stage, fp64) + (size_t)(r.B > (uint32_t)kThreads ? r.B : kThreads) *
                                                                (fp64 ? 16 : 8);
    const size_t fs = exact_finish_smem(r.B, 1, args.zcap, fp64);
    const size_t smem = gs > fs ? gs : fs;
    SFFT_CUDA(set_exact_smem_limit(smem > r.smem ? smem : r.smem, fp64), "shared memory limit");
    SFFT_CUDA(launch_exact_round(args, 1, smem, st, fp64), "hash to bins");
    return SFFT_OK;
}

sfft_status sfft_exact_decode(sfft_plan plan, uint32_t t, uint64_t sigma, uint64_t b, const double* d_u,
                              const uint32_t* d_zidx, uint32_t nz, uint32_t* d_widx, double* d_wval,
                              uint32_t* d_count, uint32_t* d_nabove, uint32_t* d_nkept, void* stream) {
    if (!plan || !d_u || !d_widx || !d_wval || !d_count || !d_nabove || !d_nkept) return SFFT_ERR_INVALID_ARG;
    if (t >= plan->rounds.size() || (nz > 0 && !d_zidx) || nz > 4096) return SFFT_ERR_INVALID_ARG;
    if (!(sigma & 1) || sigma >= plan->p.n || b >= plan->p.n) return SFFT_ERR_INVALID_ARG;
    const ExactRound& r = plan->rounds[t];
    const sfft_params& p = plan->p;
    DecodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = p.n;
    a.nmask = (uint32_t)(p.n - 1);
    a.B = r.B;
    a.logB = r.logB;
    a.H = 1 + r.nshift;
    for (uint32_t l = 0; l < r.nshift; ++l) a.shift64[l] = r.shift[l];
    a.sigma = (uint32_t)sigma;
    a.b = (uint32_t)b;
    a.wtab = plan->d_wtab + r.wtab_off;
    a.u = reinterpret_cast<const double2*>(d_u);
    a.zidx = d_zidx;
    a.nz = nz;
    a.thr = p.thr;
    a.iso_tol = p.iso_tol;
    a.gmin = p.gmin;
    a.ref_lo = p.ref_lo;
    a.ref_hi = p.ref_hi;
    a.ref_tol = p.ref_tol;
    a.widx = d_widx;
    a.wval = reinterpret_cast<double2*>(d_wval);
    a.count = d_count;
    a.nabove = d_nabove;
    a.nkept = d_nkept;
    a.fp64 = p.precision == SFFT_FP64;
    SFFT_CUDA(launch_exact_decode(a, (cudaStream_t)stream), "exact decode");
    return SFFT_OK;
}

sfft_status sfft_philox(uint32_t key0, uint32_t key1, const uint32_t* h_ctr, uint32_t count, uint32_t* d_out,
                        void* stream) {
    if (!h_ctr || (!d_out && count)) return SFFT_ERR_INVALID_ARG;
    SFFT_CUDA(launch_philox(key0, key1, h_ctr[0], h_ctr[1], h_ctr[2], h_ctr[3], count, d_out, (cudaStream_t)stream),
              "philox");
    return SFFT_OK;
}

sfft_status sfft_locate_votes(sfft_plan plan, uint32_t r, uint64_t sigma, uint64_t b, uint64_t w_fp, uint32_t nrep,
                              const uint64_t* d_beta, const double* d_u, const double* d_up, uint64_t* d_lfp,
                              uint8_t* d_valid, uint32_t* d_votes, void* stream) {
    if (!plan || plan->p.mode != SFFT_GENERAL || r >= plan->grounds.size()) return SFFT_ERR_INVALID_ARG;
    if (!d_beta || !d_u || !d_up || !d_lfp || !d_valid || !d_votes || nrep == 0 || nrep > (uint32_t)kMaxRloc)
        return SFFT_ERR_INVALID_ARG;
    if (!(sigma & 1) || sigma >= plan->p.n || b >= plan->p.n) return SFFT_ERR_INVALID_ARG;
    const GeneralRound& g = plan->grounds[r];
    VoteArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = plan->p.n;
    a.nmask = (uint32_t)(plan->p.n - 1);
    a.B = g.B;
    a.t = g.t;
    a.nrep = nrep;
    a.sigma = (uint32_t)sigma;
    a.b = (uint32_t)b;
    a.w_fp = w_fp;
    a.s = plan->p.s;
    a.u = reinterpret_cast<const double2*>(d_u);
    a.up = reinterpret_cast<const double2*>(d_up);
    a.beta = d_beta;
    a.l_fp = d_lfp;
    a.valid = d_valid;
    a.votes = d_votes;
    SFFT_CUDA(launch_locate_votes(a, (cudaStream_t)stream), "locate votes");
    return SFFT_OK;
}

sfft_status sfft_estimate_from_bins(sfft_plan plan, uint32_t r, uint32_t nrep, const uint64_t* d_sigma,
                                    const uint64_t* d_b, const uint64_t* d_a, const double* d_u, const uint32_t* d_L,
                                    uint32_t nL, uint32_t kprime, uint32_t* d_widx, double* d_wval, uint32_t* d_count,
                                    void* stream) {
    if (!plan || plan->p.mode != SFFT_GENERAL || r >= plan->grounds.size()) return SFFT_ERR_INVALID_ARG;
    if (!d_sigma || !d_b || !d_a || !d_u || (nL > 0 && !d_L) || !d_widx || !d_wval || !d_count) return SFFT_ERR_INVALID_ARG;
    if (nrep == 0 || nrep > (uint32_t)kMaxRest || nL > plan->grounds[r].B) return SFFT_ERR_INVALID_ARG;
    const GeneralRound& g = plan->grounds[r];
    EstArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = plan->p.n;
    a.nmask = (uint32_t)(plan->p.n - 1);
    a.B = g.B;
    a.logB = g.logB;
    a.nrep = nrep;
    a.nL = nL;
    a.kprime = kprime;
    a.sig = d_sigma;
    a.bb = d_b;
    a.aa = d_a;
    a.u = reinterpret_cast<const double2*>(d_u);
    a.L = d_L;
    a.wtab = plan->d_wtab + g.wtab_off;
    a.tw = plan->d_tw;
    a.tw_shift = plan->tw_shift;
    a.est_gmin = plan->p.est_gmin;
    a.widx = d_widx;
    a.wval = reinterpret_cast<double2*>(d_wval);
    a.count = d_count;
    SFFT_CUDA(launch_estimate_from_bins(a, (cudaStream_t)stream), "estimate from bins");
    return SFFT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Batch plans: mixed exact-mode requests in one persistent launch
// ------------------------------------------------------------------------------------------------
struct sfft_batch_plan_s {
    std::vector<sfft_plan> plans;
    std::vector<uint32_t> rd0, rounds, chunks0, items_of;  // per plan: first descriptor, rounds,
                                                          // round-0 chunks, items of a request
    bool fp64 = false;
    uint32_t max_req = 0;
    size_t max_items = 0;         // items of the largest batch the workspace holds
    ExactArgs* d_rdesc = nullptr;
    unsigned char* d_ctl = nullptr;  // [reqs | rd0 | rounds | head, tail, error | flags] of one call
    unsigned long long* d_items = nullptr;
    unsigned char* d_part = nullptr;
    size_t part_stride = 0;
    uint32_t* d_counter = nullptr;
    uint32_t* d_zidx = nullptr;
    double2* d_zval = nullptr;
    size_t z_stride = 0;
    uint32_t* d_zcount = nullptr;
    int32_t* d_zflag = nullptr;
    unsigned char* d_fin = nullptr;
    size_t fin_stride = 0;
    size_t smem = 0;
    int ctas = 0;
    size_t ctl_bytes = 0;
    unsigned char* h_stage[2] = {nullptr, nullptr};  // page-locked copies of the control block + items
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int cur = 0;
};

namespace {

struct CtlLayout {
    size_t reqs, rd0, rounds, ctr, flags, items, total;
};
CtlLayout ctl_layout(uint32_t nreq, size_t items0) {
    CtlLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = (off + 15) & ~size_t(15);
        off = o + bytes;
        return o;
    };
    L.reqs = take((size_t)nreq * sizeof(ReqDesc));
    L.rd0 = take((size_t)nreq * 4);
    L.rounds = take((size_t)nreq * 4);
    L.ctr = take(16);
    L.flags = take((size_t)nreq * 4);
    L.items = take(items0 * 8);
    L.total = off;
    return L;
}

void free_batch_plan(sfft_batch_plan_s* bp) {
    if (!bp) return;
    cudaFree(bp->d_rdesc);
    cudaFree(bp->d_ctl);
    cudaFree(bp->d_items);
    cudaFree(bp->d_part);
    cudaFree(bp->d_counter);
    cudaFree(bp->d_zidx);
    cudaFree(bp->d_zval);
    cudaFree(bp->d_zcount);
    cudaFree(bp->d_zflag);
    cudaFree(bp->d_fin);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(bp->h_stage[i]);
        if (bp->ev[i]) cudaEventDestroy(bp->ev[i]);
    }
    delete bp;
}

}  // namespace

extern "C" {

sfft_status sfft_batch_plan_create(const sfft_plan* plans, uint32_t nplans, uint32_t max_requests,
                                   sfft_batch_plan* out) {
    if (!out) return SFFT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || nplans == 0 || max_requests == 0 || max_requests > (1u << 24)) return SFFT_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < nplans; ++i) {
        if (!plans[i] || plans[i]->p.mode != SFFT_EXACT) return SFFT_ERR_INVALID_ARG;
        if (plans[i]->p.precision != plans[0]->p.precision) return SFFT_ERR_INVALID_ARG;
        if (plans[i]->rounds.size() > 255) return SFFT_ERR_INVALID_ARG;
    }
    auto* bp = new (std::nothrow) sfft_batch_plan_s();
    if (!bp) return SFFT_ERR_OOM;
    bp->plans.assign(plans, plans + nplans);
    bp->fp64 = plans[0]->p.precision == SFFT_FP64;
    bp->max_req = max_requests;
    const size_t csize = bp->fp64 ? 16 : 8;
    std::vector<ExactArgs> rdesc;
    uint32_t max_items_req = 0, max_chunks0 = 0;
    for (sfft_plan pl : bp->plans) {
        bp->rd0.push_back((uint32_t)rdesc.size());
        const uint32_t R = (uint32_t)pl->rounds.size();
        bp->rounds.push_back(R);
        uint32_t items = 0;
        for (uint32_t t = 0; t < R; ++t) {
            const ExactRound& r = pl->rounds[t];
            if (r.chunks > 0xFFFFu) {
                free_batch_plan(bp);
                return SFFT_ERR_K_RANGE;
            }
            ExactArgs a = base_args(pl, r, t);
            a.first_round = t == 0;
            a.last_round = t + 1 == R;
            rdesc.push_back(a);
            items += r.chunks;
            bp->smem = std::max(bp->smem, r.smem);
            if (r.fin_global) bp->fin_stride = std::max(bp->fin_stride, (r.fin_bytes + 255) & ~size_t(255));
        }
        bp->chunks0.push_back(pl->rounds[0].chunks);
        bp->items_of.push_back(items);
        max_items_req = std::max(max_items_req, items);
        max_chunks0 = std::max(max_chunks0, pl->rounds[0].chunks);
        bp->part_stride = std::max(bp->part_stride, ((pl->part_stride * csize) + 255) & ~size_t(255));
        bp->z_stride = std::max(bp->z_stride, (size_t)pl->p.z_cap);
    }
    bp->max_items = (size_t)max_items_req * max_requests;
    if (bp->max_items >= (size_t)1 << 32) {
        free_batch_plan(bp);
        return SFFT_ERR_INVALID_ARG;
    }
    bp->ctl_bytes = ctl_layout(max_requests, (size_t)max_chunks0 * max_requests).total;
    bool ok = cudaMalloc((void**)&bp->d_rdesc, rdesc.size() * sizeof(ExactArgs)) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_ctl, bp->ctl_bytes) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_items, bp->max_items * 8) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_part, bp->part_stride * max_requests) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_counter, (size_t)max_requests * 4) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_zidx, bp->z_stride * max_requests * 4) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_zval, bp->z_stride * max_requests * 16) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_zcount, (size_t)max_requests * 4) == cudaSuccess &&
              cudaMalloc((void**)&bp->d_zflag, (size_t)max_requests * 4) == cudaSuccess &&
              (bp->fin_stride == 0 || cudaMalloc((void**)&bp->d_fin, bp->fin_stride * max_requests) == cudaSuccess) &&
              cudaMallocHost((void**)&bp->h_stage[0], bp->ctl_bytes) == cudaSuccess &&
              cudaMallocHost((void**)&bp->h_stage[1], bp->ctl_bytes) == cudaSuccess &&
              cudaEventCreateWithFlags(&bp->ev[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&bp->ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        set_last_error(std::string("batch plan: ") + cudaGetErrorString(cudaGetLastError()));
        free_batch_plan(bp);
        return SFFT_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(bp->d_rdesc, rdesc.data(), rdesc.size() * sizeof(ExactArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(bp->d_counter, 0, (size_t)max_requests * 4);
    if (e != cudaSuccess) {
        set_last_error(std::string("batch plan: ") + cudaGetErrorString(e));
        free_batch_plan(bp);
        return SFFT_ERR_CUDA;
    }
    bp->ctas = exact_persistent_ctas(bp->smem, bp->fp64);
    if (bp->ctas <= 0) {
        set_last_error("batch plan: no CTA of the persistent kernel fits on the device");
        free_batch_plan(bp);
        return SFFT_ERR_K_RANGE;
    }
    *out = bp;
    return SFFT_OK;
}

sfft_status sfft_persistent_wait_check(void* stream) {
    // control block: items[1] (never published), head, tail, error
    unsigned char* d = nullptr;
    if (cudaMalloc((void**)&d, 64) != cudaSuccess) {
        cudaGetLastError();
        return SFFT_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    PersistArgs a;
    std::memset(&a, 0, sizeof(a));
    a.items = reinterpret_cast<unsigned long long*>(d);
    a.head = reinterpret_cast<uint32_t*>(d + 16);
    a.tail = a.head + 1;
    a.error = reinterpret_cast<int32_t*>(a.head + 2);
    a.total = 1;
    int32_t err = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, 64, st);
    if (e == cudaSuccess) e = launch_exact_persistent(a, 1, 0, st, false);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, a.error, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) {
        set_last_error(std::string("wait check: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return SFFT_ERR_CUDA;
    }
    return err ? SFFT_ERR_TIMEOUT : SFFT_OK;
}

sfft_status sfft_batch_plan_destroy(sfft_batch_plan bp) {
    if (!bp) return SFFT_OK;
    cudaDeviceSynchronize();
    free_batch_plan(bp);
    return SFFT_OK;
}

sfft_status sfft_batch_execute(sfft_batch_plan bp, const uint32_t* h_plan_of, const sfft_request* h_reqs,
                               uint32_t nreq, void* stream, uint32_t* d_idx, double* d_val, uint32_t cap,
                               uint32_t* d_count, int32_t* d_flag) {
    if (!bp || !h_plan_of || !h_reqs || !d_idx || !d_val || !d_count || !d_flag || cap == 0) return SFFT_ERR_INVALID_ARG;
    if (nreq == 0 || nreq > bp->max_req) return SFFT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t align = bp->fp64 ? 16 : 8;
    size_t items0 = 0, total = 0;
    for (uint32_t r = 0; r < nreq; ++r) {
        const uint32_t p = h_plan_of[r];
        if (p >= bp->plans.size() || !h_reqs[r].d_x || ((uintptr_t)h_reqs[r].d_x % align) != 0)
            return SFFT_ERR_INVALID_ARG;
        const uint32_t per = h_reqs[r].period;
        if (per != 0 && (!is_pow2(per) || per > bp->plans[p]->p.n)) return SFFT_ERR_INVALID_ARG;
        items0 += bp->chunks0[p];
        total += bp->items_of[p];
    }
    // stage the control block in this call's page-locked buffer (its previous copy has completed)
    const int cur = bp->cur;
    bp->cur ^= 1;
    SFFT_CUDA(cudaEventSynchronize(bp->ev[cur]), "staging buffer");
    unsigned char* h = bp->h_stage[cur];
    const CtlLayout L = ctl_layout(nreq, items0);
    ReqDesc* reqs = reinterpret_cast<ReqDesc*>(h + L.reqs);
    uint32_t* rd0 = reinterpret_cast<uint32_t*>(h + L.rd0);
    uint32_t* rounds = reinterpret_cast<uint32_t*>(h + L.rounds);
    uint32_t* ctr = reinterpret_cast<uint32_t*>(h + L.ctr);
    int32_t* flags = reinterpret_cast<int32_t*>(h + L.flags);
    unsigned long long* items = reinterpret_cast<unsigned long long*>(h + L.items);
    size_t q = 0;
    for (uint32_t r = 0; r < nreq; ++r) {
        const uint32_t p = h_plan_of[r];
        std::memcpy(&reqs[r], &h_reqs[r], sizeof(ReqDesc));
        rd0[r] = bp->rd0[p];
        rounds[r] = bp->rounds[p];
        flags[r] = SFFT_ERR_TIMEOUT;  // overwritten by the request's last round
        for (uint32_t c = 0; c < bp->chunks0[p]; ++c)
            items[q++] = (1ull << 63) | ((unsigned long long)r << 24) | c;
    }
    ctr[0] = 0;                 // head
    ctr[1] = (uint32_t)items0;  // tail
    ctr[2] = 0;                 // error
    ctr[3] = 0;
    unsigned char* d = bp->d_ctl;
    SFFT_CUDA(cudaMemcpyAsync(d, h, L.items, cudaMemcpyHostToDevice, st), "copy control block");
    SFFT_CUDA(cudaMemcpyAsync(bp->d_items, h + L.items, items0 * 8, cudaMemcpyHostToDevice, st), "copy items");
    SFFT_CUDA(cudaEventRecord(bp->ev[cur], st), "staging event");
    if (total > items0)
        SFFT_CUDA(cudaMemsetAsync(bp->d_items + items0, 0, (total - items0) * 8, st), "clear items");
    SFFT_CUDA(cudaMemcpyAsync(d_flag, d + L.flags, (size_t)nreq * 4, cudaMemcpyDeviceToDevice, st), "flags");
    SFFT_CUDA(cudaMemsetAsync(d_count, 0, (size_t)nreq * 4, st), "counts");
    SFFT_CUDA(cudaMemsetAsync(bp->d_zcount, 0, (size_t)nreq * 4, st), "clear zhat");
    SFFT_CUDA(cudaMemsetAsync(bp->d_zflag, 0, (size_t)nreq * 4, st), "clear flags");
    PersistArgs a;
    std::memset(&a, 0, sizeof(a));
    a.rdesc = bp->d_rdesc;
    a.reqs = reinterpret_cast<const ReqDesc*>(d + L.reqs);
    a.req_rd0 = reinterpret_cast<const uint32_t*>(d + L.rd0);
    a.req_rounds = reinterpret_cast<const uint32_t*>(d + L.rounds);
    a.items = bp->d_items;
    a.head = reinterpret_cast<uint32_t*>(d + L.ctr);
    a.tail = a.head + 1;
    a.error = reinterpret_cast<int32_t*>(a.head + 2);
    a.total = (uint32_t)total;
    a.part = bp->d_part;
    a.part_stride = bp->part_stride;
    a.counter = bp->d_counter;
    a.zidx = bp->d_zidx;
    a.zval = bp->d_zval;
    a.z_stride = bp->z_stride;
    a.zcount = bp->d_zcount;
    a.zflag = bp->d_zflag;
    a.fin = bp->d_fin;
    a.fin_stride = bp->fin_stride;
    a.out_idx = d_idx;
    a.out_val = reinterpret_cast<double2*>(d_val);
    a.out_cap = cap;
    a.out_count = d_count;
    a.out_flag = d_flag;
    const uint32_t ctas = (uint32_t)std::min<size_t>((size_t)bp->ctas, total);
    SFFT_CUDA(launch_exact_persistent(a, ctas, bp->smem, st, bp->fp64), "persistent launch");
    return SFFT_OK;
}

}  // extern "C"
