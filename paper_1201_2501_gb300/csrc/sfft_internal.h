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
constexpr uint32_t kMaxB = 4096;  // largest B of the fused exact round
constexpr uint32_t kNoIndex = 0xFFFFFFFFu;

// One round of the exact schedule (Algorithm 1's loop t = 0..log k, with this library's readings).
struct ExactRound {
    uint32_t B = 0, logB = 0;
    double alpha = 0;
    int64_t T = 0;            // taps t in [-T, T]
    uint32_t nshift = 0;      // ladder length L
    uint64_t shift[4] = {0, 0, 0, 0};
    uint32_t chunks = 0;      // CTAs per request in the gather phase
    uint32_t stage = 0;       // samples staged per CTA: kChunkTaps + largest shift
    size_t taps_off = 0;      // offset of this round's taps in the tap arrays
    size_t wtab_off = 0;      // offset of this round's W(o), o = 0..n/2B, in the W table
    size_t smem = 0;          // dynamic shared memory of the round kernel
};

// Kernel argument block of the exact round (passed by value).
struct ExactArgs {
    const void* x;             // batch x n complex values (float2 or double2)
    uint64_t n;
    uint32_t nmask;            // n - 1
    uint64_t seed;
    uint32_t round;
    uint32_t req_base;         // request index of blockIdx.y == 0 (a launch may cover part of a batch)
    uint32_t B, logB;
    int64_t T;
    uint32_t H;                // hashings: hashing h uses offset a_base + a[h]
    uint32_t a_base;           // 0 in the exact rounds; the explicit a of sfft_hash_to_bins
    uint32_t a[kMaxHash];      // a[0] = 0, a[l] = beta_l
    uint64_t shift64[kMaxHash];
    uint32_t chunks, stage, maxshift;
    const float* taps32;
    const double* taps64;
    const double* wtab;
    void* part;                // partial fold sums: request s owns [s part_stride, (s + 1) part_stride),
                               // laid out [chunks][H][B] complex R (requests may be in different rounds)
    size_t part_stride;
    uint32_t* counter;         // [batch] arrival counters (zero between launches)
    uint32_t* zidx;            // [batch][zcap]
    double2* zval;             // [batch][zcap]
    uint32_t* zcount;          // [batch]
    int32_t* zflag;            // [batch] sticky capacity flag
    uint32_t zcap;
    double thr, iso_tol, gmin, prune, ref_lo, ref_hi, ref_tol;
    uint32_t first_round, last_round;
    // outputs written by the last round
    uint32_t* out_idx;
    double2* out_val;
    uint32_t out_cap;
    uint32_t* out_count;
    int32_t* out_flag;
    // single-hashing mode (sfft_hash_to_bins): explicit (sigma, b), bins written to ubins, no decode
    int bins_only;
    uint32_t e_sigma, e_b, e_nz;
    double2* ubins;
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

}  // namespace sfft

struct sfft_plan_s {
    sfft_params p{};
    uint32_t max_batch = 0;
    int device = 0;
    std::vector<sfft::ExactRound> rounds;
    std::vector<double> taps_host;  // every round's taps, FP64
    std::vector<double> wtab_host;  // every round's W(o), o = 0..n/2B
    float* d_taps32 = nullptr;
    double* d_taps64 = nullptr;
    double* d_wtab = nullptr;
    size_t wtab_len = 0;
    void* d_part = nullptr;
    size_t part_bytes = 0;
    size_t part_stride = 0;  // elements of the partial-fold buffer owned by one request
    uint32_t* d_counter = nullptr;
    uint32_t* d_zidx = nullptr;
    double2* d_zval = nullptr;
    uint32_t* d_zcount = nullptr;
    int32_t* d_zflag = nullptr;
    // single-step helpers
    double2* d_ubins = nullptr;
    uint32_t* d_aux = nullptr;
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
// host-side plan construction (sfft_host.cpp)
sfft_status build_exact_schedule(sfft_plan_s* pl);
void window_taps_host(uint64_t n, uint32_t B, double alpha, double delta, int64_t T, double* g);
void window_table_host(uint64_t n, const double* g, int64_t T, uint64_t len, double* W);
int64_t window_halfwidth(uint32_t B, double alpha, double delta);
void draw_exact_host(uint64_t seed, uint32_t request, uint32_t round, uint64_t n, uint64_t* sigma, uint64_t* b);
void set_last_error(const std::string& s);

// device entry points (sfft_exact.cu)
cudaError_t launch_exact_round(const ExactArgs& a, uint32_t batch, size_t smem, cudaStream_t st, bool fp64);
cudaError_t launch_exact_decode(const DecodeArgs& a, cudaStream_t st);
cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t count, uint32_t* out, cudaStream_t st);
size_t exact_finish_smem(uint32_t B, uint32_t H, uint32_t zcap, bool fp64);
size_t exact_gather_smem(uint32_t stage, bool fp64);
cudaError_t set_exact_smem_limit(size_t bytes, bool fp64);
}  // namespace sfft
