// sfft_general.cu -- the general-case sparse FFT on sm_103a (Algorithms 2 and 3 of Hassanieh, Indyk,
// Katabi, Price): SparseFFT's rounds of LocateSignal (LocateInner votes over D_max levels) and
// EstimateValues (medians over R_est hashings, top-k'), for a batch of requests.
//
// The hashings of one round are non-adaptive (the intuition of Sec. 4.1): every LocateInner pair
// (a, a + beta) of every level and every EstimateValues hashing is known before any vote is counted.
// So a round is four launches for the whole batch (five with the permuted copy):
//   0. k_gen_permute  (rounds whose LocateInner pairs gather >= 2n samples) every request: x_{sigma m}
//                     for all m under the round's sigma, so that the pairs read it in order;
//   1. k_gen_gather   every (chunk range, hashing group, request): permuted gather, window,
//                     modulation, fold mod B (HashToBins steps 1-2) into partial sums; the group's
//                     last CTA to arrive sums them in chunk order;
//   2. k_gen_finish   every (hashing group, request): the fold's B-point FFT
//                     (step 3), recovered coefficients subtracted in FP64 (step 4), bins stored;
//                     for a LocateInner pair also c_j = phase(u_j / u'_j);
//   3. k_gen_locate   every (bin, request), t threads per bin (one per subregion): LocateSignal's
//                     levels in order, votes, regions, the bin's candidate for the list L;
//   4. k_gen_estimate every (candidate share, request): EstimateValues' medians; the request's last
//                     CTA takes the top k' and zhat += w_J.
// Reductions run in a fixed order; results are bit-reproducible.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "philox.cuh"
#include "sfft_device.cuh"
#include "sfft_internal.h"

namespace sfft {

// ------------------------------------------------------------------------------------------------
// hashing parameters
// ------------------------------------------------------------------------------------------------
struct HashDesc {
    uint32_t sigma, b, H;
    uint32_t a[2];
    uint64_t beta;
};

// LocateSignal's sigma, b of round r (Algorithm 3: one draw per call)
__device__ __forceinline__ void locate_sigma_b(uint64_t seed, uint32_t s, uint32_t r, uint32_t nmask, uint32_t* sigma,
                                               uint32_t* b) {
    const Words4 w = draw(seed, s, r, 0, kKindLocate);
    *sigma = (w.w[0] & nmask) | 1u;
    *b = w.w[1] & nmask;
}

// LocateInner round q of level D (g = (D - 1) R_loc + q): a uniform on [n], beta uniform on the level's range
__device__ __forceinline__ void inner_a_beta(uint64_t seed, uint32_t s, uint32_t r, uint32_t g, uint32_t nmask,
                                             uint64_t lo, uint64_t hi, uint32_t* a, uint64_t* beta) {
    const Words4 w = draw(seed, s, r, g, kKindInner);
    *a = w.w[0] & nmask;
    *beta = lo + (((uint64_t)w.w[1] * (hi - lo + 1)) >> 32);
}

// Group g of a round: g < npairs is LocateInner pair g (hashings a and a + beta under the round's
// sigma, b); g >= npairs is EstimateValues hashing q = g - npairs with fresh (sigma_q, a_q, b_q).
__device__ __forceinline__ HashDesc group_desc(const GenArgs& a, uint64_t seed, uint32_t id, uint32_t g) {
    HashDesc h;
    if (g < a.npairs) {
        locate_sigma_b(seed, id, a.round, a.nmask, &h.sigma, &h.b);
        const uint32_t D = g / a.R_loc;
        inner_a_beta(seed, id, a.round, g, a.nmask, a.beta_lo[D], a.beta_hi[D], &h.a[0], &h.beta);
        h.a[1] = (uint32_t)((h.a[0] + h.beta) & a.nmask);
        h.H = 2;
    } else {
        const Words4 w = draw(seed, id, a.round, g - a.npairs, kKindEstimate);
        h.sigma = (w.w[0] & a.nmask) | 1u;
        h.b = w.w[1] & a.nmask;
        h.a[0] = w.w[2] & a.nmask;
        h.a[1] = 0;
        h.beta = 0;
        h.H = 1;
    }
    return h;
}

// request s of a general-mode launch (signal row, seed, draw index)
__device__ __forceinline__ ReqView gen_req(const GenArgs& a, uint32_t s) {
    return req_view(a.reqs, a.x, a.n * sizeof(float2), a.seed, s, a.nmask);
}

__device__ __forceinline__ uint32_t hash_index(const GenArgs& a, uint32_t g, uint32_t h) {
    return g < a.npairs ? 2 * g + h : 2 * a.npairs + (g - a.npairs);
}

// bin and offset of a permuted position (Sec. 3 definitions)
__device__ __forceinline__ int32_t gen_offset(uint32_t p, uint32_t n, uint32_t nmask, uint32_t logNp, uint32_t* jbin) {
    const uint32_t Np = 1u << logNp;
    const uint32_t jj = ((p + (Np >> 1)) & nmask) >> logNp;
    const uint32_t dd = (p - jj * Np) & nmask;
    *jbin = jj;
    return dd > (nmask >> 1) ? (int32_t)((int64_t)dd - (int64_t)n) : (int32_t)dd;
}

// ------------------------------------------------------------------------------------------------
// 0. permuted copy (rounds whose LocateInner pairs gather >= 2n samples)
// ------------------------------------------------------------------------------------------------
// xperm[m] = x_{sigma m} for every m in [n], sigma the round's LocateInner sigma: the pairs then read
// x_{sigma (t - a)} = xperm[(t - a) mod n] in order.  Grid (CTAs, batch); 8 loads in flight per thread.
__global__ void __launch_bounds__(kThreads) k_gen_permute(const GenArgs a) {
    const uint32_t s = a.req_base + blockIdx.y;
    const ReqView rq = gen_req(a, s);
    uint32_t sigma, b;
    locate_sigma_b(rq.seed, rq.id, a.round, a.nmask, &sigma, &b);
    const float2* __restrict__ x = static_cast<const float2*>(rq.x);
    float2* __restrict__ xp = a.xperm + (size_t)s * a.n;
    constexpr uint32_t kPer = kThreads * 8;
    for (uint64_t m0 = (uint64_t)blockIdx.x * kPer; m0 < a.n; m0 += (uint64_t)gridDim.x * kPer) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint64_t m = m0 + (uint64_t)q * kThreads + threadIdx.x;
            if (m < a.n) v[q] = __ldcg(x + ((sigma * (uint32_t)m) & rq.xmask));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint64_t m = m0 + (uint64_t)q * kThreads + threadIdx.x;
            if (m < a.n) xp[m] = v[q];
        }
    }
}

// ------------------------------------------------------------------------------------------------
// 1. gather and fold
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 3) k_gen_gather(const GenArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = a.req_base + blockIdx.z, g = blockIdx.y, c = blockIdx.x, tid = threadIdx.x;
    const ReqView rq = gen_req(a, s);
    const HashDesc h = group_desc(a, rq.seed, rq.id, g);
    float2* stage = reinterpret_cast<float2*>(smem);   // [2][kChunkTaps]
    float2* red = stage + 2 * kChunkTaps;               // [H][max(B, kThreads)]
    // a pair of a round with a permuted copy reads xperm[(t - a) mod n] = x_{sigma (t - a)} in order
    const bool perm = a.xperm != nullptr && g < a.npairs;
    const float2* __restrict__ x = perm ? a.xperm + (size_t)s * a.n : static_cast<const float2*>(rq.x);
    const uint32_t xmul = perm ? 1u : h.sigma, xmask = perm ? a.nmask : rq.xmask;
    const bool big = a.B > (uint32_t)kThreads;
    if (big)
        for (uint32_t i = tid; i < h.H * a.B; i += kThreads) red[i] = make_float2(0.f, 0.f);
    float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const uint32_t sb = h.sigma * h.b;
    const float inv_half_n = 2.0f / (float)a.n;
    const uint32_t c0 = c * a.cpb, c1 = min(c0 + a.cpb, a.chunks);
    int64_t t_first = -a.T + (int64_t)c0 * kChunkTaps;
    for (uint32_t ch = c0; ch < c1; ++ch) {
        const int64_t t_lo = -a.T + (int64_t)ch * kChunkTaps;
        const uint32_t ntap = (uint32_t)(min(t_lo + (int64_t)kChunkTaps, a.T + 1) - t_lo);
        // step 1a: x_{sigma (t - a_h)} for the chunk's taps of every hashing of the group, 16 loads in
        // flight per thread (a pair's whole chunk in one batch)
        const uint32_t total = h.H * ntap;
        for (uint32_t f0 = tid; f0 < total; f0 += kThreads * 16) {
            float2 v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t f = f0 + (uint32_t)q * kThreads;
                if (f < total) {
                    const bool second = f >= ntap;
                    const uint32_t i = second ? f - ntap : f;
                    const int32_t base = (int32_t)(t_lo - (int64_t)(second ? h.a[1] : h.a[0]));
                    v[q] = __ldcg(x + ((xmul * (uint32_t)(base + (int32_t)i)) & xmask));
                }
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t f = f0 + (uint32_t)q * kThreads;
                if (f < total) stage[f < ntap ? f : kChunkTaps + (f - ntap)] = v[q];
            }
        }
        __syncthreads();
        // step 1b + 2: window, modulation w^{sigma b t}, fold mod B
        for (uint32_t k = tid; k < ntap; k += kThreads) {
            const int32_t t = (int32_t)t_lo + (int32_t)k;
            const float gv = a.taps[t < 0 ? -t : t];
            const uint32_t e = (sb * (uint32_t)t) & a.nmask;
            const int32_t es = e > (a.nmask >> 1) ? (int32_t)((int64_t)e - (int64_t)a.n) : (int32_t)e;
            float sn, cs;
            sincospif((float)es * inv_half_n, &sn, &cs);
            const float2 gt = make_float2(gv * cs, -gv * sn);
            if (!big) {
                for (uint32_t hh = 0; hh < h.H; ++hh) acc[hh] = cfma(gt, stage[hh * kChunkTaps + k], acc[hh]);
            } else {
                const uint32_t r = (uint32_t)t & (a.B - 1);
                for (uint32_t hh = 0; hh < h.H; ++hh)
                    red[hh * a.B + r] = cfma(gt, stage[hh * kChunkTaps + k], red[hh * a.B + r]);
            }
        }
        __syncthreads();
    }
    float2* part = a.part + (size_t)s * a.part_stride + ((size_t)g * a.ctas + c) * 2 * a.B;
    if (!big) {
        // every chunk starts at a multiple of B away from the first, so thread tid always folds
        // residue (t_first + tid) mod B; the threads of residue r are owner + m B
        for (uint32_t hh = 0; hh < h.H; ++hh) red[hh * kThreads + tid] = acc[hh];
        __syncthreads();
        for (uint32_t r = tid; r < a.B; r += kThreads) {
            const uint32_t owner = (r - (uint32_t)t_first) & (a.B - 1);
            for (uint32_t hh = 0; hh < h.H; ++hh) {
                float2 sum = make_float2(0.f, 0.f);
                for (uint32_t m = owner; m < (uint32_t)kThreads; m += a.B) sum = cadd(sum, red[hh * kThreads + m]);
                part[hh * a.B + r] = sum;
            }
        }
    } else {
        for (uint32_t i = tid; i < h.H * a.B; i += kThreads) part[i] = red[i];
    }
    // step 2 across CTAs: the last CTA of this (request, group) to arrive sums the partial folds in
    // chunk order into slot 0, so the finish reads one fold per hashing
    if (a.ctas == 1 || arrive(a.gcount + (size_t)s * a.ngroups + g, a.ctas) == 0) return;
    float2* part0 = a.part + (size_t)s * a.part_stride + (size_t)g * a.ctas * 2 * a.B;
    for (uint32_t i = tid; i < h.H * a.B; i += kThreads) {
        const uint32_t hh = i / a.B, r = i - hh * a.B;
        const float2* src = part0 + (size_t)hh * a.B + r;
        float2 sum = make_float2(0.f, 0.f);
        uint32_t c0 = 0;
        for (; c0 + 8 <= a.ctas; c0 += 8) {  // 8 loads in flight, added in order
            float2 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __ldcg(src + (size_t)(c0 + q) * 2 * a.B);
#pragma unroll
            for (int q = 0; q < 8; ++q) sum = cadd(sum, v[q]);
        }
        for (; c0 < a.ctas; ++c0) sum = cadd(sum, __ldcg(src + (size_t)c0 * 2 * a.B));
        part0[(size_t)hh * a.B + r] = sum;
    }
    if (tid == 0) a.gcount[(size_t)s * a.ngroups + g] = 0;  // every CTA of the group has arrived
}

// ------------------------------------------------------------------------------------------------
// 2. finish the bins of one hashing group
// ------------------------------------------------------------------------------------------------
struct GenFinLayout {
    size_t U, ent_idx, ent_bin, ent_sub, bin_cnt, bin_start, bin_list, scan, total;
};
__host__ __device__ inline size_t gtake(size_t* off, size_t bytes) {
    const size_t o = (*off + 15) & ~size_t(15);
    *off = o + bytes;
    return o;
}
__host__ __device__ inline GenFinLayout gen_fin_layout(uint32_t B, uint32_t zcap) {
    GenFinLayout L;
    size_t off = 0;
    L.U = gtake(&off, (size_t)2 * B * 8);
    L.ent_idx = gtake(&off, (size_t)zcap * 4);
    L.ent_bin = gtake(&off, (size_t)zcap * 4);
    L.ent_sub = gtake(&off, (size_t)zcap * 2 * 16);
    L.bin_cnt = gtake(&off, (size_t)(B + 1) * 4);
    L.bin_start = gtake(&off, (size_t)(B + 1) * 4);
    L.bin_list = gtake(&off, (size_t)zcap * 4);
    L.scan = gtake(&off, (size_t)(kThreads + 8) * 4);
    L.total = off;
    return L;
}
size_t general_finish_smem(uint32_t B, uint32_t zcap) { return gen_fin_layout(B, zcap).total; }

__global__ void __launch_bounds__(kThreads) k_gen_finish(const GenArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = a.req_base + blockIdx.y, g = blockIdx.x, tid = threadIdx.x;
    const ReqView rq = gen_req(a, s);
    const HashDesc h = group_desc(a, rq.seed, rq.id, g);
    const uint32_t B = a.B;
    const GenFinLayout Ly = gen_fin_layout(B, a.zcap);
    // the arrays live in shared memory, or in this (request, group)'s slice of fin_scratch when large
    unsigned char* fb = a.fin_scratch ? a.fin_scratch + ((size_t)s * a.ngroups + g) * a.fin_stride : smem;
    float2* U = reinterpret_cast<float2*>(fb + Ly.U);
    uint32_t* ent_idx = reinterpret_cast<uint32_t*>(fb + Ly.ent_idx);
    uint32_t* ent_bin = reinterpret_cast<uint32_t*>(fb + Ly.ent_bin);
    double2* ent_sub = reinterpret_cast<double2*>(fb + Ly.ent_sub);
    uint32_t* bin_cnt = reinterpret_cast<uint32_t*>(fb + Ly.bin_cnt);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(fb + Ly.bin_start);
    uint32_t* bin_list = reinterpret_cast<uint32_t*>(fb + Ly.bin_list);
    uint32_t* scan = reinterpret_cast<uint32_t*>(fb + Ly.scan);
    const uint32_t logNp = (uint32_t)(63 - __clzll((long long)a.n)) - a.logB;
    // step 3: the fold (summed over chunks by the gather's last CTA), bit-reversed, B-point FFT per
    // hashing
    const float2* part = a.part + (size_t)s * a.part_stride + (size_t)g * a.ctas * 2 * B;
    const uint32_t shift_br = 32u - a.logB;
    for (uint32_t i = tid; i < h.H * B; i += kThreads) {
        const uint32_t hh = i / B, r = i - hh * B;
        U[hh * B + (__brev(r) >> shift_br)] = __ldcg(part + (size_t)hh * B + r);
    }
    // step 4 terms of the recovered coefficients: W(-o(i)) zhat_i w^{a_h sigma i}
    const uint32_t nz = min(a.zcount[s], a.zcap);
    for (uint32_t e = tid; e < nz; e += kThreads) {
        const uint32_t i = a.zidx[(size_t)s * a.zcap + e];
        ent_idx[e] = i;
        uint32_t jb;
        const int32_t o = gen_offset((h.sigma * (i - h.b)) & a.nmask, (uint32_t)a.n, a.nmask, logNp, &jb);
        ent_bin[e] = jb;
        const double gain = a.wtab[o < 0 ? -o : o];
        const double2 z = a.zval[(size_t)s * a.zcap + e];
        const double2 gz = make_double2(gain * z.x, gain * z.y);
        for (uint32_t hh = 0; hh < h.H; ++hh) {
            const double2 w = root_pow<float>((h.a[hh] * h.sigma * i) & a.nmask, a.nmask);
            ent_sub[2 * e + hh] = make_double2(gz.x * w.x - gz.y * w.y, gz.x * w.y + gz.y * w.x);
        }
    }
    __syncthreads();
    block_fft_rows<float>(U, h.H, a.logB);
    bucket_entries(ent_bin, nz, B, bin_cnt, bin_start, bin_list, scan);
    double2* bins = a.bins + (size_t)s * a.bins_stride;
    for (uint32_t j = tid; j < B; j += kThreads) {
        double2 u[2];
        for (uint32_t hh = 0; hh < h.H; ++hh) {
            const float2 v = U[hh * B + j];
            u[hh] = make_double2((double)v.x, (double)v.y);
        }
        for (uint32_t xx = bin_start[j]; xx < bin_start[j + 1]; ++xx) {
            const uint32_t e = bin_list[xx];
            for (uint32_t hh = 0; hh < h.H; ++hh) {
                u[hh].x -= ent_sub[2 * e + hh].x;
                u[hh].y -= ent_sub[2 * e + hh].y;
            }
        }
        for (uint32_t hh = 0; hh < h.H; ++hh) bins[(size_t)hash_index(a, g, hh) * B + j] = u[hh];
        // LocateInner's c_j: an FP32 arctangent of the FP64 product (the vote arcs are s pi wide and
        // the FP32 bins carry ~1e-6 of phase noise; GB300 runs FP64 at 1/64 of the FP32 rate)
        if (h.H == 2) a.phase[(size_t)s * a.phase_stride + (size_t)g * B + j] = phase01<float>(mul_conj_rn(u[0], u[1]));
    }
}

// ------------------------------------------------------------------------------------------------
// 3. LocateSignal: votes over the levels
// ------------------------------------------------------------------------------------------------
// One LocateInner vote test (Algorithm 3: |beta theta_{j,q} - c_j| circular < s pi).  f = e / M with
// e the exact fixed-point value of beta (m + sigma b) mod n and M = n 2^F.  The test is taken on
// integers except for the (rare) e next to a boundary, where the double expression of the test
// decides, evaluated exactly as written.
struct VoteBounds {
    uint64_t ilo, len;    // e is inside iff (e - ilo) mod M <= len
    uint64_t amb0, amb1;  // integers within 0.25 of a boundary (or ~0 when none)
    uint64_t g0, g1;      // starts of the guard windows around the two arc ends (glen = 0: none)
    uint64_t glen;        // e with (e - g0) mod M <= glen or (e - g1) mod M <= glen is in a window
    double c;
};
constexpr int kVoteGuard = 16;  // extra fraction bits of the fixed-point boundaries
// Guard band of an FP32 phase.  The pipeline's c comes from an FP32 arctangent of the FP64
// product u_j conj(u'_j): rounding the product to float and atan2f's few-ulp error move it by less
// than 2e-7 of a turn from the FP64 phase.  A vote whose e lies within 2^-20 of a turn (about 1e-6)
// of an arc end of c is decided by the FP64 test on the FP64 phase instead; every other e is at
// least 2^-20 - 2e-7 of a turn from the arc ends of either phase, so both give the same vote.
constexpr int kPhaseGuardLog = 20;
// Boundaries of the vote arc (c - s/2, c + s/2) in units of 1/M, as 64-bit fixed point with
// kVoteGuard fraction bits: c M 2^G is one exact scaling of c (truncated to an integer, an error
// below 2^-G units), so only one double operation is spent per (bin, round).  guard: half width of
// the guard windows in units of 1/M (0 for an FP64 phase, which needs none).
__device__ __forceinline__ VoteBounds vote_bounds(double c, int64_t hw_fix, uint32_t logM, uint64_t guard = 0) {
    VoteBounds v;
    const int64_t one = int64_t(1) << kVoteGuard, frac_mask = one - 1;
    const int64_t xfix = (int64_t)(c * ldexp(1.0, (int)logM + kVoteGuard));
    const int64_t blf = xfix - hw_fix, bhf = xfix + hw_fix;
    const uint64_t mask = (uint64_t(1) << logM) - 1;
    const int64_t ilo = (blf >> kVoteGuard) + 1;                  // smallest integer > bl
    const int64_t ihi = ((bhf + frac_mask) >> kVoteGuard) - 1;    // largest integer < bh
    v.ilo = (uint64_t)ilo & mask;
    v.len = (uint64_t)(ihi - ilo) & mask;
    const int64_t fl = blf & frac_mask, fh = bhf & frac_mask;
    v.amb0 = fl < one / 4 ? ((uint64_t)(blf >> kVoteGuard) & mask)
                          : (fl > 3 * (one / 4) ? ((uint64_t)((blf >> kVoteGuard) + 1) & mask) : ~0ull);
    v.amb1 = fh < one / 4 ? ((uint64_t)(bhf >> kVoteGuard) & mask)
                          : (fh > 3 * (one / 4) ? ((uint64_t)((bhf >> kVoteGuard) + 1) & mask) : ~0ull);
    v.g0 = (uint64_t)((blf >> kVoteGuard) - (int64_t)guard) & mask;
    v.g1 = (uint64_t)((bhf >> kVoteGuard) - (int64_t)guard) & mask;
    v.glen = 2 * guard + 1;
    if (guard == 0) v.glen = 0;
    v.c = c;
    return v;
}
__device__ __forceinline__ bool in_guard(const VoteBounds& v, uint64_t e, uint64_t mask) {
    return v.glen != 0 && (((e - v.g0) & mask) <= v.glen || ((e - v.g1) & mask) <= v.glen);
}
// The vote test on a given phase c, as written in Algorithm 3 (circular distance below s pi), in
// double precision: the decision of a guarded e.
__device__ __forceinline__ bool vote_hit_exact(double c, uint64_t e, uint64_t M, double s) {
    const double f = (double)e / (double)M;
    double dist = fabs(f - c);
    if (dist > 0.5) dist = 1.0 - dist;
    return dist < s / 2.0;
}
// half width s M / 2 of the vote arc in the same fixed point
__device__ __forceinline__ int64_t vote_halfwidth(double s, uint32_t logM) {
    return (int64_t)llrint(0.5 * s * ldexp(1.0, (int)logM + kVoteGuard));
}
__device__ __forceinline__ bool vote_hit(const VoteBounds& v, uint64_t e, uint64_t M, double s) {
    if (e == v.amb0 || e == v.amb1) return vote_hit_exact(v.c, e, M, s);
    return ((e - v.ilo) & (M - 1)) <= v.len;
}

// Votes of bin j at one level, then its region update (the four consecutive subregions with the
// most votes among those with a majority; bottom when no subregion has one).
// phase(q) returns c_j of LocateInner round q; beta[q] its beta.  T = t subregions, a compile-time
// constant so that the vote counters live in registers.
template <int T, typename PhaseFn>
__device__ __forceinline__ void locate_bin_t(uint32_t nrep, const uint64_t* beta, PhaseFn phase, uint64_t sb_fp,
                                             uint64_t w_fp, uint32_t logM, double s, int64_t hw_fix, uint64_t& l_fp,
                                             uint8_t& valid, uint32_t* votes_out) {
    uint32_t v[T];
#pragma unroll
    for (int q = 0; q < T; ++q) v[q] = 0;
    const uint64_t M = uint64_t(1) << logM;
    const uint64_t mask = M - 1;
    const uint64_t half_step = w_fp / (2 * (uint64_t)T), step = w_fp / T;
    for (uint32_t r = 0; r < nrep; ++r) {
        const VoteBounds vb = vote_bounds(phase(r), hw_fix, logM);
        // e_q = beta (m_q + sigma b) mod M, m_q = l + (2q - 1) w / 2t, advanced by beta w / t
        uint64_t e = (beta[r] * ((l_fp + half_step + sb_fp) & mask)) & mask;
        const uint64_t de = (beta[r] * step) & mask;
#pragma unroll
        for (int q = 0; q < T; ++q) {
            if (vote_hit(vb, e, M, s)) v[q] += 1;
            e = (e + de) & mask;
        }
    }
    if (votes_out) {
#pragma unroll
        for (int q = 0; q < T; ++q) votes_out[q] = v[q];
    }
    bool any = false;
#pragma unroll
    for (int q = 0; q < T; ++q) any = any || 2u * v[q] > nrep;
    if (!any) {
        valid = 0;
        return;
    }
    uint32_t best = 0, best_sum = 0;
#pragma unroll
    for (int q0 = 0; q0 + 4 <= T; ++q0) {
        const uint32_t sum = v[q0] + v[q0 + 1] + v[q0 + 2] + v[q0 + 3];
        if (q0 == 0 || sum > best_sum) {
            best = (uint32_t)q0;
            best_sum = sum;
        }
    }
    l_fp = (l_fp + (uint64_t)best * step) & mask;
}
template <typename PhaseFn>
__device__ void locate_bin(uint32_t t, uint32_t nrep, const uint64_t* beta, PhaseFn phase, uint64_t sb_fp,
                           uint64_t w_fp, uint32_t logM, double s, int64_t hw_fix, uint64_t& l_fp, uint8_t& valid,
                           uint32_t* votes_out) {
    // the schedule admits t in {8, 16, 32} (a power of two in [8, kMaxT])
    if (t == 8)
        locate_bin_t<8>(nrep, beta, phase, sb_fp, w_fp, logM, s, hw_fix, l_fp, valid, votes_out);
    else if (t == 16)
        locate_bin_t<16>(nrep, beta, phase, sb_fp, w_fp, logM, s, hw_fix, l_fp, valid, votes_out);
    else
        locate_bin_t<32>(nrep, beta, phase, sb_fp, w_fp, logM, s, hw_fix, l_fp, valid, votes_out);
}

size_t general_locate_smem(uint32_t B) {
    (void)B;
    return 0;
}

// Ascending bitonic sort of the P keys of k[] (P a power of two), one CTA; ends with a barrier.
__device__ void block_bitonic_sort_u32(uint32_t* k, uint32_t P) {
    for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += kThreads) {
                const uint32_t j = i ^ stride;
                if (j > i) {
                    const uint32_t x = k[i], y = k[j];
                    if ((i & size) == 0 ? x > y : x < y) {
                        k[i] = y;
                        k[j] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sorts the m keys of key[0..m) ascending (key holds P >= m words, P a power of two; keys < 2^32 - 1)
// and writes the distinct ones to out[0..returned count).  keep holds m words.  Up to kThreads keys
// are ranked directly (one key per thread, ties by position); more are sorted by a bitonic network
// over the smallest power of two >= m.
__device__ uint32_t sort_unique_u32(uint32_t* key, uint32_t m, uint32_t P, uint32_t* out, uint32_t* keep,
                                    uint32_t* scan) {
    const uint32_t* sorted = key;
    if (m <= (uint32_t)kThreads) {
        if (threadIdx.x < m) {
            const uint32_t c = threadIdx.x, k = key[c];
            uint32_t r = 0;
            for (uint32_t q = 0; q < m; ++q) r += (key[q] < k || (key[q] == k && q < c)) ? 1u : 0u;
            out[r] = k;
        }
        __syncthreads();
        sorted = out;
    } else {
        uint32_t Pm = 1;
        while (Pm < m && Pm < P) Pm <<= 1;  // key holds P words and m <= P
        for (uint32_t p = m + threadIdx.x; p < Pm; p += kThreads) key[p] = 0xFFFFFFFFu;  // sort last
        __syncthreads();
        block_bitonic_sort_u32(key, Pm);
    }
    for (uint32_t p = threadIdx.x; p < m; p += kThreads) keep[p] = (p == 0 || sorted[p - 1] != sorted[p]) ? 1u : 0u;
    __syncthreads();
    const uint32_t total = block_exclusive_scan(keep, m, scan);  // keep[p]: output slot of a kept key
    // compaction: into out from key, or within out (then every kept key is read before any write)
    if (sorted == out) {
        uint32_t mine = 0, slot = 0;
        bool kept = false;
        if (threadIdx.x < m) {
            const uint32_t p = threadIdx.x;
            const uint32_t nxt = p + 1 < m ? keep[p + 1] : total;
            kept = nxt != keep[p];
            mine = out[p];
            slot = keep[p];
        }
        __syncthreads();
        if (kept) out[slot] = mine;
    } else {
        for (uint32_t p = threadIdx.x; p < m; p += kThreads) {
            const uint32_t nxt = p + 1 < m ? keep[p + 1] : total;
            if (nxt != keep[p]) out[keep[p]] = key[p];
        }
    }
    __syncthreads();
    return total;
}

// LocateSignal with t threads per bin, thread q owning subregion q: a CTA holds kThreads / t bins of
// one request (the bins are independent until L is formed).  Per level, the vote arcs of the R_loc
// rounds are formed once per bin (by threads q < R_loc, in shared memory), every thread counts the
// votes of its subregion over the rounds, and the bin's t threads take the level's decision from the
// t counts with warp shuffles (the decision of locate_bin_t, on the same integers).  The candidate of bin j
// (pi^{-1} of the integer nearest the centre of its last region, or ~0 for bottom) goes to
// L[s B + j]; EstimateValues sorts and de-duplicates them.
constexpr int kLocBins = kThreads / 8;  // bins per CTA at the smallest t
__global__ void __launch_bounds__(kThreads) k_gen_locate(const GenArgs a) {
    __shared__ uint64_t s_beta[kMaxRloc];
    __shared__ VoteBounds s_vb[kLocBins][kMaxRloc];
    const uint32_t s = a.req_base + blockIdx.y, tid = threadIdx.x;
    const uint32_t t = a.t;  // 8, 16 or 32 (the schedule checks it)
    const uint32_t q = tid & (t - 1), lb = tid / t, nb = kThreads / t;
    const uint32_t B = a.B;
    const uint32_t j = blockIdx.x * nb + lb;
    const ReqView rq = gen_req(a, s);
    uint32_t sigma, b;
    locate_sigma_b(rq.seed, rq.id, a.round, a.nmask, &sigma, &b);
    const uint64_t n = a.n, Np = n >> a.logB;
    const uint32_t logM = (uint32_t)(63 - __clzll((long long)n)) + kFracBits;
    const uint64_t M = uint64_t(1) << logM, mask = M - 1;
    const int64_t hw_fix = vote_halfwidth(a.s, logM);
    const uint64_t guard = M >> kPhaseGuardLog;
    const uint64_t sb_fp = ((uint64_t)((sigma * b) & a.nmask)) << kFracBits;
    const double2* rbins = a.bins + (size_t)s * a.bins_stride;
    // the bin's region (start l_fp, width w_D) and its bottom flag live in registers, the same in every
    // lane of the bin's group: the t lanes of a bin share a warp (t divides 32), so the level's
    // decision is taken with warp shuffles and ballots inside the group
    uint64_t l_fp = ((((uint64_t)j * Np) + n - Np / 2) & (n - 1)) << kFracBits;  // centred on the bin
    bool valid = j < B;
    const uint32_t lane = tid & 31u, gbase = lane & ~(t - 1u);
    const uint32_t gmask = t == 32u ? 0xFFFFFFFFu : ((1u << t) - 1u) << gbase;
    const double* phase = a.phase + (size_t)s * a.phase_stride;
    for (uint32_t D = 0; D < a.dmax; ++D) {
        __syncthreads();  // the previous level's readers of s_beta and s_vb are done
        if (tid < a.R_loc) {
            uint32_t aa;
            uint64_t be;
            inner_a_beta(rq.seed, rq.id, a.round, D * a.R_loc + tid, a.nmask, a.beta_lo[D], a.beta_hi[D], &aa, &be);
            s_beta[tid] = be;
        }
        const double* ph = phase + (size_t)D * a.R_loc * B;
        if (valid)
            for (uint32_t r = q; r < a.R_loc; r += t)
                s_vb[lb][r] = vote_bounds(ph[(size_t)r * B + j], hw_fix, logM, guard);
        __syncthreads();
        const uint64_t w_fp = (Np << kFracBits) >> ((uint64_t)D * a.logtp);
        const uint64_t half_step = w_fp / (2 * (uint64_t)t), step = w_fp / t;
        uint32_t v = 0;
        if (valid) {
            for (uint32_t r = 0; r < a.R_loc; ++r) {
                // e_q = beta (m_q + sigma b) mod M, m_q = l + (2q - 1) w / 2t
                const uint64_t e0 = (s_beta[r] * ((l_fp + half_step + sb_fp) & mask)) & mask;
                const uint64_t de = (s_beta[r] * step) & mask;
                const uint64_t e = (e0 + (uint64_t)q * de) & mask;
                const VoteBounds& vb = s_vb[lb][r];
                bool hit;
                if (in_guard(vb, e, mask)) {
                    // near an arc end of the FP32 phase: the FP64 phase of the pair's stored bins
                    const double2* pb = rbins + (size_t)2 * (D * a.R_loc + r) * B;
                    hit = vote_hit_exact(phase01<double>(mul_conj_rn(pb[j], pb[B + j])), e, M, a.s);
                } else {
                    hit = vote_hit(vb, e, M, a.s);
                }
                if (hit) ++v;
            }
        }
        // the level's decision (every lane of the warp takes part; a group's lanes share `valid`):
        // Q* nonempty iff some subregion has more than R_loc / 2 votes; then the window of 4
        // consecutive subregions with the most votes, the first on ties, gives the new region
        const bool any = (__ballot_sync(0xFFFFFFFFu, 2u * v > a.R_loc) & gmask) != 0u;
        uint32_t sum = v + __shfl_down_sync(0xFFFFFFFFu, v, 1, (int)t) + __shfl_down_sync(0xFFFFFFFFu, v, 2, (int)t) +
                       __shfl_down_sync(0xFFFFFFFFu, v, 3, (int)t);
        uint32_t key = q + 4u <= t ? (sum << 8) | (255u - q) : 0u;  // larger sum, then smaller q
        for (uint32_t off = t >> 1; off > 0; off >>= 1) key = max(key, __shfl_xor_sync(0xFFFFFFFFu, key, (int)off, (int)t));
        if (valid) {
            if (!any)
                valid = false;
            else
                l_fp = (l_fp + (uint64_t)(255u - (key & 255u)) * step) & mask;
        }
        if (q == 0 && j < B && a.dbg_lfp) {  // trace: the region and flag after this level
            a.dbg_lfp[((size_t)s * a.dmax + D) * B + j] = l_fp;
            a.dbg_valid[((size_t)s * a.dmax + D) * B + j] = (uint8_t)(valid ? 1 : 0);
        }
    }
    if (q != 0 || j >= B) return;
    uint32_t cand = 0xFFFFFFFFu;
    if (valid) {
        const uint64_t wlast = (Np << kFracBits) >> ((uint64_t)a.dmax * a.logtp);
        const uint32_t tau = (uint32_t)(((l_fp + wlast / 2 + (1ull << (kFracBits - 1))) >> kFracBits) & (n - 1));
        cand = ((inverse_odd(sigma) & a.nmask) * tau + b) & a.nmask;
    }
    a.L[(size_t)s * B + j] = cand;
}

// ------------------------------------------------------------------------------------------------
// 4. EstimateValues, top k', zhat += w_J
// ------------------------------------------------------------------------------------------------
struct EstLayout {
    size_t w, mag, perm, topi, topv, out_idx, out_val, keep, scan, draws, Lk, Lt, total;
    uint32_t P;
};
__host__ __device__ inline EstLayout est_layout(uint32_t B, uint32_t kprime, uint32_t zcap) {
    EstLayout L;
    size_t off = 0;
    uint32_t P = 1;
    while (P < B) P <<= 1;
    L.P = P;
    L.w = gtake(&off, (size_t)B * 16);
    L.mag = gtake(&off, (size_t)B * 8);
    L.perm = gtake(&off, (size_t)P * 4);
    L.topi = gtake(&off, (size_t)kprime * 4);
    L.topv = gtake(&off, (size_t)kprime * 16);
    L.out_idx = gtake(&off, (size_t)(zcap + kprime) * 4);
    L.out_val = gtake(&off, (size_t)(zcap + kprime) * 16);
    L.keep = gtake(&off, (size_t)(zcap + kprime > B ? zcap + kprime : B) * 4);
    L.scan = gtake(&off, (size_t)(kThreads + 8) * 4);
    L.draws = gtake(&off, (size_t)kMaxRest * 3 * 8);
    L.Lk = gtake(&off, (size_t)B * 4);
    L.Lt = gtake(&off, (size_t)B * 4);
    L.total = off;
    return L;
}
size_t general_estimate_smem(uint32_t B, uint32_t kprime, uint32_t zcap) { return est_layout(B, kprime, zcap).total; }

// w_i = median_q Re e_q + i median_q Im e_q over the hashings q whose window gain at i is >= est_gmin,
// e_q = u^{(q)}_{h_q(i)} w^{-a_q sigma_q i} / W(-o_q(i)); lower median; 0 when no hashing qualifies.
// w^e = exp(-2 pi i e / n) for an exact exponent e in [0, n) from two tables of FP64 factors,
// exp(-2 pi i (e mod 2^sh) / n) and exp(-2 pi i 2^sh (e >> sh) / n): one complex product (a few ulp
// from a direct evaluation) instead of an FP64 sincospi, which GB300 runs at 1/64 of the FP32 rate
__device__ __forceinline__ double2 root_pow_tab(uint32_t e, const double2* tw, uint32_t sh) {
    const double2 lo = tw[e & ((1u << sh) - 1u)], hi = tw[(1u << sh) + (e >> sh)];
    return make_double2(hi.x * lo.x - hi.y * lo.y, hi.x * lo.y + hi.y * lo.x);
}

template <typename BinFn>
__device__ double2 estimate_one(uint32_t i, uint32_t nrep, const uint64_t* sig, const uint64_t* bb, const uint64_t* aa,
                                BinFn bin, uint32_t n, uint32_t nmask, uint32_t logNp, const double* wtab, double gmin,
                                const double2* tw, uint32_t tw_shift) {
    double re[kMaxRest], im[kMaxRest];
    uint32_t m = 0;
    for (uint32_t q = 0; q < nrep; ++q) {
        const uint32_t sq = (uint32_t)sig[q];
        const uint32_t p = (sq * (i - (uint32_t)bb[q])) & nmask;
        uint32_t j;
        const int32_t o = gen_offset(p, n, nmask, logNp, &j);
        const double gain = wtab[o < 0 ? -o : o];
        if (!(gain >= gmin)) continue;
        const uint32_t e = ((uint32_t)aa[q] * sq * i) & nmask;
        const double2 w = root_pow_tab(e, tw, tw_shift);
        const double2 u = bin(q, j);
        const double2 v = mul_conj_rn(u, w);
        const double x = __ddiv_rn(v.x, gain), y = __ddiv_rn(v.y, gain);
        // insertion into the sorted prefixes
        uint32_t pr = m, pi = m;
        while (pr > 0 && re[pr - 1] > x) {
            re[pr] = re[pr - 1];
            --pr;
        }
        re[pr] = x;
        while (pi > 0 && im[pi - 1] > y) {
            im[pi] = im[pi - 1];
            --pi;
        }
        im[pi] = y;
        ++m;
    }
    if (m == 0) return make_double2(0.0, 0.0);
    return make_double2(re[(m - 1) / 2], im[(m - 1) / 2]);
}

// (mag2 descending, index ascending) order of candidates via a bitonic sort of a permutation over the
// smallest power of two >= m (<= P).  mag2 >= 0 is finite, so its IEEE bit pattern orders like its
// value and the comparisons run on the integer units (GB300's FP64 pipe runs at 1/64 rate).
__device__ void sort_by_magnitude(const double* mag, const uint32_t* idx, uint32_t m, uint32_t P, uint32_t* perm) {
    uint32_t Pm = 1;
    while (Pm < m && Pm < P) Pm <<= 1;
    for (uint32_t p = threadIdx.x; p < Pm; p += kThreads) perm[p] = p;
    __syncthreads();
    const unsigned long long* mb = reinterpret_cast<const unsigned long long*>(mag);
    auto before = [&](uint32_t a, uint32_t b) -> bool {  // a ranks before b
        if (a >= m) return false;
        if (b >= m) return true;
        const unsigned long long x = mb[a], y = mb[b];
        if (x != y) return x > y;
        return idx[a] < idx[b];
    };
    for (uint32_t k = 2; k <= Pm; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < Pm; i += kThreads) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t pa = perm[i], pb = perm[ixj];
                    const bool swap = up ? before(pb, pa) : before(pa, pb);
                    if (swap) {
                        perm[i] = pb;
                        perm[ixj] = pa;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Grid (E, batch): the E CTAs of a request each form L and estimate their share of its candidates;
// with E > 1 the shares go through est_w / est_mag and the last CTA to arrive takes the top k' and
// the merge.  E = 1 when the arrays live in est_scratch (one slice per request).
__global__ void __launch_bounds__(kThreads) k_gen_estimate(const GenArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = a.req_base + blockIdx.y, tid = threadIdx.x, B = a.B, E = gridDim.x;
    const EstLayout Ly = est_layout(B, a.kprime, a.zcap);
    // the arrays live in shared memory, or in this request's slice of est_scratch when large
    unsigned char* eb = a.est_scratch ? a.est_scratch + (size_t)s * a.est_stride : smem;
    double2* wv = reinterpret_cast<double2*>(eb + Ly.w);
    double* mag = reinterpret_cast<double*>(eb + Ly.mag);
    uint32_t* perm = reinterpret_cast<uint32_t*>(eb + Ly.perm);
    uint32_t* topi = reinterpret_cast<uint32_t*>(eb + Ly.topi);
    double2* topv = reinterpret_cast<double2*>(eb + Ly.topv);
    uint32_t* out_idx = reinterpret_cast<uint32_t*>(eb + Ly.out_idx);
    double2* out_val = reinterpret_cast<double2*>(eb + Ly.out_val);
    uint32_t* keep = reinterpret_cast<uint32_t*>(eb + Ly.keep);
    uint32_t* scan = reinterpret_cast<uint32_t*>(eb + Ly.scan);
    uint64_t* dr = reinterpret_cast<uint64_t*>(eb + Ly.draws);  // sigma, b, a per hashing
    const ReqView rq = gen_req(a, s);
    if (tid < a.R_est) {
        const Words4 w = draw(rq.seed, rq.id, a.round, tid, kKindEstimate);
        dr[tid] = (w.w[0] & a.nmask) | 1u;
        dr[kMaxRest + tid] = w.w[1] & a.nmask;
        dr[2 * kMaxRest + tid] = w.w[2] & a.nmask;
    }
    __syncthreads();
    // L: the candidates of the bins that LocateSignal did not reject, sorted and de-duplicated
    uint32_t* Lk = reinterpret_cast<uint32_t*>(eb + Ly.Lk);
    uint32_t* Lt = reinterpret_cast<uint32_t*>(eb + Ly.Lt);
    __shared__ uint32_t s_m;
    if (tid == 0) s_m = 0;
    __syncthreads();
    for (uint32_t j = tid; j < B; j += kThreads) {
        const uint32_t c = a.L[(size_t)s * B + j];
        if (c != 0xFFFFFFFFu) Lk[atomicAdd(&s_m, 1u)] = c;
    }
    __syncthreads();
    const uint32_t nL = sort_unique_u32(Lk, s_m, Ly.P, Lt, keep, scan);
    const uint32_t* L = Lt;
    if (tid == 0 && blockIdx.x == 0) a.nL[s] = nL;
    const double2* bins = a.bins + (size_t)s * a.bins_stride + (size_t)2 * a.npairs * B;
    const uint32_t logNp = (uint32_t)(63 - __clzll((long long)a.n)) - a.logB;
    double2* gw = a.est_w + (size_t)s * B;
    double* gmag = a.est_mag + (size_t)s * B;
    for (uint32_t c = blockIdx.x * kThreads + tid; c < nL; c += E * kThreads) {
        const double2 w = estimate_one(L[c], a.R_est, dr, dr + kMaxRest, dr + 2 * kMaxRest,
                                       [&](uint32_t q, uint32_t j) { return bins[(size_t)q * B + j]; }, (uint32_t)a.n,
                                       a.nmask, logNp, a.wtab, a.est_gmin, a.tw, a.tw_shift);
        const double m2 = __dadd_rn(__dmul_rn(w.x, w.x), __dmul_rn(w.y, w.y));
        if (E == 1) {
            wv[c] = w;
            mag[c] = m2;
        } else {
            gw[c] = w;
            gmag[c] = m2;
        }
    }
    if (E > 1) {
        if (arrive(a.ecount + s, E) == 0) return;
        for (uint32_t c = tid; c < nL; c += kThreads) {
            wv[c] = __ldcg(gw + c);
            mag[c] = __ldcg(gmag + c);
        }
        if (tid == 0) a.ecount[s] = 0;  // every CTA of the request has arrived
    }
    __syncthreads();
    sort_by_magnitude(mag, L, nL, Ly.P, perm);
    const uint32_t nJ = nL < a.kprime ? nL : a.kprime;
    // J sorted by index: the kept candidates are a subset of the ascending L, so keep L's order
    for (uint32_t c = tid; c < nL; c += kThreads) keep[c] = 0;
    __syncthreads();
    for (uint32_t r = tid; r < nJ; r += kThreads) keep[perm[r]] = 1;
    __syncthreads();
    const uint32_t total = block_exclusive_scan(keep, nL, scan);
    for (uint32_t c = tid; c < nL; c += kThreads) {
        const uint32_t nxt = c + 1 < nL ? keep[c + 1] : total;
        if (nxt != keep[c]) {
            topi[keep[c]] = L[c];
            topv[keep[c]] = wv[c];
        }
    }
    __syncthreads();
    // zhat <- zhat + w_J (zhat first on equal indices); nothing is dropped in the general case
    const uint32_t nz = min(a.zcount[s], a.zcap);
    uint32_t* zi = a.zidx + (size_t)s * a.zcap;
    double2* zv = a.zval + (size_t)s * a.zcap;
    for (uint32_t e = tid; e < nz; e += kThreads) {
        const uint32_t key = zi[e];
        const uint32_t pos = e + lower_bound_u32(topi, nJ, key);
        out_idx[pos] = key;
        out_val[pos] = zv[e];
    }
    for (uint32_t c = tid; c < nJ; c += kThreads) {
        const uint32_t pos = c + upper_bound_u32(zi, nz, topi[c]);
        out_idx[pos] = topi[c];
        out_val[pos] = topv[c];
    }
    __syncthreads();
    const uint32_t tot = nz + nJ;
    for (uint32_t p = tid; p < tot; p += kThreads) {
        const uint32_t idx = out_idx[p];
        uint32_t kp = 0;
        if (p == 0 || out_idx[p - 1] != idx) {
            if (p + 1 < tot && out_idx[p + 1] == idx) {
                out_val[p] = make_double2(out_val[p].x + out_val[p + 1].x, out_val[p].y + out_val[p + 1].y);
            }
            kp = 1;
        }
        keep[p] = kp;
    }
    __syncthreads();
    const uint32_t newcount = block_exclusive_scan(keep, tot, scan);
    const bool last = a.last_round != 0;
    for (uint32_t p = tid; p < tot; p += kThreads) {
        const uint32_t pos = keep[p];
        const uint32_t nxt = p + 1 < tot ? keep[p + 1] : newcount;
        if (nxt == pos) continue;
        if (pos < a.zcap) {
            zi[pos] = out_idx[p];
            zv[pos] = out_val[p];
        }
        if (last && pos < a.out_cap) {
            a.out_idx[(size_t)s * a.out_cap + pos] = out_idx[p];
            a.out_val[(size_t)s * a.out_cap + pos] = out_val[p];
        }
    }
    __syncthreads();
    if (tid == 0) {
        const bool overflow = newcount > a.zcap;
        if (overflow) a.zflag[s] = 1;
        a.zcount[s] = overflow ? a.zcap : newcount;
        if (last) {
            const uint32_t kept = overflow ? a.zcap : newcount;
            a.out_count[s] = kept < a.out_cap ? kept : a.out_cap;
            a.out_flag[s] = (a.zflag[s] || kept > a.out_cap) ? SFFT_ERR_CAPACITY : SFFT_OK;
        }
    }
}

// ------------------------------------------------------------------------------------------------
// single-step kernels on caller bins
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_locate_votes(const VoteArgs a) {
    const uint32_t logM = (uint32_t)(63 - __clzll((long long)a.n)) + kFracBits;
    const int64_t hw_fix = vote_halfwidth(a.s, logM);
    const uint64_t sb_fp = ((uint64_t)((a.sigma * a.b) & a.nmask)) << kFracBits;
    for (uint32_t j = threadIdx.x; j < a.B; j += kThreads) {
        for (uint32_t q = 0; q < a.t; ++q) a.votes[(size_t)j * a.t + q] = 0;
        if (!a.valid[j]) continue;
        uint64_t l = a.l_fp[j];
        uint8_t v = 1;
        locate_bin(a.t, a.nrep, a.beta,
                   [&](uint32_t r) {
                       return phase01<double>(mul_conj_rn(a.u[(size_t)r * a.B + j], a.up[(size_t)r * a.B + j]));
                   },
                   sb_fp, a.w_fp, logM, a.s, hw_fix, l, v, a.votes + (size_t)j * a.t);
        a.l_fp[j] = l;
        a.valid[j] = v;
    }
}

__global__ void __launch_bounds__(kThreads) k_estimate_from_bins(const EstArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t tid = threadIdx.x;
    const EstLayout Ly = est_layout(a.nL > 0 ? a.nL : 1, a.kprime > 0 ? a.kprime : 1, 1);
    double2* wv = reinterpret_cast<double2*>(smem + Ly.w);
    double* mag = reinterpret_cast<double*>(smem + Ly.mag);
    uint32_t* perm = reinterpret_cast<uint32_t*>(smem + Ly.perm);
    uint32_t* keep = reinterpret_cast<uint32_t*>(smem + Ly.keep);
    uint32_t* scan = reinterpret_cast<uint32_t*>(smem + Ly.scan);
    const uint32_t logNp = (uint32_t)(63 - __clzll((long long)a.n)) - a.logB;
    for (uint32_t c = tid; c < a.nL; c += kThreads) {
        const double2 w = estimate_one(a.L[c], a.nrep, a.sig, a.bb, a.aa,
                                       [&](uint32_t q, uint32_t j) { return a.u[(size_t)q * a.B + j]; }, (uint32_t)a.n,
                                       a.nmask, logNp, a.wtab, a.est_gmin, a.tw, a.tw_shift);
        wv[c] = w;
        mag[c] = __dadd_rn(__dmul_rn(w.x, w.x), __dmul_rn(w.y, w.y));
    }
    __syncthreads();
    sort_by_magnitude(mag, a.L, a.nL, Ly.P, perm);
    const uint32_t nJ = a.nL < a.kprime ? a.nL : a.kprime;
    for (uint32_t c = tid; c < a.nL; c += kThreads) keep[c] = 0;
    __syncthreads();
    for (uint32_t r = tid; r < nJ; r += kThreads) keep[perm[r]] = 1;
    __syncthreads();
    const uint32_t total = block_exclusive_scan(keep, a.nL, scan);
    for (uint32_t c = tid; c < a.nL; c += kThreads) {
        const uint32_t nxt = c + 1 < a.nL ? keep[c + 1] : total;
        if (nxt != keep[c]) {
            a.widx[keep[c]] = a.L[c];
            a.wval[keep[c]] = wv[c];
        }
    }
    if (tid == 0) *a.count = total;
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
cudaError_t general_set_smem(size_t gather, size_t finish, size_t locate, size_t estimate) {
    static std::mutex mu;  // plans may be created from several threads
    std::lock_guard<std::mutex> lk(mu);
    static size_t lim[4] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    if (gather > lim[0] && (e = cudaFuncSetAttribute(k_gen_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)gather)) == cudaSuccess)
        lim[0] = gather;
    if (e != cudaSuccess) return e;
    if (finish > lim[1] && (e = cudaFuncSetAttribute(k_gen_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)finish)) == cudaSuccess)
        lim[1] = finish;
    if (e != cudaSuccess) return e;
    if (locate > lim[2] && (e = cudaFuncSetAttribute(k_gen_locate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)locate)) == cudaSuccess)
        lim[2] = locate;
    if (e != cudaSuccess) return e;
    if (estimate > lim[3]) {
        e = cudaFuncSetAttribute(k_gen_estimate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)estimate);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_estimate_from_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)estimate);
        if (e == cudaSuccess) lim[3] = estimate;
    }
    return e;
}

cudaError_t launch_general_round(const GenArgs& a, uint32_t batch, const GeneralRound& r, cudaStream_t st) {
    if (r.perm) {
        const uint64_t per = (uint64_t)kThreads * 8, blocks = (a.n + per - 1) / per;
        k_gen_permute<<<dim3((uint32_t)(blocks < 65535 ? blocks : 65535), batch), kThreads, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_gen_gather<<<dim3(r.ctas, r.ngroups, batch), kThreads, r.smem_gather, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gen_finish<<<dim3(r.ngroups, batch), kThreads, r.fin_global ? 0 : r.smem_finish, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gen_locate<<<dim3((r.B * r.t + kThreads - 1) / kThreads, batch), kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const uint32_t E = r.est_global ? 1u : (r.B + kThreads - 1) / kThreads;
    k_gen_estimate<<<dim3(E, batch), kThreads, r.est_global ? 0 : r.smem_estimate, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_locate_votes(const VoteArgs& a, cudaStream_t st) {
    k_locate_votes<<<1, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_estimate_from_bins(const EstArgs& a, cudaStream_t st) {
    const size_t smem = est_layout(a.nL > 0 ? a.nL : 1, a.kprime > 0 ? a.kprime : 1, 1).total;
    cudaError_t e = general_set_smem(0, 0, 0, smem);
    if (e != cudaSuccess) return e;
    k_estimate_from_bins<<<1, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sfft
