// sfft_exact.cu -- the exact-mode sparse FFT on sm_103a (Algorithm 1 of Hassanieh, Indyk, Katabi,
// Price) for a whole batch of requests.
//
// Work unit: one chunk (by default 2048 consecutive window taps) of one round of one request.  Its
// CTA performs steps 1-2 of HashToBins (proof of Lemma "hashtobins") for all hashings of the round
// (a = 0 and the ladder shifts share one staged run of samples, since x_{sigma(t - beta)} is sample
// t - beta of the sigma-strided sequence): it gathers the permuted samples, applies window and
// modulation, folds them modulo B and stores the partial fold.  The last arrival of a request's round
// (arrival counter, no waiting) sums the partials in chunk order, runs the B-point FFTs (step 3),
// subtracts the recovered coefficients in FP64 (step 4), decodes locations and values
// (NoiselessSparseFFTInner's loop over J) and merges the result into zhat (NoiselessSparseFFT).
//
// k_exact_step runs every round of the batch in one launch: the sample positions of all rounds are
// known up front (sigma, b come from the counter-based draws, never from zhat), so all chunks are
// gathered at once and only the finishers are ordered, round t's by the arrival of round t - 1's.
// k_exact_round runs one round (single-hashing entry points and the persistent queue reuse its
// pieces).  Every reduction has a fixed order and no floating-point atomics exist, so results are
// bit-reproducible.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "philox.cuh"
#include "sfft_device.cuh"
#include "sfft_internal.h"

namespace sfft {

template <typename R>
__device__ __forceinline__ const R* taps_of(const ExactArgs& a);
template <>
__device__ __forceinline__ const float* taps_of<float>(const ExactArgs& a) {
    return a.taps32;
}
template <>
__device__ __forceinline__ const double* taps_of<double>(const ExactArgs& a) {
    return a.taps64;
}

// ------------------------------------------------------------------------------------------------
// shared-memory layout of the finishing phase
// ------------------------------------------------------------------------------------------------
struct FinLayout {
    size_t U, ent_idx, ent_bin, ent_val, ent_gain, ent_sub, ent_sub_f, bin_cnt, bin_start, bin_list, cand_idx, cand_bin, cand_gain,
        cand_val, srt_idx, srt_val, out_idx, out_val, keep, scan;
    size_t total;
};
__host__ __device__ inline size_t fin_take(size_t* off, size_t bytes) {
    const size_t o = (*off + 15) & ~size_t(15);
    *off = o + bytes;
    return o;
}
__host__ __device__ inline FinLayout fin_layout(uint32_t B, uint32_t H, uint32_t zcap, uint32_t csize) {
    FinLayout L;
    size_t off = 0;
    L.U = fin_take(&off, (size_t)H * B * csize);
    L.ent_idx = fin_take(&off, (size_t)zcap * 4);
    L.ent_bin = fin_take(&off, (size_t)zcap * 4);
    L.ent_val = fin_take(&off, (size_t)zcap * 16);
    L.ent_gain = fin_take(&off, (size_t)zcap * 8);
    L.ent_sub = fin_take(&off, (size_t)zcap * H * 16);
    L.ent_sub_f = fin_take(&off, (size_t)zcap * H * 8);
    L.bin_cnt = fin_take(&off, (size_t)(B + 1) * 4);
    L.bin_start = fin_take(&off, (size_t)(B + 1) * 4);
    L.bin_list = fin_take(&off, (size_t)zcap * 4);
    L.cand_idx = fin_take(&off, (size_t)B * 4);
    L.cand_bin = fin_take(&off, (size_t)B * 4);
    L.cand_gain = fin_take(&off, (size_t)B * 8);
    L.cand_val = fin_take(&off, (size_t)B * 16);
    L.srt_idx = fin_take(&off, (size_t)B * 4);
    L.srt_val = fin_take(&off, (size_t)B * 16);
    L.out_idx = fin_take(&off, (size_t)(zcap + B) * 4);
    L.out_val = fin_take(&off, (size_t)(zcap + B) * 16);
    L.keep = fin_take(&off, (size_t)(zcap + B) * 4);
    L.scan = fin_take(&off, (size_t)(kThreads + 8) * 4);
    L.total = off;
    return L;
}

size_t exact_finish_smem(uint32_t B, uint32_t H, uint32_t zcap, bool fp64) {
    return fin_layout(B, H, zcap, fp64 ? 16 : 8).total;
}
size_t exact_gather_smem(uint32_t stage, bool fp64) { return (size_t)stage * (fp64 ? 16 : 8); }

// ------------------------------------------------------------------------------------------------
// Location and estimation of one bin (NoiselessSparseFFTInner's loop body)
// ------------------------------------------------------------------------------------------------
struct DecodeCtx {
    uint32_t n, nmask, B, Np, logNp, H;
    uint32_t sigma, sigma_inv, b, sb;
    uint32_t shift[kMaxHash];  // ladder shifts beta_l (hashing l + 1)
    uint32_t logR[kMaxHash];   // log2(beta_l / B)
    const double* wtab;
    const double* winv;        // 1 / W(o) beside wtab, or null
    double thr, iso_tol, gmin, ref_lo, ref_hi, ref_tol;
    // the same thresholds for the FP32 decisions (ref_lo_f, ref_hi_f already scaled by thr)
    float thr_f, iso_tol_f, ref_lo_f, ref_hi_f, ref_tol_f, inv_n_f;
};

// bin j = round(p / Np) mod B of permuted position p, and the offset o = p - j Np in (-Np/2, Np/2]
__device__ __forceinline__ int32_t offset_of(uint32_t p, uint32_t Np, uint32_t logNp, uint32_t nmask, uint32_t* jbin) {
    const uint32_t jj = ((p + (Np >> 1)) & nmask) >> logNp;
    const uint32_t dd = (p - jj * Np) & nmask;
    *jbin = jj;
    return dd > (nmask >> 1) ? (int32_t)((int64_t)dd - (int64_t)nmask - 1) : (int32_t)dd;
}
__device__ __forceinline__ int32_t offset_of(uint32_t p, const DecodeCtx& d, uint32_t* jbin) {
    return offset_of(p, d.Np, d.logNp, d.nmask, jbin);
}

// the index part of the decode context: sizes, the hashing (sigma, sigma^-1, b) and the ladder
__device__ void fill_ctx_index(DecodeCtx& d, uint64_t n, uint32_t nmask, uint32_t B, uint32_t logB, uint32_t H,
                               const uint64_t* ladder, uint32_t sigma, uint32_t b) {
    d.n = (uint32_t)n;
    d.nmask = nmask;
    d.B = B;
    d.Np = (uint32_t)(n >> logB);
    d.logNp = ilog2_u32(d.Np);
    d.H = H;
    d.sigma = sigma;
    d.sigma_inv = inverse_odd(sigma) & nmask;
    d.b = b;
    d.sb = (sigma * b) & nmask;
    for (int l = 0; l < kMaxHash; ++l) {
        d.shift[l] = (uint32_t)ladder[l];
        d.logR[l] = ladder[l] >= B ? ilog2_u32((uint32_t)(ladder[l] / B)) : 0u;
    }
    d.inv_n_f = __int_as_float((127 - (int)ilog2_u32(d.n)) << 23);  // 2^-log2 n, exact
}

// decode context of a caller-bins decode: thresholds rounded to FP32 here, values divided by W(o)
__device__ void fill_ctx(DecodeCtx& d, uint64_t n, uint32_t nmask, uint32_t B, uint32_t logB, uint32_t H,
                         const uint64_t* ladder, uint32_t sigma, uint32_t b, const double* wtab, double thr,
                         double iso_tol, double gmin, double ref_lo, double ref_hi, double ref_tol) {
    fill_ctx_index(d, n, nmask, B, logB, H, ladder, sigma, b);
    d.wtab = wtab;
    d.winv = nullptr;
    d.thr = thr;
    d.iso_tol = iso_tol;
    d.gmin = gmin;
    d.ref_lo = ref_lo;
    d.ref_hi = ref_hi;
    d.ref_tol = ref_tol;
    d.thr_f = (float)thr;
    d.iso_tol_f = (float)iso_tol;
    d.ref_lo_f = (float)(ref_lo * thr);
    d.ref_hi_f = (float)(ref_hi * thr);
    d.ref_tol_f = (float)ref_tol;
}

// decode context of a round of the transform: the round block carries the FP32 thresholds (rounded
// on the host, so that no FP64 conversion runs here) and the table of 1 / W(o)
__device__ void fill_ctx_round(DecodeCtx& d, const ExactArgs& a, uint32_t sigma, uint32_t b) {
    uint64_t ladder[kMaxHash];
    for (int l = 0; l < kMaxHash; ++l) ladder[l] = l + 1 < kMaxHash ? a.shift64[l + 1] : 0;
    fill_ctx_index(d, a.n, a.nmask, a.B, a.logB, a.H, ladder, sigma, b);
    d.wtab = a.wtab;
    d.winv = a.winv;
    d.thr = a.thr;
    d.iso_tol = a.iso_tol;
    d.gmin = a.gmin;
    d.ref_lo = a.ref_lo;
    d.ref_hi = a.ref_hi;
    d.ref_tol = a.ref_tol;
    d.thr_f = a.thr_f;
    d.iso_tol_f = a.iso_tol_f;
    d.ref_lo_f = a.ref_lo_f;
    d.ref_hi_f = a.ref_hi_f;
    d.ref_tol_f = a.ref_tol_f;
}

// Decode of one bin (NoiselessSparseFFTInner's loop body).  u[0..H) are the bin's hashings after the
// subtraction of zhat, in the precision R of the data path.  Returns 0 (nothing), 1 (a decode of J
// kept) or 2 (a re-estimate of a known entry), with the index in *oi and the window gain that divides
// u_0 in *gain (the caller forms the FP64 value; for a decode of the FP32 path *ginv is 1 / gain from
// the table beside W, else 0, and the caller divides).  *above is set when |u_0| > thr.  The zhat entries
// hashed to bin j are list[0..nbin) (entry ids), with indices ent_idx[] and window gains ent_gain[].
//
// The FP64 data path decides in FP64.  The FP32 path takes every decision (magnitudes, phases, the
// location ladder, isolation and re-estimation tests) in FP32: its bins carry ~1e-6 of rounding, the
// ladder keeps a tolerance of at least tau_dec per level and GB300 issues FP64 at 1/64 of FP32, so FP64
// arithmetic there would cost most of the finisher's time and change no decision outside a
// measure-zero band at the thresholds.
__device__ int decode_bin_fp64(const DecodeCtx& d, uint32_t j, const double2* u, const uint32_t* list, uint32_t nbin,
                               const uint32_t* ent_idx, const double* ent_gain, uint32_t* oi, double* gout,
                               double* ginv, bool* above) {
    const double mag0 = cmag<double>(u[0]);
    *ginv = 0.0;  // the FP64 path divides
    const uint32_t L = d.H - 1;
    *above = false;
    if (!(mag0 > d.thr)) {
        // re-estimation of a known value: exactly one entry of the bin must explain the residual
        if (nbin == 0 || !(mag0 > d.ref_lo * d.thr && mag0 <= d.ref_hi * d.thr)) return 0;
        double th[kMaxHash];
        for (uint32_t l = 0; l < L; ++l) {
            if (fabs(cmag<double>(u[l + 1]) - mag0) > 0.25 * mag0) return 0;
            th[l] = phase01<double>(mul_conj(u[0], u[l + 1]));
        }
        uint32_t matches = 0, who = 0;
        double gw = 1.0;
        for (uint32_t x = 0; x < nbin; ++x) {
            const uint32_t e = list[x];
            const uint32_t i = ent_idx[e];
            const double gain = ent_gain[e];
            if (!(gain >= d.gmin)) continue;
            bool ok = true;
            for (uint32_t l = 0; l < L && ok; ++l) {
                const uint32_t ph = (d.shift[l] * d.sigma * i) & d.nmask;
                double dist = fabs(th[l] - (double)ph / (double)d.n);
                if (dist > 0.5) dist = 1.0 - dist;
                ok = dist * 6.283185307179586476925286766559 < d.ref_tol;
            }
            if (ok) {
                ++matches;
                who = i;
                gw = gain;
            }
        }
        if (matches != 1) return 0;
        *oi = who;
        *gout = gw;
        return 2;
    }
    *above = true;
    // location ladder, coarsest shift first: q = sigma i mod n/B.  Every modulus is a power of two,
    // so mod and division are masks and exact scalings.
    uint32_t logM = d.logNp - d.logR[L - 1];
    const double th = phase01<double>(mul_conj(u[0], u[L]));
    uint64_t c = (uint64_t)(int64_t)floor(th * ldexp(1.0, (int)logM) + 0.5) & ((uint64_t(1) << logM) - 1);
    for (int l = (int)L - 2; l >= 0; --l) {
        const uint32_t logMp = d.logNp - d.logR[l];
        const uint32_t logRatio = logMp - logM;
        const double thl = phase01<double>(mul_conj(u[0], u[l + 1]));
        const double y = thl * ldexp(1.0, (int)logRatio) - ldexp((double)c, -(int)logM);
        const int64_t h = (int64_t)floor(y + 0.5) & (int64_t)((uint64_t(1) << logRatio) - 1);
        c += (uint64_t(1) << logM) * (uint64_t)h;
        logM = logMp;
    }
    const uint32_t q = (uint32_t)c;
    const uint32_t dd = (q + d.Np - (d.sb & (d.Np - 1)) + (d.Np >> 1)) & (d.Np - 1);
    const int32_t o = (int32_t)dd - (int32_t)(d.Np >> 1);
    const uint32_t p = (j * d.Np + (uint32_t)o) & d.nmask;
    const uint32_t si = (p + d.sb) & d.nmask;
    const uint32_t i = (d.sigma_inv * si) & d.nmask;
    for (uint32_t l = 0; l < L; ++l)
        if (fabs(cmag<double>(u[l + 1]) - mag0) > d.iso_tol * mag0) return 0;
    const double gain = d.wtab[o < 0 ? -o : o];
    if (!(gain >= d.gmin)) return 0;
    *oi = i;
    *gout = gain;
    return 1;
}

__device__ __forceinline__ float2 mul_conj_f(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// phase(z) / 2 pi in [0, 1)
__device__ __forceinline__ float phase01_f(float2 z) {
    float p = atan2f(z.y, z.x) * 0.159154943091895336f;
    if (p < 0.0f) p += 1.0f;
    if (p >= 1.0f) p -= 1.0f;
    return p;
}
__device__ __forceinline__ float pow2_f(int e) { return __int_as_float((127 + e) << 23); }  // 2^e, |e| < 127

// Every loop over hashings is unrolled to kMaxHash with compile-time indices, so u[] and the
// phases stay in registers.
__device__ __forceinline__ int decode_bin_fp32(const DecodeCtx& d, uint32_t j, const float2* u, const uint32_t* list,
                                               uint32_t nbin, const uint32_t* ent_idx, const double* ent_gain,
                                               uint32_t* oi, double* gout, double* ginv, bool* above) {
    const float mag0 = hypotf(u[0].x, u[0].y);
    *ginv = 0.0;
    const uint32_t L = d.H - 1;
    *above = false;
    if (!(mag0 > d.thr_f)) {
        // re-estimation of a known value: exactly one entry of the bin must explain the residual
        if (nbin == 0 || !(mag0 > d.ref_lo_f && mag0 <= d.ref_hi_f)) return 0;
        float th[kMaxHash - 1];
#pragma unroll
        for (int l = 0; l < kMaxHash - 1; ++l) {
            th[l] = 0.0f;
            if ((uint32_t)l < L) {
                if (fabsf(hypotf(u[l + 1].x, u[l + 1].y) - mag0) > 0.25f * mag0) return 0;
                th[l] = phase01_f(mul_conj_f(u[0], u[l + 1]));
            }
        }
        uint32_t matches = 0, who = 0;
        double gw = 1.0;
        for (uint32_t x = 0; x < nbin; ++x) {
            const uint32_t e = list[x];
            const uint32_t i = ent_idx[e];
            const double gain = ent_gain[e];
            if (!(gain >= d.gmin)) continue;
            bool ok = true;
#pragma unroll
            for (int l = 0; l < kMaxHash - 1; ++l) {
                if ((uint32_t)l < L && ok) {
                    const uint32_t ph = (d.shift[l] * d.sigma * i) & d.nmask;
                    float dist = fabsf(th[l] - (float)ph * d.inv_n_f);
                    if (dist > 0.5f) dist = 1.0f - dist;
                    ok = dist * 6.28318530717958648f < d.ref_tol_f;
                }
            }
            if (ok) {
                ++matches;
                who = i;
                gw = gain;
            }
        }
        if (matches != 1) return 0;
        *oi = who;
        *gout = gw;
        return 2;
    }
    *above = true;
    // location ladder, coarsest shift first (as decode_bin_fp64).  Products with powers of two are
    // exact; c < 2^logM <= 2^30 and every rounded quantity fits 32 bits, so the conversions are the
    // 32-bit ones.
    float2 uL = u[1];
    uint32_t logRL = d.logR[0];
#pragma unroll
    for (int l = 2; l < kMaxHash; ++l)
        if ((uint32_t)l == L) {
            uL = u[l];
            logRL = d.logR[l - 1];
        }
    uint32_t logM = d.logNp - logRL;
    const float th = phase01_f(mul_conj_f(u[0], uL));
    uint32_t c = (uint32_t)__float2int_rd(th * pow2_f((int)logM) + 0.5f) & ((1u << logM) - 1u);
#pragma unroll
    for (int l = kMaxHash - 3; l >= 0; --l) {
        if (l > (int)L - 2) continue;
        const uint32_t logMp = d.logNp - d.logR[l];
        const uint32_t logRatio = logMp - logM;
        const float thl = phase01_f(mul_conj_f(u[0], u[l + 1]));
        const float y = thl * pow2_f((int)logRatio) - __uint2float_rn(c) * pow2_f(-(int)logM);
        const uint32_t h = (uint32_t)__float2int_rd(y + 0.5f) & ((1u << logRatio) - 1u);
        c += h << logM;
        logM = logMp;
    }
    const uint32_t q = c;
    const uint32_t dd = (q + d.Np - (d.sb & (d.Np - 1)) + (d.Np >> 1)) & (d.Np - 1);
    const int32_t o = (int32_t)dd - (int32_t)(d.Np >> 1);
    const uint32_t p = (j * d.Np + (uint32_t)o) & d.nmask;
    const uint32_t si = (p + d.sb) & d.nmask;
    const uint32_t i = (d.sigma_inv * si) & d.nmask;
#pragma unroll
    for (int l = 0; l < kMaxHash - 1; ++l)
        if ((uint32_t)l < L && fabsf(hypotf(u[l + 1].x, u[l + 1].y) - mag0) > d.iso_tol_f * mag0) return 0;
    const uint32_t oa = (uint32_t)(o < 0 ? -o : o);
    const double gain = d.wtab[oa];
    const double gi = d.winv ? d.winv[oa] : 0.0;  // loaded beside the gain: one memory latency for both
    if (!(gain >= d.gmin)) return 0;
    *oi = i;
    *gout = gain;
    *ginv = gi;
    return 1;
}

__device__ __forceinline__ int decode_bin(const DecodeCtx& d, uint32_t j, const double2* u, const uint32_t* list,
                                          uint32_t nbin, const uint32_t* ent_idx, const double* ent_gain, uint32_t* oi,
                                          double* gout, double* ginv, bool* above) {
    return decode_bin_fp64(d, j, u, list, nbin, ent_idx, ent_gain, oi, gout, ginv, above);
}
__device__ __forceinline__ int decode_bin(const DecodeCtx& d, uint32_t j, const float2* u, const uint32_t* list,
                                          uint32_t nbin, const uint32_t* ent_idx, const double* ent_gain, uint32_t* oi,
                                          double* gout, double* ginv, bool* above) {
    return decode_bin_fp32(d, j, u, list, nbin, ent_idx, ent_gain, oi, gout, ginv, above);
}

// Bin j's hashings after the subtraction of zhat, for the decisions: u_h = U_h - sum over the bin's
// entries e (in list order) of sub[e H + h], in the data path's precision (FP64 terms and sums for
// the FP64 path; the terms rounded to FP32 and summed in FP32 for the FP32 path, whose bins carry
// ~1e-6 of rounding).  The values of decoded bins are formed separately from subtracted_u0 in FP64.
__device__ __forceinline__ void subtracted_bin(const double2* U, uint32_t B, uint32_t H, uint32_t j,
                                               const uint32_t* list, uint32_t nbin, const double2* sub,
                                               const float2* /*sub_f*/, double2* u) {
    for (uint32_t h = 0; h < H; ++h) {
        double2 w = U[h * B + j];
        for (uint32_t x = 0; x < nbin; ++x) {
            const uint32_t e = list[x];
            w.x -= sub[e * H + h].x;
            w.y -= sub[e * H + h].y;
        }
        u[h] = w;
    }
}
__device__ __forceinline__ void subtracted_bin(const float2* U, uint32_t B, uint32_t H, uint32_t j,
                                               const uint32_t* list, uint32_t nbin, const double2* /*sub*/,
                                               const float2* sub_f, float2* u) {
#pragma unroll
    for (int h = 0; h < kMaxHash; ++h) u[h] = (uint32_t)h < H ? U[h * B + j] : make_float2(0.0f, 0.0f);
    for (uint32_t x = 0; x < nbin; ++x) {
        const float2* t = sub_f + list[x] * H;
#pragma unroll
        for (int h = 0; h < kMaxHash; ++h)
            if ((uint32_t)h < H) {
                u[h].x -= t[h].x;
                u[h].y -= t[h].y;
            }
    }
}
// u_0 of bin j after the subtraction, in FP64 (the first row of subtracted_bin, same order); entry e's
// FP64 term of hashing 0 is sub[e * stride]
template <typename C>
__device__ __forceinline__ double2 subtracted_u0(const C* U, uint32_t stride, uint32_t j, const uint32_t* list,
                                                 uint32_t nbin, const double2* sub) {
    const C v = U[j];
    double2 w = make_double2((double)v.x, (double)v.y);
    for (uint32_t x = 0; x < nbin; ++x) {
        const uint32_t e = list[x];
        w.x -= sub[e * stride].x;
        w.y -= sub[e * stride].y;
    }
    return w;
}

// ------------------------------------------------------------------------------------------------
// The round kernel
// ------------------------------------------------------------------------------------------------
template <typename R>
__device__ void gather_fold(const ExactArgs& a, const void* xrow, uint32_t xmask, uint32_t s, uint32_t c,
                            uint32_t sigma, uint32_t b, unsigned char* smem) {
    using C = typename Cx<R>::T;
    C* stage = reinterpret_cast<C*>(smem);
    C* red = stage + a.stage;
    const uint32_t tid = threadIdx.x;
    const C* __restrict__ x = reinterpret_cast<const C*>(xrow);
    const R* __restrict__ taps = taps_of<R>(a);
    const int64_t t_lo = -a.T + (int64_t)c * a.ctaps;
    const int64_t t_hi = min(t_lo + (int64_t)a.ctaps, a.T + 1);
    const uint32_t ntap = (uint32_t)(t_hi - t_lo);
    const int32_t base = (int32_t)(t_lo - (int64_t)a.a_base - (int64_t)a.maxshift);  // sample held by stage[0]
    const uint32_t cnt = ntap + a.maxshift;
    // step 1a: gather the sigma-strided samples x_{sigma s}, s in [base, base + cnt) (12 loads in flight)
#ifndef SFFT_GATHER_IN_FLIGHT
#define SFFT_GATHER_IN_FLIGHT 12
#endif
    constexpr int kInFlight = SFFT_GATHER_IN_FLIGHT;
    for (uint32_t i0 = tid; i0 < cnt; i0 += kThreads * kInFlight) {
        C v[kInFlight];
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            const uint32_t i = i0 + (uint32_t)q * kThreads;
            if (i < cnt) v[q] = ldg_c(x + ((sigma * (uint32_t)(base + (int32_t)i)) & xmask));
        }
#pragma unroll
        for (int q = 0; q < kInFlight; ++q) {
            const uint32_t i = i0 + (uint32_t)q * kThreads;
            if (i < cnt) stage[i] = v[q];
        }
    }
    const bool big = a.B > (uint32_t)kThreads;
    if (big)
        for (uint32_t i = tid; i < a.H * a.B; i += kThreads) red[i] = mkc((R)0, (R)0);
    __syncthreads();
    // step 1b + 2: y_t = G_t x_{sigma (t - a_h)} w^{sigma b t}, folded mod B
    C acc[kMaxHash];
#pragma unroll
    for (int h = 0; h < kMaxHash; ++h) acc[h] = mkc((R)0, (R)0);
    const uint32_t sb = sigma * b;
    const R inv_half_n = (R)2 / (R)a.n;
    for (uint32_t k = tid; k < ntap; k += kThreads) {
        const int32_t t = (int32_t)t_lo + (int32_t)k;
        const R g = taps[t < 0 ? -t : t];
        const uint32_t e = (sb * (uint32_t)t) & a.nmask;
        const int32_t es = e > (a.nmask >> 1) ? (int32_t)((int64_t)e - (int64_t)a.n) : (int32_t)e;
        R sn, cs;
        sincospi_r((R)es * inv_half_n, &sn, &cs);
        const C gt = mkc(g * cs, -g * sn);
        const uint32_t si = k + a.maxshift;
        if (!big) {
#pragma unroll
            for (int h = 0; h < kMaxHash; ++h)
                if ((uint32_t)h < a.H) acc[h] = cfma(gt, stage[si - a.a[h]], acc[h]);
        } else {
            const uint32_t r = (uint32_t)t & (a.B - 1);
            for (uint32_t h = 0; h < a.H; ++h) red[h * a.B + r] = cfma(gt, stage[si - a.a[h]], red[h * a.B + r]);
        }
    }
    if (!big) {
        for (uint32_t h = 0; h < a.H; ++h) red[h * kThreads + tid] = acc[h];
    }
    __syncthreads();
    C* part = reinterpret_cast<C*>(a.part) + (size_t)s * a.part_stride + (size_t)c * a.H * a.B;
    if (!big) {
        // residue of thread tid is (t_lo + tid) mod B; the threads of residue r are owner + m B
        for (uint32_t r = tid; r < a.B; r += kThreads) {
            const uint32_t owner = (r - (uint32_t)t_lo) & (a.B - 1);
            for (uint32_t h = 0; h < a.H; ++h) {
                C sum = mkc((R)0, (R)0);
                for (uint32_t m = owner; m < (uint32_t)kThreads; m += a.B) sum = cadd(sum, red[h * kThreads + m]);
                part[h * a.B + r] = sum;
            }
        }
    } else {
        for (uint32_t i = tid; i < a.H * a.B; i += kThreads) part[i] = red[i];
    }
}

// Step 2 across chunks: U[h][brev(r)] = sum over chunks c, in order, of part[c][h][r].  Each thread
// takes E elements of up to CM chunks with all their loads in flight at once (CM >= chunks), else
// one element at a time in batches of 16.
template <int E, int CM, typename C>
__device__ __forceinline__ void sum_partials_batched(const C* part, uint32_t chunks, uint32_t H, uint32_t logB, C* U) {
    const uint32_t B = 1u << logB, HB = H * B, shift_br = 32u - logB;
    for (uint32_t i0 = threadIdx.x; i0 < HB; i0 += (uint32_t)kThreads * E) {
        C v[E][CM];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = i0 + (uint32_t)e * kThreads;
            const uint32_t h = i >> logB, r = i & (B - 1);
#pragma unroll
            for (int c = 0; c < CM; ++c)
                if (i < HB && (uint32_t)c < chunks) v[e][c] = __ldcg(part + ((size_t)c * H + h) * B + r);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t i = i0 + (uint32_t)e * kThreads;
            if (i < HB) {
                C sum;
                sum.x = 0;
                sum.y = 0;
#pragma unroll
                for (int c = 0; c < CM; ++c)
                    if ((uint32_t)c < chunks) sum = cadd(sum, v[e][c]);
                U[(i >> logB) * B + (__brev(i & (B - 1)) >> shift_br)] = sum;
            }
        }
    }
}
template <typename C>
__device__ void sum_partials(const C* part, uint32_t chunks, uint32_t H, uint32_t logB, C* U) {
    constexpr bool f32 = sizeof(C) == sizeof(float2);  // FP64 bins: half the loads in flight (registers)
    if (chunks <= 8) {
        sum_partials_batched<f32 ? 2 : 1, 8>(part, chunks, H, logB, U);
    } else if (chunks <= 16) {
        sum_partials_batched<1, 16>(part, chunks, H, logB, U);
    } else {
        const uint32_t B = 1u << logB, shift_br = 32u - logB;
        for (uint32_t i = threadIdx.x; i < H * B; i += kThreads) {
            const uint32_t h = i >> logB, r = i & (B - 1);
            C sum;
            sum.x = 0;
            sum.y = 0;
            for (uint32_t c0 = 0; c0 < chunks; c0 += 16) {  // 16 loads in flight, summed in chunk order
                C v[16];
#pragma unroll
                for (uint32_t q = 0; q < 16; ++q)
                    if (c0 + q < chunks) v[q] = __ldcg(part + ((size_t)(c0 + q) * H + h) * B + r);
#pragma unroll
                for (uint32_t q = 0; q < 16; ++q)
                    if (c0 + q < chunks) sum = cadd(sum, v[q]);
            }
            U[h * B + (__brev(r) >> shift_br)] = sum;
        }
    }
}

// Parts of a round's finisher: the bins (partial folds summed in chunk order, bit-reversed, B-point
// FFT) and the decode (zhat subtraction, location, estimation, merge).  kFinBins leaves the bins in
// the first H B entries of the request's partial-fold area of the round; kFinDecode starts from there.
enum FinPart { kFinBins = 1, kFinDecode = 2, kFinAll = 3 };

template <typename R>
__device__ bool finish_round(const ExactArgs& a, uint32_t s, uint32_t sigma, uint32_t b, unsigned char* smem,
                             int part = kFinAll, bool carry = false, bool bins_here = false,
                             const uint32_t* next_ctr = nullptr) {
    using C = typename Cx<R>::T;
    const uint32_t tid = threadIdx.x;
    const uint32_t B = a.B, H = a.H;
    const FinLayout Ly = fin_layout(B, H, a.zcap, sizeof(C));
    C* U = reinterpret_cast<C*>(smem + Ly.U);
    uint32_t* ent_idx = reinterpret_cast<uint32_t*>(smem + Ly.ent_idx);
    uint32_t* ent_bin = reinterpret_cast<uint32_t*>(smem + Ly.ent_bin);
    double2* ent_val = reinterpret_cast<double2*>(smem + Ly.ent_val);
    double* ent_gain = reinterpret_cast<double*>(smem + Ly.ent_gain);
    double2* ent_sub = reinterpret_cast<double2*>(smem + Ly.ent_sub);
    float2* ent_sub_f = reinterpret_cast<float2*>(smem + Ly.ent_sub_f);
    uint32_t* bin_cnt = reinterpret_cast<uint32_t*>(smem + Ly.bin_cnt);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(smem + Ly.bin_start);
    uint32_t* bin_list = reinterpret_cast<uint32_t*>(smem + Ly.bin_list);
    uint32_t* cand_idx = reinterpret_cast<uint32_t*>(smem + Ly.cand_idx);
    uint32_t* cand_bin = reinterpret_cast<uint32_t*>(smem + Ly.cand_bin);
    double* cand_gain = reinterpret_cast<double*>(smem + Ly.cand_gain);
    double2* cand_val = reinterpret_cast<double2*>(smem + Ly.cand_val);
    uint32_t* srt_idx = reinterpret_cast<uint32_t*>(smem + Ly.srt_idx);
    double2* srt_val = reinterpret_cast<double2*>(smem + Ly.srt_val);
    uint32_t* out_idx = reinterpret_cast<uint32_t*>(smem + Ly.out_idx);
    double2* out_val = reinterpret_cast<double2*>(smem + Ly.out_val);
    uint32_t* keep = reinterpret_cast<uint32_t*>(smem + Ly.keep);
    uint32_t* scan = reinterpret_cast<uint32_t*>(smem + Ly.scan);
    __shared__ uint32_t s_nw, s_above, s_kept;
    C* area = reinterpret_cast<C*>(a.part) + (size_t)s * a.part_stride;  // the round's partial folds

    // steps 2 (across chunks) and 3: partial folds summed in chunk order, bit-reversed, FFT
    if (part & kFinBins) {
        sum_partials(area, a.chunks, H, a.logB, U);
        block_fft_rows<R>(U, H, a.logB);  // starts and ends with a barrier
        if (!(part & kFinDecode)) {  // every partial fold has been read: the area takes the bins
            for (uint32_t i = tid; i < H * B; i += kThreads) area[i] = U[i];
            return false;
        }
    }
    // The round's bins, when another CTA formed them (bins_here: this CTA did, just before, in place),
    // read through L2 only: each thread's first four are loaded here and stored after the entries'
    // window gains below have been requested, so that both wait out one memory latency.  The last
    // thread reads the next round's second counter (next_ctr) with an acquire load alongside: if that
    // round's bins have arrived, the caller goes on to its decode without an arrival (next_ready).
    __shared__ uint32_t s_next_ready;
    const bool load_U = !(part & kFinBins) && !bins_here;
    C uv[4];
    if (load_U) {
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
            if (tid + q * kThreads < H * B) uv[q] = __ldcg(area + tid + q * kThreads);
    }
    if (tid == kThreads - 1 && next_ctr != nullptr) s_next_ready = acquire_is(next_ctr, 1u) ? 1u : 0u;

    // zhat of this request and its per-entry subtraction terms
    // zhat is read through L2 only: in the one-launch path another CTA of this launch wrote it
    // (the first entry of each thread is fetched together with the count)
    // zhat of the previous round stays in this CTA's shared memory (up to kCarry entries) when the
    // previous round's decode of this request ran here (carry): no global load for it then
    __shared__ uint32_t c_idx[kCarry];
    __shared__ double2 c_val[kCarry];
    __shared__ uint32_t c_n;
    const bool use_carry = carry && !a.bins_only && a.zcap <= kCarry;
    const uint32_t zlim = a.bins_only ? a.e_nz : a.zcap;
    uint32_t zi0 = 0;
    double2 zv0 = make_double2(0.0, 0.0);
    if (use_carry) {
        if (tid < c_n) {
            zi0 = c_idx[tid];
            zv0 = c_val[tid];
        }
    } else if (tid < zlim) {
        zi0 = __ldcg(a.zidx + (size_t)s * a.zcap + tid);
        zv0 = __ldcg(a.zval + (size_t)s * a.zcap + tid);
    }
    const uint32_t nz = a.bins_only ? a.e_nz : (use_carry ? c_n : min(__ldcg(a.zcount + s), a.zcap));
    // the decode context is the same for every thread: one copy in shared memory (registers would
    // hold it only by spilling it to local memory)
    __shared__ DecodeCtx d;
    if (tid == kThreads - 2) fill_ctx_round(d, a, sigma, b);
    // (the entries need no part of d: their window gains are read while it is filled, by a thread that
    // holds no entry unless zhat has more than kThreads - 2)
    const uint32_t Np = (uint32_t)(a.n >> a.logB), logNp = ilog2_u32(Np);
    // The FP32 data path keeps FP64 work (issued at a small fraction of the FP32 rate) to the values:
    // entry e's FP64 term of hashing 0 goes to ent_sub[e] and its gain-scaled value, rounded to FP32,
    // to ent_gz[e] (behind the first zcap entries of ent_sub; H >= 2 outside single-hashing mode); the
    // terms of the decisions are formed in FP32 from there.  The FP64 path forms every term in FP64.
    constexpr bool f32 = sizeof(C) == sizeof(float2);
    float2* ent_gz = reinterpret_cast<float2*>(ent_sub + a.zcap);
    const uint32_t a0 = a.a_base + a.a[0];
    for (uint32_t e = tid; e < nz; e += kThreads) {
        const uint32_t i = e == tid ? zi0 : (use_carry ? c_idx[e] : __ldcg(a.zidx + (size_t)s * a.zcap + e));
        const double2 v = e == tid ? zv0 : (use_carry ? c_val[e] : __ldcg(a.zval + (size_t)s * a.zcap + e));
        ent_idx[e] = i;
        ent_val[e] = v;
        uint32_t jb;
        const int32_t o = offset_of((sigma * (i - b)) & a.nmask, Np, logNp, a.nmask, &jb);
        ent_bin[e] = jb;
        const double gain = a.wtab[o < 0 ? -o : o];
        ent_gain[e] = gain;
        if (f32) {
            const double2 gz = make_double2(gain * v.x, gain * v.y);
            double2 t0 = gz;  // hashing 0 has offset 0 in the transform's rounds: w^0 = 1
            const uint32_t e0 = (a0 * sigma * i) & a.nmask;
            if (e0 != 0) {
                const double2 w = root_pow<R>(e0, a.nmask);
                t0 = make_double2(gz.x * w.x - gz.y * w.y, gz.x * w.y + gz.y * w.x);
            }
            ent_sub[e] = t0;
            if (!a.bins_only) ent_gz[e] = make_float2((float)gz.x, (float)gz.y);
        }
    }
    if (load_U) {
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q)
            if (tid + q * kThreads < H * B) U[tid + q * kThreads] = uv[q];
        for (uint32_t i0 = tid + 4 * kThreads; i0 < H * B; i0 += 4 * kThreads) {  // B > kThreads
            C v[4];
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q)
                if (i0 + q * kThreads < H * B) v[q] = __ldcg(area + i0 + q * kThreads);
#pragma unroll
            for (uint32_t q = 0; q < 4; ++q)
                if (i0 + q * kThreads < H * B) U[i0 + q * kThreads] = v[q];
        }
    }
    if (tid == 0) {
        s_nw = 0;
        s_above = 0;
        s_kept = 0;
    }
    __syncthreads();  // d, the entries and the counts
    // read here, before thread 0 can reach the next round's write
    const bool next_ready = next_ctr != nullptr && s_next_ready != 0;
    // step 4 terms: W(-o(i)) zhat_i w^{a_h sigma i} for every (entry, hashing).  No barrier after this
    // loop: bucket_entries starts with one before anything reads the terms.
    if (f32) {
        if (!a.bins_only) {
            const float two_over_n = 2.0f * d.inv_n_f;  // exact: n is a power of two
            for (uint32_t q = tid; q < nz * H; q += kThreads) {
                const uint32_t e = q / H, h = q - e * H;
                const uint32_t ex = ((a.a_base + a.a[h]) * sigma * ent_idx[e]) & a.nmask;
                const int32_t es = ex > (a.nmask >> 1) ? (int32_t)((int64_t)ex - (int64_t)a.n) : (int32_t)ex;
                float sn, cs;
                sincospif((float)es * two_over_n, &sn, &cs);
                const float2 g = ent_gz[e];  // times w = (cs, -sn)
                ent_sub_f[q] = make_float2(g.x * cs + g.y * sn, g.y * cs - g.x * sn);
            }
        }
    } else {
        for (uint32_t q = tid; q < nz * H; q += kThreads) {
            const uint32_t e = q / H, h = q - e * H;
            const uint32_t i = ent_idx[e];
            const double2 w = root_pow<R>(((a.a_base + a.a[h]) * sigma * i) & a.nmask, a.nmask);
            const double2 gz = make_double2(ent_gain[e] * ent_val[e].x, ent_gain[e] * ent_val[e].y);
            const double2 t = make_double2(gz.x * w.x - gz.y * w.y, gz.x * w.y + gz.y * w.x);
            ent_sub[q] = t;
            ent_sub_f[q] = make_float2((float)t.x, (float)t.y);
        }
    }
    const uint32_t sub_stride = f32 ? 1u : H;  // where subtracted_u0 finds hashing 0's FP64 terms
    bucket_entries(ent_bin, nz, B, bin_cnt, bin_start, bin_list, scan);

    if (a.bins_only) {  // single-hashing mode: the subtracted bins u_0 in FP64, no decode
        for (uint32_t j = tid; j < B; j += kThreads)
            a.ubins[j] =
                subtracted_u0(U, sub_stride, j, bin_list + bin_start[j], bin_start[j + 1] - bin_start[j], ent_sub);
        return false;
    }
    // step 4 and the decode, one bin per thread: decisions in the data path's precision
    for (uint32_t j = tid; j < B; j += kThreads) {
        C u[kMaxHash];
        const uint32_t* list = bin_list + bin_start[j];
        const uint32_t nbin = bin_start[j + 1] - bin_start[j];
        subtracted_bin(U, B, H, j, list, nbin, ent_sub, ent_sub_f, u);
        uint32_t oi = 0;
        double gain = 1.0, ginv = 0.0;
        bool above;
        const int kind = decode_bin(d, j, u, list, nbin, ent_idx, ent_gain, &oi, &gain, &ginv, &above);
        // counts and candidate slots, one shared-memory atomic per warp and counter
        const unsigned m = __activemask();
        const unsigned ma = __ballot_sync(m, above), mk = __ballot_sync(m, kind == 1), mw = __ballot_sync(m, kind != 0);
        const uint32_t lane = tid & 31u, leader = (uint32_t)__ffs((int)m) - 1u;
        uint32_t base = 0;
        if (lane == leader) {
            if (ma) atomicAdd(&s_above, (uint32_t)__popc((int)ma));
            if (mk) atomicAdd(&s_kept, (uint32_t)__popc((int)mk));
            if (mw) base = atomicAdd(&s_nw, (uint32_t)__popc((int)mw));
        }
        base = __shfl_sync(m, base, (int)leader);
        if (kind != 0) {
            const uint32_t slot = base + (uint32_t)__popc((int)(mw & ((1u << lane) - 1u)));
            cand_idx[slot] = oi;
            cand_bin[slot] = j;
            cand_gain[slot] = gain;
            // its value: u_0 (step 4 in FP64) / W(-o), as a product with 1 / W(-o) from the table where
            // the decode read one (FP32 path), else as a quotient
            const double2 u0 = subtracted_u0(U, sub_stride, j, list, nbin, ent_sub);
            if (f32 && kind == 1 && d.winv)
                cand_val[slot] = make_double2(u0.x * ginv, u0.y * ginv);
            else
                cand_val[slot] = make_double2(u0.x / gain, u0.y / gain);
        }
    }
    __syncthreads();
    const uint32_t nw = s_nw;

    const bool last = a.last_round != 0;
    if (nw == 0) {
        // nothing decoded: zhat stays as it is (its entries passed the same prune test when merged)
        if (!a.bins_only && a.zcap <= kCarry && !use_carry) {  // this CTA keeps it for the next round
            for (uint32_t e = tid; e < nz; e += kThreads) {
                c_idx[e] = ent_idx[e];
                c_val[e] = ent_val[e];
            }
            if (tid == 0) c_n = nz;
        }
        if (last) {
            for (uint32_t e = tid; e < nz && e < a.out_cap; e += kThreads) {
                a.out_idx[(size_t)s * a.out_cap + e] = ent_idx[e];
                a.out_val[(size_t)s * a.out_cap + e] = ent_val[e];
            }
            if (tid == 0) {
                a.out_count[s] = nz < a.out_cap ? nz : a.out_cap;
                int32_t flag = SFFT_OK;
                if (__ldcg(a.zflag + s) || nz > a.out_cap)
                    flag = SFFT_ERR_CAPACITY;
                else if (s_above > s_kept)
                    flag = SFFT_ERR_NOT_CONVERGED;
                a.out_flag[s] = flag;
            }
        }
        return next_ready;
    }
    // merge what into zhat (NoiselessSparseFFT: zhat <- zhat + what), zhat first on equal indices,
    // then drop entries below prune * thr
    const uint32_t tot = nz + nw;
    if (nw <= (uint32_t)kThreads) {
        // positions by counting (the candidates' indices are distinct): zhat entry e goes to e + the
        // number of candidates below its index, candidate c to the number of candidates below its
        // index + the number of zhat entries at or below it
        for (uint32_t e = tid; e < nz; e += kThreads) {
            const uint32_t key = ent_idx[e];
            uint32_t r = 0;
            for (uint32_t q = 0; q < nw; ++q) r += cand_idx[q] < key ? 1u : 0u;
            out_idx[e + r] = key;
            out_val[e + r] = ent_val[e];
        }
        if (tid < nw) {
            const uint32_t key = cand_idx[tid];
            uint32_t r = 0;
            for (uint32_t q = 0; q < nw; ++q) r += cand_idx[q] < key ? 1u : 0u;
            const uint32_t pos = r + upper_bound_u32(ent_idx, nz, key);
            out_idx[pos] = key;
            out_val[pos] = cand_val[tid];
        }
    } else {  // many candidates: sorted first, then placed by binary searches
        rank_sort(cand_idx, cand_val, nw, srt_idx, srt_val);
        for (uint32_t e = tid; e < nz; e += kThreads) {
            const uint32_t pos = e + lower_bound_u32(srt_idx, nw, ent_idx[e]);
            out_idx[pos] = ent_idx[e];
            out_val[pos] = ent_val[e];
        }
        for (uint32_t c = tid; c < nw; c += kThreads) {
            const uint32_t pos = c + upper_bound_u32(ent_idx, nz, srt_idx[c]);
            out_idx[pos] = srt_idx[c];
            out_val[pos] = srt_val[c];
        }
    }
    __syncthreads();
    for (uint32_t p = tid; p < tot; p += kThreads) {
        uint32_t kp = 0;
        const uint32_t idx = out_idx[p];
        if (p == 0 || out_idx[p - 1] != idx) {
            double2 v = out_val[p];
            if (p + 1 < tot && out_idx[p + 1] == idx) {
                v.x += out_val[p + 1].x;
                v.y += out_val[p + 1].y;
                out_val[p] = v;  // the duplicate at p + 1 is never a head and is not written
            }
            // |v| < prune thr, in the data path's precision (FP32: against prune thr rounded up)
            if (f32)
                kp = hypotf((float)v.x, (float)v.y) < a.drop_f ? 0u : 1u;
            else
                kp = cmag<R>(v) < a.prune * a.thr ? 0u : 1u;
        }
        keep[p] = kp;
    }
    __syncthreads();
    const uint32_t newcount =
        tot <= (uint32_t)kThreads ? block_exclusive_scan_flags(keep, tot, scan) : block_exclusive_scan(keep, tot, scan);
    uint32_t* zi = a.zidx + (size_t)s * a.zcap;
    double2* zv = a.zval + (size_t)s * a.zcap;
    for (uint32_t p = tid; p < tot; p += kThreads) {
        const uint32_t pos = keep[p];  // exclusive prefix of the keep flags: kept iff the next differs
        const uint32_t nxt = p + 1 < tot ? keep[p + 1] : newcount;
        if (nxt == pos) continue;
        const uint32_t idx = out_idx[p];
        const double2 v = out_val[p];
        if (pos < a.zcap) {
            zi[pos] = idx;
            zv[pos] = v;
            if (a.zcap <= kCarry) {
                c_idx[pos] = idx;
                c_val[pos] = v;
            }
        }
        if (last && pos < a.out_cap) {
            a.out_idx[(size_t)s * a.out_cap + pos] = idx;
            a.out_val[(size_t)s * a.out_cap + pos] = v;
        }
    }
    if (tid == 0) {
        const bool overflow = newcount > a.zcap;
        if (overflow) a.zflag[s] = 1;
        a.zcount[s] = overflow ? a.zcap : newcount;
        c_n = overflow ? a.zcap : newcount;
        if (last) {
            const uint32_t kept_count = overflow ? a.zcap : newcount;
            a.out_count[s] = kept_count < a.out_cap ? kept_count : a.out_cap;
            int32_t flag = SFFT_OK;
            if (__ldcg(a.zflag + s) || kept_count > a.out_cap)
                flag = SFFT_ERR_CAPACITY;
            else if (s_above > s_kept)
                flag = SFFT_ERR_NOT_CONVERGED;
            a.out_flag[s] = flag;
        }
    }
    return next_ready;
}

#ifndef SFFT_ROUND_MIN_BLOCKS
#define SFFT_ROUND_MIN_BLOCKS 2  // resident CTAs per SM the register budget is sized for
#endif

template <typename R>
__global__ void __launch_bounds__(kThreads, SFFT_ROUND_MIN_BLOCKS) k_exact_round(const ExactArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = a.req_base + blockIdx.y, c = blockIdx.x;
    const ReqView rq = req_view(a.reqs, a.x, a.n * sizeof(typename Cx<R>::T), a.seed, s, a.nmask);
    uint32_t sigma, b;
    if (a.bins_only) {
        sigma = a.e_sigma;
        b = a.e_b;
    } else {
        exact_hash(rq.seed, rq.id, a.round, a.nmask, &sigma, &b);
    }
    gather_fold<R>(a, rq.x, rq.xmask, s, c, sigma, b, smem);
    // arrival: the last CTA of request s finishes the round (nobody waits)
    if (arrive(a.counter + s, a.chunks) == 0) return;
    finish_round<R>(a, s, sigma, b, a.fin_scratch ? a.fin_scratch + (size_t)s * a.fin_stride : smem);
    if (threadIdx.x == 0) a.counter[s] = 0;
}

// ------------------------------------------------------------------------------------------------
// One launch per batch: all rounds' chunks, finishers chained by arrival counters
// ------------------------------------------------------------------------------------------------
// The decodes of request s from round t on, in this CTA, for as long as the next round's bins have
// arrived.  Round t > 0's decode is the second of two arrivals at its counter2 (its bins, round t - 1's
// decode); round 0's needs no zhat and follows its bins here.  Each decode also reads the next round's
// counter2 (an acquire load that overlaps its own loads): when those bins have arrived, this chain is
// the last party of that round and goes on without an arrival of its own.  (seed, id) name the
// request's draws.
template <typename R, int NR>
__device__ __forceinline__ void decode_chain(const StepParams<NR>& sp, uint32_t t, const ExactArgs* a, uint32_t s,
                                             uint64_t seed, uint32_t id, uint32_t sigma, uint32_t b,
                                             unsigned char* smem) {
    if (t > 0 && arrive_pair(a->counter2 + s) == 0) return;
    bool bins_here = a->fin_scratch == nullptr;  // the bins just formed are in this CTA's shared memory
    for (bool carried = false;; carried = true) {
        const uint32_t* next_ctr = t + 1 < sp.R ? sp.r[t + 1].counter2 + s : nullptr;
        const bool next_ready =
            finish_round<R>(*a, s, sigma, b, a->fin_scratch ? a->fin_scratch + (size_t)s * a->fin_stride : smem,
                            kFinDecode, carried, bins_here, next_ctr);
        if (threadIdx.x == 0) a->counter2[s] = 0;  // both arrivals of round t have happened (or none, t = 0)
        if (t + 1 >= sp.R) break;
        a = &sp.r[++t];
        bins_here = false;
        // zhat of round t - 1 is published by the arrival at round t's second counter (which also
        // orders this round's shared-memory writes, the kept zhat among them, before the next reads)
        if (next_ready)
            __syncthreads();
        else if (arrive_pair(a->counter2 + s) == 0)
            break;
        exact_hash(seed, id, t, a->nmask, &sigma, &b);
    }
}

template <typename R, int NR>
__global__ void __launch_bounds__(kThreads, SFFT_ROUND_MIN_BLOCKS) k_exact_step(const __grid_constant__ StepParams<NR> sp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t tid = threadIdx.x;
    uint32_t t = 0;
    while (t + 1 < sp.R && blockIdx.x >= sp.seg[t + 1]) ++t;
    const ExactArgs* a = &sp.r[t];
    const uint32_t local = blockIdx.x - sp.seg[t];
    const uint32_t c = local % a->chunks;
    const uint32_t s = a->req_base + local / a->chunks;
    const ReqView rq = req_view(a->reqs, a->x, a->n * sizeof(typename Cx<R>::T), a->seed, s, a->nmask);
    uint32_t sigma, b;
    exact_hash(rq.seed, rq.id, t, a->nmask, &sigma, &b);
    gather_fold<R>(*a, rq.x, rq.xmask, s, c, sigma, b, smem);
    if (arrive(a->counter + s, a->chunks) == 0) return;
    // the round's bins, in this CTA's shared memory (the gather's staging area holds H B values)
    finish_round<R>(*a, s, sigma, b, smem, kFinBins);
    if (tid == 0) a->counter[s] = 0;  // every chunk of round t has arrived
    decode_chain<R, NR>(sp, t, a, s, rq.seed, rq.id, sigma, b, smem);
}

// ------------------------------------------------------------------------------------------------
// Multi-channel batches with shared hashing (see ChanParams)
// ------------------------------------------------------------------------------------------------
// Gather and fold: CTA (t, rho, c) sums, for each hashing h of round t and every channel, the terms
// G_{s + a_h} w^{sigma b (s + a_h)} x_{sigma s} over the samples s = s0 + i, i = rho' + j B (rho' the
// first index of residue class rho), j in chunk c: bin rho of hashing h.  Warp 0 issues one bulk copy
// per row (C contiguous complex values) into shared memory, then forms the rows' coefficients (one
// row per lane) while the copies are in flight; once they have landed, thread ch folds channel ch in
// row order.
constexpr uint32_t kChanWaitLimit = 1u << 22;  // tries of a bounded wait (far beyond a second)
template <int NR>
__global__ void __launch_bounds__(kThreads) k_chan_gather(const __grid_constant__ ChanParams<NR> cp) {
    extern __shared__ __align__(16) unsigned char smem[];  // bulk copies need 16-byte alignment
    __shared__ __align__(8) uint64_t bar;
    const uint32_t C = cp.C, tid = threadIdx.x;
    float2* rows = reinterpret_cast<float2*>(smem);                                       // [kChanRows][C]
    float2* coef = reinterpret_cast<float2*>(smem + (size_t)kChanRows * C * sizeof(float2));  // [kChanRows][kMaxHash]
    uint32_t t = 0;
    while (t + 1 < cp.R && blockIdx.x >= cp.cseg[t + 1]) ++t;
    const ExactArgs& a = cp.r[t];
    const uint32_t local = blockIdx.x - cp.cseg[t];
    const uint32_t rho = local & (a.B - 1), c = local / a.B;
    const int64_t s0 = -a.T - (int64_t)a.maxshift;
    const uint32_t cnt = (uint32_t)(2 * a.T + 1) + a.maxshift;
    const uint32_t i_first = (rho - (uint32_t)s0) & (a.B - 1);
    const uint32_t nrows = i_first < cnt ? (cnt - 1 - i_first) / a.B + 1 : 0;
    const uint32_t j_beg = c * kChanRows;
    const uint32_t m = nrows > j_beg ? min(kChanRows, nrows - j_beg) : 0u;  // rows of this chunk
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid < 32) {
        uint32_t sigma, b;
        exact_hash(cp.seed, cp.id, t, a.nmask, &sigma, &b);
        const uint32_t sb = sigma * b;
        const bool ok = tid < m;
        const int32_t sl = (int32_t)(s0 + (int64_t)i_first + (int64_t)(j_beg + tid) * a.B);
        // the copies first, the coefficients while they are in flight
        if (tid == 0) mbar_arrive_expect_tx(&bar, m * C * (uint32_t)sizeof(float2));
        __syncwarp();
        if (ok) {
            const uint32_t row = (sigma * (uint32_t)sl) & a.nmask;
            bulk_copy_g2s(rows + (size_t)tid * C, static_cast<const float2*>(cp.x) + (size_t)row * C,
                          C * (uint32_t)sizeof(float2), &bar);
        }
#pragma unroll
        for (int h = 0; h < kMaxHash; ++h) {
            float2 co = make_float2(0.0f, 0.0f);
            const int32_t th = sl + (int32_t)a.a[h];
            if ((uint32_t)h < a.H && ok && th >= -a.T && th <= a.T) {
                const float gt = a.taps32[th < 0 ? -th : th];
                const uint32_t e = (sb * (uint32_t)th) & a.nmask;
                const int32_t es = e > (a.nmask >> 1) ? (int32_t)((int64_t)e - (int64_t)a.n) : (int32_t)e;
                float sn, cs;
                sincospif((float)es * (2.0f / (float)a.n), &sn, &cs);
                co = make_float2(gt * cs, -gt * sn);
            }
            if (tid < kChanRows) coef[tid * kMaxHash + h] = co;
        }
    }
    __syncthreads();  // the coefficients
    if (!mbar_wait(&bar, 0, kChanWaitLimit)) {
        // never expected: flag it, give the copies a second bounded wait, leave the partial sums alone
        if (tid == 0) atomicExch(cp.error, 1u);
        mbar_wait(&bar, 0, kChanWaitLimit);
        return;
    }
    for (uint32_t ch = tid; ch < C; ch += kThreads) {
        float2 acc[kMaxHash];
#pragma unroll
        for (int h = 0; h < kMaxHash; ++h) acc[h] = make_float2(0.0f, 0.0f);
        for (uint32_t j = 0; j < m; ++j) {
            const float2 v = rows[(size_t)j * C + ch];
#pragma unroll
            for (int h = 0; h < kMaxHash; ++h) acc[h] = cfma(coef[j * kMaxHash + h], v, acc[h]);
        }
        float2* area = static_cast<float2*>(a.part) + (size_t)ch * a.part_stride;
#pragma unroll
        for (int h = 0; h < kMaxHash; ++h)
            if ((uint32_t)h < a.H) area[((size_t)c * a.H + h) * a.B + rho] = acc[h];
    }
}

// The bins of every (round, slot) at once: partial folds summed in chunk order, bit-reversed, B-point
// FFT, left at the start of the slot's area of the round.
template <int NR>
__global__ void __launch_bounds__(kThreads, SFFT_ROUND_MIN_BLOCKS) k_chan_bins(const __grid_constant__ StepParams<NR> sp,
                                                                              uint64_t seed, uint32_t id) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t t = 0;
    while (t + 1 < sp.R && blockIdx.x >= sp.seg[t + 1]) ++t;
    const ExactArgs& a = sp.r[t];
    const uint32_t s = blockIdx.x - sp.seg[t];
    uint32_t sigma, b;
    exact_hash(seed, id, t, a.nmask, &sigma, &b);
    finish_round<float>(a, s, sigma, b, smem, kFinBins);
}

// The decodes: one CTA per channel slot runs them in round order (zhat of round t feeds round t + 1).
// If the gather flagged a copy that never landed, every slot reports SFFT_ERR_TIMEOUT instead.
template <int NR>
__global__ void __launch_bounds__(kThreads, SFFT_ROUND_MIN_BLOCKS) k_chan_decode(const __grid_constant__ StepParams<NR> sp,
                                                                                uint64_t seed, uint32_t id,
                                                                                const uint32_t* error) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t s = blockIdx.x;
    if (*error) {
        if (threadIdx.x == 0) {
            const ExactArgs& a = sp.r[sp.R - 1];
            a.out_count[s] = 0;
            a.out_flag[s] = SFFT_ERR_TIMEOUT;
        }
        return;
    }
    for (uint32_t t = 0; t < sp.R; ++t) {
        const ExactArgs& a = sp.r[t];
        uint32_t sigma, b;
        exact_hash(seed, id, t, a.nmask, &sigma, &b);
        finish_round<float>(a, s, sigma, b, a.fin_scratch ? a.fin_scratch + (size_t)s * a.fin_stride : smem,
                            kFinDecode, t > 0);
        __syncthreads();  // zhat of round t is read by round t + 1 (same CTA)
    }
}

// ------------------------------------------------------------------------------------------------
// Persistent path: one launch, a device queue of (request, round, chunk) items
// ------------------------------------------------------------------------------------------------
constexpr unsigned long long kItemValid = 1ull << 63;
constexpr uint32_t kSpinLimit = 1u << 23;  // x ~128 ns: a wait gives up after about a second

__device__ __forceinline__ unsigned long long pack_item(uint32_t r, uint32_t t, uint32_t c) {
    return kItemValid | ((unsigned long long)r << 24) | ((unsigned long long)t << 16) | c;
}
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void store_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

#ifndef SFFT_PERSIST_MIN_BLOCKS
#define SFFT_PERSIST_MIN_BLOCKS 2  // resident CTAs per SM the register budget is sized for
#endif

template <typename R>
__global__ void __launch_bounds__(kThreads, SFFT_PERSIST_MIN_BLOCKS) k_exact_persistent(const PersistArgs pa) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) ExactArgs sa;
    __shared__ unsigned long long s_item;
    const uint32_t tid = threadIdx.x;
    for (;;) {
        // take the next item and wait (bounded) until it is published
        if (tid == 0) {
            const uint32_t slot = atomicAdd(pa.head, 1u);
            unsigned long long it = 0;
            if (slot < pa.total) {
                for (uint32_t spin = 0;; ++spin) {
                    it = load_acquire(pa.items + slot);
                    if (it & kItemValid) break;
                    if (spin >= kSpinLimit) {
                        atomicExch(pa.error, 1);
                        it = 0;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            s_item = it;
        }
        __syncthreads();
        const unsigned long long it = s_item;
        if (!it) return;
        const uint32_t r = (uint32_t)((it >> 24) & 0xFFFFFFFFull), t = (uint32_t)((it >> 16) & 0xFFu),
                       c = (uint32_t)(it & 0xFFFFu);
        // the (plan, round) argument block, then the request's own workspace as slot 0
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(pa.rdesc + pa.req_rd0[r] + t);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
            for (uint32_t w = tid; w < sizeof(ExactArgs) / 4; w += kThreads) dst[w] = src[w];
        }
        __syncthreads();
        if (tid == 0) {
            sa.reqs = pa.reqs + r;
            sa.req_base = 0;
            sa.part = pa.part + (size_t)r * pa.part_stride;
            sa.part_stride = 0;
            sa.counter = pa.counter + r;
            sa.zidx = pa.zidx + (size_t)r * pa.z_stride;
            sa.zval = pa.zval + (size_t)r * pa.z_stride;
            sa.zcount = pa.zcount + r;
            sa.zflag = pa.zflag + r;
            sa.fin_scratch = sa.fin_scratch ? pa.fin + (size_t)r * pa.fin_stride : nullptr;
            sa.fin_stride = 0;
            sa.out_idx = pa.out_idx + (size_t)r * pa.out_cap;
            sa.out_val = pa.out_val + (size_t)r * pa.out_cap;
            sa.out_cap = pa.out_cap;
            sa.out_count = pa.out_count + r;
            sa.out_flag = pa.out_flag + r;
        }
        __syncthreads();
        const ExactArgs& a = sa;
        const ReqView rq = req_view(a.reqs, nullptr, 0, 0, 0, a.nmask);
        uint32_t sigma, b;
        exact_hash(rq.seed, rq.id, a.round, a.nmask, &sigma, &b);
        gather_fold<R>(a, rq.x, rq.xmask, 0, c, sigma, b, smem);
        if (arrive(a.counter, a.chunks)) {
            finish_round<R>(a, 0, sigma, b, a.fin_scratch ? a.fin_scratch : smem);
            __syncthreads();  // every thread's zhat and output stores precede thread 0's release
            if (tid == 0) {
                __threadfence();
                *a.counter = 0;
                if (t + 1 < pa.req_rounds[r]) {  // publish the request's next round
                    const uint32_t nch = pa.rdesc[pa.req_rd0[r] + t + 1].chunks;
                    const uint32_t base = atomicAdd(pa.tail, nch);
                    for (uint32_t q = 0; q < nch; ++q) store_release(pa.items + base + q, pack_item(r, t + 1, q));
                }
            }
        }
        __syncthreads();  // sa and the shared arrays are rewritten by the next item
    }
}

int exact_persistent_ctas(size_t smem, bool fp64) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(k_exact_persistent<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_exact_persistent<double>, kThreads, smem);
    } else {
        e = cudaFuncSetAttribute(k_exact_persistent<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_exact_persistent<float>, kThreads, smem);
    }
    if (e != cudaSuccess) return 0;
    return sms * per;
}

cudaError_t launch_exact_persistent(const PersistArgs& a, uint32_t ctas, size_t smem, cudaStream_t st, bool fp64) {
    if (fp64)
        k_exact_persistent<double><<<ctas, kThreads, smem, st>>>(a);
    else
        k_exact_persistent<float><<<ctas, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// decode on caller bins (single CTA)
// ------------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) k_exact_decode(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_nw, s_above, s_kept;
    const uint32_t tid = threadIdx.x, B = a.B;
    const uint32_t zcap = a.nz > 0 ? a.nz : 1;
    const FinLayout Ly = fin_layout(B, a.H, zcap, 16);
    double2* U = reinterpret_cast<double2*>(smem + Ly.U);
    uint32_t* ent_idx = reinterpret_cast<uint32_t*>(smem + Ly.ent_idx);
    uint32_t* ent_bin = reinterpret_cast<uint32_t*>(smem + Ly.ent_bin);
    double* ent_gain = reinterpret_cast<double*>(smem + Ly.ent_gain);
    uint32_t* bin_cnt = reinterpret_cast<uint32_t*>(smem + Ly.bin_cnt);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(smem + Ly.bin_start);
    uint32_t* bin_list = reinterpret_cast<uint32_t*>(smem + Ly.bin_list);
    uint32_t* cand_idx = reinterpret_cast<uint32_t*>(smem + Ly.cand_idx);
    double2* cand_val = reinterpret_cast<double2*>(smem + Ly.cand_val);
    uint32_t* srt_idx = reinterpret_cast<uint32_t*>(smem + Ly.srt_idx);
    double2* srt_val = reinterpret_cast<double2*>(smem + Ly.srt_val);
    uint32_t* scan = reinterpret_cast<uint32_t*>(smem + Ly.scan);
    __shared__ DecodeCtx d;
    if (tid == 0)
        fill_ctx(d, a.n, a.nmask, B, a.logB, a.H, a.shift64, a.sigma, a.b, a.wtab, a.thr, a.iso_tol, a.gmin, a.ref_lo,
                 a.ref_hi, a.ref_tol);
    __syncthreads();
    for (uint32_t i = tid; i < a.H * B; i += kThreads) U[i] = a.u[i];
    for (uint32_t e = tid; e < a.nz; e += kThreads) {
        const uint32_t i = a.zidx[e];
        ent_idx[e] = i;
        uint32_t jb;
        const int32_t o = offset_of((a.sigma * (i - a.b)) & a.nmask, d, &jb);
        ent_bin[e] = jb;
        ent_gain[e] = a.wtab[o < 0 ? -o : o];
    }
    if (tid == 0) {
        s_nw = 0;
        s_above = 0;
        s_kept = 0;
    }
    __syncthreads();
    bucket_entries(ent_bin, a.nz, B, bin_cnt, bin_start, bin_list, scan);
    for (uint32_t j = tid; j < B; j += kThreads) {
        using C = typename Cx<R>::T;
        C u[kMaxHash];  // the caller's bins, in the precision of the decisions
        for (uint32_t h = 0; h < a.H; ++h) {
            u[h].x = U[h * B + j].x;
            u[h].y = U[h * B + j].y;
        }
        uint32_t oi = 0;
        double gain = 1.0, ginv;  // this decode divides by the gain (its context has no 1 / W table)
        bool above;
        const int kind = decode_bin(d, j, u, bin_list + bin_start[j], bin_start[j + 1] - bin_start[j], ent_idx,
                                    ent_gain, &oi, &gain, &ginv, &above);
        if (above) atomicAdd(&s_above, 1u);
        if (kind == 1) atomicAdd(&s_kept, 1u);
        if (kind != 0) {
            const uint32_t slot = atomicAdd(&s_nw, 1u);
            cand_idx[slot] = oi;
            cand_val[slot] = make_double2(U[j].x / gain, U[j].y / gain);
        }
    }
    __syncthreads();
    const uint32_t nw = s_nw;
    rank_sort(cand_idx, cand_val, nw, srt_idx, srt_val);
    for (uint32_t p = tid; p < nw; p += kThreads) {
        a.widx[p] = srt_idx[p];
        a.wval[p] = srt_val[p];
    }
    if (tid == 0) {
        *a.count = nw;
        *a.nabove = s_above;
        *a.nkept = s_kept;
    }
}

__global__ void k_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t count,
                         uint32_t* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const Words4 w = philox4x32_10(c0, c1, c2, c3 + i, k0, k1);
    for (int q = 0; q < 4; ++q) out[4 * (size_t)i + q] = w.w[q];
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
// The dynamic shared-memory ceiling of a kernel is process-wide: it is only ever raised, so a plan
// created later with smaller rounds cannot lower it under another plan's feet.
template <int NR>
static cudaError_t launch_chan_nr(const ExactArgs* rounds, uint32_t R, uint32_t C, const void* x, uint64_t seed,
                                  uint32_t id, size_t smem, uint32_t* error, cudaStream_t st, cudaEvent_t before,
                                  cudaEvent_t after) {
    ChanParams<NR> cp;
    StepParams<NR> sp;
    cp.R = sp.R = R;
    cp.C = C;
    cp.seed = seed;
    cp.id = id;
    cp.x = x;
    cp.error = error;
    cp.cseg[0] = 0;
    sp.seg[0] = 0;
    for (uint32_t t = 0; t < R; ++t) {
        const uint64_t w = (uint64_t)cp.cseg[t] + (uint64_t)rounds[t].chunks * rounds[t].B;
        if (w > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
        cp.cseg[t + 1] = (uint32_t)w;
        sp.seg[t + 1] = sp.seg[t] + C;
        cp.r[t] = sp.r[t] = rounds[t];
    }
    const size_t gsmem = (size_t)kChanRows * C * sizeof(float2) + (size_t)kChanRows * kMaxHash * sizeof(float2);
    static std::mutex mu;
    static size_t set_to = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (set_to < kChanRows * kChanMaxC * sizeof(float2) + kChanRows * kMaxHash * sizeof(float2)) {
            const int full = (int)(kChanRows * kChanMaxC * sizeof(float2) + kChanRows * kMaxHash * sizeof(float2));
            cudaError_t e = cudaFuncSetAttribute(k_chan_gather<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, full);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_chan_gather<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, full);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_chan_gather<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, full);
            if (e != cudaSuccess) return e;
            set_to = (size_t)full;
        }
    }
    cudaError_t e = cudaMemsetAsync(error, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (before && (e = cudaEventRecord(before, st)) != cudaSuccess) return e;
    k_chan_gather<NR><<<cp.cseg[R], kThreads, gsmem, st>>>(cp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (after && (e = cudaEventRecord(after, st)) != cudaSuccess) return e;
    k_chan_bins<NR><<<sp.seg[R], kThreads, smem, st>>>(sp, seed, id);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_chan_decode<NR><<<C, kThreads, smem, st>>>(sp, seed, id, error);
    return cudaGetLastError();
}

cudaError_t launch_exact_channels(const ExactArgs* rounds, uint32_t R, uint32_t C, const void* x, uint64_t seed,
                                  uint32_t id, size_t smem, uint32_t* error, cudaStream_t st, cudaEvent_t before,
                                  cudaEvent_t after) {
    if (R == 0 || R > kMaxRounds || C == 0 || C % 32 || C > kChanMaxC || !error) return cudaErrorInvalidValue;
    if (R <= 8) return launch_chan_nr<8>(rounds, R, C, x, seed, id, smem, error, st, before, after);
    if (R <= 16) return launch_chan_nr<16>(rounds, R, C, x, seed, id, smem, error, st, before, after);
    return launch_chan_nr<32>(rounds, R, C, x, seed, id, smem, error, st, before, after);
}

cudaError_t set_exact_smem_limit(size_t bytes, bool fp64) {
    static std::mutex mu;  // plans may be created from several threads
    std::lock_guard<std::mutex> lk(mu);
    static size_t limit[2] = {0, 0};
    size_t& cur = limit[fp64 ? 1 : 0];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e;
    const int b = (int)bytes;
    if (fp64) {
        e = cudaFuncSetAttribute(k_exact_round<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<double, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<double, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    } else {
        e = cudaFuncSetAttribute(k_exact_round<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<float, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<float, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_exact_step<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_bins<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_bins<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_bins<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_decode<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_decode<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chan_decode<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
    if (e == cudaSuccess) cur = bytes;
    return e;
}

cudaError_t launch_exact_round(const ExactArgs& a, uint32_t batch, size_t smem, cudaStream_t st, bool fp64) {
    const dim3 grid(a.chunks, batch);
    if (fp64)
        k_exact_round<double><<<grid, kThreads, smem, st>>>(a);
    else
        k_exact_round<float><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NR>
static cudaError_t launch_step_nr(const ExactArgs* rounds, uint32_t R, uint32_t batch, size_t smem, cudaStream_t st,
                                  bool fp64) {
    StepParams<NR> sp;
    sp.R = R;
    sp.seg[0] = 0;
    for (uint32_t t = 0; t < R; ++t) {
        const uint64_t end = (uint64_t)sp.seg[t] + (uint64_t)rounds[t].chunks * batch;
        if (end > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;  // grid limit
        sp.seg[t + 1] = (uint32_t)end;
        sp.r[t] = rounds[t];
    }
    const uint32_t ctas = sp.seg[R];
    if (ctas == 0) return cudaSuccess;
    if (fp64)
        k_exact_step<double, NR><<<ctas, kThreads, smem, st>>>(sp);
    else
        k_exact_step<float, NR><<<ctas, kThreads, smem, st>>>(sp);
    return cudaGetLastError();
}

cudaError_t launch_exact_step(const ExactArgs* rounds, uint32_t R, uint32_t batch, size_t smem, cudaStream_t st,
                              bool fp64) {
    if (R == 0 || R > kMaxRounds) return cudaErrorInvalidValue;
    if (R <= 8) return launch_step_nr<8>(rounds, R, batch, smem, st, fp64);
    if (R <= 16) return launch_step_nr<16>(rounds, R, batch, smem, st, fp64);
    return launch_step_nr<32>(rounds, R, batch, smem, st, fp64);
}

cudaError_t launch_exact_decode(const DecodeArgs& a, cudaStream_t st) {
    const size_t smem = fin_layout(a.B, a.H, a.nz > 0 ? a.nz : 1, 16).total;
    cudaError_t e;
    if (a.fp64) {
        e = cudaFuncSetAttribute(k_exact_decode<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_exact_decode<double><<<1, kThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_exact_decode<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_exact_decode<float><<<1, kThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t count, uint32_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_philox<<<(count + 255) / 256, 256, 0, st>>>(k0, k1, c0, c1, c2, c3, count, out);
    return cudaGetLastError();
}

}  // namespace sfft
