// sfft_exact.cu -- the exact-mode round of the sparse FFT on sm_103a (Algorithm 1 of Hassanieh, Indyk,
// Katabi, Price), as one kernel per round for a whole batch of requests.
//
// Grid (chunks, batch).  Every CTA performs steps 1-2 of HashToBins (proof of Lemma "hashtobins") for
// 2048 consecutive window taps of one request and all hashings of the round (a = 0 and the ladder
// shifts share one staged run of samples, since x_{sigma(t - beta)} is sample t - beta of the
// sigma-strided sequence): it gathers the permuted samples, applies window and modulation, folds
// them modulo B and stores the partial fold.  The last CTA of a request to arrive (arrival counter,
// no waiting) sums the partials in chunk order, runs the B-point FFTs (step 3), subtracts the
// recovered coefficients in FP64 (step 4), decodes locations and values
// (NoiselessSparseFFTInner's loop over J) and merges the result into zhat (NoiselessSparseFFT).
// Every reduction has a fixed order and no floating-point atomics exist, so results are
// bit-reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "sfft_internal.h"

namespace sfft {

// ------------------------------------------------------------------------------------------------
// complex helpers
// ------------------------------------------------------------------------------------------------
template <typename R>
struct Cx;
template <>
struct Cx<float> {
    using T = float2;
};
template <>
struct Cx<double> {
    using T = double2;
};

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
    a.x -= b.x;
    a.y -= b.y;
    return a;
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// acc + a * b
template <typename C>
__device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 mul_conj(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ void sincospi_r(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_r(double x, double* s, double* c) { sincospi(x, s, c); }

__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldg(p); }

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

// w^e = exp(-2 pi i e / n) in FP64 for an exact exponent e in [0, n)
__device__ __forceinline__ double2 root_pow64(uint32_t e, uint32_t nmask) {
    const uint32_t n = nmask + 1u;
    const int64_t es = e > (nmask >> 1) ? (int64_t)e - (int64_t)n : (int64_t)e;
    double s, c;
    sincospi(2.0 * (double)es / (double)n, &s, &c);
    return make_double2(c, -s);
}

__device__ __forceinline__ double phase01(double2 z) {  // phase(z) / 2 pi in [0, 1)
    double p = atan2(z.y, z.x) * 0.15915494309189533576888;  // 1 / (2 pi)
    if (p < 0.0) p += 1.0;
    if (p >= 1.0) p -= 1.0;
    return p;
}

// ------------------------------------------------------------------------------------------------
// shared-memory layout of the finishing phase
// ------------------------------------------------------------------------------------------------
struct FinLayout {
    size_t U, ent_idx, ent_bin, ent_val, bin_cnt, bin_start, bin_list, cand_idx, cand_val, key, payload, keep, scan;
    size_t total;
    uint32_t M;
};
__host__ __device__ inline size_t fin_take(size_t* off, size_t bytes) {
    const size_t o = (*off + 15) & ~size_t(15);
    *off = o + bytes;
    return o;
}
__host__ __device__ inline uint32_t pow2_ge(uint32_t v) {
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}
__host__ __device__ inline FinLayout fin_layout(uint32_t B, uint32_t H, uint32_t zcap, uint32_t csize) {
    FinLayout L;
    size_t off = 0;
    L.U = fin_take(&off, (size_t)H * B * csize);
    L.ent_idx = fin_take(&off, (size_t)zcap * 4);
    L.ent_bin = fin_take(&off, (size_t)zcap * 4);
    L.ent_val = fin_take(&off, (size_t)zcap * 16);
    L.bin_cnt = fin_take(&off, (size_t)(B + 1) * 4);
    L.bin_start = fin_take(&off, (size_t)(B + 1) * 4);
    L.bin_list = fin_take(&off, (size_t)zcap * 4);
    L.cand_idx = fin_take(&off, (size_t)B * 4);
    L.cand_val = fin_take(&off, (size_t)B * 16);
    L.M = pow2_ge(zcap + B);
    L.key = fin_take(&off, (size_t)L.M * 8);
    L.payload = fin_take(&off, (size_t)L.M * 4);
    L.keep = fin_take(&off, (size_t)L.M * 4);
    L.scan = fin_take(&off, (size_t)(kThreads + 8) * 4);
    L.total = off;
    return L;
}

size_t exact_finish_smem(uint32_t B, uint32_t H, uint32_t zcap, bool fp64) {
    return fin_layout(B, H, zcap, fp64 ? 16 : 8).total;
}
size_t exact_gather_smem(uint32_t stage, bool fp64) { return (size_t)stage * (fp64 ? 16 : 8); }

// ------------------------------------------------------------------------------------------------
// block-wide helpers (kThreads threads)
// ------------------------------------------------------------------------------------------------
// Exclusive prefix sum of v[0..len) in place; returns the total.  tmp holds kThreads + 1 words.
__device__ uint32_t block_exclusive_scan(uint32_t* v, uint32_t len, uint32_t* tmp) {
    const uint32_t tid = threadIdx.x;
    const uint32_t seg = (len + kThreads - 1) / kThreads;
    const uint32_t b0 = min(len, tid * seg), b1 = min(len, b0 + seg);
    uint32_t sum = 0;
    for (uint32_t i = b0; i < b1; ++i) sum += v[i];
    tmp[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (uint32_t i = 0; i < kThreads; ++i) {
            const uint32_t x = tmp[i];
            tmp[i] = run;
            run += x;
        }
        tmp[kThreads] = run;
    }
    __syncthreads();
    uint32_t run = tmp[tid];
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t x = v[i];
        v[i] = run;
        run += x;
    }
    const uint32_t total = tmp[kThreads];
    __syncthreads();
    return total;
}

// Ascending bitonic sort of (key, payload), M a power of two.
__device__ void block_bitonic_sort(uint64_t* key, uint32_t* pay, uint32_t M) {
    for (uint32_t k = 2; k <= M; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < M; i += kThreads) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const uint64_t a = key[i], b = key[ixj];
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ixj] = a;
                        const uint32_t t = pay[i];
                        pay[i] = pay[ixj];
                        pay[ixj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// In-place radix-2 decimation-in-time FFT of B = 2^logB points held in bit-reversed order:
// a_j <- sum_r a_r exp(-2 pi i j r / B) in natural order (Lemma "hashtobins", step 3).
template <typename R>
__device__ void block_fft(typename Cx<R>::T* a, uint32_t logB) {
    using C = typename Cx<R>::T;
    const uint32_t B = 1u << logB;
    for (uint32_t st = 1; st <= logB; ++st) {
        const uint32_t half = 1u << (st - 1);
        for (uint32_t k = threadIdx.x; k < B / 2; k += kThreads) {
            const uint32_t pos = k & (half - 1);
            const uint32_t i0 = ((k >> (st - 1)) << st) + pos;
            const uint32_t i1 = i0 + half;
            R sn, cs;
            sincospi_r(-(R)pos / (R)half, &sn, &cs);
            const C w = mkc(cs, sn);
            const C bv = cmul(a[i1], w);
            const C av = a[i0];
            a[i0] = cadd(av, bv);
            a[i1] = csub(av, bv);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------
// Location and estimation of one bin (NoiselessSparseFFTInner's loop body), FP64
// ------------------------------------------------------------------------------------------------
struct DecodeCtx {
    uint32_t n, nmask, B, Np, logNp, H;
    uint32_t sigma, sigma_inv, b, sb;
    uint64_t shift[kMaxHash];  // shift of hashing h = l + 1 is shift[l]
    const double* wtab;
    double thr, iso_tol, gmin, ref_lo, ref_hi, ref_tol;
};

__device__ __forceinline__ int32_t offset_of(uint32_t p, const DecodeCtx& d, uint32_t* jbin) {
    const uint32_t jj = ((p + (d.Np >> 1)) & d.nmask) >> d.logNp;
    const uint32_t dd = (p - jj * d.Np) & d.nmask;
    *jbin = jj;
    return dd > (d.nmask >> 1) ? (int32_t)((int64_t)dd - (int64_t)d.n) : (int32_t)dd;
}

// A known entry i of zhat explains the residual of bin j (re-estimation of known values).
__device__ bool refine_known(const DecodeCtx& d, const double2* u, double mag0, uint32_t i, double2* val) {
    const uint32_t p = (d.sigma * (i - d.b)) & d.nmask;
    uint32_t jj;
    const int32_t o = offset_of(p, d, &jj);
    const double gain = d.wtab[o < 0 ? -o : o];
    if (!(gain >= d.gmin)) return false;
    for (uint32_t l = 0; l + 1 < d.H; ++l) {
        if (fabs(hypot(u[l + 1].x, u[l + 1].y) - mag0) > 0.25 * mag0) return false;
        const uint32_t e = ((uint32_t)d.shift[l] * d.sigma * i) & d.nmask;
        const double pred = (double)e / (double)d.n;
        double dist = fabs(phase01(mul_conj(u[0], u[l + 1])) - pred);
        if (dist > 0.5) dist = 1.0 - dist;
        if (!(dist * 6.283185307179586476925286766559 < d.ref_tol)) return false;
    }
    *val = make_double2(u[0].x / gain, u[0].y / gain);
    return true;
}

// Returns 0 (nothing), 1 (a decode of J kept) or 2 (a re-estimate of a known entry).
// *above is set when |u_0| > thr.  The zhat entries hashed to bin j are ent_idx[list[0..nbin)].
__device__ int decode_bin(const DecodeCtx& d, uint32_t j, const double2* u, const uint32_t* list, uint32_t nbin,
                          const uint32_t* ent_idx, uint32_t* oi, double2* ov, bool* above) {
    const double mag0 = hypot(u[0].x, u[0].y);
    *above = false;
    if (!(mag0 > d.thr)) {
        if (nbin > 0 && mag0 > d.ref_lo * d.thr && mag0 <= d.ref_hi * d.thr) {
            uint32_t matches = 0, who = 0;
            double2 val = make_double2(0.0, 0.0);
            for (uint32_t e = 0; e < nbin; ++e) {
                double2 v;
                const uint32_t i = ent_idx[list[e]];
                if (refine_known(d, u, mag0, i, &v)) {
                    ++matches;
                    who = i;
                    val = v;
                }
            }
            if (matches == 1) {
                *oi = who;
                *ov = val;
                return 2;
            }
        }
        return 0;
    }
    *above = true;
    // location ladder, coarsest shift first: q = sigma i mod n/B
    const int L = (int)d.H - 1;
    uint64_t M = (uint64_t)d.Np / (d.shift[L - 1] / d.B);
    const double th = phase01(mul_conj(u[0], u[L]));
    uint64_t c = (uint64_t)floor(th * (double)M + 0.5) % M;
    for (int l = L - 2; l >= 0; --l) {
        const uint64_t Mp = (uint64_t)d.Np / (d.shift[l] / d.B);
        const uint64_t ratio = Mp / M;
        const double thl = phase01(mul_conj(u[0], u[l + 1]));
        const double y = thl * (double)Mp / (double)M - (double)c / (double)M;
        int64_t h = (int64_t)floor(y + 0.5);
        h %= (int64_t)ratio;
        if (h < 0) h += (int64_t)ratio;
        c += M * (uint64_t)h;
        M = Mp;
    }
    const uint32_t q = (uint32_t)c;
    const uint32_t dd = (q + d.Np - (d.sb & (d.Np - 1)) + (d.Np >> 1)) & (d.Np - 1);
    const int32_t o = (int32_t)dd - (int32_t)(d.Np >> 1);
    const uint32_t p = (j * d.Np + (uint32_t)o) & d.nmask;
    const uint32_t si = (p + d.sb) & d.nmask;
    const uint32_t i = (d.sigma_inv * si) & d.nmask;
    const double gain = d.wtab[o < 0 ? -o : o];
    if (!(gain >= d.gmin)) return 0;
    for (uint32_t l = 0; l + 1 < d.H; ++l)
        if (fabs(hypot(u[l + 1].x, u[l + 1].y) - mag0) > d.iso_tol * mag0) return 0;
    *oi = i;
    *ov = make_double2(u[0].x / gain, u[0].y / gain);
    return 1;
}

// Bucket the nz entries of zhat by bin: bin_start[B+1] (exclusive prefix), bin_list (entry ids of
// each bin, ascending).  ent_bin must be filled.
__device__ void bucket_entries(const uint32_t* ent_bin, uint32_t nz, uint32_t B, uint32_t* bin_cnt,
                               uint32_t* bin_start, uint32_t* bin_list, uint32_t* scan_tmp) {
    for (uint32_t j = threadIdx.x; j <= B; j += kThreads) bin_cnt[j] = 0;
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < nz; e += kThreads) atomicAdd(&bin_cnt[ent_bin[e]], 1u);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j <= B; j += kThreads) bin_start[j] = bin_cnt[j];
    __syncthreads();
    block_exclusive_scan(bin_start, B + 1, scan_tmp);
    for (uint32_t j = threadIdx.x; j <= B; j += kThreads) bin_cnt[j] = bin_start[j];  // fill cursor
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < nz; e += kThreads) {
        const uint32_t slot = atomicAdd(&bin_cnt[ent_bin[e]], 1u);
        bin_list[slot] = e;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < B; j += kThreads) {  // insertion sort of each (short) bin list
        const uint32_t b0 = bin_start[j], b1 = bin_start[j + 1];
        for (uint32_t x = b0 + 1; x < b1; ++x) {
            const uint32_t v = bin_list[x];
            uint32_t y = x;
            while (y > b0 && bin_list[y - 1] > v) {
                bin_list[y] = bin_list[y - 1];
                --y;
            }
            bin_list[y] = v;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------------
// The round kernel
// ------------------------------------------------------------------------------------------------
template <typename R>
__device__ void gather_fold(const ExactArgs& a, uint32_t s, uint32_t c, uint32_t sigma, uint32_t b,
                            unsigned char* smem) {
    using C = typename Cx<R>::T;
    C* stage = reinterpret_cast<C*>(smem);
    C* red = stage + a.stage;
    const uint32_t tid = threadIdx.x;
    const C* __restrict__ x = reinterpret_cast<const C*>(a.x) + (size_t)s * a.n;
    const R* __restrict__ taps = taps_of<R>(a);
    const int64_t t_lo = -a.T + (int64_t)c * kChunkTaps;
    const int64_t t_hi = min(t_lo + (int64_t)kChunkTaps, a.T + 1);
    const uint32_t ntap = (uint32_t)(t_hi - t_lo);
    const int32_t base = (int32_t)(t_lo - (int64_t)a.a_base - (int64_t)a.maxshift);  // sample held by stage[0]
    const uint32_t cnt = ntap + a.maxshift;
    // step 1a: gather the sigma-strided samples x_{sigma s}, s in [base, base + cnt) (8 loads in flight)
    for (uint32_t i0 = tid; i0 < cnt; i0 += kThreads * 8) {
        C v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t i = i0 + (uint32_t)q * kThreads;
            if (i < cnt) v[q] = ldg_c(x + ((sigma * (uint32_t)(base + (int32_t)i)) & a.nmask));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
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
    C* part = reinterpret_cast<C*>(a.part) + ((size_t)s * a.chunks + c) * a.H * a.B;
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

template <typename R>
__device__ void finish_round(const ExactArgs& a, uint32_t s, uint32_t sigma, uint32_t b, unsigned char* smem) {
    using C = typename Cx<R>::T;
    const uint32_t tid = threadIdx.x;
    const uint32_t B = a.B, H = a.H;
    const FinLayout Ly = fin_layout(B, H, a.zcap, sizeof(C));
    C* U = reinterpret_cast<C*>(smem + Ly.U);
    uint32_t* ent_idx = reinterpret_cast<uint32_t*>(smem + Ly.ent_idx);
    uint32_t* ent_bin = reinterpret_cast<uint32_t*>(smem + Ly.ent_bin);
    double2* ent_val = reinterpret_cast<double2*>(smem + Ly.ent_val);
    uint32_t* bin_cnt = reinterpret_cast<uint32_t*>(smem + Ly.bin_cnt);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(smem + Ly.bin_start);
    uint32_t* bin_list = reinterpret_cast<uint32_t*>(smem + Ly.bin_list);
    uint32_t* cand_idx = reinterpret_cast<uint32_t*>(smem + Ly.cand_idx);
    double2* cand_val = reinterpret_cast<double2*>(smem + Ly.cand_val);
    uint64_t* key = reinterpret_cast<uint64_t*>(smem + Ly.key);
    uint32_t* pay = reinterpret_cast<uint32_t*>(smem + Ly.payload);
    uint32_t* keep = reinterpret_cast<uint32_t*>(smem + Ly.keep);
    uint32_t* scan = reinterpret_cast<uint32_t*>(smem + Ly.scan);
    __shared__ uint32_t s_nw, s_above, s_kept;

    // step 2 (across chunks) and 3: partial folds summed in chunk order, bit-reversed, FFT
    const C* part = reinterpret_cast<const C*>(a.part) + (size_t)s * a.chunks * H * B;
    const uint32_t shift_br = 32u - a.logB;
    for (uint32_t i = tid; i < H * B; i += kThreads) {
        const uint32_t h = i / B, r = i - h * B;
        C sum = mkc((R)0, (R)0);
        for (uint32_t c = 0; c < a.chunks; ++c) {
            const C v = __ldcg(part + ((size_t)c * H + h) * B + r);
            sum = cadd(sum, v);
        }
        U[h * B + (__brev(r) >> shift_br)] = sum;
    }
    if (tid == 0) {
        s_nw = 0;
        s_above = 0;
        s_kept = 0;
    }
    __syncthreads();
    for (uint32_t h = 0; h < H; ++h) block_fft<R>(U + h * B, a.logB);

    // zhat of this request
    const uint32_t nz = a.bins_only ? a.e_nz : min(a.zcount[s], a.zcap);
    DecodeCtx d;
    d.n = (uint32_t)a.n;
    d.nmask = a.nmask;
    d.B = B;
    d.Np = (uint32_t)(a.n >> a.logB);
    d.logNp = 0;
    while ((1u << d.logNp) < d.Np) ++d.logNp;
    d.H = H;
    d.sigma = sigma;
    d.sigma_inv = inverse_odd(sigma) & a.nmask;
    d.b = b;
    d.sb = (sigma * b) & a.nmask;
    for (int l = 0; l < kMaxHash; ++l) d.shift[l] = l + 1 < kMaxHash ? a.shift64[l + 1] : 0;
    d.wtab = a.wtab;
    d.thr = a.thr;
    d.iso_tol = a.iso_tol;
    d.gmin = a.gmin;
    d.ref_lo = a.ref_lo;
    d.ref_hi = a.ref_hi;
    d.ref_tol = a.ref_tol;
    for (uint32_t e = tid; e < nz; e += kThreads) {
        const uint32_t i = a.zidx[(size_t)s * a.zcap + e];
        ent_idx[e] = i;
        ent_val[e] = a.zval[(size_t)s * a.zcap + e];
        uint32_t jb;
        offset_of((sigma * (i - b)) & a.nmask, d, &jb);
        ent_bin[e] = jb;
    }
    __syncthreads();
    bucket_entries(ent_bin, nz, B, bin_cnt, bin_start, bin_list, scan);

    // step 4 and the decode, one bin per thread
    for (uint32_t j = tid; j < B; j += kThreads) {
        double2 u[kMaxHash];
        for (uint32_t h = 0; h < H; ++h) {
            const C v = U[h * B + j];
            u[h] = make_double2((double)v.x, (double)v.y);
        }
        for (uint32_t x = bin_start[j]; x < bin_start[j + 1]; ++x) {
            const uint32_t e = bin_list[x];
            const uint32_t i = ent_idx[e];
            const uint32_t p = (sigma * (i - b)) & a.nmask;
            uint32_t jb;
            const int32_t o = offset_of(p, d, &jb);
            const double gain = a.wtab[o < 0 ? -o : o];
            const double2 gz = make_double2(gain * ent_val[e].x, gain * ent_val[e].y);
            for (uint32_t h = 0; h < H; ++h) {
                const double2 w = root_pow64(((a.a_base + a.a[h]) * sigma * i) & a.nmask, a.nmask);
                const double2 sub = make_double2(gz.x * w.x - gz.y * w.y, gz.x * w.y + gz.y * w.x);
                u[h].x -= sub.x;
                u[h].y -= sub.y;
            }
        }
        if (a.bins_only) {
            a.ubins[j] = u[0];
            continue;
        }
        uint32_t oi = 0;
        double2 ov;
        bool above;
        const int kind = decode_bin(d, j, u, bin_list + bin_start[j], bin_start[j + 1] - bin_start[j], ent_idx, &oi,
                                    &ov, &above);
        if (above) atomicAdd(&s_above, 1u);
        if (kind == 1) atomicAdd(&s_kept, 1u);
        if (kind != 0) {
            const uint32_t slot = atomicAdd(&s_nw, 1u);
            cand_idx[slot] = oi;
            cand_val[slot] = ov;
        }
    }
    __syncthreads();
    if (a.bins_only) return;

    // merge what into zhat: sort (index, source) and add equal indices (zhat first), prune
    const uint32_t nw = s_nw;
    const uint32_t tot = nz + nw;
    const uint32_t M = pow2_ge(tot < 2 ? 2 : tot);
    for (uint32_t p = tid; p < M; p += kThreads) {
        if (p < nz) {
            key[p] = ((uint64_t)ent_idx[p] << 1);
            pay[p] = p;
        } else if (p < tot) {
            key[p] = ((uint64_t)cand_idx[p - nz] << 1) | 1u;
            pay[p] = p;
        } else {
            key[p] = ~0ull;
            pay[p] = 0;
        }
    }
    __syncthreads();
    block_bitonic_sort(key, pay, M);
    const double drop = a.prune * a.thr;
    for (uint32_t p = tid; p < M; p += kThreads) {
        uint32_t kp = 0;
        if (p < tot) {
            const uint64_t idx = key[p] >> 1;
            const bool head = p == 0 || (key[p - 1] >> 1) != idx;
            if (head) {
                const uint32_t q0 = pay[p];
                double2 v = q0 < nz ? ent_val[q0] : cand_val[q0 - nz];
                if (p + 1 < tot && (key[p + 1] >> 1) == idx) {
                    const uint32_t q1 = pay[p + 1];
                    const double2 w = q1 < nz ? ent_val[q1] : cand_val[q1 - nz];
                    v.x += w.x;
                    v.y += w.y;
                }
                kp = hypot(v.x, v.y) < drop ? 0u : 1u;
            }
        }
        keep[p] = kp;
    }
    __syncthreads();
    const uint32_t newcount = block_exclusive_scan(keep, M, scan);
    // keep[] now holds output positions; recompute the values of kept heads and store
    uint32_t* zi = a.zidx + (size_t)s * a.zcap;
    double2* zv = a.zval + (size_t)s * a.zcap;
    const bool last = a.last_round != 0;
    for (uint32_t p = tid; p < tot; p += kThreads) {
        const uint64_t idx = key[p] >> 1;
        const bool head = p == 0 || (key[p - 1] >> 1) != idx;
        if (!head) continue;
        const uint32_t pos = keep[p];  // exclusive prefix of the keep flags: kept iff the next differs
        const uint32_t nxt = p + 1 < M ? keep[p + 1] : newcount;
        if (nxt == pos) continue;
        const uint32_t q0 = pay[p];
        double2 v = q0 < nz ? ent_val[q0] : cand_val[q0 - nz];
        if (p + 1 < tot && (key[p + 1] >> 1) == idx) {
            const uint32_t q1 = pay[p + 1];
            const double2 w = q1 < nz ? ent_val[q1] : cand_val[q1 - nz];
            v.x += w.x;
            v.y += w.y;
        }
        if (pos < a.zcap) {
            zi[pos] = (uint32_t)idx;
            zv[pos] = v;
        }
        if (last && pos < a.out_cap) {
            a.out_idx[(size_t)s * a.out_cap + pos] = (uint32_t)idx;
            a.out_val[(size_t)s * a.out_cap + pos] = v;
        }
    }
    if (tid == 0) {
        const bool overflow = newcount > a.zcap;
        if (overflow) a.zflag[s] = 1;
        a.zcount[s] = overflow ? a.zcap : newcount;
        if (last) {
            const uint32_t kept_count = overflow ? a.zcap : newcount;
            a.out_count[s] = kept_count < a.out_cap ? kept_count : a.out_cap;
            int32_t flag = SFFT_OK;
            if (a.zflag[s] || kept_count > a.out_cap)
                flag = SFFT_ERR_CAPACITY;
            else if (s_above > s_kept)
                flag = SFFT_ERR_NOT_CONVERGED;
            a.out_flag[s] = flag;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads, 4) k_exact_round(const ExactArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_last;
    const uint32_t s = blockIdx.y, c = blockIdx.x;
    uint32_t sigma, b;
    if (a.bins_only) {
        sigma = a.e_sigma;
        b = a.e_b;
    } else {
        exact_hash(a.seed, s, a.round, a.nmask, &sigma, &b);
    }
    gather_fold<R>(a, s, c, sigma, b, smem);
    // arrival: the last CTA of request s finishes the round (nobody waits)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.counter + s, 1u) == a.chunks - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    finish_round<R>(a, s, sigma, b, smem);
    if (threadIdx.x == 0) a.counter[s] = 0;
}

// ------------------------------------------------------------------------------------------------
// decode on caller bins (single CTA)
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_exact_decode(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_nw, s_above, s_kept;
    const uint32_t tid = threadIdx.x, B = a.B;
    const uint32_t zcap = a.nz > 0 ? a.nz : 1;
    const FinLayout Ly = fin_layout(B, a.H, zcap, 16);
    double2* U = reinterpret_cast<double2*>(smem + Ly.U);
    uint32_t* ent_idx = reinterpret_cast<uint32_t*>(smem + Ly.ent_idx);
    uint32_t* ent_bin = reinterpret_cast<uint32_t*>(smem + Ly.ent_bin);
    uint32_t* bin_cnt = reinterpret_cast<uint32_t*>(smem + Ly.bin_cnt);
    uint32_t* bin_start = reinterpret_cast<uint32_t*>(smem + Ly.bin_start);
    uint32_t* bin_list = reinterpret_cast<uint32_t*>(smem + Ly.bin_list);
    uint32_t* cand_idx = reinterpret_cast<uint32_t*>(smem + Ly.cand_idx);
    double2* cand_val = reinterpret_cast<double2*>(smem + Ly.cand_val);
    uint64_t* key = reinterpret_cast<uint64_t*>(smem + Ly.key);
    uint32_t* pay = reinterpret_cast<uint32_t*>(smem + Ly.payload);
    uint32_t* scan = reinterpret_cast<uint32_t*>(smem + Ly.scan);
    DecodeCtx d;
    d.n = (uint32_t)a.n;
    d.nmask = a.nmask;
    d.B = B;
    d.Np = (uint32_t)(a.n >> a.logB);
    d.logNp = 0;
    while ((1u << d.logNp) < d.Np) ++d.logNp;
    d.H = a.H;
    d.sigma = a.sigma;
    d.sigma_inv = inverse_odd(a.sigma) & a.nmask;
    d.b = a.b;
    d.sb = (a.sigma * a.b) & a.nmask;
    for (int l = 0; l < kMaxHash; ++l) d.shift[l] = a.shift64[l];
    d.wtab = a.wtab;
    d.thr = a.thr;
    d.iso_tol = a.iso_tol;
    d.gmin = a.gmin;
    d.ref_lo = a.ref_lo;
    d.ref_hi = a.ref_hi;
    d.ref_tol = a.ref_tol;
    for (uint32_t i = tid; i < a.H * B; i += kThreads) U[i] = a.u[i];
    for (uint32_t e = tid; e < a.nz; e += kThreads) {
        const uint32_t i = a.zidx[e];
        ent_idx[e] = i;
        uint32_t jb;
        offset_of((a.sigma * (i - a.b)) & a.nmask, d, &jb);
        ent_bin[e] = jb;
    }
    if (tid == 0) {
        s_nw = 0;
        s_above = 0;
        s_kept = 0;
    }
    __syncthreads();
    bucket_entries(ent_bin, a.nz, B, bin_cnt, bin_start, bin_list, scan);
    for (uint32_t j = tid; j < B; j += kThreads) {
        double2 u[kMaxHash];
        for (uint32_t h = 0; h < a.H; ++h) u[h] = U[h * B + j];
        uint32_t oi = 0;
        double2 ov;
        bool above;
        const int kind = decode_bin(d, j, u, bin_list + bin_start[j], bin_start[j + 1] - bin_start[j], ent_idx, &oi,
                                    &ov, &above);
        if (above) atomicAdd(&s_above, 1u);
        if (kind == 1) atomicAdd(&s_kept, 1u);
        if (kind != 0) {
            const uint32_t slot = atomicAdd(&s_nw, 1u);
            cand_idx[slot] = oi;
            cand_val[slot] = ov;
        }
    }
    __syncthreads();
    const uint32_t nw = s_nw;
    const uint32_t M = pow2_ge(nw < 2 ? 2 : nw);
    for (uint32_t p = tid; p < M; p += kThreads) {
        key[p] = p < nw ? (uint64_t)cand_idx[p] : ~0ull;
        pay[p] = p;
    }
    __syncthreads();
    block_bitonic_sort(key, pay, M);
    for (uint32_t p = tid; p < nw; p += kThreads) {
        a.widx[p] = (uint32_t)key[p];
        a.wval[p] = cand_val[pay[p]];
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
cudaError_t set_exact_smem_limit(size_t bytes, bool fp64) {
    static size_t limit[2] = {0, 0};
    size_t& cur = limit[fp64 ? 1 : 0];
    if (bytes <= cur) return cudaSuccess;
    cudaError_t e;
    if (fp64)
        e = cudaFuncSetAttribute(k_exact_round<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    else
        e = cudaFuncSetAttribute(k_exact_round<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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

cudaError_t launch_exact_decode(const DecodeArgs& a, cudaStream_t st) {
    const size_t smem = fin_layout(a.B, a.H, a.nz > 0 ? a.nz : 1, 16).total;
    cudaError_t e = cudaFuncSetAttribute(k_exact_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_exact_decode<<<1, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t count, uint32_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_philox<<<(count + 255) / 256, 256, 0, st>>>(k0, k1, c0, c1, c2, c3, count, out);
    return cudaGetLastError();
}

}  // namespace sfft
