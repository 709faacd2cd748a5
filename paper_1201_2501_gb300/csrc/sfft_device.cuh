// sfft_device.cuh -- device helpers shared by the exact and the general kernels: complex
// arithmetic, the precision-templated transcendental helpers, block-wide scan/sort and the batched
// bin FFT.  Everything is inline; each translation unit gets its own copy.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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

// Sample loads are cached in L2 only: the sigma-strided gather touches one 32-byte sector per sample
// and an L1 fill would fetch the whole 128-byte line.
// Request s of a launch: its signal row, its seed and the request index its random draws use.
// xmask: a permuted sample index p (already reduced mod n, or a uint32 product, n | 2^32) reads
// x[p & xmask]: n - 1, or period - 1 for a periodic extension.
struct ReqView {
    const void* x;
    uint64_t seed;
    uint32_t id;
    uint32_t xmask;
};
__device__ __forceinline__ ReqView req_view(const ReqDesc* reqs, const void* x, uint64_t row_bytes, uint64_t seed,
                                            uint32_t s, uint32_t nmask) {
    if (reqs) {
        const ReqDesc d = reqs[s];
        return ReqView{d.x, d.seed, d.id, d.period ? d.period - 1u : nmask};
    }
    return ReqView{static_cast<const unsigned char*>(x) + (size_t)s * row_bytes, seed, s, nmask};
}

__device__ __forceinline__ float2 ldg_c(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double2 ldg_c(const double2* p) { return __ldcg(p); }

// Precision of the decode.  Bins, subtraction sums, values and all index arithmetic are FP64.  The
// transcendental functions (the subtraction twiddles w^{a sigma i}, phases and magnitudes) run in
// the precision R of the data path: an FP32 bin carries ~1e-6 of accumulated rounding, so an FP32
// atan2 or sincospi (~1e-7) adds nothing measurable, while GB300's FP64 pipe is ~1/64 of FP32.
// Every phase the decode compares keeps a tolerance of at least tau_dec (1e-4 rad by default).

// w^e = exp(-2 pi i e / n) for an exact exponent e in [0, n), evaluated in precision R
template <typename R>
__device__ __forceinline__ double2 root_pow(uint32_t e, uint32_t nmask) {
    const uint32_t n = nmask + 1u;
    const int64_t es = e > (nmask >> 1) ? (int64_t)e - (int64_t)n : (int64_t)e;
    R s, c;
    sincospi_r((R)(2 * es) / (R)n, &s, &c);
    return make_double2((double)c, -(double)s);
}

// phase(z) / 2 pi in [0, 1)
template <typename R>
__device__ __forceinline__ double phase01(double2 z);
template <>
__device__ __forceinline__ double phase01<double>(double2 z) {
    double p = __ddiv_rn(atan2(z.y, z.x), 6.283185307179586476925286766559);
    if (p < 0.0) p += 1.0;
    if (p >= 1.0) p -= 1.0;
    return p;
}

// a * conj(b) with every product and sum rounded separately (no fused multiply-add), so that a
// decision taken on the result sees the same double an unfused host computation produces
__device__ __forceinline__ double2 mul_conj_rn(double2 a, double2 b) {
    return make_double2(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dsub_rn(__dmul_rn(a.y, b.x), __dmul_rn(a.x, b.y)));
}
template <>
__device__ __forceinline__ double phase01<float>(double2 z) {
    double p = (double)atan2f((float)z.y, (float)z.x) * 0.15915494309189533576888;
    if (p < 0.0) p += 1.0;
    if (p >= 1.0) p -= 1.0;
    return p;
}
template <typename R>
__device__ __forceinline__ double cmag(double2 z);
template <>
__device__ __forceinline__ double cmag<double>(double2 z) {
    return hypot(z.x, z.y);
}
template <>
__device__ __forceinline__ double cmag<float>(double2 z) {
    return (double)hypotf((float)z.x, (float)z.y);
}

__device__ __forceinline__ uint32_t ilog2_u32(uint32_t v) { return 31u - __clz(v); }

// ------------------------------------------------------------------------------------------------
// block-wide helpers (kThreads threads)
// ------------------------------------------------------------------------------------------------
// Exclusive prefix sum of v[0..len) in place; returns the total.  tmp holds kThreads + 1 words.
__device__ inline uint32_t block_exclusive_scan(uint32_t* v, uint32_t len, uint32_t* tmp) {
    const uint32_t tid = threadIdx.x;
    const uint32_t seg = (len + kThreads - 1) / kThreads;
    const uint32_t b0 = min(len, tid * seg), b1 = min(len, b0 + seg);
    uint32_t sum = 0;
    for (uint32_t i = b0; i < b1; ++i) sum += v[i];
    // inclusive scan of the per-thread sums: within each warp by shuffles, then across the 8 warps
    const uint32_t lane = tid & 31u, warp = tid >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (uint32_t off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (uint32_t w = 0; w < (uint32_t)kThreads / 32u; ++w) {
            const uint32_t x = tmp[w];
            tmp[w] = run;
            run += x;
        }
        tmp[kThreads] = run;
    }
    __syncthreads();
    uint32_t run = tmp[warp] + incl - sum;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t x = v[i];
        v[i] = run;
        run += x;
    }
    const uint32_t total = tmp[kThreads];
    __syncthreads();
    return total;
}

// The same for 0/1 flags, len <= kThreads (one per thread): warp ballots, one barrier for the warps'
// counts and one after the result.
__device__ inline uint32_t block_exclusive_scan_flags(uint32_t* v, uint32_t len, uint32_t* tmp) {
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, tid < len && v[tid] != 0u);
    if (lane == 0) tmp[warp] = (uint32_t)__popc((int)bal);
    __syncthreads();
    uint32_t off = 0, total = 0;
#pragma unroll
    for (uint32_t w = 0; w < (uint32_t)kThreads / 32u; ++w) {
        const uint32_t c = tmp[w];
        off += w < warp ? c : 0u;
        total += c;
    }
    if (tid < len) v[tid] = off + (uint32_t)__popc((int)(bal & ((1u << lane) - 1u)));
    __syncthreads();
    return total;
}

// number of entries of the ascending array a[0..len) that are < key (lower) or <= key (upper)
__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Candidates (distinct indices, any order) sorted by index into (srt_idx, srt_val) by rank counting.
__device__ inline void rank_sort(const uint32_t* idx, const double2* val, uint32_t m, uint32_t* srt_idx, double2* srt_val) {
    for (uint32_t c = threadIdx.x; c < m; c += kThreads) {
        const uint32_t key = idx[c];
        uint32_t r = 0;
        for (uint32_t q = 0; q < m; ++q) r += idx[q] < key ? 1u : 0u;
        srt_idx[r] = key;
        srt_val[r] = val[c];
    }
    __syncthreads();
}

// In-place radix-2 decimation-in-time FFTs of H rows of B = 2^logB points held in bit-reversed
// order: a_j <- sum_r a_r exp(-2 pi i j r / B) in natural order (Lemma "hashtobins", step 3).
// The first min(5, logB) stages pair elements less than 32 apart: each warp holds 32 consecutive
// elements (one per lane) and exchanges partners by shuffles, with the twiddles exp(-i pi k / 16),
// k < 16, computed once per lane and shuffled to where they are needed.  The remaining stages run
// in place in shared memory, all rows together, one barrier per stage.  Butterfly arithmetic and
// twiddle values are the same in both forms.  Ends with a barrier.
template <typename R>
__device__ void block_fft_rows(typename Cx<R>::T* a, uint32_t H, uint32_t logB) {
    using C = typename Cx<R>::T;
    const uint32_t B = 1u << logB;
    const uint32_t halfB = B >> 1;
    const uint32_t total = H * B, lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t S = logB < 5 ? logB : 5;
    __syncthreads();  // the rows are in place
    {
        R ts, tc;
        sincospi_r(-(R)(lane & 15u) / (R)16, &ts, &tc);  // exp(-i pi k / 16), k = lane mod 16
        for (uint32_t g0 = warp * 32u; g0 < total; g0 += (uint32_t)kThreads) {
            const uint32_t i = g0 + lane;
            C v = i < total ? a[i] : mkc((R)0, (R)0);
            for (uint32_t st = 1; st <= S; ++st) {
                const uint32_t half = 1u << (st - 1);
                const uint32_t pos = lane & (half - 1);
                C w;
                w.x = __shfl_sync(0xffffffffu, tc, (int)(pos << (5 - st)));
                w.y = __shfl_sync(0xffffffffu, ts, (int)(pos << (5 - st)));
                C p;
                p.x = __shfl_xor_sync(0xffffffffu, v.x, (int)half);
                p.y = __shfl_xor_sync(0xffffffffu, v.y, (int)half);
                const bool upper = (lane & half) != 0;
                const C bv = cmul(upper ? v : p, w);
                const C av = upper ? p : v;
                v = upper ? csub(av, bv) : cadd(av, bv);
            }
            if (i < total) a[i] = v;
        }
    }
    __syncthreads();
    for (uint32_t st = S + 1; st <= logB; ++st) {
        const uint32_t half = 1u << (st - 1);
        for (uint32_t idx = threadIdx.x; idx < H * halfB; idx += kThreads) {
            const uint32_t h = idx >> (logB - 1);
            const uint32_t k = idx & (halfB - 1);
            const uint32_t pos = k & (half - 1);
            const uint32_t i0 = h * B + ((k >> (st - 1)) << st) + pos;
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

// Bucket the nz entries of zhat by bin: bin_start[B+1] (exclusive prefix), bin_list (entry ids of
// each bin, ascending).  ent_bin must be filled.
__device__ inline void bucket_entries(const uint32_t* ent_bin, uint32_t nz, uint32_t B, uint32_t* bin_cnt,
                               uint32_t* bin_start, uint32_t* bin_list, uint32_t* scan_tmp) {
    if (nz == 0) {  // no entries: every bin list is empty
        for (uint32_t j = threadIdx.x; j <= B; j += kThreads) bin_start[j] = 0;
        __syncthreads();
        return;
    }
    if (nz <= (uint32_t)kThreads) {
        // one entry per thread: its place in bin_list is the number of entries before it in (bin, id)
        // order; scan_tmp receives the bins in that order, and bin_start[j] counts those below j
        if (threadIdx.x < nz) {
            const uint32_t e0 = threadIdx.x, b0 = ent_bin[e0];
            uint32_t r = 0;
            for (uint32_t e = 0; e < nz; ++e) {
                const uint32_t be = ent_bin[e];
                r += (be < b0 || (be == b0 && e < e0)) ? 1u : 0u;
            }
            bin_list[r] = e0;
            scan_tmp[r] = b0;
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j <= B; j += kThreads) bin_start[j] = lower_bound_u32(scan_tmp, nz, j);
        __syncthreads();
        return;
    }
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
// CTA arrival
// ------------------------------------------------------------------------------------------------
// Arrival of this CTA at a counter whose last arrival (the target-th) does the follow-up work.
// Returns 1 in every thread of the last arriving CTA.  Only thread 0 fences: the barrier before its
// fence orders every thread's stores before it (the fence is cumulative), and the barrier after it
// orders its fence before every thread's loads (the same pattern as a grid-wide barrier).  Data
// written by other CTAs of the same launch is then read through L2 (ld.global.cg).
// ---- bulk asynchronous copies (TMA, cp.async.bulk) completing on a shared-memory mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the async proxy
}
// one arrival that also announces `bytes` of copies to complete in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Bounded wait for the phase of parity `parity`: true once it has completed, false after `limit`
// tries (each try may suspend the thread for a short, hardware-defined time).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ uint32_t arrive(uint32_t* counter, uint32_t target) {
    __shared__ uint32_t s_arrive_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t last = atomicAdd(counter, 1u) + 1u == target ? 1u : 0u;
        if (last) __threadfence();
        s_arrive_last = last;
    }
    __syncthreads();
    return s_arrive_last;
}

// an acquire load of *p (gpu scope) compared with v
__device__ __forceinline__ bool acquire_is(const uint32_t* p, uint32_t v) {
    uint32_t seen;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(p) : "memory");
    return seen == v;
}

// Arrival of one of two parties.  When an acquire load already sees the other party's arrival, this
// CTA is the last: the other party's writes are visible through the load, and nobody reads this CTA's
// writes through the counter, so the release fence and the atomic are skipped (the counter stays at 1
// until the caller clears it).  Otherwise as arrive(counter, 2).
__device__ __forceinline__ uint32_t arrive_pair(uint32_t* counter) {
    __shared__ uint32_t s_pair_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t seen;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(counter) : "memory");
        uint32_t last = 1u;
        if (seen != 1u) {
            __threadfence();
            last = atomicAdd(counter, 1u) + 1u == 2u ? 1u : 0u;
            if (last) __threadfence();
        }
        s_pair_last = last;
    }
    __syncthreads();
    return s_pair_last;
}

}  // namespace sfft
