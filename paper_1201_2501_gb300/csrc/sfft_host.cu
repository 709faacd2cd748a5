// sfft_host.cu -- host-side plan construction: parameter defaults, the exact round schedule and the
// flat-window design (Sec. 7 of the paper), all in double precision.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "philox.cuh"
#include "sfft_internal.h"

namespace sfft {

static thread_local std::string g_last_error;

void set_last_error(const std::string& s) { g_last_error = s; }

static uint64_t pow2_at_least(double v) {
    uint64_t p = 1;
    while ((double)p < v) p <<= 1;
    return p;
}

static uint32_t ceil_log2(uint64_t v) {
    uint32_t l = 0;
    while ((uint64_t(1) << l) < v) ++l;
    return l;
}

// Sec. 7: the window is a Gaussian (frequency std sigma_f = alpha / (4 B z), z = sqrt(2 ln 1/delta))
// convolved with a box-car of half width C = (1 - alpha/2) / (2B).  In time the Gaussian factor is
// exp(-2 pi^2 sigma_f^2 t^2); it is cut where it falls to delta, at T = z / (2 pi sigma_f)
// = 4 B ln(1/delta) / (pi alpha).
int64_t window_halfwidth(uint32_t B, double alpha, double delta) {
    const double T = 4.0 * (double)B * std::log(1.0 / delta) / (M_PI * alpha);
    return (int64_t)std::floor(T);
}

// Taps g_t = n G*(t), t = 0..T, G*(t) = exp(-2 pi^2 sigma_f^2 t^2) sin(2 pi C t) / (pi t), G*(0) = 2C.
// The factor n makes an isolated tone of amplitude X land in its bin with amplitude X W(-o).
void window_taps_host(uint64_t n, uint32_t B, double alpha, double delta, int64_t T, double* g) {
    const double z = std::sqrt(2.0 * std::log(1.0 / delta));
    const double C = (1.0 - 0.5 * alpha) / (2.0 * (double)B);
    const double sf = alpha / (4.0 * (double)B * z);
    const double gauss_rate = 2.0 * M_PI * M_PI * sf * sf;
    const double nn = (double)n;
    g[0] = nn * 2.0 * C;
    for (int64_t t = 1; t <= T; ++t) {
        const double tt = (double)t;
        g[t] = nn * std::exp(-gauss_rate * tt * tt) * std::sin(2.0 * M_PI * C * tt) / (M_PI * tt);
    }
}

// Runs f(lo, hi) over [0, count) in chunks of `grain` on all host cores.
template <typename F>
void parallel_for(uint64_t count, uint64_t grain, F f) {
    const uint64_t nchunk = (count + grain - 1) / grain;
    unsigned nth = std::thread::hardware_concurrency();
    if (nth == 0) nth = 1;
    if (nth > 64) nth = 64;
    if ((uint64_t)nth > nchunk) nth = (unsigned)(nchunk ? nchunk : 1);
    std::atomic<uint64_t> next{0};
    auto work = [&]() {
        for (;;) {
            const uint64_t c = next.fetch_add(1);
            if (c >= nchunk) break;
            f(c * grain, std::min(count, (c + 1) * grain));
        }
    };
    std::vector<std::thread> pool;
    for (unsigned i = 1; i < nth; ++i) pool.emplace_back(work);
    work();
    for (auto& th : pool) th.join();
}

// W(o) for o = 0..len-1 by direct summation.  Offsets are processed in blocks; within a block
// cos(2 pi o t / n) advances by a complex rotation per step of t and is re-anchored to an exactly
// reduced phase every 128 steps.
void window_table_direct(uint64_t n, const double* g, int64_t T, uint64_t len, double* W) {
    const uint64_t blk = 256;
    parallel_for((len + blk - 1) / blk, 1, [&](uint64_t b0, uint64_t b1) {
        std::vector<double> c(blk), s(blk), cr(blk), sr(blk), acc(blk);
        for (uint64_t bi = b0; bi < b1; ++bi) {
            const uint64_t o0 = bi * blk;
            const uint64_t m = std::min<uint64_t>(blk, len - o0);
            for (uint64_t q = 0; q < m; ++q) {
                const double th = 2.0 * M_PI * (double)(o0 + q) / (double)n;
                cr[q] = std::cos(th);
                sr[q] = std::sin(th);
                acc[q] = 0.0;
            }
            for (int64_t t0 = 1; t0 <= T; t0 += 128) {
                for (uint64_t q = 0; q < m; ++q) {  // exact anchor cos/sin(2 pi ((o t0) mod n) / n)
                    const uint64_t e = ((o0 + q) * (uint64_t)t0) & (n - 1);
                    const double ph = 2.0 * M_PI * (double)e / (double)n;
                    c[q] = std::cos(ph);
                    s[q] = std::sin(ph);
                }
                const int64_t t1 = std::min<int64_t>(T, t0 + 127);
                for (int64_t t = t0; t <= t1; ++t) {
                    const double gt = g[t];
                    for (uint64_t q = 0; q < m; ++q) {
                        acc[q] += gt * c[q];
                        const double cn = c[q] * cr[q] - s[q] * sr[q];
                        const double sn = s[q] * cr[q] + c[q] * sr[q];
                        c[q] = cn;
                        s[q] = sn;
                    }
                }
            }
            for (uint64_t q = 0; q < m; ++q) W[o0 + q] = (g[0] + 2.0 * acc[q]) / (double)n;
        }
    });
}

// In-place radix-2 FFT of a power-of-two length: a_j <- sum_m a_m e^{-+2 pi i j m / N} (unscaled),
// sign - forward, + inverse.  Twiddles come from exactly reduced angles; each stage's butterflies
// run on all host cores.
void fft_pow2(std::vector<std::complex<double>>& a, bool inverse) {
    const uint64_t N = a.size();
    uint32_t logN = 0;
    while ((uint64_t(1) << logN) < N) ++logN;
    parallel_for(N, uint64_t(1) << 16, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t i = lo; i < hi; ++i) {
            uint64_t r = 0;
            for (uint32_t b = 0; b < logN; ++b) r |= ((i >> b) & 1u) << (logN - 1 - b);
            if (r > i) std::swap(a[i], a[r]);
        }
    });
    std::vector<std::complex<double>> tw(N / 2 > 0 ? N / 2 : 1);
    const double sgn = inverse ? 1.0 : -1.0;
    parallel_for(N / 2, uint64_t(1) << 16, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t j = lo; j < hi; ++j) {
            const double ang = 2.0 * M_PI * (double)j / (double)N;
            tw[j] = std::complex<double>(std::cos(ang), sgn * std::sin(ang));
        }
    });
    for (uint64_t len = 2; len <= N; len <<= 1) {
        const uint64_t half = len / 2, step = N / len;
        parallel_for(N / 2, uint64_t(1) << 15, [&](uint64_t lo, uint64_t hi) {
            for (uint64_t bf = lo; bf < hi; ++bf) {
                const uint64_t grp = bf / half, j = bf - grp * half;
                const uint64_t i0 = grp * len + j, i1 = i0 + half;
                const std::complex<double> v = a[i1] * tw[j * step];
                a[i1] = a[i0] - v;
                a[i0] = a[i0] + v;
            }
        });
    }
}

// W(o) for o = 0..len-1 as one chirp convolution (Bluestein): with c(m) = e^{-i pi m^2 / n},
// e^{-2 pi i o t / n} = c(o) c(t) conj(c(o - t)), so sum_t g_|t| e^{-2 pi i o t / n} =
// c(o) (A * H)[o + 2T] with A[t + T] = g_|t| c(t) (|t| <= T) and H[u] = conj(c(u - T)),
// 0 <= u < len + 2T; a circular convolution of length N >= len + 4T equals the linear one there.
// m^2 is reduced mod 2n in integers before the angle is formed.
void window_table_chirp(uint64_t n, const double* g, int64_t T, uint64_t len, double* W) {
    const uint64_t L = 2 * (uint64_t)T + 1, U = len + 2 * (uint64_t)T;
    uint64_t N = 1;
    while (N < len + 4 * (uint64_t)T) N <<= 1;
    const uint64_t two_n = 2 * n;
    auto chirp = [&](int64_t m) {
        const uint64_t am = (uint64_t)(m < 0 ? -m : m);
        const uint64_t r = (am * am) % two_n;  // |m| < 2^31 (len + 2T < n <= 2^30)
        const double ang = M_PI * (double)r / (double)n;
        return std::complex<double>(std::cos(ang), -std::sin(ang));
    };
    std::vector<std::complex<double>> A(N), H(N);
    parallel_for(N, uint64_t(1) << 16, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t i = lo; i < hi; ++i) {
            const int64_t t = (int64_t)i - T;
            A[i] = i < L ? g[t < 0 ? -t : t] * chirp(t) : std::complex<double>(0.0, 0.0);
            H[i] = i < U ? std::conj(chirp((int64_t)i - T)) : std::complex<double>(0.0, 0.0);
        }
    });
    fft_pow2(A, false);
    fft_pow2(H, false);
    parallel_for(N, uint64_t(1) << 16, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t i = lo; i < hi; ++i) A[i] *= H[i];
    });
    fft_pow2(A, true);
    parallel_for(len, uint64_t(1) << 16, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t o = lo; o < hi; ++o)
            W[o] = (chirp((int64_t)o) * A[o + 2 * (uint64_t)T]).real() / ((double)N * (double)n);
    });
}

// The paper's closed-form gain Ghat'(o) for o = 0..len-1 (Sec. 7): 1 for |o| <= (1 - alpha) n / 2B,
// 0 for |o| >= n / 2B, and Phi((s + C) / sig_f) - Phi((s - C) / sig_f), s = o / n, in between, with
// the window's C = (1 - alpha/2) / 2B and sig_f = alpha / (4 B z), z = sqrt(2 ln(1/delta)).
// exp(-2 pi i m / n) for an integer m in [0, n), n a power of two: the angle is reduced to the first
// octant exactly (m / n is an exact binary fraction) before one cos and one sin are taken
static double2 root_of_unity(uint64_t m, uint64_t n) {
    const uint64_t q = n / 8;  // n >= 64
    const uint64_t oct = m / q, r = m % q;
    // angle = 2 pi (oct q + r) / n = oct pi / 4 + 2 pi r / n; fold into [0, pi/4] with a sign/swap table
    const double th = 2.0 * M_PI * (double)r / (double)n;  // in [0, pi/4)
    const double c = std::cos(th), s = std::sin(th), h = std::sqrt(0.5);
    double re = 0, im = 0;  // cos and sin of the full angle
    switch (oct) {
        case 0: re = c; im = s; break;
        case 1: re = h * (c - s); im = h * (c + s); break;
        case 2: re = -s; im = c; break;
        case 3: re = -h * (c + s); im = h * (c - s); break;
        case 4: re = -c; im = -s; break;
        case 5: re = -h * (c - s); im = -h * (c + s); break;
        case 6: re = s; im = -c; break;
        default: re = h * (c + s); im = -h * (c - s); break;
    }
    return make_double2(re, -im);
}

void twiddle_tables_host(uint64_t n, uint32_t sh, std::vector<double2>* out) {
    const uint64_t lo = uint64_t(1) << sh, hi = n >> sh;
    out->resize(lo + hi);
    for (uint64_t b = 0; b < lo; ++b) (*out)[b] = root_of_unity(b, n);
    for (uint64_t a = 0; a < hi; ++a) (*out)[lo + a] = root_of_unity(a << sh, n);
}

void window_gprime_host(uint64_t n, uint32_t B, double alpha, double delta, uint64_t len, double* W) {
    const double nn = (double)n, z = std::sqrt(2.0 * std::log(1.0 / delta));
    const double C = (1.0 - alpha / 2.0) / (2.0 * (double)B), sf = alpha / (4.0 * (double)B * z);
    auto cdf = [](double v) { return 0.5 * std::erfc(-v / std::sqrt(2.0)); };
    for (uint64_t o = 0; o < len; ++o) {
        const double ao = (double)o;
        if (ao <= (1.0 - alpha) * nn / (2.0 * (double)B))
            W[o] = 1.0;
        else if (ao >= nn / (2.0 * (double)B))
            W[o] = 0.0;
        else
            W[o] = cdf((ao / nn + C) / sf) - cdf((ao / nn - C) / sf);
    }
}

// Exact response of the truncated taps, W(o) = (1/n) (g_0 + 2 sum_{t=1}^{T} g_t cos(2 pi o t / n)),
// for o = 0..len-1 (the gain HashToBins applies to a coefficient at offset o from its bin centre):
// by direct summation when len T is small, else by the chirp convolution (O((len + T) log)).
void window_table_host(uint64_t n, const double* g, int64_t T, uint64_t len, double* W) {
    uint64_t N = 1;
    while (N < len + 4 * (uint64_t)T) N <<= 1;
    uint32_t logN = 0;
    while ((uint64_t(1) << logN) < N) ++logN;
    const double direct = (double)len * (double)T, chirp = 16.0 * (double)N * (double)logN;
    if (direct <= chirp)
        window_table_direct(n, g, T, len, W);
    else
        window_table_chirp(n, g, T, len, W);
}

void draw_exact_host(uint64_t seed, uint32_t request, uint32_t round, uint64_t n, uint64_t* sigma, uint64_t* b) {
    uint32_t s, bb;
    exact_hash(seed, request, round, (uint32_t)(n - 1), &s, &bb);
    *sigma = s;
    *b = bb;
}

// Exact schedule (Algorithm 1, NoiselessSparseFFT): rounds t = 0..ceil(log2 k) (+ extra),
// k_t = ceil(k / 2^t), B_t = pow2 >= bins_per_k k_t in [B_min, n/2], alpha_t = alpha0 2^{-t/2}.
// Location ladder: shifts beta_l = B R_l, R_0 = 1, coarsest R = pow2 >= tau n / (pi B) (at most
// n/(2B)), consecutive ratios at most the largest power of two rho with pi / rho >= tau.
sfft_status build_exact_schedule(sfft_plan_s* pl) {
    const sfft_params& p = pl->p;
    const bool fp64 = p.precision == SFFT_FP64;
    const uint32_t R = ceil_log2(p.k) + 1 + p.extra_rounds;
    pl->rounds.clear();
    pl->taps_host.clear();
    pl->wtab_host.clear();
    size_t taps_off = 0, wtab_off = 0;
    for (uint32_t t = 0; t < R; ++t) {
        ExactRound r;
        uint64_t kt = ((uint64_t)p.k + (uint64_t(1) << t) - 1) >> t;
        if (kt < 1) kt = 1;
        uint64_t B = pow2_at_least(p.bins_per_k * (double)kt);
        if (B < p.B_min) B = p.B_min;
        if (B > p.n / 2) B = p.n / 2;
        if (B > kMaxB) return SFFT_ERR_K_RANGE;
        r.B = (uint32_t)B;
        r.logB = ceil_log2(B);
        r.alpha = std::ldexp(p.alpha0, -(int)(t / 2)) * ((t & 1u) ? M_SQRT1_2 : 1.0);
        r.T = window_halfwidth(r.B, r.alpha, p.delta);
        // ladder
        const uint64_t Np = p.n / B;
        uint64_t Rc = pow2_at_least(p.tau_dec * (double)p.n / (M_PI * (double)B));
        if (Rc > Np / 2) Rc = Np / 2 > 0 ? Np / 2 : 1;
        uint64_t rho = 1;
        while (M_PI / (double)(rho * 2) >= p.tau_dec) rho *= 2;
        if (rho < 2) rho = 2;
        r.nshift = 0;
        uint64_t Rl = 1;
        r.shift[r.nshift++] = B * Rl;
        while (Rl < Rc && r.nshift < 4) {
            Rl = Rl * rho < Rc ? Rl * rho : Rc;
            r.shift[r.nshift++] = B * Rl;
        }
        if (1 + r.nshift > (uint32_t)kMaxHash) return SFFT_ERR_K_RANGE;
        const uint64_t maxshift = r.shift[r.nshift - 1];
        if (maxshift > 8192) return SFFT_ERR_K_RANGE;
        const uint64_t w = 2 * (uint64_t)r.T + 1;
        r.ctaps = p.chunk_taps ? p.chunk_taps : (uint32_t)kChunkTaps;
        r.chunks = (uint32_t)((w + r.ctaps - 1) / r.ctaps);
        r.stage = (uint32_t)(r.ctaps + maxshift);
        r.taps_off = taps_off;
        r.wtab_off = wtab_off;
        const size_t gs = exact_gather_smem(r.stage, fp64) + (size_t)(1 + r.nshift) * (B > (uint64_t)kThreads ? B : kThreads) *
                                                              (fp64 ? 16 : 8);
        const size_t fs = exact_finish_smem(r.B, 1 + r.nshift, p.z_cap, fp64);
        // a finisher that does not fit next to the gather's staging keeps its arrays in device memory
        r.fin_bytes = fs;
        r.fin_global = fs > kFinSmemMax;
        r.smem = r.fin_global ? gs : (gs > fs ? gs : fs);
        if (r.smem > 200 * 1024) return SFFT_ERR_K_RANGE;
        pl->taps_host.resize(taps_off + (size_t)r.T + 1);
        window_taps_host(p.n, r.B, r.alpha, p.delta, r.T, pl->taps_host.data() + taps_off);
        pl->wtab_host.resize(wtab_off + 2 * (Np / 2 + 1));
        double* W = pl->wtab_host.data() + wtab_off;
        if (p.gain == 1)
            window_gprime_host(p.n, r.B, r.alpha, p.delta, Np / 2 + 1, W);
        else
            window_table_host(p.n, pl->taps_host.data() + taps_off, r.T, Np / 2 + 1, W);
        // 1 / W(o) beside W: the FP32 data path forms a decoded value as u_0 times this (the decode
        // reads it only where W(o) >= gmin > 0)
        for (uint64_t o = 0; o <= Np / 2; ++o) W[Np / 2 + 1 + o] = W[o] != 0.0 ? 1.0 / W[o] : 0.0;
        taps_off += (size_t)r.T + 1;
        wtab_off += 2 * (Np / 2 + 1);
        pl->rounds.push_back(r);
    }
    pl->wtab_len = wtab_off;
    return SFFT_OK;
}

// General schedule (Algorithm 2, SparseFFT): k_0 = k, k_{r+1} = floor(k_r / 4) down to 1;
// B_r = pow2 >= bins_per_k k_r / eps in [B_min, n/2]; alpha = alpha0 in every round; EstimateValues
// keeps k' = 3 k_r.  LocateSignal (Algorithm 3): t = largest power of two <= log2 n (or t_regions),
// t' = t/4, w_0 = n/B, D_max = floor(log_{t'} w_0) + 1, and at level D (width w_D = w_0 / t'^{D-1})
// beta is uniform on {ceil(s n t / 4 w_D), ..., floor(s n t / 2 w_D)}.
sfft_status build_general_schedule(sfft_plan_s* pl) {
    const sfft_params& p = pl->p;
    pl->grounds.clear();
    pl->taps_host.clear();
    pl->wtab_host.clear();
    const uint32_t logn = ceil_log2(p.n);
    uint32_t t = p.t_regions;
    if (t == 0) {
        t = 1;
        while (t * 2 <= logn) t *= 2;
    }
    if (t < 8 || t > (uint32_t)kMaxT || (t & (t - 1))) return SFFT_ERR_INVALID_ARG;
    if (p.R_loc == 0 || p.R_loc > (uint32_t)kMaxRloc || p.R_est == 0 || p.R_est > (uint32_t)kMaxRest)
        return SFFT_ERR_INVALID_ARG;
    if (p.z_cap > 4096) return SFFT_ERR_INVALID_ARG;
    const uint32_t tp = t / 4, logtp = ceil_log2(tp);
    size_t taps_off = 0, wtab_off = 0;
    for (uint64_t kr = p.k; kr >= 1; kr /= 4) {
        GeneralRound r;
        r.kr = (uint32_t)kr;
        r.kprime = 3 * r.kr;
        uint64_t B = pow2_at_least(p.bins_per_k * (double)kr / p.eps);
        if (B < p.B_min) B = p.B_min;
        if (B > p.n / 2) B = p.n / 2;
        if (B > kMaxB) return SFFT_ERR_K_RANGE;
        r.B = (uint32_t)B;
        r.logB = ceil_log2(B);
        r.T = window_halfwidth(r.B, p.alpha0, p.delta);
        r.chunks = (uint32_t)((2 * (uint64_t)r.T + 1 + kChunkTaps - 1) / kChunkTaps);
        r.cpb = r.chunks < 4 ? r.chunks : 4;  // chunks per gather CTA: 4 beat 2 and 8 at n = 2^22, k = 256
        r.ctas = (r.chunks + r.cpb - 1) / r.cpb;
        r.t = t;
        r.logtp = logtp;
        const uint32_t lw = ceil_log2(p.n / B);
        r.dmax = lw / logtp + 1;
        if (r.dmax > (uint32_t)kMaxLevels) return SFFT_ERR_K_RANGE;
        for (uint32_t D = 1; D <= r.dmax; ++D) {
            const uint64_t w = (p.n / B) >> ((uint64_t)(D - 1) * logtp);
            const double base = p.s * (double)p.n * (double)t / (double)w;
            uint64_t lo = (uint64_t)std::ceil(base / 4.0), hi = (uint64_t)std::floor(base / 2.0);
            if (hi < lo) hi = lo;
            if (hi - lo >= (uint64_t(1) << 32)) return SFFT_ERR_K_RANGE;
            r.beta_lo[D - 1] = lo;
            r.beta_hi[D - 1] = hi;
        }
        r.npairs = r.dmax * p.R_loc;
        // the pairs share the round's sigma: when they gather >= 2n samples, one in-order pass that
        // writes x_{sigma m} costs less than the random reads it replaces
        r.perm = p.permuted_copy == 0 && 2 * (uint64_t)r.npairs * (2 * (uint64_t)r.T + 1) >= 2 * p.n;
        r.ngroups = r.npairs + p.R_est;
        r.nhash = 2 * r.npairs + p.R_est;
        r.taps_off = taps_off;
        r.wtab_off = wtab_off;
        r.smem_gather = (size_t)2 * kChunkTaps * 8 + (size_t)2 * (B > (uint64_t)kThreads ? B : kThreads) * 8;
        r.smem_finish = general_finish_smem(r.B, p.z_cap);
        r.smem_locate = general_locate_smem(r.B);
        r.smem_estimate = general_estimate_smem(r.B, r.kprime, p.z_cap);
        // arrays beyond kFinSmemMax go to device memory, one slice per CTA: the finish's per (request,
        // group), the estimate's per request (its launch then gives each request a single CTA)
        r.fin_global = r.smem_finish > kFinSmemMax;
        r.est_global = r.smem_estimate > kFinSmemMax;
        if (r.smem_gather > 200 * 1024 || r.smem_locate > 200 * 1024) return SFFT_ERR_K_RANGE;
        const uint64_t Np = p.n / B;
        pl->taps_host.resize(taps_off + (size_t)r.T + 1);
        window_taps_host(p.n, r.B, p.alpha0, p.delta, r.T, pl->taps_host.data() + taps_off);
        pl->wtab_host.resize(wtab_off + Np / 2 + 1);
        if (p.gain == 1)
            window_gprime_host(p.n, r.B, p.alpha0, p.delta, Np / 2 + 1, pl->wtab_host.data() + wtab_off);
        else
            window_table_host(p.n, pl->taps_host.data() + taps_off, r.T, Np / 2 + 1, pl->wtab_host.data() + wtab_off);
        taps_off += (size_t)r.T + 1;
        wtab_off += Np / 2 + 1;
        pl->grounds.push_back(r);
        if (kr < 4) break;
    }
    pl->wtab_len = wtab_off;
    return SFFT_OK;
}

}  // namespace sfft

extern "C" {

void sfft_params_default(sfft_params* p, uint64_t n, uint32_t k, uint32_t mode) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n = n;
    p->k = k;
    p->mode = mode;
    p->precision = SFFT_FP32;
    p->delta = 1e-6;
    p->alpha0 = 0.5;
    p->bins_per_k = mode == SFFT_GENERAL ? 8.0 : 4.0;
    p->B_min = 16;
    p->extra_rounds = 0;
    p->thr = 0.5;
    p->tau_dec = 1e-4;
    p->iso_tol = 1e-3;
    p->gmin = 0.1;
    p->prune = 0.5;
    p->ref_lo = 1e-5;
    p->ref_hi = 2e-2;
    p->ref_tol = 0.1;
    p->z_cap = mode == SFFT_GENERAL ? (k * 8 > 64 ? k * 8 : 64) : (k * 4 > 64 ? k * 4 : 64);
    p->eps = 1.0;
    p->t_regions = 0;
    p->R_loc = mode == SFFT_GENERAL ? 7 : 5;
    p->R_est = 5;
    p->s = 0.25;
    p->est_gmin = 0.25;
    p->streams = mode == SFFT_GENERAL ? 4 : 1;  // exact: one launch per batch already overlaps its rounds
    p->gain = 0;
    p->chunk_taps = 2048;
}

const char* sfft_status_str(sfft_status s) {
    switch (s) {
        case SFFT_OK: return "ok";
        case SFFT_ERR_INVALID_ARG: return "invalid argument";
        case SFFT_ERR_N_NOT_POW2: return "n is not a power of two in [2^6, 2^30]";
        case SFFT_ERR_K_RANGE: return "k out of the supported range";
        case SFFT_ERR_OOM: return "device out of memory";
        case SFFT_ERR_CUDA: return "CUDA error";
        case SFFT_ERR_TIMEOUT: return "timeout";
        case SFFT_ERR_CAPACITY: return "zhat capacity exceeded";
        case SFFT_ERR_NOT_CONVERGED: return "not converged";
        case SFFT_ERR_BUSY: return "busy";
    }
    return "unknown status";
}

const char* sfft_last_error(void) { return sfft::g_last_error.c_str(); }

sfft_status sfft_window_taps(uint64_t n, uint32_t B, double alpha, double delta, int64_t* T, double* h_taps,
                             uint64_t cap) {
    if (!T || n < 64 || (n & (n - 1)) || B < 2 || (B & (B - 1)) || B > n / 2) return SFFT_ERR_INVALID_ARG;
    if (!(alpha > 0 && alpha < 1) || !(delta > 0 && delta < 0.5)) return SFFT_ERR_INVALID_ARG;
    *T = sfft::window_halfwidth(B, alpha, delta);
    if (!h_taps) return SFFT_OK;
    if (cap < (uint64_t)*T + 1) return SFFT_ERR_INVALID_ARG;
    sfft::window_taps_host(n, B, alpha, delta, *T, h_taps);
    return SFFT_OK;
}

sfft_status sfft_twiddle_tables(uint64_t n, uint64_t* len, double* h_tw, uint64_t cap) {
    if (!len || n < 64 || n > (uint64_t(1) << 30) || (n & (n - 1))) return SFFT_ERR_INVALID_ARG;
    const uint32_t sh = (sfft::ilog2_host(n) + 1) / 2;
    const uint64_t m = (uint64_t(1) << sh) + (n >> sh);
    *len = m;
    if (!h_tw) return SFFT_OK;
    if (cap < m) return SFFT_ERR_INVALID_ARG;
    std::vector<double2> tw;
    sfft::twiddle_tables_host(n, sh, &tw);
    for (uint64_t i = 0; i < m; ++i) {
        h_tw[2 * i] = tw[i].x;
        h_tw[2 * i + 1] = tw[i].y;
    }
    return SFFT_OK;
}

sfft_status sfft_window_gains(uint64_t n, uint32_t B, double alpha, double delta, uint64_t len, double* h_W) {
    int64_t T = 0;
    const sfft_status st = sfft_window_taps(n, B, alpha, delta, &T, nullptr, 0);
    if (st != SFFT_OK) return st;
    if (!h_W || len == 0 || len > n / 2 + 1) return SFFT_ERR_INVALID_ARG;
    std::vector<double> g((size_t)T + 1);
    sfft::window_taps_host(n, B, alpha, delta, T, g.data());
    sfft::window_table_host(n, g.data(), T, len, h_W);
    return SFFT_OK;
}

}  // extern "C"
