/*
 * sfft_oracle.c -- a plain, slow, FP64 CPU restatement of the sparse Fourier transform of
 * Hassanieh, Indyk, Katabi and Price, "Nearly Optimal Sparse Fourier Transform" (2012).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the CPU-baseline leg of
 * the benchmark are the only callers.  The GPU library neither links nor includes anything from
 * here; the two implementations share no code, header, table or constant generator.
 *
 * Every function below follows the paper's steps in the paper's order, in double precision,
 * without blocking, fusion or reordering.  Where the paper leaves a choice open (a Theta(.)
 * constant, a rounding rule, a tie) the reading taken is stated at the point of use.
 *
 * Conventions (Sec. 2, "Notation"):
 *   - n = 2^m; every index is 0-based and taken mod n.
 *   - w = exp(-2 pi i / n).  X = DFT(x) is the unnormalised transform X_f = sum_t x_t w^{f t};
 *     the paper's unitary spectrum is X / sqrt(n).  Only the reporting scale differs, so the
 *     window taps carry a factor n (see window_taps) and a single tone of amplitude X_i lands in
 *     its bin with amplitude X_i.
 *   - phase(z) lies in [0, 2 pi).
 *   - pi(i) = sigma (i - b) mod n; h(i) = round(pi(i) B / n) mod B with ties rounded up;
 *     o(i) = pi(i) - h(i) n / B, taken in [-n/2B, n/2B).   (Sec. 3, definitions of bin/offset)
 *
 * Random choices (sigma, a, b, beta) come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011) keyed by the request seed, with the
 * counter naming (round, sub-step, kind, request).  The mapping from 32-bit words to the ranges
 * the paper asks for is written out in draw_* below.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC 2011, Sec. 4 "Philox").                                    */
/* ------------------------------------------------------------------------------------------ */

/* One Philox-4x32 round: two 32x32->64 multiplies, the high halves xor-ed with the other two
 * counter words and the round key, the words permuted. */
static void philox_round(uint32_t c[4], const uint32_t key[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ c[1] ^ key[0];
    const uint32_t y2 = hi0 ^ c[3] ^ key[1];
    c[0] = y0;
    c[1] = lo1;
    c[2] = y2;
    c[3] = lo0;
}

/* Ten rounds; the key is bumped by the Weyl constants before every round but the first. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t kk[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            kk[0] += 0x9E3779B9u;
            kk[1] += 0xBB67AE85u;
        }
        philox_round(c, kk);
    }
    memcpy(out, c, sizeof c);
}

/* Counter layout: (c0, c1, c2, c3) = (round, sub-step, kind, request index); key = seed. */
enum { OR_KIND_EXACT = 0, OR_KIND_LOCATE = 1, OR_KIND_INNER = 2, OR_KIND_ESTIMATE = 3 };

static void draw_words(uint64_t seed, uint32_t stream, uint32_t round, uint32_t sub, uint32_t kind,
                       uint32_t out[4]) {
    const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {round, sub, kind, stream};
    or_philox4x32_10(ctr, key, out);
}

/* uniform on [0, n) (n a power of two <= 2^32) */
static uint64_t draw_mod_n(uint32_t word, uint64_t n) { return (uint64_t)word & (n - 1); }
/* uniform on the odd numbers of [0, n) */
static uint64_t draw_odd(uint32_t word, uint64_t n) { return ((uint64_t)word & (n - 1)) | 1u; }
/* uniform on the integers lo..hi (hi - lo < 2^32): multiply-shift of the 32-bit word */
static uint64_t draw_range(uint32_t word, uint64_t lo, uint64_t hi) {
    const uint64_t span = hi - lo + 1;
    return lo + (((uint64_t)word * span) >> 32);
}

/* sigma^{-1} mod 2^64 by Newton's iteration y <- y (2 - sigma y); sigma odd.  y = sigma is
 * correct to 3 bits and each step doubles the number of correct bits. */
uint64_t or_inverse_mod_pow2(uint64_t sigma, uint64_t n) {
    uint64_t y = sigma;
    for (int it = 0; it < 6; ++it) y = y * (2u - sigma * y);
    return y & (n - 1);
}

/* ------------------------------------------------------------------------------------------ */
/* Small integer helpers                                                                       */
/* ------------------------------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t n) { return ((a & (n - 1)) * (b & (n - 1))) & (n - 1); }
static uint64_t pow2ceil(double v) {
    uint64_t p = 1;
    while ((double)p < v) p <<= 1;
    return p;
}
static int ilog2(uint64_t v) {
    int l = 0;
    while (((uint64_t)1 << l) < v) ++l;
    return l;
}
/* exp(-2 pi i e / n) for an exact integer exponent e in [0, n) */
static cplx root_pow(uint64_t e, uint64_t n) {
    const double ang = OR_TWO_PI * (double)e / (double)n;
    return cos(ang) - I * sin(ang);
}
static double phase01(cplx z) { /* phase(z) / 2pi in [0, 1) */
    double p = atan2(cimag(z), creal(z)) / OR_TWO_PI;
    if (p < 0) p += 1.0;
    if (p >= 1.0) p -= 1.0;
    return p;
}

/* ------------------------------------------------------------------------------------------ */
/* Flat window (Definition in Sec. 2; construction in Sec. 7, "Efficient Constructions of      */
/* Window Functions").                                                                         */
/* ------------------------------------------------------------------------------------------ */
/*
 * Reading of the construction (its 2 pi factors are garbled in the text):
 *   z      = sqrt(2 ln(1/delta))                     (Claim "cdf", part 3: cdf(-z) < delta)
 *   C      = (1 - alpha/2) / (2B)                    (box-car half width, cycles per sample)
 *   sig_f  = alpha / (4 B z)                         (std of the Gaussian in frequency)
 *   Ghat*(s) = cdf((s + C)/sig_f) - cdf((s - C)/sig_f)   (Gaussian convolved with the box-car)
 *   G*(t)  = exp(-2 pi^2 sig_f^2 t^2) * sin(2 pi C t) / (pi t)   (its inverse transform)
 * so Ghat* drops from 1 - delta to delta across [(1-alpha)/(2B), 1/(2B)], matching the four
 * bullet properties of the flat-window definition.  The taps are truncated where the Gaussian
 * factor falls to delta:  |t| <= T = floor(z / (2 pi sig_f)) = floor(4 B ln(1/delta) / (pi alpha)).
 * The config's delta is used as the target directly (no delta -> delta/n substitution).
 */
int64_t or_window_T(uint64_t n, uint32_t B, double alpha, double delta) {
    (void)n;
    const double T = 4.0 * (double)B * log(1.0 / delta) / (M_PI * alpha);
    return (int64_t)floor(T);
}

/* taps g[t] for t = 0..T (the window is even: g[-t] = g[t]); g_t = n G*(t) */
void or_window_taps(uint64_t n, uint32_t B, double alpha, double delta, int64_t T, double* g) {
    const double z = sqrt(2.0 * log(1.0 / delta));
    const double C = (1.0 - alpha / 2.0) / (2.0 * (double)B);
    const double sf = alpha / (4.0 * (double)B * z);
    g[0] = (double)n * 2.0 * C;
    for (int64_t t = 1; t <= T; ++t) {
        const double tt = (double)t;
        const double gauss = exp(-2.0 * M_PI * M_PI * sf * sf * tt * tt);
        const double boxcar = sin(2.0 * M_PI * C * tt) / (M_PI * tt);
        g[t] = (double)n * gauss * boxcar;
    }
}

/* Exact response of the truncated taps at frequency offset l:
 *   W(l) = (1/n) sum_{t=-T}^{T} g_t w^{l t} = (1/n) (g_0 + 2 sum_{t>=1} g_t cos(2 pi l t / n)).
 * This is the Ghat that HashToBins actually applies (Lemma "hashtobins", first display). */
double or_window_response(uint64_t n, int64_t T, const double* g, int64_t l) {
    const uint64_t lm = (uint64_t)l & (n - 1);
    double s = g[0];
    for (int64_t t = 1; t <= T; ++t) {
        const uint64_t e = mulmod(lm, (uint64_t)t, n);
        s += 2.0 * g[t] * cos(OR_TWO_PI * (double)e / (double)n);
    }
    return s / (double)n;
}

static double std_normal_cdf(double x) { return 0.5 * erfc(-x / M_SQRT2); }

/* The paper's Ghat'_l (Sec. 7, the three-case definition): 1 on the pass band, 0 outside the
 * bin, the difference of Gaussian cdfs in between. */
double or_window_gprime(uint64_t n, uint32_t B, double alpha, double delta, int64_t l) {
    int64_t lc = (int64_t)((uint64_t)l & (n - 1));
    if (lc >= (int64_t)(n / 2)) lc -= (int64_t)n; /* |l| as in Sec. 2 */
    const double al = fabs((double)lc);
    const double nn = (double)n;
    if (al <= (1.0 - alpha) * nn / (2.0 * (double)B)) return 1.0;
    if (al >= nn / (2.0 * (double)B)) return 0.0;
    const double z = sqrt(2.0 * log(1.0 / delta));
    const double C = (1.0 - alpha / 2.0) / (2.0 * (double)B);
    const double sf = alpha / (4.0 * (double)B * z);
    const double s = (double)lc / nn;
    return std_normal_cdf((s + C) / sf) - std_normal_cdf((s - C) / sf);
}

/* A window with a lazily filled cache of W(o) for the offsets o in [0, n/2B]. */
typedef struct {
    uint64_t n;
    uint32_t B;
    double alpha, delta;
    int64_t T;
    double* g;       /* T+1 taps */
    double* wcache;  /* n/(2B)+1 entries */
    uint8_t* wdone;
} or_window;

static void window_init(or_window* W, uint64_t n, uint32_t B, double alpha, double delta) {
    W->n = n;
    W->B = B;
    W->alpha = alpha;
    W->delta = delta;
    W->T = or_window_T(n, B, alpha, delta);
    W->g = (double*)malloc(sizeof(double) * (size_t)(W->T + 1));
    or_window_taps(n, B, alpha, delta, W->T, W->g);
    const size_t nc = (size_t)(n / (2 * B)) + 1;
    W->wcache = (double*)calloc(nc, sizeof(double));
    W->wdone = (uint8_t*)calloc(nc, 1);
}
static void window_free(or_window* W) {
    free(W->g);
    free(W->wcache);
    free(W->wdone);
}
/* W(o) for |o| <= n/2B (the only offsets a bin ever sees); W is even. */
static double window_at(or_window* W, int64_t o) {
    const uint64_t a = (uint64_t)(o < 0 ? -o : o);
    if (!W->wdone[a]) {
        W->wcache[a] = or_window_response(W->n, W->T, W->g, (int64_t)a);
        W->wdone[a] = 1;
    }
    return W->wcache[a];
}

/* ------------------------------------------------------------------------------------------ */
/* Permutation P_{sigma,a,b} (Definition in Sec. 2)                                            */
/* ------------------------------------------------------------------------------------------ */
/* (P x)_t = x_{sigma (t - a)} w^{sigma b t} */
void or_permute(uint64_t n, const double* xin, uint64_t sigma, uint64_t a, uint64_t b, double* out) {
    const cplx* x = (const cplx*)xin;
    cplx* y = (cplx*)out;
    const uint64_t sb = mulmod(sigma, b, n);
    for (uint64_t t = 0; t < n; ++t) {
        const uint64_t src = mulmod(sigma, (t - a) & (n - 1), n);
        y[t] = x[src] * root_pow(mulmod(sb, t, n), n);
    }
}

/* bin h(i) and offset o(i) of a permuted position p = pi(i) (Sec. 3 definitions; ties of the
 * rounding go up, bin B wraps to 0, o in [-n/2B, n/2B)). */
static void bin_offset(uint64_t p, uint64_t n, uint32_t B, uint64_t* j, int64_t* o) {
    const uint64_t Np = n / B;
    const uint64_t jj = ((p + Np / 2) & (n - 1)) / Np;
    uint64_t d = (p - jj * Np) & (n - 1);
    int64_t oo = (int64_t)d;
    if (oo >= (int64_t)(n / 2)) oo -= (int64_t)n;
    *j = jj;
    *o = oo;
}
void or_bin_offset(uint64_t p, uint64_t n, uint32_t B, uint64_t* j, int64_t* o) { bin_offset(p, n, B, j, o); }

/* ------------------------------------------------------------------------------------------ */
/* HashToBins (Algorithm 1, procedure HashToBins; computed by the four-step method in the      */
/* proof of Lemma "hashtobins").                                                               */
/* ------------------------------------------------------------------------------------------ */
/*
 *   1. y_t = G_t (P_{sigma,a,b} x)_t for the 2T+1 taps t in [-T, T]
 *   2. v_r = sum_{t = r mod B} y_t
 *   3. u_j = sum_r v_r exp(-2 pi i j r / B)        (= yhat_{j n / B})
 *   4. for i in supp(zhat):  u_{h(i)} -= Ghat_{-o(i)} zhat_i w^{a sigma i}
 * Step 3 is the B-point DFT written out as its definition.  In step 4 the subtracted gain is the
 * exact response W of the taps (use_gprime = 0) or the paper's closed form Ghat' (use_gprime = 1).
 */
static void hash_to_bins(uint64_t n, const cplx* x, uint32_t nz, const uint64_t* zi, const cplx* zv,
                         uint64_t sigma, uint64_t a, uint64_t b, or_window* W, int use_gprime, cplx* u) {
    const uint32_t B = W->B;
    const int64_t T = W->T;
    cplx* v = (cplx*)calloc(B, sizeof(cplx));
    const uint64_t sb = mulmod(sigma, b, n);
    /* steps 1 and 2 */
    for (int64_t t = -T; t <= T; ++t) {
        const uint64_t tm = (uint64_t)t & (n - 1);
        const uint64_t src = mulmod(sigma, (tm - a) & (n - 1), n);
        const double g = W->g[t < 0 ? -t : t];
        const cplx y = g * x[src] * root_pow(mulmod(sb, tm, n), n);
        const uint64_t r = (uint64_t)t & (B - 1); /* t mod B, B | n */
        v[r] += y;
    }
    /* step 3 */
    for (uint32_t j = 0; j < B; ++j) {
        cplx s = 0;
        for (uint32_t r = 0; r < B; ++r) s += v[r] * root_pow(((uint64_t)j * r) & (B - 1), B);
        u[j] = s;
    }
    /* step 4 */
    for (uint32_t e = 0; e < nz; ++e) {
        const uint64_t i = zi[e] & (n - 1);
        const uint64_t p = mulmod(sigma, (i - b) & (n - 1), n);
        uint64_t j;
        int64_t o;
        bin_offset(p, n, B, &j, &o);
        const double gain = use_gprime ? or_window_gprime(n, B, W->alpha, W->delta, -o) : window_at(W, -o);
        const uint64_t ph = mulmod(mulmod(a, sigma, n), i, n);
        u[j] -= gain * zv[e] * root_pow(ph, n);
    }
    free(v);
}

/* Public wrapper: explicit taps are rebuilt from (B, alpha, delta). */
void or_hash_to_bins(uint64_t n, const double* x, uint32_t nz, const uint64_t* zi, const double* zv,
                     uint64_t sigma, uint64_t a, uint64_t b, uint32_t B, double alpha, double delta,
                     int use_gprime, double* u) {
    or_window W;
    window_init(&W, n, B, alpha, delta);
    hash_to_bins(n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, a, b, &W, use_gprime, (cplx*)u);
    window_free(&W);
}

/* ------------------------------------------------------------------------------------------ */
/* Parameters                                                                                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint64_t n;            /* signal length, a power of two */
    uint32_t k;            /* sparsity */
    uint32_t mode;         /* 0 = exactly k-sparse (Alg. 1), 1 = general (Alg. 2 and 3) */
    double delta;          /* window tolerance */
    double alpha0;         /* alpha of the first round */
    double bins_per_k;     /* B = pow2ceil(bins_per_k * k_t) (exact), pow2ceil(bins_per_k*k_r/eps) */
    uint32_t B_min;        /* smallest B used */
    uint32_t extra_rounds; /* exact: rounds after t = ceil(log2 k) */
    double thr;            /* exact: J = {j : |u_j| > thr} */
    double tau_dec;        /* exact: phase tolerance the location ladder must leave */
    double iso_tol;        /* exact: | |u^(beta)_j| - |u^(0)_j| | <= iso_tol |u^(0)_j| */
    double gmin;           /* exact: a decode needs W(-o) >= gmin */
    double prune;          /* exact: after a round drop zhat_i with |zhat_i| < prune * thr */
    double ref_lo, ref_hi; /* exact: residual window (times thr) for re-estimating a known value */
    double ref_tol;        /* exact: phase tolerance (rad) of that re-estimate */
    uint32_t z_cap;        /* capacity of zhat */
    double eps;            /* general: epsilon */
    uint32_t t_regions;    /* general: t (0 -> largest power of two <= log2 n) */
    uint32_t R_loc;        /* general: rounds of LocateInner per level */
    uint32_t R_est;        /* general: hashings of EstimateValues */
    double s;              /* general: vote half width s pi */
    double est_gmin;       /* general: a hashing joins the median only if W(-o) >= est_gmin */
} or_params;

/* ---- exact-mode schedule (Algorithm 1, procedure NoiselessSparseFFT) ---- */
/* Reading: rounds t = 0..ceil(log2 k) (+ extra); k_t = ceil(k / 2^t); B_t = pow2ceil(c k_t)
 * clamped to [B_min, n/2]; alpha_t = alpha0 2^{-t/2} (the Theta(2^{-t/2}) of the theorem's
 * running-time proof). */
uint32_t or_exact_rounds(const or_params* P) { return (uint32_t)ilog2(P->k) + 1 + P->extra_rounds; }

typedef struct {
    uint32_t B;
    double alpha;
    uint32_t nshift;      /* number of shifted hashings besides a = 0 (the ladder length L) */
    uint64_t shift[4];    /* beta_l = B R_l, finest first */
    uint64_t sigma, sigma_inv, b;
} or_exact_round;

static uint64_t exact_B(const or_params* P, uint32_t t) {
    uint64_t kt = ((uint64_t)P->k + ((uint64_t)1 << t) - 1) >> t;
    if (kt < 1) kt = 1;
    uint64_t B = pow2ceil(P->bins_per_k * (double)kt);
    if (B < P->B_min) B = P->B_min;
    if (B > P->n / 2) B = P->n / 2;
    return B;
}
static double exact_alpha(const or_params* P, uint32_t t) {
    return P->alpha0 * ldexp(1.0, -(int)(t / 2)) * ((t & 1u) ? M_SQRT1_2 : 1.0);
}

/*
 * Location ladder (reading of Algorithm 1's phase step for a delta that is not 1/(4 n^2 L)).
 * The paper compares the hashings at a = 0 and a = 1, whose phase difference 2 pi sigma i / n must
 * be known to within pi/n.  Here the shifts are beta_l = B R_l with R_0 = 1 < R_1 < ...: the phase
 * difference between a = 0 and a = beta_l is 2 pi R_l q / (n/B), q = sigma i mod n/B, and the bin
 * index supplies the rest of sigma i.  The coarsest ratio R_{L-1} is the smallest power of two with
 * pi B R_{L-1} / n >= tau_dec; consecutive ratios differ by at most the largest power of two rho
 * with pi / rho >= tau_dec, so every measurement keeps a phase tolerance of at least tau_dec.
 */
static void exact_ladder(const or_params* P, uint64_t B, or_exact_round* R) {
    const uint64_t Np = P->n / B;
    uint64_t Rc = pow2ceil(P->tau_dec * (double)P->n / (M_PI * (double)B));
    if (Rc > Np / 2) Rc = Np / 2 > 0 ? Np / 2 : 1;
    uint64_t rho = 1;
    while (M_PI / (double)(rho * 2) >= P->tau_dec) rho *= 2;
    if (rho < 2) rho = 2;
    R->nshift = 0;
    uint64_t Rl = 1;
    R->shift[R->nshift++] = B * Rl;
    while (Rl < Rc && R->nshift < 4) {
        Rl = Rl * rho < Rc ? Rl * rho : Rc;
        R->shift[R->nshift++] = B * Rl;
    }
}

void or_exact_round_params(const or_params* P, uint64_t seed, uint32_t stream, uint32_t t, uint32_t* B,
                           double* alpha, int64_t* T, uint32_t* nshift, uint64_t* shifts, uint64_t* sigma,
                           uint64_t* sigma_inv, uint64_t* b) {
    or_exact_round R;
    R.B = (uint32_t)exact_B(P, t);
    R.alpha = exact_alpha(P, t);
    exact_ladder(P, R.B, &R);
    uint32_t wd[4];
    draw_words(seed, stream, t, 0, OR_KIND_EXACT, wd);
    R.sigma = draw_odd(wd[0], P->n);
    R.b = draw_mod_n(wd[1], P->n);
    R.sigma_inv = or_inverse_mod_pow2(R.sigma, P->n);
    *B = R.B;
    *alpha = R.alpha;
    *T = or_window_T(P->n, R.B, R.alpha, P->delta);
    *nshift = R.nshift;
    for (uint32_t l = 0; l < R.nshift; ++l) shifts[l] = R.shift[l];
    *sigma = R.sigma;
    *sigma_inv = R.sigma_inv;
    *b = R.b;
}

/* ------------------------------------------------------------------------------------------ */
/* Exact location and estimation of one round (Algorithm 1, procedure                          */
/* NoiselessSparseFFTInner, loop over J), on given bins.                                       */
/* ------------------------------------------------------------------------------------------ */
/*
 * u0 = bins of P_{sigma,0,b}; us[l] = bins of P_{sigma,beta_l,b}.  For every j with |u0_j| > thr
 * in ascending j: decode q = sigma i mod n/B from the ladder (coarsest first), place pi(i) inside
 * bin j, and form i = sigma^{-1}(pi(i) + sigma b).  Reading of "v <- round(u_j)" for non-integer
 * coefficients: v = u0_j / W(-o(i)).  A decode is kept only if W(-o(i)) >= gmin and every shifted
 * bin has the magnitude of u0_j to within iso_tol (an isolated coefficient only changes phase
 * under a shift; Lemma "l:est").
 *
 * Re-estimation of known values (the non-integer counterpart of round(): with integer
 * coefficients a small contamination of a value by a neighbour at the edge of the pass band is
 * rounded away; here it would stay below thr for ever).  For a bin with ref_lo thr < |u0_j| <=
 * ref_hi thr, every entry i of zhat hashed to bin j is a candidate: it matches when the shifted
 * bins keep the magnitude of u0_j to 25% and every phase difference agrees with location i to
 * within ref_tol.  When exactly one candidate matches, u0_j / W(-o(i)) is added to zhat_i.
 *
 * Returns the number of entries written to (wi, wv); *n_above = |J|, *n_kept = kept decodes of J.
 */
static int refine_known(uint64_t n, uint32_t B, uint64_t sigma, uint64_t b, uint32_t nshift, const uint64_t* shift,
                        const cplx* u0, const cplx* const* us, or_window* W, const or_params* P, uint32_t j, uint64_t i,
                        cplx* val) {
    const double mag0 = cabs(u0[j]);
    const uint64_t p = mulmod(sigma, (i - b) & (n - 1), n);
    uint64_t jj;
    int64_t o;
    bin_offset(p, n, B, &jj, &o);
    const double gain = window_at(W, -o);
    if (!(gain >= P->gmin)) return 0;
    for (uint32_t l = 0; l < nshift; ++l) {
        if (fabs(cabs(us[l][j]) - mag0) > 0.25 * mag0) return 0;
        const double pred = (double)mulmod(mulmod(shift[l], sigma, n), i, n) / (double)n;
        double d = fabs(phase01(u0[j] * conj(us[l][j])) - pred);
        if (d > 0.5) d = 1.0 - d;
        if (!(d * OR_TWO_PI < P->ref_tol)) return 0;
    }
    *val = u0[j] / gain;
    return 1;
}

static uint32_t exact_decode(uint64_t n, uint32_t B, uint64_t sigma, uint64_t sigma_inv, uint64_t b,
                             uint32_t nshift, const uint64_t* shift, const cplx* u0, const cplx* const* us,
                             or_window* W, const or_params* P, uint32_t nz, const uint64_t* zi, uint64_t* wi, cplx* wv,
                             uint32_t* n_above, uint32_t* n_kept) {
    const uint64_t Np = n / B;
    const uint64_t sb = mulmod(sigma, b, n);
    /* the bin of every entry of zhat */
    uint64_t* zbin = (uint64_t*)malloc(sizeof(uint64_t) * (nz ? nz : 1));
    for (uint32_t e = 0; e < nz; ++e) {
        int64_t oz;
        bin_offset(mulmod(sigma, (zi[e] - b) & (n - 1), n), n, B, &zbin[e], &oz);
    }
    uint32_t cnt = 0, above = 0, kept = 0;
    for (uint32_t j = 0; j < B; ++j) {
        const double mag0 = cabs(u0[j]);
        if (!(mag0 > P->thr)) {
            if (mag0 > P->ref_lo * P->thr && mag0 <= P->ref_hi * P->thr) {
                uint32_t matches = 0;
                uint64_t who = 0;
                cplx val = 0, v;
                for (uint32_t e = 0; e < nz; ++e) {
                    if (zbin[e] != j) continue;
                    if (refine_known(n, B, sigma, b, nshift, shift, u0, us, W, P, j, zi[e] & (n - 1), &v)) {
                        ++matches;
                        who = zi[e] & (n - 1);
                        val = v;
                    }
                }
                if (matches == 1) {
                    wi[cnt] = who;
                    wv[cnt] = val;
                    ++cnt;
                }
            }
            continue;
        }
        ++above;
        /* coarsest level first */
        int L = (int)nshift;
        uint64_t M = Np / (shift[L - 1] / B);
        double th = phase01(u0[j] * conj(us[L - 1][j]));
        uint64_t c = (uint64_t)floor(th * (double)M + 0.5) % M;
        for (int l = L - 2; l >= 0; --l) {
            const uint64_t Mp = Np / (shift[l] / B);
            const uint64_t ratio = Mp / M;
            const double thl = phase01(u0[j] * conj(us[l][j]));
            const double y = thl * (double)Mp / (double)M - (double)c / (double)M;
            int64_t h = (int64_t)floor(y + 0.5);
            h %= (int64_t)ratio;
            if (h < 0) h += (int64_t)ratio;
            c += M * (uint64_t)h;
            M = Mp;
        }
        const uint64_t q = c; /* sigma i mod n/B */
        const uint64_t d = (q + Np - (sb & (Np - 1)) + Np / 2) & (Np - 1);
        const int64_t o = (int64_t)d - (int64_t)(Np / 2);
        const uint64_t p = ((uint64_t)j * Np + (uint64_t)o) & (n - 1);
        const uint64_t si = (p + sb) & (n - 1);
        const uint64_t i = mulmod(sigma_inv, si, n);
        const double gain = window_at(W, -o);
        if (!(gain >= P->gmin)) continue;
        int iso = 1;
        for (uint32_t l = 0; l < nshift; ++l)
            if (fabs(cabs(us[l][j]) - mag0) > P->iso_tol * mag0) iso = 0;
        if (!iso) continue;
        wi[cnt] = i;
        wv[cnt] = u0[j] / gain;
        ++cnt;
        ++kept;
    }
    free(zbin);
    if (n_above) *n_above = above;
    if (n_kept) *n_kept = kept;
    return cnt;
}

/* zhat <- zhat + what, kept sorted by index (a shared index adds the two values, zhat's first); entries
 * below drop_below are removed.  Capacity reading (the paper's zhat is unbounded): when more than cap
 * entries remain, the cap smallest indices are kept and *overflow is set. */
typedef struct {
    uint64_t i;
    cplx v;
} z_entry;
static int cmp_z_entry(const void* a, const void* b) {
    const uint64_t x = ((const z_entry*)a)->i, y = ((const z_entry*)b)->i;
    return x < y ? -1 : (x > y ? 1 : 0);
}
static uint32_t z_merge(uint32_t nz, uint64_t* zi, cplx* zv, uint32_t nw, const uint64_t* wi, const cplx* wv,
                        double drop_below, uint32_t cap, int* overflow) {
    z_entry* w = (z_entry*)malloc(sizeof(z_entry) * (nw ? nw : 1));
    z_entry* t = (z_entry*)malloc(sizeof(z_entry) * (nz + nw ? nz + nw : 1));
    for (uint32_t e = 0; e < nw; ++e) {
        w[e].i = wi[e];
        w[e].v = wv[e];
    }
    qsort(w, nw, sizeof(z_entry), cmp_z_entry); /* a round decodes each index at most once */
    uint32_t a = 0, b = 0, m = 0;
    while (a < nz || b < nw) {
        if (b >= nw || (a < nz && zi[a] < w[b].i)) {
            t[m].i = zi[a];
            t[m].v = zv[a];
            ++a;
        } else if (a >= nz || w[b].i < zi[a]) {
            t[m] = w[b];
            ++b;
        } else {
            t[m].i = zi[a];
            t[m].v = zv[a] + w[b].v;
            ++a;
            ++b;
        }
        ++m;
    }
    uint32_t out = 0;
    for (uint32_t e = 0; e < m; ++e) {
        if (cabs(t[e].v) < drop_below) continue;
        if (out < cap) {
            zi[out] = t[e].i;
            zv[out] = t[e].v;
        }
        ++out;
    }
    free(w);
    free(t);
    if (out > cap) {
        *overflow = 1;
        out = cap;
    }
    return out;
}

/* Public: the decode of one round on caller-supplied bins (u is nshift+1 rows of B bins: a = 0
 * first, then each beta_l). */
uint32_t or_exact_decode(const or_params* P, uint32_t B, double alpha, uint64_t sigma, uint64_t b, uint32_t nshift,
                         const uint64_t* shift, const double* u, uint32_t nz, const uint64_t* zi, uint64_t* wi, double* wv,
                         uint32_t* n_above, uint32_t* n_kept) {
    or_window W;
    window_init(&W, P->n, B, alpha, P->delta);
    const cplx* uc = (const cplx*)u;
    const cplx* us[4];
    for (uint32_t l = 0; l < nshift; ++l) us[l] = uc + (size_t)(l + 1) * B;
    const uint32_t c = exact_decode(P->n, B, sigma, or_inverse_mod_pow2(sigma, P->n), b, nshift, shift, uc, us, &W,
                                    P, nz, zi, wi, (cplx*)wv, n_above, n_kept);
    window_free(&W);
    return c;
}

/* One round of NoiselessSparseFFTInner: the 1 + L hashings and the decode; returns |what|.
 * If u_out is given it receives the (1+L) x B bins. */
uint32_t or_exact_inner(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint32_t t, uint32_t nz,
                        const uint64_t* zi, const double* zv, uint64_t* wi, double* wv, uint32_t* n_above,
                        uint32_t* n_kept, double* u_out) {
    uint32_t B, nshift;
    double alpha;
    int64_t T;
    uint64_t shifts[4], sigma, sigma_inv, b;
    or_exact_round_params(P, seed, stream, t, &B, &alpha, &T, &nshift, shifts, &sigma, &sigma_inv, &b);
    or_window W;
    window_init(&W, P->n, B, alpha, P->delta);
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)B * (nshift + 1));
    hash_to_bins(P->n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, 0, b, &W, 0, u);
    const cplx* us[4];
    for (uint32_t l = 0; l < nshift; ++l) {
        hash_to_bins(P->n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, shifts[l], b, &W, 0, u + (size_t)(l + 1) * B);
        us[l] = u + (size_t)(l + 1) * B;
    }
    const uint32_t c =
        exact_decode(P->n, B, sigma, sigma_inv, b, nshift, shifts, u, us, &W, P, nz, zi, wi, (cplx*)wv, n_above, n_kept);
    if (u_out) memcpy(u_out, u, sizeof(cplx) * (size_t)B * (nshift + 1));
    free(u);
    window_free(&W);
    return c;
}

/* ------------------------------------------------------------------------------------------ */
/* NoiselessSparseFFT (Algorithm 1, outer procedure)                                           */
/* ------------------------------------------------------------------------------------------ */
/* Returns 0, or 1 when a bin of the last round rose above thr but no coefficient could be decoded
 * from it (not converged), or 2 when zhat overflowed z_cap. */
int or_sfft_exact(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint64_t* out_i, double* out_v,
                  uint32_t* out_count) {
    const uint32_t cap = P->z_cap;
    uint64_t* zi = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    cplx* zv = (cplx*)malloc(sizeof(cplx) * cap);
    uint32_t nz = 0;
    int overflow = 0;
    uint32_t unresolved_last = 0;
    const uint32_t rounds = or_exact_rounds(P);
    const uint64_t maxB = P->n / 2;
    uint64_t* wi = (uint64_t*)malloc(sizeof(uint64_t) * maxB);
    cplx* wv = (cplx*)malloc(sizeof(cplx) * maxB);
    for (uint32_t t = 0; t < rounds; ++t) {
        uint32_t above = 0, kept = 0;
        const uint32_t nw =
            or_exact_inner(P, x, seed, stream, t, nz, zi, (const double*)zv, wi, (double*)wv, &above, &kept, NULL);
        nz = z_merge(nz, zi, zv, nw, wi, wv, P->prune * P->thr, cap, &overflow);
        unresolved_last = above - kept;
    }
    memcpy(out_i, zi, sizeof(uint64_t) * nz);
    memcpy(out_v, zv, sizeof(cplx) * nz);
    *out_count = nz;
    free(zi);
    free(zv);
    free(wi);
    free(wv);
    if (overflow) return 2;
    return unresolved_last > 0 ? 1 : 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Paper mode of Algorithm 1: the literal decode, for the paper's own input model              */
/* ------------------------------------------------------------------------------------------ */
/*
 * Algorithm 1 as printed, for spectra whose coefficients are integers (the assumption of Sec. 3:
 * every X_i lies in {-L, ..., L}; with this oracle's unnormalised scale the integers are the X_i
 * themselves).  Per round t, with the round's sigma and b (the same Philox draws as the build
 * readings, so both modes see the same hashings):
 *   u  = HashToBins(x, zhat, P_{sigma,0,b}),  u' = HashToBins(x, zhat, P_{sigma,1,b}), both
 *        subtracting zhat with the closed-form gain Ghat' of Sec. 7;
 *   J  = {j : |u_j| > thr};
 *   for j in J, ascending:  i = sigma^{-1} round(phase(u_j / u'_j) n / 2 pi) mod n,
 *                          v = round(u_j) (real and imaginary parts rounded to integers),
 *                          w_i <- v (a later j that decodes the same i overwrites it);
 *   zhat <- zhat + w.
 * round() is round-half-up.  zhat keeps every non-zero entry (the paper bounds neither its size nor
 * prunes it); an entry that cancels to exactly zero leaves the support.
 */
static double round_half_up(double v) { return floor(v + 0.5); }

/* The decode of one round on given bins u (row a = 0) and up (row a = 1): returns |w|; (wi, wv)
 * sorted by index; wj (may be NULL) receives the bin each entry was decoded from. */
uint32_t or_paper_exact_decode(const or_params* P, uint32_t B, uint64_t sigma, const double* u_re_im,
                               const double* up_re_im, uint64_t* wi, double* wv_re_im, uint32_t* wj, uint32_t* n_above) {
    const uint64_t n = P->n;
    const uint64_t sigma_inv = or_inverse_mod_pow2(sigma, n);
    const cplx* u = (const cplx*)u_re_im;
    const cplx* up = (const cplx*)up_re_im;
    cplx* wv = (cplx*)wv_re_im;
    uint32_t cnt = 0, above = 0;
    for (uint32_t j = 0; j < B; ++j) {
        if (!(cabs(u[j]) > P->thr)) continue;
        ++above;
        const double ph = phase01(u[j] / up[j]);
        const uint64_t si = (uint64_t)round_half_up(ph * (double)n) & (n - 1);
        const uint64_t i = mulmod(sigma_inv, si, n);
        const cplx v = round_half_up(creal(u[j])) + I * round_half_up(cimag(u[j]));
        uint32_t e = 0;
        while (e < cnt && wi[e] != i) ++e;
        wi[e] = i;
        wv[e] = v;
        if (wj) wj[e] = j;
        if (e == cnt) ++cnt;
    }
    /* ascending index order (insertion sort: cnt <= B) */
    for (uint32_t a = 1; a < cnt; ++a) {
        const uint64_t ki = wi[a];
        const cplx kv = wv[a];
        const uint32_t kj = wj ? wj[a] : 0;
        uint32_t b = a;
        while (b > 0 && wi[b - 1] > ki) {
            wi[b] = wi[b - 1];
            wv[b] = wv[b - 1];
            if (wj) wj[b] = wj[b - 1];
            --b;
        }
        wi[b] = ki;
        wv[b] = kv;
        if (wj) wj[b] = kj;
    }
    if (n_above) *n_above = above;
    return cnt;
}

/* One round of the literal NoiselessSparseFFTInner; u_out (may be NULL) receives the 2 x B bins. */
uint32_t or_paper_exact_inner(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint32_t t,
                              uint32_t nz, const uint64_t* zi, const double* zv, uint64_t* wi, double* wv,
                              uint32_t* wj, uint32_t* n_above, double* u_out) {
    uint32_t B, nshift;
    double alpha;
    int64_t T;
    uint64_t shifts[4], sigma, sigma_inv, b;
    or_exact_round_params(P, seed, stream, t, &B, &alpha, &T, &nshift, shifts, &sigma, &sigma_inv, &b);
    or_window W;
    window_init(&W, P->n, B, alpha, P->delta);
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)B * 2);
    hash_to_bins(P->n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, 0, b, &W, 1, u);
    hash_to_bins(P->n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, 1, b, &W, 1, u + B);
    const uint32_t c = or_paper_exact_decode(P, B, sigma, (const double*)u, (const double*)(u + B), wi, wv, wj, n_above);
    if (u_out) memcpy(u_out, u, sizeof(cplx) * (size_t)B * 2);
    free(u);
    window_free(&W);
    return c;
}

/* NoiselessSparseFFT, literal: rounds t = 0 .. ceil(log2 k) (+ extra_rounds), as or_sfft_exact.
 * Returns the number of non-zero entries of zhat written to (out_i, out_v), at most cap; -1 when zhat
 * holds more than cap entries (nothing written). */
int64_t or_sfft_exact_paper(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint64_t* out_i,
                            double* out_v, uint64_t cap) {
    const uint32_t rounds = or_exact_rounds(P);
    uint64_t total = 0; /* zhat gains at most B_t entries per round */
    for (uint32_t t = 0; t < rounds; ++t) total += exact_B(P, t);
    uint64_t* zi = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)total);
    cplx* zv = (cplx*)malloc(sizeof(cplx) * (size_t)total);
    const uint64_t maxB = P->n / 2;
    uint64_t* wi = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)maxB);
    cplx* wv = (cplx*)malloc(sizeof(cplx) * (size_t)maxB);
    uint32_t nz = 0;
    int overflow = 0;
    for (uint32_t t = 0; t < rounds; ++t) {
        const uint32_t nw = or_paper_exact_inner(P, x, seed, stream, t, nz, zi, (const double*)zv, wi, (double*)wv,
                                                 NULL, NULL, NULL);
        /* zhat + w; an entry equal to zero is not in the support (drop_below 0 keeps everything with
         * |v| >= 0, so exact zeros are removed here) */
        nz = z_merge(nz, zi, zv, nw, wi, wv, 0.0, (uint32_t)total, &overflow);
        uint32_t m = 0;
        for (uint32_t e = 0; e < nz; ++e)
            if (zv[e] != 0) {
                zi[m] = zi[e];
                zv[m] = zv[e];
                ++m;
            }
        nz = m;
    }
    int64_t ret = nz;
    if ((uint64_t)nz > cap) {
        ret = -1;
    } else {
        memcpy(out_i, zi, sizeof(uint64_t) * nz);
        memcpy(out_v, zv, sizeof(cplx) * nz);
    }
    free(zi);
    free(zv);
    free(wi);
    free(wv);
    return ret;
}

/* ------------------------------------------------------------------------------------------ */
/* General case: SparseFFT, LocateSignal, LocateInner, EstimateValues (Algorithms 2 and 3)     */
/* ------------------------------------------------------------------------------------------ */
#define OR_FRAC_BITS 16 /* fixed-point fraction bits for region positions (Alg. 3: m_{j,q}) */

/* Schedule reading: k_0 = k, k_{r+1} = floor(k_r / 4) (the k/4 step of Sec. 4.1), stop at 0;
 * B_r = pow2ceil(bins_per_k k_r / eps) clamped to [B_min, n/2]; alpha_r = alpha0. */
uint32_t or_general_rounds(const or_params* P, uint32_t* kr_out, uint32_t* B_out) {
    uint32_t r = 0;
    for (uint64_t kr = P->k; kr >= 1; kr /= 4, ++r) {
        uint64_t B = pow2ceil(P->bins_per_k * (double)kr / P->eps);
        if (B < P->B_min) B = P->B_min;
        if (B > P->n / 2) B = P->n / 2;
        if (kr_out) kr_out[r] = (uint32_t)kr;
        if (B_out) B_out[r] = (uint32_t)B;
    }
    return r;
}

static uint32_t regions_t(const or_params* P) {
    if (P->t_regions) return P->t_regions;
    const int m = ilog2(P->n);
    uint32_t t = 1;
    while (t * 2 <= (uint32_t)m) t *= 2;
    return t;
}

/* LocateSignal geometry: w0 = n/B, t' = t/4, D_max = floor(log_{t'} w0) + 1 (smallest D with
 * w0 / t'^D < 1). */
void or_locate_geometry(const or_params* P, uint32_t B, uint32_t* t_out, uint32_t* tp_out, uint32_t* dmax_out) {
    const uint32_t t = regions_t(P);
    const uint32_t tp = t / 4;
    const int lw = ilog2(P->n / B);
    const int ltp = ilog2(tp);
    *t_out = t;
    *tp_out = tp;
    *dmax_out = (uint32_t)(lw / ltp) + 1;
}

/* beta range of LocateInner: {s n t / (4 w), ..., s n t / (2 w)}, integer end points rounded inward */
void or_beta_range(const or_params* P, uint32_t t, uint64_t w, uint64_t* lo, uint64_t* hi) {
    const double base = P->s * (double)P->n * (double)t / (double)w;
    *lo = (uint64_t)ceil(base / 4.0);
    *hi = (uint64_t)floor(base / 2.0);
    if (*hi < *lo) *hi = *lo;
}

void or_locate_draws(const or_params* P, uint64_t seed, uint32_t stream, uint32_t r, uint32_t B, uint32_t D, uint32_t q,
                     uint64_t* sigma, uint64_t* b, uint64_t* a, uint64_t* beta) {
    uint32_t wd[4];
    draw_words(seed, stream, r, 0, OR_KIND_LOCATE, wd);
    *sigma = draw_odd(wd[0], P->n);
    *b = draw_mod_n(wd[1], P->n);
    uint32_t t, tp, dmax;
    or_locate_geometry(P, B, &t, &tp, &dmax);
    const uint64_t w = (P->n / B) >> ((uint64_t)(D - 1) * (uint64_t)ilog2(tp));
    uint64_t lo, hi;
    or_beta_range(P, t, w, &lo, &hi);
    draw_words(seed, stream, r, (D - 1) * P->R_loc + q, OR_KIND_INNER, wd);
    *a = draw_mod_n(wd[0], P->n);
    *beta = draw_range(wd[1], lo, hi);
}

void or_estimate_draws(const or_params* P, uint64_t seed, uint32_t stream, uint32_t r, uint32_t q, uint64_t* sigma,
                       uint64_t* b, uint64_t* a) {
    uint32_t wd[4];
    draw_words(seed, stream, r, q, OR_KIND_ESTIMATE, wd);
    *sigma = draw_odd(wd[0], P->n);
    *b = draw_mod_n(wd[1], P->n);
    *a = draw_mod_n(wd[2], P->n);
}

/*
 * LocateInner votes for one level (Algorithm 3, procedure LocateInner), on given bins.
 * u[q] / up[q] are the bins of P_{sigma,a_q,b} and P_{sigma,a_q+beta_q,b}.  Regions are fixed-point
 * positions (OR_FRAC_BITS fraction bits) mod n; valid[j] = 0 marks a bottom (no region).
 *   c_j = phase(u_j / u'_j);  m_{j,q} = l_j + (q - 1/2) w / t;  theta = 2 pi (m + sigma b) / n;
 *   vote if the circular distance of beta theta and c_j is below s pi;
 *   Q* = {q : v_{j,q} > R_loc / 2};  bottom if Q* is empty;
 *   l'_j = l_j + (q_0 - 1) w / t with [q_0, q_0 + 3] the four consecutive subregions holding the
 *   most votes.
 * Reading of the choice of l'_j: the paper takes min Q*, which the Lemma "LocateInner" shows lies
 * in [q' - 3, q'] once its constants make a far subregion's majority improbable.  With practical
 * constants (s = 1/4, R_loc = 5) a far subregion wins a majority about one time in ten, and min Q*
 * then jumps to it; the window of four subregions with the most votes keeps the Lemma's conclusion
 * (pi(i) in [l'_j, l'_j + 4w/t]) and ignores an isolated false majority.
 * Integer arithmetic is exact: beta (m + sigma b) mod n is formed in fixed point modulo n 2^F.
 * paper = 1 takes the listing's own choice instead: l'_j = l_j + (min Q* - 1) w / t.
 */
void or_locate_inner_votes_ex(const or_params* P, uint32_t B, uint64_t sigma, uint64_t b, uint32_t t, uint64_t w_fp,
                              uint32_t nrep, const uint64_t* beta, const double* u_re_im, const double* up_re_im,
                              int paper, uint64_t* l_fp, uint8_t* valid, uint32_t* votes_out) {
    const uint64_t n = P->n;
    const uint64_t modmask = (n << OR_FRAC_BITS) - 1;
    const uint64_t sb_fp = mulmod(sigma, b, n) << OR_FRAC_BITS;
    const cplx* u = (const cplx*)u_re_im;
    const cplx* up = (const cplx*)up_re_im;
    uint32_t* v = (uint32_t*)calloc((size_t)B * t, sizeof(uint32_t));
    for (uint32_t q = 0; q < nrep; ++q) {
        for (uint32_t j = 0; j < B; ++j) {
            if (!valid[j]) continue;
            const double c = phase01(u[(size_t)q * B + j] * conj(up[(size_t)q * B + j]));
            for (uint32_t qq = 1; qq <= t; ++qq) {
                const uint64_t m_fp = (l_fp[j] + (2 * (uint64_t)qq - 1) * (w_fp / (2 * (uint64_t)t))) & modmask;
                const uint64_t e = (beta[q] * ((m_fp + sb_fp) & modmask)) & modmask;
                const double f = (double)e / (double)(modmask + 1);
                double dist = fabs(f - c);
                if (dist > 0.5) dist = 1.0 - dist;
                if (dist < P->s / 2.0) v[(size_t)j * t + (qq - 1)] += 1;
            }
        }
    }
    for (uint32_t j = 0; j < B; ++j) {
        if (!valid[j]) continue;
        const uint32_t* vj = v + (size_t)j * t;
        int any = 0; /* Q* non-empty */
        for (uint32_t qq = 0; qq < t; ++qq)
            if (2 * vj[qq] > nrep) any = 1;
        if (!any) {
            valid[j] = 0;
            continue;
        }
        uint32_t best = 0;
        if (paper) {
            /* Algorithm 3 as printed: l' = l + (min Q* - 1) w / t (0-based: the first majority q) */
            while (!(2 * vj[best] > nrep)) ++best;
        } else {
            /* the four consecutive subregions with the most votes (ties to the smallest start) */
            uint32_t best_sum = 0;
            for (uint32_t q0 = 0; q0 + 4 <= t; ++q0) {
                const uint32_t sum = vj[q0] + vj[q0 + 1] + vj[q0 + 2] + vj[q0 + 3];
                if (q0 == 0 || sum > best_sum) {
                    best = q0;
                    best_sum = sum;
                }
            }
        }
        l_fp[j] = (l_fp[j] + (uint64_t)best * (w_fp / t)) & modmask;
    }
    if (votes_out) memcpy(votes_out, v, sizeof(uint32_t) * (size_t)B * t);
    free(v);
}
/* The build reading (four consecutive subregions) */
void or_locate_inner_votes(const or_params* P, uint32_t B, uint64_t sigma, uint64_t b, uint32_t t, uint64_t w_fp,
                           uint32_t nrep, const uint64_t* beta, const double* u_re_im, const double* up_re_im,
                           uint64_t* l_fp, uint8_t* valid, uint32_t* votes_out) {
    or_locate_inner_votes_ex(P, B, sigma, b, t, w_fp, nrep, beta, u_re_im, up_re_im, 0, l_fp, valid, votes_out);
}

static int cmp_u64(const void* a, const void* b) {
    const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Region start of bin j before the first level: [j n/B - n/2B, + n/B) (reading of Algorithm 3's
 * initial l^(1), centred on the bins like h) */
static uint64_t first_region_fp(uint64_t n, uint32_t B, uint32_t j) {
    const uint64_t Np = n / B;
    return ((((uint64_t)j * Np) + n - Np / 2) & (n - 1)) << OR_FRAC_BITS;
}

/* A bin's candidate after the last level: sigma^{-1}(tau) + b with tau the integer nearest the centre
 * of its last region (pi^{-1} of Algorithm 3's final l), or all ones for a bottom bin. */
static uint64_t region_candidate(uint64_t n, uint64_t Np, uint32_t tp, uint32_t dmax, uint64_t sigma, uint64_t b,
                                 uint64_t l_fp, uint8_t valid) {
    if (!valid) return ~(uint64_t)0;
    const uint64_t wlast_fp = (Np << OR_FRAC_BITS) >> ((uint64_t)dmax * (uint64_t)ilog2(tp));
    const uint64_t tau = ((l_fp + wlast_fp / 2 + ((uint64_t)1 << (OR_FRAC_BITS - 1))) >> OR_FRAC_BITS) & (n - 1);
    return (mulmod(or_inverse_mod_pow2(sigma, n), tau, n) + b) & (n - 1);
}

/*
 * LocateSignal's level loop on given bins (Algorithm 3 after its hashings): the replay entry.
 * u / up hold dmax x nrep rows of B bins, row D nrep + q being LocateInner round q of level D + 1
 * (hashings at a_q and a_q + beta_q under the call's sigma, b); beta the matching dmax x nrep shifts.
 * Outputs (each may be NULL): lfp_levels / valid_levels (dmax x B) the regions and bottom flags after
 * every level, cand (B) each bin's candidate (all ones for bottom), as or_locate_signal_ex forms them.
 */
void or_locate_replay(const or_params* P, uint32_t B, uint64_t sigma, uint64_t b, uint32_t nrep, const uint64_t* beta,
                      const double* u_re_im, const double* up_re_im, int paper, uint64_t* lfp_levels,
                      uint8_t* valid_levels, uint64_t* cand) {
    const uint64_t n = P->n;
    const uint64_t Np = n / B;
    uint32_t t, tp, dmax;
    or_locate_geometry(P, B, &t, &tp, &dmax);
    uint64_t* l_fp = (uint64_t*)malloc(sizeof(uint64_t) * B);
    uint8_t* valid = (uint8_t*)malloc(B);
    for (uint32_t j = 0; j < B; ++j) {
        l_fp[j] = first_region_fp(n, B, j);
        valid[j] = 1;
    }
    for (uint32_t D = 1; D <= dmax; ++D) {
        const uint64_t w_fp = (Np << OR_FRAC_BITS) >> ((uint64_t)(D - 1) * (uint64_t)ilog2(tp));
        const size_t row = (size_t)(D - 1) * nrep;
        or_locate_inner_votes_ex(P, B, sigma, b, t, w_fp, nrep, beta + row, u_re_im + 2 * row * B,
                                 up_re_im + 2 * row * B, paper, l_fp, valid, NULL);
        if (lfp_levels) memcpy(lfp_levels + (size_t)(D - 1) * B, l_fp, sizeof(uint64_t) * B);
        if (valid_levels) memcpy(valid_levels + (size_t)(D - 1) * B, valid, B);
    }
    if (cand)
        for (uint32_t j = 0; j < B; ++j) cand[j] = region_candidate(n, Np, tp, dmax, sigma, b, l_fp[j], valid[j]);
    free(l_fp);
    free(valid);
}

/* LocateSignal (Algorithm 3): the hashings of every level, then the level loop; returns |L| with L
 * sorted ascending and de-duplicated.  cand_out (may be NULL) receives the B per-bin candidates. */
uint32_t or_locate_signal_ex(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint32_t r, uint32_t B,
                             uint32_t nz, const uint64_t* zi, const double* zv, int paper, uint64_t* Lout,
                             uint64_t* cand_out) {
    const uint64_t n = P->n;
    uint32_t t, tp, dmax;
    or_locate_geometry(P, B, &t, &tp, &dmax);
    or_window W;
    window_init(&W, n, B, P->alpha0, P->delta);
    const uint32_t R = P->R_loc;
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)B * R * dmax);
    cplx* up = (cplx*)malloc(sizeof(cplx) * (size_t)B * R * dmax);
    uint64_t* beta = (uint64_t*)malloc(sizeof(uint64_t) * R * dmax);
    uint64_t sigma = 0, b = 0;
    for (uint32_t D = 1; D <= dmax; ++D) {
        for (uint32_t q = 0; q < R; ++q) {
            const size_t row = (size_t)(D - 1) * R + q;
            uint64_t a;
            or_locate_draws(P, seed, stream, r, B, D, q, &sigma, &b, &a, &beta[row]);
            hash_to_bins(n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, a, b, &W, 0, u + row * B);
            hash_to_bins(n, (const cplx*)x, nz, zi, (const cplx*)zv, sigma, (a + beta[row]) & (n - 1), b, &W, 0,
                         up + row * B);
        }
    }
    uint64_t* cand = (uint64_t*)malloc(sizeof(uint64_t) * B);
    or_locate_replay(P, B, sigma, b, R, beta, (const double*)u, (const double*)up, paper, NULL, NULL, cand);
    if (cand_out) memcpy(cand_out, cand, sizeof(uint64_t) * B);
    uint32_t cnt = 0;
    for (uint32_t j = 0; j < B; ++j)
        if (cand[j] != ~(uint64_t)0) Lout[cnt++] = cand[j];
    qsort(Lout, cnt, sizeof(uint64_t), cmp_u64);
    uint32_t uniq = 0;
    for (uint32_t e = 0; e < cnt; ++e)
        if (uniq == 0 || Lout[uniq - 1] != Lout[e]) Lout[uniq++] = Lout[e];
    free(cand);
    free(u);
    free(up);
    free(beta);
    window_free(&W);
    return uniq;
}
uint32_t or_locate_signal(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint32_t r, uint32_t B,
                          uint32_t nz, const uint64_t* zi, const double* zv, uint64_t* Lout) {
    return or_locate_signal_ex(P, x, seed, stream, r, B, nz, zi, zv, 0, Lout, NULL);
}

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
    uint64_t i;
    double mag2;
} or_rank;
static int cmp_rank(const void* a, const void* b) { /* |w| descending, then index ascending */
    const or_rank* x = (const or_rank*)a;
    const or_rank* y = (const or_rank*)b;
    if (x->mag2 > y->mag2) return -1;
    if (x->mag2 < y->mag2) return 1;
    return x->i < y->i ? -1 : (x->i > y->i ? 1 : 0);
}

/*
 * EstimateValues from given bins (Algorithm 2, procedure EstimateValues, after its hashing loop).
 * u holds R_est rows of B bins, hashing q with (sigma_q, a_q, b_q).  For each i in L:
 *   e_q = u^{(q)}_{h_q(i)} w^{-a_q sigma_q i} / W(-o_q(i))   for the q with W(-o_q(i)) >= est_gmin
 *   what_i = median_q Re e_q + i median_q Im e_q   (lower median; 0 if no q qualifies)
 * then J = the k' largest |what_i| (ties to the smaller index).  Reading: the division by the
 * known gain W(-o) removes the bias of hashings that put i in the transition band.
 * Returns |J|; outputs sorted by index.
 */
uint32_t or_estimate_from_bins(const or_params* P, uint32_t B, double alpha, uint32_t nrep, const uint64_t* sig,
                               const uint64_t* bb, const uint64_t* aa, const double* u_re_im, uint32_t nL,
                               const uint64_t* L, uint32_t kprime, uint64_t* wi, double* wv_re_im) {
    const uint64_t n = P->n;
    or_window W;
    window_init(&W, n, B, alpha, P->delta);
    const cplx* u = (const cplx*)u_re_im;
    cplx* est = (cplx*)malloc(sizeof(cplx) * (nL ? nL : 1));
    double* re = (double*)malloc(sizeof(double) * nrep);
    double* im = (double*)malloc(sizeof(double) * nrep);
    for (uint32_t e = 0; e < nL; ++e) {
        const uint64_t i = L[e];
        uint32_t m = 0;
        for (uint32_t q = 0; q < nrep; ++q) {
            const uint64_t p = mulmod(sig[q], (i - bb[q]) & (n - 1), n);
            uint64_t j;
            int64_t o;
            bin_offset(p, n, B, &j, &o);
            const double gain = window_at(&W, -o);
            if (!(gain >= P->est_gmin)) continue;
            const uint64_t ph = mulmod(mulmod(aa[q], sig[q], n), i, n);
            const cplx val = u[(size_t)q * B + j] * conj(root_pow(ph, n)) / gain;
            re[m] = creal(val);
            im[m] = cimag(val);
            ++m;
        }
        if (m == 0) {
            est[e] = 0;
        } else {
            qsort(re, m, sizeof(double), cmp_double);
            qsort(im, m, sizeof(double), cmp_double);
            est[e] = re[(m - 1) / 2] + I * im[(m - 1) / 2];
        }
    }
    or_rank* rk = (or_rank*)malloc(sizeof(or_rank) * (nL ? nL : 1));
    for (uint32_t e = 0; e < nL; ++e) {
        rk[e].i = L[e];
        rk[e].mag2 = creal(est[e]) * creal(est[e]) + cimag(est[e]) * cimag(est[e]);
    }
    qsort(rk, nL, sizeof(or_rank), cmp_rank);
    const uint32_t nJ = nL < kprime ? nL : kprime;
    uint64_t* keep = (uint64_t*)malloc(sizeof(uint64_t) * (nJ ? nJ : 1));
    for (uint32_t e = 0; e < nJ; ++e) keep[e] = rk[e].i;
    qsort(keep, nJ, sizeof(uint64_t), cmp_u64);
    cplx* wv = (cplx*)wv_re_im;
    for (uint32_t e = 0; e < nJ; ++e) {
        uint32_t pos = 0;
        while (L[pos] != keep[e]) ++pos; /* L is sorted and unique */
        wi[e] = keep[e];
        wv[e] = est[pos];
    }
    free(keep);
    free(rk);
    free(est);
    free(re);
    free(im);
    window_free(&W);
    return nJ;
}

/* EstimateValues with its hashings (Algorithm 2). */
uint32_t or_estimate_values(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint32_t r, uint32_t B,
                            uint32_t nz, const uint64_t* zi, const double* zv, uint32_t nL, const uint64_t* L,
                            uint32_t kprime, uint64_t* wi, double* wv) {
    const uint64_t n = P->n;
    const uint32_t R = P->R_est;
    or_window W;
    window_init(&W, n, B, P->alpha0, P->delta);
    cplx* u = (cplx*)malloc(sizeof(cplx) * (size_t)B * R);
    uint64_t* sig = (uint64_t*)malloc(sizeof(uint64_t) * R);
    uint64_t* bb = (uint64_t*)malloc(sizeof(uint64_t) * R);
    uint64_t* aa = (uint64_t*)malloc(sizeof(uint64_t) * R);
    for (uint32_t q = 0; q < R; ++q) {
        or_estimate_draws(P, seed, stream, r, q, &sig[q], &bb[q], &aa[q]);
        hash_to_bins(n, (const cplx*)x, nz, zi, (const cplx*)zv, sig[q], aa[q], bb[q], &W, 0, u + (size_t)q * B);
    }
    window_free(&W);
    const uint32_t nJ = or_estimate_from_bins(P, B, P->alpha0, R, sig, bb, aa, (const double*)u, nL, L, kprime, wi, wv);
    free(u);
    free(sig);
    free(bb);
    free(aa);
    return nJ;
}

/* SparseFFT (Algorithm 2): returns 0, or 2 when zhat overflowed z_cap.  paper = 1 runs LocateInner
 * with the listing's min Q* (or_locate_inner_votes_ex). */
int or_sfft_general_ex(const or_params* P, const double* x, uint64_t seed, uint32_t stream, int paper, uint64_t* out_i,
                       double* out_v, uint32_t* out_count) {
    const uint32_t cap = P->z_cap;
    uint64_t* zi = (uint64_t*)malloc(sizeof(uint64_t) * cap);
    cplx* zv = (cplx*)malloc(sizeof(cplx) * cap);
    uint32_t nz = 0;
    int overflow = 0;
    uint32_t krs[64], Bs[64];
    const uint32_t R = or_general_rounds(P, krs, Bs);
    const uint64_t maxB = P->n / 2;
    uint64_t* L = (uint64_t*)malloc(sizeof(uint64_t) * maxB);
    uint64_t* wi = (uint64_t*)malloc(sizeof(uint64_t) * maxB);
    cplx* wv = (cplx*)malloc(sizeof(cplx) * maxB);
    for (uint32_t r = 0; r < R; ++r) {
        const uint32_t B = Bs[r];
        const uint32_t nL = or_locate_signal_ex(P, x, seed, stream, r, B, nz, zi, (const double*)zv, paper, L, NULL);
        const uint32_t nJ = or_estimate_values(P, x, seed, stream, r, B, nz, zi, (const double*)zv, nL, L, 3 * krs[r], wi,
                                               (double*)wv);
        nz = z_merge(nz, zi, zv, nJ, wi, wv, 0.0, cap, &overflow);
    }
    memcpy(out_i, zi, sizeof(uint64_t) * nz);
    memcpy(out_v, zv, sizeof(cplx) * nz);
    *out_count = nz;
    free(zi);
    free(zv);
    free(L);
    free(wi);
    free(wv);
    return overflow ? 2 : 0;
}

int or_sfft_general(const or_params* P, const double* x, uint64_t seed, uint32_t stream, uint64_t* out_i, double* out_v,
                    uint32_t* out_count) {
    return or_sfft_general_ex(P, x, seed, stream, 0, out_i, out_v, out_count);
}

/* Number of distinct samples of x one HashToBins reads: 2T+1. */
int64_t or_samples_per_hashing(uint64_t n, uint32_t B, double alpha, double delta) {
    return 2 * or_window_T(n, B, alpha, delta) + 1;
}
