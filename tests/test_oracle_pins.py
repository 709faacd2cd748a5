"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it checks.  None of them retypes the oracle's formula: the checks use
numpy's FFT as an independent ground truth, closed forms, the paper's lemmas and claims (which hold
deterministically given the hashing events), statistics over seeds, or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, general_fields, oracle_params

# ------------------------------------------------------------------------------------------------
# Philox4x32-10 and the parameter draws (Sec. 3 "Choose sigma uniformly at random ...")
# ------------------------------------------------------------------------------------------------


def test_philox_words_are_uniform_and_counter_sensitive():
    words = []
    for c in range(4096):
        words.extend(oracle.philox4x32_10([c, 7, 1, 3], [0x1234, 0xABCD]))
    words = np.array(words, dtype=np.uint64)
    # byte histogram: chi-square with 255 dof; 99.99% quantile is about 352
    b = np.concatenate([(words >> s) & 0xFF for s in (0, 8, 16, 24)])
    hist = np.bincount(b.astype(np.int64), minlength=256)
    exp = len(b) / 256.0
    chi2 = float(np.sum((hist - exp) ** 2 / exp))
    assert chi2 < 352.0
    # each bit of the 32-bit words is set about half the time
    for bit in range(32):
        frac = float(np.mean((words >> bit) & 1))
        assert abs(frac - 0.5) < 0.02
    # every counter word and key word changes the output
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        assert oracle.philox4x32_10(c, [5, 6]) != base
    assert oracle.philox4x32_10([1, 2, 3, 4], [5, 7]) != base
    assert oracle.philox4x32_10([1, 2, 3, 4], [5, 6]) == base


@pytest.mark.parametrize("m", [4, 10, 22, 26, 32])
def test_inverse_mod_pow2(m):
    n = 1 << m
    rng = np.random.default_rng(m)
    for _ in range(200):
        s = int(rng.integers(0, n)) | 1
        si = oracle.inverse_mod_pow2(s, n)
        assert (s * si) % n == 1


def test_exact_draws_are_odd_sigma_and_uniform_b():
    P = oracle_params(exact_fields(1 << 16, 64))
    sig, bs = [], []
    for s in range(400):
        rp = oracle.exact_round_params(P, 1000 + s, 0, 0)
        sig.append(rp["sigma"])
        bs.append(rp["b"])
        assert rp["sigma"] % 2 == 1 and 0 < rp["sigma"] < (1 << 16)
        assert (rp["sigma"] * rp["sigma_inv"]) % (1 << 16) == 1
    # b spreads over [0, n): a Kolmogorov-style check on the empirical CDF
    bs = np.sort(np.array(bs) / float(1 << 16))
    dev = np.max(np.abs(bs - (np.arange(1, len(bs) + 1) / len(bs))))
    assert dev < 0.1


# ------------------------------------------------------------------------------------------------
# Claim "perm" (Sec. 2): DFT(P_{sigma,a,b} x)_{pi(i)} = X_i w^{a sigma i}
# ------------------------------------------------------------------------------------------------


def _check_perm(n, x, sigma, a, b):
    X = np.fft.fft(x)
    Y = np.fft.fft(oracle.permute(x, sigma, a, b))
    i = np.arange(n, dtype=np.int64)
    pi = (sigma * (i - b)) % n
    expect = X * np.exp(-2j * np.pi * ((a * sigma * i) % n) / n)
    assert np.max(np.abs(Y[pi] - expect)) < 1e-10 * max(1.0, np.max(np.abs(X)))


@pytest.mark.parametrize("n", [8, 16])
def test_permutation_claim_exhaustive(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sigma in range(1, n, 2):
        for a in range(n):
            for b in range(n):
                _check_perm(n, x, sigma, a, b)


@pytest.mark.parametrize("n", [256, 4096])
def test_permutation_claim_random(n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for _ in range(20):
        _check_perm(n, x, int(rng.integers(0, n)) | 1, int(rng.integers(0, n)), int(rng.integers(0, n)))


# ------------------------------------------------------------------------------------------------
# Flat window (Definition in Sec. 2, construction Lemma in Sec. 7)
# ------------------------------------------------------------------------------------------------


def _window_spectrum(n, g):
    """(1/n) DFT of the even taps g_{-T..T} placed mod n, computed by numpy's FFT."""
    T = len(g) - 1
    gp = np.zeros(n, dtype=np.float64)
    for t in range(-T, T + 1):
        gp[t % n] += g[abs(t)]
    return np.fft.fft(gp).real / n


@pytest.mark.parametrize("n,B,alpha,delta", [
    (1 << 14, 16, 0.5, 1e-6), (1 << 14, 32, 0.5, 1e-8), (1 << 14, 16, 0.25, 1e-8),
    (1 << 16, 64, 0.5, 1e-6), (1 << 16, 16, 0.125, 1e-6), (1 << 16, 256, 0.354, 1e-6),
])
def test_window_is_flat(n, B, alpha, delta):
    g = oracle.window_taps(n, B, alpha, delta)
    T = len(g) - 1
    # support size O(B/alpha log(1/delta))
    assert 2 * T + 1 <= 2 * 4 * B * math.log(1 / delta) / (math.pi * alpha) + 1
    W = _window_spectrum(n, g)
    l = np.arange(n)
    al = np.minimum(l, n - l)
    passband = al <= (1 - alpha) * n / (2 * B)
    stopband = al >= n / (2 * B)
    assert np.max(np.abs(W[passband] - 1.0)) <= delta
    assert np.max(np.abs(W[stopband])) <= delta
    assert W.min() >= -delta and W.max() <= 1 + delta
    # || Ghat' - Ghat ||_inf < delta (fourth property of the definition), on the transition band
    # and a sample of the rest
    trans = np.nonzero(~passband & ~stopband)[0]
    sample = np.concatenate([trans, np.arange(0, n, max(1, n // 512))])
    gp = np.array([oracle.window_gprime(n, B, alpha, delta, int(v)) for v in sample])
    assert np.max(np.abs(gp - W[sample])) < delta
    assert gp.min() >= 0.0 and gp.max() <= 1.0
    # the oracle's direct sum equals the FFT value
    for v in sample[:: max(1, len(sample) // 40)]:
        assert abs(oracle.window_response(n, g, int(v)) - W[v]) < 1e-12


# ------------------------------------------------------------------------------------------------
# HashToBins (Alg. 1; Lemma "hashtobins" and its four-step method)
# ------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("n,B", [(1 << 10, 8), (1 << 10, 64), (1 << 12, 16)])
def test_hash_to_bins_equals_filtered_permuted_spectrum(n, B):
    """u_j = sum_i X_i w^{a sigma i} W(j n/B - pi(i)) for any x: the exact identity behind the Lemma."""
    rng = np.random.default_rng(n + B)
    alpha, delta = 0.5, 1e-8
    g = oracle.window_taps(n, B, alpha, delta)
    Wf = _window_spectrum(n, g)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = np.fft.fft(x)
    i = np.arange(n, dtype=np.int64)
    for _ in range(6):
        sigma, a, b = int(rng.integers(0, n)) | 1, int(rng.integers(0, n)), int(rng.integers(0, n))
        u = oracle.hash_to_bins(x, sigma, a, b, B, alpha, delta)
        pi = (sigma * (i - b)) % n
        ph = np.exp(-2j * np.pi * ((a * sigma * i) % n) / n)
        expect = np.array([np.sum(X * ph * Wf[(j * (n // B) - pi) % n]) for j in range(B)])
        assert np.max(np.abs(u - expect)) < 1e-9 * np.sum(np.abs(X))


@pytest.mark.parametrize("use_gprime", [False, True])
def test_hash_to_bins_subtraction_removes_zhat(use_gprime):
    """HashToBins(x, zhat) = HashToBins(x - IDFT(zhat), 0) up to zhat's leakage outside its own bin,
    which the flat window bounds by delta ||zhat||_1 (plus delta for Ghat' - Ghat)."""
    n, B, alpha, delta = 1 << 12, 32, 0.5, 1e-7
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    zi = np.sort(rng.choice(n, 24, replace=False)).astype(np.uint64)
    zv = (rng.standard_normal(24) + 1j * rng.standard_normal(24)) * 3
    Z = np.zeros(n, dtype=np.complex128)
    Z[zi.astype(np.int64)] = zv
    xz = x - np.fft.ifft(Z)
    for _ in range(5):
        sigma, a, b = int(rng.integers(0, n)) | 1, int(rng.integers(0, n)), int(rng.integers(0, n))
        u1 = oracle.hash_to_bins(x, sigma, a, b, B, alpha, delta, zi, zv, use_gprime=use_gprime)
        u2 = oracle.hash_to_bins(xz, sigma, a, b, B, alpha, delta)
        bound = (2.0 if use_gprime else 1.0) * delta * np.sum(np.abs(zv)) + 1e-9
        assert np.max(np.abs(u1 - u2)) <= bound


# ------------------------------------------------------------------------------------------------
# NoiselessSparseFFTInner: Lemma "l:est", Claim "c:onlyS" (Sec. 3)
# ------------------------------------------------------------------------------------------------


def _events(n, B, alpha, sigma, b, support):
    Np = n // B
    pi = (sigma * (support - b)) % n
    h = ((pi + Np // 2) % n) // Np
    o = (pi - h * Np) % n
    o = np.where(o >= n // 2, o - n, o)
    coll = np.array([np.sum(h == hj) > 1 for hj in h])
    off = np.abs(o) >= (1 - alpha) * n / (2 * B)
    return h, o, coll, off


@pytest.mark.parametrize("n,k,delta", [(1 << 14, 8, 1e-8), (1 << 16, 32, 1e-7)])
def test_lemma_est_and_claim_onlyS(n, k, delta):
    P = oracle_params(exact_fields(n, k, delta=delta))
    decoded_isolated = 0
    for inst in range(25):
        sig = workloads.exact_sparse(n, k, workloads.seed_for(1, inst), dtype=np.complex128)
        res = oracle.exact_inner(P, sig.x, 77 + inst, 0, 0)
        h, o, coll, off = _events(n, res["B"], res["alpha"], res["sigma"], res["b"], sig.support)
        got = dict(zip(res["idx"].astype(np.int64).tolist(), res["val"].tolist()))
        for e, i in enumerate(sig.support.tolist()):
            if not coll[e] and not off[e]:
                assert i in got, "isolated coefficient with small offset must be decoded (Lemma l:est)"
                assert abs(got[i] - sig.values[e]) < 1e-6
                decoded_isolated += 1
        J = np.nonzero(np.abs(res["bins"][0]) > P.thr)[0]
        assert set(J.tolist()) <= set(h.tolist()), "every j in J lies in h(S) (Claim c:onlyS)"
        assert res["n_above"] == len(J) and len(res["idx"]) <= len(J) <= k
    assert decoded_isolated > 0


def test_lemma_est_brute_force_tiny():
    """All (sigma, b) at n = 64: every isolated, small-offset coefficient is decoded exactly."""
    n, k, B, alpha, delta = 64, 2, 8, 0.5, 1e-9
    P = oracle_params(exact_fields(n, k, delta=delta, bins_per_k=4.0, B_min=8))
    sig = workloads.exact_sparse(n, k, 4242, dtype=np.complex128)
    checked = 0
    for sigma in range(1, n, 2):
        for b in range(n):
            u0 = oracle.hash_to_bins(sig.x, sigma, 0, b, B, alpha, delta)
            u1 = oracle.hash_to_bins(sig.x, sigma, B, b, B, alpha, delta)
            wi, wv, above = oracle.exact_decode(P, B, alpha, sigma, b, [B], np.stack([u0, u1]))
            h, o, coll, off = _events(n, B, alpha, sigma, b, sig.support)
            got = dict(zip(wi.astype(np.int64).tolist(), wv.tolist()))
            for e, i in enumerate(sig.support.tolist()):
                if not coll[e] and not off[e]:
                    assert i in got and abs(got[i] - sig.values[e]) < 1e-6
                    checked += 1
            assert set(np.nonzero(np.abs(u0) > P.thr)[0].tolist()) <= set(h.tolist())
    assert checked > 1000


def test_claims_coll_and_off_frequencies():
    """Claim c:coll: Pr[E_coll(i)] <= 4|S|/B; Claim c:off: Pr[E_off(i)] <= alpha (here ~ alpha)."""
    n, k = 1 << 16, 32
    P = oracle_params(exact_fields(n, k))
    support = workloads.exact_sparse(n, k, 99, dtype=np.complex128).support
    n_coll = n_off = tot = 0
    for s in range(600):
        rp = oracle.exact_round_params(P, 5000 + s, 0, 0)
        _, _, coll, off = _events(n, rp["B"], rp["alpha"], rp["sigma"], rp["b"], support)
        n_coll += int(coll.sum())
        n_off += int(off.sum())
        tot += k
    B, alpha = rp["B"], rp["alpha"]
    assert n_coll / tot <= 4 * k / B
    p = n_off / tot
    assert abs(p - alpha) < 4 * math.sqrt(alpha * (1 - alpha) / tot) + 0.01


@pytest.mark.parametrize("j", [1, 3, 1 << 10, (1 << 16) // 2, 12345])
def test_limited_independence(j):
    """Lemma 3.6 of HIKP (Sec. 2): Pr[sigma j in [-C, C] mod n] <= 4C/n for random odd sigma."""
    n, C = 1 << 16, 256
    P = oracle_params(exact_fields(n, 8))
    hits = 0
    trials = 3000
    for s in range(trials):
        sigma = oracle.exact_round_params(P, 10_000 + s, 0, 0)["sigma"]
        v = (sigma * j) % n
        v = v - n if v >= n // 2 else v
        hits += abs(v) <= C
    bound = 4 * C / n
    assert hits / trials <= bound + 4 * math.sqrt(bound / trials) + 1e-3


# ------------------------------------------------------------------------------------------------
# Location ladder on synthetic bins (reading of Alg. 1's phase step at delta >> 1/(4 n^2 L))
# ------------------------------------------------------------------------------------------------


@pytest.mark.parametrize("m,B,tau", [(22, 256, 1e-4), (22, 16, 1e-4), (26, 16, 1e-4), (14, 32, 1e-4), (22, 16, 1e-2)])
def test_exact_decode_ladder_on_synthetic_bins(m, B, tau):
    n = 1 << m
    P = oracle_params(exact_fields(n, 64, tau_dec=tau))
    rng = np.random.default_rng(m * 7 + B)
    alpha = 0.5
    g = oracle.window_taps(n, B, alpha, P.delta) if m <= 22 else None
    Np = n // B
    # the ladder the oracle uses for this B
    f = exact_fields(n, 64, tau_dec=tau, B_min=B, bins_per_k=B / 64)
    rp = oracle.exact_round_params(oracle_params(f), 1, 0, 0)
    shifts = rp["shifts"]
    assert rp["B"] == B and shifts[0] == B
    assert all(s % B == 0 for s in shifts)
    # the coarsest measurement keeps a tolerance >= tau, and so does every finer one relative to
    # the next coarser (pi / ratio)
    assert math.pi * shifts[-1] / n >= tau * 0.999 or shifts[-1] == B * (Np // 2)
    for s0, s1 in zip(shifts[:-1], shifts[1:]):
        assert math.pi * s0 / s1 >= tau
    for _ in range(30):
        sigma = int(rng.integers(0, n)) | 1
        b = int(rng.integers(0, n))
        i = int(rng.integers(0, n))
        X = np.exp(2j * np.pi * rng.uniform())
        p = (sigma * (i - b)) % n
        j, o = oracle.bin_offset(p, n, B)
        if abs(o) > 0.3 * Np:  # keep the gain near one so the synthetic magnitude passes thr
            continue
        gain = oracle.window_response(n, g, -o) if g is not None else 1.0
        rows = []
        for sh in [0] + shifts:
            u = np.zeros(B, dtype=np.complex128)
            phase = np.exp(-2j * np.pi * ((sh * sigma * i) % n) / n)
            # a phase error of a fifth of the tolerance, magnitude untouched
            u[j] = X * gain * phase * np.exp(1j * 0.2 * tau * rng.standard_normal())
            rows.append(u)
        wi, wv, above = oracle.exact_decode(P, B, alpha, sigma, b, shifts, np.stack(rows))
        if g is None:
            continue  # the gain table at 2^26 is too slow to build here; location is checked below
        assert above == 1 and len(wi) == 1
        assert int(wi[0]) == i
        assert abs(wv[0] - X) < 6 * 0.2 * tau + 1e-6
    # a collision (two coefficients in one bin) is rejected by the isolation check
    if g is not None:
        sigma, b = 12345 | 1, 777
        i1 = 1000
        p1 = (sigma * (i1 - b)) % n
        j, _ = oracle.bin_offset(p1, n, B)
        i2 = (i1 + oracle.inverse_mod_pow2(sigma, n) * (Np // 4)) % n  # same bin, pi differs by n/4B
        rows = []
        for sh in [0] + shifts:
            u = np.zeros(B, dtype=np.complex128)
            for ii in (i1, i2):
                u[j] += np.exp(-2j * np.pi * ((sh * sigma * ii) % n) / n)
            rows.append(u)
        wi, wv, above = oracle.exact_decode(P, B, alpha, sigma, b, shifts, np.stack(rows))
        assert above == 1 and len(wi) == 0


# ------------------------------------------------------------------------------------------------
# NoiselessSparseFFT end to end (Theorem of Sec. 3; Sec. 5 reduction)
# ------------------------------------------------------------------------------------------------


def test_sfft_exact_config1_success_rate():
    """n = 2^14, k = 8, delta = 1e-8, B = 4k, FP64: the Theorem promises success w.p. >= 2/3."""
    n, k = 1 << 14, 8
    P = oracle_params(exact_fields(n, k, delta=1e-8))
    ok = 0
    runs = 60
    for inst in range(runs):
        sig = workloads.exact_sparse(n, k, workloads.seed_for(1, inst), dtype=np.complex128)
        zi, zv, flag = oracle.sfft_exact(P, sig.x, workloads.seed_for(1, inst))
        if np.array_equal(zi.astype(np.int64), sig.support) and np.max(np.abs(zv - sig.values)) < 1e-5:
            ok += 1
    assert ok >= 2 * runs / 3
    assert ok >= 0.9 * runs  # with these constants failures are rare (about 4% measured over 200 seeds)


def test_sfft_exact_matches_full_fft_on_complex64_input():
    """The recovered spectrum equals numpy's FFT of the very same complex64 samples."""
    n, k = 1 << 18, 64
    P = oracle_params(exact_fields(n, k))
    sig = workloads.exact_sparse(n, k, workloads.seed_for(2, 0), dtype=np.complex64)
    zi, zv, flag = oracle.sfft_exact(P, sig.x.astype(np.complex128), 11)
    X = np.fft.fft(sig.x.astype(np.complex128))
    assert np.array_equal(zi.astype(np.int64), sig.support)
    assert np.max(np.abs(zv - X[sig.support])) < 1e-5
    assert flag == 0


@pytest.mark.parametrize("kdim", [16, 64])
def test_reduction_section5(kdim):
    """Sec. 5: y_t = s_{t mod k}; DFT_n(y) = (n/k) DFT_k(s) on the multiples of n/k, zero elsewhere."""
    n = 1 << 14
    y, S = workloads.periodic_extension(n, kdim, 31 + kdim)
    scale = n // kdim
    P = oracle_params(exact_fields(n, kdim, thr=0.5 * scale, delta=1e-9))
    zi, zv, flag = oracle.sfft_exact(P, y, 2024)
    assert np.array_equal(zi.astype(np.int64), np.arange(kdim) * scale)
    assert np.max(np.abs(zv / scale - S)) < 1e-6


# ------------------------------------------------------------------------------------------------
# General case (Alg. 2 and 3)
# ------------------------------------------------------------------------------------------------


def test_locate_inner_keeps_an_isolated_tone_in_its_region():
    """Lemma "LocateInner": for an isolated tone, pi(i) stays in [l'_j, l'_j + 4w/t] at every level."""
    n, B = 1 << 14, 16
    P = oracle_params(general_fields(n, 4))
    t, tp, dmax = oracle.locate_geometry(P, B)
    assert (t, tp) == (8, 2)
    Np = n // B
    F = oracle.FRAC_BITS
    X = np.zeros(n, dtype=np.complex128)
    i0 = 5171
    X[i0] = 2.0 * np.exp(0.7j)
    x = np.fft.ifft(X)
    seed, r = 99, 0
    d = oracle.locate_draws(P, seed, 0, r, B, 1, 0)
    sigma, b = d["sigma"], d["b"]
    tau = (sigma * (i0 - b)) % n
    j0, _ = oracle.bin_offset(tau, n, B)
    l_fp = np.array([((j * Np - Np // 2) % n) << F for j in range(B)], dtype=np.uint64)
    valid = np.ones(B, dtype=np.uint8)
    for D in range(1, dmax + 1):
        w = Np >> ((D - 1) * int(math.log2(tp)))
        us, ups, betas = [], [], []
        for q in range(P.R_loc):
            dd = oracle.locate_draws(P, seed, 0, r, B, D, q)
            lo, hi = oracle.beta_range(P, t, w)
            assert lo <= dd["beta"] <= hi
            us.append(oracle.hash_to_bins(x, sigma, dd["a"], b, B, P.alpha0, P.delta))
            ups.append(oracle.hash_to_bins(x, sigma, (dd["a"] + dd["beta"]) % n, b, B, P.alpha0, P.delta))
            betas.append(dd["beta"])
        l_fp, valid, votes = oracle.locate_inner_votes(P, B, sigma, b, t, w << F, betas, np.stack(us),
                                                       np.stack(ups), l_fp, valid)
        assert valid[j0] == 1
        lo_pos = l_fp[j0] / float(1 << F)
        width = 4.0 * w / t
        rel = (tau - lo_pos) % n
        assert -1e-9 <= rel <= width + 1e-9
    L = oracle.locate_signal(P, x, seed, 0, r, B)
    assert i0 in L.tolist()


def test_estimate_values_exact_on_isolated_coefficients():
    """Lemma "indexestimate" in the noiseless limit: the median of the per-hashing estimates of an
    isolated coefficient is the coefficient, and the top-k' keeps the planted ones."""
    n, k = 1 << 14, 6
    P = oracle_params(general_fields(n, k))
    sig = workloads.exact_sparse(n, k, 321, dtype=np.complex128)
    L = np.sort(np.concatenate([sig.support, np.array([11, 777, 9000])])).astype(np.uint64)
    wi, wv = oracle.estimate_values(P, sig.x, 5, 0, 0, 64, L, k)
    assert np.array_equal(wi.astype(np.int64), sig.support)
    assert np.max(np.abs(wv - sig.values)) < 1e-5


def test_median_is_robust_to_minority_outliers():
    """Separate medians of Re and Im ignore up to (R_est-1)/2 corrupted hashings (Lemma indexestimate)."""
    n, B = 1 << 12, 16
    P = oracle_params(general_fields(n, 4))
    rng = np.random.default_rng(3)
    i = 1234
    X = 1.5 - 0.5j
    sig_, bs, as_, rows = [], [], [], []
    for q in range(5):
        sigma, b, a = int(rng.integers(0, n)) | 1, int(rng.integers(0, n)), int(rng.integers(0, n))
        p = (sigma * (i - b)) % n
        j, o = oracle.bin_offset(p, n, B)
        u = np.zeros(B, dtype=np.complex128)
        g = oracle.window_taps(n, B, P.alpha0, P.delta)
        gain = oracle.window_response(n, g, -o)
        u[j] = X * gain * np.exp(-2j * np.pi * ((a * sigma * i) % n) / n)
        if q in (1, 3):
            u[j] += 40.0 * np.exp(1j * q)  # corrupted hashings
        sig_.append(sigma)
        bs.append(b)
        as_.append(a)
        rows.append(u)
    wi, wv = oracle.estimate_from_bins(P, B, P.alpha0, sig_, bs, as_, np.stack(rows), [i], 1)
    assert list(wi) == [i]
    assert abs(wv[0] - X) < 1e-9 or abs(wv[0] - X) < 1e-6


def test_sfft_general_l2l2_guarantee():
    """Theorem of Sec. 4: ||X - zhat||_2 <= (1 + eps) Err(X, k) + delta ||X||_2 with prob. >= 2/3."""
    n, k = 1 << 13, 8
    P = oracle_params(general_fields(n, k))
    good = 0
    runs = 9
    for inst in range(runs):
        sig = workloads.general_noisy(n, k, workloads.seed_for(3, inst), dtype=np.complex128)
        X = np.fft.fft(sig.x)
        err_k = np.sqrt(np.sum(np.sort(np.abs(X) ** 2)[: n - k]))
        zi, zv, flag = oracle.sfft_general(P, sig.x, workloads.seed_for(3, inst))
        Z = np.zeros(n, dtype=np.complex128)
        Z[zi.astype(np.int64)] = zv
        lhs = np.linalg.norm(X - Z)
        if lhs <= (1 + P.eps) * err_k + P.delta * np.linalg.norm(X):
            good += 1
    assert good >= 2 * runs / 3
