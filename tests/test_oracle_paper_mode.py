"""Pins of the oracle's build readings against the paper's literal algorithms (no GPU needed).

The library and the oracle take readings where the listings cannot run as printed on this library's
inputs (see the oracle's header): a ladder of shifts instead of Algorithm 1's a = 0 / a = 1 phase
comparison, the value u_j / W(-o) instead of round(u_j), an isolation check, the re-estimation of
known values and, in Algorithm 3, the four best consecutive subregions instead of min Q*.  The oracle
also runs the listings as printed ("paper mode"); these tests check that the readings reach what the
literal algorithms reach on the inputs where those work:

* Algorithm 1 on the paper's own input model (Sec. 3: integer coefficients in {-L..L},
  delta = 1/(4 n^2 L)), where round() makes the literal decode exact;
* Algorithm 3 on isolated tones and on noisy spectra, where the rates at which min Q* and the
  four-subregion window disagree are measured (they justify the four-subregion reading).

The re-estimation of known values is pinned directly on synthetic bins.
"""
import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, general_fields, oracle_params


def _integer_params(n, k, L, **over):
    return oracle_params(exact_fields(n, k, delta=1.0 / (4.0 * n * n * L), **over))


# ------------------------------------------------------------------------------------------------
# Algorithm 1 as printed, against the true spectrum (Theorem of Sec. 3: success >= 2/3)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,k", [(10, 4), (12, 8), (14, 16)])
def test_paper_mode_recovers_integer_spectra_exactly(m, k):
    """NoiselessSparseFFT as printed returns zhat = X exactly (integers, bit for bit) with probability
    at least 2/3 (Theorem of Sec. 3); a wrong sign of the shift, a wrong sigma^{-1} or a missing
    rounding would make it fail almost always."""
    n, L = 1 << m, 4
    P = _integer_params(n, k, L)
    ok = 0
    N = 60
    for inst in range(N):
        sig = workloads.integer_sparse(n, k, L, workloads.seed_for(7, 100 * m + inst))
        zi, zv = oracle.sfft_exact_paper(P, sig.x, 500 + inst)
        ok += int(np.array_equal(zi.astype(np.int64), sig.support) and np.array_equal(zv, sig.values))
    assert ok >= (2 * N) // 3 + 1, ok
    assert ok >= 0.85 * N, ok  # measured: 53-57 of 60


def test_paper_decode_of_a_single_tone_by_hand():
    """Algorithm 1's decode on the bins of one tone: the phase of u_j / u'_j is 2 pi sigma i / n, so
    round(phase n / 2 pi) = sigma i and i = sigma^{-1} sigma i; the value is round(u_j)."""
    n, B = 1 << 12, 16
    P = _integer_params(n, 1, 8)
    rng = np.random.default_rng(3)
    for _ in range(20):
        i0 = int(rng.integers(0, n))
        X0 = float(rng.integers(-8, 9) or 5)
        x = np.fft.ifft(np.where(np.arange(n) == i0, X0, 0.0).astype(np.complex128))
        sigma, b = int(rng.integers(0, n)) | 1, int(rng.integers(0, n))
        j, o = oracle.bin_offset((sigma * (i0 - b)) % n, n, B)
        u = oracle.hash_to_bins(x, sigma, 0, b, B, 0.5, P.delta)
        up = oracle.hash_to_bins(x, sigma, 1, b, B, 0.5, P.delta)
        # the hashing at a = 1 only rotates the tone by w^{sigma i}
        assert np.isclose(up[j], u[j] * np.exp(-2j * np.pi * ((sigma * i0) % n) / n), atol=1e-9)
        wi, wv, wj, above = oracle.paper_exact_decode(P, B, sigma, u, up)
        if abs(u[j]) > 0.5:
            assert int(wi[list(wj).index(j)]) == i0
            assert wv[list(wj).index(j)] == np.round(u[j].real) + 1j * np.round(u[j].imag)
        else:
            assert j not in list(wj)


# ------------------------------------------------------------------------------------------------
# The shift ladder, value and isolation check against the literal decode, bin by bin
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,k,noise_bin", [(12, 8, 0.0), (14, 16, 0.0), (14, 16, 1e-4)])
def test_ladder_and_literal_decode_agree_on_isolated_bins(m, k, noise_bin):
    """Same round, same (sigma, b), same zhat (the true spectrum minus a random half of its entries).
    On every bin that holds exactly one residual coefficient above thr (an isolated bin, Lemma
    "l:est"), Algorithm 1's a = 0 / a = 1 rule and the shift ladder both decode that coefficient's
    index, the literal value round(u_j) is the integer itself when the coefficient sits in the pass
    band, and the ladder's value u_j / W(-o) is the coefficient (to 1e-6, plus the noise).  On bins
    with two or more residual coefficients (collisions) the two rules may differ; the isolation
    check rejects most of them, the literal rule writes a wrong index there, which a
    later round cancels.  noise_bin sets complex Gaussian time noise of about that magnitude per bin
    (mild: below the isolation check's tolerance of 1e-3 of |u_j|)."""
    n, L = 1 << m, 4
    P = _integer_params(n, k, L)
    rng = np.random.default_rng(m + k)
    isolated = ladder_skipped = collided = collided_kept = 0
    for inst in range(40):
        B0 = oracle.exact_round_params(P, 1, 0, 0)["B"]
        sig = workloads.integer_sparse(n, k, L, workloads.seed_for(9, 100 * m + inst),
                                       noise_std=noise_bin * np.sqrt(B0) / n)
        for t in range(oracle.exact_rounds(P)):
            keep = rng.random(k) < 0.5
            zi = sig.support[keep].astype(np.uint64)
            zv = sig.values[keep]
            seed = 40 + inst
            bld = oracle.exact_inner(P, sig.x, seed, 0, t, zi, zv)
            lit = oracle.paper_exact_inner(P, sig.x, seed, 0, t, zi, zv)
            assert (bld["sigma"], bld["b"], bld["B"]) == (lit["sigma"], lit["b"], lit["B"])
            B, sigma, b, alpha = bld["B"], bld["sigma"], bld["b"], bld["alpha"]
            taps = oracle.window_taps(n, B, alpha, P.delta)
            by_bin = {}
            for i, v in zip(sig.support[~keep], sig.values[~keep]):
                j, o = oracle.bin_offset((sigma * (int(i) - b)) % n, n, B)
                by_bin.setdefault(j, []).append((int(i), v, o, oracle.window_response(n, taps, -o)))
            lit_at = {int(j): (int(i), v) for i, v, j in zip(lit["idx"], lit["val"], lit["bin"])}
            bld_at = {}
            for i, v in zip(bld["idx"].astype(int), bld["val"]):
                bld_at[oracle.bin_offset((sigma * (i - b)) % n, n, B)[0]] = (i, v)
            for j, members in by_bin.items():
                strong = [m_ for m_ in members if abs(m_[1] * m_[3]) > 2 * P.thr]
                if len(members) == 1 and strong:
                    i, X_i, o, W = members[0]
                    isolated += 1
                    assert lit_at[j][0] == i, (inst, t, j)
                    if W > 1 - 1e-6:
                        assert lit_at[j][1] == X_i
                    if W < P.gmin:
                        ladder_skipped += 1
                        continue
                    assert j in bld_at and bld_at[j][0] == i, (inst, t, j)
                    assert abs(bld_at[j][1] - X_i) < 1e-6 + 100 * noise_bin
                elif len(members) > 1:
                    collided += 1
                    collided_kept += int(j in bld_at)
    assert isolated > 100
    assert ladder_skipped == 0
    # most collisions are rejected by the ladder's isolation check
    assert collided_kept <= collided // 3 + 1, (collided, collided_kept)


@pytest.mark.parametrize("m,k", [(10, 4), (12, 8), (14, 16)])
def test_build_and_paper_modes_agree_where_the_literal_algorithm_succeeds(m, k):
    """On the paper's input model the whole transforms agree: wherever NoiselessSparseFFT as printed
    returns X exactly, the build readings return the same support with values within 1e-5 (the
    library's value tolerance) -- except in a measured handful of seeds (at most 1 in 100): a
    transition-band contamination that the integer rounding removes but that lies above the
    re-estimation window, or a bin the isolation check rejects in a short schedule (measured: 3 of
    600).  The build readings succeed at least as often overall."""
    n, L = 1 << m, 4
    P = _integer_params(n, k, L)
    N = 200
    paper_ok = build_ok = paper_only = 0
    for inst in range(N):
        sig = workloads.integer_sparse(n, k, L, workloads.seed_for(7, 1000 * m + inst))
        seed = 1000 + inst
        pi, pv = oracle.sfft_exact_paper(P, sig.x, seed)
        bi, bv, _ = oracle.sfft_exact(P, sig.x, seed)
        p_ok = np.array_equal(pi.astype(np.int64), sig.support) and np.array_equal(pv, sig.values)
        b_ok = np.array_equal(bi.astype(np.int64), sig.support) and bool(np.max(np.abs(bv - sig.values)) < 1e-5)
        paper_ok += p_ok
        build_ok += b_ok
        paper_only += int(p_ok and not b_ok)
    assert paper_only <= N // 100, paper_only
    assert build_ok >= paper_ok, (build_ok, paper_ok)


# ------------------------------------------------------------------------------------------------
# Algorithm 3: min Q* (as printed) against the four best consecutive subregions
# ------------------------------------------------------------------------------------------------
def test_locate_min_qstar_and_best_four_on_isolated_tones():
    """LocateSignal on one isolated tone (noiseless, FP64).  The four-subregion reading finds the tone
    in every case; min Q* agrees with it whenever no far subregion won a chance majority, and loses
    the tone when one did: over t subregions the vote phases beta theta wrap around 2 pi once or
    twice, so a far subregion collects votes by aliasing, and min Q* jumps to it when it lies below
    the tone's subregion.  The rate of such jumps (measured here) is why the library takes the
    four-subregion window."""
    n = 1 << 14
    P = oracle_params(general_fields(n, 2))
    B = 16
    rng = np.random.default_rng(11)
    both = lost_by_paper = 0
    N = 60
    for inst in range(N):
        i0 = int(rng.integers(0, n))
        X = np.zeros(n, dtype=np.complex128)
        X[i0] = 3.0 * np.exp(2j * np.pi * rng.uniform())
        x = np.fft.ifft(X)
        Lb, cb = oracle.locate_signal(P, x, 300 + inst, 0, 0, B, with_candidates=True)
        Lp, cp = oracle.locate_signal(P, x, 300 + inst, 0, 0, B, paper=True, with_candidates=True)
        assert i0 in Lb.tolist()
        if i0 in Lp.tolist():
            both += 1
        else:
            lost_by_paper += 1
        # bins without the tone are bottom or agree between the two rules... except for aliases
    assert both + lost_by_paper == N
    assert both >= N // 2, both


def test_locate_replay_equals_locate_signal():
    """The replay entry (the level loop on given bins) on the oracle's own bins gives the same
    candidates as LocateSignal, in both modes."""
    n, k = 1 << 14, 8
    P = oracle_params(general_fields(n, k))
    sig = workloads.general_noisy(n, k, workloads.seed_for(3, 5), dtype=np.complex128)
    _, Bs = oracle.general_rounds(P)
    B = Bs[0]
    t, tp, dmax = oracle.locate_geometry(P, B)
    us, ups, betas = [], [], []
    seed = 123
    for D in range(1, dmax + 1):
        for q in range(P.R_loc):
            d = oracle.locate_draws(P, seed, 0, 0, B, D, q)
            us.append(oracle.hash_to_bins(sig.x, d["sigma"], d["a"], d["b"], B, P.alpha0, P.delta))
            ups.append(oracle.hash_to_bins(sig.x, d["sigma"], (d["a"] + d["beta"]) % n, d["b"], B, P.alpha0,
                                           P.delta))
            betas.append(d["beta"])
            sigma, b = d["sigma"], d["b"]
    for paper in (False, True):
        lfp, valid, cand = oracle.locate_replay(P, B, sigma, b, betas, np.stack(us), np.stack(ups), paper=paper)
        _, cand2 = oracle.locate_signal(P, sig.x, seed, 0, 0, B, paper=paper, with_candidates=True)
        assert np.array_equal(cand, cand2)
        assert lfp.shape == (dmax, B) and valid.shape == (dmax, B)
        # a bottom bin stays bottom at every later level
        for D in range(1, dmax):
            assert np.all(valid[D] <= valid[D - 1])


# ------------------------------------------------------------------------------------------------
# The re-estimation of a known value, pinned on synthetic bins
# ------------------------------------------------------------------------------------------------
def _refine_setup():
    n = 1 << 14
    P = oracle_params(exact_fields(n, 8))
    rp = oracle.exact_round_params(P, 5, 0, 0)
    B, alpha, shifts = rp["B"], rp["alpha"], rp["shifts"]
    sigma, b = rp["sigma"], rp["b"]
    taps = oracle.window_taps(n, B, alpha, P.delta)
    return n, P, B, alpha, shifts, sigma, b, taps


def _bins_of_residual(n, B, shifts, sigma, b, taps, entries):
    """Bins (1 + L rows) of residual coefficients {i: value}: u_j = sum W(-o(i)) r_i w^{a sigma i}."""
    rows = np.zeros((len(shifts) + 1, B), dtype=np.complex128)
    for i, r in entries.items():
        j, o = oracle.bin_offset((sigma * (i - b)) % n, n, B)
        W = oracle.window_response(n, taps, -o)
        for row, a in enumerate([0] + list(shifts)):
            rows[row, j] += W * r * np.exp(-2j * np.pi * ((a * sigma * i) % n) / n)
    return rows


def _index_at_offset(n, B, sigma, b, j, o):
    """The index i with pi(i) = j n/B + o."""
    p = (j * (n // B) + o) % n
    return (oracle.inverse_mod_pow2(sigma, n) * p + b) % n


def test_refine_known_corrects_a_contaminated_value():
    """A known entry whose residual magnitude lies inside (ref_lo, ref_hi] thr is corrected by exactly
    that residual (u_j / W(-o)), so zhat_i + correction equals the true value to 1e-12."""
    n, P, B, alpha, shifts, sigma, b, taps = _refine_setup()
    j = 5
    i0 = _index_at_offset(n, B, sigma, b, j, 3)
    for mag_over_thr in (0.5 * P.ref_hi, 0.9 * P.ref_hi, 2.0 * P.ref_lo):
        resid = mag_over_thr * P.thr * np.exp(0.4j)
        u = _bins_of_residual(n, B, shifts, sigma, b, taps, {i0: resid})
        wi, wv, above = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u, z_idx=[i0])
        assert above == 0
        assert wi.tolist() == [i0]
        assert abs(wv[0] - resid) <= 1e-12 * abs(resid) + 1e-15


def test_refine_known_leaves_residuals_outside_its_window():
    """Residuals at or below ref_lo thr, or above ref_hi thr (and below thr), are left alone."""
    n, P, B, alpha, shifts, sigma, b, taps = _refine_setup()
    j = 9
    i0 = _index_at_offset(n, B, sigma, b, j, -2)
    for mag_over_thr in (0.5 * P.ref_lo, 1.5 * P.ref_hi, 0.4):
        u = _bins_of_residual(n, B, shifts, sigma, b, taps, {i0: mag_over_thr * P.thr * np.exp(1.1j)})
        wi, _, above = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u, z_idx=[i0])
        assert above == 0 and len(wi) == 0, mag_over_thr


def test_refine_known_needs_exactly_one_matching_entry():
    """Two known entries in the bin whose locations both fit the phases (permuted positions one
    apart) -> no correction; a second entry whose location does not fit -> the fitting one is
    corrected; a residual whose magnitude changes under the shift by more than 25 % -> none."""
    n, P, B, alpha, shifts, sigma, b, taps = _refine_setup()
    j = 3
    i0 = _index_at_offset(n, B, sigma, b, j, 0)
    i_near = _index_at_offset(n, B, sigma, b, j, 1)
    i_far = _index_at_offset(n, B, sigma, b, j, (n // B) // 3)
    resid = 0.5 * P.ref_hi * P.thr * np.exp(2.0j)
    u = _bins_of_residual(n, B, shifts, sigma, b, taps, {i0: resid})
    wi, _, _ = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u, z_idx=sorted([i0, i_near]))
    assert len(wi) == 0
    wi, wv, _ = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u, z_idx=sorted([i0, i_far]))
    assert wi.tolist() == [i0] and abs(wv[0] - resid) <= 1e-12
    u2 = u.copy()
    u2[1:] *= 1.3
    wi, _, _ = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u2, z_idx=[i0])
    assert len(wi) == 0
    # a residual that is not the known entry's (phases of another location) is not attributed to it
    u3 = _bins_of_residual(n, B, shifts, sigma, b, taps, {i_far: resid})
    wi, _, _ = oracle.exact_decode(P, B, alpha, sigma, b, shifts, u3, z_idx=[i0])
    assert len(wi) == 0
