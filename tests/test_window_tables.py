"""The library's host-side window tables (sfft_window_taps / sfft_window_gains, used by every plan)
against the oracle's own construction and its direct summation of the window response, on CPU.

Small tables are summed directly; large ones come from a chirp convolution with the library's FFT.
Both must give W(o) = (1/n)(g_0 + 2 sum_t g_t cos(2 pi o t / n)) to 1e-12 absolute at every sampled
offset (ends, middle and random ones), and the taps must equal the oracle's to 1e-12 relative."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def sf():
    from paper_1201_2501_gb300 import build, sfft

    build.build()
    return sfft


@pytest.mark.parametrize("m,B,alpha,delta", [(14, 32, 0.5, 1e-8), (18, 64, 0.25, 1e-6), (22, 256, 0.5, 1e-6),
                                             (22, 16, 0.0625, 1e-6), (26, 16, 0.015625, 1e-6)])
def test_window_gains_match_direct_summation(sf, m, B, alpha, delta):
    n = 1 << m
    L = n // (2 * B) + 1
    g = sf.sfft_window_taps(n, B, alpha, delta)
    og = oracle.window_taps(n, B, alpha, delta)
    assert len(g) == len(og) == oracle.window_T(n, B, alpha, delta) + 1
    assert np.max(np.abs(g - og)) <= 1e-12 * np.max(np.abs(og))
    W = sf.sfft_window_gains(n, B, alpha, delta, L)
    rng = np.random.default_rng(m)
    offs = np.unique(np.concatenate([[0, 1, 2, L // 2, L - 2, L - 1], rng.integers(0, L, 60)]))
    want = np.array([oracle.window_response(n, og, int(o)) for o in offs])
    assert np.max(np.abs(W[offs] - want)) <= 1e-12
    # the pass band is flat to delta and the gain falls off across the transition band
    assert abs(W[0] - 1.0) <= delta
    assert W[L - 1] < W[0]


def test_window_functions_reject_bad_arguments(sf):
    import ctypes

    T = ctypes.c_int64()
    assert sf.lib().sfft_window_taps(1000, 16, 0.5, 1e-6, ctypes.byref(T), None, 0) == sf.SFFT_ERR_INVALID_ARG
    assert sf.lib().sfft_window_taps(1 << 10, 24, 0.5, 1e-6, ctypes.byref(T), None, 0) == sf.SFFT_ERR_INVALID_ARG
    assert sf.lib().sfft_window_gains(1 << 10, 16, 0.5, 1e-6, (1 << 9) + 2, None) == sf.SFFT_ERR_INVALID_ARG


@pytest.mark.parametrize("m", [6, 11, 16, 22, 26])
def test_twiddle_tables_give_the_roots_of_unity(sf, m):
    """The general mode's FP64 twiddles: w^e = T[e mod 2^sh] T[2^sh + (e >> sh)], w = exp(-2 pi i / n),
    against numpy's exp of the exact angle (e / n is an exact binary fraction) at sampled exponents."""
    n = 1 << m
    tw = sf.sfft_twiddle_tables(n)
    sh = (m + 1) // 2
    assert len(tw) == (1 << sh) + (n >> sh)
    rng = np.random.default_rng(m)
    e = np.unique(np.concatenate([[0, 1, n // 8, n // 4, n // 2, n - 1], rng.integers(0, n, 500)]))
    got = tw[e & ((1 << sh) - 1)] * tw[(1 << sh) + (e >> sh)]
    want = np.exp(-2j * np.pi * (e.astype(np.float64) / n))
    assert np.max(np.abs(got - want)) <= 4e-15  # two roundings of the factors and four of the product
    assert np.max(np.abs(np.abs(tw) - 1.0)) <= 1e-15  # each factor a unit complex number to a few ulp
