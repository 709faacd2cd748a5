"""Plain FP64 CPU oracle of the sparse FFT (Hassanieh, Indyk, Katabi, Price 2012).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The product library (``paper_1201_2501_gb300``) never imports,
links or runs anything from here, and this package imports nothing from it.

The arithmetic lives in ``sfft_oracle.c`` (plain C, double precision, each function citing the part
of the paper it restates).  This module compiles it with gcc on first use and exposes it through
ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfft_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libsfft_oracle.so")
_lock = threading.Lock()
_lib = None

MODE_EXACT = 0
MODE_GENERAL = 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsfft_oracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``or_params`` in sfft_oracle.c (field order matters)."""

    _fields_ = [
        ("n", ctypes.c_uint64),
        ("k", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("delta", ctypes.c_double),
        ("alpha0", ctypes.c_double),
        ("bins_per_k", ctypes.c_double),
        ("B_min", ctypes.c_uint32),
        ("extra_rounds", ctypes.c_uint32),
        ("thr", ctypes.c_double),
        ("tau_dec", ctypes.c_double),
        ("iso_tol", ctypes.c_double),
        ("gmin", ctypes.c_double),
        ("prune", ctypes.c_double),
        ("ref_lo", ctypes.c_double),
        ("ref_hi", ctypes.c_double),
        ("ref_tol", ctypes.c_double),
        ("z_cap", ctypes.c_uint32),
        ("eps", ctypes.c_double),
        ("t_regions", ctypes.c_uint32),
        ("R_loc", ctypes.c_uint32),
        ("R_est", ctypes.c_uint32),
        ("s", ctypes.c_double),
        ("est_gmin", ctypes.c_double),
    ]


def make_params(**fields) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        if name not in fields:
            raise KeyError(f"oracle parameter {name!r} missing")
        setattr(p, name, fields[name])
    extra = set(fields) - {f for f, _ in Params._fields_}
    if extra:
        raise KeyError(f"unknown oracle parameters {sorted(extra)}")
    return p


_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dblp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_P = ctypes.POINTER(Params)


def _declare(lib):
    u64, u32, i64, dbl, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sig = {
        "or_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "or_inverse_mod_pow2": (u64, [u64, u64]),
        "or_window_T": (i64, [u64, u32, dbl, dbl]),
        "or_window_taps": (None, [u64, u32, dbl, dbl, i64, _dblp]),
        "or_window_response": (dbl, [u64, i64, _dblp, i64]),
        "or_window_gprime": (dbl, [u64, u32, dbl, dbl, i64]),
        "or_permute": (None, [u64, _dblp, u64, u64, u64, _dblp]),
        "or_bin_offset": (None, [u64, u64, u32, _u64p, _i64p]),
        "or_hash_to_bins": (None, [u64, _dblp, u32, _u64p, _dblp, u64, u64, u64, u32, dbl, dbl, i32, _dblp]),
        "or_exact_rounds": (u32, [_P]),
        "or_exact_round_params": (None, [_P, u64, u32, u32, _u32p, _dblp, _i64p, _u32p, _u64p, _u64p, _u64p, _u64p]),
        "or_exact_decode": (u32, [_P, u32, dbl, u64, u64, u32, _u64p, _dblp, u32, _u64p, _u64p, _dblp, _u32p, _u32p]),
        "or_exact_inner": (u32, [_P, _dblp, u64, u32, u32, u32, _u64p, _dblp, _u64p, _dblp, _u32p, _u32p, _dblp]),
        "or_sfft_exact": (i32, [_P, _dblp, u64, u32, _u64p, _dblp, _u32p]),
        "or_general_rounds": (u32, [_P, _u32p, _u32p]),
        "or_locate_geometry": (None, [_P, u32, _u32p, _u32p, _u32p]),
        "or_beta_range": (None, [_P, u32, u64, _u64p, _u64p]),
        "or_locate_draws": (None, [_P, u64, u32, u32, u32, u32, u32, _u64p, _u64p, _u64p, _u64p]),
        "or_estimate_draws": (None, [_P, u64, u32, u32, u32, _u64p, _u64p, _u64p]),
        "or_locate_inner_votes": (None, [_P, u32, u64, u64, u32, u64, u32, _u64p, _dblp, _dblp, _u64p, _u8p, _u32p]),
        "or_locate_signal": (u32, [_P, _dblp, u64, u32, u32, u32, u32, _u64p, _dblp, _u64p]),
        "or_estimate_from_bins": (u32, [_P, u32, dbl, u32, _u64p, _u64p, _u64p, _dblp, u32, _u64p, u32, _u64p, _dblp]),
        "or_estimate_values": (u32, [_P, _dblp, u64, u32, u32, u32, u32, _u64p, _dblp, u32, _u64p, u32, _u64p, _dblp]),
        "or_sfft_general": (i32, [_P, _dblp, u64, u32, _u64p, _dblp, _u32p]),
        "or_samples_per_hashing": (i64, [u64, u32, dbl, dbl]),
        "or_paper_exact_decode": (u32, [_P, u32, u64, _dblp, _dblp, _u64p, _dblp, _u32p, _u32p]),
        "or_paper_exact_inner": (u32, [_P, _dblp, u64, u32, u32, u32, _u64p, _dblp, _u64p, _dblp, _u32p, _u32p,
                                       _dblp]),
        "or_sfft_exact_paper": (i64, [_P, _dblp, u64, u32, _u64p, _dblp, u64]),
        "or_locate_inner_votes_ex": (None, [_P, u32, u64, u64, u32, u64, u32, _u64p, _dblp, _dblp, i32, _u64p, _u8p,
                                            _u32p]),
        "or_locate_replay": (None, [_P, u32, u64, u64, u32, _u64p, _dblp, _dblp, i32, _u64p, _u8p, _u64p]),
        "or_locate_signal_ex": (u32, [_P, _dblp, u64, u32, u32, u32, u32, _u64p, _dblp, i32, _u64p, _u64p]),
        "or_sfft_general_ex": (i32, [_P, _dblp, u64, u32, i32, _u64p, _dblp, _u32p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            _lib = ctypes.CDLL(path)
            _declare(_lib)
    return _lib


# ---------------------------------------------------------------------------------------------
# numpy helpers
# ---------------------------------------------------------------------------------------------
def _c128(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    return a


def _dp(a):
    return a.ctypes.data_as(_dblp)


def _u64(a):
    return a.ctypes.data_as(_u64p)


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def inverse_mod_pow2(sigma, n):
    return int(lib().or_inverse_mod_pow2(sigma, n))


def window_T(n, B, alpha, delta):
    return int(lib().or_window_T(n, B, alpha, delta))


def window_taps(n, B, alpha, delta):
    T = window_T(n, B, alpha, delta)
    g = np.zeros(T + 1, dtype=np.float64)
    lib().or_window_taps(n, B, alpha, delta, T, _dp(g))
    return g


def window_response(n, taps, l):
    g = np.ascontiguousarray(taps, dtype=np.float64)
    return float(lib().or_window_response(n, len(g) - 1, _dp(g), int(l)))


def window_gprime(n, B, alpha, delta, l):
    return float(lib().or_window_gprime(n, B, alpha, delta, int(l)))


def permute(x, sigma, a, b):
    x = _c128(x)
    out = np.zeros_like(x)
    lib().or_permute(len(x), _dp(x), sigma, a, b, _dp(out))
    return out


def bin_offset(p, n, B):
    j = ctypes.c_uint64()
    o = ctypes.c_int64()
    lib().or_bin_offset(p, n, B, ctypes.byref(j), ctypes.byref(o))
    return int(j.value), int(o.value)


def _z_arrays(z_idx, z_val):
    zi = np.ascontiguousarray(np.asarray(z_idx if z_idx is not None else [], dtype=np.uint64))
    zv = _c128(z_val if z_val is not None else np.zeros(0))
    if zi.shape[0] != zv.shape[0]:
        raise ValueError("z_idx and z_val differ in length")
    return zi, zv


def hash_to_bins(x, sigma, a, b, B, alpha, delta, z_idx=None, z_val=None, use_gprime=False):
    x = _c128(x)
    zi, zv = _z_arrays(z_idx, z_val)
    u = np.zeros(B, dtype=np.complex128)
    lib().or_hash_to_bins(len(x), _dp(x), len(zi), _u64(zi), _dp(zv), sigma, a, b, B, alpha, delta,
                          1 if use_gprime else 0, _dp(u))
    return u


def exact_rounds(P):
    return int(lib().or_exact_rounds(ctypes.byref(P)))


def exact_round_params(P, seed, stream, t):
    B = ctypes.c_uint32()
    alpha = ctypes.c_double()
    T = ctypes.c_int64()
    ns = ctypes.c_uint32()
    shifts = (ctypes.c_uint64 * 4)()
    sigma, sinv, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    lib().or_exact_round_params(ctypes.byref(P), seed, stream, t, ctypes.byref(B), ctypes.byref(alpha),
                                ctypes.byref(T), ctypes.byref(ns), shifts, ctypes.byref(sigma), ctypes.byref(sinv),
                                ctypes.byref(b))
    return dict(B=B.value, alpha=alpha.value, T=T.value, shifts=[int(shifts[i]) for i in range(ns.value)],
                sigma=sigma.value, sigma_inv=sinv.value, b=b.value)


def exact_decode(P, B, alpha, sigma, b, shifts, u, z_idx=None, with_kept=False):
    """Decode of one round on given bins ``u`` (shape (1+L, B): a = 0 first, then each shift).

    ``z_idx`` are the indices already in zhat (they enable the re-estimation of known values)."""
    u = _c128(u).reshape(len(shifts) + 1, B)
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.uint64))
    zi = np.ascontiguousarray(np.asarray(z_idx if z_idx is not None else [], dtype=np.uint64))
    wi = np.zeros(B, dtype=np.uint64)
    wv = np.zeros(B, dtype=np.complex128)
    above = ctypes.c_uint32()
    kept = ctypes.c_uint32()
    c = lib().or_exact_decode(ctypes.byref(P), B, alpha, sigma, b, len(sh), _u64(sh), _dp(u), len(zi), _u64(zi),
                              _u64(wi), _dp(wv), ctypes.byref(above), ctypes.byref(kept))
    if with_kept:
        return wi[:c].copy(), wv[:c].copy(), int(above.value), int(kept.value)
    return wi[:c].copy(), wv[:c].copy(), int(above.value)


def exact_inner(P, x, seed, stream, t, z_idx=None, z_val=None):
    x = _c128(x)
    zi, zv = _z_arrays(z_idx, z_val)
    rp = exact_round_params(P, seed, stream, t)
    B = rp["B"]
    wi = np.zeros(B, dtype=np.uint64)
    wv = np.zeros(B, dtype=np.complex128)
    above = ctypes.c_uint32()
    kept = ctypes.c_uint32()
    u = np.zeros((len(rp["shifts"]) + 1) * B, dtype=np.complex128)
    c = lib().or_exact_inner(ctypes.byref(P), _dp(x), seed, stream, t, len(zi), _u64(zi), _dp(zv), _u64(wi), _dp(wv),
                             ctypes.byref(above), ctypes.byref(kept), _dp(u))
    return dict(idx=wi[:c].copy(), val=wv[:c].copy(), n_above=int(above.value), n_kept=int(kept.value),
                bins=u.reshape(len(rp["shifts"]) + 1, B), **rp)


def sfft_exact(P, x, seed, stream=0):
    x = _c128(x)
    cap = P.z_cap
    oi = np.zeros(cap, dtype=np.uint64)
    ov = np.zeros(cap, dtype=np.complex128)
    cnt = ctypes.c_uint32()
    flag = lib().or_sfft_exact(ctypes.byref(P), _dp(x), seed, stream, _u64(oi), _dp(ov), ctypes.byref(cnt))
    c = cnt.value
    return oi[:c].copy(), ov[:c].copy(), int(flag)


def general_rounds(P):
    kr = (ctypes.c_uint32 * 64)()
    Bs = (ctypes.c_uint32 * 64)()
    R = lib().or_general_rounds(ctypes.byref(P), kr, Bs)
    return [int(kr[i]) for i in range(R)], [int(Bs[i]) for i in range(R)]


def locate_geometry(P, B):
    t, tp, dmax = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    lib().or_locate_geometry(ctypes.byref(P), B, ctypes.byref(t), ctypes.byref(tp), ctypes.byref(dmax))
    return int(t.value), int(tp.value), int(dmax.value)


def beta_range(P, t, w):
    lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
    lib().or_beta_range(ctypes.byref(P), t, w, ctypes.byref(lo), ctypes.byref(hi))
    return int(lo.value), int(hi.value)


def locate_draws(P, seed, stream, r, B, D, q):
    s, b, a, be = (ctypes.c_uint64() for _ in range(4))
    lib().or_locate_draws(ctypes.byref(P), seed, stream, r, B, D, q, ctypes.byref(s), ctypes.byref(b),
                          ctypes.byref(a), ctypes.byref(be))
    return dict(sigma=s.value, b=b.value, a=a.value, beta=be.value)


def estimate_draws(P, seed, stream, r, q):
    s, b, a = (ctypes.c_uint64() for _ in range(3))
    lib().or_estimate_draws(ctypes.byref(P), seed, stream, r, q, ctypes.byref(s), ctypes.byref(b), ctypes.byref(a))
    return dict(sigma=s.value, b=b.value, a=a.value)


FRAC_BITS = 16


def locate_inner_votes(P, B, sigma, b, t, w_fp, betas, u, up, l_fp, valid, paper=False):
    """One LocateInner level on given bins; returns updated (l_fp, valid, votes).

    ``paper=True`` moves each region by the listing's min Q* instead of the four best subregions."""
    betas = np.ascontiguousarray(np.asarray(betas, dtype=np.uint64))
    nrep = len(betas)
    u = _c128(u).reshape(nrep, B)
    up = _c128(up).reshape(nrep, B)
    l_fp = np.ascontiguousarray(np.asarray(l_fp, dtype=np.uint64)).copy()
    valid = np.ascontiguousarray(np.asarray(valid, dtype=np.uint8)).copy()
    votes = np.zeros(B * t, dtype=np.uint32)
    lib().or_locate_inner_votes_ex(ctypes.byref(P), B, sigma, b, t, w_fp, nrep, _u64(betas), _dp(u), _dp(up),
                                   1 if paper else 0, _u64(l_fp), valid.ctypes.data_as(_u8p),
                                   votes.ctypes.data_as(_u32p))
    return l_fp, valid, votes.reshape(B, t)


def locate_signal(P, x, seed, stream, r, B, z_idx=None, z_val=None, paper=False, with_candidates=False):
    """LocateSignal: the sorted, de-duplicated list L (and, with ``with_candidates``, each bin's
    candidate, ``BOTTOM`` for a bin without a region)."""
    x = _c128(x)
    zi, zv = _z_arrays(z_idx, z_val)
    L = np.zeros(B, dtype=np.uint64)
    cand = np.zeros(B, dtype=np.uint64)
    c = lib().or_locate_signal_ex(ctypes.byref(P), _dp(x), seed, stream, r, B, len(zi), _u64(zi), _dp(zv),
                                  1 if paper else 0, _u64(L), _u64(cand))
    if with_candidates:
        return L[:c].copy(), cand
    return L[:c].copy()


BOTTOM = np.uint64(0xFFFFFFFFFFFFFFFF)


def locate_replay(P, B, sigma, b, betas, u, up, paper=False):
    """LocateSignal's level loop on given bins (the replay of a run's own bins).

    ``u`` / ``up``: (dmax * nrep, B) bins at a_q and a_q + beta_q, level-major; ``betas`` the matching
    shifts.  Returns (regions (dmax, B) fixed point, valid (dmax, B), candidates (B), BOTTOM for none)."""
    betas = np.ascontiguousarray(np.asarray(betas, dtype=np.uint64))
    _, _, dmax = locate_geometry(P, B)
    if len(betas) % dmax:
        raise ValueError("betas must hold dmax x nrep shifts")
    nrep = len(betas) // dmax
    u = _c128(u).reshape(dmax * nrep, B)
    up = _c128(up).reshape(dmax * nrep, B)
    lfp = np.zeros((dmax, B), dtype=np.uint64)
    valid = np.zeros((dmax, B), dtype=np.uint8)
    cand = np.zeros(B, dtype=np.uint64)
    lib().or_locate_replay(ctypes.byref(P), B, sigma, b, nrep, _u64(betas), _dp(u), _dp(up), 1 if paper else 0,
                           _u64(lfp), valid.ctypes.data_as(_u8p), _u64(cand))
    return lfp, valid, cand


def estimate_from_bins(P, B, alpha, sigmas, bs, as_, u, L, kprime):
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.uint64))
    bb = np.ascontiguousarray(np.asarray(bs, dtype=np.uint64))
    aa = np.ascontiguousarray(np.asarray(as_, dtype=np.uint64))
    nrep = len(sig)
    u = _c128(u).reshape(nrep, B)
    L = np.ascontiguousarray(np.asarray(L, dtype=np.uint64))
    wi = np.zeros(max(len(L), 1), dtype=np.uint64)
    wv = np.zeros(max(len(L), 1), dtype=np.complex128)
    c = lib().or_estimate_from_bins(ctypes.byref(P), B, alpha, nrep, _u64(sig), _u64(bb), _u64(aa), _dp(u), len(L),
                                    _u64(L), kprime, _u64(wi), _dp(wv))
    return wi[:c].copy(), wv[:c].copy()


def estimate_values(P, x, seed, stream, r, B, L, kprime, z_idx=None, z_val=None):
    x = _c128(x)
    zi, zv = _z_arrays(z_idx, z_val)
    L = np.ascontiguousarray(np.asarray(L, dtype=np.uint64))
    wi = np.zeros(max(len(L), 1), dtype=np.uint64)
    wv = np.zeros(max(len(L), 1), dtype=np.complex128)
    c = lib().or_estimate_values(ctypes.byref(P), _dp(x), seed, stream, r, B, len(zi), _u64(zi), _dp(zv), len(L),
                                 _u64(L), kprime, _u64(wi), _dp(wv))
    return wi[:c].copy(), wv[:c].copy()


def sfft_general(P, x, seed, stream=0, paper=False):
    """SparseFFT (Algorithm 2); ``paper=True`` uses LocateInner's min Q* as printed."""
    x = _c128(x)
    cap = P.z_cap
    oi = np.zeros(cap, dtype=np.uint64)
    ov = np.zeros(cap, dtype=np.complex128)
    cnt = ctypes.c_uint32()
    flag = lib().or_sfft_general_ex(ctypes.byref(P), _dp(x), seed, stream, 1 if paper else 0, _u64(oi), _dp(ov),
                                    ctypes.byref(cnt))
    c = cnt.value
    return oi[:c].copy(), ov[:c].copy(), int(flag)


def sfft(P, x, seed, stream=0):
    return sfft_exact(P, x, seed, stream) if P.mode == MODE_EXACT else sfft_general(P, x, seed, stream)


def samples_per_hashing(n, B, alpha, delta):
    return int(lib().or_samples_per_hashing(n, B, alpha, delta))


# ---------------------------------------------------------------------------------------------
# Paper mode of Algorithm 1 (the literal decode, integer coefficients)
# ---------------------------------------------------------------------------------------------
def paper_exact_decode(P, B, sigma, u, up):
    """Algorithm 1's decode on given bins at a = 0 (``u``) and a = 1 (``up``).

    Returns (indices, values, bins they came from, |J|), sorted by index."""
    u = _c128(u)
    up = _c128(up)
    wi = np.zeros(B, dtype=np.uint64)
    wv = np.zeros(B, dtype=np.complex128)
    wj = np.zeros(B, dtype=np.uint32)
    above = ctypes.c_uint32()
    c = lib().or_paper_exact_decode(ctypes.byref(P), B, sigma, _dp(u), _dp(up), _u64(wi), _dp(wv),
                                    wj.ctypes.data_as(_u32p), ctypes.byref(above))
    return wi[:c].copy(), wv[:c].copy(), wj[:c].copy(), int(above.value)


def paper_exact_inner(P, x, seed, stream, t, z_idx=None, z_val=None):
    """One literal NoiselessSparseFFTInner round (hashings at a = 0 and a = 1, Ghat' subtraction)."""
    x = _c128(x)
    zi, zv = _z_arrays(z_idx, z_val)
    rp = exact_round_params(P, seed, stream, t)
    B = rp["B"]
    wi = np.zeros(B, dtype=np.uint64)
    wv = np.zeros(B, dtype=np.complex128)
    wj = np.zeros(B, dtype=np.uint32)
    above = ctypes.c_uint32()
    u = np.zeros(2 * B, dtype=np.complex128)
    c = lib().or_paper_exact_inner(ctypes.byref(P), _dp(x), seed, stream, t, len(zi), _u64(zi), _dp(zv), _u64(wi),
                                   _dp(wv), wj.ctypes.data_as(_u32p), ctypes.byref(above), _dp(u))
    return dict(idx=wi[:c].copy(), val=wv[:c].copy(), bin=wj[:c].copy(), n_above=int(above.value),
                bins=u.reshape(2, B), **rp)


def sfft_exact_paper(P, x, seed, stream=0, cap=1 << 16):
    """NoiselessSparseFFT as printed: the non-zero entries of zhat (indices ascending)."""
    x = _c128(x)
    oi = np.zeros(cap, dtype=np.uint64)
    ov = np.zeros(cap, dtype=np.complex128)
    c = lib().or_sfft_exact_paper(ctypes.byref(P), _dp(x), seed, stream, _u64(oi), _dp(ov), cap)
    if c < 0:
        raise ValueError("zhat outgrew cap")
    return oi[:c].copy(), ov[:c].copy()
