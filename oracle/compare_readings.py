"""Measure how the oracle's readings compare with the paper's listings (test infrastructure).

    python -m oracle.compare_readings exact    # Algorithm 1: literal decode vs the build readings
    python -m oracle.compare_readings locate   # Algorithm 3: min Q* vs the four best subregions

`exact`: integer spectra (Sec. 3's input model, delta = 1/(4 n^2 L)), 200 seeds per size; counts the
seeds where both, only one, or neither of the two modes returns X exactly (values within 1e-5).
`locate`: noisy spectra at SNR 20 dB (the general workload), LocateSignal's first call in both modes
on the same hashings: bins whose candidates differ and true coordinates each list holds; then whole
transforms in both modes, mean l2/l2 ratio against Err(X, k).  Runs the oracle only.
"""
from __future__ import annotations

import collections
import sys

import numpy as np

import oracle
from paper_1201_2501_gb300 import workloads

BASE = dict(delta=1e-6, alpha0=0.5, bins_per_k=4.0, B_min=16, extra_rounds=0, thr=0.5, tau_dec=1e-4, iso_tol=1e-3,
            gmin=0.1, prune=0.5, ref_lo=1e-5, ref_hi=2e-2, ref_tol=0.1, eps=1.0, t_regions=0, R_loc=5, R_est=5,
            s=0.25, est_gmin=0.25)


def exact_report(sizes=((10, 4), (12, 8), (14, 8), (14, 16)), N=200, L=4):
    for m, k in sizes:
        n = 1 << m
        P = oracle.make_params(**dict(BASE, n=n, k=k, mode=0, z_cap=max(4 * k, 64), delta=1.0 / (4.0 * n * n * L)))
        c = collections.Counter()
        for inst in range(N):
            sig = workloads.integer_sparse(n, k, L, workloads.seed_for(7, 1000 * m + inst))
            pi, pv = oracle.sfft_exact_paper(P, sig.x, 1000 + inst)
            bi, bv, _ = oracle.sfft_exact(P, sig.x, 1000 + inst)
            p_ok = np.array_equal(pi.astype(np.int64), sig.support) and np.array_equal(pv, sig.values)
            b_ok = np.array_equal(bi.astype(np.int64), sig.support) and bool(np.max(np.abs(bv - sig.values)) < 1e-5)
            c[("both" if p_ok and b_ok else "paper only" if p_ok else "build only" if b_ok else "neither")] += 1
        print(f"n=2^{m} k={k}: {dict(c)}", flush=True)


def locate_report(cases=((16, 32, 7, 0.25), (16, 32, 31, 0.25), (16, 32, 7, 0.125)), N=40):
    for m, k, R_loc, s in cases:
        n = 1 << m
        P = oracle.make_params(**dict(BASE, n=n, k=k, mode=1, z_cap=max(8 * k, 64), bins_per_k=8.0, R_loc=R_loc, s=s))
        B = oracle.general_rounds(P)[1][0]
        c = collections.Counter()
        ratio = {False: [], True: []}
        for inst in range(N):
            sig = workloads.general_noisy(n, k, workloads.seed_for(8, inst), snr_db=20.0, dtype=np.complex128)
            seed = 77 + inst
            Lb, cb = oracle.locate_signal(P, sig.x, seed, 0, 0, B, paper=False, with_candidates=True)
            Lp, cp = oracle.locate_signal(P, sig.x, seed, 0, 0, B, paper=True, with_candidates=True)
            sup = set(sig.support.tolist())
            c["bins"] += B
            c["candidates differ"] += int(np.sum(cb != cp))
            c["true in L (four best)"] += len(sup & set(Lb.astype(int).tolist()))
            c["true in L (min Q*)"] += len(sup & set(Lp.astype(int).tolist()))
            c["true"] += k
            X = np.fft.fft(sig.x)
            err_k = np.sqrt(np.sum(np.sort(np.abs(X) ** 2)[:-k]))
            for paper in (False, True):
                oi, ov, _ = oracle.sfft_general(P, sig.x, seed, 0, paper=paper)
                Z = np.zeros(n, complex)
                Z[oi.astype(int)] = ov
                ratio[paper].append(np.linalg.norm(X - Z) / err_k)
        print(f"n=2^{m} k={k} R_loc={R_loc} s={s}: {dict(c)}; mean l2/l2 four best {np.mean(ratio[False]):.3f}, "
              f"min Q* {np.mean(ratio[True]):.3f}", flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "exact"
    exact_report() if what == "exact" else locate_report()
