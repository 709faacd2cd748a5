"""Writes tests/golden/oracle_regression.json from the oracle alone (no GPU code is imported).

The paper prints no worked numeric example, so these are regression fixtures of the oracle: values it
computes today for small, fixed inputs, stored so that any later change to its arithmetic shows up as
a failing test (tests/test_golden.py) and has to be justified against the paper.  Inputs come from the
seeded generators in paper_1201_2501_gb300/workloads.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1201_2501_gb300 import workloads  # noqa: E402
from tests.common import exact_fields, general_fields, oracle_params  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")


def cx(v):
    return [[float(z.real), float(z.imag)] for z in np.asarray(v)]


def main():
    g = {"_source": "written by tests/golden/make_golden.py from oracle/ only; regression fixtures "
                    "(the paper prints no worked numeric example)"}
    # Philox4x32-10 words for a few counters and keys (Salmon et al., SC 2011)
    g["philox"] = [{"ctr": c, "key": k, "out": [int(w) for w in oracle.philox4x32_10(c, k)]}
                   for c, k in (([0, 0, 0, 0], [0, 0]), ([1, 2, 3, 4], [5, 6]),
                                ([0xFFFFFFFF, 0, 7, 0x12345678], [0xDEADBEEF, 0xCAFEF00D]))]
    # flat window of Sec. 7 (the library's reading of its construction): T, a few taps, and the exact response W(o)
    n, B, a, d = 1 << 14, 32, 0.5, 1e-8
    taps = oracle.window_taps(n, B, a, d)
    offs = [0, 1, 64, 128, 192, 255, 256]
    g["window"] = {"n": n, "B": B, "alpha": a, "delta": d, "T": int(oracle.window_T(n, B, a, d)),
                   "taps_at": {str(t): float(taps[t]) for t in (0, 1, 2, 100, 1000, len(taps) - 1)},
                   "W_at": {str(o): oracle.window_response(n, taps, o) for o in offs},
                   "Gprime_at": {str(o): oracle.window_gprime(n, B, a, d, o) for o in offs}}
    # Algorithm 1 on three n = 2^14, k = 8 signals (FP64), request r = stream r
    f = exact_fields(1 << 14, 8, delta=1e-8)
    P = oracle_params(f)
    g["exact"] = []
    for i in range(3):
        s = workloads.exact_sparse(1 << 14, 8, workloads.seed_for(1, i), dtype=np.complex128)
        zi, zv, flag = oracle.sfft_exact(P, s.x, 4321, i)
        g["exact"].append({"instance": i, "seed": 4321, "request": i, "idx": [int(v) for v in zi],
                           "val": cx(zv), "flag": int(flag)})
    # Algorithms 2 and 3 on two noisy n = 2^14, k = 8 signals
    fg = general_fields(1 << 14, 8)
    Pg = oracle_params(fg)
    g["general"] = []
    for i in range(2):
        s = workloads.general_noisy(1 << 14, 8, workloads.seed_for(3, 40 + i))
        zi, zv, flag = oracle.sfft_general(Pg, s.x.astype(np.complex128), 555, i)
        g["general"].append({"instance": 40 + i, "seed": 555, "request": i, "idx": [int(v) for v in zi],
                             "val": cx(zv), "flag": int(flag)})
    with open(OUT, "w") as fh:
        json.dump(g, fh, indent=1)
    print(OUT)


if __name__ == "__main__":
    main()
