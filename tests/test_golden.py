"""The oracle against its stored regression fixtures (tests/golden/oracle_regression.json, written by
tests/golden/make_golden.py from oracle/ only).  Integers (Philox words, T, supports, flags) must be
equal; floating-point values equal to 1e-12 relative (the host's libm may round differently).  A
change here means the oracle's arithmetic changed and must be justified against the paper."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, general_fields, oracle_params

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_regression.json")


@pytest.fixture(scope="module")
def g():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _close(a, b, rel=1e-12):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return np.all(np.abs(a - b) <= rel * np.maximum(1.0, np.abs(b)))


def test_philox_words(g):
    for e in g["philox"]:
        assert [int(w) for w in oracle.philox4x32_10(e["ctr"], e["key"])] == e["out"]


def test_window(g):
    w = g["window"]
    n, B, a, d = w["n"], w["B"], w["alpha"], w["delta"]
    assert oracle.window_T(n, B, a, d) == w["T"]
    taps = oracle.window_taps(n, B, a, d)
    for t, v in w["taps_at"].items():
        assert _close(taps[int(t)], v)
    for o, v in w["W_at"].items():
        assert _close(oracle.window_response(n, taps, int(o)), v)
    for o, v in w["Gprime_at"].items():
        assert _close(oracle.window_gprime(n, B, a, d, int(o)), v)


def test_exact_transforms(g):
    P = oracle_params(exact_fields(1 << 14, 8, delta=1e-8))
    for e in g["exact"]:
        s = workloads.exact_sparse(1 << 14, 8, workloads.seed_for(1, e["instance"]), dtype=np.complex128)
        zi, zv, flag = oracle.sfft_exact(P, s.x, e["seed"], e["request"])
        assert [int(v) for v in zi] == e["idx"] and int(flag) == e["flag"]
        assert _close(np.stack([zv.real, zv.imag], -1), e["val"])


def test_general_transforms(g):
    P = oracle_params(general_fields(1 << 14, 8))
    for e in g["general"]:
        s = workloads.general_noisy(1 << 14, 8, workloads.seed_for(3, e["instance"]))
        zi, zv, flag = oracle.sfft_general(P, s.x.astype(np.complex128), e["seed"], e["request"])
        assert [int(v) for v in zi] == e["idx"] and int(flag) == e["flag"]
        assert _close(np.stack([zv.real, zv.imag], -1), e["val"])


@pytest.mark.gpu
def test_gpu_reproduces_the_stored_exact_results(g):
    """The FP64 device path on the stored inputs gives the stored supports, values within 1e-9."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2501_gb300 import build, sfft

    build.build()
    f = exact_fields(1 << 14, 8, delta=1e-8)
    p = sfft.sfft_params_default(1 << 14, 8, sfft.SFFT_EXACT)
    for name, _ in sfft.SfftParams._fields_:
        if name in f:
            setattr(p, name, f[name])
    p.precision = sfft.SFFT_FP64
    plan = sfft.Plan(p, 1)
    for e in g["exact"]:
        s = workloads.exact_sparse(1 << 14, 8, workloads.seed_for(1, e["instance"]), dtype=np.complex128)
        x = torch.as_tensor(s.x).cuda()
        idx, val, cnt, flag = (t.cpu().numpy() for t in
                               sfft.sfft_execute_requests(plan, [x], [e["seed"]], [e["request"]], p.z_cap))
        c = int(cnt[0])
        assert [int(v) for v in idx[0, :c].view(np.uint32)] == e["idx"] and int(flag[0]) == e["flag"]
        assert np.max(np.abs(val[0, :c] - np.asarray(e["val"]))) <= 1e-9
    plan.close()
