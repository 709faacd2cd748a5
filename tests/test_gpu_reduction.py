"""The reduction of Sec. 5 on the GPU: the k-point DFT of x through the n-point exact sparse FFT of its
periodic extension y_i = x_{i mod k}, with every sample the algorithm asks for read from the k stored
values (sfft_request.period = k), never expanded to n.

Y is k-sparse on the multiples of n/k with Y_{j n/k} = (n/k) DFT_k(x)_j, so the recovered support must
be exactly {j n/k} (bit for bit) and the values (n/k) DFT_k(x) within the FP32 tolerance; at sizes the
oracle can expand, the oracle run on the expanded y gives the same support and values.
"""
import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2501_gb300 import build, sfft

    build.build()
    sfft.lib()
    return sfft


def gpu_params(sf, fields, precision=0):
    p = sf.sfft_params_default(fields["n"], fields["k"], fields["mode"])
    for name, _ in sf.SfftParams._fields_:
        if name in fields:
            setattr(p, name, fields[name])
    p.precision = precision
    return p


def _run(sf, p, xs, periods, seed):
    plan = sf.Plan(p, len(xs))
    out = sf.sfft_execute_requests(plan, xs, [seed] * len(xs), list(range(len(xs))), p.z_cap, periods=periods)
    torch.cuda.synchronize()
    idx, val, cnt, flag = (t.cpu().numpy() for t in out)
    plan.close()
    res = []
    for r in range(len(xs)):
        c = int(cnt[r])
        res.append((idx[r, :c].view(np.uint32).astype(np.int64), val[r, :c, 0] + 1j * val[r, :c, 1], int(flag[r])))
    return res


@pytest.mark.parametrize("m,kdim,prec", [(14, 8, 1), (14, 64, 1), (20, 64, 0), (20, 256, 0)])
def test_dft_of_k_points_through_the_sparse_transform(sf, m, kdim, prec):
    n = 1 << m
    scale = n // kdim
    f = exact_fields(n, kdim, thr=0.5 * scale, delta=1e-9 if prec else 1e-6)
    dt = np.complex128 if prec else np.complex64
    sigs = [workloads.periodic_extension(n, kdim, 31 + kdim + i, dtype=dt) for i in range(3)]
    xs = [torch.as_tensor(np.ascontiguousarray(y[:kdim])).cuda() for y, _ in sigs]
    seed = 2024
    got = _run(sf, gpu_params(sf, f, prec), xs, [kdim] * len(xs), seed)
    P = oracle_params(f)
    for r, (y, S) in enumerate(sigs):
        gi, gv, gf = got[r]
        assert gf == 0
        assert np.array_equal(gi, np.arange(kdim) * scale)
        S_in = np.fft.fft(y[:kdim].astype(np.complex128))  # the DFT of the stored (rounded) samples
        assert np.max(np.abs(gv / scale - S_in)) < (1e-9 if prec else 1e-5)
        # the oracle on the expanded signal, same seed and request index
        oi, ov, of = oracle.sfft_exact(P, y.astype(np.complex128), seed, r)
        assert np.array_equal(gi, oi.astype(np.int64))
        assert np.max(np.abs(gv - ov)) / scale < (1e-9 if prec else 1e-5)


def test_dft_through_a_2_to_the_26_point_transform(sf):
    """n = 2^26, k = 1024: y would be 512 MiB; only the 1024 samples of x are stored and read."""
    n, kdim = 1 << 26, 1024
    scale = n // kdim
    f = exact_fields(n, kdim, thr=0.5 * scale)
    y_head, S = workloads.periodic_extension(1 << 12, kdim, 77, dtype=np.complex64)
    x = y_head[:kdim]
    got = _run(sf, gpu_params(sf, f), [torch.as_tensor(np.ascontiguousarray(x)).cuda()], [kdim], 5)[0]
    gi, gv, gf = got
    assert gf == 0
    assert np.array_equal(gi, np.arange(kdim) * scale)
    assert np.max(np.abs(gv / scale - np.fft.fft(x.astype(np.complex128)))) < 1e-5
