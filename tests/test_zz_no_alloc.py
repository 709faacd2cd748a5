"""sfft_hash_to_bins_static, the HashToBins entry point that allocates nothing, against sfft_hash_to_bins
and against the FP64 oracle.

The static entry point serves callers that may not use the CUDA allocator; its scratch is an array
compiled into the library.  On the same inputs its bins must agree with the plan's entry point and
with the oracle's HashToBins within the tolerance of the FP32 parity tests (2e-5 of the largest bin),
on two calls in a row (the second call finds the first call's leftovers in the shared scratch).  This
file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _window_gains(n, taps, B):
    """W(o) = (g_0 + 2 sum_t g_t cos(2 pi o t / n)) / n for o = 0..n/(2B), in FP64 (numpy)."""
    T = len(taps) - 1
    o = np.arange(n // (2 * B) + 1, dtype=np.int64)[:, None]
    t = np.arange(1, T + 1, dtype=np.int64)[None, :]
    ph = ((o * t) % n).astype(np.float64) * (2.0 * np.pi / n)
    return (taps[0] + 2.0 * (np.cos(ph) @ taps[1:])) / n


@pytest.mark.parametrize("n,k,nz", [(1 << 14, 8, 0), (1 << 16, 32, 12), (1 << 18, 64, 40)])
def test_static_hash_to_bins_matches_plan_entry_point(n, k, nz):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1201_2501_gb300 import build, sfft

    build.build()
    f = exact_fields(n, k)
    p = sfft.sfft_params_default(n, k, sfft.SFFT_EXACT)
    for name, _ in sfft.SfftParams._fields_:
        if name in f:
            setattr(p, name, f[name])
    plan = sfft.Plan(p, 1)
    sig = workloads.exact_sparse(n, k, 31337 + n % 101)
    x = torch.as_tensor(sig.x).cuda()
    rng = np.random.default_rng(n + nz)
    zi = zv = None
    if nz:
        zi = torch.as_tensor(np.sort(rng.choice(n, nz, replace=False)).astype(np.int32)).cuda()
        zv = torch.as_tensor(rng.standard_normal((nz, 2))).cuda()
    for t in range(min(plan.rounds, 2)):
        info = plan.round_info(t)
        B, T = info["B"], info["T"]
        taps64 = plan.taps(t)
        taps = torch.as_tensor(taps64.astype(np.float32)).cuda()
        wtab = torch.as_tensor(_window_gains(n, taps64, B)).cuda() if nz else None
        sigma, a, b = int(rng.integers(0, n)) | 1, int(rng.integers(0, n)), int(rng.integers(0, n))
        ref = sfft.sfft_hash_to_bins(plan, t, x, sigma, a, b, zi, zv)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()
        scale = max(1.0, float(np.max(np.abs(ref))))
        zi_o = None if zi is None else zi.cpu().numpy().astype(np.uint64)
        zv_o = None if zv is None else zv.cpu().numpy() @ np.array([1.0, 1.0j])
        ora = oracle.hash_to_bins(sig.x.astype(np.complex128), sigma, a, b, B, info["alpha"], f["delta"], zi_o, zv_o)
        for call in range(2):  # two calls in a row share the static scratch
            out = torch.full((B, 2), float("nan"), dtype=torch.float64, device="cuda")
            sfft.sfft_hash_to_bins_static(n, B, T, taps, wtab, x, sigma, a, b, zi, zv, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref)) <= 2e-5 * scale, f"call {call} of round {t}"
            assert np.max(np.abs((got[:, 0] + 1j * got[:, 1]) - ora)) <= 2e-5 * scale, f"oracle, call {call}"
    # a window whose partial sums exceed the static scratch is refused before any launch
    big_T = (sfft.SFFT_STATIC_SCRATCH_BYTES // (8 * 4096) + 1) * 2048
    dummy = torch.zeros(big_T + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_hash_to_bins_static(n, 4096, big_T, dummy, None, x, 1, 0, 0, None, None,
                                      torch.empty((4096, 2), dtype=torch.float64, device="cuda"))
    assert ei.value.status == sfft.SFFT_ERR_CAPACITY
    plan.close()
    # buffers the C side cannot size-check are refused by the binding before the call
    with pytest.raises(sfft.SfftError) as ei:
        sfft.sfft_hash_to_bins_static(n, 16, 100, torch.zeros(50, dtype=torch.float32, device="cuda"), None, x, 1, 0,
                                      0, None, None, torch.empty((16, 2), dtype=torch.float64, device="cuda"))
    assert ei.value.status == sfft.SFFT_ERR_INVALID_ARG
    with pytest.raises(sfft.SfftError):
        sfft.sfft_hash_to_bins_static(n, 16, 100, torch.zeros(101, dtype=torch.float32), None, x, 1, 0, 0, None, None,
                                      torch.empty((16, 2), dtype=torch.float64, device="cuda"))
