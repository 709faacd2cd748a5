"""Multi-channel batches with shared hashing (sfft_execute_channels) against the FP64 oracle.

C signals stored interleaved (row m = sample m of every channel) are transformed with the draws of one
request index: channel c's result must equal the oracle's Algorithm 1 on channel c's signal with that
request index -- supports and flags bit for bit, values within 1e-5 (the FP32 tolerance of the other
exact-mode tests).
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


def _plan(sf, f, batch, **over):
    p = sf.sfft_params_default(f["n"], f["k"], f["mode"])
    for name, _ in sf.SfftParams._fields_:
        if name in f:
            setattr(p, name, f[name])
    for k_, v in over.items():
        setattr(p, k_, v)
    return sf.Plan(p, batch)


STATUS = {0: 0, 1: 8, 2: 7}  # oracle flag -> C ABI status (OK, NOT_CONVERGED, CAPACITY)


def _check_channels(sf, P, x, outs, seed, rid, chans, vtol=1e-5):
    idx, val, cnt, flag = (t.cpu().numpy() for t in outs)
    idx = idx.view(np.uint32)
    for c in chans:
        xc = x[:, c].cpu().numpy().astype(np.complex128)
        oi, ov, of = oracle.sfft_exact(P, xc, seed, rid)
        k = int(cnt[c])
        assert np.array_equal(idx[c, :k].astype(np.int64), oi.astype(np.int64)), f"support of channel {c}"
        if k:
            assert np.max(np.abs((val[c, :k, 0] + 1j * val[c, :k, 1]) - ov)) <= vtol, f"values of channel {c}"
        assert int(flag[c]) == STATUS[of]


@pytest.mark.parametrize("m,k,C", [(14, 8, 32), (16, 32, 64), (18, 64, 128), (18, 16, 96)])
def test_channels_match_oracle(sf, m, k, C):
    n = 1 << m
    f = exact_fields(n, k)
    P = oracle_params(f)
    plan = _plan(sf, f, C)
    seeds = [workloads.seed_for(6, 100 * m + c) for c in range(C)]
    x, sup, val = workloads.exact_sparse_channels_device(n, k, seeds, "cuda")
    seed, rid = 8642, 5
    outs = sf.sfft_execute_channels(plan, x, seed, rid, f["z_cap"])
    torch.cuda.synchronize()
    _check_channels(sf, P, x, outs, seed, rid, range(C))
    # two calls in a row give the same bits (partial folds and counters are reused)
    outs2 = sf.sfft_execute_channels(plan, x, seed, rid, f["z_cap"])
    torch.cuda.synchronize()
    c1, c2 = outs[2].cpu(), outs2[2].cpu()
    assert torch.equal(c1, c2) and torch.equal(outs[3], outs2[3])
    for c in range(C):
        kk = int(c1[c])
        assert torch.equal(outs[0][c, :kk], outs2[0][c, :kk]) and torch.equal(outs[1][c, :kk], outs2[1][c, :kk])
    plan.close()


def test_channels_equal_their_own_requests(sf):
    """Channel c equals sfft_execute_requests on signal x[:, c] with the shared {seed, id}: the same
    support and flag, values within 1e-5 (the two fold the same products in different orders, each
    within the FP32 tolerance of the oracle)."""
    n, k, C = 1 << 18, 64, 64
    f = exact_fields(n, k)
    plan = _plan(sf, f, C)
    seeds = [workloads.seed_for(6, 900 + c) for c in range(C)]
    x, sup, val = workloads.exact_sparse_channels_device(n, k, seeds, "cuda")
    seed, rid = 77, 3
    outs = sf.sfft_execute_channels(plan, x, seed, rid, f["z_cap"])
    rows = [x[:, c].contiguous() for c in range(C)]
    ref = sf.sfft_execute_requests(plan, rows, [seed] * C, [rid] * C, f["z_cap"])
    torch.cuda.synchronize()
    gi, gv, gc, gf = (t.cpu().numpy() for t in outs)
    ri, rv, rc, rf = (t.cpu().numpy() for t in ref)
    assert np.array_equal(gc, rc) and np.array_equal(gf, rf)
    for c in range(C):
        kk = int(gc[c])
        assert np.array_equal(gi[c, :kk], ri[c, :kk])
        assert np.max(np.abs(gv[c, :kk] - rv[c, :kk]), initial=0.0) <= 1e-5
        assert np.array_equal(gi[c, :kk].view(np.uint32).astype(np.int64), sup[c])
    plan.close()


def test_channels_full_size(sf):
    """The headline transform (n = 2^22, k = 64, alpha0 = 5/8) on 256 interleaved channels (8 GiB):
    every support against the planted one, 16 channels against the oracle."""
    n, k, C = 1 << 22, 64, 256
    f = exact_fields(n, k, alpha0=0.625)
    P = oracle_params(f)
    plan = _plan(sf, f, C)
    seeds = [workloads.seed_for(2, c) for c in range(C)]
    x, sup, val = workloads.exact_sparse_channels_device(n, k, seeds, "cuda")
    seed, rid = 0x5EED2000, 0
    outs = sf.sfft_execute_channels(plan, x, seed, rid, f["z_cap"])
    torch.cuda.synchronize()
    idx = outs[0].cpu().numpy().view(np.uint32)
    cnt = outs[2].cpu().numpy()
    missed = [c for c in range(C) if not np.array_equal(idx[c, :cnt[c]].astype(np.int64), sup[c])]
    assert len(missed) <= 2, missed
    _check_channels(sf, P, x, outs, seed, rid, sorted(set(range(0, C, 16)) | set(missed)))
    plan.close()


def test_channels_argument_checks(sf):
    n, k = 1 << 14, 8
    f = exact_fields(n, k)
    plan = _plan(sf, f, 64)
    x = torch.zeros((n, 48), dtype=torch.complex64, device="cuda")  # not a multiple of 32
    with pytest.raises(sf.SfftError) as ei:
        sf.sfft_execute_channels(plan, x, 1, 0, f["z_cap"])
    assert ei.value.status == sf.SFFT_ERR_INVALID_ARG
    x = torch.zeros((n, 96), dtype=torch.complex64, device="cuda")  # more channels than the plan holds
    with pytest.raises(sf.SfftError):
        sf.sfft_execute_channels(plan, x, 1, 0, f["z_cap"])
    plan.close()
    p64 = _plan(sf, f, 32, precision=sf.SFFT_FP64)
    with pytest.raises(sf.SfftError):
        sf.sfft_execute_channels(p64, torch.zeros((n, 32), dtype=torch.complex64, device="cuda"), 1, 0, f["z_cap"])
    p64.close()
