"""Mixed exact-mode batches in one persistent launch (sfft_batch_*): requests of several plans
(different n and k, one with its end-of-round arrays in device memory) in a shuffled order give bit
for bit the results of each request's own plan run through sfft_execute, and the oracle's."""
import random

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


def _rows(outs, nreq):
    idx, val, cnt, flag = (t.cpu().numpy() for t in outs)
    return [(idx[r, :cnt[r]].view(np.uint32).astype(np.int64), val[r, :cnt[r]].copy(), int(flag[r]))
            for r in range(nreq)]


@pytest.mark.parametrize("prec", [0, 1])
def test_mixed_batch_equals_each_plans_own_execution(sf, prec):
    sizes = [(14, 8), (16, 16), (18, 64), (16, 512)] if prec == 0 else [(12, 4), (14, 8), (14, 32)]
    fields = [exact_fields(1 << m, k) for m, k in sizes]
    plans = [sf.Plan(gpu_params(sf, f, prec), 16) for f in fields]
    dt = np.complex128 if prec else np.complex64
    reqs = []
    for pi, (m, k) in enumerate(sizes):
        for i in range(4 if k < 512 else 2):
            reqs.append((pi, workloads.exact_sparse(1 << m, k, workloads.seed_for(8, 100 * pi + i), dtype=dt)))
    random.Random(5).shuffle(reqs)
    xs = [torch.as_tensor(s.x).cuda() for _, s in reqs]
    plan_of = [pi for pi, _ in reqs]
    seeds = [0x5EED8000 + r for r in range(len(reqs))]
    ids = list(range(len(reqs)))
    cap = max(f["z_cap"] for f in fields)
    bp = sf.BatchPlan(plans, 64)
    got = _rows(bp.execute(plan_of, xs, seeds, ids, cap), len(reqs))
    again = _rows(bp.execute(plan_of, xs, seeds, ids, cap), len(reqs))  # the workspace is reusable
    torch.cuda.synchronize()
    for r, (pi, s) in enumerate(reqs):
        one = _rows(sf.sfft_execute_requests(plans[pi], [xs[r]], [seeds[r]], [ids[r]], cap), 1)[0]
        for res in (got[r], again[r]):
            assert np.array_equal(res[0], one[0]), r
            assert np.array_equal(res[1], one[1]), r
            assert res[2] == one[2]
        assert np.array_equal(got[r][0], s.support)
        if r < 6:
            P = oracle_params(fields[pi])
            oi, ov, of = oracle.sfft_exact(P, s.x.astype(np.complex128), seeds[r], ids[r])
            assert np.array_equal(got[r][0], oi.astype(np.int64))
            v = got[r][1][:, 0] + 1j * got[r][1][:, 1]
            assert np.max(np.abs(v - ov)) < (1e-9 if prec else 1e-5)
    bp.close()
    for p in plans:
        p.close()


def test_persistent_headline_shape(sf):
    """The benchmark's workload shape (n = 2^22, k = 64) through one persistent launch of 32 requests,
    against sfft_execute of the same plan."""
    n, k, nreq = 1 << 22, 64, 32
    f = exact_fields(n, k)
    p = gpu_params(sf, f)
    plan = sf.Plan(p, nreq)
    x, sup, val = workloads.exact_sparse_batch_device(n, k, [workloads.seed_for(8, 500 + i) for i in range(nreq)],
                                                       "cuda")
    want = _rows(sf.sfft_execute(plan, x, 77, p.z_cap), nreq)
    bp = sf.BatchPlan([plan], nreq)
    got = _rows(bp.execute([0] * nreq, [x[r] for r in range(nreq)], [77] * nreq, list(range(nreq)), p.z_cap), nreq)
    torch.cuda.synchronize()
    for r in range(nreq):
        assert np.array_equal(got[r][0], want[r][0]) and np.array_equal(got[r][1], want[r][1])
        assert got[r][2] == want[r][2]
        assert np.array_equal(got[r][0], sup[r])
    bp.close()
    plan.close()


def test_a_wait_that_nothing_ends_gives_up_with_a_status(sf):
    """The persistent kernel's bounded wait: a CTA waiting for a queue item that is never published
    gives up after about a second, flags the launch and returns; the host reads SFFT_ERR_TIMEOUT and the
    device keeps working (a transform afterwards matches the oracle)."""
    import time

    t0 = time.perf_counter()
    assert sf.lib().sfft_persistent_wait_check(None) == sf.SFFT_ERR_TIMEOUT
    assert 0.2 < time.perf_counter() - t0 < 30.0
    n, k = 1 << 14, 8
    f = exact_fields(n, k)
    plan = sf.Plan(gpu_params(sf, f, 0), 1)
    s = workloads.exact_sparse(n, k, workloads.seed_for(2, 900), dtype=np.complex64)
    got = _rows(sf.sfft_execute(plan, torch.as_tensor(s.x[None]).cuda(), 5, f["z_cap"]), 1)[0]
    assert np.array_equal(got[0], s.support)
    plan.close()
