"""Requests with their own signals and draws, and the continuous-batching server, through the C ABI.

* sfft_execute_requests: request {row r, seed, id r} in any slot of any batch gives bit for bit the
  result of row r of sfft_execute with that seed;
* the server: jobs of several parameter sets (exact FP32 and FP64, general; host and device signals),
  submitted from two threads while earlier batches run, each give bit for bit the result of the same
  request run alone, and the exact ones recover the planted spectrum as the oracle does;
* admission by device memory: with a budget that holds only a few staged signals, every job still
  completes, correctly, and the peak of held memory stays within the budget.
"""
import random
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, general_fields, oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 0x5EED7000


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


def _rows(outputs, batch):
    idx, val, cnt, flag = (t.cpu().numpy() for t in outputs)
    res = []
    for r in range(batch):
        c = int(cnt[r])
        res.append((idx[r, :c].astype(np.int64), val[r, :c].copy(), int(flag[r])))
    return res


def test_execute_requests_equals_execute(sf):
    n, k, batch = 1 << 18, 32, 12
    p = gpu_params(sf, exact_fields(n, k))
    sigs = [workloads.exact_sparse(n, k, workloads.seed_for(7, i), dtype=np.complex64) for i in range(batch)]
    x = torch.as_tensor(np.stack([s.x for s in sigs])).cuda()
    plan = sf.Plan(p, batch)
    want = _rows(sf.sfft_execute(plan, x, SEED, p.z_cap), batch)
    perm = list(range(batch))
    random.Random(3).shuffle(perm)
    # the same requests in a shuffled order, reading the rows in place
    got = _rows(sf.sfft_execute_requests(plan, [x[r] for r in perm], [SEED] * batch, perm, p.z_cap), batch)
    torch.cuda.synchronize()
    for slot, r in enumerate(perm):
        assert np.array_equal(got[slot][0], want[r][0])
        assert np.array_equal(got[slot][1], want[r][1])
        assert got[slot][2] == want[r][2]
        assert np.array_equal(want[r][0], sigs[r].support)
    plan.close()


def _alone(sf, p, x_dev, seed, rid):
    plan = sf.Plan(p, 1)
    out = _rows(sf.sfft_execute_requests(plan, [x_dev], [seed], [rid], p.z_cap), 1)[0]
    torch.cuda.synchronize()
    plan.close()
    return out


def _job_mix():
    """(fields, precision, signal, is_exact, on_device) for a mix of parameter sets."""
    jobs = []
    for i in range(10):
        s = workloads.exact_sparse(1 << 16, 8, workloads.seed_for(7, 100 + i), dtype=np.complex64)
        jobs.append((exact_fields(1 << 16, 8), 0, s, True, i % 2 == 0))
    for i in range(8):
        s = workloads.exact_sparse(1 << 18, 32, workloads.seed_for(7, 200 + i), dtype=np.complex64)
        jobs.append((exact_fields(1 << 18, 32), 0, s, True, i % 2 == 1))
    for i in range(4):
        s = workloads.exact_sparse(1 << 14, 8, workloads.seed_for(7, 300 + i), dtype=np.complex128)
        jobs.append((exact_fields(1 << 14, 8, delta=1e-8), 1, s, True, False))
    for i in range(6):
        s = workloads.general_noisy(1 << 16, 16, workloads.seed_for(7, 400 + i))
        jobs.append((general_fields(1 << 16, 16), 0, s, False, i % 3 == 0))
    return jobs


def test_server_results_equal_alone_and_in_the_mix(sf):
    jobs = _job_mix()
    order = list(range(len(jobs)))
    random.Random(11).shuffle(order)
    srv = sf.Server(max_batch=8, instances=2)
    tickets = {}
    lock = threading.Lock()

    def submitter(part):
        rng = random.Random(part)
        for j in order[part::2]:
            fields, prec, s, _, on_dev = jobs[j]
            p = gpu_params(sf, fields, prec)
            x = torch.as_tensor(s.x)
            if on_dev:
                x = x.cuda()
            t = srv.submit(p, x, SEED + j, id=j)
            with lock:
                tickets[j] = t
            time.sleep(rng.random() * 2e-3)  # arrivals spread while earlier batches run

    th = [threading.Thread(target=submitter, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = {j: srv.wait(tickets[j], timeout_s=120) for j in range(len(jobs))}
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"]
    assert st["launches"] < len(jobs)  # some jobs shared a launch
    for j, (fields, prec, s, exact, _) in enumerate(jobs):
        idx, val, info = results[j]
        p = gpu_params(sf, fields, prec)
        a_idx, a_val, a_flag = _alone(sf, p, torch.as_tensor(s.x).cuda(), SEED + j, j)
        assert np.array_equal(idx, a_idx), j
        assert np.array_equal(val, a_val[:, 0] + 1j * a_val[:, 1]), j
        assert info["flag"] == a_flag
        if exact:
            # the oracle, with the same seed and request index, recovers the same spectrum
            P = oracle_params(fields)
            oi, ov, of = oracle.sfft_exact(P, s.x.astype(np.complex128), SEED + j, j)
            assert np.array_equal(idx, oi.astype(np.int64)), j
            assert np.max(np.abs(val - ov)) < 1e-5, j
            assert np.array_equal(idx, s.support)
        else:
            # general jobs (served as CUDA-graph batches): the oracle's support, values within 1e-5
            P = oracle_params(fields)
            oi, ov, of = oracle.sfft_general(P, s.x.astype(np.complex128), SEED + j, j)
            assert np.array_equal(idx, oi.astype(np.int64)), j
            scale = max(1.0, float(np.max(np.abs(ov), initial=0.0)))
            assert np.max(np.abs(val - ov), initial=0.0) <= 1e-5 * scale, j


def test_server_admits_by_device_memory(sf):
    n, k, njobs = 1 << 20, 16, 16
    xbytes = n * 8
    budget = 64 << 20  # the plans plus a handful of staged 8 MiB signals
    srv = sf.Server(mem_budget=budget, max_batch=4, instances=2)
    p = gpu_params(sf, exact_fields(n, k))
    sigs = [workloads.exact_sparse(n, k, workloads.seed_for(7, 500 + i), dtype=np.complex64) for i in range(njobs)]
    tick = [srv.submit(p, torch.as_tensor(s.x), SEED, id=i) for i, s in enumerate(sigs)]
    res = [srv.wait(t, timeout_s=120) for t in tick]
    st = srv.stats()
    with pytest.raises(sf.SfftError) as e:  # a signal that can never fit
        srv.submit(gpu_params(sf, exact_fields(1 << 24, 8)), torch.zeros(1 << 24, dtype=torch.complex64), SEED)
    assert e.value.status == sf.SFFT_ERR_OOM
    srv.close()
    assert st["completed"] == njobs and st["failed"] == 0
    assert st["bytes_peak"] <= budget
    assert st["bytes_peak"] >= xbytes
    for (idx, val, info), s in zip(res, sigs):
        assert np.array_equal(idx, s.support)
        assert np.max(np.abs(val - s.values)) < 1e-5
        assert info["flag"] == 0


def test_submit_many_equals_submit(sf):
    """sfft_submit_many / sfft_wait_many: a whole array of jobs queued in one call gives, job by job,
    bit for bit the results of the same jobs submitted and waited for one at a time, in ticket order;
    the planted supports are recovered; an unknown ticket and an empty array are argument errors."""
    n, k, m = 1 << 16, 16, 40
    p = gpu_params(sf, exact_fields(n, k))
    seeds = [workloads.seed_for(7, i) for i in range(m)]
    x, sup, _ = workloads.exact_sparse_batch_device(n, k, seeds, "cuda")
    xs = [x[i] for i in range(m)]
    srv = sf.Server(max_batch=16, instances=2)
    try:
        one = [srv.wait(srv.submit(p, xs[i], SEED, id=i), timeout_s=120) for i in range(m)]
        tickets = srv.submit_many(p, xs, SEED, list(range(m)))
        assert len(tickets) == m and len(set(tickets)) == m
        many = srv.wait_many(tickets, timeout_s=120)
        assert len(many) == m
        for i in range(m):
            assert np.array_equal(many[i][0], one[i][0]) and np.array_equal(many[i][1], one[i][1])
            assert many[i][2]["flag"] == one[i][2]["flag"] == 0
            assert np.array_equal(np.sort(many[i][0]), sup[i])
        # a ticket already released, and an empty array, are rejected
        with pytest.raises(sf.SfftError):
            srv.wait_many([tickets[0]], timeout_s=1)
        with pytest.raises(sf.SfftError):
            srv.submit_many(p, [], SEED, [])
    finally:
        srv.close()
