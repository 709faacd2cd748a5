"""Whole transforms captured as CUDA graphs (sfft_graph_*): replays give bit for bit the results of
the direct calls, for a batch of rows and for the plan's request table refilled between replays, in
exact and general mode."""
import numpy as np
import pytest

from paper_1201_2501_gb300 import workloads
from tests.common import exact_fields, general_fields

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


def gpu_params(sf, fields):
    p = sf.sfft_params_default(fields["n"], fields["k"], fields["mode"])
    for name, _ in sf.SfftParams._fields_:
        if name in fields:
            setattr(p, name, fields[name])
    return p


def _np(outs):
    return [t.cpu().numpy().copy() for t in outs]


def _same(a, b):
    """Same counts and flags, and the same entries up to each request's count (the rest is unwritten)."""
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    for r, c in enumerate(a[2]):
        assert np.array_equal(a[0][r, :c], b[0][r, :c])
        assert np.array_equal(a[1][r, :c], b[1][r, :c])


@pytest.mark.parametrize("mode", ["exact", "general"])
def test_graph_of_rows_equals_direct(sf, mode):
    n, k, batch = (1 << 18, 32, 8) if mode == "exact" else (1 << 16, 16, 4)
    f = exact_fields(n, k) if mode == "exact" else general_fields(n, k)
    p = gpu_params(sf, f)
    plan = sf.Plan(p, batch)
    gen = workloads.exact_sparse if mode == "exact" else workloads.general_noisy
    x = torch.as_tensor(np.stack([gen(n, k, workloads.seed_for(10, i)).x for i in range(batch)])).cuda()
    want = _np(sf.sfft_execute(plan, x, 31, p.z_cap))
    outs = (torch.zeros((batch, p.z_cap), dtype=torch.int32, device="cuda"),
            torch.zeros((batch, p.z_cap, 2), dtype=torch.float64, device="cuda"),
            torch.zeros((batch,), dtype=torch.int32, device="cuda"), torch.zeros((batch,), dtype=torch.int32, device="cuda"))
    g = sf.Graph(plan, x, batch, 31, p.z_cap, outs)
    for _ in range(3):
        g.launch()
        torch.cuda.synchronize()
        _same(_np(outs), want)
    g.close()
    plan.close()


def test_graph_of_the_request_table_follows_refills(sf):
    n, k, batch = 1 << 18, 32, 4
    f = exact_fields(n, k)
    p = gpu_params(sf, f)
    plan = sf.Plan(p, batch)
    sigs = [workloads.exact_sparse(n, k, workloads.seed_for(10, 50 + i)) for i in range(2 * batch)]
    xs = [torch.as_tensor(s.x).cuda() for s in sigs]
    outs = (torch.zeros((batch, p.z_cap), dtype=torch.int32, device="cuda"),
            torch.zeros((batch, p.z_cap, 2), dtype=torch.float64, device="cuda"),
            torch.zeros((batch,), dtype=torch.int32, device="cuda"), torch.zeros((batch,), dtype=torch.int32, device="cuda"))
    g = sf.Graph(plan, None, batch, 0, p.z_cap, outs)
    for half in (0, 1, 0):
        sel = list(range(half * batch, (half + 1) * batch))
        g.set_requests([xs[i] for i in sel], [7] * batch, sel)
        g.launch()
        torch.cuda.synchronize()
        got = _np(outs)
        want = _np(sf.sfft_execute_requests(plan, [xs[i] for i in sel], [7] * batch, sel, p.z_cap))
        _same(got, want)
        for r, i in enumerate(sel):
            assert np.array_equal(got[0][r, :got[2][r]].astype(np.int64), sigs[i].support)
    g.close()
    plan.close()
