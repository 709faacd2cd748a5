"""The autotuner (sfft_autotune): it reports every candidate with base's settings first, picks one at
least as fast as base's and at least as accurate on the planted spectra, and the chosen settings
recover fresh signals as the oracle does."""
import numpy as np
import pytest

import oracle
from paper_1201_2501_gb300 import workloads
from tests.common import oracle_params

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


@pytest.mark.parametrize("mode", [0, 1])
def test_autotune_picks_a_fast_accurate_setting(sf, mode):
    n, k = (1 << 18, 32) if mode == 0 else (1 << 16, 16)
    base = sf.sfft_params_default(n, k, mode)
    best, rep = sf.sfft_autotune(base, batch=8, reps=2)
    # the 3 x 3 x 4 (x 2 taps per CTA in exact mode) grid, which contains the base settings (listed first)
    assert len(rep) == (72 if mode == 0 else 36)
    r0 = rep[0]
    assert (r0["bins_per_k"], r0["alpha0"], r0["streams"], r0["chunk_taps"]) == \
        (base.bins_per_k, base.alpha0, base.streams, base.chunk_taps)
    chosen = [r for r in rep if r["chosen"]]
    assert len(chosen) == 1
    c = chosen[0]
    assert (best.bins_per_k, best.alpha0, best.streams, best.chunk_taps) == \
        (c["bins_per_k"], c["alpha0"], c["streams"], c["chunk_taps"])
    assert c["status"] == 0 and c["us_per_transform"] <= r0["us_per_transform"]
    if mode == 0:
        assert c["exact"] >= r0["exact"] and r0["exact"] == 8
    else:
        assert c["rel_err"] <= 1.05 * r0["rel_err"] + 1e-12
    # the chosen settings on fresh signals: exact mode against the oracle with the same settings
    if mode == 0:
        plan = sf.Plan(best, 4)
        sigs = [workloads.exact_sparse(n, k, workloads.seed_for(11, i)) for i in range(4)]
        x = torch.as_tensor(np.stack([s.x for s in sigs])).cuda()
        idx, val, cnt, flag = (t.cpu().numpy() for t in sf.sfft_execute(plan, x, 3, best.z_cap))
        fields = {f: getattr(best, f) for f, _ in sf.SfftParams._fields_
                  if f not in ("precision", "streams", "gain", "chunk_taps", "permuted_copy")}
        P = oracle_params(fields)
        for r, s in enumerate(sigs):
            gi = idx[r, :cnt[r]].view(np.uint32).astype(np.int64)
            oi, ov, of = oracle.sfft_exact(P, s.x.astype(np.complex128), 3, r)
            assert np.array_equal(gi, oi.astype(np.int64))
            assert np.array_equal(gi, s.support)
        plan.close()
