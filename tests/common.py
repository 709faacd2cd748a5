"""Parameter sets shared by the tests: both the oracle and the GPU library receive these same values."""
from __future__ import annotations

FIELDS_DEFAULT = dict(
    delta=1e-6,
    alpha0=0.5,
    bins_per_k=4.0,
    B_min=16,
    extra_rounds=0,
    thr=0.5,
    tau_dec=1e-4,
    iso_tol=1e-3,
    gmin=0.1,
    prune=0.5,
    ref_lo=1e-5,
    ref_hi=2e-2,
    ref_tol=0.1,
    eps=1.0,
    t_regions=0,
    R_loc=5,
    R_est=5,
    s=0.25,
    est_gmin=0.25,
)


def exact_fields(n, k, **over):
    f = dict(FIELDS_DEFAULT)
    f.update(n=n, k=k, mode=0, z_cap=max(4 * k, 64))
    f.update(over)
    return f


def general_fields(n, k, **over):
    f = dict(FIELDS_DEFAULT)
    f.update(n=n, k=k, mode=1, z_cap=max(8 * k, 64), bins_per_k=8.0, R_loc=7)
    f.update(over)
    return f


def oracle_params(fields):
    import oracle

    return oracle.make_params(**fields)
