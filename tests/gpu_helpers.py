"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np
import pytest

import oracle as O

# Tolerances: costs |d| <= 1e-4 max(|c|, 1e-2); threshold
# decisions closer than TAU (relative) to their threshold are set aside.
COST_TOL = 1e-4
COST_FLOOR = 1e-2
TAU = 1e-5


def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    import paper_1506_02869_gb300 as pkg
    pkg.build()
    pkg.lib()
    return torch


_wind_cache = {}


def oracle_wind(p):
    key = (p.seed, p.scenario_id, p.mpc_step, p.M, p.H, tuple(p.grid), tuple(p.box_lo),
           tuple(p.box_hi), p.dt, p.lam_t, p.beta_xy, p.gam_z, p.wind_sigma)
    if key not in _wind_cache:
        if len(_wind_cache) > 4:
            _wind_cache.clear()
        _wind_cache[key] = O.wind_field(p)
    return _wind_cache[key]


def compare_costs(got, ref, margin, smargin, what, max_excluded=0.02):
    """got/ref [N][Ls]; returns (max rel err, n compared, n excluded)."""
    keep = (margin >= TAU) & (smargin[None, :] >= TAU)
    excluded = int((~keep).sum())
    assert excluded <= max(2, max_excluded * keep.size), f"{what}: {excluded} near-threshold cases"
    g, r = got[keep], ref[keep]
    inf_g, inf_r = ~np.isfinite(g), ~np.isfinite(r)
    bad = np.nonzero(inf_g != inf_r)[0]
    assert bad.size == 0, f"{what}: feasibility differs at {bad[:10]} (got {g[bad[:5]]}, ref {r[bad[:5]]})"
    fin = ~inf_r
    err = np.abs(g[fin] - r[fin]) / np.maximum(np.abs(r[fin]), COST_FLOOR)
    emax = float(err.max()) if err.size else 0.0
    assert emax <= COST_TOL, f"{what}: max rel err {emax:.3e} (n={fin.sum()})"
    return emax, int(fin.sum()), excluded
