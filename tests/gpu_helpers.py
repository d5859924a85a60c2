"""Shared helpers of the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np
import pytest

import oracle as O

# Tolerances: costs |d| <= 1e-4 max(|c|, 1e-2) (FP32 rollout with compensated
# sums against the FP64 oracle; the floor covers costs near 0); threshold
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
           tuple(p.box_hi), p.dt, p.lam_t, p.beta_xy, p.gam_z, p.wind_sigma,
           getattr(p, "wind_stream", 3))
    if key not in _wind_cache:
        if len(_wind_cache) > 4:
            _wind_cache.clear()
        _wind_cache[key] = O.wind_field(p)
    return _wind_cache[key]


def _dump(what, **arrays):
    """Keep the arrays of a failing comparison for offline analysis, in the
    directory that TMA_TEST_DUMP_DIR names (nothing when it is unset)."""
    import os
    import re
    d = os.environ.get("TMA_TEST_DUMP_DIR", "")
    if d and os.path.isdir(d):
        np.savez(os.path.join(d, "fail_" + re.sub(r"[^A-Za-z0-9_=.-]+", "_", what) + ".npz"),
                 **arrays)


def compare_costs(got, ref, margin, smargin, what, max_excluded=0.02, max_particles=0.10):
    """got/ref [N][Ls]; returns (max rel err, n compared, n excluded).

    (l, i) is set aside when a decision of aircraft i is within TAU of its
    threshold; particle l is set aside whole when a decision that changes the
    set of flying aircraft is (it can change every other aircraft's cost)."""
    struct = smargin < TAU
    keep = (margin >= TAU) & ~struct[None, :]
    n_struct = int(struct.sum())
    n_self = int(((margin < TAU) & ~struct[None, :]).sum())
    ok_budget = n_struct <= max(1, max_particles * struct.size) and \
        n_self <= max(2, max_excluded * keep.size)
    if not ok_budget:
        _dump(what, got=got, ref=ref, margin=margin, smargin=smargin)
    assert ok_budget, f"{what}: {n_struct} particles, {n_self} aircraft near a threshold"
    g, r = got[keep], ref[keep]
    inf_g, inf_r = ~np.isfinite(g), ~np.isfinite(r)
    bad = np.nonzero(inf_g != inf_r)[0]
    if bad.size:
        _dump(what, got=got, ref=ref, margin=margin, smargin=smargin)
    assert bad.size == 0, f"{what}: feasibility differs at {bad[:10]} (got {g[bad[:5]]}, ref {r[bad[:5]]})"
    fin = ~inf_r
    err = np.abs(g[fin] - r[fin]) / np.maximum(np.abs(r[fin]), COST_FLOOR)
    emax = float(err.max()) if err.size else 0.0
    if emax > COST_TOL:
        _dump(what, got=got, ref=ref, margin=margin, smargin=smargin)
        w = int(np.argmax(err))
        what += f" worst got={g[fin][w]!r} ref={r[fin][w]!r}"
    assert emax <= COST_TOL, f"{what}: max rel err {emax:.3e} (n={fin.sum()})"
    return emax, int(fin.sum()), int((~keep).sum())


def compare_sample_costs(got, ref, margin, smargin, what, max_aside=0.1, min_compared=100):
    """got/ref [Ls][ns][N] per-sample costs; (l, m, i) is set aside when
    aircraft i of particle l has a decision within TAU of its threshold in
    sample m, or a decision that changes the set of flying aircraft does (at
    most max_aside of them); returns (max rel err, n compared)."""
    keep = (margin >= TAU) & (smargin[:, :, None] >= TAU)
    assert keep.mean() >= 1 - max_aside, (what, keep.mean())
    g, r = got[keep], ref[keep]
    assert (np.isfinite(g) == np.isfinite(r)).all(), what + ": feasibility differs"
    fin = np.isfinite(r)
    err = np.abs(g[fin] - r[fin]) / np.maximum(np.abs(r[fin]), COST_FLOOR)
    assert err.size >= min_compared and err.max() <= COST_TOL, \
        (what, err.max() if err.size else None, err.size)
    return float(err.max()), int(err.size)
