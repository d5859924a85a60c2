"""Parity at the full sizes of the 24- and 12-aircraft workloads, in the launch
configuration the solver runs them: the rollout over all particles and wind
samples on the GPU, its per-sample costs checked one by one against the FP64
oracle on sampled particles (all samples for the 12-aircraft workload; the
first and the last sample for the 24-aircraft one, whose 64x64x8 field the
oracle generates sample by sample)."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gpu_helpers import compare_sample_costs, cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda()


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_1506_02869_gb300 as pkg
    return pkg


def _run(torch, pkg, p, J, pidx, samples, rng):
    u = S.mild_controls(p, p.L, rng)
    u[: p.L // 4] = S.random_controls(p, p.L // 4, rng)
    soft = p.sep_mode != 0
    sol = pkg.Solver(p)
    cbar, _ = sol.rollout_cost(torch.from_numpy(u).cuda(), J, soft=soft)
    sc = sol.sample_costs(p.L)[samples][:, :, pidx].cpu().numpy().astype(np.float64)
    scs = sol.sample_costs(p.L, soft=True)[samples][:, :, pidx].cpu().numpy().astype(np.float64) \
        if soft else None
    sol.close()
    ref = O.rollout_at_samples(p, u[pidx], J, samples, pidx=pidx, soft=soft, nthreads=8)
    out = {"hard": compare_sample_costs(sc.transpose(2, 0, 1), ref["cost"], ref["margin"], ref["smargin"],
                                        "hard")}
    if soft:
        out["soft"] = compare_sample_costs(scs.transpose(2, 0, 1), ref["cost_soft"], ref["margin"],
                                           ref["smargin"], "soft")
    return out


def test_24_aircraft_workload_full_size(torch, pkg):
    """L 262144, M 64, N 24, H 120, 64x64x8 grid, noise cost, hard and soft."""
    p = S.config3()
    assert (p.L, p.M, p.N, p.H) == (262144, 64, 24, 120)
    rng = np.random.default_rng(70)
    pidx = np.unique(np.r_[rng.choice(p.L, 10, replace=False), [0, p.L - 1]])
    _run(torch, pkg, p, 1, pidx, [0, p.M - 1], rng)


def test_12_aircraft_workload_full_size(torch, pkg):
    """L 16384, M 16, N 12, H 60, softplus separation: every sample."""
    p = S.config4()
    assert (p.L, p.M, p.N, p.H) == (16384, 16, 12, 60)
    rng = np.random.default_rng(71)
    pidx = np.unique(np.r_[rng.choice(p.L, 40, replace=False), [0, p.L - 1]])
    _run(torch, pkg, p, 2, pidx, list(range(p.M)), rng)
