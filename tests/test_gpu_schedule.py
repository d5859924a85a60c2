"""Sample mode 1 on the GPU (the inner loop of Algorithm 1: iteration J rolls
out the first M_J = min(SampleSchedule(J), M) wind samples and weights by the
product of J_T over them), against the FP64 oracle's schedule, whose weights
are pinned to the product of the per-draw objectives on the CPU."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gpu_helpers import COST_FLOOR, COST_TOL, compare_costs, cuda, oracle_wind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda()


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_1506_02869_gb300 as pkg
    return pkg


def scheduled(p, M=12):
    return p.copy(sample_mode=1, M=M)


@pytest.mark.parametrize("J", [0, 4, 9])
def test_rollout_uses_the_first_samples(torch, pkg, J):
    p = scheduled(S.config1().copy(L=500))
    Mj = O.samples(p, J)
    assert Mj < p.M
    rng = np.random.default_rng(50 + J)
    u = S.mild_controls(p, p.L, rng)
    sol = pkg.Solver(p)
    cbar, _ = sol.rollout_cost(torch.from_numpy(u).cuda(), J)
    got = cbar.cpu().numpy().astype(np.float64)
    samp = sol.sample_costs(p.L).cpu().numpy()
    sol.close()
    assert np.isnan(samp[Mj:]).all() and not np.isnan(samp[:Mj]).any()
    W = oracle_wind(p)
    ref = O.rollout(p.copy(M=Mj), u, J, W=W[:Mj])
    emax, n, _ = compare_costs(got, ref["cbar"], ref["margin"], ref["smargin"], f"schedule J={J}")
    assert n > 100
    keep = (ref["smargin"] >= 1e-5) & (ref["margin"].min(0) >= 1e-5)
    g = samp[:Mj].transpose(2, 0, 1).astype(np.float64)[keep]
    r = ref["cost"][keep]
    fin = np.isfinite(r)
    assert (np.isfinite(g) == fin).all()
    err = np.abs(g[fin] - r[fin]) / np.maximum(np.abs(r[fin]), COST_FLOOR)
    assert err.max() <= COST_TOL


def test_solve_best_cost_reproduced_by_oracle(torch, pkg):
    p = scheduled(S.config1())
    sol = pkg.Solver(p)
    b, c, _ = sol.solve()
    b2, c2, _ = sol.solve()
    best = sol.best_index()
    sol.close()
    assert np.isfinite(c) and c == c2 and torch.equal(b, b2)
    J = p.J_max - 1
    Mj = O.samples(p, J)
    r = O.rollout(p.copy(M=Mj), b.cpu().numpy().astype(np.float64)[None], J, pidx=[best],
                  W=oracle_wind(p)[:Mj])
    if (r["margin"] >= 1e-5).all() and (r["smargin"] >= 1e-5).all():
        assert r["cbar"][:, 0].sum() == pytest.approx(c, rel=1e-4)


def test_solve_differs_from_the_fixed_sample_solve(torch, pkg):
    """The schedule changes what is computed (fewer samples, another
    exponent), so the two modes choose different controls."""
    p = scheduled(S.config1())
    out = []
    for q in (p, p.copy(sample_mode=0)):
        sol = pkg.Solver(q)
        b, c, _ = sol.solve()
        sol.close()
        out.append((b.cpu().numpy(), c))
    assert not np.array_equal(out[0][0], out[1][0])


def test_solve_quality_matches_oracle_statistically(torch, pkg):
    gpu, orc = [], []
    for step in range(3):
        p = scheduled(S.config1().copy(mpc_step=step))
        sol = pkg.Solver(p)
        sol.set_state(mpc_step=step)
        _, c, _ = sol.solve()
        sol.close()
        gpu.append(c)
        orc.append(O.smc_solve(p, nthreads=8)["best_sum"])
    gpu, orc = np.array(gpu), np.array(orc)
    assert np.isfinite(gpu).all() and np.isfinite(orc).all()
    assert abs(np.median(gpu) - np.median(orc)) <= 0.1 * np.median(orc), (gpu, orc)


def test_gradient_uses_the_iteration_samples(torch, pkg):
    p = scheduled(S.shrink(S.config4(), M=12, H=30, L=64))
    J = 6
    Mj = O.samples(p, J)
    rng = np.random.default_rng(52)
    u = S.mild_controls(p, p.L, rng)
    sol = pkg.Solver(p)
    sol.wind_field()
    cost, grad, _ = sol.rollout_grad(torch.from_numpy(u).cuda(), J, cbar=True)
    _, cs = sol.rollout_cost(torch.from_numpy(u).cuda(), J, soft=True)
    sol.close()
    cost, cs = cost.cpu().numpy(), cs.cpu().numpy().astype(np.float64)
    tot = np.where(np.isfinite(cs).all(axis=0), cs.sum(axis=0), np.inf)
    assert np.array_equal(np.isfinite(cost), np.isfinite(tot))
    fin = np.isfinite(tot)
    assert fin.sum() > 10 and np.allclose(cost[fin], tot[fin], rtol=1e-6)
    W = oracle_wind(p)[:Mj]
    l = int(np.nonzero(fin)[0][0])
    c_ref, g_ref = O.rollout_grad(p.copy(M=Mj), u[l].astype(np.float64), W, l=l, J=J)
    assert abs(cost[l] - c_ref) <= 1e-4 * max(abs(c_ref), 1e-2)
    g = grad.cpu().numpy()[l]
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)


def test_batch_equals_single_solves(torch, pkg):
    ps = S.config5(n_scen=24)
    order = sorted(range(len(ps)), key=lambda s: ps[s].N)
    pick = [order[0], order[len(order) // 2], order[-1]]
    ps = [scheduled(S.shrink(ps[k], L=512, H=24, J_max=8), M=10) for k in pick]
    Ns = [p.N for p in ps]
    b = pkg.tma_batch_create(ps)
    pkg.tma_batch_solve(b)
    res = pkg.tma_batch_results(b, Ns, ps[0].S)
    pkg.tma_batch_destroy(b)
    for k, p in enumerate(ps):
        sol = pkg.Solver(p)
        bu, c, _ = sol.solve()
        sol.close()
        assert np.array_equal(res["best_u"][k], bu.cpu().numpy()), k
        assert res["best_cost"][k] == c or (np.isinf(c) and np.isinf(res["best_cost"][k]))
