"""Varying particle count on the GPU (the speed-up the paper proposes): the
resampling of L_out ancestors from L_in weighted particles (bit-exact against
the oracle, whose ancestors are pinned by exact rational arithmetic), the
perturbation with another number of parents, and the solve with a particle
schedule."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gpu_helpers import compare_costs, cuda, oracle_wind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda()


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_1506_02869_gb300 as pkg
    return pkg


@pytest.mark.parametrize("nseg,Lin,Lout", [(8, 65536, 40000), (3, 5000, 12289), (2, 2049, 1),
                                           (1, 1, 7), (4, 6144, 6143), (24, 262144, 131072),
                                           (1, 1 << 22, 4096)])
def test_resample_to_bit_exact(torch, pkg, nseg, Lin, Lout):
    rng = np.random.default_rng(nseg + Lin + Lout)
    w = S.random_wtilde(nseg, Lin, rng)
    seed, sid, J, mpc = 777 + Lin, nseg % 3, Lout % 50, 3
    anc = torch.empty((nseg, Lout), dtype=torch.int32, device="cuda")
    st = pkg.tma_resample_to(torch.from_numpy(w).cuda(), seed, sid, J, mpc, anc)
    p = S.config1().copy(seed=seed, scenario_id=sid, mpc_step=mpc)
    ref, nd = O.resample(w, [O.resample_uniform(p, s, J) for s in range(nseg)], Lout)
    assert np.array_equal(anc.cpu().numpy(), ref)
    assert (st == pkg.TMA_WARN_DEGENERATE) == (nd > 0)


def test_resample_to_degenerate_and_concentrated(torch, pkg):
    Lin, Lout = 10000, 3001
    w = np.zeros((3, Lin))
    w[0, 4321] = 1.0
    w[1, ::9] = 0.5
    anc = torch.empty((3, Lout), dtype=torch.int32, device="cuda")
    st = pkg.tma_resample_to(torch.from_numpy(w).cuda(), 5, 0, 1, 0, anc)
    a = anc.cpu().numpy()
    assert st == pkg.TMA_WARN_DEGENERATE
    assert (a[0] == 4321).all() and (a[1] % 9 == 0).all()
    assert np.array_equal(a[2], np.arange(Lout) * Lin // Lout)
    p = S.config1().copy(seed=5)
    ref, _ = O.resample(w, [O.resample_uniform(p, s, 1) for s in range(3)], Lout)
    assert np.array_equal(a, ref)


@pytest.mark.parametrize("Lin,Lout", [(1024, 333), (300, 1024)])
def test_move_to_matches_oracle(torch, pkg, Lin, Lout):
    p = S.shrink(S.config1(), L=1024).copy(mpc_step=1)
    rng = np.random.default_rng(Lin)
    u = S.random_controls(p, Lin, rng)
    anc = rng.integers(0, Lin, (p.N, Lout)).astype(np.int32)
    sol = pkg.Solver(p)
    sol.set_state(mpc_step=1)
    out = torch.empty((Lout, p.N, p.S, 3), dtype=torch.float32, device="cuda")
    pkg.tma_move_to(sol.h, torch.from_numpy(u).cuda(), torch.from_numpy(anc).cuda(), 4, out)
    sol.close()
    out = out.cpu().numpy()
    ref = O.move(p, u.astype(np.float64), anc, 4)
    sig = np.array(p.move_sigma)
    lo, hi = np.array(p.ctrl_lo), np.array(p.ctrl_hi)
    near = (np.abs(ref - lo) < 1e-5 * sig) | (np.abs(ref - hi) < 1e-5 * sig)
    d = np.abs(out - ref)
    tol = np.broadcast_to(2e-6 * sig + 2.5e-7 * np.abs(ref), d.shape)
    assert (d[~near] <= tol[~near]).all(), d.max()


def _scheduled(L=2048, J_max=8, frac=0.25):
    p = S.shrink(S.config1(), L=L, J_max=J_max)
    return p.copy(L_sched=S.particle_schedule(L, J_max, frac))


def test_first_iterations_agree_with_the_oracle_chain(torch, pkg):
    """Iteration 0 with L_0 particles, resampled to L_1 and moved, on both sides
    from each side's own initialisation."""
    p = _scheduled()
    L0, L1 = p.L_sched[0], p.L_sched[1]
    assert L1 < L0
    sol = pkg.Solver(p)
    u0 = sol.init_controls(L0)
    cbar, _ = sol.rollout_cost(u0, 0)
    wt, _, _ = pkg.lse(cbar, O.kappa(0))
    anc = torch.empty((p.N, L1), dtype=torch.int32, device="cuda")
    pkg.tma_resample_to(wt, p.seed, p.scenario_id, 0, p.mpc_step, anc)
    u1 = torch.empty((L1, p.N, p.S, 3), dtype=torch.float32, device="cuda")
    pkg.tma_move_to(sol.h, u0, anc, 0, u1)
    sol.close()
    ru0 = O.init_controls(p, L0)
    rr = O.rollout(p, ru0, 0, W=oracle_wind(p))
    compare_costs(cbar.cpu().numpy().astype(np.float64), rr["cbar"], rr["margin"], rr["smargin"], "J0")
    # the resampling of the GPU's own weights is exact
    ref_anc, _ = O.resample(wt.cpu().numpy(), [O.resample_uniform(p, s, 0) for s in range(p.N)], L1)
    assert np.array_equal(anc.cpu().numpy(), ref_anc)
    rwt, _, _ = O.lse(rr["cbar"], O.kappa(0))
    ranc, _ = O.resample(rwt, [O.resample_uniform(p, s, 0) for s in range(p.N)], L1)
    same = anc.cpu().numpy() == ranc
    assert same.mean() > 0.97, same.mean()
    ru1 = O.move(p, ru0, ranc, 0)
    g1 = u1.cpu().numpy()
    for i in range(p.N):
        ok = same[i]
        assert np.allclose(g1[ok, i], ru1[ok, i], rtol=1e-5, atol=1e-5 * np.array(p.move_sigma).max())


def test_solve_with_schedule_is_deterministic_and_reproduced(torch, pkg):
    p = _scheduled()
    sol = pkg.Solver(p)
    b, c, _ = sol.solve()
    b2, c2, _ = sol.solve()
    best = sol.best_index()
    parts = sol.particles()
    sol.close()
    Lf = p.L_sched[-1]
    assert parts.shape[0] == Lf and 0 <= best < Lf
    assert np.isfinite(c) and c == c2 and torch.equal(b, b2)
    assert torch.equal(parts[best], b)
    r = O.rollout(p, b.cpu().numpy().astype(np.float64)[None], p.J_max - 1, pidx=[best],
                  W=oracle_wind(p))
    if (r["margin"] >= 1e-5).all() and (r["smargin"] >= 1e-5).all():
        assert r["cbar"][:, 0].sum() == pytest.approx(c, rel=1e-4)


def test_solve_quality_matches_oracle_statistically(torch, pkg):
    gpu, orc = [], []
    for step in range(3):
        p = _scheduled(L=1024, J_max=10, frac=0.25).copy(mpc_step=step)
        sol = pkg.Solver(p)
        sol.set_state(mpc_step=step)
        _, c, _ = sol.solve()
        sol.close()
        gpu.append(c)
        orc.append(O.smc_solve(p, nthreads=8)["best_sum"])
    gpu, orc = np.array(gpu), np.array(orc)
    assert np.isfinite(gpu).all() and np.isfinite(orc).all()
    assert abs(np.median(gpu) - np.median(orc)) <= 0.1 * np.median(orc), (gpu, orc)


def test_schedule_with_moves_and_sample_schedule(torch, pkg):
    """The particle schedule composes with the accepted moves and the sample
    schedule: the solve runs, the move counts acceptances out of L_{J+1}."""
    p = S.shrink(S.config4(), M=12, H=30, L=2048, J_max=5)
    p = p.copy(L_sched=(2048, 1024, 1024, 512, 512), sample_mode=1)
    sol = pkg.Solver(p)
    sol.set_move(2, 1e-4)
    _, c, _ = sol.solve()
    acc, _ = sol.mh_stats()
    sol.close()
    assert np.isfinite(c)
    assert (acc > 0).all() and (acc <= np.array(p.L_sched[1:])).all()
    assert acc[0] > 0.97 * p.L_sched[1]
