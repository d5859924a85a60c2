"""Rolling window on the GPU (the paper's rolling-window section): aircraft
that enter at preset MPC steps, late entrants scored over their active steps,
finished aircraft out of the problem, the plant retiring arrivals in the
landing sector, and the batched kernel with a varying active set -- against
the FP64 oracle's rolling window, pinned on the CPU against the same
situations stated without the window."""
import math

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


def windowed(t=4, H=30, L=600, M=3, finished=1 << 5):
    """Six aircraft of the 12-aircraft traffic at MPC step t: two present, one
    entering in 3 steps, one in 10, one after the horizon, one finished."""
    p = S.shrink(S.config4(), L=L, M=M, H=H)
    ac = p.aircraft[:6].copy()
    ac["t_enter"] = [0, t, t + 3, t + 10, t + H + 5, 0]
    return p.copy(N=6, aircraft=ac, rolling=1, mpc_step=t, finished=finished)


def _solver(pkg, p):
    sol = pkg.Solver(p)
    sol.set_state(mpc_step=p.mpc_step)
    sol.set_finished(p.finished)
    return sol


@pytest.mark.parametrize("J,soft", [(0, False), (3, True)])
def test_rollout_matches_oracle(torch, pkg, J, soft):
    p = windowed()
    rng = np.random.default_rng(60 + J)
    u = S.mild_controls(p, p.L, rng)
    sol = _solver(pkg, p)
    cbar, cs = sol.rollout_cost(torch.from_numpy(u).cuda(), J, soft=soft)
    samp = sol.sample_costs(p.L).cpu().numpy().astype(np.float64).transpose(2, 0, 1)
    live = sol.live_steps()
    status, fin = sol.status()
    sol.close()
    assert list(status) == [1, 1, 0, 0, 0, 2] and fin == 1 << 5
    ref = O.rollout(p, u, J, W=oracle_wind(p), soft=soft)
    got = cbar.cpu().numpy().astype(np.float64)
    emax, n, _ = compare_costs(got, ref["cbar"], ref["margin"], ref["smargin"], f"rolling J={J}")
    assert n > 1000
    if soft:
        compare_costs(cs.cpu().numpy().astype(np.float64), ref["cbar_soft"], ref["margin"],
                      ref["smargin"], "rolling soft")
    # absent aircraft cost exactly 0 in every particle and sample
    assert (got[4] == 0).all() and (got[5] == 0).all() and (samp[:, :, 4:] == 0).all()
    assert abs(live - ref["live"]) <= 0.001 * ref["live"]
    keep = (ref["smargin"] >= 1e-5) & (ref["margin"].min(0) >= 1e-5)
    g, r = samp[keep], ref["cost"][keep]
    fin_r = np.isfinite(r)
    assert (np.isfinite(g) == fin_r).all()
    err = np.abs(g[fin_r] - r[fin_r]) / np.maximum(np.abs(r[fin_r]), COST_FLOOR)
    assert err.max() <= COST_TOL


def test_rolling_window_with_corner_wind_and_sample_schedule(torch, pkg):
    """The combination the paper's standard problem uses (Sec. 4.4, Sec. 5.1):
    rolling window, each particle's wind on the 2x2x2 corner grid drawn in the
    kernel, and iteration J rolling out min(SampleSchedule(J), M) samples."""
    p = windowed(H=12, L=256, M=12).copy(grid=(2, 2, 2), wind_mode=1, sample_mode=1)
    rng = np.random.default_rng(61)
    u = S.mild_controls(p, p.L, rng)
    J = 5                                        # SampleSchedule(5) = 9 < M
    sol = _solver(pkg, p)
    cbar, _ = sol.rollout_cost(torch.from_numpy(u).cuda(), J)
    sol.close()
    # the oracle's rollout averages over all of p.M: hand it the iteration's samples
    ref = O.rollout(p.copy(M=O.samples(p, J)), u, J, soft=False)
    got = cbar.cpu().numpy().astype(np.float64)
    emax, n, _ = compare_costs(got, ref["cbar"], ref["margin"], ref["smargin"], "rolling corner wind")
    assert n > 300
    assert (got[4] == 0).all() and (got[5] == 0).all()


def test_everyone_present_is_the_plain_rollout(torch, pkg):
    p = windowed(finished=0)
    ac = p.aircraft.copy()
    ac["t_enter"] = 0
    p = p.copy(aircraft=ac)
    u = torch.from_numpy(S.mild_controls(p, p.L, np.random.default_rng(61))).cuda()
    out = []
    for q in (p, p.copy(rolling=0)):
        sol = _solver(pkg, q)
        c, _ = sol.rollout_cost(u, 2)
        out.append(c.cpu().numpy())
        sol.close()
    assert np.array_equal(out[0], out[1])


def test_plant_moves_active_aircraft_and_retires_landed_arrivals(torch, pkg):
    p = windowed(t=4, finished=0)
    ac = p.aircraft.copy()
    # aircraft 0: an arrival placed in the landing sector (it lands during the step)
    ac[0]["type"], ac[0]["x"], ac[0]["y"], ac[0]["z"] = 0, 5000.0, 0.0, 300.0
    ac[0]["v"], ac[0]["chi"] = 85.0, math.pi
    p = p.copy(aircraft=ac)
    rng = np.random.default_rng(62)
    u = S.mild_controls(p, 1, rng)[0]
    u[0] = 0.0
    sol = _solver(pkg, p)
    pkg.tma_plant_step(sol.h, torch.from_numpy(u).cuda())
    x, mpc = pkg.tma_get_state(sol.h, p.N)
    status, fin = sol.status()
    sol.close()
    x0 = np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])
    ref = O.plant_step(p, x0, oracle_wind(p)[0, 0], u[:, 0, :])
    scale = np.array([1e4, 1e4, 1e3, 1e2, 1.0, 1e4])
    assert np.all(np.abs(x - ref) <= 2e-6 * np.maximum(np.abs(ref), scale)), (x, ref)
    for i in (2, 3, 4):                    # not entered: kept in place
        assert np.array_equal(x[i], x0[i].astype(np.float32).astype(np.float64))
    assert mpc == 5
    want = O.plant_finished(p, ref)
    assert want & 1 and fin == want
    assert status[0] == 2 and status[1] == 1


def test_solve_best_cost_reproduced_by_oracle(torch, pkg):
    p = windowed(L=2048, M=4)
    sol = _solver(pkg, p)
    b, c, _ = sol.solve()
    best = sol.best_index()
    b2, c2, _ = sol.solve()
    sol.close()
    assert np.isfinite(c) and c == c2 and torch.equal(b, b2)
    r = O.rollout(p, b.cpu().numpy().astype(np.float64)[None], p.J_max - 1, pidx=[best],
                  W=oracle_wind(p))
    if (r["margin"] >= 1e-5).all() and (r["smargin"] >= 1e-5).all():
        assert r["cbar"][:, 0].sum() == pytest.approx(c, rel=1e-4)


def test_mpc_loop_brings_aircraft_in(torch, pkg):
    """Over the receding-horizon loop the waiting aircraft stay put until their
    entry step and move afterwards."""
    p = windowed(t=0, L=1024, M=3, H=24, finished=0)
    ac = p.aircraft.copy()
    ac["t_enter"] = [0, 0, 2, 3, 40, 1]
    p = p.copy(aircraft=ac)
    sol = _solver(pkg, p)
    T, costs, _ = pkg.tma_mpc_run(sol.h, 4, p.N)      # states [steps][N][6] after each plant step
    status, _ = sol.status()
    sol.close()
    x0 = np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])
    for t in range(4):
        for i in range(p.N):
            moved = not np.allclose(T[t, i], x0[i].astype(np.float32))
            assert moved == (ac["t_enter"][i] <= t), (t, i)
    assert np.isfinite(costs).all()
    assert list(status) == [1, 1, 1, 1, 0, 1]


def test_gradient_and_langevin_refuse_the_window(torch, pkg):
    p = windowed(L=64)
    sol = _solver(pkg, p)
    u = torch.zeros((p.L, p.N, p.S, 3), device="cuda")
    with pytest.raises(pkg.TmaError):
        sol.rollout_grad(u, 0)
    with pytest.raises(pkg.TmaError):
        sol.set_move(2, 0.1)
    sol.set_move(1, 0.5)                    # the random-walk move needs no gradient
    _, c, _ = sol.solve()
    sol.close()
    assert np.isfinite(c)


def test_batch_equals_single_solves_with_varying_active_sets(torch, pkg):
    ps = S.config5(n_scen=24)
    order = sorted(range(len(ps)), key=lambda s: ps[s].N)
    pick = [order[0], order[len(order) // 2], order[-1]]
    out = []
    for n, k in enumerate(pick):
        q = S.shrink(ps[k], L=512, M=3, H=24, J_max=3)
        ac = q.aircraft.copy()
        ac["t_enter"] = (np.arange(q.N) * (n + 2)) % 30     # some now, some later, some beyond H
        out.append(q.copy(aircraft=ac, rolling=1, mpc_step=2))
    Ns = [p.N for p in out]
    b = pkg.tma_batch_create(out)
    pkg.tma_batch_set_state(b, None, [p.mpc_step for p in out])
    pkg.tma_batch_solve(b)
    res = pkg.tma_batch_results(b, Ns, out[0].S)
    pkg.tma_batch_destroy(b)
    for k, p in enumerate(out):
        sol = _solver(pkg, p)
        bu, c, _ = sol.solve()
        sol.close()
        assert np.array_equal(res["best_u"][k], bu.cpu().numpy()), k
        assert res["best_cost"][k] == c or (np.isinf(c) and np.isinf(res["best_cost"][k]))
