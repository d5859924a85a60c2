"""Batched MPC on the GPU: many scenarios with uneven aircraft counts in one
persistent launch per stage, the receding-horizon loop (plant step) and its
CUDA-graph capture.  The batched solve shares the single-scenario arithmetic,
so it must reproduce single-scenario solves bit for bit; the plant step is
checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gpu_helpers import compare_sample_costs, cuda, oracle_wind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda()


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_1506_02869_gb300 as pkg
    return pkg


def mixed_batch(n, L=1024, M=4, H=24, J=4):
    """Scenarios of the batched workload spanning the aircraft counts: 2 (16
    tiles per CTA), around 10 (3 tiles), above 16 (1 tile) and the largest."""
    ps = S.config5(n_scen=48)
    order = sorted(range(len(ps)), key=lambda s: ps[s].N)
    pick = [order[0], order[len(order) // 3], order[len(order) // 2], order[-1],
            order[len(order) // 4], order[-2], order[1], order[-3]][:n]
    return [S.shrink(ps[k], L=L, M=M, H=H, J_max=J) for k in pick]


def _states(p):
    return np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])


@pytest.mark.parametrize("dispatch", [0, 1])
def test_batch_solve_equals_single_solves(torch, pkg, dispatch):
    """Both rollout dispatch forms (one persistent launch; a launch per
    scenario)."""
    ps = mixed_batch(6)
    Ns = [p.N for p in ps]
    assert min(Ns) <= 3 and max(Ns) > 16
    b = pkg.tma_batch_create(ps)
    form, timed = pkg.tma_batch_get_dispatch(b)
    assert form in (0, 1) and timed[0] > 0 and timed[1] > 0
    assert form == (1 if timed[1] < timed[0] else 0)
    pkg.tma_batch_set_dispatch(b, dispatch)
    pkg.tma_batch_solve(b)
    res = pkg.tma_batch_results(b, Ns, ps[0].S)
    live = pkg.tma_batch_live_steps(b)
    lat = pkg.tma_batch_latency(b, len(ps))
    pkg.tma_batch_destroy(b)
    live_single = 0
    for k, p in enumerate(ps):
        sol = pkg.Solver(p)
        bu, c, _ = sol.solve()
        best = sol.best_index()
        live_single += sol.live_steps()
        sol.close()
        assert np.array_equal(res["best_u"][k], bu.cpu().numpy()), k
        assert res["best_cost"][k] == c or (np.isinf(c) and np.isinf(res["best_cost"][k]))
        assert res["best"][k] == best
    assert live == live_single
    assert (lat > 0).all() and np.isfinite(lat).all()


def test_batched_rollout_matches_oracle_at_full_size(torch, pkg):
    """The batched persistent rollout against the FP64 oracle directly (not
    only through the single-scenario path): scenarios of the batched workload
    with 2, about 17 and 32 aircraft at its full sizes (L 16384, M 16, H 60),
    one persistent launch; the per-sample costs of 32 sampled particles per
    scenario, every sample, compared one by one."""
    ps_all = S.config5(n_scen=256)
    Ns_all = np.array([p.N for p in ps_all])
    pick = [int(np.nonzero(Ns_all == 2)[0][0]), int(np.argmin(np.abs(Ns_all - 17))),
            int(np.nonzero(Ns_all == 32)[0][0])]
    ps = [ps_all[k] for k in pick]
    Ns = [p.N for p in ps]
    L, M = ps[0].L, ps[0].M
    assert (L, M, ps[0].H) == (16384, 16, 60) and Ns[0] == 2 and Ns[2] == 32
    rng = np.random.default_rng(80)
    us = []
    for p in ps:
        u = S.mild_controls(p, L, rng)
        u[: L // 4] = S.random_controls(p, L // 4, rng)
        us.append(u)
    J = 2
    b = pkg.tma_batch_create(ps)
    packed = torch.from_numpy(np.concatenate([u.reshape(-1) for u in us])).cuda()
    costs = []
    for form in (0, 1):                        # the persistent launch, then a launch per scenario
        pkg.tma_batch_set_dispatch(b, form)
        c = torch.full((M * L * sum(Ns),), float("nan"), dtype=torch.float32, device="cuda")
        pkg.tma_batch_rollout_cost(b, packed, J, c)
        torch.cuda.synchronize()
        costs.append(c.cpu().numpy())
    pkg.tma_batch_destroy(b)
    assert np.array_equal(costs[0], costs[1])
    cost = costs[0].astype(np.float64)
    off = 0
    for k, p in enumerate(ps):
        block = cost[off: off + M * p.N * L].reshape(M, p.N, L)
        off += M * p.N * L
        assert not np.isnan(block).any()
        pidx = np.unique(np.r_[rng.choice(L, 30, replace=False), [0, L - 1]])
        ref = O.rollout_at_samples(p, us[k][pidx].astype(np.float64), J, list(range(M)), pidx=pidx,
                                   soft=False, nthreads=8)
        compare_sample_costs(block[:, :, pidx].transpose(2, 0, 1), ref["cost"], ref["margin"],
                             ref["smargin"], f"batched N={p.N}")


def test_batch_solve_with_five_segments_equals_single_solves(torch, pkg):
    """S = 5 (15 controls per aircraft) takes the batched move's general form
    (four segments take the unrolled one)."""
    ps = [p.copy(S=5) for p in mixed_batch(3, L=512, M=3, H=20, J=3)]
    Ns = [p.N for p in ps]
    b = pkg.tma_batch_create(ps)
    pkg.tma_batch_solve(b)
    res = pkg.tma_batch_results(b, Ns, 5)
    pkg.tma_batch_destroy(b)
    for k, p in enumerate(ps):
        sol = pkg.Solver(p)
        bu, c, _ = sol.solve()
        sol.close()
        assert np.array_equal(res["best_u"][k], bu.cpu().numpy()), k
        assert res["best_cost"][k] == c or (np.isinf(c) and np.isinf(res["best_cost"][k]))


def test_batch_mpc_graph_equals_eager_and_single_loop(torch, pkg):
    ps = mixed_batch(4, L=512, M=3, H=20, J=3)
    Ns = [p.N for p in ps]
    bg = pkg.tma_batch_create(ps)
    be = pkg.tma_batch_create(ps)
    pkg.tma_batch_mpc(bg, 2, use_graph=True)
    pkg.tma_batch_mpc(be, 2, use_graph=False)
    rg = pkg.tma_batch_results(bg, Ns, ps[0].S)
    re = pkg.tma_batch_results(be, Ns, ps[0].S)
    for k in range(len(ps)):
        assert np.array_equal(rg["states"][k], re["states"][k])
        assert np.array_equal(rg["best_u"][k], re["best_u"][k])
    assert (rg["mpc"] == np.array([p.mpc_step + 2 for p in ps])).all()
    # replaying the captured graph continues from the advanced state
    pkg.tma_batch_mpc(bg, 2, use_graph=True)
    pkg.tma_batch_mpc(be, 2, use_graph=False)
    rg = pkg.tma_batch_results(bg, Ns, ps[0].S)
    re = pkg.tma_batch_results(be, Ns, ps[0].S)
    for k in range(len(ps)):
        assert np.array_equal(rg["states"][k], re["states"][k])
    pkg.tma_batch_destroy(bg)
    pkg.tma_batch_destroy(be)
    # the same loop through single-scenario solvers: solve, then the plant step
    for k, p in enumerate(ps):
        sol = pkg.Solver(p)
        for _ in range(4):
            bu, _, _ = sol.solve()
            pkg.tma_plant_step(sol.h, bu)
        x, mpc = pkg.tma_get_state(sol.h, p.N)
        sol.close()
        assert mpc == p.mpc_step + 4
        assert np.array_equal(x.astype(np.float32), re["states"][k].astype(np.float32)), k


def test_plant_step_matches_oracle(torch, pkg):
    p = S.config1().copy(mpc_step=2)
    sol = pkg.Solver(p)
    sol.set_state(mpc_step=2)
    rng = np.random.default_rng(31)
    u = S.mild_controls(p, 1, rng)[0]
    pkg.tma_plant_step(sol.h, torch.from_numpy(u).cuda())
    x, mpc = pkg.tma_get_state(sol.h, p.N)
    sol.close()
    ref = O.plant_step(p, _states(p), oracle_wind(p)[0, 0], u[:, 0, :])
    assert mpc == 3
    scale = np.array([1e4, 1e4, 1e3, 1e2, 1.0, 1e4])
    assert np.all(np.abs(x - ref) <= 2e-6 * np.maximum(np.abs(ref), scale)), (x, ref)


def test_plant_step_limits_thrust_like_the_oracle(torch, pkg):
    # a steep descent needs negative thrust: the plant applies Tmin and slows down
    p = S.config1()
    sol = pkg.Solver(p)
    u = np.zeros((p.N, p.S, 3), np.float32)
    u[:, :, 1] = -15.0
    u[:, :, 2] = -1.0
    pkg.tma_plant_step(sol.h, torch.from_numpy(u).cuda())
    x, _ = pkg.tma_get_state(sol.h, p.N)
    sol.close()
    ref = O.plant_step(p, _states(p), oracle_wind(p)[0, 0], u[:, 0, :])
    assert np.allclose(x, ref, rtol=2e-6, atol=1e-3)
    assert (ref[:, 5] == _states(p)[:, 5]).all()          # idle thrust burns no fuel


def test_batch_rejects_mismatched_shapes(torch, pkg):
    ps = mixed_batch(2)
    ps[1] = ps[1].copy(M=ps[0].M + 1)
    with pytest.raises(pkg.TmaError):
        pkg.tma_batch_create(ps)


def test_mpc_run_equals_the_solve_and_plant_loop(torch, pkg):
    p = S.shrink(S.config1(), L=512, M=3, H=20, J_max=4)
    sol = pkg.Solver(p)
    traj, costs, st = pkg.tma_mpc_run(sol.h, 3, p.N)
    assert pkg.tma_get_error(sol.h) == 0
    sol.close()
    sol = pkg.Solver(p)
    for t in range(3):
        bu, c, _ = sol.solve()
        pkg.tma_plant_step(sol.h, bu)
        x, mpc = pkg.tma_get_state(sol.h, p.N)
        assert np.array_equal(x, traj[t]) and c == costs[t]
    assert mpc == p.mpc_step + 3
    sol.close()


def test_error_word_reports_an_infeasible_choice(torch, pkg):
    p = S.shrink(S.config1(), L=256, M=2, H=10, J_max=2).copy(z_min=5500.0)
    sol = pkg.Solver(p)
    sol.solve()
    sol.solve()
    assert pkg.tma_get_error(sol.h) & 2
    assert pkg.tma_get_error(sol.h) == 0        # cleared by the read
    sol.close()


def test_batch_full_size_in_one_launch_equals_single_solves(torch, pkg):
    """The batched workload at full size -- 256 scenarios of 2 to 32 aircraft,
    L 16384, M 16, H 60, all in one persistent launch per stage -- for one
    iteration (J_max = 1: initial controls, rollout, selection), against the
    single-scenario solver on sampled scenarios (the smallest, the largest and
    two between); the chosen controls and their costs are the same bits."""
    ps = [p.copy(J_max=1) for p in S.config5(n_scen=256)]
    assert len(ps) == 256 and ps[0].L == 16384 and ps[0].M == 16 and ps[0].H == 60
    Ns = [p.N for p in ps]
    b = pkg.tma_batch_create(ps)
    pkg.tma_batch_solve(b)
    res = pkg.tma_batch_results(b, Ns, ps[0].S)
    pkg.tma_batch_destroy(b)
    order = sorted(range(len(ps)), key=lambda s: ps[s].N)
    for k in (order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]):
        sol = pkg.Solver(ps[k])
        bu, c, _ = sol.solve()
        best = sol.best_index()
        sol.close()
        assert np.array_equal(res["best_u"][k], bu.cpu().numpy()), k
        assert res["best_cost"][k] == c or (np.isinf(c) and np.isinf(res["best_cost"][k])), k
        assert res["best"][k] == best, k
