"""The gradient of the soft cost and the Metropolis-Hastings moves on the GPU,
against the FP64 oracle (its reverse-mode gradient, pinned by finite
differences; its proposal and accept step, pinned by the Metropolis-Hastings
ratio and Gaussian-target invariance).

Gradient bar: relative L2 error per particle <= 1e-3 of the oracle's gradient,
for every particle whose threshold decisions are not within 1e-5 (relative) of
their thresholds in the oracle.  (A gradient also has kinks -- |.|, the
wrapped angle, the min of the separation gap -- where FP32 and FP64 could take
opposite sides; on these seeded cases no particle comes near the bar: the
largest error is 1.8e-4, so no allowance for them is made.)"""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from gpu_helpers import TAU, cuda, oracle_wind

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def torch():
    return cuda()


@pytest.fixture(scope="module")
def pkg(torch):
    import paper_1506_02869_gb300 as pkg
    return pkg


def _close_pair_problem():
    import math
    p = S.shrink(S.config4(), M=4, H=30, L=96)
    p = p.copy(aircraft=p.aircraft[:3].copy(), N=3, sp_beta=4.0, mu_sep=0.5)
    a = p.aircraft
    a[0]["x"], a[0]["y"], a[0]["z"], a[0]["chi"] = 8000.0, 0.0, 3000.0, math.pi
    a[1]["x"], a[1]["y"], a[1]["z"], a[1]["chi"] = 8000.0 + 1.1 * p.sep_h, 200.0, 3100.0, math.pi
    a[2]["x"], a[2]["y"], a[2]["z"], a[2]["chi"] = 8000.0, 1.2 * p.sep_h, 3050.0, math.pi
    return p


CASES = {
    "config4": lambda: S.shrink(S.config4(), M=4, H=40, L=100),
    "close_pair": _close_pair_problem,
    "noise": lambda: S.shrink(S.config3(), M=3, H=30, L=70, grid=(16, 16, 4)).copy(sep_mode=1),
    "config1": lambda: S.shrink(S.config1(), M=5, H=20, L=64).copy(sep_mode=1),
}


def _grad_case(torch, pkg, p, J=2, seed=0):
    rng = np.random.default_rng(seed)
    u = S.mild_controls(p, p.L, rng)
    sol = pkg.Solver(p)
    sol.wind_field()
    cost, grad, cb = sol.rollout_grad(torch.from_numpy(u).cuda(), J, cbar=True)
    torch.cuda.synchronize()
    out = dict(cost=cost.cpu().numpy(), grad=grad.cpu().numpy(), cbar=cb.cpu().numpy(), sol=sol, u=u)
    return out


@pytest.mark.parametrize("case", list(CASES))
def test_gradient_matches_oracle_adjoint(torch, pkg, case):
    p = CASES[case]()
    J = 2
    g = _grad_case(torch, pkg, p, J)
    g["sol"].close()
    W = oracle_wind(p)
    ref = O.rollout(p, g["u"].astype(np.float64), J, W=W)
    keep = (ref["smargin"] >= TAU) & (ref["margin"].min(axis=0) >= TAU)
    feas = np.isfinite(ref["cbar_soft"]).all(axis=0)
    cmp = keep & feas
    assert cmp.sum() >= 0.5 * p.L, (case, cmp.sum())
    # feasibility agrees wherever decisions are clear
    assert np.array_equal(np.isfinite(g["cost"])[keep], feas[keep])
    errs = []
    for l in np.nonzero(cmp)[0]:
        c_ref, g_ref = O.rollout_grad(p, g["u"][l].astype(np.float64), W, l=int(l), J=J)
        assert abs(g["cost"][l] - c_ref) <= 1e-4 * max(abs(c_ref), 1e-2)
        e = np.linalg.norm(g["grad"][l] - g_ref) / max(np.linalg.norm(g_ref), 1e-30)
        errs.append(e)
    errs = np.array(errs)
    n_bad = int((errs > GRAD_TOL).sum())
    print(f"gradient {case}: {errs.size} particles compared, {n_bad} above {GRAD_TOL}, "
          f"median {np.median(errs):.2e}, max {errs.max():.2e}")
    assert n_bad == 0, (case, n_bad, errs.size, float(np.median(errs)), float(errs.max()))
    # infeasible particles: +inf cost and a zero gradient
    inf = ~np.isfinite(g["cost"])
    assert not g["grad"][inf].any()


def test_gradient_matches_oracle_adjoint_at_full_size(torch, pkg):
    """The 12-aircraft workload at its full size (L 16384, M 16, H 60,
    softplus separation, checkpoints every 10 steps) in the launch the solver
    runs; the gradients of 64 sampled particles against the oracle's adjoint
    (the compared ones: those without a decision near its threshold and
    feasible)."""
    p = S.config4()
    assert (p.L, p.M, p.N, p.H) == (16384, 16, 12, 60)
    J = 3
    g = _grad_case(torch, pkg, p, J, seed=21)
    g["sol"].close()
    rng = np.random.default_rng(22)
    pidx = np.unique(np.r_[rng.choice(p.L, 62, replace=False), [0, p.L - 1]])
    W = oracle_wind(p)
    ref = O.rollout(p, g["u"][pidx].astype(np.float64), J, pidx=pidx, W=W, nthreads=8)
    keep = (ref["smargin"] >= TAU) & (ref["margin"].min(axis=0) >= TAU)
    feas = np.isfinite(ref["cbar_soft"]).all(axis=0)
    assert np.array_equal(np.isfinite(g["cost"][pidx])[keep], feas[keep])
    errs = []
    for q in np.nonzero(keep & feas)[0]:
        l = int(pidx[q])
        c_ref, g_ref = O.rollout_grad(p, g["u"][l].astype(np.float64), W, l=l, J=J)
        assert abs(g["cost"][l] - c_ref) <= 1e-4 * max(abs(c_ref), 1e-2)
        errs.append(np.linalg.norm(g["grad"][l] - g_ref) / max(np.linalg.norm(g_ref), 1e-30))
    errs = np.array(errs)
    n_bad = int((errs > GRAD_TOL).sum())
    print(f"full-size gradient: {errs.size} particles compared, {n_bad} above {GRAD_TOL}, "
          f"median {np.median(errs):.2e}, max {errs.max():.2e}")
    assert errs.size >= 20
    assert n_bad == 0, (n_bad, errs.size, float(errs.max()))


def test_gradient_pass_costs_are_the_rollout_costs(torch, pkg):
    """Same step function as the rollout: the same feasibility, and costs equal
    up to the order of the separation-penalty sum (accumulated backwards in the
    gradient pass)."""
    p = S.shrink(S.config4(), M=4, H=40, L=200)
    g = _grad_case(torch, pkg, p, J=3, seed=4)
    sol = g["sol"]
    _, cs = sol.rollout_cost(torch.from_numpy(g["u"]).cuda(), 3, soft=True)
    cs = cs.cpu().numpy()
    sol.close()
    assert np.array_equal(np.isfinite(cs), np.isfinite(g["cbar"]))
    fin = np.isfinite(cs)
    assert np.allclose(g["cbar"][fin], cs[fin], rtol=2e-6, atol=1e-7)
    tot = np.where(np.isfinite(cs).all(axis=0), cs.astype(np.float64).sum(axis=0), np.inf)
    assert np.allclose(g["cost"], tot, rtol=1e-6, atol=0)


def test_gradient_is_deterministic_and_ragged(torch, pkg):
    p = S.shrink(S.config4(), M=3, H=25, L=37)
    a = _grad_case(torch, pkg, p, J=1, seed=9)
    b = _grad_case(torch, pkg, p, J=1, seed=9)
    a["sol"].close()
    b["sol"].close()
    assert np.array_equal(a["grad"], b["grad"]) and np.array_equal(a["cost"], b["cost"])
    # the first particles of a larger call are the same computation
    p2 = p.copy(L=37 + 64)
    c = _grad_case(torch, pkg, p2, J=1, seed=9)
    c["sol"].close()
    rng = np.random.default_rng(9)
    assert np.array_equal(c["u"][:37], S.mild_controls(p, 37, rng))
    assert np.allclose(c["grad"][:37], a["grad"], rtol=1e-6, atol=1e-9)


def test_autograd_wrapper(torch, pkg):
    p = S.shrink(S.config4(), M=2, H=20, L=64)
    rng = np.random.default_rng(5)
    u = torch.from_numpy(S.mild_controls(p, p.L, rng)).cuda().requires_grad_(True)
    sol = pkg.Solver(p)
    sol.wind_field()
    cost = pkg.rollout_cost_autograd(u, sol, 1)
    w = torch.linspace(0.5, 1.5, p.L, device="cuda")
    fin = torch.isfinite(cost)
    (torch.where(fin, cost, torch.zeros_like(cost)) * w).sum().backward()
    c2, g2, _ = sol.rollout_grad(u.detach(), 1)
    sol.close()
    assert torch.equal(cost.detach(), c2)
    assert torch.allclose(u.grad, w.reshape(-1, 1, 1, 1) * g2)


def test_gradient_rejects_long_horizons(torch, pkg):
    p = S.shrink(S.config4(), M=1, H=330, L=32)
    sol = pkg.Solver(p)
    u = torch.zeros((32, p.N, p.S, 3), device="cuda")
    with pytest.raises(pkg.TmaError):
        sol.rollout_grad(u, 0)
    sol.close()


@pytest.mark.parametrize("kind", [1, 2])
def test_mh_propose_and_accept_match_oracle(torch, pkg, kind):
    p = S.shrink(S.config4(), M=2, H=20, L=300)
    rng = np.random.default_rng(kind)
    u = S.mild_controls(p, p.L, rng)
    u[:40, :, :, 0] = np.float32(p.ctrl_hi[0]) * np.float32(0.999)   # proposals leave the box
    sg = np.asarray(p.move_sigma, np.float32)
    g = (0.05 * rng.standard_normal(u.shape) / sg).astype(np.float32)
    gp = (0.05 * rng.standard_normal(u.shape) / sg).astype(np.float32)
    cb = rng.exponential(1.0, (p.N, p.L)).astype(np.float32)
    cbp = (cb + rng.normal(0, 0.05, cb.shape)).astype(np.float32)
    cb[0, :5] = np.inf
    cbp[1, 5:10] = np.inf
    kappa, eps, J = 9.0, 1.3, 4
    sol = pkg.Solver(p)
    du = torch.from_numpy(u).cuda()
    dup = torch.empty_like(du)
    inbox = torch.empty(p.L, dtype=torch.uint8, device="cuda")
    pkg.tma_mh_propose(sol.h, du, torch.from_numpy(g).cuda(), J, kappa, eps, kind, dup, inbox)
    up_ref, inbox_ref = O.mh_propose(p, u.astype(np.float64), g.astype(np.float64), J, kappa, eps, kind)
    up = dup.cpu().numpy()
    lo, hi = np.asarray(p.ctrl_lo), np.asarray(p.ctrl_hi)
    scale = (hi - lo)
    assert np.all(np.abs(up - up_ref) <= 2e-6 * scale)
    near = (np.abs(up_ref - lo) < 1e-5 * scale) | (np.abs(up_ref - hi) < 1e-5 * scale)
    clear = ~near.reshape(p.L, -1).any(axis=1)
    ib = inbox.cpu().numpy()
    assert np.array_equal(ib[clear], inbox_ref[clear])
    assert 0 < ib.sum() < p.L
    # accept from identical FP32 inputs
    dout = torch.empty_like(du)
    acc = torch.empty(p.L, dtype=torch.uint8, device="cuda")
    pkg.tma_mh_accept(sol.h, du, dup, torch.from_numpy(cb).cuda(), torch.from_numpy(cbp).cuda(),
                      torch.from_numpy(g).cuda(), torch.from_numpy(gp).cuda(), inbox, J, kappa, eps,
                      kind, dout, acc)
    sol.close()
    out_ref, acc_ref, la = O.mh_accept(p, u.astype(np.float64), up.astype(np.float64), cb, cbp, g, gp,
                                       ib, J, kappa, eps, kind)
    a = acc.cpu().numpy().astype(bool)
    U = np.array([O.uniform23(O.draw(p, l, 0, 0, 6, J)[0]) for l in range(p.L)])
    decided = np.abs(la - np.log(U)) > 1e-9
    assert np.array_equal(a[decided], acc_ref[decided])
    assert 0 < a.sum() < p.L
    o = dout.cpu().numpy()
    assert np.array_equal(o[a], up[a]) and np.array_equal(o[~a], u[~a])


@pytest.mark.parametrize("kind,eps0", [(1, 1.0), (2, 1e-4)])
def test_solve_with_accepted_moves(torch, pkg, kind, eps0):
    """The move inside the solve: with a small first step nearly every Langevin
    proposal is accepted (the proposal density ratio and the cost change both
    vanish), which fails if the gradient, costs or random streams of the
    current and proposed particles are mismatched; the step then adapts by the
    stated rule; the solve is deterministic."""
    p = S.shrink(S.config4(), M=4, H=30, L=2048, J_max=6)
    sol = pkg.Solver(p)
    sol.set_move(kind, eps0)
    bu, c, st = sol.solve()
    acc, eps = sol.mh_stats()
    bu2, c2, _ = sol.solve()
    sol.close()
    assert np.isfinite(c) and c == c2 and torch.equal(bu, bu2)
    assert (acc > 0).all() and (acc <= p.L).all()
    assert eps[0] == eps0
    rate = acc / p.L
    if kind == 2:
        assert rate[0] > 0.97, rate
    for j in range(len(eps) - 1):
        want = 0.8 if rate[j] < 0.5 else (1.25 if rate[j] > 0.7 else 1.0)
        assert eps[j + 1] == pytest.approx(eps[j] * want, rel=1e-12)
