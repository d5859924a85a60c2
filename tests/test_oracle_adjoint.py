"""Pins of the oracle's reverse-mode gradient of the soft cost (the gradient
that the Langevin move of the particles uses).

The gradient routine re-runs the rollout with the reduced forms of the
dynamics (z' = z + dt hdot, v' = v + dt a, chi' = chi + dt w, drag in closed
form).  The forward rollout it is checked against uses the literal forms of
Eq. (hor) (lift coefficient from the coordinated turn, drag polar), so the
value test below also pins the reduction.  Derivatives are pinned by central
finite differences of that independent forward rollout."""
import math

import numpy as np
import pytest

import oracle as O
import scenarios as S


def soft_objective(p, u, W, l=0, J=0):
    """sum_i mean_m c_soft[i][m] by the forward rollout (Sec. 3.3-3.6)."""
    r = O.rollout(p, u[None], J, pidx=np.array([l]), W=W, soft=True)
    return float(r["cbar_soft"][:, 0].sum()), r


def close_pair():
    """Two aircraft 1.1 separation radii apart at nearly the same altitude, so
    that the softplus separation term carries a sizeable gradient."""
    p = S.shrink(S.config1(), M=2, H=16)
    p = p.copy(sep_mode=1, sp_beta=4.0, mu_sep=0.5)
    a = p.aircraft
    a[0]["x"], a[0]["y"], a[0]["z"], a[0]["chi"] = 8000.0, 0.0, 3000.0, math.pi
    a[1]["type"] = 1
    a[1]["x"], a[1]["y"], a[1]["z"], a[1]["chi"] = 8000.0 + 1.1 * p.sep_h, 200.0, 3100.0, math.pi
    a[1]["v"] = 170.0
    return p


SCALES = np.array([1.5 * math.pi / 180.0, 15.0, 1.0])


def _feasible_controls(p, W, seed, need_margin=1e-3, tries=50):
    rng = np.random.default_rng(seed)
    for _ in range(tries):
        u = S.mild_controls(p, 1, rng)[0].astype(np.float64)
        c, r = soft_objective(p, u, W)
        if np.isfinite(c) and r["margin"].min() > need_margin:
            return u
    raise AssertionError("no feasible controls found")


def _fd(p, u, W, n, h):
    up, um = u.copy(), u.copy()
    up.flat[n] += h
    um.flat[n] -= h
    return (soft_objective(p, up, W)[0] - soft_objective(p, um, W)[0]) / (2 * h)


@pytest.mark.parametrize("which", ["config1", "config4", "close_pair", "noise"])
def test_gradient_matches_central_differences(which):
    if which == "config1":
        p = S.shrink(S.config1(), M=2, H=20)
    elif which == "config4":
        p = S.shrink(S.config4(), M=2, H=24)
        p = p.copy(aircraft=p.aircraft[:5], N=5)
    elif which == "close_pair":
        p = close_pair()
    else:
        p = S.shrink(S.config3(), M=2, H=24, grid=(16, 16, 4))
        p = p.copy(aircraft=p.aircraft[:4], N=4)
    W = O.wind_field(p)
    u = _feasible_controls(p, W, seed=7)
    c, g = O.rollout_grad(p, u, W)
    c_fwd, _ = soft_objective(p, u, W)
    assert abs(c - c_fwd) <= 1e-11 * max(1.0, abs(c_fwd))
    fd = np.empty_like(g)
    for n in range(g.size):
        h = 1e-6 * SCALES[n % 3]
        fd.flat[n] = _fd(p, u, W, n, h)
    scale = np.abs(fd).reshape(-1, 3).max(axis=0)           # per control kind
    err = np.abs(g - fd).reshape(-1, 3) / np.maximum(scale, 1e-300)
    assert err.max() <= 2e-5, (which, err.max(), np.unravel_index(err.argmax(), err.shape))
    # every control kind of every aircraft influences the cost
    assert (np.abs(g).reshape(p.N, -1).max(axis=1) > 0).all()


def test_separation_gradient_pushes_the_pair_apart():
    """The separation part of the gradient (the difference between mu > 0 and
    mu = 0, the cost being linear in mu) is non-zero for a close pair, raises
    the cost, and matches the same difference of finite differences."""
    p = close_pair()
    W = O.wind_field(p)
    u = np.zeros((p.N, p.S, 3))
    u[:, :, 1] = 1.0
    c0, g0 = O.rollout_grad(p, u, W)
    p2 = p.copy(mu_sep=0.0)
    c1, g1 = O.rollout_grad(p2, u, W)
    gsep = g0 - g1                      # the separation part, by linearity in mu
    assert np.isfinite(c0) and c0 > c1
    assert np.abs(gsep).max() > 0
    fd = []
    for n in (0 * p.S * 3 + 2, 1 * p.S * 3 + 2):
        fd.append((_fd(p, u, W, n, 1e-6) - _fd(p2, u, W, n, 1e-6)))
    assert np.allclose([gsep[0, 0, 2], gsep[1, 0, 2]], fd, rtol=1e-4, atol=1e-9)


def test_directional_derivative():
    """<grad, d> equals the central difference along a random direction d."""
    p = S.shrink(S.config4(), M=3, H=20)
    p = p.copy(aircraft=p.aircraft[:6], N=6)
    W = O.wind_field(p)
    u = _feasible_controls(p, W, seed=11)
    _, g = O.rollout_grad(p, u, W, l=3, J=2)
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.standard_normal(u.shape) * SCALES
        eps = 1e-6
        cp = O.rollout(p, (u + eps * d)[None], 2, pidx=np.array([3]), W=W)["cbar_soft"].sum()
        cm = O.rollout(p, (u - eps * d)[None], 2, pidx=np.array([3]), W=W)["cbar_soft"].sum()
        fd = (cp - cm) / (2 * eps)
        assert abs(float(np.sum(g * d)) - fd) <= 1e-5 * max(abs(fd), 1e-3)


def test_infeasible_particle_has_infinite_cost_and_zero_gradient():
    p = S.shrink(S.config1(), M=2, H=20)
    W = O.wind_field(p)
    u = np.zeros((p.N, p.S, 3))
    u[:, :, 1] = 15.0 * 5          # climb far beyond sin(gamma_max) v
    c, g = O.rollout_grad(p, u, W)
    assert math.isinf(c) and not g.any()


def test_wind_free_gradient_of_straight_flight():
    """Without wind and turbulence, a departure scored on altitude alone has a
    negative climb-rate gradient in every segment while below its target
    altitude (climbing reduces |Z - z|), larger in magnitude for earlier
    segments (they act on more steps of the sum); scored on fuel alone, its
    speed-change and climb-rate gradients are positive (both raise thrust)."""
    base = S.shrink(S.config1(), M=1, H=20).copy(wind_sigma=0.0, turb_sigma=0.0)
    base = base.copy(aircraft=base.aircraft[1:], N=1)
    u = np.zeros((1, base.S, 3))
    u[0, :, 1] = 2.0
    p = base.copy(alpha_dep=(0.0, 0.0, 1.0, 0.0))
    c, g = O.rollout_grad(p, u, O.wind_field(p))
    assert np.isfinite(c)
    assert (g[0, :, 1] < 0).all()
    assert (np.diff(np.abs(g[0, :, 1])) < 0).all()
    assert not g[0, :, 0].any() and not g[0, :, 2].any()
    p = base.copy(alpha_dep=(0.0, 1.0, 0.0, 0.0))
    c, g = O.rollout_grad(p, u, O.wind_field(p))
    assert (g[0, :, 1] > 0).all() and (g[0, :, 2] > 0).all()
