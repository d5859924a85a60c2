"""Pins of the oracle's Metropolis-Hastings moves (random walk and Langevin
proposal with accept step; an extension of the perturbation of Algorithm 1).

The accept ratio is checked against the textbook Metropolis-Hastings ratio
written with the Gaussian proposal densities in the original control units
(scipy's normal log-density); the chain is checked to leave a Gaussian
target invariant (an unadjusted Langevin chain, or a wrong correction, does
not); the proposal's moments are checked; and on the real soft cost a small
step is accepted almost always."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import scenarios as S


def tiny_problem(N=1, S_=1, box=1e3):
    p = S.shrink(S.config1(), M=1, H=4).copy(S=S_, N=N)
    p.aircraft = p.aircraft[:N].copy() if N <= 2 else np.resize(p.aircraft, N)
    return p.copy(ctrl_lo=(-box * 0.03, -box * 15.0, -box), ctrl_hi=(box * 0.03, box * 15.0, box))


def langevin_logq(p, to, frm, g_frm, kappa, eps):
    """log q(to | frm) of the Langevin proposal N(frm - (eps^2/2) kappa Sigma grad,
    eps^2 Sigma), Sigma = diag(move_sigma^2), in control units."""
    sg = np.broadcast_to(np.asarray(p.move_sigma), to.shape)
    mean = frm - 0.5 * eps * eps * kappa * sg * sg * g_frm
    return stats.norm.logpdf(to, loc=mean, scale=eps * sg).reshape(to.shape[0], -1).sum(axis=1)


@pytest.mark.parametrize("kind", [1, 2])
def test_accept_ratio_is_the_metropolis_hastings_ratio(kind):
    p = tiny_problem(N=2, S_=3)
    rng = np.random.default_rng(3)
    L = 64
    sg = np.asarray(p.move_sigma)
    u = rng.standard_normal((L, p.N, p.S, 3)) * sg * 3
    up = u + rng.standard_normal(u.shape) * sg
    g = rng.standard_normal(u.shape) / sg
    gp = rng.standard_normal(u.shape) / sg
    cb = rng.exponential(1.0, (p.N, L))
    cbp = rng.exponential(1.0, (p.N, L))
    kappa, eps = 7.0, 0.8
    inbox = np.ones(L, np.uint8)
    _, _, la = O.mh_accept(p, u, up, cb, cbp, g, gp, inbox, 0, kappa, eps, kind)
    ref = -kappa * (cbp.sum(axis=0) - cb.sum(axis=0))
    if kind == 2:
        ref += langevin_logq(p, u, up, gp, kappa, eps) - langevin_logq(p, up, u, g, kappa, eps)
    assert np.allclose(la, ref, rtol=1e-10, atol=1e-10)
    # the reverse move has the opposite log ratio
    _, _, la_r = O.mh_accept(p, up, u, cbp, cb, gp, g, inbox, 0, kappa, eps, kind)
    assert np.allclose(la_r, -la, rtol=1e-10, atol=1e-10)


def test_accept_rules_for_box_and_infinite_costs():
    p = tiny_problem(N=1, S_=1)
    L = 4
    u = np.zeros((L, 1, 1, 3))
    up = u + 0.01
    cb = np.array([[1.0, np.inf, 1.0, 1.0]])
    cbp = np.array([[np.inf, 0.5, 0.5, 0.5]])
    inbox = np.array([1, 1, 0, 1], np.uint8)
    out, acc, la = O.mh_accept(p, u, up, cb, cbp, None, None, inbox, 0, 3.0, 1.0, 1)
    assert list(acc[:3]) == [False, True, False]
    assert la[0] == -np.inf and la[1] == np.inf and la[2] == -np.inf
    assert acc[3]               # lower cost: log alpha > 0 > ln U
    assert np.array_equal(out[acc], up[acc]) and np.array_equal(out[~acc], u[~acc])


def test_proposal_moments():
    p = tiny_problem(N=2, S_=4)
    L = 20000
    sg = np.asarray(p.move_sigma)
    u = np.zeros((L, p.N, p.S, 3))
    g = np.ones_like(u) / sg            # grad_z = 1 in every coordinate
    kappa, eps = 2.0, 0.5
    up, inbox = O.mh_propose(p, u, None, 3, kappa, eps, 1)
    z = (up / sg).reshape(L, -1)
    assert inbox.all()
    assert abs(z.mean()) < 4 * eps / math.sqrt(z.size)
    assert abs(z.std() / eps - 1.0) < 0.01
    assert stats.kstest(z[:, 5] / eps, "norm").pvalue > 1e-3
    # independent coordinates and particles
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.03
    up2, _ = O.mh_propose(p, u, g, 3, kappa, eps, 2)
    drift = ((up2 - up) / sg).reshape(L, -1)    # same normals, drift -(eps^2/2) kappa
    assert np.allclose(drift, -0.5 * eps * eps * kappa, atol=1e-12)
    # the move of iteration J differs from iteration J+1
    up3, _ = O.mh_propose(p, u, None, 4, kappa, eps, 1)
    assert not np.allclose(up3, up)


def _gaussian_chain(kind, eps, steps, L, correct=True, seed=0):
    """Chain on the target exp(-C), C = sum (u / s)^2 / 2, started at the target."""
    p = tiny_problem(N=1, S_=1)
    sg = np.asarray(p.move_sigma)
    s = 2.0 * sg
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((L, 1, 1, 3)) * s
    ones = np.ones((1, L))

    def cost(x):
        return 0.5 * ((x / s) ** 2).reshape(L, -1).sum(axis=1)

    for t in range(steps):
        g = u / (s * s)
        up, inbox = O.mh_propose(p, u, g, 100 + t, 1.0, eps, kind)
        gp = up / (s * s)
        if correct:
            u, _, _ = O.mh_accept(p, u, up, cost(u) * ones, cost(up) * ones, g, gp, inbox,
                                  100 + t, 1.0, eps, kind)
        else:
            u = up                                   # unadjusted Langevin
    return (u / s).reshape(L, -1)


@pytest.mark.parametrize("kind", [1, 2])
def test_gaussian_target_is_invariant(kind):
    z = _gaussian_chain(kind, eps=1.2, steps=8, L=40000)
    assert abs(z.mean()) < 0.03
    assert abs(z.var() - 1.0) < 0.03


def test_unadjusted_langevin_is_detectably_biased():
    """The invariance test above has the power to see a missing correction: the
    unadjusted chain inflates the variance by about 1 / (1 - eps^2 / 16)."""
    z = _gaussian_chain(2, eps=1.2, steps=8, L=40000, correct=False)
    assert z.var() > 1.06


def test_small_steps_are_almost_always_accepted():
    p = S.shrink(S.config4(), M=2, H=20, L=32)
    p = p.copy(aircraft=p.aircraft[:4], N=4)
    W = O.wind_field(p)
    rng = np.random.default_rng(2)
    u = S.mild_controls(p, 32, rng).astype(np.float64)
    J, kappa = 1, float(O.kappa(1))

    def soft_and_grad(x):
        r = O.rollout(p, x, J, W=W)
        g = np.stack([O.rollout_grad(p, x[l], W, l=l, J=J)[1] for l in range(x.shape[0])])
        return r["cbar_soft"], g

    cb, g = soft_and_grad(u)
    feas = np.isfinite(cb).all(axis=0)
    assert feas.sum() >= 16
    rates = []
    for eps in (1e-3, 0.3):
        up, inbox = O.mh_propose(p, u, g, J, kappa, eps, 2)
        cbp, gp = soft_and_grad(up)
        _, acc, la = O.mh_accept(p, u, up, cb, cbp, g, gp, inbox, J, kappa, eps, 2)
        rates.append(acc[feas].mean())
        if eps == 1e-3:
            assert np.abs(la[feas & np.isfinite(la)]).max() < 1e-2
    assert rates[0] == 1.0 and rates[1] < rates[0]
