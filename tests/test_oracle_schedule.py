"""Pins of the oracle's sample mode 1, the inner loop of Algorithm 1: iteration
J draws SampleSchedule(J) = floor(3 + 5 exp(0.05 J)) disturbance realisations
(Sec. 5.1), at most M, and the weight of an aircraft is the product of its
objective J_T over those draws (Sec. 3.6).

The product is formed here directly from the per-sample objectives
exp(-c_m) and compared with exp(-exponent * cbar), the form the solve uses;
the schedule against hand-evaluated values; the solve's per-iteration costs
against rollouts of exactly the first M_J samples."""
import math

import numpy as np
import pytest

import oracle as O
import scenarios as S


def small(**kw):
    p = S.shrink(S.config1(), L=48, M=12, H=16, J_max=12)
    return p.copy(**kw)


def test_schedule_values_and_cap():
    p = small(sample_mode=1)
    # floor(3 + 5 e^{0.05 J}) by hand: J = 0 -> 8, J = 4 -> 9.107, J = 7 -> 10.095, J = 11 -> 11.67
    want = [8, 8, 8, 8, 9, 9, 9, 10, 10, 10, 11, 11]
    assert [O.samples(p, J) for J in range(12)] == want
    assert [O.exponent(p, J) for J in range(12)] == want
    capped = p.copy(M=9)
    assert [O.samples(capped, J) for J in range(12)] == [min(w, 9) for w in want]
    assert [O.exponent(capped, J) for J in range(12)] == [min(w, 9) for w in want]
    # sample mode 0: all M samples, annealing exponent kappa_J
    p0 = small()
    assert all(O.samples(p0, J) == p0.M for J in range(12))
    assert [O.exponent(p0, J) for J in range(12)] == want
    # far along the schedule: J = 40 -> 3 + 5 e^2 = 39.9
    big = p.copy(M=64)
    assert O.samples(big, 40) == 39 and O.samples(big, 100) == 64


def test_weight_is_the_product_of_objectives_over_the_draws():
    p = small(sample_mode=1)
    rng = np.random.default_rng(3)
    u = S.mild_controls(p, p.L, rng).astype(np.float64)
    W = O.wind_field(p)
    for J in (0, 5, 11):
        Mj = O.samples(p, J)
        r = O.rollout(p.copy(M=Mj), u, J, W=W[:Mj])
        c = r["cost"]                                  # [L][Mj][N] = -ln J_T per draw
        fin = np.isfinite(c).all(axis=1)               # [L][N]
        prod = np.prod(np.exp(-c), axis=1)             # product of J_T over the draws
        lw = -O.exponent(p, J) * r["cbar"].T           # log-weight of the solve
        assert fin.sum() > 0.5 * fin.size
        assert np.allclose(np.exp(lw[fin]), prod[fin], rtol=1e-12, atol=0)
        # an infeasible draw makes the product zero: cbar is +inf there
        assert np.all(np.isinf(r["cbar"].T[~fin]))


def test_iteration_uses_the_first_samples_of_the_field():
    p = small(sample_mode=1)
    rng = np.random.default_rng(4)
    u = S.mild_controls(p, 20, rng).astype(np.float64)
    W = O.wind_field(p)
    full = O.rollout(p, u, 7, W=W)
    Mj = O.samples(p, 7)
    part = O.rollout(p.copy(M=Mj), u, 7, W=W[:Mj])
    assert np.array_equal(part["cost"], full["cost"][:, :Mj])
    with np.errstate(invalid="ignore"):
        want = np.where(np.isfinite(full["cost"][:, :Mj]).all(axis=1),
                        full["cost"][:, :Mj].mean(axis=1), np.inf).T
    fin = np.isfinite(want)
    assert np.allclose(part["cbar"][fin], want[fin], rtol=1e-13)


def test_solve_follows_the_schedule():
    """Each iteration of the solve scores its particles on the first M_J
    samples, and the weights of the next resampling use the exponent M_J."""
    p = small(sample_mode=1, L=32, J_max=6)
    W = O.wind_field(p)
    res = O.smc_solve(p, W=W, history=True)
    for h in res["history"]:
        J = h["J"]
        Mj = O.samples(p, J)
        r = O.rollout(p, h["u"], J, W=W)
        c = r["cost"][:, :Mj]
        with np.errstate(invalid="ignore"):
            want = np.where(np.isfinite(c).all(axis=1), c.mean(axis=1), np.inf).T
        fin = np.isfinite(want)
        assert fin.mean() > 0.25
        assert np.array_equal(np.isfinite(h["cbar"]), fin)
        assert np.allclose(h["cbar"][fin], want[fin], rtol=1e-12)
    # the next particles are the resampled (exponent M_J) and perturbed ones
    h0, h1 = res["history"][0], res["history"][1]
    wt, _, _ = O.lse(h0["cbar"], O.samples(p, 0))
    anc, _ = O.resample(wt, [O.resample_uniform(p, i, 0) for i in range(p.N)])
    assert np.array_equal(O.move(p, h0["u"], anc, 0), h1["u"])


def test_mode_0_solve_is_unchanged_by_the_schedule_functions():
    p = small(L=32, J_max=4)
    W = O.wind_field(p)
    res = O.smc_solve(p, W=W, history=True)
    h = res["history"][2]
    r = O.rollout(p, h["u"], 2, W=W)
    assert np.array_equal(np.isfinite(h["cbar"]), np.isfinite(r["cbar"]))
    fin = np.isfinite(r["cbar"])
    assert np.array_equal(h["cbar"][fin], r["cbar"][fin])
    assert math.isclose(O.exponent(p, 2), O.kappa(2))
