"""Pins of the oracle's weighting, resampling, perturbation and selection
(Sec. 3.6-3.8, Algorithm 1, schedule of Sec. 5.1)."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle as O
import scenarios as S


# --------------------------------------------------------------- schedule

def test_sample_schedule_values():
    # floor(3 + 5 e^{0.05 J}) evaluated by hand
    expect = {0: 8, 5: 9, 10: 11, 20: 16, 29: 24, 99: 708}
    for J, k in expect.items():
        assert O.kappa(J) == k
    assert sum(O.kappa(J) for J in range(100)) == 14625
    ks = [O.kappa(J) for J in range(200)]
    assert all(b >= a for a, b in zip(ks, ks[1:]))              # monotonically increasing


# -------------------------------------------------------------------- LSE

def test_lse_against_library_logsumexp(rng):
    c = S.random_cbar(5, 3001, rng).astype(np.float64)
    for kap in (1.0, 8.0, 24.0, 708.0):
        wt, lm, ws = O.lse(c, kap)
        for s in range(5):
            fin = np.isfinite(c[s])
            ref = logsumexp(-kap * c[s][fin])
            assert lm[s] + math.log(ws[s]) == pytest.approx(ref, rel=1e-13, abs=1e-13)
            assert wt[s].max() == 1.0
            assert (wt[s][~fin] == 0).all()
            assert wt[s].sum() == pytest.approx(ws[s], rel=1e-14)


def test_lse_shift_invariance_and_normalisation(rng):
    c = S.random_cbar(3, 500, rng, frac_inf=0.0).astype(np.float64)
    wt1, _, ws1 = O.lse(c, 8.0)
    wt2, _, ws2 = O.lse(c + 3.0, 8.0)                  # exp(-8*3) cancels in the ratio
    assert np.allclose(wt1, wt2, rtol=1e-12)
    assert np.allclose((wt1 / ws1[:, None]).sum(1), 1.0, rtol=1e-14)


def test_lse_degenerate_segment():
    c = np.full((2, 7), np.inf)
    c[1, 3] = 0.5
    wt, lm, ws = O.lse(c, 10.0)
    assert lm[0] == -np.inf and ws[0] == 0 and (wt[0] == 0).all()
    assert lm[1] == -5.0 and wt[1, 3] == 1.0 and ws[1] == 1.0


# ------------------------------------------------------------- resampling

def _counts(anc, L):
    return np.bincount(anc, minlength=L)


def _brute_ancestors(w, r):
    """a_l = #{j : S_j <= t_l} with exact rational arithmetic (an equivalent
    form of min{j : S_j > t_l} for a non-decreasing S)."""
    L = len(w)
    q = [0 if not (x > 0) else (1 << 40 if x >= 1 else int(Fraction(x) * (1 << 40))) for x in w]
    Ssum = np.cumsum(np.array(q, dtype=object))
    Q = int(Ssum[-1])
    out = []
    for l in range(L):
        t = Fraction((l << 32) + r) * Q / (L << 32)
        t = t.numerator // t.denominator
        out.append(sum(1 for s in Ssum if s <= t))
    return out


@pytest.mark.parametrize("L", [1, 2, 3, 5, 8])
def test_resample_brute_force_tiny(L, rng):
    for trial in range(40):
        w = rng.random(L) * (rng.random(L) > 0.3)
        w[rng.integers(L)] = 1.0
        r = int(rng.integers(0, 2 ** 32))
        anc, nd = O.resample(w[None, :], [r])
        assert nd == 0
        assert list(anc[0]) == _brute_ancestors(list(w), r)


def test_resample_equal_weights_is_identity(rng):
    for L in (1, 7, 1000, 4096):
        for r in (0, 1, 2 ** 31, 2 ** 32 - 1, int(rng.integers(0, 2 ** 32))):
            anc, _ = O.resample(np.full((1, L), 0.37), [r])
            assert (anc[0] == np.arange(L)).all()


def test_resample_counts_are_floor_or_ceil_of_expectation(rng):
    L = 2000
    w = S.random_wtilde(4, L, rng)
    r = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
    anc, _ = O.resample(w, r)
    for s in range(4):
        q = np.floor(w[s] * 2.0 ** 40)
        expect = L * q / q.sum()
        cnt = _counts(anc[s], L)
        assert cnt.sum() == L
        assert (cnt >= np.floor(expect) - 1e-9).all() and (cnt <= np.ceil(expect) + 1e-9).all()
        assert (cnt[w[s] == 0] == 0).all()                   # zero weight is never drawn
        assert (np.diff(anc[s]) >= 0).all()                  # systematic: ancestors sorted


def test_resample_is_unbiased_over_the_uniform(rng):
    L = 6
    w = np.array([0.1, 0.0, 0.55, 1.0, 0.02, 0.3])
    q = np.floor(w * 2.0 ** 40)
    acc = np.zeros(L)
    n = 4000
    for r in rng.integers(0, 2 ** 32, n):
        anc, _ = O.resample(w[None, :], [int(r)])
        acc += _counts(anc[0], L)
    assert np.allclose(acc / n, L * q / q.sum(), atol=0.03)


def test_resample_matches_textbook_systematic_scheme(rng):
    # the fixed-point CDF equals the usual FP64 systematic scheme except where a
    # threshold falls within rounding of a CDF step
    L = 5000
    w = S.random_wtilde(1, L, rng)[0]
    r = int(rng.integers(0, 2 ** 32))
    anc, _ = O.resample(w[None, :], [r])
    cdf = np.cumsum(w) / w.sum()
    u = (np.arange(L) + r / 2 ** 32) / L
    ref = np.searchsorted(cdf, u, side="right")
    assert (anc[0] != ref).sum() <= 2


def test_resample_all_zero_segment_is_identity():
    w = np.zeros((2, 9))
    w[1, 4] = 1.0
    anc, nd = O.resample(w, [123, 456])
    assert nd == 1
    assert (anc[0] == np.arange(9)).all() and (anc[1] == 4).all()


def test_resample_uniform_stream():
    p = S.config1()
    r = O.resample_uniform(p, 1, 3)
    assert r == O.draw(p, 0, 1, 0, 2, 3)[0]


# ------------------------------------------------------------ perturbation

def test_move_without_noise_copies_ancestors(rng):
    p = S.config1().copy(move_sigma=(0.0, 0.0, 0.0))
    L = 300
    u = S.random_controls(p, L, rng).astype(np.float64)
    anc = S.random_ancestors(p.N, L, rng)
    out = O.move(p, u, anc, 2)
    for i in range(p.N):
        assert np.array_equal(out[:, i], u[anc[i], i])


def test_move_noise_is_gaussian_with_sigma(rng):
    p = S.config1().copy(ctrl_lo=(-1e3, -1e3, -1e3), ctrl_hi=(1e3, 1e3, 1e3))
    L = 4000
    u = np.zeros((L, p.N, p.S, 3))
    anc = np.tile(np.arange(L, dtype=np.int32), (p.N, 1))
    out = O.move(p, u, anc, 5)
    for c in range(3):
        z = out[..., c].ravel() / p.move_sigma[c]
        assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03
    # iterations draw fresh noise
    out2 = O.move(p, u, anc, 6)
    assert abs(np.corrcoef(out.ravel(), out2.ravel())[0, 1]) < 0.03


def test_move_clips_to_box(rng):
    p = S.config1().copy(move_sigma=(10.0, 1e3, 1e3))
    L = 200
    u = S.random_controls(p, L, rng).astype(np.float64)
    anc = S.random_ancestors(p.N, L, rng)
    out = O.move(p, u, anc, 0)
    lo, hi = np.array(p.ctrl_lo), np.array(p.ctrl_hi)
    assert (out >= lo).all() and (out <= hi).all()
    assert np.isclose(out, lo).any() and np.isclose(out, hi).any()


def test_init_controls_uniform_in_box():
    p = S.config1()
    u = O.init_controls(p, 5000)
    lo, hi = np.array(p.ctrl_lo), np.array(p.ctrl_hi)
    assert (u >= lo).all() and (u <= hi).all()
    z = (u - lo) / (hi - lo)
    assert abs(z.mean() - 0.5) < 0.01 and abs(z.var() - 1 / 12) < 0.005


# -------------------------------------------------------------- selection

def test_select_brute_force(rng):
    N, L = 3, 1000
    c = S.random_cbar(N, L, rng, frac_inf=0.3).astype(np.float64)
    best, bsum, ninf = O.select(c)
    ninf_l = (~np.isfinite(c)).sum(0)
    sums = np.where(np.isfinite(c), c, 0).sum(0)
    order = sorted(range(L), key=lambda l: (ninf_l[l], sums[l], l))
    assert best == order[0] and ninf == ninf_l[best]
    if ninf == 0:
        assert bsum == pytest.approx(sums[best], rel=1e-15)


def test_select_ties_take_lowest_index_and_all_infeasible():
    c = np.array([[1.0, 0.5, 0.5, 2.0], [1.0, 1.0, 1.0, 0.0]])
    assert O.select(c)[0] == 1
    c2 = np.full((2, 4), np.inf)
    c2[0, 2] = 3.0
    best, bsum, ninf = O.select(c2)
    assert best == 2 and ninf == 1 and bsum == np.inf


# ------------------------------------------------------------------ chain

def test_smc_solve_config1_improves_and_selects_feasible():
    p = S.config1()
    W = O.wind_field(p)
    res = O.smc_solve(p, W=W, nthreads=4, history=True)
    assert res["n_inf"] == 0 and np.isfinite(res["best_sum"])
    first, last = res["history"][0]["cbar"], res["history"][-1]["cbar"]
    feas = lambda c: np.isfinite(c).all(0)                      # noqa: E731
    assert feas(last).mean() > feas(first).mean()              # the population becomes feasible
    f0 = first[:, feas(first)].sum(0)
    f1 = last[:, feas(last)].sum(0)
    assert np.median(f1) < np.median(f0)                       # and cheaper
    # the selected controls reproduce the selected cost
    r = O.rollout(p, res["u"][res["best"]][None], p.J_max - 1, pidx=[res["best"]], W=W)
    assert r["cbar"][:, 0].sum() == pytest.approx(res["best_sum"], rel=1e-12)
