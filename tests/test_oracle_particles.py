"""Pins of the oracle's varying particle count (the speed-up the paper
proposes: many particles early, fewer once the search narrows): systematic
resampling of L_out ancestors from L_in weighted particles, and the solve's
particle schedule.

The ancestors are checked against exact rational arithmetic on tiny inputs,
the floor/ceil count property of systematic resampling, unbiasedness over the
uniform, the textbook FP64 scheme, and the degenerate rule; the solve against
its stages applied by hand."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import scenarios as S


@pytest.fixture
def rng():
    return np.random.default_rng(77)


def _brute(w, r, Lout):
    """a_l = #{j : S_j <= t_l}, t_l = floor((l 2^32 + r) Q / (Lout 2^32)), exact."""
    q = [0 if not (x > 0) else (1 << 40 if x >= 1 else int(Fraction(x) * (1 << 40))) for x in w]
    S_ = np.cumsum(np.array(q, dtype=object))
    Q = int(S_[-1])
    out = []
    for l in range(Lout):
        t = ((l << 32) + r) * Q // (Lout << 32)
        out.append(sum(1 for s in S_ if s <= t))
    return out


@pytest.mark.parametrize("Lin,Lout", [(1, 3), (3, 1), (5, 2), (2, 7), (8, 5), (6, 6)])
def test_brute_force_tiny(Lin, Lout, rng):
    for _ in range(40):
        w = rng.random(Lin) * (rng.random(Lin) > 0.3)
        w[rng.integers(Lin)] = 1.0
        r = int(rng.integers(0, 2 ** 32))
        anc, nd = O.resample(w[None, :], [r], Lout)
        assert nd == 0 and anc.shape == (1, Lout)
        assert list(anc[0]) == _brute(list(w), r, Lout)


@pytest.mark.parametrize("Lin,Lout", [(2000, 700), (700, 2000), (4096, 4095)])
def test_counts_are_floor_or_ceil_of_expectation(Lin, Lout, rng):
    w = S.random_wtilde(3, Lin, rng)
    r = [int(x) for x in rng.integers(0, 2 ** 32, 3)]
    anc, _ = O.resample(w, r, Lout)
    for s in range(3):
        q = np.floor(w[s] * 2.0 ** 40)
        expect = Lout * q / q.sum()
        cnt = np.bincount(anc[s], minlength=Lin)
        assert cnt.sum() == Lout and cnt.size == Lin
        assert (cnt >= np.floor(expect) - 1e-9).all() and (cnt <= np.ceil(expect) + 1e-9).all()
        assert (cnt[w[s] == 0] == 0).all()
        assert (np.diff(anc[s]) >= 0).all()


def test_unbiased_over_the_uniform(rng):
    w = np.array([0.1, 0.0, 0.55, 1.0, 0.02, 0.3])
    q = np.floor(w * 2.0 ** 40)
    for Lout in (4, 11):
        acc = np.zeros(w.size)
        n = 3000
        for r in rng.integers(0, 2 ** 32, n):
            anc, _ = O.resample(w[None, :], [int(r)], Lout)
            acc += np.bincount(anc[0], minlength=w.size)
        assert np.allclose(acc / n, Lout * q / q.sum(), atol=0.03)


def test_matches_textbook_systematic_scheme(rng):
    Lin, Lout = 5000, 1234
    w = S.random_wtilde(1, Lin, rng)[0]
    r = int(rng.integers(0, 2 ** 32))
    anc, _ = O.resample(w[None, :], [r], Lout)
    cdf = np.cumsum(w) / w.sum()
    u = (np.arange(Lout) + r / 2 ** 32) / Lout
    ref = np.searchsorted(cdf, u, side="right")
    assert (anc[0] != ref).sum() <= 2


def test_same_count_is_the_plain_resampler(rng):
    w = S.random_wtilde(2, 999, rng)
    r = [5, 2 ** 32 - 1]
    a1, n1 = O.resample(w, r)
    a2, n2 = O.resample(w, r, 999)
    assert np.array_equal(a1, a2) and n1 == n2


def test_degenerate_segment_spreads_evenly():
    w = np.zeros((2, 10))
    w[1, 3] = 0.5
    anc, nd = O.resample(w, [1, 2], 4)
    assert nd == 1
    assert list(anc[0]) == [0, 2, 5, 7]           # floor(l * 10 / 4)
    assert (anc[1] == 3).all()
    anc, _ = O.resample(np.zeros((1, 3)), [9], 7)
    assert list(anc[0]) == [0, 0, 0, 1, 1, 2, 2]    # floor(l * 3 / 7)


def test_move_makes_one_child_per_ancestor_entry(rng):
    p = S.shrink(S.config1(), L=10).copy(move_sigma=(0.0, 0.0, 0.0))
    u = S.mild_controls(p, 10, rng).astype(np.float64)
    anc = rng.integers(0, 10, (p.N, 4)).astype(np.int32)
    out = O.move(p, u, anc, 3)
    assert out.shape == (4, p.N, p.S, 3)
    for i in range(p.N):
        assert np.array_equal(out[:, i], u[anc[i], i])


def test_schedule_helper():
    s = S.particle_schedule(65536, 30, 0.125)
    assert s[0] == 65536 and s[-1] == 8192 and len(s) == 30
    assert all(a >= b for a, b in zip(s, s[1:])) and all(x % 32 == 0 for x in s)


def test_solve_follows_the_particle_schedule():
    p = S.shrink(S.config1(), L=96, M=4, H=16, J_max=5)
    p = p.copy(L_sched=(96, 70, 64, 33, 40))
    W = O.wind_field(p)
    res = O.smc_solve(p, W=W, history=True)
    hist = res["history"]
    assert [h["u"].shape[0] for h in hist] == list(p.L_sched)
    assert [h["cbar"].shape[1] for h in hist] == list(p.L_sched)
    assert np.array_equal(hist[0]["u"], O.init_controls(p, 96))
    for J in range(p.J_max - 1):
        h = hist[J]
        wt, _, _ = O.lse(h["cbar"], O.kappa(J))
        anc, _ = O.resample(wt, [O.resample_uniform(p, i, J) for i in range(p.N)], p.L_sched[J + 1])
        assert np.array_equal(O.move(p, h["u"], anc, J), hist[J + 1]["u"])
    assert res["u"].shape[0] == 40 and 0 <= res["best"] < 40
