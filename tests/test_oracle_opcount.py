"""The operation-counting build of the oracle (oracle/opcount.cpp): the same
arithmetic as the oracle, so the same costs bit for bit, and a count that is
additive over particles and constant per step of a steady
flight.  The count per live aircraft-step-sample is the algorithmic work the
benchmark's roofline uses."""
import numpy as np

import oracle as O
import scenarios as S
from conftest import make_problem, one_aircraft, zero_wind


def _case():
    p = S.shrink(S.config3(), L=6, M=3, H=30)
    rng = np.random.default_rng(5)
    u = S.mild_controls(p, p.L, rng).astype(np.float64)
    return p, u, O.wind_field(p)


def test_counting_build_computes_the_oracle_costs():
    p, u, W = _case()
    ref = O.rollout(p, u, 1, W=W)
    ops, live = O.rollout_opcount(p, u, 1, W)
    assert live == ref["live"] and ops > 0
    # the counting library's own outputs (run again through the plain entry point)
    import ctypes as C
    lib = O._opcount_lib()
    ch = np.empty((p.L, p.M, p.N))
    cs = np.empty((p.L, p.M, p.N))
    mg = np.empty((p.L, p.M, p.N))
    sm = np.empty((p.L, p.M))
    lv = C.c_int64(0)
    m = O._Marshalled(p)
    pidx = np.arange(p.L, dtype=np.int64)
    Wc = np.ascontiguousarray(W)
    lib.orc_rollout(m.ps, m.ac, O._ptr(Wc, C.c_double), 0, p.M, O._ptr(u, C.c_double),
                    O._ptr(pidx, C.c_int64), p.L, 1, 1, O._ptr(ch, C.c_double), O._ptr(cs, C.c_double),
                    O._ptr(mg, C.c_double), O._ptr(sm, C.c_double), C.byref(lv))
    assert np.array_equal(ch, ref["cost"]) and np.array_equal(cs, ref["cost_soft"])
    assert np.array_equal(mg.min(axis=1).T, ref["margin"])


def test_count_is_additive_over_particles():
    p, u, W = _case()
    ops, live = O.rollout_opcount(p, u, 1, W)
    a = O.rollout_opcount(p, u[:2], 1, W, pidx=np.arange(2))
    b = O.rollout_opcount(p, u[2:], 1, W, pidx=np.arange(2, p.L))
    assert (a[0] + b[0], a[1] + b[1]) == (ops, live)


def test_steady_flight_costs_the_same_every_step():
    ac = one_aircraft(kind=1, x=-20000.0, y=5000.0, z=3000.0, v=150.0, chi=0.3, CD2=0.03)
    counts = []
    for H in (4, 5, 6, 7):
        p = make_problem([ac], H=H)
        u = np.zeros((1, 1, p.S, 3))
        counts.append(O.rollout_opcount(p, u, 0, zero_wind(p), soft=False))
    steps = np.diff([c[0] for c in counts])
    assert [c[1] for c in counts] == [4, 5, 6, 7]
    assert (steps == steps[0]).all() and 100 < steps[0] < 400, steps


def test_hard_only_counts_less_than_hard_and_soft():
    p, u, W = _case()
    hard = O.rollout_opcount(p, u, 1, W, soft=False)
    both = O.rollout_opcount(p, u, 1, W, soft=True)
    assert hard[1] == both[1] and hard[0] < both[0]
