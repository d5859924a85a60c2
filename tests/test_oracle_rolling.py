"""Pins of the oracle's rolling window (the paper's rolling-window section):
aircraft enter the problem at preset MPC steps and leave it once finished; a
late entrant is optimised from its entry step over its remaining steps.

Checked against problems that state the same situation without the window:
an aircraft that is out of the problem leaves the others' costs exactly as if
it were absent; a late entrant flying straight without disturbances scores
what the same flight scores over a horizon of its active steps; separation
with an aircraft that has not entered is not checked; the plant keeps waiting
and finished aircraft in place and retires arrivals in the landing sector."""
import math

import numpy as np
import pytest

import oracle as O
import scenarios as S
from conftest import controls, make_problem, one_aircraft, zero_wind


def traffic(n=5, H=20, **kw):
    p = S.shrink(S.config4(), L=40, M=3, H=H)
    p = p.copy(aircraft=p.aircraft[:n].copy(), N=n, **kw)
    return p


def costs(p, u, J=1):
    r = O.rollout(p, u, J, W=O.wind_field(p))
    return r


def test_window_with_everyone_present_changes_nothing():
    p = traffic()
    u = S.mild_controls(p, p.L, np.random.default_rng(1)).astype(np.float64)
    a = costs(p, u)
    b = costs(p.copy(rolling=1, mpc_step=2), u)          # t_enter = 0 <= mpc_step
    c = costs(p.copy(mpc_step=2), u)
    for k in ("cbar", "cbar_soft"):
        assert np.array_equal(b[k], c[k])
    assert b["live"] == c["live"]
    assert not np.array_equal(a["cbar"], b["cbar"])        # mpc_step keys the streams


@pytest.mark.parametrize("how", ["not_entered", "finished"])
def test_absent_aircraft_costs_zero_and_leaves_the_others_alone(how):
    p = traffic(n=5)
    rng = np.random.default_rng(2)
    u = S.mild_controls(p, p.L, rng).astype(np.float64)
    ac = p.aircraft.copy()
    if how == "not_entered":
        ac["t_enter"][4] = p.mpc_step + p.H              # enters after this horizon
        q = p.copy(rolling=1, aircraft=ac)
    else:
        q = p.copy(rolling=1, finished=1 << 4)
    r = costs(q, u)
    assert (r["cbar"][4] == 0).all() and (r["cbar_soft"][4] == 0).all()
    # the same problem without aircraft 4 (the last: the others keep their indices)
    p4 = p.copy(N=4, aircraft=p.aircraft[:4].copy())
    r4 = costs(p4, u[:, :4])
    for k in ("cbar", "cbar_soft"):
        fin = np.isfinite(r4[k])
        assert np.array_equal(np.isfinite(r[k][:4]), fin)
        assert np.array_equal(r[k][:4][fin], r4[k][fin])
    assert r["live"] == r4["live"]


@pytest.mark.parametrize("kind", [0, 1])
def test_late_entrant_scores_its_active_steps(kind):
    """No wind, no turbulence, zero controls: the entrant waits k_in steps,
    then flies straight; its cost equals the cost of the same flight over a
    horizon of H - k_in steps (per-step means, fuel bound and departure
    altitude bounds over the active steps)."""
    H, kin = 16, 6
    ac = one_aircraft(kind=kind, x=-20000.0, y=15000.0, z=3000.0, v=150.0, chi=0.3,
                      CD2=0.03, theta_F=1.0)
    ac["t_enter"] = 7 + kin
    p = make_problem([ac], H=H, rolling=1, mpc_step=7, wind_sigma=0.0)
    traj, ch, cs = O.trajectory(p, controls(p)[0], zero_wind(p)[0], l=0, m=0, J=0)
    assert np.array_equal(traj[kin, 0, :6], traj[0, 0, :6])      # waited at its entry state
    assert not np.array_equal(traj[kin + 1, 0, :6], traj[kin, 0, :6])
    q = make_problem([ac], H=H - kin, wind_sigma=0.0)
    traj_q, ch_q, _ = O.trajectory(q, controls(q)[0], zero_wind(q)[0], l=0, m=0, J=0)
    assert np.allclose(traj[-1, 0, :7], traj_q[-1, 0, :7], rtol=1e-12, atol=1e-9)
    assert ch[0] == pytest.approx(ch_q[0], rel=1e-12)
    # the waiting steps count as neither flown nor scored
    full = make_problem([ac], H=H, wind_sigma=0.0)
    _, ch_full, _ = O.trajectory(full, controls(full)[0], zero_wind(full)[0], l=0, m=0, J=0)
    assert abs(ch_full[0] - ch[0]) > 1e-6


def test_no_separation_with_an_aircraft_that_has_not_entered():
    # B starts on top of A's waiting position and flies away at 150 m/s;
    # A enters after B is beyond the horizontal separation
    A = one_aircraft(kind=1, x=0.0, y=0.0, z=3000.0, v=150.0, chi=0.0, CD2=0.0)
    B = one_aircraft(kind=1, x=0.0, y=0.0, z=3100.0, v=150.0, chi=math.pi, CD2=0.0)
    p = make_problem([A, B], H=10, wind_sigma=0.0)
    need = int(math.ceil(p.sep_h / (150.0 * p.dt))) + 1
    A2 = A.copy()
    A2["t_enter"] = need
    q = make_problem([A2, B], H=10, rolling=1, wind_sigma=0.0)
    _, ch_p, _ = O.trajectory(p, controls(p)[0], zero_wind(p)[0], l=0, m=0, J=0)
    _, ch_q, _ = O.trajectory(q, controls(q)[0], zero_wind(q)[0], l=0, m=0, J=0)
    assert np.isinf(ch_p).all()                  # both present from the start: violation
    assert np.isfinite(ch_q).all()               # A waits: no conflict


def test_plant_keeps_absent_aircraft_and_moves_the_rest():
    p = traffic(n=4, rolling=1, mpc_step=5)
    ac = p.aircraft.copy()
    ac["t_enter"][1] = 6                         # enters next step
    p = p.copy(aircraft=ac, finished=1 << 2)
    x0 = np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])
    u = S.mild_controls(p, 1, np.random.default_rng(3))[0, :, 0, :].astype(np.float64)
    W0 = O.wind_field(p)[0, 0]
    x1 = O.plant_step(p, x0, W0, u)
    ref = O.plant_step(p.copy(rolling=0, finished=0), x0, W0, u)
    for i in range(4):
        if i in (1, 2):
            assert np.array_equal(x1[i], x0[i])
        else:
            assert np.array_equal(x1[i], ref[i])


def test_plant_retires_arrivals_in_the_landing_sector():
    land = one_aircraft(kind=0, x=5000.0, y=0.0, z=300.0, v=85.0, chi=math.pi)
    far = one_aircraft(kind=0, x=30000.0, y=0.0, z=3000.0, v=150.0, chi=math.pi)
    dep = one_aircraft(kind=1, x=5000.0, y=0.0, z=300.0, v=85.0, chi=math.pi)
    wait = land.copy()
    wait["t_enter"] = 9
    p = make_problem([land, far, dep, wait], H=5, rolling=1, mpc_step=3)
    x = np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])
    assert O.plant_finished(p, x) == 0b0001      # departures and waiting aircraft never finish
    assert O.plant_finished(p.copy(finished=0b0100), x) == 0b0101
    assert O.plant_finished(p.copy(rolling=0), x) == 0
    x2 = x.copy()
    x2[0, 3] = 95.0                              # too fast for the sector
    assert O.plant_finished(p, x2) == 0


def test_gradient_refuses_the_rolling_window():
    p = traffic(n=2, rolling=1)
    u = S.mild_controls(p, 1, np.random.default_rng(4))[0].astype(np.float64)
    c, _ = O.rollout_grad(p, u, O.wind_field(p), l=0, J=0)
    assert math.isnan(c)
