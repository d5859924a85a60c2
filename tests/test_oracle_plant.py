"""Pins of the oracle's plant step (Sec. 2, Fig. 1: the true system flies the
chosen first-segment controls for one step dt; Eq. (hor) with the plant's
clamps |sin gamma| <= 0.999 and Tmin <= T <= Tmax).

Each check comes from something other than the oracle's own formula: the
reduced forms that Eq. (hor) takes under a coordinated turn (chi' = chi + dt w,
z' = z + dt hdot, v' = v + dt a while the thrust is not clamped), the fuel burn
of a clamped thrust (dt eta Tmax, eta = Cf1 (1 + v / Cf2), independent of the
drag), the ISA density table, a linear wind field that trilinear interpolation
reproduces exactly, and the turbulence pair of random stream 7 formed here from
the Philox block function and the Box-Muller transform written out.  Several
aircraft with different controls go through one call, so that a transposed
operand, a wrong sign of the heading rate, a wrong stream or a missing clamp
fails one of them."""
import math

import numpy as np
import pytest

import oracle as O
from conftest import make_problem, one_aircraft

G0 = 9.80665
DEG = math.pi / 180
GOLDEN = 0x9E3779B97F4A7C15


def states(p):
    return np.array([[a[k] for k in ("x", "y", "z", "v", "chi", "m")] for a in p.aircraft])


def zero_field(p):
    return np.zeros((p.n_grid, 2))


def eta(a, v):
    return a["Cf1"] * (1.0 + v / a["Cf2"])


def three_aircraft(**kw):
    acs = [one_aircraft(kind=1, x=-8000.0, y=3000.0, z=3000.0, v=150.0, chi=0.4, CD2=0.0),
           one_aircraft(kind=0, x=20000.0, y=-5000.0, z=4500.0, v=180.0, chi=2.9, CD2=0.03,
                        m=70000.0),
           one_aircraft(kind=1, x=1000.0, y=12000.0, z=1000.0, v=120.0, chi=-1.3, CD2=0.04,
                        m=52000.0)]
    return make_problem(acs, H=6, **kw)


def test_straight_level_step_and_fuel_against_the_isa_table():
    """w = hdot = a = 0, CD2 = 0, no wind: one step along the heading at constant
    altitude and speed, and the thrust equals the drag 1/2 rho v^2 S CD0 with
    rho from the ISA table (1000 m: 1.1117, 3000 m: 0.90925 kg/m^3)."""
    for z, rho_tab in ((1000.0, 1.1117), (3000.0, 0.90925)):
        ac = one_aircraft(kind=1, x=-5000.0, y=2000.0, z=z, v=150.0, chi=0.4, CD2=0.0)
        p = make_problem([ac], H=4)
        x0 = states(p)
        x1 = O.plant_step(p, x0, zero_field(p), np.zeros((1, 3)))[0]
        assert x1[0] == pytest.approx(-5000.0 + p.dt * 150.0 * math.cos(0.4), abs=1e-9)
        assert x1[1] == pytest.approx(2000.0 + p.dt * 150.0 * math.sin(0.4), abs=1e-9)
        assert x1[2] == z and x1[3] == pytest.approx(150.0, abs=1e-12)
        assert x1[4] == 0.4
        burn = ac["m"] - x1[5]
        D = burn / (p.dt * eta(ac, 150.0))
        assert D / (0.5 * 150.0 ** 2 * ac["S"] * ac["CD0"]) == pytest.approx(rho_tab, rel=5e-4)


def test_turn_climb_and_acceleration_take_their_reduced_forms():
    """Under the coordinated turn the heading changes by dt w (lift L = m g cos
    gamma / cos phi, chi' = chi + dt L sin phi / (m v)), the altitude by dt hdot
    (v sin gamma = hdot) and the speed by dt a while Tmin < T < Tmax; each
    aircraft flies its own row of controls, left and right turns alike."""
    p = three_aircraft()
    x0 = states(p)
    u0 = np.array([[1.2 * DEG, 8.0, 0.6],
                   [-0.9 * DEG, -3.0, 0.2],
                   [0.5 * DEG, 3.0, 0.9]])
    x1 = O.plant_step(p, x0, zero_field(p), u0)
    for i in range(3):
        assert x1[i, 4] - x0[i, 4] == pytest.approx(p.dt * u0[i, 0], abs=1e-12)
        assert x1[i, 2] - x0[i, 2] == pytest.approx(p.dt * u0[i, 1], abs=1e-9)
        assert x1[i, 3] - x0[i, 3] == pytest.approx(p.dt * u0[i, 2], abs=1e-9)
        # the position moves along the step-k heading with the horizontal speed v cos gamma
        cg = math.sqrt(1.0 - (u0[i, 1] / x0[i, 3]) ** 2)
        assert x1[i, 0] - x0[i, 0] == pytest.approx(p.dt * x0[i, 3] * cg * math.cos(x0[i, 4]), abs=1e-9)
        assert x1[i, 1] - x0[i, 1] == pytest.approx(p.dt * x0[i, 3] * cg * math.sin(x0[i, 4]), abs=1e-9)
    # a left turn (w > 0) raises the heading in the mathematical convention
    assert x1[0, 4] > x0[0, 4] and x1[1, 4] < x0[1, 4]


def test_thrust_held_at_tmax_and_tmin():
    """A hard acceleration asks for more than Tmax: the plant applies Tmax, so
    the burn is exactly dt eta(v) Tmax and the speed gains dt ((Tmax - D)/m -
    g sin gamma) with D from the ISA density.  A steep descent with braking asks
    for less than Tmin: the plant applies Tmin (burn dt eta Tmin; no burn at
    Tmin = 0)."""
    fast = one_aircraft(kind=1, z=3000.0, v=150.0, chi=0.0, CD2=0.0, Tmax=200e3)
    brake = one_aircraft(kind=1, x=9000.0, z=3000.0, v=150.0, chi=0.0, CD2=0.0, Tmin=0.0)
    idle = one_aircraft(kind=1, x=-9000.0, z=3000.0, v=150.0, chi=0.0, CD2=0.0, Tmin=15e3)
    p = make_problem([fast, brake, idle], H=4)
    x0 = states(p)
    u0 = np.array([[0.0, 0.0, 4.0],          # m a = 240 kN alone, above Tmax = 200 kN
                   [0.0, -20.0, -3.0],       # T_req = m (a + g sin gamma) + D < 0
                   [0.0, -20.0, -3.0]])
    x1 = O.plant_step(p, x0, zero_field(p), u0)
    m = x0[0, 5]
    assert m - x1[0, 5] == pytest.approx(p.dt * eta(fast, 150.0) * 200e3, rel=1e-10)
    D = 0.5 * 0.90925 * 150.0 ** 2 * fast["S"] * fast["CD0"]      # ISA table, 3000 m
    assert x1[0, 3] - 150.0 == pytest.approx(p.dt * (200e3 - D) / m, rel=2e-4)
    assert x1[0, 3] - 150.0 < p.dt * 4.0                           # short of the command
    assert x1[1, 5] == x0[1, 5]                                    # Tmin = 0: no burn
    sg = -20.0 / 150.0
    assert x1[1, 3] - 150.0 == pytest.approx(p.dt * (-D / m - G0 * sg), rel=2e-4)
    assert x1[1, 3] - 150.0 > p.dt * -3.0                          # gravity helps: above the command
    assert x0[2, 5] - x1[2, 5] == pytest.approx(p.dt * eta(idle, 150.0) * 15e3, rel=1e-10)
    assert x1[2, 3] - 150.0 == pytest.approx(p.dt * ((15e3 - D) / m - G0 * sg), rel=2e-4)


def test_climb_angle_held_below_ninety_degrees():
    """|hdot / v| above 0.999 is flown at sin gamma = +-0.999 exactly."""
    up = one_aircraft(kind=1, z=3000.0, v=100.0, CD2=0.0, Tmax=5e6)
    down = one_aircraft(kind=1, x=5000.0, z=6000.0, v=100.0, CD2=0.0, Tmax=5e6)
    p = make_problem([up, down], H=4)
    x0 = states(p)
    u0 = np.array([[0.0, 150.0, 0.0], [0.0, -250.0, 0.0]])
    x1 = O.plant_step(p, x0, zero_field(p), u0)
    assert x1[0, 2] - 3000.0 == pytest.approx(p.dt * 100.0 * 0.999, rel=1e-12)
    assert x1[1, 2] - 6000.0 == pytest.approx(-p.dt * 100.0 * 0.999, rel=1e-12)
    cg = math.sqrt(1.0 - 0.999 ** 2)
    assert x1[0, 0] == pytest.approx(p.dt * 100.0 * cg, rel=1e-12)
    # the speed equation sees g sin gamma at the held angle (thrust not clamped)
    assert x1[0, 3] - 100.0 == pytest.approx(0.0, abs=1e-9)


def test_wind_of_sample_zero_step_zero_at_the_pre_step_position():
    """A wind field linear in the coordinates is reproduced exactly by the
    trilinear interpolation: the displacement gains dt w(x, y, z) at the state
    before the step."""
    p = three_aircraft(turb_sigma=0.0)
    X, Y, Z = O.grid_nodes(p)
    XX, YY, ZZ = np.meshgrid(X, Y, Z, indexing="ij")
    wx = 3.0 + 4e-5 * XX - 2e-4 * ZZ + 1e-5 * YY
    wy = -2.0 + 6e-5 * YY + 1e-4 * ZZ
    W0 = np.stack([wx.ravel(), wy.ravel()], axis=1)
    x0 = states(p)
    u0 = np.array([[0.3 * DEG, 2.0, 0.1], [-0.2 * DEG, -4.0, 0.0], [0.0, 1.0, -0.2]])
    calm = O.plant_step(p, x0, zero_field(p), u0)
    windy = O.plant_step(p, x0, W0, u0)
    for i in range(3):
        x, y, z = x0[i, :3]
        assert windy[i, 0] - calm[i, 0] == pytest.approx(
            p.dt * (3.0 + 4e-5 * x - 2e-4 * z + 1e-5 * y), abs=1e-9)
        assert windy[i, 1] - calm[i, 1] == pytest.approx(p.dt * (-2.0 + 6e-5 * y + 1e-4 * z), abs=1e-9)
        assert np.array_equal(windy[i, 2:], calm[i, 2:])


def _philox(ctr, key):
    return O.philox(ctr, key)


def _stream7_pair(p, i):
    """Box-Muller pair of words 0, 1 of the Philox draw with counter
    (0, i, 7 << 24, mpc_step << 16) under key seed + scenario_id * golden."""
    s = (p.seed + p.scenario_id * GOLDEN) % 2 ** 64
    x = _philox([0, i, 7 << 24, (p.mpc_step & 0xFFFF) << 16], [s & 0xFFFFFFFF, s >> 32])
    ua = ((x[0] >> 9) + 0.5) / 2 ** 23
    ub = ((x[1] >> 9) + 0.5) / 2 ** 23
    r = math.sqrt(-2.0 * math.log(ua))
    return r * math.cos(2 * math.pi * ub), r * math.sin(2 * math.pi * ub)


@pytest.mark.parametrize("mpc_step,sid", [(0, 0), (5, 3)])
def test_turbulence_is_the_stream_7_pair_of_each_aircraft(mpc_step, sid):
    p = three_aircraft(turb_sigma=1.7, mpc_step=mpc_step, scenario_id=sid, seed=777)
    x0 = states(p)
    u0 = np.array([[0.3 * DEG, 2.0, 0.1], [-0.2 * DEG, -4.0, 0.0], [0.0, 1.0, -0.2]])
    calm = O.plant_step(p.copy(turb_sigma=0.0), x0, zero_field(p), u0)
    gust = O.plant_step(p, x0, zero_field(p), u0)
    for i in range(3):
        n0, n1 = _stream7_pair(p, i)
        assert (gust[i, 0] - calm[i, 0]) == pytest.approx(p.dt * 1.7 * n0, abs=1e-8)
        assert (gust[i, 1] - calm[i, 1]) == pytest.approx(p.dt * 1.7 * n1, abs=1e-8)
    # the rollout's turbulence stream (0) would give other numbers
    s = (p.seed + p.scenario_id * GOLDEN) % 2 ** 64
    x = _philox([0, 0, 0, (p.mpc_step & 0xFFFF) << 16], [s & 0xFFFFFFFF, s >> 32])
    assert x != _philox([0, 0, 7 << 24, (p.mpc_step & 0xFFFF) << 16], [s & 0xFFFFFFFF, s >> 32])


def test_fuel_burn_of_an_unclamped_thrust():
    """With CD2 = 0: T = m (a + g sin gamma) + 1/2 rho v^2 S CD0 (ISA table), the
    burn is dt eta(v) T and the new mass is m - burn."""
    ac = one_aircraft(kind=1, z=3000.0, v=160.0, CD2=0.0)
    p = make_problem([ac], H=4)
    x0 = states(p)
    u0 = np.array([[0.0, 6.0, 0.5]])
    x1 = O.plant_step(p, x0, zero_field(p), u0)[0]
    D = 0.5 * 0.90925 * 160.0 ** 2 * ac["S"] * ac["CD0"]
    T = ac["m"] * (0.5 + G0 * 6.0 / 160.0) + D
    assert ac["m"] - x1[5] == pytest.approx(p.dt * eta(ac, 160.0) * T, rel=3e-4)
