"""Pins of the oracle's rollout: dynamics (Sec. 3.3, Eq. (hor)), constraints
(Sec. 3.4), landing (Eq. (TO_init)), objectives (Sec. 3.5, Sec. 7.1) and the
per-sample cost, against closed forms and the paper's worked values."""
import math

import numpy as np
import pytest

import oracle as O
import scenarios as S
from conftest import controls, make_problem, one_aircraft, zero_wind

G0 = 9.80665
DEG = math.pi / 180


def run(p, u=None, W=None, l=0, m=0, J=0):
    if W is None:
        W = zero_wind(p)
    if u is None:
        u = controls(p)[0]
    return O.trajectory(p, u, W[m], l=l, m=m, J=J)


# ---------------------------------------------------------------- dynamics

def test_straight_level_flight_and_fuel_closed_form():
    v, z, H = 150.0, 3000.0, 12
    ac = one_aircraft(kind=1, x=-5000.0, y=2000.0, z=z, v=v, chi=0.4, CD2=0.0)
    p = make_problem([ac], H=H)
    traj, ch, _ = run(p)
    k = np.arange(H + 1)
    assert np.allclose(traj[:, 0, 0], -5000.0 + k * p.dt * v * math.cos(0.4), rtol=0, atol=1e-8)
    assert np.allclose(traj[:, 0, 1], 2000.0 + k * p.dt * v * math.sin(0.4), rtol=0, atol=1e-8)
    assert np.allclose(traj[:, 0, 2], z) and np.allclose(traj[:, 0, 3], v)
    # with CD2 = 0 and a = 0 the thrust equals the drag, which does not depend on mass:
    # F = H dt eta(v) * 1/2 rho v^2 S CD0
    F = traj[-1, 0, 6]
    eta = ac["Cf1"] * (1 + v / ac["Cf2"])
    rho_eff = F / (H * p.dt * eta * 0.5 * v * v * ac["S"] * ac["CD0"])
    assert rho_eff == pytest.approx(0.90925, rel=3e-4)          # ISA table, 3000 m
    assert traj[-1, 0, 5] == pytest.approx(ac["m"] - F, rel=1e-15)
    # departure with only the fuel term weighted: cost = -ln(1 - F/Fmax)
    p2 = p.copy(alpha_dep=(0.0, 1.0, 0.0, 0.0))
    _, ch2, _ = run(p2)
    Fmax = H * p.dt * ac["Tmax"] * ac["Cf1"] * (1 + p.v_max / ac["Cf2"])
    assert ch2[0] == pytest.approx(-math.log(1 - F / Fmax), rel=1e-12)


def test_isa_density_at_other_altitudes():
    # 1000 m: 1.1117, 5000 m: 0.7364 kg/m^3 (ISA table)
    for z, rho_tab in ((1000.0, 1.1117), (5000.0, 0.7364)):
        ac = one_aircraft(kind=1, z=z, v=160.0, CD2=0.0)
        p = make_problem([ac], H=1)
        traj, _, _ = run(p)
        eta = ac["Cf1"] * (1 + 160.0 / ac["Cf2"])
        rho = traj[-1, 0, 6] / (p.dt * eta * 0.5 * 160.0 ** 2 * ac["S"] * ac["CD0"])
        assert rho == pytest.approx(rho_tab, rel=5e-4)


def test_constant_turn_rate_gives_polygon_on_circle():
    w, v, H = 1.2 * DEG, 140.0, 16
    ac = one_aircraft(kind=1, x=0.0, y=0.0, z=4000.0, v=v, chi=0.25, CD2=0.04)
    p = make_problem([ac], H=H)
    traj, ch, _ = run(p, controls(p, w=w)[0])
    assert np.isfinite(ch[0])
    k = np.arange(H + 1)
    # the lift/bank relations produce exactly the commanded turn rate
    assert np.allclose(traj[:, 0, 4], 0.25 + k * p.dt * w, rtol=0, atol=1e-12)
    assert np.allclose(traj[:, 0, 3], v, atol=1e-9)              # a = 0 keeps the speed
    b = w * p.dt
    sx = np.sin(k * b / 2) / math.sin(b / 2) * np.cos(0.25 + (k - 1) * b / 2)
    sy = np.sin(k * b / 2) / math.sin(b / 2) * np.sin(0.25 + (k - 1) * b / 2)
    assert np.allclose(traj[:, 0, 0], p.dt * v * sx, atol=1e-7)
    assert np.allclose(traj[:, 0, 1], p.dt * v * sy, atol=1e-7)
    # vertices of the Euler polygon lie on a circle of radius dt v / (2 sin(w dt / 2))
    R = p.dt * v / (2 * math.sin(b / 2))
    xy = traj[:, 0, :2]
    A = np.c_[2 * xy, np.ones(len(xy))]
    c = np.linalg.lstsq(A, (xy ** 2).sum(1), rcond=None)[0]
    radius = np.sqrt(c[2] + c[0] ** 2 + c[1] ** 2)
    assert radius == pytest.approx(R, rel=1e-9)


def test_climb_and_acceleration():
    hd, a, v0, H = 6.0, 0.5, 130.0, 10
    ac = one_aircraft(kind=1, x=0.0, y=0.0, z=2000.0, v=v0, chi=0.0, CD2=0.03)
    p = make_problem([ac], H=H)
    traj, ch, _ = run(p, controls(p, hdot=hd, acc=a)[0])
    assert np.isfinite(ch[0])
    k = np.arange(H + 1)
    vk = v0 + k * p.dt * a
    assert np.allclose(traj[:, 0, 2], 2000.0 + k * p.dt * hd, atol=1e-8)
    assert np.allclose(traj[:, 0, 3], vk, atol=1e-8)
    # horizontal speed v cos(gamma) = sqrt(v^2 - hdot^2)
    xk = np.r_[0.0, np.cumsum(p.dt * np.sqrt(vk[:-1] ** 2 - hd ** 2))]
    assert np.allclose(traj[:, 0, 0], xk, atol=1e-7)


def test_turbulence_is_white_with_sigma():
    ac = one_aircraft(kind=1, x=0.0, y=0.0, z=3000.0, v=150.0, chi=0.0)
    p = make_problem([ac], H=2, turb_sigma=1.5)
    base = run(p.copy(turb_sigma=0.0))[0]
    dx = []
    for l in range(3000):
        t = run(p, l=l)[0]
        dx.append([(t[1, 0, 0] - base[1, 0, 0]) / p.dt, (t[1, 0, 1] - base[1, 0, 1]) / p.dt,
                   (t[2, 0, 0] - t[1, 0, 0] - (base[2, 0, 0] - base[1, 0, 0])) / p.dt])
    dx = np.array(dx)
    assert np.allclose(dx.std(0), 1.5, rtol=0.05)
    assert np.allclose(dx.mean(0), 0.0, atol=0.1)
    assert abs(np.corrcoef(dx[:, 0], dx[:, 2])[0, 1]) < 0.06     # independent across steps


# ------------------------------------------------------------- constraints

@pytest.mark.parametrize("eps,viol", [(-1e-6, True), (1e-6, False)])
def test_separation_flips_at_analytic_closest_approach(eps, viol):
    # A flies east from the origin, B north from (X, -Y); the closest approach is at
    # t* = (X+Y)/(2v) with d_min = |X-Y|/sqrt(2) (t* = -dp.dv/|dv|^2, d = |dp + t* dv|)
    v = 150.0
    p0 = make_problem([one_aircraft()], H=10)
    Sh = p0.sep_h
    tstar = 5 * p0.dt
    s = 2 * v * tstar
    d = math.sqrt(2) * Sh * (1 + eps)
    X, Y = (s + d) / 2, (s - d) / 2
    A = one_aircraft(kind=1, x=0.0, y=0.0, z=3000.0, v=v, chi=0.0)
    B = one_aircraft(kind=1, x=X, y=-Y, z=3000.0, v=v, chi=math.pi / 2)
    p = make_problem([A, B], H=10)
    traj, ch, _ = run(p)
    dk = np.hypot(traj[:, 0, 0] - traj[:, 1, 0], traj[:, 0, 1] - traj[:, 1, 1])
    assert dk.argmin() == 5 and dk.min() == pytest.approx(Sh * (1 + eps), rel=1e-9)
    assert (not np.isfinite(ch[0])) == viol and (not np.isfinite(ch[1])) == viol
    assert bool(int(traj[-1, 0, 7]) & 4) == viol


@pytest.mark.parametrize("eps,viol", [(-1e-6, True), (1e-6, False)])
def test_vertical_separation_flips_at_sep_v(eps, viol):
    p0 = make_problem([one_aircraft()], H=4)
    dz = p0.sep_v * (1 + eps)
    A = one_aircraft(kind=1, x=0.0, y=0.0, z=3000.0, v=150.0, chi=0.0)
    B = one_aircraft(kind=1, x=100.0, y=0.0, z=3000.0 + dz, v=150.0, chi=0.0)
    p = make_problem([A, B], H=4)
    _, ch, _ = run(p)
    assert (not np.isfinite(ch[0])) == viol and (not np.isfinite(ch[1])) == viol


def test_unary_altitude_bounds_inclusive_and_freeze():
    # sin(gamma) = -10/160 is exact, so z reaches z_min = 150 exactly: allowed
    ac = one_aircraft(kind=1, z=250.0, v=160.0, CD2=0.0)
    p = make_problem([ac], H=3)
    traj, ch, _ = run(p, controls(p, hdot=-10.0)[0])
    assert traj[1, 0, 2] == 150.0 and int(traj[1, 0, 7]) & 1 == 0
    # the next step goes below: infeasible from then on and frozen
    assert int(traj[2, 0, 7]) & 1 == 1 and not np.isfinite(ch[0])
    assert np.array_equal(traj[3, 0, :7], traj[2, 0, :7])
    # the upper bound
    ac2 = one_aircraft(kind=1, z=9900.0, v=160.0)
    p2 = make_problem([ac2], H=2)
    traj2, ch2, _ = run(p2, controls(p2, hdot=15.0)[0])
    assert not np.isfinite(ch2[0]) and int(traj2[1, 0, 7]) & 1 == 1


@pytest.mark.parametrize("f,ok", [(1 - 1e-9, True), (1 + 1e-9, False)])
def test_bank_angle_limit(f, ok):
    v = 150.0
    ac = one_aircraft(kind=1, v=v)
    p = make_problem([ac], H=2)
    w = f * math.tan(p.phi_max) * G0 / v
    _, ch, _ = run(p, controls(p, w=w)[0])
    assert np.isfinite(ch[0]) == ok


@pytest.mark.parametrize("f,ok", [(1 - 1e-9, True), (1 + 1e-9, False)])
def test_climb_angle_limit(f, ok):
    v = 150.0
    ac = one_aircraft(kind=1, v=v)
    p = make_problem([ac], H=1)
    _, ch, _ = run(p, controls(p, hdot=f * v * math.sin(p.gamma_max))[0])
    assert np.isfinite(ch[0]) == ok


def test_thrust_limits():
    # steep idle descent needs negative thrust: infeasible
    ac = one_aircraft(kind=1, v=150.0, z=5000.0)
    p = make_problem([ac], H=1)
    _, ch, _ = run(p, controls(p, hdot=-15.0, acc=-1.0)[0])
    assert not np.isfinite(ch[0])
    # a heavy aircraft with a small engine cannot accelerate while climbing
    ac2 = one_aircraft(kind=1, v=150.0, z=3000.0, m=80000.0, Tmax=120e3)
    p2 = make_problem([ac2], H=1)
    _, ch2, _ = run(p2, controls(p2, hdot=15.0, acc=1.0)[0])
    assert not np.isfinite(ch2[0])


def test_min_mass_constraint():
    ac = one_aircraft(kind=1, v=150.0, m=45010.0, m_empty=45000.0)     # 10 kg of fuel left
    p = make_problem([ac], H=3)
    traj, ch, _ = run(p)
    assert not np.isfinite(ch[0])
    # level flight burns a constant dt*eta*D per step (CD2 = 0): the limit is crossed
    # at the first step whose cumulative burn exceeds 10 kg
    burn = traj[1, 0, 6]
    k_dead = int(np.floor(10.0 / burn)) + 1
    flags = traj[:, 0, 7].astype(int) & 1
    assert list(flags) == [0] * k_dead + [1] * (p.H + 1 - k_dead)


# ----------------------------------------------------------------- landing

def _lander(v=85.0, **kw):
    base = dict(kind=0, x=5000.0, y=0.0, z=300.0, v=v, chi=math.pi, CD2=0.0)
    base.update(kw)
    return one_aircraft(**base)


def test_landing_in_sector_gives_best_per_step_cost():
    ac = _lander()
    p = make_problem([ac], H=8)
    traj, ch, _ = run(p)
    assert int(traj[1, 0, 7]) & 2            # landed after the first step
    assert np.array_equal(traj[-1, 0, :7], traj[1, 0, :7])      # frozen
    # all deviation terms are zero (best value); only one step of fuel was burned
    F1 = traj[1, 0, 6]
    eta = ac["Cf1"] * (1 + 85.0 / ac["Cf2"])
    rho = 1.225 * (1 - 2.2558e-5 * 300.0) ** 4.2559
    assert F1 == pytest.approx(p.dt * eta * 0.5 * rho * 85.0 ** 2 * ac["S"] * ac["CD0"], rel=1e-12)
    Fmax = p.H * p.dt * ac["Tmax"] * ac["Cf1"] * (1 + p.v_max / ac["Cf2"])
    a1, a2, a3 = p.alpha_arr
    assert ch[0] == pytest.approx(-math.log(a1 + a2 + a3 * (1 - F1 / Fmax)), rel=1e-12)


@pytest.mark.parametrize("change", [dict(v=95.0), dict(z=1200.0), dict(x=15000.0),
                                    dict(chi=math.pi - 25 * DEG), dict(x=3000.0, y=1500.0),
                                    dict(x=-5000.0, chi=0.0)])
def test_each_landing_condition_is_required(change):
    ac = _lander(**change)
    p = make_problem([ac], H=2)
    traj, _, _ = run(p)
    assert not int(traj[1, 0, 7]) & 2


def test_landed_aircraft_leaves_separation_checks():
    A = _lander()
    # B flies level through A's landing point two steps later at the same height
    B = one_aircraft(kind=1, x=4150.0 + 2 * 10 * 150.0, y=0.0, z=300.0 + 50.0, v=150.0,
                     chi=math.pi, CD2=0.0)
    p = make_problem([A, B], H=4)
    traj, ch, _ = run(p)
    assert int(traj[1, 0, 7]) & 2
    d = np.hypot(traj[3, 0, 0] - traj[3, 1, 0], traj[3, 0, 1] - traj[3, 1, 1])
    assert d < p.sep_h
    assert np.isfinite(ch[1])


# ---------------------------------------------------------------- objectives

def test_worked_example_bearing_term():
    # on the desired bearing for the whole horizon: J1 = 1; 90 degrees off: J1 = 0.5
    ac = one_aircraft(kind=1, x=1000.0, y=0.0, z=3000.0, v=150.0, chi=0.0)
    for thF, J1 in ((0.0, 1.0), (math.pi / 2, 0.5), (-math.pi / 2, 0.5), (math.pi, 0.0 + 1e-300)):
        ac["theta_F"] = thF
        p = make_problem([ac], H=6, alpha_dep=(1.0, 0.0, 0.0, 0.0))
        _, ch, _ = run(p)
        if J1 > 1e-100:
            assert ch[0] == pytest.approx(-math.log(J1), abs=1e-12)
        else:
            assert ch[0] == pytest.approx(-math.log(1e-30))


def test_speed_and_altitude_terms():
    ac = one_aircraft(kind=1, x=1000.0, z=3000.0, v=180.0, v_D=200.0, Z=3000.0)
    p = make_problem([ac], H=5, alpha_dep=(0.0, 0.0, 0.0, 1.0))
    _, ch, _ = run(p)
    Cmax = max(p.v_max - 200.0, 200.0 - p.v_min)
    assert ch[0] == pytest.approx(-math.log(1 - 20.0 / Cmax), rel=1e-12)
    # at the target altitude all horizon: B = inf B = 0, J3 = 1
    p3 = make_problem([ac], H=5, alpha_dep=(0.0, 0.0, 1.0, 0.0))
    _, ch3, _ = run(p3)
    assert ch3[0] == pytest.approx(0.0, abs=1e-14)
    # 2 km below the target, flying level: B = 2000, sup/inf from the max climb rate
    ac["Z"] = 5000.0
    _, ch4, _ = run(make_problem([ac], H=5, alpha_dep=(0.0, 0.0, 1.0, 0.0)))
    c = p.v_max * math.sin(p.gamma_max) * p.dt
    sup = np.mean([2000 + k * c for k in range(1, 6)])
    inf = np.mean([max(2000 - k * c, 0) for k in range(1, 6)])
    assert ch4[0] == pytest.approx(-math.log((sup - 2000) / (sup - inf)), rel=1e-12)


def test_zero_fuel_burn_scores_one():
    # level flight with a = -D/m needs zero thrust, so nothing is burned: J_fuel = 1
    ac = one_aircraft(kind=1, v=150.0, CD2=0.0, Tmin=-1.0)
    p = make_problem([ac], H=1, alpha_dep=(0.0, 1.0, 0.0, 0.0))
    traj, _, _ = run(p)
    D = traj[1, 0, 6] / (p.dt * ac["Cf1"] * (1 + 150.0 / ac["Cf2"]))
    traj0, ch, _ = run(p, controls(p, acc=-D / ac["m"])[0])
    assert abs(traj0[1, 0, 6]) < 1e-9
    assert ch[0] == pytest.approx(0.0, abs=1e-12)


def test_arrival_flow_heading_and_glide_terms():
    # on the +x axis flying west the flow-field heading is pi (D = 0); glide angle
    # atan(z / x) against beta_f
    ac = one_aircraft(kind=0, x=20000.0, y=0.0, z=1000.0, v=150.0, chi=math.pi, CD2=0.0)
    p = make_problem([ac], H=3, alpha_arr=(1.0, 0.0, 0.0))
    _, ch, _ = run(p)
    assert ch[0] == pytest.approx(0.0, abs=1e-14)
    p2 = make_problem([ac], H=3, alpha_arr=(0.0, 1.0, 0.0))
    traj, ch2, _ = run(p2)
    E = np.mean([abs(math.atan2(1000.0, traj[k, 0, 0]) - p.beta_f) for k in range(1, 4)])
    assert ch2[0] == pytest.approx(-math.log(1 - E / (math.pi / 2)), rel=1e-12)
    # due north of the runway the flow arc is a half circle: heading chi_hat = pi + 2*(pi/2) = 0
    ac3 = one_aircraft(kind=0, x=0.0, y=20000.0, z=1000.0, v=150.0, chi=0.0, CD2=0.0)
    p3 = make_problem([ac3], H=1, alpha_arr=(1.0, 0.0, 0.0))
    traj3, ch3, _ = run(p3)
    th = math.atan2(traj3[1, 0, 1], traj3[1, 0, 0])
    D = abs(math.remainder(0.0 - (math.pi + 2 * th), 2 * math.pi))
    assert ch3[0] == pytest.approx(-math.log(1 - D / math.pi), abs=1e-12)


def test_noise_cost():
    n = 8
    pd = np.full((n, n), 0.5)
    base = dict(w_noise=1.0, popdense=pd, pop_n=(n, n), pop_lo=(-40000.0, -40000.0),
                pop_hi=(40000.0, 40000.0))
    # below the cutoff: each step scores 1 - (1 - (z/A_c)^2) * 0.5
    ac = one_aircraft(kind=1, x=0.0, z=2000.0, v=150.0)
    p = make_problem([ac], H=4, **base)
    _, ch, _ = run(p)
    assert ch[0] == pytest.approx(-math.log(1 - 0.75 * 0.5), rel=1e-12)
    # above the cutoff the noise term is 1 whatever the density
    ac2 = one_aircraft(kind=1, x=0.0, z=4500.0, v=150.0)
    _, ch2, _ = run(make_problem([ac2], H=4, **base))
    assert ch2[0] == pytest.approx(0.0, abs=1e-14)
    # outside the population grid there is nobody to disturb
    ac3 = one_aircraft(kind=1, x=45000.0, z=1000.0, v=150.0)
    _, ch3, _ = run(make_problem([ac3], H=4, **base))
    assert ch3[0] == pytest.approx(0.0, abs=1e-14)


def test_soft_separation_penalty_closed_form():
    d = 1.3 * make_problem([one_aircraft()]).sep_h
    A = one_aircraft(kind=1, x=0.0, y=0.0, z=3000.0, v=150.0, chi=0.0, theta_F=0.0)
    B = one_aircraft(kind=1, x=0.0, y=d, z=3000.0, v=150.0, chi=0.0, theta_F=0.0)
    p = make_problem([A, B], H=6, sep_mode=1)
    _, ch, cs = run(p)
    g = 1 - d / p.sep_h
    pen = p.H * np.logaddexp(0.0, p.sp_beta * g) / p.sp_beta
    assert np.isfinite(ch).all()
    assert cs - ch == pytest.approx([p.mu_sep * pen] * 2, rel=1e-10)


def test_costs_are_nonnegative_and_bounded():
    # 0 <= J_T <= 1 (Sec. 3.5) means finite costs are >= 0
    p = S.config2().copy(M=2, H=30, grid=(8, 8, 4))
    rng = np.random.default_rng(5)
    u = S.mild_controls(p, 64, rng)
    r = O.rollout(p, u, 0, soft=True)
    c = r["cost"][np.isfinite(r["cost"])]
    assert c.size > 100 and (c >= 0).all() and (c < -math.log(1e-30) + 1e-9).all()
    assert (r["cbar_soft"][np.isfinite(r["cbar"])] >= r["cbar"][np.isfinite(r["cbar"])]).all()
