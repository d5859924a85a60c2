"""Pins of the oracle's wind model (Sec. 3.9.1) and of its trilinear
interpolation, through factorisation identities, statistics and exact
reproduction of constant and linear fields."""
import math

import numpy as np
import pytest

import oracle as O
import scenarios as S
from conftest import controls, make_problem, one_aircraft, zero_wind


def small(**kw):
    p = S.config1().copy(grid=(3, 3, 2), H=4, M=1, box_lo=(-20000.0, -20000.0, 0.0),
                         box_hi=(20000.0, 20000.0, 6000.0))
    return p.copy(**kw)


def test_cholesky_factors_reproduce_covariance():
    p = S.config1()
    Rxy, Rz = O.wind_covariance_factors(p)
    Lxy, Lz = np.linalg.cholesky(Rxy), np.linalg.cholesky(Rz)
    assert np.abs(Lxy @ Lxy.T - Rxy).max() < 1e-10
    assert np.abs(Lz @ Lz.T - Rz).max() < 1e-12
    # the Kronecker factor of the full grid covariance
    L = p.wind_sigma * np.kron(Lxy, Lz)
    assert np.abs(L @ L.T - O.wind_covariance(p)).max() < 1e-8


def test_covariance_entries_follow_eq_cov():
    p = small()
    R = O.wind_covariance(p)
    xs, ys, zs = O.grid_nodes(p)
    # node (ix, iy, iz) has index (ix*ny + iy)*nz + iz
    a, b = (0, 0, 0), (2, 1, 1)
    ia = (a[0] * 3 + a[1]) * 2 + a[2]
    ib = (b[0] * 3 + b[1]) * 2 + b[2]
    dxy = math.hypot(xs[2] - xs[0], ys[1] - ys[0])
    dz = zs[1] - zs[0]
    expect = p.wind_sigma ** 2 * math.exp(-p.beta_xy * dxy) * math.exp(-p.gam_z * dz)
    assert R[ia, ib] == pytest.approx(expect, rel=1e-14)
    assert np.allclose(np.diag(R), p.wind_sigma ** 2)


def test_kronecker_field_equals_literal_recursion():
    p = S.config1().copy(H=6, M=2, lam_t=2e-2)      # a visible time decay
    W1 = O.wind_field(p)
    W2 = O.wind_field_literal(p)
    assert np.abs(W1 - W2).max() < 1e-9


def test_field_covariance_matches_r_hat_statistically():
    p = small(M=4000, H=1)
    W = O.wind_field(p)                               # [M][1][P][2]
    R = O.wind_covariance(p)
    for c in range(2):
        X = W[:, 0, :, c]
        C = X.T @ X / X.shape[0]
        assert np.abs(C - R).max() < 0.08 * p.wind_sigma ** 2
    # X and Y components uncorrelated
    cxy = (W[:, 0, :, 0] * W[:, 0, :, 1]).mean()
    assert abs(cxy) < 0.05 * p.wind_sigma ** 2


def test_time_correlation_is_a():
    p = small(M=3000, H=3, lam_t=math.log(2.0) / 10.0)   # a = exp(-dt*lam) = 0.5
    assert O.wind_ar_coefficient(p) == pytest.approx(0.5)
    W = O.wind_field(p)
    x0, x1, x2 = W[:, 0, :, 0].ravel(), W[:, 1, :, 0].ravel(), W[:, 2, :, 0].ravel()
    assert np.corrcoef(x0, x1)[0, 1] == pytest.approx(0.5, abs=0.03)
    assert np.corrcoef(x0, x2)[0, 1] == pytest.approx(0.25, abs=0.03)
    # stationary: every step keeps the variance sigma^2
    for x in (x0, x1, x2):
        assert x.var() == pytest.approx(p.wind_sigma ** 2, rel=0.05)


def test_a_equal_one_freezes_the_field():
    p = small(M=2, H=5, lam_t=0.0)
    W = O.wind_field(p)
    for k in range(1, 5):
        assert np.array_equal(W[:, k], W[:, 0])


def _straight(p, W, u=None):
    if u is None:
        u = controls(p)[0]
    return O.trajectory(p, u, W[0])[0]


def test_constant_wind_field_displaces_track_exactly():
    ac = one_aircraft(kind=1, x=1000.0, y=-2000.0, z=3000.0, v=150.0, chi=0.3)
    p = make_problem([ac], H=8)
    W = zero_wind(p)
    traj0 = _straight(p, W)
    W[..., 0], W[..., 1] = 7.0, -3.0           # same value at every node
    traj1 = _straight(p, W)
    k = np.arange(p.H + 1)
    assert np.allclose(traj1[:, 0, 0] - traj0[:, 0, 0], 7.0 * p.dt * k, atol=1e-9)
    assert np.allclose(traj1[:, 0, 1] - traj0[:, 0, 1], -3.0 * p.dt * k, atol=1e-9)


def test_linear_wind_field_is_reproduced_exactly():
    # w_x = alpha * x at the nodes; trilinear interpolation of a linear function is exact,
    # so x_{k+1} = x_k + dt (v cos(chi) + alpha x_k) has a closed form
    ac = one_aircraft(kind=1, x=1000.0, y=500.0, z=3000.0, v=150.0, chi=0.0)
    p = make_problem([ac], H=10)
    xs, ys, zs = O.grid_nodes(p)
    alpha, beta = 1e-4, 2e-4
    W = zero_wind(p)
    X = np.repeat(xs, p.grid[1] * p.grid[2])
    Z = np.tile(zs, p.grid[0] * p.grid[1])
    W[..., 0] = alpha * X
    W[..., 1] = beta * Z
    traj = _straight(p, W)
    r = 1.0 + alpha * p.dt
    k = np.arange(p.H + 1)
    v = 150.0
    x_expect = r ** k * 1000.0 + p.dt * v * (r ** k - 1.0) / (alpha * p.dt)
    assert np.allclose(traj[:, 0, 0], x_expect, rtol=1e-12, atol=1e-7)
    assert np.allclose(traj[:, 0, 1], 500.0 + beta * 3000.0 * p.dt * k, atol=1e-7)


def test_positions_outside_box_use_face_values():
    ac = one_aircraft(kind=1, x=60000.0, y=0.0, z=3000.0, v=100.0, chi=0.0)   # beyond x_hi
    p = make_problem([ac], H=3)
    xs, ys, zs = O.grid_nodes(p)
    W = zero_wind(p)
    X = np.repeat(xs, p.grid[1] * p.grid[2])
    W[..., 1] = np.where(X == xs[-1], 4.0, -9.0)     # only the x_hi face blows +4 in y
    traj = _straight(p, W)
    assert np.allclose(traj[:, 0, 1], 4.0 * p.dt * np.arange(p.H + 1), atol=1e-9)


def test_held_out_wind_stream_is_independent():
    """Stream 8 gives the same distribution as stream 3 (the model of Sec. 3.9.1)
    and independent draws."""
    p = S.shrink(S.config1(), M=4, H=6)
    v3 = O.wind_normals(p)
    v8 = O.wind_normals(p.copy(wind_stream=8))
    assert v3.shape == v8.shape
    assert abs(np.corrcoef(v3.ravel(), v8.ravel())[0, 1]) < 0.05
    assert abs(v8.std() - 1.0) < 0.05 and abs(v8.mean()) < 0.05
    assert np.array_equal(O.wind_normals(p.copy(wind_stream=3)), v3)


# ---------------------------------------------------------------- per-particle wind (mode 1)

def _mode1(p=None, **kw):
    base = S.shrink(S.config1(), M=3, H=8, grid=(2, 2, 2)) if p is None else p
    return base.copy(wind_mode=1, **kw)


def test_particle_wind_is_the_paper_recursion():
    """W(0) = Qhat v(0), W(k+1) = a W(k) + Q v(k+1) with QQ^T = (1-a^2) R_hat and
    Qhat Qhat^T = R_hat (Sec. 3.9.1), factorised here independently, with the
    normals of random stream 9 re-derived from the counter layout."""
    p = _mode1()
    R = O.wind_covariance(p)
    a = O.wind_ar_coefficient(p)
    Qhat = np.linalg.cholesky(R)
    Q = np.linalg.cholesky((1 - a * a) * R)
    for l, m in ((0, 0), (7, 2), (2 ** 31 + 5, 1)):
        got = O.particle_wind(p, l, m)
        W = np.zeros((8, 2))
        for k in range(p.H):
            v = np.empty((8, 2))
            for r in range(4):
                w = O.draw(p, l & 0xFFFFFFFF, 4 * m + r, k, 9, 0)
                v[2 * r] = O.box_muller(w[0], w[1])
                v[2 * r + 1] = O.box_muller(w[2], w[3])
            W = Qhat @ v if k == 0 else a * W + Q @ v
            assert np.allclose(got[k], W, rtol=1e-12, atol=1e-12), (l, m, k)


def test_particle_wind_statistics():
    """Across particles the field at every step has covariance R_hat, and the
    lag-one correlation of a node is a."""
    p = _mode1(S.shrink(S.config1(), M=1, H=4, grid=(2, 2, 2)).copy(lam_t=0.02))
    R = O.wind_covariance(p)
    a = O.wind_ar_coefficient(p)
    n = 6000
    F = np.stack([O.particle_wind(p, l, 0) for l in range(n)])      # [n][H][8][2]
    for k in (0, 3):
        X = F[:, k, :, 0]
        C = np.cov(X.T)
        assert np.allclose(C, R, atol=5 * R[0, 0] * np.sqrt(2.0 / n)), k
    x0, x1 = F[:, 2, 3, 1], F[:, 3, 3, 1]
    rho = np.corrcoef(x0, x1)[0, 1]
    assert abs(rho - a) < 4 * (1 - a * a) / np.sqrt(n) + 0.01


def test_particle_wind_differs_between_particles_and_samples():
    p = _mode1()
    w00, w10, w01 = O.particle_wind(p, 0, 0), O.particle_wind(p, 1, 0), O.particle_wind(p, 0, 1)
    assert not np.allclose(w00, w10) and not np.allclose(w00, w01)
    assert np.array_equal(w00, O.particle_wind(p, 0, 0))


def test_mode1_rollout_uses_each_particles_own_field():
    """With the control sequence shared, two particles differ only by their
    random streams; with turbulence off, two samples of one particle differ
    only by their wind field, and the rollout's interpolation of that field is
    the trilinear interpolation of the corner values."""
    p = _mode1(turb_sigma=0.0)
    rng = np.random.default_rng(3)
    u = np.repeat(S.mild_controls(p, 1, rng).astype(np.float64), 2, axis=0)
    r = O.rollout(p, u, 0, pidx=np.array([4, 9]))
    assert not np.allclose(r["cost_soft"][0], r["cost_soft"][1])
    r2 = O.rollout(p, u[:1], 0, pidx=np.array([4]))
    assert np.array_equal(r2["cost_soft"][0], r["cost_soft"][0])
    # the trajectory of sample m under mode 1 equals the mode-0 trajectory run
    # on that particle's field
    Wl = O.particle_wind(p, 4, 1)
    t1, _, _ = O.trajectory(p, u[0], np.zeros((p.H, 8, 2)), l=4, m=1)
    t0, _, _ = O.trajectory(p.copy(wind_mode=0), u[0], Wl, l=4, m=1)
    assert np.array_equal(t1, t0)
