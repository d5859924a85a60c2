"""Pins against what the paper prints (tests/golden/paper_constants.txt, each
value with its place in the paper): the oracle and the synthetic workloads use
the paper's objective weights, wind-correlation constants, noise cutoff and
sample schedule, and the layout table's rows all cover the same 10240
particles.  No GPU needed."""
import math
import os

import numpy as np

import oracle as O
import scenarios as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.txt")


def paper():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0] if line.lstrip().startswith("#") else line
        if "=" not in line:
            continue
        name, rest = line.split("=", 1)
        value = rest.split("|", 1)[0].split()
        out[name.strip()] = value
    return out


def test_fixture_is_complete_and_cited():
    names = {"alpha_dep", "alpha_arr", "lambda", "beta", "gamma", "A_c", "schedule", "J_max", "L",
             "layout_rows", "layout_best", "layout_used"}
    assert names <= set(paper())
    for line in open(GOLDEN):
        if "=" in line and not line.lstrip().startswith("#"):
            assert "| Sec." in line, line


def test_objective_weights_are_the_papers():
    g = paper()
    dep = [float(v) for v in g["alpha_dep"]]
    arr = [float(v) for v in g["alpha_arr"]]
    assert math.isclose(sum(dep), 1.0) and math.isclose(sum(arr), 1.0)   # Eq. (maxcost): weights sum to 1
    for p in (S.config1(), S.config2(), S.config3(), S.config4(), S.config5(n_scen=2)[1]):
        assert tuple(p.alpha_dep) == tuple(dep)
        assert tuple(p.alpha_arr) == tuple(arr)


def test_wind_correlation_constants_and_covariance():
    g = paper()
    lam, beta, gam = (float(g[k][0]) for k in ("lambda", "beta", "gamma"))
    p = S.shrink(S.config1(), L=8, M=1, H=2, grid=(3, 3, 2))
    assert (p.lam_t, p.beta_xy, p.gam_z) == (lam, beta, gam)
    # the oracle's covariance between two grid nodes is Eq. (cov) at equal times
    R = O.wind_covariance(p)
    xs, ys, zs = O.grid_nodes(p)
    ny, nz = p.grid[1], p.grid[2]

    def idx(ix, iy, iz):
        return (ix * ny + iy) * nz + iz

    for (a, b) in (((0, 0, 0), (2, 1, 1)), ((1, 2, 0), (0, 0, 1)), ((2, 2, 1), (2, 2, 1))):
        d = math.hypot(xs[a[0]] - xs[b[0]], ys[a[1]] - ys[b[1]])
        want = p.wind_sigma ** 2 * math.exp(-beta * d) * math.exp(-gam * abs(zs[a[2]] - zs[b[2]]))
        assert math.isclose(R[idx(*a), idx(*b)], want, rel_tol=1e-12)
    # the AR(1) coefficient exp(-dt lambda) (reading of G_t = 1/lambda)
    assert math.isclose(O.wind_ar_coefficient(p), math.exp(-p.dt * lam), rel_tol=1e-15)


def test_noise_cutoff_is_the_papers():
    assert S.config3().A_c == float(paper()["A_c"][0])


def test_sample_schedule_uses_the_printed_constants():
    a, b, c = (float(v) for v in paper()["schedule"])
    J_max = int(paper()["J_max"][0])
    for J in range(J_max):
        assert O.kappa(J) == math.floor(a + b * math.exp(c * J)), J
    # monotonically increasing, as Algorithm 1 requires of the schedule
    ks = [O.kappa(J) for J in range(J_max)]
    assert all(x <= y for x, y in zip(ks, ks[1:])) and ks[0] == 8


def test_layout_table_rows_cover_the_same_particles():
    g = paper()
    L = int(g["L"][0])
    rows = [tuple(int(v) for v in r.split("x")) for r in g["layout_rows"]]
    assert len(rows) == 17 and all(t * b == L for t, b in rows)
    for k in ("layout_best", "layout_used"):
        t, b = (int(v) for v in g[k][0].split("x"))
        assert (t, b) in rows
