"""Seeded synthetic TMA traffic and stage inputs.

This module only *creates inputs*: scenario parameters, initial aircraft
states, aircraft coefficients, a population-density grid and random arrays
for stage-level tests.  It holds none of the method's arithmetic (no
dynamics, costs, wind model, weights or resampling).  Both the CUDA path and
the CPU oracle consume what it produces; neither imports the other.

The traffic stands in for the Gatwick/FlightRadar24 data of the paper (Sec. 6),
which is not available here.  Shapes follow the paper: a TMA of 30-40 km
radius around a single East-West runway at the origin (Sec. 5.1), departures
that have completed their initial climb (Sec. 3.3), arrivals entering on the
TMA boundary (Sec. 3.3), and a population-density map built from Gaussian
population centres on a 1 km grid (Sec. 7.1).

Units are SI throughout (m, s, kg, N, rad).  Headings use the mathematical
convention (0 = +x = East, counter-clockwise positive), the convention of the
discrete dynamics of Sec. 3.3.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BASE_SEED = 20150601

# Per-aircraft record layout shared (as data) by both consumers.
AIRCRAFT_DTYPE = np.dtype([
    ("type", np.int32),          # 0 = arrival, 1 = departure
    ("x", np.float64), ("y", np.float64), ("z", np.float64),
    ("v", np.float64), ("chi", np.float64), ("m", np.float64),
    ("theta_F", np.float64),     # departure: desired bearing from the airport
    ("Z", np.float64),           # departure: desired altitude
    ("v_D", np.float64),         # departure: desired airspeed
    ("m_empty", np.float64),     # mass of the aircraft without fuel
    ("S", np.float64), ("CD0", np.float64), ("CD2", np.float64),
    ("Cf1", np.float64), ("Cf2", np.float64),
    ("Tmin", np.float64), ("Tmax", np.float64),
    ("t_enter", np.int32),       # rolling window: MPC step at which the aircraft enters
])

NM = 1852.0
FT = 0.3048
DEG = math.pi / 180.0


@dataclasses.dataclass
class Problem:
    """One TMA scenario: sizes, model constants and the aircraft."""
    N: int
    H: int
    L: int
    M: int
    J_max: int
    S: int = 4
    dt: float = 10.0
    seed: int = BASE_SEED
    scenario_id: int = 0
    mpc_step: int = 0
    box_lo: tuple = (-30000.0, -30000.0, 0.0)
    box_hi: tuple = (30000.0, 30000.0, 6000.0)
    grid: tuple = (16, 16, 4)
    wind_sigma: float = 5.0
    turb_sigma: float = 1.0
    lam_t: float = 6e-6           # time-correlation rate (read as 1/s)
    beta_xy: float = 1.6e-6       # horizontal correlation rate (1/m)
    gam_z: float = 1.5e-5         # vertical correlation rate (1/m)
    sep_h: float = 3 * NM
    sep_v: float = 1000 * FT
    sep_mode: int = 0             # 0 hard, 1 soft, 2 both
    sp_beta: float = 10.0
    mu_sep: float = 1.0
    z_min: float = 150.0
    z_max: float = 6000.0
    gamma_max: float = 10 * DEG
    phi_max: float = 30 * DEG
    v_min: float = 60.0
    v_max: float = 260.0
    ctrl_lo: tuple = (-1.5 * DEG, -15.0, -1.0)   # turn rate, climb rate, speed change
    ctrl_hi: tuple = (1.5 * DEG, 15.0, 1.0)
    move_sigma: tuple = (0.05 * 3.0 * DEG, 0.05 * 30.0, 0.05 * 2.0)
    alpha_dep: tuple = (0.4, 0.1, 0.25, 0.25)    # bearing, fuel, altitude, speed
    alpha_arr: tuple = (0.25, 0.65, 0.1)         # flow heading, glide path, fuel
    w_noise: float = 0.0
    A_c: float = 4000.0
    pop_n: tuple = (0, 0)
    pop_lo: tuple = (0.0, 0.0)
    pop_hi: tuple = (0.0, 0.0)
    popdense: Optional[np.ndarray] = None        # [pop_n[0]][pop_n[1]] float64, x-major
    P_runway: float = 10000.0
    P_beta: float = 6 * DEG
    P_chi: float = 20 * DEG
    P_vs: float = 90.0
    beta_f: float = 3 * DEG
    wind_stream: int = 3                         # 8: held-out evaluation wind samples
    wind_mode: int = 0                           # 1: a field per (particle, sample), 2x2x2 grid
    sample_mode: int = 0                         # 1: iteration J draws min(kappa_J, M) samples
    L_sched: Optional[tuple] = None              # particles per iteration (J_max entries, <= L)
    rolling: int = 0                             # 1: rolling window (t_enter, finished aircraft)
    finished: int = 0                            # rolling window: bit i = aircraft i has left
    aircraft: Optional[np.ndarray] = None        # AIRCRAFT_DTYPE[N]

    def copy(self, **kw) -> "Problem":
        p = dataclasses.replace(self, **kw)
        if p.aircraft is not None:
            p.aircraft = p.aircraft.copy()
        return p

    @property
    def n_grid(self) -> int:
        return int(self.grid[0] * self.grid[1] * self.grid[2])


# --------------------------------------------------------------------------
# aircraft synthesis
# --------------------------------------------------------------------------

def _coefficients(rng: np.random.Generator, rec, m0: float) -> None:
    """Seeded BADA-like coefficients (ranges typical of an A320-class jet)."""
    rec["m"] = m0
    rec["m_empty"] = 0.75 * m0
    rec["S"] = rng.uniform(115.0, 130.0)
    rec["CD0"] = rng.uniform(0.020, 0.030)
    rec["CD2"] = rng.uniform(0.035, 0.050)
    rec["Cf1"] = rng.uniform(1.0e-5, 1.3e-5)
    rec["Cf2"] = rng.uniform(400.0, 520.0)
    rec["Tmin"] = 0.0
    rec["Tmax"] = rng.uniform(200e3, 260e3)


def _separated(recs, cand, sep_h, sep_v) -> bool:
    for r in recs:
        dh = math.hypot(r["x"] - cand["x"], r["y"] - cand["y"])
        if dh < 1.5 * sep_h and abs(r["z"] - cand["z"]) < 2.0 * sep_v:
            return False
    return True


def _arrival(rng, ring, z_rng, v_rng, m_rng):
    rec = np.zeros((), AIRCRAFT_DTYPE)
    th = rng.uniform(-math.pi, math.pi)
    rec["type"] = 0
    rec["x"] = ring * math.cos(th)
    rec["y"] = ring * math.sin(th)
    rec["z"] = rng.uniform(*z_rng)
    rec["v"] = rng.uniform(*v_rng)
    rec["chi"] = th + math.pi + rng.uniform(-20, 20) * DEG   # roughly towards the airport
    _coefficients(rng, rec, rng.uniform(*m_rng) * 1000.0)
    return rec


def _departure(rng, r_rng, v_rng, m_rng, z_top):
    rec = np.zeros((), AIRCRAFT_DTYPE)
    th = rng.uniform(-math.pi, math.pi)
    r = rng.uniform(*r_rng)
    rec["type"] = 1
    rec["x"] = r * math.cos(th)
    rec["y"] = r * math.sin(th)
    rec["z"] = min(400.0 + 0.08 * r, 0.8 * z_top)
    rec["v"] = rng.uniform(*v_rng)
    rec["chi"] = th + rng.uniform(-30, 30) * DEG             # outbound
    rec["theta_F"] = th + rng.uniform(-60, 60) * DEG
    rec["Z"] = rng.uniform(0.7, 0.9) * z_top
    rec["v_D"] = rng.uniform(200.0, 230.0)
    _coefficients(rng, rec, rng.uniform(*m_rng) * 1000.0)
    return rec


def _traffic(rng, n_arr, n_dep, *, ring, z_top, sep_h, sep_v,
             v_rng=(150.0, 220.0), m_rng=(50.0, 75.0), dep_r=(2000.0, 22000.0)):
    recs: List[np.ndarray] = []
    kinds = [0] * n_arr + [1] * n_dep
    for kind in kinds:
        for attempt in range(2000):
            if kind == 0:
                rr = ring if attempt < 1000 else ring * rng.uniform(0.8, 1.1)
                cand = _arrival(rng, rr, (3000.0, min(6000.0, 0.85 * z_top)), v_rng, m_rng)
            else:
                cand = _departure(rng, dep_r, (120.0, 180.0), m_rng, z_top)
            if _separated(recs, cand, sep_h, sep_v):
                break
        recs.append(cand)
    out = np.zeros(len(recs), AIRCRAFT_DTYPE)
    for i, r in enumerate(recs):
        out[i] = r
    return out


def popdense_grid(rng, n=128, spacing=1000.0, n_centres=20, half_box=50000.0):
    """Population-density map of Sec. 7.1 on an n x n grid with 1 km spacing.

    Centres are uniform in the TMA box; radii are log-normal (median 2 km,
    sigma_ln 0.4).  The map is the clipped sum of normalised Gaussians of the
    distance to each centre, with distances and radii in km.
    Returns (grid[n][n] float64 x-major, lo, hi).
    """
    half = 0.5 * (n - 1) * spacing
    xs = np.linspace(-half, half, n)
    cx = rng.uniform(-half_box, half_box, n_centres)
    cy = rng.uniform(-half_box, half_box, n_centres)
    c = 2.0 * np.exp(0.4 * rng.standard_normal(n_centres))       # km
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    acc = np.zeros_like(X)
    for k in range(n_centres):
        b = np.hypot(X - cx[k], Y - cy[k]) / 1000.0
        acc += np.exp(-b * b / (2 * c[k] ** 2)) / (c[k] * math.sqrt(2 * math.pi))
    return np.minimum(acc, 1.0), (-half, -half), (half, half)


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def config1(seed: int = BASE_SEED + 1) -> Problem:
    """2 aircraft (1 arrival, 1 departure), 60x60 km x 6 km box, 16x16x4 wind grid,
    H=20, L=1024, M=8, 10 annealing iterations, hard separation."""
    rng = np.random.default_rng(seed)
    p = Problem(N=2, H=20, L=1024, M=8, J_max=10, seed=seed,
                box_lo=(-30000.0, -30000.0, 0.0), box_hi=(30000.0, 30000.0, 6000.0),
                grid=(16, 16, 4), z_max=6000.0)
    ac = np.zeros(2, AIRCRAFT_DTYPE)
    th = rng.uniform(-math.pi, math.pi)
    a = ac[0]
    a["type"] = 0
    a["x"], a["y"] = 30000.0 * math.cos(th), 30000.0 * math.sin(th)
    a["z"] = rng.uniform(3000.0, 5000.0)
    a["v"] = rng.uniform(150.0, 200.0)
    a["chi"] = th + math.pi
    _coefficients(rng, a, rng.uniform(55.0, 70.0) * 1000.0)
    d = ac[1]
    d["type"] = 1
    d["x"], d["y"], d["z"] = 0.0, 0.0, 400.0
    d["chi"] = math.pi
    d["v"] = 120.0
    d["theta_F"] = rng.uniform(-math.pi, math.pi)
    d["Z"] = 5000.0
    d["v_D"] = 200.0
    _coefficients(rng, d, rng.uniform(55.0, 70.0) * 1000.0)
    ac[0], ac[1] = a, d
    p.aircraft = ac
    return p


def config2(seed: int = BASE_SEED + 2) -> Problem:
    """8 aircraft, mixed arrivals/departures, 100x100 km x 8 km box, 64x64x8 wind grid,
    H=60, L=65536, M=32, 30 annealing iterations, hard separation, no noise cost."""
    rng = np.random.default_rng(seed)
    n_arr = int(rng.integers(3, 6))
    p = Problem(N=8, H=60, L=65536, M=32, J_max=30, seed=seed,
                box_lo=(-50000.0, -50000.0, 0.0), box_hi=(50000.0, 50000.0, 8000.0),
                grid=(64, 64, 8), z_max=8000.0)
    p.aircraft = _traffic(rng, n_arr, 8 - n_arr, ring=40000.0, z_top=8000.0,
                          sep_h=p.sep_h, sep_v=p.sep_v)
    return p


def config3(seed: int = BASE_SEED + 3) -> Problem:
    """24 aircraft (14 arrivals, 10 departures), H=120, L=262144, M=64, 64x64x8 grid,
    fuel + ground-noise cost (w_n = 0.1) on a 128x128 population grid, hard and
    softplus separation both evaluated."""
    rng = np.random.default_rng(seed)
    p = Problem(N=24, H=120, L=262144, M=64, J_max=30, seed=seed,
                box_lo=(-50000.0, -50000.0, 0.0), box_hi=(50000.0, 50000.0, 8000.0),
                grid=(64, 64, 8), z_max=8000.0, sep_mode=2, w_noise=0.1)
    p.aircraft = _traffic(rng, 14, 10, ring=40000.0, z_top=8000.0, sep_h=p.sep_h,
                          sep_v=p.sep_v, v_rng=(120.0, 250.0), m_rng=(50.0, 80.0))
    pd, lo, hi = popdense_grid(rng)
    p.popdense, p.pop_n, p.pop_lo, p.pop_hi = pd, pd.shape, lo, hi
    return p


def config4(seed: int = BASE_SEED + 4) -> Problem:
    """12 aircraft, H=60, L=16384, M=16, 16x16x4 grid, softplus separation (beta=10)."""
    rng = np.random.default_rng(seed)
    p = Problem(N=12, H=60, L=16384, M=16, J_max=30, seed=seed,
                box_lo=(-50000.0, -50000.0, 0.0), box_hi=(50000.0, 50000.0, 8000.0),
                grid=(16, 16, 4), z_max=8000.0, sep_mode=1)
    p.aircraft = _traffic(rng, 6, 6, ring=40000.0, z_top=8000.0,
                          sep_h=p.sep_h, sep_v=p.sep_v)
    return p


def config5(seed: int = BASE_SEED + 5, n_scen: int = 256) -> List[Problem]:
    """n_scen independent scenarios with N ~ U{2..32}, H=60, L=16384, M=16,
    20 annealing iterations, 16x16x4 grid."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scen):
        n = int(rng.integers(2, 33))
        n_arr = int(rng.integers(1, n)) if n > 1 else 1
        p = Problem(N=n, H=60, L=16384, M=16, J_max=20, seed=seed, scenario_id=s,
                    box_lo=(-60000.0, -60000.0, 0.0), box_hi=(60000.0, 60000.0, 9000.0),
                    grid=(16, 16, 4), z_max=9000.0)
        p.aircraft = _traffic(rng, n_arr, n - n_arr, ring=45000.0, z_top=9000.0,
                              sep_h=p.sep_h, sep_v=p.sep_v, dep_r=(2000.0, 30000.0))
        out.append(p)
    return out


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


def make_config(k: int, **kw):
    return CONFIGS[k](**kw)


def particle_schedule(L: int, J_max: int, final_frac: float, multiple: int = 32) -> tuple:
    """A decreasing particle count: geometric from L at J = 0 to final_frac * L
    at J = J_max - 1, each rounded down to a multiple of `multiple` (at least
    one multiple), never increasing."""
    out, prev = [], L
    for J in range(J_max):
        x = L * final_frac ** (J / max(J_max - 1, 1))
        n = max(multiple, int(x) // multiple * multiple) if J else L
        prev = min(prev, n)
        out.append(prev)
    return tuple(out)


def shrink(p: Problem, *, L=None, M=None, H=None, J_max=None, grid=None) -> Problem:
    """Same traffic and constants at smaller sizes (for tests)."""
    kw = {}
    for name, val in (("L", L), ("M", M), ("H", H), ("J_max", J_max), ("grid", grid)):
        if val is not None:
            kw[name] = val
    return p.copy(**kw)


# --------------------------------------------------------------------------
# stage inputs (plain seeded random arrays)
# --------------------------------------------------------------------------

def random_controls(p: Problem, L: int, rng: np.random.Generator) -> np.ndarray:
    """Controls u[L][N][S][3] (float32), uniform in the control box."""
    lo = np.asarray(p.ctrl_lo, np.float64)
    hi = np.asarray(p.ctrl_hi, np.float64)
    u = lo + (hi - lo) * rng.random((L, p.N, p.S, 3))
    return u.astype(np.float32)


def mild_controls(p: Problem, L: int, rng: np.random.Generator, frac: float = 0.3) -> np.ndarray:
    """Controls drawn in the central `frac` of the box, so that most trajectories
    stay feasible (exercises the full cost path rather than early violations)."""
    lo = np.asarray(p.ctrl_lo, np.float64)
    hi = np.asarray(p.ctrl_hi, np.float64)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) * frac
    u = mid + half * (2 * rng.random((L, p.N, p.S, 3)) - 1)
    # keep the climb rate mostly non-negative so that thrust stays positive
    u[..., 1] = np.abs(u[..., 1]) * 0.5
    return u.astype(np.float32)


def random_cbar(nseg: int, L: int, rng: np.random.Generator, frac_inf: float = 0.1,
                scale: float = 2.0) -> np.ndarray:
    """Per-(segment, particle) mean costs (float32) with a fraction of +inf."""
    c = (scale * rng.exponential(1.0, (nseg, L))).astype(np.float32)
    c[rng.random((nseg, L)) < frac_inf] = np.inf
    return c


def random_wtilde(nseg: int, L: int, rng: np.random.Generator, frac_zero: float = 0.2,
                  spread: float = 30.0) -> np.ndarray:
    """Unnormalised weights in [0, 1] (float64) with max 1 per segment and zeros."""
    w = np.exp(-spread * rng.random((nseg, L)))
    w[rng.random((nseg, L)) < frac_zero] = 0.0
    for s in range(nseg):
        if L:
            w[s, rng.integers(0, L)] = 1.0
    return w


def random_ancestors(nseg: int, L: int, rng: np.random.Generator) -> np.ndarray:
    return rng.integers(0, max(L, 1), (nseg, L), dtype=np.int32)
