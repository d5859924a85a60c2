"""FP64 CPU oracle of the SMC-MPC hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path
(`paper_1506_02869_gb300`), and never imports it.

The per-particle arithmetic lives in plain C (`oracle.c`, FP64); the wind
model's linear algebra (Sec. 3.9.1: covariance, Cholesky factors, the AR(1)
recursion) is written here with numpy, using library Cholesky and matmul as
steps.  Every function names the passage of Eele & Maciejowski (TR.693, 2015)
it restates.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_OPC_PATH = os.path.join(_LIBDIR, "liboracle_opcount.so")
_OPC_SRC = _SRC + [os.path.join(_HERE, "opcount.cpp")]
_lock = threading.Lock()
_lib = None
_opc = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    stale = force or not os.path.exists(_LIBPATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIBPATH) for s in _SRC)
    if stale:
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC[0], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def build_opcount(force: bool = False) -> str:
    """Compile the operation-counting build of the oracle (opcount.cpp: oracle.c
    as C++ with a counting double, single-threaded) into
    oracle/_lib/liboracle_opcount.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    stale = force or not os.path.exists(_OPC_PATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_OPC_PATH) for s in _OPC_SRC)
    if stale:
        tmp = _OPC_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-Wno-unknown-pragmas", "-o", tmp, _OPC_SRC[2], "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OPC_PATH)
    return _OPC_PATH


class OrcProblem(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("H", C.c_int), ("S", C.c_int), ("L", C.c_int), ("M", C.c_int),
        ("J_max", C.c_int), ("dt", C.c_double), ("seed", C.c_uint64),
        ("scenario_id", C.c_uint32), ("mpc_step", C.c_uint32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("grid", C.c_int * 3),
        ("wind_sigma", C.c_double), ("turb_sigma", C.c_double), ("lam_t", C.c_double),
        ("beta_xy", C.c_double), ("gam_z", C.c_double),
        ("sep_h", C.c_double), ("sep_v", C.c_double), ("sep_mode", C.c_int),
        ("sp_beta", C.c_double), ("mu_sep", C.c_double),
        ("z_min", C.c_double), ("z_max", C.c_double), ("gamma_max", C.c_double),
        ("phi_max", C.c_double), ("v_min", C.c_double), ("v_max", C.c_double),
        ("ctrl_lo", C.c_double * 3), ("ctrl_hi", C.c_double * 3), ("move_sigma", C.c_double * 3),
        ("alpha_dep", C.c_double * 4), ("alpha_arr", C.c_double * 3),
        ("w_noise", C.c_double), ("A_c", C.c_double),
        ("pop_n", C.c_int * 2), ("pop_lo", C.c_double * 2), ("pop_hi", C.c_double * 2),
        ("popdense", C.POINTER(C.c_double)),
        ("P_runway", C.c_double), ("P_beta", C.c_double), ("P_chi", C.c_double),
        ("P_vs", C.c_double), ("beta_f", C.c_double), ("wind_stream", C.c_uint32),
        ("wind_mode", C.c_int), ("wind_chol", C.POINTER(C.c_double)),
        ("rolling", C.c_int), ("finished", C.c_uint32),
    ]


class OrcAircraft(C.Structure):
    _fields_ = [("type", C.c_int32), ("t_enter", C.c_int32)] + [
        (n, C.c_double) for n in ("x", "y", "z", "v", "chi", "m", "theta_F", "Z", "v_D",
                                  "m_empty", "S", "CD0", "CD2", "Cf1", "Cf2", "Tmin", "Tmax")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            d, i32, u32, i64 = C.c_double, C.c_int, C.c_uint32, C.c_int64
            P = C.POINTER
            _lib.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            _lib.orc_uniform23.argtypes = [u32]
            _lib.orc_uniform23.restype = d
            _lib.orc_box_muller.argtypes = [u32, u32, P(d), P(d)]
            _lib.orc_draw.argtypes = [P(OrcProblem), u32, u32, u32, u32, u32, P(u32)]
            _lib.orc_wind_normals.argtypes = [P(OrcProblem), i32, i32, P(d)]
            _lib.orc_rollout.argtypes = [P(OrcProblem), P(OrcAircraft), P(d), i32, i32, P(d),
                                         P(i64), i32, i32, i32, P(d), P(d), P(d), P(d), P(i64)]
            _lib.orc_trajectory.argtypes = [P(OrcProblem), P(OrcAircraft), P(d), i32, P(d), i64,
                                            i32, P(d), P(d), P(d)]
            _lib.orc_rollout_grad.argtypes = [P(OrcProblem), P(OrcAircraft), P(d), P(d), i64, i32, P(d)]
            _lib.orc_rollout_grad.restype = d
            _lib.orc_mh_propose.argtypes = [P(OrcProblem), P(d), P(d), i64, i32, d, d, i32, P(d),
                                            P(C.c_uint8)]
            _lib.orc_mh_propose.restype = None
            _lib.orc_mh_accept.argtypes = [P(OrcProblem), P(d), P(d), P(d), P(d), P(d), P(d),
                                           P(C.c_uint8), i64, i32, d, d, i32, P(d), P(C.c_uint8),
                                           P(d)]
            _lib.orc_mh_accept.restype = None
            _lib.orc_plant_step.argtypes = [P(OrcProblem), P(OrcAircraft), P(d), P(d), P(d), P(d)]
            _lib.orc_plant_finished.argtypes = [P(OrcProblem), P(OrcAircraft), P(d)]
            _lib.orc_plant_finished.restype = u32
            _lib.orc_particle_wind.argtypes = [P(OrcProblem), i64, i32, P(d)]
            _lib.orc_particle_wind.restype = None
            _lib.orc_kappa.argtypes = [i32]
            _lib.orc_kappa.restype = i32
            _lib.orc_lse.argtypes = [P(d), i32, i32, d, P(d), P(d), P(d)]
            _lib.orc_resample_uniform.argtypes = [P(OrcProblem), i32, i32]
            _lib.orc_resample_uniform.restype = u32
            _lib.orc_resample.argtypes = [P(d), i32, i32, P(u32), P(C.c_int32)]
            _lib.orc_resample.restype = i32
            _lib.orc_resample_to.argtypes = [P(d), i32, i32, i32, P(u32), P(C.c_int32)]
            _lib.orc_resample_to.restype = i32
            _lib.orc_move.argtypes = [P(OrcProblem), P(d), P(C.c_int32), i32, i32, P(d)]
            _lib.orc_init_controls.argtypes = [P(OrcProblem), i32, P(d)]
            _lib.orc_select.argtypes = [P(d), i32, i32, P(d), P(i32)]
            _lib.orc_select.restype = i64
    return _lib


def _opcount_lib():
    global _opc
    with _lock:
        if _opc is None:
            _opc = C.CDLL(build_opcount())
            d, i32, i64, P = C.c_double, C.c_int, C.c_int64, C.POINTER
            _opc.orc_rollout.argtypes = [P(OrcProblem), P(OrcAircraft), P(d), i32, i32, P(d),
                                         P(i64), i32, i32, i32, P(d), P(d), P(d), P(d), P(i64)]
            _opc.orc_opcount_read.argtypes = [C.c_int]
            _opc.orc_opcount_read.restype = C.c_uint64
    return _opc


def rollout_opcount(p, u, J, W, pidx=None, soft=True):
    """Floating-point operations of the oracle's rollout (every wind sample of
    W, costs included; counting rule in opcount.cpp) of controls
    u[Lsub][N][S][3], and the aircraft-steps it simulated: (ops, live)."""
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    Ls = u.shape[0]
    pidx = np.arange(Ls, dtype=np.int64) if pidx is None else np.ascontiguousarray(pidx, np.int64)
    W = np.ascontiguousarray(W, np.float64)
    mc = W.shape[0]
    ch = np.empty((Ls, mc, p.N))
    cs = np.empty((Ls, mc, p.N)) if soft else None
    mg = np.empty((Ls, mc, p.N))
    sm = np.empty((Ls, mc))
    live = C.c_int64(0)
    m = _Marshalled(p)
    L = _opcount_lib()
    L.orc_opcount_read(1)
    L.orc_rollout(m.ps, m.ac, _ptr(W, C.c_double), 0, mc, _ptr(u, C.c_double), _ptr(pidx, C.c_int64),
                  Ls, J, 1, _ptr(ch, C.c_double), _ptr(cs, C.c_double) if soft else None,
                  _ptr(mg, C.c_double), _ptr(sm, C.c_double), C.byref(live))
    return int(L.orc_opcount_read(1)), int(live.value)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class _Marshalled:
    """Keeps the ctypes structures and the arrays they point into alive."""

    def __init__(self, p):
        self.p = p
        s = OrcProblem()
        s.N, s.H, s.S, s.L, s.M, s.J_max = p.N, p.H, p.S, p.L, p.M, p.J_max
        s.dt = p.dt
        s.seed = p.seed & 0xFFFFFFFFFFFFFFFF
        s.scenario_id, s.mpc_step = p.scenario_id, p.mpc_step
        s.box_lo[:], s.box_hi[:], s.grid[:] = p.box_lo, p.box_hi, p.grid
        for n in ("wind_sigma", "turb_sigma", "lam_t", "beta_xy", "gam_z", "sep_h", "sep_v",
                  "sp_beta", "mu_sep", "z_min", "z_max", "gamma_max", "phi_max", "v_min",
                  "v_max", "w_noise", "A_c", "P_runway", "P_beta", "P_chi", "P_vs", "beta_f"):
            setattr(s, n, float(getattr(p, n)))
        s.sep_mode = p.sep_mode
        s.wind_stream = int(getattr(p, "wind_stream", 3))
        s.rolling = int(getattr(p, "rolling", 0))
        s.finished = int(getattr(p, "finished", 0)) & 0xFFFFFFFF
        s.wind_mode = int(getattr(p, "wind_mode", 0))
        if s.wind_mode == 1:
            # Qhat: lower Cholesky factor of R_hat on the 2x2x2 corner grid (a library step)
            if tuple(p.grid) != (2, 2, 2):
                raise ValueError("wind mode 1 uses the 2x2x2 grid of the box corners")
            self.chol = np.ascontiguousarray(np.linalg.cholesky(wind_covariance(p)), np.float64)
            s.wind_chol = _ptr(self.chol, C.c_double)
        s.ctrl_lo[:], s.ctrl_hi[:], s.move_sigma[:] = p.ctrl_lo, p.ctrl_hi, p.move_sigma
        s.alpha_dep[:], s.alpha_arr[:] = p.alpha_dep, p.alpha_arr
        if p.popdense is not None:
            self.pop = np.ascontiguousarray(p.popdense, np.float64)
            s.pop_n[:] = self.pop.shape
            s.pop_lo[:], s.pop_hi[:] = p.pop_lo, p.pop_hi
            s.popdense = _ptr(self.pop, C.c_double)
        else:
            self.pop = None
            s.pop_n[:] = (0, 0)
        self.s = s
        ac = p.aircraft
        self.ac = (OrcAircraft * p.N)()
        for i in range(p.N):
            r = ac[i]
            self.ac[i].type = int(r["type"])
            self.ac[i].t_enter = int(r["t_enter"]) if "t_enter" in r.dtype.names else 0
            for n in ("x", "y", "z", "v", "chi", "m", "theta_F", "Z", "v_D", "m_empty", "S",
                      "CD0", "CD2", "Cf1", "Cf2", "Tmin", "Tmax"):
                setattr(self.ac[i], n, float(r[n]))

    @property
    def ps(self):
        return C.byref(self.s)


# ----------------------------------------------------------------------
# random numbers (Philox4x32-10, Salmon et al. SC'11; Box-Muller)
# ----------------------------------------------------------------------

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def uniform23(x: int) -> float:
    return lib().orc_uniform23(x)


def box_muller(xa: int, xb: int):
    a, b = C.c_double(), C.c_double()
    lib().orc_box_muller(xa, xb, C.byref(a), C.byref(b))
    return a.value, b.value


def draw(p, c0, c1, q, stream, J):
    m = _Marshalled(p)
    o = (C.c_uint32 * 4)()
    lib().orc_draw(m.ps, c0, c1, q, stream, J, o)
    return list(o)


# ----------------------------------------------------------------------
# wind model, Sec. 3.9.1
# ----------------------------------------------------------------------

def grid_nodes(p):
    """Node coordinates, inclusive of the box faces (reading R11)."""
    return [np.linspace(p.box_lo[d], p.box_hi[d], p.grid[d]) for d in range(3)]


def wind_covariance_factors(p):
    """Horizontal and vertical correlation matrices of Eq. (cov).

    R_xy[a, b] = exp(-beta |P_a - P_b|) over the (x, y) nodes (index ix*ny+iy),
    R_z[a, b] = exp(-gamma |z_a - z_b|); the full covariance of the grid
    vector (index (ix*ny+iy)*nz+iz) is sigma^2 (R_xy kron R_z).
    """
    xs, ys, zs = grid_nodes(p)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    dxy = np.hypot(X[:, None] - X[None, :], Y[:, None] - Y[None, :])
    Rxy = np.exp(-p.beta_xy * dxy)
    Rz = np.exp(-p.gam_z * np.abs(zs[:, None] - zs[None, :]))
    return Rxy, Rz


def wind_covariance(p):
    """Full covariance R_hat of the grid vector (Eq. (cov), time lag 0)."""
    Rxy, Rz = wind_covariance_factors(p)
    return p.wind_sigma ** 2 * np.kron(Rxy, Rz)


def wind_ar_coefficient(p):
    """a = exp(-dt / G_t), with G_t = 1/lam_t (reading R11)."""
    return math.exp(-p.dt * p.lam_t)


def particle_wind(p, l, m):
    """Mode-1 wind of particle l, sample m: [H][8][2] on the box corners (reading R19)."""
    out = np.empty((p.H, 8, 2), np.float64)
    mm = _Marshalled(p)
    lib().orc_particle_wind(mm.ps, int(l), int(m), _ptr(out, C.c_double))
    return out


def wind_normals(p, m0=0, mc=None):
    """v_X(k), v_Y(k) for samples m0..m0+mc-1 as an array [mc][H][P][2]."""
    if mc is None:
        mc = p.M - m0
    out = np.empty((mc, p.H, p.n_grid, 2), np.float64)
    m = _Marshalled(p)
    lib().orc_wind_normals(m.ps, m0, mc, _ptr(out, C.c_double))
    return out


def wind_field_literal(p, m0=0, mc=None):
    """W(k) by the recursion of Sec. 3.9.1 with the full covariance matrix:
    W(0) = Qhat v(0), W(k+1) = a W(k) + Q v(k+1), Qhat Qhat^T = R_hat,
    Q Q^T = (1 - a^2) R_hat.  Only for small grids (dense P x P Cholesky)."""
    V = wind_normals(p, m0, mc)
    R = wind_covariance(p)
    a = wind_ar_coefficient(p)
    Qhat = np.linalg.cholesky(R)
    Q = np.linalg.cholesky((1.0 - a * a) * R)
    W = np.empty_like(V)
    for mm in range(V.shape[0]):
        for c in range(2):
            W[mm, 0, :, c] = Qhat @ V[mm, 0, :, c]
            for k in range(1, p.H):
                W[mm, k, :, c] = a * W[mm, k - 1, :, c] + Q @ V[mm, k, :, c]
    return W


def wind_field(p, m0=0, mc=None):
    """Same field as `wind_field_literal`, using chol(A kron B) = chol(A) kron chol(B)
    and Q = sqrt(1 - a^2) Qhat, so that large grids stay tractable:
    W(k) = sigma (L_xy kron L_z) B(k), B(0) = v(0), B(k) = a B(k-1) + sqrt(1-a^2) v(k)."""
    V = wind_normals(p, m0, mc)
    mc = V.shape[0]
    nx, ny, nz = p.grid
    Rxy, Rz = wind_covariance_factors(p)
    Lxy = np.linalg.cholesky(Rxy)
    Lz = np.linalg.cholesky(Rz)
    a = wind_ar_coefficient(p)
    b = math.sqrt(1.0 - a * a)
    B = V  # recursion in place
    for k in range(1, p.H):
        B[:, k] = a * B[:, k - 1] + b * B[:, k]
    B = B.reshape(mc, p.H, nx * ny, nz, 2)
    # vertical factor: B'[.., q, y, c] = sum_z Lz[y, z] B[.., q, z, c]
    B = np.einsum("yz,mkqzc->mkqyc", Lz, B, optimize=True)
    # horizontal factor as one matrix product over q
    Bq = np.ascontiguousarray(B.transpose(2, 0, 1, 3, 4)).reshape(nx * ny, -1)
    del B
    Wq = Lxy @ Bq
    del Bq
    W = Wq.reshape(nx * ny, mc, p.H, nz, 2).transpose(1, 2, 0, 3, 4)
    return p.wind_sigma * np.ascontiguousarray(W).reshape(mc, p.H, p.n_grid, 2)


# ----------------------------------------------------------------------
# rollout and costs (Algorithm 1 inner loop; Sec. 3.3-3.6, 7.1)
# ----------------------------------------------------------------------

def rollout(p, u, J, pidx=None, W=None, nthreads=1, m_chunk=None, soft=True):
    """Per-(aircraft, particle) mean costs of controls u[Lsub][N][S][3].

    Returns a dict with
      cbar[N][Lsub]       mean over wind samples of -ln J_T, +inf when infeasible (hard),
      cbar_soft[N][Lsub]  same with the softplus separation penalty (if soft),
      cost[Lsub][M][N]    per-sample hard costs,
      margin[N][Lsub]     smallest relative threshold margin of each aircraft,
      smargin[Lsub]       smallest margin of decisions that change the flying set,
      live                number of simulated aircraft-steps.
    `pidx` gives the global particle indices (they key the turbulence streams).
    """
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    Ls = u.shape[0]
    if pidx is None:
        pidx = np.arange(Ls, dtype=np.int64)
    pidx = np.ascontiguousarray(pidx, np.int64)
    cost = np.empty((Ls, p.M, p.N))
    costs = np.empty((Ls, p.M, p.N)) if soft else None
    marg = np.empty((Ls, p.M, p.N))
    smarg = np.empty((Ls, p.M))
    live_total = 0
    mstep = p.M if (W is not None or m_chunk is None) else m_chunk
    m = _Marshalled(p)
    for m0 in range(0, p.M, mstep):
        mc = min(mstep, p.M - m0)
        Wc = W[m0:m0 + mc] if W is not None else wind_field(p, m0, mc)
        Wc = np.ascontiguousarray(Wc, np.float64)
        ch = np.empty((Ls, mc, p.N))
        cs = np.empty((Ls, mc, p.N)) if soft else None
        mg = np.empty((Ls, mc, p.N))
        sm = np.empty((Ls, mc))
        live = C.c_int64(0)
        lib().orc_rollout(m.ps, m.ac, _ptr(Wc, C.c_double), m0, mc, _ptr(u, C.c_double),
                          _ptr(pidx, C.c_int64), Ls, J, nthreads, _ptr(ch, C.c_double),
                          _ptr(cs, C.c_double) if soft else None, _ptr(mg, C.c_double),
                          _ptr(sm, C.c_double), C.byref(live))
        cost[:, m0:m0 + mc] = ch
        if soft:
            costs[:, m0:m0 + mc] = cs
        marg[:, m0:m0 + mc] = mg
        smarg[:, m0:m0 + mc] = sm
        live_total += live.value
    out = {
        "cbar": cost.mean(axis=1).T.copy(),
        "cost": cost,
        "margin": marg.min(axis=1).T.copy(),
        "smargin": smarg.min(axis=1),
        "live": live_total,
    }
    if soft:
        out["cbar_soft"] = costs.mean(axis=1).T.copy()
        out["cost_soft"] = costs
    return out


def rollout_at_samples(p, u, J, samples, pidx=None, soft=True, nthreads=1):
    """Per-sample costs of controls u[Lsub][N][S][3] under the listed wind
    samples only (each field generated alone, so that full-size problems stay
    tractable): dict of cost / cost_soft [Lsub][len(samples)][N] and margin /
    smargin as `rollout` returns them per sample ([Lsub][len][N], [Lsub][len])."""
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    Ls = u.shape[0]
    if pidx is None:
        pidx = np.arange(Ls, dtype=np.int64)
    pidx = np.ascontiguousarray(pidx, np.int64)
    ns = len(samples)
    out = {"cost": np.empty((Ls, ns, p.N)), "margin": np.empty((Ls, ns, p.N)),
           "smargin": np.empty((Ls, ns))}
    if soft:
        out["cost_soft"] = np.empty((Ls, ns, p.N))
    m = _Marshalled(p)
    for q, ms in enumerate(samples):
        Wc = np.ascontiguousarray(wind_field(p, int(ms), 1), np.float64)
        ch = np.empty((Ls, 1, p.N))
        cs = np.empty((Ls, 1, p.N)) if soft else None
        mg = np.empty((Ls, 1, p.N))
        sm = np.empty((Ls, 1))
        live = C.c_int64(0)
        lib().orc_rollout(m.ps, m.ac, _ptr(Wc, C.c_double), int(ms), 1, _ptr(u, C.c_double),
                          _ptr(pidx, C.c_int64), Ls, J, nthreads, _ptr(ch, C.c_double),
                          _ptr(cs, C.c_double) if soft else None, _ptr(mg, C.c_double),
                          _ptr(sm, C.c_double), C.byref(live))
        out["cost"][:, q] = ch[:, 0]
        out["margin"][:, q] = mg[:, 0]
        out["smargin"][:, q] = sm[:, 0]
        if soft:
            out["cost_soft"][:, q] = cs[:, 0]
    return out


def trajectory(p, u_l, W_m, l=0, m=0, J=0):
    """States of one (particle, sample) rollout: (traj[H+1][N][8], cost_hard[N],
    cost_soft[N]); traj columns x, y, z, v, chi, m, F, flags (1 violated,
    2 landed, 4 separation violated).  W_m = W[H][P][2]."""
    u = np.ascontiguousarray(u_l, np.float64).reshape(p.N, p.S, 3)
    Wm = np.ascontiguousarray(W_m, np.float64).reshape(p.H, p.n_grid, 2)
    traj = np.empty((p.H + 1, p.N, 8))
    ch = np.empty(p.N)
    cs = np.empty(p.N)
    mm = _Marshalled(p)
    lib().orc_trajectory(mm.ps, mm.ac, _ptr(Wm, C.c_double), m, _ptr(u, C.c_double), l, J,
                         _ptr(traj, C.c_double), _ptr(ch, C.c_double), _ptr(cs, C.c_double))
    return traj, ch, cs


def rollout_grad(p, u_l, W, l=0, J=0):
    """(C, dC/du) of one particle: C = sum_i mean_m c_soft (softplus separation),
    gradient by reverse mode; (inf, 0) if the particle is infeasible."""
    u = np.ascontiguousarray(u_l, np.float64).reshape(p.N, p.S, 3)
    Wc = np.ascontiguousarray(W, np.float64)
    g = np.empty((p.N, p.S, 3))
    mm = _Marshalled(p)
    c = lib().orc_rollout_grad(mm.ps, mm.ac, _ptr(Wc, C.c_double), _ptr(u, C.c_double), l, J,
                               _ptr(g, C.c_double))
    return c, g


def mh_propose(p, u, grad, J, kappa, eps, kind):
    """Proposal of the Metropolis-Hastings move (kind 1 random walk, 2 Langevin):
    (u_prop [L][N][S][3], inbox [L])."""
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    L = u.shape[0]
    g = np.ascontiguousarray(grad if grad is not None else np.zeros_like(u), np.float64)
    up = np.empty_like(u)
    inbox = np.empty(L, np.uint8)
    mm = _Marshalled(p)
    lib().orc_mh_propose(mm.ps, _ptr(u, C.c_double), _ptr(g, C.c_double), L, J, kappa, eps, kind,
                         _ptr(up, C.c_double), _ptr(inbox, C.c_uint8))
    return up, inbox


def mh_accept(p, u, up, cbar, cbarp, g, gp, inbox, J, kappa, eps, kind):
    """Accept step: (u_out, accepted [L], log_alpha [L])."""
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    L = u.shape[0]
    up = np.ascontiguousarray(up, np.float64).reshape(u.shape)
    z = np.zeros_like(u)
    g = np.ascontiguousarray(g if g is not None else z, np.float64).reshape(u.shape)
    gp = np.ascontiguousarray(gp if gp is not None else z, np.float64).reshape(u.shape)
    cb = np.ascontiguousarray(cbar, np.float64).reshape(p.N, L)
    cbp = np.ascontiguousarray(cbarp, np.float64).reshape(p.N, L)
    ib = np.ascontiguousarray(inbox, np.uint8)
    out = np.empty_like(u)
    acc = np.empty(L, np.uint8)
    la = np.empty(L)
    mm = _Marshalled(p)
    lib().orc_mh_accept(mm.ps, _ptr(u, C.c_double), _ptr(up, C.c_double), _ptr(cb, C.c_double),
                        _ptr(cbp, C.c_double), _ptr(g, C.c_double), _ptr(gp, C.c_double),
                        _ptr(ib, C.c_uint8), L, J, kappa, eps, kind, _ptr(out, C.c_double),
                        _ptr(acc, C.c_uint8), _ptr(la, C.c_double))
    return out, acc.astype(bool), la


def plant_finished(p, x):
    """Rolling window (reading R22): the finished mask after a plant step that
    produced the states x[N][6]: p.finished plus every active arrival inside
    the landing sector."""
    xi = np.ascontiguousarray(x, np.float64).reshape(p.N, 6)
    mm = _Marshalled(p)
    return int(lib().orc_plant_finished(mm.ps, mm.ac, _ptr(xi, C.c_double)))


def plant_step(p, x, W0, u0):
    """One step of the true system (Sec. 2, Fig. 1): states x[N][6] (x, y, z,
    v, chi, m), wind field W0[P][2] of sample 0 at step 0, first-segment
    controls u0[N][3]; returns the new states.  With a rolling window, aircraft
    that have not entered (t_enter > mpc_step) or have finished keep theirs."""
    xi = np.ascontiguousarray(x, np.float64).reshape(p.N, 6)
    W = np.ascontiguousarray(W0, np.float64).reshape(p.n_grid, 2)
    uu = np.ascontiguousarray(u0, np.float64).reshape(p.N, 3)
    out = np.empty_like(xi)
    mm = _Marshalled(p)
    lib().orc_plant_step(mm.ps, mm.ac, _ptr(xi, C.c_double), _ptr(W, C.c_double),
                         _ptr(uu, C.c_double), _ptr(out, C.c_double))
    return out


# ----------------------------------------------------------------------
# weights, resampling, perturbation, selection (Sec. 3.6-3.8)
# ----------------------------------------------------------------------

def kappa(J: int) -> int:
    """SampleSchedule(J) = floor(3 + 5 exp(0.05 J)) of Sec. 5.1, used as the
    annealing exponent (reading R10)."""
    return lib().orc_kappa(J)


def samples(p, J: int) -> int:
    """Wind samples of iteration J: all M (sample mode 0), or the paper's inner
    loop of Algorithm 1, SampleSchedule(J) draws, at most M (sample mode 1;
    reading R20)."""
    return min(kappa(J), p.M) if getattr(p, "sample_mode", 0) == 1 else p.M


def exponent(p, J: int) -> int:
    """The factor of the mean cost in the log-weight l = -exponent * cbar: the
    annealing exponent kappa_J with M fixed samples (reading R10); with the
    inner loop of Algorithm 1 the weight is the product of J_T over the
    iteration's draws (Sec. 3.6), l = -sum_m c_m = -samples(p, J) * cbar
    (reading R20)."""
    return samples(p, J) if getattr(p, "sample_mode", 0) == 1 else kappa(J)


def lse(cbar, kappa_J):
    """w~ = exp(l - max l) with l = -kappa * cbar per segment (row); returns
    (wtilde[nseg][L], lmax[nseg], wsum[nseg])."""
    c = np.ascontiguousarray(cbar, np.float64)
    nseg, L = c.shape
    wt = np.empty_like(c)
    lm = np.empty(nseg)
    ws = np.empty(nseg)
    lib().orc_lse(_ptr(c, C.c_double), nseg, L, float(kappa_J), _ptr(wt, C.c_double),
                  _ptr(lm, C.c_double), _ptr(ws, C.c_double))
    return wt, lm, ws


def resample_uniform(p, seg: int, J: int) -> int:
    m = _Marshalled(p)
    return lib().orc_resample_uniform(m.ps, seg, J)


def resample(wtilde, r, L_out=None):
    """Ancestors anc[nseg][L_out] of systematic resampling (reading R12; L_out
    thresholds over the L weighted particles, reading R21; L_out = L by
    default); returns (anc, number of degenerate segments)."""
    w = np.ascontiguousarray(wtilde, np.float64)
    nseg, L = w.shape
    Lo = L if L_out is None else int(L_out)
    rr = np.ascontiguousarray(np.asarray(r, np.uint64).astype(np.uint32))
    anc = np.empty((nseg, Lo), np.int32)
    nd = lib().orc_resample_to(_ptr(w, C.c_double), nseg, L, Lo, _ptr(rr, C.c_uint32),
                               _ptr(anc, C.c_int32))
    return anc, nd


def move(p, u, anc, J):
    """u'[l][i] = clip(u[anc[i][l]][i] + sigma * xi) (Algorithm 1, perturbation);
    one child per ancestor entry, l < anc.shape[1]."""
    u = np.ascontiguousarray(u, np.float64).reshape(-1, p.N, p.S, 3)
    a = np.ascontiguousarray(anc, np.int32).reshape(p.N, -1)
    L = a.shape[1]
    assert a.size == 0 or (a.min() >= 0 and a.max() < u.shape[0])
    out = np.empty((L, p.N, p.S, 3))
    m = _Marshalled(p)
    lib().orc_move(m.ps, _ptr(u, C.c_double), _ptr(a, C.c_int32), L, J, _ptr(out, C.c_double))
    return out


def init_controls(p, L=None):
    """Uniform initial controls (Sec. 3.2) from random stream 4."""
    L = p.L if L is None else L
    out = np.empty((L, p.N, p.S, 3))
    m = _Marshalled(p)
    lib().orc_init_controls(m.ps, L, _ptr(out, C.c_double))
    return out


def select(cbar):
    """Best particle of Sec. 3.8: (index, cost sum, number of infeasible aircraft)."""
    c = np.ascontiguousarray(cbar, np.float64)
    N, L = c.shape
    bs = C.c_double()
    ni = C.c_int()
    best = lib().orc_select(_ptr(c, C.c_double), N, L, C.byref(bs), C.byref(ni))
    return int(best), bs.value, ni.value


def particles(p, J: int) -> int:
    """Particles evaluated in iteration J: L, or the particle schedule's entry
    (reading R21)."""
    sched = getattr(p, "L_sched", None)
    return int(sched[J]) if sched is not None else p.L


def smc_solve(p, W=None, nthreads=1, history=False):
    """One SMC optimisation (Algorithm 1) with the readings of oracle.c:
    J_max evaluations; between them per-aircraft resampling and perturbation;
    final selection from the last evaluation."""
    if W is None:
        W = wind_field(p)
    u = init_controls(p, particles(p, 0))
    hist = []
    r = None
    for J in range(p.J_max):
        Mj = samples(p, J)      # the first Mj samples of the solve's field
        r = rollout(p.copy(M=Mj), u, J, W=W[:Mj], nthreads=nthreads, soft=(p.sep_mode != 0))
        cb = r["cbar_soft"] if p.sep_mode == 1 else r["cbar"]
        if history:
            hist.append({"J": J, "cbar": cb.copy(), "u": u.copy()})
        if J < p.J_max - 1:
            wt, _, _ = lse(cb, exponent(p, J))
            rr = [resample_uniform(p, i, J) for i in range(p.N)]
            anc, _ = resample(wt, rr, particles(p, J + 1))
            u = move(p, u, anc, J)
    cb = r["cbar_soft"] if p.sep_mode == 1 else r["cbar"]
    best, bsum, ninf = select(cb)
    return {"best": best, "best_sum": bsum, "n_inf": ninf, "best_u": u[best].copy(),
            "cbar": cb, "u": u, "history": hist}
