"""Python binding of the GB300 SMC-MPC hot path (include/tma_smc.h).

Argument marshalling only: every step of the path runs in the CUDA kernels
of `_lib/libtma_smc.so`.  Functions carry the names of the C-ABI entry
points; PyTorch provides device memory and streams.  If the library has not
been built, every call raises -- there is no CPU fallback.

A problem is any object (or dict) with the fields of `tma_problem` plus an
`aircraft` record array with the fields type, x, y, z, v, chi, m, theta_F,
Z, v_D, m_empty, S, CD0, CD2, Cf1, Cf2, Tmin, Tmax.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libtma_smc.so")

TMA_OK, TMA_ERR_INVALID_ARG, TMA_ERR_OOM, TMA_ERR_CUDA = 0, 1, 2, 3
TMA_ERR_BOUNDS, TMA_ERR_TIMEOUT, TMA_WARN_DEGENERATE, TMA_ERR_UNSUPPORTED = 4, 5, 6, 7
TMA_MAX_AIRCRAFT = 32
TMA_MAX_PARTICLES = 1 << 22
TMA_MAX_GRAD_HORIZON = 320
TMA_MOVE_PAPER, TMA_MOVE_RWMH, TMA_MOVE_MALA = 0, 1, 2
TMA_DEVERR_DEGENERATE, TMA_DEVERR_INFEASIBLE, TMA_DEVERR_BOUNDS = 1, 2, 4

EXPORTS = [
    "tma_status_str", "tma_last_error_string", "tma_launch_count", "tma_create", "tma_destroy",
    "tma_set_state", "tma_wind_field", "tma_rollout_cost", "tma_sample_costs", "tma_live_steps",
    "tma_move", "tma_init_controls", "tma_solve", "tma_solve_host", "tma_best_index",
    "tma_lse_workspace", "tma_lse", "tma_resample_workspace", "tma_resample",
    "tma_select_workspace", "tma_select", "tma_profile_enable", "tma_profile_read",
    "tma_resample_noalloc", "tma_get_tuning", "tma_plant_step", "tma_get_state",
    "tma_batch_create", "tma_batch_destroy", "tma_batch_set_state", "tma_batch_solve",
    "tma_batch_mpc", "tma_batch_results", "tma_batch_latency", "tma_batch_live_steps",
    "tma_set_wind_stream", "tma_rollout_grad", "tma_set_move", "tma_mh_propose", "tma_mh_accept",
    "tma_mh_stats", "tma_get_grad_tuning", "tma_get_particles", "tma_mpc_run", "tma_get_error",
    "tma_resample_to", "tma_move_to", "tma_set_finished", "tma_get_status", "tma_set_tuning",
    "tma_lse_resample_workspace", "tma_lse_resample", "tma_batch_rollout_cost",
    "tma_batch_get_dispatch", "tma_batch_set_dispatch",
]


class TmaError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{msg}: status {status} ({_status_str(status)})")
        self.status = status


class TmaProblem(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("H", C.c_int32), ("S", C.c_int32), ("L", C.c_int32), ("M", C.c_int32),
        ("J_max", C.c_int32), ("dt", C.c_double), ("seed", C.c_uint64),
        ("scenario_id", C.c_uint32), ("mpc_step", C.c_uint32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("grid", C.c_int32 * 3),
        ("wind_sigma", C.c_double), ("turb_sigma", C.c_double), ("lam_t", C.c_double),
        ("beta_xy", C.c_double), ("gam_z", C.c_double), ("sep_h", C.c_double),
        ("sep_v", C.c_double), ("sep_mode", C.c_int32), ("sp_beta", C.c_double),
        ("mu_sep", C.c_double), ("z_min", C.c_double), ("z_max", C.c_double),
        ("gamma_max", C.c_double), ("phi_max", C.c_double), ("v_min", C.c_double),
        ("v_max", C.c_double), ("ctrl_lo", C.c_double * 3), ("ctrl_hi", C.c_double * 3),
        ("move_sigma", C.c_double * 3), ("alpha_dep", C.c_double * 4),
        ("alpha_arr", C.c_double * 3), ("w_noise", C.c_double), ("A_c", C.c_double),
        ("pop_n", C.c_int32 * 2), ("pop_lo", C.c_double * 2), ("pop_hi", C.c_double * 2),
        ("popdense", C.POINTER(C.c_double)), ("P_runway", C.c_double), ("P_beta", C.c_double),
        ("P_chi", C.c_double), ("P_vs", C.c_double), ("beta_f", C.c_double),
        ("wind_mode", C.c_int32), ("sample_mode", C.c_int32),
        ("L_sched", C.POINTER(C.c_int64)), ("rolling", C.c_int32),
    ]


class TmaState(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("x", "y", "z", "v", "chi", "m")]


class TmaProfile(C.Structure):
    _fields_ = [("ms", C.c_double * 10), ("launches", C.c_uint64 * 10)]


STAGES = ("wind", "init", "rollout", "sample_mean", "lse", "resample", "move", "select", "grad",
          "mh")


class TmaAircraft(C.Structure):
    _fields_ = [("type", C.c_int32), ("t_enter", C.c_int32), ("x0", TmaState)] + [
        (n, C.c_double) for n in ("theta_F", "Z", "v_D", "m_empty", "S", "CD0", "CD2", "Cf1",
                                  "Cf2", "Tmin", "Tmax")]


_lib = None
_lock = threading.Lock()


def build(force=False, verbose=False):
    """Compile the CUDA library for sm_103a (in-tree)."""
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIBPATH):
                raise RuntimeError(f"CUDA library not built ({LIBPATH}); run build() first")
            L = C.CDLL(LIBPATH)
            P, vp, st = C.POINTER, C.c_void_p, C.c_void_p
            i32, i64, u32, u64, d, sz = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double, C.c_size_t
            sig = {
                "tma_status_str": ([C.c_int], C.c_char_p),
                "tma_last_error_string": ([], C.c_char_p),
                "tma_launch_count": ([], u64),
                "tma_create": ([P(TmaProblem), P(TmaAircraft), P(vp)], C.c_int),
                "tma_destroy": ([vp], None),
                "tma_set_state": ([vp, P(TmaState), u32, st], C.c_int),
                "tma_wind_field": ([vp, vp, st], C.c_int),
                "tma_rollout_cost": ([vp, vp, i64, i32, vp, vp, st], C.c_int),
                "tma_sample_costs": ([vp, vp, i64, C.c_int, st], C.c_int),
                "tma_live_steps": ([vp, P(u64), st], C.c_int),
                "tma_move": ([vp, vp, vp, i64, i32, vp, st], C.c_int),
                "tma_move_to": ([vp, vp, i64, vp, i64, i32, vp, st], C.c_int),
                "tma_init_controls": ([vp, vp, i64, st], C.c_int),
                "tma_solve": ([vp, vp, P(d), st], C.c_int),
                "tma_solve_host": ([vp, P(TmaState), u32, vp, P(d), st], C.c_int),
                "tma_best_index": ([vp, P(i64), st], C.c_int),
                "tma_get_particles": ([vp, vp, i64, st], C.c_int),
                "tma_lse_workspace": ([i32, i64], sz),
                "tma_lse": ([vp, i32, i64, d, vp, vp, vp, vp, sz, st], C.c_int),
                "tma_resample_workspace": ([i32, i64], sz),
                "tma_resample": ([vp, i32, i64, u64, u32, u32, u32, vp, vp, sz, st], C.c_int),
                "tma_resample_to": ([vp, i32, i64, i64, u64, u32, u32, u32, vp, vp, sz, st], C.c_int),
                "tma_lse_resample_workspace": ([i32, i64], sz),
                "tma_lse_resample": ([vp, i32, i64, i64, d, u64, u32, u32, u32, vp, vp, vp, vp, sz, st],
                                     C.c_int),
                "tma_select_workspace": ([i64], sz),
                "tma_select": ([vp, i32, i64, vp, vp, vp, vp, sz, st], C.c_int),
                "tma_profile_enable": ([vp, C.c_int], C.c_int),
                "tma_get_tuning": ([vp, P(i32), P(i32), P(i32), P(C.c_float)], C.c_int),
                "tma_get_grad_tuning": ([vp, P(i32), P(i32), P(i32), P(C.c_float)], C.c_int),
                "tma_plant_step": ([vp, vp, st], C.c_int),
                "tma_get_state": ([vp, P(TmaState), P(u32), st], C.c_int),
                "tma_set_finished": ([vp, u32, st], C.c_int),
                "tma_set_tuning": ([vp, i32], C.c_int),
                "tma_get_status": ([vp, P(i32), P(u32), st], C.c_int),
                "tma_mpc_run": ([vp, i32, P(TmaState), P(d), st], C.c_int),
                "tma_get_error": ([vp, P(u32), st], C.c_int),
                "tma_batch_create": ([P(TmaProblem), P(P(TmaAircraft)), i32, P(vp)], C.c_int),
                "tma_batch_destroy": ([vp], None),
                "tma_batch_set_state": ([vp, P(TmaState), P(u32), st], C.c_int),
                "tma_batch_solve": ([vp, st], C.c_int),
                "tma_batch_mpc": ([vp, i32, i32, st], C.c_int),
                "tma_batch_results": ([vp, vp, P(d), P(i64), P(TmaState), P(u32), st], C.c_int),
                "tma_batch_latency": ([vp, P(d), st], C.c_int),
                "tma_batch_live_steps": ([vp, P(u64), st], C.c_int),
                "tma_batch_rollout_cost": ([vp, vp, i32, vp, vp, st], C.c_int),
                "tma_batch_get_dispatch": ([vp, P(i32), P(C.c_float), P(C.c_float)], C.c_int),
                "tma_batch_set_dispatch": ([vp, i32], C.c_int),
                "tma_resample_noalloc": ([vp, i32, i64, u64, u32, u32, u32, vp, st], C.c_int),
                "tma_profile_read": ([vp, P(TmaProfile), C.c_int], C.c_int),
                "tma_set_wind_stream": ([vp, u32], C.c_int),
                "tma_rollout_grad": ([vp, vp, i64, i32, vp, vp, vp, st], C.c_int),
                "tma_set_move": ([vp, i32, d], C.c_int),
                "tma_mh_propose": ([vp, vp, vp, i64, i32, d, d, i32, vp, vp, st], C.c_int),
                "tma_mh_accept": ([vp, vp, vp, vp, vp, vp, vp, vp, i64, i32, d, d, i32, vp, vp, st],
                                  C.c_int),
                "tma_mh_stats": ([vp, P(u32), P(d), i32, st], C.c_int),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _status_str(s):
    try:
        return lib().tma_status_str(s).decode()
    except Exception:
        return "?"


def _check(status, what, allow=(TMA_OK,)):
    if status not in allow:
        extra = ""
        if status == TMA_ERR_CUDA:
            extra = " / " + lib().tma_last_error_string().decode()
        raise TmaError(status, what + extra)
    return status


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _get(p, name, default=None):
    if isinstance(p, dict):
        return p.get(name, default)
    return getattr(p, name, default)


def problem_struct(p):
    """Marshal a problem object into (TmaProblem, TmaAircraft[N], keep-alive)."""
    s = TmaProblem()
    for n in ("N", "H", "S", "L", "M", "J_max"):
        setattr(s, n, int(_get(p, n)))
    s.dt = float(_get(p, "dt"))
    s.seed = int(_get(p, "seed")) & 0xFFFFFFFFFFFFFFFF
    s.scenario_id = int(_get(p, "scenario_id", 0))
    s.mpc_step = int(_get(p, "mpc_step", 0))
    s.box_lo[:] = [float(v) for v in _get(p, "box_lo")]
    s.box_hi[:] = [float(v) for v in _get(p, "box_hi")]
    s.grid[:] = [int(v) for v in _get(p, "grid")]
    for n in ("wind_sigma", "turb_sigma", "lam_t", "beta_xy", "gam_z", "sep_h", "sep_v",
              "sp_beta", "mu_sep", "z_min", "z_max", "gamma_max", "phi_max", "v_min", "v_max",
              "w_noise", "A_c", "P_runway", "P_beta", "P_chi", "P_vs", "beta_f"):
        setattr(s, n, float(_get(p, n)))
    s.sep_mode = int(_get(p, "sep_mode"))
    s.wind_mode = int(_get(p, "wind_mode", 0))
    s.sample_mode = int(_get(p, "sample_mode", 0))
    s.rolling = int(_get(p, "rolling", 0))
    s.ctrl_lo[:] = [float(v) for v in _get(p, "ctrl_lo")]
    s.ctrl_hi[:] = [float(v) for v in _get(p, "ctrl_hi")]
    s.move_sigma[:] = [float(v) for v in _get(p, "move_sigma")]
    s.alpha_dep[:] = [float(v) for v in _get(p, "alpha_dep")]
    s.alpha_arr[:] = [float(v) for v in _get(p, "alpha_arr")]
    keep = []
    pd = _get(p, "popdense")
    if pd is not None:
        pd = np.ascontiguousarray(pd, np.float64)
        keep.append(pd)
        s.pop_n[:] = list(pd.shape)
        s.pop_lo[:] = [float(v) for v in _get(p, "pop_lo")]
        s.pop_hi[:] = [float(v) for v in _get(p, "pop_hi")]
        s.popdense = pd.ctypes.data_as(C.POINTER(C.c_double))
    ls = _get(p, "L_sched", None)
    if ls is not None:
        ls = np.ascontiguousarray(ls, np.int64)
        keep.append(ls)
        s.L_sched = ls.ctypes.data_as(C.POINTER(C.c_int64))
    ac = _get(p, "aircraft")
    arr = (TmaAircraft * s.N)()
    for i in range(s.N):
        r = ac[i]
        a = arr[i]
        a.type = int(r["type"])
        a.t_enter = int(r["t_enter"]) if "t_enter" in r.dtype.names else 0
        for n in ("x", "y", "z", "v", "chi", "m"):
            setattr(a.x0, n, float(r[n]))
        for n in ("theta_F", "Z", "v_D", "m_empty", "S", "CD0", "CD2", "Cf1", "Cf2", "Tmin", "Tmax"):
            setattr(a, n, float(r[n]))
    return s, arr, keep


def states_struct(x0):
    """x0: array-like [N][6] (x, y, z, v, chi, m) -> TmaState[N]."""
    x0 = np.asarray(x0, np.float64).reshape(-1, 6)
    arr = (TmaState * len(x0))()
    for i, r in enumerate(x0):
        arr[i].x, arr[i].y, arr[i].z, arr[i].v, arr[i].chi, arr[i].m = (float(v) for v in r)
    return arr


# ---------------------------------------------------------------- solver

def tma_create(problem):
    """Create a solver on the current CUDA device; returns an opaque handle."""
    s, arr, keep = problem_struct(problem)
    h = C.c_void_p()
    _check(lib().tma_create(C.byref(s), arr, C.byref(h)), "tma_create")
    return h


def tma_destroy(h):
    if h:
        lib().tma_destroy(h)


def tma_set_state(h, x0=None, mpc_step=0, stream=None):
    arr = states_struct(x0) if x0 is not None else None
    _check(lib().tma_set_state(h, arr, int(mpc_step), _stream(stream)), "tma_set_state")


def tma_wind_field(h, out=None, stream=None):
    _check(lib().tma_wind_field(h, _dptr(out), _stream(stream)), "tma_wind_field")
    return out


def tma_set_wind_stream(h, stream):
    _check(lib().tma_set_wind_stream(h, int(stream)), "tma_set_wind_stream")


def tma_rollout_cost(h, u, J, cbar, cbar_soft=None, stream=None):
    """u: cuda float32 [L][N][S][3]; writes cbar (and cbar_soft) [N][L]."""
    L = u.shape[0]
    _check(lib().tma_rollout_cost(h, _dptr(u), L, int(J), _dptr(cbar), _dptr(cbar_soft),
                                  _stream(stream)), "tma_rollout_cost")


def tma_sample_costs(h, out, soft=False, stream=None):
    """out: cuda float32 [M][N][L]."""
    _check(lib().tma_sample_costs(h, _dptr(out), out.shape[2], int(soft), _stream(stream)),
           "tma_sample_costs")


def tma_live_steps(h, stream=None):
    v = C.c_uint64()
    _check(lib().tma_live_steps(h, C.byref(v), _stream(stream)), "tma_live_steps")
    return v.value


def tma_move(h, u, anc, J, u_out, stream=None):
    _check(lib().tma_move(h, _dptr(u), _dptr(anc), u.shape[0], int(J), _dptr(u_out),
                          _stream(stream)), "tma_move")


def tma_move_to(h, u, anc, J, u_out, stream=None):
    """u: parents [L_in][N][S][3], anc: int32 [N][L] -> u_out: children [L][N][S][3]."""
    _check(lib().tma_move_to(h, _dptr(u), u.shape[0], _dptr(anc), anc.shape[1], int(J), _dptr(u_out),
                             _stream(stream)), "tma_move_to")


def tma_init_controls(h, u, stream=None):
    _check(lib().tma_init_controls(h, _dptr(u), u.shape[0], _stream(stream)), "tma_init_controls")


def tma_solve(h, best_u=None, stream=None, want_cost=True):
    """One SMC solve; returns (status, best cost or None)."""
    c = C.c_double()
    st = lib().tma_solve(h, _dptr(best_u), C.byref(c) if want_cost else None, _stream(stream))
    _check(st, "tma_solve", allow=(TMA_OK, TMA_WARN_DEGENERATE))
    return st, (c.value if want_cost else None)


def tma_solve_host(h, x0, mpc_step, best_u_host, stream=None):
    """Solve through host buffers; best_u_host: float32 numpy [N][S][3] (written)."""
    assert best_u_host.dtype == np.float32 and best_u_host.flags.c_contiguous
    c = C.c_double()
    arr = states_struct(x0)
    st = lib().tma_solve_host(h, arr, int(mpc_step), best_u_host.ctypes.data_as(C.c_void_p),
                              C.byref(c), _stream(stream))
    _check(st, "tma_solve_host", allow=(TMA_OK, TMA_WARN_DEGENERATE))
    return st, c.value


def tma_get_particles(h, out, stream=None):
    """Copy the last solve's particle set into out (cuda float32 [L][N][S][3])."""
    _check(lib().tma_get_particles(h, _dptr(out), out.shape[0], _stream(stream)),
           "tma_get_particles")
    return out


def tma_best_index(h, stream=None):
    v = C.c_int64()
    _check(lib().tma_best_index(h, C.byref(v), _stream(stream)), "tma_best_index")
    return v.value


def tma_get_tuning(h):
    """(chosen rollout variant, {variant: ms per rollout} timed by the autotuner)."""
    v, n = C.c_int32(), C.c_int32()
    vs, ms = (C.c_int32 * 24)(), (C.c_float * 24)()
    _check(lib().tma_get_tuning(h, C.byref(v), C.byref(n), vs, ms), "tma_get_tuning")
    return v.value, {vs[k]: ms[k] for k in range(n.value)}


def tma_get_grad_tuning(h):
    """(chosen gradient-kernel variant, {variant: ms per launch} timed by its autotuner)."""
    v, n = C.c_int32(), C.c_int32()
    vs, ms = (C.c_int32 * 8)(), (C.c_float * 8)()
    _check(lib().tma_get_grad_tuning(h, C.byref(v), C.byref(n), vs, ms), "tma_get_grad_tuning")
    return v.value, {vs[k]: ms[k] for k in range(n.value)}


def tma_profile_enable(h, on=True):
    _check(lib().tma_profile_enable(h, int(bool(on))), "tma_profile_enable")


def tma_profile_read(h, reset=True):
    """Per-stage device time {stage: (ms, launches)} since the last reset."""
    prof = TmaProfile()
    _check(lib().tma_profile_read(h, C.byref(prof), int(bool(reset))), "tma_profile_read")
    return {name: (prof.ms[k], prof.launches[k]) for k, name in enumerate(STAGES)}


# -------------------------------------------------- gradient and accepted moves

def tma_rollout_grad(h, u, J, cost, grad, cbar_soft=None, stream=None):
    """u: cuda float32 [L][N][S][3]; writes cost [L], grad [L][N][S][3] (and the
    per-aircraft soft means [N][L])."""
    _check(lib().tma_rollout_grad(h, _dptr(u), u.shape[0], int(J), _dptr(cost), _dptr(grad),
                                  _dptr(cbar_soft), _stream(stream)), "tma_rollout_grad")


def tma_set_move(h, kind, eps0=1.0):
    _check(lib().tma_set_move(h, int(kind), float(eps0)), "tma_set_move")


def tma_mh_propose(h, u, grad, J, kappa, eps, kind, u_prop, inbox, stream=None):
    _check(lib().tma_mh_propose(h, _dptr(u), _dptr(grad), u.shape[0], int(J), float(kappa),
                                float(eps), int(kind), _dptr(u_prop), _dptr(inbox),
                                _stream(stream)), "tma_mh_propose")


def tma_mh_accept(h, u, u_prop, cbar, cbar_prop, grad, grad_prop, inbox, J, kappa, eps, kind,
                  u_out, accepted=None, stream=None):
    _check(lib().tma_mh_accept(h, _dptr(u), _dptr(u_prop), _dptr(cbar), _dptr(cbar_prop),
                               _dptr(grad), _dptr(grad_prop), _dptr(inbox), u.shape[0], int(J),
                               float(kappa), float(eps), int(kind), _dptr(u_out), _dptr(accepted),
                               _stream(stream)), "tma_mh_accept")


def tma_mh_stats(h, n, stream=None):
    """(accepted particles, step) per iteration of the last solve, n entries."""
    acc = (C.c_uint32 * max(n, 1))()
    eps = (C.c_double * max(n, 1))()
    _check(lib().tma_mh_stats(h, acc, eps, int(n), _stream(stream)), "tma_mh_stats")
    return np.array(acc[:n], np.int64), np.array(eps[:n])


def _rollout_cost_function():
    """torch.autograd.Function over tma_rollout_grad: C(u) [L] with dC/du."""
    torch = _torch()

    class RolloutCost(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u, solver, J):
            u = u.detach().contiguous()
            cost = torch.empty(u.shape[0], dtype=torch.float32, device=u.device)
            grad = torch.empty_like(u)
            tma_rollout_grad(solver.h, u, J, cost, grad)
            ctx.save_for_backward(grad)
            return cost

        @staticmethod
        def backward(ctx, g_cost):
            (grad,) = ctx.saved_tensors
            return g_cost.reshape(-1, 1, 1, 1) * grad, None, None

    return RolloutCost


_RolloutCost = None


def rollout_cost_autograd(u, solver, J):
    """Differentiable soft objective C(u) = sum_i cbar_soft[i] of each particle
    (float32 [L]); backward multiplies the kernel's gradient."""
    global _RolloutCost
    if _RolloutCost is None:
        _RolloutCost = _rollout_cost_function()
    return _RolloutCost.apply(u, solver, J)


# ------------------------------------------------------------- MPC plant

def tma_plant_step(h, u, stream=None):
    """Advance the solver's true state by one step with the segment-0 controls of
    u (cuda float32 [N][S][3])."""
    _check(lib().tma_plant_step(h, _dptr(u), _stream(stream)), "tma_plant_step")


def tma_mpc_run(h, n_steps, N, stream=None):
    """n receding-horizon steps (solve + plant): (states [n][N][6], best costs [n], status)."""
    traj = (TmaState * max(n_steps * N, 1))()
    costs = (C.c_double * max(n_steps, 1))()
    st = lib().tma_mpc_run(h, int(n_steps), traj, costs, _stream(stream))
    _check(st, "tma_mpc_run", allow=(TMA_OK, TMA_WARN_DEGENERATE))
    x = np.array([[getattr(traj[t * N + i], f) for f in ("x", "y", "z", "v", "chi", "m")]
                  for t in range(n_steps) for i in range(N)]).reshape(n_steps, N, 6)
    return x, np.array(costs[:n_steps]), st


def tma_get_error(h, stream=None):
    """The solver's sticky device error word (TMA_DEVERR_* bits), cleared by
    the call; the word is returned also when its bounds bit makes the call
    return TMA_ERR_BOUNDS."""
    v = C.c_uint32()
    _check(lib().tma_get_error(h, C.byref(v), _stream(stream)), "tma_get_error",
           allow=(TMA_OK, TMA_ERR_BOUNDS))
    return v.value


def tma_get_state(h, N, stream=None):
    """(states [N][6] as numpy, MPC step) of the solver."""
    arr = (TmaState * N)()
    mpc = C.c_uint32()
    _check(lib().tma_get_state(h, arr, C.byref(mpc), _stream(stream)), "tma_get_state")
    return np.array([[a.x, a.y, a.z, a.v, a.chi, a.m] for a in arr]), mpc.value


def tma_set_tuning(h, variant):
    _check(lib().tma_set_tuning(h, int(variant)), "tma_set_tuning")


def tma_set_finished(h, mask, stream=None):
    _check(lib().tma_set_finished(h, int(mask) & 0xFFFFFFFF, _stream(stream)), "tma_set_finished")


def tma_get_status(h, N, stream=None):
    """(per-aircraft status [N]: 0 not entered, 1 active, 2 finished; finished mask)."""
    st = (C.c_int32 * N)()
    fin = C.c_uint32()
    _check(lib().tma_get_status(h, st, C.byref(fin), _stream(stream)), "tma_get_status")
    return np.array(list(st), np.int32), fin.value


# ----------------------------------------------------------------- batches

def tma_batch_create(problems):
    """One batch handle for a list of problems sharing sizes and wind model."""
    structs = [problem_struct(p) for p in problems]
    n = len(structs)
    parr = (TmaProblem * n)(*[s for s, _, _ in structs])
    aptrs = (C.POINTER(TmaAircraft) * n)(*[C.cast(a, C.POINTER(TmaAircraft)) for _, a, _ in structs])
    h = C.c_void_p()
    _check(lib().tma_batch_create(parr, aptrs, n, C.byref(h)), "tma_batch_create")
    return h


def tma_batch_destroy(h):
    if h:
        lib().tma_batch_destroy(h)


def tma_batch_set_state(h, x0=None, mpc=None, stream=None):
    arr = states_struct(x0) if x0 is not None else None
    m = (C.c_uint32 * len(mpc))(*[int(v) for v in mpc]) if mpc is not None else None
    _check(lib().tma_batch_set_state(h, arr, m, _stream(stream)), "tma_batch_set_state")


def tma_batch_solve(h, stream=None):
    _check(lib().tma_batch_solve(h, _stream(stream)), "tma_batch_solve")


def tma_batch_mpc(h, n_steps, use_graph=True, stream=None):
    _check(lib().tma_batch_mpc(h, int(n_steps), int(bool(use_graph)), _stream(stream)), "tma_batch_mpc")


def tma_batch_get_dispatch(h):
    """(form in use: 0 persistent launch, 1 a launch per scenario; timed ms of
    each form on one rollout of the batch at creation)."""
    d, a, b = C.c_int32(), C.c_float(), C.c_float()
    _check(lib().tma_batch_get_dispatch(h, C.byref(d), C.byref(a), C.byref(b)), "tma_batch_get_dispatch")
    return d.value, {0: a.value, 1: b.value}


def tma_batch_set_dispatch(h, dispatch):
    _check(lib().tma_batch_set_dispatch(h, int(dispatch)), "tma_batch_set_dispatch")


def tma_batch_rollout_cost(h, u, J, cost_ms, cost_ms_soft=None, stream=None):
    """The batched rollout alone on packed controls u (scenario after
    scenario, [L][N_s][S][3] each) -> packed per-sample costs ([M][N_s][L] each)."""
    _check(lib().tma_batch_rollout_cost(h, _dptr(u), int(J), _dptr(cost_ms),
                                        _dptr(cost_ms_soft) if cost_ms_soft is not None else None,
                                        _stream(stream)), "tma_batch_rollout_cost")


def tma_batch_results(h, Ns, S, stream=None):
    """dict with best_u (list of [N_s][S][3]), best_cost [n], best [n], states
    (list of [N_s][6]) and mpc [n]."""
    n, tot = len(Ns), int(sum(Ns))
    bu = np.empty((tot, S, 3), np.float32)
    bc = np.empty(n, np.float64)
    bi = np.empty(n, np.int64)
    xs = (TmaState * tot)()
    mp = np.empty(n, np.uint32)
    _check(lib().tma_batch_results(h, bu.ctypes.data_as(C.c_void_p), bc.ctypes.data_as(C.POINTER(C.c_double)),
                                   bi.ctypes.data_as(C.POINTER(C.c_int64)), xs,
                                   mp.ctypes.data_as(C.POINTER(C.c_uint32)), _stream(stream)),
           "tma_batch_results")
    st = np.array([[a.x, a.y, a.z, a.v, a.chi, a.m] for a in xs])
    offs = np.r_[0, np.cumsum(Ns)]
    return {"best_u": [bu[offs[k]:offs[k + 1]] for k in range(n)], "best_cost": bc, "best": bi,
            "states": [st[offs[k]:offs[k + 1]] for k in range(n)], "mpc": mp}


def tma_batch_latency(h, n, stream=None):
    out = np.empty(n, np.float64)
    _check(lib().tma_batch_latency(h, out.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)),
           "tma_batch_latency")
    return out


def tma_batch_live_steps(h, stream=None):
    v = C.c_uint64()
    _check(lib().tma_batch_live_steps(h, C.byref(v), _stream(stream)), "tma_batch_live_steps")
    return v.value


# --------------------------------------------------------- stateless stages

def _workspace(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


def tma_lse(cbar, kappa, wtilde, lmax=None, wsum=None, work=None, stream=None):
    """cbar: cuda float32 [nseg][L] -> wtilde float64 [nseg][L] (+ lmax, wsum [nseg])."""
    nseg, L = cbar.shape
    need = lib().tma_lse_workspace(nseg, L)
    if work is None:
        work = _workspace(need, cbar.device)
    _check(lib().tma_lse(_dptr(cbar), nseg, L, float(kappa), _dptr(wtilde), _dptr(lmax),
                         _dptr(wsum), _dptr(work), work.numel(), _stream(stream)), "tma_lse")


def tma_resample(wtilde, seed, scenario_id, J, mpc_step, anc, work=None, stream=None):
    """wtilde: cuda float64 [nseg][L] -> anc int32 [nseg][L]; returns the status
    (TMA_WARN_DEGENERATE when a segment was all zero)."""
    nseg, L = wtilde.shape
    need = lib().tma_resample_workspace(nseg, L)
    if work is None:
        work = _workspace(need, wtilde.device)
    return _check(lib().tma_resample(_dptr(wtilde), nseg, L, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                     int(scenario_id), int(J), int(mpc_step), _dptr(anc),
                                     _dptr(work), work.numel(), _stream(stream)),
                  "tma_resample", allow=(TMA_OK, TMA_WARN_DEGENERATE))


def tma_resample_to(wtilde, seed, scenario_id, J, mpc_step, anc, work=None, stream=None):
    """wtilde: cuda float64 [nseg][L] -> anc int32 [nseg][L_out] (L_out = anc.shape[1]);
    returns the status."""
    nseg, L = wtilde.shape
    need = lib().tma_resample_workspace(nseg, L)
    if work is None:
        work = _workspace(need, wtilde.device)
    return _check(lib().tma_resample_to(_dptr(wtilde), nseg, L, anc.shape[1],
                                        int(seed) & 0xFFFFFFFFFFFFFFFF, int(scenario_id), int(J),
                                        int(mpc_step), _dptr(anc), _dptr(work), work.numel(),
                                        _stream(stream)),
                  "tma_resample_to", allow=(TMA_OK, TMA_WARN_DEGENERATE))


def tma_lse_resample(cbar, kappa, seed, scenario_id, J, mpc_step, wtilde, anc, degenerate=None,
                     work=None, stream=None):
    """cbar: cuda float32 [nseg][L] -> wtilde float64 [nseg][L] and anc int32
    [nseg][L_out] (L_out = anc.shape[1]) in one stream-ordered call; bit 0 of
    degenerate (cuda int32 [1], zeroed by the caller) marks an all-zero segment."""
    nseg, L = cbar.shape
    need = lib().tma_lse_resample_workspace(nseg, L)
    if work is None:
        work = _workspace(need, cbar.device)
    _check(lib().tma_lse_resample(_dptr(cbar), nseg, L, anc.shape[1], float(kappa),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(scenario_id), int(J),
                                  int(mpc_step), _dptr(wtilde), _dptr(anc), _dptr(degenerate),
                                  _dptr(work), work.numel(), _stream(stream)), "tma_lse_resample")


def tma_resample_noalloc(wtilde, seed, scenario_id, J, mpc_step, anc, stream=None):
    """tma_resample without a workspace (library-owned fixed scratch; see the
    header for its size limit and the serialisation rule); returns the status."""
    nseg, L = wtilde.shape
    return _check(lib().tma_resample_noalloc(_dptr(wtilde), nseg, L, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                             int(scenario_id), int(J), int(mpc_step), _dptr(anc),
                                             _stream(stream)),
                  "tma_resample_noalloc", allow=(TMA_OK, TMA_WARN_DEGENERATE))


def tma_select(cbar, best, best_sum=None, ninf=None, work=None, stream=None):
    """cbar: cuda float32 [N][L] -> best int64 [1], best_sum float64 [1], ninf int32 [1]."""
    N, L = cbar.shape
    need = lib().tma_select_workspace(L)
    if work is None:
        work = _workspace(need, cbar.device)
    _check(lib().tma_select(_dptr(cbar), N, L, _dptr(best), _dptr(best_sum), _dptr(ninf),
                            _dptr(work), work.numel(), _stream(stream)), "tma_select")


# ------------------------------------------------------------ convenience

class Solver:
    """Owns a tma_solver handle and allocates outputs with torch."""

    def __init__(self, problem, device=None):
        torch = _torch()
        self.problem = problem
        self.N, self.S, self.L, self.M, self.H = (int(_get(problem, n)) for n in ("N", "S", "L", "M", "H"))
        self.J_max = int(_get(problem, "J_max"))
        ls = _get(problem, "L_sched", None)
        # particles after the last iteration (the set the selection chooses from)
        self.L_final = int(ls[self.J_max - 1]) if ls is not None else self.L
        self.sep_mode = int(_get(problem, "sep_mode"))
        self.grid = tuple(int(v) for v in _get(problem, "grid"))
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.h = tma_create(problem)

    def close(self):
        if getattr(self, "h", None):
            tma_destroy(self.h)
            self.h = None

    __del__ = close

    def set_state(self, x0=None, mpc_step=0):
        tma_set_state(self.h, x0, mpc_step)

    def set_finished(self, mask):
        tma_set_finished(self.h, mask)

    def status(self):
        return tma_get_status(self.h, self.N)

    def wind_field(self):
        torch = _torch()
        P = self.grid[0] * self.grid[1] * self.grid[2]
        out = torch.empty((self.M, self.H, P, 2), dtype=torch.float32, device=self.device)
        tma_wind_field(self.h, out)
        return out

    def rollout_cost(self, u, J, soft=False):
        torch = _torch()
        L = u.shape[0]
        cbar = torch.empty((self.N, L), dtype=torch.float32, device=self.device)
        cs = torch.empty_like(cbar) if soft else None
        tma_rollout_cost(self.h, u, J, cbar, cs)
        return cbar, cs

    def sample_costs(self, L, soft=False):
        torch = _torch()
        out = torch.empty((self.M, self.N, L), dtype=torch.float32, device=self.device)
        tma_sample_costs(self.h, out, soft)
        return out

    def live_steps(self):
        return tma_live_steps(self.h)

    def move(self, u, anc, J):
        torch = _torch()
        out = torch.empty_like(u)
        tma_move(self.h, u, anc, J, out)
        return out

    def init_controls(self, L=None):
        torch = _torch()
        L = self.L if L is None else L
        u = torch.empty((L, self.N, self.S, 3), dtype=torch.float32, device=self.device)
        tma_init_controls(self.h, u)
        return u

    def solve(self):
        torch = _torch()
        best_u = torch.empty((self.N, self.S, 3), dtype=torch.float32, device=self.device)
        st, cost = tma_solve(self.h, best_u)
        return best_u, cost, st

    def best_index(self):
        return tma_best_index(self.h)

    def particles(self, L=None):
        torch = _torch()
        L = self.L_final if L is None else L
        out = torch.empty((L, self.N, self.S, 3), dtype=torch.float32, device=self.device)
        return tma_get_particles(self.h, out)

    def rollout_grad(self, u, J, cbar=False):
        """(cost [L], grad [L][N][S][3], per-aircraft soft means [N][L] or None)."""
        torch = _torch()
        L = u.shape[0]
        cost = torch.empty(L, dtype=torch.float32, device=self.device)
        grad = torch.empty_like(u)
        cb = torch.empty((self.N, L), dtype=torch.float32, device=self.device) if cbar else None
        tma_rollout_grad(self.h, u, J, cost, grad, cb)
        return cost, grad, cb

    def set_wind_stream(self, stream):
        tma_set_wind_stream(self.h, stream)

    def set_move(self, kind, eps0=1.0):
        tma_set_move(self.h, kind, eps0)

    def mh_stats(self):
        return tma_mh_stats(self.h, self.J_max - 1)


def lse(cbar, kappa):
    torch = _torch()
    nseg, L = cbar.shape
    wt = torch.empty((nseg, L), dtype=torch.float64, device=cbar.device)
    lm = torch.empty(nseg, dtype=torch.float64, device=cbar.device)
    ws = torch.empty(nseg, dtype=torch.float64, device=cbar.device)
    tma_lse(cbar, kappa, wt, lm, ws)
    return wt, lm, ws


def resample(wtilde, seed, scenario_id, J, mpc_step):
    torch = _torch()
    anc = torch.empty(wtilde.shape, dtype=torch.int32, device=wtilde.device)
    st = tma_resample(wtilde, seed, scenario_id, J, mpc_step, anc)
    return anc, st


def select(cbar):
    torch = _torch()
    dev = cbar.device
    best = torch.empty(1, dtype=torch.int64, device=dev)
    bs = torch.empty(1, dtype=torch.float64, device=dev)
    ni = torch.empty(1, dtype=torch.int32, device=dev)
    tma_select(cbar, best, bs, ni)
    return int(best.item()), float(bs.item()), int(ni.item())
