"""The C-ABI library loads and exports every entry point of include/tma_smc.h;
the Python mirror of its structures matches the C layout; invalid arguments
are rejected before any CUDA call.  No GPU needed."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1506_02869_gb300 as pkg
import scenarios as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tma_smc.h")


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tma_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIBPATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tma_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(pkg.EXPORTS) == names
    for n in names:
        assert callable(getattr(pkg, n, None)) or n in (
            "tma_status_str", "tma_last_error_string", "tma_launch_count", "tma_lse_workspace",
            "tma_lse_resample_workspace", "tma_resample_workspace", "tma_select_workspace"), n
        getattr(lib, n)


def test_struct_layout_matches_header(tmp_path):
    fields = {"tma_problem": (pkg.TmaProblem, ["N", "dt", "seed", "scenario_id", "box_lo", "grid",
                                               "wind_sigma", "sep_mode", "sp_beta", "ctrl_lo",
                                               "alpha_dep", "w_noise", "pop_n", "pop_lo",
                                               "popdense", "P_runway", "beta_f", "wind_mode",
                                               "sample_mode", "L_sched", "rolling"]),
              "tma_aircraft": (pkg.TmaAircraft, ["type", "t_enter", "x0", "theta_F", "m_empty", "Tmax"]),
              "tma_state": (pkg.TmaState, ["x", "m"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(){"]
    for st, (_, fs) in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(c)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for st, (cls, fs) in fields.items():
        assert int(out[st]) == C.sizeof(cls), st
        for f in fs:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_status_strings(lib):
    for s in range(8):
        assert lib.tma_status_str(s).decode() not in ("", "unknown status")


def _create(p):
    s, arr, keep = pkg.problem_struct(p)
    h = C.c_void_p()
    st = pkg.lib().tma_create(C.byref(s), arr, C.byref(h))
    return st, h


@pytest.mark.parametrize("change", [dict(N=0), dict(N=33), dict(L=0), dict(L=(1 << 22) + 1),
                                    dict(M=0), dict(H=0), dict(S=0), dict(grid=(1, 4, 4)),
                                    dict(grid=(4, 4, 17)), dict(sep_mode=3), dict(dt=0.0),
                                    dict(J_max=0), dict(mpc_step=1 << 16), dict(sep_h=0.0),
                                    dict(v_min=300.0), dict(wind_mode=2), dict(wind_mode=-1),
                                    dict(wind_mode=1, grid=(2, 2, 3)), dict(wind_mode=1, grid=(4, 4, 4)),
                                    dict(sample_mode=2), dict(sample_mode=-1),
                                    dict(L_sched=(1024,) * 9 + (0,)), dict(L_sched=(2048,) + (1024,) * 9),
                                    dict(rolling=2), dict(rolling=-1)])
def test_create_rejects_invalid_problems(lib, change):
    p = S.config1().copy(**change)
    if "N" in change and change["N"] > 2:
        p.aircraft = np.resize(p.aircraft, change["N"])
    st, h = _create(p)
    assert st == pkg.TMA_ERR_INVALID_ARG and not h.value


def test_stage_calls_reject_invalid_arguments(lib):
    L = lib
    null = C.c_void_p()
    assert L.tma_lse(null, 2, 10, 0.0, null, null, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_lse(null, 2, 10, 8.0, null, null, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample(null, 2, 10, 0, 0, 1 << 16, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample(null, 2, 10, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_select(null, 0, 10, null, null, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_rollout_cost(null, null, 1, 0, null, null, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_solve(null, null, None, null) == pkg.TMA_ERR_INVALID_ARG
    # empty inputs are valid no-ops
    assert L.tma_resample(null, 0, 10, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_OK
    assert L.tma_resample(null, 3, 0, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_OK
    # resampling to another count: both counts empty or both positive
    assert L.tma_resample_to(null, 2, 10, 0, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample_to(null, 2, 0, 5, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample_to(null, 2, 10, -1, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample_to(null, 2, 10, 7, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_resample_to(null, 0, 10, 7, 0, 0, 0, 0, null, null, 0, null) == pkg.TMA_OK
    # the fused weights + resampling call: kappa, counts and buffers checked first
    assert L.tma_lse_resample(null, 2, 10, 10, 0.0, 0, 0, 0, 0, null, null, null, null, 0, null) == \
        pkg.TMA_ERR_INVALID_ARG
    assert L.tma_lse_resample(null, 2, 10, 10, 8.0, 0, 0, 0, 0, null, null, null, null, 0, null) == \
        pkg.TMA_ERR_INVALID_ARG
    assert L.tma_lse_resample(null, 2, 10, 0, 8.0, 0, 0, 0, 0, null, null, null, null, 0, null) == \
        pkg.TMA_ERR_INVALID_ARG
    assert L.tma_lse_resample(null, 0, 10, 10, 8.0, 0, 0, 0, 0, null, null, null, null, 0, null) == pkg.TMA_OK
    assert L.tma_move_to(null, null, 4, null, 4, 0, null, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_set_finished(null, 0, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_get_status(null, None, None, null) == pkg.TMA_ERR_INVALID_ARG


def test_workspace_sizes(lib):
    for nseg, L in ((1, 1), (8, 65536), (24, 262144), (1, 1 << 22)):
        for f in (lib.tma_lse_workspace, lib.tma_resample_workspace):
            assert f(nseg, L) >= 16
        assert lib.tma_resample_workspace(nseg, L) >= lib.tma_resample_workspace(1, 1)
        assert lib.tma_lse_resample_workspace(nseg, L) >= \
            lib.tma_lse_workspace(nseg, L) + lib.tma_resample_workspace(nseg, L) - 16
    assert lib.tma_select_workspace(1 << 22) > 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIBPATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()


def test_batch_create_rejects_invalid_batches(lib):
    import scenarios as S
    ps = [S.shrink(p, L=64, M=2, H=10, J_max=2) for p in S.config5(n_scen=3)]
    structs = [pkg.problem_struct(p) for p in ps]

    def create(plist):
        n = len(plist)
        parr = (pkg.TmaProblem * max(n, 1))(*[s for s, _, _ in plist])
        aptrs = (C.POINTER(pkg.TmaAircraft) * max(n, 1))(
            *[C.cast(a, C.POINTER(pkg.TmaAircraft)) for _, a, _ in plist])
        h = C.c_void_p()
        return lib.tma_batch_create(parr, aptrs, n, C.byref(h)), h

    assert create([])[0] == pkg.TMA_ERR_INVALID_ARG
    bad = pkg.problem_struct(ps[1].copy(M=3))
    st, h = create([structs[0], bad])
    assert st == pkg.TMA_ERR_INVALID_ARG and not h.value
    bad_grid = pkg.problem_struct(ps[1].copy(grid=(8, 8, 4)))
    assert create([structs[0], bad_grid])[0] == pkg.TMA_ERR_INVALID_ARG
    # a particle schedule is for single solvers only
    sched = pkg.problem_struct(ps[1].copy(L_sched=(64, 32)))
    assert create([structs[0], sched])[0] == pkg.TMA_ERR_UNSUPPORTED
    assert lib.tma_batch_mpc(None, 1, 1, None) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_batch_rollout_cost(None, None, 0, None, None, None) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_batch_get_dispatch(None, None, None, None) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_batch_set_dispatch(None, 0) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_plant_step(None, None, None) == pkg.TMA_ERR_INVALID_ARG


def test_gradient_and_move_calls_reject_invalid_arguments(lib):
    null = C.c_void_p()
    L = lib
    assert L.tma_rollout_grad(null, null, 1, 0, null, null, null, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_set_move(null, pkg.TMA_MOVE_MALA, 1.0) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_mh_propose(null, null, null, 1, 0, 1.0, 1.0, 2, null, null, null) == \
        pkg.TMA_ERR_INVALID_ARG
    assert L.tma_mh_accept(null, null, null, null, null, null, null, null, 1, 0, 1.0, 1.0, 2, null,
                           null, null) == pkg.TMA_ERR_INVALID_ARG
    assert L.tma_mh_stats(null, None, None, 1, null) == pkg.TMA_ERR_INVALID_ARG


def test_profile_struct_has_every_stage():
    src = open(HEADER).read()
    n = int(re.search(r"#define TMA_N_STAGES (\d+)", src).group(1))
    assert len(pkg.TmaProfile._fields_[0][1]()) == n == len(pkg.STAGES)


def test_mpc_and_error_calls_reject_invalid_arguments(lib):
    null = C.c_void_p()
    assert lib.tma_mpc_run(null, 1, None, None, null) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_get_error(null, None, null) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_get_particles(null, null, 1, null) == pkg.TMA_ERR_INVALID_ARG
    assert lib.tma_set_wind_stream(null, 8) == pkg.TMA_ERR_INVALID_ARG
