import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scenarios as S  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) on a machine without a GPU only when
    # they were deselected by the caller; an explicit `-m gpu` run must fail
    # loudly if no device is present.
    pass


def one_aircraft(kind=1, **kw):
    """A single-aircraft record with plain A320-like coefficients."""
    a = np.zeros((), S.AIRCRAFT_DTYPE)
    base = dict(type=kind, x=0.0, y=0.0, z=3000.0, v=150.0, chi=0.0, m=60000.0,
                theta_F=0.0, Z=5000.0, v_D=200.0, m_empty=45000.0, S=122.6, CD0=0.024,
                CD2=0.0, Cf1=1.1e-5, Cf2=450.0, Tmin=0.0, Tmax=240e3)
    base.update(kw)
    for k, v in base.items():
        a[k] = v
    return a


def make_problem(aircraft, H=10, L=1, M=1, **kw):
    """A small problem around explicit aircraft, with turbulence off."""
    ac = np.zeros(len(aircraft), S.AIRCRAFT_DTYPE)
    for i, a in enumerate(aircraft):
        ac[i] = a
    base = dict(N=len(aircraft), H=H, L=L, M=M, J_max=1, turb_sigma=0.0,
                box_lo=(-50000.0, -50000.0, 0.0), box_hi=(50000.0, 50000.0, 10000.0),
                grid=(4, 4, 3), z_max=10000.0)
    base.update(kw)
    p = S.Problem(**base)
    p.aircraft = ac
    return p


def zero_wind(p):
    return np.zeros((p.M, p.H, p.n_grid, 2))


def controls(p, w=0.0, hdot=0.0, acc=0.0, L=1):
    u = np.zeros((L, p.N, p.S, 3))
    u[..., 0], u[..., 1], u[..., 2] = w, hdot, acc
    return u


ISA = lambda z: 1.225 * (1.0 - 2.2558e-5 * z) ** 4.2559  # noqa: E731


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)
