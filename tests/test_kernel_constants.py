"""Constants the kernels carry: the arctangent polynomial of the rollout is the
fit that paper_1506_02869_gb300/csrc/fit_atan.py computes, and its FP32
evaluation stays within 1.2e-7 rad of arctan on [0, 1] (no GPU needed)."""
import os
import re
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1506_02869_gb300", "csrc")


def kernel_coefficients():
    src = open(os.path.join(CSRC, "rollout_tile.cuh")).read()
    body = src[src.index("atan2_poly"):src.index("return copysignf(a, y);")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return vals[::-1]          # Horner order in the source: highest degree first


def test_atan_polynomial_is_the_fit():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "fit_atan.py"), "8"], capture_output=True,
                         text=True, check=True).stdout
    err = float(re.search(r"max abs error \(FP32 evaluation\) (\S+)", out).group(1))
    fit = [float(v) for v in re.findall(r"^\s+([-+]?\d\.\d+e[-+]\d+)$", out, re.M)]
    assert len(fit) == 9 and err < 1.2e-7
    assert np.allclose(kernel_coefficients(), fit, rtol=1e-9, atol=0)


def test_atan2_octants_in_fp32():
    """The kernel's octant reconstruction, evaluated in FP32 with numpy."""
    c = np.array(kernel_coefficients(), np.float32)
    rng = np.random.default_rng(0)
    y = rng.normal(size=200000).astype(np.float32) * np.float32(3e4)
    x = rng.normal(size=200000).astype(np.float32) * np.float32(3e4)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    t = (mn / mx).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.float32(c[8])
    for k in range(7, -1, -1):
        p = (p * s + c[k]).astype(np.float32)
    a = (t * p).astype(np.float32)
    a = np.where(ay > ax, np.float32(np.pi / 2) - a, a).astype(np.float32)
    a = np.where(x < 0, np.float32(np.pi) - a, a).astype(np.float32)
    a = np.copysign(a, y)
    assert np.abs(a.astype(np.float64) - np.arctan2(y.astype(np.float64), x.astype(np.float64))).max() < 5e-7


# ---- the normalisation's FP64 exponential (exp_table.h, exp_nonpos in resample.cu)

def _exp_table():
    src = open(os.path.join(CSRC, "exp_table.h")).read()
    L1 = float.fromhex(re.search(r"kExpL1 = (\S+);", src).group(1))
    L2 = float.fromhex(re.search(r"kExpL2 = (\S+);", src).group(1))
    body = src[src.index("kExp2Frac[256] = {"):]
    tab = [float.fromhex(v) for v in re.findall(r"(0x1\.[0-9a-f]+p[+-]\d+)", body)]
    return L1, L2, tab


def test_exp_table_is_the_generator_output():
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp_table.py")], capture_output=True,
                         text=True, check=True).stdout
    assert out.strip() == open(os.path.join(CSRC, "exp_table.h")).read().strip()
    L1, L2, tab = _exp_table()
    assert len(tab) == 256 and tab[0] == 1.0
    j = np.arange(256)
    # every entry within half an ulp of 2^(j/256) (numpy's exp2 is within one)
    assert np.all(np.abs(np.array(tab) - np.exp2(j / 256.0)) <= np.spacing(np.array(tab)))
    assert abs((L1 + L2) - np.log(2.0) / 256) < 1e-18 and abs(L2) < 2.0 ** -60


def _fma(a, b, c):
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _exp_nonpos(x, xf, L1, tab):
    """The kernel's steps: FP64 where it uses FP64 (fused multiply-adds
    emulated exactly), FP32 where it uses FP32; the reduction takes the head L1
    of ln2/256 alone."""
    f32 = np.float32
    if not np.float32(xf) > np.float32(-746.0):
        return 0.0
    k = int(np.rint(f32(xf) * f32(369.329794)))
    r = _fma(-float(k), L1, x)
    rf = f32(r)
    h = f32(f32(f32(rf * f32(1.0 / 24.0)) + f32(1.0 / 6.0)) * rf) + f32(0.5)
    small = f32(f32(rf * rf) * f32(h))
    p = r + float(small)
    t = tab[k & 255]
    y = _fma(t, p, t)
    return float(np.ldexp(y, k >> 8))


def test_exp_nonpos_meets_its_error_bound():
    """Relative error below 5e-13 against the correctly rounded exp over the
    range the weights use (kappa (cmin - c) from 0 down to -740), including
    table boundaries and the subnormal end."""
    import math
    L1, _, tab = _exp_table()
    rng = np.random.default_rng(3)
    kappa = 11.0
    c = np.float32(rng.uniform(0, 60, 3000))
    xs = [(-kappa * float(ci), np.float32(kappa) * (np.float32(0) - ci)) for ci in c]
    # multiples of ln2/256 and half-way points, and the far end
    for k in (1, 2, 255, 256, 257, 5000, 100000, 275000):
        for d in (0.0, 0.5, -0.5, 1e-9):
            x = -(k + d) * math.log(2.0) / 256
            xs.append((x, np.float32(x)))
    xs += [(0.0, np.float32(0.0)), (-744.0, np.float32(-744.0)), (-700.0, np.float32(-700.0))]
    worst = 0.0
    for x, xf in xs:
        got = _exp_nonpos(x, xf, L1, tab)
        ref = math.exp(x)
        if ref > 1e-300:
            worst = max(worst, abs(got - ref) / ref)
        else:
            assert abs(got - ref) <= 2 * 5e-324 + 1e-12 * ref
    assert worst < 5e-13, worst
    assert _exp_nonpos(0.0, np.float32(0.0), L1, tab) == 1.0
