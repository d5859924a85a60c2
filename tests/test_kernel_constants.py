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
