"""Coefficients of the rollout's arctangent: atan(t) ~ t P(t^2) on [0, 1].

P is fitted by weighted least squares on Chebyshev nodes of t (relative error
of atan(t) / t, which approximates the minimax fit); the printed FP32 Horner
evaluation error is the figure quoted beside the coefficients in
rollout_tile.cuh.  Run: python fit_atan.py [degree]
"""
import sys

import numpy as np

deg = int(sys.argv[1]) if len(sys.argv) > 1 else 8
n = 4000
t = np.cos(np.pi * (np.arange(n) + 0.5) / n) * 0.5 + 0.5      # Chebyshev nodes on [0, 1]
t = np.concatenate([t, [1.0]])
s = t * t
f = np.where(t > 0, np.arctan(t) / np.where(t > 0, t, 1.0), 1.0)
A = np.vander(s, deg + 1, increasing=True)
c, *_ = np.linalg.lstsq(A, f, rcond=None)
# evaluate in FP32 Horner as the kernel does
tt = np.linspace(0.0, 1.0, 2_000_001, dtype=np.float32)
ss = (tt * tt).astype(np.float32)
p = np.float32(c[-1])
for k in range(deg - 1, -1, -1):
    p = (p * ss + np.float32(c[k])).astype(np.float32)
approx = (tt * p).astype(np.float32)
err = np.abs(approx.astype(np.float64) - np.arctan(tt.astype(np.float64)))
print("degree", deg, "max abs error (FP32 evaluation)", err.max())
print("coefficients (s^0 .. s^%d):" % deg)
for k, v in enumerate(c):
    print("  %.9e" % v)
