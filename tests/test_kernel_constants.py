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


# ---- the normalisation's exponential (exp_table.h, exp_fixed in resample.cu)

def _exp_table():
    src = open(os.path.join(CSRC, "exp_table.h")).read()
    C1 = int(re.search(r"kExpC1 = (-?\d+)LL;", src).group(1))
    C2 = int(re.search(r"kExpC2 = (-?\d+)LL;", src).group(1))
    body = src[src.index("kExp2Frac63[256] = {"):]
    tab = [int(v, 16) for v in re.findall(r"0x([0-9a-f]{16})ull", body)]
    return C1, C2, tab


def test_exp_table_is_the_generator_output():
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    out = subprocess.run([sys.executable, os.path.join(CSRC, "gen_exp_table.py")], capture_output=True,
                         text=True, check=True).stdout
    assert out.strip() == open(os.path.join(CSRC, "exp_table.h")).read().strip()
    C1, C2, tab = _exp_table()
    assert len(tab) == 256 and tab[0] == 1 << 63 and all(t < 1 << 64 for t in tab)
    # every entry within half a unit of 2^(j/256) 2^63, checked against numpy's
    # exp2 (within one ulp) and, for a few entries, 60-digit decimals
    j = np.arange(256)
    assert np.all(np.abs(np.array(tab, dtype=np.float64) - np.exp2(j / 256.0 + 63)) <= 2.0 ** 11)
    for jj in (1, 77, 128, 255):
        exact = Decimal(2) ** (Decimal(jj) / 256) * Decimal(2) ** 63
        assert abs(Decimal(tab[jj]) - exact) <= Decimal("0.5")
    # ln2/256 at the scale 2^53 = C1 + C2 / 2^32 within 2^-33
    step53 = Decimal(2).ln() / 256 * Decimal(2) ** 53
    assert abs(Decimal(C1) + Decimal(C2) / Decimal(2) ** 32 - step53) <= Decimal(2) ** -33
    assert abs(C2) < 1 << 31


def _kappa_times(d, kappa):
    """|d| kappa at the scale 2^53, truncated, with the kernel's integers."""
    d = np.float32(d)
    if d == 0:
        return 0
    u = int(np.array(d).view(np.uint32))
    E = (u >> 23) & 0xFF
    M = (u & 0x7FFFFF) | 0x800000
    mant, ex = np.frexp(kappa)                  # kappa = mant 2^ex, mant in [0.5, 1)
    K = int(mant * 2.0 ** 53)
    e = int(ex) - 53
    sh = 150 - 53 - E - e
    # the kernel forms floor(M K / 2^13) first: every in-range result has sh >= 13
    assert sh >= 13 or (M * K) >> sh >= 746 << 53
    return (M * K) >> sh if sh < 77 else 0


def exp_fixed(cmin, c, kappa, tail=True, half=True):
    """The kernel's steps: FP32 where it uses FP32, its 64-bit integers exactly
    (Python integers; the 128-bit products' high halves by shifts).  tail and
    half off plant a mistake: the tail of ln2/256 dropped, r^2 for r^2/2."""
    f32 = np.float32
    cmin, c = f32(cmin), f32(c)
    xf = f32(f32(min(kappa, 3.0e38)) * f32(cmin - c))
    if not xf > f32(-746.0):
        return 0.0
    dh = f32(cmin - c)
    bb = f32(dh - cmin)
    dl = f32(f32(cmin - f32(dh - bb)) + f32(f32(-c) - bb))
    ah, al = _kappa_times(dh, kappa), _kappa_times(abs(dl), kappa)
    x53 = (-ah if dh < 0 else ah) + (-al if dl < 0 else al)
    C1, C2, tab = _exp_table()
    k = int(np.rint(f32(xf * f32(369.329794))))
    r53 = x53 - k * C1 - (((k * C2) >> 32) if tail else 0)
    r62 = r53 * 512
    s62 = ((abs(r62) * abs(r62)) >> 64) << (1 if half else 2)
    rf = f32(f32(int(r53 >> 13)) * f32(2.0 ** -40))
    t = f32(f32(f32(rf * rf) * rf) * f32(f32(rf * f32(1.0 / 24.0)) + f32(1.0 / 6.0)))
    t62 = int(np.rint(f32(t * f32(2.0 ** 60)))) * 4
    e62 = (1 << 62) + r62 + s62 + t62
    y61 = (tab[k & 255] * e62) >> 64
    p = y61.bit_length() - 1
    shm = p - 52
    m = (y61 + (1 << (shm - 1))) >> shm
    E = 1023 + (k >> 8) + (p - 61)
    if E < -60:
        return 0.0
    return float(np.ldexp(float(m), E - 1023 - 52))


def test_exp_fixed_meets_its_error_bound():
    """Relative error below 1e-15 against exp of the exact x = kappa (cmin - c)
    (60-digit decimals) over the range the weights use, from 0 down to -745:
    table boundaries, half-way points, the subnormal end; exactly 1 at the
    minimum."""
    from decimal import Decimal, getcontext
    from fractions import Fraction
    getcontext().prec = 60
    rng = np.random.default_rng(3)
    cases = []
    for kappa in (0.37, 11.0, 23.7, 708.0):
        cmin = np.float32(rng.uniform(0, 3))
        for c in np.float32(cmin + rng.exponential(1.0, 600) * (40.0 / kappa)):
            cases.append((cmin, c, kappa))
    # x on multiples of ln2/256 and half-way between them (c chosen in FP32 near them)
    for kstep in (1, 2, 255, 256, 257, 5000, 100000, 275000):
        for dd in (0.0, 0.5, -0.5):
            x = -(kstep + dd) * np.log(2.0) / 256
            cases.append((np.float32(0.0), np.float32(-x / 3.0), 3.0))
    # x down to the cut-off, where the product's shift is smallest
    for kappa in (1.0, 1.37, 708.0, 3.3e-5):
        for xx in (-745.9, -700.0, -512.5, -511.9):
            cases.append((np.float32(0.0), np.float32(-xx / kappa), kappa))
    cases += [(np.float32(1.5), np.float32(1.5), 708.0), (np.float32(0.0), np.float32(248.0), 3.0),
              (np.float32(2.0), np.float32(2.0 + 744.0 / 11.0), 11.0), (np.float32(-4.0), np.float32(9.0), 5.5)]
    worst = 0.0
    for cmin, c, kappa in cases:
        got = exp_fixed(cmin, c, kappa)
        x = Fraction(kappa) * (Fraction(float(cmin)) - Fraction(float(c)))
        ref = (Decimal(x.numerator) / Decimal(x.denominator)).exp()
        if ref > Decimal("1e-300"):
            worst = max(worst, abs(Decimal(got) - ref) / ref)
        else:
            assert Decimal(got) <= ref * 2 + Decimal("1e-323")
    assert worst < Decimal("1e-15"), worst
    assert exp_fixed(np.float32(1.5), np.float32(1.5), 708.0) == 1.0
    assert exp_fixed(np.float32(0.0), np.float32(1e30), 1.0) == 0.0
    # kappa beyond the FP32 range: 1 at the minimum, 0 elsewhere; kappa tiny: 1
    assert exp_fixed(np.float32(2.0), np.float32(2.0), 1e300) == 1.0
    assert exp_fixed(np.float32(2.0), np.float32(2.5), 1e300) == 0.0
    assert exp_fixed(np.float32(2.0), np.float32(9.0), 1e-300) == 1.0


def _worst_rel_error(cases, **kw):
    from decimal import Decimal, getcontext
    from fractions import Fraction
    getcontext().prec = 60
    worst = Decimal(0)
    for cmin, c, kappa in cases:
        got = exp_fixed(cmin, c, kappa, **kw)
        x = Fraction(kappa) * (Fraction(float(cmin)) - Fraction(float(c)))
        ref = (Decimal(x.numerator) / Decimal(x.denominator)).exp()
        if ref > Decimal("1e-300"):
            worst = max(worst, abs(Decimal(got) - ref) / ref)
    return worst


def test_exp_fixed_emulation_catches_planted_mistakes():
    """The error bound fails when a step of the emulated algorithm is wrong:
    the tail of ln2/256 dropped, or the r^2/2 term taken as r^2."""
    rng = np.random.default_rng(5)
    cases = [(np.float32(0.0), np.float32(c), 23.7) for c in rng.uniform(0.5, 30.0, 200)]
    assert _worst_rel_error(cases) < 1e-15
    assert _worst_rel_error(cases, tail=False) > 1e-13
    assert _worst_rel_error(cases, half=False) > 1e-8
