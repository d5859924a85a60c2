"""The resampling kernel's count arithmetic (`count_from_base` and the chunk
base in `res_expand`, paper_1506_02869_gb300/csrc/resample.cu), emulated on
the CPU step by step -- every FP32 operation correctly rounded from exact
rationals, the 64-bit products wrapping -- against exact integer counts.

Systematic resampling on the fixed-point CDF (Sec. 3.7): with the segment
total Q, the uniform r and Rhi = floor(r Q / 2^32), the number of particle
thresholds below an inclusive prefix S is #{l < Lout : l Q + Rhi < S Lout}.
The kernel takes it relative to its chunk's start Sb (count nb, residual
Eb = nb Q + Rhi - Sb Lout): an FP32 estimate of (D Lout - Eb)/Q for
D = S - Sb, then one exact test of D Lout - Eb - cr Q > 0 in wrapping 64-bit
arithmetic.  The cases put the real bound on and beside integers, take the
largest segment total (2^62) and the largest output count of this path
(2^20), and check the estimate's error against its bound: 6 2^-24 (Lout + 1)
to first order (Df and the ratio Lout/Q within 2^-23 and 3 2^-24 relative, eb
within 5 2^-24, one rounding of the fused result), taken here as
7 2^-24 (Lout + 1), below 1/2 for Lout <= 2^20 as the count needs.  No GPU."""
import math
import random
from fractions import Fraction

M64 = (1 << 64) - 1


def est_bound(Lout):
    return Fraction(7, 1 << 24) * (Lout + 1)


def f32(x):
    """x (a Fraction or int) rounded to the nearest FP32 value, ties to even."""
    x = Fraction(x)
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = a / Fraction(2) ** (e - 23)          # in [2^23, 2^24)
    m = math.floor(q)
    rem = q - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return s * Fraction(m) * Fraction(2) ** (e - 23)


def u64_to_float(v):
    # fmaf(float(v >> 32), 2^32, float(v & 0xffffffff)): one rounding of the sum
    return f32(f32(v >> 32) * (1 << 32) + f32(v & 0xFFFFFFFF))


def exact_count(S, Q, Rhi, Lout):
    x = S * Lout - Rhi
    if x <= 0:
        return 0
    return min(Lout, -(-x // Q))


def chunk_base(Sb, Q, Rhi, Lout):
    nb = exact_count(Sb, Q, Rhi, Lout)
    Eb = (nb * Q + Rhi - Sb * Lout) & M64        # the kernel keeps the low 64 bits
    eb = f32(u64_to_float(Eb) / u64_to_float(Q))
    return nb, Eb, eb


def kernel_count(D, nb, Eb, eb, Q, Lout, ratio, diff_test=True, with_eb=True, half=True):
    """count_from_base as the kernel evaluates it (the switches plant mistakes)."""
    est = f32(u64_to_float(D) * ratio - (eb if with_eb else 0))
    cr = max(math.ceil(f32(est - Fraction(1, 2))) if half else math.ceil(est), 0)
    c = nb + cr
    if c >= Lout:
        return Lout, est
    if not diff_test:
        return c, est
    diff = (D * Lout - (Eb if with_eb else 0) - cr * Q) & M64
    if diff >> 63:
        diff -= 1 << 64
    return c + (1 if diff > 0 else 0), est


def make_cases(seed, n):
    rnd = random.Random(seed)
    cases = []
    for k in range(n):
        Q = rnd.choice([rnd.randint(1, 1 << 20), rnd.randint(1, 1 << 62), (1 << 62) - rnd.randint(0, 1 << 20),
                        1 << 62, rnd.randint(1, 7)])
        Lout = rnd.choice([1, 2, 3, rnd.randint(1, 1 << 20), 1 << 20, (1 << 20) - 1, 262144])
        r = rnd.choice([0, rnd.getrandbits(32), 0xFFFFFFFF])
        Rhi = (r * Q) >> 32
        Sb = rnd.choice([0, rnd.randint(0, Q), Q])
        if k % 3 == 0:
            # S with its real bound on or beside an integer n
            n = rnd.randint(0, Lout)
            S = -(-(n * Q + Rhi) // Lout) + rnd.choice([-1, 0, 1])
            S = min(max(S, Sb), Q)
        else:
            S = rnd.randint(Sb, Q)
        cases.append((Q, Lout, Rhi, Sb, S))
    return cases


def mismatches(cases, **kw):
    bad = 0
    for Q, Lout, Rhi, Sb, S in cases:
        nb, Eb, eb = chunk_base(Sb, Q, Rhi, Lout)
        ratio = f32(Fraction(f32(Lout)) / u64_to_float(Q))
        got, _ = kernel_count(S - Sb, nb, Eb, eb, Q, Lout, ratio, **kw)
        bad += got != exact_count(S, Q, Rhi, Lout)
    return bad


def test_chunk_base_residual_fits_below_the_total():
    for Q, Lout, Rhi, Sb, S in make_cases(1, 3000):
        nb, Eb, _ = chunk_base(Sb, Q, Rhi, Lout)
        assert 0 <= nb * Q + Rhi - Sb * Lout < Q            # so its low 64 bits are the value
        assert Eb == nb * Q + Rhi - Sb * Lout


def test_counts_equal_the_exact_counts_and_the_estimate_meets_its_bound():
    cases = make_cases(2, 6000)
    for Q, Lout, Rhi, Sb, S in cases:
        nb, Eb, eb = chunk_base(Sb, Q, Rhi, Lout)
        ratio = f32(Fraction(f32(Lout)) / u64_to_float(Q))
        D = S - Sb
        got, est = kernel_count(D, nb, Eb, eb, Q, Lout, ratio)
        assert got == exact_count(S, Q, Rhi, Lout), (Q, Lout, Rhi, Sb, S)
        x_rel = Fraction(D * Lout - (nb * Q + Rhi - Sb * Lout), Q)
        assert abs(est - x_rel) <= est_bound(Lout), (Q, Lout, Sb, S, float(est - x_rel))
    assert est_bound(1 << 20) < Fraction(1, 2)


def test_the_cases_catch_planted_mistakes():
    cases = make_cases(3, 3000)
    assert mismatches(cases) == 0
    assert mismatches(cases, diff_test=False) > 0        # the estimate alone is not enough
    assert mismatches(cases, with_eb=False) > 0          # the chunk's residual dropped
    assert mismatches(cases, half=False) > 0             # ceil(est) in place of ceil(est - 1/2)
