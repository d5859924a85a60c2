"""Pins of the oracle's random streams (Philox4x32-10, 23-bit uniforms,
Box-Muller) against a library implementation and against statistics."""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O
import scenarios as S


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            path = os.path.join(d, name) if d else name
            try:
                return ctypes.CDLL(path)
            except OSError:
                continue
    return None


def _curand_host_philox(seed, offset_words, n_words):
    """Raw 32-bit outputs of cuRAND's host Philox4_32_10 generator."""
    lib = _curand()
    if lib is None:
        pytest.skip("cuRAND host library not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


# cuRAND's host generator emits block b of its stream from the counter
# (b div 2^16 mod 2^32, b div 2^48, b mod 2^16, 0) under key (seed lo, seed hi);
# its generator offset moves b.  This reaches counter words c0, c1, c2 and both
# key words of the block function.
@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 20150601])
def test_philox_matches_curand_host_stream(seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = _curand_host_philox(seed, 0, 4 * 70000).reshape(-1, 4)
    for b in list(range(0, 70000, 997)) + [65535, 65536, 65537]:
        ctr = [(b >> 16) & 0xFFFFFFFF, b >> 48, b & 0xFFFF, 0]
        assert O.philox(ctr, key) == list(got[b]), (seed, b)


@pytest.mark.parametrize("b", [(1 << 48) + 5, (3 << 48) + (7 << 16) + 9, (1 << 40) + 123,
                               (0xFFFF << 16) | 0xFFFF, ((1 << 14) - 1 << 48) | (0xFFFFFFFF << 16)])
def test_philox_matches_curand_high_counter_words(b):
    seed = 0xDEADBEEFCAFEF00D
    got = _curand_host_philox(seed, 4 * b, 4)
    ctr = [(b >> 16) & 0xFFFFFFFF, (b >> 48) & 0xFFFFFFFF, b & 0xFFFF, 0]
    assert O.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]) == list(got)


def test_uniform23_exact_in_float32_and_open_interval():
    xs = [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]
    for x in xs:
        u = O.uniform23(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u       # representable in FP32: both sides see it exactly
    assert O.uniform23(0) == 2.0 ** -24
    assert O.uniform23(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # only the top 23 bits matter
    assert O.uniform23(0x12345600) == O.uniform23(0x123457FF)
    # uniform on the 2^23 cells: mean and variance of U(0,1)
    rng = np.random.default_rng(3)
    u = np.array([O.uniform23(int(x)) for x in rng.integers(0, 2 ** 32, 40000, dtype=np.uint64)])
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005


def test_box_muller_is_standard_normal():
    rng = np.random.default_rng(7)
    w = rng.integers(0, 2 ** 32, size=(60000, 2), dtype=np.uint64)
    z = np.array([O.box_muller(int(a), int(b)) for a, b in w])
    z0, z1 = z[:, 0], z[:, 1]
    for v in (z0, z1):
        assert abs(v.mean()) < 0.02
        assert abs(v.std() - 1.0) < 0.02
        assert stats.kstest(v, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 0.02     # the pair is independent
    assert abs(stats.kurtosis(z0)) < 0.1


def test_box_muller_inverts_to_its_uniforms():
    """The inverse of the polar transform recovers the two uniforms: the
    squared radius z0^2 + z1^2 = -2 ln u_a and the angle atan2(z1, z0) = 2 pi u_b
    (mod 2 pi), u_a from the first word and u_b from the second.  A swapped
    word, a swapped sine and cosine, a sign or a factor in the radius fails."""
    rng = np.random.default_rng(11)
    words = [(int(a), int(b)) for a, b in rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64)]
    words += [(0, 0), (0xFFFFFFFF, 0x80000000), (0x80000000, 0xFFFFFFFF), (12345, 0x40000000)]
    for xa, xb in words:
        z0, z1 = O.box_muller(xa, xb)
        ua, ub = O.uniform23(xa), O.uniform23(xb)
        assert math.exp(-0.5 * (z0 * z0 + z1 * z1)) == pytest.approx(ua, rel=1e-12, abs=1e-300)
        ang = math.atan2(z1, z0) / (2 * math.pi) % 1.0
        d = abs(ang - ub)
        assert min(d, 1.0 - d) < 1e-12, (xa, xb, ang, ub)


def test_draw_counter_layout_and_scenario_key():
    p = S.config1().copy(mpc_step=3, scenario_id=5)
    s = (p.seed + 5 * 0x9E3779B97F4A7C15) & (2 ** 64 - 1)
    key = [s & 0xFFFFFFFF, s >> 32]
    got = O.draw(p, 11, 2 | (7 << 8), 9, 1, 4)
    assert got == O.philox([11, 2 | (7 << 8), 9 | (1 << 24), 4 | (3 << 16)], key)
    # distinct streams, samples and iterations give distinct blocks
    seen = {tuple(O.draw(p, 0, 0, 0, st, J)) for st in range(9) for J in range(4)}
    assert len(seen) == 36
