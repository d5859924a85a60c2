// Device utilities of the CUDA path: counter-based random numbers and
// compensated accumulation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tma {

// One Philox round: the two 32x32->64 bit products, each formed by one widening
// multiply, both halves used.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                      (uint32_t)p0);
}

// Philox4x32-10 block function (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 bit
// multiplies with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        c = philox_round(c, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same block function with the round keys given: rk[2r], rk[2r + 1] =
// (k0, k1) + r (0x9E3779B9, 0xBB67AE85), the key of round r (a kernel that has
// them in its parameter space reads them as constant operands instead of
// forming them round by round).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, rk[2 * r], rk[2 * r + 1]);
    return c;
}

// Counter layout of every random stream: (c0, c1, q | stream << 24, J | mpc << 16).
__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                      uint32_t q, uint32_t stream, uint32_t J, uint32_t mpc)
{
    return philox4x32_10(make_uint4(c0, c1, (q & 0xFFFFFFu) | (stream << 24),
                                    (J & 0xFFFFu) | (mpc << 16)),
                         k0, k1);
}

__device__ __forceinline__ uint4 draw_rk(const uint32_t *rk, uint32_t c0, uint32_t c1, uint32_t q,
                                         uint32_t stream, uint32_t J, uint32_t mpc)
{
    return philox4x32_10_rk(make_uint4(c0, c1, (q & 0xFFFFFFu) | (stream << 24), (J & 0xFFFFu) | (mpc << 16)),
                            rk);
}

// Uniform in (0, 1) from the top 23 bits: ((x >> 9) + 1/2) / 2^23, exact in FP32.
__device__ __forceinline__ float uniform23(uint32_t x)
{
    return __fmaf_rn((float)(x >> 9), 1.0f / 8388608.0f, 1.0f / 16777216.0f);
}

// Box-Muller transform of two words into two independent standard normals.
__device__ __forceinline__ float2 box_muller(uint32_t xa, uint32_t xb)
{
    const float r = sqrtf(-2.0f * logf(uniform23(xa)));
    float s, c;
    sincospif(2.0f * uniform23(xb), &s, &c);
    return make_float2(r * c, r * s);
}

// The same transform with the hardware approximations of log, sin and cos
// (absolute errors near 2^-21 on these argument ranges); the angle is taken in
// [-pi, pi) so that no range reduction is needed.  Near u = 1 the approximate
// logarithm can come out just above 0; the radius argument is clamped at 0 so
// that it never yields NaN.
__device__ __forceinline__ float2 box_muller_fast(uint32_t xa, uint32_t xb)
{
    const float r = sqrtf(fmaxf(-2.0f * __logf(uniform23(xa)), 0.0f));
    float s, c;
    __sincosf(fmaf(6.28318530717958647692f, uniform23(xb), -3.14159265358979323846f), &s, &c);
    return make_float2(-r * c, -r * s);
}

// sin and cos of an angle of moderate size: reduced to [-pi, pi] with one
// rounding, then the hardware approximation.
__device__ __forceinline__ void sincos_reduced(float a, float *s, float *c)
{
    const float r = fmaf(-6.28318530717958647692f, rintf(a * 0.159154943091895335769f), a);
    __sincosf(r, s, c);
}

// Kahan-compensated FP32 accumulator.
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float y)
    {
        const float yy = y - c;
        const float t = s + yy;
        c = (t - s) - yy;
        s = t;
    }
};

// Absolute angular distance of an angle difference, in [0, pi].
__device__ __forceinline__ float angdist(float a)
{
    const float twopi = 6.28318530717958647692f;
    const float r = a - twopi * rintf(a * (1.0f / twopi));
    return fabsf(r);
}

// 128-bit unsigned product and comparison helpers (fixed-point CDF).
struct U128 {
    unsigned long long hi, lo;
};
__device__ __forceinline__ U128 mul64x64(unsigned long long a, unsigned long long b)
{
    return U128{__umul64hi(a, b), a * b};
}
__device__ __forceinline__ bool lt128(U128 a, U128 b)
{
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

}  // namespace tma
