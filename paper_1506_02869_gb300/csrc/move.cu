// Perturbation of the resampled controls (Algorithm 1) and their uniform
// initialisation (Sec. 3.2).
//
// One thread per (particle l, aircraft i), aircraft fastest, so that a warp
// writes a contiguous run of u_out[l][i][S*3].  The parent record
// u[anc[i][l]][i] is gathered with 16-byte loads (S*3 = 12 floats = 3 x float4
// when S = 4); the Gaussian noise comes from random stream 1.
#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {

namespace {

struct MoveC {
    int N, nc;             // nc = S*3 controls per (particle, aircraft)
    float lo[3], hi[3], sigma[3];
    uint32_t key0, key1;
    uint32_t rk[20];       // Philox round keys of (key0, key1)
};

__device__ __forceinline__ float clip(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// kNC: the number of controls per (particle, aircraft) when fixed at compile
// time (12 = four segments: the loop unrolls and the per-control constants
// become fixed operands), 0 when taken from C.nc.
template <bool kVec, int kNC = 0>
__global__ void __launch_bounds__(256) move_kernel(const MoveC C, const DynState *__restrict__ dyn,
                                                   const float *__restrict__ u,
                                                   const int32_t *__restrict__ anc, long long L,
                                                   long long Lin, int J, float *__restrict__ u_out,
                                                   unsigned int *__restrict__ err)
{
    // L children from Lin parents
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * C.N) return;
    const long long l = t / C.N;
    const int i = (int)(t - l * C.N);
    int a = __ldg(anc + (size_t)i * L + l);
    if ((unsigned long long)a >= (unsigned long long)Lin) {
        // out-of-range ancestor: reported in the sticky error word, and the
        // child still gets a defined parent (its own index, clamped)
        if (err) atomicOr(err, TMA_DEVERR_BOUNDS);
        a = (int)(l < Lin ? l : Lin - 1);
    }
    const uint32_t mpc = dyn ? dyn->mpc_step : 0u;
    const int nc = kNC > 0 ? kNC : C.nc;
    const float *src = u + ((size_t)a * C.N + i) * nc;
    float *dst = u_out + ((size_t)l * C.N + i) * nc;
    const int nq = (nc + 3) / 4;
#pragma unroll
    for (int q = 0; q < nq; ++q) {
        const uint4 r = draw_rk(C.rk, (uint32_t)l, (uint32_t)i, (uint32_t)q, 1u, (uint32_t)J, mpc);
        const float2 z01 = box_muller(r.x, r.y), z23 = box_muller(r.z, r.w);
        const float z[4] = {z01.x, z01.y, z23.x, z23.y};
        if (kVec) {
            const float4 p = __ldg(reinterpret_cast<const float4 *>(src) + q);
            const float pv[4] = {p.x, p.y, p.z, p.w};
            float ov[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = (4 * q + e) % 3;
                ov[e] = clip(fmaf(C.sigma[c], z[e], pv[e]), C.lo[c], C.hi[c]);
            }
            reinterpret_cast<float4 *>(dst)[q] = make_float4(ov[0], ov[1], ov[2], ov[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int n = 4 * q + e;
                if (n < nc) {
                    const int c = n % 3;
                    dst[n] = clip(fmaf(C.sigma[c], z[e], __ldg(src + n)), C.lo[c], C.hi[c]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) init_kernel(const MoveC C, const DynState *__restrict__ dyn,
                                                   long long L, float *__restrict__ u)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * C.N) return;
    const long long l = t / C.N;
    const int i = (int)(t - l * C.N);
    const uint32_t mpc = dyn ? dyn->mpc_step : 0u;
    float *dst = u + ((size_t)l * C.N + i) * C.nc;
    const int nq = (C.nc + 3) / 4;
    for (int q = 0; q < nq; ++q) {
        const uint4 r = draw(C.key0, C.key1, (uint32_t)l, (uint32_t)i, (uint32_t)q, 4u, 0u, mpc);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int n = 4 * q + e;
            if (n < C.nc) {
                const int c = n % 3;
                dst[n] = fmaf(C.hi[c] - C.lo[c], uniform23(w[e]), C.lo[c]);
            }
        }
    }
}

MoveC make_move(const ProblemC &P, const float lo[3], const float hi[3], const float sigma[3])
{
    MoveC C;
    C.N = P.N;
    C.nc = P.S * 3;
    for (int c = 0; c < 3; ++c) {
        C.lo[c] = lo[c];
        C.hi[c] = hi[c];
        C.sigma[c] = sigma ? sigma[c] : 0.0f;
    }
    C.key0 = P.key0;
    C.key1 = P.key1;
    for (int r = 0; r < 20; ++r) C.rk[r] = P.rk[r];
    return C;
}

}  // namespace

cudaError_t launch_move(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                        const float ctrl_hi[3], const float sigma[3], const float *u,
                        const int32_t *anc, int64_t L, int64_t Lin, int J, float *u_out, cudaStream_t st,
                        unsigned int *err)
{
    if (L <= 0 || Lin <= 0) return cudaSuccess;
    const MoveC C = make_move(P, ctrl_lo, ctrl_hi, sigma);
    const long long n = (long long)L * P.N;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (C.nc == 12) move_kernel<true, 12><<<grid, 256, 0, st>>>(C, dyn, u, anc, L, Lin, J, u_out, err);
    else if (C.nc % 4 == 0) move_kernel<true><<<grid, 256, 0, st>>>(C, dyn, u, anc, L, Lin, J, u_out, err);
    else move_kernel<false><<<grid, 256, 0, st>>>(C, dyn, u, anc, L, Lin, J, u_out, err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init_controls(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                                 const float ctrl_hi[3], float *u, int64_t L, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    const MoveC C = make_move(P, ctrl_lo, ctrl_hi, nullptr);
    const long long n = (long long)L * P.N;
    init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C, dyn, L, u);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
