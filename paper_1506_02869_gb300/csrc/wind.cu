// Wind-field generation (Sec. 3.9.1): W(0) = Qhat v(0), W(k+1) = a W(k) + Q v(k+1)
// with Qhat = sigma (L_xy kron L_z) and Q = sqrt(1 - a^2) Qhat.  Because the
// recursion is linear, W(k) = sigma (L_xy kron L_z) B(k) with
// B(0) = v(0), B(k) = a B(k-1) + sqrt(1 - a^2) v(k).
//
// Kernel 1 draws v (Philox stream 3, Box-Muller), runs the AR(1) recursion
// over k and applies the small vertical factor L_z, writing
// Btmp[q][((m H + k) nz + iz) 2 + c] for horizontal node q.
// Kernel 2 applies the horizontal factor as one lower-triangular matrix
// product over q (an FP32 register-tiled GEMM) and scatters into the
// rollout's packed layout: float4 per node; kernel 3 turns the upper half of
// every record into the difference to the node one level up, so that the
// trilinear interpolation needs four aligned 16-byte loads and no subtraction
// in the vertical direction.
#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {

namespace {

__global__ void __launch_bounds__(128) wind_normals_ar_kernel(const WindC w,
                                                              const DynState *__restrict__ dyn,
                                                              float *__restrict__ Btmp)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)w.M * w.nxy) return;
    const int m = (int)(t / w.nxy);
    const int q = (int)(t - (long long)m * w.nxy);
    const uint32_t mpc = dyn->mpc_step;
    const int nz = w.nz;
    float B[2][TMA_MAX_GRID_Z];
#pragma unroll
    for (int iz = 0; iz < TMA_MAX_GRID_Z; ++iz) B[0][iz] = B[1][iz] = 0.0f;
    float *row = Btmp + (size_t)q * w.ldb;
    for (int k = 0; k < w.H; ++k) {
#pragma unroll
        for (int iz = 0; iz < TMA_MAX_GRID_Z; ++iz) {
            if (iz < nz) {
                const uint4 r = draw(w.key0, w.key1, (uint32_t)(q * nz + iz), (uint32_t)m << 8,
                                     (uint32_t)k, w.stream, 0u, mpc);
                const float2 n = box_muller(r.x, r.y);
                if (k == 0) {
                    B[0][iz] = n.x;
                    B[1][iz] = n.y;
                } else {
                    B[0][iz] = fmaf(w.a, B[0][iz], w.b * n.x);
                    B[1][iz] = fmaf(w.a, B[1][iz], w.b * n.y);
                }
            }
        }
        float *o = row + ((size_t)m * w.H + k) * (size_t)(2 * nz);
#pragma unroll
        for (int iz = 0; iz < TMA_MAX_GRID_Z; ++iz) {
            if (iz < nz) {
                float ax = 0.0f, ay = 0.0f;
#pragma unroll
                for (int jz = 0; jz <= iz; ++jz) {
                    const float lz = w.Lz[iz * TMA_MAX_GRID_Z + jz];
                    ax = fmaf(lz, B[0][jz], ax);
                    ay = fmaf(lz, B[1][jz], ay);
                }
                o[2 * iz] = ax;
                o[2 * iz + 1] = ay;
            }
        }
    }
}

// C[p][col] = sum_{q <= p} A[p][q] Btmp[q][col]; W[(col / 2nz) nxy + p][col % 2nz] = sigma C.
// 128 x 128 tiles, K step 8, 8 x 8 outputs per thread.  A is zero-padded to a
// multiple of 128 rows and lda columns; Btmp is zero-padded to a multiple of 8
// rows and ldb (multiple of 128) columns, so the main loop needs no guards.
__global__ void __launch_bounds__(256) wind_gemm_kernel(const WindC w, const float *__restrict__ A,
                                                        int lda, const float *__restrict__ Bm,
                                                        float *__restrict__ W)
{
    __shared__ __align__(16) float As[8][128];
    __shared__ __align__(16) float Bs[8][128];
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int row0 = blockIdx.y * 128, col0 = blockIdx.x * 128;
    const int kend = min(((w.nxy + 7) / 8) * 8, row0 + 128);
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;

    const int ar = t >> 1, ak = (t & 1) * 4;     // A tile: row ar, k offset ak
    const int bk = t >> 5, bc = (t & 31) * 4;    // B tile: k row bk, column offset bc
    for (int k0 = 0; k0 < kend; k0 += 8) {
        const float4 av = __ldg(reinterpret_cast<const float4 *>(A + (size_t)(row0 + ar) * lda + k0 + ak));
        const float4 bv = __ldg(reinterpret_cast<const float4 *>(Bm + (size_t)(k0 + bk) * w.ldb + col0 + bc));
        As[ak + 0][ar] = av.x;
        As[ak + 1][ar] = av.y;
        As[ak + 2][ar] = av.z;
        As[ak + 3][ar] = av.w;
        *reinterpret_cast<float4 *>(&Bs[bk][bc]) = bv;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
            const float ar8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float br8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(ar8[a], br8[b], acc[a][b]);
        }
        __syncthreads();
    }
    // scatter into the packed layout: node q of field (m, k) holds
    // (W_x(q), W_y(q), W_x(q + 1 level), W_y(q + 1 level)); the top level
    // repeats its own value in the upper half (never read by interpolation)
    const int two_nz = 2 * w.nz;
    const int P = w.nxy * w.nz;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int row = row0 + ty * 8 + a;
        if (row >= w.nxy) continue;
#pragma unroll
        for (int b = 0; b < 8; b += 2) {
            const int col = col0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
            if (col >= w.ncol) continue;   // ncol is even: a pair (x, y) is never split
            const int mk = col / two_nz;
            const int iz = (col - mk * two_nz) >> 1;
            const float2 val = make_float2(w.sigma * acc[a][b], w.sigma * acc[a][b + 1]);
            float2 *rec = reinterpret_cast<float2 *>(W + ((size_t)mk * P + (size_t)row * w.nz + iz) * 4);
            rec[0] = val;
            if (iz == w.nz - 1) rec[1] = val;
            if (iz > 0) rec[-1] = val;      // upper half of the record one level below
        }
    }
}

// rec = (W_x, W_y, W_x one level up, W_y one level up) -> (W_x, W_y, dW_x, dW_y)
__global__ void __launch_bounds__(256) wind_diff_kernel(float4 *__restrict__ W, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float4 r = W[t];
    r.z -= r.x;
    r.w -= r.y;
    W[t] = r;
}

}  // namespace

cudaError_t launch_wind_normals_ar(const WindC &w, const DynState *dyn, float *Btmp,
                                   cudaStream_t st)
{
    const long long n = (long long)w.M * w.nxy;
    if (n <= 0) return cudaSuccess;
    wind_normals_ar_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(w, dyn, Btmp);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_wind_gemm(const WindC &w, const float *Lxy, int lda, const float *Btmp,
                             float *W, cudaStream_t st)
{
    dim3 grid(w.ldb / 128, (w.nxy + 127) / 128);
    wind_gemm_kernel<<<grid, 256, 0, st>>>(w, Lxy, lda, Btmp, W);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)(w.ncol / (2 * w.nz)) * w.nxy * w.nz;   // records
    wind_diff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<float4 *>(W), n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
