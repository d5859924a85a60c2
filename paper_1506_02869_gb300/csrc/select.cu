// Final sample selection (Sec. 3.8): the particle with the fewest infeasible
// aircraft, then the smallest sum of mean costs (the largest product of
// weights), ties to the lowest index.  Two passes: per-block candidates, then
// one block over the candidates.  Sums run over aircraft in index order in
// FP64, so the decision is exact and independent of the launch shape.
#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {

namespace {

struct Cand {
    int ninf;
    double sum;
    long long l;
};

__device__ __forceinline__ bool better(const Cand &a, const Cand &b)
{
    if (a.ninf != b.ninf) return a.ninf < b.ninf;
    if (a.sum != b.sum) return a.sum < b.sum;
    return a.l < b.l;
}

__device__ Cand block_best(Cand c)
{
    __shared__ int sn[256];
    __shared__ double ss[256];
    __shared__ long long sl[256];
    sn[threadIdx.x] = c.ninf;
    ss[threadIdx.x] = c.sum;
    sl[threadIdx.x] = c.l;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const Cand a{sn[threadIdx.x], ss[threadIdx.x], sl[threadIdx.x]};
            const Cand b{sn[threadIdx.x + o], ss[threadIdx.x + o], sl[threadIdx.x + o]};
            if (better(b, a)) {
                sn[threadIdx.x] = b.ninf;
                ss[threadIdx.x] = b.sum;
                sl[threadIdx.x] = b.l;
            }
        }
        __syncthreads();
    }
    return Cand{sn[0], ss[0], sl[0]};
}

__global__ void __launch_bounds__(256) select_partial(const float *__restrict__ cbar, int N,
                                                      long long L, Cand *__restrict__ part)
{
    Cand best{1 << 30, 0.0, 1ll << 62};
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < L;
         l += (long long)gridDim.x * blockDim.x) {
        int ni = 0;
        double sum = 0.0;
        for (int i = 0; i < N; ++i) {
            const float c = __ldg(cbar + (size_t)i * L + l);
            if (isinf(c) || isnan(c)) ++ni;
            else sum += (double)c;
        }
        const Cand c{ni, sum, l};
        if (better(c, best)) best = c;
    }
    best = block_best(best);
    if (threadIdx.x == 0) part[blockIdx.x] = best;
}

__global__ void __launch_bounds__(256) select_final(const Cand *__restrict__ part, int nparts,
                                                    long long *__restrict__ out_best,
                                                    double *__restrict__ out_sum,
                                                    int *__restrict__ out_ninf)
{
    Cand best{1 << 30, 0.0, 1ll << 62};
    for (int j = threadIdx.x; j < nparts; j += blockDim.x)
        if (better(part[j], best)) best = part[j];
    best = block_best(best);
    if (threadIdx.x == 0) {
        *out_best = best.l;
        if (out_sum) *out_sum = best.ninf == 0 ? best.sum : __longlong_as_double(0x7ff0000000000000ll);
        if (out_ninf) *out_ninf = best.ninf;
    }
}

// Copies the chosen particle's controls; when err is given, also ORs the
// solve's status into the sticky error word: bit 0 a weight segment was all
// zero (flags bit 0), bit 1 the chosen particle has an infeasible aircraft.
__global__ void gather_best_kernel(const float *__restrict__ u, const long long *__restrict__ best,
                                   int n, float *__restrict__ out, const unsigned int *flags,
                                   const int *ninf, unsigned int *err)
{
    const long long b = *best;
    for (int j = threadIdx.x; j < n; j += blockDim.x) out[j] = u[(size_t)b * n + j];
    if (err && threadIdx.x == 0) *err |= (*flags & 1u) | (*ninf > 0 ? 2u : 0u);
}

constexpr int kSelBlocks = 592;   // 4 x 148 resident blocks; the second pass reads 592 candidates

}  // namespace

size_t select_workspace(int64_t L)
{
    (void)L;
    return kSelBlocks * sizeof(Cand) + 16;
}

cudaError_t launch_select(const float *cbar, int N, int64_t L, int64_t *best, double *best_sum,
                          int *ninf, void *work, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    auto *part = reinterpret_cast<Cand *>((reinterpret_cast<uintptr_t>(work) + 15) & ~uintptr_t(15));
    const long long need = (L + 255) / 256;
    const int nb = (int)(need < kSelBlocks ? need : kSelBlocks);
    select_partial<<<nb, 256, 0, st>>>(cbar, N, L, part);
    select_final<<<1, 256, 0, st>>>(part, nb, reinterpret_cast<long long *>(best), best_sum, ninf);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_gather_best(const float *u, const int64_t *best, int n, float *best_u,
                               cudaStream_t st, const unsigned int *flags, const int *ninf,
                               unsigned int *err)
{
    gather_best_kernel<<<1, 256, 0, st>>>(u, reinterpret_cast<const long long *>(best), n, best_u,
                                          flags, ninf, err);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
