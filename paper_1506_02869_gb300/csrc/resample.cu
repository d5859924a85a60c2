// Annealed weights, FP64 normalisation (Sec. 3.6, schedule of Sec. 5.1) and
// systematic resampling on a fixed-point CDF (Sec. 3.7).
//
// Each segment (one aircraft of one scenario) of length L is cut into chunks
// of kChunk particles; one 256-thread block handles one (chunk, segment).
//
//   LSE:      (1) chunk minima of the finite costs; (2) every block reduces its
//             segment's minima to lmax = -kappa * min c (exact: multiplying by
//             kappa > 0 is monotone), writes wtilde = exp(-kappa c - lmax) in
//             FP64 and a chunk partial sum; (3) the partial sums are added in
//             chunk order into wsum.
//   Resample: (1) chunk sums of q = floor(wtilde 2^40) (uint64, exact);
//             (2) every block forms its chunk's inclusive prefix S_j in shared
//             memory, finds the range of particles l whose threshold
//             t_l = floor((l 2^32 + r) Q / (Lout 2^32)) falls in the chunk, and
//             assigns a_l = min{j : S_j > t_l} by binary search.  Because
//             S_j > floor(y) <=> S_j > y for integer S_j, both searches compare
//             128-bit products S_j * Lout 2^32 against (l 2^32 + r) * Q and need
//             no division.  Integer arithmetic makes the result independent of
//             the summation order.  Lout ancestors are drawn from the Lin weighted
//             particles of the segment (Lout = Lin for a fixed particle count).
#include <cfloat>
#include <mutex>

#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 8;
constexpr int kChunk = kThreads * kPer;  // 2048

// padded shared-memory index of chunk element j (one extra word per 16)
__device__ __forceinline__ int spad(int j) { return j + (j >> 4); }

// q = floor(w 2^40) for w in (0, 1); w >= 1 (and +inf) counts as 2^40; NaN,
// zero, subnormals and negative values as 0.  Scaling by a power of two is
// exact, so the floor is read from the IEEE bits with integer instructions
// only: w = m 2^(e - 1075) with the 53-bit significand m and the exponent field
// e, hence w 2^40 = m 2^(e - 1035) and floor = m >> (1035 - e).
__device__ __forceinline__ unsigned long long qfix(double w)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(w);
    const unsigned long long frac = u & ((1ull << 52) - 1);
    const int e = (int)((u >> 52) & 0x7ff);
    if (u >> 63) return 0ull;                                 // negative
    if (e >= 1023) return (e == 0x7ff && frac) ? 0ull : 1ull << 40;   // NaN, or w >= 1
    const int shift = 1035 - e;
    if (e == 0 || shift >= 64) return 0ull;                   // zero, subnormal, below 2^-40
    return (frac | (1ull << 52)) >> shift;
}

// Block-wide reduction; `identity` pads the lanes beyond the number of warps.
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T *sh, T identity)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : identity;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

struct MinOp {
    __device__ float operator()(float a, float b) const { return fminf(a, b); }
};
struct AddU64 {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const
    {
        return a + b;
    }
};

__global__ void __launch_bounds__(kThreads) lse_chunk_min(const float *__restrict__ cbar, long long L,
                                                          int nchunk, float *__restrict__ cmin)
{
    __shared__ float sh[32];
    const int s = blockIdx.y, c = blockIdx.x;
    const float *row = cbar + (size_t)s * L;
    const long long base = (long long)c * kChunk;
    float mn = __int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const long long idx = base + threadIdx.x + j * kThreads;
        if (idx < L) {
            const float v = __ldg(row + idx);
            if (v < mn) mn = v;             // +inf and NaN never lower the minimum
        }
    }
    mn = block_reduce(mn, MinOp(), sh, __int_as_float(0x7f800000));
    if (threadIdx.x == 0) cmin[(size_t)s * nchunk + c] = mn;
}

__global__ void __launch_bounds__(kThreads) lse_exp(const float *__restrict__ cbar, long long L,
                                                    int nchunk, double kappa,
                                                    const float *__restrict__ cmin,
                                                    double *__restrict__ wtilde,
                                                    double *__restrict__ csum)
{
    __shared__ float shf[32];
    const int s = blockIdx.y, c = blockIdx.x;
    float mn = __int_as_float(0x7f800000);
    for (int j = threadIdx.x; j < nchunk; j += kThreads) mn = fminf(mn, cmin[(size_t)s * nchunk + j]);
    mn = block_reduce(mn, MinOp(), shf, __int_as_float(0x7f800000));
    const bool any = !isinf(mn);
    const double lmax = -kappa * (double)mn;
    const float *row = cbar + (size_t)s * L;
    double *out = wtilde + (size_t)s * L;
    const long long base = (long long)c * kChunk;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const long long idx = base + threadIdx.x + j * kThreads;
        if (idx < L) {
            const float v = __ldg(row + idx);
            double w = 0.0;
            if (any && !isinf(v) && !isnan(v)) w = exp(-kappa * (double)v - lmax);
            out[idx] = w;
            acc += w;
        }
    }
    // fixed-order block sum: per-thread partials through shared memory
    __shared__ double part[kThreads];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) csum[(size_t)s * nchunk + c] = part[0];
}

__global__ void lse_finish(const float *__restrict__ cmin, const double *__restrict__ csum, int nseg,
                           int nchunk, double kappa, double *__restrict__ lmax,
                           double *__restrict__ wsum)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    float mn = __int_as_float(0x7f800000);
    double sum = 0.0;
    for (int c = 0; c < nchunk; ++c) {
        mn = fminf(mn, cmin[(size_t)s * nchunk + c]);
        sum += csum[(size_t)s * nchunk + c];
    }
    if (lmax) lmax[s] = isinf(mn) ? -__longlong_as_double(0x7ff0000000000000ll) : -kappa * (double)mn;
    if (wsum) wsum[s] = sum;
}

__global__ void __launch_bounds__(kThreads) res_chunk_sum(const double *__restrict__ wtilde,
                                                          long long L, int nchunk,
                                                          unsigned long long *__restrict__ cq)
{
    __shared__ unsigned long long sh[32];
    const int s = blockIdx.y, c = blockIdx.x;
    const double *row = wtilde + (size_t)s * L;
    const long long base = (long long)c * kChunk;
    unsigned long long acc = 0;
    if (base + kChunk <= L && (((size_t)s * L + base) & 1) == 0) {
        // full chunk, 16-byte aligned: two values per load
        const double2 *row2 = reinterpret_cast<const double2 *>(row + base);
#pragma unroll
        for (int j = 0; j < kPer / 2; ++j) {
            const double2 v = __ldg(row2 + threadIdx.x + j * kThreads);
            acc += qfix(v.x) + qfix(v.y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const long long idx = base + threadIdx.x + j * kThreads;
            if (idx < L) acc += qfix(__ldg(row + idx));
        }
    }
    acc = block_reduce(acc, AddU64(), sh, 0ull);
    if (threadIdx.x == 0) cq[(size_t)s * nchunk + c] = acc;
}

// number of particles l in [0, L) with (l 2^32 + r) Q < X D, D = L 2^32
__device__ long long count_below(unsigned long long X, unsigned long long Q, unsigned long long D,
                                 uint32_t r, long long L)
{
    const U128 rhs = mul64x64(X, D);
    long long lo = 0, hi = L;  // answer in [lo, hi]
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        const U128 lhs = mul64x64(((unsigned long long)mid << 32) + r, Q);
        if (lt128(lhs, rhs)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) res_expand(const double *__restrict__ wtilde, long long L,
                                                       long long Lout, int nchunk,
                                                       const unsigned long long *__restrict__ cq,
                                                       uint32_t key0, uint32_t key1, uint32_t J,
                                                       const uint32_t *__restrict__ d_mpc,
                                                       uint32_t mpc_host, int32_t *__restrict__ anc,
                                                       unsigned int *__restrict__ flags,
                                                       const SegKey *__restrict__ seg_keys,
                                                       const DynState *__restrict__ dyns)
{
    // S_j * D of the chunk (128-bit, hi and lo words), padded; the chunk's last S_j
    __shared__ unsigned long long SDh[kChunk + kChunk / 16], SDl[kChunk + kChunk / 16];
    __shared__ unsigned long long s_last;
    __shared__ unsigned long long wtot[kThreads / 32];
    __shared__ unsigned long long sh[32];
    __shared__ long long range[2];
    const int s = blockIdx.y, c = blockIdx.x;
    const long long base = (long long)c * kChunk;
    const int len = (int)min((long long)kChunk, L - base);

    // offset of this chunk and the segment total (integer, order-free)
    unsigned long long before = 0, total = 0;
    for (int j = threadIdx.x; j < nchunk; j += kThreads) {
        const unsigned long long v = cq[(size_t)s * nchunk + j];
        total += v;
        if (j < c) before += v;
    }
    before = block_reduce(before, AddU64(), sh, 0ull);
    total = block_reduce(total, AddU64(), sh, 0ull);
    int32_t *a = anc + (size_t)s * Lout;

    if (total == 0) {
        // degenerate segment: ancestors floor(l L / Lout) spread evenly (the
        // identity when Lout = L); this chunk writes the l that map into it
        const long long l0 = (base * Lout + L - 1) / L, l1 = ((base + len) * Lout + L - 1) / L;
        for (long long l = l0 + threadIdx.x; l < l1; l += kThreads) a[l] = (int32_t)(l * L / Lout);
        if (c == 0 && threadIdx.x == 0 && flags) atomicOr(flags, 1u);
        return;
    }

    // inclusive prefix of q over the chunk: every thread loads its kPer
    // consecutive values (16-byte loads where aligned), scans them in registers;
    // warp scan of the thread totals, block scan of the warp totals.  The chunk's
    // prefix goes to shared memory padded by one word per 16 (no bank conflicts)
    // for the searches.
    const double *row = wtilde + (size_t)s * L;
    const int j0 = threadIdx.x * kPer;
    unsigned long long qv[kPer];
    if (len == kChunk && (((size_t)s * L + base) & 1) == 0) {
        const double2 *p2 = reinterpret_cast<const double2 *>(row + base + j0);
#pragma unroll
        for (int j = 0; j < kPer / 2; ++j) {
            const double2 v = __ldg(p2 + j);
            qv[2 * j] = qfix(v.x);
            qv[2 * j + 1] = qfix(v.y);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) qv[j] = j0 + j < len ? qfix(__ldg(row + base + j0 + j)) : 0ull;
    }
    unsigned long long run = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        run += qv[j];
        qv[j] = run;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    unsigned long long woff = 0;
    for (int w = 0; w < wid; ++w) woff += wtot[w];
    const unsigned long long add = before + woff + (incl - run);
    // the searches compare thresholds against S_j * D: form the products once
    const unsigned long long D = (unsigned long long)Lout << 32;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const unsigned long long S = qv[j] + add;
        const U128 p = mul64x64(S, D);
        SDh[spad(j0 + j)] = p.hi;
        SDl[spad(j0 + j)] = p.lo;
        if (j0 + j == len - 1) s_last = S;
    }
    __syncthreads();

    uint32_t r;
    if (seg_keys) {
        // batched: the segment's scenario key and aircraft index, its scenario's MPC step
        const SegKey sk = seg_keys[s];
        r = draw(sk.key0, sk.key1, 0u, sk.c1, 0u, 2u, J, dyns[sk.scen].mpc_step).x;
    } else {
        const uint32_t mpc = d_mpc ? *d_mpc : mpc_host;
        r = draw(key0, key1, 0u, (uint32_t)s, 0u, 2u, J, mpc).x;
    }
    if (threadIdx.x == 0) range[0] = count_below(before, total, D, r, Lout);
    if (threadIdx.x == 32) range[1] = count_below(s_last, total, D, r, Lout);
    __syncthreads();
    const long long lo = range[0], hi = range[1];
    for (long long l = lo + threadIdx.x; l < hi; l += kThreads) {
        const U128 target = mul64x64(((unsigned long long)l << 32) + r, total);
        int jlo = 0, jhi = len - 1;  // smallest j with S_j * D > target
        while (jlo < jhi) {
            const int mid = (jlo + jhi) >> 1;
            if (lt128(target, U128{SDh[spad(mid)], SDl[spad(mid)]})) jhi = mid;
            else jlo = mid + 1;
        }
        a[l] = (int32_t)(base + jlo);
    }
}

}  // namespace

static int n_chunks(int64_t L) { return (int)((L + kChunk - 1) / kChunk); }

size_t lse_workspace(int nseg, int64_t L)
{
    const size_t n = (size_t)nseg * (size_t)n_chunks(L);
    return n * sizeof(float) + 16 + n * sizeof(double) + 16;
}

size_t resample_workspace(int nseg, int64_t L)
{
    return (size_t)nseg * (size_t)n_chunks(L) * sizeof(unsigned long long) + 16;
}

cudaError_t launch_lse(const float *cbar, int nseg, int64_t L, double kappa, double *wtilde,
                       double *lmax, double *wsum, void *work, cudaStream_t st)
{
    if (nseg <= 0 || L <= 0) return cudaSuccess;
    const int nc = n_chunks(L);
    const size_t n = (size_t)nseg * nc;
    float *cmin = reinterpret_cast<float *>(work);
    double *csum = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(cmin + n) + 15) & ~uintptr_t(15));
    dim3 grid(nc, nseg);
    lse_chunk_min<<<grid, kThreads, 0, st>>>(cbar, L, nc, cmin);
    lse_exp<<<grid, kThreads, 0, st>>>(cbar, L, nc, kappa, cmin, wtilde, csum);
    count_launch(2);
    if (lmax || wsum) {
        lse_finish<<<(nseg + 127) / 128, 128, 0, st>>>(cmin, csum, nseg, nc, kappa, lmax, wsum);
        count_launch();
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Resampling without any allocation by the caller or the library.
//
// The scratch of tma_resample (one uint64 partial sum per (segment, chunk) and
// a status word) lives here in a file-scope device array instead of a
// caller-provided workspace.  Every GPU that loads this library keeps the
// array (about 512 KB) until the process exits.  Host code must not use the
// array's name as a device address: its device address is fetched once per
// device with cudaGetSymbolAddress and passed to the kernels.

namespace {
constexpr long long kNoAllocMaxPartials = 65536;   // nseg * ceil(L / 2048) at most
static __device__ __align__(256) unsigned long long g_resample_scratch[kNoAllocMaxPartials + 2];
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (set up on first use).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_resample_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_resample(const double *wtilde, int nseg, int64_t L, int64_t Lout, uint32_t key0,
                            uint32_t key1, uint32_t J, const uint32_t *d_mpc, uint32_t mpc_host,
                            int32_t *anc, void *work, unsigned int *d_flags, cudaStream_t st,
                            const SegKey *seg_keys, const DynState *dyns)
{
    if (nseg <= 0 || L <= 0 || Lout <= 0) return cudaSuccess;
    const int nc = n_chunks(L);
    auto *cq = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(work) + 15) & ~uintptr_t(15));
    dim3 grid(nc, nseg);
    res_chunk_sum<<<grid, kThreads, 0, st>>>(wtilde, L, nc, cq);
    res_expand<<<grid, kThreads, 0, st>>>(wtilde, L, Lout, nc, cq, key0, key1, J, d_mpc, mpc_host,
                                          anc, d_flags, seg_keys, dyns);
    count_launch(2);
    return cudaGetLastError();
}

// See include/tma_smc.h.
extern "C" tma_status tma_resample_noalloc(const double *d_wtilde, int32_t nseg, int64_t L,
                                           uint64_t seed, uint32_t scenario_id, uint32_t J,
                                           uint32_t mpc_step, int32_t *d_anc, tma_stream_t stream)
{
    if (nseg < 0 || L < 0 || L > TMA_MAX_PARTICLES || J > 0xFFFF || mpc_step > 0xFFFF)
        return TMA_ERR_INVALID_ARG;
    if (nseg == 0 || L == 0) return TMA_OK;
    if (!d_wtilde || !d_anc) return TMA_ERR_INVALID_ARG;
    if ((long long)nseg * n_chunks(L) > kNoAllocMaxPartials) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return record_cuda_error(e);
    // the status word follows the partial sums; it must start at zero
    unsigned int *flags =
        reinterpret_cast<unsigned int *>(static_cast<unsigned long long *>(scratch) + kNoAllocMaxPartials);
    if ((e = cudaMemsetAsync(flags, 0, sizeof(unsigned int), st)) != cudaSuccess)
        return record_cuda_error(e);
    const uint64_t key = seed + (uint64_t)scenario_id * 0x9E3779B97F4A7C15ull;
    if ((e = launch_resample(d_wtilde, nseg, L, L, (uint32_t)key, (uint32_t)(key >> 32), J, nullptr,
                             mpc_step, d_anc, scratch, flags, st)) != cudaSuccess)
        return record_cuda_error(e);
    unsigned int h = 0;
    if ((e = cudaMemcpyAsync(&h, flags, sizeof h, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return record_cuda_error(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return record_cuda_error(e);
    return (h & 1u) ? TMA_WARN_DEGENERATE : TMA_OK;
}

}  // namespace tma
