// Annealed weights, FP64 normalisation (Sec. 3.6, schedule of Sec. 5.1) and
// systematic resampling on a fixed-point CDF (Sec. 3.7).
//
// Each segment (one aircraft of one scenario) of length L is cut into chunks
// of kChunk particles; one 256-thread block handles one (chunk, segment).
//
//   LSE:      (1) chunk minima of the finite costs; (2) every block reduces its
//             segment's minima to cmin (lmax = -kappa cmin: multiplying by
//             kappa > 0 is monotone), writes wtilde = exp(kappa (cmin - c)) as
//             FP64 values (table-driven exponential in integer fixed point, no
//             FP64 arithmetic) and, when asked, a chunk partial sum; (3) the
//             partial sums are added in chunk order into wsum.
//   Resample: (1) chunk sums of q = floor(wtilde 2^40) (uint64, exact), by
//             their own pass or by the LSE pass that writes wtilde;
//             (2) every block forms its chunk's inclusive prefix S_j, and for
//             every j the number n_j of particles l whose threshold
//             t_l = floor((l 2^32 + r) Q / (Lout 2^32)) lies below S_j; the
//             chunk's particles are l in [n_(before), n_(last)), element j's
//             copies [n_(j-1), n_j), so a_l = min{j : S_j > t_l} = min{j :
//             n_j > l}: each element with copies marks its first particle in a
//             shared-memory window and a running maximum fills in the rest.
//             Because S_j > floor(y) <=> S_j > y for integer S_j, a count is
//             settled by comparing integers (S_j Lout against
//             l Q + floor(r Q / 2^32), no division); an FP32 estimate within
//             one of the count says which l to compare.  The comparison is
//             taken relative to the chunk's start, where the difference fits
//             in 64 bits (output counts up to 2^20), else in 128 bits.
//             Integer arithmetic makes the result independent of the
//             summation order.  Lout
//             ancestors are drawn from the Lin weighted particles of the
//             segment (Lout = Lin for a fixed particle count).
#include <cfloat>
#include <cuda.h>

#include <mutex>

#include "device_common.cuh"
#include "exp_table.h"
#include "tma_internal.h"

namespace tma {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 8;
constexpr int kChunk = kThreads * kPer;  // 2048


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

// The normalisation's exponential w = exp(x), x = kappa (cmin - c) <= 0, with
// no FP64 instruction (GB300 issues FP64 at a small fraction of its FP32 and
// integer rate): the table-driven method of Tang (ACM TOMS 15(2), 1989) with
// 256 entries, carried out in 64-bit integer fixed point.
//   x:  cmin - c = dh + dl exactly (FP32 two-sum), kappa = K 2^eK with the
//       53-bit integer K, so kappa dh and kappa dl are integer products below
//       2^77, taken to the scale 2^53 by a shift (truncated, error below 2^-52).
//   k = rint(x 256 / ln 2) from the FP32 copy xf of x; r = x - k ln2/256 at the
//       scale 2^53 with ln2/256 = (kExpC1 + kExpC2 / 2^32) 2^-53 (error below
//       2^-52), |r| < 1.5e-3.
//   exp(r) = 1 + r + r^2/2 + (r^3/6 + r^4/24) + O(r^5/120 < 7e-17): r^2/2 from
//       a 64 x 64-bit product at the scale 2^62, the last bracket (< 5e-10) in
//       FP32 (absolute error below 2e-16).
//   y = 2^((k & 255)/256) exp(r) as the high half of the 128-bit product of
//       the table entry (scale 2^63) and exp(r) (scale 2^62), rounded to 53
//       bits, times 2^(k >> 8) in the exponent field; results below the
//       smallest normal double through one FP64 multiply by 2^-64 (rare).
// Relative error below 1e-15.  x = 0 gives exactly 1.
struct KappaFix {
    unsigned long long K;  // 53-bit significand of kappa (kappa > 0 finite)
    int e;                 // kappa = K 2^e
};

__device__ __forceinline__ KappaFix kappa_fix(double kappa)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(kappa);
    const int ex = (int)((u >> 52) & 0x7ff);
    KappaFix f;
    f.K = ex ? ((u & ((1ull << 52) - 1)) | (1ull << 52)) : (u & ((1ull << 52) - 1));
    f.e = (ex ? ex : 1) - 1075;
    return f;
}

// |d| kappa at the scale 2^53, truncated, for a finite FP32 d with |d kappa| < 2^10
__device__ __forceinline__ long long kappa_times(float d, const KappaFix &kf)
{
    const uint32_t u = __float_as_uint(d);
    const int E = (int)((u >> 23) & 0xff);
    if (E == 0) return 0;                                  // zero (subnormals are flushed)
    const uint32_t M = (u & 0x7fffffu) | 0x800000u;        // |d| = M 2^(E - 150)
    // |d| kappa 2^53 = M K 2^(E - 150 + e + 53) = floor(M K / 2^sh); M K >= 2^75
    // and a result below 746 2^53 < 2^62.6 give sh >= 13; with K = Kh 2^21 + Kl,
    // floor(M K / 2^13) = M Kh 2^8 + floor(M Kl / 2^13), below 2^64 as M K < 2^77
    const int sh = 150 - 53 - E - kf.e;
    if (sh < 13) return 0x7fffffffffffffffLL;              // out of range (not reached)
    if (sh >= 77) return 0;
    const unsigned long long p13 = (((unsigned long long)M * (uint32_t)(kf.K >> 21)) << 8) +
                                   (((unsigned long long)M * (uint32_t)(kf.K & 0x1fffffu)) >> 13);
    return (long long)(p13 >> (sh - 13));
}

// Also gives q = floor(w 2^40), the resampling's fixed-point weight (qfix(w)).
__device__ __forceinline__ double exp_fixed(float cmin, float c, float xf, const KappaFix &kf,
                                            const unsigned long long *tab, unsigned long long &q)
{
    q = 0ull;
    if (!(xf > -746.0f)) return 0.0;                       // below half the smallest subnormal
    // cmin - c = dh + dl exactly
    const float dh = cmin - c;
    const float bb = dh - cmin;
    const float dl = (cmin - (dh - bb)) + (-c - bb);
    const long long ah = kappa_times(dh, kf), al = kappa_times(dl, kf);
    const long long x53 = (dh < 0.0f ? -ah : ah) + (dl < 0.0f ? -al : al);
    const int k = __float2int_rn(xf * 369.329794f);        // 256 / ln 2
    const long long r53 = x53 - (long long)k * kExpC1 - (((long long)k * kExpC2) >> 32);
    const long long r62 = r53 * 512;
    const unsigned long long ar = (unsigned long long)(r62 < 0 ? -r62 : r62);
    const long long s62 = (long long)(__umul64hi(ar, ar) << 1);           // r^2 / 2
    const float rf = (float)(int)(r53 >> 13) * 0x1p-40f;
    const float t = rf * rf * rf * fmaf(rf, 1.0f / 24.0f, 1.0f / 6.0f);  // r^3/6 + r^4/24
    const long long t62 = (long long)__float2int_rn(t * 0x1p60f) * 4;
    const unsigned long long e62 = (unsigned long long)((1LL << 62) + r62 + s62 + t62);
    const unsigned long long y61 = __umul64hi(tab[k & 255], e62);         // y 2^61, y in (0.99, 2.01)
    const int p = 63 - __clzll((long long)y61);                           // 60, 61 or 62
    const int shm = p - 52;
    const unsigned long long m = (y61 + (1ull << (shm - 1))) >> shm;      // in [2^52, 2^53]
    const int E = 1023 + (k >> 8) + (p - 61);
    // w = m 2^(E - 1075), so floor(w 2^40) = m >> (1035 - E) (w <= 1: E <= 1023)
    if (E > 971) q = m >> (1035 - E);
    if (E >= 1) return __longlong_as_double((long long)(((unsigned long long)(E - 1) << 52) + m));
    if (E < -60) return 0.0;
    return __longlong_as_double((long long)(((unsigned long long)(E + 63) << 52) + m)) * 0x1p-64;
}

// Writes wtilde; csum (chunk sums of wtilde, fixed order) and cq (chunk sums
// of q = floor(wtilde 2^40) for the resampling) when given.
__global__ void __launch_bounds__(kThreads) lse_exp(const float *__restrict__ cbar, long long L,
                                                    int nchunk, double kappa,
                                                    const float *__restrict__ cmin,
                                                    double *__restrict__ wtilde,
                                                    double *__restrict__ csum,
                                                    unsigned long long *__restrict__ cq)
{
    __shared__ float shf[32];
    __shared__ unsigned long long shq[32];
    __shared__ unsigned long long tab[256];
    const int s = blockIdx.y, c = blockIdx.x;
    for (int j = threadIdx.x; j < 256; j += kThreads) tab[j] = kExp2Frac63[j];
    float mn = __int_as_float(0x7f800000);
    for (int j = threadIdx.x; j < nchunk; j += kThreads) mn = fminf(mn, cmin[(size_t)s * nchunk + j]);
    mn = block_reduce(mn, MinOp(), shf, __int_as_float(0x7f800000));   // its barriers also cover tab
    const bool any = !isinf(mn);
    const float kf = (float)fmin(kappa, 3.0e38);   // finite, so that xf is 0 at the minimum
    const KappaFix kfix = kappa_fix(kappa);
    const float *row = cbar + (size_t)s * L;
    double *out = wtilde + (size_t)s * L;
    const long long base = (long long)c * kChunk;
    const bool want_sum = csum != nullptr;
    double acc = 0.0;
    unsigned long long qacc = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const long long idx = base + threadIdx.x + j * kThreads;
        if (idx < L) {
            const float v = __ldg(row + idx);
            double w = 0.0;
            unsigned long long q = 0ull;
            // -kappa c - lmax = kappa (cmin - c) <= 0 (exactly 0 at the
            // minimum); its FP32 copy picks the table entry
            if (any && !isinf(v) && !isnan(v)) w = exp_fixed(mn, v, kf * (mn - v), kfix, tab, q);
            out[idx] = w;
            if (want_sum) acc += w;
            qacc += q;
        }
    }
    if (cq) {
        qacc = block_reduce(qacc, AddU64(), shq, 0ull);
        if (threadIdx.x == 0) cq[(size_t)s * nchunk + c] = qacc;
    }
    if (!csum) return;
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

// a * b for a < 2^64, b < 2^32 (exact, 128-bit)
__device__ __forceinline__ U128 mul64x32(unsigned long long a, uint32_t b)
{
    const uint32_t alo = (uint32_t)a, ahi = (uint32_t)(a >> 32);
    const unsigned long long lo = (unsigned long long)alo * b;   // 32 x 32 -> 64
    const unsigned long long hi = (unsigned long long)ahi * b;
    const unsigned long long rlo = lo + (hi << 32);
    return U128{(hi >> 32) + (rlo < lo ? 1ull : 0ull), rlo};
}

__device__ __forceinline__ U128 add64(U128 a, unsigned long long b)
{
    const unsigned long long lo = a.lo + b;
    return U128{a.hi + (lo < b ? 1ull : 0ull), lo};
}

// The thresholds of a segment.  With r Q = Rhi 2^32 + Rlo (Rlo < 2^32),
//   t_l = floor((l 2^32 + r) Q / (Lout 2^32)) = floor((l Q + Rhi) / Lout)
// (the multiple l Q 2^32 leaves the inner floor exact), and for an integer S
//   S > t_l  <=>  S Lout > X_l = l Q + Rhi,
// so a threshold is never formed: X_l steps by Q from particle to particle,
// and S_j Lout is compared against it in 128-bit integers (no division; the
// products stay below 2^85 for Q < 2^62 and Lout <= 2^22).
struct Thresholds {
    unsigned long long Q, Rhi;
    uint32_t Lout;
    float ratio;          // Lout / Q
    float shift;          // r 2^-32
};

// a 64-bit value as FP32 (relative error 2^-23 at most)
__device__ __forceinline__ float u64_to_float(unsigned long long v)
{
    return fmaf(__uint2float_rn((uint32_t)(v >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)v));
}

// S above particle l's threshold: S Lout > l Q + Rhi
__device__ __forceinline__ bool above(const U128 &SL, unsigned long long Q, unsigned long long Rhi, int l)
{
    return lt128(add64(mul64x32(Q, (uint32_t)l), Rhi), SL);
}

// Number of particles l in [0, Lout) whose threshold lies below S (S Lout >
// l Q + Rhi): the condition holds up to the count and fails beyond.  The FP32
// estimate S Lout / Q - r 2^-32 has a relative error below 2^-22, so for
// Lout <= 2^21 it lies within 1/2 of the count's real bound x (the count is
// ceil(x), or x when x is an integer): the count is c0 = ceil(est - 1/2) or
// c0 + 1, told apart by the exact condition at c0.  Larger Lout steps from
// ceil(est) until the conditions agree with the count.
__device__ __forceinline__ int count_below(unsigned long long S, const Thresholds &T)
{
    const U128 SL = mul64x32(S, T.Lout);
    const float est = fminf(fmaxf(fmaf(u64_to_float(S), T.ratio, -T.shift), 0.0f), (float)T.Lout);
    if (T.Lout <= (1u << 21)) {
        // the true bound x lies within 1/2 of est, so with c0 = ceil(est - 1/2)
        // the particles below c0 - 1 < x all count and the count is c0 or
        // c0 + 1: one exact comparison, at c0, tells them apart
        const int c0 = max(__float2int_ru(est - 0.5f), 0);
        return c0 >= (int)T.Lout ? (int)T.Lout : c0 + (above(SL, T.Q, T.Rhi, c0) ? 1 : 0);
    }
    int n = __float2int_ru(est);
    while (n < (int)T.Lout && above(SL, T.Q, T.Rhi, n)) ++n;
    while (n > 0 && !above(SL, T.Q, T.Rhi, n - 1)) --n;
    return n;
}

// Count below S_j = Sb + D for a chunk whose start Sb has the count nb and
// the residual Eb = X_nb - Sb Lout (0 <= Eb < Q): with x the real bound of S_j
// (count = ceil(x)), x - nb = (D Lout - Eb) / Q.  The FP32 estimate est of
// x - nb is within 6 2^-24 (Lout + 1) of it to first order (D and the ratio
// Lout / Q as FP32 within 2^-23 and 3 2^-24 relative, D <= Q so the product is
// at most Lout; Eb / Q within 5 2^-24; one rounding of the fused result), below
// 1/2 for Lout <= 2^20, hence c = nb + max(ceil(est - 1/2), 0) lies within one
// of x, the count is c or c + 1, and S_j Lout > X_c is decided by
//   S_j Lout - X_c = D Lout - Eb - (c - nb) Q,
// a difference below Q < 2^62 in magnitude: it is exact in 64-bit two's
// complement although its terms wrap.
struct ChunkBase {
    unsigned long long Eb;
    float eb;       // Eb / Q
    int nb;
};

__device__ __forceinline__ int count_from_base(unsigned long long D, const ChunkBase &B,
                                               unsigned long long Q, uint32_t Lout, float ratio)
{
    const float est = fmaf(u64_to_float(D), ratio, -B.eb);
    const int cr = max(__float2int_ru(est - 0.5f), 0);
    const int c = B.nb + cr;
    if (c >= (int)Lout) return (int)Lout;
    const long long diff = (long long)(D * (unsigned long long)Lout - B.Eb - (unsigned long long)(uint32_t)cr * Q);
    return c + (diff > 0 ? 1 : 0);
}

constexpr int kWin = 4096;                 // ancestors written per window
constexpr int kWinPer = kWin / kThreads;   // 16 per thread, four 16-byte vectors
// window entry k -> shared word: four padding words per 32, so that the
// 16-byte vectors of the eight threads of a quarter warp (entries 16 t ..
// 16 t + 15 per thread) fall in distinct banks and stay 16-byte aligned
__device__ __forceinline__ int wpad(int k) { return k + ((k >> 5) << 2); }

// Copies of element j are the particles [n_(j-1), n_j), n_j the number of
// thresholds below S_j.  Every element's count is formed independently (eight
// per thread, no chain between them); the chunk's particles [lo, hi) are
// then written in windows of kWin starting at lo rounded down to a multiple
// of 4: each element with copies marks its first particle with j + 1, a
// running maximum over the window fills in the rest (each thread takes 16
// consecutive entries in registers, then a warp scan and the warps' maxima),
// and every thread stores its entries that lie in [lo, hi), as 16-byte
// vectors where the ancestor row is 16-byte aligned.
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
    __shared__ __align__(16) int win[kWin + kWin / 8];   // padded: wpad(k)
    __shared__ int lastc[kThreads];
    __shared__ int wmax[kThreads / 32];
    __shared__ unsigned long long wtot[kThreads / 32];
    __shared__ unsigned long long seg_before, seg_total;
    __shared__ Thresholds Tsh;
    __shared__ ChunkBase Bsh;
    const int s = blockIdx.y, c = blockIdx.x;
    const long long base = (long long)c * kChunk;
    const int len = (int)min((long long)kChunk, L - base);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    // this thread's kPer consecutive weights (16-byte loads where aligned;
    // zero past the chunk), issued before anything else
    const double *row = wtilde + (size_t)s * L;
    const int j0 = threadIdx.x * kPer;
    const bool full = len == kChunk && (((size_t)s * L + base) & 1) == 0;
    double wv[kPer];
    if (full) {
        const double2 *p2 = reinterpret_cast<const double2 *>(row + base + j0);
#pragma unroll
        for (int j = 0; j < kPer / 2; ++j) {
            const double2 v = __ldg(p2 + j);
            wv[2 * j] = v.x;
            wv[2 * j + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) wv[j] = j0 + j < len ? __ldg(row + base + j0 + j) : 0.0;
    }
    // this thread's window entries start at zero (ordered before any mark by
    // the barriers below)
    {
        int4 *w4 = reinterpret_cast<int4 *>(win + wpad(kWinPer * threadIdx.x));
#pragma unroll
        for (int g = 0; g < kWinPer / 4; ++g) w4[g] = make_int4(0, 0, 0, 0);
    }

    if (wid == 0) {
        // the segment's bookkeeping, while the loads are in flight: the chunk's
        // offset and the segment total (integer, order-free), the uniform, the
        // thresholds, the count below the chunk's start and its residual
        unsigned long long before = 0, total = 0;
        for (int j = lane; j < nchunk; j += 32) {
            const unsigned long long v = cq[(size_t)s * nchunk + j];
            total += v;
            if (j < c) before += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            total += __shfl_xor_sync(0xffffffffu, total, o);
        }
        if (lane == 0) {
            seg_before = before;
            seg_total = total;
            if (total != 0) {
                uint32_t r;
                if (seg_keys) {
                    // batched: the segment's scenario key and aircraft index, its scenario's MPC step
                    const SegKey sk = seg_keys[s];
                    r = draw(sk.key0, sk.key1, 0u, sk.c1, 0u, 2u, J, dyns[sk.scen].mpc_step).x;
                } else {
                    const uint32_t mpc = d_mpc ? *d_mpc : mpc_host;
                    r = draw(key0, key1, 0u, (uint32_t)s, 0u, 2u, J, mpc).x;
                }
                Thresholds T;
                T.Q = total;
                const U128 rQ = mul64x32(total, r);
                T.Rhi = (rQ.hi << 32) | (rQ.lo >> 32);     // floor(r Q / 2^32) < 2^62
                T.Lout = (uint32_t)Lout;
                T.ratio = __fdiv_rn((float)(uint32_t)Lout, u64_to_float(total));
                T.shift = (float)r * 2.3283064365386963e-10f;
                Tsh = T;
                ChunkBase B;
                B.nb = count_below(before, T);
                // X_nb - before Lout lies in [0, Q): its low 64 bits are the value
                const U128 Xn = add64(mul64x32(T.Q, (uint32_t)B.nb), T.Rhi);
                B.Eb = Xn.lo - mul64x32(before, T.Lout).lo;
                B.eb = __fdiv_rn(u64_to_float(B.Eb), u64_to_float(T.Q));
                Bsh = B;
            }
        }
    }

    // inclusive prefix of q over the chunk: every thread scans its kPer
    // values in registers; warp scan of the thread totals, block scan of the
    // warp totals
    unsigned long long qv[kPer];
    unsigned long long run = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        run += qfix(wv[j]);
        qv[j] = run;
    }
    unsigned long long incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    const unsigned long long before = seg_before, total = seg_total;
    int32_t *a = anc + (size_t)s * Lout;
    if (total == 0) {
        // degenerate segment: ancestors floor(l L / Lout) spread evenly (the
        // identity when Lout = L); this chunk writes the l that map into it
        const long long l0 = (base * Lout + L - 1) / L, l1 = ((base + len) * Lout + L - 1) / L;
        for (long long l = l0 + threadIdx.x; l < l1; l += kThreads) a[l] = (int32_t)(l * L / Lout);
        if (c == 0 && threadIdx.x == 0 && flags) atomicOr(flags, 1u);
        return;
    }
    unsigned long long woff = 0;
    for (int w = 0; w < wid; ++w) woff += wtot[w];
    // prefix of q within the chunk before this thread's first element
    const unsigned long long add = woff + (incl - run);
    const Thresholds T = Tsh;
    // the counts of this thread's elements, independent of each other (the
    // elements past the chunk repeat the chunk's last prefix)
    int nc[kPer];
    if (T.Lout <= (1u << 20)) {
        const ChunkBase B = Bsh;
#pragma unroll
        for (int j = 0; j < kPer; ++j) nc[j] = count_from_base(qv[j] + add, B, T.Q, T.Lout, T.ratio);
    } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) nc[j] = count_below(qv[j] + add + before, T);
    }
    lastc[threadIdx.x] = nc[kPer - 1];
    __syncthreads();
    const int lo = Bsh.nb, hi = lastc[kThreads - 1];
    const int nprev0 = threadIdx.x == 0 ? lo : lastc[threadIdx.x - 1];
    // 16-byte stores need the row start aligned (Lout a multiple of 4 and an
    // aligned output array); the window starts are multiples of 4
    const bool vec = (reinterpret_cast<uintptr_t>(a) & 15) == 0;
    const int k0 = kWinPer * threadIdx.x;
    int4 *mine = reinterpret_cast<int4 *>(win + wpad(k0));

    int carry = 0;
    for (int w0 = lo & ~3; lo < hi && w0 < hi; w0 += kWin) {
        const int wl = min(kWin, hi - w0);
        int np = nprev0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            if (nc[j] > np && np >= w0 && np < w0 + wl) win[wpad(np - w0)] = j0 + j + 1;
            np = nc[j];
        }
        __syncthreads();
        // inclusive running maximum over the window: this thread's 16 entries
        // (zero beyond wl) in registers, read and cleared for the next window
        int v[kWinPer];
        int m = 0;
        if (k0 < wl) {
#pragma unroll
            for (int g = 0; g < kWinPer / 4; ++g) {
                const int4 t = mine[g];
                mine[g] = make_int4(0, 0, 0, 0);
                v[4 * g] = t.x;
                v[4 * g + 1] = t.y;
                v[4 * g + 2] = t.z;
                v[4 * g + 3] = t.w;
            }
#pragma unroll
            for (int q = 0; q < kWinPer; ++q) {
                m = max(m, v[q]);
                v[q] = m;
            }
        }
        int inc = m;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = max(inc, t);
        }
        if (lane == 31) wmax[wid] = inc;
        int ex = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) ex = 0;
        __syncthreads();
        int pre = carry, all = carry;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const int t = wmax[w];
            if (w < wid) pre = t > pre ? t : pre;
            all = t > all ? t : all;
        }
        ex = max(ex, pre);
        carry = all;
        if (k0 < wl) {
            // entries w0 + k0 + q; the ancestor of particle p is base + value - 1
            const int b1 = (int)base - 1;
#pragma unroll
            for (int g = 0; g < kWinPer / 4; ++g) {
                const int p0 = w0 + k0 + 4 * g;
                const int4 o = make_int4(b1 + max(v[4 * g], ex), b1 + max(v[4 * g + 1], ex),
                                         b1 + max(v[4 * g + 2], ex), b1 + max(v[4 * g + 3], ex));
                if (vec && p0 >= lo && p0 + 4 <= hi) {
                    *reinterpret_cast<int4 *>(a + p0) = o;
                } else {
                    if (p0 >= lo && p0 < hi) a[p0] = o.x;
                    if (p0 + 1 >= lo && p0 + 1 < hi) a[p0 + 1] = o.y;
                    if (p0 + 2 >= lo && p0 + 2 < hi) a[p0 + 2] = o.z;
                    if (p0 + 3 >= lo && p0 + 3 < hi) a[p0 + 3] = o.w;
                }
            }
        }
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

unsigned long long *resample_partials(void *work)
{
    return reinterpret_cast<unsigned long long *>((reinterpret_cast<uintptr_t>(work) + 15) & ~uintptr_t(15));
}

cudaError_t launch_lse(const float *cbar, int nseg, int64_t L, double kappa, double *wtilde,
                       double *lmax, double *wsum, void *work, cudaStream_t st,
                       unsigned long long *cq)
{
    if (nseg <= 0 || L <= 0) return cudaSuccess;
    const int nc = n_chunks(L);
    const size_t n = (size_t)nseg * nc;
    float *cmin = reinterpret_cast<float *>(work);
    double *csum = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(cmin + n) + 15) & ~uintptr_t(15));
    dim3 grid(nc, nseg);
    lse_chunk_min<<<grid, kThreads, 0, st>>>(cbar, L, nc, cmin);
    lse_exp<<<grid, kThreads, 0, st>>>(cbar, L, nc, kappa, cmin, wtilde, (lmax || wsum) ? csum : nullptr, cq);
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
// device with cudaGetSymbolAddress and passed to the kernels.  The address
// belongs to the device's context: after cudaDeviceReset the next call finds a
// new context (its driver ID differs) and fetches the address again.

namespace {
constexpr long long kNoAllocMaxPartials = 65536;   // nseg * ceil(L / 2048) at most
static __device__ __align__(256) unsigned long long g_resample_scratch[kNoAllocMaxPartials + 2];
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
struct ScratchSetUp {
    void *addr = nullptr;
    unsigned long long ctx_id = 0;   // driver ID of the context the address belongs to
};
ScratchSetUp g_scratch[kMaxDevices];

// Driver ID of the current context (0 if the driver cannot tell), through the
// driver's entry points (this library links only the runtime).
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f);
            get_id = reinterpret_cast<GetId>(g);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the array on the current device: set up on the first call
// with this device current, and again when the device's context has changed
// (or had not been created yet at the previous set-up: its ID then read 0).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    ScratchSetUp &su = g_scratch[dev];
    if (!su.addr || su.ctx_id != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_resample_scratch);
        if (e != cudaSuccess) return e;
        su.addr = p;
        su.ctx_id = ctx;
    }
    *out = su.addr;
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_resample(const double *wtilde, int nseg, int64_t L, int64_t Lout, uint32_t key0,
                            uint32_t key1, uint32_t J, const uint32_t *d_mpc, uint32_t mpc_host,
                            int32_t *anc, void *work, unsigned int *d_flags, cudaStream_t st,
                            const SegKey *seg_keys, const DynState *dyns, bool sums_ready)
{
    if (nseg <= 0 || L <= 0 || Lout <= 0) return cudaSuccess;
    const int nc = n_chunks(L);
    unsigned long long *cq = resample_partials(work);
    dim3 grid(nc, nseg);
    if (!sums_ready) {
        res_chunk_sum<<<grid, kThreads, 0, st>>>(wtilde, L, nc, cq);
        count_launch();
    }
    res_expand<<<grid, kThreads, 0, st>>>(wtilde, L, Lout, nc, cq, key0, key1, J, d_mpc, mpc_host,
                                          anc, d_flags, seg_keys, dyns);
    count_launch();
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
