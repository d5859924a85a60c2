// Particle-parallel rollout and costing: the inner loop of Algorithm 1
// (Sec. 3.3-3.6, Sec. 7.1) for every (particle, wind sample, aircraft).
//
// Thread mapping: one block simulates 32 particles under one wind sample m;
// warp i of the block is aircraft i, lane j is particle 32*b + j.  Every thread
// keeps its aircraft's state (position, airspeed, heading, fuel burned) and
// cost accumulators in registers for the whole horizon.  Aircraft type,
// constants and the wind field are uniform over a warp, so warps do not
// diverge on the arrival/departure terms and the constants are broadcast.
// The pairwise separation check of Eq. (avoidance) reads the other aircraft's
// positions of the same particle from shared memory (double-buffered by step,
// one barrier per step).  Blocks are ordered with the wind sample slowest, so
// the blocks resident at one time read the same wind field and share it in L2.
#include "rollout_tile.cuh"

namespace tma {

namespace {

// Launch-bound variants (block size cap, minimum resident blocks per SM): the
// register budget per thread is 65536 / (cap * blocks); the autotuner picks
// among the variants whose cap fits the block (32 * N threads).  OwnWind is
// wind mode 1 (per-particle fields) and Rolling the rolling window, each a
// kernel of its own so that the plain problem keeps its register allocation;
// Soft the softplus form; TP the particles of a tile (32, or 16: the half tile,
// a warp holding two aircraft, so that the blocks of a large N are half as big).
template <int kMaxThreads, int kMinBlocks, bool OwnWind, bool Rolling, bool Soft, int TP = kPB>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks) rollout_kernel(const ProblemC P,
                                                       const DynState *__restrict__ dyn,
                                                       const float *__restrict__ u,
                                                       const float4 *__restrict__ W, long long L,
                                                       int nLb, int J, float *__restrict__ cost_ms,
                                                       float *__restrict__ cost_ms_soft,
                                                       unsigned long long *__restrict__ live)
{
    extern __shared__ float spos[];
    const int m = blockIdx.x / nLb;            // wind sample: block-uniform
    const long long l0 = (long long)(blockIdx.x - m * nLb) * TP;
    const int i = threadIdx.x / TP, j = threadIdx.x % TP;
    const TileResult r = rollout_tile_mode<OwnWind, Rolling, Soft, true, TP>(
        P, dyn, u, W + (size_t)m * P.H * P.P, L, l0, i, j, m, J, spos, 0, blockDim.x);
    store_tile(r, P.N, L, l0 + j, i, j, m, cost_ms, cost_ms_soft, live);
}

// Mean over wind samples: cbar[i][l] = (1/M) sum_m cost_ms[m][i][l], +inf when any
// sample was infeasible.  Samples are summed in order with compensation.
__global__ void __launch_bounds__(256) sample_mean_kernel(const float *__restrict__ cost_ms,
                                                          long long L, int M, int N,
                                                          float *__restrict__ cbar)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L * N) return;
    Kahan s;
    bool inf = false;
    const size_t stride = (size_t)N * L;
    for (int m = 0; m < M; ++m) {
        const float v = __ldg(cost_ms + (size_t)m * stride + t);
        if (isinf(v)) inf = true;
        else s.add(v);
    }
    cbar[t] = inf ? __int_as_float(0x7f800000) : s.s / (float)M;
}

}  // namespace

struct Variant {
    int max_threads, min_blocks;
};
// registers per thread: 64, 85, 64, 128, 64, 128, 85, 85
constexpr Variant kVariants[] = {{256, 4}, {256, 3}, {512, 2}, {512, 1}, {1024, 1},
                                 {256, 2}, {384, 2}, {768, 1}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
// the smaller tiles (TP particles, block TP N, 32 / TP aircraft per warp):
// shared wind field, no rolling window, N a multiple of 32 / TP (full warps).
// Half tiles (16): registers per thread 85, 85, 64; quarter tiles (8): 64, 85.
constexpr Variant kHalfVariants[] = {{768, 1}, {384, 2}, {512, 2}};
constexpr int kNumHalfVariants = sizeof(kHalfVariants) / sizeof(kHalfVariants[0]);
constexpr Variant kQuarterVariants[] = {{512, 2}, {384, 2}};
constexpr int kNumQuarterVariants = sizeof(kQuarterVariants) / sizeof(kQuarterVariants[0]);
static_assert(kHalfVariantBase + kNumHalfVariants <= kQuarterVariantBase, "variant table");
static_assert(kQuarterVariantBase + kNumQuarterVariants <= kMaxRolloutVariants, "variant table");

static bool small_tile_valid(const ProblemC &P, int tp, int cap)
{
    return P.wind_mode == 0 && !P.rolling && P.N % (32 / tp) == 0 && cap >= P.N * tp;
}

int rollout_variants(const ProblemC &P, int *out)
{
    int n = 0;
    for (int v = 0; v < kNumVariants; ++v)
        if (kVariants[v].max_threads >= P.N * kPB) out[n++] = v;
    int pv[kMaxRolloutVariants];
    const int np = rollout_pair_variants(P, pv);
    for (int c = 0; c < np; ++c) out[n++] = kPairVariantBase + pv[c];
    for (int v = 0; v < kNumHalfVariants; ++v)
        if (small_tile_valid(P, 16, kHalfVariants[v].max_threads)) out[n++] = kHalfVariantBase + v;
    for (int v = 0; v < kNumQuarterVariants; ++v)
        if (small_tile_valid(P, 8, kQuarterVariants[v].max_threads)) out[n++] = kQuarterVariantBase + v;
    return n;
}

// The one-sample kernel on tiles of TP < 32 particles with launch bounds (T, B).
template <int T, int B, int TP>
static void launch_small_tile(const ProblemC &P, const DynState *dyn, const float *u, const float4 *W4,
                              int64_t L, int J, float *cost_ms, float *cost_ms_soft,
                              unsigned long long *live, cudaStream_t st)
{
    const long long nLb = (L + TP - 1) / TP;
    const unsigned grid = (unsigned)(nLb * P.M);
    const int block = P.N * TP;
    const size_t smem = (size_t)tile_smem_words(P.N, 0, TP) * sizeof(float);
    if (cost_ms_soft) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(rollout_kernel<T, B, false, false, true, TP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        rollout_kernel<T, B, false, false, true, TP><<<grid, block, smem, st>>>(P, dyn, u, W4, L, (int)nLb, J,
                                                                              cost_ms, cost_ms_soft, live);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(rollout_kernel<T, B, false, false, false, TP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        rollout_kernel<T, B, false, false, false, TP><<<grid, block, smem, st>>>(P, dyn, u, W4, L, (int)nLb, J,
                                                                               cost_ms, cost_ms_soft, live);
    }
}

cudaError_t launch_rollout(const ProblemC &P, const DynState *dyn, const float *u, const float *W,
                           int64_t L, int J, float *cost_ms, float *cost_ms_soft,
                           unsigned long long *live, cudaStream_t st, int variant)
{
    if (L <= 0) return cudaSuccess;
    if (variant >= kHalfVariantBase) {
        const float4 *W4 = reinterpret_cast<const float4 *>(W);
        const int hv = variant - kHalfVariantBase, qv = variant - kQuarterVariantBase;
        bool done = true;
        if (hv >= 0 && hv < kNumHalfVariants && small_tile_valid(P, 16, kHalfVariants[hv].max_threads)) {
            if (hv == 0) launch_small_tile<768, 1, 16>(P, dyn, u, W4, L, J, cost_ms, cost_ms_soft, live, st);
            else if (hv == 1) launch_small_tile<384, 2, 16>(P, dyn, u, W4, L, J, cost_ms, cost_ms_soft, live, st);
            else launch_small_tile<512, 2, 16>(P, dyn, u, W4, L, J, cost_ms, cost_ms_soft, live, st);
        } else if (qv >= 0 && qv < kNumQuarterVariants &&
                   small_tile_valid(P, 8, kQuarterVariants[qv].max_threads)) {
            if (qv == 0) launch_small_tile<512, 2, 8>(P, dyn, u, W4, L, J, cost_ms, cost_ms_soft, live, st);
            else launch_small_tile<384, 2, 8>(P, dyn, u, W4, L, J, cost_ms, cost_ms_soft, live, st);
        } else {
            done = false;
        }
        if (done) {
            count_launch();
            return cudaGetLastError();
        }
        variant = -1;                  // not valid for this problem: the one-sample kernel
    } else if (variant >= kPairVariantBase) {
        int pv[kMaxRolloutVariants];
        const int np = rollout_pair_variants(P, pv);
        for (int c = 0; c < np; ++c)
            if (pv[c] == variant - kPairVariantBase)
                return launch_rollout_pair(P, dyn, u, W, L, J, cost_ms, cost_ms_soft, live, st, pv[c]);
        variant = -1;                  // not valid for this problem: the one-sample kernel
    }
    if (variant < 0 || variant >= kNumVariants || kVariants[variant].max_threads < P.N * kPB) {
        int cand[kMaxRolloutVariants];
        rollout_variants(P, cand);
        variant = cand[0];
    }
    const long long nLb = (L + kPB - 1) / kPB;
    const unsigned grid = (unsigned)(nLb * P.M);
    const int block = P.N * kPB;
    const size_t smem = (size_t)tile_smem_words(P.N, P.wind_mode) * sizeof(float);
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
    // above the default 48 KB of dynamic shared memory the kernel must opt in
#define TMA_ROLLOUT_KS(T, B, O, R, F)                                                            \
    do {                                                                                         \
        if (smem > 48 * 1024)                                                                    \
            cudaFuncSetAttribute(rollout_kernel<T, B, O, R, F>,                                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
        rollout_kernel<T, B, O, R, F><<<grid, block, smem, st>>>(P, dyn, u, W4, L, (int)nLb, J,  \
                                                                 cost_ms, cost_ms_soft, live);   \
    } while (0)
#define TMA_ROLLOUT_K(T, B, O, R)                                                                \
    do {                                                                                         \
        if (cost_ms_soft) TMA_ROLLOUT_KS(T, B, O, R, true);                                      \
        else TMA_ROLLOUT_KS(T, B, O, R, false);                                                  \
    } while (0)
#define TMA_ROLLOUT(T, B)                                                                        \
    do {                                                                                         \
        if (P.wind_mode == 1) {                                                                  \
            if (P.rolling) TMA_ROLLOUT_K(T, B, true, true);                                      \
            else TMA_ROLLOUT_K(T, B, true, false);                                               \
        } else {                                                                                 \
            if (P.rolling) TMA_ROLLOUT_K(T, B, false, true);                                     \
            else TMA_ROLLOUT_K(T, B, false, false);                                              \
        }                                                                                        \
    } while (0)
    switch (variant) {
    case 0: TMA_ROLLOUT(256, 4); break;
    case 1: TMA_ROLLOUT(256, 3); break;
    case 2: TMA_ROLLOUT(512, 2); break;
    case 3: TMA_ROLLOUT(512, 1); break;
    case 5: TMA_ROLLOUT(256, 2); break;
    case 6: TMA_ROLLOUT(384, 2); break;
    case 7: TMA_ROLLOUT(768, 1); break;
    default: TMA_ROLLOUT(1024, 1); break;
    }
#undef TMA_ROLLOUT
#undef TMA_ROLLOUT_K
#undef TMA_ROLLOUT_KS
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sample_mean(const float *cost_ms, int64_t L, int M, int N, float *cbar,
                               cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    const long long n = (long long)L * N;
    sample_mean_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cost_ms, L, M, N, cbar);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
