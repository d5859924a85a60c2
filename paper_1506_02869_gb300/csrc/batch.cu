// Batched receding-horizon MPC over many independent TMA scenarios with
// uneven aircraft counts (one SMC solve per scenario per MPC step, Sec. 2 and
// Algorithm 1), all scenarios in single launches.
//
//   rollout_batched   persistent kernel: a CTA of 32 warps holds
//                     min(15, floor(32 / N_s)) tile slots of N_s warps; each slot
//                     claims tiles (wind sample m, 32 particles) of the current
//                     scenario from that scenario's atomic counter and
//                     synchronises only its own warps (a named barrier per
//                     slot), so a slow tile does not hold the others.  All CTAs
//                     walk the scenarios in the same order; small and large
//                     scenarios share the machine without a launch per
//                     scenario.  The arithmetic is the single-scenario tile's.
//   batch_*           the remaining stages over all scenarios at once; weight
//                     segments are (scenario, aircraft) pairs, so LSE and
//                     resampling reuse the segmented kernels.
//   plant_step        applies each scenario's chosen first control to its
//                     true state (the "Plant" of Fig. 1) and advances its MPC
//                     step on the device, so that MPC steps can be replayed as
//                     one CUDA graph.
#include <algorithm>

#include "rollout_tile.cuh"

namespace tma {

namespace {

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// ------------------------------------------------------------------ rollout


// OwnWind: wind mode 1 and Soft: the softplus penalties evaluated (both the
// same for every scenario of a batch), fixed at compile time so that the
// kernel holds only the two tile forms it can run (with and without the
// rolling window) within its 64 registers.
template <bool OwnWind, bool Soft>
__global__ void __launch_bounds__(1024, 1) rollout_batched_kernel(
    const ProblemC *__restrict__ probs, const BatchScen *__restrict__ scen, int n_scen,
    const DynState *__restrict__ dyns, const float *__restrict__ u, const float4 *__restrict__ W,
    long long L, int nLb, int J, int Mj, float *__restrict__ cost_ms, float *__restrict__ cost_ms_soft,
    unsigned long long *__restrict__ live, unsigned long long *__restrict__ claimed)
{
    // this iteration's tiles: wind samples 0 .. Mj-1 (the cost rows keep the stride M)
    const long long items = (long long)Mj * nLb;
    __shared__ ProblemC Ps;
    __shared__ BatchScen Sc;
    __shared__ long long slot_item[15];
    __shared__ int skip_sh;
    extern __shared__ float spos[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Every CTA walks the scenarios in the same order, so the CTAs of the device
    // share one scenario (and its wind field in L2) at a time.
    for (int s = 0; s < n_scen; ++s) {
        if (threadIdx.x == 0)
            skip_sh = *reinterpret_cast<volatile unsigned long long *>(claimed + s) >=
                      (unsigned long long)items;
        __syncthreads();            // also: the previous scenario's slots are done with Ps
        if (skip_sh) continue;
        {
            const int nw = (int)(sizeof(ProblemC) / sizeof(int));
            const int *src = reinterpret_cast<const int *>(probs + s);
            int *dst = reinterpret_cast<int *>(&Ps);
            for (int t = threadIdx.x; t < nw; t += blockDim.x) dst[t] = src[t];
            if (threadIdx.x == 0) Sc = scen[s];
        }
        __syncthreads();
        const int Ns = Sc.N;
        if (w < Sc.T * Ns) {
            // tile slot q of N warps: claims tiles (wind sample, 32 particles) of
            // this scenario one at a time and synchronises its own warps only;
            // the scenario's offsets stay in shared memory (Sc), not in registers
            const int q = w / Ns, i = w - q * Ns;
            const int bar = 1 + q, cnt = Ns * 32;
            for (;;) {
                if (i == 0 && lane == 0) slot_item[q] = (long long)atomicAdd(claimed + s, 1ull);
                tile_barrier(bar, cnt);
                const long long it = slot_item[q];
                if (it >= items) break;
                const int m = (int)(it / nLb);
                const long long l0 = (it - (long long)m * nLb) * kPB;
                const float4 *Wm = W + Sc.w_off + (size_t)m * Ps.H * Ps.P;
                float *sp = spos + (size_t)q * tile_smem_words(Ns, Ps.wind_mode);
                const TileResult r =
                    Ps.rolling ? rollout_tile_mode<OwnWind, true, Soft, false>(Ps, dyns + s, u + Sc.u_off, Wm, L,
                                                                               l0, i, lane, m, J, sp, bar, cnt)
                               : rollout_tile_mode<OwnWind, false, Soft, false>(Ps, dyns + s, u + Sc.u_off, Wm, L,
                                                                                l0, i, lane, m, J, sp, bar, cnt);
                const size_t cbase = (size_t)Sc.seg_off * Ps.M * (size_t)L;
                store_tile(r, Ns, L, l0 + lane, i, lane, m, cost_ms + cbase,
                           cost_ms_soft ? cost_ms_soft + cbase : nullptr, live);
            }
        }
    }
}

// ------------------------------------------------------------- sample means

__global__ void __launch_bounds__(256) batch_sample_mean(const float *__restrict__ cost_ms,
                                                         const BatchScen *__restrict__ scen,
                                                         const int *__restrict__ seg_scen,
                                                         long long nseg, long long L, int M,
                                                         int Mj, float *__restrict__ cbar)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg * L) return;
    const long long seg = t / L, l = t - seg * L;
    const int s = seg_scen[seg];
    const BatchScen sc = scen[s];
    const int i = (int)(seg - sc.seg_off);
    const float *c = cost_ms + (size_t)sc.seg_off * M * L + (size_t)i * L + l;
    const size_t stride = (size_t)sc.N * L;
    Kahan acc;
    bool inf = false;
    for (int m = 0; m < Mj; ++m) {
        const float v = __ldg(c + (size_t)m * stride);
        if (isinf(v)) inf = true;
        else acc.add(v);
    }
    cbar[t] = inf ? __int_as_float(0x7f800000) : acc.s / (float)Mj;
}

// ----------------------------------------------------------- move and init

// kS: the segment count when fixed at compile time (4: the loop unrolls and
// every control's component is known), 0 when taken from S.
template <int kS = 0>
__global__ void __launch_bounds__(256) batch_move(const BatchScen *__restrict__ scen,
                                                  const int *__restrict__ seg_scen,
                                                  const DynState *__restrict__ dyns, long long nseg,
                                                  long long L, int S, const float *__restrict__ u,
                                                  const int32_t *__restrict__ anc, int J,
                                                  float *__restrict__ u_out, unsigned int *__restrict__ err)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg * L) return;
    const long long seg = t / L, l = t - seg * L;
    const int s = seg_scen[seg];
    const BatchScen sc = scen[s];
    const int i = (int)(seg - sc.seg_off);
    int a = __ldg(anc + t);
    if ((unsigned long long)a >= (unsigned long long)L) {   // reported, and a defined parent kept
        if (err) atomicOr(err, TMA_DEVERR_BOUNDS);
        a = (int)l;
    }
    const int nc = 3 * (kS > 0 ? kS : S);
    const float *src = u + sc.u_off + ((size_t)a * sc.N + i) * nc;
    float *dst = u_out + sc.u_off + ((size_t)l * sc.N + i) * nc;
    const uint32_t mpc = dyns[s].mpc_step;
#pragma unroll
    for (int q = 0; q < (nc + 3) / 4; ++q) {
        const uint4 r = draw(sc.key0, sc.key1, (uint32_t)l, (uint32_t)i, (uint32_t)q, 1u, (uint32_t)J, mpc);
        const float2 z01 = box_muller(r.x, r.y), z23 = box_muller(r.z, r.w);
        const float z[4] = {z01.x, z01.y, z23.x, z23.y};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int n = 4 * q + e;
            if (n < nc) {
                const int c = n % 3;
                dst[n] = clampf(fmaf(sc.move_sigma[c], z[e], __ldg(src + n)), sc.ctrl_lo[c], sc.ctrl_hi[c]);
            }
        }
    }
}

__global__ void __launch_bounds__(256) batch_init(const BatchScen *__restrict__ scen,
                                                  const int *__restrict__ seg_scen,
                                                  const DynState *__restrict__ dyns, long long nseg,
                                                  long long L, int S, float *__restrict__ u)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nseg * L) return;
    const long long seg = t / L, l = t - seg * L;
    const int s = seg_scen[seg];
    const BatchScen sc = scen[s];
    const int i = (int)(seg - sc.seg_off);
    const int nc = 3 * S;
    float *dst = u + sc.u_off + ((size_t)l * sc.N + i) * nc;
    const uint32_t mpc = dyns[s].mpc_step;
    for (int q = 0; q < (nc + 3) / 4; ++q) {
        const uint4 r = draw(sc.key0, sc.key1, (uint32_t)l, (uint32_t)i, (uint32_t)q, 4u, 0u, mpc);
        const uint32_t wv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int n = 4 * q + e;
            if (n < nc) {
                const int c = n % 3;
                dst[n] = fmaf(sc.ctrl_hi[c] - sc.ctrl_lo[c], uniform23(wv[e]), sc.ctrl_lo[c]);
            }
        }
    }
}

// ------------------------------------------------------------ wind normals

// As the single-scenario kernel, over (scenario of the group, sample, node);
// every scenario keys its own normals and uses its own MPC step.  w.M is the
// group's sample count (scenarios x M_scen).
__global__ void __launch_bounds__(128) batch_wind_normals_ar(const WindC w, int s0, int M_scen,
                                                             const BatchScen *__restrict__ scen,
                                                             const DynState *__restrict__ dyns,
                                                             float *__restrict__ Btmp)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)w.M * w.nxy) return;
    const int ms = (int)(t / w.nxy);           // (scenario in group, sample) < w.M
    const int q = (int)(t - (long long)ms * w.nxy);
    const int sl = ms / M_scen, m = ms - sl * M_scen;
    const int s = s0 + sl;
    const uint32_t mpc = dyns[s].mpc_step;
    const uint32_t k0 = scen[s].key0, k1 = scen[s].key1;
    const int nz = w.nz;
    float B[2][TMA_MAX_GRID_Z];
#pragma unroll
    for (int iz = 0; iz < TMA_MAX_GRID_Z; ++iz) B[0][iz] = B[1][iz] = 0.0f;
    float *row = Btmp + (size_t)q * w.ldb;
    for (int k = 0; k < w.H; ++k) {
#pragma unroll
        for (int iz = 0; iz < TMA_MAX_GRID_Z; ++iz) {
            if (iz < nz) {
                const uint4 r = draw(k0, k1, (uint32_t)(q * nz + iz), (uint32_t)m << 8, (uint32_t)k, 3u, 0u, mpc);
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
        float *o = row + ((size_t)ms * w.H + k) * (size_t)(2 * nz);
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

// --------------------------------------------------------------- selection

// One block per scenario: the particle with the fewest infeasible aircraft,
// then the smallest sum of mean costs (aircraft summed in order, FP64), ties
// to the lowest index (Sec. 3.8).  Copies the chosen controls and stamps the
// device clock when the scenario's solve is complete.
__global__ void __launch_bounds__(256) batch_select(const BatchScen *__restrict__ scen,
                                                    const float *__restrict__ cbar, long long L,
                                                    int S, const float *__restrict__ u,
                                                    long long *__restrict__ best,
                                                    double *__restrict__ best_sum,
                                                    int *__restrict__ ninf,
                                                    float *__restrict__ best_u,
                                                    unsigned long long *__restrict__ t_end)
{
    __shared__ int sn[256];
    __shared__ double ss[256];
    __shared__ long long sl[256];
    const int s = blockIdx.x;
    const BatchScen sc = scen[s];
    int bn = 1 << 30;
    double bs = 0.0;
    long long bl = 1ll << 62;
    for (long long l = threadIdx.x; l < L; l += blockDim.x) {
        int ni = 0;
        double sum = 0.0;
        for (int i = 0; i < sc.N; ++i) {
            const float c = __ldg(cbar + (size_t)(sc.seg_off + i) * L + l);
            if (isinf(c) || isnan(c)) ++ni;
            else sum += (double)c;
        }
        if (ni < bn || (ni == bn && (sum < bs || (sum == bs && l < bl)))) {
            bn = ni;
            bs = sum;
            bl = l;
        }
    }
    sn[threadIdx.x] = bn;
    ss[threadIdx.x] = bs;
    sl[threadIdx.x] = bl;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            const int n2 = sn[threadIdx.x + o];
            const double s2 = ss[threadIdx.x + o];
            const long long l2 = sl[threadIdx.x + o];
            const int n1 = sn[threadIdx.x];
            const double s1 = ss[threadIdx.x];
            const long long l1 = sl[threadIdx.x];
            if (n2 < n1 || (n2 == n1 && (s2 < s1 || (s2 == s1 && l2 < l1)))) {
                sn[threadIdx.x] = n2;
                ss[threadIdx.x] = s2;
                sl[threadIdx.x] = l2;
            }
        }
        __syncthreads();
    }
    const long long b = sl[0];
    const int nc = sc.N * S * 3;
    for (int j = threadIdx.x; j < nc; j += blockDim.x)
        best_u[(size_t)sc.seg_off * S * 3 + j] = u[sc.u_off + (size_t)b * nc + j];
    __syncthreads();
    if (threadIdx.x == 0) {
        best[s] = b;
        best_sum[s] = sn[0] == 0 ? ss[0] : __longlong_as_double(0x7ff0000000000000ll);
        ninf[s] = sn[0];
        __threadfence();
        t_end[s] = globaltimer();
    }
}

__global__ void stamp_start(unsigned long long *t0)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t0 = globaltimer();
}

// ------------------------------------------------------------------- plant

// The true system of Fig. 1: every aircraft flies its scenario's chosen
// controls of the first segment for one step dt.  The disturbance is the
// scenario's wind field of sample 0 at step 0 (in wind mode 1: step 0 of the
// corner-grid field of the reserved particle index 0xFFFFFFFF, sample 0) plus
// white turbulence from random stream 7; the climb angle is kept below 90 degrees and the thrust
// within its limits (the plant cannot refuse a command), and the speed and
// fuel follow from the applied thrust.  The state is written back for the
// next MPC step.  Rolling window: an aircraft that has not entered
// (t_enter > MPC step) or has finished keeps its state; an arrival that ends
// the step in the landing sector is marked finished.
__global__ void __launch_bounds__(128) plant_step_kernel(const ProblemC *__restrict__ probs,
                                                         const BatchScen *__restrict__ scen,
                                                         const int *__restrict__ seg_scen,
                                                         long long nseg, DynState *__restrict__ dyns,
                                                         const float4 *__restrict__ W,
                                                         const float *__restrict__ best_u, int S)
{
    const long long seg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (seg >= nseg) return;
    const int s = seg_scen[seg];
    const BatchScen sc = scen[s];
    const ProblemC &P = probs[s];
    const int i = (int)(seg - sc.seg_off);
    const AircraftC &A = P.ac[i];
    DynState &d = dyns[s];
    if (P.rolling && ((((d.finished >> i) & 1u) != 0u) || (long long)A.t_enter > (long long)d.mpc_step))
        return;
    const float x = d.x0[i][0], y = d.x0[i][1], z = d.x0[i][2];
    const float v = d.x0[i][3], chi = d.x0[i][4], mass = d.x0[i][5];
    const float *uu = best_u + (size_t)seg * S * 3;   // segment 0 of this aircraft
    const float uw = uu[0], uh = uu[1], ua = uu[2];
    const float dt = P.dt;
    const float sg = fmaxf(fminf(uh / v, 0.999f), -0.999f);
    const float cg = sqrtf(1.0f - sg * sg);
    const float tp = uw * v / (kG0 * cg);
    const float secphi = sqrtf(fmaf(tp, tp, 1.0f));
    const float rho = 1.225f * exp2f(4.2559f * __log2f(fmaxf(fmaf(-2.2558e-5f, z, 1.0f), 1e-30f)));
    const float qS = A.halfS * rho * v * v;
    const float CL = mass * kG0 * cg * secphi / qS;
    const float D = qS * fmaf(A.CD2, CL * CL, A.CD0);
    const float T = clampf(fmaf(mass, fmaf(kG0, sg, ua), D), A.Tmin, A.Tmax);
    float2 w;
    if (P.wind_mode == 1) {
        float B[16];                   // B(0) = v(0): draws r = 0..3 of stream 9
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 e = draw(P.key0, P.key1, 0xFFFFFFFFu, (uint32_t)q, 0u, 9u, 0u, d.mpc_step);
            const float2 v0 = box_muller(e.x, e.y), v1 = box_muller(e.z, e.w);
            B[4 * q] = v0.x;
            B[4 * q + 1] = v0.y;
            B[4 * q + 2] = v1.x;
            B[4 * q + 3] = v1.y;
        }
        w = particle_wind_at<1>(P, B, x, y, z);
    } else {
        w = wind_interp(wind_fetch(P, W + sc.w_off, x, y, z));
    }
    const uint4 r = draw(P.key0, P.key1, 0u, (uint32_t)i, 0u, 7u, 0u, d.mpc_step);
    const float2 n = box_muller(r.x, r.y);
    w.x = fmaf(P.turb_sigma, n.x, w.x);
    w.y = fmaf(P.turb_sigma, n.y, w.y);
    float sc_, cc_;
    sincosf(chi, &sc_, &cc_);
    const float eta = A.Cf1 * fmaf(v, A.invCf2, 1.0f);
    // Eq. (hor) with the applied (possibly limited) thrust T
    d.x0[i][0] = fmaf(dt, fmaf(v * cg, cc_, w.x), x);
    d.x0[i][1] = fmaf(dt, fmaf(v * cg, sc_, w.y), y);
    d.x0[i][2] = fmaf(dt, v * sg, z);
    d.x0[i][3] = fmaf(dt, (T - D) / mass - kG0 * sg, v);
    d.x0[i][4] = fmaf(dt, uw, chi);
    d.x0[i][5] = mass - dt * eta * T;
    if (P.rolling && A.type == 0) {
        // only this thread sets bit i; the others read their own bits
        const float x1 = d.x0[i][0], y1 = d.x0[i][1];
        const float th = atan2_poly(y1, x1);
        float r, ath;
        const float beta = arc_glide(x1, y1, d.x0[i][2], th, r, ath);
        if (in_landing_sector(P, x1, r, ath, beta, d.x0[i][4], d.x0[i][3])) atomicOr(&d.finished, 1u << i);
    }
}

__global__ void advance_mpc_step(DynState *__restrict__ dyns, int n_scen)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_scen) dyns[s].mpc_step += 1u;
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// A CTA of 32 warps holds floor(32 / N) tiles of N warps: the most shared
// memory over every aircraft count.
size_t batch_rollout_smem()
{
    size_t best = 0;
    for (int n = 1; n <= kMaxN; ++n)
        best = std::max(best, (size_t)std::min(15, 32 / n) * tile_smem_words(n, 1) * sizeof(float));
    return best;
}

cudaError_t launch_batch_rollout(const ProblemC *probs, const BatchScen *scen, int n_scen,
                                 const DynState *dyns, const float *u, const float *W, long long L,
                                 int J, int Mj, float *cost_ms, float *cost_ms_soft,
                                 unsigned long long *live, unsigned long long *claimed, int grid,
                                 int wind_mode, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(claimed, 0, sizeof(unsigned long long) * (size_t)n_scen, st);
    if (e != cudaSuccess) return e;
    const int nLb = (int)((L + kPB - 1) / kPB);
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
#define TMA_BATCH_K(O, F)                                                                        \
    rollout_batched_kernel<O, F><<<grid, 1024, batch_rollout_smem(), st>>>(                      \
        probs, scen, n_scen, dyns, u, W4, L, nLb, J, Mj, cost_ms, cost_ms_soft, live, claimed)
    if (wind_mode == 1) {
        if (cost_ms_soft) TMA_BATCH_K(true, true);
        else TMA_BATCH_K(true, false);
    } else {
        if (cost_ms_soft) TMA_BATCH_K(false, true);
        else TMA_BATCH_K(false, false);
    }
#undef TMA_BATCH_K
    count_launch();
    return cudaGetLastError();
}

int batch_rollout_grid()
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // every instance: 1024 threads, the same shared memory, 64 registers
    const void *kernels[] = {(const void *)rollout_batched_kernel<false, false>,
                             (const void *)rollout_batched_kernel<false, true>,
                             (const void *)rollout_batched_kernel<true, false>,
                             (const void *)rollout_batched_kernel<true, true>};
    per_sm = 1 << 30;
    for (const void *k : kernels) {
        int n = 0;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_rollout_smem());
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 1024, batch_rollout_smem()) != cudaSuccess) n = 1;
        per_sm = std::min(per_sm, n);
    }
    per_sm = std::max(1, per_sm);
    return sms * per_sm;
}

cudaError_t launch_batch_sample_mean(const float *cost_ms, const BatchScen *scen,
                                     const int *seg_scen, long long nseg, long long L, int M,
                                     int Mj, float *cbar, cudaStream_t st)
{
    batch_sample_mean<<<blocks_for(nseg * L, 256), 256, 0, st>>>(cost_ms, scen, seg_scen, nseg, L, M,
                                                                 Mj, cbar);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_move(const BatchScen *scen, const int *seg_scen, const DynState *dyns,
                              long long nseg, long long L, int S, const float *u,
                              const int32_t *anc, int J, float *u_out, cudaStream_t st, unsigned int *err)
{
    if (S == 4)
        batch_move<4><<<blocks_for(nseg * L, 256), 256, 0, st>>>(scen, seg_scen, dyns, nseg, L, S, u, anc, J,
                                                                 u_out, err);
    else
        batch_move<<<blocks_for(nseg * L, 256), 256, 0, st>>>(scen, seg_scen, dyns, nseg, L, S, u, anc, J, u_out,
                                                              err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_init(const BatchScen *scen, const int *seg_scen, const DynState *dyns,
                              long long nseg, long long L, int S, float *u, cudaStream_t st)
{
    batch_init<<<blocks_for(nseg * L, 256), 256, 0, st>>>(scen, seg_scen, dyns, nseg, L, S, u);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_wind_normals(const WindC &w, int s0, int M_scen, const BatchScen *scen,
                                      const DynState *dyns, float *Btmp, cudaStream_t st)
{
    batch_wind_normals_ar<<<blocks_for((long long)w.M * w.nxy, 128), 128, 0, st>>>(w, s0, M_scen, scen, dyns, Btmp);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_select(const BatchScen *scen, int n_scen, const float *cbar, long long L,
                                int S, const float *u, long long *best, double *best_sum, int *ninf,
                                float *best_u, unsigned long long *t_end, cudaStream_t st)
{
    batch_select<<<n_scen, 256, 0, st>>>(scen, cbar, L, S, u, best, best_sum, ninf, best_u, t_end);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stamp_start(unsigned long long *t0, cudaStream_t st)
{
    stamp_start<<<1, 32, 0, st>>>(t0);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_plant_step(const ProblemC *probs, const BatchScen *scen, const int *seg_scen,
                              long long nseg, int n_scen, DynState *dyns, const float *W,
                              const float *best_u, int S, cudaStream_t st)
{
    plant_step_kernel<<<blocks_for(nseg, 128), 128, 0, st>>>(probs, scen, seg_scen, nseg, dyns,
                                                              reinterpret_cast<const float4 *>(W), best_u, S);
    advance_mpc_step<<<blocks_for(n_scen, 128), 128, 0, st>>>(dyns, n_scen);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace tma
