// Metropolis-Hastings moves of whole particles (an extension of the
// perturbation step of Algorithm 1; the paper's own move has no accept step).
// Target at iteration J: pi_J(u) proportional to exp(-kappa_J C(u)),
// C(u) = sum_i cbar_soft[i](u), with the iteration's wind samples.  The
// controls are scaled by the move step sigma of each control kind (turn rate,
// climb rate, speed change): with z = u / sigma the proposals are
//   random walk   z' = z + eps xi
//   Langevin      z' = z - (eps^2 / 2) kappa grad_z C(z) + eps xi,
//                 grad_z C = sigma * grad_u C,
// xi standard normal from random stream 5; proposals outside the control box
// are rejected; the accept test uses one uniform of stream 6 and is taken in
// FP64.  One warp per particle: lanes run over the N * S * 3 controls.
#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {

namespace {

// normal number e of aircraft i of particle l (e = s * 3 + c): word e % 4 of
// draw q = e / 4 of stream 5; words (0, 1) and (2, 3) each give one
// Box-Muller pair.
__device__ __forceinline__ float mh_normal(uint32_t k0, uint32_t k1, uint32_t l, uint32_t i,
                                           uint32_t e, uint32_t J, uint32_t mpc)
{
    const uint4 r = draw(k0, k1, l, i, e >> 2, 5u, J, mpc);
    const uint32_t w = e & 3u;
    const float2 p = w < 2 ? box_muller(r.x, r.y) : box_muller(r.z, r.w);
    return (w & 1u) ? p.y : p.x;
}

__global__ void __launch_bounds__(256) mh_propose_kernel(MhParams h, const DynState *__restrict__ dyn,
                                                         const float *__restrict__ u,
                                                         const float *__restrict__ grad, long long L,
                                                         int J, float kappa,
                                                         const double *__restrict__ d_eps,
                                                         float *__restrict__ u_prop,
                                                         uint8_t *__restrict__ inbox)
{
    const long long l = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= L) return;
    const uint32_t mpc = dyn->mpc_step;
    const float eps = (float)*d_eps;
    const float drift = h.langevin ? 0.5f * eps * eps * kappa : 0.0f;
    const int nS3 = h.S * 3;
    const int nel = h.N * nS3;
    bool ok = true;
    for (int n = lane; n < nel; n += 32) {
        const int i = n / nS3, e = n - i * nS3, c = e % 3;
        const size_t o = (size_t)l * nel + n;
        const float sg = h.sigma[c];
        const float xi = mh_normal(h.key0, h.key1, (uint32_t)l, (uint32_t)i, (uint32_t)e, (uint32_t)J, mpc);
        float v = u[o];
        if (h.langevin) v = fmaf(-drift * sg * sg, grad[o], v);
        v = fmaf(eps * sg, xi, v);
        u_prop[o] = v;
        ok = ok && v >= h.lo[c] && v <= h.hi[c];
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) inbox[l] = ok ? 1 : 0;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) mh_accept_kernel(
    MhParams h, const DynState *__restrict__ dyn, const float *__restrict__ u,
    const float *__restrict__ up, const float *__restrict__ cbar, const float *__restrict__ cbarp,
    const float *__restrict__ g, const float *__restrict__ gp, const uint8_t *__restrict__ inbox,
    long long L, int J, float kappa, const double *__restrict__ d_eps, float *__restrict__ u_out,
    float *__restrict__ cbar_out, uint8_t *__restrict__ accepted,
    unsigned int *__restrict__ n_accept)
{
    const long long l = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= L) return;
    const int N = h.N, nS3 = h.S * 3, nel = N * nS3;
    // C(u) and C(u') summed over aircraft (FP64)
    double c = 0.0, cp = 0.0;
    bool inf = false, infp = false;
    if (lane < N) {
        const float a = cbar[(size_t)lane * L + l], b = cbarp[(size_t)lane * L + l];
        inf = isinf(a);
        infp = isinf(b);
        c = inf ? 0.0 : (double)a;
        cp = infp ? 0.0 : (double)b;
    }
    inf = __any_sync(0xffffffffu, inf);
    infp = __any_sync(0xffffffffu, infp);
    c = warp_sum(c);
    cp = warp_sum(cp);
    const double eps = *d_eps;
    double lq = 0.0;
    if (h.langevin) {
        // log q(u | u') - log q(u' | u) in the scaled coordinates
        const double d = 0.5 * eps * eps * (double)kappa;
        double fw = 0.0, bw = 0.0;
        for (int n = lane; n < nel; n += 32) {
            const size_t o = (size_t)l * nel + n;
            const double sg = (double)h.sigma[n % nS3 % 3];
            const double dz = ((double)up[o] - (double)u[o]) / sg;
            const double b = -dz + d * sg * (double)gp[o];     // z - z' + d grad_z(z')
            const double f = dz + d * sg * (double)g[o];       // z' - z + d grad_z(z)
            bw = fma(b, b, bw);
            fw = fma(f, f, fw);
        }
        bw = warp_sum(bw);
        fw = warp_sum(fw);
        lq = -(bw - fw) / (2.0 * eps * eps);
    }
    bool acc;
    if (!inbox[l] || infp) {
        acc = false;
    } else if (inf) {
        acc = true;
    } else {
        const double log_alpha = -(double)kappa * (cp - c) + lq;
        const uint4 r = draw(h.key0, h.key1, (uint32_t)l, 0u, 0u, 6u, (uint32_t)J, dyn->mpc_step);
        const double U = ((double)(r.x >> 9) + 0.5) * (1.0 / 8388608.0);
        acc = log(U) < log_alpha;
    }
    for (int n = lane; n < nel; n += 32) {
        const size_t o = (size_t)l * nel + n;
        u_out[o] = acc ? up[o] : u[o];
    }
    if (cbar_out && lane < N)
        cbar_out[(size_t)lane * L + l] = acc ? cbarp[(size_t)lane * L + l] : cbar[(size_t)lane * L + l];
    if (lane == 0) {
        if (accepted) accepted[l] = acc ? 1 : 0;
        if (acc && n_accept) atomicAdd(n_accept, 1u);
    }
}

// Step-size adaptation between iterations: eps is scaled by 0.8 when the
// acceptance rate of the last move fell below 0.5 and by 1.25 above 0.7; the
// count is kept in the per-iteration history and reset.
__global__ void mh_adapt_kernel(double *eps, unsigned int *n_accept, unsigned int *history,
                                double *eps_history, int J, long long L)
{
    const double rate = (double)*n_accept / (double)L;
    if (history) history[J] = *n_accept;
    if (eps_history) eps_history[J] = *eps;
    if (rate < 0.5) *eps *= 0.8;
    else if (rate > 0.7) *eps *= 1.25;
    *n_accept = 0;
}

}  // namespace

cudaError_t launch_mh_propose(const MhParams &h, const DynState *dyn, const float *u,
                              const float *grad, int64_t L, int J, float kappa, const double *d_eps,
                              float *u_prop, uint8_t *inbox, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    mh_propose_kernel<<<(unsigned)((L * 32 + 255) / 256), 256, 0, st>>>(h, dyn, u, grad, L, J, kappa,
                                                                        d_eps, u_prop, inbox);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mh_accept(const MhParams &h, const DynState *dyn, const float *u, const float *up,
                             const float *cbar, const float *cbarp, const float *g, const float *gp,
                             const uint8_t *inbox, int64_t L, int J, float kappa,
                             const double *d_eps, float *u_out, float *cbar_out, uint8_t *accepted,
                             unsigned int *n_accept, cudaStream_t st)
{
    if (L <= 0) return cudaSuccess;
    mh_accept_kernel<<<(unsigned)((L * 32 + 255) / 256), 256, 0, st>>>(
        h, dyn, u, up, cbar, cbarp, g, gp, inbox, L, J, kappa, d_eps, u_out, cbar_out, accepted,
        n_accept);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mh_adapt(double *eps, unsigned int *n_accept, unsigned int *history,
                            double *eps_history, int J, int64_t L, cudaStream_t st)
{
    mh_adapt_kernel<<<1, 1, 0, st>>>(eps, n_accept, history, eps_history, J, L);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
