// One rollout tile: 32 particles x N aircraft under one wind sample (the inner
// loop of Algorithm 1; Sec. 3.3-3.6, Sec. 7.1).  Shared by the single-scenario
// kernel (rollout.cu) and the batched persistent kernel (batch.cu).
//
// The N warps of a tile each simulate one aircraft (warp-uniform type,
// constants and wind field) for 32 particles (lane j = particle l0 + j), with
// the aircraft state and cost accumulators in registers for the whole
// horizon.  The pairwise separation check of Eq. (avoidance) reads the other
// aircraft's positions of the same particle from the tile's shared-memory
// buffer, double-buffered by step, behind one barrier per step.
#pragma once

#include "device_common.cuh"
#include "tma_internal.h"

namespace tma {


constexpr float kG0 = 9.80665f;
constexpr float kPi = 3.14159265358979323846f;

// Trilinear interpolation of one wind field (Sec. 3.9.1) at a position clamped
// into the grid box: wind_fetch locates the cell and loads its four packed
// columns (float4 per node: own (x, y) value and the value one level up),
// wind_interp combines them.
struct WindFetch {
    float4 a00, a01, a10, a11;
    float tx, ty, tz;
};

__device__ __forceinline__ WindFetch wind_fetch(const ProblemC &P, const float4 *__restrict__ Wk,
                                                float x, float y, float z)
{
    const float pos[3] = {x, y, z};
    int idx[3];
    float t[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float c = fminf(fmaxf(pos[d], P.box_lo[d]), P.box_hi[d]);
        const float f = (c - P.box_lo[d]) * P.inv_h[d];
        const int i = min((int)f, P.grid[d] - 2);
        idx[d] = i;
        t[d] = f - (float)i;
    }
    const int nz = P.grid[2];
    const int nyz = P.grid[1] * nz;
    const int p = (idx[0] * P.grid[1] + idx[1]) * nz + idx[2];
    WindFetch r;
    r.a00 = __ldg(Wk + p);
    r.a01 = __ldg(Wk + p + nz);
    r.a10 = __ldg(Wk + p + nyz);
    r.a11 = __ldg(Wk + p + nyz + nz);
    r.tx = t[0];
    r.ty = t[1];
    r.tz = t[2];
    return r;
}

__device__ __forceinline__ float2 wind_interp(const WindFetch &f)
{
    float2 c00, c01, c10, c11, c0, c1, r;
    c00.x = fmaf(f.tz, f.a00.z - f.a00.x, f.a00.x); c00.y = fmaf(f.tz, f.a00.w - f.a00.y, f.a00.y);
    c01.x = fmaf(f.tz, f.a01.z - f.a01.x, f.a01.x); c01.y = fmaf(f.tz, f.a01.w - f.a01.y, f.a01.y);
    c10.x = fmaf(f.tz, f.a10.z - f.a10.x, f.a10.x); c10.y = fmaf(f.tz, f.a10.w - f.a10.y, f.a10.y);
    c11.x = fmaf(f.tz, f.a11.z - f.a11.x, f.a11.x); c11.y = fmaf(f.tz, f.a11.w - f.a11.y, f.a11.y);
    c0.x = fmaf(f.ty, c01.x - c00.x, c00.x); c0.y = fmaf(f.ty, c01.y - c00.y, c00.y);
    c1.x = fmaf(f.ty, c11.x - c10.x, c10.x); c1.y = fmaf(f.ty, c11.y - c10.y, c10.y);
    r.x = fmaf(f.tx, c1.x - c0.x, c0.x);
    r.y = fmaf(f.tx, c1.y - c0.y, c0.y);
    return r;
}

// Population density of Sec. 7.1: bilinear between grid nodes, 0 outside.
__device__ __forceinline__ float popdense_at(const ProblemC &P, float x, float y)
{
    if (P.popdense == nullptr) return 0.0f;
    if (!(x >= P.pop_lo[0] && x <= P.pop_hi[0] && y >= P.pop_lo[1] && y <= P.pop_hi[1]))
        return 0.0f;
    const float f0 = (x - P.pop_lo[0]) * P.pop_inv_h[0];
    const float f1 = (y - P.pop_lo[1]) * P.pop_inv_h[1];
    const int i0 = min((int)f0, P.pop_n[0] - 2), i1 = min((int)f1, P.pop_n[1] - 2);
    const float t0 = f0 - (float)i0, t1 = f1 - (float)i1;
    const float *g = P.popdense + (size_t)i0 * P.pop_n[1] + i1;
    const float g00 = __ldg(g), g01 = __ldg(g + 1);
    const float g10 = __ldg(g + P.pop_n[1]), g11 = __ldg(g + P.pop_n[1] + 1);
    const float a = fmaf(t1, g01 - g00, g00), b = fmaf(t1, g11 - g10, g10);
    return fmaf(t0, b - a, a);
}

__device__ __forceinline__ float softplus(float g, float beta, float inv_beta)
{
    const float bg = beta * g;
    return bg > 0.0f ? (bg + log1pf(__expf(-bg))) * inv_beta : log1pf(__expf(bg)) * inv_beta;
}

constexpr int kPB = kTileParticles;

__device__ __forceinline__ void tile_barrier(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Simulates aircraft i (this warp) of particles l0..l0+31 (lane j) under the
// packed wind field Wm of sample m, and writes the per-sample costs
// cost_ms[(m N + i) L + l] (and the softplus variant when cost_ms_soft is not
// null).  spos is the tile's [2][3][N][32] float buffer; every warp of the
// tile must call this with the same barrier (bar_id, bar_count threads).
__device__ __forceinline__ void rollout_tile(const ProblemC &P, const DynState *__restrict__ dyn,
                                             const float *__restrict__ u,
                                             const float4 *__restrict__ Wm, long long L,
                                             long long l0, int i, int j, int m, int J,
                                             float *__restrict__ cost_ms,
                                             float *__restrict__ cost_ms_soft,
                                             unsigned long long *__restrict__ live, float *spos,
                                             int bar_id, int bar_count)
{
    const int N = P.N;
    const long long l = l0 + j;
    const bool exists = l < L;
    const AircraftC &A = P.ac[i];
    const uint32_t mpc = dyn->mpc_step;
    const float dt = P.dt;

    float x = dyn->x0[i][0], y = dyn->x0[i][1], z = dyn->x0[i][2];
    float v = dyn->x0[i][3], chi = dyn->x0[i][4];
    const float m0 = dyn->x0[i][5];
    // departure altitude term: sup / inf of the per-step distance to Z reachable
    // from the current altitude at the maximum climb rate c (Sec. 3.5), in closed
    // form: sup = d0 + c (H+1)/2, inf = (K d0 - c K (K+1)/2) / H, K = min(H, floor(d0/c))
    const float d0 = fabsf(A.Z - z);
    const float supB = fmaf(P.climb_step, 0.5f * (float)(P.H + 1), d0);
    const float Kf = fminf((float)P.H, floorf(__fdividef(d0, P.climb_step)));
    const float infB = (Kf * d0 - P.climb_step * 0.5f * Kf * (Kf + 1.0f)) / (float)P.H;
    const float invSupInf = 1.0f / (supB - infB);
    Kahan F, sA, sB, sC;
    float sN = 0.0f, soft = 0.0f;
    bool dead = !exists, landed = false, sepv = false;
    int seg = -1, ks = 0, knext = 0;
    float uw = 0.0f, uh = 0.0f, ua = 0.0f;
    // within a control segment z, v and chi are linear in time: evaluate them
    // from the segment's start values so that rounding does not accumulate
    float zb = 0.0f, vb = 0.0f, cb = 0.0f;
    const float *ul = u + ((size_t)(exists ? l : 0) * N + i) * (size_t)(P.S * 3);
    float2 turb_next = make_float2(0.0f, 0.0f);
    unsigned int nlive = 0;
    const bool soft_on = cost_ms_soft != nullptr;
    const int plane = N * kPB;

    for (int k = 0; k < P.H; ++k) {
        if (!dead && !landed) {
            ++nlive;
            if (k >= knext) {
                // segment s = floor(k S / H) starts at step ceil(s H / S)
                seg = (k * P.S) / P.H;
                knext = ((seg + 1) * P.H + P.S - 1) / P.S;
                ks = k;
                uw = __ldg(ul + 3 * seg);
                uh = __ldg(ul + 3 * seg + 1);
                ua = __ldg(ul + 3 * seg + 2);
                zb = z;
                vb = v;
                cb = chi;
            }
            const float mass = m0 - F.s;
            // control-derived quantities and their limits (Sec. 3.4)
            const float sg = __fdividef(uh, v);
            bool ok = fabsf(sg) <= P.sgmax;
            const float cg = sqrtf(fmaxf(1.0f - sg * sg, 0.0f));
            const float tp = __fdividef(uw * v, kG0 * cg);
            ok = ok && (fabsf(tp) < P.tpmax);
            const float secphi = sqrtf(fmaf(tp, tp, 1.0f));
            const float rho = 1.225f * exp2f(4.2559f * __log2f(fmaxf(fmaf(-2.2558e-5f, z, 1.0f), 1e-30f)));
            const float qS = A.halfS * rho * v * v;
            const float CL = __fdividef(mass * kG0 * cg * secphi, qS);
            const float D = qS * fmaf(A.CD2, CL * CL, A.CD0);
            const float T = fmaf(mass, fmaf(kG0, sg, ua), D);
            ok = ok && (T >= A.Tmin) && (T <= A.Tmax);
            if (!ok) {
                dead = true;
            } else {
                // disturbance: wind field of sample m plus white turbulence
                float2 w = wind_interp(wind_fetch(P, Wm + (size_t)k * P.P, x, y, z));
                float2 n;
                if ((k & 1) == 0) {
                    const uint4 r = draw(P.key0, P.key1, (uint32_t)l, (uint32_t)i | ((uint32_t)m << 8),
                                         (uint32_t)(k >> 1), 0u, (uint32_t)J, mpc);
                    n = box_muller_fast(r.x, r.y);
                    turb_next = box_muller_fast(r.z, r.w);
                } else {
                    n = turb_next;
                }
                w.x = fmaf(P.turb_sigma, n.x, w.x);
                w.y = fmaf(P.turb_sigma, n.y, w.y);
                // explicit Euler step of Eq. (hor); v sin(gamma) = hdot, the
                // speed equation reduces to v += dt a and the heading equation
                // to chi += dt w (coordinated turn)
                float sc, cc;
                sincos_reduced(chi, &sc, &cc);
                const float vh = v * cg;
                x = fmaf(dt, fmaf(vh, cc, w.x), x);
                y = fmaf(dt, fmaf(vh, sc, w.y), y);
                const float nk = (float)(k + 1 - ks) * dt;
                z = fmaf(nk, uh, zb);
                const float eta = A.Cf1 * fmaf(v, A.invCf2, 1.0f);
                F.add(dt * eta * T);
                v = fmaf(nk, ua, vb);
                chi = fmaf(nk, uw, cb);
                const float mass1 = m0 - F.s;
                if (!(z >= P.z_min && z <= P.z_max && v >= P.v_min && v <= P.v_max &&
                      mass1 >= A.m_empty)) {
                    dead = true;
                } else {
                    const float th = atan2f(y, x);
                    if (A.type == 0) {
                        // arrival: flow-field arc, glide angle and landing sector
                        const float r = sqrtf(fmaf(x, x, y * y));
                        const float ath = fabsf(th);
                        const float ratio = ath < 1e-3f ? fmaf(th * th, 1.0f / 6.0f, 1.0f)
                                                        : __fdividef(ath, fmaxf(__sinf(ath), 0.25f * ath));
                        const float beta = atan2f(z, r * ratio);
                        const float hdg = angdist(chi - kPi);
                        if (r <= P.P_runway && beta <= P.P_beta && x > 0.0f && ath <= P.P_chi &&
                            hdg <= P.P_chi && v <= P.P_vs) {
                            landed = true;
                        } else {
                            sA.add(angdist(chi - fmaf(2.0f, th, kPi)));
                            sB.add(fabsf(beta - P.beta_f));
                        }
                    } else {
                        sA.add(angdist(th - A.thF));
                        sB.add(fabsf(A.Z - z));
                        sC.add(fabsf(v - A.vD));
                    }
                    if (P.w_noise != 0.0f && !landed) {
                        const float za = z * P.Ac_inv;
                        const float h = fmaxf(fmaf(-za, za, 1.0f), 0.0f);
                        sN = fmaf(h, popdense_at(P, x, y), sN);
                    }
                }
            }
        }
        // binary separation constraints at step k+1 among flying aircraft: every
        // thread publishes its position (a far-away altitude when not flying)
        const bool act = !dead && !landed;
        float *buf = spos + (k & 1) * 3 * plane;
        buf[i * kPB + j] = x;
        buf[plane + i * kPB + j] = y;
        buf[2 * plane + i * kPB + j] = act ? z : 1e30f;
        tile_barrier(bar_id, bar_count);
        if (act) {
            for (int i2 = 0; i2 < N; ++i2) {
                if (i2 == i) continue;
                const float dx = x - buf[i2 * kPB + j];
                const float dy = y - buf[plane + i2 * kPB + j];
                const float adz = fabsf(z - buf[2 * plane + i2 * kPB + j]);
                const float dh2 = fmaf(dx, dx, dy * dy);
                if (dh2 < P.Sh2 && adz < P.Sv) sepv = true;
                if (soft_on) {
                    const float g = fminf(fmaf(-sqrtf(dh2), P.Sh_inv, 1.0f),
                                          fmaf(-adz, P.Sv_inv, 1.0f));
                    soft += softplus(g, P.sp_beta, P.sp_inv_beta);
                }
            }
        }
    }

    // objectives (Sec. 3.5, Sec. 7.1) and the per-sample cost -ln J_T
    const float invH = 1.0f / (float)P.H;
    const float Jf = fmaf(-F.s, A.invFmax, 1.0f);
    float Jsum;
    if (A.type == 1) {
        const float J1 = fmaf(-sA.s * invH, 1.0f / kPi, 1.0f);
        const float J3 = (supB - sB.s * invH) * invSupInf;
        const float J4 = fmaf(-sC.s * invH, A.invCmax, 1.0f);
        Jsum = P.a_dep[0] * J1 + P.a_dep[1] * Jf + P.a_dep[2] * J3 + P.a_dep[3] * J4;
    } else {
        const float J1 = fmaf(-sA.s * invH, 1.0f / kPi, 1.0f);
        const float J3 = fmaf(-sB.s * invH, 2.0f / kPi, 1.0f);
        Jsum = P.a_arr[0] * J1 + P.a_arr[1] * J3 + P.a_arr[2] * Jf;
    }
    const float JT = (1.0f - P.w_noise) * Jsum + P.w_noise * fmaf(-sN, invH, 1.0f);
    const float c = -logf(fmaxf(JT, 1e-30f));
    if (exists) {
        const size_t o = ((size_t)m * N + i) * (size_t)L + l;
        cost_ms[o] = (dead || sepv) ? __int_as_float(0x7f800000) : c;
        if (soft_on) cost_ms_soft[o] = dead ? __int_as_float(0x7f800000) : fmaf(P.mu_sep, soft, c);
    }
    if (live != nullptr) {
        const unsigned int tot = __reduce_add_sync(0xffffffffu, exists ? nlive : 0u);
        if (j == 0 && tot) atomicAdd(live, (unsigned long long)tot);
    }
}

}  // namespace tma
