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
// columns (float4 per node: own (x, y) value and the difference to the node one
// level up), wind_interp combines them.
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
    c00.x = fmaf(f.tz, f.a00.z, f.a00.x); c00.y = fmaf(f.tz, f.a00.w, f.a00.y);
    c01.x = fmaf(f.tz, f.a01.z, f.a01.x); c01.y = fmaf(f.tz, f.a01.w, f.a01.y);
    c10.x = fmaf(f.tz, f.a10.z, f.a10.x); c10.y = fmaf(f.tz, f.a10.w, f.a10.y);
    c11.x = fmaf(f.tz, f.a11.z, f.a11.x); c11.y = fmaf(f.tz, f.a11.w, f.a11.y);
    c0.x = fmaf(f.ty, c01.x - c00.x, c00.x); c0.y = fmaf(f.ty, c01.y - c00.y, c00.y);
    c1.x = fmaf(f.ty, c11.x - c10.x, c10.x); c1.y = fmaf(f.ty, c11.y - c10.y, c10.y);
    r.x = fmaf(f.tx, c1.x - c0.x, c0.x);
    r.y = fmaf(f.tx, c1.y - c0.y, c0.y);
    return r;
}

// Angle of (x, y) in (-pi, pi], as atan2: t = min/max of |x|, |y| in [0, 1],
// atan(t) = t P(t^2) with the degree-8 polynomial of a weighted least-squares
// fit on Chebyshev nodes (fit_atan.py beside this file; 1e-7 rad in FP32),
// then the octant.  (0, 0) gives 0.
__device__ __forceinline__ float atan2_poly(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float s = t * t;
    float p = 2.932487579e-03f;
    p = fmaf(p, s, -1.641217540e-02f);
    p = fmaf(p, s, 4.327672817e-02f);
    p = fmaf(p, s, -7.556783848e-02f);
    p = fmaf(p, s, 1.066743802e-01f);
    p = fmaf(p, s, -1.421109512e-01f);
    p = fmaf(p, s, 1.999369316e-01f);
    p = fmaf(p, s, -3.333313793e-01f);
    p = fmaf(p, s, 9.999999938e-01f);
    float a = t * p;
    if (ay > ax) a = 1.57079632679489662f - a;
    if (x < 0.0f) a = 3.14159265358979324f - a;
    return copysignf(a, y);
}

// 2^x by the hardware approximation (relative error near 2^-22).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Population density of Sec. 7.1: bilinear between grid nodes, 0 outside (the
// cell's four corners in one load).
__device__ __forceinline__ float popdense_at(const ProblemC &P, float x, float y)
{
    if (P.popcell == nullptr) return 0.0f;
    if (!(x >= P.pop_lo[0] && x <= P.pop_hi[0] && y >= P.pop_lo[1] && y <= P.pop_hi[1]))
        return 0.0f;
    const float f0 = (x - P.pop_lo[0]) * P.pop_inv_h[0];
    const float f1 = (y - P.pop_lo[1]) * P.pop_inv_h[1];
    const int i0 = min((int)f0, P.pop_n[0] - 2), i1 = min((int)f1, P.pop_n[1] - 2);
    const float t0 = f0 - (float)i0, t1 = f1 - (float)i1;
    const float4 g = __ldg(P.popcell + (size_t)i0 * (P.pop_n[1] - 1) + i1);   // g00, g01, g10, g11
    const float a = fmaf(t1, g.y - g.x, g.x), b = fmaf(t1, g.w - g.z, g.z);
    return fmaf(t0, b - a, a);
}

// ln(1 + e) for 0 <= e <= 1: e itself below 2^-12 (error below e^2/2 < 2^-13 e),
// else the hardware logarithm of 1 + e (absolute error near 2^-24).
__device__ __forceinline__ float log1p_unit(float e)
{
    return e < 2.44140625e-4f ? e : __logf(1.0f + e);
}

// Softplus penalty ln(1 + exp(beta g)) / beta of Eq. (avoidance) in soft form,
// as max(beta g, 0) + ln(1 + exp(-|beta g|)).
__device__ __forceinline__ float softplus(float g, float beta, float inv_beta)
{
    const float bg = beta * g;
    return (fmaxf(bg, 0.0f) + log1p_unit(__expf(-fabsf(bg)))) * inv_beta;
}

constexpr int kPB = kTileParticles;
// partners screened per group (the group's loads in flight together)
constexpr int kScreen = 2;

// Mode-1 wind (a field per (particle, sample) on the 2x2x2 grid of the box
// corners, the paper's scheme): the state B of the particle's eight nodes lives
// in the tile's shared buffer pw[2 (step parity)][16 (node * 2 + component)][32
// lanes].  Draw r = 0..3 of random stream 9 (counter l, 4 m + r, step k) gives
// nodes 2r and 2r + 1; warp r mod N draws it.  B(0) = v(0), B(k) = a B(k-1) +
// sqrt(1 - a^2) v(k), W(k) = Qhat B(k) (Sec. 3.9.1).
__device__ __forceinline__ void particle_wind_step(const ProblemC &P, float *pw, int i, int N, int j,
                                                   uint32_t l, int m, int k, uint32_t mpc)
{
    float *dst = pw + (k & 1) * 16 * kPB + j;
    const float *src = pw + ((k + 1) & 1) * 16 * kPB + j;     // B(k-1)
    for (int r = i; r < 4; r += N) {
        const uint4 d = draw(P.key0, P.key1, l, (uint32_t)(4 * m + r), (uint32_t)k, 9u, 0u, mpc);
        const float2 v0 = box_muller_fast(d.x, d.y), v1 = box_muller_fast(d.z, d.w);
        const float v[4] = {v0.x, v0.y, v1.x, v1.y};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int row = 4 * r + e;        // node 2r + e / 2, component e % 2
            dst[row * kPB] = k == 0 ? v[e] : fmaf(P.wind_a, src[row * kPB], P.wind_b * v[e]);
        }
    }
}

// Wind of that field at a position (clamped into the box): with the trilinear
// weights w_n of the corners, W = sum_n w_n sum_j Qhat[n][j] B_j = sum_j g_j B_j,
// g_j = sum_(n >= j) w_n Qhat[n][j].  B holds row (node * 2 + component) at
// B[row * Stride]: pw[k & 1] + lane with Stride kPB in the tile.
template <int Stride = kPB>
__device__ __forceinline__ float2 particle_wind_at(const ProblemC &P, const float *B, float x, float y,
                                                   float z)
{
    const float tx = fminf(fmaxf((x - P.box_lo[0]) * P.inv_h[0], 0.0f), 1.0f);
    const float ty = fminf(fmaxf((y - P.box_lo[1]) * P.inv_h[1], 0.0f), 1.0f);
    const float tz = fminf(fmaxf((z - P.box_lo[2]) * P.inv_h[2], 0.0f), 1.0f);
    float wn[8];
#pragma unroll
    for (int n = 0; n < 8; ++n)
        wn[n] = ((n & 4) ? tx : 1.0f - tx) * ((n & 2) ? ty : 1.0f - ty) * ((n & 1) ? tz : 1.0f - tz);
    float2 w = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int jn = 0; jn < 8; ++jn) {
        float g = 0.0f;
#pragma unroll
        for (int n = jn; n < 8; ++n) g = fmaf(wn[n], P.wchol[n * (n + 1) / 2 + jn], g);
        w.x = fmaf(g, B[(2 * jn) * Stride], w.x);
        w.y = fmaf(g, B[(2 * jn + 1) * Stride], w.y);
    }
    return w;
}

__device__ __forceinline__ void tile_barrier(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// State of one aircraft of one particle during a rollout (registers).
struct AcState {
    float x, y, z, v, chi;
    Kahan F;                 // fuel burned
    float zb, vb, cb;        // z, v, chi at the start of the current control segment
    int seg, ks, knext;      // current segment, its first step, first step of the next
    int srem;                // ((seg + 1) H + S - 1) mod S: knext's remainder
    float uw, uh, ua;        // controls of the current segment
    bool dead, landed;
    float2 turb_next;        // second normal pair of the last even-step draw
    float th;                // bearing atan2(y, x) of the step-(k+1) state
    float beta;              // arrivals: glide angle of the step-(k+1) state
};

__device__ __forceinline__ void ac_init(AcState &s, const DynState *__restrict__ dyn, int i,
                                        bool exists, int S)
{
    s.x = dyn->x0[i][0];
    s.y = dyn->x0[i][1];
    s.z = dyn->x0[i][2];
    s.v = dyn->x0[i][3];
    s.chi = dyn->x0[i][4];
    s.F = Kahan();
    s.zb = s.vb = s.cb = 0.0f;
    s.seg = -1;
    s.srem = S - 1;
    s.ks = 0;
    s.knext = 0;
    s.uw = s.uh = s.ua = 0.0f;
    s.dead = !exists;
    s.landed = false;
    s.turb_next = make_float2(0.0f, 0.0f);
    s.th = s.beta = 0.0f;
}

// Arrival geometry (Eq. (flow)): the arc tangent to the runway through the
// aircraft at bearing th = atan2(y, x) has length s = r th / sin th (capped at
// 4 r); returns the glide angle atan2(z, s) and r, |th|.
__device__ __forceinline__ float arc_glide(float x, float y, float z, float th, float &r, float &ath)
{
    r = sqrtf(fmaf(x, x, y * y));
    ath = fabsf(th);
    const float ratio = ath < 1e-3f ? fmaf(th * th, 1.0f / 6.0f, 1.0f)
                                    : __fdividef(ath, fmaxf(__sinf(ath), 0.25f * ath));
    return atan2_poly(z, r * ratio);
}

// The landing sector of Eq. (TO_init): range, glide angle, bearing cone on the
// approach side (x > 0), heading within P_chi of the runway, speed.
__device__ __forceinline__ bool in_landing_sector(const ProblemC &P, float x, float r, float ath,
                                                  float beta, float chi, float v)
{
    const float hdg = angdist(chi - kPi);
    return r <= P.P_runway && beta <= P.P_beta && x > 0.0f && ath <= P.P_chi && hdg <= P.P_chi &&
           v <= P.P_vs;
}

// Per-step deviation sums of the objectives (Sec. 3.5, Sec. 7.1).
struct CostSums {
    Kahan sA, sB, sC;
    float sN = 0.0f;
    __device__ __forceinline__ void arrival(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        sA.add(angdist(s.chi - fmaf(2.0f, s.th, kPi)));
        sB.add(fabsf(s.beta - P.beta_f));
    }
    __device__ __forceinline__ void departure(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        sA.add(angdist(s.th - A.thF));
        sB.add(fabsf(A.Z - s.z));
        sC.add(fabsf(s.v - A.vD));
    }
    __device__ __forceinline__ void noise(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        const float za = s.z * P.Ac_inv;
        const float h = fmaxf(fmaf(-za, za, 1.0f), 0.0f);
        // above A_c the term is 0 (h = 0): the density is not looked up
        if (h > 0.0f) sN = fmaf(h, popdense_at(P, s.x, s.y), sN);
    }
};

// Advances one flying aircraft (not stopped before step k) by step k
// (Sec. 3.3-3.4): control limits on the step-k values, explicit Euler step of
// Eq. (hor) under wind and turbulence, unary limits and (arrivals) the landing
// sector of Eq. (TO_init) on the step-(k+1) state.  When the aircraft is still
// flying after the step, the visitor sees the new state (s.th, s.beta set):
// visit.arrival or visit.departure, then visit.noise when the noise cost is
// on.  Returns false when the control limits failed (the aircraft did not
// move); otherwise s.dead / s.landed tell whether it stopped at this step.
// ul = this particle's controls of this aircraft [S][3]; the wind is the
// sample's shared field Wk, or the particle's own field when pwk is given.
// ParamP: P is the kernel's parameter (the turbulence draw takes the round
// keys precomputed in it).
template <bool ParamP = false, class Visit>
__device__ __forceinline__ bool ac_step(const ProblemC &P, const AircraftC &A, AcState &s,
                                        const float *__restrict__ ul,
                                        const float4 *__restrict__ Wk, float m0, uint32_t l,
                                        uint32_t i, uint32_t m, int k, int J, uint32_t mpc,
                                        Visit &visit, const float *pwk = nullptr)
{
    const float dt = P.dt;
    if (k >= s.knext) {
        // segment s covers the steps [ceil(s H / S), ceil((s + 1) H / S)) (every
        // segment has a step: S <= H); knext = ceil((seg + 1) H / S) advances by
        // H = seg_q S + seg_r with its remainder carried, so no division (a late
        // entrant passes several segments at its first step)
        do {
            ++s.seg;
            s.knext += P.seg_q;
            s.srem += P.seg_r;
            if (s.srem >= P.S) {
                s.srem -= P.S;
                ++s.knext;
            }
        } while (k >= s.knext);
        s.ks = k;
        s.uw = __ldg(ul + 3 * s.seg);
        s.uh = __ldg(ul + 3 * s.seg + 1);
        s.ua = __ldg(ul + 3 * s.seg + 2);
        s.zb = s.z;
        s.vb = s.v;
        s.cb = s.chi;
    }
    const float mass = m0 - s.F.s;
    // control-derived quantities and their limits (Sec. 3.4)
    const float sg = __fdividef(s.uh, s.v);
    bool ok = fabsf(sg) <= P.sgmax;
    const float cg = sqrtf(fmaxf(1.0f - sg * sg, 0.0f));
    const float tp = __fdividef(s.uw * s.v, kG0 * cg);
    ok = ok && (fabsf(tp) < P.tpmax);
    const float secphi = sqrtf(fmaf(tp, tp, 1.0f));
    const float rho = 1.225f * ex2_approx(4.2559f * __log2f(fmaxf(fmaf(-2.2558e-5f, s.z, 1.0f), 1e-30f)));
    const float qS = A.halfS * rho * s.v * s.v;
    const float CL = __fdividef(mass * kG0 * cg * secphi, qS);
    const float D = qS * fmaf(A.CD2, CL * CL, A.CD0);
    const float T = fmaf(mass, fmaf(kG0, sg, s.ua), D);
    ok = ok && (T >= A.Tmin) && (T <= A.Tmax);
    if (!ok) {
        s.dead = true;
        return false;
    }
    // disturbance: wind field of sample m plus white turbulence
    float2 w = pwk ? particle_wind_at(P, pwk, s.x, s.y, s.z)
                   : wind_interp(wind_fetch(P, Wk, s.x, s.y, s.z));
    float2 n;
    if ((k & 1) == 0) {
        const uint4 r = ParamP ? draw_rk(P.rk, l, i | (m << 8), (uint32_t)(k >> 1), 0u, (uint32_t)J, mpc)
                               : draw(P.key0, P.key1, l, i | (m << 8), (uint32_t)(k >> 1), 0u, (uint32_t)J, mpc);
        n = box_muller_fast(r.x, r.y);
        s.turb_next = box_muller_fast(r.z, r.w);
    } else {
        n = s.turb_next;
    }
    w.x = fmaf(P.turb_sigma, n.x, w.x);
    w.y = fmaf(P.turb_sigma, n.y, w.y);
    // explicit Euler step of Eq. (hor); v sin(gamma) = hdot, the speed equation
    // reduces to v += dt a and the heading equation to chi += dt w (coordinated
    // turn).  Within a control segment z, v and chi are linear in time: they are
    // evaluated from the segment's start values so that rounding does not
    // accumulate.
    float sc, cc;
    sincos_reduced(s.chi, &sc, &cc);
    const float vh = s.v * cg;
    s.x = fmaf(dt, fmaf(vh, cc, w.x), s.x);
    s.y = fmaf(dt, fmaf(vh, sc, w.y), s.y);
    const float nk = (float)(k + 1 - s.ks) * dt;
    s.z = fmaf(nk, s.uh, s.zb);
    const float eta = A.Cf1 * fmaf(s.v, A.invCf2, 1.0f);
    s.F.add(dt * eta * T);
    s.v = fmaf(nk, s.ua, s.vb);
    s.chi = fmaf(nk, s.uw, s.cb);
    const float mass1 = m0 - s.F.s;
    if (!(s.z >= P.z_min && s.z <= P.z_max && s.v >= P.v_min && s.v <= P.v_max &&
          mass1 >= A.m_empty)) {
        s.dead = true;
    } else {
        s.th = atan2_poly(s.y, s.x);
        if (A.type == 0) {
            // arrival: flow-field arc, glide angle and landing sector
            float r, ath;
            s.beta = arc_glide(s.x, s.y, s.z, s.th, r, ath);
            if (in_landing_sector(P, s.x, r, ath, s.beta, s.chi, s.v)) {
                s.landed = true;
            } else {
                visit.arrival(P, A, s);
            }
        } else {
            visit.departure(P, A, s);
        }
        if (P.w_noise != 0.0f && !s.landed) visit.noise(P, A, s);
    }
    return true;
}

// Departure altitude term: sup / inf of the per-step distance to Z reachable
// from the current altitude at the maximum climb rate c (Sec. 3.5), in closed
// form over the Ha scored steps (Ha = H, or a late entrant's active steps):
// sup = d0 + c (Ha+1)/2, inf = (K d0 - c K (K+1)/2) / Ha, K = min(Ha, floor(d0/c)).
struct AltBounds {
    float supB, invSupInf;
};

__device__ __forceinline__ AltBounds alt_bounds(const ProblemC &P, const AircraftC &A, float z0, int Ha)
{
    const float d0 = fabsf(A.Z - z0);
    const float supB = fmaf(P.climb_step, 0.5f * (float)(Ha + 1), d0);
    const float Kf = fminf((float)Ha, floorf(__fdividef(d0, P.climb_step)));
    const float infB = (Kf * d0 - P.climb_step * 0.5f * Kf * (Kf + 1.0f)) / (float)Ha;
    return AltBounds{supB, 1.0f / (supB - infB)};
}

// J_T of Sec. 3.5 and Sec. 7.1 from the deviation sums and the fuel burned,
// per-step means over the Ha scored steps (the fuel bound too: A.invFmax is
// for H steps).
__device__ __forceinline__ float total_objective(const ProblemC &P, const AircraftC &A,
                                                 const CostSums &c, float Fs, AltBounds ab, int Ha)
{
    const float invH = 1.0f / (float)Ha;
    const float Jf = Ha == P.H ? fmaf(-Fs, A.invFmax, 1.0f)
                               : fmaf(-Fs, A.invFmax * ((float)P.H * invH), 1.0f);
    float Jsum;
    if (A.type == 1) {
        const float J1 = fmaf(-c.sA.s * invH, 1.0f / kPi, 1.0f);
        const float J3 = (ab.supB - c.sB.s * invH) * ab.invSupInf;
        const float J4 = fmaf(-c.sC.s * invH, A.invCmax, 1.0f);
        Jsum = P.a_dep[0] * J1 + P.a_dep[1] * Jf + P.a_dep[2] * J3 + P.a_dep[3] * J4;
    } else {
        const float J1 = fmaf(-c.sA.s * invH, 1.0f / kPi, 1.0f);
        const float J3 = fmaf(-c.sB.s * invH, 2.0f / kPi, 1.0f);
        Jsum = P.a_arr[0] * J1 + P.a_arr[1] * J3 + P.a_arr[2] * Jf;
    }
    return (1.0f - P.w_noise) * Jsum + P.w_noise * fmaf(-c.sN, invH, 1.0f);
}

// Shared memory of one tile (32-bit words): positions float4 [2][2N + 4][32]
// (double-buffered by step; every aircraft's row written twice, at i and
// i + N, so that the partners i+1 .. i+N/2 are consecutive rows without a
// wrap; the screening pass reads partners in groups, up to kScreen - 1 rows
// past the last, which the four spare rows hold), separation flags [N][32],
// the soft form's received penalties [2][N][floor((N-1)/2) + 1][32] with a
// word per (step parity, aircraft, particle) marking the slots written
// [2][N][32], and in wind mode 1 the particles' wind state [2][16][32].
__host__ __device__ constexpr int tile_pair_slots(int N) { return (N - 1) / 2 + 1; }
__host__ __device__ constexpr int tile_pos_rows(int N) { return 2 * N + 4; }
// tp: particles of the tile (32, or 16 for the half tile)
__host__ __device__ constexpr int tile_smem_words(int N, int wind_mode, int tp = kTileParticles)
{
    return (4 * 2 * tile_pos_rows(N) + N + 2 * N + 2 * N * tile_pair_slots(N) + (wind_mode == 1 ? 32 : 0)) * tp;
}

// Simulates aircraft i (this warp) of particles l0..l0+31 (lane j) under the
// packed wind field Wm of sample m and returns its per-sample costs (the
// softplus variant too when Soft); the caller stores them (store_tile), so
// that no output pointer is live during the steps.  spos is the tile's
// tile_smem_words(N, P.wind_mode) buffer; every warp of the tile must call this
// with the same barrier (bar_id, bar_count threads).
//
// Separation (Eq. (avoidance)) checks every unordered pair once: warp i takes
// the partners i+d, d = 1 .. floor((N-1)/2) (mod N), and for even N also
// d = N/2 when i < N/2, so every warp has the same load.  A violation marks
// both aircraft (the partner through its flag in shared memory).  In the soft
// form a branch-free screening pass first marks the partners within reach (the
// distance beyond which the penalty is below e^-30 / beta, a region that
// contains the hard one); only a warp with a lane within reach of some partner
// evaluates those pairs (the softplus and the hard test).  The softplus
// penalty of a pair enters both aircraft's costs: the owner adds it, stores it
// in the partner's slot d and sets bit d of the partner's mark word; after the
// next step's barrier every aircraft adds its marked slots in increasing d and
// clears the word (deterministic sums; a pair out of reach has penalty 0,
// which neither side adds).
struct TileResult {
    float cost;         // -ln J_T, +inf if infeasible or separation violated (hard)
    float cost_soft;    // with the softplus penalty, +inf if infeasible
    unsigned int live;  // aircraft-steps simulated by this thread
};

// OwnWind: wind mode 1; Rolling: the rolling window; Soft: the softplus
// penalties are evaluated and exchanged besides the hard test (each compiled
// apart, so the plain problem keeps its register budget).
// ParamP: P is the kernel's parameter (the plain kernels): the aircraft's
// constants are copied into registers once (a reference into the parameter
// space reloads them at every use) and the turbulence draws take the
// precomputed round keys.  The batched kernel holds P in shared memory and
// keeps the reference, its register budget is full.
// TP: particles of the tile, 32 (one warp per aircraft), 16 or 8 (a warp holds
// 32 / TP consecutive aircraft, TP lanes each; every warp of the block is full
// when N is a multiple of 32 / TP), so that several blocks of a large N share
// an SM.  The shared buffers are laid out the same way with TP particles per
// row.
template <bool OwnWind, bool Rolling, bool Soft, bool ParamP = true, int TP = kTileParticles>
__device__ __forceinline__ TileResult rollout_tile_mode(const ProblemC &P, const DynState *__restrict__ dyn,
                                                        const float *__restrict__ u,
                                                        const float4 *__restrict__ Wm, long long L,
                                                        long long l0, int i, int j, int m, int J,
                                                        float *spos, int bar_id,
                                                        int bar_count)
{
    static_assert(TP == kTileParticles || ((TP == 16 || TP == 8) && !OwnWind),
                  "smaller tiles: shared wind field only");
    constexpr int kPB = TP;     // particles per row of every shared buffer of this tile
    const int N = P.N;
    const long long l = l0 + j;
    const bool exists = l < L;
    AircraftC Acopy;
    if constexpr (ParamP) Acopy = P.ac[i];
    const AircraftC &A = ParamP ? Acopy : P.ac[i];
    const uint32_t mpc = dyn->mpc_step;
    // rolling window: the first step this aircraft flies, and whether it is in
    // the problem at all during this horizon (warp-uniform)
    int k_in = 0;
    bool out = false;
    if (Rolling) {
        const long long d = (long long)A.t_enter - (long long)mpc;
        k_in = d > 0 ? (int)min(d, (long long)P.H) : 0;
        out = ((dyn->finished >> i) & 1u) != 0u || k_in >= P.H;
    }
    const int Ha = P.H - k_in;
    AcState s;
    ac_init(s, dyn, i, exists && !out, P.S);
    if (Rolling && (k_in & 1) && exists && !out) {
        // entering at an odd step: the turbulence pair of that step comes from
        // the draw of the even step before it, which this aircraft did not fly
        const uint4 r = draw(P.key0, P.key1, (uint32_t)l, (uint32_t)i | ((uint32_t)m << 8),
                             (uint32_t)(k_in >> 1), 0u, (uint32_t)J, mpc);
        s.turb_next = box_muller_fast(r.z, r.w);
    }
    const float m0 = dyn->x0[i][5];
    const AltBounds ab = alt_bounds(P, A, s.z, Ha);
    CostSums cs;
    float soft = 0.0f;
    bool sepv = false;
    const float *ul = u + ((size_t)(exists ? l : 0) * N + i) * (size_t)(P.S * 3);
    unsigned int nlive = 0;
    const int plane = N * kPB;
    const int rows = tile_pos_rows(N);
    float4 *pos = reinterpret_cast<float4 *>(spos);                          // [2][2N + 4][TP]
    int *vflag = reinterpret_cast<int *>(spos + 8 * rows * kPB);            // [N][TP]
    unsigned *rmark = reinterpret_cast<unsigned *>(vflag + plane);         // [2][N][TP]
    float *recv = reinterpret_cast<float *>(rmark + 2 * plane);           // [2][N][slots][TP]
    const int slots = tile_pair_slots(N);
    // ordered before any partner's mark by the step-0 (and step-1) barrier
    vflag[i * kPB + j] = 0;
    if constexpr (Soft) {
        rmark[i * kPB + j] = 0u;
        rmark[plane + i * kPB + j] = 0u;
    }
    const int n_half = (N - 1) >> 1;
    const bool even = (N & 1) == 0;
    const int n_pairs = n_half + ((even && i < (N >> 1)) ? 1 : 0);   // at most 16
    const unsigned pair_bits = (1u << n_pairs) - 1u;
    constexpr bool own_wind = OwnWind;
    float *pw = recv + 2 * N * slots * kPB;                               // mode 1: [2][16][32]
    if constexpr (own_wind) {
        particle_wind_step(P, pw, i, N, j, (uint32_t)l, m, 0, mpc);
        tile_barrier(bar_id, bar_count);
    }

    for (int k = 0; k < P.H; ++k) {
        const bool entered = k >= k_in;
        if (!s.dead && !s.landed && entered) {
            ++nlive;
            ac_step<ParamP>(P, A, s, ul, Wm + (size_t)k * P.P, m0, (uint32_t)l, (uint32_t)i, (uint32_t)m,
                            k, J, mpc, cs, own_wind ? pw + (k & 1) * 16 * kPB + j : nullptr);
        }
        // the particles' wind state of the next step, read after this step's barrier
        if (own_wind && k + 1 < P.H) particle_wind_step(P, pw, i, N, j, (uint32_t)l, m, k + 1, mpc);
        // binary separation constraints at step k+1 among flying aircraft: every
        // thread publishes its position (a far-away altitude when not flying)
        const bool act = !s.dead && !s.landed && entered;
        float4 *buf = pos + (k & 1) * rows * kPB;
        const float4 me = make_float4(s.x, s.y, act ? s.z : 1e30f, 0.0f);
        buf[i * kPB + j] = me;
        buf[(i + N) * kPB + j] = me;
        tile_barrier(bar_id, bar_count);
        // partner i + 1 + d is row i + 1 + d of buf (no wrap); its index mod N
        // only where a mark or a penalty slot is written
        const float4 *qrow = buf + (i + 1) * kPB + j;
        if constexpr (Soft) {
            // penalties the partners marked for this aircraft at the previous step
            if (k > 0) {
                unsigned *mw = rmark + ((k - 1) & 1) * plane + i * kPB + j;
                unsigned rm = *mw;
                if (rm != 0u) {
                    *mw = 0u;
                    const float *rr = recv + ((((k - 1) & 1) * N + i) * slots) * kPB + j;
                    do {
                        soft += rr[(__ffs(rm) - 1) * kPB];
                        rm &= rm - 1u;
                    } while (rm != 0u);
                }
            }
            // screening in groups of kScreen partners: bit d set when partner d
            // is within reach
            unsigned near = 0u;
#pragma unroll
            for (int d0 = 0; d0 < 16; d0 += kScreen) {
                if (d0 < n_pairs) {
#pragma unroll
                    for (int e = 0; e < kScreen; ++e) {
                        const float4 q = qrow[(d0 + e) * kPB];
                        const float dx = s.x - q.x, dy = s.y - q.y;
                        if (fmaf(dx, dx, dy * dy) < P.sp_far_h2 && fabsf(s.z - q.z) < P.sp_far_v)
                            near |= 1u << (d0 + e);
                    }
                }
            }
            near = act ? (near & pair_bits) : 0u;
            if (__any_sync(0xffffffffu, near != 0u)) {
                float *rw = recv + ((k & 1) * N * slots) * kPB + j;
                unsigned *mark = rmark + (k & 1) * plane + j;
                while (near != 0u) {
                    const int d = __ffs(near) - 1;
                    near &= near - 1u;
                    const int i2 = i + 1 + d < N ? i + 1 + d : i + 1 + d - N;
                    const float4 q = qrow[d * kPB];
                    const float dx = s.x - q.x, dy = s.y - q.y, adz = fabsf(s.z - q.z);
                    const float dh2 = fmaf(dx, dx, dy * dy);
                    if (dh2 < P.Sh2 && adz < P.Sv) {
                        sepv = true;
                        vflag[i2 * kPB + j] = 1;
                    }
                    const float pen = softplus(fminf(fmaf(-sqrtf(dh2), P.Sh_inv, 1.0f), fmaf(-adz, P.Sv_inv, 1.0f)),
                                               P.sp_beta, P.sp_inv_beta);
                    soft += pen;
                    rw[(i2 * slots + d) * kPB] = pen;
                    atomicOr(mark + i2 * kPB, 1u << d);
                }
            }
        } else if (act) {
            // hard form: a violation is rare, its branch almost never taken
            for (int d = 0; d < n_pairs; ++d) {
                const float4 q = qrow[d * kPB];
                const float dx = s.x - q.x, dy = s.y - q.y;
                if (fmaf(dx, dx, dy * dy) < P.Sh2 && fabsf(s.z - q.z) < P.Sv) {
                    sepv = true;
                    const int i2 = i + 1 + d < N ? i + 1 + d : i + 1 + d - N;
                    vflag[i2 * kPB + j] = 1;
                }
            }
        }
    }
    // marks and penalties the partners wrote at the last step
    tile_barrier(bar_id, bar_count);
    sepv = sepv || vflag[i * kPB + j] != 0;
    if constexpr (Soft) {
        unsigned rm = rmark[((P.H - 1) & 1) * plane + i * kPB + j];
        const float *rr = recv + ((((P.H - 1) & 1) * N + i) * slots) * kPB + j;
        for (; rm != 0u; rm &= rm - 1u) soft += rr[(__ffs(rm) - 1) * kPB];
    }

    // the per-sample cost -ln J_T (Sec. 3.6)
    const float JT = total_objective(P, A, cs, s.F.s, ab, Ha);
    const float c = -logf(fmaxf(JT, 1e-30f));
    TileResult r;
    r.cost = (s.dead || sepv) ? __int_as_float(0x7f800000) : c;
    r.cost_soft = s.dead ? __int_as_float(0x7f800000) : fmaf(P.mu_sep, soft, c);
    if (out) {                      // not in the problem this horizon: J_T = 1
        r.cost = 0.0f;
        r.cost_soft = 0.0f;
    }
    r.live = exists ? nlive : 0u;
    return r;
}

// Stores one thread's tile result: cost_ms[(m N + i) L + l] (and the soft
// variant when cost_ms_soft is not null); adds the warp's live steps.
__device__ __forceinline__ void store_tile(const TileResult &r, int N, long long L, long long l,
                                           int i, int j, int m, float *__restrict__ cost_ms,
                                           float *__restrict__ cost_ms_soft,
                                           unsigned long long *__restrict__ live)
{
    if (l < L) {
        const size_t o = ((size_t)m * N + i) * (size_t)L + l;
        cost_ms[o] = r.cost;
        if (cost_ms_soft) cost_ms_soft[o] = r.cost_soft;
    }
    if (live != nullptr) {
        // one atomic per warp (a warp of a smaller tile holds several aircraft)
        const unsigned int tot = __reduce_add_sync(0xffffffffu, r.live);
        if ((threadIdx.x & 31) == 0 && tot) atomicAdd(live, (unsigned long long)tot);
    }
}

}  // namespace tma
