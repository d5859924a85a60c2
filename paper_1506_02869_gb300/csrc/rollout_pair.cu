// Rollout of one tile for two wind samples per thread (the inner loop of
// Algorithm 1, Sec. 3.3-3.6, Sec. 7.1), for the plain problem: the shared
// wind field of Sec. 3.9.1 and no rolling window.
//
// Of an aircraft's state only the position (x, y) depends on the wind: the
// altitude, airspeed and heading follow the controls alone (Eq. (hor) with
// v sin(gamma) = hdot, dv/dt = a, dchi/dt = w), and the thrust, the fuel flow
// and so the mass follow from those.  The control and state limits are
// therefore the same under every wind sample.  This kernel gives each thread
// the samples m and m + ceil(M/2) of one (particle, aircraft): the
// wind-independent part of a step (limits, drag, thrust, fuel, the new
// altitude, airspeed and heading, the departure's altitude and speed terms)
// is computed once for both, the rest (wind, turbulence, position, bearing,
// glide angle, landing, separation) per sample, the (x, y) pairs with the
// packed two-lane FP32 instructions.  The mapping is otherwise the one of
// rollout_tile.cuh: warp i = aircraft i, lane j = particle l0 + j, positions
// exchanged through shared memory behind one barrier per step.  Every
// operation is the one the single-sample tile performs, in the same order, so
// the two kernels return the same bits.
#include "rollout_tile.cuh"

namespace tma {

namespace {

// ---- packed two-lane FP32 arithmetic (per lane the IEEE single operation)
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding, as the subtraction: (-1) b + a
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float lane(float2 v, int g) { return g ? v.y : v.x; }
__device__ __forceinline__ void set_lane(float2 &v, int g, float a)
{
    if (g) v.y = a;
    else v.x = a;
}

// Kahan-compensated sums of the two samples, lane by lane the scalar Kahan.
struct Kahan2 {
    float2 s = make_float2(0.0f, 0.0f), c = make_float2(0.0f, 0.0f);
    // add in the lanes whose flag is set, keep the others unchanged
    __device__ __forceinline__ void add_masked(float2 y, bool on0, bool on1)
    {
        const float2 yy = sub2(y, c);
        const float2 t = add2(s, yy);
        const float2 cn = sub2(sub2(t, s), yy);
        if (on0) {
            s.x = t.x;
            c.x = cn.x;
        }
        if (on1) {
            s.y = t.y;
            c.y = cn.y;
        }
    }
    __device__ __forceinline__ Kahan lane_sum(int g) const
    {
        Kahan k;
        k.s = lane(s, g);
        k.c = lane(c, g);
        return k;
    }
};

// Trilinear interpolation of the packed field (own value and difference to
// the level above per node) with the (x, y) components in the two lanes.
__device__ __forceinline__ float2 wind_interp_packed(const WindFetch &f)
{
    const float2 tz = dup2(f.tz);
    const float2 c00 = fma2(tz, make_float2(f.a00.z, f.a00.w), make_float2(f.a00.x, f.a00.y));
    const float2 c01 = fma2(tz, make_float2(f.a01.z, f.a01.w), make_float2(f.a01.x, f.a01.y));
    const float2 c10 = fma2(tz, make_float2(f.a10.z, f.a10.w), make_float2(f.a10.x, f.a10.y));
    const float2 c11 = fma2(tz, make_float2(f.a11.z, f.a11.w), make_float2(f.a11.x, f.a11.y));
    const float2 ty = dup2(f.ty);
    const float2 c0 = fma2(ty, sub2(c01, c00), c00);
    const float2 c1 = fma2(ty, sub2(c11, c10), c10);
    return fma2(dup2(f.tx), sub2(c1, c0), c0);
}

// atan2_poly of rollout_tile.cuh for the two samples, the polynomial packed.
__device__ __forceinline__ float2 atan2_poly2(float2 y, float2 x)
{
    float2 t;
    bool swap[2], neg[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const float xg = lane(x, g), yg = lane(y, g);
        const float ax = fabsf(xg), ay = fabsf(yg);
        const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
        set_lane(t, g, mx > 0.0f ? __fdividef(mn, mx) : 0.0f);
        swap[g] = ay > ax;
        neg[g] = xg < 0.0f;
    }
    const float2 s = mul2(t, t);
    float2 p = dup2(2.932487579e-03f);
    p = fma2(p, s, dup2(-1.641217540e-02f));
    p = fma2(p, s, dup2(4.327672817e-02f));
    p = fma2(p, s, dup2(-7.556783848e-02f));
    p = fma2(p, s, dup2(1.066743802e-01f));
    p = fma2(p, s, dup2(-1.421109512e-01f));
    p = fma2(p, s, dup2(1.999369316e-01f));
    p = fma2(p, s, dup2(-3.333313793e-01f));
    p = fma2(p, s, dup2(9.999999938e-01f));
    const float2 a2 = mul2(t, p);
    float2 r;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        float a = lane(a2, g);
        if (swap[g]) a = 1.57079632679489662f - a;
        if (neg[g]) a = 3.14159265358979324f - a;
        set_lane(r, g, copysignf(a, lane(y, g)));
    }
    return r;
}

// The two samples' part of an aircraft's state (lane g = sample g).
struct PairState {
    // wind-independent
    float z, v, chi;
    Kahan F;
    float zb, vb, cb;
    int seg, ks, knext, srem;
    float uw, uh, ua;
    // per sample
    float2 P[2];             // (x, y) of sample g
    bool fly[2];             // still flying (not stopped, in the problem)
    bool dead[2];            // stopped by a limit: infeasible
    float2 turb_next[2];
    float Ffin[2];           // fuel burned when the sample stopped
};

// One step of both samples (the samples that are no longer flying keep their
// state).  Same operations as ac_step of rollout_tile.cuh.
__device__ __forceinline__ void pair_step(const ProblemC &P, const AircraftC &A, PairState &s,
                                          const float *__restrict__ ul,
                                          const float4 *__restrict__ Wk0,
                                          const float4 *__restrict__ Wk1, float m0, uint32_t l,
                                          uint32_t i, uint32_t mA, uint32_t mB, int k, int J,
                                          uint32_t mpc, Kahan2 &sA, Kahan2 &sB, Kahan &dB,
                                          Kahan &dC, float2 &sN)
{
    const float dt = P.dt;
    if (k >= s.knext) {
        // the next segment(s), as ac_step advances them (no division)
        do {
            ++s.seg;
            s.knext += P.seg_q;
            s.srem += P.seg_r;
            if (s.srem >= P.S) {
                s.srem -= P.S;
                ++s.knext;
            }
        } while (k >= s.knext);
        const int seg = s.seg;
        s.ks = k;
        s.uw = __ldg(ul + 3 * seg);
        s.uh = __ldg(ul + 3 * seg + 1);
        s.ua = __ldg(ul + 3 * seg + 2);
        s.zb = s.z;
        s.vb = s.v;
        s.cb = s.chi;
    }
    const float mass = m0 - s.F.s;
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
        s.dead[0] = s.dead[0] || s.fly[0];
        s.dead[1] = s.dead[1] || s.fly[1];
        s.fly[0] = s.fly[1] = false;
        return;
    }
    float2 w0 = wind_interp_packed(wind_fetch(P, Wk0, s.P[0].x, s.P[0].y, s.z));
    float2 w1 = wind_interp_packed(wind_fetch(P, Wk1, s.P[1].x, s.P[1].y, s.z));
    float2 n0 = make_float2(0.0f, 0.0f), n1 = n0;
    if ((k & 1) == 0) {
        if (s.fly[0]) {
            const uint4 r = draw_rk(P.rk, l, i | (mA << 8), (uint32_t)(k >> 1), 0u, (uint32_t)J, mpc);
            n0 = box_muller_fast(r.x, r.y);
            s.turb_next[0] = box_muller_fast(r.z, r.w);
        }
        if (s.fly[1]) {
            const uint4 r = draw_rk(P.rk, l, i | (mB << 8), (uint32_t)(k >> 1), 0u, (uint32_t)J, mpc);
            n1 = box_muller_fast(r.x, r.y);
            s.turb_next[1] = box_muller_fast(r.z, r.w);
        }
    } else {
        n0 = s.turb_next[0];
        n1 = s.turb_next[1];
    }
    const float2 sig = dup2(P.turb_sigma);
    w0 = fma2(sig, n0, w0);
    w1 = fma2(sig, n1, w1);
    float sc, cc;
    sincos_reduced(s.chi, &sc, &cc);
    const float vh = s.v * cg;
    const float2 vh2 = dup2(vh), dt2 = dup2(dt), cs = make_float2(cc, sc);
    const float2 p0 = fma2(dt2, fma2(vh2, cs, w0), s.P[0]);
    const float2 p1 = fma2(dt2, fma2(vh2, cs, w1), s.P[1]);
    if (s.fly[0]) s.P[0] = p0;
    if (s.fly[1]) s.P[1] = p1;
    const float nk = (float)(k + 1 - s.ks) * dt;
    s.z = fmaf(nk, s.uh, s.zb);
    const float eta = A.Cf1 * fmaf(s.v, A.invCf2, 1.0f);
    s.F.add(dt * eta * T);
    s.v = fmaf(nk, s.ua, s.vb);
    s.chi = fmaf(nk, s.uw, s.cb);
    const float mass1 = m0 - s.F.s;
    if (!(s.z >= P.z_min && s.z <= P.z_max && s.v >= P.v_min && s.v <= P.v_max &&
          mass1 >= A.m_empty)) {
        s.dead[0] = s.dead[0] || s.fly[0];
        s.dead[1] = s.dead[1] || s.fly[1];
        s.fly[0] = s.fly[1] = false;
        return;
    }
    const float2 X = make_float2(s.P[0].x, s.P[1].x), Y = make_float2(s.P[0].y, s.P[1].y);
    const float2 th = atan2_poly2(Y, X);
    bool score0 = s.fly[0], score1 = s.fly[1];
    if (A.type == 0) {
        float2 beta;
        float2 dA;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float r, ath;
            const float tg = lane(th, g);
            const float b = arc_glide(lane(X, g), lane(Y, g), s.z, tg, r, ath);
            set_lane(beta, g, b);
            set_lane(dA, g, angdist(s.chi - fmaf(2.0f, tg, kPi)));
            if (s.fly[g] && in_landing_sector(P, lane(X, g), r, ath, b, s.chi, s.v)) {
                s.fly[g] = false;            // landed: frozen, its cost is final
                s.Ffin[g] = s.F.s;
                if (g == 0) score0 = false;
                else score1 = false;
            }
        }
        sA.add_masked(dA, score0, score1);
        sB.add_masked(make_float2(fabsf(beta.x - P.beta_f), fabsf(beta.y - P.beta_f)), score0, score1);
    } else {
        sA.add_masked(make_float2(angdist(th.x - A.thF), angdist(th.y - A.thF)), score0, score1);
        dB.add(fabsf(A.Z - s.z));
        dC.add(fabsf(s.v - A.vD));
    }
    if (P.w_noise != 0.0f) {
        const float za = s.z * P.Ac_inv;
        const float h = fmaxf(fmaf(-za, za, 1.0f), 0.0f);
        if (score0) sN.x = fmaf(h, popdense_at(P, X.x, Y.x), sN.x);
        if (score1) sN.y = fmaf(h, popdense_at(P, X.y, Y.y), sN.y);
    }
}

// Shared memory of one pair tile (32-bit words): positions float4
// [2 (step parity)][2 (sample)][N][32], separation flags [2][N][32], the
// received softplus penalties [2 (parity)][2 (sample)][N][slots][32].
__host__ __device__ constexpr int pair_smem_words(int N)
{
    return (16 * N + 2 * N + 4 * N * tile_pair_slots(N)) * kTileParticles;
}

template <int kMaxThreads, int kMinBlocks>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks)
    rollout_pair_kernel(const ProblemC P, const DynState *__restrict__ dyn, const float *__restrict__ u,
                        const float4 *__restrict__ W, long long L, int nLb, int J,
                        float *__restrict__ cost_ms, float *__restrict__ cost_ms_soft,
                        unsigned long long *__restrict__ live)
{
    extern __shared__ float sh[];
    const int N = P.N;
    const int Mh = (P.M + 1) >> 1;
    const int pb = blockIdx.x / nLb;                      // sample pair: block-uniform
    const int mA = pb, mB = pb + Mh;
    const bool hasB = mB < P.M;
    const long long l0 = (long long)(blockIdx.x - pb * nLb) * kPB;
    const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
    const long long l = l0 + j;
    const bool exists = l < L;
    const bool soft_on = cost_ms_soft != nullptr;
    const AircraftC A = P.ac[i];   // a copy: the warp-uniform constants stay in registers
    const uint32_t mpc = dyn->mpc_step;
    const float4 *WA = W + (size_t)mA * P.H * P.P;
    const float4 *WB = W + (size_t)(hasB ? mB : mA) * P.H * P.P;

    PairState s;
    s.z = dyn->x0[i][2];
    s.v = dyn->x0[i][3];
    s.chi = dyn->x0[i][4];
    s.F = Kahan();
    s.zb = s.vb = s.cb = 0.0f;
    s.ks = 0;
    s.knext = 0;
    s.seg = -1;
    s.srem = P.S - 1;
    s.uw = s.uh = s.ua = 0.0f;
    s.P[0] = s.P[1] = make_float2(dyn->x0[i][0], dyn->x0[i][1]);
    s.fly[0] = exists;
    s.fly[1] = exists && hasB;
    s.dead[0] = s.dead[1] = false;
    s.turb_next[0] = s.turb_next[1] = make_float2(0.0f, 0.0f);
    s.Ffin[0] = s.Ffin[1] = 0.0f;
    const float m0 = dyn->x0[i][5];
    const AltBounds ab = alt_bounds(P, A, s.z, P.H);
    Kahan2 sA, sB;
    Kahan dB, dC;
    float2 sN = make_float2(0.0f, 0.0f);
    float soft[2] = {0.0f, 0.0f};
    bool sepv[2] = {false, false};
    unsigned int nlive[2] = {0u, 0u};
    const float *ul = u + ((size_t)(exists ? l : 0) * N + i) * (size_t)(P.S * 3);

    const int plane = N * kPB;                                       // words of one [N][32] plane
    float4 *pos = reinterpret_cast<float4 *>(sh);                    // [2][2][N][32]
    int *vflag = reinterpret_cast<int *>(sh + 16 * plane);           // [2][N][32]
    float *recv = sh + 18 * plane;                                   // [2][2][N][slots][32]
    const int slots = tile_pair_slots(N);
    vflag[i * kPB + j] = 0;
    vflag[plane + i * kPB + j] = 0;
    const int n_half = (N - 1) >> 1;
    const bool even = (N & 1) == 0;
    const int n_pairs = n_half + ((even && i < (N >> 1)) ? 1 : 0);
    const int n_recv = n_half + ((even && i >= (N >> 1)) ? 1 : 0);

    for (int k = 0; k < P.H; ++k) {
        if (s.fly[0] || s.fly[1]) {
            nlive[0] += s.fly[0];
            nlive[1] += s.fly[1];
            pair_step(P, A, s, ul, WA + (size_t)k * P.P, WB + (size_t)k * P.P, m0, (uint32_t)l,
                      (uint32_t)i, (uint32_t)mA, (uint32_t)mB, k, J, mpc, sA, sB, dB, dC, sN);
        }
        const bool act0 = s.fly[0], act1 = s.fly[1];
        float4 *buf = pos + (k & 1) * 2 * plane;
        buf[i * kPB + j] = make_float4(s.P[0].x, s.P[0].y, act0 ? s.z : 1e30f, 0.0f);
        buf[plane + i * kPB + j] = make_float4(s.P[1].x, s.P[1].y, act1 ? s.z : 1e30f, 0.0f);
        tile_barrier(0, blockDim.x);
        if (soft_on) {
            if (k > 0) {
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const float *rr = recv + ((((k - 1) & 1) * 2 + g) * N + i) * slots * kPB + j;
                    for (int d = 0; d < n_recv; ++d) soft[g] += rr[d * kPB];
                }
            }
            int i2 = i;
            for (int d = 0; d < n_pairs; ++d) {
                i2 = (i2 + 1 == N) ? 0 : i2 + 1;
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const bool act = g ? act1 : act0;
                    const float4 q = buf[g * plane + i2 * kPB + j];
                    const float2 dxy = sub2(s.P[g], make_float2(q.x, q.y));
                    const float adz = fabsf(s.z - q.z);
                    const float dh2 = fmaf(dxy.x, dxy.x, dxy.y * dxy.y);
                    float pen = 0.0f;
                    if (act) {
                        if (dh2 < P.Sh2 && adz < P.Sv) {
                            sepv[g] = true;
                            vflag[g * plane + i2 * kPB + j] = 1;
                        }
                        if (dh2 < P.sp_far_h2 && adz < P.sp_far_v)   // else below e^-30 / beta
                            pen = softplus(fminf(fmaf(-sqrtf(dh2), P.Sh_inv, 1.0f), fmaf(-adz, P.Sv_inv, 1.0f)),
                                           P.sp_beta, P.sp_inv_beta);
                        soft[g] += pen;
                    }
                    recv[((((k & 1) * 2 + g) * N + i2) * slots + d) * kPB + j] = pen;
                }
            }
        } else if (act0 || act1) {
            int i2 = i;
            for (int d = 0; d < n_pairs; ++d) {
                i2 = (i2 + 1 == N) ? 0 : i2 + 1;
                const float4 q0 = buf[i2 * kPB + j];
                const float4 q1 = buf[plane + i2 * kPB + j];
                const float2 d0 = sub2(s.P[0], make_float2(q0.x, q0.y));
                const float2 d1 = sub2(s.P[1], make_float2(q1.x, q1.y));
                if (act0 && fmaf(d0.x, d0.x, d0.y * d0.y) < P.Sh2 && fabsf(s.z - q0.z) < P.Sv) {
                    sepv[0] = true;
                    vflag[i2 * kPB + j] = 1;
                }
                if (act1 && fmaf(d1.x, d1.x, d1.y * d1.y) < P.Sh2 && fabsf(s.z - q1.z) < P.Sv) {
                    sepv[1] = true;
                    vflag[plane + i2 * kPB + j] = 1;
                }
            }
        }
    }
    tile_barrier(0, blockDim.x);
    if (soft_on) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const float *rr = recv + ((((P.H - 1) & 1) * 2 + g) * N + i) * slots * kPB + j;
            for (int d = 0; d < n_recv; ++d) soft[g] += rr[d * kPB];
        }
    }
    unsigned int tot = 0;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const bool valid = exists && (g == 0 || hasB);
        const bool sv = sepv[g] || vflag[g * plane + i * kPB + j] != 0;
        const float Fs = (s.fly[g] || s.dead[g]) ? s.F.s : s.Ffin[g];
        CostSums cs;
        cs.sA = sA.lane_sum(g);
        if (A.type == 0) {
            cs.sB = sB.lane_sum(g);
        } else {
            cs.sB = dB;
            cs.sC = dC;
        }
        cs.sN = lane(sN, g);
        const float JT = total_objective(P, A, cs, Fs, ab, P.H);
        const float c = -logf(fmaxf(JT, 1e-30f));
        if (valid) {
            const size_t o = ((size_t)(g ? mB : mA) * N + i) * (size_t)L + l;
            cost_ms[o] = (s.dead[g] || sv) ? __int_as_float(0x7f800000) : c;
            if (cost_ms_soft)
                cost_ms_soft[o] = s.dead[g] ? __int_as_float(0x7f800000) : fmaf(P.mu_sep, soft[g], c);
            tot += nlive[g];
        }
    }
    if (live != nullptr) {
        tot = __reduce_add_sync(0xffffffffu, tot);
        if (j == 0 && tot) atomicAdd(live, (unsigned long long)tot);
    }
}

}  // namespace

struct PairVariant {
    int max_threads, min_blocks;
};
// registers per thread: 85, 128, 85, 128, 85
constexpr PairVariant kPairVariants[] = {{256, 3}, {256, 2}, {384, 2}, {512, 1}, {768, 1}};
constexpr int kNumPairVariants = sizeof(kPairVariants) / sizeof(kPairVariants[0]);

int rollout_pair_variants(const ProblemC &P, int *out)
{
    if (P.wind_mode != 0 || P.rolling || P.M < 2) return 0;
    int n = 0;
    for (int v = 0; v < kNumPairVariants; ++v)
        if (kPairVariants[v].max_threads >= P.N * kPB) out[n++] = v;
    return n;
}

cudaError_t launch_rollout_pair(const ProblemC &P, const DynState *dyn, const float *u, const float *W,
                                int64_t L, int J, float *cost_ms, float *cost_ms_soft,
                                unsigned long long *live, cudaStream_t st, int variant)
{
    if (L <= 0) return cudaSuccess;
    if (variant < 0 || variant >= kNumPairVariants || kPairVariants[variant].max_threads < P.N * kPB ||
        P.wind_mode != 0 || P.rolling || P.M < 2)
        return cudaErrorInvalidValue;   // callers pick among rollout_pair_variants
    const long long nLb = (L + kPB - 1) / kPB;
    const unsigned grid = (unsigned)(nLb * ((P.M + 1) / 2));
    const int block = P.N * kPB;
    const size_t smem = (size_t)pair_smem_words(P.N) * sizeof(float);
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
#define TMA_PAIR_K(T, B)                                                                         \
    do {                                                                                         \
        if (smem > 48 * 1024)                                                                    \
            cudaFuncSetAttribute(rollout_pair_kernel<T, B>,                                      \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
        rollout_pair_kernel<T, B><<<grid, block, smem, st>>>(P, dyn, u, W4, L, (int)nLb, J,       \
                                                             cost_ms, cost_ms_soft, live);        \
    } while (0)
    switch (variant) {
    case 0: TMA_PAIR_K(256, 3); break;
    case 1: TMA_PAIR_K(256, 2); break;
    case 2: TMA_PAIR_K(384, 2); break;
    case 3: TMA_PAIR_K(512, 1); break;
    default: TMA_PAIR_K(768, 1); break;
    }
#undef TMA_PAIR_K
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
