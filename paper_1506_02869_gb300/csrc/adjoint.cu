// Reverse-mode derivative of the soft cost with respect to the controls: the
// gradient of C_l = sum_i (1/M) sum_m c_soft[i][m] (the rollout of Sec. 3.3-3.6
// and Sec. 7.1 with the softplus separation penalty; unary and control limits
// stay hard) for every particle l, used by the Langevin move.
//
// Mapping: as the rollout, one block is 32 particles (lanes) x N aircraft
// (warps); a block takes a contiguous range of wind samples.  For each sample:
//   pass 1  the forward rollout of each aircraft alone (the step function of
//           the rollout kernel), saving a checkpoint of the aircraft state
//           every 10 steps; its J_T fixes the cost coefficients of the
//           reverse sweep.  No exchange between aircraft is needed yet;
//   pass 2  for each checkpoint interval, last to first: recompute its steps
//           from the checkpoint, keeping the pre-step states and the
//           derivative of the per-step cost terms at the post-step state
//           (deviation terms, and the separation penalty with its value, the
//           partner positions coming through a shared-memory exchange as in
//           the rollout); then run the interval's steps backwards, carrying
//           the adjoint (x, y, z, v, chi, F) of this aircraft and summing the
//           control gradient of each segment.
// Limit, landing and interpolation-cell decisions keep their forward values.
// Once the forward pass is stored, the reverse sweep needs nothing from the
// other aircraft: the separation derivative with respect to this aircraft's
// position depends only on forward positions.
#include "rollout_tile.cuh"

namespace tma {

namespace {

constexpr int kCkEvery = 10;
constexpr int kMaxCk = TMA_MAX_GRAD_HORIZON / kCkEvery;

struct Checkpoint {
    float x, y, z, v, chi, Fs, Fc, zb, vb, cb;
    int ks, segflags;     // segment + 1 in bits 0..19, dead bit 20, landed bit 21
};

__device__ __forceinline__ Checkpoint save(const AcState &s)
{
    Checkpoint c;
    c.x = s.x; c.y = s.y; c.z = s.z; c.v = s.v; c.chi = s.chi;
    c.Fs = s.F.s; c.Fc = s.F.c;
    c.zb = s.zb; c.vb = s.vb; c.cb = s.cb;
    c.ks = s.ks;
    c.segflags = (s.seg + 1) | (s.dead ? 1 << 20 : 0) | (s.landed ? 1 << 21 : 0);
    return c;
}

__device__ __forceinline__ void restore(const ProblemC &P, AcState &s, const Checkpoint &c,
                                        const float *__restrict__ ul)
{
    s.x = c.x; s.y = c.y; s.z = c.z; s.v = c.v; s.chi = c.chi;
    s.F.s = c.Fs; s.F.c = c.Fc;
    s.zb = c.zb; s.vb = c.vb; s.cb = c.cb;
    s.ks = c.ks;
    s.seg = (c.segflags & 0xFFFFF) - 1;
    s.dead = (c.segflags >> 20) & 1;
    s.landed = (c.segflags >> 21) & 1;
    if (s.seg >= 0) {
        const long long B = (long long)(s.seg + 1) * P.H + P.S - 1;
        s.knext = (int)(B / P.S);
        s.srem = (int)(B % P.S);
        s.uw = __ldg(ul + 3 * s.seg);
        s.uh = __ldg(ul + 3 * s.seg + 1);
        s.ua = __ldg(ul + 3 * s.seg + 2);
    } else {
        s.knext = 0;
        s.srem = P.S - 1;
    }
}

__device__ __forceinline__ float sgnf(float a) { return a > 0.0f ? 1.0f : (a < 0.0f ? -1.0f : 0.0f); }

// wrapped angle in [-pi, pi] (the signed counterpart of angdist)
__device__ __forceinline__ float wrapf(float a)
{
    const float twopi = 6.28318530717958647692f;
    return a - twopi * rintf(a * (1.0f / twopi));
}

// Trilinear wind and its derivative with respect to position; zero along an
// axis where the position lies outside the box (it is clamped there).
__device__ __forceinline__ void wind_grad(const ProblemC &P, const float4 *__restrict__ Wk, float x,
                                          float y, float z, float2 &dwx, float2 &dwy, float2 &dwz)
{
    const WindFetch f = wind_fetch(P, Wk, x, y, z);
    float2 c00, c01, c10, c11, e00, e01, e10, e11;
    // records hold (value, difference to the node one level up)
    c00.x = fmaf(f.tz, f.a00.z, f.a00.x); c00.y = fmaf(f.tz, f.a00.w, f.a00.y);
    c01.x = fmaf(f.tz, f.a01.z, f.a01.x); c01.y = fmaf(f.tz, f.a01.w, f.a01.y);
    c10.x = fmaf(f.tz, f.a10.z, f.a10.x); c10.y = fmaf(f.tz, f.a10.w, f.a10.y);
    c11.x = fmaf(f.tz, f.a11.z, f.a11.x); c11.y = fmaf(f.tz, f.a11.w, f.a11.y);
    e00 = make_float2(f.a00.z, f.a00.w);
    e01 = make_float2(f.a01.z, f.a01.w);
    e10 = make_float2(f.a10.z, f.a10.w);
    e11 = make_float2(f.a11.z, f.a11.w);
    float2 c0, c1, e0, e1;
    c0.x = fmaf(f.ty, c01.x - c00.x, c00.x); c0.y = fmaf(f.ty, c01.y - c00.y, c00.y);
    c1.x = fmaf(f.ty, c11.x - c10.x, c10.x); c1.y = fmaf(f.ty, c11.y - c10.y, c10.y);
    e0.x = fmaf(f.ty, e01.x - e00.x, e00.x); e0.y = fmaf(f.ty, e01.y - e00.y, e00.y);
    e1.x = fmaf(f.ty, e11.x - e10.x, e10.x); e1.y = fmaf(f.ty, e11.y - e10.y, e10.y);
    const bool ix = x > P.box_lo[0] && x < P.box_hi[0];
    const bool iy = y > P.box_lo[1] && y < P.box_hi[1];
    const bool iz = z > P.box_lo[2] && z < P.box_hi[2];
    // d/dx: difference across the x cell; d/dy: across y, bilinear in x; d/dz likewise
    dwx = ix ? make_float2((c1.x - c0.x) * P.inv_h[0], (c1.y - c0.y) * P.inv_h[0]) : make_float2(0.f, 0.f);
    const float2 dy0 = make_float2(c01.x - c00.x, c01.y - c00.y);
    const float2 dy1 = make_float2(c11.x - c10.x, c11.y - c10.y);
    dwy = iy ? make_float2(fmaf(f.tx, dy1.x - dy0.x, dy0.x) * P.inv_h[1],
                           fmaf(f.tx, dy1.y - dy0.y, dy0.y) * P.inv_h[1])
             : make_float2(0.f, 0.f);
    dwz = iz ? make_float2(fmaf(f.tx, e1.x - e0.x, e0.x) * P.inv_h[2],
                           fmaf(f.tx, e1.y - e0.y, e0.y) * P.inv_h[2])
             : make_float2(0.f, 0.f);
}

// Population density (Sec. 7.1) and its gradient; 0 outside the grid.
__device__ __forceinline__ float popdense_grad(const ProblemC &P, float x, float y, float &gx, float &gy)
{
    gx = gy = 0.0f;
    if (P.popcell == nullptr) return 0.0f;
    if (!(x >= P.pop_lo[0] && x <= P.pop_hi[0] && y >= P.pop_lo[1] && y <= P.pop_hi[1]))
        return 0.0f;
    const float f0 = (x - P.pop_lo[0]) * P.pop_inv_h[0];
    const float f1 = (y - P.pop_lo[1]) * P.pop_inv_h[1];
    const int i0 = min((int)f0, P.pop_n[0] - 2), i1 = min((int)f1, P.pop_n[1] - 2);
    const float t0 = f0 - (float)i0, t1 = f1 - (float)i1;
    const float4 g = __ldg(P.popcell + (size_t)i0 * (P.pop_n[1] - 1) + i1);
    const float g00 = g.x, g01 = g.y, g10 = g.z, g11 = g.w;
    gx = fmaf(t1, (g11 - g01) - (g10 - g00), g10 - g00) * P.pop_inv_h[0];
    gy = fmaf(t0, (g11 - g10) - (g01 - g00), g01 - g00) * P.pop_inv_h[1];
    const float a = fmaf(t1, g01 - g00, g00), b = fmaf(t1, g11 - g10, g10);
    return fmaf(t0, b - a, a);
}

// Coefficients d c / d (deviation sums, fuel) of one aircraft's per-sample cost
// c = -ln J_T, already divided by M.
struct CostGrad {
    float gA, gB, gC, gN, gF;
};

__device__ __forceinline__ CostGrad cost_grad(const ProblemC &P, const AircraftC &A, float JT,
                                              AltBounds ab, float invM)
{
    CostGrad g{0.f, 0.f, 0.f, 0.f, 0.f};
    if (!(JT > 1e-30f)) return g;            // the cost is clamped there
    const float invH = 1.0f / (float)P.H;
    const float s = -invM / JT;              // d c / d J_T, over M
    const float wj = (1.0f - P.w_noise) * s;
    if (A.type == 1) {
        g.gA = wj * (-P.a_dep[0] * invH / kPi);
        g.gB = wj * (-P.a_dep[2] * invH * ab.invSupInf);
        g.gC = wj * (-P.a_dep[3] * invH * A.invCmax);
        g.gF = wj * (-P.a_dep[1] * A.invFmax);
    } else {
        g.gA = wj * (-P.a_arr[0] * invH / kPi);
        g.gB = wj * (-P.a_arr[1] * invH * (2.0f / kPi));
        g.gF = wj * (-P.a_arr[2] * A.invFmax);
    }
    g.gN = s * (-P.w_noise * invH);
    return g;
}

// Derivative of this aircraft's per-step deviation terms at a flying
// step-(k+1) state, as a step visitor: the sources (x, y, z, v, chi) that enter
// the adjoint at step k+1.
struct TermGrad {
    CostGrad cg;
    float sx = 0.f, sy = 0.f, sz = 0.f, sv = 0.f, sc = 0.f;

    __device__ __forceinline__ void bearing(const AcState &s, float coef)
    {
        const float r2 = fmaf(s.x, s.x, s.y * s.y);
        const float ir2 = r2 > 0.0f ? 1.0f / r2 : 0.0f;
        sx = fmaf(coef, -s.y * ir2, sx);
        sy = fmaf(coef, s.x * ir2, sy);
    }
    __device__ __forceinline__ void departure(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        bearing(s, sgnf(wrapf(s.th - A.thF)) * cg.gA);
        sz = fmaf(cg.gB, sgnf(s.z - A.Z), sz);
        sv = fmaf(cg.gC, sgnf(s.v - A.vD), sv);
    }
    __device__ __forceinline__ void arrival(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        const float se = sgnf(wrapf(s.chi - fmaf(2.0f, s.th, kPi))) * cg.gA;
        sc += se;
        bearing(s, -2.0f * se);
        // glide angle beta = atan2(z, r ratio(theta)), ratio = |theta| / sin|theta|
        const float x = s.x, y = s.y, z = s.z;
        const float r2 = fmaf(x, x, y * y);
        const float r = sqrtf(r2);
        const float ath = fabsf(s.th);
        float ratio, dratio;
        if (ath < 1e-3f) {
            ratio = fmaf(s.th * s.th, 1.0f / 6.0f, 1.0f);
            dratio = s.th * (1.0f / 3.0f);
        } else {
            float sn, cs;
            __sincosf(ath, &sn, &cs);                 // ath in [0, pi]: no range reduction needed
            if (sn >= 0.25f * ath) {
                ratio = ath / sn;
                dratio = sgnf(s.th) * (sn - ath * cs) / (sn * sn);
            } else {
                ratio = 4.0f;
                dratio = 0.0f;
            }
        }
        const float sa = r * ratio;
        const float den = fmaf(z, z, sa * sa);
        const float bb = cg.gB * sgnf(s.beta - P.beta_f);
        sz = fmaf(bb, sa / den, sz);
        // d(sa)/dx = ratio x / r + r ratio'(theta) dtheta/dx, likewise for y
        const float bsa = -bb * z / den;
        const float ir = r > 0.0f ? 1.0f / r : 0.0f;
        sx = fmaf(bsa, ratio * x * ir, sx);
        sy = fmaf(bsa, ratio * y * ir, sy);
        bearing(s, bsa * r * dratio);
    }
    __device__ __forceinline__ void noise(const ProblemC &P, const AircraftC &A, const AcState &s)
    {
        float gx, gy;
        const float pd = popdense_grad(P, s.x, s.y, gx, gy);
        const float za = s.z * P.Ac_inv;
        const float h = fmaf(-za, za, 1.0f);
        if (h > 0.0f) {
            sx = fmaf(cg.gN * h, gx, sx);
            sy = fmaf(cg.gN * h, gy, sy);
            sz = fmaf(cg.gN * pd, -2.0f * s.z * P.Ac_inv * P.Ac_inv, sz);
        }
    }
};

// Adjoint of step k of one aircraft (Eq. (hor) with the drag of the
// coordinated turn in closed form, D = q CD0 + CD2 m^2 (g^2 cos^2(gamma) +
// w^2 v^2) / q, q = rho v^2 S / 2): maps the adjoint at k+1 to the adjoint at
// k and adds the step's control derivative to (gw, gh, ga).
__device__ __forceinline__ void step_adjoint(const ProblemC &P, const AircraftC &A,
                                             const float4 *__restrict__ Wk, float x, float y,
                                             float z, float v, float chi, float mass, float uw,
                                             float uh, float ua, float &X, float &Y, float &Z,
                                             float &V, float &CH, float &FF, float &gw, float &gh,
                                             float &ga)
{
    const float dt = P.dt;
    const float iv = 1.0f / v;
    const float sg = uh * iv;
    const float cg = sqrtf(fmaxf(1.0f - sg * sg, 1e-12f));
    const float icg = 1.0f / cg;
    const float dcg_dv = uh * uh * iv * iv * iv * icg;
    const float dcg_dh = -uh * iv * iv * icg;
    const float base = fmaxf(fmaf(-2.2558e-5f, z, 1.0f), 1e-30f);
    const float rho = 1.225f * ex2_approx(4.2559f * __log2f(base));   // as the forward step
    const float q = A.halfS * rho * v * v;
    const float iq = 1.0f / q;
    const float dq_dz = q * (4.2559f * -2.2558e-5f) / base;
    const float dq_dv = 2.0f * q * iv;
    const float g2 = kG0 * kG0;
    const float A2 = fmaf(g2, 1.0f - sg * sg, uw * uw * v * v);
    const float dA2_dv = 2.0f * g2 * uh * uh * iv * iv * iv + 2.0f * uw * uw * v;
    const float dA2_dh = -2.0f * g2 * uh * iv * iv;
    const float dA2_dw = 2.0f * uw * v * v;
    const float K2 = A.CD2 * mass * mass;
    const float D = fmaf(q, A.CD0, K2 * A2 * iq);
    const float T = fmaf(mass, fmaf(kG0, sg, ua), D);
    const float dD_dv = fmaf(A.CD0, dq_dv, K2 * (dA2_dv * iq - A2 * dq_dv * iq * iq));
    const float dD_dz = fmaf(A.CD0, dq_dz, -K2 * A2 * dq_dz * iq * iq);
    const float dD_dm = 2.0f * A.CD2 * mass * A2 * iq;
    const float dT_dv = fmaf(-mass * kG0 * uh, iv * iv, dD_dv);
    const float dT_dm = ua + kG0 * sg + dD_dm;
    const float dT_dh = fmaf(mass * kG0, iv, K2 * dA2_dh * iq);
    const float dT_dw = K2 * dA2_dw * iq;
    const float eta = A.Cf1 * fmaf(v, A.invCf2, 1.0f);
    const float deta_dv = A.Cf1 * A.invCf2;
    float2 dwx, dwy, dwz;
    wind_grad(P, Wk, x, y, z, dwx, dwy, dwz);
    float sc, cc;
    sincos_reduced(chi, &sc, &cc);
    const float proj = fmaf(cc, X, sc * Y);            // along-track adjoint
    const float fe = FF * dt * eta;                     // fuel adjoint times d F'/d T
    const float nX = X + dt * fmaf(X, dwx.x, Y * dwx.y);
    const float nY = Y + dt * fmaf(X, dwy.x, Y * dwy.y);
    const float nZ = Z + dt * fmaf(X, dwz.x, Y * dwz.y) + fe * dD_dz;
    const float nV = V + dt * (cg + v * dcg_dv) * proj + FF * dt * fmaf(deta_dv, T, eta * dT_dv);
    const float nC = CH + dt * v * cg * fmaf(-sc, X, cc * Y);
    const float nF = FF - fe * dT_dm;
    gw += fmaf(dt, CH, fe * dT_dw);
    gh += dt * Z + dt * v * dcg_dh * proj + fe * dT_dh;
    ga += fmaf(dt, V, fe * mass);
    X = nX; Y = nY; Z = nZ; V = nV; CH = nC; FF = nF;
}

// Derivative of one pair's separation penalty (weight w = 2 mu sigma(beta g) / M)
// with respect to this aircraft's position, from the differences own - partner.
__device__ __forceinline__ void pair_grad(const ProblemC &P, float w, float dx, float dy, float dz,
                                          float &sx, float &sy, float &sz)
{
    const float dh = sqrtf(fmaf(dx, dx, dy * dy));
    const float ghh = fmaf(-dh, P.Sh_inv, 1.0f);
    const float gvv = fmaf(-fabsf(dz), P.Sv_inv, 1.0f);
    if (ghh <= gvv) {
        if (dh > 0.0f) {
            const float eh = w * P.Sh_inv / dh;
            sx = fmaf(-eh, dx, sx);
            sy = fmaf(-eh, dy, sy);
        }
    } else {
        sz = fmaf(-w * P.Sv_inv, sgnf(dz), sz);
    }
}

// The penalty of a pair and the logistic weight of its derivative, from one
// exponential of -|beta g| (0, 0 when either aircraft is not flying: its
// published altitude is far away).
__device__ __forceinline__ float2 pair_penalty(const ProblemC &P, float dx, float dy, float dz)
{
    const float dh = sqrtf(fmaf(dx, dx, dy * dy));
    const float gmin = fminf(fmaf(-dh, P.Sh_inv, 1.0f), fmaf(-fabsf(dz), P.Sv_inv, 1.0f));
    const float bg = P.sp_beta * gmin;
    const float e = __expf(-fabsf(bg));
    return make_float2((fmaxf(bg, 0.0f) + log1p_unit(e)) * P.sp_inv_beta,
                       (bg >= 0.0f ? 1.0f : e) / (1.0f + e));
}

// Pairs are computed once (as in the rollout) when the received slots fit in
// shared memory; above this aircraft count every aircraft computes its N-1.
constexpr int kGradPairOnceMaxN = 16;

// Positions are triple-buffered by step: a receiver reads its partners'
// positions of step k-1 at step k, after the step-k barrier; a partner can
// overwrite that buffer only at step k+2, after the step-(k+1) barrier, which
// the receiver reaches after its read.
__host__ __device__ constexpr int grad_smem_words(int N)
{
    return 12 * N * kTileParticles +                                              // positions
           (N <= kGradPairOnceMaxN ? 4 * N * tile_pair_slots(N) * kTileParticles : 0);  // slots
}

template <int kMaxThreads, int kMinBlocks>
__global__ void __launch_bounds__(kMaxThreads, kMinBlocks)
rollout_grad_kernel(const ProblemC P, const DynState *__restrict__ dyn, const float *__restrict__ u,
                    const float4 *__restrict__ W, long long L, int nLb, int m_per_block, int J,
                    float *__restrict__ cost_ms, float *__restrict__ gpart)
{
    extern __shared__ float spos[];
    const int N = P.N;
    const int i = threadIdx.x >> 5, j = threadIdx.x & 31;
    const int chunk = blockIdx.x / nLb;
    const long long l = (long long)(blockIdx.x - chunk * nLb) * kPB + j;
    const bool exists = l < L;
    const AircraftC A = P.ac[i];   // a copy: the warp-uniform constants stay in registers
    const uint32_t mpc = dyn->mpc_step;
    const float m0 = dyn->x0[i][5];
    const float *ul = u + ((size_t)(exists ? l : 0) * N + i) * (size_t)(P.S * 3);
    const int nS3 = P.S * 3;
    float *gout = gpart + (((size_t)chunk * L + (exists ? l : 0)) * N + i) * (size_t)nS3;
    if (exists)
        for (int n = 0; n < nS3; ++n) gout[n] = 0.0f;
    const int plane = N * kPB;
    // shared memory: positions float4 [3][N][32], then (pair-once) the received
    // (penalty, logistic weight) float2 [2][N][slots][32]
    float4 *pos = reinterpret_cast<float4 *>(spos);
    float2 *slots = reinterpret_cast<float2 *>(spos + 12 * plane);
    const bool pair_once = N <= kGradPairOnceMaxN;
    const int n_slots = tile_pair_slots(N);
    const int n_half = (N - 1) >> 1;
    const bool even_n = (N & 1) == 0;
    const int n_pairs = n_half + ((even_n && i < (N >> 1)) ? 1 : 0);
    const int n_recv = n_half + ((even_n && i >= (N >> 1)) ? 1 : 0);
    const float invM = 1.0f / (float)P.M;
    const float sep_c = 2.0f * P.mu_sep * invM;        // each pair enters two aircraft's costs
    const int mb = chunk * m_per_block, me = min(P.M, mb + m_per_block);
    const int nck = (P.H + kCkEvery - 1) / kCkEvery;

    Checkpoint ck[kMaxCk];
    float hx[kCkEvery], hy[kCkEvery], hz[kCkEvery], hv[kCkEvery], hc[kCkEvery], hF[kCkEvery];
    float rx[kCkEvery], ry[kCkEvery], rz[kCkEvery], rv[kCkEvery], rc[kCkEvery];

    for (int m = mb; m < me; ++m) {
        const float4 *Wm = W + (size_t)m * P.H * P.P;
        // ---------------- pass 1: forward rollout of this aircraft alone, with
        // checkpoints; J_T fixes the cost coefficients of the reverse sweep
        AcState s;
        ac_init(s, dyn, i, exists, P.S);
        const AltBounds ab = alt_bounds(P, A, s.z, P.H);
        CostSums cs;
        for (int k = 0; k < P.H; ++k) {
            if (k % kCkEvery == 0) ck[k / kCkEvery] = save(s);
            if (!s.dead && !s.landed)
                ac_step<true>(P, A, s, ul, Wm + (size_t)k * P.P, m0, (uint32_t)l, (uint32_t)i,
                        (uint32_t)m, k, J, mpc, cs);
        }
        const float JT = total_objective(P, A, cs, s.F.s, ab, P.H);
        const float c = -logf(fmaxf(JT, 1e-30f));
        const bool dead = s.dead;
        const CostGrad cg = cost_grad(P, A, JT, ab, invM);
        float soft = 0.0f;     // separation penalty, summed in pass 2

        // ---------------- pass 2: interval by interval, last to first
        float X = 0.f, Y = 0.f, Z = 0.f, V = 0.f, CH = 0.f, FF = cg.gF;
        int gseg = -1;
        float gw = 0.f, gh = 0.f, ga = 0.f;
        for (int c_i = nck - 1; c_i >= 0; --c_i) {
            const int k0 = c_i * kCkEvery, k1 = min(P.H, k0 + kCkEvery);
            AcState r;
            ac_init(r, dyn, i, exists, P.S);
            restore(P, r, ck[c_i], ul);
            unsigned upd = 0;
            // the previous interval's last exchange may still be read
            tile_barrier(0, blockDim.x);
            for (int k = k0; k < k1; ++k) {
                const int t = k - k0;
                hx[t] = r.x; hy[t] = r.y; hz[t] = r.z; hv[t] = r.v; hc[t] = r.chi; hF[t] = r.F.s;
                TermGrad tg;
                tg.cg = cg;
                if (!r.dead && !r.landed &&
                    ac_step<true>(P, A, r, ul, Wm + (size_t)k * P.P, m0, (uint32_t)l, (uint32_t)i,
                            (uint32_t)m, k, J, mpc, tg))
                    upd |= 1u << t;
                const bool act = !r.dead && !r.landed;
                float sx = tg.sx, sy = tg.sy, sz = tg.sz, sv = tg.sv, sc = tg.sc;
                float4 *buf = pos + (k % 3) * plane;
                buf[i * kPB + j] = make_float4(r.x, r.y, act ? r.z : 1e30f, 0.0f);
                tile_barrier(0, blockDim.x);
                if (pair_once) {
                    // pairs the partners computed for this aircraft at the previous
                    // step: penalty, and the derivative from both positions of then
                    if (k > k0) {
                        const float2 *rr = slots + ((((k - 1) & 1) * N + i) * n_slots) * kPB + j;
                        const float4 *pb = pos + ((k - 1) % 3) * plane;
                        float px = 0.f, py = 0.f, pz = 0.f;
                        int o = i;
                        for (int d = 0; d < n_recv; ++d) {
                            o = (o == 0) ? N - 1 : o - 1;
                            const float2 ps = rr[d * kPB];
                            soft += ps.x;
                            if (ps.y != 0.0f) {
                                const float4 q = pb[o * kPB + j];
                                pair_grad(P, sep_c * ps.y, hx[t] - q.x, hy[t] - q.y, hz[t] - q.z,
                                          px, py, pz);
                            }
                        }
                        rx[t - 1] += px; ry[t - 1] += py; rz[t - 1] += pz;
                    }
                    float2 *rw = slots + ((k & 1) * N * n_slots) * kPB + j;
                    int i2 = i;
                    for (int d = 0; d < n_pairs; ++d) {
                        i2 = (i2 + 1 == N) ? 0 : i2 + 1;
                        float2 ps = make_float2(0.0f, 0.0f);
                        const float4 q = buf[i2 * kPB + j];
                        const float dx = r.x - q.x, dy = r.y - q.y, dz = r.z - q.z;
                        // beyond reach the penalty and its weight are below e^-30: 0,
                        // as in the rollout; only a warp with a lane in reach evaluates
                        const bool near = act && fmaf(dx, dx, dy * dy) < P.sp_far_h2 && fabsf(dz) < P.sp_far_v;
                        if (__any_sync(0xffffffffu, near) && near) {
                            ps = pair_penalty(P, dx, dy, dz);
                            soft += ps.x;
                            if (ps.y != 0.0f) pair_grad(P, sep_c * ps.y, dx, dy, dz, sx, sy, sz);
                        }
                        rw[(i2 * n_slots + d) * kPB] = ps;
                    }
                } else if (act) {
                    for (int i2 = 0; i2 < N; ++i2) {
                        if (i2 == i) continue;
                        const float4 q = buf[i2 * kPB + j];
                        const float dx = r.x - q.x, dy = r.y - q.y, dz = r.z - q.z;
                        if (fmaf(dx, dx, dy * dy) >= P.sp_far_h2 || fabsf(dz) >= P.sp_far_v) continue;   // out of reach
                        const float2 ps = pair_penalty(P, dx, dy, dz);
                        soft += ps.x;
                        if (ps.y != 0.0f) pair_grad(P, sep_c * ps.y, dx, dy, dz, sx, sy, sz);
                    }
                }
                rx[t] = sx; ry[t] = sy; rz[t] = sz; rv[t] = sv; rc[t] = sc;
            }
            if (pair_once) {
                // pairs of the interval's last step, received after one more barrier
                tile_barrier(0, blockDim.x);
                const int k = k1 - 1, t = k - k0;
                const float2 *rr = slots + (((k & 1) * N + i) * n_slots) * kPB + j;
                const float4 *pb = pos + (k % 3) * plane;
                float px = 0.f, py = 0.f, pz = 0.f;
                int o = i;
                for (int d = 0; d < n_recv; ++d) {
                    o = (o == 0) ? N - 1 : o - 1;
                    const float2 ps = rr[d * kPB];
                    soft += ps.x;
                    if (ps.y != 0.0f) {
                        const float4 q = pb[o * kPB + j];
                        pair_grad(P, sep_c * ps.y, r.x - q.x, r.y - q.y, r.z - q.z, px, py, pz);
                    }
                }
                rx[t] += px; ry[t] += py; rz[t] += pz;
            }
            // reverse sweep of the interval
            for (int k = k1 - 1; k >= k0; --k) {
                const int t = k - k0;
                if (!((upd >> t) & 1u)) continue;
                X += rx[t]; Y += ry[t]; Z += rz[t]; V += rv[t]; CH += rc[t];
                const int sg = (k * P.S) / P.H;
                if (sg != gseg) {
                    if (gseg >= 0 && exists) {
                        gout[3 * gseg] += gw;
                        gout[3 * gseg + 1] += gh;
                        gout[3 * gseg + 2] += ga;
                    }
                    gseg = sg;
                    gw = gh = ga = 0.f;
                }
                step_adjoint(P, A, Wm + (size_t)k * P.P, hx[t], hy[t], hz[t], hv[t], hc[t],
                             m0 - hF[t], __ldg(ul + 3 * sg), __ldg(ul + 3 * sg + 1),
                             __ldg(ul + 3 * sg + 2), X, Y, Z, V, CH, FF, gw, gh, ga);
            }
        }
        if (gseg >= 0 && exists) {
            gout[3 * gseg] += gw;
            gout[3 * gseg + 1] += gh;
            gout[3 * gseg + 2] += ga;
        }
        if (exists)
            cost_ms[((size_t)m * N + i) * (size_t)L + l] =
                dead ? __int_as_float(0x7f800000) : fmaf(P.mu_sep, soft, c);
    }
}

// One warp per particle: per-aircraft sample means (as the rollout's sample
// mean: compensated, in sample order, +inf when any sample was infeasible),
// their sum C_l, and the gradient summed over the sample ranges (zero when the
// particle is infeasible).
__global__ void __launch_bounds__(256) grad_reduce_kernel(const float *__restrict__ cost_ms,
                                                          const float *__restrict__ gpart,
                                                          long long L, int M, int N, int nS3,
                                                          int nchunk, float *__restrict__ cost,
                                                          float *__restrict__ grad,
                                                          float *__restrict__ cbar)
{
    const long long l = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= L) return;
    float cb = 0.0f;
    bool inf = false;
    if (lane < N) {
        Kahan s;
        for (int m = 0; m < M; ++m) {
            const float v = __ldg(cost_ms + ((size_t)m * N + lane) * (size_t)L + l);
            if (isinf(v)) inf = true;
            else s.add(v);
        }
        cb = inf ? __int_as_float(0x7f800000) : s.s / (float)M;
        if (cbar) cbar[(size_t)lane * L + l] = cb;
    }
    const bool infeasible = __any_sync(0xffffffffu, inf);
    double tot = lane < N && !inf ? (double)cb : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) cost[l] = infeasible ? __int_as_float(0x7f800000) : (float)tot;
    const int nel = N * nS3;
    const size_t stride = (size_t)L * nel;
    for (int n = lane; n < nel; n += 32) {
        float g = 0.0f;
        if (!infeasible)
            for (int c = 0; c < nchunk; ++c) g += __ldg(gpart + c * stride + (size_t)l * nel + n);
        grad[(size_t)l * nel + n] = g;
    }
}

}  // namespace

// Launch-bound variants (block size cap, minimum resident blocks per SM); the
// register budget per thread is 65536 / (cap * blocks).  The variant is chosen
// by timing (host side) among those whose cap fits the block (32 N threads).
struct GradVariant {
    int max_threads, min_blocks;
};
constexpr GradVariant kGradVariants[] = {{256, 1}, {256, 2}, {256, 3}, {384, 1}, {384, 2},
                                         {512, 1}, {768, 1}, {1024, 1}};
constexpr int kNumGradVariants = sizeof(kGradVariants) / sizeof(kGradVariants[0]);

int rollout_grad_variants(int N, int *out)
{
    int n = 0;
    for (int v = 0; v < kNumGradVariants; ++v)
        if (kGradVariants[v].max_threads >= N * kPB) out[n++] = v;
    return n;
}

#define TMA_GRAD_VARIANT_SWITCH(V, CALL)                              \
    switch (V) {                                                      \
    case 0: CALL(256, 1); break;                                      \
    case 1: CALL(256, 2); break;                                      \
    case 2: CALL(256, 3); break;                                      \
    case 3: CALL(384, 1); break;                                      \
    case 4: CALL(384, 2); break;                                      \
    case 5: CALL(512, 1); break;                                      \
    case 6: CALL(768, 1); break;                                      \
    default: CALL(1024, 1); break;                                    \
    }

static int valid_variant(int N, int variant)
{
    if (variant >= 0 && variant < kNumGradVariants && kGradVariants[variant].max_threads >= N * kPB)
        return variant;
    int cand[kNumGradVariants];
    rollout_grad_variants(N, cand);
    return cand[0];
}

cudaError_t rollout_grad_occupancy(int N, int variant, int *blocks_per_sm)
{
    const int block = N * kPB;
    const size_t smem = (size_t)2 * 3 * N * kPB * sizeof(float);
#define TMA_OCC(T, B)                                                                            \
    do {                                                                                         \
        if (smem > 48 * 1024)                                                                    \
            cudaFuncSetAttribute(rollout_grad_kernel<T, B>,                                      \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, rollout_grad_kernel<T, B>, \
                                                             block, smem);                       \
    } while (0)
    TMA_GRAD_VARIANT_SWITCH(valid_variant(N, variant), TMA_OCC)
#undef TMA_OCC
    return cudaSuccess;
}

cudaError_t launch_rollout_grad(const ProblemC &P, const DynState *dyn, const float *u,
                                const float *W, int64_t L, int J, int nchunk, float *cost_ms,
                                float *gpart, float *cost, float *grad, float *cbar,
                                cudaStream_t st, int variant)
{
    if (L <= 0) return cudaSuccess;
    const long long nLb = (L + kPB - 1) / kPB;
    const int m_per_block = (P.M + nchunk - 1) / nchunk;
    nchunk = (P.M + m_per_block - 1) / m_per_block;
    const unsigned grid = (unsigned)(nLb * nchunk);
    const int block = P.N * kPB;
    const size_t smem = (size_t)grad_smem_words(P.N) * sizeof(float);
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
#define TMA_LAUNCH(T, B)                                                                   \
    do {                                                                                   \
        if (smem > 48 * 1024)                                                              \
            cudaFuncSetAttribute(rollout_grad_kernel<T, B>,                                \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
        rollout_grad_kernel<T, B><<<grid, block, smem, st>>>(P, dyn, u, W4, L, (int)nLb,   \
                                                             m_per_block, J, cost_ms, gpart); \
    } while (0)
    TMA_GRAD_VARIANT_SWITCH(valid_variant(P.N, variant), TMA_LAUNCH)
#undef TMA_LAUNCH
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !cost) return e;
    grad_reduce_kernel<<<(unsigned)((L * 32 + 255) / 256), 256, 0, st>>>(
        cost_ms, gpart, L, P.M, P.N, P.S * 3, nchunk, cost, grad, cbar);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tma
