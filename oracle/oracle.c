/*
 * oracle.c -- plain FP64 CPU oracle of the SMC-MPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the
 * benchmark).  It shares no code with the CUDA path.  Loops are written in
 * the order of the paper's definitions, with no blocking or fusion; OpenMP
 * over independent particles is the only parallelism (timing only).
 *
 * Readings of the paper (Eele & Maciejowski, TR.693, 2015) used here:
 *  R1  Controls are (turn rate w, climb rate hdot, speed change a), piecewise
 *      constant over S equal segments, segment s = floor(k*S/H).  They map to
 *      the paper's (gamma, phi, T) of Sec. 3.3 by sin(gamma) = hdot/v,
 *      tan(phi) = w v / (g cos(gamma)) (coordinated turn) and
 *      T = m (a + g sin(gamma)) + D.
 *  R2  "Standard aerodynamic relations" (Sec. 3.3): lift from the coordinated
 *      turn, L = m g cos(gamma)/cos(phi) = C_L q S; drag polar
 *      D = q S (CD0 + CD2 C_L^2); ISA troposphere density
 *      rho = 1.225 (1 - 2.2558e-5 z)^4.2559; fuel flow eta = Cf1 (1 + v/Cf2)
 *      (Sec. 6.2, Eq. (blah)).
 *  R3  Control constraints (gamma, phi, T of Sec. 3.4) are checked on the
 *      step-k values, unary state constraints (z, v, m) on the step-(k+1)
 *      state.  A violating aircraft gets weight 0 (cost +inf) and is frozen
 *      from that step on: it takes no part in later separation checks.
 *  R4  Landing (Eq. (TO_init)) is tested on the step-(k+1) state of arrivals;
 *      the bearing cone uses atan2(y, x) with x > 0, the heading test
 *      |wrap(chi - pi)| <= P_chi.  A landed aircraft is frozen, leaves the
 *      separation checks and scores the best per-step value for the remaining
 *      steps (Sec. 3.9).
 *  R5  Separation (Eq. (avoidance)) is violated when d_h^2 < sep_h^2 and
 *      |dz| < sep_v, checked at steps 1..H between flying aircraft.  Soft form:
 *      mu * sum_k sum_j softplus_beta(min(1 - d_h/sep_h, 1 - |dz|/sep_v)).
 *  R6  Deviation sums run over steps 1..H and are divided by H (the paper's
 *      sum from k to k+H has H+1 terms).  The extra 1/H in J_T is dropped so
 *      that 0 <= J_T <= 1 as the paper states.  The fuel term is
 *      1 - F/(H dt Tmax eta(vmax)) (the printed form grows with fuel burned).
 *  R7  Departure: A = bearing error |wrap(atan2(y,x) - theta_F)| (sup pi,
 *      inf 0); B = |Z - z| with sup/inf the per-step means of
 *      d0 +/- k dt vmax sin(gamma_max) (inf clipped at 0); C = |v - v_D| with
 *      sup max(vmax - v_D, v_D - vmin).
 *  R8  Arrival flow field (Eq. (flow)) restated in the mathematical heading
 *      convention: the arc through the aircraft tangent to the runway at the
 *      origin has central angle 2*theta_p (theta_p = atan2(y,x)), heading
 *      chi_hat = pi + 2*theta_p, remaining arc length
 *      s = r*theta_p/sin(theta_p) capped at 4r (continuous cap), glide angle
 *      beta = atan2(z, s).  D = |wrap(chi - chi_hat)| (sup pi),
 *      E = |beta - beta_f| (sup pi/2).
 *  R9  Weights of Table coeff attach to the named terms: departure
 *      (bearing, fuel, altitude, speed), arrival (flow heading, glide path,
 *      fuel).  J_T = (1 - w_n) sum alpha J + w_n J_noise (Sec. 7.1).
 *  R10 Per-sample cost c = -ln J_T; the product of Sec. 3.6 over M samples
 *      becomes the mean cost, and the annealed log-weight is
 *      l = -kappa_J * mean_m c with kappa_J = floor(3 + 5 exp(0.05 J))
 *      (SampleSchedule of Sec. 5.1), J = 0..J_max-1.
 *  R11 Wind (Sec. 3.9.1): grid nodes inclusive over the box; covariance
 *      sigma^2 exp(-beta |dxy|) exp(-gamma |dz|) (sigma constant); time
 *      factor a = exp(-dt*lam_t), lam_t read in 1/s.  The field is shared by
 *      all particles of a solve (common random numbers); white turbulence is
 *      drawn per particle, sample, aircraft and step.  Positions are clamped
 *      into the box before trilinear interpolation.
 *  R12 Resampling (Sec. 3.7) is systematic on a fixed-point CDF:
 *      q_j = floor(w_j 2^40), S = inclusive prefix sum, Q = S_{L-1},
 *      t_l = floor((l 2^32 + r) Q / (L 2^32)), a_l = min{j : S_j > t_l}.
 *  R13 Perturbation (Algorithm 1): Gaussian random walk, clipped to the
 *      control box.  Final selection (Sec. 3.8): the particle with the fewest
 *      infeasible aircraft, then the smallest sum of mean costs (= the largest
 *      product of weights), ties to the lowest index.
 *  R14 Random numbers: Philox4x32-10, key = seed + scenario_id*0x9E3779B97F4A7C15,
 *      counter (c0, c1, q | stream<<24, J | mpc_step<<16); uniforms use the
 *      top 23 bits, ((x>>9)+0.5)/2^23 (an odd multiple of 2^-24, exact in FP32
 *      and FP64); normals by Box-Muller.
 *  R15 Plant (Fig. 1): one step dt of the chosen first-segment controls
 *      under the wind of sample 0 at step 0 plus turbulence (stream 7), with
 *      |sin(gamma)| held at 0.999 and T held within [Tmin, Tmax].
 *  R16 Gradient (an extension): reverse mode of the soft objective over the
 *      discrete dynamics; every limit, landing, cell and min/|.| decision keeps
 *      its forward value.
 *  R17 Metropolis-Hastings moves (an extension): target exp(-kappa C(u)) per
 *      particle, coordinates scaled by the move step of their kind.
 *  R18 Held-out evaluation winds: the wind model drawn from stream 8.
 *  R19 Wind mode 1: one field per (particle, sample) on the 2x2x2 grid of the
 *      box corners, drawn from stream 9 (see orc_particle_wind).
 *  R20 Sample mode 1 (the inner loop of Algorithm 1): iteration J uses the
 *      first M_J = min(SampleSchedule(J), M) samples and the log-weight is
 *      the log of the product of J_T over them, -M_J * (mean cost).  The
 *      driver of the solve (oracle/__init__.py) applies it; the rollout here
 *      takes the sample count as P->M.
 *  R22 Rolling window (the paper's rolling-window section): aircraft i enters
 *      at MPC step t_enter and, at MPC step t, flies the horizon steps
 *      k >= k_in = max(0, t_enter - t) from its entry state; its objective
 *      is the mean of its per-step terms over its H - k_in active steps
 *      (the fuel bound and the departure altitude bounds over those steps).
 *      An aircraft with k_in >= H, or one that has finished, is not in the
 *      problem: cost 0 (J_T = 1), no simulation, no separation checks.  The
 *      plant moves only active aircraft and marks an arrival finished once
 *      it is in the landing sector of Eq. (TO_init).
 *  R21 Particle schedule: iteration J evaluates L_J particles; the systematic
 *      resampling after it draws L_{J+1} ancestors from the L_J weighted ones
 *      (orc_resample_to); the perturbation makes L_{J+1} children.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static const double G0 = 9.80665;

/* ------------------------------------------------------------------ */
/* random numbers                                                       */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {              /* Weyl key schedule */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform23(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) / 8388608.0;
}

void orc_box_muller(uint32_t xa, uint32_t xb, double *z0, double *z1)
{
    double ua = orc_uniform23(xa), ub = orc_uniform23(xb);
    double r = sqrt(-2.0 * log(ua));
    *z0 = r * cos(2.0 * M_PI * ub);
    *z1 = r * sin(2.0 * M_PI * ub);
}

void orc_draw(const orc_problem *P, uint32_t c0, uint32_t c1, uint32_t q, uint32_t stream,
              uint32_t J, uint32_t out[4])
{
    uint64_t s = P->seed + (uint64_t)P->scenario_id * 0x9E3779B97F4A7C15ull;
    uint32_t key[2] = {(uint32_t)s, (uint32_t)(s >> 32)};
    uint32_t ctr[4] = {c0, c1, (q & 0xFFFFFFu) | (stream << 24),
                       (J & 0xFFFFu) | (P->mpc_step << 16)};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* wind model, Sec. 3.9.1: the standard normals v_X(k), v_Y(k)           */
/* ------------------------------------------------------------------ */

void orc_wind_normals(const orc_problem *P, int m0, int mc, double *out)
{
    const int64_t Pn = (int64_t)P->grid[0] * P->grid[1] * P->grid[2];
    for (int mm = 0; mm < mc; mm++) {
        int m = m0 + mm;
        for (int k = 0; k < P->H; k++) {
            for (int64_t p = 0; p < Pn; p++) {
                uint32_t w[4];
                orc_draw(P, (uint32_t)p, (uint32_t)m << 8, (uint32_t)k,
                         P->wind_stream ? P->wind_stream : 3u, 0u, w);
                double z0, z1;
                orc_box_muller(w[0], w[1], &z0, &z1);
                double *o = out + (((int64_t)mm * P->H + k) * Pn + p) * 2;
                o[0] = z0;
                o[1] = z1;
            }
        }
    }
}

/* Mode 1 (reading R19): a wind field per (particle, sample) on the 2x2x2 grid of
 * the box corners, as the paper draws it inside its GPU kernel (Sec. 6).  The
 * recursion W(0) = Qhat v(0), W(k+1) = a W(k) + Q v(k+1), Q = sqrt(1 - a^2) Qhat,
 * is written W(k) = Qhat B(k) with B(0) = v(0), B(k) = a B(k-1) + sqrt(1-a^2) v(k).
 * The normals come from random stream 9: counter (c0 = l, c1 = 4 m + r, q = k) for
 * r = 0..3; draw r gives node 2r (words 0, 1: v_X, v_Y) and node 2r+1 (words 2, 3). */
void orc_particle_wind(const orc_problem *P, int64_t l, int m, double *out)
{
    const double a = exp(-P->dt * P->lam_t), b = sqrt(1.0 - a * a);
    double B[8][2];
    for (int k = 0; k < P->H; k++) {
        for (int r = 0; r < 4; r++) {
            uint32_t w[4];
            orc_draw(P, (uint32_t)l, (uint32_t)(4 * m + r), (uint32_t)k, 9u, 0u, w);
            double v[4];
            orc_box_muller(w[0], w[1], &v[0], &v[1]);
            orc_box_muller(w[2], w[3], &v[2], &v[3]);
            for (int h = 0; h < 2; h++)
                for (int c = 0; c < 2; c++) {
                    const int n = 2 * r + h;
                    B[n][c] = k == 0 ? v[2 * h + c] : a * B[n][c] + b * v[2 * h + c];
                }
        }
        for (int n = 0; n < 8; n++)
            for (int c = 0; c < 2; c++) {
                double s = 0.0;
                for (int j = 0; j <= n; j++) s += P->wind_chol[n * 8 + j] * B[j][c];
                out[((int64_t)k * 8 + n) * 2 + c] = s;
            }
    }
}

/* trilinear interpolation of one wind field W_k[p][2] */
static void trilinear(const orc_problem *P, const double *Wk, double x, double y, double z,
                      double *wx, double *wy)
{
    double pos[3] = {x, y, z};
    int idx[3];
    double t[3];
    for (int d = 0; d < 3; d++) {
        double lo = P->box_lo[d], hi = P->box_hi[d];
        int n = P->grid[d];
        double h = (hi - lo) / (n - 1);
        double c = pos[d] < lo ? lo : (pos[d] > hi ? hi : pos[d]);
        double f = (c - lo) / h;
        int i = (int)floor(f);
        if (i > n - 2) i = n - 2;
        if (i < 0) i = 0;
        idx[d] = i;
        t[d] = f - i;
    }
    const int ny = P->grid[1], nz = P->grid[2];
    double ax = 0.0, ay = 0.0;
    for (int dx = 0; dx < 2; dx++)
        for (int dy = 0; dy < 2; dy++)
            for (int dz = 0; dz < 2; dz++) {
                double w = (dx ? t[0] : 1.0 - t[0]) * (dy ? t[1] : 1.0 - t[1]) *
                           (dz ? t[2] : 1.0 - t[2]);
                int64_t p = ((int64_t)(idx[0] + dx) * ny + (idx[1] + dy)) * nz + (idx[2] + dz);
                ax += w * Wk[2 * p];
                ay += w * Wk[2 * p + 1];
            }
    *wx = ax;
    *wy = ay;
}

/* population density of Sec. 7.1, bilinear between grid nodes, 0 outside */
static double popdense_at(const orc_problem *P, double x, double y)
{
    if (!P->popdense || P->pop_n[0] < 2 || P->pop_n[1] < 2) return 0.0;
    if (x < P->pop_lo[0] || x > P->pop_hi[0] || y < P->pop_lo[1] || y > P->pop_hi[1]) return 0.0;
    const int n0 = P->pop_n[0], n1 = P->pop_n[1];
    double f0 = (x - P->pop_lo[0]) / ((P->pop_hi[0] - P->pop_lo[0]) / (n0 - 1));
    double f1 = (y - P->pop_lo[1]) / ((P->pop_hi[1] - P->pop_lo[1]) / (n1 - 1));
    int i0 = (int)floor(f0), i1 = (int)floor(f1);
    if (i0 > n0 - 2) i0 = n0 - 2;
    if (i1 > n1 - 2) i1 = n1 - 2;
    if (i0 < 0) i0 = 0;
    if (i1 < 0) i1 = 0;
    double t0 = f0 - i0, t1 = f1 - i1;
    const double *g = P->popdense;
    return (1 - t0) * (1 - t1) * g[(int64_t)i0 * n1 + i1] + (1 - t0) * t1 * g[(int64_t)i0 * n1 + i1 + 1] +
           t0 * (1 - t1) * g[(int64_t)(i0 + 1) * n1 + i1] + t0 * t1 * g[(int64_t)(i0 + 1) * n1 + i1 + 1];
}

/* absolute angular distance of an angle difference, in [0, pi] */
static double angdist(double a)
{
    double r = fmod(fabs(a), 2.0 * M_PI);
    return r > M_PI ? 2.0 * M_PI - r : r;
}

/* ------------------------------------------------------------------ */
/* decision margins (used by the tests to set aside near-threshold      */
/* cases, where FP32 and FP64 may legitimately decide differently)      */
/* ------------------------------------------------------------------ */

/* The margins are bookkeeping of the parity protocol, not part of the method.
 * orc_margin_t and ORC_MARGIN(expr) (the evaluation of a margin) are double and
 * (expr) here; the operation-counting build of opcount.cpp redefines them so
 * that this bookkeeping stays out of its count. */
#ifndef ORC_MARGIN_T
#define ORC_MARGIN_T double
#define ORC_MARGIN(expr) (expr)
#endif
typedef ORC_MARGIN_T orc_margin_t;

typedef struct {
    int n_false;
    orc_margin_t min_true, max_false;
} conj_t;

static void conj_init(conj_t *c) { c->n_false = 0; c->min_true = INFINITY; c->max_false = 0.0; }
static void conj_add(conj_t *c, int ok, orc_margin_t margin)
{
    if (ok) {
        if (margin < c->min_true) c->min_true = margin;
    } else {
        c->n_false++;
        if (margin > c->max_false) c->max_false = margin;
    }
}
static int conj_ok(const conj_t *c) { return c->n_false == 0; }
/* a true conjunction flips when any member flips; a false one only when every false member does */
static orc_margin_t conj_margin(const conj_t *c) { return c->n_false == 0 ? c->min_true : c->max_false; }
static double rel(double a, double b, double scale) { return fabs(a - b) / fabs(scale); }

/* ------------------------------------------------------------------ */
/* rollout of one (particle, wind sample): Algorithm 1, inner loop body */
/* ------------------------------------------------------------------ */

typedef struct {
    double x, y, z, v, chi, m, F;
    int dead, landed, sepv;
    double sA, sB, sC, sN, soft;
    orc_margin_t margin, smargin;
} acst;

static double softplus(double g, double beta)
{
    double bg = beta * g;
    return bg > 0 ? (bg + log1p(exp(-bg))) / beta : log1p(exp(bg)) / beta;
}

static void record(const acst *st, int N, double *traj)
{
    for (int i = 0; i < N; i++) {
        double *o = traj + (int64_t)i * 8;
        o[0] = st[i].x; o[1] = st[i].y; o[2] = st[i].z; o[3] = st[i].v;
        o[4] = st[i].chi; o[5] = st[i].m; o[6] = st[i].F;
        o[7] = st[i].dead + 2 * st[i].landed + 4 * st[i].sepv;
    }
}

static void rollout_sample(const orc_problem *P, const orc_aircraft *A, const double *Wm, int m,
                           const double *ul, int64_t l, int J, acst *st, double *ch, double *cs,
                           double *mg, double *smg, int64_t *live, double *traj)
{
    const int N = P->N, H = P->H, S = P->S;
    const int64_t Pn = (int64_t)P->grid[0] * P->grid[1] * P->grid[2];
    const double dt = P->dt;
    const double sgmax = sin(P->gamma_max), tpmax = tan(P->phi_max);
    const double Sh2 = P->sep_h * P->sep_h, Sv = P->sep_v;
    int64_t nlive = 0;
    double *own = NULL;
    if (P->wind_mode == 1) {      /* this particle's own field for this sample */
        own = (double *)malloc(sizeof(double) * (size_t)H * 16);
        orc_particle_wind(P, l, m, own);
        Wm = own;
    }

    /* rolling window (reading R22): first active step, and whether the
     * aircraft is in the problem at all during this horizon */
    int kin[256], out[256];
    for (int i = 0; i < N; i++) {
        kin[i] = 0;
        out[i] = 0;
        if (P->rolling) {
            const int64_t d = (int64_t)A[i].t_enter - (int64_t)P->mpc_step;
            kin[i] = d > 0 ? (d < H ? (int)d : H) : 0;
            out[i] = ((P->finished >> i) & 1u) || kin[i] >= H;
        }
    }
    for (int i = 0; i < N; i++) {
        acst *s = &st[i];
        memset(s, 0, sizeof(*s));
        s->x = A[i].x; s->y = A[i].y; s->z = A[i].z;
        s->v = A[i].v; s->chi = A[i].chi; s->m = A[i].m;
        s->margin = INFINITY;
        s->smargin = INFINITY;
    }
    if (traj) record(st, N, traj);

    for (int k = 0; k < H; k++) {
        const double *Wk = Wm + (int64_t)k * Pn * 2;
        for (int i = 0; i < N; i++) {
            acst *s = &st[i];
            const orc_aircraft *a = &A[i];
            if (s->dead || s->landed || out[i] || k < kin[i]) continue;
            nlive++;
            const int seg = (int)(((int64_t)k * S) / H);
            const double *uu = ul + ((int64_t)i * S + seg) * 3;
            const double w = uu[0], hd = uu[1], acc = uu[2];

            /* control constraints on the step-k values (Sec. 3.4) */
            double sg = hd / s->v;
            conj_t cc;
            conj_init(&cc);
            conj_add(&cc, fabs(sg) <= sgmax, ORC_MARGIN(rel(fabs(sg), sgmax, sgmax)));
            if (!(fabs(sg) < 1.0)) {
                orc_margin_t cm = conj_margin(&cc);
                if (cm < s->margin) s->margin = cm;
                if (cm < s->smargin) s->smargin = cm;
                s->dead = 1;
                continue;
            }
            double cg = sqrt(1.0 - sg * sg);
            double tp = w * s->v / (G0 * cg);
            conj_add(&cc, fabs(tp) < tpmax, ORC_MARGIN(rel(fabs(tp), tpmax, tpmax)));
            double cphi = 1.0 / sqrt(1.0 + tp * tp);
            double sphi = tp * cphi;
            double base = 1.0 - 2.2558e-5 * s->z;
            double rho = 1.225 * pow(base > 0.0 ? base : 0.0, 4.2559);
            double qS = 0.5 * rho * s->v * s->v * a->S;
            double CL = s->m * G0 * cg / (qS * cphi);
            double D = qS * (a->CD0 + a->CD2 * CL * CL);
            double T = s->m * (acc + G0 * sg) + D;
            conj_add(&cc, T >= a->Tmin, ORC_MARGIN(rel(T, a->Tmin, a->Tmax)));
            conj_add(&cc, T <= a->Tmax, ORC_MARGIN(rel(T, a->Tmax, a->Tmax)));
            {
                orc_margin_t cm = conj_margin(&cc);
                if (cm < s->margin) s->margin = cm;
                if (cm < s->smargin) s->smargin = cm;
            }
            if (!conj_ok(&cc)) { s->dead = 1; continue; }
            double Lift = CL * qS;
            double eta = a->Cf1 * (1.0 + s->v / a->Cf2);

            /* disturbance: wind field plus white turbulence */
            double wx, wy;
            trilinear(P, Wk, s->x, s->y, s->z, &wx, &wy);
            uint32_t tb[4];
            orc_draw(P, (uint32_t)l, (uint32_t)i | ((uint32_t)m << 8), (uint32_t)(k >> 1), 0u,
                     (uint32_t)J, tb);
            double n0, n1;
            if ((k & 1) == 0) orc_box_muller(tb[0], tb[1], &n0, &n1);
            else              orc_box_muller(tb[2], tb[3], &n0, &n1);
            wx += P->turb_sigma * n0;
            wy += P->turb_sigma * n1;

            /* explicit Euler step, Eq. (hor) */
            double x1 = s->x + dt * (s->v * cos(s->chi) * cg) + wx * dt;
            double y1 = s->y + dt * (s->v * sin(s->chi) * cg) + wy * dt;
            double z1 = s->z + dt * (s->v * sg);
            double v1 = s->v + dt * ((T - D) / s->m - G0 * sg);
            double chi1 = s->chi + dt * (Lift * sphi / (s->m * s->v));
            double burn = dt * (eta * T);
            double m1 = s->m - burn;
            s->F += burn;
            s->x = x1; s->y = y1; s->z = z1; s->v = v1; s->chi = chi1; s->m = m1;

            /* unary state constraints on the step-(k+1) state (Sec. 3.4) */
            conj_t cu;
            conj_init(&cu);
            conj_add(&cu, z1 >= P->z_min, ORC_MARGIN(rel(z1, P->z_min, P->z_min)));
            conj_add(&cu, z1 <= P->z_max, ORC_MARGIN(rel(z1, P->z_max, P->z_max)));
            conj_add(&cu, v1 >= P->v_min, ORC_MARGIN(rel(v1, P->v_min, P->v_min)));
            conj_add(&cu, v1 <= P->v_max, ORC_MARGIN(rel(v1, P->v_max, P->v_max)));
            conj_add(&cu, m1 >= a->m_empty, ORC_MARGIN(rel(m1, a->m_empty, a->m_empty)));
            {
                orc_margin_t cm = conj_margin(&cu);
                if (cm < s->margin) s->margin = cm;
                if (cm < s->smargin) s->smargin = cm;
            }
            if (!conj_ok(&cu)) { s->dead = 1; continue; }

            double th = atan2(y1, x1);
            if (a->type == 0) {
                /* arrival: flow-field geometry and landing sector */
                double r = sqrt(x1 * x1 + y1 * y1);
                double ath = fabs(th);
                double ratio = ath < 1e-3 ? 1.0 + th * th / 6.0 : ath / fmax(sin(ath), 0.25 * ath);
                double sarc = r * ratio;
                double beta = atan2(z1, sarc);
                double chihat = M_PI + 2.0 * th;
                double hdg = angdist(chi1 - M_PI);
                conj_t cl;
                conj_init(&cl);
                conj_add(&cl, r <= P->P_runway, ORC_MARGIN(rel(r, P->P_runway, P->P_runway)));
                conj_add(&cl, beta <= P->P_beta, ORC_MARGIN(rel(beta, P->P_beta, P->P_beta)));
                conj_add(&cl, x1 > 0.0, ORC_MARGIN(fabs(x1) / P->P_runway));
                conj_add(&cl, ath <= P->P_chi, ORC_MARGIN(rel(ath, P->P_chi, P->P_chi)));
                conj_add(&cl, hdg <= P->P_chi, ORC_MARGIN(rel(hdg, P->P_chi, P->P_chi)));
                conj_add(&cl, v1 <= P->P_vs, ORC_MARGIN(rel(v1, P->P_vs, P->P_vs)));
                {
                    orc_margin_t cm = conj_margin(&cl);
                    if (cm < s->margin) s->margin = cm;
                    if (cm < s->smargin) s->smargin = cm;
                }
                if (conj_ok(&cl)) { s->landed = 1; continue; }
                s->sA += angdist(chi1 - chihat);
                s->sB += fabs(beta - P->beta_f);
            } else {
                s->sA += angdist(th - a->theta_F);
                s->sB += fabs(a->Z - z1);
                s->sC += fabs(v1 - a->v_D);
            }
            if (P->w_noise != 0.0) {
                double za = z1 / P->A_c;
                double h = 1.0 - za * za;
                if (h < 0.0) h = 0.0;
                s->sN += h * popdense_at(P, x1, y1);
            }
        }

        /* binary separation constraints at step k+1, Eq. (avoidance) */
        for (int i = 0; i < N; i++) {
            if (st[i].dead || st[i].landed || out[i] || k < kin[i]) continue;
            for (int j = i + 1; j < N; j++) {
                if (st[j].dead || st[j].landed || out[j] || k < kin[j]) continue;
                double dx = st[i].x - st[j].x, dy = st[i].y - st[j].y, dz = st[i].z - st[j].z;
                double dh2 = dx * dx + dy * dy, adz = fabs(dz);
                conj_t cp;
                conj_init(&cp);
                conj_add(&cp, dh2 < Sh2, ORC_MARGIN(rel(dh2, Sh2, Sh2)));
                conj_add(&cp, adz < Sv, ORC_MARGIN(rel(adz, Sv, Sv)));
                orc_margin_t cm = conj_margin(&cp);
                if (cm < st[i].margin) st[i].margin = cm;
                if (cm < st[j].margin) st[j].margin = cm;
                if (conj_ok(&cp)) { st[i].sepv = 1; st[j].sepv = 1; }
                if (cs) {
                    double g = fmin(1.0 - sqrt(dh2) / P->sep_h, 1.0 - adz / Sv);
                    double pen = softplus(g, P->sp_beta);
                    st[i].soft += pen;
                    st[j].soft += pen;
                }
            }
        }
        if (traj) record(st, N, traj + (int64_t)(k + 1) * N * 8);
    }

    /* objectives (Sec. 3.5, Sec. 7.1) and per-sample cost (Sec. 3.6) */
    orc_margin_t smin = INFINITY;
    for (int i = 0; i < N; i++) {
        const acst *s = &st[i];
        const orc_aircraft *a = &A[i];
        if (out[i]) {                 /* not in the problem this horizon: J_T = 1 */
            if (ch) ch[i] = 0.0;
            if (cs) cs[i] = 0.0;
            if (mg) mg[i] = s->margin;
            continue;
        }
        const int Ha = H - kin[i];    /* active steps (H without a rolling window) */
        const double eta_max = a->Cf1 * (1.0 + P->v_max / a->Cf2);
        const double Fmax = Ha * dt * a->Tmax * eta_max;
        const double Jf = 1.0 - s->F / Fmax;
        double Jsum;
        if (a->type == 1) {
            double d0 = fabs(a->Z - a->z), c = P->v_max * sgmax * dt;
            double supB = 0.0, infB = 0.0;
            for (int k = 1; k <= Ha; k++) {
                supB += d0 + k * c;
                infB += (d0 - k * c) > 0.0 ? d0 - k * c : 0.0;
            }
            supB /= Ha;
            infB /= Ha;
            double J1 = 1.0 - (s->sA / Ha) / M_PI;
            double J3 = (supB - s->sB / Ha) / (supB - infB);
            double Cmax = fmax(P->v_max - a->v_D, a->v_D - P->v_min);
            double J4 = 1.0 - (s->sC / Ha) / Cmax;
            Jsum = P->alpha_dep[0] * J1 + P->alpha_dep[1] * Jf + P->alpha_dep[2] * J3 +
                   P->alpha_dep[3] * J4;
        } else {
            double J1 = 1.0 - (s->sA / Ha) / M_PI;
            double J3 = 1.0 - (s->sB / Ha) / (0.5 * M_PI);
            Jsum = P->alpha_arr[0] * J1 + P->alpha_arr[1] * J3 + P->alpha_arr[2] * Jf;
        }
        double JT = (1.0 - P->w_noise) * Jsum + P->w_noise * (1.0 - s->sN / Ha);
        double base = -log(JT > 1e-30 ? JT : 1e-30);
        if (ch) ch[i] = (s->dead || s->sepv) ? INFINITY : base;
        if (cs) cs[i] = s->dead ? INFINITY : base + P->mu_sep * s->soft;
        if (mg) mg[i] = s->margin;
        if (s->smargin < smin) smin = s->smargin;
    }
    if (smg) *smg = smin;
    if (live) *live += nlive;
    free(own);
}

void orc_rollout(const orc_problem *P, const orc_aircraft *A, const double *W, int m0, int mc,
                 const double *u, const int64_t *pidx, int Lsub, int J, int nthreads,
                 double *cost_hard, double *cost_soft, double *margin, double *smargin,
                 int64_t *live)
{
    const int N = P->N;
    const int64_t Pn = (int64_t)P->grid[0] * P->grid[1] * P->grid[2];
    const int64_t wstride = (int64_t)P->H * Pn * 2;
    const int64_t ustride = (int64_t)N * P->S * 3;
    int64_t total_live = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads) reduction(+ : total_live)
    for (int ll = 0; ll < Lsub; ll++) {
        acst st[256];
        int64_t nl = 0;
        for (int mm = 0; mm < mc; mm++) {
            int64_t o = ((int64_t)ll * mc + mm) * N;
            rollout_sample(P, A, W + (int64_t)mm * wstride, m0 + mm, u + (int64_t)ll * ustride,
                           pidx[ll], J, st, cost_hard ? cost_hard + o : NULL,
                           cost_soft ? cost_soft + o : NULL, margin ? margin + o : NULL,
                           smargin ? smargin + (int64_t)ll * mc + mm : NULL, &nl, NULL);
        }
        total_live += nl;
    }
    if (live) *live = total_live;
}

void orc_trajectory(const orc_problem *P, const orc_aircraft *A, const double *Wm, int m,
                    const double *ul, int64_t l, int J, double *traj, double *cost_hard,
                    double *cost_soft)
{
    acst st[256];
    int64_t nl = 0;
    rollout_sample(P, A, Wm, m, ul, l, J, st, cost_hard, cost_soft, NULL, NULL, &nl, traj);
}

/* ------------------------------------------------------------------ */
/* reverse-mode derivative of the soft cost (gradient for the MALA move)   */
/* ------------------------------------------------------------------ */

/* wind interpolation with its gradient with respect to position (zero along
 * an axis where the position is clamped to the box) */
static void trilinear_grad(const orc_problem *P, const double *Wk, double x, double y, double z,
                           double w[2], double dw[2][3])
{
    double pos[3] = {x, y, z};
    int idx[3], inside[3];
    double t[3], ih[3];
    for (int d = 0; d < 3; d++) {
        double lo = P->box_lo[d], hi = P->box_hi[d];
        int n = P->grid[d];
        double h = (hi - lo) / (n - 1);
        inside[d] = pos[d] > lo && pos[d] < hi;
        double c = pos[d] < lo ? lo : (pos[d] > hi ? hi : pos[d]);
        double f = (c - lo) / h;
        int i = (int)floor(f);
        if (i > n - 2) i = n - 2;
        if (i < 0) i = 0;
        idx[d] = i;
        t[d] = f - i;
        ih[d] = 1.0 / h;
    }
    const int ny = P->grid[1], nz = P->grid[2];
    for (int c = 0; c < 2; c++) {
        w[c] = 0.0;
        dw[c][0] = dw[c][1] = dw[c][2] = 0.0;
    }
    for (int dx = 0; dx < 2; dx++)
        for (int dy = 0; dy < 2; dy++)
            for (int dz = 0; dz < 2; dz++) {
                double fx = dx ? t[0] : 1.0 - t[0], fy = dy ? t[1] : 1.0 - t[1], fz = dz ? t[2] : 1.0 - t[2];
                double gx = (dx ? 1.0 : -1.0) * ih[0], gy = (dy ? 1.0 : -1.0) * ih[1], gz = (dz ? 1.0 : -1.0) * ih[2];
                int64_t p = ((int64_t)(idx[0] + dx) * ny + (idx[1] + dy)) * nz + (idx[2] + dz);
                for (int c = 0; c < 2; c++) {
                    double v = Wk[2 * p + c];
                    w[c] += fx * fy * fz * v;
                    dw[c][0] += gx * fy * fz * v;
                    dw[c][1] += fx * gy * fz * v;
                    dw[c][2] += fx * fy * gz * v;
                }
            }
    for (int c = 0; c < 2; c++)
        for (int d = 0; d < 3; d++)
            if (!inside[d]) dw[c][d] = 0.0;
}

/* population density and its gradient (0 outside the grid) */
static double popdense_grad(const orc_problem *P, double x, double y, double *gx, double *gy)
{
    *gx = *gy = 0.0;
    if (!P->popdense || P->pop_n[0] < 2 || P->pop_n[1] < 2) return 0.0;
    if (x < P->pop_lo[0] || x > P->pop_hi[0] || y < P->pop_lo[1] || y > P->pop_hi[1]) return 0.0;
    const int n0 = P->pop_n[0], n1 = P->pop_n[1];
    double h0 = (P->pop_hi[0] - P->pop_lo[0]) / (n0 - 1), h1 = (P->pop_hi[1] - P->pop_lo[1]) / (n1 - 1);
    double f0 = (x - P->pop_lo[0]) / h0, f1 = (y - P->pop_lo[1]) / h1;
    int i0 = (int)floor(f0), i1 = (int)floor(f1);
    if (i0 > n0 - 2) i0 = n0 - 2;
    if (i1 > n1 - 2) i1 = n1 - 2;
    if (i0 < 0) i0 = 0;
    if (i1 < 0) i1 = 0;
    double t0 = f0 - i0, t1 = f1 - i1;
    const double *g = P->popdense;
    double g00 = g[(int64_t)i0 * n1 + i1], g01 = g[(int64_t)i0 * n1 + i1 + 1];
    double g10 = g[(int64_t)(i0 + 1) * n1 + i1], g11 = g[(int64_t)(i0 + 1) * n1 + i1 + 1];
    *gx = ((1 - t1) * (g10 - g00) + t1 * (g11 - g01)) / h0;
    *gy = ((1 - t0) * (g01 - g00) + t0 * (g11 - g10)) / h1;
    return (1 - t0) * (1 - t1) * g00 + (1 - t0) * t1 * g01 + t0 * (1 - t1) * g10 + t0 * t1 * g11;
}

static double wrap_pi(double a)  /* to (-pi, pi] */
{
    double r = fmod(a, 2.0 * M_PI);
    if (r > M_PI) r -= 2.0 * M_PI;
    if (r <= -M_PI) r += 2.0 * M_PI;
    return r;
}

static double sgn(double a) { return a > 0 ? 1.0 : (a < 0 ? -1.0 : 0.0); }

typedef struct {
    double x, y, z, v, chi, F;
    int upd;       /* the aircraft was advanced at this step */
    int active;    /* flying (not violated, not landed) after the step */
} gstep;

/* The soft objective of one particle, C = sum_i (1/M) sum_m c_soft[i][m]
 * (softplus separation of reading R5, unary and control constraints hard), and
 * its gradient with respect to the controls u[N][S][3], by the reverse mode of
 * the rollout (Sec. 3.3-3.5, Sec. 7.1).  The forward pass is the rollout of
 * orc_rollout written with the identities of reading R1 (z' = z + dt hdot,
 * v' = v + dt a, chi' = chi + dt w) and the drag of reading R2 in closed form,
 * D = q CD0 + CD2 m^2 (g^2 (1 - hdot^2/v^2) + w^2 v^2) / q, q = rho v^2 S / 2.
 * Decisions (limits, landing, kinks of |.| and of the interpolation) are held
 * at their forward values.  Returns +inf (gradient 0) when any aircraft
 * violates a hard constraint in any sample. */
double orc_rollout_grad(const orc_problem *P, const orc_aircraft *A, const double *W,
                        const double *ul, int64_t l, int J, double *grad)
{
    const int N = P->N, H = P->H, S = P->S, M = P->M;
    const int64_t Pn = (int64_t)P->grid[0] * P->grid[1] * P->grid[2];
    const double dt = P->dt, sgmax = sin(P->gamma_max), tpmax = tan(P->phi_max);
    const double Sh = P->sep_h, Sv = P->sep_v, bet = P->sp_beta, mu = P->mu_sep;
    for (int n = 0; n < N * S * 3; n++) grad[n] = 0.0;
    if (P->wind_mode != 0 || P->rolling) return NAN;   /* shared wind field, fixed aircraft set */
    gstep *tr = (gstep *)malloc(sizeof(gstep) * (size_t)(H + 1) * N);
    double *gs = (double *)calloc((size_t)N * S * 3, sizeof(double));
    double total = 0.0;
    int infeasible = 0;

    for (int m = 0; m < M && !infeasible; m++) {
        const double *Wm = W + (int64_t)m * H * Pn * 2;
        double sA[64], sB[64], sC[64], sN[64], soft[64], nz[64][2];
        int dead[64], landed[64];
        /* turbulence normals of the sample (as the forward rollout draws them) */
        double *turb = (double *)malloc(sizeof(double) * (size_t)H * N * 2);
        for (int i = 0; i < N; i++) {
            gstep *g = &tr[i];
            g->x = A[i].x; g->y = A[i].y; g->z = A[i].z; g->v = A[i].v; g->chi = A[i].chi; g->F = 0.0;
            g->upd = 0; g->active = 1;
            sA[i] = sB[i] = sC[i] = sN[i] = soft[i] = 0.0;
            dead[i] = landed[i] = 0;
            for (int k = 0; k < H; k += 2) {
                uint32_t tb[4];
                orc_draw(P, (uint32_t)l, (uint32_t)i | ((uint32_t)m << 8), (uint32_t)(k >> 1), 0u, (uint32_t)J, tb);
                double a0, a1, b0, b1;
                orc_box_muller(tb[0], tb[1], &a0, &a1);
                orc_box_muller(tb[2], tb[3], &b0, &b1);
                turb[((int64_t)k * N + i) * 2] = a0;
                turb[((int64_t)k * N + i) * 2 + 1] = a1;
                if (k + 1 < H) {
                    turb[((int64_t)(k + 1) * N + i) * 2] = b0;
                    turb[((int64_t)(k + 1) * N + i) * 2 + 1] = b1;
                }
            }
            (void)nz;
        }
        /* ---------------- forward */
        for (int k = 0; k < H; k++) {
            for (int i = 0; i < N; i++) {
                const orc_aircraft *a = &A[i];
                gstep *c = &tr[(int64_t)k * N + i], *n1 = &tr[(int64_t)(k + 1) * N + i];
                *n1 = *c;
                n1->upd = 0;
                c->upd = 0;
                if (dead[i] || landed[i]) { n1->active = 0; continue; }
                const int seg = (int)(((int64_t)k * S) / H);
                const double *uu = ul + ((int64_t)i * S + seg) * 3;
                const double w = uu[0], hd = uu[1], acc = uu[2];
                const double mass = a->m - c->F;
                double sg = hd / c->v;
                int ok = fabs(sg) <= sgmax && fabs(sg) < 1.0;
                double cg = ok ? sqrt(1.0 - sg * sg) : 1.0;
                double tp = w * c->v / (G0 * cg);
                ok = ok && fabs(tp) < tpmax;
                double rho = 1.225 * pow(fmax(1.0 - 2.2558e-5 * c->z, 0.0), 4.2559);
                double q = 0.5 * rho * c->v * c->v * a->S;
                double A2 = G0 * G0 * (1.0 - sg * sg) + w * w * c->v * c->v;
                double D = q * a->CD0 + a->CD2 * mass * mass * A2 / q;
                double T = mass * (acc + G0 * sg) + D;
                ok = ok && T >= a->Tmin && T <= a->Tmax;
                if (!ok) { dead[i] = 1; n1->active = 0; continue; }
                c->upd = 1;
                double wv[2], dw[2][3];
                trilinear_grad(P, Wm + (int64_t)k * Pn * 2, c->x, c->y, c->z, wv, dw);
                const double *tn = &turb[((int64_t)k * N + i) * 2];
                n1->x = c->x + dt * (c->v * cg * cos(c->chi) + wv[0] + P->turb_sigma * tn[0]);
                n1->y = c->y + dt * (c->v * cg * sin(c->chi) + wv[1] + P->turb_sigma * tn[1]);
                n1->z = c->z + dt * hd;
                n1->v = c->v + dt * acc;
                n1->chi = c->chi + dt * w;
                n1->F = c->F + dt * a->Cf1 * (1.0 + c->v / a->Cf2) * T;
                if (!(n1->z >= P->z_min && n1->z <= P->z_max && n1->v >= P->v_min && n1->v <= P->v_max &&
                      a->m - n1->F >= a->m_empty)) { dead[i] = 1; n1->active = 0; continue; }
                double th = atan2(n1->y, n1->x);
                if (a->type == 0) {
                    double r = sqrt(n1->x * n1->x + n1->y * n1->y), ath = fabs(th);
                    double ratio = ath < 1e-3 ? 1.0 + th * th / 6.0 : ath / fmax(sin(ath), 0.25 * ath);
                    double beta = atan2(n1->z, r * ratio);
                    if (r <= P->P_runway && beta <= P->P_beta && n1->x > 0.0 && ath <= P->P_chi &&
                        angdist(n1->chi - M_PI) <= P->P_chi && n1->v <= P->P_vs) {
                        landed[i] = 1; n1->active = 0; continue;
                    }
                    sA[i] += angdist(n1->chi - M_PI - 2.0 * th);
                    sB[i] += fabs(beta - P->beta_f);
                } else {
                    sA[i] += angdist(th - a->theta_F);
                    sB[i] += fabs(a->Z - n1->z);
                    sC[i] += fabs(n1->v - a->v_D);
                }
                if (P->w_noise != 0.0) {
                    double za = n1->z / P->A_c, h = fmax(1.0 - za * za, 0.0);
                    sN[i] += h * popdense_at(P, n1->x, n1->y);
                }
                n1->active = 1;
            }
            for (int i = 0; i < N; i++) {
                const gstep *pi_ = &tr[(int64_t)(k + 1) * N + i];
                if (!pi_->active) continue;
                for (int j = i + 1; j < N; j++) {
                    const gstep *pj = &tr[(int64_t)(k + 1) * N + j];
                    if (!pj->active) continue;
                    double dx = pi_->x - pj->x, dy = pi_->y - pj->y, dz = pi_->z - pj->z;
                    double g = fmin(1.0 - sqrt(dx * dx + dy * dy) / Sh, 1.0 - fabs(dz) / Sv);
                    double pen = softplus(g, bet);
                    soft[i] += pen;
                    soft[j] += pen;
                }
            }
        }
        for (int i = 0; i < N; i++)
            if (dead[i]) infeasible = 1;
        if (infeasible) { free(turb); break; }
        /* objective and its sensitivity to the accumulated sums */
        double gA[64], gB[64], gC[64], gN[64], gF[64];
        for (int i = 0; i < N; i++) {
            const orc_aircraft *a = &A[i];
            const double Fmax = H * dt * a->Tmax * a->Cf1 * (1.0 + P->v_max / a->Cf2);
            const double FH = tr[(int64_t)H * N + i].F;
            double Jsum, dA, dB, dC = 0.0, dF;
            if (a->type == 1) {
                double d0 = fabs(a->Z - a->z), cl = P->v_max * sgmax * dt, sup = 0.0, inf = 0.0;
                for (int k = 1; k <= H; k++) {
                    sup += d0 + k * cl;
                    inf += (d0 - k * cl) > 0.0 ? d0 - k * cl : 0.0;
                }
                sup /= H;
                inf /= H;
                double Cmax = fmax(P->v_max - a->v_D, a->v_D - P->v_min);
                Jsum = P->alpha_dep[0] * (1.0 - sA[i] / H / M_PI) + P->alpha_dep[1] * (1.0 - FH / Fmax) +
                       P->alpha_dep[2] * (sup - sB[i] / H) / (sup - inf) +
                       P->alpha_dep[3] * (1.0 - sC[i] / H / Cmax);
                dA = -P->alpha_dep[0] / (H * M_PI);
                dB = -P->alpha_dep[2] / (H * (sup - inf));
                dC = -P->alpha_dep[3] / (H * Cmax);
                dF = -P->alpha_dep[1] / Fmax;
            } else {
                Jsum = P->alpha_arr[0] * (1.0 - sA[i] / H / M_PI) + P->alpha_arr[1] * (1.0 - sB[i] / H / (0.5 * M_PI)) +
                       P->alpha_arr[2] * (1.0 - FH / Fmax);
                dA = -P->alpha_arr[0] / (H * M_PI);
                dB = -P->alpha_arr[1] / (H * 0.5 * M_PI);
                dF = -P->alpha_arr[2] / Fmax;
            }
            double JT = (1.0 - P->w_noise) * Jsum + P->w_noise * (1.0 - sN[i] / H);
            double gJ = JT > 1e-30 ? -1.0 / JT : 0.0;
            total += (-log(JT > 1e-30 ? JT : 1e-30) + mu * soft[i]) / M;
            gA[i] = gJ * (1.0 - P->w_noise) * dA / M;
            gB[i] = gJ * (1.0 - P->w_noise) * dB / M;
            gC[i] = gJ * (1.0 - P->w_noise) * dC / M;
            gN[i] = gJ * (-P->w_noise / H) / M;
            gF[i] = gJ * (1.0 - P->w_noise) * dF / M;
        }
        /* ---------------- reverse */
        double bx[64], by[64], bz[64], bv[64], bc[64], bF[64];
        for (int i = 0; i < N; i++) {
            bx[i] = by[i] = bz[i] = bv[i] = bc[i] = 0.0;
            bF[i] = gF[i];
        }
        for (int k = H - 1; k >= 0; k--) {
            /* separation terms at step k+1: dC/dp_ij = 2 mu / M */
            for (int i = 0; i < N; i++) {
                const gstep *pi_ = &tr[(int64_t)(k + 1) * N + i];
                if (!pi_->active) continue;
                for (int j = i + 1; j < N; j++) {
                    const gstep *pj = &tr[(int64_t)(k + 1) * N + j];
                    if (!pj->active) continue;
                    double dx = pi_->x - pj->x, dy = pi_->y - pj->y, dz = pi_->z - pj->z;
                    double dh = sqrt(dx * dx + dy * dy);
                    double gh = 1.0 - dh / Sh, gv = 1.0 - fabs(dz) / Sv, g = fmin(gh, gv);
                    double sig = 1.0 / (1.0 + exp(-bet * g));
                    double s = 2.0 * mu / M * sig;
                    if (gh <= gv) {
                        if (dh > 0.0) {
                            double ex = dx / dh / Sh, ey = dy / dh / Sh;
                            bx[i] -= s * ex; by[i] -= s * ey;
                            bx[j] += s * ex; by[j] += s * ey;
                        }
                    } else {
                        double ez = sgn(dz) / Sv;
                        bz[i] -= s * ez;
                        bz[j] += s * ez;
                    }
                }
            }
            for (int i = 0; i < N; i++) {
                const orc_aircraft *a = &A[i];
                const gstep *c = &tr[(int64_t)k * N + i], *n1 = &tr[(int64_t)(k + 1) * N + i];
                if (!c->upd) continue;
                /* per-step terms on the step-(k+1) state (only while flying) */
                if (n1->active) {
                    double x = n1->x, y = n1->y, z = n1->z, r2 = x * x + y * y;
                    double th = atan2(y, x), dthx = -y / r2, dthy = x / r2;
                    if (a->type == 1) {
                        double s = sgn(wrap_pi(th - a->theta_F)) * gA[i];
                        bx[i] += s * dthx; by[i] += s * dthy;
                        bz[i] += gB[i] * sgn(z - a->Z);
                        bv[i] += gC[i] * sgn(n1->v - a->v_D);
                    } else {
                        double se = sgn(wrap_pi(n1->chi - M_PI - 2.0 * th)) * gA[i];
                        bc[i] += se;
                        bx[i] += -2.0 * se * dthx; by[i] += -2.0 * se * dthy;
                        double r = sqrt(r2), ath = fabs(th), ratio, dratio;
                        if (ath < 1e-3) { ratio = 1.0 + th * th / 6.0; dratio = th / 3.0; }
                        else if (sin(ath) >= 0.25 * ath) {
                            ratio = ath / sin(ath);
                            dratio = sgn(th) * (sin(ath) - ath * cos(ath)) / (sin(ath) * sin(ath));
                        } else { ratio = 4.0; dratio = 0.0; }
                        double sa = r * ratio, beta = atan2(z, sa), den = z * z + sa * sa;
                        double bb = gB[i] * sgn(beta - P->beta_f);
                        bz[i] += bb * sa / den;
                        double bsa = -bb * z / den;
                        bx[i] += bsa * ratio * x / r + bsa * r * dratio * dthx;
                        by[i] += bsa * ratio * y / r + bsa * r * dratio * dthy;
                    }
                    if (P->w_noise != 0.0) {
                        double gx, gy, pd = popdense_grad(P, x, y, &gx, &gy);
                        double za = z / P->A_c, h = 1.0 - za * za;
                        if (h > 0.0) {
                            bx[i] += gN[i] * h * gx;
                            by[i] += gN[i] * h * gy;
                            bz[i] += gN[i] * pd * (-2.0 * z / (P->A_c * P->A_c));
                        }
                    }
                }
                /* the step map k -> k+1 */
                const int seg = (int)(((int64_t)k * S) / H);
                const double *uu = ul + ((int64_t)i * S + seg) * 3;
                const double w = uu[0], hd = uu[1], acc = uu[2];
                const double v = c->v, mass = a->m - c->F, chi = c->chi;
                const double sg = hd / v, cg = sqrt(1.0 - sg * sg);
                const double dcg_dv = (hd * hd / (v * v * v)) / cg, dcg_dh = -(hd / (v * v)) / cg;
                const double base = 1.0 - 2.2558e-5 * c->z;
                const double rho = 1.225 * pow(base, 4.2559);
                const double q = 0.5 * rho * v * v * a->S;
                const double dq_dz = q * (4.2559 * -2.2558e-5 / base), dq_dv = 2.0 * q / v;
                const double A2 = G0 * G0 * (1.0 - sg * sg) + w * w * v * v;
                const double dA2_dv = 2.0 * G0 * G0 * hd * hd / (v * v * v) + 2.0 * w * w * v;
                const double dA2_dh = -2.0 * G0 * G0 * hd / (v * v), dA2_dw = 2.0 * w * v * v;
                const double K2 = a->CD2 * mass * mass;
                const double D = q * a->CD0 + K2 * A2 / q;
                const double T = mass * (acc + G0 * sg) + D;
                const double dD_dv = a->CD0 * dq_dv + K2 * (dA2_dv / q - A2 * dq_dv / (q * q));
                const double dD_dz = a->CD0 * dq_dz - K2 * A2 * dq_dz / (q * q);
                const double dD_dm = 2.0 * a->CD2 * mass * A2 / q;
                const double dT_dv = -mass * G0 * hd / (v * v) + dD_dv;
                const double dT_dz = dD_dz;
                const double dT_dm = acc + G0 * sg + dD_dm;
                const double dT_dh = mass * G0 / v + K2 * dA2_dh / q;
                const double dT_dw = K2 * dA2_dw / q;
                const double dT_da = mass;
                const double eta = a->Cf1 * (1.0 + v / a->Cf2), deta_dv = a->Cf1 / a->Cf2;
                double wv[2], dw[2][3];
                trilinear_grad(P, Wm + (int64_t)k * Pn * 2, c->x, c->y, c->z, wv, dw);
                const double X = bx[i], Y = by[i], Z = bz[i], V = bv[i], CH = bc[i], FF = bF[i];
                double nbx = X + dt * (X * dw[0][0] + Y * dw[1][0]);
                double nby = Y + dt * (X * dw[0][1] + Y * dw[1][1]);
                double nbz = Z + dt * (X * dw[0][2] + Y * dw[1][2]) + FF * dt * eta * dT_dz;
                double nbv = V + dt * cos(chi) * (cg + v * dcg_dv) * X + dt * sin(chi) * (cg + v * dcg_dv) * Y +
                             FF * dt * (deta_dv * T + eta * dT_dv);
                double nbc = CH + dt * (-v * cg * sin(chi)) * X + dt * (v * cg * cos(chi)) * Y;
                double nbF = FF * (1.0 - dt * eta * dT_dm);
                double *gu = gs + ((int64_t)i * S + seg) * 3;
                gu[0] += dt * CH + FF * dt * eta * dT_dw;
                gu[1] += dt * Z + dt * v * dcg_dh * (cos(chi) * X + sin(chi) * Y) + FF * dt * eta * dT_dh;
                gu[2] += dt * V + FF * dt * eta * dT_da;
                bx[i] = nbx; by[i] = nby; bz[i] = nbz; bv[i] = nbv; bc[i] = nbc; bF[i] = nbF;
            }
        }
        for (int n = 0; n < N * S * 3; n++) {
            grad[n] += gs[n];
            gs[n] = 0.0;
        }
        free(turb);
    }
    free(tr);
    free(gs);
    if (infeasible) {
        for (int n = 0; n < N * S * 3; n++) grad[n] = 0.0;
        return INFINITY;
    }
    return total;
}

/* ------------------------------------------------------------------ */
/* Metropolis-Hastings moves of whole particles (extension of the        */
/* perturbation of Algorithm 1).  Target pi(u) ~ exp(-kappa C(u)),       */
/* C = sum_i cbar_soft[i]; controls scaled by the move step sigma of     */
/* their kind (z = u / sigma).                                           */
/* ------------------------------------------------------------------ */

/* standard normal number e of aircraft i of particle l for the proposal:
 * random stream 5, draw e/4, words (0,1) -> first pair, (2,3) -> second */
static double mh_normal(const orc_problem *P, int64_t l, int i, int e, int J)
{
    uint32_t r[4];
    orc_draw(P, (uint32_t)l, (uint32_t)i, (uint32_t)(e / 4), 5u, (uint32_t)J, r);
    double a, b;
    if (e % 4 < 2) orc_box_muller(r[0], r[1], &a, &b);
    else orc_box_muller(r[2], r[3], &a, &b);
    return (e % 2 == 0) ? a : b;
}

void orc_mh_propose(const orc_problem *P, const double *u, const double *grad, int64_t L, int J,
                    double kappa, double eps, int kind, double *u_prop, uint8_t *inbox)
{
    const int N = P->N, S = P->S;
    for (int64_t l = 0; l < L; l++) {
        int ok = 1;
        for (int i = 0; i < N; i++)
            for (int e = 0; e < 3 * S; e++) {
                const int c = e % 3;
                const int64_t o = (l * N + i) * 3 * S + e;
                const double sg = P->move_sigma[c];
                /* Langevin: z' = z - (eps^2/2) kappa grad_z C + eps xi, grad_z = sigma grad_u */
                double z = u[o] / sg;
                if (kind == 2) z -= 0.5 * eps * eps * kappa * sg * grad[o];
                z += eps * mh_normal(P, l, i, e, J);
                u_prop[o] = sg * z;
                if (!(u_prop[o] >= P->ctrl_lo[c] && u_prop[o] <= P->ctrl_hi[c])) ok = 0;
            }
        inbox[l] = (uint8_t)ok;
    }
}

void orc_mh_accept(const orc_problem *P, const double *u, const double *up, const double *cbar,
                   const double *cbarp, const double *g, const double *gp, const uint8_t *inbox,
                   int64_t L, int J, double kappa, double eps, int kind, double *u_out,
                   uint8_t *accepted, double *log_alpha)
{
    const int N = P->N, S = P->S, nel = N * 3 * S;
    for (int64_t l = 0; l < L; l++) {
        double C = 0.0, Cp = 0.0;
        int inf = 0, infp = 0;
        for (int i = 0; i < N; i++) {
            if (isinf(cbar[(int64_t)i * L + l])) inf = 1; else C += cbar[(int64_t)i * L + l];
            if (isinf(cbarp[(int64_t)i * L + l])) infp = 1; else Cp += cbarp[(int64_t)i * L + l];
        }
        /* log of the Metropolis-Hastings ratio pi(u') q(u|u') / (pi(u) q(u'|u)) */
        double la = -kappa * (Cp - C);
        if (kind == 2) {
            /* Gaussian proposal densities in z: q(z'|z) ~ exp(-|z' - m(z)|^2 / (2 eps^2)),
             * m(z) = z - (eps^2/2) kappa grad_z C(z) */
            const double d = 0.5 * eps * eps * kappa;
            double fw = 0.0, bw = 0.0;
            for (int n = 0; n < nel; n++) {
                const int64_t o = l * nel + n;
                const double sg = P->move_sigma[n % 3];
                const double z = u[o] / sg, zp = up[o] / sg;
                const double f = zp - (z - d * sg * g[o]);      /* z' - m(z)  */
                const double b = z - (zp - d * sg * gp[o]);     /* z  - m(z') */
                fw += f * f;
                bw += b * b;
            }
            la += -(bw - fw) / (2.0 * eps * eps);
        }
        int acc;
        if (!inbox[l] || infp) acc = 0;
        else if (inf) acc = 1;
        else {
            uint32_t r[4];
            orc_draw(P, (uint32_t)l, 0u, 0u, 6u, (uint32_t)J, r);
            acc = log(orc_uniform23(r[0])) < la;
        }
        if (log_alpha) log_alpha[l] = (!inbox[l] || infp) ? -INFINITY : (inf ? INFINITY : la);
        if (accepted) accepted[l] = (uint8_t)acc;
        for (int n = 0; n < nel; n++) u_out[l * nel + n] = acc ? up[l * nel + n] : u[l * nel + n];
    }
}

/* ------------------------------------------------------------------ */
/* the plant of the MPC loop (Sec. 2, Fig. 1)                            */
/* ------------------------------------------------------------------ */

/* One step dt of the true system under the first-segment controls u0[N][3]:
 * Eq. (hor) with the climb angle kept below 90 degrees (|sin gamma| <= 0.999)
 * and the thrust held within [Tmin, Tmax]; disturbance = wind field W0[P][2]
 * (sample 0, step 0) plus white turbulence from random stream 7. */
static int plant_active(const orc_problem *P, const orc_aircraft *A, int i)
{
    return !P->rolling ||
           (!((P->finished >> i) & 1u) && (int64_t)A[i].t_enter <= (int64_t)P->mpc_step);
}

/* Rolling window (reading R22): the finished mask after a plant step that
 * produced the states x[N][6] -- the previous mask plus every active arrival
 * inside the landing sector of Eq. (TO_init) (range, glide angle, bearing cone
 * with x > 0, heading, speed). */
uint32_t orc_plant_finished(const orc_problem *P, const orc_aircraft *A, const double *x)
{
    uint32_t f = P->finished;
    if (!P->rolling) return f;
    for (int i = 0; i < P->N; i++) {
        if (A[i].type != 0 || !plant_active(P, A, i)) continue;
        const double *s = x + 6 * i;
        const double r = sqrt(s[0] * s[0] + s[1] * s[1]);
        const double th = atan2(s[1], s[0]), ath = fabs(th);
        const double ratio = ath < 1e-3 ? 1.0 + th * th / 6.0 : ath / fmax(sin(ath), 0.25 * ath);
        const double beta = atan2(s[2], r * ratio);
        const double hdg = angdist(s[4] - M_PI);
        if (r <= P->P_runway && beta <= P->P_beta && s[0] > 0.0 && ath <= P->P_chi &&
            hdg <= P->P_chi && s[3] <= P->P_vs)
            f |= 1u << i;
    }
    return f;
}

/* Rolling window: an aircraft that has not entered or has finished keeps its
 * state. */
void orc_plant_step(const orc_problem *P, const orc_aircraft *A, const double *x_in,
                    const double *W0, const double *u0, double *x_out)
{
    for (int i = 0; i < P->N; i++) {
        const orc_aircraft *a = &A[i];
        const double *s = x_in + 6 * i;
        if (!plant_active(P, A, i)) {
            for (int c = 0; c < 6; c++) x_out[6 * i + c] = s[c];
            continue;
        }
        double x = s[0], y = s[1], z = s[2], v = s[3], chi = s[4], m = s[5];
        double w = u0[3 * i], hd = u0[3 * i + 1], acc = u0[3 * i + 2];
        double sg = hd / v;
        if (sg > 0.999) sg = 0.999;
        if (sg < -0.999) sg = -0.999;
        double cg = sqrt(1.0 - sg * sg);
        double tp = w * v / (G0 * cg);
        double cphi = 1.0 / sqrt(1.0 + tp * tp), sphi = tp * cphi;
        double base = 1.0 - 2.2558e-5 * z;
        double rho = 1.225 * pow(base > 0.0 ? base : 0.0, 4.2559);
        double qS = 0.5 * rho * v * v * a->S;
        double CL = m * G0 * cg / (qS * cphi);
        double D = qS * (a->CD0 + a->CD2 * CL * CL);
        double T = m * (acc + G0 * sg) + D;
        if (T < a->Tmin) T = a->Tmin;
        if (T > a->Tmax) T = a->Tmax;
        double Lift = CL * qS, eta = a->Cf1 * (1.0 + v / a->Cf2);
        double wx, wy;
        trilinear(P, W0, x, y, z, &wx, &wy);
        uint32_t tb[4];
        orc_draw(P, 0u, (uint32_t)i, 0u, 7u, 0u, tb);
        double n0, n1;
        orc_box_muller(tb[0], tb[1], &n0, &n1);
        wx += P->turb_sigma * n0;
        wy += P->turb_sigma * n1;
        double *o = x_out + 6 * i;
        o[0] = x + P->dt * (v * cos(chi) * cg) + wx * P->dt;
        o[1] = y + P->dt * (v * sin(chi) * cg) + wy * P->dt;
        o[2] = z + P->dt * (v * sg);
        o[3] = v + P->dt * ((T - D) / m - G0 * sg);
        o[4] = chi + P->dt * (Lift * sphi / (m * v));
        o[5] = m - P->dt * (eta * T);
    }
}

/* ------------------------------------------------------------------ */
/* weights (Sec. 3.6 with the schedule of Sec. 5.1)                      */
/* ------------------------------------------------------------------ */

int orc_kappa(int J)
{
    return (int)floor(3.0 + 5.0 * exp(0.05 * J));
}

void orc_lse(const double *cbar, int nseg, int L, double kappa, double *wtilde, double *lmax,
             double *wsum)
{
    for (int s = 0; s < nseg; s++) {
        const double *c = cbar + (int64_t)s * L;
        double mx = -INFINITY;
        for (int j = 0; j < L; j++) {
            if (isfinite(c[j])) {
                double l = -kappa * c[j];
                if (l > mx) mx = l;
            }
        }
        double sum = 0.0;
        for (int j = 0; j < L; j++) {
            double w = 0.0;
            if (isfinite(c[j]) && mx > -INFINITY) w = exp(-kappa * c[j] - mx);
            wtilde[(int64_t)s * L + j] = w;
            sum += w;
        }
        if (lmax) lmax[s] = mx;
        if (wsum) wsum[s] = sum;
    }
}

/* ------------------------------------------------------------------ */
/* systematic resampling on a fixed-point CDF (Sec. 3.7)                  */
/* ------------------------------------------------------------------ */

uint32_t orc_resample_uniform(const orc_problem *P, int seg, int J)
{
    uint32_t w[4];
    orc_draw(P, 0u, (uint32_t)seg, 0u, 2u, (uint32_t)J, w);
    return w[0];
}

/* Systematic resampling of Lout ancestors from Lin weighted particles (reading
 * R12 with L_out thresholds t_l = floor((l 2^32 + r) Q / (Lout 2^32)),
 * l < Lout; reading R21).  A segment with Q = 0 gets the evenly spread
 * ancestors floor(l Lin / Lout) (the identity when Lout = Lin). */
int orc_resample_to(const double *wtilde, int nseg, int Lin, int Lout, const uint32_t *r, int32_t *anc)
{
    int ndeg = 0;
    uint64_t *S = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(Lin > 0 ? Lin : 1));
    for (int s = 0; s < nseg; s++) {
        const double *w = wtilde + (int64_t)s * Lin;
        uint64_t acc = 0;
        for (int j = 0; j < Lin; j++) {
            uint64_t q = 0;
            if (w[j] >= 1.0) q = 1ull << 40;
            else if (w[j] > 0.0) q = (uint64_t)(w[j] * 1099511627776.0);
            acc += q;
            S[j] = acc;
        }
        int32_t *a = anc + (int64_t)s * Lout;
        if (acc == 0) {
            for (int l = 0; l < Lout; l++) a[l] = (int32_t)((int64_t)l * Lin / Lout);
            ndeg++;
            continue;
        }
        const unsigned __int128 den = (unsigned __int128)(uint64_t)Lout << 32;
        int j = 0;
        for (int l = 0; l < Lout; l++) {
            unsigned __int128 num = (unsigned __int128)((((uint64_t)l) << 32) + r[s]) * acc;
            uint64_t t = (uint64_t)(num / den);
            while (S[j] <= t) j++;
            a[l] = j;
        }
    }
    free(S);
    return ndeg;
}

int orc_resample(const double *wtilde, int nseg, int L, const uint32_t *r, int32_t *anc)
{
    return orc_resample_to(wtilde, nseg, L, L, r, anc);
}

/* ------------------------------------------------------------------ */
/* perturbation (Algorithm 1) and initialisation (Sec. 3.2)              */
/* ------------------------------------------------------------------ */

/* L = the number of children (anc[N][L]); ancestors index the parents in u. */
void orc_move(const orc_problem *P, const double *u, const int32_t *anc, int L, int J,
              double *u_out)
{
    const int N = P->N, nc = 3 * P->S, nq = (nc + 3) / 4;
    for (int l = 0; l < L; l++) {
        for (int i = 0; i < N; i++) {
            const int32_t a = anc[(int64_t)i * L + l];
            const double *src = u + ((int64_t)a * N + i) * nc;
            double *dst = u_out + ((int64_t)l * N + i) * nc;
            for (int q = 0; q < nq; q++) {
                uint32_t w[4];
                orc_draw(P, (uint32_t)l, (uint32_t)i, (uint32_t)q, 1u, (uint32_t)J, w);
                double z[4];
                orc_box_muller(w[0], w[1], &z[0], &z[1]);
                orc_box_muller(w[2], w[3], &z[2], &z[3]);
                for (int t = 0; t < 4; t++) {
                    int n = 4 * q + t;
                    if (n >= nc) break;
                    int c = n % 3;
                    double v = src[n] + P->move_sigma[c] * z[t];
                    if (v < P->ctrl_lo[c]) v = P->ctrl_lo[c];
                    if (v > P->ctrl_hi[c]) v = P->ctrl_hi[c];
                    dst[n] = v;
                }
            }
        }
    }
}

void orc_init_controls(const orc_problem *P, int L, double *u)
{
    const int N = P->N, nc = 3 * P->S, nq = (nc + 3) / 4;
    for (int l = 0; l < L; l++)
        for (int i = 0; i < N; i++) {
            double *dst = u + ((int64_t)l * N + i) * nc;
            for (int q = 0; q < nq; q++) {
                uint32_t w[4];
                orc_draw(P, (uint32_t)l, (uint32_t)i, (uint32_t)q, 4u, 0u, w);
                for (int t = 0; t < 4; t++) {
                    int n = 4 * q + t;
                    if (n >= nc) break;
                    int c = n % 3;
                    dst[n] = P->ctrl_lo[c] + (P->ctrl_hi[c] - P->ctrl_lo[c]) * orc_uniform23(w[t]);
                }
            }
        }
}

/* ------------------------------------------------------------------ */
/* final selection (Sec. 3.8)                                            */
/* ------------------------------------------------------------------ */

int64_t orc_select(const double *cbar, int N, int L, double *best_sum, int *n_inf)
{
    int64_t best = -1;
    int bn = N + 1;
    double bs = INFINITY;
    for (int l = 0; l < L; l++) {
        int ni = 0;
        double sum = 0.0;
        for (int i = 0; i < N; i++) {
            double c = cbar[(int64_t)i * L + l];
            if (!isfinite(c)) ni++;
            else sum += c;
        }
        if (ni < bn || (ni == bn && sum < bs)) {
            best = l;
            bn = ni;
            bs = sum;
        }
    }
    if (best_sum) *best_sum = (bn == 0) ? bs : INFINITY;
    if (n_inf) *n_inf = bn;
    return best;
}
