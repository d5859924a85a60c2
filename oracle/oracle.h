/*
 * oracle.h -- plain FP64 CPU oracle of the SMC-MPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; the product never
 * calls it.
 *
 * Every function restates the method of Eele & Maciejowski, "Sequential Monte
 * Carlo Optimisation for Air Traffic Management" (CUED/F-INFENG/TR.693, 2015):
 *   dynamics            Sec. 3.3, Eq. (hor)
 *   landing sector      Sec. 3.3, Eq. (TO_init)
 *   unary constraints   Sec. 3.4
 *   separation          Sec. 3.4, Eq. (avoidance)
 *   objectives          Sec. 3.5 (departure J^D, arrival J^A, Eq. (flow))
 *   weight scaling      Sec. 3.6
 *   resampling/perturb  Sec. 3.7, Algorithm 1
 *   final selection     Sec. 3.8
 *   wind model          Sec. 3.9.1, Eq. (cov)
 *   noise cost          Sec. 7.1
 * The readings taken where the paper is silent or garbled are listed in the
 * header comment of oracle.c.
 */
#ifndef TMA_ORACLE_H
#define TMA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int N, H, S, L, M, J_max;
    double dt;
    uint64_t seed;
    uint32_t scenario_id, mpc_step;
    double box_lo[3], box_hi[3];
    int grid[3];
    double wind_sigma, turb_sigma, lam_t, beta_xy, gam_z;
    double sep_h, sep_v;
    int sep_mode;                 /* 0 hard, 1 soft, 2 both */
    double sp_beta, mu_sep;
    double z_min, z_max, gamma_max, phi_max, v_min, v_max;
    double ctrl_lo[3], ctrl_hi[3], move_sigma[3];
    double alpha_dep[4], alpha_arr[3], w_noise, A_c;
    int pop_n[2];
    double pop_lo[2], pop_hi[2];
    const double *popdense;       /* [pop_n[0]][pop_n[1]] or NULL */
    double P_runway, P_beta, P_chi, P_vs, beta_f;
    uint32_t wind_stream;         /* random stream of the wind normals: 3, or 8 for held-out
                                     evaluation samples (0 reads as 3) */
    int wind_mode;                /* 0 one field per wind sample shared by all particles;
                                     1 a field per (particle, sample) on the 2x2x2 grid of
                                     the box corners (the paper's scheme) */
    const double *wind_chol;      /* mode 1: lower Cholesky factor of R_hat, 8 x 8 row-major */
    int rolling;                  /* 1: rolling window (aircraft enter at t_enter, finished
                                     aircraft have left; reading R22) */
    uint32_t finished;            /* rolling window: bit i = aircraft i has left the problem */
} orc_problem;

typedef struct {
    int32_t type;                 /* 0 arrival, 1 departure */
    int32_t t_enter;              /* rolling window: MPC step at which the aircraft enters */
    double x, y, z, v, chi, m;
    double theta_F, Z, v_D;
    double m_empty, S, CD0, CD2, Cf1, Cf2, Tmin, Tmax;
} orc_aircraft;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 23-bit uniform in (0,1) from one 32-bit word, exact in FP32. */
double orc_uniform23(uint32_t x);
/* Box-Muller pair from two 32-bit words. */
void orc_box_muller(uint32_t xa, uint32_t xb, double *z0, double *z1);
/* One draw of the counter layout used by every random stream. */
void orc_draw(const orc_problem *P, uint32_t c0, uint32_t c1, uint32_t q, uint32_t stream,
              uint32_t J, uint32_t out[4]);

/* Standard normals v_X, v_Y of the wind model for samples m0..m0+mc-1:
 * out[mc][H][P][2]. */
void orc_wind_normals(const orc_problem *P, int m0, int mc, double *out);

/* Mode 1 wind of particle l, sample m: out[H][8][2] = (W_X, W_Y) at the eight
 * box-corner nodes, W(k) = Qhat B(k), B(0) = v(0), B(k) = a B(k-1) + sqrt(1-a^2) v(k)
 * (the recursion of Sec. 3.9.1), v from random stream 9. */
void orc_particle_wind(const orc_problem *P, int64_t l, int m, double *out);

/* Rollout of particles `pidx` (global indices) under wind samples m0..m0+mc-1.
 * W holds those samples: W[mc][H][P][2].  u[Lsub][N][S][3].
 * Outputs per (particle, sample, aircraft): cost_hard/cost_soft [Lsub][mc][N];
 * margin [Lsub][mc][N] (smallest relative distance of any threshold decision
 * of that aircraft to its threshold); smargin [Lsub][mc] (same, restricted to
 * decisions that change the set of flying aircraft).  live counts simulated
 * aircraft-steps.  Any output pointer may be NULL.  N <= 256. */
void orc_rollout(const orc_problem *P, const orc_aircraft *A, const double *W, int m0, int mc,
                 const double *u, const int64_t *pidx, int Lsub, int J, int nthreads,
                 double *cost_hard, double *cost_soft, double *margin, double *smargin,
                 int64_t *live);

/* One (particle l, sample m) rollout with its trajectory:
 * traj[H+1][N][8] = (x, y, z, v, chi, m, F, flags) after each step, flags =
 * violated + 2*landed + 4*separation-violated.  Wm = W[H][P][2] of sample m. */
void orc_trajectory(const orc_problem *P, const orc_aircraft *A, const double *Wm, int m,
                    const double *ul, int64_t l, int J, double *traj, double *cost_hard,
                    double *cost_soft);

/* Soft objective C = sum_i mean_m c_soft[i][m] of particle l (controls
 * ul[N][S][3], all M wind samples W[M][H][P][2], iteration J) and its
 * gradient grad[N][S][3] by reverse mode; +inf (gradient 0) if infeasible.
 * N <= 64. */
double orc_rollout_grad(const orc_problem *P, const orc_aircraft *A, const double *W,
                        const double *ul, int64_t l, int J, double *grad);

/* Metropolis-Hastings move of whole particles u[L][N][S][3] (kind 1 random
 * walk, 2 Langevin): proposal from random stream 5 of iteration J, in-box
 * flag per particle; accept with the 23-bit uniform of stream 6.  cbar and
 * cbarp are per-aircraft soft means [N][L]; g, gp gradients [L][N][S][3]
 * (kind 2 only).  log_alpha (may be NULL) receives the log acceptance ratio
 * (-inf for a rejected-by-rule proposal, +inf for a forced accept). */
void orc_mh_propose(const orc_problem *P, const double *u, const double *grad, int64_t L, int J,
                    double kappa, double eps, int kind, double *u_prop, uint8_t *inbox);
void orc_mh_accept(const orc_problem *P, const double *u, const double *up, const double *cbar,
                   const double *cbarp, const double *g, const double *gp, const uint8_t *inbox,
                   int64_t L, int J, double kappa, double eps, int kind, double *u_out,
                   uint8_t *accepted, double *log_alpha);

/* One step of the true system (plant of the MPC loop): x_in/x_out[N][6]
 * (x, y, z, v, chi, m), W0 = wind field of sample 0 at step 0, u0[N][3]. */
uint32_t orc_plant_finished(const orc_problem *P, const orc_aircraft *A, const double *x);
void orc_plant_step(const orc_problem *P, const orc_aircraft *A, const double *x_in,
                    const double *W0, const double *u0, double *x_out);

/* Annealed log-weights and their segment-wise normalisation. */
int orc_kappa(int J);
void orc_lse(const double *cbar, int nseg, int L, double kappa, double *wtilde, double *lmax,
             double *wsum);
/* Systematic resampling on a fixed-point CDF (bit-exact definition). */
uint32_t orc_resample_uniform(const orc_problem *P, int seg, int J);
int orc_resample(const double *wtilde, int nseg, int L, const uint32_t *r, int32_t *anc);
int orc_resample_to(const double *wtilde, int nseg, int Lin, int Lout, const uint32_t *r, int32_t *anc);
/* Perturbation of the resampled controls. */
void orc_move(const orc_problem *P, const double *u, const int32_t *anc, int L, int J,
              double *u_out);
void orc_init_controls(const orc_problem *P, int L, double *u);
/* Final selection: index of the best particle; *best_sum = its cost sum. */
int64_t orc_select(const double *cbar, int N, int L, double *best_sum, int *n_inf);

#ifdef __cplusplus
}
#endif
#endif
