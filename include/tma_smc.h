/*
 * tma_smc.h -- C-ABI of the GB300 (sm_103a) implementation of the data-parallel
 * hot path of Sequential Monte Carlo optimisation inside Model Predictive
 * Control for multi-aircraft Terminal Manoeuvring Area trajectories
 * (Eele & Maciejowski, CUED/F-INFENG/TR.693, 2015).
 *
 * Conventions shared by every entry point
 *   - Units are SI (m, s, kg, N, rad); headings use the mathematical
 *     convention (0 = +x, counter-clockwise positive).
 *   - "d_" pointers are device pointers on the current CUDA device, "h_"
 *     pointers are host pointers.  All device pointers are caller-owned unless
 *     stated otherwise; the library never frees them.
 *   - Every launch goes on the caller's stream (`tma_stream_t` is a
 *     cudaStream_t; NULL is the legacy default stream) and is stream-ordered;
 *     nothing synchronises unless the entry point writes a host output.
 *   - The ABI never aborts, throws or prints; it returns a tma_status.  Invalid
 *     sizes or NULL required pointers give TMA_ERR_INVALID_ARG before any
 *     launch; a failed CUDA call gives TMA_ERR_CUDA (the CUDA error string is
 *     available from tma_last_error_string()).
 *   - Layouts are row-major C arrays:
 *       controls  u[L][N][S][3] float32, per segment (turn rate w [rad/s],
 *                 climb rate hdot [m/s], speed change a [m/s^2]), piecewise
 *                 constant over S equal segments of the horizon;
 *       costs     cbar[N][L] float32 (aircraft-major, one segment per aircraft);
 *       weights   wtilde[N][L] float64;  ancestors anc[N][L] int32;
 *       wind      W[M][H][P][2] float32, P = nx*ny*nz grid nodes, node index
 *                 (ix*ny + iy)*nz + iz, components (x, y).
 */
#ifndef TMA_SMC_H
#define TMA_SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tma_stream_t;
typedef struct tma_solver tma_solver;

typedef enum {
    TMA_OK = 0,
    TMA_ERR_INVALID_ARG = 1,
    TMA_ERR_OOM = 2,
    TMA_ERR_CUDA = 3,
    TMA_ERR_BOUNDS = 4,
    TMA_ERR_TIMEOUT = 5,
    TMA_WARN_DEGENERATE = 6,   /* a weight segment was all zero; identity ancestors were used */
    TMA_ERR_UNSUPPORTED = 7
} tma_status;

/* Limits of the library. */
#define TMA_MAX_AIRCRAFT 32          /* N: one warp lane per aircraft */
#define TMA_MAX_PARTICLES (1 << 22)  /* L: keeps the fixed-point CDF products in 128 bits */
#define TMA_MAX_GRID_Z 16
#define TMA_MAX_GRAD_HORIZON 320     /* H of tma_rollout_grad: checkpoints kept per thread */

/* Move kinds of tma_set_move. */
/* Bits of the sticky device error word (tma_get_error, tma_batch_results). */
#define TMA_DEVERR_DEGENERATE 1u  /* some weight segment was all zero: identity ancestors used */
#define TMA_DEVERR_INFEASIBLE 2u  /* the chosen particle had an infeasible aircraft */
#define TMA_DEVERR_BOUNDS 4u      /* a perturbation read an ancestor index out of range */

#define TMA_MOVE_PAPER 0   /* Gaussian random walk, clipped, no accept step (Algorithm 1) */
#define TMA_MOVE_RWMH 1    /* random walk with a Metropolis-Hastings accept step */
#define TMA_MOVE_MALA 2    /* Langevin proposal (gradient of the soft cost) with accept step */

/* Scenario: the optimal-control problem of Sec. 2 and Sec. 3 (all host values). */
typedef struct {
    int32_t N;                /* aircraft (Sec. 2), 1..TMA_MAX_AIRCRAFT */
    int32_t H;                /* prediction horizon in steps (Sec. 2) */
    int32_t S;                /* control segments over the horizon */
    int32_t L;                /* particles (Sec. 3.2), 1..TMA_MAX_PARTICLES */
    int32_t M;                /* wind samples per particle (Sec. 3.3, inner loop) */
    int32_t J_max;            /* SMC iterations (Algorithm 1) */
    double dt;                /* step length delta t [s] (Eq. (hor)) */
    uint64_t seed;            /* key of every random stream */
    uint32_t scenario_id;     /* mixed into the key: seed + scenario_id * 0x9E3779B97F4A7C15 */
    uint32_t mpc_step;        /* receding-horizon step (Sec. 2), part of every counter */
    double box_lo[3], box_hi[3];  /* wind grid box (x, y, z) */
    int32_t grid[3];          /* wind grid nodes nx, ny, nz (each >= 2, nz <= 16) */
    double wind_sigma;        /* std of the forecast error [m/s] (Eq. (cov)) */
    double turb_sigma;        /* std of white turbulence per step [m/s] */
    double lam_t;             /* time correlation rate [1/s]: a = exp(-dt*lam_t) */
    double beta_xy, gam_z;    /* horizontal / vertical correlation rates [1/m] */
    double sep_h, sep_v;      /* separation minima 2P_r, 2P_h (Eq. (avoidance)) */
    int32_t sep_mode;         /* 0 hard, 1 softplus, 2 both (weights use hard) */
    double sp_beta, mu_sep;   /* softplus sharpness and weight */
    double z_min, z_max, gamma_max, phi_max, v_min, v_max;  /* envelope (Sec. 3.4) */
    double ctrl_lo[3], ctrl_hi[3];  /* control box (initial uniform draw, clipping) */
    double move_sigma[3];     /* std of the Gaussian perturbation (Algorithm 1) */
    double alpha_dep[4];      /* departure weights: bearing, fuel, altitude, speed (Table coeff) */
    double alpha_arr[3];      /* arrival weights: flow heading, glide path, fuel (Table coeff) */
    double w_noise, A_c;      /* noise-cost weight and altitude cut-off (Sec. 7.1) */
    int32_t pop_n[2];         /* population grid nodes (0 = no noise map) */
    double pop_lo[2], pop_hi[2];
    const double *popdense;   /* host [pop_n[0]][pop_n[1]]; copied by tma_create */
    double P_runway, P_beta, P_chi, P_vs, beta_f;  /* landing sector (Eq. (TO_init)), glide angle */
    int32_t wind_mode;        /* 0: one wind field per sample, shared by all particles (grid as
                                 above); 1: a field per (particle, sample) on the 2x2x2 grid of the
                                 box corners (grid must be 2,2,2), drawn inside the rollout from
                                 random stream 9 -- the paper's scheme (Sec. 3.9.1, Sec. 6).
                                 tma_rollout_grad and the accepted moves need mode 0. */
    int32_t sample_mode;      /* 0: every iteration rolls out all M wind samples and weights by
                                 l = -kappa_J * cbar (kappa_J = SampleSchedule(J), Sec. 5.1);
                                 1: the inner loop of Algorithm 1 -- iteration J rolls out samples
                                 0 .. M_J-1, M_J = min(SampleSchedule(J), M), and the weight is the
                                 product of J_T over those draws (Sec. 3.6): l = -M_J * cbar.
                                 tma_rollout_cost, tma_rollout_grad and the moves of iteration J
                                 use M_J samples in mode 1. */
    const int64_t *L_sched;   /* NULL: every iteration evaluates L particles.  Otherwise host
                                 [J_max], 1 <= L_sched[J] <= L: iteration J evaluates L_sched[J]
                                 particles and the resampling after it draws L_sched[J+1]
                                 ancestors (tma_resample_to) -- the varying particle count the
                                 paper proposes (Sec. 9).  Copied by tma_create; single solvers
                                 only (tma_batch_create rejects it). */
    int32_t rolling;          /* 1: rolling window (the paper's rolling-window section).  At MPC
                                 step t aircraft i flies the horizon steps k >= max(0, t_enter - t)
                                 from its entry state, its objective is the mean of its per-step
                                 terms over those steps, and an aircraft that enters after the
                                 horizon, or has finished, is out of the problem (cost 0, not
                                 simulated, not in separation checks).  The plant moves only
                                 active aircraft and marks an arrival finished once it is in the
                                 landing sector of Eq. (TO_init).  tma_rollout_grad and the
                                 Langevin move need rolling = 0. */
} tma_problem;

typedef struct {
    double x, y, z, v, chi, m;   /* X_0 of Sec. 3.3: position, airspeed, heading, mass */
} tma_state;

typedef struct {
    int32_t type;             /* 0 arrival, 1 departure */
    int32_t t_enter;          /* rolling window (tma_problem.rolling = 1): the MPC step at which
                                 the aircraft enters the problem; ignored otherwise */
    tma_state x0;             /* initial state (the entry state of a late entrant) */
    double theta_F, Z, v_D;   /* departure targets: bearing, altitude, airspeed (Sec. 3.5) */
    double m_empty;           /* minimum mass m_Aircraft (Sec. 3.4) */
    double S, CD0, CD2;       /* wing area and drag polar */
    double Cf1, Cf2;          /* fuel flow eta = Cf1 (1 + v/Cf2) (Sec. 6.2, Eq. (blah)) */
    double Tmin, Tmax;        /* thrust limits (Sec. 3.4) */
} tma_aircraft;

const char *tma_status_str(tma_status s);
/* Text of the last CUDA error seen by this thread's last failing call ("" if none). */
const char *tma_last_error_string(void);
/* Number of CUDA kernels this library has launched in this process. */
uint64_t tma_launch_count(void);

/* ---------------------------------------------------------------- solver */

/* Create a solver for one scenario on the current device.  Copies `prob`,
 * `aircraft[prob->N]` and the population map; factorises the wind covariance
 * of Eq. (cov) (host FP64 Cholesky of the Kronecker factors, Sec. 3.9.1) and
 * allocates the device buffers it owns (wind field, controls, costs, weights,
 * ancestors, scratch).  Errors: TMA_ERR_INVALID_ARG (sizes, limits above),
 * TMA_ERR_OOM, TMA_ERR_CUDA.  On error *out is NULL. */
tma_status tma_create(const tma_problem *prob, const tma_aircraft *aircraft, tma_solver **out);
void tma_destroy(tma_solver *s);

/* Set the measured states X_0 (host, N entries; NULL keeps the current ones)
 * and the receding-horizon step (Sec. 2, Fig. 1).  Stream-ordered copy. */
tma_status tma_set_state(tma_solver *s, const tma_state *h_x0, uint32_t mpc_step,
                         tma_stream_t stream);

/* Generate the solver's wind field for its current mpc_step (Sec. 3.9.1):
 * W(0) = Qhat v(0), W(k+1) = a W(k) + Q v(k+1) with Qhat = sigma (L_xy kron L_z),
 * Q = sqrt(1 - a^2) Qhat.  If d_W is not NULL the field is also copied there
 * (float32 [M][H][P][2]).  Uses solver-owned scratch. */
tma_status tma_wind_field(tma_solver *s, float *d_W, tma_stream_t stream);

/* Random stream of the wind normals of this solver: 3 (default, the samples of
 * the optimisation) or 8 (held-out samples, for evaluating a chosen control
 * sequence on winds the optimisation did not see).  The next wind generation
 * uses it; the current field is dropped. */
tma_status tma_set_wind_stream(tma_solver *s, uint32_t stream);

/* Rollout and costs (Algorithm 1 inner loop; Sec. 3.3-3.6, Sec. 7.1): for every
 * particle l < L of d_u (u[L][N][S][3]), every wind sample m < M of the
 * solver's current field and every aircraft, simulate H steps of Eq. (hor)
 * under wind + turbulence, check constraints (Sec. 3.4), landing (Eq. (TO_init))
 * and separation (Eq. (avoidance)), and score -ln J_T.  Outputs the sample
 * means d_cbar[N][L] (+inf when the aircraft violated a constraint in any
 * sample), and, if d_cbar_soft is not NULL, the softplus-separation variant.
 * J is the SMC iteration (keys the turbulence stream).  Particle l keys its
 * streams with index l.  L <= the solver's L.  Uses solver-owned scratch. */
tma_status tma_rollout_cost(tma_solver *s, const float *d_u, int64_t L, int32_t J, float *d_cbar,
                            float *d_cbar_soft, tma_stream_t stream);

/* Per-sample costs of the last tma_rollout_cost call: d_out[M][N][L] float32
 * (wind sample, aircraft, particle), L <= the L of that call. */
tma_status tma_sample_costs(tma_solver *s, float *d_out, int64_t L, int soft, tma_stream_t stream);

/* Number of simulated (not frozen) aircraft-steps in the last tma_rollout_cost
 * call, or summed over all rollouts of the last tma_solve; syncs. */
tma_status tma_live_steps(tma_solver *s, uint64_t *h_live, tma_stream_t stream);

/* Perturbation (Algorithm 1): d_u_out[l][i] = clip(d_u[d_anc[i][l]][i] + sigma xi)
 * with xi from random stream 1 of iteration J.  d_u_out must not alias d_u.
 * Ancestors must lie in [0, L); an out-of-range ancestor is replaced by l. */
tma_status tma_move(tma_solver *s, const float *d_u, const int32_t *d_anc, int64_t L, int32_t J,
                    float *d_u_out, tma_stream_t stream);

/* The perturbation with another number of parents (varying particle count,
 * Sec. 9): L children d_u_out[L][N][S][3] from the L_in parents d_u[L_in],
 * d_anc[N][L] in [0, L_in) (tma_resample_to's output).  An out-of-range
 * ancestor sets TMA_DEVERR_BOUNDS in the solver's sticky device error word
 * (tma_get_error then returns TMA_ERR_BOUNDS) and the child takes the parent
 * min(l, L_in - 1), so every output is defined; nothing traps.  L, L_in <= the
 * solver's L; tma_move is this call with L_in = L. */
tma_status tma_move_to(tma_solver *s, const float *d_u, int64_t L_in, const int32_t *d_anc, int64_t L,
                       int32_t J, float *d_u_out, tma_stream_t stream);

/* Uniform initial controls (Sec. 3.2) from random stream 4: d_u[L][N][S][3]. */
tma_status tma_init_controls(tma_solver *s, float *d_u, int64_t L, tma_stream_t stream);

/* One SMC optimisation (Algorithm 1) from the solver's current state: wind
 * field, uniform initialisation, J_max rollouts with annealed weighting, FP64
 * normalisation, systematic resampling and perturbation between them, and the
 * final selection (Sec. 3.8).  Writes the chosen controls d_best_u[N][S][3]
 * (device, caller-owned, may be NULL) and, if h_best_cost is not NULL, syncs
 * the stream and writes the chosen particle's cost sum (host).  Returns
 * TMA_WARN_DEGENERATE when some weight segment was all zero. */
tma_status tma_solve(tma_solver *s, float *d_best_u, double *h_best_cost, tma_stream_t stream);

/* The same solve through host buffers: copies h_x0[N] in, solves, copies the
 * chosen controls h_best_u[N][S][3] and their cost out; syncs the stream. */
tma_status tma_solve_host(tma_solver *s, const tma_state *h_x0, uint32_t mpc_step, float *h_best_u,
                          double *h_best_cost, tma_stream_t stream);

/* The particle set of the last tma_solve after its final iteration (the set
 * the selection of Sec. 3.8 chose from): d_u_out[L][N][S][3] (device,
 * caller-owned), L <= the solver's L (the first L particles). */
tma_status tma_get_particles(tma_solver *s, float *d_u_out, int64_t L, tma_stream_t stream);

/* Index of the particle chosen by the last tma_solve (host); syncs. */
tma_status tma_best_index(tma_solver *s, int64_t *h_best, tma_stream_t stream);

/* Launch configuration of the rollout kernel chosen by the autotuner that
 * tma_create runs (Sec. 4.4 sweeps thread/block layouts by hand; here every
 * valid launch-bound variant -- block-size cap and minimum resident blocks --
 * is timed on the solver's own workload and the fastest kept; the choice is
 * cached per device, aircraft count, problem kind and workload size class).
 * *n_timed is 0 when the choice came from the cache; h_variants/h_ms (up to 24
 * entries, may be NULL) receive the
 * candidates and their mean time per rollout in ms. */
tma_status tma_get_tuning(tma_solver *s, int32_t *variant, int32_t *n_timed, int32_t *h_variants,
                          float *h_ms);

/* Force the rollout kernel's launch variant for this solver, e.g. to sweep
 * the layouts as Sec. 4.4 does.  0-7: one wind sample per thread, block-size
 * cap x minimum resident blocks = 256x4, 256x3, 512x2, 512x1, 1024x1, 256x2,
 * 384x2, 768x1.  8-12: two wind samples per thread (m and m + ceil(M/2); the
 * wind-independent part of each step -- limits, drag, thrust, fuel, altitude,
 * airspeed, heading -- computed once for both), 256x3, 256x2, 384x2, 512x1,
 * 768x1; only for the shared wind field (wind mode 0) without the rolling
 * window and M >= 2.  13-15: the one-sample kernel on tiles of 16 particles (a
 * warp holds two aircraft; block 16 N threads), 768x1, 384x2, 512x2; 16-17: on
 * tiles of 8 particles (four aircraft per warp; block 8 N threads), 512x2,
 * 384x2; both for the shared wind field only and for N a multiple of 2 or 4
 * (full warps).  Every variant returns the same bits.  A variant whose cap is
 * below the block or that does not apply to the problem returns
 * TMA_ERR_INVALID_ARG. */
tma_status tma_set_tuning(tma_solver *s, int32_t variant);

/* The same record for the kernel of tma_rollout_grad, tuned on its first use
 * (tma_rollout_grad or tma_set_move with TMA_MOVE_MALA); *variant is -1 before. */
tma_status tma_get_grad_tuning(tma_solver *s, int32_t *variant, int32_t *n_timed,
                               int32_t *h_variants, float *h_ms);

/* Per-stage device time of the solver's launches (CUDA events recorded on the
 * launching stream around each stage when profiling is on).  Stages:
 * 0 wind generation, 1 initial controls, 2 rollout, 3 sample means, 4 LSE,
 * 5 resampling, 6 move, 7 selection, 8 gradient of the soft cost,
 * 9 Metropolis-Hastings proposal and accept.  tma_profile_read synchronises on
 * the recorded events, adds their durations to the totals and, if reset != 0,
 * clears the totals after copying them out. */
#define TMA_N_STAGES 10
typedef struct {
    double ms[TMA_N_STAGES];
    uint64_t launches[TMA_N_STAGES];
} tma_profile;
tma_status tma_profile_enable(tma_solver *s, int on);
tma_status tma_profile_read(tma_solver *s, tma_profile *h_out, int reset);

/* ------------------------------------------- gradient and accepted moves */

/* Gradient of the soft cost (an extension: the paper's perturbation uses no
 * gradient).  For particles l < L of d_u[L][N][S][3] (device) and the
 * solver's current wind field, iteration J (keys the turbulence as in
 * tma_rollout_cost): the objective C_l = sum_i (1/M) sum_m c_soft[i][m], the
 * per-sample cost -ln J_T of Sec. 3.5-3.6 plus the softplus separation penalty
 * mu sum sp_beta(min(1 - d_h/S_h, 1 - |dz|/S_v)) of Eq. (avoidance) in soft
 * form, with the unary and control limits of Sec. 3.4 kept hard.  Writes
 * d_cost[L] (+inf when any aircraft violates a hard limit in any sample),
 * d_grad[L][N][S][3] = dC_l/du_l (zero for infeasible particles) and, if
 * d_cbar_soft is not NULL, the per-aircraft means [N][L] (the same values as
 * tma_rollout_cost's soft means).  Reverse mode over the discrete dynamics of
 * Eq. (hor): limit, landing and interpolation-cell decisions are held at their
 * forward values; states are recomputed from checkpoints taken every 10
 * steps.  Valid for any sep_mode.  H must be <= TMA_MAX_GRAD_HORIZON
 * (TMA_ERR_UNSUPPORTED otherwise).  Uses solver-owned scratch, allocated on the
 * first call (not inside stream capture). */
tma_status tma_rollout_grad(tma_solver *s, const float *d_u, int64_t L, int32_t J, float *d_cost,
                            float *d_grad, float *d_cbar_soft, tma_stream_t stream);

/* Chooses the move between the iterations of tma_solve (Algorithm 1's
 * perturbation step).  TMA_MOVE_PAPER (default): the paper's clipped Gaussian
 * random walk.  TMA_MOVE_RWMH / TMA_MOVE_MALA (extensions, sep_mode != 0):
 * after resampling, one Metropolis-Hastings step per particle with target
 * exp(-kappa_J C(u)) (C as in tma_rollout_grad) and step eps (in units of the
 * problem's move_sigma per control kind), starting at eps0 > 0 and adapted
 * after every iteration: times 0.8 when fewer than half of the particles
 * accepted, times 1.25 when more than 70 %.  See tma_mh_propose / tma_mh_accept
 * for the proposal and the accept rule.  Allocates the move's scratch. */
tma_status tma_set_move(tma_solver *s, int32_t kind, double eps0);

/* Proposal of one Metropolis-Hastings move for particles l < L (device
 * buffers [L][N][S][3]): with sigma = the problem's move_sigma per control kind
 * and xi standard normal from random stream 5 of iteration J,
 *   TMA_MOVE_RWMH   u' = u + eps sigma xi
 *   TMA_MOVE_MALA   u' = u - (eps^2/2) kappa sigma^2 d_grad + eps sigma xi.
 * d_inbox[l] = 1 when every control of u'_l lies in the control box (else the
 * proposal will be rejected).  d_grad may be NULL for TMA_MOVE_RWMH. */
tma_status tma_mh_propose(tma_solver *s, const float *d_u, const float *d_grad, int64_t L,
                          int32_t J, double kappa, double eps, int32_t kind, float *d_u_prop,
                          uint8_t *d_inbox, tma_stream_t stream);

/* Accept step of that move: with C = sum_i d_cbar[i][l] and C' = sum_i
 * d_cbar_prop[i][l] (per-aircraft soft means [N][L]),
 *   log alpha = -kappa (C' - C) - (|z - z' + d g'|^2 - |z' - z + d g|^2) / (2 eps^2)
 * for TMA_MOVE_MALA (z = u / sigma, g = sigma d_grad, g' = sigma d_grad_prop,
 * d = (eps^2/2) kappa), -kappa (C' - C) for TMA_MOVE_RWMH; the particle moves
 * when ln U < log alpha, U the 23-bit uniform of random stream 6 (FP64).  A
 * proposal outside the box or with C' = +inf is rejected; from C = +inf any
 * finite in-box proposal is accepted.  Writes d_u_out (may alias d_u) and,
 * if not NULL, d_accepted[L] (0/1).  Gradients may be NULL for RWMH. */
tma_status tma_mh_accept(tma_solver *s, const float *d_u, const float *d_u_prop,
                         const float *d_cbar, const float *d_cbar_prop, const float *d_grad,
                         const float *d_grad_prop, const uint8_t *d_inbox, int64_t L, int32_t J,
                         double kappa, double eps, int32_t kind, float *d_u_out,
                         uint8_t *d_accepted, tma_stream_t stream);

/* Per-iteration record of the last tma_solve with an accepted move: for
 * J < n, h_accepts[J] = particles that moved after iteration J and h_eps[J] =
 * the step used there (either pointer may be NULL); n <= J_max - 1; syncs. */
tma_status tma_mh_stats(tma_solver *s, uint32_t *h_accepts, double *h_eps, int32_t n,
                        tma_stream_t stream);

/* ------------------------------------------------------------ MPC plant */

/* The plant of Fig. 1 (Sec. 2): every aircraft flies the first-segment controls
 * d_u[N][S][3] (device; only segment 0 is used) for one step dt from the
 * solver's current state, under the wind field of sample 0 at step 0 plus white
 * turbulence from random stream 7, thrust held within [Tmin, Tmax].  The new
 * state replaces the solver's state on the device and the MPC step advances by
 * one (the next solve draws new random numbers).  Syncs the stream. */
tma_status tma_plant_step(tma_solver *s, const float *d_u, tma_stream_t stream);
/* Receding-horizon control of Fig. 1 (Sec. 2): n_steps times, one tma_solve
 * from the current state followed by tma_plant_step with the chosen controls.
 * h_traj[n_steps][N] (host) receives the state after each plant step and, if
 * not NULL, h_costs[n_steps] the chosen particle's cost sum of each solve.
 * Syncs once per step.  Returns TMA_WARN_DEGENERATE when some solve had an all-
 * zero weight segment. */
tma_status tma_mpc_run(tma_solver *s, int32_t n_steps, tma_state *h_traj, double *h_costs,
                       tma_stream_t stream);

/* Sticky device status of the solves and stage calls since the last call, in
 * *h_err: TMA_DEVERR_DEGENERATE (bit 0) some weight segment was all zero
 * (identity ancestors were used), TMA_DEVERR_INFEASIBLE (bit 1) the chosen
 * particle had an infeasible aircraft (no particle satisfied every limit),
 * TMA_DEVERR_BOUNDS (bit 2) a perturbation met an ancestor index out of range.
 * Clears the word; syncs.  Returns TMA_ERR_BOUNDS when bit 2 was set (the word
 * is written all the same), else TMA_OK. */
tma_status tma_get_error(tma_solver *s, uint32_t *h_err, tma_stream_t stream);

/* Rolling window: set the mask of aircraft that have left the problem (bit i =
 * aircraft i; bits at or above N must be zero); tma_set_state with states
 * clears it, the plant step sets bits of arrivals that landed.  Syncs. */
tma_status tma_set_finished(tma_solver *s, uint32_t mask, tma_stream_t stream);

/* Rolling window: per aircraft h_status[N] (may be NULL) at the current MPC
 * step -- 0 not yet entered (t_enter > MPC step), 1 active, 2 finished -- and
 * the finished mask (may be NULL).  Without a rolling window every aircraft is
 * 1.  Syncs. */
tma_status tma_get_status(tma_solver *s, int32_t *h_status, uint32_t *h_finished, tma_stream_t stream);

/* The solver's current state h_x[N] (host) and MPC step; syncs. */
tma_status tma_get_state(tma_solver *s, tma_state *h_x, uint32_t *h_mpc, tma_stream_t stream);

/* --------------------------------------------------------------- batches */

/* Many independent TMA scenarios solved together (receding-horizon MPC per
 * scenario, Sec. 2; Algorithm 1 each).  Scenarios may differ in aircraft
 * (N_s = 1..32, states, targets, coefficients), weights, control box and
 * seeds; they must share L, M, H, S, J_max, dt, sep_mode, sample_mode and the
 * wind model (wind_mode, grid, box, rates, sigma); otherwise
 * TMA_ERR_INVALID_ARG.  Weight segments are (scenario, aircraft) pairs,
 * at most 65535 in total.  aircraft[s] points to probs[s].N records.
 * The rollout of all scenarios is one persistent launch over a work queue. */
typedef struct tma_batch tma_batch;
tma_status tma_batch_create(const tma_problem *probs, const tma_aircraft *const *aircraft,
                            int32_t n_scen, tma_batch **out);
void tma_batch_destroy(tma_batch *b);
/* States h_x0 (sum of N_s entries, scenario-major; NULL keeps the device
 * states) and MPC steps h_mpc[n_scen] (NULL keeps them); syncs. */
tma_status tma_batch_set_state(tma_batch *b, const tma_state *h_x0, const uint32_t *h_mpc,
                               tma_stream_t stream);
/* One SMC solve of every scenario from its current state (device only). */
tma_status tma_batch_solve(tma_batch *b, tma_stream_t stream);
/* n_steps receding-horizon steps: each solves every scenario, then the plant
 * advances every scenario by one step with its chosen first control (as
 * tma_plant_step).  With use_graph != 0 the whole sequence is captured once
 * into a CUDA graph (re-captured when n_steps changes) and launched; the
 * results equal those without the graph. */
tma_status tma_batch_mpc(tma_batch *b, int32_t n_steps, int32_t use_graph, tma_stream_t stream);
/* The batch's rollout dispatch (the paper's layout sweep of Sec. 4.4 done by
 * measurement): at creation every scenario's launch variant of the
 * single-scenario rollout kernel is tuned (cached like the solvers'), and two
 * forms are timed on one rollout of the whole batch -- 0: one persistent
 * launch over a work queue of every scenario's tiles; 1: one launch of the
 * single-scenario kernel per scenario, spread over four streams forked from and
 * joined to the caller's (also inside a graph capture) -- and the
 * faster is kept.  get: the form in use and the two timings (ms; any pointer
 * may be NULL).  set: forces a form (0 or 1, else TMA_ERR_INVALID_ARG); a
 * captured MPC loop of the other form is discarded.  Both forms compute the
 * same bits. */
tma_status tma_batch_get_dispatch(tma_batch *b, int32_t *dispatch, float *ms_persistent, float *ms_per_scenario);
tma_status tma_batch_set_dispatch(tma_batch *b, int32_t dispatch);
/* The batched rollout alone (the rollout inside tma_batch_solve, in the
 * batch's dispatch form; Sec. 3.3-3.6 for every scenario), on given controls:
 * generates every
 * scenario's wind field for its current MPC step, then rolls out d_u at
 * iteration J (the first SampleSchedule(J) samples in sample mode 1, else all
 * M) and writes the per-sample costs.  Packed layouts, scenario after scenario
 * (offsets by the aircraft counts N_s' of the scenarios s' before s):
 *   d_u            [L][N_s][S][3] at float offset L * 3S * sum N_s' (device, in)
 *   d_cost_ms      [M][N_s][L] at float offset M * L * sum N_s' (device, out):
 *                  -ln J_T, +inf when infeasible or separated too little
 *   d_cost_ms_soft the softplus form in the same layout (device, out; may be
 *                  NULL; ignored when sep_mode = 0)
 * All caller-owned; stream-ordered, no synchronisation.  Rows of samples not
 * rolled out (sample mode 1) are left as they were. */
tma_status tma_batch_rollout_cost(tma_batch *b, const float *d_u, int32_t J, float *d_cost_ms,
                                  float *d_cost_ms_soft, tma_stream_t stream);
/* Results of the last solve: chosen controls h_best_u (sum N_s x S x 3,
 * scenario-major), cost sums h_best_cost[n_scen], particle indices
 * h_best[n_scen]; current states h_x (sum N_s) and MPC steps h_mpc[n_scen].
 * Any pointer may be NULL; syncs.  Returns TMA_ERR_BOUNDS (the outputs are
 * written all the same) when a perturbation since the last call met an
 * ancestor index out of range (the batch's sticky error word, cleared here). */
tma_status tma_batch_results(tma_batch *b, float *h_best_u, double *h_best_cost, int64_t *h_best,
                             tma_state *h_x, uint32_t *h_mpc, tma_stream_t stream);
/* Per-scenario solve latency of the last solve in ms: device clock from the
 * start of the solve to the end of that scenario's selection; syncs. */
tma_status tma_batch_latency(tma_batch *b, double *h_ms, tma_stream_t stream);
/* Simulated aircraft-steps of the last batched solve (all rollouts); syncs. */
tma_status tma_batch_live_steps(tma_batch *b, uint64_t *h_live, tma_stream_t stream);

/* ------------------------------------------------------ stateless stages */

/* Annealed log-weights and their FP64 normalisation per segment (Sec. 3.6,
 * schedule of Sec. 5.1): l_j = -kappa * (double)cbar_j, lmax = max over finite
 * l_j, d_wtilde[s][j] = exp(l_j - lmax) = exp(kappa (cmin - cbar_j)) (0 for
 * +inf cost; relative error below 1e-15 against the exact value, evaluated in
 * integer fixed point), d_lmax[s], d_wsum[s] = sum_j wtilde.  A segment with
 * no finite cost gets lmax = -inf, wtilde = 0.  d_lmax / d_wsum may be NULL.
 * Scratch: d_work of tma_lse_workspace() bytes. */
size_t tma_lse_workspace(int32_t nseg, int64_t L);
tma_status tma_lse(const float *d_cbar, int32_t nseg, int64_t L, double kappa, double *d_wtilde,
                   double *d_lmax, double *d_wsum, void *d_work, size_t work_bytes,
                   tma_stream_t stream);

/* Systematic resampling per segment (Sec. 3.7) on a fixed-point CDF:
 * q_j = floor(wtilde_j 2^40), S = inclusive prefix sum, Q = S_{L-1},
 * t_l = floor((l 2^32 + r) Q / (L 2^32)), d_anc[s][l] = min{j : S_j > t_l}.
 * r is word 0 of Philox4x32-10 under key seed + scenario_id*0x9E3779B97F4A7C15
 * and counter (0, s, 2<<24, J | mpc_step<<16).  A segment with Q = 0 gets
 * identity ancestors and the call returns TMA_WARN_DEGENERATE.  wtilde must
 * lie in [0, 1] (values above 1 count as 1, NaN and negatives as 0).
 * Scratch: d_work of tma_resample_workspace() bytes. */
size_t tma_resample_workspace(int32_t nseg, int64_t L);
tma_status tma_resample(const double *d_wtilde, int32_t nseg, int64_t L, uint64_t seed,
                        uint32_t scenario_id, uint32_t J, uint32_t mpc_step, int32_t *d_anc,
                        void *d_work, size_t work_bytes, tma_stream_t stream);

/* Systematic resampling to another particle count (the varying particle count
 * the paper proposes as a speed-up, Sec. 9): L_out ancestors per segment from
 * the L weighted particles, t_l = floor((l 2^32 + r) Q / (L_out 2^32)) for
 * l < L_out, d_anc[s][l] = min{j : S_j > t_l} in [0, L); d_anc is
 * [nseg][L_out].  A segment with Q = 0 gets ancestors floor(l L / L_out) and
 * the call returns TMA_WARN_DEGENERATE.  L and L_out are both zero or both in
 * [1, TMA_MAX_PARTICLES].  Uniform r, weights and workspace as tma_resample
 * (workspace sized by L); tma_resample is this call with L_out = L. */
tma_status tma_resample_to(const double *d_wtilde, int32_t nseg, int64_t L, int64_t L_out,
                           uint64_t seed, uint32_t scenario_id, uint32_t J, uint32_t mpc_step,
                           int32_t *d_anc, void *d_work, size_t work_bytes, tma_stream_t stream);

/* The annealed weights and the resampling of one SMC iteration in one
 * stream-ordered call (Sec. 3.6-3.7; the stages between two rollouts of
 * Algorithm 1): d_wtilde as tma_lse, then d_anc as tma_resample with L_out
 * ancestors, the resampling's chunk sums of q formed by the pass that writes
 * wtilde (one read of wtilde less than the two calls).  Neither synchronises:
 * when d_degenerate (device int32, caller-owned, may be NULL) is given, bit 0
 * is set there if a segment had Q = 0 (the caller zeroes it).  Scratch: d_work
 * of tma_lse_resample_workspace(nseg, L) bytes; other arguments and errors as
 * tma_lse and tma_resample_to. */
size_t tma_lse_resample_workspace(int32_t nseg, int64_t L);
tma_status tma_lse_resample(const float *d_cbar, int32_t nseg, int64_t L, int64_t L_out, double kappa,
                            uint64_t seed, uint32_t scenario_id, uint32_t J, uint32_t mpc_step,
                            double *d_wtilde, int32_t *d_anc, uint32_t *d_degenerate, void *d_work,
                            size_t work_bytes, tma_stream_t stream);

/* Systematic resampling exactly as tma_resample, for callers that cannot
 * allocate device memory: a control loop that must never block in (or fail
 * inside) the CUDA allocator once it is running, or a host application whose
 * device memory is entirely owned by another allocator and which cannot hand
 * out a workspace.  The paper has no counterpart; this is a deployment
 * variant.
 *   - Scratch: a fixed array inside this library (about 512 KB; every GPU that
 *     loads the library holds it until the process exits).  The call itself
 *     allocates nothing and needs no workspace.
 *   - Limit: nseg * ceil(L / 2048) <= 65536 (e.g. 32 segments of 4,194,304
 *     particles); larger sizes return TMA_ERR_INVALID_ARG.  Other arguments
 *     and errors as tma_resample; synchronises the stream to read the
 *     degenerate-segment status.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     After cudaDeviceReset the next call on that device sees a new context
 *     and looks the address up again (so does the first call after the
 *     context was created, when an earlier call ran before it existed).
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls that overlap on the GPU (different streams or threads at the same
 *     time) race and must be serialised by the caller. */
tma_status tma_resample_noalloc(const double *d_wtilde, int32_t nseg, int64_t L, uint64_t seed,
                                uint32_t scenario_id, uint32_t J, uint32_t mpc_step, int32_t *d_anc,
                                tma_stream_t stream);

/* Final selection (Sec. 3.8): over particles l < L, the fewest aircraft with
 * infinite cost, then the smallest sum_i (double)cbar[i][l] summed in order
 * i = 0..N-1, ties to the lowest l.  Writes d_best (int64), d_best_sum (double;
 * +inf when the chosen particle has an infeasible aircraft), d_ninf (int32).
 * Scratch: d_work of tma_select_workspace() bytes. */
size_t tma_select_workspace(int64_t L);
tma_status tma_select(const float *d_cbar, int32_t N, int64_t L, int64_t *d_best, double *d_best_sum,
                      int32_t *d_ninf, void *d_work, size_t work_bytes, tma_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TMA_SMC_H */
