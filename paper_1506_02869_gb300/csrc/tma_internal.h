// Internal declarations of the CUDA path: kernel parameter blocks, the solver
// object and the launchers implemented by each .cu file.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tma_smc.h"

namespace tma {

constexpr int kMaxN = TMA_MAX_AIRCRAFT;
constexpr int kTileParticles = 32;   // particles per rollout tile (one warp per aircraft)
constexpr int kPairVariantBase = 8;  // first rollout variant index of the two-sample kernel
constexpr int kHalfVariantBase = 13; // first rollout variant index of the 16-particle (half) tile
constexpr int kQuarterVariantBase = 16; // first rollout variant index of the 8-particle tile
constexpr int kMaxRolloutVariants = 24;

// Per-aircraft constants in FP32 (derived on the host in FP64).
struct AircraftC {
    int type;              // 0 arrival, 1 departure
    float halfS, CD0, CD2;
    float Cf1, invCf2, Tmin, Tmax, m_empty;
    float thF, Z, vD;
    float invFmax;         // 1 / (H dt Tmax eta(vmax))
    float invCmax;         // departure speed-term normalisation
    int t_enter;           // rolling window: MPC step at which the aircraft enters
};

// Problem constants passed by value to the rollout kernels.
struct ProblemC {
    int N, H, S, M, G;     // G = lanes per (particle, sample) group = next_pow2(N)
    int seg_q, seg_r;      // H = seg_q S + seg_r: the control segments' lengths step by these
    int P;                 // wind grid nodes
    int grid[3];
    float dt;
    float box_lo[3], box_hi[3], inv_h[3];
    float turb_sigma;
    float sgmax, tpmax;    // sin(gamma_max), tan(phi_max)
    float climb_step;      // vmax sin(gamma_max) dt: largest altitude change per step
    float Sh2, Sh_inv, Sv, Sv_inv;
    int sep_mode;
    float sp_beta, sp_inv_beta, mu_sep;
    // beyond these (d_h^2 above sp_far_h2 or |dz| above sp_far_v) the margin g
    // lies below -30 / beta and the softplus penalty below e^-30 / beta: it is
    // taken as 0 without evaluating it
    float sp_far_h2, sp_far_v;
    float z_min, z_max, v_min, v_max;
    float a_dep[4], a_arr[3];
    float w_noise, Ac_inv;
    int pop_n[2];
    float pop_lo[2], pop_hi[2], pop_inv_h[2];
    // device, or nullptr: the density's cells [pop_n0 - 1][pop_n1 - 1], each
    // holding its four corner values (g[a][b], g[a][b+1], g[a+1][b], g[a+1][b+1])
    // so that one 16-byte load gives a bilinear lookup
    const float4 *popcell;
    float P_runway, P_beta, P_chi, P_vs, beta_f;
    int rolling;           // 1: rolling window (t_enter, finished aircraft)
    int wind_mode;         // 1: a wind field per (particle, sample) on the box corners
    float wind_a, wind_b;  // AR(1) coefficients a, sqrt(1 - a^2) of that field
    float wchol[36];       // its Qhat: lower Cholesky factor of R_hat (8 x 8, packed rows)
    uint32_t key0, key1;   // Philox key (seed + scenario_id * golden)
    uint32_t rk[20];       // its ten round keys (k0, k1 of round r at 2r, 2r + 1)
    AircraftC ac[kMaxN];
};

// Per-solve dynamic state in device memory (updated between graph replays).
struct DynState {
    float x0[kMaxN][6];
    uint32_t mpc_step;
    uint32_t finished;     // rolling window: bit i = aircraft i has left the problem
};

// Parameters of the wind-field generation kernels.
struct WindC {
    int M, H, nxy, nz, ncol, ldb;
    uint32_t stream;       // random stream of the normals: 3, or 8 for held-out samples
    float a, b, sigma;
    float Lz[TMA_MAX_GRID_Z * TMA_MAX_GRID_Z];
    uint32_t key0, key1;
};

// One scenario of a batch: offsets into the packed batch buffers.
struct BatchScen {
    long long u_off;      // floats: controls u_s[L][N][S][3]
    long long seg_off;    // first segment (aircraft) of the scenario
    long long w_off;      // float4s: packed wind field [M][H][P]
    long long items;      // its tiles: M * ceil(L / 32) (wind sample, 32 particles)
    int N, T;             // aircraft; tile slots per CTA
    float ctrl_lo[3], ctrl_hi[3], move_sigma[3];
    uint32_t key0, key1;
};

// Parameters of the Metropolis-Hastings move kernels (mala.cu).
struct MhParams {
    int N, S;
    int langevin;          // 1: Langevin proposal and its proposal-density ratio
    float sigma[3], lo[3], hi[3];
    uint32_t key0, key1;
};

// Per-segment key of the resampling uniform (batched form).
struct SegKey {
    uint32_t key0, key1, c1;
    int scen;
};

// ------------------------------------------------------------------ launchers
// Each returns cudaSuccess or the launch error.

cudaError_t launch_wind_normals_ar(const WindC &w, const DynState *dyn, float *Btmp,
                                   cudaStream_t st);
cudaError_t launch_wind_gemm(const WindC &w, const float *Lxy, int lda, const float *Btmp,
                             float *W, cudaStream_t st);

cudaError_t launch_rollout(const ProblemC &P, const DynState *dyn, const float *u, const float *W,
                           int64_t L, int J, float *cost_ms, float *cost_ms_soft,
                           unsigned long long *live, cudaStream_t st, int variant);
// Launch-bound variants of the rollout kernel valid for the problem (indices
// into the variant table: 0-7 the one-sample kernel, kPairVariantBase + v the
// two-sample kernel of rollout_pair.cu, kHalfVariantBase + v and
// kQuarterVariantBase + v the one-sample kernel on 16- and 8-particle tiles);
// returns their number (at least 1, at most kMaxRolloutVariants).
int rollout_variants(const ProblemC &P, int *out);
// The two-sample kernel (shared wind field, no rolling window, M >= 2): its
// variants valid for the problem (0-based) and its launcher.
int rollout_pair_variants(const ProblemC &P, int *out);
cudaError_t launch_rollout_pair(const ProblemC &P, const DynState *dyn, const float *u, const float *W,
                                int64_t L, int J, float *cost_ms, float *cost_ms_soft,
                                unsigned long long *live, cudaStream_t st, int variant);
cudaError_t launch_sample_mean(const float *cost_ms, int64_t L, int M, int N, float *cbar,
                               cudaStream_t st);

// cq: when given, the LSE pass also writes the resampling's chunk sums of
// q = floor(wtilde 2^40) there (resample_partials of the resampling's
// workspace), and launch_resample is then called with sums_ready.
cudaError_t launch_lse(const float *cbar, int nseg, int64_t L, double kappa, double *wtilde,
                       double *lmax, double *wsum, void *work, cudaStream_t st,
                       unsigned long long *cq = nullptr);
size_t lse_workspace(int nseg, int64_t L);
cudaError_t launch_resample(const double *wtilde, int nseg, int64_t L, int64_t Lout, uint32_t key0,
                            uint32_t key1, uint32_t J, const uint32_t *d_mpc, uint32_t mpc_host,
                            int32_t *anc, void *work, unsigned int *d_flags, cudaStream_t st,
                            const SegKey *seg_keys = nullptr, const DynState *dyns = nullptr,
                            bool sums_ready = false);
size_t resample_workspace(int nseg, int64_t L);
// The chunk sums' place in a resampling workspace.
unsigned long long *resample_partials(void *work);

cudaError_t launch_move(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                        const float ctrl_hi[3], const float sigma[3], const float *u,
                        const int32_t *anc, int64_t L, int64_t Lin, int J, float *u_out,
                        cudaStream_t st, unsigned int *err = nullptr);
cudaError_t launch_init_controls(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                                 const float ctrl_hi[3], float *u, int64_t L, cudaStream_t st);

cudaError_t launch_select(const float *cbar, int N, int64_t L, int64_t *best, double *best_sum,
                          int *ninf, void *work, cudaStream_t st);
size_t select_workspace(int64_t L);
cudaError_t launch_gather_best(const float *u, const int64_t *best, int nctl_per_particle,
                               float *best_u, cudaStream_t st, const unsigned int *flags = nullptr,
                               const int *ninf = nullptr, unsigned int *err = nullptr);

// gradient of the soft cost (adjoint.cu): per-sample costs cost_ms[M][N][L],
// partial gradients gpart[nchunk][L][N][S][3] over nchunk ranges of samples
// (cost == nullptr: the main kernel only, for timing); variant indexes the
// launch-bound table (rollout_grad_variants lists those valid for N)
cudaError_t launch_rollout_grad(const ProblemC &P, const DynState *dyn, const float *u,
                                const float *W, int64_t L, int J, int nchunk, float *cost_ms,
                                float *gpart, float *cost, float *grad, float *cbar,
                                cudaStream_t st, int variant);
cudaError_t rollout_grad_occupancy(int N, int variant, int *blocks_per_sm);
int rollout_grad_variants(int N, int *out);

// Metropolis-Hastings moves (mala.cu)
cudaError_t launch_mh_propose(const MhParams &h, const DynState *dyn, const float *u,
                              const float *grad, int64_t L, int J, float kappa, const double *d_eps,
                              float *u_prop, uint8_t *inbox, cudaStream_t st);
cudaError_t launch_mh_accept(const MhParams &h, const DynState *dyn, const float *u, const float *up,
                             const float *cbar, const float *cbarp, const float *g, const float *gp,
                             const uint8_t *inbox, int64_t L, int J, float kappa,
                             const double *d_eps, float *u_out, float *cbar_out, uint8_t *accepted,
                             unsigned int *n_accept, cudaStream_t st);
cudaError_t launch_mh_adapt(double *eps, unsigned int *n_accept, unsigned int *history,
                            double *eps_history, int J, int64_t L, cudaStream_t st);

// batched MPC (batch.cu)
size_t batch_rollout_smem();
int batch_rollout_grid();
// claimed: one tile counter per scenario (zeroed by the launcher)
cudaError_t launch_batch_rollout(const ProblemC *probs, const BatchScen *scen, int n_scen,
                                 const DynState *dyns, const float *u, const float *W, long long L,
                                 int J, int Mj, float *cost_ms, float *cost_ms_soft,
                                 unsigned long long *live, unsigned long long *claimed, int grid,
                                 int wind_mode, cudaStream_t st);
cudaError_t launch_batch_sample_mean(const float *cost_ms, const BatchScen *scen,
                                     const int *seg_scen, long long nseg, long long L, int M,
                                     int Mj, float *cbar, cudaStream_t st);
cudaError_t launch_batch_move(const BatchScen *scen, const int *seg_scen, const DynState *dyns,
                              long long nseg, long long L, int S, const float *u,
                              const int32_t *anc, int J, float *u_out, cudaStream_t st,
                              unsigned int *err = nullptr);
cudaError_t launch_batch_init(const BatchScen *scen, const int *seg_scen, const DynState *dyns,
                              long long nseg, long long L, int S, float *u, cudaStream_t st);
cudaError_t launch_batch_wind_normals(const WindC &w, int s0, int M_scen, const BatchScen *scen,
                                      const DynState *dyns, float *Btmp, cudaStream_t st);
cudaError_t launch_batch_select(const BatchScen *scen, int n_scen, const float *cbar, long long L,
                                int S, const float *u, long long *best, double *best_sum, int *ninf,
                                float *best_u, unsigned long long *t_end, cudaStream_t st);
cudaError_t launch_stamp_start(unsigned long long *t0, cudaStream_t st);
cudaError_t launch_plant_step(const ProblemC *probs, const BatchScen *scen, const int *seg_scen,
                              long long nseg, int n_scen, DynState *dyns, const float *W,
                              const float *best_u, int S, cudaStream_t st);

void count_launch(int n = 1);

// Store the CUDA error text for tma_last_error_string(); returns TMA_ERR_CUDA.
tma_status record_cuda_error(cudaError_t e);

// Host FP64 Cholesky (lower), row-major n x n, in place; returns false if not
// positive definite.
bool cholesky_lower(std::vector<double> &A, int n);

}  // namespace tma

struct tma_solver {
    tma_problem prob;
    std::vector<tma_aircraft> aircraft;
    std::vector<double> popdense_host;
    std::vector<int64_t> L_sched;   // particles per iteration (empty: L every iteration)
    tma::ProblemC P;
    tma::WindC wind;
    int device;
    // device buffers (owned)
    tma::DynState *d_dyn = nullptr;
    float *d_Lxy = nullptr;
    int lda = 0;
    float *d_Btmp = nullptr;
    float *d_W = nullptr;
    float *d_u[2] = {nullptr, nullptr};
    float *d_cost_ms = nullptr, *d_cost_ms_soft = nullptr;
    float *d_cbar = nullptr, *d_cbar_soft = nullptr;
    double *d_wtilde = nullptr;
    int32_t *d_anc = nullptr;
    float *d_popdense = nullptr;          // population density cells (ProblemC::popcell), or nullptr
    void *d_work = nullptr;             // LSE workspace, then the resampling's at lse_work_bytes
    size_t work_bytes = 0, lse_work_bytes = 0;
    int64_t *d_best = nullptr;
    double *d_best_sum = nullptr;
    int32_t *d_ninf = nullptr;
    unsigned int *d_flags = nullptr;
    unsigned int *d_err = nullptr;      // sticky error word (tma_get_error)
    unsigned long long *d_live = nullptr;
    float *d_best_u = nullptr;
    int cur_u = 0;
    int64_t last_L = 0;
    int last_M = 0;             // wind samples of the last rollout (M_J in sample mode 1)
    uint32_t mpc_step = 0;
    bool wind_ready = false;
    // stage profiling (CUDA events)
    bool prof = false;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[TMA_N_STAGES] = {0};
    uint64_t prof_n[TMA_N_STAGES] = {0};
    // one-scenario tables for the plant step (the batched plant kernel)
    tma::ProblemC *d_probs1 = nullptr;
    tma::BatchScen *d_scen1 = nullptr;
    int *d_seg_scen1 = nullptr;
    // gradient scratch (allocated on first use)
    float *d_gcost_ms = nullptr;        // [M][N][L]
    float *d_gpart = nullptr;           // [nchunk][L][N][S][3]
    size_t gpart_elems = 0;
    int grad_variant = -1;              // autotuned launch variant of the gradient kernel
    int n_grad_tuned = 0;
    int grad_tuned_variant[8] = {0};
    float grad_tuned_ms[8] = {0};
    // accepted moves (tma_set_move)
    int move_kind = 0;
    double eps0 = 1.0;
    double *d_eps = nullptr;            // [0] adapted step, [1] step of a stage call
    unsigned int *d_nacc = nullptr;
    unsigned int *d_acc_hist = nullptr; // [J_max]
    double *d_eps_hist = nullptr;       // [J_max]
    float *d_u_prop = nullptr, *d_grad0 = nullptr, *d_grad1 = nullptr;
    float *d_cbar0 = nullptr, *d_cbar1 = nullptr, *d_cost0 = nullptr, *d_cost1 = nullptr;
    uint8_t *d_inbox = nullptr;
    // autotuned launch variant of the rollout kernel and the timings behind it
    int rollout_variant = -1;
    int n_tuned = 0;
    int tuned_variant[tma::kMaxRolloutVariants] = {0};
    float tuned_ms[tma::kMaxRolloutVariants] = {0};
};

struct tma_batch {
    int n_scen = 0;
    int device = 0;
    int L = 0, M = 0, H = 0, S = 0, J_max = 0, sep_mode = 0;
    long long nseg = 0, n_items = 0;
    int grid = 0;
    std::vector<tma_problem> probs;
    std::vector<std::vector<tma_aircraft>> aircraft;
    std::vector<std::vector<double>> pop;
    std::vector<tma::BatchScen> scen;
    std::vector<int> seg_scen;
    std::vector<tma::DynState> dyn_h;
    std::vector<tma::WindC> wind_groups;   // one GEMM per group of scenarios
    std::vector<int> group_start;
    int lda = 0;
    // device buffers (owned)
    tma::ProblemC *d_probs = nullptr;
    tma::BatchScen *d_scen = nullptr;
    int *d_seg_scen = nullptr;
    tma::SegKey *d_segkeys = nullptr;
    tma::DynState *d_dyns = nullptr;
    float *d_Lxy = nullptr, *d_Btmp = nullptr, *d_W = nullptr;
    float *d_u[2] = {nullptr, nullptr};
    float *d_cost_ms = nullptr, *d_cost_ms_soft = nullptr, *d_cbar = nullptr, *d_cbar_soft = nullptr;
    double *d_wtilde = nullptr;
    int32_t *d_anc = nullptr;
    void *d_work = nullptr;             // LSE workspace, then the resampling's at lse_work_bytes
    size_t lse_work_bytes = 0;
    long long *d_best = nullptr;
    double *d_best_sum = nullptr;
    int *d_ninf = nullptr;
    float *d_best_u = nullptr;
    unsigned long long *d_t_start = nullptr, *d_t_end = nullptr, *d_live = nullptr, *d_queue = nullptr;
    unsigned int *d_flags = nullptr;
    unsigned int *d_err = nullptr;      // sticky error word (TMA_DEVERR_BOUNDS), read by tma_batch_results
    // rollout dispatch, chosen at creation by timing both forms on the batch:
    // 0 one persistent launch over every scenario's tiles, 1 one launch of the
    // single-scenario kernel per scenario (its autotuned variant each)
    int dispatch = 0;
    float dispatch_ms[2] = {0.f, 0.f};
    std::vector<tma::ProblemC> pc_h;    // every scenario's kernel problem (host copy)
    std::vector<int> scen_variant;      // its variant of the single-scenario rollout kernel
    // form 1 spreads the per-scenario launches over these streams (forked from
    // and joined to the caller's stream by events, also inside a capture)
    static constexpr int kAuxStreams = 4;
    cudaStream_t aux[kAuxStreams] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kAuxStreams] = {};
    std::vector<float *> d_pops;
    int final_u = 0;
    // captured MPC loop
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
};
