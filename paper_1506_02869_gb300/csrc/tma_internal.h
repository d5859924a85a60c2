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

// Per-aircraft constants in FP32 (derived on the host in FP64).
struct AircraftC {
    int type;              // 0 arrival, 1 departure
    float halfS, CD0, CD2;
    float Cf1, invCf2, Tmin, Tmax, m_empty;
    float thF, Z, vD;
    float invFmax;         // 1 / (H dt Tmax eta(vmax))
    float supB, invSupInf; // departure altitude-term normalisation
    float invCmax;         // departure speed-term normalisation
};

// Problem constants passed by value to the rollout kernels.
struct ProblemC {
    int N, H, S, M, G;     // G = lanes per (particle, sample) group = next_pow2(N)
    int P;                 // wind grid nodes
    int grid[3];
    float dt;
    float box_lo[3], box_hi[3], inv_h[3];
    float turb_sigma;
    float sgmax, tpmax;    // sin(gamma_max), tan(phi_max)
    float Sh2, Sh_inv, Sv, Sv_inv;
    int sep_mode;
    float sp_beta, sp_inv_beta, mu_sep;
    float z_min, z_max, v_min, v_max;
    float a_dep[4], a_arr[3];
    float w_noise, Ac_inv;
    int pop_n[2];
    float pop_lo[2], pop_hi[2], pop_inv_h[2];
    const float *popdense; // device [pop_n0][pop_n1] or nullptr
    float P_runway, P_beta, P_chi, P_vs, beta_f;
    uint32_t key0, key1;   // Philox key (seed + scenario_id * golden)
    AircraftC ac[kMaxN];
};

// Per-solve dynamic state in device memory (updated between graph replays).
struct DynState {
    float x0[kMaxN][6];
    uint32_t mpc_step;
};

// Parameters of the wind-field generation kernels.
struct WindC {
    int M, H, nxy, nz, ncol, ldb;
    float a, b, sigma;
    float Lz[TMA_MAX_GRID_Z * TMA_MAX_GRID_Z];
    uint32_t key0, key1;
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
// Launch-bound variants of the rollout kernel valid for N aircraft (indices
// into the variant table); returns their number (at least 1).
int rollout_variants(int N, int *out);
cudaError_t launch_sample_mean(const float *cost_ms, int64_t L, int M, int N, float *cbar,
                               cudaStream_t st);

cudaError_t launch_lse(const float *cbar, int nseg, int64_t L, double kappa, double *wtilde,
                       double *lmax, double *wsum, void *work, cudaStream_t st);
size_t lse_workspace(int nseg, int64_t L);
cudaError_t launch_resample(const double *wtilde, int nseg, int64_t L, uint32_t key0,
                            uint32_t key1, uint32_t J, const uint32_t *d_mpc, uint32_t mpc_host,
                            int32_t *anc, void *work, unsigned int *d_flags, cudaStream_t st);
size_t resample_workspace(int nseg, int64_t L);

cudaError_t launch_move(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                        const float ctrl_hi[3], const float sigma[3], const float *u,
                        const int32_t *anc, int64_t L, int J, float *u_out, cudaStream_t st);
cudaError_t launch_init_controls(const ProblemC &P, const DynState *dyn, const float ctrl_lo[3],
                                 const float ctrl_hi[3], float *u, int64_t L, cudaStream_t st);

cudaError_t launch_select(const float *cbar, int N, int64_t L, int64_t *best, double *best_sum,
                          int *ninf, void *work, cudaStream_t st);
size_t select_workspace(int64_t L);
cudaError_t launch_gather_best(const float *u, const int64_t *best, int nctl_per_particle,
                               float *best_u, cudaStream_t st);

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
    float *d_popdense = nullptr;
    void *d_work = nullptr;
    size_t work_bytes = 0;
    int64_t *d_best = nullptr;
    double *d_best_sum = nullptr;
    int32_t *d_ninf = nullptr;
    unsigned int *d_flags = nullptr;
    unsigned long long *d_live = nullptr;
    float *d_best_u = nullptr;
    int cur_u = 0;
    int64_t last_L = 0;
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
    double prof_ms[8] = {0};
    uint64_t prof_n[8] = {0};
    // autotuned launch variant of the rollout kernel and the timings behind it
    int rollout_variant = -1;
    int n_tuned = 0;
    int tuned_variant[8] = {0};
    float tuned_ms[8] = {0};
};
