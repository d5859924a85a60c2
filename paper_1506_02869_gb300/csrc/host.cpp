// Host runtime of the CUDA path: scenario validation, derived constants, the
// FP64 Cholesky factors of the wind covariance, the solver object and every
// entry point of include/tma_smc.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "tma_internal.h"

namespace tma {

static std::atomic<unsigned long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

static thread_local std::string g_last_error;

static tma_status cuda_fail(cudaError_t e)
{
    g_last_error = cudaGetErrorString(e);
    return TMA_ERR_CUDA;
}

tma_status record_cuda_error(cudaError_t e) { return cuda_fail(e); }

#define TMA_CUDA(expr)                             \
    do {                                           \
        cudaError_t e_ = (expr);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// ------------------------------------------------------------------ Cholesky

// Right-looking blocked Cholesky, lower triangle, row-major; the panel solve
// and the trailing update are split over threads by rows.
bool cholesky_lower(std::vector<double> &A, int n)
{
    const int NB = 64;
    unsigned hw = std::thread::hardware_concurrency();
    const int nth = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
    auto at = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    auto parallel_rows = [&](int r0, int r1, auto &&fn) {
        const int rows = r1 - r0;
        if (rows <= 0) return;
        const int T = std::min(nth, std::max(1, rows / 16));
        if (T == 1) {
            for (int i = r0; i < r1; ++i) fn(i);
            return;
        }
        std::vector<std::thread> th;
        for (int t = 0; t < T; ++t)
            th.emplace_back([&, t]() {
                for (int i = r0 + t; i < r1; i += T) fn(i);
            });
        for (auto &x : th) x.join();
    };
    bool ok = true;
    for (int kb = 0; kb < n && ok; kb += NB) {
        const int ke = std::min(n, kb + NB);
        for (int j = kb; j < ke; ++j) {
            double d = at(j, j);
            for (int t = kb; t < j; ++t) d -= at(j, t) * at(j, t);
            if (!(d > 0.0)) {
                ok = false;
                break;
            }
            const double ljj = std::sqrt(d);
            at(j, j) = ljj;
            for (int i = j + 1; i < ke; ++i) {
                double s = at(i, j);
                for (int t = kb; t < j; ++t) s -= at(i, t) * at(j, t);
                at(i, j) = s / ljj;
            }
        }
        if (!ok) break;
        parallel_rows(ke, n, [&](int i) {
            for (int j = kb; j < ke; ++j) {
                double s = at(i, j);
                for (int t = kb; t < j; ++t) s -= at(i, t) * at(j, t);
                at(i, j) = s / at(j, j);
            }
        });
        parallel_rows(ke, n, [&](int i) {
            const double *ri = &A[(size_t)i * n + kb];
            for (int j = ke; j <= i; ++j) {
                const double *rj = &A[(size_t)j * n + kb];
                double s = 0.0;
                for (int t = 0; t < ke - kb; ++t) s += ri[t] * rj[t];
                at(i, j) -= s;
            }
        });
    }
    if (!ok) return false;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) at(i, j) = 0.0;
    return true;
}

// Horizontal factor L_xy (FP32, zero-padded) cached per grid and rate.
struct LxyEntry {
    std::vector<float> L;
    int lda;
};
static std::mutex g_lxy_mu;
static std::map<std::string, std::shared_ptr<LxyEntry>> g_lxy;

static std::shared_ptr<LxyEntry> horizontal_factor(const tma_problem &p)
{
    char key[256];
    snprintf(key, sizeof key, "%d %d %.17g %.17g %.17g %.17g %.17g", p.grid[0], p.grid[1],
             p.box_lo[0], p.box_hi[0], p.box_lo[1], p.box_hi[1], p.beta_xy);
    {
        std::lock_guard<std::mutex> g(g_lxy_mu);
        auto it = g_lxy.find(key);
        if (it != g_lxy.end()) return it->second;
    }
    const int nx = p.grid[0], ny = p.grid[1], n = nx * ny;
    std::vector<double> xs(nx), ys(ny);
    for (int i = 0; i < nx; ++i) xs[i] = p.box_lo[0] + (p.box_hi[0] - p.box_lo[0]) * i / (nx - 1);
    for (int i = 0; i < ny; ++i) ys[i] = p.box_lo[1] + (p.box_hi[1] - p.box_lo[1]) * i / (ny - 1);
    std::vector<double> R((size_t)n * n);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b <= a; ++b) {
            const double dx = xs[a / ny] - xs[b / ny], dy = ys[a % ny] - ys[b % ny];
            R[(size_t)a * n + b] = std::exp(-p.beta_xy * std::sqrt(dx * dx + dy * dy));
        }
    if (!cholesky_lower(R, n)) return nullptr;
    auto e = std::make_shared<LxyEntry>();
    e->lda = ((n + 127) / 128) * 128;
    e->L.assign((size_t)e->lda * e->lda, 0.0f);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b <= a; ++b) e->L[(size_t)a * e->lda + b] = (float)R[(size_t)a * n + b];
    std::lock_guard<std::mutex> g(g_lxy_mu);
    g_lxy[key] = e;
    return e;
}

static int next_pow2(int n)
{
    int g = 1;
    while (g < n) g <<= 1;
    return g;
}

static bool finite(double x) { return std::isfinite(x); }

static tma_status validate(const tma_problem *p, const tma_aircraft *ac)
{
    if (!p || !ac) return TMA_ERR_INVALID_ARG;
    if (p->N < 1 || p->N > TMA_MAX_AIRCRAFT || p->H < 1 || p->S < 1 || p->S > p->H ||
        p->L < 1 || p->L > TMA_MAX_PARTICLES || p->M < 1 || p->M >= (1 << 24) ||
        p->J_max < 1 || p->J_max > 0xFFFF || p->H > (1 << 25) || p->mpc_step > 0xFFFF)
        return TMA_ERR_INVALID_ARG;
    if (!(p->dt > 0) || !finite(p->dt)) return TMA_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (p->grid[d] < 2 || !(p->box_hi[d] > p->box_lo[d])) return TMA_ERR_INVALID_ARG;
    if (p->grid[2] > TMA_MAX_GRID_Z) return TMA_ERR_INVALID_ARG;
    if (p->wind_mode != 0 && p->wind_mode != 1) return TMA_ERR_INVALID_ARG;
    if (p->sample_mode != 0 && p->sample_mode != 1) return TMA_ERR_INVALID_ARG;
    if (p->rolling != 0 && p->rolling != 1) return TMA_ERR_INVALID_ARG;
    if (p->L_sched)
        for (int J = 0; J < p->J_max; ++J)
            if (p->L_sched[J] < 1 || p->L_sched[J] > p->L) return TMA_ERR_INVALID_ARG;
    if (p->wind_mode == 1 && (p->grid[0] != 2 || p->grid[1] != 2 || p->grid[2] != 2))
        return TMA_ERR_INVALID_ARG;
    if ((long long)p->grid[0] * p->grid[1] > 16384) return TMA_ERR_INVALID_ARG;
    if (!(p->sep_h > 0) || !(p->sep_v > 0) || p->sep_mode < 0 || p->sep_mode > 2)
        return TMA_ERR_INVALID_ARG;
    if (!(p->lam_t >= 0) || !(p->wind_sigma >= 0) || !(p->turb_sigma >= 0)) return TMA_ERR_INVALID_ARG;
    if (!(p->gamma_max > 0 && p->gamma_max < M_PI / 2) || !(p->phi_max > 0 && p->phi_max < M_PI / 2))
        return TMA_ERR_INVALID_ARG;
    if (!(p->v_max > p->v_min) || !(p->v_min > 0)) return TMA_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(p->ctrl_hi[c] >= p->ctrl_lo[c])) return TMA_ERR_INVALID_ARG;
    if (p->w_noise != 0.0 && !(p->A_c > 0)) return TMA_ERR_INVALID_ARG;
    if (p->pop_n[0] != 0 || p->pop_n[1] != 0) {
        if (p->pop_n[0] < 2 || p->pop_n[1] < 2 || !p->popdense || !(p->pop_hi[0] > p->pop_lo[0]) ||
            !(p->pop_hi[1] > p->pop_lo[1]))
            return TMA_ERR_INVALID_ARG;
    }
    for (int i = 0; i < p->N; ++i) {
        const tma_aircraft &a = ac[i];
        if (a.type != 0 && a.type != 1) return TMA_ERR_INVALID_ARG;
        if (!(a.x0.v > 0) || !(a.x0.m > 0) || !(a.S > 0) || !(a.Cf1 > 0) || !(a.Cf2 > 0) ||
            !(a.Tmax > 0))
            return TMA_ERR_INVALID_ARG;
    }
    return TMA_OK;
}

// The population density's cells with their four corner values, the layout
// of ProblemC::popcell: cell (a, b) of the row-major [n0][n1] grid g holds
// g[a][b], g[a][b+1], g[a+1][b], g[a+1][b+1] (FP32).
static std::vector<float> pack_popcells(const double *g, int n0, int n1)
{
    std::vector<float> c((size_t)(n0 - 1) * (n1 - 1) * 4);
    for (int a = 0; a + 1 < n0; ++a)
        for (int b = 0; b + 1 < n1; ++b) {
            float *o = &c[((size_t)a * (n1 - 1) + b) * 4];
            o[0] = (float)g[(size_t)a * n1 + b];
            o[1] = (float)g[(size_t)a * n1 + b + 1];
            o[2] = (float)g[(size_t)(a + 1) * n1 + b];
            o[3] = (float)g[(size_t)(a + 1) * n1 + b + 1];
        }
    return c;
}

static ProblemC derive_problem(const tma_problem &p, const tma_aircraft *aircraft,
                               const float *d_popcell)
{
    ProblemC P;
    std::memset(&P, 0, sizeof P);
    P.N = p.N;
    P.H = p.H;
    P.S = p.S;
    P.M = p.M;
    P.G = next_pow2(p.N);
    P.P = p.grid[0] * p.grid[1] * p.grid[2];
    for (int d = 0; d < 3; ++d) {
        P.grid[d] = p.grid[d];
        P.box_lo[d] = (float)p.box_lo[d];
        P.box_hi[d] = (float)p.box_hi[d];
        P.inv_h[d] = (float)((p.grid[d] - 1) / (p.box_hi[d] - p.box_lo[d]));
    }
    P.dt = (float)p.dt;
    P.wind_mode = p.wind_mode;
    if (p.wind_mode == 1) {
        // Qhat for the field of one (particle, sample): Cholesky factor (FP64) of
        // R_hat = sigma^2 exp(-beta |dxy|) exp(-gamma |dz|) over the eight box
        // corners, node index (ix * 2 + iy) * 2 + iz
        std::vector<double> R(64);
        for (int a = 0; a < 8; ++a)
            for (int b = 0; b < 8; ++b) {
                const int ax = a >> 2, ay = (a >> 1) & 1, az = a & 1;
                const int bx = b >> 2, by = (b >> 1) & 1, bz = b & 1;
                const double dx = (ax - bx) * (p.box_hi[0] - p.box_lo[0]);
                const double dy = (ay - by) * (p.box_hi[1] - p.box_lo[1]);
                const double dz = (az - bz) * (p.box_hi[2] - p.box_lo[2]);
                R[a * 8 + b] = p.wind_sigma * p.wind_sigma * std::exp(-p.beta_xy * std::sqrt(dx * dx + dy * dy)) *
                               std::exp(-p.gam_z * std::fabs(dz));
            }
        if (cholesky_lower(R, 8))
            for (int n = 0, k = 0; n < 8; ++n)
                for (int j = 0; j <= n; ++j) P.wchol[k++] = (float)R[n * 8 + j];
        const double a = std::exp(-p.dt * p.lam_t);
        P.wind_a = (float)a;
        P.wind_b = (float)std::sqrt(std::max(0.0, 1.0 - a * a));
    }
    P.turb_sigma = (float)p.turb_sigma;
    P.sgmax = (float)std::sin(p.gamma_max);
    P.tpmax = (float)std::tan(p.phi_max);
    P.climb_step = (float)(p.v_max * std::sin(p.gamma_max) * p.dt);
    P.Sh2 = (float)(p.sep_h * p.sep_h);
    P.Sh_inv = (float)(1.0 / p.sep_h);
    P.Sv = (float)p.sep_v;
    P.Sv_inv = (float)(1.0 / p.sep_v);
    P.sep_mode = p.sep_mode;
    P.sp_beta = (float)p.sp_beta;
    P.sp_inv_beta = (float)(p.sp_beta != 0 ? 1.0 / p.sp_beta : 0.0);
    {
        // g = min(1 - d_h/S_h, 1 - |dz|/S_v) < -30/beta when d_h > S_h (1 + 30/beta)
        // or |dz| > S_v (1 + 30/beta)
        const double f = p.sp_beta > 0 ? 1.0 + 30.0 / p.sp_beta : 1e30;
        const double fh = p.sep_h * f;
        P.sp_far_h2 = (float)std::min(fh * fh, 1e30);
        P.sp_far_v = (float)std::min(p.sep_v * f, 1e30);
    }
    P.mu_sep = (float)p.mu_sep;
    P.z_min = (float)p.z_min;
    P.z_max = (float)p.z_max;
    P.v_min = (float)p.v_min;
    P.v_max = (float)p.v_max;
    for (int j = 0; j < 4; ++j) P.a_dep[j] = (float)p.alpha_dep[j];
    for (int j = 0; j < 3; ++j) P.a_arr[j] = (float)p.alpha_arr[j];
    P.w_noise = (float)p.w_noise;
    P.Ac_inv = (float)(p.A_c > 0 ? 1.0 / p.A_c : 0.0);
    P.popcell = reinterpret_cast<const float4 *>(d_popcell);
    for (int d = 0; d < 2; ++d) {
        P.pop_n[d] = p.pop_n[d];
        P.pop_lo[d] = (float)p.pop_lo[d];
        P.pop_hi[d] = (float)p.pop_hi[d];
        P.pop_inv_h[d] = p.pop_n[d] >= 2 ? (float)((p.pop_n[d] - 1) / (p.pop_hi[d] - p.pop_lo[d])) : 0.f;
    }
    P.P_runway = (float)p.P_runway;
    P.P_beta = (float)p.P_beta;
    P.P_chi = (float)p.P_chi;
    P.P_vs = (float)p.P_vs;
    P.beta_f = (float)p.beta_f;
    const uint64_t key = p.seed + (uint64_t)p.scenario_id * 0x9E3779B97F4A7C15ull;
    P.seg_q = p.H / p.S;
    P.seg_r = p.H % p.S;
    P.key0 = (uint32_t)key;
    P.key1 = (uint32_t)(key >> 32);
    for (int r = 0; r < 10; ++r) {      // the round keys: (k0, k1) + r (Weyl constants)
        P.rk[2 * r] = P.key0 + (uint32_t)r * 0x9E3779B9u;
        P.rk[2 * r + 1] = P.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    for (int i = 0; i < p.N; ++i) {
        const tma_aircraft &a = aircraft[i];
        AircraftC &c = P.ac[i];
        c.type = a.type;
        c.halfS = (float)(0.5 * a.S);
        c.CD0 = (float)a.CD0;
        c.CD2 = (float)a.CD2;
        c.Cf1 = (float)a.Cf1;
        c.invCf2 = (float)(1.0 / a.Cf2);
        c.Tmin = (float)a.Tmin;
        c.Tmax = (float)a.Tmax;
        c.m_empty = (float)a.m_empty;
        c.thF = (float)a.theta_F;
        c.Z = (float)a.Z;
        c.vD = (float)a.v_D;
        const double Fmax = p.H * p.dt * a.Tmax * a.Cf1 * (1.0 + p.v_max / a.Cf2);
        c.invFmax = (float)(1.0 / Fmax);
        c.invCmax = (float)(1.0 / std::max(p.v_max - a.v_D, a.v_D - p.v_min));
        c.t_enter = a.t_enter;
    }
    P.rolling = p.rolling;
    return P;
}

static void derive(tma_solver *s)
{
    s->P = derive_problem(s->prob, s->aircraft.data(), s->d_popdense);
}

static void upload_x0(tma_solver *s, DynState &d)
{
    std::memset(&d, 0, sizeof d);
    for (int i = 0; i < s->prob.N; ++i) {
        const tma_state &x = s->aircraft[i].x0;
        d.x0[i][0] = (float)x.x;
        d.x0[i][1] = (float)x.y;
        d.x0[i][2] = (float)x.z;
        d.x0[i][3] = (float)x.v;
        d.x0[i][4] = (float)x.chi;
        d.x0[i][5] = (float)x.m;
    }
    d.mpc_step = s->mpc_step;
}

static void free_all(tma_solver *s)
{
    void *ptrs[] = {s->d_dyn, s->d_Lxy, s->d_Btmp, s->d_W, s->d_u[0], s->d_u[1], s->d_cost_ms,
                    s->d_cost_ms_soft, s->d_cbar, s->d_cbar_soft, s->d_wtilde, s->d_anc,
                    s->d_popdense, s->d_work, s->d_best, s->d_best_sum, s->d_ninf, s->d_flags, s->d_err,
                    s->d_live, s->d_best_u, s->d_probs1, s->d_scen1, s->d_seg_scen1,
                    s->d_gcost_ms, s->d_gpart, s->d_eps, s->d_nacc, s->d_acc_hist,
                    s->d_eps_hist, s->d_u_prop, s->d_grad0, s->d_grad1, s->d_cbar0, s->d_cbar1,
                    s->d_cost0, s->d_cost1, s->d_inbox};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <typename T>
static cudaError_t alloc(T **p, size_t bytes)
{
    return cudaMalloc(reinterpret_cast<void **>(p), bytes > 0 ? bytes : 16);
}

// Static (FP32) copies of the control box and move sigma.
static void ctrl_f(const tma_problem &p, float lo[3], float hi[3], float sg[3])
{
    for (int c = 0; c < 3; ++c) {
        lo[c] = (float)p.ctrl_lo[c];
        hi[c] = (float)p.ctrl_hi[c];
        sg[c] = (float)p.move_sigma[c];
    }
}

// Optional CUDA-event timing of one stage on the launching stream.
struct StageTimer {
    tma_solver *s;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    static cudaEvent_t take(tma_solver *s)
    {
        if (!s->event_pool.empty()) {
            cudaEvent_t e = s->event_pool.back();
            s->event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    StageTimer(tma_solver *s_, int stage_, cudaStream_t st_) : s(s_), stage(stage_), st(st_)
    {
        if (s->prof && (a = take(s)) != nullptr) cudaEventRecord(a, st);
    }
    void done()
    {
        if (!a) return;
        cudaEvent_t b = take(s);
        if (!b) return;
        cudaEventRecord(b, st);
        s->pending.push_back({stage, a, b});
        a = nullptr;
    }
    ~StageTimer() { done(); }
};

static int kappa_of(int J) { return (int)std::floor(3.0 + 5.0 * std::exp(0.05 * J)); }

// Wind samples of iteration J: all M, or in sample mode 1 the inner loop of
// Algorithm 1, SampleSchedule(J) draws (at most M).
static int samples_of(const tma_problem &p, int J)
{
    return p.sample_mode == 1 ? std::min(kappa_of(J), p.M) : p.M;
}

// Factor of the mean cost in the log-weight: kappa_J with M fixed samples; in
// sample mode 1 the product of J_T over the iteration's M_J draws (Sec. 3.6).
static double exponent_of(const tma_problem &p, int J)
{
    return p.sample_mode == 1 ? (double)samples_of(p, J) : (double)kappa_of(J);
}

// Particles evaluated in iteration J (the particle schedule, else L).
static int64_t particles_of(const tma_solver *s, int J)
{
    return s->L_sched.empty() ? s->prob.L : s->L_sched[(size_t)J];
}

// The problem as the kernels of iteration J see it (M = that iteration's samples).
static ProblemC problem_at(const tma_solver *s, int J)
{
    ProblemC P = s->P;
    P.M = samples_of(s->prob, J);
    return P;
}

// the resampling's part of the solver's workspace (after the LSE's)
static void *res_work(const tma_solver *s) { return static_cast<char *>(s->d_work) + s->lse_work_bytes; }

// device address of DynState::mpc_step (pointer arithmetic only)
static const uint32_t *dyn_mpc(const tma_solver *s)
{
    return reinterpret_cast<const uint32_t *>(reinterpret_cast<const char *>(s->d_dyn) +
                                              offsetof(DynState, mpc_step));
}

// ------------------------------------------------------------------ autotuner

static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

static std::string tune_key_of(const tma_problem &p, int device)
{
    cudaDeviceProp prop;
    char key[320];
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) prop.name[0] = 0;
    // the workload's size class: tiles of the tuning launch (32 particles x one
    // wind sample each, at most 8192 particles), by power of two -- a small
    // solver's choice is not reused for a large one
    const long long tiles = (std::min<long long>(p.L, 8192) + 31) / 32 * (long long)p.M;
    int lg = 0;
    while ((2LL << lg) <= tiles) ++lg;
    snprintf(key, sizeof key, "%s|N=%d|pop=%d|wind=%d|rolling=%d|sep=%d|tiles=2^%d", prop.name, p.N,
             p.pop_n[0] > 0, p.wind_mode, p.rolling, p.sep_mode, lg);
    return key;
}

static std::string tune_key(const tma_solver *s) { return tune_key_of(s->prob, s->device); }

// Times every launch variant of the rollout kernel valid for P on the given
// buffers (Lp particles, all wind samples, iteration 0, the hard costs only):
// one untimed launch and three timed per variant; *best = the fastest, and the
// timings in tv[] / tms[] (*nt entries).
static cudaError_t time_rollout_variants(const ProblemC &P, const DynState *dyn, const float *u,
                                         const float *W, int64_t Lp, float *cost, cudaStream_t st,
                                         cudaEvent_t e0, cudaEvent_t e1, int *best, int *nt, int *tv,
                                         float *tms)
{
    int cand[kMaxRolloutVariants];
    const int nc = rollout_variants(P, cand);
    *best = cand[0];
    *nt = 0;
    float best_ms = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        e = launch_rollout(P, dyn, u, W, Lp, 0, cost, nullptr, nullptr, st, cand[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
            e = launch_rollout(P, dyn, u, W, Lp, 0, cost, nullptr, nullptr, st, cand[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        tv[*nt] = cand[c];
        tms[*nt] = ms / 3.0f;
        ++*nt;
        if (ms < best_ms) {
            best_ms = ms;
            *best = cand[c];
        }
    }
    return e;
}

}  // namespace tma

using namespace tma;

extern "C" {

static tma_status autotune_rollout(tma_solver *s);

const char *tma_status_str(tma_status s)
{
    switch (s) {
    case TMA_OK: return "ok";
    case TMA_ERR_INVALID_ARG: return "invalid argument";
    case TMA_ERR_OOM: return "out of memory";
    case TMA_ERR_CUDA: return "CUDA error";
    case TMA_ERR_BOUNDS: return "index out of bounds";
    case TMA_ERR_TIMEOUT: return "timeout";
    case TMA_WARN_DEGENERATE: return "degenerate weights (identity resampling used)";
    case TMA_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *tma_last_error_string(void) { return g_last_error.c_str(); }

uint64_t tma_launch_count(void) { return g_launches.load(); }

tma_status tma_create(const tma_problem *prob, const tma_aircraft *aircraft, tma_solver **out)
{
    if (!out) return TMA_ERR_INVALID_ARG;
    *out = nullptr;
    tma_status v = validate(prob, aircraft);
    if (v != TMA_OK) return v;
    tma_solver *s = nullptr;
    try {
        s = new tma_solver();
        s->prob = *prob;
        s->aircraft.assign(aircraft, aircraft + prob->N);
        if (prob->pop_n[0] >= 2) {
            s->popdense_host.assign(prob->popdense,
                                    prob->popdense + (size_t)prob->pop_n[0] * prob->pop_n[1]);
        }
        s->prob.popdense = nullptr;
        if (prob->L_sched) s->L_sched.assign(prob->L_sched, prob->L_sched + prob->J_max);
        s->prob.L_sched = nullptr;
        s->mpc_step = prob->mpc_step;
        cudaGetDevice(&s->device);
        const tma_problem &p = s->prob;
        const size_t L = (size_t)p.L, N = (size_t)p.N, M = (size_t)p.M, H = (size_t)p.H;
        const int nx = p.grid[0], ny = p.grid[1], nz = p.grid[2];
        const int nxy = nx * ny;
        const size_t P = (size_t)nxy * nz;
        auto fail = [&](cudaError_t e) {
            free_all(s);
            delete s;
            return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : cuda_fail(e);
        };
        cudaError_t e;
        // population density to device: FP32 cells with their four corners
        if (!s->popdense_host.empty()) {
            const std::vector<float> pf = pack_popcells(s->popdense_host.data(), p.pop_n[0], p.pop_n[1]);
            if ((e = alloc(&s->d_popdense, pf.size() * 4))) return fail(e);
            if ((e = cudaMemcpy(s->d_popdense, pf.data(), pf.size() * 4, cudaMemcpyHostToDevice)))
                return fail(e);
        }
        derive(s);
        // wind factors
        auto lxy = horizontal_factor(p);
        if (!lxy) {
            free_all(s);
            delete s;
            return TMA_ERR_INVALID_ARG;
        }
        std::vector<double> Rz((size_t)nz * nz);
        for (int a = 0; a < nz; ++a)
            for (int b = 0; b <= a; ++b) {
                const double za = p.box_lo[2] + (p.box_hi[2] - p.box_lo[2]) * a / (nz - 1);
                const double zb = p.box_lo[2] + (p.box_hi[2] - p.box_lo[2]) * b / (nz - 1);
                Rz[(size_t)a * nz + b] = std::exp(-p.gam_z * std::fabs(za - zb));
            }
        if (!cholesky_lower(Rz, nz)) {
            free_all(s);
            delete s;
            return TMA_ERR_INVALID_ARG;
        }
        WindC &w = s->wind;
        std::memset(&w, 0, sizeof w);
        w.M = p.M;
        w.H = p.H;
        w.nxy = nxy;
        w.nz = nz;
        w.ncol = (int)(M * H * 2 * nz);
        w.ldb = ((w.ncol + 127) / 128) * 128;
        const double a = std::exp(-p.dt * p.lam_t);
        w.a = (float)a;
        w.b = (float)std::sqrt(std::max(0.0, 1.0 - a * a));
        w.sigma = (float)p.wind_sigma;
        for (int r = 0; r < nz; ++r)
            for (int c = 0; c <= r; ++c) w.Lz[r * TMA_MAX_GRID_Z + c] = (float)Rz[(size_t)r * nz + c];
        w.key0 = s->P.key0;
        w.key1 = s->P.key1;
        w.stream = 3u;
        s->lda = lxy->lda;
        if ((e = alloc(&s->d_Lxy, lxy->L.size() * 4))) return fail(e);
        if ((e = cudaMemcpy(s->d_Lxy, lxy->L.data(), lxy->L.size() * 4, cudaMemcpyHostToDevice)))
            return fail(e);
        const size_t brows = (size_t)s->lda;
        if ((e = alloc(&s->d_Btmp, brows * w.ldb * 4))) return fail(e);
        if ((e = cudaMemset(s->d_Btmp, 0, brows * w.ldb * 4))) return fail(e);
        if ((e = alloc(&s->d_W, M * H * P * 4 * 4))) return fail(e);   // packed float4 per node
        const size_t ubytes = L * N * p.S * 3 * 4;
        if ((e = alloc(&s->d_u[0], ubytes))) return fail(e);
        if ((e = alloc(&s->d_u[1], ubytes))) return fail(e);
        if ((e = alloc(&s->d_cost_ms, L * M * N * 4))) return fail(e);
        if (p.sep_mode != 0 && (e = alloc(&s->d_cost_ms_soft, L * M * N * 4))) return fail(e);
        if ((e = alloc(&s->d_cbar, L * N * 4))) return fail(e);
        if (p.sep_mode != 0 && (e = alloc(&s->d_cbar_soft, L * N * 4))) return fail(e);
        if ((e = alloc(&s->d_wtilde, L * N * 8))) return fail(e);
        if ((e = alloc(&s->d_anc, L * N * 4))) return fail(e);
        // the LSE's and the resampling's workspaces side by side: the LSE pass
        // writes the resampling's chunk sums
        s->lse_work_bytes = (lse_workspace(p.N, p.L) + 255) / 256 * 256;
        s->work_bytes = std::max(s->lse_work_bytes + resample_workspace(p.N, p.L), select_workspace(p.L));
        if ((e = alloc(&s->d_work, s->work_bytes))) return fail(e);
        if ((e = alloc(&s->d_best, 8))) return fail(e);
        if ((e = alloc(&s->d_best_sum, 8))) return fail(e);
        if ((e = alloc(&s->d_ninf, 4))) return fail(e);
        if ((e = alloc(&s->d_flags, 4))) return fail(e);
        if ((e = alloc(&s->d_err, 4))) return fail(e);
        if ((e = cudaMemset(s->d_err, 0, 4))) return fail(e);
        if ((e = alloc(&s->d_live, 8))) return fail(e);
        if ((e = alloc(&s->d_best_u, N * p.S * 3 * 4))) return fail(e);
        if ((e = alloc(&s->d_dyn, sizeof(DynState)))) return fail(e);
        DynState d;
        upload_x0(s, d);
        if ((e = cudaMemcpy(s->d_dyn, &d, sizeof d, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemset(s->d_flags, 0, 4))) return fail(e);
        if ((e = cudaMemset(s->d_live, 0, 8))) return fail(e);
        const tma_status tr = autotune_rollout(s);
        if (tr != TMA_OK) {
            free_all(s);
            delete s;
            return tr;
        }
    } catch (const std::bad_alloc &) {
        if (s) {
            free_all(s);
            delete s;
        }
        return TMA_ERR_OOM;
    }
    *out = s;
    return TMA_OK;
}

static void release_events(tma_solver *s)
{
    for (auto &p : s->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    s->pending.clear();
    for (auto e : s->event_pool) cudaEventDestroy(e);
    s->event_pool.clear();
}

void tma_destroy(tma_solver *s)
{
    if (!s) return;
    release_events(s);
    free_all(s);
    delete s;
}

tma_status tma_get_tuning(tma_solver *s, int32_t *variant, int32_t *n_timed, int32_t *h_variants,
                          float *h_ms)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    if (variant) *variant = s->rollout_variant;
    if (n_timed) *n_timed = s->n_tuned;
    for (int c = 0; c < s->n_tuned; ++c) {
        if (h_variants) h_variants[c] = s->tuned_variant[c];
        if (h_ms) h_ms[c] = s->tuned_ms[c];
    }
    return TMA_OK;
}

tma_status tma_set_tuning(tma_solver *s, int32_t variant)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    int cand[kMaxRolloutVariants];
    const int n = rollout_variants(s->P, cand);
    for (int c = 0; c < n; ++c)
        if (cand[c] == variant) {
            s->rollout_variant = variant;
            return TMA_OK;
        }
    return TMA_ERR_INVALID_ARG;
}

tma_status tma_get_grad_tuning(tma_solver *s, int32_t *variant, int32_t *n_timed,
                               int32_t *h_variants, float *h_ms)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    if (variant) *variant = s->grad_variant;
    if (n_timed) *n_timed = s->n_grad_tuned;
    for (int c = 0; c < s->n_grad_tuned; ++c) {
        if (h_variants) h_variants[c] = s->grad_tuned_variant[c];
        if (h_ms) h_ms[c] = s->grad_tuned_ms[c];
    }
    return TMA_OK;
}

tma_status tma_profile_enable(tma_solver *s, int on)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    s->prof = on != 0;
    return TMA_OK;
}

tma_status tma_profile_read(tma_solver *s, tma_profile *h_out, int reset)
{
    if (!s || !h_out) return TMA_ERR_INVALID_ARG;
    for (auto &p : s->pending) {
        TMA_CUDA(cudaEventSynchronize(p.b));
        float ms = 0.0f;
        TMA_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        s->prof_ms[p.stage] += ms;
        s->prof_n[p.stage] += 1;
        s->event_pool.push_back(p.a);
        s->event_pool.push_back(p.b);
    }
    s->pending.clear();
    for (int k = 0; k < TMA_N_STAGES; ++k) {
        h_out->ms[k] = s->prof_ms[k];
        h_out->launches[k] = s->prof_n[k];
        if (reset) {
            s->prof_ms[k] = 0.0;
            s->prof_n[k] = 0;
        }
    }
    return TMA_OK;
}

tma_status tma_set_state(tma_solver *s, const tma_state *h_x0, uint32_t mpc_step, tma_stream_t stream)
{
    if (!s || mpc_step > 0xFFFF) return TMA_ERR_INVALID_ARG;
    if (h_x0) {
        for (int i = 0; i < s->prob.N; ++i)
            if (!(h_x0[i].v > 0) || !(h_x0[i].m > 0)) return TMA_ERR_INVALID_ARG;
        for (int i = 0; i < s->prob.N; ++i) s->aircraft[i].x0 = h_x0[i];
        derive(s);   // departure altitude normalisation depends on the initial altitude
    }
    s->mpc_step = mpc_step;
    if (h_x0) {
        DynState d;
        upload_x0(s, d);
        TMA_CUDA(cudaMemcpyAsync(s->d_dyn, &d, sizeof d, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    } else {
        // keep the device state (it may have been advanced by tma_plant_step)
        TMA_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(s->d_dyn) + offsetof(DynState, mpc_step),
                                 &mpc_step, sizeof mpc_step, cudaMemcpyHostToDevice,
                                 (cudaStream_t)stream));
    }
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    s->wind_ready = false;
    return TMA_OK;
}

static tma_status gen_wind(tma_solver *s, cudaStream_t st);

// Choose the rollout kernel's launch-bound variant by timing every valid
// candidate on this solver's workload (uniform initial controls, at most 8192
// particles, all wind samples); the choice is cached per device, aircraft
// count, problem kind and workload size class for the life of the process.
static tma_status autotune_rollout(tma_solver *s)
{
    int cand[kMaxRolloutVariants];
    const int nc = rollout_variants(s->P, cand);
    s->rollout_variant = cand[0];
    s->n_tuned = 0;
    if (nc <= 1) return TMA_OK;
    const std::string key = tune_key(s);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->rollout_variant = it->second;
            return TMA_OK;
        }
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // time on an idle device: work still running on other streams (the caller's
    // own kernels) would make a slower variant look faster
    TMA_CUDA(cudaDeviceSynchronize());
    TMA_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(st);
    };
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e);
    }
    tma_status r = gen_wind(s, st);
    const int64_t Lp = std::min<int64_t>(s->prob.L, 8192);
    float lo[3], hi[3], sg[3];
    ctrl_f(s->prob, lo, hi, sg);
    if (r == TMA_OK) {
        e = launch_init_controls(s->P, s->d_dyn, lo, hi, s->d_u[0], Lp, st);
        if (e == cudaSuccess)
            e = time_rollout_variants(s->P, s->d_dyn, s->d_u[0], s->d_W, Lp, s->d_cost_ms, st, e0, e1,
                                      &s->rollout_variant, &s->n_tuned, s->tuned_variant, s->tuned_ms);
        if (e != cudaSuccess) r = cuda_fail(e);
    }
    cleanup();
    if (r == TMA_OK) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = s->rollout_variant;
    }
    return r;
}

static tma_status gen_wind(tma_solver *s, cudaStream_t st)
{
    StageTimer t(s, 0, st);
    TMA_CUDA(launch_wind_normals_ar(s->wind, s->d_dyn, s->d_Btmp, st));
    TMA_CUDA(launch_wind_gemm(s->wind, s->d_Lxy, s->lda, s->d_Btmp, s->d_W, st));
    s->wind_ready = true;
    return TMA_OK;
}

tma_status tma_wind_field(tma_solver *s, float *d_W, tma_stream_t stream)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    tma_status r = gen_wind(s, st);
    if (r != TMA_OK) return r;
    if (d_W) {
        // the solver keeps float4 (own value, value one level up) per node; copy the own values
        const size_t rows = (size_t)s->prob.M * s->prob.H * s->P.P;
        TMA_CUDA(cudaMemcpy2DAsync(d_W, 8, s->d_W, 16, 8, rows, cudaMemcpyDeviceToDevice, st));
    }
    return TMA_OK;
}

static tma_status rollout_into(tma_solver *s, const float *d_u, int64_t L, int32_t J, float *cbar,
                               float *cbar_soft, cudaStream_t st, bool reset_live)
{
    // wind mode 1 draws each particle's field inside the rollout: no shared field
    if (!s->wind_ready && s->P.wind_mode == 0) {
        tma_status r = gen_wind(s, st);
        if (r != TMA_OK) return r;
    }
    const bool soft = cbar_soft != nullptr;
    const ProblemC Pj = problem_at(s, J);
    if (reset_live) TMA_CUDA(cudaMemsetAsync(s->d_live, 0, 8, st));
    {
        StageTimer t(s, 2, st);
        TMA_CUDA(launch_rollout(Pj, s->d_dyn, d_u, s->d_W, L, J, s->d_cost_ms,
                                soft ? s->d_cost_ms_soft : nullptr, s->d_live, st,
                                s->rollout_variant));
    }
    {
        StageTimer t(s, 3, st);
        TMA_CUDA(launch_sample_mean(s->d_cost_ms, L, Pj.M, s->prob.N, cbar, st));
        if (soft)
            TMA_CUDA(launch_sample_mean(s->d_cost_ms_soft, L, Pj.M, s->prob.N, cbar_soft, st));
    }
    s->last_L = L;
    s->last_M = Pj.M;
    return TMA_OK;
}

tma_status tma_rollout_cost(tma_solver *s, const float *d_u, int64_t L, int32_t J, float *d_cbar,
                            float *d_cbar_soft, tma_stream_t stream)
{
    if (!s || !d_u || !d_cbar || L < 0 || L > s->prob.L || J < 0 || J > 0xFFFF)
        return TMA_ERR_INVALID_ARG;
    if (d_cbar_soft && s->prob.sep_mode == 0) return TMA_ERR_INVALID_ARG;
    return rollout_into(s, d_u, L, J, d_cbar, d_cbar_soft, (cudaStream_t)stream, true);
}

tma_status tma_sample_costs(tma_solver *s, float *d_out, int64_t L, int soft, tma_stream_t stream)
{
    if (!s || !d_out || L < 0 || L > s->last_L) return TMA_ERR_INVALID_ARG;
    const float *src = soft ? s->d_cost_ms_soft : s->d_cost_ms;
    if (!src) return TMA_ERR_INVALID_ARG;
    // the buffer holds [M][N][last_L]; copy out the first L particles of each row
    // of the last call's samples, and NaN for the samples it did not use
    TMA_CUDA(cudaMemcpy2DAsync(d_out, (size_t)L * 4, src, (size_t)s->last_L * 4, (size_t)L * 4,
                               (size_t)s->last_M * s->prob.N, cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
    if (s->last_M < s->prob.M)
        TMA_CUDA(cudaMemsetAsync(d_out + (size_t)s->last_M * s->prob.N * L, 0xFF,
                                 (size_t)(s->prob.M - s->last_M) * s->prob.N * L * 4,
                                 (cudaStream_t)stream));
    return TMA_OK;
}

tma_status tma_live_steps(tma_solver *s, uint64_t *h_live, tma_stream_t stream)
{
    if (!s || !h_live) return TMA_ERR_INVALID_ARG;
    unsigned long long v = 0;
    TMA_CUDA(cudaMemcpyAsync(&v, s->d_live, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *h_live = v;
    return TMA_OK;
}

tma_status tma_move(tma_solver *s, const float *d_u, const int32_t *d_anc, int64_t L, int32_t J,
                    float *d_u_out, tma_stream_t stream)
{
    return tma_move_to(s, d_u, L, d_anc, L, J, d_u_out, stream);
}

tma_status tma_move_to(tma_solver *s, const float *d_u, int64_t L_in, const int32_t *d_anc, int64_t L,
                       int32_t J, float *d_u_out, tma_stream_t stream)
{
    if (!s || !d_u || !d_anc || !d_u_out || d_u == d_u_out || L < 0 || L > s->prob.L || L_in < 0 ||
        L_in > s->prob.L || (L > 0 && L_in == 0) || J < 0 || J > 0xFFFF)
        return TMA_ERR_INVALID_ARG;
    float lo[3], hi[3], sg[3];
    ctrl_f(s->prob, lo, hi, sg);
    TMA_CUDA(launch_move(s->P, s->d_dyn, lo, hi, sg, d_u, d_anc, L, L_in, J, d_u_out,
                         (cudaStream_t)stream, s->d_err));
    return TMA_OK;
}

tma_status tma_init_controls(tma_solver *s, float *d_u, int64_t L, tma_stream_t stream)
{
    if (!s || !d_u || L < 0 || L > s->prob.L) return TMA_ERR_INVALID_ARG;
    float lo[3], hi[3], sg[3];
    ctrl_f(s->prob, lo, hi, sg);
    TMA_CUDA(launch_init_controls(s->P, s->d_dyn, lo, hi, d_u, L, (cudaStream_t)stream));
    return TMA_OK;
}

// ------------------------------------------------------------------ gradient

// Ranges of wind samples per gradient block: enough blocks for about two
// waves of the device, at most one range per sample.
static int grad_chunks(tma_solver *s, int64_t L, int variant, int M)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (rollout_grad_occupancy(s->prob.N, variant, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    const long long tiles = (L + kTileParticles - 1) / kTileParticles;
    const long long want = 2LL * std::max(sms, 1) * per_sm;
    long long c = (want + tiles - 1) / std::max(tiles, 1LL);
    return (int)std::max(1LL, std::min<long long>(c, M));
}

static tma_status ensure_grad_scratch(tma_solver *s, int64_t L, int nchunk)
{
    const tma_problem &p = s->prob;
    if (!s->d_gcost_ms) {
        cudaError_t e = alloc(&s->d_gcost_ms, (size_t)p.M * p.N * p.L * sizeof(float));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : record_cuda_error(e);
    }
    const size_t need = (size_t)nchunk * L * p.N * p.S * 3;
    if (need > s->gpart_elems) {
        if (s->d_gpart) cudaFree(s->d_gpart);
        s->d_gpart = nullptr;
        s->gpart_elems = 0;
        cudaError_t e = alloc(&s->d_gpart, need * sizeof(float));
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : record_cuda_error(e);
        s->gpart_elems = need;
    }
    return TMA_OK;
}

// Choose the gradient kernel's launch-bound variant by timing every valid
// candidate on this solver's workload (uniform controls, at most 4096
// particles); cached per device and aircraft count.  The variants compute
// the same arithmetic.
static tma_status autotune_grad(tma_solver *s)
{
    if (s->grad_variant >= 0) return TMA_OK;
    int cand[8];
    const int nc = rollout_grad_variants(s->prob.N, cand);
    s->grad_variant = cand[0];
    s->n_grad_tuned = 0;
    if (nc <= 1) return TMA_OK;
    const std::string key = tune_key(s) + "|grad";
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->grad_variant = it->second;
            return TMA_OK;
        }
    }
    const int64_t Lp = std::min<int64_t>(s->prob.L, 4096);
    const size_t nu = (size_t)Lp * s->prob.N * s->prob.S * 3;
    int max_chunks = 1;
    for (int c = 0; c < nc; ++c) max_chunks = std::max(max_chunks, grad_chunks(s, Lp, cand[c], s->prob.M));
    tma_status r = ensure_grad_scratch(s, Lp, max_chunks);
    if (r != TMA_OK) return r;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float *d_u = nullptr;
    // time on an idle device: work still running on other streams (the caller's
    // own kernels) would make a slower variant look faster
    TMA_CUDA(cudaDeviceSynchronize());
    TMA_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = alloc(&d_u, nu * sizeof(float));
    float lo[3], hi[3], sg[3];
    ctrl_f(s->prob, lo, hi, sg);
    if (e == cudaSuccess && !s->wind_ready) {
        r = gen_wind(s, st);
        if (r != TMA_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = launch_init_controls(s->P, s->d_dyn, lo, hi, d_u, Lp, st);
    float best = 1e30f;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        const int nch = grad_chunks(s, Lp, cand[c], s->prob.M);
        // one untimed launch, then two timed
        e = launch_rollout_grad(s->P, s->d_dyn, d_u, s->d_W, Lp, 0, nch, s->d_gcost_ms, s->d_gpart,
                                nullptr, nullptr, nullptr, st, cand[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
            e = launch_rollout_grad(s->P, s->d_dyn, d_u, s->d_W, Lp, 0, nch, s->d_gcost_ms,
                                    s->d_gpart, nullptr, nullptr, nullptr, st, cand[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) break;
        s->grad_tuned_variant[s->n_grad_tuned] = cand[c];
        s->grad_tuned_ms[s->n_grad_tuned] = ms / 2.0f;
        ++s->n_grad_tuned;
        if (ms < best) {
            best = ms;
            s->grad_variant = cand[c];
        }
    }
    if (d_u) cudaFree(d_u);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (r != TMA_OK) return r;
    if (e != cudaSuccess) return cuda_fail(e);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = s->grad_variant;
    return TMA_OK;
}

static tma_status grad_into(tma_solver *s, const float *d_u, int64_t L, int32_t J, float *cost,
                            float *grad, float *cbar, cudaStream_t st)
{
    if (!s->wind_ready) {
        tma_status r = gen_wind(s, st);
        if (r != TMA_OK) return r;
    }
    tma_status r = autotune_grad(s);
    if (r != TMA_OK) return r;
    const ProblemC Pj = problem_at(s, J);
    const int nchunk = grad_chunks(s, L, s->grad_variant, Pj.M);
    r = ensure_grad_scratch(s, L, nchunk);
    if (r != TMA_OK) return r;
    StageTimer t(s, 8, st);
    TMA_CUDA(launch_rollout_grad(Pj, s->d_dyn, d_u, s->d_W, L, J, nchunk, s->d_gcost_ms,
                                 s->d_gpart, cost, grad, cbar, st, s->grad_variant));
    return TMA_OK;
}

extern "C" tma_status tma_set_wind_stream(tma_solver *s, uint32_t stream)
{
    if (!s || (stream != 3u && stream != 8u)) return TMA_ERR_INVALID_ARG;
    s->wind.stream = stream;
    s->wind_ready = false;
    return TMA_OK;
}

extern "C" tma_status tma_rollout_grad(tma_solver *s, const float *d_u, int64_t L, int32_t J,
                                       float *d_cost, float *d_grad, float *d_cbar_soft,
                                       tma_stream_t stream)
{
    if (!s || !d_u || !d_cost || !d_grad || L < 0 || L > s->prob.L || J < 0 || J > 0xFFFF)
        return TMA_ERR_INVALID_ARG;
    if (s->prob.H > TMA_MAX_GRAD_HORIZON || s->prob.wind_mode != 0 || s->prob.rolling != 0)
        return TMA_ERR_UNSUPPORTED;
    if (L == 0) return TMA_OK;
    return grad_into(s, d_u, L, J, d_cost, d_grad, d_cbar_soft, (cudaStream_t)stream);
}

// ------------------------------------------------------- accepted moves

static MhParams mh_params(const tma_solver *s, int kind)
{
    MhParams h;
    std::memset(&h, 0, sizeof h);
    h.N = s->prob.N;
    h.S = s->prob.S;
    h.langevin = kind == TMA_MOVE_MALA;
    ctrl_f(s->prob, h.lo, h.hi, h.sigma);
    h.key0 = s->P.key0;
    h.key1 = s->P.key1;
    return h;
}

static tma_status ensure_mh_scalars(tma_solver *s)
{
    if (s->d_eps) return TMA_OK;
    const size_t nj = (size_t)std::max(s->prob.J_max, 1);
    cudaError_t e = alloc(&s->d_eps, 2 * sizeof(double));
    if (e == cudaSuccess) e = alloc(&s->d_nacc, sizeof(unsigned int));
    if (e == cudaSuccess) e = alloc(&s->d_acc_hist, nj * sizeof(unsigned int));
    if (e == cudaSuccess) e = alloc(&s->d_eps_hist, nj * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(s->d_nacc, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(s->d_acc_hist, 0, nj * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(s->d_eps_hist, 0, nj * sizeof(double));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : record_cuda_error(e);
    return TMA_OK;
}

extern "C" tma_status tma_set_move(tma_solver *s, int32_t kind, double eps0)
{
    if (!s || kind < TMA_MOVE_PAPER || kind > TMA_MOVE_MALA) return TMA_ERR_INVALID_ARG;
    if (kind == TMA_MOVE_PAPER) {
        s->move_kind = kind;
        return TMA_OK;
    }
    if (!(eps0 > 0.0) || !std::isfinite(eps0) || s->prob.sep_mode == 0) return TMA_ERR_INVALID_ARG;
    if (kind == TMA_MOVE_MALA &&
        (s->prob.H > TMA_MAX_GRAD_HORIZON || s->prob.wind_mode != 0 || s->prob.rolling != 0))
        return TMA_ERR_UNSUPPORTED;
    tma_status r = ensure_mh_scalars(s);
    if (r != TMA_OK) return r;
    const tma_problem &p = s->prob;
    const size_t nu = (size_t)p.L * p.N * p.S * 3, nc = (size_t)p.N * p.L;
    cudaError_t e = cudaSuccess;
    if (!s->d_u_prop) e = alloc(&s->d_u_prop, nu * 4);
    if (e == cudaSuccess && !s->d_cbar0) e = alloc(&s->d_cbar0, nc * 4);
    if (e == cudaSuccess && !s->d_cbar1) e = alloc(&s->d_cbar1, nc * 4);
    if (e == cudaSuccess && !s->d_inbox) e = alloc(&s->d_inbox, (size_t)p.L);
    if (kind == TMA_MOVE_MALA) {
        if (e == cudaSuccess && !s->d_grad0) e = alloc(&s->d_grad0, nu * 4);
        if (e == cudaSuccess && !s->d_grad1) e = alloc(&s->d_grad1, nu * 4);
        if (e == cudaSuccess && !s->d_cost0) e = alloc(&s->d_cost0, (size_t)p.L * 4);
        if (e == cudaSuccess && !s->d_cost1) e = alloc(&s->d_cost1, (size_t)p.L * 4);
    }
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : record_cuda_error(e);
    if (kind == TMA_MOVE_MALA) {
        r = autotune_grad(s);
        if (r == TMA_OK) r = ensure_grad_scratch(s, p.L, grad_chunks(s, p.L, s->grad_variant, p.M));
        if (r != TMA_OK) return r;
    }
    s->move_kind = kind;
    s->eps0 = eps0;
    return TMA_OK;
}

static bool valid_mh(const tma_solver *s, int64_t L, int32_t J, double kappa, double eps, int kind)
{
    return s && L >= 0 && L <= s->prob.L && J >= 0 && J <= 0xFFFF && std::isfinite(kappa) &&
           kappa >= 0.0 && eps > 0.0 && std::isfinite(eps) &&
           (kind == TMA_MOVE_RWMH || kind == TMA_MOVE_MALA);
}

extern "C" tma_status tma_mh_propose(tma_solver *s, const float *d_u, const float *d_grad, int64_t L,
                                     int32_t J, double kappa, double eps, int32_t kind,
                                     float *d_u_prop, uint8_t *d_inbox, tma_stream_t stream)
{
    if (!valid_mh(s, L, J, kappa, eps, kind) || !d_u || !d_u_prop || !d_inbox ||
        (kind == TMA_MOVE_MALA && !d_grad))
        return TMA_ERR_INVALID_ARG;
    if (L == 0) return TMA_OK;
    tma_status r = ensure_mh_scalars(s);
    if (r != TMA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    TMA_CUDA(cudaMemcpyAsync(s->d_eps + 1, &eps, sizeof(double), cudaMemcpyHostToDevice, st));
    TMA_CUDA(launch_mh_propose(mh_params(s, kind), s->d_dyn, d_u, d_grad, L, J, (float)kappa,
                               s->d_eps + 1, d_u_prop, d_inbox, st));
    TMA_CUDA(cudaStreamSynchronize(st));     // the step lives in a stack variable
    return TMA_OK;
}

extern "C" tma_status tma_mh_accept(tma_solver *s, const float *d_u, const float *d_u_prop,
                                    const float *d_cbar, const float *d_cbar_prop,
                                    const float *d_grad, const float *d_grad_prop,
                                    const uint8_t *d_inbox, int64_t L, int32_t J, double kappa,
                                    double eps, int32_t kind, float *d_u_out, uint8_t *d_accepted,
                                    tma_stream_t stream)
{
    if (!valid_mh(s, L, J, kappa, eps, kind) || !d_u || !d_u_prop || !d_cbar || !d_cbar_prop ||
        !d_inbox || !d_u_out || (kind == TMA_MOVE_MALA && (!d_grad || !d_grad_prop)))
        return TMA_ERR_INVALID_ARG;
    if (L == 0) return TMA_OK;
    tma_status r = ensure_mh_scalars(s);
    if (r != TMA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    TMA_CUDA(cudaMemcpyAsync(s->d_eps + 1, &eps, sizeof(double), cudaMemcpyHostToDevice, st));
    TMA_CUDA(launch_mh_accept(mh_params(s, kind), s->d_dyn, d_u, d_u_prop, d_cbar, d_cbar_prop,
                              d_grad, d_grad_prop, d_inbox, L, J, (float)kappa, s->d_eps + 1,
                              d_u_out, nullptr, d_accepted, nullptr, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    return TMA_OK;
}

extern "C" tma_status tma_mh_stats(tma_solver *s, uint32_t *h_accepts, double *h_eps, int32_t n,
                                   tma_stream_t stream)
{
    if (!s || n < 0 || n > std::max(s->prob.J_max - 1, 0)) return TMA_ERR_INVALID_ARG;
    if (n == 0) return TMA_OK;
    if (!s->d_acc_hist) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (h_accepts)
        TMA_CUDA(cudaMemcpyAsync(h_accepts, s->d_acc_hist, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    if (h_eps)
        TMA_CUDA(cudaMemcpyAsync(h_eps, s->d_eps_hist, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    return TMA_OK;
}

// One accepted move of all particles at iteration J: u_cur holds the resampled
// particles on entry and the moved ones on exit.
static tma_status mh_move(tma_solver *s, float *u_cur, int J, int64_t L, cudaStream_t st)
{
    const tma_problem &p = s->prob;
    const int kind = s->move_kind;
    const float kappa = (float)exponent_of(p, J);
    const MhParams h = mh_params(s, kind);
    if (kind == TMA_MOVE_MALA) {
        tma_status r = grad_into(s, u_cur, L, J, s->d_cost0, s->d_grad0, s->d_cbar0, st);
        if (r != TMA_OK) return r;
    } else {
        tma_status r = rollout_into(s, u_cur, L, J, s->d_cbar, s->d_cbar0, st, false);
        if (r != TMA_OK) return r;
    }
    {
        StageTimer t(s, 9, st);
        TMA_CUDA(launch_mh_propose(h, s->d_dyn, u_cur, s->d_grad0, L, J, kappa, s->d_eps,
                                   s->d_u_prop, s->d_inbox, st));
    }
    if (kind == TMA_MOVE_MALA) {
        tma_status r = grad_into(s, s->d_u_prop, L, J, s->d_cost1, s->d_grad1, s->d_cbar1, st);
        if (r != TMA_OK) return r;
    } else {
        tma_status r = rollout_into(s, s->d_u_prop, L, J, s->d_cbar, s->d_cbar1, st, false);
        if (r != TMA_OK) return r;
    }
    {
        StageTimer t(s, 9, st);
        TMA_CUDA(launch_mh_accept(h, s->d_dyn, u_cur, s->d_u_prop, s->d_cbar0, s->d_cbar1,
                                  s->d_grad0, s->d_grad1, s->d_inbox, L, J, kappa, s->d_eps,
                                  u_cur, nullptr, nullptr, s->d_nacc, st));
        TMA_CUDA(launch_mh_adapt(s->d_eps, s->d_nacc, s->d_acc_hist, s->d_eps_hist, J, L, st));
    }
    return TMA_OK;
}

static tma_status solve_device(tma_solver *s, cudaStream_t st, bool *degenerate)
{
    const tma_problem &p = s->prob;
    float lo[3], hi[3], sg[3];
    ctrl_f(p, lo, hi, sg);
    tma_status r = gen_wind(s, st);
    if (r != TMA_OK) return r;
    TMA_CUDA(cudaMemsetAsync(s->d_flags, 0, 4, st));
    TMA_CUDA(cudaMemsetAsync(s->d_live, 0, 8, st));
    if (s->move_kind != TMA_MOVE_PAPER) {
        TMA_CUDA(cudaMemcpyAsync(s->d_eps, &s->eps0, sizeof(double), cudaMemcpyHostToDevice, st));
        TMA_CUDA(cudaMemsetAsync(s->d_nacc, 0, sizeof(unsigned int), st));
    }
    {
        StageTimer t(s, 1, st);
        TMA_CUDA(launch_init_controls(s->P, s->d_dyn, lo, hi, s->d_u[0], particles_of(s, 0), st));
    }
    int cur = 0;
    const bool use_soft = p.sep_mode == 1;
    float *cb = use_soft ? s->d_cbar_soft : s->d_cbar;
    for (int J = 0; J < p.J_max; ++J) {
        // every stage of iteration J sees its particles packed: [L_J] or [N][L_J]
        const int64_t Lj = particles_of(s, J);
        r = rollout_into(s, s->d_u[cur], Lj, J, s->d_cbar, p.sep_mode != 0 ? s->d_cbar_soft : nullptr,
                         st, false);
        if (r != TMA_OK) return r;
        if (J < p.J_max - 1) {
            const int64_t Ln = particles_of(s, J + 1);
            {
                StageTimer t(s, 4, st);
                TMA_CUDA(launch_lse(cb, p.N, Lj, exponent_of(p, J), s->d_wtilde, nullptr, nullptr,
                                    s->d_work, st, resample_partials(res_work(s))));
            }
            {
                StageTimer t(s, 5, st);
                TMA_CUDA(launch_resample(s->d_wtilde, p.N, Lj, Ln, s->P.key0, s->P.key1, (uint32_t)J,
                                         dyn_mpc(s), 0u, s->d_anc, res_work(s), s->d_flags, st, nullptr,
                                         nullptr, true));
            }
            {
                StageTimer t(s, 6, st);
                // the accepted moves start from the resampled particles themselves
                const float zero[3] = {0.0f, 0.0f, 0.0f};
                TMA_CUDA(launch_move(s->P, s->d_dyn, lo, hi, s->move_kind == TMA_MOVE_PAPER ? sg : zero,
                                     s->d_u[cur], s->d_anc, Ln, Lj, J, s->d_u[cur ^ 1], st, s->d_err));
            }
            cur ^= 1;
            if (s->move_kind != TMA_MOVE_PAPER) {
                r = mh_move(s, s->d_u[cur], J, Ln, st);
                if (r != TMA_OK) return r;
            }
        }
    }
    s->cur_u = cur;
    {
        StageTimer t(s, 7, st);
        const int64_t Lf = particles_of(s, p.J_max - 1);
        TMA_CUDA(launch_select(cb, p.N, Lf, s->d_best, s->d_best_sum, s->d_ninf, s->d_work, st));
        TMA_CUDA(launch_gather_best(s->d_u[cur], s->d_best, p.N * p.S * 3, s->d_best_u, st,
                                    s->d_flags, s->d_ninf, s->d_err));
    }
    (void)degenerate;
    return TMA_OK;
}

tma_status tma_solve(tma_solver *s, float *d_best_u, double *h_best_cost, tma_stream_t stream)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    bool deg = false;
    tma_status r = solve_device(s, st, &deg);
    if (r != TMA_OK) return r;
    if (d_best_u)
        TMA_CUDA(cudaMemcpyAsync(d_best_u, s->d_best_u, (size_t)s->prob.N * s->prob.S * 3 * 4,
                                 cudaMemcpyDeviceToDevice, st));
    if (h_best_cost) {
        unsigned int flags = 0;
        TMA_CUDA(cudaMemcpyAsync(h_best_cost, s->d_best_sum, 8, cudaMemcpyDeviceToHost, st));
        TMA_CUDA(cudaMemcpyAsync(&flags, s->d_flags, 4, cudaMemcpyDeviceToHost, st));
        TMA_CUDA(cudaStreamSynchronize(st));
        if (flags & 1u) return TMA_WARN_DEGENERATE;
    }
    return TMA_OK;
}

tma_status tma_solve_host(tma_solver *s, const tma_state *h_x0, uint32_t mpc_step, float *h_best_u,
                          double *h_best_cost, tma_stream_t stream)
{
    if (!s || !h_best_u) return TMA_ERR_INVALID_ARG;
    tma_status r = tma_set_state(s, h_x0, mpc_step, stream);
    if (r != TMA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    bool deg = false;
    r = solve_device(s, st, &deg);
    if (r != TMA_OK) return r;
    unsigned int flags = 0;
    double cost = 0.0;
    TMA_CUDA(cudaMemcpyAsync(h_best_u, s->d_best_u, (size_t)s->prob.N * s->prob.S * 3 * 4,
                             cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemcpyAsync(&cost, s->d_best_sum, 8, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemcpyAsync(&flags, s->d_flags, 4, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    if (h_best_cost) *h_best_cost = cost;
    return (flags & 1u) ? TMA_WARN_DEGENERATE : TMA_OK;
}

tma_status tma_get_particles(tma_solver *s, float *d_u_out, int64_t L, tma_stream_t stream)
{
    if (!s || !d_u_out || L < 0 || L > particles_of(s, s->prob.J_max - 1)) return TMA_ERR_INVALID_ARG;
    const size_t bytes = (size_t)L * s->prob.N * s->prob.S * 3 * sizeof(float);
    TMA_CUDA(cudaMemcpyAsync(d_u_out, s->d_u[s->cur_u], bytes, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return TMA_OK;
}

tma_status tma_best_index(tma_solver *s, int64_t *h_best, tma_stream_t stream)
{
    if (!s || !h_best) return TMA_ERR_INVALID_ARG;
    TMA_CUDA(cudaMemcpyAsync(h_best, s->d_best, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TMA_OK;
}

size_t tma_lse_workspace(int32_t nseg, int64_t L)
{
    return (nseg < 0 || L < 0) ? 0 : lse_workspace(nseg, L);
}

tma_status tma_lse(const float *d_cbar, int32_t nseg, int64_t L, double kappa, double *d_wtilde,
                   double *d_lmax, double *d_wsum, void *d_work, size_t work_bytes, tma_stream_t stream)
{
    if (nseg < 0 || L < 0 || L > TMA_MAX_PARTICLES || !(kappa > 0) || !std::isfinite(kappa))
        return TMA_ERR_INVALID_ARG;
    if (nseg == 0 || L == 0) {
        if (nseg > 0 && (d_lmax || d_wsum)) {
            std::vector<double> lm(nseg, -INFINITY), ws(nseg, 0.0);
            if (d_lmax) TMA_CUDA(cudaMemcpyAsync(d_lmax, lm.data(), nseg * 8, cudaMemcpyHostToDevice, (cudaStream_t)stream));
            if (d_wsum) TMA_CUDA(cudaMemcpyAsync(d_wsum, ws.data(), nseg * 8, cudaMemcpyHostToDevice, (cudaStream_t)stream));
            TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        }
        return TMA_OK;
    }
    if (!d_cbar || !d_wtilde || !d_work || work_bytes < lse_workspace(nseg, L)) return TMA_ERR_INVALID_ARG;
    TMA_CUDA(launch_lse(d_cbar, nseg, L, kappa, d_wtilde, d_lmax, d_wsum, d_work, (cudaStream_t)stream));
    return TMA_OK;
}

size_t tma_resample_workspace(int32_t nseg, int64_t L)
{
    return (nseg < 0 || L < 0) ? 0 : resample_workspace(nseg, L) + 16;
}

tma_status tma_resample(const double *d_wtilde, int32_t nseg, int64_t L, uint64_t seed,
                        uint32_t scenario_id, uint32_t J, uint32_t mpc_step, int32_t *d_anc,
                        void *d_work, size_t work_bytes, tma_stream_t stream)
{
    return tma_resample_to(d_wtilde, nseg, L, L, seed, scenario_id, J, mpc_step, d_anc, d_work,
                           work_bytes, stream);
}

tma_status tma_resample_to(const double *d_wtilde, int32_t nseg, int64_t L, int64_t L_out,
                           uint64_t seed, uint32_t scenario_id, uint32_t J, uint32_t mpc_step,
                           int32_t *d_anc, void *d_work, size_t work_bytes, tma_stream_t stream)
{
    if (nseg < 0 || L < 0 || L > TMA_MAX_PARTICLES || L_out < 0 || L_out > TMA_MAX_PARTICLES ||
        J > 0xFFFF || mpc_step > 0xFFFF || (L == 0) != (L_out == 0))
        return TMA_ERR_INVALID_ARG;
    if (nseg == 0 || L == 0) return TMA_OK;
    if (!d_wtilde || !d_anc || !d_work || work_bytes < tma_resample_workspace(nseg, L))
        return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t key = seed + (uint64_t)scenario_id * 0x9E3779B97F4A7C15ull;
    // the last 16 bytes of the workspace hold the degenerate flag
    char *base = reinterpret_cast<char *>(d_work);
    const size_t rw = resample_workspace(nseg, L);
    unsigned int *flags = reinterpret_cast<unsigned int *>(
        (reinterpret_cast<uintptr_t>(base + rw) + 3) & ~uintptr_t(3));
    TMA_CUDA(cudaMemsetAsync(flags, 0, 4, st));
    TMA_CUDA(launch_resample(d_wtilde, nseg, L, L_out, (uint32_t)key, (uint32_t)(key >> 32), J,
                             nullptr, mpc_step, d_anc, d_work, flags, st));
    unsigned int h = 0;
    TMA_CUDA(cudaMemcpyAsync(&h, flags, 4, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    return (h & 1u) ? TMA_WARN_DEGENERATE : TMA_OK;
}

size_t tma_lse_resample_workspace(int32_t nseg, int64_t L)
{
    if (nseg < 0 || L < 0) return 0;
    return (lse_workspace(nseg, L) + 255) / 256 * 256 + resample_workspace(nseg, L);
}

tma_status tma_lse_resample(const float *d_cbar, int32_t nseg, int64_t L, int64_t L_out, double kappa,
                            uint64_t seed, uint32_t scenario_id, uint32_t J, uint32_t mpc_step,
                            double *d_wtilde, int32_t *d_anc, uint32_t *d_degenerate, void *d_work,
                            size_t work_bytes, tma_stream_t stream)
{
    if (nseg < 0 || L < 0 || L > TMA_MAX_PARTICLES || L_out < 0 || L_out > TMA_MAX_PARTICLES ||
        J > 0xFFFF || mpc_step > 0xFFFF || (L == 0) != (L_out == 0) || !(kappa > 0) ||
        !std::isfinite(kappa))
        return TMA_ERR_INVALID_ARG;
    if (nseg == 0 || L == 0) return TMA_OK;
    if (!d_cbar || !d_wtilde || !d_anc || !d_work || work_bytes < tma_lse_resample_workspace(nseg, L))
        return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t key = seed + (uint64_t)scenario_id * 0x9E3779B97F4A7C15ull;
    void *rwork = static_cast<char *>(d_work) + (lse_workspace(nseg, L) + 255) / 256 * 256;
    TMA_CUDA(launch_lse(d_cbar, nseg, L, kappa, d_wtilde, nullptr, nullptr, d_work, st,
                        resample_partials(rwork)));
    TMA_CUDA(launch_resample(d_wtilde, nseg, L, L_out, (uint32_t)key, (uint32_t)(key >> 32), J, nullptr,
                             mpc_step, d_anc, rwork, d_degenerate, st, nullptr, nullptr, true));
    return TMA_OK;
}

size_t tma_select_workspace(int64_t L) { return L < 0 ? 0 : select_workspace(L); }

tma_status tma_select(const float *d_cbar, int32_t N, int64_t L, int64_t *d_best, double *d_best_sum,
                      int32_t *d_ninf, void *d_work, size_t work_bytes, tma_stream_t stream)
{
    if (N < 1 || L < 1 || !d_cbar || !d_best || !d_work || work_bytes < select_workspace(L))
        return TMA_ERR_INVALID_ARG;
    TMA_CUDA(launch_select(d_cbar, N, L, d_best, d_best_sum, d_ninf, d_work, (cudaStream_t)stream));
    return TMA_OK;
}


// --------------------------------------------------------------- MPC plant

// The plant step of Fig. 1, stream-ordered (no sync).
static tma_status plant_async(tma_solver *s, const float *d_u, cudaStream_t st)
{
    if (!s->d_probs1) {
        cudaError_t e = alloc(&s->d_probs1, sizeof(ProblemC));
        if (!e) e = alloc(&s->d_scen1, sizeof(BatchScen));
        if (!e) e = alloc(&s->d_seg_scen1, sizeof(int) * TMA_MAX_AIRCRAFT);
        if (!e) e = cudaMemset(s->d_seg_scen1, 0, sizeof(int) * TMA_MAX_AIRCRAFT);
        if (e) return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : cuda_fail(e);
    }
    if (!s->wind_ready && s->P.wind_mode == 0) {
        tma_status r = gen_wind(s, st);
        if (r != TMA_OK) return r;
    }
    BatchScen sc;
    std::memset(&sc, 0, sizeof sc);
    sc.N = s->prob.N;
    TMA_CUDA(cudaMemcpyAsync(s->d_probs1, &s->P, sizeof(ProblemC), cudaMemcpyHostToDevice, st));
    TMA_CUDA(cudaMemcpyAsync(s->d_scen1, &sc, sizeof sc, cudaMemcpyHostToDevice, st));
    TMA_CUDA(launch_plant_step(s->d_probs1, s->d_scen1, s->d_seg_scen1, s->prob.N, 1, s->d_dyn,
                               s->d_W, d_u, s->prob.S, st));
    s->mpc_step += 1;
    s->wind_ready = false;
    return TMA_OK;
}

tma_status tma_plant_step(tma_solver *s, const float *d_u, tma_stream_t stream)
{
    if (!s || !d_u) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    tma_status r = plant_async(s, d_u, st);
    if (r != TMA_OK) return r;
    TMA_CUDA(cudaStreamSynchronize(st));
    return TMA_OK;
}

tma_status tma_mpc_run(tma_solver *s, int32_t n_steps, tma_state *h_traj, double *h_costs,
                       tma_stream_t stream)
{
    if (!s || n_steps < 0 || (n_steps > 0 && !h_traj) ||
        (uint64_t)s->mpc_step + (uint64_t)n_steps > 0xFFFFu)
        return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<DynState> states((size_t)n_steps);
    std::vector<double> costs((size_t)n_steps);
    unsigned int deg = 0;
    for (int t = 0; t < n_steps; ++t) {
        bool d = false;
        tma_status r = solve_device(s, st, &d);
        if (r != TMA_OK) return r;
        TMA_CUDA(cudaMemcpyAsync(&costs[t], s->d_best_sum, 8, cudaMemcpyDeviceToHost, st));
        unsigned int flags = 0;
        TMA_CUDA(cudaMemcpyAsync(&flags, s->d_flags, 4, cudaMemcpyDeviceToHost, st));
        r = plant_async(s, s->d_best_u, st);
        if (r != TMA_OK) return r;
        TMA_CUDA(cudaMemcpyAsync(&states[t], s->d_dyn, sizeof(DynState), cudaMemcpyDeviceToHost, st));
        TMA_CUDA(cudaStreamSynchronize(st));
        deg |= flags & 1u;
    }
    for (int t = 0; t < n_steps; ++t) {
        for (int i = 0; i < s->prob.N; ++i) {
            tma_state &x = h_traj[(size_t)t * s->prob.N + i];
            x.x = states[t].x0[i][0];
            x.y = states[t].x0[i][1];
            x.z = states[t].x0[i][2];
            x.v = states[t].x0[i][3];
            x.chi = states[t].x0[i][4];
            x.m = states[t].x0[i][5];
        }
        if (h_costs) h_costs[t] = costs[t];
    }
    return deg ? TMA_WARN_DEGENERATE : TMA_OK;
}

tma_status tma_get_error(tma_solver *s, uint32_t *h_err, tma_stream_t stream)
{
    if (!s || !h_err) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    TMA_CUDA(cudaMemcpyAsync(h_err, s->d_err, 4, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemsetAsync(s->d_err, 0, 4, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    return (*h_err & TMA_DEVERR_BOUNDS) ? TMA_ERR_BOUNDS : TMA_OK;
}

tma_status tma_get_state(tma_solver *s, tma_state *h_x, uint32_t *h_mpc, tma_stream_t stream)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    DynState d;
    TMA_CUDA(cudaMemcpyAsync(&d, s->d_dyn, sizeof d, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; h_x && i < s->prob.N; ++i) {
        h_x[i].x = d.x0[i][0];
        h_x[i].y = d.x0[i][1];
        h_x[i].z = d.x0[i][2];
        h_x[i].v = d.x0[i][3];
        h_x[i].chi = d.x0[i][4];
        h_x[i].m = d.x0[i][5];
    }
    if (h_mpc) *h_mpc = d.mpc_step;
    return TMA_OK;
}

tma_status tma_set_finished(tma_solver *s, uint32_t mask, tma_stream_t stream)
{
    if (!s || (s->prob.N < 32 && (mask >> s->prob.N) != 0u)) return TMA_ERR_INVALID_ARG;
    TMA_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(s->d_dyn) + offsetof(DynState, finished), &mask,
                             sizeof mask, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TMA_OK;
}

tma_status tma_get_status(tma_solver *s, int32_t *h_status, uint32_t *h_finished, tma_stream_t stream)
{
    if (!s) return TMA_ERR_INVALID_ARG;
    DynState d;
    TMA_CUDA(cudaMemcpyAsync(&d, s->d_dyn, sizeof d, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    for (int i = 0; h_status && i < s->prob.N; ++i) {
        if ((d.finished >> i) & 1u) h_status[i] = 2;
        else if (s->prob.rolling && (int64_t)s->aircraft[i].t_enter > (int64_t)d.mpc_step) h_status[i] = 0;
        else h_status[i] = 1;
    }
    if (h_finished) *h_finished = d.finished;
    return TMA_OK;
}

// ------------------------------------------------------------------ batches

static void batch_free(tma_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int q = 0; q < tma_batch::kAuxStreams; ++q) {
        if (b->aux[q]) cudaStreamDestroy(b->aux[q]);
        if (b->join_ev[q]) cudaEventDestroy(b->join_ev[q]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    void *ptrs[] = {b->d_probs, b->d_scen, b->d_seg_scen, b->d_segkeys, b->d_dyns, b->d_Lxy,
                    b->d_Btmp, b->d_W, b->d_u[0], b->d_u[1], b->d_cost_ms, b->d_cost_ms_soft,
                    b->d_cbar, b->d_cbar_soft, b->d_wtilde, b->d_anc, b->d_work, b->d_best,
                    b->d_best_sum, b->d_ninf, b->d_best_u, b->d_t_start, b->d_t_end, b->d_live,
                    b->d_queue, b->d_flags, b->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (float *p : b->d_pops)
        if (p) cudaFree(p);
}

static bool same_shape(const tma_problem &a, const tma_problem &b)
{
    bool ok = a.L == b.L && a.M == b.M && a.H == b.H && a.S == b.S && a.J_max == b.J_max &&
              a.dt == b.dt && a.beta_xy == b.beta_xy && a.gam_z == b.gam_z && a.lam_t == b.lam_t &&
              a.wind_sigma == b.wind_sigma && a.sep_mode == b.sep_mode && a.wind_mode == b.wind_mode &&
              a.sample_mode == b.sample_mode;
    for (int d = 0; d < 3; ++d)
        ok = ok && a.grid[d] == b.grid[d] && a.box_lo[d] == b.box_lo[d] && a.box_hi[d] == b.box_hi[d];
    return ok;
}

// Every scenario's wind field for its current MPC step (wind mode 1, the same
// for the whole batch, draws each particle's field in the rollout instead).
static tma_status batch_wind(tma_batch *b, cudaStream_t st)
{
    const size_t P = (size_t)b->probs[0].grid[0] * b->probs[0].grid[1] * b->probs[0].grid[2];
    for (size_t g = 0; g < b->wind_groups.size() && b->probs[0].wind_mode == 0; ++g) {
        const WindC &w = b->wind_groups[g];
        const int s0 = b->group_start[g];
        TMA_CUDA(launch_batch_wind_normals(w, s0, b->M, b->d_scen, b->d_dyns, b->d_Btmp, st));
        TMA_CUDA(launch_wind_gemm(w, b->d_Lxy, b->lda, b->d_Btmp,
                                  b->d_W + (size_t)s0 * b->M * b->H * P * 4, st));
    }
    return TMA_OK;
}

// One rollout of every scenario at iteration J (Mj wind samples), in the
// batch's dispatch form.
static cudaError_t batch_rollout(tma_batch *b, const float *d_u, int J, int Mj, float *cost,
                                 float *cost_soft, int dispatch, cudaStream_t st)
{
    if (dispatch == 0)
        return launch_batch_rollout(b->d_probs, b->d_scen, b->n_scen, b->d_dyns, d_u, b->d_W, b->L, J, Mj,
                                    cost, cost_soft, b->d_live, b->d_queue, b->grid, b->probs[0].wind_mode, st);
    // scenarios round-robin over the auxiliary streams, so that one launch's
    // last wave overlaps the next scenario's first
    const int ns = tma_batch::kAuxStreams;
    cudaError_t e = cudaEventRecord(b->fork_ev, st);
    for (int q = 0; q < ns && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(b->aux[q], b->fork_ev, 0);
    for (int s = 0; s < b->n_scen && e == cudaSuccess; ++s) {
        const BatchScen &sc = b->scen[s];
        ProblemC Ps = b->pc_h[s];
        Ps.M = Mj;
        const size_t co = (size_t)sc.seg_off * b->M * (size_t)b->L;
        e = launch_rollout(Ps, b->d_dyns + s, d_u + sc.u_off, b->d_W + (size_t)sc.w_off * 4, b->L, J, cost + co,
                           cost_soft ? cost_soft + co : nullptr, b->d_live, b->aux[s % ns], b->scen_variant[s]);
    }
    for (int q = 0; q < ns && e == cudaSuccess; ++q) e = cudaEventRecord(b->join_ev[q], b->aux[q]);
    for (int q = 0; q < ns && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(st, b->join_ev[q], 0);
    return e;
}

static tma_status batch_solve_device(tma_batch *b, cudaStream_t st)
{
    const long long L = b->L;
    TMA_CUDA(launch_stamp_start(b->d_t_start, st));
    {
        tma_status r = batch_wind(b, st);
        if (r != TMA_OK) return r;
    }
    TMA_CUDA(launch_batch_init(b->d_scen, b->d_seg_scen, b->d_dyns, b->nseg, L, b->S, b->d_u[0], st));
    TMA_CUDA(cudaMemsetAsync(b->d_flags, 0, 4, st));
    TMA_CUDA(cudaMemsetAsync(b->d_live, 0, 8, st));
    int cur = 0;
    const bool soft = b->sep_mode != 0;
    float *cb = b->sep_mode == 1 ? b->d_cbar_soft : b->d_cbar;
    for (int J = 0; J < b->J_max; ++J) {
        const int Mj = samples_of(b->probs[0], J);
        TMA_CUDA(batch_rollout(b, b->d_u[cur], J, Mj, b->d_cost_ms, soft ? b->d_cost_ms_soft : nullptr,
                               b->dispatch, st));
        TMA_CUDA(launch_batch_sample_mean(b->d_cost_ms, b->d_scen, b->d_seg_scen, b->nseg, L, b->M,
                                          Mj, b->d_cbar, st));
        if (soft)
            TMA_CUDA(launch_batch_sample_mean(b->d_cost_ms_soft, b->d_scen, b->d_seg_scen, b->nseg, L,
                                              b->M, Mj, b->d_cbar_soft, st));
        if (J < b->J_max - 1) {
            void *rwork = static_cast<char *>(b->d_work) + b->lse_work_bytes;
            TMA_CUDA(launch_lse(cb, (int)b->nseg, L, exponent_of(b->probs[0], J), b->d_wtilde, nullptr,
                                nullptr, b->d_work, st, resample_partials(rwork)));
            TMA_CUDA(launch_resample(b->d_wtilde, (int)b->nseg, L, L, 0u, 0u, (uint32_t)J, nullptr, 0u,
                                     b->d_anc, rwork, b->d_flags, st, b->d_segkeys, b->d_dyns, true));
            TMA_CUDA(launch_batch_move(b->d_scen, b->d_seg_scen, b->d_dyns, b->nseg, L, b->S,
                                       b->d_u[cur], b->d_anc, J, b->d_u[cur ^ 1], st, b->d_err));
            cur ^= 1;
        }
    }
    TMA_CUDA(launch_batch_select(b->d_scen, b->n_scen, cb, L, b->S, b->d_u[cur], b->d_best,
                                 b->d_best_sum, b->d_ninf, b->d_best_u, b->d_t_end, st));
    b->final_u = cur;
    return TMA_OK;
}

// The batch's rollout dispatch: every scenario's variant of the single-scenario
// kernel (the solvers' autotuner and cache, timed on the scenario's own first
// 8192 particles), then both dispatch forms timed on the whole batch at
// iteration 0 (uniform initial controls; one untimed and one timed rollout
// each); the faster form is kept.  On an idle device, like the solvers' tuner.
static tma_status batch_tune(tma_batch *b)
{
    const int n = b->n_scen;
    b->scen_variant.assign(n, 0);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TMA_CUDA(cudaDeviceSynchronize());
    TMA_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    auto cleanup = [&]() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(st);
    };
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    tma_status r = e == cudaSuccess ? batch_wind(b, st) : cuda_fail(e);
    if (r == TMA_OK) e = launch_batch_init(b->d_scen, b->d_seg_scen, b->d_dyns, b->nseg, b->L, b->S, b->d_u[0], st);
    const int64_t Lp = std::min<int64_t>(b->L, 8192);
    for (int s = 0; s < n && r == TMA_OK && e == cudaSuccess; ++s) {
        const std::string key = tune_key_of(b->probs[s], b->device);
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                b->scen_variant[s] = it->second;
                continue;
            }
        }
        const BatchScen &sc = b->scen[s];
        int best = 0, nt = 0, tv[kMaxRolloutVariants];
        float tms[kMaxRolloutVariants];
        e = time_rollout_variants(b->pc_h[s], b->d_dyns + s, b->d_u[0] + sc.u_off, b->d_W + (size_t)sc.w_off * 4,
                                  Lp, b->d_cost_ms + (size_t)sc.seg_off * b->M * (size_t)b->L, st, e0, e1, &best,
                                  &nt, tv, tms);
        if (e == cudaSuccess) {
            b->scen_variant[s] = best;
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = best;
        }
    }
    const int M0 = samples_of(b->probs[0], 0);
    for (int form = 0; form < 2 && r == TMA_OK && e == cudaSuccess; ++form) {
        e = batch_rollout(b, b->d_u[0], 0, M0, b->d_cost_ms, nullptr, form, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = batch_rollout(b, b->d_u[0], 0, M0, b->d_cost_ms, nullptr, form, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b->dispatch_ms[form], e0, e1);
    }
    if (r == TMA_OK && e != cudaSuccess) r = cuda_fail(e);
    if (r == TMA_OK) b->dispatch = b->dispatch_ms[1] < b->dispatch_ms[0] ? 1 : 0;
    cleanup();
    return r;
}

static tma_status batch_mpc_steps(tma_batch *b, int n_steps, cudaStream_t st)
{
    for (int n = 0; n < n_steps; ++n) {
        tma_status r = batch_solve_device(b, st);
        if (r != TMA_OK) return r;
        TMA_CUDA(launch_plant_step(b->d_probs, b->d_scen, b->d_seg_scen, b->nseg, b->n_scen,
                                   b->d_dyns, b->d_W, b->d_best_u, b->S, st));
    }
    return TMA_OK;
}

tma_status tma_batch_create(const tma_problem *probs, const tma_aircraft *const *aircraft,
                            int32_t n_scen, tma_batch **out)
{
    if (!out || !probs || !aircraft || n_scen < 1 || n_scen > (1 << 20)) return TMA_ERR_INVALID_ARG;
    *out = nullptr;
    for (int s = 0; s < n_scen; ++s) {
        tma_status v = validate(&probs[s], aircraft[s]);
        if (v != TMA_OK) return v;
        if (!same_shape(probs[0], probs[s])) return TMA_ERR_INVALID_ARG;
        if (probs[s].L_sched) return TMA_ERR_UNSUPPORTED;    // fixed particle count per batch
    }
    tma_batch *b = nullptr;
    try {
        b = new tma_batch();
        cudaGetDevice(&b->device);
        const tma_problem &p0 = probs[0];
        b->n_scen = n_scen;
        b->L = p0.L;
        b->M = p0.M;
        b->H = p0.H;
        b->S = p0.S;
        b->J_max = p0.J_max;
        b->sep_mode = p0.sep_mode;
        const int nx = p0.grid[0], ny = p0.grid[1], nz = p0.grid[2], nxy = nx * ny;
        const size_t P = (size_t)nxy * nz;
        const long long nLb = ((long long)p0.L + kTileParticles - 1) / kTileParticles;
        auto fail = [&](cudaError_t e) {
            batch_free(b);
            delete b;
            return e == cudaErrorMemoryAllocation ? TMA_ERR_OOM : cuda_fail(e);
        };
        cudaError_t e;
        std::vector<ProblemC> pc(n_scen);
        std::vector<SegKey> segkeys;
        long long u_off = 0, items = 0;
        for (int s = 0; s < n_scen; ++s) {
            const tma_problem &p = probs[s];
            b->probs.push_back(p);
            b->aircraft.emplace_back(aircraft[s], aircraft[s] + p.N);
            float *dpop = nullptr;
            if (p.pop_n[0] >= 2) {
                const std::vector<float> pf = pack_popcells(p.popdense, p.pop_n[0], p.pop_n[1]);
                if ((e = alloc(&dpop, pf.size() * 4))) return fail(e);
                b->d_pops.push_back(dpop);
                if ((e = cudaMemcpy(dpop, pf.data(), pf.size() * 4, cudaMemcpyHostToDevice))) return fail(e);
            }
            b->probs.back().popdense = nullptr;
            pc[s] = derive_problem(p, aircraft[s], dpop);
            BatchScen sc;
            std::memset(&sc, 0, sizeof sc);
            sc.u_off = u_off;
            sc.seg_off = b->nseg;
            sc.w_off = (long long)s * p.M * p.H * (long long)P;
            sc.N = p.N;
            sc.T = std::min(15, 32 / p.N);   // one named barrier (ids 1..15) per tile
            sc.items = (long long)p.M * nLb;
            for (int c = 0; c < 3; ++c) {
                sc.ctrl_lo[c] = (float)p.ctrl_lo[c];
                sc.ctrl_hi[c] = (float)p.ctrl_hi[c];
                sc.move_sigma[c] = (float)p.move_sigma[c];
            }
            sc.key0 = pc[s].key0;
            sc.key1 = pc[s].key1;
            b->scen.push_back(sc);
            for (int i = 0; i < p.N; ++i) {
                b->seg_scen.push_back(s);
                segkeys.push_back(SegKey{sc.key0, sc.key1, (uint32_t)i, s});
            }
            DynState d;
            std::memset(&d, 0, sizeof d);
            for (int i = 0; i < p.N; ++i) {
                const tma_state &x = aircraft[s][i].x0;
                d.x0[i][0] = (float)x.x;
                d.x0[i][1] = (float)x.y;
                d.x0[i][2] = (float)x.z;
                d.x0[i][3] = (float)x.v;
                d.x0[i][4] = (float)x.chi;
                d.x0[i][5] = (float)x.m;
            }
            d.mpc_step = p.mpc_step;
            b->dyn_h.push_back(d);
            u_off += (long long)p.L * p.N * p.S * 3;
            items += sc.items;
            b->nseg += p.N;
        }
        b->n_items = items;
        if (b->nseg > 65535) {
            batch_free(b);
            delete b;
            return TMA_ERR_INVALID_ARG;   // one resampling block row per segment
        }
        // wind factors shared by all scenarios (same grid and rates)
        auto lxy = horizontal_factor(p0);
        std::vector<double> Rz((size_t)nz * nz);
        for (int a = 0; a < nz; ++a)
            for (int c = 0; c <= a; ++c) {
                const double za = p0.box_lo[2] + (p0.box_hi[2] - p0.box_lo[2]) * a / (nz - 1);
                const double zc = p0.box_lo[2] + (p0.box_hi[2] - p0.box_lo[2]) * c / (nz - 1);
                Rz[(size_t)a * nz + c] = std::exp(-p0.gam_z * std::fabs(za - zc));
            }
        if (!lxy || !cholesky_lower(Rz, nz)) {
            batch_free(b);
            delete b;
            return TMA_ERR_INVALID_ARG;
        }
        b->lda = lxy->lda;
        const long long per_scen = (long long)p0.M * p0.H * 2 * nz;
        int gsz = (int)std::max(1LL, std::min(64LL, (1LL << 28) / ((long long)b->lda * per_scen)));
        gsz = std::min(gsz, n_scen);
        const int max_ldb = (int)(((gsz * per_scen) + 127) / 128 * 128);
        const double a = std::exp(-p0.dt * p0.lam_t);
        for (int s0 = 0; s0 < n_scen; s0 += gsz) {
            const int nsc = std::min(gsz, n_scen - s0);
            WindC w;
            std::memset(&w, 0, sizeof w);
            w.stream = 3u;
            w.M = nsc * p0.M;
            w.H = p0.H;
            w.nxy = nxy;
            w.nz = nz;
            w.ncol = (int)(nsc * per_scen);
            w.ldb = max_ldb;
            w.a = (float)a;
            w.b = (float)std::sqrt(std::max(0.0, 1.0 - a * a));
            w.sigma = (float)p0.wind_sigma;
            for (int r = 0; r < nz; ++r)
                for (int c = 0; c <= r; ++c) w.Lz[r * TMA_MAX_GRID_Z + c] = (float)Rz[(size_t)r * nz + c];
            b->wind_groups.push_back(w);
            b->group_start.push_back(s0);
        }
        const size_t L = (size_t)p0.L, M = (size_t)p0.M, nseg = (size_t)b->nseg;
        if ((e = alloc(&b->d_probs, sizeof(ProblemC) * n_scen))) return fail(e);
        if ((e = alloc(&b->d_scen, sizeof(BatchScen) * n_scen))) return fail(e);
        if ((e = alloc(&b->d_seg_scen, sizeof(int) * nseg))) return fail(e);
        if ((e = alloc(&b->d_segkeys, sizeof(SegKey) * nseg))) return fail(e);
        if ((e = alloc(&b->d_dyns, sizeof(DynState) * n_scen))) return fail(e);
        if ((e = alloc(&b->d_Lxy, lxy->L.size() * 4))) return fail(e);
        if ((e = alloc(&b->d_Btmp, (size_t)b->lda * max_ldb * 4))) return fail(e);
        if ((e = cudaMemset(b->d_Btmp, 0, (size_t)b->lda * max_ldb * 4))) return fail(e);
        if ((e = alloc(&b->d_W, (size_t)n_scen * M * p0.H * P * 16))) return fail(e);
        if ((e = alloc(&b->d_u[0], (size_t)u_off * 4))) return fail(e);
        if ((e = alloc(&b->d_u[1], (size_t)u_off * 4))) return fail(e);
        if ((e = alloc(&b->d_cost_ms, M * nseg * L * 4))) return fail(e);
        if (b->sep_mode && (e = alloc(&b->d_cost_ms_soft, M * nseg * L * 4))) return fail(e);
        if ((e = alloc(&b->d_cbar, nseg * L * 4))) return fail(e);
        if (b->sep_mode && (e = alloc(&b->d_cbar_soft, nseg * L * 4))) return fail(e);
        if ((e = alloc(&b->d_wtilde, nseg * L * 8))) return fail(e);
        if ((e = alloc(&b->d_anc, nseg * L * 4))) return fail(e);
        b->lse_work_bytes = (lse_workspace((int)nseg, L) + 255) / 256 * 256;
        if ((e = alloc(&b->d_work, b->lse_work_bytes + resample_workspace((int)nseg, L))))
            return fail(e);
        if ((e = alloc(&b->d_best, 8 * (size_t)n_scen))) return fail(e);
        if ((e = alloc(&b->d_best_sum, 8 * (size_t)n_scen))) return fail(e);
        if ((e = alloc(&b->d_ninf, 4 * (size_t)n_scen))) return fail(e);
        if ((e = alloc(&b->d_best_u, nseg * p0.S * 3 * 4))) return fail(e);
        if ((e = alloc(&b->d_t_start, 8))) return fail(e);
        if ((e = alloc(&b->d_t_end, 8 * (size_t)n_scen))) return fail(e);
        if ((e = alloc(&b->d_live, 8))) return fail(e);
        if ((e = alloc(&b->d_queue, 8 * (size_t)n_scen))) return fail(e);
        if ((e = alloc(&b->d_flags, 4))) return fail(e);
        if ((e = alloc(&b->d_err, 4))) return fail(e);
        if ((e = cudaMemset(b->d_err, 0, 4))) return fail(e);
        if ((e = cudaMemcpy(b->d_probs, pc.data(), sizeof(ProblemC) * n_scen, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemcpy(b->d_scen, b->scen.data(), sizeof(BatchScen) * n_scen, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemcpy(b->d_seg_scen, b->seg_scen.data(), sizeof(int) * nseg, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemcpy(b->d_segkeys, segkeys.data(), sizeof(SegKey) * nseg, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemcpy(b->d_dyns, b->dyn_h.data(), sizeof(DynState) * n_scen, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaMemcpy(b->d_Lxy, lxy->L.data(), lxy->L.size() * 4, cudaMemcpyHostToDevice))) return fail(e);
        if ((e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking))) return fail(e);
        for (int q = 0; q < tma_batch::kAuxStreams; ++q) {
            if ((e = cudaStreamCreateWithFlags(&b->aux[q], cudaStreamNonBlocking))) return fail(e);
            if ((e = cudaEventCreateWithFlags(&b->join_ev[q], cudaEventDisableTiming))) return fail(e);
        }
        if ((e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming))) return fail(e);
        b->grid = batch_rollout_grid();
        b->pc_h = pc;
    } catch (const std::bad_alloc &) {
        if (b) {
            batch_free(b);
            delete b;
        }
        return TMA_ERR_OOM;
    }
    const tma_status r = batch_tune(b);
    if (r != TMA_OK) {
        batch_free(b);
        delete b;
        return r;
    }
    *out = b;
    return TMA_OK;
}

tma_status tma_batch_get_dispatch(tma_batch *b, int32_t *dispatch, float *ms_persistent, float *ms_per_scenario)
{
    if (!b) return TMA_ERR_INVALID_ARG;
    if (dispatch) *dispatch = b->dispatch;
    if (ms_persistent) *ms_persistent = b->dispatch_ms[0];
    if (ms_per_scenario) *ms_per_scenario = b->dispatch_ms[1];
    return TMA_OK;
}

tma_status tma_batch_set_dispatch(tma_batch *b, int32_t dispatch)
{
    if (!b || (dispatch != 0 && dispatch != 1)) return TMA_ERR_INVALID_ARG;
    if (dispatch != b->dispatch && b->graph) {      // a captured loop holds the other form
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_steps = 0;
    }
    b->dispatch = dispatch;
    return TMA_OK;
}

void tma_batch_destroy(tma_batch *b)
{
    if (!b) return;
    batch_free(b);
    delete b;
}

tma_status tma_batch_set_state(tma_batch *b, const tma_state *h_x0, const uint32_t *h_mpc,
                               tma_stream_t stream)
{
    if (!b) return TMA_ERR_INVALID_ARG;
    // start from the device state so that plant-advanced states are kept
    TMA_CUDA(cudaMemcpyAsync(b->dyn_h.data(), b->d_dyns, sizeof(DynState) * b->n_scen,
                             cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    long long k = 0;
    for (int s = 0; s < b->n_scen; ++s) {
        for (int i = 0; i < b->probs[s].N; ++i, ++k) {
            if (!h_x0) continue;
            const tma_state &x = h_x0[k];
            if (!(x.v > 0) || !(x.m > 0)) return TMA_ERR_INVALID_ARG;
            float *d = b->dyn_h[s].x0[i];
            d[0] = (float)x.x;
            d[1] = (float)x.y;
            d[2] = (float)x.z;
            d[3] = (float)x.v;
            d[4] = (float)x.chi;
            d[5] = (float)x.m;
        }
        if (h_x0) b->dyn_h[s].finished = 0u;     // new states: every aircraft back in the problem
        if (h_mpc) {
            if (h_mpc[s] > 0xFFFF) return TMA_ERR_INVALID_ARG;
            b->dyn_h[s].mpc_step = h_mpc[s];
        }
    }
    TMA_CUDA(cudaMemcpyAsync(b->d_dyns, b->dyn_h.data(), sizeof(DynState) * b->n_scen,
                             cudaMemcpyHostToDevice, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TMA_OK;
}

tma_status tma_batch_solve(tma_batch *b, tma_stream_t stream)
{
    if (!b) return TMA_ERR_INVALID_ARG;
    return batch_solve_device(b, (cudaStream_t)stream);
}

tma_status tma_batch_mpc(tma_batch *b, int32_t n_steps, int32_t use_graph, tma_stream_t stream)
{
    if (!b || n_steps < 0) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_steps == 0) return TMA_OK;
    if (!use_graph) return batch_mpc_steps(b, n_steps, st);
    if (!b->graph || b->graph_steps != n_steps) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        TMA_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
        tma_status r = batch_mpc_steps(b, n_steps, b->capture_stream);
        const cudaError_t ec = cudaStreamEndCapture(b->capture_stream, &g);
        if (r != TMA_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (ec != cudaSuccess) return cuda_fail(ec);
        const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            b->graph = nullptr;
            return cuda_fail(ei);
        }
        b->graph_steps = n_steps;
    }
    TMA_CUDA(cudaGraphLaunch(b->graph, st));
    return TMA_OK;
}

tma_status tma_batch_rollout_cost(tma_batch *b, const float *d_u, int32_t J, float *d_cost_ms,
                                  float *d_cost_ms_soft, tma_stream_t stream)
{
    if (!b || !d_u || !d_cost_ms || J < 0 || J > 0xFFFF) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    tma_status r = batch_wind(b, st);
    if (r != TMA_OK) return r;
    const bool soft = b->sep_mode != 0 && d_cost_ms_soft != nullptr;
    TMA_CUDA(cudaMemsetAsync(b->d_live, 0, 8, st));
    TMA_CUDA(batch_rollout(b, d_u, J, samples_of(b->probs[0], J), d_cost_ms, soft ? d_cost_ms_soft : nullptr,
                           b->dispatch, st));
    return TMA_OK;
}

tma_status tma_batch_results(tma_batch *b, float *h_best_u, double *h_best_cost, int64_t *h_best,
                             tma_state *h_x, uint32_t *h_mpc, tma_stream_t stream)
{
    if (!b) return TMA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (h_best_u)
        TMA_CUDA(cudaMemcpyAsync(h_best_u, b->d_best_u, (size_t)b->nseg * b->S * 3 * 4,
                                 cudaMemcpyDeviceToHost, st));
    if (h_best_cost)
        TMA_CUDA(cudaMemcpyAsync(h_best_cost, b->d_best_sum, 8 * (size_t)b->n_scen, cudaMemcpyDeviceToHost, st));
    if (h_best)
        TMA_CUDA(cudaMemcpyAsync(h_best, b->d_best, 8 * (size_t)b->n_scen, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemcpyAsync(b->dyn_h.data(), b->d_dyns, sizeof(DynState) * b->n_scen,
                             cudaMemcpyDeviceToHost, st));
    unsigned int err = 0;
    TMA_CUDA(cudaMemcpyAsync(&err, b->d_err, 4, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemsetAsync(b->d_err, 0, 4, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    long long k = 0;
    for (int s = 0; s < b->n_scen; ++s) {
        if (h_mpc) h_mpc[s] = b->dyn_h[s].mpc_step;
        for (int i = 0; i < b->probs[s].N; ++i, ++k) {
            if (!h_x) continue;
            const float *d = b->dyn_h[s].x0[i];
            h_x[k] = tma_state{d[0], d[1], d[2], d[3], d[4], d[5]};
        }
    }
    return (err & TMA_DEVERR_BOUNDS) ? TMA_ERR_BOUNDS : TMA_OK;
}

tma_status tma_batch_latency(tma_batch *b, double *h_ms, tma_stream_t stream)
{
    if (!b || !h_ms) return TMA_ERR_INVALID_ARG;
    std::vector<unsigned long long> t(b->n_scen);
    unsigned long long t0 = 0;
    cudaStream_t st = (cudaStream_t)stream;
    TMA_CUDA(cudaMemcpyAsync(&t0, b->d_t_start, 8, cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaMemcpyAsync(t.data(), b->d_t_end, 8 * t.size(), cudaMemcpyDeviceToHost, st));
    TMA_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < b->n_scen; ++s) h_ms[s] = (double)(long long)(t[s] - t0) * 1e-6;
    return TMA_OK;
}

tma_status tma_batch_live_steps(tma_batch *b, uint64_t *h_live, tma_stream_t stream)
{
    if (!b || !h_live) return TMA_ERR_INVALID_ARG;
    unsigned long long v = 0;
    TMA_CUDA(cudaMemcpyAsync(&v, b->d_live, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TMA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    *h_live = v;
    return TMA_OK;
}

}  // extern "C"
