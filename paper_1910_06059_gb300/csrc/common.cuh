// Internal declarations of the GB300 black-oil library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "bo.h"

namespace bo {

// ---------------------------------------------------------------------------
// Error handling: every C entry point catches bo::Error and maps it to a
// status plus a thread-local message.
// ---------------------------------------------------------------------------
struct Error {
    bo_status status;
    std::string msg;
};

[[noreturn]] void fail(bo_status st, const std::string& msg);
bo_status set_last_error(bo_status st, const std::string& msg);   // returns st
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define BO_CUDA(call) ::bo::check_cuda((call), #call, __FILE__, __LINE__)
#define BO_LAUNCH_CHECK(name) ::bo::check_cuda(cudaGetLastError(), name, __FILE__, __LINE__)

// ---------------------------------------------------------------------------
// Data layout in HBM (n cells, natural order c = i + nx*(j + ny*k)):
//   cell vectors of 3 components: structure of arrays v[e*n + c]
//   Jacobian A: 7 blocks per cell, block-major then entry-major:
//     A[(b*9 + e)*n + c],  b: 0 diag, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z,
//     e = 3*r + s for dR_r,c / dy_s,neighbour(b); zero where no neighbour.
//   ILU(0) data P in tile order (see tiles.cuh, pidx): b: 0 D^-1,
//     1..3 D^-1 A_{c,-x/-y/-z}, 4..6 D^-1 A_{c,+x/+y/+z}.
// ---------------------------------------------------------------------------
enum { NB_DIAG = 0, NB_MX = 1, NB_PX = 2, NB_MY = 3, NB_PY = 4, NB_MZ = 5, NB_PZ = 6 };
constexpr int NPROP = 28;   // per-cell face quantities: rho_a, b_a lam_a (3 x 4), r_go b_o lam_o (4)

struct DevFluid {
    double g, rho_s[3], p_ref, bw_ref, c_w, mu_w, R_sb, p_b, Bo_slope, c_o, mu_o0, mu_o_r, c_mu,
        p_sc, Z, mu_g0, mu_g_p, c_r, s_wco, s_orw, s_org, n_corey;
};

struct Geom {
    int nx, ny, nz, n;
};

// Equilibration input (depths positive downward, SI units).
struct EquilDev {
    double datum_z, datum_p, woc, goc, rgo, swc;
};

// Well description and per-step state, in device memory.
struct WellDev {
    int kind, phase, ctl0, ctl;   // ctl: 0 rate, 1 bhp
    int off, ncon;
    double target, limit, bhp, bhp_bk;
    double z_datum, rho_well;
    double Rw, Dw, xw;
    double qs[3];   // surface rates (w, o, g) summed over the connections at the last assembly
    // full standard well (Section 2.2.1; wells_std.cu), when full != 0
    int full;
    int singular;        // D_w had a zero pivot at the last assembly
    double vw;           // wellbore volume of the storage term (0: no storage)
    double xs[4];        // Q_t, F_w, F_g, p_bhp (p_bhp mirrors bhp)
    double xs_bk[4];     // at the step start (restored on a cut)
    double A0s[3];       // wellbore storage at the step start
    double Rs[4];        // well residual: three component balances, control
    double D[16];        // D_w = dR_w / dx_w, row-major
    double Dinv[16];     // D_w^-1
    double dxs[4];       // solution of the well rows, x_w = D_w^-1 (R_w - B_w x_r)
};
enum { BO_WELL_MODEL_REDUCED = 0, BO_WELL_MODEL_STANDARD = 1 };
// weights g_w, g_o, g_g of the weighted total rate Q_t (a small gas weight)
__host__ __device__ __forceinline__ double std_well_g(int a) { return a == 2 ? 0.01 : 1.0; }

// Scalars of the BiCGStab recurrence, kept on the device.
struct KrylovScalars {
    double rho, rho_old, alpha, omega, beta, nr0, tol;
    double last_nr;
    int it, maxit, state, status;   // state: 0 running, 1 half-step exit pending, 2 done
    int half_exit;                  // the solve ended on the half step (no second apply)
    int restarts;                   // restarts from the true residual
    double true_nr;                 // ||b - Op x||_2 at the last check
    double stop;                    // the recurrence stops at ||r|| <= stop
    double inner;                   // per-cycle relative target (0: tol alone)
};
enum { KS_RUN = 0, KS_HALF = 1, KS_DONE = 2 };
enum { LS_OK = 0, LS_NOT_CONVERGED = 1, LS_BREAKDOWN = 2 };

// Device-to-host status block read once per Newton iteration.
struct NewtonStatus {
    double norms[7];
    int dead_wells;   // rate wells with D_w == 0 in the last assembly
    int pad;
    int singular_wells;   // full standard wells whose D_w had a zero pivot
    int pad2;
};

constexpr int MAX_TIMERS = 16;

// A timed interval outside the solver graphs: two events on the sim's stream,
// read back at the next flush.
struct EagerTimer {
    cudaEvent_t a, b;
    int id;
};

// One Newton system kept for offline training of the learned stage: its
// Jacobian, ILU(0) data, FP32 features, per-cell scalings and nr residuals
// of its BiCGStab solve ([nr][3n]).
struct LearnSystem {
    double* A = nullptr;
    double* P = nullptr;
    float* featf = nullptr;
    float4* cell = nullptr;
    double* r = nullptr;
    int nr = 0;
};

struct CprData;   // CPR preconditioner data (cpr.cu)
struct DdData;    // K-subdomain solver data (dd.cu)

}  // namespace bo

// The opaque object of the C ABI.
struct bo_sim {
    bo::Geom geo{};
    int nlev = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool props_set = false;
    bool assembled = false;
    bool factored = false;
    bool solved = false;
    double dt_last = 0.0;
    double dt_next = 0.0;   // sub-step length carried between report steps

    std::vector<double> dx, dy, dz;
    double top = 0.0;
    bo::DevFluid fluid{};

    // wells (host mirror of the static part)
    int nw = 0, ncon = 0, nrate = 0;
    std::vector<bo::WellDev> wells_h;
    std::vector<int> con_cell_h;
    std::vector<double> well_volume;   // wellbore volume per well (pi r_w^2 x perforated thickness)


    // device memory
    double *d_dx = nullptr, *d_dy = nullptr, *d_dz = nullptr;
    double *d_perm = nullptr, *d_poro = nullptr;
    double *d_T = nullptr;       // 3n: +x, +y, +z face transmissibility
    double *d_pv = nullptr, *d_depth = nullptr;
    double *d_p = nullptr, *d_sw = nullptr, *d_x = nullptr;
    uint8_t* d_flag = nullptr;
    double* d_bk = nullptr;      // 3n backup of (p, sw, x)
    uint8_t* d_bkflag = nullptr;
    double* d_A0 = nullptr;      // 3n
    double* d_props = nullptr;   // NPROP * n
    double* d_R = nullptr;       // 3n
    double* d_A = nullptr;       // 63n
    double* d_P = nullptr;       // 63 x tile-order ILU(0) data
    double* d_yt = nullptr;      // forward-sweep result, tile order [slot][3][32]
    double* d_qt = nullptr;      // forward-sweep right-hand side D^-1 r, tile order
    int* d_order = nullptr;      // sweep tile lists: forward [T], backward [T]
    float* d_P32 = nullptr;      // FP32 factors in the FP32 sweep layout (mixed mode)
    float* d_r32 = nullptr;      // FP32 sweep input, tile order (mixed mode)
    float* d_y32 = nullptr;      // FP32 sweep work vector, tile order (mixed mode)
    bool mixed = false;          // preconditioner applies in FP32
    int last_restarts = 0;       // BiCGStab restarts from the true residual, last solve
    double last_rel_res = 0.0;   // ||b - Op x|| / ||b||, last solve
    double* d_face = nullptr;    // tile-face buffers of the wavefront sweeps
    int* d_sweep_sync = nullptr; // [2]: a bounded wait of a sweep ran out
    int* d_cellcon = nullptr;    // c -> connection index or -1
    bo::WellDev* d_wells = nullptr;
    int* d_con_cell = nullptr;
    double* d_con_wi = nullptr;
    double* d_wB = nullptr;      // 3 * ncon
    double* d_wC = nullptr;      // 3 * ncon
    // full standard wells (wells_std.cu)
    int well_model = 0;          // BO_WELL_MODEL_*
    bool well_storage = true;
    double* d_wB4 = nullptr;     // [ncon][4][3]: B_w, dR_w / dx_c of the connection cell
    double* d_wC4 = nullptr;     // [ncon][3][4]: C_w, dR_c / dx_w
    double* d_wcorr = nullptr;   // [ncon][3]: C_w D_w^-1 B_w x of the last operator
    // Krylov vectors (3n each) and reduction scratch
    double *d_b = nullptr, *d_xs = nullptr, *d_r = nullptr, *d_rh = nullptr, *d_pk = nullptr,
           *d_v = nullptr, *d_s = nullptr, *d_t = nullptr, *d_ph = nullptr, *d_sh = nullptr;
    double* d_part = nullptr;    // reduction partials
    int part_blocks = 0;
    bo::KrylovScalars* d_ks = nullptr;
    bo::NewtonStatus* d_ns = nullptr;
    bo::NewtonStatus* h_ns = nullptr;   // pinned
    bo::KrylovScalars* h_ks = nullptr;  // pinned

    // learned preconditioner stage (learned.cu)
    float* d_ml_theta = nullptr;   // FP32 parameters (BO_LEARN_NPARAM)
    float* d_ml_grad = nullptr;    // gradient accumulator
    float* d_ml_m = nullptr;       // Adam moments
    float* d_ml_v = nullptr;
    void* d_ml_wbf = nullptr;      // BF16 weight image of the tensor-core kernel
    void* d_ml_feat = nullptr;     // [n][64] BF16 block features of the last factorisation
    float* d_ml_featf = nullptr;   // [n][64] FP32 block features (training only)
    float4* d_ml_cell = nullptr;   // [n] (1/rho_0, 1/rho_1, 1/rho_2, sigma_x)
    float* d_ml_W = nullptr;       // [9][n] per-cell matrices of the network
    double* d_ml_part = nullptr;   // reduction partials
    double *d_ml_delta = nullptr, *d_ml_u = nullptr, *d_ml_z0 = nullptr, *d_ml_e = nullptr,
           *d_ml_dd = nullptr;     // training vectors (3n)
    double* d_ml_scal = nullptr;   // training scalars
    int* d_ml_count = nullptr;     // samples stored by the last solve
    double* d_ml_samples = nullptr;  // [cap][3n] residual samples
    int ml_cap = 0;
    int ml_adam_t = 0;
    int ml_engine = 1;             // BO_LEARN_ENGINE_*: tensor-core kernel of the network
    bool ml_params = false;        // parameters set
    bool ml_on = false;            // the stage runs inside BiCGStab
    bool ml_online = false;        // collect residuals and train after each solve
    int ml_epochs = 1;
    double ml_lr = 1e-3;
    long long ml_systems = 0, ml_steps = 0, ml_fallbacks = 0;
    int ml_guard_left = 0, ml_guard_state = 0;          // bo_learn_guard window and decision
    long long ml_guard_stage_its = 0, ml_guard_plain_its = 0;
    double ml_first_loss = -1.0, ml_last_loss = -1.0, ml_train_ms = 0.0;
    int ml_collect_max = 0;                   // systems to keep for offline training (0: off)
    std::vector<bo::LearnSystem> ml_set;      // the kept systems
    cudaGraphExec_t g_iter_ml = nullptr;
    cudaGraphExec_t g_iter64 = nullptr;   // FP64 sweeps in mixed mode (fallback solves)
    int last_fallback = 0;                // bo_solve_report::fallback of the last solve

    // CPR two-stage preconditioner (cpr.cu); precond: BO_PRECOND_*
    int precond = 0;
    int solve_schedule = 0;   // BO_SCHEDULE_*: tiled kernels or one CTA per solve
    bo::CprData* cpr = nullptr;
    bo::DdData* dd = nullptr;   // K-subdomain solver (dd.cu)

    // CUDA graphs of one BiCGStab iteration block and of the factorisation
    cudaGraphExec_t g_iter = nullptr;
    cudaGraphExec_t g_factor = nullptr;
    cudaGraphExec_t g_iter_timed = nullptr;
    int iters_per_graph = 4;
    int sweep_ctas_per_sm = 2;   // persistent CTAs of the FP64 sweeps per SM (1 or 2)
    int ysub = 0;                // block-Jacobi slabs of ysub cell rows in y (0: no cut in y)
    int zsub = 0;                // and of zsub cell layers in z (0: no cut in z)

    // timing
    bool timing = false;
    int ntimers = 0;
    std::string timer_name[bo::MAX_TIMERS];
    double timer_ms[bo::MAX_TIMERS] = {};
    long long timer_n[bo::MAX_TIMERS] = {};
    std::vector<cudaEvent_t> iter_events;  // per iteration-in-graph: begin/end pairs
    std::vector<bo::EagerTimer> pending_timers;   // this object's open intervals

    // kernels launched for this object (direct launches, plus the kernel
    // nodes of every graph launch)
    long long launches = 0;
    std::vector<std::pair<cudaGraphExec_t, int>> graph_kernels;  // kernel nodes per graph
};

namespace bo {

// ---- launchers (defined in the .cu files) ---------------------------------
void launch_static(bo_sim* s);
void launch_hydrostatic(bo_sim* s, double p_top, double sw, double rgo);
void launch_equilibrium(bo_sim* s, const EquilDev& e);
void launch_begin_step(bo_sim* s);
void launch_begin_wells(bo_sim* s);   // datum, wellbore density, step-start well values
void launch_assemble(bo_sim* s, double dt);
void launch_norms(bo_sim* s, double dt);
void launch_fix_dead_wells(bo_sim* s);
void launch_well_init_bhp(bo_sim* s);
void launch_restore(bo_sim* s);

void setup_sweeps(bo_sim* s);
int sweep_timeout(bo_sim* s);
size_t ilu_storage(const bo_sim* s);
int tile_count(const bo_sim* s);                 // tiles of the wavefront schedule
void update_sweep_order(bo_sim* s);              // sweep tile lists after a block-Jacobi change
void setup_sweeps64(bo_sim* s);                  // FP64 sweep grid: residency check, tile lists
size_t face_storage(const bo_sim* s);
void enqueue_factor(bo_sim* s, cudaStream_t st, int* bad);
void enqueue_fwd(bo_sim* s, cudaStream_t st, const double* r, double* y, const KrylovScalars* ks);
void enqueue_bwd(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks);
void export_dinv(bo_sim* s, double* dinv);
size_t factors32_floats(const bo_sim* s);        // size of d_P32 (FP32 sweep layout)
size_t vec32_floats(const bo_sim* s);            // size of d_r32, d_y32 (tile order)
void convert_factors32(bo_sim* s, cudaStream_t st);
void reset_sweep_faces(bo_sim* s);                // sentinels of the current precision
void fill_sweep_faces(bo_sim* s, bool fp32);      // sentinels of the given precision
double wait_selftest(bo_sim* s);
void build_graphs(bo_sim* s);
void destroy_graphs(bo_sim* s);
void launch_factor(bo_sim* s);                       // graph of level kernels
void launch_precond(bo_sim* s, const double* r, double* z);
void launch_op(bo_sim* s, const double* x, double* y);
// returns LS_*; fp64: FP64 sweeps even in mixed mode (the fallback solve)
int run_bicgstab(bo_sim* s, double tol, int maxit, int* its, bool use_ml, bool fp64 = false);
// one-CTA solve of a small model (block_solve.cu)
bool block_solve_fits(const bo_sim* s);
bool block_solve_active(const bo_sim* s);
int run_block_bicgstab(bo_sim* s, double tol, int maxit, int max_restarts, int* its);
void launch_block_precond(bo_sim* s, const double* r, double* z);
void launch_well_recover(bo_sim* s);
// the preconditioner application of BiCGStab: ILU(0) or CPR, z = M^-1 r
void enqueue_precond_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                           const KrylovScalars* ks);
// the BiCGStab graphs store their iterations' residuals (online training or
// the offline set's collection)
inline bool learn_collecting(const bo_sim* s) { return s->ml_online || s->ml_collect_max > 0; }
void learn_set_clear(bo_sim* s);
// right-hand side of the well-reduced system into d_b
void enqueue_reduced_rhs(bo_sim* s, cudaStream_t st);
// K-subdomain solve (dd.cu): returns LS_*
int dd_bicgstab(bo_sim* s, double tol, int maxit, int* its);
void dd_free(bo_sim* s);
// y = b - S x with the well-reduced operator S (dot partials clobbered)
void enqueue_op_resid(bo_sim* s, cudaStream_t st, const double* x, double* y, const double* b,
                      const KrylovScalars* ks);

// The wells' part of the reduced operator for x: reduced wells write per rate
// well sop_w = (B_w . x) / D_w into the reduction scratch and return it (the
// cell rows subtract wC sop); full standard wells write C_w D_w^-1 B_w x per
// connection into d_wcorr and return null (the cell rows subtract d_wcorr).
const double* enqueue_well_dots(bo_sim* s, cudaStream_t st, const double* x,
                                const KrylovScalars* ks);
// the correction the cell rows read: d_wcorr for full wells, else null
inline const double* well_corr(const bo_sim* s) {
    return s->well_model == BO_WELL_MODEL_STANDARD ? s->d_wcorr : nullptr;
}

// full standard wells (wells_std.cu)
void std_wells_setup(bo_sim* s);                 // buffers, volumes, flags
void launch_std_wells_assemble(bo_sim* s, double dt);
void launch_std_wells_init(bo_sim* s);           // Q_t, F from the inflow after a state change
void enqueue_std_well_corr(bo_sim* s, cudaStream_t st, const double* x, const KrylovScalars* ks);
void enqueue_std_wells_rhs(bo_sim* s, cudaStream_t st, double* b);
void launch_std_wells_recover(bo_sim* s);
void launch_std_wells_update(bo_sim* s, const bo_newton_opts& o);

// CPR (cpr.cu)
void cpr_build(bo_sim* s);                   // aggregation hierarchy, once per model
void cpr_free(bo_sim* s);
void enqueue_cpr_setup(bo_sim* s, cudaStream_t st);   // per factorisation
void enqueue_cpr_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                       const KrylovScalars* ks);
void cpr_vcycle_host(bo_sim* s, const double* b, double* x);
void cpr_export_pressure(bo_sim* s, double* w, double* ap);
int cpr_levels(const bo_sim* s);
int cpr_level_size(const bo_sim* s, int l);
const std::vector<int>& cpr_aggregation(const bo_sim* s, int l);
int* cpr_status_ptr(bo_sim* s);
void launch_newton_update(bo_sim* s, const bo_newton_opts& o);

// learned preconditioner stage (learned.cu)
void learn_setup(bo_sim* s);                 // parameters, features, kernel attributes
void learn_setup_training(bo_sim* s);        // FP32 features and training vectors
void learn_set_params(bo_sim* s, const float* host);
void learn_get_params(bo_sim* s, float* host);
void learn_get_grad(bo_sim* s, float* host);
void learn_clear_grad(bo_sim* s);
void enqueue_learn_features(bo_sim* s, cudaStream_t st);
void enqueue_learn_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                         const KrylovScalars* ks);
void enqueue_learn_collect(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks);
double learn_loss_grad(bo_sim* s, const double* r);   // one sample; returns the loss
void learn_adam(bo_sim* s, double lr);

// Launch accounting: one kernel launched on st (not counted while st is being
// captured into a graph: a graph's kernels count when the graph is launched).
void count_launch(bo_sim* s, cudaStream_t st, int k = 1);
// Record the number of kernel nodes of a captured graph for its executable.
void note_graph(bo_sim* s, cudaGraph_t g, cudaGraphExec_t exec);
void graph_launch(bo_sim* s, cudaGraphExec_t exec, cudaStream_t st);

int timer_id(bo_sim* s, const char* name);
void timer_begin(bo_sim* s, int id);
void timer_end(bo_sim* s, int id);
void timers_flush(bo_sim* s);
void launch_wi(bo_sim* s, const int* d_con_well, const double* d_rw, const double* d_skin);
int props_blocks(const bo_sim* s);
int norm_blocks(const bo_sim* s);

void residual_norms_noalloc(const double* R, const double* pv, const double* b, int n, double dt,
                            double* out6, cudaStream_t stream);

// Convert between cell-major host vectors (3c+e) and SoA device vectors.
void upload_aos3(bo_sim* s, const double* host, double* dev);
void download_aos3(const bo_sim* s, const double* dev, double* host);

}  // namespace bo
