/*
 * bo.h -- C ABI of the GB300 black-oil Newton-step library (libbo.so).
 *
 * The library implements the fully-implicit black-oil Newton step of
 * arXiv 1910.06059 (OPM Flow): residual and Jacobian assembly by forward-mode
 * automatic differentiation over the cells and two-point-flux faces of a
 * Cartesian grid (Section 2.1.1, Eqs. materialbalance, acc, flux1, flux2,
 * head; Section 2.4), reduced standard wells coupled through the Schur
 * complement (Section 2.2.1, Eqs. wellinflow, wellequation), and the linear
 * solve by BiCGStab preconditioned with block ILU(0) (Section 2.3.1), inside a
 * Newton loop with Appleyard chop, variable switching and time-step cutting
 * (Section 2.3, Eq. linsystem).
 *
 * Conventions shared by every entry point
 *  - Units are SI: Pa, m, s, m^2 (permeability), Pa.s, surface m^3.
 *  - Cell index c = i + nx*(j + ny*k), 0-based, k counts layers downward.
 *  - Unknowns per cell y = (p_o, s_w, x) with x = s_g in state SAT (flag 0,
 *    gas present) or x = r_go in state USAT (flag 1, no free gas), following
 *    Eq. (primaryVariableMeaning).  Equations per cell are ordered
 *    (water, oil, gas) components.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Entry
 *    points named *_dev take device pointers (for example a torch tensor's
 *    data_ptr()) and read or write them on the library's stream; the caller
 *    keeps them alive until that stream has passed the call.
 *  - Every call returns a bo_status and never aborts the process.  On error
 *    bo_last_error() returns a message for the calling thread.  A CUDA error
 *    maps to BO_ERR_CUDA and leaves the object usable only for bo_destroy.
 *  - The library allocates its own device memory on the current device at
 *    bo_create_grid / bo_set_properties and frees it in bo_destroy.
 *  - Calls on one bo_sim are not thread-safe; distinct objects are independent.
 */
#ifndef BO_H
#define BO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bo_sim bo_sim; /* opaque; owns all of its device memory */

typedef enum {
    BO_OK = 0,
    BO_ERR_INVALID_ARG = 1,
    BO_ERR_CUDA = 2,
    BO_ERR_OOM = 3,
    BO_ERR_NOT_CONVERGED = 4,     /* Newton failed after all time-step cuts */
    BO_ERR_LINEAR_BREAKDOWN = 5,  /* BiCGStab breakdown or non-finite scalar */
    BO_ERR_DEVICE_TIMEOUT = 6,    /* a bounded device-side wait ran out */
    BO_ERR_STATE = 7              /* call out of order (e.g. solve before assemble) */
} bo_status;

/* Fluid and rock parameters (Sections 2.1.4-2.1.6).  The paper gives the
 * forms, not the values; the library evaluates:
 *   b_w = bw_ref exp(c_w (p - p_ref)), mu_w constant;
 *   r_s(p) = R_sb p / p_b; p_sat(r) = p_b r / R_sb;
 *   b_o = exp(c_o (p - p_sat(r_go))) / (1 + Bo_slope r_go);
 *   mu_o = mu_o0 / (1 + mu_o_r r_go) * exp(c_mu (p - p_sat(r_go)));
 *   b_g = p / (p_sc Z); mu_g = mu_g0 (1 + p / mu_g_p);  rho_a as in the
 *   paper's nomenclature; m_phi = exp(c_r (p - p_ref));
 *   Corey curves of exponent n_corey with end points s_wco, s_orw, s_org,
 *   combined by Eq. (gwseg).  rho_s = surface densities (w, o, g). */
typedef struct {
    double g, rho_s[3], p_ref, bw_ref, c_w, mu_w, R_sb, p_b, Bo_slope, c_o, mu_o0, mu_o_r, c_mu,
        p_sc, Z, mu_g0, mu_g_p, c_r, s_wco, s_orw, s_org, n_corey;
} bo_fluid;

/* One vertical standard well (Section 2.2.1) in reduced form: the only well
 * unknown is the bottom-hole pressure of a rate-controlled well.  Producing
 * connections carry every phase at its own mobility; injecting connections
 * carry the injected phase at the total mobility; reverse flow through a
 * connection is set to zero.  cells[0] is the datum (top) connection.  A
 * cell may belong to at most one connection of one well. */
typedef struct {
    int kind;          /* 0 injector, 1 producer */
    int phase;         /* injected phase of an injector: 0 water, 2 gas */
    int control;       /* 0 surface-rate control, 1 BHP control */
    int ncon;          /* number of connections */
    const int* cells;  /* ncon cell indices (host memory, copied) */
    double target;     /* rate control: surface m^3/s (> 0); BHP control: Pa */
    double bhp_limit;  /* rate control: BHP bound that switches the well to BHP control */
    double rw, skin;   /* well radius (m) and skin for the Peaceman index */
} bo_well;

/* Newton controls (Section 2.3).  Convergence: max_a MB_a <= tol_mb,
 * max_a CNV_a <= tol_cnv and every rate-controlled well's |R_w|/target <=
 * tol_well.  Appleyard chop per cell: |dp| <= dp_rel_max * p; (ds_w, ds_g)
 * scaled so that max |ds| <= ds_max; in USAT cells |dr_go| <= drs_rel_max *
 * R_sb, and the pressure may fall at most a fraction bp_overshoot below the
 * saturation pressure of the updated r_go (no far jump across the
 * saturated/undersaturated boundary).  Switching: SAT -> USAT when s_g < 0
 * (r_go = r_s(p)); USAT -> SAT when r_go > r_s(p) (1 + eps_switch) (s_g = 0).
 * Rate-controlled wells: the BHP may at most halve its distance to the
 * opening pressure (the BHP at which the first connection flows) per
 * iteration; a well assembled without any flowing connection is moved 0.1%
 * past its opening pressure and assembled again.
 * Linear solve to relative residual tol_lin within max_lin iterations; a
 * linear solve that misses it fails the Newton solve.  Sub-steps: the first
 * sub-step of a simulation is dt_init (<= 0: the whole report step); the
 * sub-step length is carried between report steps, multiplied after a
 * converged sub-step of k Newton iterations by 2 (k <= 4), 1.5 (k <= 8),
 * 1 (k <= 12) or 0.7, capped at the report step, and multiplied by
 * cut_factor after a failed one (at most max_cuts failures per report step). */
typedef struct {
    double tol_mb, tol_cnv, tol_well;
    int max_newton;
    double tol_lin;
    int max_lin, max_cuts;
    double ds_max, dp_rel_max, drs_rel_max, eps_switch;
    double bp_overshoot, dt_init, cut_factor;
} bo_newton_opts;

typedef struct {
    double tol;   /* stop when ||r||_2 <= tol * ||r_0||_2 */
    int max_it;
} bo_solve_opts;

typedef struct {
    int iterations;  /* BiCGStab iterations (a half-iteration exit counts as one) */
    int status;      /* 0 converged, 1 not converged in max_it, 2 breakdown */
    int restarts;    /* restarts from the true residual (see bo_solve) */
    double rel_res;  /* FP64 true residual ||b - Op x||_2 / ||b||_2 at exit */
    int fallback;    /* repeats after a failed attempt, bit mask: 1 without the
                        learned stage (bo_learn_enable), 2 with the FP64 sweeps
                        (BO_PRECISION_MIXED); iterations counts every attempt,
                        status, restarts and rel_res are the last attempt's */
} bo_solve_report;

typedef struct {
    int newton_its, lin_its, cuts, substeps, status;
    double mb[3], cnv[3], well_res;       /* last accepted norms */
    double ms_assemble, ms_factor, ms_solve, ms_update;  /* host-timed phases (ms) */
} bo_step_report;

/* Thread-local message describing the last failing call. */
const char* bo_last_error(void);

/* Grid of nx*ny*nz box cells; dx[nx], dy[ny], dz[nz] in m; top_depth is the
 * depth of the top face (depth increases downward).  Allocates the device
 * state on the current CUDA device. */
bo_status bo_create_grid(int nx, int ny, int nz, const double* dx, const double* dy,
                         const double* dz, double top_depth, bo_sim** out);

/* Rock, fluid and wells.  perm[3n] holds the permeability (m^2) along x, y
 * and z, component-major: perm[c] = kx, perm[n + c] = ky, perm[2n + c] = kz
 * of cell c (an isotropic rock repeats one array three times); every value
 * must be > 0 and finite.  poro[n] is the reference porosity.  Computes on
 * the device the static data of Appendix B -- transmissibilities as harmonic
 * means of half transmissibilities |F| k_d / (h_d / 2), k_d the
 * permeability along the face normal d -- pore volumes, depths and Peaceman
 * well indices WI = 2 pi k h / (ln(r_o / r_w) + skin) of the vertical
 * connections: k = kx and r_o = 0.14 sqrt(dx^2 + dy^2) when kx = ky, else
 * k = sqrt(kx ky) and r_o = 0.28 sqrt(sqrt(ky/kx) dx^2 + sqrt(kx/ky) dy^2) /
 * ((ky/kx)^(1/4) + (kx/ky)^(1/4)).  The arrays are copied; the caller keeps
 * ownership. */
bo_status bo_set_properties(bo_sim* sim, const double* perm, const double* poro,
                            const bo_fluid* fluid, const bo_well* wells, int nwells);

/* Static data for checking: Tx, Ty, Tz (transmissibility of each cell's
 * +x, +y, +z face, 0 on the boundary), pv, depth (each [n]); wi[total
 * connections] in well order.  Any pointer may be NULL. */
bo_status bo_get_static(const bo_sim* sim, double* Tx, double* Ty, double* Tz, double* pv,
                        double* depth, double* wi);

/* Initial state: USAT cells with r_go = rgo and s_w = sw; pressure in
 * discrete hydrostatic equilibrium of the oil column (Section 2.1.3 with the
 * face density of Eq. head), p = p_top at the centre of the top layer.  Well
 * BHPs start at their target (BHP control) or limit (rate control); a
 * rate-controlled injector starts at the BHP that meets its target by the
 * linear inflow relation with all connections injecting, capped by its limit. */
bo_status bo_init_hydrostatic(bo_sim* sim, double p_top, double sw, double rgo);

/* Initial state in vertical equilibrium (Section 2.1.3) from a datum
 * pressure and the water-oil and gas-oil contact depths (depths positive
 * downward, SI units).  Each zone's phase pressure solves dp/dz = rho(p) g by
 * classical 4th-order Runge-Kutta in max(1, ceil(|dz| / 1 m)) equal steps:
 * the datum's zone from the datum, the zones above and below from the
 * contacts, where the phase pressures are equal (this model has no capillary
 * pressure).  Zones: gas above goc_depth, oil between, water below
 * woc_depth.  Cells: oil zone s_w = swc; gas zone s_w = swc, s_g = 1 - swc -
 * s_org (saturated); water zone s_w = 1 - s_orw; oil carries
 * min(rgo, r_s(p)) and is undersaturated (x = rgo) when rgo < r_s(p), else
 * saturated with s_g = 0.  Wells start as after bo_init_hydrostatic.
 * BO_ERR_INVALID_ARG unless datum_pressure > 0, goc_depth <= woc_depth,
 * rgo >= 0 and 0 <= swc < 1 - s_orw - s_org. */
typedef struct {
    double datum_depth, datum_pressure, woc_depth, goc_depth, rgo, swc;
} bo_equil;
bo_status bo_init_equilibrium(bo_sim* sim, const bo_equil* eq);

/* State I/O.  p, sw, x are [n] doubles, flag [n] bytes (0 SAT, 1 USAT),
 * well_bhp [nwells] (may be NULL when there are no wells). */
bo_status bo_set_state(bo_sim* sim, const double* p, const double* sw, const double* x,
                       const unsigned char* flag, const double* well_bhp);
bo_status bo_get_state(const bo_sim* sim, double* p, double* sw, double* x,
                       unsigned char* flag, double* well_bhp);
bo_status bo_set_state_dev(bo_sim* sim, const double* p, const double* sw, const double* x,
                           const unsigned char* flag, const double* well_bhp);
bo_status bo_get_state_dev(const bo_sim* sim, double* p, double* sw, double* x,
                           unsigned char* flag, double* well_bhp);

/* Stream for every subsequent device operation (a cudaStream_t, e.g. torch's
 * current stream); NULL selects the legacy default stream. */
bo_status bo_set_stream(bo_sim* sim, void* cuda_stream);

/* Start of a time step: stores the accumulation terms A0 at the current
 * state, freezes each well's datum density (explicit over the step,
 * Section 2.2.1), resets well controls, and saves the state for a cut. */
bo_status bo_begin_step(bo_sim* sim);

/* Residual R and Jacobian J at the current state for step length dt
 * (Eq. materialbalance); stays on the device. */
bo_status bo_assemble(bo_sim* sim, double dt);

/* Convergence measures of the last assembly: out[0..2] MB_a, out[3..5]
 * CNV_a (a = w, o, g), out[6] max relative rate-well residual.
 * MB_a = dt Bavg_a |sum_i R_a,i| / sum_i PV_i; CNV_a = dt Bavg_a max_i |R_a,i| / PV_i,
 * Bavg_a = mean over cells of 1/b_a. */
bo_status bo_norms(bo_sim* sim, double dt, double* out7);

/* Copy-out of the last assembly as 3x3-block CSR with row-major blocks
 * (J[r][c] = dR_r,i / dy_c,j), natural cell order, columns ascending:
 * rowptr[n+1], colind[nnzb], vals[9*nnzb], res[3n] (cell-major).  Any
 * pointer may be NULL.  *nnzb_out (may be NULL) receives nnzb. */
bo_status bo_get_system(const bo_sim* sim, int* rowptr, int* colind, double* vals, double* res,
                        int* nnzb_out);

/* Well linearisation of the last assembly: per well R_w, D_w, control, and
 * per connection B (3 = dR_w/dy) and C (3 = dR/dp_bhp), packed in well order. */
bo_status bo_get_wells(const bo_sim* sim, double* Rw, double* Dw, double* B, double* C,
                       int* control);

/* Well model (Section 2.2.1).  BO_WELL_REDUCED (default): the reduced
 * standard well, one unknown per rate-controlled well (its BHP), no
 * cross-flow.  BO_WELL_STANDARD: the full standard well -- four unknowns per
 * well, the weighted total rate Q_t, the weighted fractions F_w, F_g
 * (Eq. weighted_total_rate, weights g = (1, 1, 0.01)) and p_bhp; connection
 * inflow by Eq. (wellinflow) with cross-flow (an injecting connection of a
 * producer carries the wellbore mixture); one balance per component with,
 * when storage != 0, the wellbore storage A_a = V_w F_a / g_a, V_w = pi r_w^2
 * times the perforated thickness (Eq. conseq-swell); the control of
 * Eqs. (well-control-bhp/rate); the Schur complement of Eq. (wellequation)
 * with a 4x4 D_w per well.  An injector's wellbore holds its injected phase
 * (F fixed).  The well unknowns are initialised by the next bo_set_state,
 * bo_init_hydrostatic or bo_init_equilibrium (a producer's Q_t and F from
 * its inflow at that state and BHP), which must follow this call.
 * BO_ERR_STATE before bo_set_properties; BO_ERR_INVALID_ARG for another
 * model. */
/* Residency of the FP64 triangular sweeps' persistent CTAs: k = 1 or 2 per
 * SM (default 2).  With two, the row warps of the two CTAs on an SM share the
 * sub-partitions' FP64 pipes; with one, fewer tiles of the wavefront are in
 * flight at once.  Re-records the solver graphs.  BO_ERR_INVALID_ARG for
 * another k, BO_ERR_STATE before bo_set_properties. */
bo_status bo_set_sweep_ctas_per_sm(bo_sim* sim, int k);

#define BO_WELL_REDUCED 0
#define BO_WELL_STANDARD 1
bo_status bo_set_well_model(bo_sim* sim, int model, int storage);
bo_status bo_get_well_model(const bo_sim* sim, int* model);

/* Full standard wells (BO_WELL_STANDARD): the blocks of Eq. (wellequation)
 * at the last assembly -- B[ncon][4][3] = dR_w / dy_c of each connection's
 * cell, C[ncon][3][4] = dR_c / dx_w of the cell row, both in connection
 * order (well by well, the connections in the order given), D[nw][4][4] =
 * dR_w / dx_w and Rw[nw][4] (rows: the water, oil and gas balances -- for
 * an injector the injected phase's balance, F_w - F_w,inj, F_g - F_g,inj --
 * then the control) -- and the current unknowns xw[nw][4] = (Q_t, F_w, F_g,
 * p_bhp).  x_w variables are ordered (Q_t, F_w, F_g, p_bhp), cell variables
 * (p_o, s_w, x).  Any pointer may be NULL; B, C, D, Rw need an assembly
 * (BO_ERR_STATE otherwise, and when the model is not selected). */
bo_status bo_get_std_wells(const bo_sim* sim, double* B, double* C, double* D, double* Rw,
                           double* xw);

/* Well production report (Section 2.2.1): per well the surface rates of
 * water, oil and gas (m^3/s at surface conditions, the connection inflows of
 * Eq. (wellinflow) summed over the well's connections, gas including the
 * dissolved gas of the produced oil) at the state of the last assembly, production positive
 * and injection negative; after a successful bo_step that is the converged
 * state of its last sub-step.  rates[3*nwells] (well-major), bhp[nwells]
 * (Pa, current), control[nwells] (0 rate, 1 BHP, current); any pointer may
 * be NULL.  Zero rates before the first assembly.  Requires
 * bo_set_properties (BO_ERR_STATE otherwise). */
bo_status bo_get_well_rates(const bo_sim* sim, double* rates, double* bhp, int* control);

/* Block ILU(0) of the last assembly's reservoir matrix A in natural order.
 * On the 7-point pattern only the diagonal blocks change (the grid graph is
 * bipartite, so no fill position of ILU(0) lies in the pattern), giving
 * M = (L_A + D) D^-1 (D + U_A) with D_i = A_ii - sum_k A_ik D_k^-1 A_ki.
 * dinv (may be NULL) receives D_i^-1, [n][3][3] row-major. */
bo_status bo_factor(bo_sim* sim, double* dinv);

/* z = M^-1 r with the factors of the last bo_factor; r, z are [3n] host
 * arrays in cell-major order.  In BO_PRECISION_MIXED the sweeps run on the
 * FP32 factors in FP32 arithmetic (r and z stay FP64). */
bo_status bo_precond_apply(bo_sim* sim, const double* r, double* z);

/* y = (A - sum_w C_w D_w^-1 B_w) x, the well-reduced operator of
 * Eq. (wellequation); x, y are [3n] host arrays in cell-major order. */
bo_status bo_apply_op(bo_sim* sim, const double* x, double* y);

/* Linear solve J sol = R of the last assembly: factors, then right-
 * preconditioned BiCGStab on the reduced system, then the well unknowns.
 * The iteration stops on the recurrence's residual; the FP64 true residual
 * ||b - Op x|| is then computed and must meet the same tolerance, else
 * BiCGStab restarts from it (at most 8 times, within max_it) and the solve
 * reports not converged if it still misses.  A solve that fails with the
 * learned stage on is repeated without it, and one that fails with the FP32
 * sweeps of BO_PRECISION_MIXED is repeated with the FP64 sweeps (each repeat
 * from a zero initial guess with a fresh max_it; report->fallback says which
 * ran).
 * sol (may be NULL) receives [3n + nwells] (cell-major, then one entry per
 * well, 0 for wells without an unknown); with BO_WELL_STANDARD [3n + 4
 * nwells], four entries per well (Q_t, F_w, F_g, p_bhp). */
bo_status bo_solve(bo_sim* sim, const bo_solve_opts* opts, bo_solve_report* report,
                   double* sol);

/* The same linear solve as K subdomains (Section 2.5: each process owns the
 * rows of its subdomain, exchanges one ghost layer before every operator
 * product, applies ILU(0) to its own block and joins the inner products by
 * an all-reduce), emulated on one GPU.  The subdomains are the y slabs set
 * by bo_set_subdomains (ysub > 0, zsub = 0; K = ceil(ny / ysub)); the
 * Krylov vectors and the Jacobian rows live in a subdomain-local layout with
 * ghost rows, the halo exchange is a device copy, each inner product is a
 * per-subdomain sum followed by a sum over the subdomains in order, and the
 * preconditioner is the same block-Jacobi ILU(0) as bo_solve's (so the
 * iteration equals bo_solve's up to the grouping of the inner products).
 * The scalars of the iteration come back to the host once per
 * half-iteration (no CUDA graph).  Requires FP64 sweeps, ILU(0), the reduced
 * well model and no learned stage (BO_ERR_STATE otherwise); sol and report
 * as for bo_solve (restarts, rel_res and fallback are reported as 0). */
bo_status bo_dd_solve(bo_sim* sim, const bo_solve_opts* opts, bo_solve_report* report,
                      double* sol);

/* Newton update from the last bo_solve: dy = -sol with chop and variable
 * switching as in bo_newton_opts; wells on rate control that pass their BHP
 * limit switch to BHP control. */
bo_status bo_newton_update(bo_sim* sim, const bo_newton_opts* opts);

/* One report step of length dt with Newton iterations and time-step cuts.
 * On BO_ERR_NOT_CONVERGED the state is restored to the start of the step. */
bo_status bo_step(bo_sim* sim, double dt, const bo_newton_opts* opts, bo_step_report* report);

/* Sub-step length carried into the next report step (s; 0 = not started),
 * part of the simulation state for checkpoint and restart. */
bo_status bo_get_step_control(const bo_sim* sim, double* dt_next);
bo_status bo_set_step_control(bo_sim* sim, double dt_next);

/* Per-kernel timing of the device kernels launched inside bo_step/bo_solve
 * while enabled (CUDA events on the library stream).  names receive up to
 * max entries of "name\0", ms_total and launches are per entry. */
bo_status bo_set_timing(bo_sim* sim, int enabled);
bo_status bo_get_timing(const bo_sim* sim, int max, char (*names)[32], double* ms_total,
                        long long* launches, int* count);

/* Preconditioner of BiCGStab (Section 2.3.1).  BO_PRECOND_ILU0 (default):
 * block ILU(0) (block-Jacobi boxes when bo_set_subdomains cuts them).
 * BO_PRECOND_CPR: the two-stage constrained-pressure-residual method the
 * section names for large cases: quasi-IMPES weights w_c = A_cc^-T e_p, the
 * 7-point pressure matrix A_p = W^T A E_p, one V-cycle of plain-aggregation
 * AMG on A_p (two damped-Jacobi sweeps, omega 2/3, each way; exact solve on
 * the coarsest level) as the first stage, block ILU(0) on the remaining
 * residual as the second: z = x1 + M^-1 (r - S x1), x1 = E_p V(W^T r).  The
 * aggregation hierarchy is built once per model from the face
 * transmissibilities (strength 0.25, greedy aggregates, down to 200
 * unknowns) on the first selection; each factorisation recomputes the
 * weights, A_p and its Galerkin coarse operators.  Switching re-records the
 * BiCGStab graphs.  Errors: BO_ERR_INVALID_ARG for an unknown kind,
 * BO_ERR_STATE before bo_set_properties. */
#define BO_PRECOND_ILU0 0
#define BO_PRECOND_CPR 1
bo_status bo_set_preconditioner(bo_sim* sim, int kind);
bo_status bo_get_preconditioner(const bo_sim* sim, int* kind);

/* Schedule of the linear solve (Section 2.3.1's ILU0-BiCGStab; the paper runs
 * it as a sequence of parallel kernels, which is BO_SCHEDULE_TILED here).
 * BO_SCHEDULE_TILED (default): the wavefront-tiled sweeps and vector kernels
 * over the whole GPU, replayed as CUDA graphs of a few iterations each.
 * BO_SCHEDULE_BLOCK: the whole solve (reduced right-hand side aside) is ONE
 * launch of ONE 256-thread CTA: triangular sweeps by levels i + j + k inside
 * the CTA, the operator, the dot products, the recurrence and its true
 * residual checks and restarts, with the tiled factorisation's ILU(0) data;
 * meant for small models stepped side by side (an ensemble), where it frees
 * the rest of the GPU for the other models.  Same recurrence and stopping
 * rules, results equal to rounding.  It applies while the preconditioner is
 * FP64 ILU(0) without block-Jacobi cuts, the wells are the reduced standard
 * wells (at most 128), no learned stage runs and ceil(ny/8) ceil(nz/4) <= 128;
 * otherwise the tiled schedule runs.  bo_precond_apply follows the schedule.
 * Errors: BO_ERR_INVALID_ARG for an unknown kind or a NULL sim. */
#define BO_SCHEDULE_TILED 0
#define BO_SCHEDULE_BLOCK 1
bo_status bo_set_solve_schedule(bo_sim* sim, int kind);
bo_status bo_get_solve_schedule(const bo_sim* sim, int* kind);

/* The CPR aggregation hierarchy (for checking): *nlevels levels, sizes[l]
 * unknowns on level l (up to max_levels entries), agg = the maps of levels
 * 0 .. nlevels-2 concatenated (agg[off_l + i] = aggregate of node i of level
 * l, off_l = sizes[0] + ... + sizes[l-1]); agg may be NULL.  BO_ERR_STATE
 * when CPR has never been selected. */
bo_status bo_cpr_hierarchy(const bo_sim* sim, int max_levels, int* nlevels, int* sizes, int* agg);

/* CPR pressure system of the last bo_factor (for checking): w [n][3]
 * quasi-IMPES weights and ap [n][7] pressure-matrix entries per cell in the
 * order diag, -x, +x, -y, +y, -z, +z (zero where no neighbour).  Host arrays,
 * either may be NULL.  BO_ERR_STATE without a CPR factorisation. */
bo_status bo_cpr_pressure_system(bo_sim* sim, double* w, double* ap);

/* One CPR V-cycle on the pressure matrix of the last bo_factor: x = V(A_p) b,
 * b and x host arrays of n values.  BO_ERR_STATE without a CPR
 * factorisation. */
bo_status bo_cpr_vcycle(bo_sim* sim, const double* b, double* x);

/* Kernels the library has launched for this object since it was created:
 * every direct launch counts one, every launch of a captured CUDA graph
 * counts the graph's kernel nodes (a kernel that returns at once because its
 * solve has finished still counts).  Diagnostics for benchmarks, no
 * counterpart in the paper.  count: host pointer, required. */
bo_status bo_get_launch_count(const bo_sim* sim, long long* count);

/* Precision of the ILU(0) preconditioner.  BO_PRECISION_FP64 (the default):
 * factors stored and applied in FP64.  BO_PRECISION_MIXED: the factors are
 * computed in FP64; the scaled off-diagonal blocks are stored rounded to
 * FP32 (a second copy, 56 x 4 bytes per cell slot, allocated at the first
 * switch) and both triangular sweeps run in FP32 (the pivot inverse is
 * applied in FP64 before the forward sweep); residual assembly, the Krylov vectors and scalars, the operator,
 * the true-residual check of bo_solve and the Newton convergence test stay
 * FP64.  The preconditioner is only an approximation of J^-1, so the
 * precision of its application changes iteration counts, not the converged
 * Newton state beyond the tolerances.  A solve the FP32 sweeps fail is
 * repeated with the FP64 factors and sweeps (bo_solve).  Switching re-records the solver's
 * CUDA graphs and converts factors already computed.  Requires
 * bo_set_properties; BO_ERR_INVALID_ARG for another value. */
enum { BO_PRECISION_FP64 = 0, BO_PRECISION_MIXED = 1 };
bo_status bo_set_precision(bo_sim* sim, int precision);
bo_status bo_get_precision(const bo_sim* sim, int* precision);

/* Block-Jacobi ILU(0), the parallel preconditioner of Section 2.5 (one
 * ILU(0) block per subdomain), on one GPU: the grid is cut into slabs of
 * ysub cell rows in y and of zsub cell layers in z (the last slab in each
 * direction may be shorter; the subdomains are the boxes the two sets of
 * cuts make) and the factorisation leaves out every block that couples two
 * subdomains; the operator keeps them.  The subdomains' wavefronts then run
 * side by side, so a sweep takes about nx + min(ny, ysub) + min(nz, zsub)
 * levels instead of nx + ny + nz.  0 means no cut in that direction, so
 * (0, 0) restores plain ILU(0).  ysub must be 0 or a positive multiple of 8
 * and zsub 0 or a positive multiple of 4 (the tile extents of the sweeps);
 * BO_ERR_INVALID_ARG otherwise.  Requires bo_set_properties; the factors of
 * an earlier bo_factor are dropped (factor again).  bo_get_subdomains
 * writes either value to a non-NULL pointer. */
bo_status bo_set_subdomains(bo_sim* sim, int ysub, int zsub);
bo_status bo_get_subdomains(const bo_sim* sim, int* ysub, int* zsub);
/* Learned correction of the preconditioner, an extension of the ILU(0)-
 * preconditioned BiCGStab of Section 2.3.1.  With the stage on, every
 * preconditioner application inside BiCGStab becomes
 *     z = M^-1 r + delta(r),  delta_c = sigma_c (W_c rhat_c),  W_c = N(f_c),
 * N a 63 -> 128 -> 128 -> 9 ReLU MLP of the cell's normalised Jacobian row
 * (diagonal block and the -x, +x, -y, +y, -z, +z blocks, each entry
 * A[e][v] sigma_nb[v] / rho_e with sigma = (1e6 Pa, 0.05, 0.05 for s_g or 5
 * for r_go) and rho_e = max_v |A_cc[e][v]| sigma_c[v]); W_c[v][e] =
 * N[3 v + e] acts on the row-scaled residual rhat_c[e] = r_c[e] / rho_e.
 * The correction is linear in r, so for one Jacobian the preconditioner is
 * one fixed linear map.  The network runs once per factorisation on the
 * tensor cores (BF16 weights and activations, FP32 accumulation); each
 * application is a per-cell 3x3 product.  A solve that fails with the
 * stage is repeated with plain ILU(0) (counted as a fallback).
 *
 * Parameters: BO_LEARN_NPARAM values, flat, in the order W1[128][63],
 * b1[128], W2[128][128], b2[128], W3[9][128], b3[9] (row-major, h = W x + b).
 * Training (FP32, on the device) minimises ||r - A (M^-1 r + delta(r))||^2 /
 * ||r||^2 with Adam over residuals the solver produces, A being the
 * reservoir Jacobian of the last assembly (the well coupling is left out). */
#define BO_LEARN_NPARAM 25865
typedef struct {
    int samples;    /* residuals kept per linear solve (the first iterations'), 1..64 */
    int epochs;     /* passes over them after each solve, 1..100 */
    double lr;      /* Adam step size, 0 < lr < 1 */
} bo_learn_opts;
typedef struct {
    long long systems;      /* linear systems trained on */
    long long steps;        /* Adam steps */
    long long fallbacks;    /* solves repeated with plain ILU(0) */
    double first_loss;      /* mean loss over the first epoch on the first system (-1: none) */
    double last_loss;       /* mean loss over the last epoch on the last system (-1: none) */
    double train_ms;        /* host wall time spent training */
    long long guard_stage_its;   /* BiCGStab iterations with the stage over the guard window */
    long long guard_plain_its;   /* and with plain ILU(0) on the same systems */
    int guard_state;        /* 0 no guard, 1 probing, 2 stage kept, 3 stage turned off */
} bo_learn_report;

/* Parameters from / to host doubles (rounded to FP32 on the device); nparam
 * must be BO_LEARN_NPARAM.  Setting them resets the Adam state. */
bo_status bo_learn_set_params(bo_sim* sim, const double* theta, int nparam);
bo_status bo_learn_get_params(bo_sim* sim, double* theta, int nparam);
/* Stage on (1) or off (0) inside BiCGStab (bo_solve, bo_step); re-records the
 * solver graphs.  Requires parameters. */
bo_status bo_learn_enable(bo_sim* sim, int on);
/* Tensor-core kernel of the network (run once per factorisation):
 * BO_LEARN_ENGINE_TCGEN05 (default) issues tcgen05.mma kind::f16 from one
 * thread per CTA on 128-cell tiles with the accumulators in tensor memory;
 * BO_LEARN_ENGINE_MMA_SYNC uses warp-level mma.sync m16n8k16.  Both take BF16
 * weights and activations with FP32 accumulation (results equal up to the
 * order of the FP32 sums).  A tcgen05 layer that does not complete within its
 * bounded wait fails the factorisation (the linear solve reports a
 * breakdown).  BO_ERR_INVALID_ARG for another value. */
/* Offline training set of the learned stage (the simulator's own earlier
 * systems).  bo_learn_collect with max_systems > 0 clears the set and, from
 * then on, keeps every linear solve's system -- its Jacobian, ILU(0) data,
 * FP32 features and per-cell scalings -- with the first `samples` (1..64)
 * BiCGStab residuals of its solve, until max_systems are kept or the device
 * has no room left; max_systems = 0 stops collecting and keeps the set.
 * Needs parameters (BO_ERR_STATE); with online training on, samples must be
 * its own count.  Memory: about 0.9 KB per cell plus 24 B per cell and
 * residual for every kept system.
 * bo_learn_set_info: the kept systems and residuals (either pointer may be
 * NULL).
 * bo_learn_train_offline: `epochs` passes of one Adam step (step size lr) per
 * kept residual, each on its own system (the loss of bo_learn_loss_grad);
 * first_loss / last_loss (may be NULL) receive the mean loss over the first
 * and over the last pass.  Needs a non-empty set, parameters and the FP64
 * ILU(0) preconditioner (BO_ERR_STATE). */
bo_status bo_learn_collect(bo_sim* sim, int max_systems, int samples);
bo_status bo_learn_set_info(const bo_sim* sim, int* systems, int* residuals);
bo_status bo_learn_train_offline(bo_sim* sim, int epochs, double lr, double* first_loss,
                                 double* last_loss);

#define BO_LEARN_ENGINE_MMA_SYNC 0
#define BO_LEARN_ENGINE_TCGEN05 1
bo_status bo_learn_set_engine(bo_sim* sim, int engine);
bo_status bo_learn_get_engine(const bo_sim* sim, int* engine);
/* Online training: with opts non-NULL every later linear solve (bo_solve,
 * bo_step) keeps its first opts->samples BiCGStab residuals and then takes
 * opts->epochs Adam passes over them on that system; NULL turns it off.
 * Requires parameters; BO_ERR_INVALID_ARG for values out of range. */
bo_status bo_learn_online(bo_sim* sim, const bo_learn_opts* opts);
bo_status bo_learn_get_report(const bo_sim* sim, bo_learn_report* report);
/* Guard of the stage: with the stage on, each of the next `probe` linear
 * solves is repeated with plain ILU(0) on the same system (the plain
 * solution is the one used, so the Newton path is the method's own); after
 * the window the stage stays on only if it needed fewer BiCGStab iterations
 * in total than plain ILU(0), else it is turned off (bo_learn_report's
 * guard fields record the counts and the decision).  probe = 0 cancels a
 * window.  BO_ERR_INVALID_ARG for probe < 0, BO_ERR_STATE without the stage
 * on.  (The paper has no learned stage; this is the stage's own check that
 * it pays, against the Section 2.3.1 method it corrects.) */
bo_status bo_learn_guard(bo_sim* sim, int probe);
/* delta(r) on the last assembly with the tensor-core kernel; r, delta are
 * [3n] host arrays in cell-major order.  Requires a factorisation of the
 * last assembly and parameters. */
bo_status bo_learn_delta(bo_sim* sim, const double* r, double* delta);
/* One FP32 training pass on the last assembly and factorisation for the
 * host residual r [3n]: *loss (may be NULL) and the gradient grad
 * [BO_LEARN_NPARAM] (may be NULL); parameters are not changed. */
bo_status bo_learn_loss_grad(bo_sim* sim, const double* r, double* loss, double* grad);

/* Ensembles (the batched form): many independent models of uneven size
 * advanced together on one GPU.  Each member keeps its own Newton loop,
 * time-step control and solver (Section 2.3 per member); the ensemble steps
 * the members concurrently from a pool of host workers, each on its own CUDA
 * stream, handing out members largest first (or in the given order).  The
 * caller creates, initialises and destroys the members; the ensemble holds
 * pointers to them and must be destroyed first.  A member is stepped by one
 * worker at a time; while it is being stepped its stream is the worker's.
 *
 * bo_ensemble_create: count distinct members (bo_set_properties done),
 *   `streams` concurrent workers (1..256); BO_ERR_INVALID_ARG / BO_ERR_STATE.
 * bo_ensemble_set_schedule / get_schedule: workers (1..256) and order
 *   (largest_first = 1: by decreasing cell count, 0: the members' order).
 * bo_ensemble_step: one report step of length dt for every member, as
 *   bo_step would take it; reports[count] and statuses[count] (each may be
 *   NULL) receive each member's report and status; returns BO_OK if every
 *   member succeeded, else the first failing member's status (its message is
 *   not kept: call bo_step on that member alone to see it).
 * bo_ensemble_autotune: times one probe report step of length dt_probe for
 *   every candidate worker count (candidates[ncand], each 1..256) in both
 *   orders, putting every member's state and step control back after each
 *   probe, and keeps the fastest schedule whose probe succeeded;
 *   seconds[2 * ncand] (may be NULL) receives the probe times, largest-first
 *   order first.  BO_ERR_NOT_CONVERGED if no probe succeeded.
 * bo_ensemble_last_step_ms: device time of the last bo_ensemble_step (or
 *   autotune probe) in milliseconds, measured with CUDA events: from an
 *   event every worker stream waits on before its first member to an event
 *   recorded after every worker stream's last member; -1 when it could not
 *   be measured. */
typedef struct bo_ensemble bo_ensemble;
bo_status bo_ensemble_create(bo_sim* const* members, int count, int streams, bo_ensemble** out);
bo_status bo_ensemble_set_schedule(bo_ensemble* ens, int streams, int largest_first);
bo_status bo_ensemble_get_schedule(const bo_ensemble* ens, int* streams, int* largest_first);
bo_status bo_ensemble_step(bo_ensemble* ens, double dt, const bo_newton_opts* opts,
                           bo_step_report* reports, bo_status* statuses);
bo_status bo_ensemble_autotune(bo_ensemble* ens, double dt_probe, const bo_newton_opts* opts,
                               const int* candidates, int ncand, double* seconds);
bo_status bo_ensemble_last_step_ms(const bo_ensemble* ens, double* ms);
/* Preconditioner per member size class: members up to the median cell count
 * and the larger ones each get BO_PRECOND_ILU0 or BO_PRECOND_CPR; one probe
 * report step of length dt_probe (with the current worker schedule) times
 * each of the four combinations, putting every member's state and step
 * control back after each, and the fastest one whose probe stepped every
 * member is kept.  seconds[4] (may be NULL) receives the probe times in the
 * order (ILU0, ILU0), (ILU0, CPR), (CPR, ILU0), (CPR, CPR) for (small,
 * large); small_kind / large_kind (may be NULL) the choice.
 * BO_ERR_NOT_CONVERGED if no combination stepped every member (the members'
 * preconditioners are then as before). */
bo_status bo_ensemble_autotune_precond(bo_ensemble* ens, double dt_probe, const bo_newton_opts* opts,
                                      double* seconds, int* small_kind, int* large_kind);
/* Solve schedule of the small members (up to the median cell count; the
 * larger ones keep BO_SCHEDULE_TILED) and the number of worker streams: one
 * probe report step of length dt_probe times each of (BO_SCHEDULE_TILED, w),
 * (BO_SCHEDULE_BLOCK, w), (BO_SCHEDULE_TILED, w4), (BO_SCHEDULE_BLOCK, w4),
 * w the current worker count and w4 = min(256, 4 w) (one-CTA solves leave
 * the SMs to other members, so more of them can run at once), putting every
 * member's state and step control back after each; the fastest combination
 * whose probe stepped every member is kept.  seconds[4] (may be NULL)
 * receives the probe times in that order, *small_schedule and *streams (may
 * be NULL) the choice.  BO_ERR_NOT_CONVERGED if no combination stepped every
 * member (schedules and worker count are then as before). */
bo_status bo_ensemble_autotune_schedule(bo_ensemble* ens, double dt_probe, const bo_newton_opts* opts,
                                       double* seconds, int* small_schedule, int* streams);
bo_status bo_ensemble_destroy(bo_ensemble* ens);

/* Self-test of failure detection: runs the bounded device-side wait of the
 * wavefront sweeps on a face slot that nothing ever writes.  The wait runs
 * out after about one second, the kernel records it and returns, and the
 * call reports BO_ERR_DEVICE_TIMEOUT with *seconds (may be NULL) = the time
 * the wait took; the context stays usable.  Any other status is a failure
 * of the mechanism.  (The paper has no counterpart; Section 2.3's
 * time-step cutting is the host-side part of failure handling.) */
bo_status bo_selftest_bounded_wait(bo_sim* sim, double* seconds);

/* Convergence measures of a residual for callers that cannot allocate device
 * memory (for example a host application or plugin that owns the whole
 * device memory budget and hands out only its own buffers, or code that
 * must not let an allocation synchronise the device).  The paper has no
 * counterpart: it is the measure of bo_norms on caller-owned buffers.
 * All pointers are device pointers owned by the caller:
 *   R    [3][n] residual, component-major (R[a*n + i], a = w, o, g);
 *   pv   [n]    pore volumes;
 *   b    [3][n] shrinkage factors b_a of every cell;
 *   out6 [6]    receives MB_a (0..2) and CNV_a (3..5) as defined at bo_norms.
 * n must be 1 .. 8,388,608: the per-block partial sums live in a fixed
 * file-scope device array of 4096 x 10 doubles (320 KB), held in every CUDA
 * context that has loaded the library's device code until that context
 * ends; larger n is rejected with BO_ERR_INVALID_ARG.  The call itself
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library
 * routine).  First call in a context: CUDA loads a library's device code
 * lazily, so the first call in each context (the device's primary context,
 * a caller's own driver-API context, or a context re-created after
 * cudaDeviceReset) loads the module, which places the array in device
 * memory, and looks up the array's address in that context; make it once
 * at start-up, before the memory budget is fixed and before any stream
 * capture (CUDA_MODULE_LOADING=EAGER loads the module with the context
 * instead).  Later calls in the same context reuse the address.  It runs
 * asynchronously on `stream` (a cudaStream_t or NULL).  A NaN anywhere in R
 * makes the MB and CNV results NaN.  Every call shares the one array and
 * overwrites what it reads, so nothing needs clearing, but calls that
 * overlap on the GPU race on it. */
bo_status bo_residual_norms_noalloc(const double* R, const double* pv, const double* b, int n,
                                    double dt, double* out6, void* stream);

/* Number of cells, wells, connections, and nonzero blocks of the pattern. */
bo_status bo_sizes(const bo_sim* sim, int* n, int* nwells, int* ncon, int* nnzb);

/* Release all device memory of the object. */
bo_status bo_destroy(bo_sim* sim);

#ifdef __cplusplus
}
#endif
#endif /* BO_H */
