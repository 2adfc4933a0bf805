// CPU FP64 oracle for the fully-implicit black-oil Newton step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, sequential
// reference that the CUDA library is checked against.  Only the test suite,
// the smoke check and the benchmark's CPU-baseline leg may build, load or call
// it; the product path never does.  It shares no code with the CUDA library.
//
// What it computes, with the paper's notation (arXiv 1910.06059):
//   * Discrete residual, Eq. (materialbalance), Section 2.1.1:
//       R_a,i = phi_ref,i V_i / dt (A_a,i - A0_a,i) + sum_j u_a,ij + q_a,i
//     with the accumulation terms of Eq. (acc) for dry gas (r_og = 0):
//       A_w = m_phi b_w s_w, A_o = m_phi b_o s_o, A_g = m_phi (b_g s_g + r_go b_o s_o).
//   * TPFA fluxes, Eqs. (flux1), (flux2), (head): upwinded b lambda times
//     T_ij times the potential difference, with the arithmetic-mean density
//     and the upwind cell chosen on the sign of the potential (>= 0: cell i).
//   * Transmissibility, Appendix B: harmonic combination of the two
//     half-transmissibilities t = |F| k / (distance centre to face).
//   * Three-phase oil relative permeability by segregation, Eq. (gwseg).
//   * Standard-well inflow, Eq. (wellinflow), in the reduced one-unknown
//     form (BHP only) and the Schur complement of Eq. (wellequation).
//   * Jacobian by forward-mode automatic differentiation (Section 2.4):
//     a value carried together with its derivatives; products by the
//     product rule.
//   * Newton iteration, Eq. (linsystem), with Appleyard chop, variable
//     switching with a threshold, time-step cutting (Section 2.3), and the
//     MB / CNV convergence measures of Section 2.3.
//   * ILU0 preconditioned BiCGStab (Section 2.3.1): textbook block ILU(0)
//     on the matrix pattern in natural order, right-preconditioned
//     BiCGStab of van der Vorst.
//
// Threads (orc_set_threads, default 1): the loops whose iterations are
// independent -- cell properties, accumulation, the face fluxes, the operator's
// rows and the vector updates -- may run on several host threads.  Every
// floating-point sum keeps its sequential order (dot products and the norms
// stay sequential; each cell gathers its face terms in the order of the
// sequential face loop), so the results do not depend on the thread count.
// The ILU(0) factorisation and sweeps are sequential, as in the paper's
// per-process ILU(0).
//
// Parity: the functions are pinned by the CPU test suite against finite
// differences, mass conservation, hydrostatic equilibrium, the 1-D
// incompressible closed form, the ILU(0) identity and dense LU on tiny grids.
// Full three-phase trajectories are pinned only through those invariants.

#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>
#include <algorithm>

namespace orc {

// Host threads of the loops with independent iterations (1: sequential).
static int g_threads = 1;
#define ORC_PARALLEL_FOR _Pragma("omp parallel for num_threads(g_threads) schedule(static)")

// ---------------------------------------------------------------------------
// Forward-mode dual number: value plus N first derivatives.
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
    double v;
    double d[N];
    Dual() : v(0.0) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
    Dual(double c) : v(c) { for (int k = 0; k < N; ++k) d[k] = 0.0; }  // NOLINT
    static Dual var(double val, int slot) { Dual r(val); r.d[slot] = 1.0; return r; }
};

template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v + b.v; for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v - b.v; for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k]; return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r; r.v = -a.v; for (int k = 0; k < N; ++k) r.d[k] = -a.d[k]; return r;
}
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v * b.v;
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r; r.v = a.v / b.v;
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
    return r;
}
template <int N> Dual<N> operator*(double s, const Dual<N>& a) { return Dual<N>(s) * a; }
template <int N> Dual<N> operator*(const Dual<N>& a, double s) { return a * Dual<N>(s); }
template <int N> Dual<N> operator+(double s, const Dual<N>& a) { return Dual<N>(s) + a; }
template <int N> Dual<N> operator-(double s, const Dual<N>& a) { return Dual<N>(s) - a; }
template <int N> Dual<N> operator-(const Dual<N>& a, double s) { return a - Dual<N>(s); }
template <int N> Dual<N> operator/(const Dual<N>& a, double s) { return a / Dual<N>(s); }
template <int N> Dual<N> operator/(double s, const Dual<N>& a) { return Dual<N>(s) / a; }

template <int N> Dual<N> dexp(const Dual<N>& a) {
    Dual<N> r; r.v = std::exp(a.v);
    for (int k = 0; k < N; ++k) r.d[k] = r.v * a.d[k];
    return r;
}
// a^n for a >= 0 (n > 1), derivative n a^(n-1).
template <int N> Dual<N> dpow(const Dual<N>& a, double n) {
    Dual<N> r; r.v = std::pow(a.v, n);
    double dd = n * std::pow(a.v, n - 1.0);
    for (int k = 0; k < N; ++k) r.d[k] = dd * a.d[k];
    return r;
}
// clamp to [0, 1]; derivative zero where the clamp is active.
template <int N> Dual<N> clamp01(const Dual<N>& a) {
    if (a.v <= 0.0) return Dual<N>(0.0);
    if (a.v >= 1.0) return Dual<N>(1.0);
    return a;
}
// Re-seat a 3-derivative cell dual into slots [off, off+3) of an M-dual.
template <int M> Dual<M> lift(const Dual<3>& a, int off) {
    Dual<M> r(a.v); for (int k = 0; k < 3; ++k) r.d[off + k] = a.d[k]; return r;
}

// ---------------------------------------------------------------------------
// Parameters.  The order of the flat array matches synth.fluid_params().
// ---------------------------------------------------------------------------
struct Fluid {
    double g, rho_s[3], p_ref, bw_ref, c_w, mu_w, R_sb, p_b, Bo_slope, c_o, mu_o0, mu_o_r,
        c_mu, p_sc, Z, mu_g0, mu_g_p, c_r, s_wco, s_orw, s_org, n_corey;
};
static Fluid fluid_from(const double* f) {
    Fluid F;
    F.g = f[0]; F.rho_s[0] = f[1]; F.rho_s[1] = f[2]; F.rho_s[2] = f[3];
    F.p_ref = f[4]; F.bw_ref = f[5]; F.c_w = f[6]; F.mu_w = f[7]; F.R_sb = f[8]; F.p_b = f[9];
    F.Bo_slope = f[10]; F.c_o = f[11]; F.mu_o0 = f[12]; F.mu_o_r = f[13]; F.c_mu = f[14];
    F.p_sc = f[15]; F.Z = f[16]; F.mu_g0 = f[17]; F.mu_g_p = f[18]; F.c_r = f[19];
    F.s_wco = f[20]; F.s_orw = f[21]; F.s_org = f[22]; F.n_corey = f[23];
    return F;
}

enum { W = 0, O = 1, G = 2 };
enum { SAT = 0, USAT = 1 };

// Cell quantities with derivatives with respect to the cell's own primary
// variables (p_o, s_w, x) -- Section 2.1.2 primary-variable choice.
struct CellProps {
    Dual<3> b[3], lam[3], rho[3], mphi, rgo, s[3];
    Dual<3> A[3];  // accumulation terms (Eq. acc)
};

// Dissolution limit r_s(p): linear up to the bubble point (reading of the
// configuration "Rs(p) linear to bubble point").
static Dual<3> rs_of(const Fluid& F, const Dual<3>& p) { return p * (F.R_sb / F.p_b); }

static CellProps cell_props(const Fluid& F, double p_, double sw_, double x_, int flag) {
    CellProps c;
    Dual<3> p = Dual<3>::var(p_, 0), sw = Dual<3>::var(sw_, 1), x = Dual<3>::var(x_, 2);
    Dual<3> sg, rgo;
    if (flag == SAT) { sg = x; rgo = rs_of(F, p); }      // gas present: x = s_g, oil saturated
    else             { sg = Dual<3>(0.0); rgo = x; }     // no gas: x = r_go
    Dual<3> so = 1.0 - sw - sg;
    c.s[W] = sw; c.s[O] = so; c.s[G] = sg; c.rgo = rgo;

    // Water: b_w(p; c_w, p_ref, b_ref), constant viscosity (Section 2.1.6).
    c.b[W] = F.bw_ref * dexp(F.c_w * (p - F.p_ref));
    Dual<3> mu_w(F.mu_w);
    // Live oil: saturated FVF B_o,sat(r) and undersaturated compressibility
    // about the saturation pressure p_sat(r) of the dissolved gas ratio.
    Dual<3> psat = rgo * (F.p_b / F.R_sb);
    Dual<3> Bsat = 1.0 + F.Bo_slope * rgo;
    c.b[O] = dexp(F.c_o * (p - psat)) / Bsat;
    Dual<3> mu_o = (F.mu_o0 / (1.0 + F.mu_o_r * rgo)) * dexp(F.c_mu * (p - psat));
    // Dry gas.
    c.b[G] = p / (F.p_sc * F.Z);
    Dual<3> mu_g = F.mu_g0 * (1.0 + p / F.mu_g_p);
    // Rock: phi = m_phi(p) phi_ref (Section 2.1.4).
    c.mphi = dexp(F.c_r * (p - F.p_ref));
    // Densities (nomenclature): rho_w = b_w rho_Sw, rho_o = b_o (rho_So + r_go rho_Sg), rho_g = b_g rho_Sg.
    c.rho[W] = c.b[W] * F.rho_s[W];
    c.rho[O] = c.b[O] * (F.rho_s[O] + rgo * F.rho_s[G]);
    c.rho[G] = c.b[G] * F.rho_s[G];

    // Relative permeabilities: Corey two-phase curves combined by Eq. (gwseg).
    double n = F.n_corey;
    Dual<3> krw = dpow(clamp01((sw - F.s_wco) / (1.0 - F.s_wco - F.s_orw)), n);
    Dual<3> krg = dpow(clamp01(sg / (1.0 - F.s_wco - F.s_org)), n);
    Dual<3> krow = dpow(clamp01((so - F.s_orw) / (1.0 - F.s_wco - F.s_orw)), n);
    Dual<3> krog = dpow(clamp01((so - F.s_org) / (1.0 - F.s_wco - F.s_org)), n);
    Dual<3> ww = sw - F.s_wco;
    if (ww.v < 0.0) ww = Dual<3>(0.0);
    Dual<3> den = ww + sg;
    Dual<3> kro = (den.v <= 1e-14) ? krow : (ww * krow + sg * krog) / den;
    c.lam[W] = krw / mu_w;
    c.lam[O] = kro / mu_o;
    c.lam[G] = krg / mu_g;

    c.A[W] = c.mphi * c.b[W] * sw;
    c.A[O] = c.mphi * c.b[O] * so;
    c.A[G] = c.mphi * (c.b[G] * sg + rgo * c.b[O] * so);
    return c;
}

// ---------------------------------------------------------------------------
// Model
// ---------------------------------------------------------------------------
struct Well {
    int kind;      // 0 injector, 1 producer
    int phase;     // injected phase (W or G) for injectors
    int control0;  // 0 rate, 1 bhp (as given)
    int control;   // current control within a step
    double target, bhp_limit, rw, skin;
    std::vector<int> cells;
    std::vector<double> WI;
    double z_datum = 0.0, rho_well = 0.0;
    double bhp = 0.0;
    // Linearisation of the well (rate-controlled wells only).
    double Rw = 0.0, Dw = 0.0;
    // Surface rates (w, o, g) summed over the connections at the last assembly.
    double qs[3] = {0.0, 0.0, 0.0};
    std::vector<double> B;  // 3 per connection: dR_w/dy_cell
    std::vector<double> C;  // 3 per connection: dR_cell/dbhp
};

// One TPFA face between cell i and its higher-index neighbour j: the three
// component fluxes u_a (Eqs. flux1, flux2) and their derivatives with respect
// to the primary variables of i (bi) and of j (bj), row-major [a][v].
struct FaceTerm {
    double u[3], bi[9], bj[9];
};

struct Model {
    int nx, ny, nz, n;
    double top_depth = 0.0;
    Fluid F;
    std::vector<double> dx, dy, dz;
    std::vector<double> perm, poro, pv, depth, vol;   // perm [3][n]: kx, ky, kz
    // Transmissibility of the +x, +y, +z face of each cell (0 at the boundary).
    std::vector<double> Tx, Ty, Tz;
    std::vector<Well> wells;
    // State
    std::vector<double> p, sw, x;
    std::vector<uint8_t> flag;
    // Step-start data
    std::vector<double> A0;  // 3n
    std::vector<double> bk_p, bk_sw, bk_x, bk_bhp;
    std::vector<uint8_t> bk_flag;
    // Linear system (BCSR, 3x3 row-major blocks) and residual
    std::vector<int> rowptr, colind, diagpos;
    std::vector<double> vals, R;
    // ILU(0) factors in the same pattern (strict L blocks and U blocks incl. diagonal)
    std::vector<double> lu;
    std::vector<double> Uinv;  // inverse of U diagonal blocks, 9n
    double dt_last = 0.0;
    double dt_next = 0.0;  // sub-step length carried between report steps (0: unset)
    // Block-Jacobi ILU(0) over boxes of ysub cell rows in y and zsub cell
    // layers in z (0: no cut in that direction): the parallel preconditioner
    // of Section 2.5 (one ILU(0) block per subdomain; the couplings between
    // subdomains are left out of M, the operator keeps them).
    int ysub = 0, zsub = 0;
    // Face terms of the last assembly, 3 per cell (+x, +y, +z), filled only
    // where the face exists.
    std::vector<FaceTerm> faces;
};

static inline int cidx(const Model& m, int i, int j, int k) { return i + m.nx * (j + m.ny * k); }

static void build_pattern(Model& m) {
    int n = m.n;
    m.rowptr.assign(n + 1, 0);
    m.colind.clear();
    m.diagpos.assign(n, 0);
    for (int k = 0; k < m.nz; ++k)
        for (int j = 0; j < m.ny; ++j)
            for (int i = 0; i < m.nx; ++i) {
                int c = cidx(m, i, j, k);
                std::vector<int> cols;
                if (k > 0) cols.push_back(c - m.nx * m.ny);
                if (j > 0) cols.push_back(c - m.nx);
                if (i > 0) cols.push_back(c - 1);
                cols.push_back(c);
                if (i < m.nx - 1) cols.push_back(c + 1);
                if (j < m.ny - 1) cols.push_back(c + m.nx);
                if (k < m.nz - 1) cols.push_back(c + m.nx * m.ny);
                for (int q : cols) {
                    if (q == c) m.diagpos[c] = (int)m.colind.size();
                    m.colind.push_back(q);
                }
                m.rowptr[c + 1] = (int)m.colind.size();
            }
    m.vals.assign(9 * m.colind.size(), 0.0);
}

static int find_block(const Model& m, int row, int col) {
    for (int q = m.rowptr[row]; q < m.rowptr[row + 1]; ++q)
        if (m.colind[q] == col) return q;
    return -1;
}

// Appendix B: half-transmissibility of a box cell towards a face normal to
// axis d is |F| k_d / (h_d / 2) with the permeability along d; T_ij =
// t_ij t_ji / (t_ij + t_ji).
static void compute_static(Model& m) {
    int n = m.n;
    m.pv.assign(n, 0); m.depth.assign(n, 0); m.vol.assign(n, 0);
    m.Tx.assign(n, 0); m.Ty.assign(n, 0); m.Tz.assign(n, 0);
    std::vector<double> ztop(m.nz + 1, m.top_depth);
    for (int k = 0; k < m.nz; ++k) ztop[k + 1] = ztop[k] + m.dz[k];
    for (int k = 0; k < m.nz; ++k)
        for (int j = 0; j < m.ny; ++j)
            for (int i = 0; i < m.nx; ++i) {
                int c = cidx(m, i, j, k);
                m.vol[c] = m.dx[i] * m.dy[j] * m.dz[k];
                m.pv[c] = m.poro[c] * m.vol[c];
            }
    for (int k = 0; k < m.nz; ++k)
        for (int j = 0; j < m.ny; ++j)
            for (int i = 0; i < m.nx; ++i)
                m.depth[cidx(m, i, j, k)] = ztop[k] + 0.5 * m.dz[k];
    for (int k = 0; k < m.nz; ++k)
        for (int j = 0; j < m.ny; ++j)
            for (int i = 0; i < m.nx; ++i) {
                int c = cidx(m, i, j, k);
                if (i + 1 < m.nx) {
                    int e = c + 1;
                    double area = m.dy[j] * m.dz[k];
                    double t1 = area * m.perm[c] / (0.5 * m.dx[i]);
                    double t2 = area * m.perm[e] / (0.5 * m.dx[i + 1]);   // kx
                    m.Tx[c] = t1 * t2 / (t1 + t2);
                }
                if (j + 1 < m.ny) {
                    int e = c + m.nx;
                    double area = m.dx[i] * m.dz[k];
                    double t1 = area * m.perm[n + c] / (0.5 * m.dy[j]);
                    double t2 = area * m.perm[n + e] / (0.5 * m.dy[j + 1]);   // ky
                    m.Ty[c] = t1 * t2 / (t1 + t2);
                }
                if (k + 1 < m.nz) {
                    int e = c + m.nx * m.ny;
                    double area = m.dx[i] * m.dy[j];
                    double t1 = area * m.perm[2 * n + c] / (0.5 * m.dz[k]);
                    double t2 = area * m.perm[2 * n + e] / (0.5 * m.dz[k + 1]);   // kz
                    m.Tz[c] = t1 * t2 / (t1 + t2);
                }
            }
}

// Peaceman well index for a vertical connection in a box cell:
// WI = 2 pi k h / (ln(r_o / r_w) + skin), r_o = 0.14 sqrt(dx^2 + dy^2)
// (Peaceman 1978).  With kx != ky (Peaceman 1983): k = sqrt(kx ky) and
// r_o = 0.28 sqrt(sqrt(ky/kx) dx^2 + sqrt(kx/ky) dy^2) /
//       ((ky/kx)^(1/4) + (kx/ky)^(1/4)).
static double peaceman(double kx, double ky, double dx, double dy, double h, double rw,
                       double skin) {
    if (kx == ky) {
        double ro = 0.14 * std::sqrt(dx * dx + dy * dy);
        return 2.0 * M_PI * kx * h / (std::log(ro / rw) + skin);
    }
    const double ryx = std::sqrt(ky / kx), rxy = std::sqrt(kx / ky);
    const double ro = 0.28 * std::sqrt(ryx * dx * dx + rxy * dy * dy) /
                      (std::sqrt(ryx) + std::sqrt(rxy));
    return 2.0 * M_PI * std::sqrt(kx * ky) * h / (std::log(ro / rw) + skin);
}

// ---------------------------------------------------------------------------
// Well terms.  Connection inflow (Eq. wellinflow) in surface volumes, with
// derivatives with respect to the cell's (p, s_w, x) (slots 0..2) and the
// well BHP (slot 3).  Reading of the paper's M_{a,j}: producing connections
// carry each phase at its own mobility; injecting connections carry the
// injected phase at the total mobility; reverse flow is set to zero.
// ---------------------------------------------------------------------------
static void connection_rates(const Model& m, const Well& w, int con, Dual<4> q[3]) {
    const Fluid& F = m.F;
    int c = w.cells[con];
    CellProps cp = cell_props(F, m.p[c], m.sw[c], m.x[c], m.flag[c]);
    Dual<4> pc = lift<4>(Dual<3>::var(m.p[c], 0), 0);
    Dual<4> bhp = (w.control == 0) ? Dual<4>::var(w.bhp, 3) : Dual<4>(w.bhp);
    double h = F.g * w.rho_well * (m.depth[c] - w.z_datum);
    Dual<4> dp = pc - bhp - h;
    for (int a = 0; a < 3; ++a) q[a] = Dual<4>(0.0);
    double WI = w.WI[con];
    if (w.kind == 1) {  // producer
        if (dp.v > 0.0) {
            for (int a = 0; a < 3; ++a) q[a] = WI * lift<4>(cp.b[a] * cp.lam[a], 0) * dp;
            q[G] = q[G] + WI * lift<4>(cp.rgo * cp.b[O] * cp.lam[O], 0) * dp;
        }
    } else {            // injector
        if (dp.v < 0.0) {
            Dual<3> lt = cp.lam[W] + cp.lam[O] + cp.lam[G];
            q[w.phase] = WI * lift<4>(lt * cp.b[w.phase], 0) * dp;
        }
    }
}

// Surface rate that a rate control acts on: the injected component for an
// injector (positive when injecting), the oil rate for a producer.
static Dual<4> controlled_rate(const Well& w, const Dual<4> q[3]) {
    if (w.kind == 0) return -q[w.phase];
    return q[O];
}

// ---------------------------------------------------------------------------
// Assembly
// ---------------------------------------------------------------------------
static void add_block(Model& m, int q, const double blk[9], double sgn) {
    for (int e = 0; e < 9; ++e) m.vals[9 * q + e] += sgn * blk[e];
}

static void begin_step(Model& m) {
    int n = m.n;
    m.A0.assign(3 * n, 0.0);
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) {
        CellProps cp = cell_props(m.F, m.p[c], m.sw[c], m.x[c], m.flag[c]);
        for (int a = 0; a < 3; ++a) m.A0[3 * c + a] = cp.A[a].v;
    }
    // Well datum and wellbore density, explicit over the step (Section 2.2.1).
    for (Well& w : m.wells) {
        w.control = w.control0;
        if (w.control == 1) w.bhp = w.target;
        int c0 = w.cells[0];
        w.z_datum = m.depth[c0];
        if (w.kind == 0) {
            CellProps cp = cell_props(m.F, m.p[c0], m.sw[c0], m.x[c0], m.flag[c0]);
            w.rho_well = cp.rho[w.phase].v;
        } else {
            double num = 0.0, den = 0.0;
            for (int c : w.cells) {
                CellProps cp = cell_props(m.F, m.p[c], m.sw[c], m.x[c], m.flag[c]);
                for (int a = 0; a < 3; ++a) { num += cp.lam[a].v * cp.rho[a].v; den += cp.lam[a].v; }
            }
            w.rho_well = den > 0.0 ? num / den : 0.0;
        }
    }
    m.bk_p = m.p; m.bk_sw = m.sw; m.bk_x = m.x; m.bk_flag = m.flag;
    m.bk_bhp.clear();
    for (Well& w : m.wells) m.bk_bhp.push_back(w.bhp);
}

static FaceTerm face_term(const Model& m, const std::vector<CellProps>& props, int i, int j,
                          double T) {
    const Fluid& F = m.F;
    const CellProps& ci = props[i];
    const CellProps& cj = props[j];
    Dual<6> pi = lift<6>(Dual<3>::var(m.p[i], 0), 0);
    Dual<6> pj = lift<6>(Dual<3>::var(m.p[j], 0), 3);
    double dz = m.depth[i] - m.depth[j];
    Dual<6> u[3];
    Dual<6> dphi[3];
    bool up_i[3];
    for (int a = 0; a < 3; ++a) {
        Dual<6> rho_ij = 0.5 * (lift<6>(ci.rho[a], 0) + lift<6>(cj.rho[a], 3));
        dphi[a] = pi - pj - F.g * rho_ij * dz;
        up_i[a] = dphi[a].v >= 0.0;
        Dual<6> mob = up_i[a] ? lift<6>(ci.b[a] * ci.lam[a], 0) : lift<6>(cj.b[a] * cj.lam[a], 3);
        u[a] = mob * T * dphi[a];
    }
    // Dissolved gas travels with the oil phase (Eq. flux2).
    Dual<6> rmob = up_i[O] ? lift<6>(ci.rgo * ci.b[O] * ci.lam[O], 0)
                           : lift<6>(cj.rgo * cj.b[O] * cj.lam[O], 3);
    u[G] = u[G] + rmob * T * dphi[O];
    FaceTerm f;
    for (int a = 0; a < 3; ++a) {
        f.u[a] = u[a].v;
        for (int v = 0; v < 3; ++v) { f.bi[3 * a + v] = u[a].d[v]; f.bj[3 * a + v] = u[a].d[3 + v]; }
    }
    return f;
}

static void assemble(Model& m, double dt) {
    int n = m.n;
    std::fill(m.vals.begin(), m.vals.end(), 0.0);
    m.R.assign(3 * n, 0.0);
    m.dt_last = dt;
    std::vector<CellProps> props(n);
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) props[c] = cell_props(m.F, m.p[c], m.sw[c], m.x[c], m.flag[c]);

    // Accumulation: (phi_ref V / dt) (A - A0) into R and the diagonal block.
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) {
        double s = m.pv[c] / dt;
        double blk[9];
        for (int a = 0; a < 3; ++a) {
            m.R[3 * c + a] += s * (props[c].A[a].v - m.A0[3 * c + a]);
            for (int v = 0; v < 3; ++v) blk[3 * a + v] = s * props[c].A[a].d[v];
        }
        add_block(m, m.diagpos[c], blk, 1.0);
    }

    // Faces: each connection once, oriented from the lower to the higher index
    // (+x, +y, +z of every cell), u_ij added to R_i and subtracted from R_j.
    // The terms are formed first; then every cell adds its six faces in the
    // order of a sequential sweep over the lower cells (k, j, i outermost to
    // innermost; +x, +y, +z within a cell): -z, -y, -x, +x, +y, +z.
    const int plane = m.nx * m.ny;
    std::vector<FaceTerm>& ft = m.faces;
    ft.resize(3 * (size_t)n);
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) {
        const int ii = c % m.nx, jj = (c / m.nx) % m.ny, k = c / plane;
        if (ii + 1 < m.nx) ft[3 * (size_t)c + 0] = face_term(m, props, c, c + 1, m.Tx[c]);
        if (jj + 1 < m.ny) ft[3 * (size_t)c + 1] = face_term(m, props, c, c + m.nx, m.Ty[c]);
        if (k + 1 < m.nz) ft[3 * (size_t)c + 2] = face_term(m, props, c, c + plane, m.Tz[c]);
    }
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) {
        const int ii = c % m.nx, jj = (c / m.nx) % m.ny, k = c / plane;
        const int dq = m.diagpos[c];
        // faces from the lower neighbours: this cell is their j
        const int lower[3] = {c - plane, c - m.nx, c - 1};
        const bool has_lower[3] = {k > 0, jj > 0, ii > 0};
        const int ldir[3] = {2, 1, 0};
        for (int q = 0; q < 3; ++q) {
            if (!has_lower[q]) continue;
            const FaceTerm& f = ft[3 * (size_t)lower[q] + ldir[q]];
            for (int a = 0; a < 3; ++a) m.R[3 * c + a] -= f.u[a];
            add_block(m, find_block(m, c, lower[q]), f.bi, -1.0);
            add_block(m, dq, f.bj, -1.0);
        }
        // own faces: this cell is their i
        const int upper[3] = {c + 1, c + m.nx, c + plane};
        const bool has_upper[3] = {ii + 1 < m.nx, jj + 1 < m.ny, k + 1 < m.nz};
        for (int q = 0; q < 3; ++q) {
            if (!has_upper[q]) continue;
            const FaceTerm& f = ft[3 * (size_t)c + q];
            for (int a = 0; a < 3; ++a) m.R[3 * c + a] += f.u[a];
            add_block(m, dq, f.bi, 1.0);
            add_block(m, find_block(m, c, upper[q]), f.bj, 1.0);
        }
    }

    // Wells: q_a,i adds to R_a,i; rate-controlled wells add an equation.
    for (Well& w : m.wells) {
        int nc = (int)w.cells.size();
        w.B.assign(3 * nc, 0.0); w.C.assign(3 * nc, 0.0);
        w.qs[0] = w.qs[1] = w.qs[2] = 0.0;
        Dual<4> rate(0.0);
        for (int con = 0; con < nc; ++con) {
            int c = w.cells[con];
            Dual<4> q[3];
            connection_rates(m, w, con, q);
            double blk[9];
            for (int a = 0; a < 3; ++a) {
                m.R[3 * c + a] += q[a].v;
                w.qs[a] += q[a].v;
                for (int v = 0; v < 3; ++v) blk[3 * a + v] = q[a].d[v];
                w.C[3 * con + a] = q[a].d[3];
            }
            add_block(m, m.diagpos[c], blk, 1.0);
            Dual<4> r = controlled_rate(w, q);
            for (int v = 0; v < 3; ++v) w.B[3 * con + v] = r.d[v];
            rate = rate + r;
        }
        if (w.control == 0) {
            // Eq. (well-control-rate): R_c = Q - Q_target.
            w.Rw = rate.v - w.target;
            w.Dw = rate.d[3];
        } else {
            w.Rw = 0.0; w.Dw = 1.0;
            std::fill(w.B.begin(), w.B.end(), 0.0);
            std::fill(w.C.begin(), w.C.end(), 0.0);
        }
    }
}

// Section 2.3 convergence measures (per component a):
//   MB_a  = dt * Bavg_a * |sum_i R_a,i| / sum_i PV_i
//   CNV_a = dt * Bavg_a * max_i |R_a,i| / PV_i,   Bavg_a = mean_i 1 / b_a,i
// out[0..2] = MB, out[3..5] = CNV, out[6] = max relative well-equation residual.
static void norms(const Model& m, double dt, double* out) {
    int n = m.n;
    double sumR[3] = {0, 0, 0}, maxR[3] = {0, 0, 0}, sumB[3] = {0, 0, 0}, pvt = 0.0;
    std::vector<double> b(3 * (size_t)n);
    ORC_PARALLEL_FOR
    for (int c = 0; c < n; ++c) {
        CellProps cp = cell_props(m.F, m.p[c], m.sw[c], m.x[c], m.flag[c]);
        for (int a = 0; a < 3; ++a) b[3 * (size_t)c + a] = cp.b[a].v;
    }
    for (int c = 0; c < n; ++c) {
        pvt += m.pv[c];
        for (int a = 0; a < 3; ++a) {
            sumR[a] += m.R[3 * c + a];
            maxR[a] = std::max(maxR[a], std::fabs(m.R[3 * c + a]) / m.pv[c]);
            sumB[a] += 1.0 / b[3 * (size_t)c + a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        double Bavg = sumB[a] / n;
        out[a] = dt * Bavg * std::fabs(sumR[a]) / pvt;
        out[3 + a] = dt * Bavg * maxR[a];
    }
    double wr = 0.0;
    for (const Well& w : m.wells)
        if (w.control == 0) wr = std::max(wr, std::fabs(w.Rw) / std::max(std::fabs(w.target), 1e-300));
    out[6] = wr;
}

// ---------------------------------------------------------------------------
// Linear algebra on 3x3 blocks (row-major)
// ---------------------------------------------------------------------------
static void mm3(const double* a, const double* b, double* c) {
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += a[3 * r + k] * b[3 * k + s];
            c[3 * r + s] = acc;
        }
}
static void mv3(const double* a, const double* x, double* y) {
    for (int r = 0; r < 3; ++r) y[r] = a[3 * r] * x[0] + a[3 * r + 1] * x[1] + a[3 * r + 2] * x[2];
}
// Inverse by Gaussian elimination with partial pivoting.
static bool inv3(const double* a, double* out) {
    double m[3][6];
    for (int r = 0; r < 3; ++r) {
        for (int s = 0; s < 3; ++s) { m[r][s] = a[3 * r + s]; m[r][3 + s] = (r == s) ? 1.0 : 0.0; }
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r) if (std::fabs(m[r][col]) > std::fabs(m[piv][col])) piv = r;
        if (m[piv][col] == 0.0) return false;
        if (piv != col) for (int s = 0; s < 6; ++s) std::swap(m[col][s], m[piv][s]);
        double d = m[col][col];
        for (int s = 0; s < 6; ++s) m[col][s] /= d;
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            double f = m[r][col];
            for (int s = 0; s < 6; ++s) m[r][s] -= f * m[col][s];
        }
    }
    for (int r = 0; r < 3; ++r) for (int s = 0; s < 3; ++s) out[3 * r + s] = m[r][3 + s];
    return true;
}

// Textbook block ILU(0) in natural row order, restricted to the pattern of A:
// for each row i and each k < i in the pattern: L_ik = A_ik U_kk^-1, then
// A_ij -= L_ik U_kj for every j > k present in both row i and row k.
static bool ilu0(Model& m) {
    int n = m.n;
    m.lu = m.vals;
    if (m.ysub > 0 || m.zsub > 0) {   // block-Jacobi: drop the blocks that couple two subdomains
        // subdomain of a cell: (slab in y, slab in z); a direction without cuts is one slab
        auto dom = [&](int c) {
            const int j = (c / m.nx) % m.ny, k = c / (m.nx * m.ny);
            const int sy = m.ysub > 0 ? j / m.ysub : 0, sz = m.zsub > 0 ? k / m.zsub : 0;
            return sy + m.ny * sz;
        };
        for (int i = 0; i < n; ++i) {
            const int si = dom(i);
            for (int q = m.rowptr[i]; q < m.rowptr[i + 1]; ++q)
                if (dom(m.colind[q]) != si)
                    for (int e = 0; e < 9; ++e) m.lu[9 * q + e] = 0.0;
        }
    }
    m.Uinv.assign(9 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int q = m.rowptr[i]; q < m.rowptr[i + 1]; ++q) {
            int k = m.colind[q];
            if (k >= i) break;
            double L[9];
            mm3(&m.lu[9 * q], &m.Uinv[9 * k], L);
            std::memcpy(&m.lu[9 * q], L, sizeof(L));
            for (int qk = m.rowptr[k]; qk < m.rowptr[k + 1]; ++qk) {
                int j = m.colind[qk];
                if (j <= k) continue;
                int qi = find_block(m, i, j);
                if (qi < 0) continue;
                double P[9];
                mm3(L, &m.lu[9 * qk], P);
                for (int e = 0; e < 9; ++e) m.lu[9 * qi + e] -= P[e];
            }
        }
        if (!inv3(&m.lu[9 * m.diagpos[i]], &m.Uinv[9 * i])) return false;
    }
    return true;
}

// z = (LU)^-1 r: forward substitution with unit-lower L, back substitution with U.
static void ilu_apply(const Model& m, const double* r, double* z) {
    int n = m.n;
    std::vector<double> y(3 * n);
    for (int i = 0; i < n; ++i) {
        double acc[3] = {r[3 * i], r[3 * i + 1], r[3 * i + 2]};
        for (int q = m.rowptr[i]; q < m.diagpos[i]; ++q) {
            double t[3];
            mv3(&m.lu[9 * q], &y[3 * m.colind[q]], t);
            for (int e = 0; e < 3; ++e) acc[e] -= t[e];
        }
        for (int e = 0; e < 3; ++e) y[3 * i + e] = acc[e];
    }
    for (int i = n - 1; i >= 0; --i) {
        double acc[3] = {y[3 * i], y[3 * i + 1], y[3 * i + 2]};
        for (int q = m.diagpos[i] + 1; q < m.rowptr[i + 1]; ++q) {
            double t[3];
            mv3(&m.lu[9 * q], &z[3 * m.colind[q]], t);
            for (int e = 0; e < 3; ++e) acc[e] -= t[e];
        }
        mv3(&m.Uinv[9 * i], acc, &z[3 * i]);
    }
}

// Reduced operator of Eq. (wellequation): y = A x - sum_w C_w D_w^-1 (B_w x).
static void apply_op(const Model& m, const double* x, double* y) {
    int n = m.n;
    ORC_PARALLEL_FOR
    for (int i = 0; i < n; ++i) {
        double acc[3] = {0, 0, 0};
        for (int q = m.rowptr[i]; q < m.rowptr[i + 1]; ++q) {
            double t[3];
            mv3(&m.vals[9 * q], &x[3 * m.colind[q]], t);
            for (int e = 0; e < 3; ++e) acc[e] += t[e];
        }
        for (int e = 0; e < 3; ++e) y[3 * i + e] = acc[e];
    }
    for (const Well& w : m.wells) {
        if (w.control != 0) continue;
        double bx = 0.0;
        for (size_t con = 0; con < w.cells.size(); ++con)
            for (int v = 0; v < 3; ++v) bx += w.B[3 * con + v] * x[3 * w.cells[con] + v];
        double s = bx / w.Dw;
        for (size_t con = 0; con < w.cells.size(); ++con)
            for (int e = 0; e < 3; ++e) y[3 * w.cells[con] + e] -= w.C[3 * con + e] * s;
    }
}

static double dot(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

enum { LIN_OK = 0, LIN_NOT_CONVERGED = 1, LIN_BREAKDOWN = 2, LIN_FACTOR_FAIL = 3 };

// Right-preconditioned BiCGStab (van der Vorst) on the reduced system
// S x = b, b = R_r - sum_w C_w D_w^-1 R_w; then x_w = D_w^-1 (R_w - B_w x_r).
// Output sol has 3n reservoir entries followed by one entry per well
// (zero for wells without an unknown).  Stops when ||r|| <= tol ||r0|| and
// the true residual ||b - S x|| meets the same bound (see the restarts below).
static int solve(Model& m, double tol, int maxit, double* sol, int* its_out) {
    int n = m.n, N = 3 * n;
    *its_out = 0;
    if (!ilu0(m)) return LIN_FACTOR_FAIL;
    std::vector<double> b(m.R);
    for (const Well& w : m.wells) {
        if (w.control != 0) continue;
        double s = w.Rw / w.Dw;
        for (size_t con = 0; con < w.cells.size(); ++con)
            for (int e = 0; e < 3; ++e) b[3 * w.cells[con] + e] -= w.C[3 * con + e] * s;
    }
    std::vector<double> x(N, 0.0), r(b), rh(b), p(N, 0.0), v(N, 0.0), ph(N), s(N), sh(N), t(N);
    const double nr0 = std::sqrt(dot(r, r));
    // One BiCGStab cycle from the current r (with rh = r, p = v = 0), until the
    // recurrence's residual meets tol ||r0||, a breakdown, or maxit iterations
    // in total.
    auto cycle = [&]() -> int {
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        for (int it = *its_out + 1; it <= maxit; ++it) {
            double rho = dot(rh, r);
            if (rho == 0.0 || !std::isfinite(rho)) return LIN_BREAKDOWN;
            double beta = (rho / rho_old) * (alpha / omega);
            ORC_PARALLEL_FOR
            for (int i = 0; i < N; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            ilu_apply(m, p.data(), ph.data());
            apply_op(m, ph.data(), v.data());
            double rv = dot(rh, v);
            if (rv == 0.0 || !std::isfinite(rv)) return LIN_BREAKDOWN;
            alpha = rho / rv;
            ORC_PARALLEL_FOR
            for (int i = 0; i < N; ++i) s[i] = r[i] - alpha * v[i];
            double ns = std::sqrt(dot(s, s));
            if (ns <= tol * nr0) {
                for (int i = 0; i < N; ++i) x[i] += alpha * ph[i];
                *its_out = it;
                return LIN_OK;
            }
            ilu_apply(m, s.data(), sh.data());
            apply_op(m, sh.data(), t.data());
            double tt = dot(t, t);
            if (tt == 0.0 || !std::isfinite(tt)) return LIN_BREAKDOWN;
            omega = dot(t, s) / tt;
            if (omega == 0.0 || !std::isfinite(omega)) return LIN_BREAKDOWN;
            ORC_PARALLEL_FOR
            for (int i = 0; i < N; ++i) { x[i] += alpha * ph[i] + omega * sh[i]; r[i] = s[i] - omega * t[i]; }
            double nr = std::sqrt(dot(r, r));
            *its_out = it;
            if (nr <= tol * nr0) return LIN_OK;
            rho_old = rho;
        }
        return LIN_NOT_CONVERGED;
    };
    int status = nr0 == 0.0 ? LIN_OK : cycle();
    // Acceptance on the true residual b - S x: the recurrence's residual can
    // drift from it.  A miss restarts BiCGStab from the true residual (at most
    // 8 times, iterations counted on); with the budget spent the solve is not
    // converged.
    for (int restarts = 0; status == LIN_OK && nr0 > 0.0; ++restarts) {
        apply_op(m, x.data(), t.data());
        for (int i = 0; i < N; ++i) r[i] = b[i] - t[i];
        double nt = std::sqrt(dot(r, r));
        if (nt <= tol * nr0) break;
        if (restarts >= 8 || *its_out >= maxit || !std::isfinite(nt)) {
            status = LIN_NOT_CONVERGED;
            break;
        }
        rh = r;
        std::fill(p.begin(), p.end(), 0.0);
        std::fill(v.begin(), v.end(), 0.0);
        status = cycle();
    }
    if (status == LIN_NOT_CONVERGED) *its_out = maxit;
    for (int i = 0; i < N; ++i) sol[i] = x[i];
    int wi = 0;
    for (const Well& w : m.wells) {
        double xw = 0.0;
        if (w.control == 0) {
            double bx = 0.0;
            for (size_t con = 0; con < w.cells.size(); ++con)
                for (int v2 = 0; v2 < 3; ++v2) bx += w.B[3 * con + v2] * x[3 * w.cells[con] + v2];
            xw = (w.Rw - bx) / w.Dw;
        }
        sol[N + wi] = xw;
        ++wi;
    }
    return status;
}

// ---------------------------------------------------------------------------
// Domain decomposition (Section 2.5) emulated with K host threads, one per
// subdomain: slabs of ysub cell rows in y (the block-Jacobi slabs of the
// preconditioner).  Each rank keeps its interior rows of the operator with
// columns in its own index space (interior plus one ghost row on each side
// that has a neighbour), its own ILU(0) block factorised from those rows, the
// wells whose columns it holds, and its slice of every Krylov vector.  Before
// each operator product the ranks exchange their boundary rows (halo); every
// inner product is a local sum in row order followed by an all-reduce (the
// K local sums added in rank order by every rank).  The iteration is the
// BiCGStab of `solve` step for step, so with K = 1 it is `solve` bit for bit;
// with K > 1 only the grouping of the inner products' sums differs.
// ---------------------------------------------------------------------------
struct DdBarrier {
    std::mutex mu;
    std::condition_variable cv;
    int n, count = 0;
    long gen = 0;
    explicit DdBarrier(int k) : n(k) {}
    void wait() {
        std::unique_lock<std::mutex> lock(mu);
        const long g = gen;
        if (++count == n) {
            count = 0;
            ++gen;
            cv.notify_all();
        } else {
            cv.wait(lock, [&] { return gen != g; });
        }
    }
};

struct DdRank {
    int nx = 0, j0 = 0, j1 = 0, gl = 0, gh = 0, nyl = 0, nint = 0, ntot = 0;
    std::vector<int> gcell;   // interior index -> global cell
    std::vector<int> lpos;    // interior index -> position in the ghosted local layout
    std::vector<int> rp, ci, diag;   // local operator rows (columns: local positions)
    std::vector<double> val, lu, Uinv;
    std::vector<int> wells;   // wells whose connection cells lie in this slab
    std::vector<double> send_lo, send_hi;   // boundary rows for the neighbours
};

// global cell (inside the rank's slab or its ghost rows) -> ghosted position
static int local_of(const Model& m, const DdRank& d, int c) {
    const int i = c % m.nx, j = (c / m.nx) % m.ny, k = c / (m.nx * m.ny);
    return i + m.nx * (j - d.j0 + d.gl + d.nyl * k);
}
// global cell of the slab -> interior index (natural order inside the slab)
static int interior_of(const Model& m, const DdRank& d, int c) {
    const int i = c % m.nx, j = (c / m.nx) % m.ny, k = c / (m.nx * m.ny);
    return i + m.nx * (j - d.j0 + (d.j1 - d.j0) * k);
}
// ghosted position -> interior index, -1 for a ghost
static int interior_pos(const DdRank& d, int pos) {
    const int jl = (pos / d.nx) % d.nyl;
    if (jl < d.gl || jl >= d.nyl - d.gh) return -1;
    const int i = pos % d.nx, k = pos / (d.nx * d.nyl);
    return i + d.nx * (jl - d.gl + (d.j1 - d.j0) * k);
}

static int dd_solve(Model& m, double tol, int maxit, double* sol, int* its_out) {
    const int n = m.n, nx = m.nx, ny = m.ny, nz = m.nz;
    *its_out = 0;
    if (m.ysub <= 0 || m.zsub > 0) return LIN_FACTOR_FAIL;   // y slabs only
    const int K = (ny + m.ysub - 1) / m.ysub;
    std::vector<DdRank> R(K);
    for (int k = 0; k < K; ++k) {
        DdRank& d = R[k];
        d.nx = nx;
        d.j0 = k * m.ysub;
        d.j1 = std::min(ny, d.j0 + m.ysub);
        d.gl = k > 0 ? 1 : 0;
        d.gh = k + 1 < K ? 1 : 0;
        d.nyl = d.j1 - d.j0 + d.gl + d.gh;
        d.ntot = nx * d.nyl * nz;
        auto local = [&](int c) {   // global cell -> local position (inside the ghosted slab)
            const int i = c % nx, j = (c / nx) % ny, kk = c / (nx * ny);
            return i + nx * (j - d.j0 + d.gl + d.nyl * kk);
        };
        for (int kk = 0; kk < nz; ++kk)
            for (int j = d.j0; j < d.j1; ++j)
                for (int i = 0; i < nx; ++i) {
                    const int c = cidx(m, i, j, kk);
                    d.gcell.push_back(c);
                    d.lpos.push_back(local(c));
                }
        d.nint = (int)d.gcell.size();
        // local operator rows (all blocks) and the ILU(0) block (in-slab blocks)
        d.rp.push_back(0);
        for (int ii = 0; ii < d.nint; ++ii) {
            const int c = d.gcell[ii];
            for (int q = m.rowptr[c]; q < m.rowptr[c + 1]; ++q) {
                d.ci.push_back(local(m.colind[q]));
                d.val.insert(d.val.end(), &m.vals[9 * q], &m.vals[9 * q] + 9);
                if (m.colind[q] == c) d.diag.push_back((int)d.ci.size() - 1);
            }
            d.rp.push_back((int)d.ci.size());
        }
        for (size_t w = 0; w < m.wells.size(); ++w) {
            const int c0 = m.wells[w].cells[0];
            const int j = (c0 / nx) % ny;
            if (j >= d.j0 && j < d.j1) d.wells.push_back((int)w);
        }
    }
    // ILU(0) of each block: the textbook elimination on the rank's rows with
    // the blocks of other slabs left out (they are zero in the block-Jacobi M)
    auto in_slab = [&](const DdRank& d, int pos) {
        const int jl = (pos / nx) % d.nyl;
        return jl >= d.gl && jl < d.nyl - d.gh;
    };
    std::vector<int> pos2int;
    for (DdRank& d : R) {
        pos2int.assign(d.ntot, -1);
        for (int ii = 0; ii < d.nint; ++ii) pos2int[d.lpos[ii]] = ii;
        d.lu = d.val;
        for (int ii = 0; ii < d.nint; ++ii)
            for (int q = d.rp[ii]; q < d.rp[ii + 1]; ++q)
                if (!in_slab(d, d.ci[q]))
                    for (int e = 0; e < 9; ++e) d.lu[9 * q + e] = 0.0;
        d.Uinv.assign(9 * (size_t)d.nint, 0.0);
        auto find = [&](int row, int colpos) {
            for (int q = d.rp[row]; q < d.rp[row + 1]; ++q)
                if (d.ci[q] == colpos) return q;
            return -1;
        };
        for (int ii = 0; ii < d.nint; ++ii) {
            for (int q = d.rp[ii]; q < d.rp[ii + 1]; ++q) {
                const int kk = pos2int[d.ci[q]];
                if (d.ci[q] >= d.lpos[ii]) break;
                if (kk < 0) continue;   // a ghost column: its block is zero
                double L[9];
                mm3(&d.lu[9 * q], &d.Uinv[9 * kk], L);
                std::memcpy(&d.lu[9 * q], L, sizeof(L));
                for (int qk = d.rp[kk]; qk < d.rp[kk + 1]; ++qk) {
                    if (d.ci[qk] <= d.lpos[kk]) continue;
                    const int qi = find(ii, d.ci[qk]);
                    if (qi < 0) continue;
                    double P[9];
                    mm3(L, &d.lu[9 * qk], P);
                    for (int e = 0; e < 9; ++e) d.lu[9 * qi + e] -= P[e];
                }
            }
            if (!inv3(&d.lu[9 * d.diag[ii]], &d.Uinv[9 * ii])) return LIN_FACTOR_FAIL;
        }
    }
    // right-hand side of the reduced system, sliced per rank
    std::vector<double> bglob(m.R);
    for (const Well& w : m.wells) {
        if (w.control != 0) continue;
        const double s = w.Rw / w.Dw;
        for (size_t con = 0; con < w.cells.size(); ++con)
            for (int e = 0; e < 3; ++e) bglob[3 * w.cells[con] + e] -= w.C[3 * con + e] * s;
    }
    DdBarrier bar(K);
    std::vector<double> partial(K, 0.0);
    std::vector<int> status(K, LIN_OK), its(K, 0);
    auto rank_main = [&](int k) {
        DdRank& d = R[k];
        const int Ni = 3 * d.nint;
        auto allreduce = [&](double v) {
            partial[k] = v;
            bar.wait();
            double s = 0.0;
            for (int q = 0; q < K; ++q) s += partial[q];
            bar.wait();
            return s;
        };
        auto dotl = [&](const std::vector<double>& a, const std::vector<double>& b) {
            double s = 0.0;
            for (int q = 0; q < Ni; ++q) s += a[q] * b[q];
            return allreduce(s);
        };
        // x in the ghosted layout (3 per position); interior vectors are [3 nint]
        const int plane = nx;   // cells of one x-line
        auto halo = [&](std::vector<double>& xl) {
            // send: the first and the last interior row of every z layer
            const int rows = d.j1 - d.j0;
            d.send_lo.resize(3 * (size_t)plane * nz);
            d.send_hi.resize(3 * (size_t)plane * nz);
            for (int kk = 0; kk < nz; ++kk)
                for (int i = 0; i < nx; ++i)
                    for (int e = 0; e < 3; ++e) {
                        d.send_lo[3 * (i + nx * kk) + e] = xl[3 * (i + nx * (d.gl + d.nyl * kk)) + e];
                        d.send_hi[3 * (i + nx * kk) + e] =
                            xl[3 * (i + nx * (d.gl + rows - 1 + d.nyl * kk)) + e];
                    }
            bar.wait();
            for (int kk = 0; kk < nz; ++kk)
                for (int i = 0; i < nx; ++i)
                    for (int e = 0; e < 3; ++e) {
                        if (d.gl) xl[3 * (i + nx * (0 + d.nyl * kk)) + e] = R[k - 1].send_hi[3 * (i + nx * kk) + e];
                        if (d.gh) xl[3 * (i + nx * (d.nyl - 1 + d.nyl * kk)) + e] = R[k + 1].send_lo[3 * (i + nx * kk) + e];
                    }
            bar.wait();
        };
        std::vector<double> gx(3 * (size_t)d.ntot, 0.0);   // ghosted work vector
        // y = S x for interior x (halo exchanged inside); wells of this rank
        auto op = [&](const std::vector<double>& xi, std::vector<double>& y) {
            for (int ii = 0; ii < d.nint; ++ii)
                for (int e = 0; e < 3; ++e) gx[3 * d.lpos[ii] + e] = xi[3 * ii + e];
            halo(gx);
            for (int ii = 0; ii < d.nint; ++ii) {
                double acc[3] = {0, 0, 0};
                for (int q = d.rp[ii]; q < d.rp[ii + 1]; ++q) {
                    double t[3];
                    mv3(&d.val[9 * q], &gx[3 * d.ci[q]], t);
                    for (int e = 0; e < 3; ++e) acc[e] += t[e];
                }
                for (int e = 0; e < 3; ++e) y[3 * ii + e] = acc[e];
            }
            for (int wi : d.wells) {
                const Well& w = m.wells[wi];
                if (w.control != 0) continue;
                double bx = 0.0;
                for (size_t con = 0; con < w.cells.size(); ++con)
                    for (int v = 0; v < 3; ++v) bx += w.B[3 * con + v] * gx[3 * (size_t)local_of(m, d, w.cells[con]) + v];
                const double s = bx / w.Dw;
                for (size_t con = 0; con < w.cells.size(); ++con) {
                    const int ii = interior_of(m, d, w.cells[con]);
                    for (int e = 0; e < 3; ++e) y[3 * ii + e] -= w.C[3 * con + e] * s;
                }
            }
        };
        // z = M_k^-1 r on the rank's block
        std::vector<double> yv(Ni);
        auto prec = [&](const std::vector<double>& r, std::vector<double>& z) {
            for (int ii = 0; ii < d.nint; ++ii) {
                double acc[3] = {r[3 * ii], r[3 * ii + 1], r[3 * ii + 2]};
                for (int q = d.rp[ii]; q < d.diag[ii]; ++q) {
                    const int kk = interior_pos(d, d.ci[q]);
                    if (kk < 0) continue;
                    double t[3];
                    mv3(&d.lu[9 * q], &yv[3 * kk], t);
                    for (int e = 0; e < 3; ++e) acc[e] -= t[e];
                }
                for (int e = 0; e < 3; ++e) yv[3 * ii + e] = acc[e];
            }
            for (int ii = d.nint - 1; ii >= 0; --ii) {
                double acc[3] = {yv[3 * ii], yv[3 * ii + 1], yv[3 * ii + 2]};
                for (int q = d.diag[ii] + 1; q < d.rp[ii + 1]; ++q) {
                    const int kk = interior_pos(d, d.ci[q]);
                    if (kk < 0) continue;
                    double t[3];
                    mv3(&d.lu[9 * q], &z[3 * kk], t);
                    for (int e = 0; e < 3; ++e) acc[e] -= t[e];
                }
                mv3(&d.Uinv[9 * ii], acc, &z[3 * ii]);
            }
        };
        std::vector<double> b(Ni);
        for (int ii = 0; ii < d.nint; ++ii)
            for (int e = 0; e < 3; ++e) b[3 * ii + e] = bglob[3 * d.gcell[ii] + e];
        std::vector<double> x(Ni, 0.0), r(b), rh(b), p(Ni, 0.0), v(Ni, 0.0), ph(Ni), s(Ni), sh(Ni), t(Ni);
        const double nr0 = std::sqrt(dotl(r, r));
        int it_done = 0;
        auto cycle = [&]() -> int {
            double rho_old = 1.0, alpha = 1.0, omega = 1.0;
            for (int it = it_done + 1; it <= maxit; ++it) {
                const double rho = dotl(rh, r);
                if (rho == 0.0 || !std::isfinite(rho)) return LIN_BREAKDOWN;
                const double beta = (rho / rho_old) * (alpha / omega);
                for (int i = 0; i < Ni; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
                prec(p, ph);
                op(ph, v);
                const double rv = dotl(rh, v);
                if (rv == 0.0 || !std::isfinite(rv)) return LIN_BREAKDOWN;
                alpha = rho / rv;
                for (int i = 0; i < Ni; ++i) s[i] = r[i] - alpha * v[i];
                const double ns = std::sqrt(dotl(s, s));
                if (ns <= tol * nr0) {
                    for (int i = 0; i < Ni; ++i) x[i] += alpha * ph[i];
                    it_done = it;
                    return LIN_OK;
                }
                prec(s, sh);
                op(sh, t);
                const double tt = dotl(t, t);
                if (tt == 0.0 || !std::isfinite(tt)) return LIN_BREAKDOWN;
                omega = dotl(t, s) / tt;
                if (omega == 0.0 || !std::isfinite(omega)) return LIN_BREAKDOWN;
                for (int i = 0; i < Ni; ++i) {
                    x[i] += alpha * ph[i] + omega * sh[i];
                    r[i] = s[i] - omega * t[i];
                }
                const double nr = std::sqrt(dotl(r, r));
                it_done = it;
                if (nr <= tol * nr0) return LIN_OK;
                rho_old = rho;
            }
            return LIN_NOT_CONVERGED;
        };
        int st = nr0 == 0.0 ? LIN_OK : cycle();
        for (int restarts = 0; st == LIN_OK && nr0 > 0.0; ++restarts) {
            op(x, t);
            for (int i = 0; i < Ni; ++i) r[i] = b[i] - t[i];
            const double nt = std::sqrt(dotl(r, r));
            if (nt <= tol * nr0) break;
            if (restarts >= 8 || it_done >= maxit || !std::isfinite(nt)) {
                st = LIN_NOT_CONVERGED;
                break;
            }
            rh = r;
            std::fill(p.begin(), p.end(), 0.0);
            std::fill(v.begin(), v.end(), 0.0);
            st = cycle();
        }
        if (st == LIN_NOT_CONVERGED) it_done = maxit;
        for (int ii = 0; ii < d.nint; ++ii)
            for (int e = 0; e < 3; ++e) sol[3 * d.gcell[ii] + e] = x[3 * ii + e];
        // the owned wells' unknowns
        for (int wi : d.wells) {
            const Well& w = m.wells[wi];
            double xw = 0.0;
            if (w.control == 0) {
                double bx = 0.0;
                for (size_t con = 0; con < w.cells.size(); ++con)
                    for (int v2 = 0; v2 < 3; ++v2)
                        bx += w.B[3 * con + v2] * x[3 * interior_of(m, d, w.cells[con]) + v2];
                xw = (w.Rw - bx) / w.Dw;
            }
            sol[3 * n + wi] = xw;
        }
        status[k] = st;
        its[k] = it_done;
    };
    std::vector<std::thread> th;
    for (int k = 1; k < K; ++k) th.emplace_back(rank_main, k);
    rank_main(0);
    for (auto& t : th) t.join();
    *its_out = its[0];
    return status[0];
}

// ---------------------------------------------------------------------------
// Newton update (Section 2.3): dy = -sol; Appleyard chop; variable switching.
// ---------------------------------------------------------------------------
struct Opts {
    double tol_mb, tol_cnv, tol_well;
    int max_newton;
    double tol_lin;
    int max_lin, max_cuts;
    double ds_max, dp_rel_max, drs_rel_max, eps_switch;
    double bp_overshoot, dt_init, cut_factor;
};
static Opts opts_from(const double* o) {
    Opts r;
    r.tol_mb = o[0]; r.tol_cnv = o[1]; r.tol_well = o[2]; r.max_newton = (int)o[3];
    r.tol_lin = o[4]; r.max_lin = (int)o[5]; r.max_cuts = (int)o[6];
    r.ds_max = o[7]; r.dp_rel_max = o[8]; r.drs_rel_max = o[9]; r.eps_switch = o[10];
    r.bp_overshoot = o[11]; r.dt_init = o[12]; r.cut_factor = o[13];
    return r;
}

// Opening pressure of a well at the current cell pressures: the BHP at which
// the first connection starts to flow, min_j (p_j - h_j) for an injector
// (it injects through connection j when BHP + h_j > p_j), max_j for a
// producer.
static double opening_bhp(const Model& m, const Well& w) {
    double v = (w.kind == 0) ? 1e300 : -1e300;
    for (int c : w.cells) {
        double ph = m.p[c] - m.F.g * w.rho_well * (m.depth[c] - w.z_datum);
        v = (w.kind == 0) ? std::min(v, ph) : std::max(v, ph);
    }
    return v;
}

static void newton_update(Model& m, const Opts& o, const double* sol) {
    const Fluid& F = m.F;
    int n = m.n;
    for (int c = 0; c < n; ++c) {
        double dp = -sol[3 * c], dsw = -sol[3 * c + 1], dx = -sol[3 * c + 2];
        double p = m.p[c];
        double dpmax = o.dp_rel_max * p;
        if (std::fabs(dp) > dpmax) dp = (dp > 0 ? dpmax : -dpmax);
        if (m.flag[c] == SAT) {
            double mx = std::max(std::fabs(dsw), std::fabs(dx));
            if (mx > o.ds_max) { double f = o.ds_max / mx; dsw *= f; dx *= f; }
        } else {
            if (std::fabs(dsw) > o.ds_max) { double f = o.ds_max / std::fabs(dsw); dsw *= f; }
            double drmax = o.drs_rel_max * F.R_sb;
            if (std::fabs(dx) > drmax) dx = (dx > 0 ? drmax : -drmax);
            // Section 2.3: do not let an undersaturated cell jump far across the
            // saturation boundary in one iteration -- its pressure may fall at
            // most a fraction bp_overshoot below the saturation pressure of its
            // updated dissolved-gas ratio.
            double pfloor = (1.0 - o.bp_overshoot) * (F.p_b * (m.x[c] + dx) / F.R_sb);
            if (p + dp < pfloor && pfloor < p) dp = pfloor - p;
        }
        double pn = p + dp, swn = m.sw[c] + dsw, xn = m.x[c] + dx;
        swn = std::min(std::max(swn, 0.0), 1.0);
        uint8_t fl = m.flag[c];
        if (fl == SAT) {
            if (xn > 1.0 - swn) xn = 1.0 - swn;
            if (xn < 0.0) { fl = USAT; xn = pn * (F.R_sb / F.p_b); }
        } else {
            double rs = pn * (F.R_sb / F.p_b);
            if (xn > rs * (1.0 + o.eps_switch)) { fl = SAT; xn = 0.0; }
        }
        m.p[c] = pn; m.sw[c] = swn; m.x[c] = xn; m.flag[c] = fl;
    }
    int wi = 0;
    for (Well& w : m.wells) {
        if (w.control == 0) {
            double d = -sol[3 * n + wi];
            double dmax = o.dp_rel_max * w.bhp;
            if (std::fabs(d) > dmax) d = (d > 0 ? dmax : -dmax);
            double old = w.bhp;
            double nb = old + d;
            // well chop: a rate-controlled well must keep flowing -- the BHP may
            // at most halve its distance to the opening pressure (at the
            // updated cell pressures) per iteration
            double po = opening_bhp(m, w);
            if (w.kind == 0) {
                double floor_ = (old > po) ? po + 0.5 * (old - po) : po + 1e-3 * std::fabs(po);
                if (nb < floor_) nb = floor_;
            } else {
                double ceil_ = (old < po) ? po - 0.5 * (po - old) : po - 1e-3 * std::fabs(po);
                if (nb > ceil_) nb = ceil_;
            }
            w.bhp = nb;
            bool viol = (w.kind == 0) ? (w.bhp > w.bhp_limit) : (w.bhp < w.bhp_limit);
            if (viol) { w.control = 1; w.bhp = w.bhp_limit; }
        }
        ++wi;
    }
}

// After assembly: a rate-controlled well with no flowing connection (D_w = 0)
// has no sensitivity to its BHP; its BHP is moved just past the opening
// pressure (0.1% of it) and the system is assembled again.
static bool fix_dead_wells(Model& m) {
    bool changed = false;
    for (Well& w : m.wells)
        if (w.control == 0 && w.Dw == 0.0) {
            double po = opening_bhp(m, w);
            w.bhp = (w.kind == 0) ? po + 1e-3 * std::fabs(po) : po - 1e-3 * std::fabs(po);
            changed = true;
        }
    return changed;
}

static void restore(Model& m) {
    m.p = m.bk_p; m.sw = m.bk_sw; m.x = m.bk_x; m.flag = m.bk_flag;
    for (size_t i = 0; i < m.wells.size(); ++i) m.wells[i].bhp = m.bk_bhp[i];
}

// Sub-step growth after a converged Newton solve of nits iterations: easy
// steps grow, hard ones shrink (an iteration-count step controller).
static double step_growth(int nits) {
    if (nits <= 4) return 2.0;
    if (nits <= 8) return 1.5;
    if (nits <= 12) return 1.0;
    return 0.7;
}

// One Newton solve of a (sub)step of length dt; returns 0 when converged.
// rep: [newton_its, lin_its]
static int newton(Model& m, double dt, const Opts& o, int* nits, int* lits) {
    begin_step(m);
    std::vector<double> sol(3 * m.n + m.wells.size());
    double nrm[7];
    for (int it = 0;; ++it) {
        assemble(m, dt);
        if (fix_dead_wells(m)) assemble(m, dt);
        norms(m, dt, nrm);
        bool finite = true;
        for (double v : nrm) if (!std::isfinite(v)) finite = false;
        if (!finite) return 2;
        bool conv = true;
        for (int a = 0; a < 3; ++a) if (nrm[a] > o.tol_mb || nrm[3 + a] > o.tol_cnv) conv = false;
        if (nrm[6] > o.tol_well) conv = false;
        if (conv) { *nits = it; return 0; }
        if (it == o.max_newton) { *nits = it; return 1; }
        int li = 0;
        int st = solve(m, o.tol_lin, o.max_lin, sol.data(), &li);
        *lits += li;
        // a linear solve that breaks down or misses its tolerance fails the
        // Newton solve (the step is then cut)
        if (st != LIN_OK) { *nits = it + 1; return 3; }
        newton_update(m, o, sol.data());
    }
}

}  // namespace orc

using namespace orc;

extern "C" {

// fluid: 24 values in the order of synth.fluid_params(); wells: per well
// wint[4*w] = {kind, phase, control, ncon}, wdbl[4*w] = {target, bhp_limit, rw, skin},
// wcells = concatenated connection cell indices.
void* orc_create(int nx, int ny, int nz, const double* dx, const double* dy, const double* dz,
                 double top_depth, const double* perm, const double* poro, const double* fluid, int nwells,
                 const int* wint, const double* wdbl, const int* wcells) {
    Model* m = new Model();
    m->nx = nx; m->ny = ny; m->nz = nz; m->n = nx * ny * nz;
    m->F = fluid_from(fluid);
    m->dx.assign(dx, dx + nx); m->dy.assign(dy, dy + ny); m->dz.assign(dz, dz + nz);
    m->perm.assign(perm, perm + 3 * (size_t)m->n); m->poro.assign(poro, poro + m->n);
    m->top_depth = top_depth;
    compute_static(*m);
    build_pattern(*m);
    int off = 0;
    for (int w = 0; w < nwells; ++w) {
        Well wl;
        wl.kind = wint[4 * w]; wl.phase = wint[4 * w + 1]; wl.control0 = wl.control = wint[4 * w + 2];
        int ncon = wint[4 * w + 3];
        wl.target = wdbl[4 * w]; wl.bhp_limit = wdbl[4 * w + 1]; wl.rw = wdbl[4 * w + 2]; wl.skin = wdbl[4 * w + 3];
        for (int q = 0; q < ncon; ++q) {
            int c = wcells[off + q];
            wl.cells.push_back(c);
            int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
            wl.WI.push_back(peaceman(m->perm[c], m->perm[m->n + c], m->dx[i], m->dy[j], m->dz[k],
                                     wl.rw, wl.skin));
        }
        off += ncon;
        wl.bhp = (wl.control == 1) ? wl.target : wl.bhp_limit;
        m->wells.push_back(wl);
    }
    m->p.assign(m->n, 0.0); m->sw.assign(m->n, 0.0); m->x.assign(m->n, 0.0); m->flag.assign(m->n, 0);
    m->A0.assign(3 * m->n, 0.0);
    m->R.assign(3 * m->n, 0.0);
    return m;
}

void orc_destroy(void* h) { delete static_cast<Model*>(h); }
int orc_nnzb(void* h) { return (int)static_cast<Model*>(h)->colind.size(); }

void orc_static(void* h, double* Tx, double* Ty, double* Tz, double* pv, double* depth, double* wi) {
    Model* m = static_cast<Model*>(h);
    std::memcpy(Tx, m->Tx.data(), sizeof(double) * m->n);
    std::memcpy(Ty, m->Ty.data(), sizeof(double) * m->n);
    std::memcpy(Tz, m->Tz.data(), sizeof(double) * m->n);
    std::memcpy(pv, m->pv.data(), sizeof(double) * m->n);
    std::memcpy(depth, m->depth.data(), sizeof(double) * m->n);
    int q = 0;
    for (const Well& w : m->wells) for (double v : w.WI) wi[q++] = v;
}

void orc_set_state(void* h, const double* p, const double* sw, const double* x,
                   const uint8_t* flag, const double* bhp) {
    Model* m = static_cast<Model*>(h);
    m->p.assign(p, p + m->n); m->sw.assign(sw, sw + m->n); m->x.assign(x, x + m->n);
    m->flag.assign(flag, flag + m->n);
    for (size_t w = 0; w < m->wells.size(); ++w) m->wells[w].bhp = bhp[w];
}

void orc_get_state(void* h, double* p, double* sw, double* x, uint8_t* flag, double* bhp) {
    Model* m = static_cast<Model*>(h);
    std::memcpy(p, m->p.data(), sizeof(double) * m->n);
    std::memcpy(sw, m->sw.data(), sizeof(double) * m->n);
    std::memcpy(x, m->x.data(), sizeof(double) * m->n);
    std::memcpy(flag, m->flag.data(), m->n);
    for (size_t w = 0; w < m->wells.size(); ++w) bhp[w] = m->wells[w].bhp;
}

// Well start-up after an initial state is set: BHP-controlled wells at their
// target, rate-controlled ones first at their limit, then a rate-controlled
// injector at the BHP that meets its target by the linear inflow relation of
// the initial state (all connections injecting), capped by its limit;
// begin_step's datum density is used.
static void start_wells(Model* m) {
    const Fluid& F = m->F;
    for (Well& w : m->wells) w.bhp = (w.control0 == 1) ? w.target : w.bhp_limit;
    begin_step(*m);
    for (Well& w : m->wells) {
        if (w.control0 != 0 || w.kind != 0) continue;
        double num = w.target, den = 0.0;
        for (size_t q = 0; q < w.cells.size(); ++q) {
            int c = w.cells[q];
            CellProps cp = cell_props(F, m->p[c], m->sw[c], m->x[c], m->flag[c]);
            double mob = w.WI[q] * (cp.lam[W].v + cp.lam[O].v + cp.lam[G].v) * cp.b[w.phase].v;
            double h = F.g * w.rho_well * (m->depth[c] - w.z_datum);
            num += mob * (m->p[c] - h);
            den += mob;
        }
        if (den > 0.0) w.bhp = std::min(w.bhp_limit, num / den);
    }
}

// Initial state: undersaturated oil at dissolved ratio rgo, water saturation
// sw, and pressure in discrete hydrostatic equilibrium of the oil phase in
// every column, p = p_top at the centre of the top layer:
//   p_{k+1} = p_k + g (rho_o(p_k) + rho_o(p_{k+1}))/2 (z_{k+1} - z_k)
// (the equilibrium equation dp/dz = rho g of Section 2.1.3 written with the
// face density of Eq. (head)), solved by fixed-point iteration.
void orc_init_hydrostatic(void* h, double p_top, double sw, double rgo) {
    Model* m = static_cast<Model*>(h);
    const Fluid& F = m->F;
    for (int j = 0; j < m->ny; ++j)
        for (int i = 0; i < m->nx; ++i) {
            double pk = p_top;
            for (int k = 0; k < m->nz; ++k) {
                int c = cidx(*m, i, j, k);
                if (k > 0) {
                    int cu = cidx(*m, i, j, k - 1);
                    double dzz = m->depth[c] - m->depth[cu];
                    double rho_u = cell_props(F, pk, sw, rgo, USAT).rho[O].v;
                    double pn = pk;
                    for (int it = 0; it < 200; ++it) {
                        double rho_n = cell_props(F, pn, sw, rgo, USAT).rho[O].v;
                        double nxt = pk + F.g * 0.5 * (rho_u + rho_n) * dzz;
                        bool done = std::fabs(nxt - pn) <= 1e-15 * std::fabs(nxt);
                        pn = nxt;
                        if (done) break;
                    }
                    pk = pn;
                }
                m->p[c] = pk; m->sw[c] = sw; m->x[c] = rgo; m->flag[c] = USAT;
            }
        }
    start_wells(m);
}

// ---------------------------------------------------------------------------
// Equilibration (Section 2.1.3): vertical equilibrium from a datum pressure
// and the water-oil and gas-oil contact depths.  Each zone's phase pressure
// solves dp/dz = rho_alpha(p) g; the datum's zone is integrated from the
// datum, the zones above and below from the contacts, where the phase
// pressures are equal (the capillary pressure of this model is zero).  The
// ODEs are integrated with the classical 4th-order Runge-Kutta method in
// N = max(1, ceil(|dz| / 1 m)) equal steps.
//   zones: gas above the GOC, oil between the contacts, water below the WOC;
//   oil carries the dissolved ratio r = min(rgo, r_s(p)).
// Cell states: oil zone s_w = swc; gas zone s_w = swc, s_g = 1 - swc - s_org
// (saturated, residual oil); water zone s_w = 1 - s_orw (residual oil).  Oil
// with rgo < r_s(p) is undersaturated (x = rgo), else saturated with s_g = 0
// (gas zone aside).
// ---------------------------------------------------------------------------
enum { ZGAS = 0, ZOIL = 1, ZWAT = 2 };
struct Equil { double datum_z, datum_p, woc, goc, rgo, swc; };

static int zone_of(const Equil& e, double z) { return z < e.goc ? ZGAS : (z < e.woc ? ZOIL : ZWAT); }

static double zone_density(const Fluid& F, int zone, double p, double rgo) {
    if (zone == ZWAT) return F.rho_s[W] * F.bw_ref * std::exp(F.c_w * (p - F.p_ref));
    if (zone == ZGAS) return F.rho_s[G] * p / (F.p_sc * F.Z);
    const double rs = (F.R_sb / F.p_b) * p;
    const double r = rgo < rs ? rgo : rs;
    const double psat = r * (F.p_b / F.R_sb);
    const double bo = std::exp(F.c_o * (p - psat)) / (1.0 + F.Bo_slope * r);
    return bo * (F.rho_s[O] + r * F.rho_s[G]);
}

static double rk4_pressure(const Fluid& F, int zone, double rgo, double z0, double p0, double z) {
    const int N = std::max(1, (int)std::ceil(std::fabs(z - z0) / 1.0));
    const double h = (z - z0) / N;
    double p = p0;
    for (int q = 0; q < N; ++q) {
        const double k1 = F.g * zone_density(F, zone, p, rgo);
        const double k2 = F.g * zone_density(F, zone, p + 0.5 * h * k1, rgo);
        const double k3 = F.g * zone_density(F, zone, p + 0.5 * h * k2, rgo);
        const double k4 = F.g * zone_density(F, zone, p + h * k3, rgo);
        p += (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }
    return p;
}

// Anchor (depth, pressure) of every zone's phase-pressure curve.
static void zone_anchors(const Fluid& F, const Equil& e, double za[3], double pa[3]) {
    const int zd = zone_of(e, e.datum_z);
    za[zd] = e.datum_z;
    pa[zd] = e.datum_p;
    if (zd == ZOIL) {
        za[ZGAS] = e.goc;
        pa[ZGAS] = rk4_pressure(F, ZOIL, e.rgo, e.datum_z, e.datum_p, e.goc);
        za[ZWAT] = e.woc;
        pa[ZWAT] = rk4_pressure(F, ZOIL, e.rgo, e.datum_z, e.datum_p, e.woc);
    } else if (zd == ZGAS) {
        za[ZOIL] = e.goc;
        pa[ZOIL] = rk4_pressure(F, ZGAS, e.rgo, e.datum_z, e.datum_p, e.goc);
        za[ZWAT] = e.woc;
        pa[ZWAT] = rk4_pressure(F, ZOIL, e.rgo, e.goc, pa[ZOIL], e.woc);
    } else {
        za[ZOIL] = e.woc;
        pa[ZOIL] = rk4_pressure(F, ZWAT, e.rgo, e.datum_z, e.datum_p, e.woc);
        za[ZGAS] = e.goc;
        pa[ZGAS] = rk4_pressure(F, ZOIL, e.rgo, e.woc, pa[ZOIL], e.goc);
    }
}

// e6 = {datum depth, datum pressure, WOC depth, GOC depth, rgo, swc}
void orc_init_equilibrium(void* h, const double* e6) {
    Model* m = static_cast<Model*>(h);
    const Fluid& F = m->F;
    const Equil e{e6[0], e6[1], e6[2], e6[3], e6[4], e6[5]};
    double za[3], pa[3];
    zone_anchors(F, e, za, pa);
    for (int c = 0; c < m->n; ++c) {
        const double z = m->depth[c];
        const int zone = zone_of(e, z);
        const double p = rk4_pressure(F, zone, e.rgo, za[zone], pa[zone], z);
        m->p[c] = p;
        if (zone == ZGAS) {
            m->sw[c] = e.swc;
            m->x[c] = 1.0 - e.swc - F.s_org;
            m->flag[c] = SAT;
            continue;
        }
        m->sw[c] = zone == ZWAT ? 1.0 - F.s_orw : e.swc;
        const double rs = (F.R_sb / F.p_b) * p;
        if (e.rgo < rs) {
            m->x[c] = e.rgo;
            m->flag[c] = USAT;
        } else {
            m->x[c] = 0.0;
            m->flag[c] = SAT;
        }
    }
    start_wells(m);
}

void orc_begin_step(void* h) { begin_step(*static_cast<Model*>(h)); }

void orc_assemble(void* h, double dt) {
    Model* m = static_cast<Model*>(h);
    assemble(*m, dt);
}

void orc_get_system(void* h, int* rowptr, int* colind, double* vals, double* res) {
    Model* m = static_cast<Model*>(h);
    std::memcpy(rowptr, m->rowptr.data(), sizeof(int) * (m->n + 1));
    std::memcpy(colind, m->colind.data(), sizeof(int) * m->colind.size());
    std::memcpy(vals, m->vals.data(), sizeof(double) * m->vals.size());
    std::memcpy(res, m->R.data(), sizeof(double) * 3 * m->n);
}

// Per well: Rw, Dw, then B (3 per connection) and C (3 per connection),
// packed well after well; control[w] is the current control.
void orc_get_wells(void* h, double* rw, double* dw, double* B, double* C, int* control) {
    Model* m = static_cast<Model*>(h);
    int q = 0;
    for (size_t w = 0; w < m->wells.size(); ++w) {
        const Well& wl = m->wells[w];
        rw[w] = wl.Rw; dw[w] = wl.Dw; control[w] = wl.control;
        for (size_t k = 0; k < wl.B.size(); ++k) { B[q + k] = wl.B[k]; C[q + k] = wl.C[k]; }
        q += (int)wl.B.size();
    }
}

// Per well: surface rates (w, o, g) of the last assembly, current BHP and control.
void orc_well_rates(void* h, double* rates, double* bhp, int* control) {
    Model* m = static_cast<Model*>(h);
    for (size_t w = 0; w < m->wells.size(); ++w) {
        const Well& wl = m->wells[w];
        for (int a = 0; a < 3; ++a) rates[3 * w + a] = wl.qs[a];
        bhp[w] = wl.bhp;
        control[w] = wl.control;
    }
}

void orc_set_well_control(void* h, int w, int control, double bhp) {
    Model* m = static_cast<Model*>(h);
    m->wells[w].control = control;
    m->wells[w].bhp = bhp;
}

void orc_norms(void* h, double dt, double* out) { norms(*static_cast<Model*>(h), dt, out); }

// Residual of the full (reservoir + well) system at a given solution vector,
// computed with the unreduced blocks: out = J sol - [R; R_w].
void orc_residual_check(void* h, const double* sol, double* out) {
    Model* m = static_cast<Model*>(h);
    int n = m->n;
    for (int i = 0; i < n; ++i) {
        double acc[3] = {0, 0, 0};
        for (int q = m->rowptr[i]; q < m->rowptr[i + 1]; ++q) {
            double t[3];
            mv3(&m->vals[9 * q], &sol[3 * m->colind[q]], t);
            for (int e = 0; e < 3; ++e) acc[e] += t[e];
        }
        for (int e = 0; e < 3; ++e) out[3 * i + e] = acc[e] - m->R[3 * i + e];
    }
    int wi = 0;
    for (const Well& w : m->wells) {
        double xw = sol[3 * n + wi];
        double r = 0.0;
        if (w.control == 0) {
            for (size_t con = 0; con < w.cells.size(); ++con) {
                int c = w.cells[con];
                for (int e = 0; e < 3; ++e) out[3 * c + e] += w.C[3 * con + e] * xw;
                for (int v = 0; v < 3; ++v) r += w.B[3 * con + v] * sol[3 * c + v];
            }
            r += w.Dw * xw - w.Rw;
        }
        out[3 * n + wi] = r;
        ++wi;
    }
}

int orc_ilu0(void* h, double* lu_vals, double* uinv) {
    Model* m = static_cast<Model*>(h);
    if (!ilu0(*m)) return 1;
    std::memcpy(lu_vals, m->lu.data(), sizeof(double) * m->lu.size());
    std::memcpy(uinv, m->Uinv.data(), sizeof(double) * 9 * m->n);
    return 0;
}

// z = M^-1 r with M the ILU(0) factors from the last orc_ilu0 call.
void orc_ilu_apply(void* h, const double* r, double* z) { ilu_apply(*static_cast<Model*>(h), r, z); }

// y = reduced operator applied to x (after orc_assemble).
void orc_apply_op(void* h, const double* x, double* y) { apply_op(*static_cast<Model*>(h), x, y); }

int orc_solve(void* h, double tol, int maxit, double* sol, int* its) {
    return solve(*static_cast<Model*>(h), tol, maxit, sol, its);
}

// The same solve with one host thread per y slab of the block-Jacobi
// subdomains (orc_set_subdomains with ysub > 0, zsub = 0): local rows,
// halo exchange and all-reduced inner products.
int orc_dd_solve(void* h, double tol, int maxit, double* sol, int* its) {
    return dd_solve(*static_cast<Model*>(h), tol, maxit, sol, its);
}

void orc_newton_update(void* h, const double* opts, const double* sol) {
    newton_update(*static_cast<Model*>(h), opts_from(opts), sol);
}

// One report step of length dt with adaptive sub-steps (Section 2.3 time-step
// cutting): the sub-step length is carried between report steps; a
// converged sub-step grows it by step_growth, a failed Newton solve restores
// the state and multiplies it by cut_factor (at most max_cuts failures per
// report step).  report: [newton_its, lin_its, cuts, substeps, status(0 ok)].
int orc_step(void* h, double dt, const double* opts, double* report) {
    Model* m = static_cast<Model*>(h);
    Opts o = opts_from(opts);
    double t = 0.0;
    if (m->dt_next <= 0.0) m->dt_next = (o.dt_init > 0.0) ? o.dt_init : dt;
    int nits_tot = 0, lits_tot = 0, cuts = 0, subs = 0;
    int status = 0;
    while (t < dt * (1.0 - 1e-12)) {
        double dts = std::min(m->dt_next, dt - t);
        int nits = 0, lits = 0;
        int st = newton(*m, dts, o, &nits, &lits);
        nits_tot += nits; lits_tot += lits;
        if (st == 0) {
            t += dts;
            ++subs;
            m->dt_next = std::min(dts * step_growth(nits), dt);
            continue;
        }
        restore(*m);
        ++cuts;
        m->dt_next = dts * o.cut_factor;
        if (cuts > o.max_cuts) { status = 1; break; }
    }
    report[0] = nits_tot; report[1] = lits_tot; report[2] = cuts; report[3] = subs; report[4] = status;
    return status;
}

// Host threads of the independent loops (1 = sequential); returns the count set.
int orc_set_threads(int threads) {
    g_threads = threads < 1 ? 1 : threads;
    return g_threads;
}

double orc_get_dt_next(void* h) { return static_cast<Model*>(h)->dt_next; }
void orc_set_dt_next(void* h, double v) { static_cast<Model*>(h)->dt_next = v; }
void orc_set_subdomains(void* h, int ysub, int zsub) {
    static_cast<Model*>(h)->ysub = ysub > 0 ? ysub : 0;
    static_cast<Model*>(h)->zsub = zsub > 0 ? zsub : 0;
}

// Single-cell property evaluation with derivatives (for pin tests).
// out: for each quantity value then d/dp, d/dsw, d/dx; quantities in order
// b_w b_o b_g lam_w lam_o lam_g rho_w rho_o rho_g m_phi r_go A_w A_o A_g  (14 x 4)
void orc_cell_props(const double* fluid, double p, double sw, double x, int flag, double* out) {
    Fluid F = fluid_from(fluid);
    CellProps c = cell_props(F, p, sw, x, flag);
    const Dual<3>* q[14] = {&c.b[0], &c.b[1], &c.b[2], &c.lam[0], &c.lam[1], &c.lam[2],
                            &c.rho[0], &c.rho[1], &c.rho[2], &c.mphi, &c.rgo,
                            &c.A[0], &c.A[1], &c.A[2]};
    for (int k = 0; k < 14; ++k) {
        out[4 * k] = q[k]->v;
        for (int v = 0; v < 3; ++v) out[4 * k + 1 + v] = q[k]->d[v];
    }
}

}  // extern "C"
