// Residual and Jacobian assembly of the black-oil equations on the GPU
// (arXiv 1910.06059, Section 2.1.1 Eqs. materialbalance, acc, flux1, flux2,
// head; Section 2.2.1 Eq. wellinflow; Section 2.4 forward-mode AD), plus the
// static precompute of Appendix B, the hydrostatic initial state, the
// convergence measures of Section 2.3 and the Newton update with Appleyard
// chop and variable switching.
//
// Kernels and their data:
//   k_props  one thread per cell: cell quantities with derivatives (D3 duals),
//            accumulation residual and the accumulation part of the diagonal
//            block; writes the 28 face quantities per cell (SoA) for k_flux.
//   k_flux   one thread per cell: the six faces of the cell in the order
//            -z, -y, -x, +x, +y, +z; every face is evaluated in its canonical
//            orientation (lower cell index first), so both cells see bitwise
//            the same flux and derivatives (skew symmetry holds exactly).
//            Each thread owns its row: residual, diagonal block and its six
//            off-diagonal blocks; no atomics.
//   k_wells  one block per well: connection inflow and its derivatives,
//            well-equation residual and Schur pieces B_w, C_w, D_w.
#include <cmath>

#include "cell.cuh"

namespace bo {

// ---------------------------------------------------------------------------
// a1: static data (Appendix B) -- one thread per cell.  perm is [3][n]
// (kx, ky, kz); a face normal to axis d takes the permeability along d.
// ---------------------------------------------------------------------------
__global__ void k_static(Geom g, const double* __restrict__ dx, const double* __restrict__ dy,
                         const double* __restrict__ dz, double top,
                         const double* __restrict__ perm, const double* __restrict__ poro,
                         double* __restrict__ T, double* __restrict__ pv,
                         double* __restrict__ depth) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n) return;
    int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    double zt = top;
    for (int q = 0; q < k; ++q) zt += dz[q];
    depth[c] = zt + 0.5 * dz[k];
    pv[c] = poro[c] * (dx[i] * dy[j] * dz[k]);
    double tx = 0.0, ty = 0.0, tz = 0.0;
    if (i + 1 < g.nx) {
        double a = dy[j] * dz[k];
        double t1 = a * perm[c] / (0.5 * dx[i]);
        double t2 = a * perm[c + 1] / (0.5 * dx[i + 1]);
        tx = t1 * t2 / (t1 + t2);
    }
    if (j + 1 < g.ny) {
        double a = dx[i] * dz[k];
        double t1 = a * perm[g.n + c] / (0.5 * dy[j]);
        double t2 = a * perm[g.n + c + g.nx] / (0.5 * dy[j + 1]);
        ty = t1 * t2 / (t1 + t2);
    }
    if (k + 1 < g.nz) {
        double a = dx[i] * dy[j];
        double t1 = a * perm[2 * g.n + c] / (0.5 * dz[k]);
        double t2 = a * perm[2 * g.n + c + g.nx * g.ny] / (0.5 * dz[k + 1]);
        tz = t1 * t2 / (t1 + t2);
    }
    T[c] = tx;
    T[g.n + c] = ty;
    T[2 * g.n + c] = tz;
}

// Peaceman index of each vertical connection: WI = 2 pi k h / (ln(r_o/r_w) +
// skin).  With kx = ky, k = kx and r_o = 0.14 sqrt(dx^2 + dy^2) (Peaceman
// 1978); otherwise k = sqrt(kx ky) and r_o = 0.28 sqrt(sqrt(ky/kx) dx^2 +
// sqrt(kx/ky) dy^2) / ((ky/kx)^(1/4) + (kx/ky)^(1/4)) (Peaceman 1983).
__global__ void k_wi(Geom g, int ncon, const int* __restrict__ con_cell,
                     const int* __restrict__ con_well, const WellDev* __restrict__ wells,
                     const double* __restrict__ dx, const double* __restrict__ dy,
                     const double* __restrict__ dz, const double* __restrict__ perm,
                     const double* __restrict__ rw, const double* __restrict__ skin,
                     double* __restrict__ wi) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= ncon) return;
    int c = con_cell[q];
    int w = con_well[q];
    int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    const double kx = perm[c], ky = perm[g.n + c];
    if (kx == ky) {
        const double ro = 0.14 * sqrt(dx[i] * dx[i] + dy[j] * dy[j]);
        wi[q] = 2.0 * M_PI * kx * dz[k] / (log(ro / rw[w]) + skin[w]);
    } else {
        const double ryx = sqrt(ky / kx), rxy = sqrt(kx / ky);
        const double ro = 0.28 * sqrt(ryx * dx[i] * dx[i] + rxy * dy[j] * dy[j]) /
                          (sqrt(ryx) + sqrt(rxy));
        wi[q] = 2.0 * M_PI * sqrt(kx * ky) * dz[k] / (log(ro / rw[w]) + skin[w]);
    }
    (void)wells;
}

// Hydrostatic oil column per (i, j): p_{k+1} = p_k + g (rho(p_k) + rho(p_{k+1}))/2 dz.
__global__ void k_hydrostatic(Geom g, DevFluid F, double p_top, double sw, double rgo,
                              const double* __restrict__ depth, double* __restrict__ p,
                              double* __restrict__ s, double* __restrict__ x,
                              uint8_t* __restrict__ flag) {
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= g.nx * g.ny) return;
    double pk = p_top;
    int plane = g.nx * g.ny;
    CellD cd;
    for (int k = 0; k < g.nz; ++k) {
        int c = col + k * plane;
        if (k > 0) {
            double dzz = depth[c] - depth[c - plane];
            cell_eval(F, pk, sw, rgo, 1, cd);
            double rho_u = cd.rho[O_].v;
            double pn = pk;
            for (int it = 0; it < 200; ++it) {
                cell_eval(F, pn, sw, rgo, 1, cd);
                double nxt = pk + F.g * 0.5 * (rho_u + cd.rho[O_].v) * dzz;
                bool done = fabs(nxt - pn) <= 1e-15 * fabs(nxt);
                pn = nxt;
                if (done) break;
            }
            pk = pn;
        }
        p[c] = pk;
        s[c] = sw;
        x[c] = rgo;
        flag[c] = 1;
    }
}

// ---------------------------------------------------------------------------
// Equilibration (Section 2.1.3): each zone's phase pressure solves
// dp/dz = rho_alpha(p) g by classical RK4 in N = max(1, ceil(|dz| / 1 m))
// equal steps, the datum's zone from the datum and the other zones from the
// contacts (equal phase pressures there: this model has no capillary
// pressure).  Zones: gas above the GOC, oil between the contacts, water
// below the WOC; oil carries r = min(rgo, r_s(p)).
// ---------------------------------------------------------------------------
enum { ZGAS = 0, ZOIL = 1, ZWAT = 2 };

__device__ __forceinline__ int zone_of(const EquilDev& e, double z) {
    return z < e.goc ? ZGAS : (z < e.woc ? ZOIL : ZWAT);
}

__device__ double zone_density(const DevFluid& F, int zone, double p, double rgo) {
    if (zone == ZWAT) return F.rho_s[W_] * F.bw_ref * exp(F.c_w * (p - F.p_ref));
    if (zone == ZGAS) return F.rho_s[G_] * p / (F.p_sc * F.Z);
    const double rs = (F.R_sb / F.p_b) * p;
    const double r = rgo < rs ? rgo : rs;
    const double psat = r * (F.p_b / F.R_sb);
    const double bo = exp(F.c_o * (p - psat)) / (1.0 + F.Bo_slope * r);
    return bo * (F.rho_s[O_] + r * F.rho_s[G_]);
}

__device__ double rk4_pressure(const DevFluid& F, int zone, double rgo, double z0, double p0,
                               double z) {
    const int N = max(1, (int)ceil(fabs(z - z0) / 1.0));
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

// Anchor (depth, pressure) of every zone: out[zone] = depth, out[3 + zone] = pressure.
__global__ void k_equil_anchors(DevFluid F, EquilDev e, double* __restrict__ out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double za[3], pa[3];
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
    for (int q = 0; q < 3; ++q) {
        out[q] = za[q];
        out[3 + q] = pa[q];
    }
}

// Cell states of the zones: connate water in the oil and gas zones, residual
// oil in the water and gas zones; oil undersaturated when rgo < r_s(p).
__global__ void k_equil_cells(int n, DevFluid F, EquilDev e, const double* __restrict__ anchors,
                              const double* __restrict__ depth, double* __restrict__ p,
                              double* __restrict__ sw, double* __restrict__ x,
                              uint8_t* __restrict__ flag) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const double z = depth[c];
        const int zone = zone_of(e, z);
        const double pc = rk4_pressure(F, zone, e.rgo, anchors[zone], anchors[3 + zone], z);
        p[c] = pc;
        if (zone == ZGAS) {
            sw[c] = e.swc;
            x[c] = 1.0 - e.swc - F.s_org;
            flag[c] = 0;
            continue;
        }
        sw[c] = zone == ZWAT ? 1.0 - F.s_orw : e.swc;
        const double rs = (F.R_sb / F.p_b) * pc;
        if (e.rgo < rs) {
            x[c] = e.rgo;
            flag[c] = 1;
        } else {
            x[c] = 0.0;
            flag[c] = 0;
        }
    }
}

void launch_equilibrium(bo_sim* s, const EquilDev& e) {
    k_equil_anchors<<<1, 32, 0, s->stream>>>(s->fluid, e, s->d_part);
    count_launch(s, s->stream);
    k_equil_cells<<<152 * 4, 256, 0, s->stream>>>(s->geo.n, s->fluid, e, s->d_part, s->d_depth,
                                                  s->d_p, s->d_sw, s->d_x, s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_equil");
}

// ---------------------------------------------------------------------------
// Step start: accumulation A0 and the saved state.
// ---------------------------------------------------------------------------
__global__ void k_begin_cells(int n, DevFluid F, const double* __restrict__ p,
                              const double* __restrict__ sw, const double* __restrict__ x,
                              const uint8_t* __restrict__ flag, double* __restrict__ A0,
                              double* __restrict__ bk, uint8_t* __restrict__ bkflag) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    CellD cd;
    cell_eval(F, p[c], sw[c], x[c], flag[c], cd);
    A0[c] = cd.A[0].v;
    A0[n + c] = cd.A[1].v;
    A0[2 * n + c] = cd.A[2].v;
    bk[c] = p[c];
    bk[n + c] = sw[c];
    bk[2 * n + c] = x[c];
    bkflag[c] = flag[c];
}

// One thread per well, sequential over connections (a handful of values).
__global__ void k_begin_wells(int nw, DevFluid F, WellDev* __restrict__ wells,
                              const int* __restrict__ con_cell, const double* __restrict__ depth,
                              const double* __restrict__ p, const double* __restrict__ sw,
                              const double* __restrict__ x, const uint8_t* __restrict__ flag) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    WellDev& W = wells[w];
    W.ctl = W.ctl0;
    if (W.ctl == 1) W.bhp = W.target;
    int c0 = con_cell[W.off];
    W.z_datum = depth[c0];
    CellD cd;
    if (W.kind == 0) {
        cell_eval(F, p[c0], sw[c0], x[c0], flag[c0], cd);
        W.rho_well = cd.rho[W.phase].v;
    } else {
        double num = 0.0, den = 0.0;
        for (int q = 0; q < W.ncon; ++q) {
            int c = con_cell[W.off + q];
            cell_eval(F, p[c], sw[c], x[c], flag[c], cd);
            for (int a = 0; a < 3; ++a) {
                num += cd.lam[a].v * cd.rho[a].v;
                den += cd.lam[a].v;
            }
        }
        W.rho_well = den > 0.0 ? num / den : 0.0;
    }
    W.bhp_bk = W.bhp;
    if (W.full) {   // full standard well: storage at the step start, backup
        W.xs[3] = W.bhp;
        const double frac[3] = {W.xs[1], (1.0 - W.xs[1]) - W.xs[2], W.xs[2]};
        for (int a = 0; a < 3; ++a) W.A0s[a] = (W.vw * frac[a]) / std_well_g(a);
        for (int k = 0; k < 4; ++k) W.xs_bk[k] = W.xs[k];
    }
}

__global__ void k_restore(int n, double* __restrict__ p, double* __restrict__ sw,
                          double* __restrict__ x, uint8_t* __restrict__ flag,
                          const double* __restrict__ bk, const uint8_t* __restrict__ bkflag,
                          int nw, WellDev* __restrict__ wells) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        p[c] = bk[c];
        sw[c] = bk[n + c];
        x[c] = bk[2 * n + c];
        flag[c] = bkflag[c];
    }
    if (c < nw) {
        WellDev& W = wells[c];
        W.bhp = W.bhp_bk;
        if (W.full)
            for (int k = 0; k < 4; ++k) W.xs[k] = W.xs_bk[k];
    }
}

// ---------------------------------------------------------------------------
// a2 + a3: cell quantities and accumulation (one thread per cell).
// ---------------------------------------------------------------------------
constexpr int PROPS_BS = 256;

__global__ void __launch_bounds__(PROPS_BS)
k_props(int n, DevFluid F, const double* __restrict__ p, const double* __restrict__ sw,
        const double* __restrict__ x, const uint8_t* __restrict__ flag,
        const double* __restrict__ pv, const double* __restrict__ A0, double dt,
        double* __restrict__ props, double* __restrict__ R, double* __restrict__ A,
        double* __restrict__ part_binv) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    double binv[3] = {0.0, 0.0, 0.0};
    if (c < n) {
        CellD cd;
        cell_eval(F, p[c], sw[c], x[c], flag[c], cd);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            props[(4 * a + 0) * n + c] = cd.rho[a].v;
            props[(4 * a + 1) * n + c] = cd.rho[a].d0;
            props[(4 * a + 2) * n + c] = cd.rho[a].d1;
            props[(4 * a + 3) * n + c] = cd.rho[a].d2;
            D3 m = cd.b[a] * cd.lam[a];
            props[(12 + 4 * a + 0) * n + c] = m.v;
            props[(12 + 4 * a + 1) * n + c] = m.d0;
            props[(12 + 4 * a + 2) * n + c] = m.d1;
            props[(12 + 4 * a + 3) * n + c] = m.d2;
            binv[a] = 1.0 / cd.b[a].v;
        }
        D3 rm = cd.rgo * cd.b[O_] * cd.lam[O_];
        props[24 * n + c] = rm.v;
        props[25 * n + c] = rm.d0;
        props[26 * n + c] = rm.d1;
        props[27 * n + c] = rm.d2;
        double s = pv[c] / dt;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R[a * n + c] = s * (cd.A[a].v - A0[a * n + c]);
            A[(3 * a + 0) * n + c] = s * cd.A[a].d0;
            A[(3 * a + 1) * n + c] = s * cd.A[a].d1;
            A[(3 * a + 2) * n + c] = s * cd.A[a].d2;
        }
    }
    // block partial sums of 1/b_a for the convergence measures
    __shared__ double sh[3][PROPS_BS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = binv[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[a][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int q = 0; q < PROPS_BS / 32; ++q) v += sh[threadIdx.x][q];
        part_binv[blockIdx.x * 3 + threadIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------
// a4: face fluxes with upwinding (one thread per cell, six faces).
// ---------------------------------------------------------------------------
struct FaceSide {
    double rho[3][4];   // value + 3 derivatives
    double mob[3][4];   // b_a lam_a
    double rmob[4];     // r_go b_o lam_o
    double p, z;
};

__device__ __forceinline__ void load_side(const double* __restrict__ props,
                                          const double* __restrict__ p,
                                          const double* __restrict__ depth, int n, int c,
                                          FaceSide& s) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s.rho[a][k] = props[(4 * a + k) * n + c];
            s.mob[a][k] = props[(12 + 4 * a + k) * n + c];
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) s.rmob[k] = props[(24 + k) * n + c];
    s.p = p[c];
    s.z = depth[c];
}

// Flux of Eqs. (flux1), (flux2), (head) from L (lower index) to H, with its
// derivatives with respect to y_L (dl) and y_H (dh).
__device__ __forceinline__ void face_flux(const FaceSide& L, const FaceSide& H, double T,
                                          double g, double u[3], double dl[3][3],
                                          double dh[3][3]) {
    double dz = L.z - H.z;
    double phv[3], phl[3][3], phh[3][3];
    bool upl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double rij = 0.5 * (L.rho[a][0] + H.rho[a][0]);
        double grav = g * rij;
        phv[a] = (L.p - H.p) - grav * dz;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            phl[a][k] = (k == 0 ? 1.0 : 0.0) - (g * (0.5 * L.rho[a][1 + k])) * dz;
            phh[a][k] = (k == 0 ? -1.0 : 0.0) - (g * (0.5 * H.rho[a][1 + k])) * dz;
        }
        upl[a] = phv[a] >= 0.0;
        const double* m = upl[a] ? L.mob[a] : H.mob[a];
        double mt = m[0] * T;
        u[a] = mt * phv[a];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double up = (m[1 + k] * T) * phv[a];
            dl[a][k] = mt * phl[a][k] + (upl[a] ? up : 0.0);
            dh[a][k] = mt * phh[a][k] + (upl[a] ? 0.0 : up);
        }
    }
    // dissolved gas moves with the oil phase
    const double* rm = upl[O_] ? L.rmob : H.rmob;
    double rt = rm[0] * T;
    u[G_] = u[G_] + rt * phv[O_];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double up = (rm[1 + k] * T) * phv[O_];
        dl[G_][k] = dl[G_][k] + (rt * phl[O_][k] + (upl[O_] ? up : 0.0));
        dh[G_][k] = dh[G_][k] + (rt * phh[O_][k] + (upl[O_] ? 0.0 : up));
    }
}

constexpr int FLUX_BS = 128;

__global__ void __launch_bounds__(FLUX_BS)
k_flux(Geom g, double grav, const double* __restrict__ props, const double* __restrict__ p,
       const double* __restrict__ depth, const double* __restrict__ T,
       double* __restrict__ R, double* __restrict__ A) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int n = g.n;
    if (c >= n) return;
    int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    int plane = g.nx * g.ny;
    FaceSide me, nb;
    load_side(props, p, depth, n, c, me);
    double r[3], jd[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) r[a] = R[a * n + c];
#pragma unroll
    for (int e = 0; e < 9; ++e) jd[e] = A[e * n + c];
    // directions in accumulation order: -z, -y, -x, +x, +y, +z
    const int dirs[6] = {NB_MZ, NB_MY, NB_MX, NB_PX, NB_PY, NB_PZ};
#pragma unroll 1
    for (int q = 0; q < 6; ++q) {
        int b = dirs[q];
        int other;
        bool exists;
        double Tf;
        switch (b) {
            case NB_MZ: exists = k > 0; other = c - plane; break;
            case NB_MY: exists = j > 0; other = c - g.nx; break;
            case NB_MX: exists = i > 0; other = c - 1; break;
            case NB_PX: exists = i + 1 < g.nx; other = c + 1; break;
            case NB_PY: exists = j + 1 < g.ny; other = c + g.nx; break;
            default:    exists = k + 1 < g.nz; other = c + plane; break;
        }
        double* blk = A + (size_t)(b * 9) * n + c;
        if (!exists) {
#pragma unroll
            for (int e = 0; e < 9; ++e) blk[(size_t)e * n] = 0.0;
            continue;
        }
        int axis = (b - 1) >> 1;               // 0 x, 1 y, 2 z
        bool minus = (b & 1) == 1;             // -x, -y, -z
        int lo = minus ? other : c;
        Tf = T[axis * n + lo];
        load_side(props, p, depth, n, other, nb);
        double u[3], dl[3][3], dh[3][3];
        if (minus) face_flux(nb, me, Tf, grav, u, dl, dh);
        else       face_flux(me, nb, Tf, grav, u, dl, dh);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!minus) {          // this cell is the lower one: +u, own derivs dl
                r[a] += u[a];
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    jd[3 * a + s] += dl[a][s];
                    blk[(size_t)(3 * a + s) * n] = dh[a][s];
                }
            } else {               // this cell is the higher one: -u, own derivs dh
                r[a] -= u[a];
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    jd[3 * a + s] -= dh[a][s];
                    blk[(size_t)(3 * a + s) * n] = -dl[a][s];
                }
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) R[a * n + c] = r[a];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e * n + c] = jd[e];
}

// ---------------------------------------------------------------------------
// a5: wells (one block per well, one thread per connection).
// ---------------------------------------------------------------------------
constexpr int WELL_BS = 128;

__global__ void __launch_bounds__(WELL_BS)
k_wells(Geom g, DevFluid F, WellDev* __restrict__ wells, const int* __restrict__ con_cell,
        const double* __restrict__ con_wi, const double* __restrict__ depth,
        const double* __restrict__ p, const double* __restrict__ sw,
        const double* __restrict__ x, const uint8_t* __restrict__ flag,
        double* __restrict__ R, double* __restrict__ A, double* __restrict__ wB,
        double* __restrict__ wC, NewtonStatus* __restrict__ ns) {
    int n = g.n;
    WellDev& W = wells[blockIdx.x];
    const bool rate = (W.ctl == 0);
    double rsum = 0.0, dsum = 0.0, qsum[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
        int con = W.off + q;
        int c = con_cell[con];
        CellD cd;
        cell_eval(F, p[c], sw[c], x[c], flag[c], cd);
        double h = F.g * W.rho_well * (depth[c] - W.z_datum);
        double dp = p[c] - W.bhp - h;   // d/dp_c = 1, d/dbhp = -1
        double WI = con_wi[con];
        double qv[3] = {0, 0, 0}, qd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, qb[3] = {0, 0, 0};
        if (W.kind == 1) {
            if (dp > 0.0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    D3 m = cd.b[a] * cd.lam[a];
                    double wm = WI * m.v;
                    qv[a] = wm * dp;
                    qd[a][0] = (WI * m.d0) * dp + wm;
                    qd[a][1] = (WI * m.d1) * dp;
                    qd[a][2] = (WI * m.d2) * dp;
                    qb[a] = -wm;
                }
                D3 rm = cd.rgo * cd.b[O_] * cd.lam[O_];
                double wr = WI * rm.v;
                qv[G_] = qv[G_] + wr * dp;
                qd[G_][0] = qd[G_][0] + ((WI * rm.d0) * dp + wr);
                qd[G_][1] = qd[G_][1] + (WI * rm.d1) * dp;
                qd[G_][2] = qd[G_][2] + (WI * rm.d2) * dp;
                qb[G_] = qb[G_] - wr;
            }
        } else {
            if (dp < 0.0) {
                D3 lt = cd.lam[W_] + cd.lam[O_] + cd.lam[G_];
                D3 m = lt * cd.b[W.phase];
                double wm = WI * m.v;
                int a = W.phase;
                qv[a] = wm * dp;
                qd[a][0] = (WI * m.d0) * dp + wm;
                qd[a][1] = (WI * m.d1) * dp;
                qd[a][2] = (WI * m.d2) * dp;
                qb[a] = -wm;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R[a * n + c] += qv[a];
            qsum[a] += qv[a];
#pragma unroll
            for (int s = 0; s < 3; ++s) A[(size_t)(3 * a + s) * n + c] += qd[a][s];
        }
        // the controlled surface rate: injected component (positive when
        // injecting) for an injector, oil for a producer
        double rv, rd[3], rb;
        if (W.kind == 0) {
            int a = W.phase;
            rv = -qv[a]; rd[0] = -qd[a][0]; rd[1] = -qd[a][1]; rd[2] = -qd[a][2]; rb = -qb[a];
        } else {
            rv = qv[O_]; rd[0] = qd[O_][0]; rd[1] = qd[O_][1]; rd[2] = qd[O_][2]; rb = qb[O_];
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            wB[3 * con + s] = rate ? rd[s] : 0.0;
            wC[3 * con + s] = rate ? qb[s] : 0.0;
        }
        rsum += rv;
        dsum += rb;
    }
    __shared__ double sr[WELL_BS], sd[WELL_BS], sq[3][WELL_BS];
    sr[threadIdx.x] = rsum;
    sd[threadIdx.x] = dsum;
#pragma unroll
    for (int a = 0; a < 3; ++a) sq[a][threadIdx.x] = qsum[a];
    __syncthreads();
    for (int o = WELL_BS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sr[threadIdx.x] += sr[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
#pragma unroll
            for (int a = 0; a < 3; ++a) sq[a][threadIdx.x] += sq[a][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) W.qs[a] = sq[a][0];
        if (rate) {
            W.Rw = sr[0] - W.target;
            W.Dw = sd[0];
            if (W.Dw == 0.0) atomicAdd(&ns->dead_wells, 1);
        } else {
            W.Rw = 0.0;
            W.Dw = 1.0;
        }
    }
}

// Opening pressure of a well (one block, all threads get the result): the
// BHP at which the first connection starts to flow, min_j (p_j - h_j) for an
// injector, max_j for a producer.
__device__ double opening_bhp(const WellDev& W, const int* __restrict__ con_cell,
                              const double* __restrict__ p, const double* __restrict__ depth,
                              double g) {
    __shared__ double sh[128];
    double v = (W.kind == 0) ? 1e300 : -1e300;
    for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
        int c = con_cell[W.off + q];
        double ph = p[c] - g * W.rho_well * (depth[c] - W.z_datum);
        v = (W.kind == 0) ? fmin(v, ph) : fmax(v, ph);
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] = (W.kind == 0) ? fmin(sh[threadIdx.x], sh[threadIdx.x + o])
                                            : fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// A rate-controlled well without a flowing connection (D_w = 0) has no
// sensitivity to its BHP: move the BHP just past the opening pressure.
__global__ void k_fix_dead_wells(WellDev* __restrict__ wells, const int* __restrict__ con_cell,
                                 const double* __restrict__ p, const double* __restrict__ depth,
                                 double g) {
    WellDev& W = wells[blockIdx.x];
    if (!(W.ctl == 0 && W.Dw == 0.0)) return;   // uniform over the block
    double po = opening_bhp(W, con_cell, p, depth, g);
    if (threadIdx.x == 0) {
        W.bhp = (W.kind == 0) ? po + 1e-3 * fabs(po) : po - 1e-3 * fabs(po);
        if (W.full) W.xs[3] = W.bhp;
    }
}

// Initial BHP of a rate-controlled injector: the BHP that meets the target by
// the linear inflow relation with every connection injecting, capped by the
// limit (after k_begin_wells has set the datum and wellbore density).
__global__ void k_well_init_bhp(DevFluid F, WellDev* __restrict__ wells,
                                const int* __restrict__ con_cell,
                                const double* __restrict__ con_wi,
                                const double* __restrict__ depth, const double* __restrict__ p,
                                const double* __restrict__ sw, const double* __restrict__ x,
                                const uint8_t* __restrict__ flag) {
    WellDev& W = wells[blockIdx.x];
    if (W.ctl0 != 0 || W.kind != 0) return;
    __shared__ double sn[128], sd[128];
    double num = 0.0, den = 0.0;
    for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
        int con = W.off + q;
        int c = con_cell[con];
        CellD cd;
        cell_eval(F, p[c], sw[c], x[c], flag[c], cd);
        double mob = con_wi[con] * (cd.lam[W_].v + cd.lam[O_].v + cd.lam[G_].v) * cd.b[W.phase].v;
        double h = F.g * W.rho_well * (depth[c] - W.z_datum);
        num += mob * (p[c] - h);
        den += mob;
    }
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sn[threadIdx.x] += sn[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && sd[0] > 0.0) W.bhp = fmin(W.limit, (W.target + sn[0]) / sd[0]);
}

// ---------------------------------------------------------------------------
// a6: convergence measures (Section 2.3).
// ---------------------------------------------------------------------------
constexpr int NORM_BS = 256;

__global__ void __launch_bounds__(NORM_BS)
k_norm_partials(int n, const double* __restrict__ R, const double* __restrict__ pv,
                double* __restrict__ part) {
    // part[block*7 + {0..2 sum R, 3..5 max |R|/pv, 6 sum pv}]
    double s[3] = {0, 0, 0}, mx[3] = {0, 0, 0}, spv = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double v = pv[c];
        spv += v;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double r = R[a * n + c];
            s[a] += r;
            mx[a] = fmax(mx[a], fabs(r) / v);
        }
    }
    __shared__ double sh[7][NORM_BS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double vals[7] = {s[0], s[1], s[2], mx[0], mx[1], mx[2], spv};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double v = vals[q];
        for (int o = 16; o > 0; o >>= 1) {
            double w = __shfl_down_sync(0xffffffffu, v, o);
            v = (q >= 3 && q < 6) ? fmax(v, w) : v + w;
        }
        if (lane == 0) sh[q][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        int q = threadIdx.x;
        double v = sh[q][0];
        for (int w = 1; w < NORM_BS / 32; ++w) v = (q >= 3 && q < 6) ? fmax(v, sh[q][w]) : v + sh[q][w];
        part[blockIdx.x * 7 + q] = v;
    }
}

__global__ void k_norm_final(int n, int nb_norm, const double* __restrict__ part,
                             int nb_props, const double* __restrict__ part_binv, double dt,
                             int nw, const WellDev* __restrict__ wells,
                             NewtonStatus* __restrict__ ns) {
    // single warp, fixed-order reduction
    __shared__ double acc[10];
    if (threadIdx.x < 10) {
        int q = threadIdx.x;
        double v = 0.0;
        if (q < 7) {
            for (int b = 0; b < nb_norm; ++b) {
                double w = part[b * 7 + q];
                v = (q >= 3 && q < 6) ? fmax(v, w) : v + w;
            }
        } else {
            for (int b = 0; b < nb_props; ++b) v += part_binv[b * 3 + (q - 7)];
        }
        acc[q] = v;
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        double pvt = acc[6];
        for (int a = 0; a < 3; ++a) {
            double bavg = acc[7 + a] / n;
            ns->norms[a] = dt * bavg * fabs(acc[a]) / pvt;
            ns->norms[3 + a] = dt * bavg * acc[3 + a];
        }
        double wr = 0.0;
        for (int w = 0; w < nw; ++w) {
            const WellDev& W = wells[w];
            if (W.full) {
                // balances relative to the well's rate scale, fixed fractions
                // absolute, the control relative to its target
                const double qs = fmax(fabs(W.xs[0]), 1e-12);
                if (W.kind == 0) {
                    wr = fmax(wr, fabs(W.Rs[0]) / qs);
                    wr = fmax(wr, fmax(fabs(W.Rs[1]), fabs(W.Rs[2])));
                } else {
                    wr = fmax(wr, fmax(fmax(fabs(W.Rs[0]), fabs(W.Rs[1])), fabs(W.Rs[2])) / qs);
                }
                const double scale =
                    (W.ctl == 0) ? W.target : fmax(W.ctl0 == 1 ? W.target : W.limit, 1.0);
                wr = fmax(wr, fabs(W.Rs[3]) / scale);
            } else if (W.ctl == 0) {
                wr = fmax(wr, fabs(W.Rw) / fmax(fabs(W.target), 1e-300));
            }
        }
        ns->norms[6] = wr;
    }
}

// ---------------------------------------------------------------------------
// a9: Newton update with Appleyard chop and variable switching.
// ---------------------------------------------------------------------------
__global__ void k_newton_update(int n, DevFluid F, bo_newton_opts o,
                                const double* __restrict__ sol, double* __restrict__ p,
                                double* __restrict__ sw, double* __restrict__ x,
                                uint8_t* __restrict__ flag) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double dp = -sol[c], dsw = -sol[n + c], dx = -sol[2 * n + c];
    double pc = p[c];
    double dpmax = o.dp_rel_max * pc;
    if (fabs(dp) > dpmax) dp = (dp > 0 ? dpmax : -dpmax);
    uint8_t fl = flag[c];
    if (fl == 0) {
        double mx = fmax(fabs(dsw), fabs(dx));
        if (mx > o.ds_max) {
            double f = o.ds_max / mx;
            dsw *= f;
            dx *= f;
        }
    } else {
        if (fabs(dsw) > o.ds_max) {
            double f = o.ds_max / fabs(dsw);
            dsw *= f;
        }
        double drmax = o.drs_rel_max * F.R_sb;
        if (fabs(dx) > drmax) dx = (dx > 0 ? drmax : -drmax);
        // no far jump across the saturation boundary: the pressure may fall
        // at most bp_overshoot below the saturation pressure of the new r_go
        double pfloor = (1.0 - o.bp_overshoot) * (F.p_b * (x[c] + dx) / F.R_sb);
        if (pc + dp < pfloor && pfloor < pc) dp = pfloor - pc;
    }
    double pn = pc + dp, swn = sw[c] + dsw, xn = x[c] + dx;
    swn = fmin(fmax(swn, 0.0), 1.0);
    if (fl == 0) {
        if (xn > 1.0 - swn) xn = 1.0 - swn;
        if (xn < 0.0) {
            fl = 1;
            xn = pn * (F.R_sb / F.p_b);
        }
    } else {
        double rs = pn * (F.R_sb / F.p_b);
        if (xn > rs * (1.0 + o.eps_switch)) {
            fl = 0;
            xn = 0.0;
        }
    }
    p[c] = pn;
    sw[c] = swn;
    x[c] = xn;
    flag[c] = fl;
}

// BHP update of rate-controlled wells (one block per well, after the cell
// update): chopped Newton step, then the well chop -- the BHP may at most
// halve its distance to the opening pressure per iteration, so the well keeps
// flowing -- then the switch to BHP control past the limit.
__global__ void k_well_update(bo_newton_opts o, WellDev* __restrict__ wells,
                              const int* __restrict__ con_cell, const double* __restrict__ p,
                              const double* __restrict__ depth, double g) {
    WellDev& W = wells[blockIdx.x];
    if (W.ctl != 0) return;   // uniform over the block
    double po = opening_bhp(W, con_cell, p, depth, g);
    if (threadIdx.x != 0) return;
    double d = -W.xw;
    double dmax = o.dp_rel_max * W.bhp;
    if (fabs(d) > dmax) d = (d > 0 ? dmax : -dmax);
    double old = W.bhp;
    double nb = old + d;
    if (W.kind == 0) {
        double fl = (old > po) ? po + 0.5 * (old - po) : po + 1e-3 * fabs(po);
        if (nb < fl) nb = fl;
    } else {
        double cl = (old < po) ? po - 0.5 * (po - old) : po - 1e-3 * fabs(po);
        if (nb > cl) nb = cl;
    }
    W.bhp = nb;
    bool viol = (W.kind == 0) ? (W.bhp > W.limit) : (W.bhp < W.limit);
    if (viol) {
        W.ctl = 1;
        W.bhp = W.limit;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(int n, int bs) { return (n + bs - 1) / bs; }

void launch_static(bo_sim* s) {
    Geom g = s->geo;
    k_static<<<blocks_for(g.n, 256), 256, 0, s->stream>>>(g, s->d_dx, s->d_dy, s->d_dz, s->top,
                                                         s->d_perm, s->d_poro, s->d_T, s->d_pv,
                                                         s->d_depth);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_static");
}

void launch_wi(bo_sim* s, const int* d_con_well, const double* d_rw, const double* d_skin) {
    if (s->ncon == 0) return;
    k_wi<<<blocks_for(s->ncon, 128), 128, 0, s->stream>>>(s->geo, s->ncon, s->d_con_cell,
                                                         d_con_well, s->d_wells, s->d_dx,
                                                         s->d_dy, s->d_dz, s->d_perm, d_rw,
                                                         d_skin, s->d_con_wi);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_wi");
}

void launch_hydrostatic(bo_sim* s, double p_top, double sw, double rgo) {
    Geom g = s->geo;
    int cols = g.nx * g.ny;
    k_hydrostatic<<<blocks_for(cols, 128), 128, 0, s->stream>>>(g, s->fluid, p_top, sw, rgo,
                                                               s->d_depth, s->d_p, s->d_sw,
                                                               s->d_x, s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_hydrostatic");
}

void launch_begin_step(bo_sim* s) {
    int n = s->geo.n;
    k_begin_cells<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, s->fluid, s->d_p, s->d_sw,
                                                            s->d_x, s->d_flag, s->d_A0,
                                                            s->d_bk, s->d_bkflag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_begin_cells");
    launch_begin_wells(s);
}

void launch_begin_wells(bo_sim* s) {
    if (s->nw == 0) return;
    k_begin_wells<<<blocks_for(s->nw, 32), 32, 0, s->stream>>>(
        s->nw, s->fluid, s->d_wells, s->d_con_cell, s->d_depth, s->d_p, s->d_sw, s->d_x,
        s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_begin_wells");
}

void launch_restore(bo_sim* s) {
    int n = s->geo.n;
    int m = n > s->nw ? n : s->nw;
    k_restore<<<blocks_for(m, 256), 256, 0, s->stream>>>(n, s->d_p, s->d_sw, s->d_x, s->d_flag,
                                                        s->d_bk, s->d_bkflag, s->nw,
                                                        s->d_wells);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_restore");
}

int props_blocks(const bo_sim* s) { return blocks_for(s->geo.n, PROPS_BS); }
int norm_blocks(const bo_sim* s) {
    int b = blocks_for(s->geo.n, NORM_BS);
    return b < 1024 ? b : 1024;
}

void launch_assemble(bo_sim* s, double dt) {
    int n = s->geo.n;
    int tp = timer_id(s, "assemble_props");
    int tf = timer_id(s, "assemble_flux");
    timer_begin(s, tp);
    k_props<<<props_blocks(s), PROPS_BS, 0, s->stream>>>(
        n, s->fluid, s->d_p, s->d_sw, s->d_x, s->d_flag, s->d_pv, s->d_A0, dt, s->d_props,
        s->d_R, s->d_A, s->d_part /* binv partials live at the start of d_part */);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_props");
    timer_end(s, tp);
    timer_begin(s, tf);
    k_flux<<<blocks_for(n, FLUX_BS), FLUX_BS, 0, s->stream>>>(s->geo, s->fluid.g, s->d_props,
                                                             s->d_p, s->d_depth, s->d_T, s->d_R,
                                                             s->d_A);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_flux");
    timer_end(s, tf);
    BO_CUDA(cudaMemsetAsync(&s->d_ns->dead_wells, 0, sizeof(int), s->stream));
    if (s->well_model == BO_WELL_MODEL_STANDARD) {
        launch_std_wells_assemble(s, dt);
    } else if (s->nw > 0) {
        k_wells<<<s->nw, WELL_BS, 0, s->stream>>>(s->geo, s->fluid, s->d_wells, s->d_con_cell,
                                                  s->d_con_wi, s->d_depth, s->d_p, s->d_sw,
                                                  s->d_x, s->d_flag, s->d_R, s->d_A, s->d_wB,
                                                  s->d_wC, s->d_ns);
        count_launch(s, s->stream);
        BO_LAUNCH_CHECK("k_wells");
    }
}

void launch_fix_dead_wells(bo_sim* s) {
    if (s->nw == 0) return;
    k_fix_dead_wells<<<s->nw, 128, 0, s->stream>>>(s->d_wells, s->d_con_cell, s->d_p, s->d_depth,
                                                    s->fluid.g);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_fix_dead_wells");
}

void launch_well_init_bhp(bo_sim* s) {
    if (s->nw == 0) return;
    k_well_init_bhp<<<s->nw, 128, 0, s->stream>>>(s->fluid, s->d_wells, s->d_con_cell,
                                                   s->d_con_wi, s->d_depth, s->d_p, s->d_sw,
                                                   s->d_x, s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_well_init_bhp");
}

void launch_norms(bo_sim* s, double dt) {
    int n = s->geo.n;
    int nb = norm_blocks(s);
    int npb = props_blocks(s);
    double* part_norm = s->d_part + 3 * (size_t)npb;
    k_norm_partials<<<nb, NORM_BS, 0, s->stream>>>(n, s->d_R, s->d_pv, part_norm);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_norm_partials");
    k_norm_final<<<1, 32, 0, s->stream>>>(n, nb, part_norm, npb, s->d_part, dt, s->nw,
                                          s->d_wells, s->d_ns);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_norm_final");
}

void launch_newton_update(bo_sim* s, const bo_newton_opts& o) {
    int n = s->geo.n;
    k_newton_update<<<blocks_for(n, 256), 256, 0, s->stream>>>(n, s->fluid, o, s->d_xs, s->d_p,
                                                              s->d_sw, s->d_x, s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_newton_update");
    if (s->well_model == BO_WELL_MODEL_STANDARD) {
        launch_std_wells_update(s, o);
    } else if (s->nw > 0) {
        k_well_update<<<s->nw, 128, 0, s->stream>>>(o, s->d_wells, s->d_con_cell, s->d_p,
                                                     s->d_depth, s->fluid.g);
        count_launch(s, s->stream);
        BO_LAUNCH_CHECK("k_well_update");
    }
}

}  // namespace bo
