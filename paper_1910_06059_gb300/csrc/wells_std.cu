// Full standard well model on the GPU (arXiv 1910.06059, Section 2.2.1):
// four unknowns per well -- the weighted total rate Q_t, the weighted
// fractions F_w and F_g (Eq. weighted_total_rate, g = (1, 1, 0.01)) and the
// bottom-hole pressure -- with connection inflow by Eq. (wellinflow),
// cross-flow, one wellbore balance per component with a storage term
// (Eq. conseq-swell), the control equation (Eqs. well-control-bhp/rate),
// and the Schur complement of Eq. (wellequation) with a 4x4 D_w per well.
//
// Readings where the section is silent (the same in the oracle):
//  * Q_a = F_a Q_t / g_a, F_o = 1 - F_w - F_g; production positive.
//  * A producing connection (p_j > p_bhp + h_j, producers only) carries each
//    phase at the cell's mobility, gas adding r_go times the oil term.  An
//    injecting connection carries the total reservoir volume rate
//    WI lambda_t dp split by the wellbore mixture: q_a = WI lambda_t dp
//    Q_a / V, V = Q_w/b_w + Q_o/b_o + (Q_g - r Q_o)/b_g at the cell's
//    pressure, r = min(r_s(p), Q_g/Q_o) the gas the oil can hold.
//  * An injector's wellbore holds its injected phase: its equations are that
//    phase's balance, F_w and F_g fixed, and the control; its connections
//    only inject.
//  * Storage A_a,w = V_w F_a / g_a, V_w = pi r_w^2 times the perforated
//    thickness.  Heads and datum as for the reduced well.
//
// Layout: B_w (dR_w / dx_c) as [ncon][4][3], C_w (dR_c / dx_w) as
// [ncon][3][4], D_w and D_w^-1 row-major in the well's descriptor.  Each
// kernel runs one block per well, one thread per connection; the sums over
// connections are fixed-order tree reductions.
#include <cmath>

#include "cell.cuh"

namespace bo {

constexpr int SW_BS = 128;
constexpr int NV = 7;   // dual slots: cell (p, s_w, x), well (Q_t, F_w, F_g, p_bhp)

struct D7 {
    double v;
    double d[NV];
};

__device__ __forceinline__ D7 c7(double v) {
    D7 r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = 0.0;
    return r;
}
__device__ __forceinline__ D7 var7(double v, int slot) {
    D7 r = c7(v);
    r.d[slot] = 1.0;
    return r;
}
__device__ __forceinline__ D7 cell7(const D3& a) {
    D7 r = c7(a.v);
    r.d[0] = a.d0;
    r.d[1] = a.d1;
    r.d[2] = a.d2;
    return r;
}
__device__ __forceinline__ D7 operator+(const D7& a, const D7& b) {
    D7 r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
__device__ __forceinline__ D7 operator-(const D7& a, const D7& b) {
    D7 r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
__device__ __forceinline__ D7 operator-(const D7& a, double s) {
    D7 r = a;
    r.v = a.v - s;
    return r;
}
__device__ __forceinline__ D7 operator-(double s, const D7& a) {
    D7 r;
    r.v = s - a.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = -a.d[k];
    return r;
}
__device__ __forceinline__ D7 operator*(const D7& a, const D7& b) {
    D7 r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
__device__ __forceinline__ D7 operator*(double s, const D7& a) {
    D7 r;
    r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = s * a.d[k];
    return r;
}
__device__ __forceinline__ D7 operator/(const D7& a, const D7& b) {
    D7 r;
    r.v = a.v / b.v;
    const double den = b.v * b.v;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / den;
    return r;
}
__device__ __forceinline__ D7 operator/(const D7& a, double s) {
    D7 r;
    r.v = a.v / s;
#pragma unroll
    for (int k = 0; k < NV; ++k) r.d[k] = a.d[k] / s;
    return r;
}

// Surface rates q[3] of one connection into the well, as duals over the
// connection cell's and the well's unknowns.
__device__ void conn_rates(const DevFluid& F, const WellDev& W, double wi, double pc_,
                           double sw, double x, int flag, double depth_c, D7 (&q)[3]) {
    CellD cd;
    cell_eval(F, pc_, sw, x, flag, cd);
    const D7 pc = var7(pc_, 0);
    const D7 bhp = var7(W.xs[3], 6);
    const D7 fw = var7(W.xs[1], 4), fg = var7(W.xs[2], 5);
    const double h = F.g * W.rho_well * (depth_c - W.z_datum);
    const D7 dp = (pc - bhp) - h;
    q[0] = q[1] = q[2] = c7(0.0);
    if (dp.v > 0.0) {
        if (W.kind == 0) return;   // an injector's connections only inject
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = ((wi * cell7(cd.b[a])) * cell7(cd.lam[a])) * dp;
        q[2] = q[2] + cell7(cd.rgo) * q[1];
    } else if (dp.v < 0.0) {
        const D7 qres = (wi * ((cell7(cd.lam[0]) + cell7(cd.lam[1])) + cell7(cd.lam[2]))) * dp;
        const D7 Qw[3] = {fw / std_well_g(0), ((1.0 - fw) - fg) / std_well_g(1),
                          fg / std_well_g(2)};
        D7 rmix = c7(0.0);
        if (fabs(Qw[1].v) > 0.0) {
            const D7 rs = (F.R_sb / F.p_b) * pc;
            const D7 ratio = (Qw[2].v / Qw[1].v > 0.0) ? Qw[2] / Qw[1] : c7(0.0);
            rmix = rs.v < ratio.v ? rs : ratio;
        }
        const D7 V = (Qw[0] / cell7(cd.b[0]) + Qw[1] / cell7(cd.b[1])) +
                     (Qw[2] - rmix * Qw[1]) / cell7(cd.b[2]);
        if (V.v != 0.0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) q[a] = (qres * Qw[a]) / V;
        }
    }
}

// Gauss-Jordan inverse of a 4x4 matrix with partial pivoting; false on a
// zero pivot (inv is then zero).
__device__ bool inv4(const double* A, double* inv) {
    double m[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            m[r][c] = A[4 * r + c];
            m[r][4 + c] = (r == c) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(m[r][c]) > fabs(m[piv][c])) piv = r;
        if (!(fabs(m[piv][c]) > 0.0)) {
            for (int k = 0; k < 16; ++k) inv[k] = 0.0;
            return false;
        }
        if (piv != c)
            for (int k = 0; k < 8; ++k) {
                const double t = m[c][k];
                m[c][k] = m[piv][k];
                m[piv][k] = t;
            }
        const double ip = 1.0 / m[c][c];
        for (int k = 0; k < 8; ++k) m[c][k] *= ip;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const double f = m[r][c];
            if (f != 0.0)
                for (int k = 0; k < 8; ++k) m[r][k] -= f * m[c][k];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) inv[4 * r + c] = m[r][4 + c];
    return true;
}

// Fixed-order block sum of K values per thread into red[0..K) (all threads
// read the result after the call).
template <int K>
__device__ void block_sum(double (&v)[K], double (*sh)[SW_BS], double* red) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int o = SW_BS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < K) red[threadIdx.x] = sh[threadIdx.x][0];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Assembly: connection terms into the cell rows, B_w, C_w, the well residual
// and D_w, D_w^-1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SW_BS)
k_swells(int n, DevFluid F, WellDev* __restrict__ wells, const int* __restrict__ con_cell,
         const double* __restrict__ con_wi, const double* __restrict__ depth,
         const double* __restrict__ p, const double* __restrict__ sw,
         const double* __restrict__ x, const uint8_t* __restrict__ flag, double dt,
         double* __restrict__ R, double* __restrict__ A, double* __restrict__ wB4,
         double* __restrict__ wC4, NewtonStatus* __restrict__ ns) {
    WellDev& W = wells[blockIdx.x];
    const bool inj = (W.kind == 0);
    const int ph = W.phase;
    double acc[15];   // sum_j q_a (3), sum_j dq_a / dx_w (12)
#pragma unroll
    for (int k = 0; k < 15; ++k) acc[k] = 0.0;
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int con = W.off + j;
        const int c = con_cell[con];
        D7 q[3];
        conn_rates(F, W, con_wi[con], p[c], sw[c], x[c], flag[c], depth[c], q);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R[(size_t)a * n + c] += q[a].v;
#pragma unroll
            for (int s = 0; s < 3; ++s) A[(size_t)(3 * a + s) * n + c] += q[a].d[s];
#pragma unroll
            for (int k = 0; k < 4; ++k) wC4[12 * (size_t)con + 4 * a + k] = q[a].d[3 + k];
            acc[a] += q[a].v;
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[3 + 4 * a + k] += q[a].d[3 + k];
        }
        // B_w: the balances lose the connection's rates; an injector keeps
        // its injected phase's balance (row 0) and fixes F (rows 1, 2)
        double* b = wB4 + 12 * (size_t)con;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            if (inj) {
                b[s] = -q[ph].d[s];
                b[3 + s] = 0.0;
                b[6 + s] = 0.0;
            } else {
                b[s] = -q[0].d[s];
                b[3 + s] = -q[1].d[s];
                b[6 + s] = -q[2].d[s];
            }
            b[9 + s] = 0.0;
        }
    }
    __shared__ double sh[15][SW_BS];
    __shared__ double red[15];
    block_sum<15>(acc, sh, red);
    if (threadIdx.x != 0) return;
    // wellbore balances R_a = (A_a - A0_a)/dt + Q_a - sum_j q_a
    const D7 qt = var7(W.xs[0], 3), fw = var7(W.xs[1], 4), fg = var7(W.xs[2], 5);
    const D7 frac[3] = {fw, (1.0 - fw) - fg, fg};
    double Rw[4], D[16];
    for (int a = 0; a < 3; ++a) {
        const D7 bal = ((W.vw * frac[a]) / std_well_g(a) - W.A0s[a]) / dt +
                       (frac[a] * qt) / std_well_g(a);
        Rw[a] = bal.v - red[a];
        for (int k = 0; k < 4; ++k) D[4 * a + k] = bal.d[3 + k] - red[3 + 4 * a + k];
    }
    if (inj) {
        Rw[0] = Rw[ph];
        for (int k = 0; k < 4; ++k) D[k] = D[4 * ph + k];
        Rw[1] = W.xs[1] - (ph == 0 ? 1.0 : 0.0);
        Rw[2] = W.xs[2] - (ph == 2 ? 1.0 : 0.0);
        for (int k = 0; k < 4; ++k) {
            D[4 + k] = (k == 1) ? 1.0 : 0.0;
            D[8 + k] = (k == 2) ? 1.0 : 0.0;
        }
    }
    if (W.ctl == 1) {   // the BHP target, or the limit after a switch from rate control
        Rw[3] = W.xs[3] - (W.ctl0 == 1 ? W.target : W.limit);
        for (int k = 0; k < 4; ++k) D[12 + k] = (k == 3) ? 1.0 : 0.0;
    } else {
        const int a = inj ? ph : 1;
        const D7 Qa = (frac[a] * qt) / std_well_g(a);
        const D7 ctl = inj ? (c7(0.0) - Qa) - W.target : Qa - W.target;
        Rw[3] = ctl.v;
        for (int k = 0; k < 4; ++k) D[12 + k] = ctl.d[3 + k];
    }
    for (int k = 0; k < 4; ++k) W.Rs[k] = Rw[k];
    for (int k = 0; k < 16; ++k) W.D[k] = D[k];
    const bool ok = inv4(D, W.Dinv);
    W.singular = ok ? 0 : 1;
    // the reduced-well fields the shared host logic reads
    W.Rw = 0.0;
    W.Dw = ok ? 1.0 : 0.0;
    for (int a = 0; a < 3; ++a) W.qs[a] = (frac[a].v * qt.v) / std_well_g(a);
    if (!ok) {
        if (W.ctl == 0) atomicAdd(&ns->dead_wells, 1);
        atomicAdd(&ns->singular_wells, 1);
    }
}

// ---------------------------------------------------------------------------
// Reduced operator: corr_j = C_j D_w^-1 (sum_i B_i x_ci) per connection.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SW_BS)
k_swcorr(int n, const WellDev* __restrict__ wells, const int* __restrict__ con_cell,
         const double* __restrict__ wB4, const double* __restrict__ wC4,
         const double* __restrict__ xv, double* __restrict__ corr,
         const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const WellDev& W = wells[blockIdx.x];
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int con = W.off + j;
        const int c = con_cell[con];
        const double xc[3] = {xv[c], xv[(size_t)n + c], xv[2 * (size_t)n + c]};
        const double* b = wB4 + 12 * (size_t)con;
#pragma unroll
        for (int r = 0; r < 4; ++r) u[r] += b[3 * r] * xc[0] + b[3 * r + 1] * xc[1] + b[3 * r + 2] * xc[2];
    }
    __shared__ double sh[4][SW_BS];
    __shared__ double red[4];
    block_sum<4>(u, sh, red);
    double t[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        t[r] = W.Dinv[4 * r] * red[0] + W.Dinv[4 * r + 1] * red[1] + W.Dinv[4 * r + 2] * red[2] +
               W.Dinv[4 * r + 3] * red[3];
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int con = W.off + j;
        const double* cc = wC4 + 12 * (size_t)con;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            corr[3 * (size_t)con + a] =
                cc[4 * a] * t[0] + cc[4 * a + 1] * t[1] + cc[4 * a + 2] * t[2] + cc[4 * a + 3] * t[3];
    }
}

// Right-hand side: b_c -= C_j D_w^-1 R_w.
__global__ void __launch_bounds__(SW_BS)
k_swrhs(int n, const WellDev* __restrict__ wells, const int* __restrict__ con_cell,
        const double* __restrict__ wC4, double* __restrict__ b) {
    const WellDev& W = wells[blockIdx.x];
    double t[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        t[r] = W.Dinv[4 * r] * W.Rs[0] + W.Dinv[4 * r + 1] * W.Rs[1] +
               W.Dinv[4 * r + 2] * W.Rs[2] + W.Dinv[4 * r + 3] * W.Rs[3];
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int con = W.off + j;
        const int c = con_cell[con];
        const double* cc = wC4 + 12 * (size_t)con;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            b[(size_t)a * n + c] -=
                cc[4 * a] * t[0] + cc[4 * a + 1] * t[1] + cc[4 * a + 2] * t[2] + cc[4 * a + 3] * t[3];
    }
}

// Well rows of the solution: x_w = D_w^-1 (R_w - B_w x_r).
__global__ void __launch_bounds__(SW_BS)
k_swrecover(int n, WellDev* __restrict__ wells, const int* __restrict__ con_cell,
            const double* __restrict__ wB4, const double* __restrict__ xv) {
    WellDev& W = wells[blockIdx.x];
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int con = W.off + j;
        const int c = con_cell[con];
        const double xc[3] = {xv[c], xv[(size_t)n + c], xv[2 * (size_t)n + c]};
        const double* b = wB4 + 12 * (size_t)con;
#pragma unroll
        for (int r = 0; r < 4; ++r) u[r] += b[3 * r] * xc[0] + b[3 * r + 1] * xc[1] + b[3 * r + 2] * xc[2];
    }
    __shared__ double sh[4][SW_BS];
    __shared__ double red[4];
    block_sum<4>(u, sh, red);
    if (threadIdx.x != 0) return;
    double rr[4];
    for (int r = 0; r < 4; ++r) rr[r] = W.Rs[r] - red[r];
    for (int r = 0; r < 4; ++r)
        W.dxs[r] = W.Dinv[4 * r] * rr[0] + W.Dinv[4 * r + 1] * rr[1] + W.Dinv[4 * r + 2] * rr[2] +
                   W.Dinv[4 * r + 3] * rr[3];
}

// Opening pressure (all threads get it): min_j (p_j - h_j) for an injector,
// max_j for a producer.
__device__ double std_opening_bhp(const WellDev& W, const int* __restrict__ con_cell,
                                  const double* __restrict__ p, const double* __restrict__ depth,
                                  double g) {
    __shared__ double sh[SW_BS];
    double v = (W.kind == 0) ? 1e300 : -1e300;
    for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
        const int c = con_cell[W.off + j];
        const double ph = p[c] - g * W.rho_well * (depth[c] - W.z_datum);
        v = (W.kind == 0) ? fmin(v, ph) : fmax(v, ph);
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = SW_BS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] = (W.kind == 0) ? fmin(sh[threadIdx.x], sh[threadIdx.x + o])
                                            : fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Newton update of the well unknowns (after the cell update): the BHP step
// chopped to dp_rel_max of the BHP; a rate-controlled well's BHP at most
// halves its distance to the opening pressure (it keeps flowing); F_w in
// [0, 1], F_g in [0, 1 - F_w]; past its BHP limit a rate well switches to
// BHP control for the rest of the step.
__global__ void __launch_bounds__(SW_BS)
k_swupdate(bo_newton_opts o, WellDev* __restrict__ wells, const int* __restrict__ con_cell,
           const double* __restrict__ p, const double* __restrict__ depth, double g) {
    WellDev& W = wells[blockIdx.x];
    const double po = std_opening_bhp(W, con_cell, p, depth, g);
    if (threadIdx.x != 0) return;
    double d[4];
    for (int k = 0; k < 4; ++k) d[k] = -W.dxs[k];
    const double dmax = o.dp_rel_max * W.xs[3];
    if (fabs(d[3]) > dmax) d[3] = d[3] > 0 ? dmax : -dmax;
    const double old = W.xs[3];
    for (int k = 0; k < 4; ++k) W.xs[k] += d[k];
    if (W.ctl == 0) {
        if (W.kind == 0) {
            const double fl = (old > po) ? po + 0.5 * (old - po) : po + 1e-3 * fabs(po);
            W.xs[3] = fmax(W.xs[3], fl);
        } else {
            const double cl = (old < po) ? po - 0.5 * (po - old) : po - 1e-3 * fabs(po);
            W.xs[3] = fmin(W.xs[3], cl);
        }
    }
    W.xs[1] = fmin(fmax(W.xs[1], 0.0), 1.0);
    W.xs[2] = fmin(fmax(W.xs[2], 0.0), 1.0 - W.xs[1]);
    if (W.ctl == 0) {
        const bool viol = (W.kind == 0) ? (W.xs[3] > W.limit) : (W.xs[3] < W.limit);
        if (viol) {
            W.ctl = 1;
            W.xs[3] = W.limit;
        }
    }
    W.bhp = W.xs[3];
}

// Before the datum pass of a new state: control from the well's
// specification, the BHP of a BHP-controlled well at its target, Q_t and the
// fractions cleared, an injector's fraction of its injected phase at one.
__global__ void k_swreset(int nw, WellDev* __restrict__ wells) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    WellDev& W = wells[w];
    W.ctl = W.ctl0;
    if (W.ctl == 1) W.bhp = W.target;
    W.xs[0] = W.xs[1] = W.xs[2] = 0.0;
    W.xs[3] = W.bhp;
    if (W.kind == 0) W.xs[W.phase == 0 ? 1 : 2] = 1.0;
}

// After the datum pass: a producer's Q_t and fractions from its inflow at the
// current state and BHP (when it produces), an injector's Q_t from a rate
// target (zero under BHP control).
__global__ void __launch_bounds__(SW_BS)
k_swinit(DevFluid F, WellDev* __restrict__ wells, const int* __restrict__ con_cell,
         const double* __restrict__ con_wi, const double* __restrict__ depth,
         const double* __restrict__ p, const double* __restrict__ sw,
         const double* __restrict__ x, const uint8_t* __restrict__ flag) {
    WellDev& W = wells[blockIdx.x];
    double acc[3] = {0.0, 0.0, 0.0};
    if (W.kind == 1) {
        for (int j = threadIdx.x; j < W.ncon; j += blockDim.x) {
            const int con = W.off + j;
            const int c = con_cell[con];
            D7 q[3];
            conn_rates(F, W, con_wi[con], p[c], sw[c], x[c], flag[c], depth[c], q);
            for (int a = 0; a < 3; ++a) acc[a] += q[a].v;
        }
    }
    __shared__ double sh[3][SW_BS];
    __shared__ double red[3];
    block_sum<3>(acc, sh, red);
    if (threadIdx.x != 0) return;
    if (W.kind == 1) {
        const double qt = (std_well_g(0) * red[0] + std_well_g(1) * red[1]) + std_well_g(2) * red[2];
        if (qt > 0.0) {
            W.xs[0] = qt;
            W.xs[1] = std_well_g(0) * red[0] / qt;
            W.xs[2] = std_well_g(2) * red[2] / qt;
        }
    } else {
        W.xs[0] = (W.ctl == 0) ? -W.target * std_well_g(W.phase) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void std_wells_setup(bo_sim* s) {
    if (s->ncon == 0) return;
    if (!s->d_wB4) {
        BO_CUDA(cudaMalloc(&s->d_wB4, sizeof(double) * 12 * s->ncon));
        BO_CUDA(cudaMalloc(&s->d_wC4, sizeof(double) * 12 * s->ncon));
        BO_CUDA(cudaMalloc(&s->d_wcorr, sizeof(double) * 3 * s->ncon));
        BO_CUDA(cudaMemset(s->d_wB4, 0, sizeof(double) * 12 * s->ncon));
        BO_CUDA(cudaMemset(s->d_wC4, 0, sizeof(double) * 12 * s->ncon));
        BO_CUDA(cudaMemset(s->d_wcorr, 0, sizeof(double) * 3 * s->ncon));
    }
}

void launch_std_wells_assemble(bo_sim* s, double dt) {
    if (s->nw == 0) return;
    BO_CUDA(cudaMemsetAsync(&s->d_ns->singular_wells, 0, sizeof(int), s->stream));
    k_swells<<<s->nw, SW_BS, 0, s->stream>>>(s->geo.n, s->fluid, s->d_wells, s->d_con_cell,
                                              s->d_con_wi, s->d_depth, s->d_p, s->d_sw, s->d_x,
                                              s->d_flag, dt, s->d_R, s->d_A, s->d_wB4, s->d_wC4,
                                              s->d_ns);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_swells");
}

void launch_std_wells_init(bo_sim* s) {
    if (s->nw == 0) return;
    k_swreset<<<(s->nw + 31) / 32, 32, 0, s->stream>>>(s->nw, s->d_wells);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_swreset");
    launch_begin_wells(s);
    k_swinit<<<s->nw, SW_BS, 0, s->stream>>>(s->fluid, s->d_wells, s->d_con_cell, s->d_con_wi,
                                             s->d_depth, s->d_p, s->d_sw, s->d_x, s->d_flag);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_swinit");
}

void enqueue_std_well_corr(bo_sim* s, cudaStream_t st, const double* x, const KrylovScalars* ks) {
    if (s->nw == 0) return;
    k_swcorr<<<s->nw, SW_BS, 0, st>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB4, s->d_wC4, x,
                                      s->d_wcorr, ks);
    count_launch(s, st);
}

void enqueue_std_wells_rhs(bo_sim* s, cudaStream_t st, double* b) {
    if (s->nw == 0) return;
    k_swrhs<<<s->nw, SW_BS, 0, st>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wC4, b);
    count_launch(s, st);
}

void launch_std_wells_recover(bo_sim* s) {
    if (s->nw == 0) return;
    k_swrecover<<<s->nw, SW_BS, 0, s->stream>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB4,
                                                s->d_xs);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_swrecover");
}

void launch_std_wells_update(bo_sim* s, const bo_newton_opts& o) {
    if (s->nw == 0) return;
    k_swupdate<<<s->nw, SW_BS, 0, s->stream>>>(o, s->d_wells, s->d_con_cell, s->d_p, s->d_depth,
                                               s->fluid.g);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_swupdate");
}

}  // namespace bo
