// Linear solver of the Newton step (arXiv 1910.06059, Section 2.3.1):
// block ILU(0)-preconditioned BiCGStab on the well-reduced system of
// Eq. (wellequation).
//
// ILU(0) on the 7-point pattern.  In natural order the lower neighbours of a
// cell are -x, -y, -z and the upper ones +x, +y, +z.  The grid graph is
// bipartite (neighbours differ in the parity of i+j+k) so every fill position
// of ILU(0), reached through two edges, is the cell itself or a cell outside
// the pattern: only the diagonal blocks change,
//     D_c = A_cc - sum_{k lower} A_ck D_k^-1 A_kc,
// and M = (L_A + D) D^-1 (D + U_A).  The factorisation stores, in wavefront
// order, D_c^-1 and the scaled blocks D_c^-1 A_ck (lower) and D_c^-1 A_cj
// (upper), so that
//     forward  y_c = D_c^-1 r_c - sum_lower (D_c^-1 A_ck) y_k
//     backward z_c = y_c       - sum_upper (D_c^-1 A_cj) z_j
// Cells with equal i+j+k (a wavefront level) are independent in both
// recurrences; levels run in order.
//
// BiCGStab (van der Vorst), right preconditioned, all scalars on the device:
// every kernel reads the recurrence state and returns at once when the solve
// has finished, so a fixed CUDA graph of several iterations can be replayed
// until the host sees the finished flag.  Reductions are deterministic:
// per-block partials in a fixed grid, summed in a fixed order.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace bo {

constexpr int VEC_BS = 256;
constexpr int VEC_GRID = 152 * 4;   // one wave of 4 blocks per SM

__device__ __forceinline__ void cell_ijk(const Geom& g, int c, int& i, int& j, int& k) {
    i = c % g.nx;
    j = (c / g.nx) % g.ny;
    k = c / (g.nx * g.ny);
}

__device__ __forceinline__ bool ks_skip(const KrylovScalars* ks) {
    return ks != nullptr && ks->state != KS_RUN;
}

// ---------------------------------------------------------------------------
// Reduced operator y = A x - sum_w C_w D_w^-1 (B_w x)  (+ fused dot partials)
// ---------------------------------------------------------------------------
// Per rate well: sop_w = (B_w . x) / D_w.  One block per well.
__global__ void k_wdot(int n, const WellDev* __restrict__ wells, const int* __restrict__ con_cell,
                       const double* __restrict__ wB, const double* __restrict__ x,
                       double* __restrict__ sop, const KrylovScalars* __restrict__ ks) {
    if (ks_skip(ks)) return;
    const WellDev& W = wells[blockIdx.x];
    double acc = 0.0;
    if (W.ctl == 0) {
        for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
            int con = W.off + q;
            int c = con_cell[con];
            acc += wB[3 * con] * x[c] + wB[3 * con + 1] * x[n + c] + wB[3 * con + 2] * x[2 * n + c];
        }
    }
    __shared__ double sh[128];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sop[blockIdx.x] = (W.ctl == 0) ? sh[0] / W.Dw : 0.0;
}

// mode 0: no dots; 1: part0 = (rh, y); 2: part0 = (y, s), part1 = (y, y);
// 3: y = o1 - Op x (the true residual of b = o1), part0 = (y, y)
template <int MODE>
__global__ void __launch_bounds__(VEC_BS)
k_spmv(Geom g, const double* __restrict__ A, const double* __restrict__ x,
       double* __restrict__ y, const int* __restrict__ cellcon,
       const int* __restrict__ con_well, const double* __restrict__ wC,
       const double* __restrict__ sop, const double* __restrict__ ccorr,
       const double* __restrict__ o1, double* __restrict__ part,
       const KrylovScalars* __restrict__ ks) {
    if (ks_skip(ks)) return;
    const int n = g.n;
    const int plane = g.nx * g.ny;
    double d0 = 0.0, d1 = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        double xv[3] = {x[c], x[n + c], x[2 * n + c]};
        double acc[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            acc[r] = A[(size_t)(3 * r) * n + c] * xv[0] + A[(size_t)(3 * r + 1) * n + c] * xv[1] +
                     A[(size_t)(3 * r + 2) * n + c] * xv[2];
        const bool has[6] = {i > 0, i + 1 < g.nx, j > 0, j + 1 < g.ny, k > 0, k + 1 < g.nz};
        const int nbc[6] = {c - 1, c + 1, c - g.nx, c + g.nx, c - plane, c + plane};
#pragma unroll
        for (int b = 1; b <= 6; ++b) {
            if (!has[b - 1]) continue;
            int q = nbc[b - 1];
            double xn[3] = {x[q], x[n + q], x[2 * n + q]};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double* Ab = A + (size_t)(b * 9 + 3 * r) * n + c;
                acc[r] += Ab[0] * xn[0] + Ab[(size_t)n] * xn[1] + Ab[2 * (size_t)n] * xn[2];
            }
        }
        int con = cellcon[c];
        if (con >= 0) {
            if (ccorr != nullptr) {   // full standard wells: C_j D^-1 B x per connection
#pragma unroll
                for (int r = 0; r < 3; ++r) acc[r] -= ccorr[3 * con + r];
            } else {
                double sw = sop[con_well[con]];
#pragma unroll
                for (int r = 0; r < 3; ++r) acc[r] -= wC[3 * con + r] * sw;
            }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            if (MODE == 3) {
                acc[r] = o1[r * n + c] - acc[r];
                d0 += acc[r] * acc[r];
            }
            y[r * n + c] = acc[r];
            if (MODE == 1) d0 += o1[r * n + c] * acc[r];
            if (MODE == 2) {
                d0 += acc[r] * o1[r * n + c];
                d1 += acc[r] * acc[r];
            }
        }
    }
    if (MODE == 0) return;
    __shared__ double sh[2][VEC_BS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
    }
    if (lane == 0) {
        sh[0][wid] = d0;
        sh[1][wid] = d1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < VEC_BS / 32; ++w) v += sh[threadIdx.x][w];
        part[threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

// ---------------------------------------------------------------------------
// BLAS-1 kernels with fused dot partials (vectors of length N = 3n)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void block_partials(double (&v)[K], double* __restrict__ part) {
    __shared__ double sh[K][VEC_BS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double x = 0.0;
        for (int w = 0; w < VEC_BS / 32; ++w) x += sh[threadIdx.x][w];
        part[threadIdx.x * gridDim.x + blockIdx.x] = x;
    }
}

// b = R - sum_w C_w (R_w / D_w); x = 0; r = rh = b; p = v = 0; part0 = (r, r)
__global__ void __launch_bounds__(VEC_BS)
k_krylov_init(int N, const double* __restrict__ R, double* __restrict__ b,
              double* __restrict__ x, double* __restrict__ r, double* __restrict__ rh,
              double* __restrict__ p, double* __restrict__ v, double* __restrict__ part) {
    double d[1] = {0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
        double bv = b[q];
        x[q] = 0.0;
        r[q] = bv;
        rh[q] = bv;
        p[q] = 0.0;
        v[q] = 0.0;
        d[0] += bv * bv;
    }
    block_partials<1>(d, part);
    (void)R;
}

__global__ void k_rhs_copy(int N, const double* __restrict__ R, double* __restrict__ b) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x)
        b[q] = R[q];
}

__global__ void k_rhs_wells(int n, const WellDev* __restrict__ wells,
                            const int* __restrict__ con_cell, const double* __restrict__ wC,
                            double* __restrict__ b) {
    const WellDev& W = wells[blockIdx.x];
    if (W.ctl != 0) return;
    double s = W.Rw / W.Dw;
    for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
        int con = W.off + q;
        int c = con_cell[con];
#pragma unroll
        for (int e = 0; e < 3; ++e) b[e * n + c] -= wC[3 * con + e] * s;
    }
}

// p = r + beta (p - omega v)
__global__ void __launch_bounds__(VEC_BS)
k_p_update(int N, const double* __restrict__ r, double* __restrict__ p,
           const double* __restrict__ v, const KrylovScalars* __restrict__ ks) {
    if (ks->state != KS_RUN) return;
    double beta = ks->beta, omega = ks->omega;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x)
        p[q] = r[q] + beta * (p[q] - omega * v[q]);
}

// s = r - alpha v ; part0 = (s, s)
__global__ void __launch_bounds__(VEC_BS)
k_s_update(int N, const double* __restrict__ r, const double* __restrict__ v,
           double* __restrict__ s, double* __restrict__ part,
           const KrylovScalars* __restrict__ ks) {
    if (ks->state != KS_RUN) return;
    double alpha = ks->alpha;
    double d[1] = {0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
        double sv = r[q] - alpha * v[q];
        s[q] = sv;
        d[0] += sv * sv;
    }
    block_partials<1>(d, part);
}

// RUN:  x += alpha ph + omega sh ; r = s - omega t ; part0 = (r, r), part1 = (rh, r)
// HALF: x += alpha ph
__global__ void __launch_bounds__(VEC_BS)
k_xr_update(int N, double* __restrict__ x, const double* __restrict__ ph,
            const double* __restrict__ sh, const double* __restrict__ s,
            const double* __restrict__ t, double* __restrict__ r,
            const double* __restrict__ rh, double* __restrict__ part,
            const KrylovScalars* __restrict__ ks) {
    int st = ks->state;
    if (st == KS_DONE) return;
    double alpha = ks->alpha, omega = ks->omega;
    if (st == KS_HALF) {
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x)
            x[q] += alpha * ph[q];
        return;
    }
    double d[2] = {0.0, 0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
        x[q] += alpha * ph[q] + omega * sh[q];
        double rv = s[q] - omega * t[q];
        r[q] = rv;
        d[0] += rv * rv;
        d[1] += rh[q] * rv;
    }
    block_partials<2>(d, part);
}

// ---------------------------------------------------------------------------
// Scalar steps of the recurrence (one block; fixed-order sums of partials)
// ---------------------------------------------------------------------------
__device__ double sum_partials(const double* __restrict__ part, int nb) {
    // called by the whole block of 256 threads; returns the sum in thread 0
    __shared__ double sh[256];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void breakdown(KrylovScalars* ks) {
    ks->state = KS_DONE;
    ks->status = LS_BREAKDOWN;
    ks->it -= 1;
}

// setup: nr0 = ||b||, rho = (rh, r) = ||b||^2
__global__ void k_s_setup(KrylovScalars* ks, const double* __restrict__ part, int nb, double tol,
                          int maxit, double inner) {
    double rr = sum_partials(part, nb);
    if (threadIdx.x != 0) return;
    ks->tol = tol;
    ks->maxit = maxit;
    ks->it = 0;
    ks->rho_old = 1.0;
    ks->alpha = 1.0;
    ks->omega = 1.0;
    ks->beta = 0.0;
    ks->nr0 = sqrt(rr);
    ks->rho = rr;
    ks->last_nr = ks->nr0;
    ks->status = LS_NOT_CONVERGED;
    ks->state = KS_RUN;
    ks->half_exit = 0;
    ks->restarts = 0;
    ks->true_nr = ks->nr0;
    ks->inner = inner;
    ks->stop = fmax(tol, inner) * ks->nr0;
    if (ks->nr0 == 0.0) {
        ks->state = KS_DONE;
        ks->status = LS_OK;
    }
}

// iteration start: rho (already in ks->rho), beta
__global__ void k_s1(KrylovScalars* ks) {
    if (ks->state != KS_RUN) return;
    if (ks->it == ks->maxit) {
        ks->state = KS_DONE;
        ks->status = LS_NOT_CONVERGED;
        return;
    }
    ks->it += 1;
    double rho = ks->rho;
    if (rho == 0.0 || !isfinite(rho)) {
        breakdown(ks);
        return;
    }
    ks->beta = (rho / ks->rho_old) * (ks->alpha / ks->omega);
}

// alpha = rho / (rh, v)
__global__ void k_s2(KrylovScalars* ks, const double* __restrict__ part, int nb) {
    if (ks->state != KS_RUN) return;
    double rv = sum_partials(part, nb);
    if (threadIdx.x != 0) return;
    if (rv == 0.0 || !isfinite(rv)) {
        breakdown(ks);
        return;
    }
    ks->alpha = ks->rho / rv;
}

// ||s|| <= tol ||r0||: finish with the half step
__global__ void k_s3(KrylovScalars* ks, const double* __restrict__ part, int nb) {
    if (ks->state != KS_RUN) return;
    double ss = sum_partials(part, nb);
    if (threadIdx.x != 0) return;
    double ns = sqrt(ss);
    if (ns <= ks->stop) {
        ks->state = KS_HALF;
        ks->half_exit = 1;
        ks->last_nr = ns;
    }
}

// omega = (t, s) / (t, t)
__global__ void k_s4(KrylovScalars* ks, const double* __restrict__ part, int nb) {
    if (ks->state != KS_RUN) return;
    double ts = sum_partials(part, nb);
    double tt = sum_partials(part + nb, nb);
    if (threadIdx.x != 0) return;
    if (tt == 0.0 || !isfinite(tt)) {
        breakdown(ks);
        return;
    }
    double om = ts / tt;
    if (om == 0.0 || !isfinite(om)) {
        breakdown(ks);
        return;
    }
    ks->omega = om;
}

// convergence on ||r||; next rho = (rh, r)
__global__ void k_s5(KrylovScalars* ks, const double* __restrict__ part, int nb) {
    int st = ks->state;
    if (st == KS_DONE) return;
    if (st == KS_HALF) {
        if (threadIdx.x == 0) {
            ks->state = KS_DONE;
            ks->status = LS_OK;
        }
        return;
    }
    double rr = sum_partials(part, nb);
    double rhr = sum_partials(part + nb, nb);
    if (threadIdx.x != 0) return;
    double nr = sqrt(rr);
    ks->last_nr = nr;
    if (nr <= ks->stop) {
        ks->state = KS_DONE;
        ks->status = LS_OK;
        return;
    }
    ks->rho_old = ks->rho;
    ks->rho = rhr;
}

// The recurrence's residual decides when to stop, the true residual
// ||b - Op x|| (FP64, computed after the stop) decides whether to accept.
// Otherwise BiCGStab restarts from the true residual with the iteration count
// carried on: after drift of the recurrence, or after a cycle of the mixed-
// precision solver that stopped at its own target inner * ||r_start||
// (an FP32 preconditioner is not exactly the same linear map at every
// application, which limits how far one BiCGStab cycle can reduce the
// residual).  With allow == 0 the solve is reported as not converged instead.
__global__ void k_s_restart(KrylovScalars* ks, const double* __restrict__ part, int nb, int allow) {
    double rr = sum_partials(part, nb);
    if (threadIdx.x != 0) return;
    double nr = sqrt(rr);
    ks->true_nr = nr;
    if (ks->status != LS_OK) return;
    if (nr <= ks->tol * ks->nr0) return;
    if (!allow || ks->it >= ks->maxit || !isfinite(nr)) {
        ks->status = LS_NOT_CONVERGED;
        return;
    }
    ks->restarts += 1;
    ks->stop = fmax(ks->tol * ks->nr0, ks->inner * nr);
    ks->rho = rr;
    ks->rho_old = 1.0;
    ks->alpha = 1.0;
    ks->omega = 1.0;
    ks->beta = 0.0;
    ks->last_nr = nr;
    ks->half_exit = 0;
    ks->status = LS_NOT_CONVERGED;
    ks->state = KS_RUN;
}

// restart vectors: rh = r, p = v = 0 (only when k_s_restart restarted)
__global__ void k_restart_vectors(int N, const double* __restrict__ r, double* __restrict__ rh,
                                  double* __restrict__ p, double* __restrict__ v,
                                  const KrylovScalars* __restrict__ ks) {
    if (ks->state != KS_RUN) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
        rh[q] = r[q];
        p[q] = 0.0;
        v[q] = 0.0;
    }
}

// x_w = (R_w - B_w x_r) / D_w
__global__ void k_well_recover(int n, WellDev* __restrict__ wells,
                               const int* __restrict__ con_cell, const double* __restrict__ wB,
                               const double* __restrict__ x) {
    WellDev& W = wells[blockIdx.x];
    double acc = 0.0;
    if (W.ctl == 0) {
        for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
            int con = W.off + q;
            int c = con_cell[con];
            acc += wB[3 * con] * x[c] + wB[3 * con + 1] * x[n + c] + wB[3 * con + 2] * x[2 * n + c];
        }
    }
    __shared__ double sh[128];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) W.xw = (W.ctl == 0) ? (W.Rw - sh[0]) / W.Dw : 0.0;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static inline int blocks_for(int n, int bs) { return (n + bs - 1) / bs; }

static int* factor_bad(bo_sim* s) { return reinterpret_cast<int*>(&s->d_ns->pad); }

void enqueue_precond_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                           const KrylovScalars* ks) {
    if (s->precond == BO_PRECOND_CPR) {
        enqueue_cpr_apply(s, st, r, z, ks);
        return;
    }
    enqueue_fwd(s, st, r, z, ks);
    enqueue_bwd(s, st, z, ks);
}

static double* d_sop(bo_sim* s) { return s->d_part + 8 * VEC_GRID; }

template <int MODE>
static void enqueue_op(bo_sim* s, cudaStream_t st, const double* x, double* y, const double* o1,
                       const KrylovScalars* ks) {
    enqueue_well_dots(s, st, x, ks);
    k_spmv<MODE><<<VEC_GRID, VEC_BS, 0, st>>>(s->geo, s->d_A, x, y, s->d_cellcon,
                                              s->d_cellcon + s->geo.n, s->d_wC, d_sop(s),
                                              well_corr(s), o1, s->d_part, ks);
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_spmv");
}

void count_launch(bo_sim* s, cudaStream_t st, int k) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return;
    s->launches += k;
}

void note_graph(bo_sim* s, cudaGraph_t g, cudaGraphExec_t exec) {
    size_t count = 0;
    BO_CUDA(cudaGraphGetNodes(g, nullptr, &count));
    std::vector<cudaGraphNode_t> nodes(count);
    if (count) BO_CUDA(cudaGraphGetNodes(g, nodes.data(), &count));
    int kernels = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        BO_CUDA(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel) kernels += 1;
    }
    s->graph_kernels.emplace_back(exec, kernels);
}

void graph_launch(bo_sim* s, cudaGraphExec_t exec, cudaStream_t st) {
    BO_CUDA(cudaGraphLaunch(exec, st));
    for (const auto& gk : s->graph_kernels)
        if (gk.first == exec) {
            s->launches += gk.second;
            break;
        }
}

// Timers: event pairs recorded on the launching stream (graph nodes when captured).
int timer_id(bo_sim* s, const char* name) {
    for (int q = 0; q < s->ntimers; ++q)
        if (s->timer_name[q] == name) return q;
    if (s->ntimers >= MAX_TIMERS) return -1;
    s->timer_name[s->ntimers] = name;
    return s->ntimers++;
}


void timer_begin(bo_sim* s, int id) {
    if (!s->timing || id < 0) return;
    EagerTimer t{};
    t.id = id;
    BO_CUDA(cudaEventCreate(&t.a));
    BO_CUDA(cudaEventCreate(&t.b));
    BO_CUDA(cudaEventRecord(t.a, s->stream));
    s->pending_timers.push_back(t);   // per object: ensemble workers time members concurrently
}
void timer_end(bo_sim* s, int id) {
    if (!s->timing || id < 0) return;
    for (auto it = s->pending_timers.rbegin(); it != s->pending_timers.rend(); ++it)
        if (it->id == id) {
            BO_CUDA(cudaEventRecord(it->b, s->stream));
            return;
        }
}
void timers_flush(bo_sim* s) {
    if (s->pending_timers.empty()) return;
    BO_CUDA(cudaStreamSynchronize(s->stream));
    for (auto& t : s->pending_timers) {
        float ms = 0.f;
        BO_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        s->timer_ms[t.id] += ms;
        s->timer_n[t.id] += 1;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    s->pending_timers.clear();
}

// One BiCGStab iteration enqueued on st (captured into a graph).
// ev (may be null): 2 events per timed op, ops: 0 fwd+bwd sweeps (2 applies),
// recorded as [fwd1, bwd1, spmv1, fwd2, bwd2, spmv2, blas] pairs.
enum { TI_FWD = 0, TI_BWD = 1, TI_SPMV = 2, TI_BLAS = 3, TI_N = 4 };

// ml: the learned correction follows each preconditioner apply (z += delta);
// collect: the residual of every iteration is stored as a training sample.
static void enqueue_iteration(bo_sim* s, cudaStream_t st, cudaEvent_t* ev, bool ml, bool collect) {
    const int N = 3 * s->geo.n;
    KrylovScalars* ks = s->d_ks;
    double* part = s->d_part;
    auto rec = [&](int k) {
        // an external event node: a plain record inside stream capture would
        // only mark a dependency
        if (ev) BO_CUDA(cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal));
    };
    // events: 0,1 blas(p); 2,3 fwd1; 4,5 bwd1; 6,7 spmv1; 8,9 blas(s); 10,11 fwd2; 12,13 bwd2;
    //         14,15 spmv2; 16,17 blas(xr)
    k_s1<<<1, 1, 0, st>>>(ks);
    count_launch(s, st);
    rec(0);
    k_p_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_r, s->d_pk, s->d_v, ks);
    count_launch(s, st);
    rec(1);
    // ph = M^-1 p
    rec(2);
    if (s->precond == BO_PRECOND_CPR) {   // the whole two-stage apply is timed as one
        enqueue_cpr_apply(s, st, s->d_pk, s->d_ph, ks);
        rec(3);
        rec(4);
    } else {
        enqueue_fwd(s, st, s->d_pk, s->d_ph, ks);
        rec(3);
        rec(4);
        enqueue_bwd(s, st, s->d_ph, ks);
    }
    rec(5);
    rec(18);
    if (ml) enqueue_learn_apply(s, st, s->d_pk, s->d_ph, ks);
    rec(19);
    rec(6);
    enqueue_op<1>(s, st, s->d_ph, s->d_v, s->d_rh, ks);
    rec(7);
    k_s2<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    count_launch(s, st);
    rec(8);
    k_s_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_r, s->d_v, s->d_s, part, ks);
    count_launch(s, st);
    rec(9);
    k_s3<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    count_launch(s, st);
    rec(10);
    if (s->precond == BO_PRECOND_CPR) {
        enqueue_cpr_apply(s, st, s->d_s, s->d_sh, ks);
        rec(11);
        rec(12);
    } else {
        enqueue_fwd(s, st, s->d_s, s->d_sh, ks);
        rec(11);
        rec(12);
        enqueue_bwd(s, st, s->d_sh, ks);
    }
    rec(13);
    rec(20);
    if (ml) enqueue_learn_apply(s, st, s->d_s, s->d_sh, ks);
    rec(21);
    rec(14);
    enqueue_op<2>(s, st, s->d_sh, s->d_t, s->d_s, ks);
    rec(15);
    k_s4<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    count_launch(s, st);
    rec(16);
    k_xr_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_xs, s->d_ph, s->d_sh, s->d_s, s->d_t,
                                             s->d_r, s->d_rh, part, ks);
    count_launch(s, st);
    rec(17);
    if (collect) enqueue_learn_collect(s, st, s->d_r, ks);
    k_s5<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    count_launch(s, st);
    BO_LAUNCH_CHECK("bicgstab iteration");
}

static constexpr int EV_PER_ITER = 22;

static cudaGraphExec_t capture(bo_sim* s, int iters, cudaEvent_t* ev, bool ml, bool collect) {
    cudaStream_t cs;
    BO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    BO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < iters; ++q)
        enqueue_iteration(s, cs, ev ? ev + q * EV_PER_ITER : nullptr, ml, collect);
    BO_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec;
    BO_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    note_graph(s, graph, exec);
    BO_CUDA(cudaGraphDestroy(graph));
    BO_CUDA(cudaStreamDestroy(cs));
    return exec;
}

static cudaGraphExec_t capture_factor(bo_sim* s) {
    cudaStream_t cs;
    BO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    BO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    enqueue_factor(s, cs, factor_bad(s));
    if (s->precond == BO_PRECOND_CPR) enqueue_cpr_setup(s, cs);
    if (s->ml_on || learn_collecting(s)) enqueue_learn_features(s, cs);
    BO_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec;
    BO_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    note_graph(s, graph, exec);
    BO_CUDA(cudaGraphDestroy(graph));
    BO_CUDA(cudaStreamDestroy(cs));
    return exec;
}

void build_graphs(bo_sim* s) {
    destroy_graphs(s);
    s->g_factor = capture_factor(s);
    s->g_iter = capture(s, s->iters_per_graph, nullptr, false, learn_collecting(s));
    if (s->ml_on) s->g_iter_ml = capture(s, s->iters_per_graph, nullptr, true, learn_collecting(s));
    if (s->mixed) {   // FP64 sweeps for a solve the FP32 sweeps fail
        s->mixed = false;
        try {
            s->g_iter64 = capture(s, s->iters_per_graph, nullptr, false, false);
        } catch (...) {
            s->mixed = true;
            throw;
        }
        s->mixed = true;
    }
}

void destroy_graphs(bo_sim* s) {
    if (s->g_iter) cudaGraphExecDestroy(s->g_iter);
    if (s->g_factor) cudaGraphExecDestroy(s->g_factor);
    if (s->g_iter_timed) cudaGraphExecDestroy(s->g_iter_timed);
    if (s->g_iter_ml) cudaGraphExecDestroy(s->g_iter_ml);
    if (s->g_iter64) cudaGraphExecDestroy(s->g_iter64);
    s->g_iter = s->g_factor = s->g_iter_timed = s->g_iter_ml = s->g_iter64 = nullptr;
    for (cudaEvent_t e : s->iter_events) cudaEventDestroy(e);
    s->iter_events.clear();
    s->graph_kernels.clear();
}

static void ensure_timed_graph(bo_sim* s) {
    if (s->g_iter_timed) return;
    s->iter_events.resize((size_t)EV_PER_ITER * s->iters_per_graph);
    for (auto& e : s->iter_events) BO_CUDA(cudaEventCreate(&e));
    s->g_iter_timed = capture(s, s->iters_per_graph, s->iter_events.data(), s->ml_on, learn_collecting(s));
}


void launch_factor(bo_sim* s) {
    int t = timer_id(s, "ilu_factor");
    BO_CUDA(cudaMemsetAsync(factor_bad(s), 0, sizeof(int), s->stream));
    if (s->precond == BO_PRECOND_CPR)
        BO_CUDA(cudaMemsetAsync(cpr_status_ptr(s), 0, sizeof(int), s->stream));
    timer_begin(s, t);
    graph_launch(s, s->g_factor, s->stream);
    timer_end(s, t);
}

void launch_precond(bo_sim* s, const double* r, double* z) {
    if (block_solve_active(s)) {
        launch_block_precond(s, r, z);
        return;
    }
    enqueue_precond_apply(s, s->stream, r, z, nullptr);
}

void enqueue_op_resid(bo_sim* s, cudaStream_t st, const double* x, double* y, const double* b,
                      const KrylovScalars* ks) {
    enqueue_op<3>(s, st, x, y, b, ks);
}

const double* enqueue_well_dots(bo_sim* s, cudaStream_t st, const double* x,
                                const KrylovScalars* ks) {
    if (s->well_model == BO_WELL_MODEL_STANDARD) {
        enqueue_std_well_corr(s, st, x, ks);
        return nullptr;
    }
    if (s->nw > 0) {
        k_wdot<<<s->nw, 128, 0, st>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB, x, d_sop(s), ks);
        count_launch(s, st);
    }
    return d_sop(s);
}

void launch_op(bo_sim* s, const double* x, double* y) {
    enqueue_op<0>(s, s->stream, x, y, nullptr, nullptr);
}

void launch_well_recover(bo_sim* s) {
    if (s->nw == 0) return;
    if (s->well_model == BO_WELL_MODEL_STANDARD) {
        launch_std_wells_recover(s);
        return;
    }
    k_well_recover<<<s->nw, 128, 0, s->stream>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB,
                                                 s->d_xs);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_well_recover");
}

constexpr int MAX_RESTARTS = 8;
constexpr double MIXED_INNER = 1e-4;   // per-cycle reduction target with FP32 sweeps

// Replays the iteration graph until the recurrence stops (or the iteration
// limit is reached), adding the per-kernel event times when timing is on.
static void replay_iterations(bo_sim* s, cudaGraphExec_t g, bool timed, int* prev_it) {
    cudaStream_t st = s->stream;
    // with CPR the whole two-stage apply is one timer (its events 2-3, 10-11)
    const bool cpr = s->precond == BO_PRECOND_CPR;
    const int t_fwd = timer_id(s, cpr ? "cpr_apply" : "ilu_fwd_sweep");
    const int t_bwd = cpr ? -1 : timer_id(s, "ilu_bwd_sweep");
    const int t_spmv = timer_id(s, "spmv_wells"), t_blas = timer_id(s, "blas1_fused");
    const int t_ml = s->ml_on ? timer_id(s, "learned_stage") : -1;
    const int left = s->h_ks->maxit - s->h_ks->it;
    for (int guard = 0; guard < left + 2; guard += s->iters_per_graph) {
        graph_launch(s, g, st);
        BO_CUDA(cudaMemcpyAsync(s->h_ks, s->d_ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
        BO_CUDA(cudaStreamSynchronize(st));
        const KrylovScalars& k = *s->h_ks;
        if (timed) {
            // iterations that did work in this launch (a half step counts as one)
            int ran = k.it - *prev_it;
            for (int q = 0; q < ran && q < s->iters_per_graph; ++q) {
                cudaEvent_t* e = s->iter_events.data() + q * EV_PER_ITER;
                float ms;
                auto add = [&](int id, int a, int b) {
                    if (id < 0) return;
                    BO_CUDA(cudaEventElapsedTime(&ms, e[a], e[b]));
                    s->timer_ms[id] += ms;
                    s->timer_n[id] += 1;
                };
                add(t_fwd, 2, 3);
                add(t_bwd, 4, 5);
                if (t_ml >= 0) add(t_ml, 18, 19);
                add(t_spmv, 6, 7);
                add(t_blas, 0, 1);
                add(t_blas, 8, 9);
                bool second_half = !(q == ran - 1 && k.state == KS_DONE && k.half_exit);
                if (second_half) {
                    add(t_fwd, 10, 11);
                    add(t_bwd, 12, 13);
                    if (t_ml >= 0) add(t_ml, 20, 21);
                    add(t_spmv, 14, 15);
                }
                add(t_blas, 16, 17);
            }
        }
        *prev_it = k.it;
        if (k.state == KS_DONE) break;
    }
}

// Right-hand side of the reduced system into d_b: b = R - sum_w C_w D_w^-1 R_w.
void enqueue_reduced_rhs(bo_sim* s, cudaStream_t st) {
    const int n = s->geo.n, N = 3 * n;
    k_rhs_copy<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_R, s->d_b);
    count_launch(s, st);
    if (s->well_model == BO_WELL_MODEL_STANDARD) {
        enqueue_std_wells_rhs(s, st, s->d_b);
    } else if (s->nw > 0) {
        k_rhs_wells<<<s->nw, 128, 0, st>>>(n, s->d_wells, s->d_con_cell, s->d_wC, s->d_b);
        count_launch(s, st);
    }
}

int run_bicgstab(bo_sim* s, double tol, int maxit, int* its, bool use_ml, bool fp64) {
    if (block_solve_active(s)) return run_block_bicgstab(s, tol, maxit, MAX_RESTARTS, its);
    const int N = 3 * s->geo.n;
    cudaStream_t st = s->stream;
    enqueue_reduced_rhs(s, st);
    k_krylov_init<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_R, s->d_b, s->d_xs, s->d_r, s->d_rh,
                                               s->d_pk, s->d_v, s->d_part);
    count_launch(s, st);
    // the learned stage (like the FP32 sweeps) is not the same linear map at
    // every application: cycles stop at the inner target, the true residual decides
    const bool ml = use_ml && s->ml_on && !fp64;
    const bool fp32 = s->mixed && !fp64;
    k_s_setup<<<1, 256, 0, st>>>(s->d_ks, s->d_part, VEC_GRID, tol, maxit,
                                 (fp32 || ml) ? MIXED_INNER : 0.0);
    count_launch(s, st);
    BO_LAUNCH_CHECK("bicgstab setup");
    if (learn_collecting(s)) BO_CUDA(cudaMemsetAsync(s->d_ml_count, 0, sizeof(int), st));
    s->h_ks->it = 0;
    s->h_ks->maxit = maxit;
    // the timed graph carries the configured stage; a fallback solve runs untimed
    const bool timed = s->timing && ml == s->ml_on && fp32 == s->mixed;
    if (timed) ensure_timed_graph(s);
    cudaGraphExec_t g = timed ? s->g_iter_timed
                        : (s->mixed && !fp32) ? s->g_iter64
                        : (ml ? s->g_iter_ml : s->g_iter);
    const int t_check = timer_id(s, "true_residual");
    int prev_it = 0;
    for (int round = 0;; ++round) {
        replay_iterations(s, g, timed, &prev_it);
        if (s->h_ks->state != KS_DONE || s->h_ks->status == LS_BREAKDOWN) break;
        // FP64 true residual r = b - Op x; accept, restart from it, or give up
        timer_begin(s, t_check);
        enqueue_op<3>(s, st, s->d_xs, s->d_r, s->d_b, nullptr);
        k_s_restart<<<1, 256, 0, st>>>(s->d_ks, s->d_part, VEC_GRID, round < MAX_RESTARTS);
        count_launch(s, st);
        k_restart_vectors<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_r, s->d_rh, s->d_pk, s->d_v,
                                                       s->d_ks);
        count_launch(s, st);
        timer_end(s, t_check);
        BO_LAUNCH_CHECK("true residual");
        BO_CUDA(cudaMemcpyAsync(s->h_ks, s->d_ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
        BO_CUDA(cudaStreamSynchronize(st));
        if (s->h_ks->state != KS_RUN) break;
    }
    timers_flush(s);
    *its = s->h_ks->it;
    s->last_restarts = s->h_ks->restarts;
    s->last_rel_res = s->h_ks->nr0 > 0.0 ? s->h_ks->true_nr / s->h_ks->nr0 : 0.0;
    if (s->h_ks->state != KS_DONE) return LS_NOT_CONVERGED;
    return s->h_ks->status;
}

}  // namespace bo
