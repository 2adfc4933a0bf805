// Block-per-model linear solve: the whole ILU(0)-preconditioned BiCGStab of
// one small model (arXiv 1910.06059, Section 2.3.1, on the well-reduced
// system of Eq. (wellequation)) in ONE launch of ONE CTA.
//
// Why.  A small model's solve on the tiled schedule is a chain of short,
// latency-bound kernels (about fourteen launches per iteration, a host read
// of the recurrence state every few iterations); many small models side by
// side (an ensemble) leave most of the GPU idle in launch gaps.  Here a CTA
// keeps the recurrence scalars in registers, synchronises with __syncthreads
// only, and never returns to the host until the solve has finished, so one
// small model occupies one SM for the length of its solve and the others fill
// the remaining SMs.  On GB300 an FP64 warp instruction holds its SM
// sub-partition for about 64 cycles, so a handful of warps keep the SM's FP64
// pipe busy: one 256-thread CTA per model is enough.
//
// Triangular sweeps inside the CTA.  The factor data are the tiled
// factorisation's (tile order, tiles.cuh): lane (jj, kk) of tile (J, K) owns
// the x-line (j, k) = (TJ J + jj, TK K + kk), warp w owns tiles w, w + 8, ...
// At CTA level L every line handles the cell with i + j + k = L (forward
// ascending, backward descending); its three lower (upper) neighbours were
// handled at level L - 1 (L + 1) by its own line and by the lines (j -+ 1, k)
// and (j, k -+ 1).  Each line leaves its value in a two-level ring in shared
// memory (level parity), read by its neighbours after one __syncthreads.
//
// Everything else follows the tiled schedule's recurrence step by step
// (linsolve.cu: the same scalar tests, breakdown rules, half-step exit, true
// residual check and restarts), with deterministic block reductions in a
// fixed order.  Only the order of the dot-product sums differs, so results
// agree with the tiled schedule to rounding.
//
// Scope: the FP64 ILU(0) preconditioner, reduced standard wells, no
// block-Jacobi cuts; other configurations keep the tiled schedule.
#include <cmath>

#include "tiles.cuh"

namespace bo {

constexpr int BLK_THREADS = 256;
constexpr int BLK_WARPS = BLK_THREADS / 32;
constexpr int BLK_MAXW = 128;   // wells whose (B_w x) / D_w sit in shared memory
constexpr int BLK_MAXT = 128;   // tiles of the ring: 2 x 3 x 32 x T doubles (192 KB at 128)

struct BlockArgs {
    Geom g;
    int NJ, NK, T, NL, NLEV;
    const double* __restrict__ A;   // 63 n, block entries structure-of-arrays
    const double* __restrict__ P;   // tile-order ILU(0) data
    const WellDev* __restrict__ wells;
    int nw;
    const int* __restrict__ con_cell;
    const int* __restrict__ cellcon;    // c -> connection or -1
    const int* __restrict__ con_well;   // connection -> well
    const double* __restrict__ wB;
    const double* __restrict__ wC;
    const double* __restrict__ b;   // right-hand side of the reduced system
    // Krylov vectors (written inside the launch: no read-only loads on them)
    double *x, *r, *rh, *p, *v, *s, *t, *ph, *sh;
    KrylovScalars* ks;
    double tol;
    int maxit, max_restarts;
    const double* ain;   // non-null: apply the preconditioner once, aout = M^-1 ain
    double* aout;
};

// ---------------------------------------------------------------------------
// Deterministic block sums: warp sums by shuffles in a fixed order, then every
// thread adds the warp partials in the same order (the same bits everywhere).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void blk_sum2(double& a, double& b, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(FULL, a, o);
        b += __shfl_down_sync(FULL, b, o);
    }
    if (lane == 0) {
        red[w] = a;
        red[BLK_WARPS + w] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
#pragma unroll
    for (int q = 0; q < BLK_WARPS; ++q) {
        a += red[q];
        b += red[BLK_WARPS + q];
    }
    __syncthreads();
}

__device__ __forceinline__ int blk_line(const BlockArgs& a, int j, int k) {
    return ((j / TJ) + a.NJ * (k / TK)) * 32 + (j % TJ) + TJ * (k % TK);
}

// acc -= B v with B the q0-th 3x3 block of the lane's factor row
__device__ __forceinline__ void blk_sub(double acc[3], const double* Pl, int q0, double v0,
                                        double v1, double v2) {
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
        const double* B = Pl + (size_t)(q0 + 3 * rr) * 32;
        acc[rr] -= B[0] * v0 + B[32] * v1 + B[64] * v2;
    }
}

// z = M^-1 q: forward y = D^-1 q - sum_lower (D^-1 A_ck) y_k into z, then
// backward z = y - sum_upper (D^-1 A_cj) z_j in place.  The caller has
// synchronised after writing q; the last level ends with a __syncthreads.
__device__ void blk_precond(const BlockArgs& a, const double* q, double* z, double* ring) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int jj = lane % TJ, kk = lane / TJ;
    const int n = a.g.n, nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int RL = a.T * 32;   // lines of one ring level and component
    for (int pass = 0; pass < 2; ++pass) {
        const bool fwd = pass == 0;
        for (int step = 0; step < a.NLEV; ++step) {
            const int L = fwd ? step : a.NLEV - 1 - step;
            double* cur = ring + (L & 1) * 3 * RL;
            const double* prev = ring + ((L & 1) ^ 1) * 3 * RL;
            for (int t = warp; t < a.T; t += BLK_WARPS) {
                const int J = t % a.NJ, K = t / a.NJ;
                const int l = L - TJ * J - TK * K;   // tile level of this line set
                if (l < 0 || l >= a.NL) continue;   // the whole tile is idle at L
                const int i = l - jj - kk, j = TJ * J + jj, k = TK * K + kk;
                const int line = t * 32 + lane;
                double y[3] = {0.0, 0.0, 0.0};
                if (i >= 0 && i < nx && j < ny && k < nz) {
                    const int c = i + nx * (j + ny * k);
                    const double* Pl = a.P + ((size_t)(t * a.NL + l) * NPE) * 32 + lane;
                    if (fwd) {
                        const double r0 = q[c], r1 = q[n + c], r2 = q[2 * n + c];
#pragma unroll
                        for (int rr = 0; rr < 3; ++rr)
                            y[rr] = Pl[(size_t)(3 * rr) * 32] * r0 + Pl[(size_t)(3 * rr + 1) * 32] * r1 +
                                    Pl[(size_t)(3 * rr + 2) * 32] * r2;
                        if (i > 0)
                            blk_sub(y, Pl, 9, prev[line], prev[RL + line], prev[2 * RL + line]);
                        if (j > 0) {
                            const int m = blk_line(a, j - 1, k);
                            blk_sub(y, Pl, 18, prev[m], prev[RL + m], prev[2 * RL + m]);
                        }
                        if (k > 0) {
                            const int m = blk_line(a, j, k - 1);
                            blk_sub(y, Pl, 27, prev[m], prev[RL + m], prev[2 * RL + m]);
                        }
                    } else {
                        y[0] = z[c];
                        y[1] = z[n + c];
                        y[2] = z[2 * n + c];
                        if (i + 1 < nx)
                            blk_sub(y, Pl, 36, prev[line], prev[RL + line], prev[2 * RL + line]);
                        if (j + 1 < ny) {
                            const int m = blk_line(a, j + 1, k);
                            blk_sub(y, Pl, 45, prev[m], prev[RL + m], prev[2 * RL + m]);
                        }
                        if (k + 1 < nz) {
                            const int m = blk_line(a, j, k + 1);
                            blk_sub(y, Pl, 54, prev[m], prev[RL + m], prev[2 * RL + m]);
                        }
                    }
                    z[c] = y[0];
                    z[n + c] = y[1];
                    z[2 * n + c] = y[2];
                }
                cur[line] = y[0];
                cur[RL + line] = y[1];
                cur[2 * RL + line] = y[2];
            }
            __syncthreads();
        }
    }
}

// Reduced operator y = A x - sum_w C_w D_w^-1 (B_w x) with fused dot partials
// (per thread; the caller sums them with blk_sum2):
// MODE 1: d0 = (o1, y); 2: d0 = (y, o1), d1 = (y, y); 3: y = o1 - Op x, d0 = (y, y).
template <int MODE>
__device__ void blk_op(const BlockArgs& a, const double* x, double* y, const double* o1,
                       double* sop, double& d0, double& d1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.g.n, nx = a.g.nx, ny = a.g.ny, nz = a.g.nz, plane = nx * ny;
    // per rate well: sop_w = (B_w . x) / D_w
    for (int w = warp; w < a.nw; w += BLK_WARPS) {
        const WellDev& W = a.wells[w];
        double acc = 0.0;
        if (W.ctl == 0)
            for (int q = lane; q < W.ncon; q += 32) {
                const int con = W.off + q, c = a.con_cell[con];
                acc += a.wB[3 * con] * x[c] + a.wB[3 * con + 1] * x[n + c] +
                       a.wB[3 * con + 2] * x[2 * n + c];
            }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o);
        if (lane == 0) sop[w] = (W.ctl == 0) ? acc / W.Dw : 0.0;
    }
    __syncthreads();
    d0 = 0.0;
    d1 = 0.0;
    for (int c = threadIdx.x; c < n; c += BLK_THREADS) {
        const int i = c % nx, j = (c / nx) % ny, k = c / plane;
        const double xv[3] = {x[c], x[n + c], x[2 * n + c]};
        double acc[3];
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
            acc[rr] = a.A[(size_t)(3 * rr) * n + c] * xv[0] + a.A[(size_t)(3 * rr + 1) * n + c] * xv[1] +
                      a.A[(size_t)(3 * rr + 2) * n + c] * xv[2];
        const bool has[6] = {i > 0, i + 1 < nx, j > 0, j + 1 < ny, k > 0, k + 1 < nz};
        const int nbc[6] = {c - 1, c + 1, c - nx, c + nx, c - plane, c + plane};
#pragma unroll
        for (int bb = 1; bb <= 6; ++bb) {
            if (!has[bb - 1]) continue;
            const int qn = nbc[bb - 1];
            const double xn[3] = {x[qn], x[n + qn], x[2 * n + qn]};
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                const double* Ab = a.A + (size_t)(bb * 9 + 3 * rr) * n + c;
                acc[rr] += Ab[0] * xn[0] + Ab[(size_t)n] * xn[1] + Ab[2 * (size_t)n] * xn[2];
            }
        }
        const int con = a.cellcon[c];
        if (con >= 0) {
            const double sw = sop[a.con_well[con]];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) acc[rr] -= a.wC[3 * con + rr] * sw;
        }
#pragma unroll
        for (int rr = 0; rr < 3; ++rr) {
            if (MODE == 3) {
                acc[rr] = o1[rr * n + c] - acc[rr];
                d0 += acc[rr] * acc[rr];
            }
            y[rr * n + c] = acc[rr];
            if (MODE == 1) d0 += o1[rr * n + c] * acc[rr];
            if (MODE == 2) {
                d0 += acc[rr] * o1[rr * n + c];
                d1 += acc[rr] * acc[rr];
            }
        }
    }
}

// The recurrence scalars, one copy per thread (every thread computes the same
// values from the same block sums).
struct BlkState {
    double rho, rho_old, alpha, omega, beta, nr0, last_nr, true_nr, stop;
    int it, state, status, half_exit, restarts;
};

__global__ void __launch_bounds__(BLK_THREADS)
k_block_bicgstab(BlockArgs a) {
    extern __shared__ double ring[];   // 2 levels x 3 components x 32 T lines
    __shared__ double red[2 * BLK_WARPS];
    __shared__ double sop[BLK_MAXW];
    if (a.ain != nullptr) {   // one preconditioner application
        blk_precond(a, a.ain, a.aout, ring);
        return;
    }
    const int N = 3 * a.g.n;
    const int tid = threadIdx.x;
    double d0 = 0.0, d1 = 0.0;
    // b is the reduced right-hand side; x = 0, r = rh = b, p = v = 0
    for (int q = tid; q < N; q += BLK_THREADS) {
        const double bv = a.b[q];
        a.x[q] = 0.0;
        a.r[q] = bv;
        a.rh[q] = bv;
        a.p[q] = 0.0;
        a.v[q] = 0.0;
        d0 += bv * bv;
    }
    blk_sum2(d0, d1, red);
    BlkState k;
    k.it = 0;
    k.rho_old = 1.0;
    k.alpha = 1.0;
    k.omega = 1.0;
    k.beta = 0.0;
    k.nr0 = sqrt(d0);
    k.rho = d0;
    k.last_nr = k.nr0;
    k.status = LS_NOT_CONVERGED;
    k.state = KS_RUN;
    k.half_exit = 0;
    k.restarts = 0;
    k.true_nr = k.nr0;
    k.stop = a.tol * k.nr0;
    if (k.nr0 == 0.0) {
        k.state = KS_DONE;
        k.status = LS_OK;
    }
    auto breakdown = [&]() {
        k.state = KS_DONE;
        k.status = LS_BREAKDOWN;
        k.it -= 1;
    };
    for (int round = 0;; ++round) {
        while (k.state == KS_RUN) {
            if (k.it == a.maxit) {
                k.state = KS_DONE;
                k.status = LS_NOT_CONVERGED;
                break;
            }
            k.it += 1;
            if (k.rho == 0.0 || !isfinite(k.rho)) {
                breakdown();
                break;
            }
            k.beta = (k.rho / k.rho_old) * (k.alpha / k.omega);
            // p = r + beta (p - omega v); ph = M^-1 p; v = Op ph
            for (int q = tid; q < N; q += BLK_THREADS)
                a.p[q] = a.r[q] + k.beta * (a.p[q] - k.omega * a.v[q]);
            __syncthreads();
            blk_precond(a, a.p, a.ph, ring);
            blk_op<1>(a, a.ph, a.v, a.rh, sop, d0, d1);
            blk_sum2(d0, d1, red);
            if (d0 == 0.0 || !isfinite(d0)) {
                breakdown();
                break;
            }
            k.alpha = k.rho / d0;
            // s = r - alpha v; the half step ends the solve when ||s|| is small
            d0 = 0.0;
            d1 = 0.0;
            for (int q = tid; q < N; q += BLK_THREADS) {
                const double sv = a.r[q] - k.alpha * a.v[q];
                a.s[q] = sv;
                d0 += sv * sv;
            }
            blk_sum2(d0, d1, red);
            const double ns = sqrt(d0);
            if (ns <= k.stop) {
                for (int q = tid; q < N; q += BLK_THREADS) a.x[q] += k.alpha * a.ph[q];
                k.half_exit = 1;
                k.last_nr = ns;
                k.state = KS_DONE;
                k.status = LS_OK;
                break;
            }
            // sh = M^-1 s; t = Op sh; omega = (t, s) / (t, t)
            blk_precond(a, a.s, a.sh, ring);
            blk_op<2>(a, a.sh, a.t, a.s, sop, d0, d1);
            blk_sum2(d0, d1, red);
            if (d1 == 0.0 || !isfinite(d1)) {
                breakdown();
                break;
            }
            const double om = d0 / d1;
            if (om == 0.0 || !isfinite(om)) {
                breakdown();
                break;
            }
            k.omega = om;
            // x += alpha ph + omega sh; r = s - omega t
            d0 = 0.0;
            d1 = 0.0;
            for (int q = tid; q < N; q += BLK_THREADS) {
                a.x[q] += k.alpha * a.ph[q] + k.omega * a.sh[q];
                const double rv = a.s[q] - k.omega * a.t[q];
                a.r[q] = rv;
                d0 += rv * rv;
                d1 += a.rh[q] * rv;
            }
            blk_sum2(d0, d1, red);
            const double nr = sqrt(d0);
            k.last_nr = nr;
            if (nr <= k.stop) {
                k.state = KS_DONE;
                k.status = LS_OK;
                break;
            }
            k.rho_old = k.rho;
            k.rho = d1;
        }
        __syncthreads();   // x of the half step
        if (k.status == LS_BREAKDOWN) break;
        // true residual r = b - Op x: accept, restart from it, or give up
        blk_op<3>(a, a.x, a.r, a.b, sop, d0, d1);
        blk_sum2(d0, d1, red);
        const double nr = sqrt(d0);
        k.true_nr = nr;
        if (k.status != LS_OK) break;
        if (nr <= a.tol * k.nr0) break;
        if (round >= a.max_restarts || k.it >= a.maxit || !isfinite(nr)) {
            k.status = LS_NOT_CONVERGED;
            break;
        }
        k.restarts += 1;
        k.stop = a.tol * k.nr0;
        k.rho = d0;
        k.rho_old = 1.0;
        k.alpha = 1.0;
        k.omega = 1.0;
        k.beta = 0.0;
        k.last_nr = nr;
        k.half_exit = 0;
        k.status = LS_NOT_CONVERGED;
        k.state = KS_RUN;
        for (int q = tid; q < N; q += BLK_THREADS) {
            a.rh[q] = a.r[q];
            a.p[q] = 0.0;
            a.v[q] = 0.0;
        }
        __syncthreads();
    }
    if (tid == 0) {
        KrylovScalars* o = a.ks;
        o->rho = k.rho;
        o->rho_old = k.rho_old;
        o->alpha = k.alpha;
        o->omega = k.omega;
        o->beta = k.beta;
        o->nr0 = k.nr0;
        o->tol = a.tol;
        o->last_nr = k.last_nr;
        o->it = k.it;
        o->maxit = a.maxit;
        o->state = k.state;
        o->status = k.status;
        o->half_exit = k.half_exit;
        o->restarts = k.restarts;
        o->true_nr = k.true_nr;
        o->stop = k.stop;
        o->inner = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static BlockArgs block_args(bo_sim* s) {
    BlockArgs a{};
    a.g = s->geo;
    a.NJ = (s->geo.ny + TJ - 1) / TJ;
    a.NK = (s->geo.nz + TK - 1) / TK;
    a.T = a.NJ * a.NK;
    a.NL = s->geo.nx + TJ + TK - 2;
    a.NLEV = s->geo.nx + s->geo.ny + s->geo.nz - 2;
    a.A = s->d_A;
    a.P = s->d_P;
    a.wells = s->d_wells;
    a.nw = s->nw;
    a.con_cell = s->d_con_cell;
    a.cellcon = s->d_cellcon;
    a.con_well = s->d_cellcon + s->geo.n;
    a.wB = s->d_wB;
    a.wC = s->d_wC;
    a.b = s->d_b;
    a.x = s->d_xs;
    a.r = s->d_r;
    a.rh = s->d_rh;
    a.p = s->d_pk;
    a.v = s->d_v;
    a.s = s->d_s;
    a.t = s->d_t;
    a.ph = s->d_ph;
    a.sh = s->d_sh;
    a.ks = s->d_ks;
    return a;
}

bool block_solve_fits(const bo_sim* s) {
    const int T = ((s->geo.ny + TJ - 1) / TJ) * ((s->geo.nz + TK - 1) / TK);
    return T <= BLK_MAXT && s->nw <= BLK_MAXW;
}

bool block_solve_active(const bo_sim* s) {
    return s->solve_schedule == BO_SCHEDULE_BLOCK && block_solve_fits(s) &&
           s->precond == BO_PRECOND_ILU0 && !s->mixed && !s->ml_on && !learn_collecting(s) &&
           s->well_model == BO_WELL_MODEL_REDUCED && s->ysub == 0 && s->zsub == 0;
}

static void launch_block(bo_sim* s, const BlockArgs& a) {
    const size_t smem = (size_t)2 * 3 * 32 * a.T * sizeof(double);
    // Above 48 KB of static + dynamic shared memory a launch needs the opt-in,
    // an attribute of the current context: it is set before every such launch
    // (a new context after a reset needs it again), always to the same value
    // (the ring of BLK_MAXT tiles), so concurrent callers (ensemble workers)
    // cannot lower it under each other.
    if (smem + 2048 > 48 * 1024)
        BO_CUDA(cudaFuncSetAttribute(k_block_bicgstab, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)2 * 3 * 32 * BLK_MAXT * sizeof(double))));
    k_block_bicgstab<<<1, BLK_THREADS, smem, s->stream>>>(a);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_block_bicgstab");
}

int run_block_bicgstab(bo_sim* s, double tol, int maxit, int max_restarts, int* its) {
    enqueue_reduced_rhs(s, s->stream);
    BlockArgs a = block_args(s);
    a.tol = tol;
    a.maxit = maxit;
    a.max_restarts = max_restarts;
    const int t = timer_id(s, "block_bicgstab");
    timer_begin(s, t);
    launch_block(s, a);
    timer_end(s, t);
    BO_CUDA(cudaMemcpyAsync(s->h_ks, s->d_ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    timers_flush(s);
    const KrylovScalars& k = *s->h_ks;
    *its = k.it;
    s->last_restarts = k.restarts;
    s->last_rel_res = k.nr0 > 0.0 ? k.true_nr / k.nr0 : 0.0;
    if (k.state != KS_DONE) return LS_NOT_CONVERGED;
    return k.status;
}

void launch_block_precond(bo_sim* s, const double* r, double* z) {
    BlockArgs a = block_args(s);
    a.ain = r;
    a.aout = z;
    launch_block(s, a);
}

}  // namespace bo
