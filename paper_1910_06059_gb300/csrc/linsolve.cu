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

// ---------------------------------------------------------------------------
// Wavefront levels: cells sorted by L = i + j + k, then k, then j.
// ---------------------------------------------------------------------------
void build_levels(bo_sim* s) {
    const Geom& g = s->geo;
    s->nlev = g.nx + g.ny + g.nz - 2;
    std::vector<int> cnt(s->nlev + 1, 0);
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) cnt[i + j + k + 1]++;
    for (int L = 0; L < s->nlev; ++L) cnt[L + 1] += cnt[L];
    s->lvl_ptr = cnt;
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    std::vector<int> perm(g.n), iperm(g.n);
    for (int L = 0; L < s->nlev; ++L) {
        // enumerate (k, j) ascending with i = L - j - k in range
        for (int k = 0; k < g.nz; ++k)
            for (int j = 0; j < g.ny; ++j) {
                int i = L - j - k;
                if (i < 0 || i >= g.nx) continue;
                int c = i + g.nx * (j + g.ny * k);
                perm[pos[L]] = c;
                iperm[c] = pos[L];
                pos[L]++;
            }
    }
    BO_CUDA(cudaMemcpy(s->d_perm_lvl, perm.data(), sizeof(int) * g.n, cudaMemcpyHostToDevice));
    BO_CUDA(cudaMemcpy(s->d_perm_lvl + g.n, iperm.data(), sizeof(int) * g.n,
                       cudaMemcpyHostToDevice));
}

// ---------------------------------------------------------------------------
// 3x3 block helpers (row-major, e = 3r + s)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ld_blk_nat(const double* __restrict__ A, int b, int n, int c,
                                           double m[9]) {
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = A[(size_t)(b * 9 + e) * n + c];
}
__device__ __forceinline__ void mm3(const double a[9], const double b[9], double c[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s)
            c[3 * r + s] = a[3 * r] * b[s] + a[3 * r + 1] * b[3 + s] + a[3 * r + 2] * b[6 + s];
}
// Inverse by the adjugate.
__device__ __forceinline__ void inv3(const double a[9], double o[9]) {
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    double id = 1.0 / det;
    o[0] = c00 * id;
    o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
    o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    o[3] = c01 * id;
    o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
    o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    o[6] = c02 * id;
    o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
    o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
}

__device__ __forceinline__ void cell_ijk(const Geom& g, int c, int& i, int& j, int& k) {
    i = c % g.nx;
    j = (c / g.nx) % g.ny;
    k = c / (g.nx * g.ny);
}

__device__ __forceinline__ bool ks_skip(const KrylovScalars* ks) {
    return ks != nullptr && ks->state != KS_RUN;
}

// ---------------------------------------------------------------------------
// Dataflow sweeps.  One persistent, co-resident grid walks the cells in
// wavefront order (each thread takes cells m = t, t + T, t + 2T, ... of the
// level-sorted order, T threads in all), so every cell a thread waits for
// sits earlier in that order and is owned by a running thread: the wait
// always ends.  A cell waits only for its three neighbours on the previous
// level, through per-cell ready flags: the producer stores its result and
// then releases flag[c] = seq (st.release.gpu); the consumer acquires the
// flag (ld.acquire.gpu) and reads the neighbour's values from L2
// (ld.global.cg), never from a possibly stale L1 line.  seq is the sweep
// number: read from sync[0] at kernel entry, advanced by the last block to
// finish, so flags never need clearing.  Every wait is bounded; on timeout
// the kernel records sync[2] = 1 and returns instead of hanging.
// ---------------------------------------------------------------------------
struct SweepArgs {
    Geom g;
    const int* perm;   // m -> c
    const int* iperm;  // c -> m
    int* flag;         // per cell (natural index)
    int* sync;         // [0] sweep epoch, [1] finished blocks, [2] timeout
};

constexpr int SWP_BS = 128;
constexpr long long SPIN_LIMIT = 1LL << 24;

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *f == seq.  Returns false (and records the timeout) when the
// bounded wait runs out or another thread has already timed out.
__device__ __noinline__ bool wait_ready(const int* f, int seq, int* sync) {
    if (ld_acquire_gpu(f) == seq) return true;
    for (long long s = 1; s <= SPIN_LIMIT; ++s) {
        __nanosleep(64);
        if (ld_acquire_gpu(f) == seq) return true;
        if ((s & 1023) == 0 && ld_acquire_gpu(sync + 2) != 0) return false;
    }
    atomicExch(sync + 2, 1);
    return false;
}

__device__ __forceinline__ int sweep_begin(const int* sync) { return ld_acquire_gpu(sync) + 1; }

__device__ __forceinline__ void sweep_end(int* sync) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int done = atomicAdd(sync + 1, 1);
        if (done == (int)gridDim.x - 1) {  // last block out: reset, advance the epoch
            sync[1] = 0;
            __threadfence();
            atomicAdd(sync, 1);
        }
    }
}

__device__ __forceinline__ void ldcg3(const double* v, int n, int c, double out[3]) {
    out[0] = __ldcg(v + c);
    out[1] = __ldcg(v + n + c);
    out[2] = __ldcg(v + 2 * n + c);
}

// ---------------------------------------------------------------------------
// a7: ILU(0) factorisation.  A cell needs the scaled upper blocks
// D_k^-1 A_kc of its lower neighbours; it publishes its own scaled upper
// blocks first (the only data others wait for), then D^-1 and the scaled
// lower blocks.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SWP_BS)
k_factor_sweep(SweepArgs a, const double* __restrict__ A, double* __restrict__ P,
               int* __restrict__ bad) {
    const int seq = sweep_begin(a.sync);
    const int n = a.g.n;
    const int lowb[3] = {NB_MX, NB_MY, NB_MZ};
    const int uppb[3] = {NB_PX, NB_PY, NB_PZ};
    bool alive = true;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; alive && m < n; m += gridDim.x * blockDim.x) {
        int c = a.perm[m];
        int i, j, k;
        cell_ijk(a.g, c, i, j, k);
        const bool has_lo[3] = {i > 0, j > 0, k > 0};
        const bool has_up[3] = {i + 1 < a.g.nx, j + 1 < a.g.ny, k + 1 < a.g.nz};
        const int lo_nb[3] = {c - 1, c - a.g.nx, c - a.g.nx * a.g.ny};
        double D[9];
        ld_blk_nat(A, NB_DIAG, n, c, D);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!has_lo[d]) continue;
            double Ack[9], Ukc[9], prod[9];
            ld_blk_nat(A, lowb[d], n, c, Ack);
            int nb = lo_nb[d];
            if (!wait_ready(a.flag + nb, seq, a.sync)) {
                alive = false;
                break;
            }
            int mk = a.iperm[nb];
#pragma unroll
            for (int e = 0; e < 9; ++e) Ukc[e] = __ldcg(P + (size_t)((4 + d) * 9 + e) * n + mk);
            mm3(Ack, Ukc, prod);
#pragma unroll
            for (int e = 0; e < 9; ++e) D[e] -= prod[e];
        }
        if (!alive) break;
        double Di[9];
        inv3(D, Di);
        double blk[9], sc[9];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (has_up[d]) {
                ld_blk_nat(A, uppb[d], n, c, blk);
                mm3(Di, blk, sc);
            } else {
#pragma unroll
                for (int e = 0; e < 9; ++e) sc[e] = 0.0;
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) P[(size_t)((4 + d) * 9 + e) * n + m] = sc[e];
        }
        st_release_gpu(a.flag + c, seq);
        bool finite = true;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            finite = finite && isfinite(Di[e]);
            P[(size_t)e * n + m] = Di[e];
        }
        if (!finite) atomicAdd(bad, 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (has_lo[d]) {
                ld_blk_nat(A, lowb[d], n, c, blk);
                mm3(Di, blk, sc);
            } else {
#pragma unroll
                for (int e = 0; e < 9; ++e) sc[e] = 0.0;
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) P[(size_t)((1 + d) * 9 + e) * n + m] = sc[e];
        }
    }
    sweep_end(a.sync);
}

// ---------------------------------------------------------------------------
// a8: forward sweep y = (L_A + D)^-1 r, i.e. y_c = D_c^-1 r_c - sum_lower
// (D_c^-1 A_ck) y_k.  The matrix blocks and D^-1 r are loaded and formed
// before the wait; only the three neighbour products follow it.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SWP_BS)
k_fwd_sweep(SweepArgs a, const double* __restrict__ P, const double* __restrict__ r,
            double* __restrict__ y, const KrylovScalars* __restrict__ ks) {
    if (ks_skip(ks)) return;
    const int seq = sweep_begin(a.sync);
    const int n = a.g.n;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        int c = a.perm[m];
        int i, j, k;
        cell_ijk(a.g, c, i, j, k);
        double rv[3] = {r[c], r[n + c], r[2 * n + c]};
        double acc[3];
#pragma unroll
        for (int row = 0; row < 3; ++row)
            acc[row] = P[(size_t)(3 * row) * n + m] * rv[0] + P[(size_t)(3 * row + 1) * n + m] * rv[1] +
                       P[(size_t)(3 * row + 2) * n + m] * rv[2];
        const bool has_lo[3] = {i > 0, j > 0, k > 0};
        const int lo_nb[3] = {c - 1, c - a.g.nx, c - a.g.nx * a.g.ny};
        double Lb[3][9];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int e = 0; e < 9; ++e)
                Lb[d][e] = has_lo[d] ? P[(size_t)((1 + d) * 9 + e) * n + m] : 0.0;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!has_lo[d]) continue;
            int q = lo_nb[d];
            ok = ok && wait_ready(a.flag + q, seq, a.sync);
            double yv[3];
            ldcg3(y, n, q, yv);
#pragma unroll
            for (int row = 0; row < 3; ++row)
                acc[row] -= Lb[d][3 * row] * yv[0] + Lb[d][3 * row + 1] * yv[1] + Lb[d][3 * row + 2] * yv[2];
        }
        if (!ok) break;
        y[c] = acc[0];
        y[n + c] = acc[1];
        y[2 * n + c] = acc[2];
        st_release_gpu(a.flag + c, seq);
    }
    sweep_end(a.sync);
}

// backward sweep in place: z_c = y_c - sum_upper (D_c^-1 A_cj) z_j
__global__ void __launch_bounds__(SWP_BS)
k_bwd_sweep(SweepArgs a, const double* __restrict__ P, double* __restrict__ z,
            const KrylovScalars* __restrict__ ks) {
    if (ks_skip(ks)) return;
    const int seq = sweep_begin(a.sync);
    const int n = a.g.n;
    const int T = gridDim.x * blockDim.x;
    // walk the wavefront order backwards: thread t takes m = n-1-t, n-1-t-T, ...
    for (int mm = blockIdx.x * blockDim.x + threadIdx.x; mm < n; mm += T) {
        int m = n - 1 - mm;
        int c = a.perm[m];
        int i, j, k;
        cell_ijk(a.g, c, i, j, k);
        double acc[3];
        ldcg3(z, n, c, acc);
        const bool has_up[3] = {i + 1 < a.g.nx, j + 1 < a.g.ny, k + 1 < a.g.nz};
        const int up_nb[3] = {c + 1, c + a.g.nx, c + a.g.nx * a.g.ny};
        double Ub[3][9];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int e = 0; e < 9; ++e)
                Ub[d][e] = has_up[d] ? P[(size_t)((4 + d) * 9 + e) * n + m] : 0.0;
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!has_up[d]) continue;
            int q = up_nb[d];
            ok = ok && wait_ready(a.flag + q, seq, a.sync);
            double zv[3];
            ldcg3(z, n, q, zv);
#pragma unroll
            for (int row = 0; row < 3; ++row)
                acc[row] -= Ub[d][3 * row] * zv[0] + Ub[d][3 * row + 1] * zv[1] + Ub[d][3 * row + 2] * zv[2];
        }
        if (!ok) break;
        z[c] = acc[0];
        z[n + c] = acc[1];
        z[2 * n + c] = acc[2];
        st_release_gpu(a.flag + c, seq);
    }
    sweep_end(a.sync);
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

// mode 0: no dots; 1: part0 = (rh, y); 2: part0 = (y, s), part1 = (y, y)
template <int MODE>
__global__ void __launch_bounds__(VEC_BS)
k_spmv(Geom g, const double* __restrict__ A, const double* __restrict__ x,
       double* __restrict__ y, const int* __restrict__ cellcon,
       const int* __restrict__ con_well, const double* __restrict__ wC,
       const double* __restrict__ sop, const double* __restrict__ o1,
       double* __restrict__ part, const KrylovScalars* __restrict__ ks) {
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
            double sw = sop[con_well[con]];
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r] -= wC[3 * con + r] * sw;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
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
                          int maxit) {
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
    if (ns <= ks->tol * ks->nr0) {
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
    if (nr <= ks->tol * ks->nr0) {
        ks->state = KS_DONE;
        ks->status = LS_OK;
        return;
    }
    ks->rho_old = ks->rho;
    ks->rho = rhr;
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

static SweepArgs sweep_args(bo_sim* s) {
    SweepArgs a;
    a.g = s->geo;
    a.perm = s->d_perm_lvl;
    a.iperm = s->d_perm_lvl + s->geo.n;
    a.flag = s->d_flag_sweep;
    a.sync = s->d_sweep_sync;
    return a;
}

static int* factor_bad(bo_sim* s) { return reinterpret_cast<int*>(&s->d_ns->pad); }

// Co-resident grid for the dataflow sweeps: a cooperative launch, which fails
// with an error instead of starting a grid that cannot be resident at once.
template <class... Args>
static void launch_coop(bo_sim* s, cudaStream_t st, void (*kern)(Args...), Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(s->sweep_grid);
    cfg.blockDim = dim3(SWP_BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BO_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

void setup_sweeps(bo_sim* s) {
    int dev, sms, per_sm = 0;
    BO_CUDA(cudaGetDevice(&dev));
    BO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int lim = 1 << 30;
    for (const void* k : {(const void*)k_factor_sweep, (const void*)k_fwd_sweep, (const void*)k_bwd_sweep}) {
        BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, SWP_BS, 0));
        lim = std::min(lim, per_sm);
    }
    int want = std::max(1, std::min(lim, s->sweep_blocks_per_sm));
    s->sweep_grid = want * sms;
    BO_CUDA(cudaMemset(s->d_flag_sweep, 0, sizeof(int) * (size_t)s->geo.n));
    BO_CUDA(cudaMemset(s->d_sweep_sync, 0, sizeof(int) * 4));
}

static void enqueue_factor(bo_sim* s, cudaStream_t st) {
    launch_coop(s, st, k_factor_sweep, sweep_args(s), (const double*)s->d_A, s->d_P, factor_bad(s));
}

static void enqueue_fwd(bo_sim* s, cudaStream_t st, const double* r, double* y,
                        const KrylovScalars* ks) {
    launch_coop(s, st, k_fwd_sweep, sweep_args(s), (const double*)s->d_P, r, y, ks);
}

static void enqueue_bwd(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks) {
    launch_coop(s, st, k_bwd_sweep, sweep_args(s), (const double*)s->d_P, z, ks);
}

static void enqueue_precond(bo_sim* s, cudaStream_t st, const double* r, double* z,
                            const KrylovScalars* ks) {
    enqueue_fwd(s, st, r, z, ks);
    enqueue_bwd(s, st, z, ks);
}

static double* d_sop(bo_sim* s) { return s->d_part + 8 * VEC_GRID; }

template <int MODE>
static void enqueue_op(bo_sim* s, cudaStream_t st, const double* x, double* y, const double* o1,
                       const KrylovScalars* ks) {
    if (s->nw > 0) {
        k_wdot<<<s->nw, 128, 0, st>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB, x, d_sop(s),
                                      ks);
    }
    k_spmv<MODE><<<VEC_GRID, VEC_BS, 0, st>>>(s->geo, s->d_A, x, y, s->d_cellcon,
                                              s->d_cellcon + s->geo.n, s->d_wC, d_sop(s), o1,
                                              s->d_part, ks);
    BO_LAUNCH_CHECK("k_spmv");
}

// Timers: event pairs recorded on the launching stream (graph nodes when captured).
int timer_id(bo_sim* s, const char* name) {
    for (int q = 0; q < s->ntimers; ++q)
        if (s->timer_name[q] == name) return q;
    if (s->ntimers >= MAX_TIMERS) return -1;
    s->timer_name[s->ntimers] = name;
    return s->ntimers++;
}

struct EagerTimer {
    cudaEvent_t a, b;
    int id;
};
static std::vector<EagerTimer> g_pending;  // per process; flushed after each sync

void timer_begin(bo_sim* s, int id) {
    if (!s->timing || id < 0) return;
    EagerTimer t{};
    t.id = id;
    BO_CUDA(cudaEventCreate(&t.a));
    BO_CUDA(cudaEventCreate(&t.b));
    BO_CUDA(cudaEventRecord(t.a, s->stream));
    g_pending.push_back(t);
}
void timer_end(bo_sim* s, int id) {
    if (!s->timing || id < 0) return;
    for (auto it = g_pending.rbegin(); it != g_pending.rend(); ++it)
        if (it->id == id) {
            BO_CUDA(cudaEventRecord(it->b, s->stream));
            return;
        }
}
void timers_flush(bo_sim* s) {
    if (g_pending.empty()) return;
    BO_CUDA(cudaStreamSynchronize(s->stream));
    for (auto& t : g_pending) {
        float ms = 0.f;
        BO_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
        s->timer_ms[t.id] += ms;
        s->timer_n[t.id] += 1;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_pending.clear();
}

// One BiCGStab iteration enqueued on st (captured into a graph).
// ev (may be null): 2 events per timed op, ops: 0 fwd+bwd sweeps (2 applies),
// recorded as [fwd1, bwd1, spmv1, fwd2, bwd2, spmv2, blas] pairs.
enum { TI_FWD = 0, TI_BWD = 1, TI_SPMV = 2, TI_BLAS = 3, TI_N = 4 };

static void enqueue_iteration(bo_sim* s, cudaStream_t st, cudaEvent_t* ev) {
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
    rec(0);
    k_p_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_r, s->d_pk, s->d_v, ks);
    rec(1);
    // ph = M^-1 p
    rec(2);
    enqueue_fwd(s, st, s->d_pk, s->d_ph, ks);
    rec(3);
    rec(4);
    enqueue_bwd(s, st, s->d_ph, ks);
    rec(5);
    rec(6);
    enqueue_op<1>(s, st, s->d_ph, s->d_v, s->d_rh, ks);
    rec(7);
    k_s2<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    rec(8);
    k_s_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_r, s->d_v, s->d_s, part, ks);
    rec(9);
    k_s3<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    rec(10);
    enqueue_fwd(s, st, s->d_s, s->d_sh, ks);
    rec(11);
    rec(12);
    enqueue_bwd(s, st, s->d_sh, ks);
    rec(13);
    rec(14);
    enqueue_op<2>(s, st, s->d_sh, s->d_t, s->d_s, ks);
    rec(15);
    k_s4<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    rec(16);
    k_xr_update<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_xs, s->d_ph, s->d_sh, s->d_s, s->d_t,
                                             s->d_r, s->d_rh, part, ks);
    rec(17);
    k_s5<<<1, 256, 0, st>>>(ks, part, VEC_GRID);
    BO_LAUNCH_CHECK("bicgstab iteration");
}

static constexpr int EV_PER_ITER = 18;

static cudaGraphExec_t capture(bo_sim* s, int iters, cudaEvent_t* ev) {
    cudaStream_t cs;
    BO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    BO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < iters; ++q) enqueue_iteration(s, cs, ev ? ev + q * EV_PER_ITER : nullptr);
    BO_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec;
    BO_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    BO_CUDA(cudaGraphDestroy(graph));
    BO_CUDA(cudaStreamDestroy(cs));
    return exec;
}

static cudaGraphExec_t capture_factor(bo_sim* s) {
    cudaStream_t cs;
    BO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    BO_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    enqueue_factor(s, cs);
    BO_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec;
    BO_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    BO_CUDA(cudaGraphDestroy(graph));
    BO_CUDA(cudaStreamDestroy(cs));
    return exec;
}

void build_graphs(bo_sim* s) {
    destroy_graphs(s);
    s->g_factor = capture_factor(s);
    s->g_iter = capture(s, s->iters_per_graph, nullptr);
}

void destroy_graphs(bo_sim* s) {
    if (s->g_iter) cudaGraphExecDestroy(s->g_iter);
    if (s->g_factor) cudaGraphExecDestroy(s->g_factor);
    if (s->g_iter_timed) cudaGraphExecDestroy(s->g_iter_timed);
    s->g_iter = s->g_factor = s->g_iter_timed = nullptr;
    for (cudaEvent_t e : s->iter_events) cudaEventDestroy(e);
    s->iter_events.clear();
}

static void ensure_timed_graph(bo_sim* s) {
    if (s->g_iter_timed) return;
    s->iter_events.resize((size_t)EV_PER_ITER * s->iters_per_graph);
    for (auto& e : s->iter_events) BO_CUDA(cudaEventCreate(&e));
    s->g_iter_timed = capture(s, s->iters_per_graph, s->iter_events.data());
}

int sweep_timeout(bo_sim* s) {
    int v = 0;
    BO_CUDA(cudaMemcpyAsync(&v, s->d_sweep_sync + 2, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    return v;
}

void launch_factor(bo_sim* s) {
    int t = timer_id(s, "ilu_factor");
    BO_CUDA(cudaMemsetAsync(factor_bad(s), 0, sizeof(int), s->stream));
    timer_begin(s, t);
    BO_CUDA(cudaGraphLaunch(s->g_factor, s->stream));
    timer_end(s, t);
}

void launch_precond(bo_sim* s, const double* r, double* z) { enqueue_precond(s, s->stream, r, z, nullptr); }

void launch_op(bo_sim* s, const double* x, double* y) {
    enqueue_op<0>(s, s->stream, x, y, nullptr, nullptr);
}

void launch_well_recover(bo_sim* s) {
    if (s->nw == 0) return;
    k_well_recover<<<s->nw, 128, 0, s->stream>>>(s->geo.n, s->d_wells, s->d_con_cell, s->d_wB,
                                                 s->d_xs);
    BO_LAUNCH_CHECK("k_well_recover");
}

int run_bicgstab(bo_sim* s, double tol, int maxit, int* its) {
    const int n = s->geo.n, N = 3 * n;
    cudaStream_t st = s->stream;
    // right-hand side of the reduced system
    k_rhs_copy<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_R, s->d_b);
    if (s->nw > 0) k_rhs_wells<<<s->nw, 128, 0, st>>>(n, s->d_wells, s->d_con_cell, s->d_wC, s->d_b);
    k_krylov_init<<<VEC_GRID, VEC_BS, 0, st>>>(N, s->d_R, s->d_b, s->d_xs, s->d_r, s->d_rh,
                                               s->d_pk, s->d_v, s->d_part);
    k_s_setup<<<1, 256, 0, st>>>(s->d_ks, s->d_part, VEC_GRID, tol, maxit);
    BO_LAUNCH_CHECK("bicgstab setup");
    const bool timed = s->timing;
    if (timed) ensure_timed_graph(s);
    cudaGraphExec_t g = timed ? s->g_iter_timed : s->g_iter;
    int prev_it = 0;
    int t_fwd = timer_id(s, "ilu_fwd_sweep"), t_bwd = timer_id(s, "ilu_bwd_sweep");
    int t_spmv = timer_id(s, "spmv_wells"), t_blas = timer_id(s, "blas1_fused");
    for (int guard = 0; guard < maxit + 2; guard += s->iters_per_graph) {
        BO_CUDA(cudaGraphLaunch(g, st));
        BO_CUDA(cudaMemcpyAsync(s->h_ks, s->d_ks, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
        BO_CUDA(cudaStreamSynchronize(st));
        const KrylovScalars& k = *s->h_ks;
        if (timed) {
            // iterations that did work in this launch (a half step counts as one)
            int ran = k.it - prev_it;
            for (int q = 0; q < ran && q < s->iters_per_graph; ++q) {
                cudaEvent_t* e = s->iter_events.data() + q * EV_PER_ITER;
                float ms;
                auto add = [&](int id, int a, int b) {
                    BO_CUDA(cudaEventElapsedTime(&ms, e[a], e[b]));
                    s->timer_ms[id] += ms;
                    s->timer_n[id] += 1;
                };
                add(t_fwd, 2, 3);
                add(t_bwd, 4, 5);
                add(t_spmv, 6, 7);
                add(t_blas, 0, 1);
                add(t_blas, 8, 9);
                bool second_half = !(q == ran - 1 && k.state == KS_DONE && k.half_exit);
                if (second_half) {
                    add(t_fwd, 10, 11);
                    add(t_bwd, 12, 13);
                    add(t_spmv, 14, 15);
                }
                add(t_blas, 16, 17);
            }
        }
        prev_it = k.it;
        if (k.state == KS_DONE) break;
    }
    timers_flush(s);
    *its = s->h_ks->it;
    if (s->h_ks->state != KS_DONE) return LS_NOT_CONVERGED;
    return s->h_ks->status;
}

}  // namespace bo
