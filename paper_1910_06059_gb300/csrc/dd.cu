// Domain decomposition of the linear solve (arXiv 1910.06059, Section 2.5:
// each process owns the rows of its subdomain, exchanges a ghost layer
// before every operator product, applies ILU(0) to its own block and joins
// the inner products by an all-reduce), emulated as K subdomains on one GPU.
//
// The subdomains are the block-Jacobi slabs of ysub cell rows in y.  Every
// vector of the Krylov method lives in a subdomain-local layout: subdomain k
// holds its rows j0..j1-1 plus one ghost row on each side that has a
// neighbour, concatenated over k (positions off_k + i + nx (j - j0 + gl +
// nyl kz)); the Jacobian rows are copied into the same per-subdomain order.
// Kernels run with blockIdx.y = subdomain:
//   k_dd_halo     the ghost rows from the neighbours' boundary rows (a device
//                 copy in place of the message exchange)
//   k_dd_spmv     the subdomain's rows of the well-reduced operator on its
//                 ghosted vector, with per-subdomain partial inner products
//   k_dd_*        vector updates with per-subdomain partials
//   k_dd_allreduce  each subdomain's sum of its blocks' partials, then the
//                 sum over the subdomains in subdomain order
// The preconditioner is each subdomain's ILU(0) block: the FP64 tiled sweeps
// with the slab cuts, which couple no two subdomains, applied to the
// subdomains' rows gathered into the natural layout.  The BiCGStab iteration
// is the one of the single-domain solver (right preconditioning, early exit
// on ||s||, the true-residual acceptance with restarts); its scalars come
// back to the host once per half-iteration.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace bo {

constexpr int DD_BS = 256;
constexpr int DD_GX = 64;        // blocks per subdomain (grid-stride)
constexpr int DD_MAXK = 1024;

struct DdPart {
    int j0, j1, gl, gh, nyl, off, ioff, nint;
};

struct DdData {
    int K = 0, ysub = 0;
    long long Ntot = 0, Nint = 0;     // ghosted positions, interior cells
    std::vector<DdPart> h_parts;
    DdPart* parts = nullptr;
    double* A = nullptr;              // [63][Nint] rows in subdomain order
    // Krylov vectors in the ghosted layout, [3][Ntot] each
    double *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
           *t = nullptr, *ph = nullptr, *sh = nullptr, *b = nullptr;
    double* gsc = nullptr;            // [3][n] natural-layout scratch for the sweeps
    double* gz = nullptr;             // [3][n]
    double* part = nullptr;           // [2][K][DD_GX] partials
    double* red = nullptr;            // [2] all-reduced sums
    double* sop = nullptr;            // [nw] per-well (B . x) / D
};

struct DdGeom {
    int nx, ny, nz, n, K;
    long long Ntot, Nint;
};

__device__ __forceinline__ void dd_cell(const DdGeom& G, const DdPart& P, int ii, int& i, int& j,
                                        int& kz) {
    const int rows = P.j1 - P.j0;
    i = ii % G.nx;
    j = P.j0 + (ii / G.nx) % rows;
    kz = ii / (G.nx * rows);
}
__device__ __forceinline__ long long dd_pos(const DdGeom& G, const DdPart& P, int i, int j, int kz) {
    return P.off + i + (long long)G.nx * (j - P.j0 + P.gl + (long long)P.nyl * kz);
}

// fixed-order block partials of K values into part[q][k][bx]
template <int Q>
__device__ void dd_partials(double (&v)[Q], double* __restrict__ part, int K) {
    __shared__ double sh[Q][DD_BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < Q) {
        double x = 0.0;
        for (int w = 0; w < DD_BS / 32; ++w) x += sh[threadIdx.x][w];
        part[((size_t)threadIdx.x * K + blockIdx.y) * gridDim.x + blockIdx.x] = x;
    }
}

// natural [3][n] -> subdomain layout (interior positions); ghosts untouched
__global__ void __launch_bounds__(DD_BS)
k_dd_in(DdGeom G, const DdPart* __restrict__ parts, const double* __restrict__ g,
        double* __restrict__ d) {
    const DdPart P = parts[blockIdx.y];
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < P.nint; ii += gridDim.x * blockDim.x) {
        int i, j, kz;
        dd_cell(G, P, ii, i, j, kz);
        const int c = i + G.nx * (j + G.ny * kz);
        const long long q = dd_pos(G, P, i, j, kz);
#pragma unroll
        for (int e = 0; e < 3; ++e) d[e * G.Ntot + q] = g[(size_t)e * G.n + c];
    }
}
// subdomain layout -> natural [3][n]
__global__ void __launch_bounds__(DD_BS)
k_dd_out(DdGeom G, const DdPart* __restrict__ parts, const double* __restrict__ d,
         double* __restrict__ g) {
    const DdPart P = parts[blockIdx.y];
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < P.nint; ii += gridDim.x * blockDim.x) {
        int i, j, kz;
        dd_cell(G, P, ii, i, j, kz);
        const int c = i + G.nx * (j + G.ny * kz);
        const long long q = dd_pos(G, P, i, j, kz);
#pragma unroll
        for (int e = 0; e < 3; ++e) g[(size_t)e * G.n + c] = d[e * G.Ntot + q];
    }
}
// the Jacobian rows of each subdomain, [63][Nint] in subdomain order
__global__ void __launch_bounds__(DD_BS)
k_dd_rows(DdGeom G, const DdPart* __restrict__ parts, const double* __restrict__ A,
          double* __restrict__ Ad) {
    const DdPart P = parts[blockIdx.y];
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < P.nint; ii += gridDim.x * blockDim.x) {
        int i, j, kz;
        dd_cell(G, P, ii, i, j, kz);
        const int c = i + G.nx * (j + G.ny * kz);
        for (int e = 0; e < 63; ++e) Ad[(size_t)e * G.Nint + P.ioff + ii] = A[(size_t)e * G.n + c];
    }
}

// ghost rows <- the neighbours' boundary rows (one thread per (i, kz, comp))
__global__ void __launch_bounds__(DD_BS)
k_dd_halo(DdGeom G, const DdPart* __restrict__ parts, double* __restrict__ x,
          const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const int k = blockIdx.y;
    const DdPart P = parts[k];
    const int m = G.nx * G.nz;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 3 * m; q += gridDim.x * blockDim.x) {
        const int e = q / m, i = q % G.nx, kz = (q % m) / G.nx;
        if (P.gl) {   // row j0 - 1 is the last row of subdomain k - 1
            const DdPart L = parts[k - 1];
            x[e * G.Ntot + dd_pos(G, P, i, P.j0 - 1, kz)] = x[e * G.Ntot + dd_pos(G, L, i, P.j0 - 1, kz)];
        }
        if (P.gh) {   // row j1 is the first row of subdomain k + 1
            const DdPart U = parts[k + 1];
            x[e * G.Ntot + dd_pos(G, P, i, P.j1, kz)] = x[e * G.Ntot + dd_pos(G, U, i, P.j1, kz)];
        }
    }
}

// per rate well sop_w = (B_w . x) / D_w with x in the subdomain layout (the
// connection cells are rows of the subdomain holding the well's column)
__global__ void k_dd_wdot(DdGeom G, const DdPart* __restrict__ parts, int ysub,
                          const WellDev* __restrict__ wells, const int* __restrict__ con_cell,
                          const double* __restrict__ wB, const double* __restrict__ x,
                          double* __restrict__ sop, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const WellDev& W = wells[blockIdx.x];
    double acc = 0.0;
    if (W.ctl == 0)
        for (int q = threadIdx.x; q < W.ncon; q += blockDim.x) {
            const int con = W.off + q, c = con_cell[con];
            const int i = c % G.nx, j = (c / G.nx) % G.ny, kz = c / (G.nx * G.ny);
            const long long p = dd_pos(G, parts[j / ysub], i, j, kz);
            acc += wB[3 * con] * x[p] + wB[3 * con + 1] * x[G.Ntot + p] + wB[3 * con + 2] * x[2 * G.Ntot + p];
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

// y = S x on each subdomain's rows; MODE 1: part0 = (rh, y); 2: part0 = (y, s),
// part1 = (y, y); 3: y = o1 - S x, part0 = (y, y)
template <int MODE>
__global__ void __launch_bounds__(DD_BS)
k_dd_spmv(DdGeom G, const DdPart* __restrict__ parts, const double* __restrict__ Ad,
          const double* __restrict__ x, double* __restrict__ y, const int* __restrict__ cellcon,
          const int* __restrict__ con_well, const double* __restrict__ wC,
          const double* __restrict__ sop, const double* __restrict__ o1,
          double* __restrict__ part, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const DdPart P = parts[blockIdx.y];
    double d[2] = {0.0, 0.0};
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < P.nint; ii += gridDim.x * blockDim.x) {
        int i, j, kz;
        dd_cell(G, P, ii, i, j, kz);
        const long long p0 = dd_pos(G, P, i, j, kz);
        const long long row = P.ioff + ii;
        const long long pl = (long long)G.nx * P.nyl;
        const bool has[7] = {true, i > 0, i + 1 < G.nx, j > 0, j + 1 < G.ny, kz > 0, kz + 1 < G.nz};
        const long long nb[7] = {p0, p0 - 1, p0 + 1, p0 - G.nx, p0 + G.nx, p0 - pl, p0 + pl};
        double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            if (!has[b]) continue;
            const double xn[3] = {x[nb[b]], x[G.Ntot + nb[b]], x[2 * G.Ntot + nb[b]]};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double* Ab = Ad + (size_t)(b * 9 + 3 * r) * G.Nint + row;
                acc[r] += Ab[0] * xn[0] + Ab[(size_t)G.Nint] * xn[1] + Ab[2 * (size_t)G.Nint] * xn[2];
            }
        }
        const int c = i + G.nx * (j + G.ny * kz);
        const int con = cellcon[c];
        if (con >= 0) {
            const double sw = sop[con_well[con]];
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r] -= wC[3 * con + r] * sw;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const long long q = r * G.Ntot + p0;
            if (MODE == 3) {
                acc[r] = o1[q] - acc[r];
                d[0] += acc[r] * acc[r];
            }
            y[q] = acc[r];
            if (MODE == 1) d[0] += o1[q] * acc[r];
            if (MODE == 2) {
                d[0] += acc[r] * o1[q];
                d[1] += acc[r] * acc[r];
            }
        }
    }
    if (MODE == 0) return;
    dd_partials<2>(d, part, G.K);
}

// vector kernels over the interior positions with per-subdomain partials
// OP 0: part0 = (a, b); 1: p = r + beta (p - omega v); 2: s = r - alpha v,
// part0 = (s, s); 3: x += alpha ph + omega sh, r = s - omega t, part0 = (r, r);
// 4: x += alpha ph; 5: r = b, rh = b, x = p = v = 0, part0 = (b, b);
// 6: rh = r, p = v = 0
template <int OP>
__global__ void __launch_bounds__(DD_BS)
k_dd_vec(DdGeom G, const DdPart* __restrict__ parts, double* __restrict__ a,
         double* __restrict__ b, double* __restrict__ c, double* __restrict__ d5,
         double* __restrict__ e5, double* __restrict__ f5, double s1, double s2,
         double* __restrict__ part) {
    const DdPart P = parts[blockIdx.y];
    double acc[2] = {0.0, 0.0};
    for (int ii = blockIdx.x * blockDim.x + threadIdx.x; ii < P.nint; ii += gridDim.x * blockDim.x) {
        int i, j, kz;
        dd_cell(G, P, ii, i, j, kz);
        const long long p0 = dd_pos(G, P, i, j, kz);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const long long q = r * G.Ntot + p0;
            if (OP == 0) acc[0] += a[q] * b[q];
            if (OP == 1) a[q] = b[q] + s1 * (a[q] - s2 * c[q]);                 // p, r, v
            if (OP == 2) {                                                       // s, r, v
                a[q] = b[q] - s1 * c[q];
                acc[0] += a[q] * a[q];
            }
            if (OP == 3) {                                                       // x, ph, sh, r, s, t
                a[q] += s1 * b[q] + s2 * c[q];
                d5[q] = e5[q] - s2 * f5[q];
                acc[0] += d5[q] * d5[q];
            }
            if (OP == 4) a[q] += s1 * b[q];                                      // x, ph
            if (OP == 5) {                                                       // b, r, rh, x, p, v
                const double bv = a[q];
                b[q] = bv;
                c[q] = bv;
                d5[q] = 0.0;
                e5[q] = 0.0;
                f5[q] = 0.0;
                acc[0] += bv * bv;
            }
            if (OP == 6) {                                                       // r, rh, p, v
                b[q] = a[q];
                c[q] = 0.0;
                d5[q] = 0.0;
            }
        }
    }
    if (OP == 0 || OP == 2 || OP == 3 || OP == 5) dd_partials<2>(acc, part, G.K);
}

// all-reduce: each subdomain's sum of its blocks, then over the subdomains
// in subdomain order (thread q for partial q)
__global__ void k_dd_allreduce(int K, int gx, const double* __restrict__ part,
                               double* __restrict__ red) {
    const int q = threadIdx.x;
    if (q >= 2) return;
    double tot = 0.0;
    for (int k = 0; k < K; ++k) {
        double sub = 0.0;
        for (int bx = 0; bx < gx; ++bx) sub += part[((size_t)q * K + k) * gx + bx];
        tot += sub;
    }
    red[q] = tot;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void dd_free(bo_sim* s) {
    DdData* d = s->dd;
    if (!d) return;
    void* ptrs[] = {d->parts, d->A, d->x, d->r, d->rh, d->p, d->v, d->s, d->t, d->ph, d->sh,
                    d->b, d->gsc, d->gz, d->part, d->red, d->sop};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete d;
    s->dd = nullptr;
}

static void dd_setup(bo_sim* s) {
    const Geom& g = s->geo;
    if (s->dd && s->dd->ysub == s->ysub) return;
    dd_free(s);
    DdData* d = new DdData();
    s->dd = d;
    d->ysub = s->ysub;
    d->K = (g.ny + s->ysub - 1) / s->ysub;
    if (d->K > DD_MAXK) fail(BO_ERR_INVALID_ARG, "bo_dd_solve: more than 1024 subdomains");
    long long off = 0, ioff = 0;
    for (int k = 0; k < d->K; ++k) {
        DdPart P{};
        P.j0 = k * s->ysub;
        P.j1 = std::min(g.ny, P.j0 + s->ysub);
        P.gl = k > 0 ? 1 : 0;
        P.gh = k + 1 < d->K ? 1 : 0;
        P.nyl = P.j1 - P.j0 + P.gl + P.gh;
        P.off = (int)off;
        P.ioff = (int)ioff;
        P.nint = g.nx * (P.j1 - P.j0) * g.nz;
        off += (long long)g.nx * P.nyl * g.nz;
        ioff += P.nint;
        d->h_parts.push_back(P);
    }
    d->Ntot = off;
    d->Nint = ioff;
    if (off >= (1LL << 31)) fail(BO_ERR_INVALID_ARG, "bo_dd_solve: model too large");
    auto zeros = [&](double** p, size_t count) {
        BO_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(double) * std::max<size_t>(count, 1)));
        BO_CUDA(cudaMemset(*p, 0, sizeof(double) * std::max<size_t>(count, 1)));
    };
    BO_CUDA(cudaMalloc(reinterpret_cast<void**>(&d->parts), sizeof(DdPart) * d->K));
    BO_CUDA(cudaMemcpy(d->parts, d->h_parts.data(), sizeof(DdPart) * d->K, cudaMemcpyHostToDevice));
    zeros(&d->A, 63 * (size_t)d->Nint);
    double** vecs[] = {&d->x, &d->r, &d->rh, &d->p, &d->v, &d->s, &d->t, &d->ph, &d->sh, &d->b};
    for (double** v : vecs) zeros(v, 3 * (size_t)d->Ntot);
    zeros(&d->gsc, 3 * (size_t)g.n);
    zeros(&d->gz, 3 * (size_t)g.n);
    zeros(&d->part, 2 * (size_t)d->K * DD_GX);
    zeros(&d->red, 2);
    zeros(&d->sop, std::max(s->nw, 1));
}

int dd_bicgstab(bo_sim* s, double tol, int maxit, int* its) {
    dd_setup(s);
    DdData* d = s->dd;
    const Geom& g = s->geo;
    cudaStream_t st = s->stream;
    const DdGeom G{g.nx, g.ny, g.nz, g.n, d->K, d->Ntot, d->Nint};
    const dim3 grid(DD_GX, d->K);
    const int hgrid = std::max(1, std::min(DD_GX, (3 * g.nx * g.nz + DD_BS - 1) / DD_BS));
    auto red = [&](double out[2]) {
        k_dd_allreduce<<<1, 32, 0, st>>>(d->K, DD_GX, d->part, d->red);
        count_launch(s, st);
        BO_CUDA(cudaMemcpyAsync(out, d->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        BO_CUDA(cudaStreamSynchronize(st));
    };
    // z = M^-1 r: the subdomains' ILU(0) blocks (tiled sweeps with the slab cuts)
    auto prec = [&](const double* r, double* z) {
        k_dd_out<<<grid, DD_BS, 0, st>>>(G, d->parts, r, d->gsc);
        count_launch(s, st);
        enqueue_fwd(s, st, d->gsc, d->gz, nullptr);
        enqueue_bwd(s, st, d->gz, nullptr);
        k_dd_in<<<grid, DD_BS, 0, st>>>(G, d->parts, d->gz, z);
        count_launch(s, st);
    };
    // y = S x (halo exchange first), MODE as in k_dd_spmv
    auto op = [&](auto mode, double* x, double* y, const double* o1) {
        constexpr int MODE = decltype(mode)::value;
        k_dd_halo<<<dim3(hgrid, d->K), DD_BS, 0, st>>>(G, d->parts, x, nullptr);
        count_launch(s, st);
        if (s->nw > 0) {
            k_dd_wdot<<<s->nw, 128, 0, st>>>(G, d->parts, d->ysub, s->d_wells, s->d_con_cell,
                                             s->d_wB, x, d->sop, nullptr);
            count_launch(s, st);
        }
        k_dd_spmv<MODE><<<grid, DD_BS, 0, st>>>(G, d->parts, d->A, x, y, s->d_cellcon,
                                                s->d_cellcon + g.n, s->d_wC, d->sop, o1, d->part,
                                                nullptr);
        count_launch(s, st);
    };
    using M1 = std::integral_constant<int, 1>;
    using M2 = std::integral_constant<int, 2>;
    using M3 = std::integral_constant<int, 3>;
    // the subdomains' rows and right-hand side
    k_dd_rows<<<grid, DD_BS, 0, st>>>(G, d->parts, s->d_A, d->A);
    count_launch(s, st);
    enqueue_reduced_rhs(s, st);
    k_dd_in<<<grid, DD_BS, 0, st>>>(G, d->parts, s->d_b, d->b);
    count_launch(s, st);
    k_dd_vec<5><<<grid, DD_BS, 0, st>>>(G, d->parts, d->b, d->r, d->rh, d->x, d->p, d->v, 0.0, 0.0,
                                        d->part);
    count_launch(s, st);
    double sums[2];
    red(sums);
    const double nr0 = std::sqrt(sums[0]);
    int it_done = 0;
    auto cycle = [&]() -> int {
        double rho_old = 1.0, alpha = 1.0, omega = 1.0;
        for (int it = it_done + 1; it <= maxit; ++it) {
            k_dd_vec<0><<<grid, DD_BS, 0, st>>>(G, d->parts, d->rh, d->r, nullptr, nullptr, nullptr,
                                                nullptr, 0.0, 0.0, d->part);
            count_launch(s, st);
            red(sums);
            const double rho = sums[0];
            if (rho == 0.0 || !std::isfinite(rho)) return LS_BREAKDOWN;
            const double beta = (rho / rho_old) * (alpha / omega);
            k_dd_vec<1><<<grid, DD_BS, 0, st>>>(G, d->parts, d->p, d->r, d->v, nullptr, nullptr,
                                                nullptr, beta, omega, d->part);
            count_launch(s, st);
            prec(d->p, d->ph);
            op(M1{}, d->ph, d->v, d->rh);
            red(sums);
            const double rv = sums[0];
            if (rv == 0.0 || !std::isfinite(rv)) return LS_BREAKDOWN;
            alpha = rho / rv;
            k_dd_vec<2><<<grid, DD_BS, 0, st>>>(G, d->parts, d->s, d->r, d->v, nullptr, nullptr,
                                                nullptr, alpha, 0.0, d->part);
            count_launch(s, st);
            red(sums);
            if (std::sqrt(sums[0]) <= tol * nr0) {
                k_dd_vec<4><<<grid, DD_BS, 0, st>>>(G, d->parts, d->x, d->ph, nullptr, nullptr,
                                                    nullptr, nullptr, alpha, 0.0, d->part);
                count_launch(s, st);
                it_done = it;
                return LS_OK;
            }
            prec(d->s, d->sh);
            op(M2{}, d->sh, d->t, d->s);
            red(sums);
            const double ts = sums[0], tt = sums[1];
            if (tt == 0.0 || !std::isfinite(tt)) return LS_BREAKDOWN;
            omega = ts / tt;
            if (omega == 0.0 || !std::isfinite(omega)) return LS_BREAKDOWN;
            k_dd_vec<3><<<grid, DD_BS, 0, st>>>(G, d->parts, d->x, d->ph, d->sh, d->r, d->s, d->t,
                                                alpha, omega, d->part);
            count_launch(s, st);
            red(sums);
            it_done = it;
            if (std::sqrt(sums[0]) <= tol * nr0) return LS_OK;
            rho_old = rho;
        }
        return LS_NOT_CONVERGED;
    };
    int status = nr0 == 0.0 ? LS_OK : cycle();
    for (int restarts = 0; status == LS_OK && nr0 > 0.0; ++restarts) {
        op(M3{}, d->x, d->r, d->b);   // r = b - S x
        red(sums);
        const double nt = std::sqrt(sums[0]);
        if (nt <= tol * nr0) break;
        if (restarts >= 8 || it_done >= maxit || !std::isfinite(nt)) {
            status = LS_NOT_CONVERGED;
            break;
        }
        k_dd_vec<6><<<grid, DD_BS, 0, st>>>(G, d->parts, d->r, d->rh, d->p, d->v, nullptr, nullptr,
                                            0.0, 0.0, d->part);
        count_launch(s, st);
        status = cycle();
    }
    if (status == LS_NOT_CONVERGED) it_done = maxit;
    *its = it_done;
    // the solution in the natural layout (the wells' rows follow from it)
    k_dd_out<<<grid, DD_BS, 0, st>>>(G, d->parts, d->x, s->d_xs);
    count_launch(s, st);
    BO_LAUNCH_CHECK("dd bicgstab");
    return status;
}

}  // namespace bo
