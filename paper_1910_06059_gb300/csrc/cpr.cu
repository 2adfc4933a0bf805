// CPR (constrained pressure residual) two-stage preconditioner with an
// aggregation AMG for its pressure stage (arXiv 1910.06059, Section 2.3.1:
// for large cases CPR with algebraic multigrid for the pressure is
// preferable to ILU(0); the decoupling is quasi-IMPES).
//
//   weights   w_c = D_c^-T e_p   (D_c = A_cc, the Jacobian's diagonal block):
//             w_c^T A_cc = e_p^T, the weighted equation has no diagonal
//             dependence on s_w or x
//   pressure  A_p[c, j] = w_c^T A_cj e_p on the 7-point pattern, r_p = w^T r
//   stage 1   x1 = E_p V(A_p, r_p): one V-cycle of plain-aggregation AMG,
//             two damped-Jacobi sweeps (omega 2/3) before and after the
//             coarse correction, an exact solve on the coarsest level
//   stage 2   z = x1 + M_ILU^-1 (r - S x1), S the well-reduced operator
//
// Aggregation.  The aggregates are built once per model on the host from
// the graph Laplacian of the face transmissibilities (strength
// |a_ij| >= 0.25 max_k |a_ik|, symmetrised; greedy passes in natural
// order: seeds whose strong neighbours are all free, attachment to a
// neighbouring aggregate, singletons), level by level on the Galerkin
// coarse Laplacians, down to at most 200 unknowns.  Each Newton system's
// pressure matrix is carried by these fixed piecewise-constant
// prolongators: its coarse operators P^T A_p P are segmented sums over
// precomputed lists of fine entries (fixed order, deterministic).
//
// GPU layout: level 0 is the 7-point pressure matrix in the Jacobian's
// layout ap[b][n] (b: diag, -x, +x, -y, +y, -z, +z; zero where no
// neighbour); coarser levels are CSR (what the Galerkin sums and the
// coarsest inverse read) with an ELL copy for the V-cycle (one thread per
// row, coalesced).  Restriction forms each level's residual once and sums
// each aggregate's members in ascending order (no atomics); prolongation
// adds each node's aggregate value.  The coarsest matrix is inverted per Newton
// system by one CTA (Gauss-Jordan, partial pivoting) and applied as a dense
// product.  All kernels are memory-bound streaming kernels; the V-cycle is
// captured in the BiCGStab iteration's CUDA graph.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace bo {

constexpr double CPR_OMEGA = 2.0 / 3.0;
constexpr double CPR_THETA = 0.25;
constexpr int CPR_COARSE = 200;
constexpr int CPR_MAX_LEVELS = 12;
constexpr int CPR_BS = 256;
constexpr int CPR_GRID = 152 * 4;
constexpr int CPR_GRID_ROWS = 152 * 8;   // coarse-level rows: latency-bound gathers, full occupancy
// levels whose rows are short (the first coarse level: up to 32 entries, 12
// on average) get an ELL copy and one thread per row; the longer rows of the
// coarser levels are read by a warp per row
constexpr int CPR_ELL_MAX = 32, CPR_ELL_AVG = 12;

struct CprLevel {
    int n = 0, nnz = 0;
    // levels >= 1: CSR pattern of the coarse operator, its diagonal positions
    int *rowptr = nullptr, *colind = nullptr, *diag = nullptr;
    double *val = nullptr, *dinv = nullptr;
    // Galerkin lists: entry e of this level = sum of the previous level's
    // entries cidx[cptr[e] .. cptr[e + 1])
    int *cptr = nullptr, *cidx = nullptr;
    // the same operator in ELL form for the V-cycle: width W (the longest
    // row), entry e of row i at e n + i; padding has column i and value 0
    int W = 0;
    bool ell = false;
    int* ecol = nullptr;
    double* eval = nullptr;
    // to the next level: agg[i] = aggregate of node i; members of aggregate I
    // are mem[mptr[I] .. mptr[I + 1]) (ascending)
    int *agg = nullptr, *mptr = nullptr, *mem = nullptr;
    double *x = nullptr, *y = nullptr, *b = nullptr;   // V-cycle vectors
};

struct CprData {
    std::vector<CprLevel> lv;
    std::vector<std::vector<int>> h_agg;   // host copies of the aggregation maps
    int nc = 0;                            // size of the coarsest level
    double* cwork = nullptr;               // [nc][2 nc] Gauss-Jordan work
    double* cinv = nullptr;                // [nc][nc] inverse of the coarsest operator
    double* w = nullptr;                   // [3][n] quasi-IMPES weights
    double* x1 = nullptr;                  // [3][n] E_p x_p (components 1, 2 stay zero)
    double* r2 = nullptr;                  // [3][n] second-stage residual
    int* status = nullptr;                 // [1] a singular coarsest pivot
};

// ---------------------------------------------------------------------------
// Host: the transmissibility Laplacian and its aggregation hierarchy
// ---------------------------------------------------------------------------
struct HostCsr {
    int n = 0;
    std::vector<int> rp, ci;
    std::vector<double> v;
};

// Graph Laplacian of the face transmissibilities (T of the +x, +y, +z face
// of every cell), off-diagonals -T, diagonal (sum T)(1 + 1e-12) + 1e-300;
// columns ascending.
static HostCsr transmissibility_laplacian(const std::vector<double>& T, int nx, int ny, int nz) {
    const int n = nx * ny * nz, plane = nx * ny;
    HostCsr A;
    A.n = n;
    A.rp.assign(n + 1, 0);
    A.ci.reserve((size_t)7 * n);
    A.v.reserve((size_t)7 * n);
    for (int c = 0; c < n; ++c) {
        const int i = c % nx, j = (c / nx) % ny, k = c / plane;
        const int cols[7] = {c - plane, c - nx, c - 1, c, c + 1, c + nx, c + plane};
        const bool has[7] = {k > 0, j > 0, i > 0, true, i + 1 < nx, j + 1 < ny, k + 1 < nz};
        const double tv[7] = {k > 0 ? T[2 * (size_t)n + c - plane] : 0.0, j > 0 ? T[(size_t)n + c - nx] : 0.0,
                              i > 0 ? T[c - 1] : 0.0, 0.0, T[c], T[(size_t)n + c], T[2 * (size_t)n + c]};
        double d = 0.0;
        for (int q = 0; q < 7; ++q)
            if (has[q] && q != 3) d += tv[q];
        for (int q = 0; q < 7; ++q) {
            if (!has[q]) continue;
            A.ci.push_back(cols[q]);
            A.v.push_back(q == 3 ? d * (1.0 + 1e-12) + 1e-300 : -tv[q]);
        }
        A.rp[c + 1] = (int)A.ci.size();
    }
    return A;
}

// Symmetrised strong-connection graph: j strong for i when
// |a_ij| >= theta max_{k != i} |a_ik| (and a_ij != 0); neighbour lists ascending.
static void strong_graph(const HostCsr& A, std::vector<int>& sp, std::vector<int>& sc) {
    const int n = A.n;
    std::vector<std::vector<int>> nb(n);
    for (int i = 0; i < n; ++i) {
        double mx = 0.0;
        for (int q = A.rp[i]; q < A.rp[i + 1]; ++q)
            if (A.ci[q] != i) mx = std::max(mx, std::fabs(A.v[q]));
        for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
            const int j = A.ci[q];
            const double m = std::fabs(A.v[q]);
            if (j != i && m >= CPR_THETA * mx && m > 0.0) {
                nb[i].push_back(j);
                nb[j].push_back(i);
            }
        }
    }
    sp.assign(n + 1, 0);
    sc.clear();
    for (int i = 0; i < n; ++i) {
        std::sort(nb[i].begin(), nb[i].end());
        nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
        sc.insert(sc.end(), nb[i].begin(), nb[i].end());
        sp[i + 1] = (int)sc.size();
    }
}

// Greedy aggregation in natural order; returns the number of aggregates.
static int aggregate(const std::vector<int>& sp, const std::vector<int>& sc, std::vector<int>& agg) {
    const int n = (int)sp.size() - 1;
    agg.assign(n, -1);
    int na = 0;
    for (int i = 0; i < n; ++i) {   // pass 1: a free node whose strong neighbours are all free
        if (agg[i] >= 0) continue;
        bool free = true;
        for (int q = sp[i]; q < sp[i + 1] && free; ++q) free = agg[sc[q]] < 0;
        if (!free) continue;
        agg[i] = na;
        for (int q = sp[i]; q < sp[i + 1]; ++q) agg[sc[q]] = na;
        ++na;
    }
    for (int i = 0; i < n; ++i) {   // pass 2: join the first neighbouring aggregate
        if (agg[i] >= 0) continue;
        for (int q = sp[i]; q < sp[i + 1]; ++q)
            if (agg[sc[q]] >= 0) {
                agg[i] = agg[sc[q]];
                break;
            }
    }
    for (int i = 0; i < n; ++i)     // pass 3: what is left stands alone
        if (agg[i] < 0) agg[i] = na++;
    return na;
}

// Galerkin coarse operator P^T A P of a piecewise-constant P (columns ascending).
static HostCsr galerkin(const HostCsr& A, const std::vector<int>& agg, int nc) {
    std::vector<std::vector<int>> members(nc);
    for (int i = 0; i < A.n; ++i) members[agg[i]].push_back(i);
    HostCsr C;
    C.n = nc;
    C.rp.assign(nc + 1, 0);
    std::vector<int> pos(nc, -1), cols;
    std::vector<double> acc(nc, 0.0);
    for (int I = 0; I < nc; ++I) {
        cols.clear();
        for (int i : members[I])
            for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
                const int J = agg[A.ci[q]];
                if (pos[J] < 0) {
                    pos[J] = 1;
                    cols.push_back(J);
                    acc[J] = 0.0;
                }
                acc[J] += A.v[q];
            }
        std::sort(cols.begin(), cols.end());
        for (int J : cols) {
            C.ci.push_back(J);
            C.v.push_back(acc[J]);
            pos[J] = -1;
        }
        C.rp[I + 1] = (int)C.ci.size();
    }
    return C;
}

template <class T>
static T* upload(const std::vector<T>& h) {
    T* d = nullptr;
    BO_CUDA(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(T) * std::max<size_t>(h.size(), 1)));
    if (!h.empty()) BO_CUDA(cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    return d;
}
template <class T>
static T* dzeros(size_t count) {
    T* d = nullptr;
    BO_CUDA(cudaMalloc(reinterpret_cast<void**>(&d), sizeof(T) * std::max<size_t>(count, 1)));
    BO_CUDA(cudaMemset(d, 0, sizeof(T) * std::max<size_t>(count, 1)));
    return d;
}

// Index of the 7-point block of cell i towards column j (level-0 layout b n + i).
static int l0_entry(int i, int j, const Geom& g) {
    const int plane = g.nx * g.ny;
    const int d = j - i;
    const int b = d == 0 ? NB_DIAG : d == -1 ? NB_MX : d == 1 ? NB_PX : d == -g.nx ? NB_MY
                : d == g.nx ? NB_PY : d == -plane ? NB_MZ : NB_PZ;
    return b * g.n + i;
}

void cpr_build(bo_sim* s) {
    if (s->cpr) return;
    const Geom& g = s->geo;
    const int n = g.n;
    std::vector<double> T(3 * (size_t)n);
    BO_CUDA(cudaMemcpy(T.data(), s->d_T, sizeof(double) * T.size(), cudaMemcpyDeviceToHost));
    std::vector<HostCsr> A;
    std::vector<std::vector<int>> aggs;
    A.push_back(transmissibility_laplacian(T, g.nx, g.ny, g.nz));
    while ((int)A.size() < CPR_MAX_LEVELS && A.back().n > CPR_COARSE) {
        std::vector<int> sp, sc, agg;
        strong_graph(A.back(), sp, sc);
        const int nc = aggregate(sp, sc, agg);
        if (nc >= A.back().n) break;
        A.push_back(galerkin(A.back(), agg, nc));
        aggs.push_back(std::move(agg));
    }
    CprData* c = new CprData();
    s->cpr = c;
    const int L = (int)A.size();
    c->lv.resize(L);
    c->h_agg = aggs;
    // position of entry (I, J) in a level's CSR row
    auto find = [](const HostCsr& M, int I, int J) {
        const int* b = M.ci.data() + M.rp[I];
        const int* e = M.ci.data() + M.rp[I + 1];
        const int* p = std::lower_bound(b, e, J);
        return (int)(p - M.ci.data());
    };
    for (int l = 0; l < L; ++l) {
        CprLevel& v = c->lv[l];
        v.n = A[l].n;
        if (l == 0) {
            v.nnz = 7 * n;
            v.val = dzeros<double>(7 * (size_t)n);
        } else {
            v.nnz = A[l].rp[v.n];
            v.rowptr = upload(A[l].rp);
            v.colind = upload(A[l].ci);
            std::vector<int> dg(v.n);
            for (int I = 0; I < v.n; ++I) dg[I] = find(A[l], I, I);
            v.diag = upload(dg);
            v.val = dzeros<double>(v.nnz);
            // Galerkin lists from level l - 1: fine entries in row order
            const HostCsr& F = A[l - 1];
            const std::vector<int>& ag = aggs[l - 1];
            std::vector<int> cnt(v.nnz + 1, 0), target(F.rp[F.n]);
            for (int i = 0; i < F.n; ++i)
                for (int q = F.rp[i]; q < F.rp[i + 1]; ++q) {
                    target[q] = find(A[l], ag[i], ag[F.ci[q]]);
                    cnt[target[q] + 1] += 1;
                }
            for (int e = 0; e < v.nnz; ++e) cnt[e + 1] += cnt[e];
            std::vector<int> idx(F.rp[F.n]), fill(cnt.begin(), cnt.end() - 1);
            for (int i = 0; i < F.n; ++i)
                for (int q = F.rp[i]; q < F.rp[i + 1]; ++q)
                    idx[fill[target[q]]++] = (l == 1) ? l0_entry(i, F.ci[q], g) : q;
            v.cptr = upload(cnt);
            v.cidx = upload(idx);
            int W = 0;
            for (int I = 0; I < v.n; ++I) W = std::max(W, A[l].rp[I + 1] - A[l].rp[I]);
            v.W = W;
            v.ell = W <= CPR_ELL_MAX && v.nnz <= CPR_ELL_AVG * (long long)v.n;
            if (v.ell) {
                std::vector<int> ec((size_t)W * v.n);
                for (int I = 0; I < v.n; ++I)
                    for (int e = 0; e < W; ++e) {
                        const int q = A[l].rp[I] + e;
                        ec[(size_t)e * v.n + I] = q < A[l].rp[I + 1] ? A[l].ci[q] : I;
                    }
                v.ecol = upload(ec);
                v.eval = dzeros<double>((size_t)W * v.n);
            }
        }
        v.dinv = dzeros<double>(v.n);
        v.x = (l == 0) ? nullptr : dzeros<double>(v.n);   // level 0: the pressure column of x1
        v.y = dzeros<double>(v.n);
        v.b = dzeros<double>(v.n);
        if (l + 1 < L) {
            const std::vector<int>& ag = aggs[l];
            const int nc = A[l + 1].n;
            std::vector<int> mp(nc + 1, 0), mem(v.n);
            for (int i = 0; i < v.n; ++i) mp[ag[i] + 1] += 1;
            for (int I = 0; I < nc; ++I) mp[I + 1] += mp[I];
            std::vector<int> fill(mp.begin(), mp.end() - 1);
            for (int i = 0; i < v.n; ++i) mem[fill[ag[i]]++] = i;
            v.agg = upload(ag);
            v.mptr = upload(mp);
            v.mem = upload(mem);
        }
    }
    c->nc = A[L - 1].n;
    c->cwork = dzeros<double>((size_t)c->nc * 2 * c->nc);
    c->cinv = dzeros<double>((size_t)c->nc * c->nc);
    c->w = dzeros<double>(3 * (size_t)n);
    c->x1 = dzeros<double>(3 * (size_t)n);
    c->lv[0].x = c->x1;   // x1 = E_p x_p: its s_w and x columns stay zero
    c->r2 = dzeros<double>(3 * (size_t)n);
    c->status = dzeros<int>(1);
}

void cpr_free(bo_sim* s) {
    CprData* c = s->cpr;
    if (!c) return;
    for (CprLevel& v : c->lv) {
        void* ptrs[] = {v.rowptr, v.colind, v.diag, v.val, v.dinv, v.cptr, v.cidx, v.ecol,
                        v.eval,   v.agg,    v.mptr, v.mem, v.x == c->x1 ? nullptr : v.x,
                        v.y,      v.b};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    void* ptrs[] = {c->cwork, c->cinv, c->w, c->x1, c->r2, c->status};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c;
    s->cpr = nullptr;
}

// ---------------------------------------------------------------------------
// Per Newton system: weights, pressure matrix, coarse operators, coarsest inverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CPR_BS)
k_cpr_level0(int n, const double* __restrict__ A, double* __restrict__ w, double* __restrict__ ap,
             double* __restrict__ dinv) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double a[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) a[e] = A[(size_t)(NB_DIAG * 9 + e) * n + c];
        // w = first row of A_cc^-1 (w^T A_cc = e_p^T), by cofactors
        const double c00 = a[4] * a[8] - a[5] * a[7];
        const double c01 = a[5] * a[6] - a[3] * a[8];
        const double c02 = a[3] * a[7] - a[4] * a[6];
        const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
        const double w0 = c00 / det;
        const double w1 = (a[2] * a[7] - a[1] * a[8]) / det;
        const double w2 = (a[1] * a[5] - a[2] * a[4]) / det;
        w[c] = w0;
        w[(size_t)n + c] = w1;
        w[2 * (size_t)n + c] = w2;
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            const double* Ab = A + (size_t)(b * 9) * n + c;   // column 0 of block b: entries 0, 3, 6
            const double v = w0 * Ab[0] + w1 * Ab[(size_t)3 * n] + w2 * Ab[(size_t)6 * n];
            ap[(size_t)b * n + c] = v;
            if (b == NB_DIAG) dinv[c] = 1.0 / v;
        }
    }
}

__global__ void __launch_bounds__(CPR_BS)
k_cpr_galerkin(int nc, const int* __restrict__ rowptr, const int* __restrict__ diag,
               const int* __restrict__ cptr, const int* __restrict__ cidx,
               const double* __restrict__ fine, double* __restrict__ val, double* __restrict__ eval,
               double* __restrict__ dinv) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        for (int e = rowptr[I]; e < rowptr[I + 1]; ++e) {
            double s = 0.0;
            for (int q = cptr[e]; q < cptr[e + 1]; ++q) s += fine[cidx[q]];
            val[e] = s;
            if (eval) eval[(size_t)(e - rowptr[I]) * nc + I] = s;
        }
        dinv[I] = 1.0 / val[diag[I]];
    }
}

struct Nb7 {
    int nb[7];
    bool has[7];
};
__device__ __forceinline__ Nb7 nb7(const Geom& g, int c) {
    const int plane = g.nx * g.ny, i = c % g.nx, j = (c / g.nx) % g.ny, k = c / plane;
    Nb7 r;
    r.nb[NB_DIAG] = c;
    r.has[NB_DIAG] = true;
    r.nb[NB_MX] = c - 1;
    r.has[NB_MX] = i > 0;
    r.nb[NB_PX] = c + 1;
    r.has[NB_PX] = i + 1 < g.nx;
    r.nb[NB_MY] = c - g.nx;
    r.has[NB_MY] = j > 0;
    r.nb[NB_PY] = c + g.nx;
    r.has[NB_PY] = j + 1 < g.ny;
    r.nb[NB_MZ] = c - plane;
    r.has[NB_MZ] = k > 0;
    r.nb[NB_PZ] = c + plane;
    r.has[NB_PZ] = k + 1 < g.nz;
    return r;
}
// Coarsest operator to dense [A | I] and Gauss-Jordan with partial pivoting
// by one CTA; the inverse lands in cinv.  A zero pivot sets status.
__global__ void __launch_bounds__(1024)
k_cpr_coarse_inverse(Geom g0, int nc, const int* __restrict__ rowptr, const int* __restrict__ colind,
                     const double* __restrict__ val, double* __restrict__ M,
                     double* __restrict__ cinv, int* __restrict__ status) {
    const int m2 = 2 * nc;
    for (int q = threadIdx.x; q < nc * m2; q += blockDim.x) {
        const int r = q / m2, col = q % m2;
        M[q] = (col >= nc && col - nc == r) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (rowptr) {
        for (int r = threadIdx.x; r < nc; r += blockDim.x)
            for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) M[(size_t)r * m2 + colind[e]] = val[e];
    } else {   // the coarsest level is level 0: the 7-point layout val[b][n]
        for (int r = threadIdx.x; r < nc; r += blockDim.x) {
            const Nb7 q = nb7(g0, r);
            for (int b = 0; b < 7; ++b)
                if (q.has[b]) M[(size_t)r * m2 + q.nb[b]] = val[(size_t)b * nc + r];
        }
    }
    __syncthreads();
    __shared__ double red_v[1024];
    __shared__ int red_i[1024];
    __shared__ int piv_s;
    for (int k = 0; k < nc; ++k) {
        // pivot: the largest |M[i][k]|, i >= k (first index on ties)
        double best = -1.0;
        int bi = k;
        for (int i = k + threadIdx.x; i < nc; i += blockDim.x) {
            const double v = fabs(M[(size_t)i * m2 + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        red_v[threadIdx.x] = best;
        red_i[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) {
                const double v2 = red_v[threadIdx.x + o];
                const int i2 = red_i[threadIdx.x + o];
                if (v2 > red_v[threadIdx.x] || (v2 == red_v[threadIdx.x] && i2 < red_i[threadIdx.x])) {
                    red_v[threadIdx.x] = v2;
                    red_i[threadIdx.x] = i2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            piv_s = red_i[0];
            if (!(red_v[0] > 0.0)) *status = 1;
        }
        __syncthreads();
        const int p = piv_s;
        if (p != k)
            for (int col = threadIdx.x; col < m2; col += blockDim.x) {
                const double t = M[(size_t)k * m2 + col];
                M[(size_t)k * m2 + col] = M[(size_t)p * m2 + col];
                M[(size_t)p * m2 + col] = t;
            }
        __syncthreads();
        const double inv = 1.0 / M[(size_t)k * m2 + k];
        __syncthreads();
        for (int col = threadIdx.x; col < m2; col += blockDim.x) M[(size_t)k * m2 + col] *= inv;
        __syncthreads();
        for (int q = threadIdx.x; q < nc * m2; q += blockDim.x) {
            const int i = q / m2, col = q % m2;
            if (i == k) continue;
            const double f = M[(size_t)i * m2 + k];
            if (col != k) M[q] -= f * M[(size_t)k * m2 + col];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nc; i += blockDim.x)
            if (i != k) M[(size_t)i * m2 + k] = 0.0;
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        const int r = q / nc, col = q % nc;
        cinv[q] = M[(size_t)r * m2 + nc + col];
    }
}

// ---------------------------------------------------------------------------
// V-cycle kernels.  Level 0: the 7-point matrix ap[b][n]; levels >= 1: CSR.
// ---------------------------------------------------------------------------
// (A x)_c on level 0, x read through f(j)
template <class F>
__device__ __forceinline__ double ax0(const Geom& g, const double* __restrict__ ap, int c, F f) {
    const Nb7 q = nb7(g, c);
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 7; ++b)
        if (q.has[b]) s += ap[(size_t)b * g.n + c] * f(q.nb[b]);
    return s;
}

// first pre-smoothing from x = 0 on level 0: b = w^T r, x = omega dinv b
__global__ void __launch_bounds__(CPR_BS)
k_cpr_pre0(int n, const double* __restrict__ w, const double* __restrict__ r,
           const double* __restrict__ dinv, double* __restrict__ b, double* __restrict__ x,
           const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const double bv = w[c] * r[c] + w[(size_t)n + c] * r[(size_t)n + c] +
                          w[2 * (size_t)n + c] * r[2 * (size_t)n + c];
        b[c] = bv;
        x[c] = CPR_OMEGA * dinv[c] * bv;
    }
}
// first pre-smoothing from x = 0 on a coarse level
__global__ void __launch_bounds__(CPR_BS)
k_cpr_pre(int n, const double* __restrict__ b, const double* __restrict__ dinv,
          double* __restrict__ x, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x[c] = CPR_OMEGA * dinv[c] * b[c];
}

// y = x + omega dinv (b - A x) on level 0
__global__ void __launch_bounds__(CPR_BS)
k_cpr_jac0(Geom g, const double* __restrict__ ap, const double* __restrict__ dinv,
           const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ y,
           const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += gridDim.x * blockDim.x) {
        const double s = ax0(g, ap, c, [&](int j) { return x[j]; });
        y[c] = x[c] + CPR_OMEGA * dinv[c] * (b[c] - s);
    }
}
// Prolongation folded into the last kernel that writes a coarse level's x:
// each coarse row I adds its final value to the finer level's x at the
// members of aggregate I (every fine node has one aggregate: no conflicts).
struct Prolong {
    const int* mptr = nullptr;
    const int* mem = nullptr;
    double* xf = nullptr;
};
__device__ __forceinline__ void prolong_row(const Prolong& up, int I, double xI) {
    if (up.xf == nullptr) return;
    for (int q = up.mptr[I]; q < up.mptr[I + 1]; ++q) up.xf[up.mem[q]] += xI;
}

// Levels >= 1 in ELL form: one thread per row, the W entries of a row read
// at e n + i (coalesced over the rows of a warp), all loads of a row
// independent of each other.
__device__ __forceinline__ double ell_dot(int n, int W, int i, const int* __restrict__ col,
                                          const double* __restrict__ val,
                                          const double* __restrict__ x) {
    double s = 0.0;
    for (int e = 0; e < W; ++e) s += val[(size_t)e * n + i] * x[col[(size_t)e * n + i]];
    return s;
}

// y = x + omega dinv (b - A x); with up, y is also added into the finer level
__global__ void __launch_bounds__(CPR_BS)
k_cpr_jac(int n, int W, const int* __restrict__ col, const double* __restrict__ val,
          const double* __restrict__ dinv, const double* __restrict__ b,
          const double* __restrict__ x, double* __restrict__ y, Prolong up,
          const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double yi = x[i] + CPR_OMEGA * dinv[i] * (b[i] - ell_dot(n, W, i, col, val, x));
        y[i] = yi;
        prolong_row(up, i, yi);
    }
}

// residual y = b - A x
__global__ void __launch_bounds__(CPR_BS)
k_cpr_res(int n, int W, const int* __restrict__ col, const double* __restrict__ val,
          const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ y,
          const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        y[i] = b[i] - ell_dot(n, W, i, col, val, x);
}

// Levels whose rows are long (the coarse ones): 32 lanes per row, the row's
// entries strided over the lanes and summed by shuffles.  The loops run
// warp-uniform so every lane reaches the shuffles.
__device__ __forceinline__ double row_dot32(int i, bool active, int lane,
                                            const int* __restrict__ rowptr,
                                            const int* __restrict__ colind,
                                            const double* __restrict__ val,
                                            const double* __restrict__ x) {
    double s = 0.0;
    if (active)
        for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) s += val[e] * x[colind[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}
// y = x + omega dinv (b - A x) (RES = false) or y = b - A x (RES = true)
template <bool RES>
__global__ void __launch_bounds__(CPR_BS)
k_cpr_csr32(int n, const int* __restrict__ rowptr, const int* __restrict__ colind,
            const double* __restrict__ val, const double* __restrict__ dinv,
            const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ y,
            Prolong up, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nwarps) {   // warp-uniform
        const double s = row_dot32(i, true, lane, rowptr, colind, val, x);
        if (lane == 0) {
            const double yi = RES ? b[i] - s : x[i] + CPR_OMEGA * dinv[i] * (b[i] - s);
            y[i] = yi;
            if (!RES) prolong_row(up, i, yi);
        }
    }
}

// residual y = b - A x on level 0 (one thread per cell, coalesced)
__global__ void __launch_bounds__(CPR_BS)
k_cpr_res0(Geom g, const double* __restrict__ ap, const double* __restrict__ b,
           const double* __restrict__ x, double* __restrict__ y,
           const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.n; c += gridDim.x * blockDim.x)
        y[c] = b[c] - ax0(g, ap, c, [&](int j) { return x[j]; });
}

// coarse right-hand side: bc[I] = sum over the members of I (ascending) of y;
// with yc, also the coarse level's first pre-smoothing sweep from zero,
// yc = omega dinv_c bc
__global__ void __launch_bounds__(CPR_BS)
k_cpr_sum(int nc, const int* __restrict__ mptr, const int* __restrict__ mem,
          const double* __restrict__ y, double* __restrict__ bc,
          const double* __restrict__ dinv_c, double* __restrict__ yc,
          const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = mptr[I]; q < mptr[I + 1]; ++q) s += y[mem[q]];
        bc[I] = s;
        if (yc) yc[I] = CPR_OMEGA * dinv_c[I] * s;
    }
}

// coarsest level: x = A^-1 b (dense)
__global__ void __launch_bounds__(CPR_BS)
k_cpr_coarse_apply(int nc, const double* __restrict__ cinv, const double* __restrict__ b,
                   double* __restrict__ x, Prolong up, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nc; r += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < nc; ++q) s += cinv[(size_t)r * nc + q] * b[q];
        x[r] = s;
        prolong_row(up, r, s);
    }
}

// Second-stage residual r2 = r - S E_p x_p: only the pressure column of each
// block enters (x1 = E_p x_p has no s_w or x components), and the well term
// C_w (B_w . x1) / D_w with the per-well dots already in sop.
__global__ void __launch_bounds__(CPR_BS)
k_cpr_resid(Geom g, const double* __restrict__ A, const double* __restrict__ xp,
            const double* __restrict__ r, const int* __restrict__ cellcon,
            const int* __restrict__ con_well, const double* __restrict__ wC,
            const double* __restrict__ sop, const double* __restrict__ ccorr,
            double* __restrict__ r2, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    const int n = g.n;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const Nb7 q = nb7(g, c);
        double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            if (!q.has[b]) continue;
            const double x = xp[q.nb[b]];
#pragma unroll
            for (int e = 0; e < 3; ++e) acc[e] += A[(size_t)(b * 9 + 3 * e) * n + c] * x;
        }
        const int con = cellcon[c];
        if (con >= 0) {
            if (ccorr != nullptr) {   // full standard wells
#pragma unroll
                for (int e = 0; e < 3; ++e) acc[e] -= ccorr[3 * con + e];
            } else {
                const double sw = sop[con_well[con]];
#pragma unroll
                for (int e = 0; e < 3; ++e) acc[e] -= wC[3 * con + e] * sw;
            }
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) r2[(size_t)e * n + c] = r[(size_t)e * n + c] - acc[e];
    }
}

// z += E_p x_p
__global__ void __launch_bounds__(CPR_BS)
k_cpr_add(int n, const double* __restrict__ xp, double* __restrict__ z,
          const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        z[c] += xp[c];
}

// ---------------------------------------------------------------------------
// Host enqueue
// ---------------------------------------------------------------------------
static int grid_for(int n) { return std::max(1, std::min(CPR_GRID, (n + CPR_BS - 1) / CPR_BS)); }

void enqueue_cpr_setup(bo_sim* s, cudaStream_t st) {
    CprData* c = s->cpr;
    const int n = s->geo.n;
    k_cpr_level0<<<grid_for(n), CPR_BS, 0, st>>>(n, s->d_A, c->w, c->lv[0].val, c->lv[0].dinv);
    count_launch(s, st);
    for (size_t l = 1; l < c->lv.size(); ++l) {
        CprLevel& v = c->lv[l];
        k_cpr_galerkin<<<grid_for(v.n), CPR_BS, 0, st>>>(v.n, v.rowptr, v.diag, v.cptr, v.cidx,
                                                        c->lv[l - 1].val, v.val, v.eval, v.dinv);
        count_launch(s, st);
    }
    const CprLevel& last = c->lv.back();
    k_cpr_coarse_inverse<<<1, 1024, 0, st>>>(s->geo, c->nc, last.rowptr, last.colind, last.val,
                                             c->cwork, c->cinv, c->status);
    count_launch(s, st);
    BO_LAUNCH_CHECK("cpr setup");
}

static int grid_for_rows(int n) {
    return std::max(1, std::min(CPR_GRID_ROWS, (n + CPR_BS - 1) / CPR_BS));
}
// short rows (the first coarse level): one thread per row over the ELL copy;
// long rows: a warp per row over the CSR arrays
static int grid_warps(int n) {
    return std::max(1, std::min(CPR_GRID_ROWS, (n + CPR_BS / 32 - 1) / (CPR_BS / 32)));
}
static void jac_ell(bo_sim* s, cudaStream_t st, const CprLevel& v, const double* x, double* y,
                    const KrylovScalars* ks, Prolong up = Prolong{}) {
    if (v.ell)
        k_cpr_jac<<<grid_for_rows(v.n), CPR_BS, 0, st>>>(v.n, v.W, v.ecol, v.eval, v.dinv, v.b, x,
                                                        y, up, ks);
    else
        k_cpr_csr32<false><<<grid_warps(v.n), CPR_BS, 0, st>>>(v.n, v.rowptr, v.colind, v.val,
                                                              v.dinv, v.b, x, y, up, ks);
    count_launch(s, st);
}
static void res_ell(bo_sim* s, cudaStream_t st, const CprLevel& v, const double* x, double* y,
                    const KrylovScalars* ks) {
    if (v.ell)
        k_cpr_res<<<grid_for_rows(v.n), CPR_BS, 0, st>>>(v.n, v.W, v.ecol, v.eval, v.b, x, y, ks);
    else
        k_cpr_csr32<true><<<grid_warps(v.n), CPR_BS, 0, st>>>(v.n, v.rowptr, v.colind, v.val,
                                                             v.dinv, v.b, x, y, Prolong{}, ks);
    count_launch(s, st);
}

// One V-cycle of levels l.. on lv[l].b, result in lv[l].x; on level 0 the
// right-hand side is w^T r (or lv[0].b as it stands when r is null).
// Pre-smoothing: two sweeps from zero (-> y -> x; on the coarse levels the
// first comes with the restriction into the level); restriction: the residual
// b - A x into y, summed per aggregate into the next level's b; the coarser
// levels' last kernel adds P xc into x; post-smoothing: two sweeps x -> y -> x.
static void vcycle(bo_sim* s, cudaStream_t st, size_t l, const double* r,
                   const KrylovScalars* ks, Prolong up = Prolong{}) {
    CprData* c = s->cpr;
    CprLevel& v = c->lv[l];
    const Geom& g = s->geo;
    const int gr = grid_for(v.n);
    if (l + 1 == c->lv.size()) {   // coarsest: exact solve (a single-level hierarchy too)
        if (l == 0 && r) {
            k_cpr_pre0<<<gr, CPR_BS, 0, st>>>(v.n, c->w, r, v.dinv, v.b, v.y, ks);
            count_launch(s, st);
        }
        k_cpr_coarse_apply<<<gr, CPR_BS, 0, st>>>(v.n, c->cinv, v.b, v.x, up, ks);
        count_launch(s, st);
        return;
    }
    CprLevel& w = c->lv[l + 1];
    const bool w_coarsest = l + 2 == c->lv.size();
    if (l == 0) {
        if (r)
            k_cpr_pre0<<<gr, CPR_BS, 0, st>>>(v.n, c->w, r, v.dinv, v.b, v.y, ks);
        else
            k_cpr_pre<<<gr, CPR_BS, 0, st>>>(v.n, v.b, v.dinv, v.y, ks);
        count_launch(s, st);
        k_cpr_jac0<<<gr, CPR_BS, 0, st>>>(g, v.val, v.dinv, v.b, v.y, v.x, ks);
        count_launch(s, st);
        k_cpr_res0<<<gr, CPR_BS, 0, st>>>(g, v.val, v.b, v.x, v.y, ks);
        count_launch(s, st);
    } else {   // the first sweep from zero came with the restriction into this level
        jac_ell(s, st, v, v.y, v.x, ks);
        res_ell(s, st, v, v.x, v.y, ks);
    }
    k_cpr_sum<<<grid_for(w.n), CPR_BS, 0, st>>>(w.n, v.mptr, v.mem, v.y, w.b, w.dinv,
                                               w_coarsest ? nullptr : w.y, ks);
    count_launch(s, st);
    vcycle(s, st, l + 1, r, ks, Prolong{v.mptr, v.mem, v.x});   // adds P xc into v.x
    if (l == 0) {
        k_cpr_jac0<<<gr, CPR_BS, 0, st>>>(g, v.val, v.dinv, v.b, v.x, v.y, ks);
        count_launch(s, st);
        k_cpr_jac0<<<gr, CPR_BS, 0, st>>>(g, v.val, v.dinv, v.b, v.y, v.x, ks);
        count_launch(s, st);
    } else {
        jac_ell(s, st, v, v.x, v.y, ks);
        jac_ell(s, st, v, v.y, v.x, ks, up);
    }
}

// The pressure stage alone: x_p = V(A_p, w^T r) into lv[0].x (r null: the
// right-hand side already in lv[0].b).
void enqueue_cpr_pressure(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks) {
    vcycle(s, st, 0, r, ks);
    BO_LAUNCH_CHECK("cpr v-cycle");
}

// One V-cycle on a host pressure right-hand side b[n] into x[n] (checking).
void cpr_vcycle_host(bo_sim* s, const double* b, double* x) {
    CprData* c = s->cpr;
    const int n = s->geo.n;
    BO_CUDA(cudaMemcpyAsync(c->lv[0].b, b, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
    enqueue_cpr_pressure(s, s->stream, nullptr, nullptr);
    BO_CUDA(cudaMemcpyAsync(x, c->lv[0].x, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
}

// Both stages: z = x1 + M_ILU^-1 (r - S x1), x1 = E_p x_p.
void enqueue_cpr_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                       const KrylovScalars* ks) {
    CprData* c = s->cpr;
    const int n = s->geo.n;
    enqueue_cpr_pressure(s, st, r, ks);
    // r2 = r - S x1, x1 = E_p x_p (the wells' dots read x1's pressure part)
    const double* sop = enqueue_well_dots(s, st, c->x1, ks);
    k_cpr_resid<<<grid_for(n), CPR_BS, 0, st>>>(s->geo, s->d_A, c->lv[0].x, r, s->d_cellcon,
                                               s->d_cellcon + n, s->d_wC, sop, well_corr(s),
                                               c->r2, ks);
    count_launch(s, st);
    enqueue_fwd(s, st, c->r2, z, ks);
    enqueue_bwd(s, st, z, ks);
    k_cpr_add<<<grid_for(n), CPR_BS, 0, st>>>(n, c->lv[0].x, z, ks);
    count_launch(s, st);
    BO_LAUNCH_CHECK("cpr apply");
}

// Host views for checking (after a factorisation with CPR selected).
void cpr_export_pressure(bo_sim* s, double* w, double* ap) {
    CprData* c = s->cpr;
    const int n = s->geo.n;
    std::vector<double> hw(3 * (size_t)n), ha(7 * (size_t)n);
    BO_CUDA(cudaMemcpy(hw.data(), c->w, sizeof(double) * hw.size(), cudaMemcpyDeviceToHost));
    BO_CUDA(cudaMemcpy(ha.data(), c->lv[0].val, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost));
    for (int q = 0; q < n; ++q) {
        if (w)
            for (int e = 0; e < 3; ++e) w[3 * (size_t)q + e] = hw[(size_t)e * n + q];
        if (ap)
            for (int b = 0; b < 7; ++b) ap[7 * (size_t)q + b] = ha[(size_t)b * n + q];
    }
}

int cpr_levels(const bo_sim* s) { return s->cpr ? (int)s->cpr->lv.size() : 0; }
int cpr_level_size(const bo_sim* s, int l) { return s->cpr->lv[l].n; }
const std::vector<int>& cpr_aggregation(const bo_sim* s, int l) { return s->cpr->h_agg[l]; }
int* cpr_status_ptr(bo_sim* s) { return s->cpr->status; }

}  // namespace bo
