// Block ILU(0) factorisation and triangular sweeps of the 7-point pattern as
// warp-tiled wavefronts (arXiv 1910.06059, Section 2.3.1: ILU0 is the default
// preconditioner and takes most of the solve time).
//
// ILU(0) on this pattern changes only the diagonal blocks (the grid graph is
// bipartite, so no fill position lies in the pattern):
//     D_c = A_cc - sum_{k in {-x,-y,-z}} A_ck D_k^-1 A_kc,
//     M   = (L_A + D) D^-1 (D + U_A).
// Forward  y_c = D_c^-1 r_c - sum_lower (D_c^-1 A_ck) y_k
// Backward z_c = y_c       - sum_upper (D_c^-1 A_cj) z_j
//
// Schedule of the factorisation.  The (j, k) plane is cut into tiles of
// TJ x TK x-lines; one warp owns a tile, one lane owns an x-line
// (lane = jj + TJ kk).  At tile level l
// lane (jj, kk) handles the cell i = l - jj - kk, so the three lower
// neighbours of that cell were handled one level earlier by the lane itself
// (i-1, kept in registers), by lane jj-1 and by lane kk-1 (exchanged with
// warp shuffles).  Only the tile faces j = j0 and k = k0 depend on another
// warp: the producing warp writes its face values into write-once face
// buffers whose slots hold a NaN sentinel; the consuming warp polls (bounded)
// until the value appears and puts the sentinel back, so the buffers are
// ready for the next sweep without clearing.  A warp only waits for tiles
// with smaller (J, K), and all warps are co-resident (cooperative launch), so
// every wait ends.  A wait that runs out of its bound records an error and
// the sweep finishes with zeros for the missing values.
//
// The factor data P is stored in tile order (pidx in tiles.cuh): a tile
// level's 63 entries x 32 lanes are contiguous, so the sweeps move a level
// with one bulk copy; b: 0 D^-1, 1..3 D^-1 A_{c,-x/-y/-z}, 4..6 D^-1
// A_{c,+x/+y/+z}.  The sweeps themselves are in sweep64.cu.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tiles.cuh"

namespace bo {

#ifndef BO_TILE_WARPS
#define BO_TILE_WARPS 4
#endif
constexpr int TILE_WARPS = BO_TILE_WARPS;  // warps (tiles) per CTA of the factorisation

// Wait for K values of a face slot, return them, and put the sentinel back.
// The poll backs off exponentially (64 ns doubling to 1 us) so waiting lanes
// keep the load/store unit free for the warps doing work.
template <int K>
__device__ __forceinline__ void take_face(double* slot, double (&out)[K], int* err) {
    unsigned ns = 64;
    for (long long s = 0;; ++s) {
        bool ready = true;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            out[q] = ld_relaxed(slot + q);
            ready = ready && !is_sentinel(out[q]);
        }
        if (ready) break;
        if (s >= POLL_LIMIT || ((s & 255) == 255 && ld_relaxed_i(err) != 0)) {
            atomicExch(err, 1);
#pragma unroll
            for (int q = 0; q < K; ++q) out[q] = 0.0;
            return;
        }
        if (BO_POLL_SLEEP_NS > 0) {
            __nanosleep(ns);
            ns = ns < 1024u ? 2u * ns : 1024u;
        }
    }
    const double sent = __longlong_as_double((long long)SENTINEL_BITS);
#pragma unroll
    for (int q = 0; q < K; ++q) st_relaxed(slot + q, sent);
}

template <int K>
__device__ __forceinline__ void put_face(double* slot, const double* v) {
#pragma unroll
    for (int q = 0; q < K; ++q) st_relaxed(slot + q, v[q]);
}

// 3x3 helpers, row-major e = 3r + s
__device__ __forceinline__ void mm3t(const double a[9], const double b[9], double c[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s)
            c[3 * r + s] = a[3 * r] * b[s] + a[3 * r + 1] * b[3 + s] + a[3 * r + 2] * b[6 + s];
}
__device__ __forceinline__ void inv3t(const double a[9], double o[9]) {
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
__device__ __forceinline__ void ldA(const double* __restrict__ A, int b, int n, int c, double m[9]) {
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = A[(size_t)(b * 9 + e) * n + c];
}
// acc -= B v  (B row-major 3x3)
__device__ __forceinline__ void sub_mv(double acc[3], const double B[9], const double v[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) acc[r] -= B[3 * r] * v[0] + B[3 * r + 1] * v[1] + B[3 * r + 2] * v[2];
}

__device__ __forceinline__ double zsel(bool keep, double v) { return keep ? v : 0.0; }

struct LaneTile {
    int t, J, K, jj, kk, j, k;
    bool valid;
};

__device__ __forceinline__ bool lane_tile(const TileArgs& a, LaneTile& L) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    L.t = blockIdx.x + gridDim.x * warp;   // tiles of one CTA are far apart in (J, K)
    if (L.t >= a.T) return false;
    L.J = L.t % a.NJ;
    L.K = L.t / a.NJ;
    L.jj = lane % TJ;
    L.kk = lane / TJ;
    L.j = L.J * TJ + L.jj;
    L.k = L.K * TK + L.kk;
    L.valid = L.j < a.g.ny && L.k < a.g.nz;
    return true;
}


// ---------------------------------------------------------------------------
// a7: factorisation.  Lane state: the scaled upper blocks D^-1 A_{c,+x/+y/+z}
// of its previous cell; the +y and +z ones go to the neighbouring lanes or
// faces.  Only D, D^-1 and these blocks are on the wavefront's critical path
// (branch-free FP64, missing neighbours through zero blocks of A); the scaled
// lower blocks follow in k_factor_lower with full warps.
// ---------------------------------------------------------------------------
// D -= B U, as FMA chains
__device__ __forceinline__ void fnma_mm(double D[9], const double B[9], const double U[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double v = D[3 * r + s];
            v = fma(-B[3 * r], U[s], v);
            v = fma(-B[3 * r + 1], U[3 + s], v);
            v = fma(-B[3 * r + 2], U[6 + s], v);
            D[3 * r + s] = v;
        }
}

__global__ void __launch_bounds__(32 * TILE_WARPS)
k_factor_tiled(TileArgs a, const double* __restrict__ A, double* __restrict__ P,
               double* __restrict__ fJ, double* __restrict__ fK, int* __restrict__ bad) {
    LaneTile L;
    if (!lane_tile(a, L)) return;
    const int n = a.g.n, nx = a.g.nx;
    const int lane = threadIdx.x & 31;
    const bool feedJ = L.jj == TJ - 1 && L.J + 1 < a.NJ && !ycut(a, (L.J + 1) * TJ);
    const bool feedK = L.kk == TK - 1 && L.K + 1 < a.NK && !zcut(a, (L.K + 1) * TK);
    const bool hasJ = L.j > 0 && !ycut(a, L.j), hasK = L.k > 0 && !zcut(a, L.k);
    const bool upJ = !ycut(a, L.j + 1);   // the +y coupling stays in the slab
    const bool upK = !zcut(a, L.k + 1);   // the +z coupling stays in the slab
    double Ux[9], Uy[9], Uz[9];   // this lane's scaled upper blocks of its last cell
#pragma unroll
    for (int e = 0; e < 9; ++e) Ux[e] = Uy[e] = Uz[e] = 0.0;
    for (int l = 0; l < a.NL; ++l) {
        const int i = l - L.jj - L.kk;
        const bool act = L.valid && i >= 0 && i < nx;
        double Uyn[9], Uzn[9];   // neighbours' upper blocks pointing at this cell
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            Uyn[e] = zsel(hasJ, __shfl_up_sync(FULL, Uy[e], 1));
            Uzn[e] = zsel(hasK, __shfl_up_sync(FULL, Uz[e], TJ));
        }
        const int c = act ? i + nx * (L.j + a.g.ny * L.k) : 0;
        if (act && hasJ && L.jj == 0) take_face<9>(fJ + jslot(a, L.t - 1, i, L.kk, 9), Uyn, a.err);
        if (act && hasK && L.kk == 0) take_face<9>(fK + kslot(a, L.t - a.NJ, i, L.jj, 9), Uzn, a.err);
        double D[9], Bx[9], By[9], Bz[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            D[e] = act ? A[(size_t)(NB_DIAG * 9 + e) * n + c] : (e % 4 == 0 ? 1.0 : 0.0);
            Bx[e] = act ? A[(size_t)(NB_MX * 9 + e) * n + c] : 0.0;
            By[e] = act && hasJ ? A[(size_t)(NB_MY * 9 + e) * n + c] : 0.0;
            Bz[e] = act && hasK ? A[(size_t)(NB_MZ * 9 + e) * n + c] : 0.0;
        }
        __syncwarp();
        fnma_mm(D, Bx, Ux);
        fnma_mm(D, By, Uyn);
        fnma_mm(D, Bz, Uzn);
        double Di[9];
        inv3t(D, Di);
        // scaled upper blocks: the data the next cells wait for
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            Bx[e] = act ? A[(size_t)(NB_PX * 9 + e) * n + c] : 0.0;
            By[e] = act && upJ ? A[(size_t)(NB_PY * 9 + e) * n + c] : 0.0;
            Bz[e] = act && upK ? A[(size_t)(NB_PZ * 9 + e) * n + c] : 0.0;
        }
        double Ux2[9], Uy2[9], Uz2[9];
        mm3t(Di, Bx, Ux2);
        mm3t(Di, By, Uy2);
        mm3t(Di, Bz, Uz2);
        if (act) {
            const size_t slot = (size_t)L.t * a.NL + l;
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                Ux[e] = Ux2[e];
                Uy[e] = Uy2[e];
                Uz[e] = Uz2[e];
            }
            if (feedJ) put_face<9>(fJ + jslot(a, L.t, i, L.kk, 9), Uy);
            if (feedK) put_face<9>(fK + kslot(a, L.t, i, L.jj, 9), Uz);
            bool finite = true;
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                finite = finite && isfinite(Di[e]);
                P[pidx(slot, e, lane)] = Di[e];
                P[pidx(slot, 36 + e, lane)] = Ux[e];
                P[pidx(slot, 45 + e, lane)] = Uy[e];
                P[pidx(slot, 54 + e, lane)] = Uz[e];
            }
            if (!finite) atomicAdd(bad, 1);
        }
    }
}

// Scaled lower blocks D_c^-1 A_{c,-x/-y/-z} for every tile-order slot (one
// thread per slot, full warps; zero for idle slots and missing neighbours).
__global__ void __launch_bounds__(256)
k_factor_lower(TileArgs a, const double* __restrict__ A, double* __restrict__ P) {
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < a.NP;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int lane = (int)(idx & 31);
        const size_t tl = idx >> 5;
        const int t = (int)(tl / a.NL), l = (int)(tl % a.NL);
        const int J = t % a.NJ, K = t / a.NJ, jj = lane % TJ, kk = lane / TJ;
        const int j = J * TJ + jj, k = K * TK + kk, i = l - jj - kk;
        const bool act = j < a.g.ny && k < a.g.nz && i >= 0 && i < a.g.nx;
        const int c = act ? i + a.g.nx * (j + a.g.ny * k) : 0;
        double Di[9], B[9], S[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) Di[e] = act ? P[pidx(tl, e, lane)] : 0.0;
        const int lowb[3] = {NB_MX, NB_MY, NB_MZ};
        const bool keep[3] = {true, !ycut(a, j), !zcut(a, k)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int e = 0; e < 9; ++e)
                B[e] = act && keep[d] ? A[(size_t)(lowb[d] * 9 + e) * a.g.n + c] : 0.0;
            mm3t(Di, B, S);
#pragma unroll
            for (int e = 0; e < 9; ++e) P[pidx(tl, (1 + d) * 9 + e, lane)] = S[e];
        }
    }
}

__global__ void k_fill_sentinel(double* __restrict__ p, size_t count) {
    const double sent = __longlong_as_double((long long)SENTINEL_BITS);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
         q += (size_t)gridDim.x * blockDim.x)
        p[q] = sent;
}

// Self-test of the bounded wait: poll a face slot that nothing writes.
__global__ void k_wait_selftest(double* slot, int* err, long long* ns_out) {
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    double v[3];
    take_face<3>(slot, v, err);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    *ns_out = (long long)(t1 - t0);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
TileArgs tile_args(const bo_sim* s) {
    TileArgs a;
    a.g = s->geo;
    a.NJ = (s->geo.ny + TJ - 1) / TJ;
    a.NK = (s->geo.nz + TK - 1) / TK;
    a.T = a.NJ * a.NK;
    a.NL = s->geo.nx + TJ + TK - 2;
    a.NP = (size_t)a.T * a.NL * 32;
    a.err = s->d_sweep_sync + 2;
    a.ysub = s->ysub;
    a.zsub = s->zsub;
    return a;
}

int tile_count(const bo_sim* s) {
    return ((s->geo.ny + TJ - 1) / TJ) * ((s->geo.nz + TK - 1) / TK);
}

size_t ilu_storage(const bo_sim* s) {
    int NJ = (s->geo.ny + TJ - 1) / TJ, NK = (s->geo.nz + TK - 1) / TK;
    return (size_t)NJ * NK * (s->geo.nx + TJ + TK - 2) * 32;
}

// face buffers: factor j/k faces (9 values per slot), sweep j/k faces (3)
size_t face_storage(const bo_sim* s) {
    int NJ = (s->geo.ny + TJ - 1) / TJ, NK = (s->geo.nz + TK - 1) / TK;
    size_t T = (size_t)NJ * NK;
    return T * s->geo.nx * (TK * 9 + TJ * 9 + TK * 3 + TJ * 3);
}

static double* faceJ9(bo_sim* s) { return s->d_face; }
static double* faceK9(bo_sim* s) {
    TileArgs a = tile_args(s);
    return s->d_face + (size_t)a.T * s->geo.nx * TK * 9;
}
double* faceJ3(bo_sim* s) {
    TileArgs a = tile_args(s);
    return faceK9(s) + (size_t)a.T * s->geo.nx * TJ * 9;
}
double* faceK3(bo_sim* s) {
    TileArgs a = tile_args(s);
    return faceJ3(s) + (size_t)a.T * s->geo.nx * TK * 3;
}

static int tile_grid(bo_sim* s) {
    TileArgs a = tile_args(s);
    return (a.T + TILE_WARPS - 1) / TILE_WARPS;
}

void setup_sweeps(bo_sim* s) {
    size_t fc = face_storage(s);
    k_fill_sentinel<<<1024, 256>>>(s->d_face, fc);
    count_launch(s, nullptr);
    BO_LAUNCH_CHECK("k_fill_sentinel");
    BO_CUDA(cudaMemset(s->d_sweep_sync, 0, sizeof(int) * 4));
    BO_CUDA(cudaDeviceSynchronize());
    // every tile warp must be resident at once
    int dev, sms, per_sm = 0;
    BO_CUDA(cudaGetDevice(&dev));
    BO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor_tiled, 32 * TILE_WARPS, 0));
    if ((long long)per_sm * sms < tile_grid(s))
        fail(BO_ERR_INVALID_ARG, "grid too large for one co-resident wavefront factorisation");
    setup_sweeps64(s);
    setup_sweeps32(s);
}

void enqueue_factor(bo_sim* s, cudaStream_t st, int* bad) {
    TileArgs a = tile_args(s);
    launch_coop(st, tile_grid(s), 32 * TILE_WARPS, k_factor_tiled, a, (const double*)s->d_A,
                s->d_P, faceJ9(s), faceK9(s), bad);
    count_launch(s, st);
    k_factor_lower<<<152 * 8, 256, 0, st>>>(a, (const double*)s->d_A, s->d_P);
    count_launch(s, st);
    if (s->mixed) convert_factors32(s, st);
}

static void refill_faces3(bo_sim* s, cudaStream_t st) {
    TileArgs a = tile_args(s);
    k_fill_sentinel<<<304, 256, 0, st>>>(faceJ3(s), (size_t)a.T * s->geo.nx * (TK + TJ) * 3);
    count_launch(s, st);
}

// Sentinels of the current precision in the 3-value face buffers (after a
// precision switch or an abandoned sweep).
void reset_sweep_faces(bo_sim* s) { fill_sweep_faces(s, s->mixed); }

void fill_sweep_faces(bo_sim* s, bool fp32) {
    if (fp32)
        reset_faces32(s, s->stream);
    else
        refill_faces3(s, s->stream);
    BO_LAUNCH_CHECK("fill_sweep_faces");
}

// The forward sweep leaves y in a tile-order work vector (FP64: d_yt; mixed
// mode: the FP32 one) and the backward sweep writes z in natural order; the
// two always run as a pair (y is not needed in natural order).
void enqueue_fwd(bo_sim* s, cudaStream_t st, const double* r, double* y, const KrylovScalars* ks) {
    (void)y;
    if (s->mixed) {
        enqueue_fwd32(s, st, r, ks);
        return;
    }
    enqueue_fwd64(s, st, r, ks);
}

void enqueue_bwd(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks) {
    if (s->mixed) {
        enqueue_bwd32(s, st, z, ks);
        return;
    }
    enqueue_bwd64(s, st, z, ks);
}

int sweep_timeout(bo_sim* s) {
    int v = 0;
    BO_CUDA(cudaMemcpyAsync(&v, s->d_sweep_sync + 2, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    return v;
}

// Runs one bounded face wait that can only time out; returns the wait time.
double wait_selftest(bo_sim* s) {
    int* err = s->d_sweep_sync + 3;   // a flag of its own: the sweeps' flag stays clear
    long long* ns = nullptr;
    double* slot = nullptr;           // a face slot of its own that nothing writes
    BO_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s->stream));
    BO_CUDA(cudaMalloc(&ns, sizeof(long long)));
    BO_CUDA(cudaMalloc(&slot, 3 * sizeof(double)));
    k_fill_sentinel<<<1, 32, 0, s->stream>>>(slot, 3);
    count_launch(s, s->stream);
    k_wait_selftest<<<1, 1, 0, s->stream>>>(slot, err, ns);
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_wait_selftest");
    long long h = 0;
    int e = 0;
    BO_CUDA(cudaMemcpyAsync(&h, ns, sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
    cudaFree(ns);
    cudaFree(slot);
    BO_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s->stream));
    if (e == 0) fail(BO_ERR_STATE, "bounded-wait self-test: the wait did not run out");
    return h * 1e-9;
}

// D^-1 of every cell in natural order, [n][9].
void export_dinv(bo_sim* s, double* dinv) {
    TileArgs a = tile_args(s);
    std::vector<double> P(NPE * a.NP);
    BO_CUDA(cudaMemcpy(P.data(), s->d_P, sizeof(double) * P.size(), cudaMemcpyDeviceToHost));
    const Geom& g = s->geo;
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) {
                int J = j / TJ, K = k / TK, jj = j % TJ, kk = k % TK;
                int t = J + a.NJ * K;
                int l = i + jj + kk;
                size_t slot = (size_t)t * a.NL + l;
                int c = i + g.nx * (j + g.ny * k);
                for (int e = 0; e < 9; ++e) dinv[9 * (size_t)c + e] = P[pidx(slot, e, jj + TJ * kk)];
            }
}

}  // namespace bo
