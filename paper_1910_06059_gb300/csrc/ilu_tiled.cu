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
// Schedule.  The (j, k) plane is cut into tiles of TJ x TK x-lines; one warp
// owns a tile, one lane owns an x-line (lane = jj + TJ kk).  At tile level l
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
// The factor data P is stored in tile order, P[(b*9 + e) * NP + (t*NL + l)*32
// + lane], so every tile level reads and writes 256 contiguous bytes per
// block entry; b: 0 D^-1, 1..3 D^-1 A_{c,-x/-y/-z}, 4..6 D^-1 A_{c,+x/+y/+z}.
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
            const size_t idx = ((size_t)L.t * a.NL + l) * 32 + lane;
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
                P[(size_t)e * a.NP + idx] = Di[e];
                P[(size_t)(36 + e) * a.NP + idx] = Ux[e];
                P[(size_t)(45 + e) * a.NP + idx] = Uy[e];
                P[(size_t)(54 + e) * a.NP + idx] = Uz[e];
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
        for (int e = 0; e < 9; ++e) Di[e] = act ? P[(size_t)e * a.NP + idx] : 0.0;
        const int lowb[3] = {NB_MX, NB_MY, NB_MZ};
        const bool keep[3] = {true, !ycut(a, j), !zcut(a, k)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int e = 0; e < 9; ++e)
                B[e] = act && keep[d] ? A[(size_t)(lowb[d] * 9 + e) * a.g.n + c] : 0.0;
            mm3t(Di, B, S);
#pragma unroll
            for (int e = 0; e < 9; ++e) P[(size_t)((1 + d) * 9 + e) * a.NP + idx] = S[e];
        }
    }
}

// ---------------------------------------------------------------------------
// a8: forward sweep y = (L_A + D)^-1 r.  The loads of the next tile level (36
// factor entries and r) are issued before the current level waits and
// computes, so their latency overlaps the dependent FP64 chain.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tile_cell(const TileArgs& a, const LaneTile& L, int l, int& c,
                                          size_t& idx) {
    int i = l - L.jj - L.kk;
    if (!L.valid || i < 0 || i >= a.g.nx) return false;
    c = i + a.g.nx * (L.j + a.g.ny * L.k);
    idx = ((size_t)L.t * a.NL + l) * 32 + (threadIdx.x & 31);
    return true;
}

template <int NB, int B0>
__device__ __forceinline__ void ld_P(const TileArgs& a, const double* __restrict__ P, size_t idx,
                                     double (&out)[NB * 9]) {
#pragma unroll
    for (int q = 0; q < NB * 9; ++q) out[q] = P[(size_t)(B0 * 9 + q) * a.NP + idx];
}

// The FP64 part of every tile level is written without branches: on GB300 an
// FP64 warp instruction occupies its sub-partition for about 64 cycles
// however many lanes are active, so a divergent FP64 section would cost its
// instructions once per lane group.  Missing neighbours contribute through
// zero blocks (stored as zeros by the factorisation) and zeroed values.

// acc_r += sum_s (-B[r][s]) v[s] as one fused multiply-add chain per row
__device__ __forceinline__ void fnma_mv(double acc[3], const double* B, const double v[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        acc[r] = fma(-B[3 * r], v[0], acc[r]);
        acc[r] = fma(-B[3 * r + 1], v[1], acc[r]);
        acc[r] = fma(-B[3 * r + 2], v[2], acc[r]);
    }
}

// Sweeps with three warps per tile: warp r computes row r of the 3x3 block
// products for the tile's 32 lines, so each warp issues a third of the FP64
// instructions of a tile level and the three warps run on different
// sub-partitions.  The level's results go through a double-buffered shared
// array (all three components per line) with one named barrier per level;
// face values are read by all three warps, so face slots are refilled with
// the sentinel by k_fill_sentinel after the sweep instead of being reset.
constexpr int ROW_WARPS = 3;
constexpr int SWEEP_THREADS = 32 * ROW_WARPS;

struct RowTile {
    int t, J, K, jj, kk, j, k, row, lane;
    bool valid;
};

__device__ __forceinline__ RowTile row_tile(const TileArgs& a) {
    RowTile R;
    R.t = blockIdx.x;
    R.row = threadIdx.x >> 5;
    R.lane = threadIdx.x & 31;
    R.J = R.t % a.NJ;
    R.K = R.t / a.NJ;
    R.jj = R.lane % TJ;
    R.kk = R.lane / TJ;
    R.j = R.J * TJ + R.jj;
    R.k = R.K * TK + R.kk;
    R.valid = R.j < a.g.ny && R.k < a.g.nz;
    return R;
}

__device__ __forceinline__ bool row_cell(const TileArgs& a, const RowTile& R, int l, int& c,
                                         size_t& idx) {
    int i = l - R.jj - R.kk;
    if (!R.valid || i < 0 || i >= a.g.nx) return false;
    c = i + a.g.nx * (R.j + a.g.ny * R.k);
    idx = ((size_t)R.t * a.NL + l) * 32 + R.lane;
    return true;
}

__device__ __forceinline__ void named_barrier() {
    asm volatile("bar.sync 1, %0;" ::"r"(SWEEP_THREADS) : "memory");
}

// Wait for the three values of a face slot (no reset; see above).
template <typename T>
__device__ __forceinline__ void peek_face(const T* slot, T out[3], int* err) {
    unsigned ns = 64;
    for (long long s = 0;; ++s) {
        bool ready = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            out[q] = ld_relaxed(slot + q);
            ready = ready && !is_sentinel(out[q]);
        }
        if (ready) return;
        if (s >= POLL_LIMIT || ((s & 255) == 255 && ld_relaxed_i(err) != 0)) {
            atomicExch(err, 1);
            out[0] = out[1] = out[2] = T(0);
            return;
        }
        if (BO_POLL_SLEEP_NS > 0) {
            __nanosleep(ns);
            ns = ns < 1024u ? 2u * ns : 1024u;
        }
    }
}

// a8: forward sweep y = (L_A + D)^-1 r, row r of
//     y_c = D_c^-1 r_c - L_x y_{i-1} - L_y y_{j-1} - L_z y_{k-1}   (FP64).
// Every index of the level loop is affine in the level, so the loop only
// advances pointers: the factor slot by 32 entries, the cell by one, the face
// slots by one row of the face.  Factor rows, r and face values of the next
// level are loaded while the current level computes.
__global__ void __launch_bounds__(SWEEP_THREADS)
k_fwd_tiled(TileArgs a, const double* __restrict__ P, const double* __restrict__ r,
            double* __restrict__ y, double* __restrict__ fJ, double* __restrict__ fK,
            const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    __shared__ double ys[2][32][3];
    const RowTile R = row_tile(a);
    const int n = a.g.n, nx = a.g.nx;
    const int rw = R.row;
    const bool feedJ = R.valid && R.jj == TJ - 1 && R.J + 1 < a.NJ && !ycut(a, (R.J + 1) * TJ);
    const bool feedK = R.valid && R.kk == TK - 1 && R.K + 1 < a.NK && !zcut(a, (R.K + 1) * TK);
    const bool hasJ = R.j > 0 && !ycut(a, R.j), hasK = R.k > 0 && !zcut(a, R.k);
    const bool takeJ = R.valid && hasJ && R.jj == 0, takeK = R.valid && hasK && R.kk == 0;
    const int l0 = R.jj + R.kk;                   // first level of this line (i = 0)
    const size_t NP = a.NP;
    // level l of this line: factor slot, cell, face slots (valid when 0 <= i < nx)
    const double* Pl = P + (size_t)(3 * rw) * NP + ((size_t)R.t * a.NL) * 32 + R.lane;
    const int c0 = nx * (R.j + a.g.ny * R.k) - l0;   // cell index at level l is c0 + l
    const double* fjin = fJ + jslot(a, R.t - 1 < 0 ? 0 : R.t - 1, 0, R.kk, 3) - (size_t)l0 * TK * 3;
    const double* fkin = fK + kslot(a, R.t - a.NJ < 0 ? 0 : R.t - a.NJ, 0, R.jj, 3) - (size_t)l0 * TJ * 3;
    double* fjout = fJ + jslot(a, R.t, 0, R.kk, 3) - (size_t)l0 * TK * 3 + rw;
    double* fkout = fK + kslot(a, R.t, 0, R.jj, 3) - (size_t)l0 * TJ * 3 + rw;
    // P entries of row rw: block b, column s at offset (9 b + s) NP from Pl
    auto loadP = [&](int l, double out[12], double rin[3], double fj[3], double fk[3]) {
        const int i = l - l0;
        const bool act = R.valid && i >= 0 && i < nx;
        const double* p = Pl + (size_t)l * 32;
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) out[3 * b2 + s2] = act ? p[(size_t)(9 * b2 + s2) * NP] : 0.0;
        const int c = c0 + l;
#pragma unroll
        for (int e = 0; e < 3; ++e) rin[e] = act ? r[(size_t)e * n + c] : 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fj[e] = (act && takeJ) ? ld_relaxed(fjin + (size_t)l * TK * 3 + e) : 0.0;
            fk[e] = (act && takeK) ? ld_relaxed(fkin + (size_t)l * TJ * 3 + e) : 0.0;
        }
        return act;
    };
    double Pc[12], rc[3], fjc[3], fkc[3];
    bool actc = loadP(0, Pc, rc, fjc, fkc);
    ys[1][R.lane][rw] = 0.0;
    named_barrier();
    for (int l = 0; l < a.NL; ++l) {
        const int pb = (l + 1) & 1, cb = l & 1;
        double Pn[12], rn[3], fjn[3], fkn[3];
        const bool actn = (l + 1 < a.NL) ? loadP(l + 1, Pn, rn, fjn, fkn) : false;
        if (l + 1 >= a.NL) {
#pragma unroll
            for (int q = 0; q < 12; ++q) Pn[q] = 0.0;
            rn[0] = rn[1] = rn[2] = 0.0;
            fjn[0] = fjn[1] = fjn[2] = fkn[0] = fkn[1] = fkn[2] = 0.0;
        }
        double yp[3], yj[3], yk[3];
        const int lj = R.jj > 0 ? R.lane - 1 : R.lane;
        const int lk = R.kk > 0 ? R.lane - TJ : R.lane;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            yp[e] = ys[pb][R.lane][e];
            yj[e] = (hasJ && R.jj > 0) ? ys[pb][lj][e] : 0.0;
            yk[e] = (hasK && R.kk > 0) ? ys[pb][lk][e] : 0.0;
        }
        if (actc && takeJ) {
            if (is_sentinel(fjc[0]) || is_sentinel(fjc[1]) || is_sentinel(fjc[2]))
                peek_face(fjin + (size_t)l * TK * 3, fjc, a.err);
            yj[0] = fjc[0]; yj[1] = fjc[1]; yj[2] = fjc[2];
        }
        if (actc && takeK) {
            if (is_sentinel(fkc[0]) || is_sentinel(fkc[1]) || is_sentinel(fkc[2]))
                peek_face(fkin + (size_t)l * TJ * 3, fkc, a.err);
            yk[0] = fkc[0]; yk[1] = fkc[1]; yk[2] = fkc[2];
        }
        __syncwarp();
        double acc = Pc[0] * rc[0];
        acc = fma(Pc[1], rc[1], acc);
        acc = fma(Pc[2], rc[2], acc);
        double t = -Pc[3] * yp[0];
        t = fma(-Pc[4], yp[1], t);
        t = fma(-Pc[5], yp[2], t);
        t = fma(-Pc[6], yj[0], t);
        t = fma(-Pc[7], yj[1], t);
        t = fma(-Pc[8], yj[2], t);
        double u = -Pc[9] * yk[0];
        u = fma(-Pc[10], yk[1], u);
        u = fma(-Pc[11], yk[2], u);
        acc = acc + (t + u);
        ys[cb][R.lane][rw] = actc ? acc : 0.0;
        if (actc) {
            y[(size_t)rw * n + c0 + l] = acc;
            if (feedJ) st_relaxed(fjout + (size_t)l * TK * 3, acc);
            if (feedK) st_relaxed(fkout + (size_t)l * TJ * 3, acc);
        }
        named_barrier();
#pragma unroll
        for (int q = 0; q < 12; ++q) Pc[q] = Pn[q];
        rc[0] = rn[0]; rc[1] = rn[1]; rc[2] = rn[2];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fjc[e] = fjn[e];
            fkc[e] = fkn[e];
        }
        actc = actn;
    }
}

// a8: backward sweep in place, row r of z_c = y_c - sum_upper (D^-1 A_cj) z_j
// (FP64); levels run downward, same pointer stepping in the other direction.
__global__ void __launch_bounds__(SWEEP_THREADS)
k_bwd_tiled(TileArgs a, const double* __restrict__ P, double* __restrict__ z,
            double* __restrict__ fJ, double* __restrict__ fK, const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    __shared__ double zs[2][32][3];
    const RowTile R = row_tile(a);
    const int n = a.g.n, nx = a.g.nx;
    const int rw = R.row;
    const bool feedJ = R.valid && R.jj == 0 && R.J > 0 && !ycut(a, R.J * TJ);
    const bool feedK = R.valid && R.kk == 0 && R.K > 0 && !zcut(a, R.K * TK);
    const bool hasJ = R.j + 1 < a.g.ny && !ycut(a, R.j + 1),
               hasK = R.k + 1 < a.g.nz && !zcut(a, R.k + 1);
    const bool takeJ = R.valid && hasJ && R.jj == TJ - 1, takeK = R.valid && hasK && R.kk == TK - 1;
    const int l0 = R.jj + R.kk;
    const size_t NP = a.NP;
    const double* Pl = P + (size_t)(36 + 3 * rw) * NP + ((size_t)R.t * a.NL) * 32 + R.lane;
    const int c0 = nx * (R.j + a.g.ny * R.k) - l0;
    const int tJ = (R.t + 1 < a.T) ? R.t + 1 : R.t, tK = (R.t + a.NJ < a.T) ? R.t + a.NJ : R.t;
    const double* fjin = fJ + jslot(a, tJ, 0, R.kk, 3) - (size_t)l0 * TK * 3;
    const double* fkin = fK + kslot(a, tK, 0, R.jj, 3) - (size_t)l0 * TJ * 3;
    double* fjout = fJ + jslot(a, R.t, 0, R.kk, 3) - (size_t)l0 * TK * 3 + rw;
    double* fkout = fK + kslot(a, R.t, 0, R.jj, 3) - (size_t)l0 * TJ * 3 + rw;
    // next[0..8]: P entries of row rw; next[9]: y of the cell (row rw)
    auto load = [&](int l, double next[10], double fj[3], double fk[3]) {
        const int i = l - l0;
        const bool act = R.valid && i >= 0 && i < nx;
        const double* p = Pl + (size_t)l * 32;
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2)
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) next[3 * b2 + s2] = act ? p[(size_t)(9 * b2 + s2) * NP] : 0.0;
        next[9] = act ? z[(size_t)rw * n + c0 + l] : 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fj[e] = (act && takeJ) ? ld_relaxed(fjin + (size_t)l * TK * 3 + e) : 0.0;
            fk[e] = (act && takeK) ? ld_relaxed(fkin + (size_t)l * TJ * 3 + e) : 0.0;
        }
        return act;
    };
    double Pc[10], fjc[3], fkc[3];
    bool actc = load(a.NL - 1, Pc, fjc, fkc);
    zs[1][R.lane][rw] = 0.0;
    named_barrier();
    const int lj = R.jj < TJ - 1 ? R.lane + 1 : R.lane;
    const int lk = R.kk < TK - 1 ? R.lane + TJ : R.lane;
    const bool inJ = hasJ && R.jj < TJ - 1, inK = hasK && R.kk < TK - 1;
    int step = 0;
    for (int l = a.NL - 1; l >= 0; --l, ++step) {
        const int pb = (step + 1) & 1, cb = step & 1;
        double Pn[10], fjn[3], fkn[3];
        bool actn = false;
        if (l > 0) {
            actn = load(l - 1, Pn, fjn, fkn);
        } else {
#pragma unroll
            for (int q = 0; q < 10; ++q) Pn[q] = 0.0;
            fjn[0] = fjn[1] = fjn[2] = fkn[0] = fkn[1] = fkn[2] = 0.0;
        }
        double zp[3], zj[3], zk[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            zp[e] = zs[pb][R.lane][e];
            zj[e] = inJ ? zs[pb][lj][e] : 0.0;
            zk[e] = inK ? zs[pb][lk][e] : 0.0;
        }
        if (actc && takeJ) {
            if (is_sentinel(fjc[0]) || is_sentinel(fjc[1]) || is_sentinel(fjc[2]))
                peek_face(fjin + (size_t)l * TK * 3, fjc, a.err);
            zj[0] = fjc[0]; zj[1] = fjc[1]; zj[2] = fjc[2];
        }
        if (actc && takeK) {
            if (is_sentinel(fkc[0]) || is_sentinel(fkc[1]) || is_sentinel(fkc[2]))
                peek_face(fkin + (size_t)l * TJ * 3, fkc, a.err);
            zk[0] = fkc[0]; zk[1] = fkc[1]; zk[2] = fkc[2];
        }
        __syncwarp();
        double t = -Pc[0] * zp[0];
        t = fma(-Pc[1], zp[1], t);
        t = fma(-Pc[2], zp[2], t);
        t = fma(-Pc[3], zj[0], t);
        t = fma(-Pc[4], zj[1], t);
        t = fma(-Pc[5], zj[2], t);
        double u = -Pc[6] * zk[0];
        u = fma(-Pc[7], zk[1], u);
        u = fma(-Pc[8], zk[2], u);
        const double acc = Pc[9] + (t + u);
        zs[cb][R.lane][rw] = actc ? acc : 0.0;
        if (actc) {
            z[(size_t)rw * n + c0 + l] = acc;
            if (feedJ) st_relaxed(fjout + (size_t)l * TK * 3, acc);
            if (feedK) st_relaxed(fkout + (size_t)l * TJ * 3, acc);
        }
        named_barrier();
#pragma unroll
        for (int q = 0; q < 10; ++q) Pc[q] = Pn[q];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fjc[e] = fjn[e];
            fkc[e] = fkn[e];
        }
        actc = actn;
    }
}

__global__ void k_fill_sentinel(double* __restrict__ p, size_t count) {
    const double sent = __longlong_as_double((long long)SENTINEL_BITS);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
         q += (size_t)gridDim.x * blockDim.x)
        p[q] = sent;
}

// Self-test of the bounded wait: poll a face slot that nothing writes.
__global__ void k_wait_selftest(const double* slot, int* err, long long* ns_out) {
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    double v[3];
    peek_face(slot, v, err);
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
    int lim = 1 << 30;
    for (const void* k : {(const void*)k_fwd_tiled, (const void*)k_bwd_tiled}) {
        BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, SWEEP_THREADS, 0));
        lim = std::min(lim, per_sm);
    }
    if ((long long)lim * sms < tile_args(s).T)
        fail(BO_ERR_INVALID_ARG, "grid too large for one co-resident wavefront sweep");
    setup_sweeps32(s);
}

void enqueue_factor(bo_sim* s, cudaStream_t st, int* bad) {
    TileArgs a = tile_args(s);
    launch_coop(st, tile_grid(s), 32 * TILE_WARPS, k_factor_tiled, a, (const double*)s->d_A,
                s->d_P, faceJ9(s), faceK9(s), bad);
    k_factor_lower<<<152 * 8, 256, 0, st>>>(a, (const double*)s->d_A, s->d_P);
    if (s->mixed) convert_factors32(s, st);
}

static void refill_faces3(bo_sim* s, cudaStream_t st) {
    TileArgs a = tile_args(s);
    k_fill_sentinel<<<304, 256, 0, st>>>(faceJ3(s), (size_t)a.T * s->geo.nx * (TK + TJ) * 3);
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

// In mixed mode the forward sweep leaves y in the FP32 tile-order work
// vector and the backward sweep converts its result into z; the two always
// run as a pair.
void enqueue_fwd(bo_sim* s, cudaStream_t st, const double* r, double* y, const KrylovScalars* ks) {
    if (s->mixed) {
        enqueue_fwd32(s, st, r, ks);
        return;
    }
    TileArgs a = tile_args(s);
    launch_coop(st, a.T, SWEEP_THREADS, k_fwd_tiled, a, (const double*)s->d_P, r, y, faceJ3(s),
                faceK3(s), ks);
    refill_faces3(s, st);
}

void enqueue_bwd(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks) {
    if (s->mixed) {
        enqueue_bwd32(s, st, z, ks);
        return;
    }
    TileArgs a = tile_args(s);
    launch_coop(st, a.T, SWEEP_THREADS, k_bwd_tiled, a, (const double*)s->d_P, z, faceJ3(s),
                faceK3(s), ks);
    refill_faces3(s, st);
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
    k_wait_selftest<<<1, 1, 0, s->stream>>>(slot, err, ns);
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
    std::vector<double> P(9 * a.NP);
    for (int e = 0; e < 9; ++e)
        BO_CUDA(cudaMemcpy(P.data() + e * a.NP, s->d_P + e * a.NP, sizeof(double) * a.NP,
                           cudaMemcpyDeviceToHost));
    const Geom& g = s->geo;
    for (int k = 0; k < g.nz; ++k)
        for (int j = 0; j < g.ny; ++j)
            for (int i = 0; i < g.nx; ++i) {
                int J = j / TJ, K = k / TK, jj = j % TJ, kk = k % TK;
                int t = J + a.NJ * K;
                int l = i + jj + kk;
                size_t idx = ((size_t)t * a.NL + l) * 32 + jj + TJ * kk;
                int c = i + g.nx * (j + g.ny * k);
                for (int e = 0; e < 9; ++e) dinv[9 * (size_t)c + e] = P[e * a.NP + idx];
            }
}

}  // namespace bo
