// FP32 triangular sweeps of the mixed-precision solver (arXiv 1910.06059,
// Section 2.3.1: the ILU(0) preconditioner of BiCGStab, here applied in FP32
// while the Krylov method, the operator and the Newton test stay FP64).
//
// Same wavefront as the FP64 sweeps (tiles of TJ x TK x-lines, lane (jj, kk)
// handles cell i = l - jj - kk at tile level l), but one warp owns a whole
// tile and computes all three rows of its cell: the values of the lower (or
// upper) neighbours come from the lane itself (i -+ 1), from lanes jj -+ 1
// and kk -+ 1 by warp shuffles, or from the face buffers written by the
// neighbouring tiles.  Nothing in the level loop is FP64 and nothing waits on
// a barrier.
//
// Data in tile order.  For tile t and level l (slot s = t NL + l) the factor
// rows of the 32 lanes are one contiguous chunk, and so are the vector values:
//   forward factors  F[s][g][lane][4], g < 7: entries q = 4g + e of
//                    D^-1 A_-x, D^-1 A_-y, D^-1 A_-z (q = 9 (b-1) + 3 row + col,
//                    q = 27 is padding)
//   backward factors B[s][g][lane][4], g < 7: D^-1 A_+x, D^-1 A_+y, D^-1 A_+z
//                    (q = 9 (b-4) + 3 row + col, q = 27 is padding)
//   vectors          V[s][lane][4] (three rows and a zero)
// so a single TMA bulk copy per chunk moves a tile level into shared memory.
// The copies run D32 levels ahead through a ring of shared-memory stages,
// each with an mbarrier that the copy completes.  Bulk conversion kernels
// move the FP64 Krylov vectors into and out of tile order (all lanes busy,
// off the wavefront).
//
// The pivot inverse D^-1 is not rounded to FP32: the forward sweep's input is
// q_c = D_c^-1 r_c, formed in FP64 by the conversion kernel and then rounded.
// Rounding the entries of an explicit inverse of an ill-conditioned 3x3 pivot
// block (per-cell Skeel condition numbers reach 1e7 at the initial state of
// the undersaturated models) and applying it in FP32 loses the small unknown
// families to cancellation; the scaled off-diagonal blocks do not have this
// problem.
//
// Face values are floats with their own sentinel; a consumer takes a value
// and puts the sentinel back, so the buffers need no refill between sweeps.
#include <algorithm>

#include "tiles.cuh"

namespace bo {

constexpr int D32 = 8;                    // levels in flight per tile
constexpr int FWD_G = 7, BWD_G = 7;       // float4 groups of factor rows per lane
constexpr int FWD_CHUNK = (FWD_G + 1) * 32;   // float4 per stage: factors + vector
constexpr int BWD_CHUNK = (BWD_G + 1) * 32;
constexpr long long MBAR_LIMIT = 1LL << 22;   // bounded mbarrier waits

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bounded wait for a stage; a wait that runs out records the error.
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
    for (long long s = 0; s < MBAR_LIMIT; ++s)
        if (mbar_try_wait(bar, parity)) return;
    atomicExch(err, 1);
}

// Take the three values of a face slot: poll (bounded) until none holds the
// sentinel, then put the sentinel back.  Short waits spin; long ones (a tile
// the wavefront has not reached yet) back off up to 256 ns.
__device__ __forceinline__ void take3(float* slot, float v[3], int* err) {
    if (is_sentinel(v[0]) || is_sentinel(v[1]) || is_sentinel(v[2])) {
        unsigned ns = 32;
        for (long long s = 0;; ++s) {
            v[0] = ld_relaxed(slot);
            v[1] = ld_relaxed(slot + 1);
            v[2] = ld_relaxed(slot + 2);
            if (!is_sentinel(v[0]) && !is_sentinel(v[1]) && !is_sentinel(v[2])) break;
            if (s >= POLL_LIMIT * 4 || ((s & 255) == 255 && ld_relaxed_i(err) != 0)) {
                atomicExch(err, 1);
                v[0] = v[1] = v[2] = 0.f;
                return;
            }
            if (s >= 16) {
                __nanosleep(ns);
                ns = ns < 256u ? 2u * ns : 256u;
            }
        }
    }
    const float sent = __uint_as_float(SENTINEL_BITS32);
    st_relaxed(slot, sent);
    st_relaxed(slot + 1, sent);
    st_relaxed(slot + 2, sent);
}

struct WarpTile {
    int t, J, K, jj, kk, j, k, lane;
    bool valid;
};

__device__ __forceinline__ WarpTile warp_tile(const TileArgs& a) {
    WarpTile W;
    W.t = blockIdx.x;
    W.lane = threadIdx.x;
    W.J = W.t % a.NJ;
    W.K = W.t / a.NJ;
    W.jj = W.lane % TJ;
    W.kk = W.lane / TJ;
    W.j = W.J * TJ + W.jj;
    W.k = W.K * TK + W.kk;
    W.valid = W.j < a.g.ny && W.k < a.g.nz;
    return W;
}

// acc[row] -= M[row][:] v  with M the 9 entries q0..q0+8 of a lane's chunk
__device__ __forceinline__ void sub_block(float acc[3], const float* m, const float v[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        acc[r] = fmaf(-m[3 * r], v[0], acc[r]);
        acc[r] = fmaf(-m[3 * r + 1], v[1], acc[r]);
        acc[r] = fmaf(-m[3 * r + 2], v[2], acc[r]);
    }
}

// a8 forward sweep in FP32: Y = (L_A + D)^-1 R in tile order, from
// Q = D^-1 R: y_c = q_c - sum_lower (D_c^-1 A_ck) y_k.
__global__ void __launch_bounds__(32)
k_fwd32(TileArgs a, const float4* __restrict__ F, const float4* __restrict__ Rt,
        float4* __restrict__ Yt, float* __restrict__ fJ, float* __restrict__ fK,
        const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    __shared__ __align__(128) float4 ring[D32][FWD_CHUNK];
    __shared__ __align__(8) unsigned long long bar[D32];
    const WarpTile W = warp_tile(a);
    const int nx = a.g.nx, lane = W.lane;
    const bool feedJ = W.valid && W.jj == TJ - 1 && W.J + 1 < a.NJ && !ycut(a, (W.J + 1) * TJ);
    const bool feedK = W.valid && W.kk == TK - 1 && W.K + 1 < a.NK && !zcut(a, (W.K + 1) * TK);
    const bool takeJ = W.valid && W.j > 0 && !ycut(a, W.j) && W.jj == 0;
    const bool takeK = W.valid && W.k > 0 && !zcut(a, W.k) && W.kk == 0;
    const bool inJ = W.j > 0 && W.jj > 0, inK = W.k > 0 && W.kk > 0;
    const int l0 = W.jj + W.kk;
    const size_t s0 = (size_t)W.t * a.NL;
    float* fjin = fJ + jslot(a, W.t - 1 < 0 ? 0 : W.t - 1, 0, W.kk, 3) - (size_t)l0 * TK * 3;
    float* fkin = fK + kslot(a, W.t - a.NJ < 0 ? 0 : W.t - a.NJ, 0, W.jj, 3) - (size_t)l0 * TJ * 3;
    float* fjout = fJ + jslot(a, W.t, 0, W.kk, 3) - (size_t)l0 * TK * 3;
    float* fkout = fK + kslot(a, W.t, 0, W.jj, 3) - (size_t)l0 * TJ * 3;
    auto active = [&](int l) { return W.valid && l - l0 >= 0 && l - l0 < nx; };
    auto issue = [&](int l) {   // lane 0: stage of level l
        const int st = l % D32;
        mbar_expect_tx(&bar[st], FWD_CHUNK * 16);
        bulk_load(&ring[st][0], F + (s0 + l) * (FWD_G * 32), FWD_G * 32 * 16, &bar[st]);
        bulk_load(&ring[st][FWD_G * 32], Rt + (s0 + l) * 32, 32 * 16, &bar[st]);
    };
    if (lane == 0) {
        for (int d = 0; d < D32; ++d) mbar_init(&bar[d], 1);
        mbar_init_fence();
        for (int d = 0; d < D32 && d < a.NL; ++d) issue(d);
    }
    __syncwarp();
    auto faces = [&](int l, float fj[3], float fk[3]) {
        const bool act = l < a.NL && active(l);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fj[e] = (act && takeJ) ? ld_relaxed(fjin + (size_t)l * TK * 3 + e) : 0.f;
            fk[e] = (act && takeK) ? ld_relaxed(fkin + (size_t)l * TJ * 3 + e) : 0.f;
        }
    };
    float fjc[3], fkc[3], yprev[3] = {0.f, 0.f, 0.f};
    faces(0, fjc, fkc);
    for (int l = 0; l < a.NL; ++l) {
        const int st = l % D32;
        const bool act = active(l);
        float fjn[3], fkn[3];
        faces(l + 1, fjn, fkn);
        float yj[3], yk[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float a1 = __shfl_up_sync(FULL, yprev[e], 1);
            const float a8 = __shfl_up_sync(FULL, yprev[e], TJ);
            yj[e] = inJ ? a1 : 0.f;
            yk[e] = inK ? a8 : 0.f;
        }
        mbar_wait(&bar[st], (unsigned)(l / D32) & 1u, a.err);
        float m[4 * FWD_G];
#pragma unroll
        for (int g = 0; g < FWD_G; ++g) {
            const float4 v = ring[st][g * 32 + lane];
            m[4 * g] = v.x;
            m[4 * g + 1] = v.y;
            m[4 * g + 2] = v.z;
            m[4 * g + 3] = v.w;
        }
        const float4 rv = ring[st][FWD_G * 32 + lane];
        __syncwarp();   // every lane has read the stage
        if (lane == 0 && l + D32 < a.NL) issue(l + D32);
        float acc[3] = {rv.x, rv.y, rv.z};   // q = D^-1 r (formed in FP64)
        sub_block(acc, m, yprev);
        if (act && takeJ) {
            take3(fjin + (size_t)l * TK * 3, fjc, a.err);
            yj[0] = fjc[0]; yj[1] = fjc[1]; yj[2] = fjc[2];
        }
        sub_block(acc, m + 9, yj);
        if (act && takeK) {
            take3(fkin + (size_t)l * TJ * 3, fkc, a.err);
            yk[0] = fkc[0]; yk[1] = fkc[1]; yk[2] = fkc[2];
        }
        sub_block(acc, m + 18, yk);
#pragma unroll
        for (int e = 0; e < 3; ++e) yprev[e] = act ? acc[e] : 0.f;
        Yt[(s0 + l) * 32 + lane] = make_float4(yprev[0], yprev[1], yprev[2], 0.f);
        if (act && feedJ) {
            float* o = fjout + (size_t)l * TK * 3;
            st_relaxed(o, yprev[0]);
            st_relaxed(o + 1, yprev[1]);
            st_relaxed(o + 2, yprev[2]);
        }
        if (act && feedK) {
            float* o = fkout + (size_t)l * TJ * 3;
            st_relaxed(o, yprev[0]);
            st_relaxed(o + 1, yprev[1]);
            st_relaxed(o + 2, yprev[2]);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fjc[e] = fjn[e];
            fkc[e] = fkn[e];
        }
    }
}

// a8 backward sweep in FP32, in place: Z = (D + U_A)^-1 D Y in tile order.
__global__ void __launch_bounds__(32)
k_bwd32(TileArgs a, const float4* __restrict__ B, float4* __restrict__ Yt, float* __restrict__ fJ,
        float* __restrict__ fK, const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    __shared__ __align__(128) float4 ring[D32][BWD_CHUNK];
    __shared__ __align__(8) unsigned long long bar[D32];
    const WarpTile W = warp_tile(a);
    const int nx = a.g.nx, lane = W.lane;
    const bool feedJ = W.valid && W.jj == 0 && W.J > 0 && !ycut(a, W.J * TJ);
    const bool feedK = W.valid && W.kk == 0 && W.K > 0 && !zcut(a, W.K * TK);
    const bool hasJ = W.j + 1 < a.g.ny && !ycut(a, W.j + 1),
               hasK = W.k + 1 < a.g.nz && !zcut(a, W.k + 1);
    const bool takeJ = W.valid && hasJ && W.jj == TJ - 1, takeK = W.valid && hasK && W.kk == TK - 1;
    const bool inJ = hasJ && W.jj < TJ - 1, inK = hasK && W.kk < TK - 1;
    const int l0 = W.jj + W.kk;
    const size_t s0 = (size_t)W.t * a.NL;
    const int tJ = (W.t + 1 < a.T) ? W.t + 1 : W.t, tK = (W.t + a.NJ < a.T) ? W.t + a.NJ : W.t;
    float* fjin = fJ + jslot(a, tJ, 0, W.kk, 3) - (size_t)l0 * TK * 3;
    float* fkin = fK + kslot(a, tK, 0, W.jj, 3) - (size_t)l0 * TJ * 3;
    float* fjout = fJ + jslot(a, W.t, 0, W.kk, 3) - (size_t)l0 * TK * 3;
    float* fkout = fK + kslot(a, W.t, 0, W.jj, 3) - (size_t)l0 * TJ * 3;
    auto active = [&](int l) { return W.valid && l - l0 >= 0 && l - l0 < nx; };
    auto issue = [&](int step) {   // lane 0: stage of level NL - 1 - step
        const int st = step % D32;
        const size_t sl = s0 + (size_t)(a.NL - 1 - step);
        mbar_expect_tx(&bar[st], BWD_CHUNK * 16);
        bulk_load(&ring[st][0], B + sl * (BWD_G * 32), BWD_G * 32 * 16, &bar[st]);
        bulk_load(&ring[st][BWD_G * 32], Yt + sl * 32, 32 * 16, &bar[st]);
    };
    if (lane == 0) {
        for (int d = 0; d < D32; ++d) mbar_init(&bar[d], 1);
        mbar_init_fence();
        for (int d = 0; d < D32 && d < a.NL; ++d) issue(d);
    }
    __syncwarp();
    auto faces = [&](int l, float fj[3], float fk[3]) {
        const bool act = l >= 0 && active(l);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fj[e] = (act && takeJ) ? ld_relaxed(fjin + (size_t)l * TK * 3 + e) : 0.f;
            fk[e] = (act && takeK) ? ld_relaxed(fkin + (size_t)l * TJ * 3 + e) : 0.f;
        }
    };
    float fjc[3], fkc[3], zprev[3] = {0.f, 0.f, 0.f};
    faces(a.NL - 1, fjc, fkc);
    for (int step = 0; step < a.NL; ++step) {
        const int l = a.NL - 1 - step, st = step % D32;
        const bool act = active(l);
        float fjn[3], fkn[3];
        faces(l - 1, fjn, fkn);
        float zj[3], zk[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float a1 = __shfl_down_sync(FULL, zprev[e], 1);
            const float a8 = __shfl_down_sync(FULL, zprev[e], TJ);
            zj[e] = inJ ? a1 : 0.f;
            zk[e] = inK ? a8 : 0.f;
        }
        mbar_wait(&bar[st], (unsigned)(step / D32) & 1u, a.err);
        float m[28];
#pragma unroll
        for (int g = 0; g < BWD_G; ++g) {
            const float4 v = ring[st][g * 32 + lane];
            m[4 * g] = v.x;
            m[4 * g + 1] = v.y;
            m[4 * g + 2] = v.z;
            m[4 * g + 3] = v.w;
        }
        const float4 yv = ring[st][BWD_G * 32 + lane];
        __syncwarp();
        if (lane == 0 && step + D32 < a.NL) issue(step + D32);
        float acc[3] = {yv.x, yv.y, yv.z};
        sub_block(acc, m, zprev);
        if (act && takeJ) {
            take3(fjin + (size_t)l * TK * 3, fjc, a.err);
            zj[0] = fjc[0]; zj[1] = fjc[1]; zj[2] = fjc[2];
        }
        sub_block(acc, m + 9, zj);
        if (act && takeK) {
            take3(fkin + (size_t)l * TJ * 3, fkc, a.err);
            zk[0] = fkc[0]; zk[1] = fkc[1]; zk[2] = fkc[2];
        }
        sub_block(acc, m + 18, zk);
#pragma unroll
        for (int e = 0; e < 3; ++e) zprev[e] = act ? acc[e] : 0.f;
        Yt[(s0 + l) * 32 + lane] = make_float4(zprev[0], zprev[1], zprev[2], 0.f);
        if (act && feedJ) {
            float* o = fjout + (size_t)l * TK * 3;
            st_relaxed(o, zprev[0]);
            st_relaxed(o + 1, zprev[1]);
            st_relaxed(o + 2, zprev[2]);
        }
        if (act && feedK) {
            float* o = fkout + (size_t)l * TJ * 3;
            st_relaxed(o, zprev[0]);
            st_relaxed(o + 1, zprev[1]);
            st_relaxed(o + 2, zprev[2]);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            fjc[e] = fjn[e];
            fkc[e] = fkn[e];
        }
    }
}

// ---------------------------------------------------------------------------
// Layout conversions (bulk, all lanes busy)
// ---------------------------------------------------------------------------
// FP64 factors (tile order, pidx) -> FP32 chunks F (blocks 1-3) and B
// (blocks 4-6).
__global__ void k_factors32(const double* __restrict__ P, size_t NP, float4* __restrict__ F,
                            float4* __restrict__ Bk) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NP;
         q += (size_t)gridDim.x * blockDim.x) {
        const size_t s = q >> 5;
        const int lane = (int)(q & 31);
        auto Pq = [&](int e) { return P[pidx(s, e, lane)]; };
#pragma unroll
        for (int g = 0; g < FWD_G; ++g) {
            float4 v;
            v.x = (float)Pq(9 + 4 * g);
            v.y = (float)Pq(9 + 4 * g + 1);
            v.z = (float)Pq(9 + 4 * g + 2);
            v.w = (g < FWD_G - 1) ? (float)Pq(9 + 4 * g + 3) : 0.f;
            F[(s * FWD_G + g) * 32 + lane] = v;
        }
#pragma unroll
        for (int g = 0; g < BWD_G; ++g) {
            float4 v;
            v.x = (float)Pq(36 + 4 * g);
            v.y = (float)Pq(36 + 4 * g + 1);
            v.z = (float)Pq(36 + 4 * g + 2);
            v.w = (g < BWD_G - 1) ? (float)Pq(36 + 4 * g + 3) : 0.f;
            Bk[(s * BWD_G + g) * 32 + lane] = v;
        }
    }
}

// Thread g of the conversions handles line (t, lane) at level l, g = (t*32 + lane)*NL + l,
// so neighbouring threads touch neighbouring cells of one x-line.
__device__ __forceinline__ bool line_cell(const TileArgs& a, size_t g, size_t& slot, int& c) {
    const int l = (int)(g % a.NL);
    const size_t tl = g / a.NL;
    const int lane = (int)(tl & 31), t = (int)(tl >> 5);
    const int jj = lane % TJ, kk = lane / TJ;
    const int j = (t % a.NJ) * TJ + jj, k = (t / a.NJ) * TK + kk, i = l - jj - kk;
    slot = ((size_t)t * a.NL + l) * 32 + lane;
    if (j >= a.g.ny || k >= a.g.nz || i < 0 || i >= a.g.nx) return false;
    c = i + a.g.nx * (j + a.g.ny * k);
    return true;
}

// Cell of tile-order slot q (slot-major: neighbouring threads are the lanes of
// one tile level, so the factor reads are coalesced).
__device__ __forceinline__ bool slot_cell(const TileArgs& a, size_t q, int& c) {
    const int lane = (int)(q & 31);
    const size_t s = q >> 5;
    const int l = (int)(s % a.NL), t = (int)(s / a.NL);
    const int jj = lane % TJ, kk = lane / TJ;
    const int j = (t % a.NJ) * TJ + jj, k = (t / a.NJ) * TK + kk, i = l - jj - kk;
    if (j >= a.g.ny || k >= a.g.nz || i < 0 || i >= a.g.nx) return false;
    c = i + a.g.nx * (j + a.g.ny * k);
    return true;
}

// Q = D^-1 r in FP64 (r[e*n + c], D^-1 = block 0 of the FP64 factors), rounded
// into the FP32 tile-order vector; slots without a cell get zeros.
__global__ void k_to_tiles32(TileArgs a, const double* __restrict__ P, const double* __restrict__ r,
                             float4* __restrict__ V, const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    const size_t NP = a.NP;
    const int n = a.g.n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < NP;
         q += (size_t)gridDim.x * blockDim.x) {
        int c;
        const int lane = (int)(q & 31);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (slot_cell(a, q, c)) {
            const double r0 = r[c], r1 = r[(size_t)n + c], r2 = r[2 * (size_t)n + c];
            double o[3];
#pragma unroll
            for (int e = 0; e < 3; ++e)
                o[e] = fma(P[pidx(q >> 5, 3 * e, lane)], r0,
                           fma(P[pidx(q >> 5, 3 * e + 1, lane)], r1, P[pidx(q >> 5, 3 * e + 2, lane)] * r2));
            v.x = (float)o[0];
            v.y = (float)o[1];
            v.z = (float)o[2];
        }
        V[q] = v;
    }
}

// V (FP32 tile order) -> z (FP64, z[e*n + c])
__global__ void k_from_tiles64(TileArgs a, const float4* __restrict__ V, double* __restrict__ z,
                               const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    const size_t total = a.NP;
    const int n = a.g.n;
    for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total;
         g += (size_t)gridDim.x * blockDim.x) {
        size_t slot;
        int c;
        if (!line_cell(a, g, slot, c)) continue;
        const float4 v = V[slot];
        z[c] = (double)v.x;
        z[(size_t)n + c] = (double)v.y;
        z[2 * (size_t)n + c] = (double)v.z;
    }
}

__global__ void k_fill_sentinel32(float* __restrict__ p, size_t count) {
    const float sent = __uint_as_float(SENTINEL_BITS32);
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < count;
         q += (size_t)gridDim.x * blockDim.x)
        p[q] = sent;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
size_t factors32_floats(const bo_sim* s) {
    TileArgs a = tile_args(s);
    return (size_t)a.T * a.NL * 32 * 4 * (FWD_G + BWD_G);
}
size_t vec32_floats(const bo_sim* s) {
    TileArgs a = tile_args(s);
    return (size_t)a.T * a.NL * 32 * 4;
}

static float4* fwd_factors(bo_sim* s) { return reinterpret_cast<float4*>(s->d_P32); }
static float4* bwd_factors(bo_sim* s) {
    TileArgs a = tile_args(s);
    return reinterpret_cast<float4*>(s->d_P32) + (size_t)a.T * a.NL * FWD_G * 32;
}
static float* faceJ3f(bo_sim* s) { return reinterpret_cast<float*>(faceJ3(s)); }
static float* faceK3f(bo_sim* s) {
    TileArgs a = tile_args(s);
    return faceJ3f(s) + (size_t)a.T * s->geo.nx * TK * 3;
}

void setup_sweeps32(bo_sim* s) {
    int dev, sms, per_sm = 0, lim = 1 << 30;
    BO_CUDA(cudaGetDevice(&dev));
    BO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (const void* k : {(const void*)k_fwd32, (const void*)k_bwd32}) {
        // the stage rings want the whole shared-memory carveout
        BO_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
        BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32, 0));
        lim = std::min(lim, per_sm);
    }
    if ((long long)lim * sms < tile_args(s).T)
        fail(BO_ERR_INVALID_ARG, "grid too large for one co-resident FP32 wavefront sweep");
}

void convert_factors32(bo_sim* s, cudaStream_t st) {
    TileArgs a = tile_args(s);
    k_factors32<<<152 * 8, 256, 0, st>>>(s->d_P, a.NP, fwd_factors(s), bwd_factors(s));
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_factors32");
}

void reset_faces32(bo_sim* s, cudaStream_t st) {
    TileArgs a = tile_args(s);
    k_fill_sentinel32<<<304, 256, 0, st>>>(faceJ3f(s), (size_t)a.T * s->geo.nx * (TK + TJ) * 3);
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_fill_sentinel32");
}

void enqueue_fwd32(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks) {
    TileArgs a = tile_args(s);
    float4* R = reinterpret_cast<float4*>(s->d_r32);
    float4* Y = reinterpret_cast<float4*>(s->d_y32);
    k_to_tiles32<<<152 * 8, 256, 0, st>>>(a, (const double*)s->d_P, r, R, ks);
    count_launch(s, st);
    launch_coop(st, a.T, 32, k_fwd32, a, (const float4*)fwd_factors(s), (const float4*)R, Y,
                faceJ3f(s), faceK3f(s), ks);
    count_launch(s, st);
}

void enqueue_bwd32(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks) {
    TileArgs a = tile_args(s);
    float4* Y = reinterpret_cast<float4*>(s->d_y32);
    launch_coop(st, a.T, 32, k_bwd32, a, (const float4*)bwd_factors(s), Y, faceJ3f(s), faceK3f(s),
                ks);
    count_launch(s, st);
    k_from_tiles64<<<152 * 8, 256, 0, st>>>(a, (const float4*)Y, z, ks);
    count_launch(s, st);
}

}  // namespace bo
