// FP64 triangular sweeps of the block ILU(0) preconditioner (arXiv
// 1910.06059, Section 2.3.1: ILU0 is BiCGStab's default preconditioner and
// takes most of the solve time).
//
//   forward  y_c = D_c^-1 r_c - sum_lower (D_c^-1 A_ck) y_k
//   backward z_c = y_c       - sum_upper (D_c^-1 A_cj) z_j
//
// Wavefront over tiles of TJ x TK x-lines, as in the factorisation: at tile
// level l, lane (jj, kk) of a tile handles cell i = l - jj - kk, so the three
// lower (upper) neighbours of its cell were handled one level earlier (later)
// by the lane itself, by lane jj -+ 1 and by lane kk -+ 1, or by the
// neighbouring tile for the lanes on the tile's faces.
//
// GB300 design.  An FP64 warp instruction holds its SM sub-partition for
// about 64 cycles however many lanes are active, so a tile level costs what
// its FP64 instructions cost; everything else is kept off that path:
//   * q = D^-1 r is formed before the wavefront by a fully parallel kernel,
//     in tile order; one CTA of four warps per tile; warps 0-2 compute rows
//     0-2 of the level (three block products, two FMA chains), each on its
//     own sub-partition; warp 3 (the helper) fetches the face values of the
//     neighbouring tiles and keeps the stage ring full;
//   * the factor rows of a tile level are one contiguous chunk in HBM
//     (ILU data in tile order, 63 entries x 32 lanes per level) and reach
//     shared memory by cp.async.bulk copies (the level's three scaled
//     blocks and its 3-vector q or y) into a ring of S64 stages, each
//     completed on its own mbarrier, S64 - 1 levels ahead of the arithmetic;
//   * the level's results are exchanged through a zero-padded plane in
//     shared memory whose border row and column hold the neighbouring tiles'
//     face values (written by the helper), so every lane reads its three
//     neighbours with the same three loads: no selects, no shuffles;
//   * the CTAs are persistent: 2 per SM, each taking its tiles from a list in
//     topological order (sorted by the level at which a tile can start);
//     the ring runs on across a CTA's tiles.  A tile waits only for tiles
//     earlier in the list, every CTA is resident (cooperative launch), so
//     every wait ends;
//   * face values pass through write-once slots holding a NaN sentinel; the
//     helper polls (bounded) until a value appears and puts the sentinel back,
//     so no refill kernel runs between sweeps.
// Idle slots of the tile order (ragged tiles, i outside the line) hold zero
// factors; inactive lanes produce zero, so the padding needs no predicates
// in the arithmetic.  The forward result y stays in tile order (the
// backward sweep's bulk copies read it); the backward result z is written in
// natural order.
#include <algorithm>
#include <vector>

#include "tiles.cuh"

namespace bo {

constexpr int S64 = 8;                          // stages of the ring
constexpr int SW_THREADS = 128;                 // 3 row warps + the helper warp
constexpr int HELPER = 3;                       // warp index of the helper
constexpr int BLK_ENT = 27;                     // 3 scaled off-diagonal blocks
constexpr int STAGE = (BLK_ENT + 3) * 32;       // doubles per stage: blocks + a 3-vector
constexpr int HJ = TJ + 1, HK = TK + 1;         // padded exchange plane
constexpr int YPL = HK * HJ;                    // one component of the plane
constexpr int YBUF = 3 * YPL;                   // one level of the plane
constexpr long long MBAR_LIMIT64 = 1LL << 22;   // bounded mbarrier waits

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy primitives (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned sa(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mb_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for a stage; gives up at once when another wait of the sweep
// has already given up (the error flag is set), so a failed sweep ends fast.
__device__ __forceinline__ bool mb_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(sa(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mb_wait(unsigned long long* bar, unsigned parity, int* err) {
    if (mb_test(bar, parity)) return;   // the usual case: the copy landed levels ago
    for (long long q = 0; q < MBAR_LIMIT64; ++q) {
        if (mb_try(bar, parity)) return;
        if ((q & 1023) == 1023 && ld_relaxed_i(err) != 0) return;
    }
    atomicExch(err, 1);
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(sa(dst)),
        "l"(src), "r"(bytes), "r"(sa(bar))
        : "memory");
}

struct SweepArgs {
    TileArgs a;
    const int* order;   // tiles in topological order of the sweep's direction
    int G;              // CTAs of the launch
};

// Geometry of one lane of tile t.
struct LaneGeo {
    int t, J, K, j, k, l0, cbase;   // cell at level l: cbase + l (when active)
    bool valid;
};
__device__ __forceinline__ LaneGeo lane_geo(const TileArgs& a, int t, int lane) {
    LaneGeo G;
    G.t = t;
    G.J = t % a.NJ;
    G.K = t / a.NJ;
    const int jj = lane % TJ, kk = lane / TJ;
    G.j = G.J * TJ + jj;
    G.k = G.K * TK + kk;
    G.l0 = jj + kk;
    G.valid = G.j < a.g.ny && G.k < a.g.nz;
    G.cbase = a.g.nx * (G.j + a.g.ny * G.k) - G.l0;
    return G;
}
__device__ __forceinline__ bool lane_active(const TileArgs& a, const LaneGeo& G, int l) {
    const int i = l - G.l0;
    return G.valid && i >= 0 && i < a.g.nx;
}

// Poll a face slot (bounded) until none of its three values is the sentinel,
// then put the sentinel back.  v holds the prefetched values on entry.
__device__ __forceinline__ void take_slot(double* slot, double v[3], int* err) {
    if (is_sentinel(v[0]) || is_sentinel(v[1]) || is_sentinel(v[2])) {
        unsigned ns = 32;
        for (long long q = 0;; ++q) {
            v[0] = ld_relaxed(slot);
            v[1] = ld_relaxed(slot + 1);
            v[2] = ld_relaxed(slot + 2);
            if (!is_sentinel(v[0]) && !is_sentinel(v[1]) && !is_sentinel(v[2])) break;
            if (q >= POLL_LIMIT * 4 || ((q & 255) == 255 && ld_relaxed_i(err) != 0)) {
                atomicExch(err, 1);
                v[0] = v[1] = v[2] = 0.0;
                return;
            }
            if (q >= 32) {
                __nanosleep(ns);
                ns = ns < 256u ? 2u * ns : 256u;
            }
        }
    }
    const double sent = __longlong_as_double((long long)SENTINEL_BITS);
    st_relaxed(slot, sent);
    st_relaxed(slot + 1, sent);
    st_relaxed(slot + 2, sent);
}

// A helper lane's face slot for one tile: at level l the slot is
// base + (l - off) stride, to be read when need and 0 <= l - off < nx; hp is
// the slot's place in the padded exchange plane (-1: this lane has no face).
struct FaceLane {
    double* base;
    int off, stride, hp;
    bool need;
};
// Forward: lanes 0..TK-1 take the j-face of row kk = lane from tile J - 1,
// lanes TK..TK+TJ-1 the k-face of column jj = lane - TK from tile K - 1.
__device__ __forceinline__ FaceLane face_lane_fwd(const TileArgs& a, const LaneGeo& G, int lane,
                                                  double* fJ, double* fK) {
    FaceLane f{nullptr, 0, 0, -1, false};
    if (lane < TK) {
        const int kk = lane;
        f.off = kk;
        f.stride = TK * 3;
        f.hp = (kk + 1) * HJ;
        f.need = G.J > 0 && !ycut(a, G.J * TJ) && G.K * TK + kk < a.g.nz;
        if (f.need) f.base = fJ + jslot(a, G.t - 1, 0, kk, 3);
    } else if (lane < TK + TJ) {
        const int jj = lane - TK;
        f.off = jj;
        f.stride = TJ * 3;
        f.hp = jj + 1;
        f.need = G.K > 0 && !zcut(a, G.K * TK) && G.J * TJ + jj < a.g.ny;
        if (f.need) f.base = fK + kslot(a, G.t - a.NJ, 0, jj, 3);
    }
    return f;
}
// Backward: the upper neighbours of lane (TJ - 1, kk) in tile J + 1 and of
// lane (jj, TK - 1) in tile K + 1.
__device__ __forceinline__ FaceLane face_lane_bwd(const TileArgs& a, const LaneGeo& G, int lane,
                                                  double* fJ, double* fK) {
    FaceLane f{nullptr, 0, 0, -1, false};
    if (lane < TK) {
        const int kk = lane;
        f.off = TJ - 1 + kk;
        f.stride = TK * 3;
        f.hp = kk * HJ + TJ;
        f.need = G.J + 1 < a.NJ && !ycut(a, (G.J + 1) * TJ) && G.K * TK + kk < a.g.nz;
        if (f.need) f.base = fJ + jslot(a, G.t + 1, 0, kk, 3);
    } else if (lane < TK + TJ) {
        const int jj = lane - TK;
        f.off = jj + TK - 1;
        f.stride = TJ * 3;
        f.hp = TK * HJ + jj;
        f.need = G.K + 1 < a.NK && !zcut(a, (G.K + 1) * TK) && G.J * TJ + jj < a.g.ny;
        if (f.need) f.base = fK + kslot(a, G.t + a.NJ, 0, jj, 3);
    }
    return f;
}
__device__ __forceinline__ double* face_at(const FaceLane& f, int l, int nx) {
    const int i = l - f.off;
    return (f.need && i >= 0 && i < nx) ? f.base + (size_t)i * f.stride : nullptr;
}

// The helper warp's view of one stage: which tile and level it belongs to.
struct StageCursor {
    int m, l;   // m-th tile of this CTA, level (forward) or step (backward)
};
__device__ __forceinline__ void advance(StageCursor& c, int NL) {
    if (++c.l == NL) {
        c.l = 0;
        ++c.m;
    }
}

constexpr int MAX_CTA_TILES = 64;   // tiles of one CTA (checked on the host)

// ---------------------------------------------------------------------------
// q = D^-1 r in tile order, Qt[slot][3][32] (zero for idle slots): the
// forward sweep's right-hand side, formed by all SMs before the wavefront.
// Threads follow the tile order (a warp is one tile level), so the factor
// reads and the writes are coalesced; neighbouring warps are neighbouring
// levels of one tile and reuse each other's sectors of r.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_q_tiles(TileArgs a, const double* __restrict__ P, const double* __restrict__ r,
          double* __restrict__ Qt, const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    const int n = a.g.n;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < a.NP;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int lane = (int)(idx & 31);
        const size_t slot = idx >> 5;
        const int t = (int)(slot / a.NL), l = (int)(slot % a.NL);
        const LaneGeo G = lane_geo(a, t, lane);
        double rv[3] = {0.0, 0.0, 0.0};
        if (lane_active(a, G, l)) {
            const int c = G.cbase + l;
#pragma unroll
            for (int e = 0; e < 3; ++e) rv[e] = r[(size_t)e * n + c];
        }
        const double* D = P + slot * (NPE * 32) + lane;
        double* q = Qt + slot * 96 + lane;
#pragma unroll
        for (int row = 0; row < 3; ++row) {
            double v = D[(3 * row) * 32] * rv[0];
            v = fma(D[(3 * row + 1) * 32], rv[1], v);
            v = fma(D[(3 * row + 2) * 32], rv[2], v);
            q[row * 32] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// a8 forward sweep: Yt = (L_A + D)^-1 r, from Qt = D^-1 r; Yt in tile order.
// Row warp rw of a level: acc = q[rw] - L_x[rw][:] y_{i-1} - L_y[rw][:] y_{j-1}
// - L_z[rw][:] y_{k-1} (ten FP64 operations in two chains).  A stage is the
// level's three scaled lower blocks and q; the helper stages the face values
// and issues the bulk copies.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SW_THREADS, 2)
k_fwd64(SweepArgs A, const double* __restrict__ P, const double* __restrict__ Qt,
        double* __restrict__ Yt, double* __restrict__ fJ, double* __restrict__ fK,
        const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    extern __shared__ __align__(128) double smem[];
    double* ring = smem;                                   // [S64][STAGE]
    double* ysh = ring + S64 * STAGE;                      // [2][3][HK][HJ]
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(ysh + 2 * YBUF);
    int* tiles = reinterpret_cast<int*>(bar + S64);        // [MAX_CTA_TILES]
    const TileArgs& a = A.a;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int jj = lane % TJ, kk = lane / TJ;
    const int NL = a.NL;
    const int ntiles = blockIdx.x < a.T ? (a.T - 1 - blockIdx.x) / A.G + 1 : 0;
    const long long total = (long long)ntiles * NL;
    for (int q = threadIdx.x; q < ntiles; q += SW_THREADS) tiles[q] = A.order[blockIdx.x + q * A.G];
    for (int q = threadIdx.x; q < 2 * YBUF; q += SW_THREADS) ysh[q] = 0.0;
    __syncthreads();
    // issue cursor (helper lane 0): stage (tile m, level l) copies slot t NL + l
    StageCursor ic{0, 0};
    size_t islot = (size_t)tiles[0] * NL;
    long long issued = 0;
    auto issue = [&]() {
        const int st = (int)(issued % S64);
        mb_expect(&bar[st], STAGE * 8);
        double* dst = ring + (size_t)st * STAGE;
        bulk_g2s(dst, P + islot * (NPE * 32) + 9 * 32, BLK_ENT * 32 * 8, &bar[st]);
        bulk_g2s(dst + BLK_ENT * 32, Qt + islot * 96, 96 * 8, &bar[st]);
        ++issued;
        advance(ic, NL);
        if (ic.l == 0) {
            if (ic.m < ntiles) islot = (size_t)tiles[ic.m] * NL;
        } else {
            ++islot;
        }
    };
    if (threadIdx.x == HELPER * 32) {
        for (int d = 0; d < S64; ++d) mb_init(&bar[d], 1);
        mb_fence_init();
        while (issued < S64 - 1 && issued < total) issue();
    }
    __syncthreads();
    if (total == 0) return;

    if (warp == HELPER) {
        // ---- helper: face values and the ring -------------------------------
        StageCursor nx{0, 0};   // the stage being prepared
        LaneGeo G = lane_geo(a, tiles[0], lane);
        FaceLane F = face_lane_fwd(a, G, lane, fJ, fK);
        double fv[3] = {0.0, 0.0, 0.0};
        auto load_faces = [&](int l) {
            const double* sl = face_at(F, l, a.g.nx);
#pragma unroll
            for (int e = 0; e < 3; ++e) fv[e] = sl ? ld_relaxed(sl + e) : 0.0;
        };
        auto prepare = [&](long long g) {   // face values of stage g into the plane it reads
            double* sl = face_at(F, nx.l, a.g.nx);
            if (sl) take_slot(sl, fv, a.err);
            if (F.hp >= 0) {
                double* yb = ysh + (((int)(g & 1)) ^ 1) * YBUF + F.hp;
                yb[0] = fv[0];
                yb[YPL] = fv[1];
                yb[2 * YPL] = fv[2];
            }
            advance(nx, NL);
            if (g + 1 < total) {
                if (nx.l == 0) {
                    G = lane_geo(a, tiles[nx.m], lane);
                    F = face_lane_fwd(a, G, lane, fJ, fK);
                }
                load_faces(nx.l);
            }
        };
        // A tile's first stage is prepared only after the previous tile has
        // finished (the barrier before it): the helper then waits only for
        // tiles earlier in the list than the one the CTA is working on.
        load_faces(0);
        long long g = 0;
        for (int m = 0; m < ntiles; ++m) {
            prepare(g);
            __syncthreads();
            for (int l = 0; l < NL; ++l, ++g) {
                if (lane == 0 && issued < total) issue();
                if (l + 1 < NL) prepare(g + 1);
                __syncthreads();
            }
        }
        return;
    }

    // ---- row warps ---------------------------------------------------------
    const int rw = warp;
    const int op = (kk + 1) * HJ + jj + 1;   // this lane in the padded plane
    long long g = 0;
    for (int m = 0; m < ntiles; ++m) {
        __syncthreads();   // the helper has prepared the tile's first stage
        const LaneGeo G = lane_geo(a, tiles[m], lane);
        const bool feedJ = G.valid && jj == TJ - 1 && G.J + 1 < a.NJ && !ycut(a, (G.J + 1) * TJ);
        const bool feedK = G.valid && kk == TK - 1 && G.K + 1 < a.NK && !zcut(a, (G.K + 1) * TK);
        double* yout = Yt + ((size_t)G.t * NL * 3 + rw) * 32 + lane;
        double* fjo = fJ + jslot(a, G.t, 0, kk, 3) + rw - (size_t)G.l0 * TK * 3;
        double* fko = fK + kslot(a, G.t, 0, jj, 3) + rw - (size_t)G.l0 * TJ * 3;
        for (int l = 0; l < NL; ++l, ++g) {
            const int st = (int)(g % S64);
            mb_wait(&bar[st], (unsigned)((g / S64) & 1), a.err);
            const double* L = ring + (size_t)st * STAGE + 3 * rw * 32 + lane;   // row rw of D^-1 A_-x
            const double* yb = ysh + (((int)(g & 1)) ^ 1) * YBUF + op;
            // three independent chains (q and the -x block, the -y block, the -z
            // block) of three dependent FP64 operations each, then two adds
            double u = ring[(size_t)st * STAGE + (BLK_ENT + rw) * 32 + lane];
            double v = -L[9 * 32] * yb[-1];
            double w = -L[18 * 32] * yb[-HJ];
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) u = fma(-L[s2 * 32], yb[s2 * YPL], u);          // -x
#pragma unroll
            for (int s2 = 1; s2 < 3; ++s2) v = fma(-L[(9 + s2) * 32], yb[s2 * YPL - 1], v);   // -y
#pragma unroll
            for (int s2 = 1; s2 < 3; ++s2) w = fma(-L[(18 + s2) * 32], yb[s2 * YPL - HJ], w); // -z
            const bool act = lane_active(a, G, l);
            const double acc = act ? u + (v + w) : 0.0;
            ysh[(int)(g & 1) * YBUF + rw * YPL + op] = acc;
            yout[(size_t)l * 96] = acc;
            if (act && feedJ) st_relaxed(fjo + (size_t)l * TK * 3, acc);
            if (act && feedK) st_relaxed(fko + (size_t)l * TJ * 3, acc);
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// a8 backward sweep: z = (D + U_A)^-1 D y, y from Yt (tile order), z natural.
// Levels run downward; the tile list is the forward list reversed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SW_THREADS, 2)
k_bwd64(SweepArgs A, const double* __restrict__ P, const double* __restrict__ Yt,
        double* __restrict__ z, double* __restrict__ fJ, double* __restrict__ fK,
        const KrylovScalars* __restrict__ ks) {
    if (ks_skip_t(ks)) return;
    extern __shared__ __align__(128) double smem[];
    double* ring = smem;                                   // [S64][STAGE]
    double* ysh = ring + S64 * STAGE;                      // [2][3][HK][HJ]
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(ysh + 2 * YBUF);
    int* tiles = reinterpret_cast<int*>(bar + S64);        // [MAX_CTA_TILES]
    const TileArgs& a = A.a;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int jj = lane % TJ, kk = lane / TJ;
    const int NL = a.NL, n = a.g.n;
    const int ntiles = blockIdx.x < a.T ? (a.T - 1 - blockIdx.x) / A.G + 1 : 0;
    const long long total = (long long)ntiles * NL;
    for (int q = threadIdx.x; q < ntiles; q += SW_THREADS) tiles[q] = A.order[blockIdx.x + q * A.G];
    for (int q = threadIdx.x; q < 2 * YBUF; q += SW_THREADS) ysh[q] = 0.0;
    __syncthreads();
    // issue cursor: stage (tile m, step l) copies slot t NL + NL - 1 - l
    StageCursor ic{0, 0};
    size_t islot = (size_t)tiles[0] * NL + NL - 1;
    long long issued = 0;
    auto issue = [&]() {
        const int st = (int)(issued % S64);
        mb_expect(&bar[st], STAGE * 8);
        double* dst = ring + (size_t)st * STAGE;
        bulk_g2s(dst, P + islot * (NPE * 32) + 36 * 32, BLK_ENT * 32 * 8, &bar[st]);
        bulk_g2s(dst + BLK_ENT * 32, Yt + islot * 96, 96 * 8, &bar[st]);
        ++issued;
        advance(ic, NL);
        if (ic.l == 0) {
            if (ic.m < ntiles) islot = (size_t)tiles[ic.m] * NL + NL - 1;
        } else {
            --islot;
        }
    };
    if (threadIdx.x == HELPER * 32) {
        for (int d = 0; d < S64; ++d) mb_init(&bar[d], 1);
        mb_fence_init();
        while (issued < S64 - 1 && issued < total) issue();
    }
    __syncthreads();
    if (total == 0) return;

    if (warp == HELPER) {
        StageCursor nx{0, 0};
        LaneGeo G = lane_geo(a, tiles[0], lane);
        FaceLane F = face_lane_bwd(a, G, lane, fJ, fK);
        double fv[3] = {0.0, 0.0, 0.0};
        auto load_faces = [&](int l) {
            const double* sl = face_at(F, l, a.g.nx);
#pragma unroll
            for (int e = 0; e < 3; ++e) fv[e] = sl ? ld_relaxed(sl + e) : 0.0;
        };
        auto prepare = [&](long long g) {
            double* sl = face_at(F, NL - 1 - nx.l, a.g.nx);
            if (sl) take_slot(sl, fv, a.err);
            if (F.hp >= 0) {
                double* yb = ysh + (((int)(g & 1)) ^ 1) * YBUF + F.hp;
                yb[0] = fv[0];
                yb[YPL] = fv[1];
                yb[2 * YPL] = fv[2];
            }
            advance(nx, NL);
            if (g + 1 < total) {
                if (nx.l == 0) {
                    G = lane_geo(a, tiles[nx.m], lane);
                    F = face_lane_bwd(a, G, lane, fJ, fK);
                }
                load_faces(NL - 1 - nx.l);
            }
        };
        load_faces(NL - 1);
        long long g = 0;
        for (int m = 0; m < ntiles; ++m) {   // first stage of a tile: as in the forward sweep
            prepare(g);
            __syncthreads();
            for (int step = 0; step < NL; ++step, ++g) {
                if (lane == 0 && issued < total) issue();
                if (step + 1 < NL) prepare(g + 1);
                __syncthreads();
            }
        }
        return;
    }

    const int rw = warp;
    const int op = kk * HJ + jj;   // interior at [kk][jj], borders at row TK and column TJ
    long long g = 0;
    for (int m = 0; m < ntiles; ++m) {
        __syncthreads();
        const LaneGeo G = lane_geo(a, tiles[m], lane);
        const bool feedJ = G.valid && jj == 0 && G.J > 0 && !ycut(a, G.J * TJ);
        const bool feedK = G.valid && kk == 0 && G.K > 0 && !zcut(a, G.K * TK);
        double* fjo = fJ + jslot(a, G.t, 0, kk, 3) + rw - (size_t)G.l0 * TK * 3;
        double* fko = fK + kslot(a, G.t, 0, jj, 3) + rw - (size_t)G.l0 * TJ * 3;
        double* zo = z + (size_t)rw * n + G.cbase;
        for (int step = 0; step < NL; ++step, ++g) {
            const int l = NL - 1 - step;
            const int st = (int)(g % S64);
            mb_wait(&bar[st], (unsigned)((g / S64) & 1), a.err);
            const double* U = ring + (size_t)st * STAGE + 3 * rw * 32 + lane;
            const double* yb = ysh + (((int)(g & 1)) ^ 1) * YBUF + op;
            // three independent chains (y and the +x block, the +y block, the +z
            // block), then two adds
            double u = ring[(size_t)st * STAGE + (BLK_ENT + rw) * 32 + lane];
            double v = -U[9 * 32] * yb[1];
            double w = -U[18 * 32] * yb[HJ];
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) u = fma(-U[s2 * 32], yb[s2 * YPL], u);            // +x
#pragma unroll
            for (int s2 = 1; s2 < 3; ++s2) v = fma(-U[(9 + s2) * 32], yb[s2 * YPL + 1], v);   // +y
#pragma unroll
            for (int s2 = 1; s2 < 3; ++s2) w = fma(-U[(18 + s2) * 32], yb[s2 * YPL + HJ], w); // +z
            const bool act = lane_active(a, G, l);
            const double acc = act ? u + (v + w) : 0.0;
            ysh[(int)(g & 1) * YBUF + rw * YPL + op] = acc;
            if (act) {
                zo[l] = acc;
                if (feedJ) st_relaxed(fjo + (size_t)l * TK * 3, acc);
                if (feedK) st_relaxed(fko + (size_t)l * TJ * 3, acc);
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
constexpr size_t SWEEP_SMEM = sizeof(double) * (S64 * STAGE + 2 * YBUF) +
                              sizeof(unsigned long long) * S64 + sizeof(int) * MAX_CTA_TILES;

// Tiles in the order a wavefront reaches them: the level at which tile
// (J, K) can start is TJ (J - J0) + TK (K - K0) within its block-Jacobi box
// (J0, K0: the box's first tile), ties by (K, J).  Every dependency of a tile
// (J - 1, K), (J, K - 1) in the same box comes earlier in the list.
std::vector<int> sweep_tile_order(const TileArgs& a) {
    const int bj = a.ysub > 0 ? a.ysub / TJ : a.NJ, bk = a.zsub > 0 ? a.zsub / TK : a.NK;
    std::vector<int> t(a.T);
    for (int q = 0; q < a.T; ++q) t[q] = q;
    auto key = [&](int q) {
        const int J = q % a.NJ, K = q / a.NJ;
        return std::make_tuple(TJ * (J % bj) + TK * (K % bk), K, J);
    };
    std::sort(t.begin(), t.end(), [&](int x, int y) { return key(x) < key(y); });
    return t;
}

// Persistent CTAs of the sweeps: sweep_ctas_per_sm per SM (1 or 2; with two,
// the row warps of the two CTAs share the SM sub-partitions' FP64 pipes).
int sweep_ctas(const bo_sim* s) {
    int dev, sms;
    BO_CUDA(cudaGetDevice(&dev));
    BO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return std::min(tile_args(s).T, s->sweep_ctas_per_sm * sms);
}

void setup_sweeps64(bo_sim* s) {
    BO_CUDA(cudaFuncSetAttribute(k_fwd64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM));
    BO_CUDA(cudaFuncSetAttribute(k_bwd64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM));
    // two CTAs per SM need the whole shared-memory carveout
    for (const void* k : {(const void*)k_fwd64, (const void*)k_bwd64})
        BO_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    int dev, sms, pf = 0, pb = 0;
    BO_CUDA(cudaGetDevice(&dev));
    BO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pf, k_fwd64, SW_THREADS, SWEEP_SMEM));
    BO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, k_bwd64, SW_THREADS, SWEEP_SMEM));
    if ((long long)std::min(pf, pb) * sms < sweep_ctas(s))
        fail(BO_ERR_INVALID_ARG, "sweep CTAs cannot all be resident at once");
    const TileArgs a = tile_args(s);
    if ((a.T + sweep_ctas(s) - 1) / sweep_ctas(s) > MAX_CTA_TILES)
        fail(BO_ERR_INVALID_ARG, "grid too large: more wavefront tiles per CTA than the sweeps hold");
    update_sweep_order(s);
}

// Tile lists of both directions for the current block-Jacobi boxes.
void update_sweep_order(bo_sim* s) {
    const TileArgs a = tile_args(s);
    std::vector<int> f = sweep_tile_order(a);
    std::vector<int> both(2 * (size_t)a.T);
    for (int q = 0; q < a.T; ++q) {
        both[q] = f[q];
        both[a.T + q] = f[a.T - 1 - q];
    }
    BO_CUDA(cudaMemcpy(s->d_order, both.data(), sizeof(int) * both.size(), cudaMemcpyHostToDevice));
}

void enqueue_fwd64(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks) {
    SweepArgs A{tile_args(s), s->d_order, sweep_ctas(s)};
    k_q_tiles<<<152 * 8, 256, 0, st>>>(A.a, (const double*)s->d_P, r, s->d_qt, ks);
    count_launch(s, st);
    launch_coop_smem(st, A.G, SW_THREADS, SWEEP_SMEM, k_fwd64, A, (const double*)s->d_P,
                     (const double*)s->d_qt, s->d_yt, faceJ3(s), faceK3(s), ks);
    count_launch(s, st);
}

void enqueue_bwd64(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks) {
    SweepArgs A{tile_args(s), s->d_order + tile_args(s).T, sweep_ctas(s)};
    launch_coop_smem(st, A.G, SW_THREADS, SWEEP_SMEM, k_bwd64, A, (const double*)s->d_P,
                     (const double*)s->d_yt, z, faceJ3(s), faceK3(s), ks);
    count_launch(s, st);
}

}  // namespace bo
