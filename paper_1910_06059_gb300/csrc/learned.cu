// Learned correction of the ILU(0) preconditioner (an extension of the
// ILU(0)-preconditioned BiCGStab of arXiv 1910.06059 Section 2.3.1):
//     z = M^-1 r + delta(r),  delta_c = sigma_c * (W_c rhat_c),  W_c = N(f_c)
// N: 63 -> 128 -> 128 -> 9 ReLU MLP of the 63 normalised entries of the
// cell's Jacobian row (diagonal block, then the -x, +x, -y, +y, -z, +z
// blocks); W_c[v][e] = N[3 v + e] is a 3x3 matrix acting on the cell's
// row-scaled residual:
//     sigma_c      = (1e6 Pa, 0.05, 0.05 | 5)   (x = s_g | r_go)
//     rho_{c,e}    = max_v |A_cc[e][v]| sigma_{c,v}
//     F_{c,b}[e,v] = A_{c,b}[e][v] sigma_{nb,v} / rho_{c,e}
//     rhat_c[e]    = r_c[e] / rho_{c,e}
// The correction is linear in r: for one Jacobian the preconditioner is one
// fixed linear map, which BiCGStab's recurrences need.
//
// The network runs once per factorisation, on the tensor cores (BF16 weights
// and activations, FP32 accumulation, mma.sync m16n8k16 with the accumulators
// of one layer re-packed in registers as the A operand of the next; each warp
// takes 16 cells, a CTA keeps the weights in shared memory), and stores W_c.
// Each application inside BiCGStab is then a per-cell 3x3 product.
//
// Training minimises L = ||e - A delta||^2 / ||r||^2, e = r - A M^-1 r, over
// residuals the solver itself produces (the recurrence residuals of its
// BiCGStab iterations), in FP32 on the CUDA cores: a forward kernel (delta),
// the plain Jacobian operator and its transpose, a backward kernel that
// recomputes the forward pass per chunk of cells and accumulates the weight
// gradients in registers, and Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace bo {

constexpr int MLH = 128, MLF = 63, MLO = 9;
constexpr float SIG_P = 1e6f, SIG_S = 0.05f, SIG_SG = 0.05f, SIG_RGO = 5.0f;
// flat parameter offsets: W1[128][63], b1, W2[128][128], b2, W3[9][128], b3
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLH * MLF, OFF_W2 = OFF_B1 + MLH,
              OFF_B2 = OFF_W2 + MLH * MLH, OFF_W3 = OFF_B2 + MLH, OFF_B3 = OFF_W3 + MLO * MLH,
              NPARAM = OFF_B3 + MLO;
static_assert(NPARAM == BO_LEARN_NPARAM, "parameter count");

// BF16 weight image in shared memory, n-major with padded k so that the
// 32-bit operand loads of a warp hit 32 distinct banks (row strides of 36 and
// 68 words).  Layer 1 has K = 64 (63 features and a zero), layer 3 N = 16
// (9 outputs and zero rows).
constexpr int K1 = 64, K1P = 72, K2P = 136, N3 = 16;
constexpr int W1S = MLH * K1P, W2S = MLH * K2P, W3S = N3 * K2P;
constexpr int WBF_ELEMS = W1S + W2S + W3S;              // 28,800 bf16 (56.3 KB)
constexpr int XS = 16 * K1P;                             // per-warp feature tile (bf16)
constexpr int INF_WARPS = 4;
constexpr size_t INF_SMEM = (size_t)(WBF_ELEMS + INF_WARPS * XS) * 2 + (2 * MLH + N3) * 4 + 64;

constexpr int ML_BS = 256;
constexpr int ML_GRID = 152 * 4;                         // fixed grid of the reductions

static __nv_bfloat16* wbf_of(bo_sim* s) { return static_cast<__nv_bfloat16*>(s->d_ml_wbf); }
static __nv_bfloat16* feat_of(bo_sim* s) { return static_cast<__nv_bfloat16*>(s->d_ml_feat); }

// ---------------------------------------------------------------------------
// Features of the last assembly
// ---------------------------------------------------------------------------
__device__ __forceinline__ float sig_x(uint8_t flag) { return flag == 0 ? SIG_SG : SIG_RGO; }

// Block features (BF16 for the network, FP32 for training when ff is given;
// [n][64], entry 63 zero) and per-cell (1/rho_0, 1/rho_1, 1/rho_2, sigma_x).
__global__ void __launch_bounds__(ML_BS)
k_ml_feat(Geom g, const double* __restrict__ A, const uint8_t* __restrict__ flag,
          __nv_bfloat16* __restrict__ fbf, float* __restrict__ ff, float4* __restrict__ cell) {
    const int n = g.n, plane = g.nx * g.ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / plane;
        const int nbc[7] = {c, c - 1, c + 1, c - g.nx, c + g.nx, c - plane, c + plane};
        const bool has[7] = {true, i > 0, i + 1 < g.nx, j > 0, j + 1 < g.ny, k > 0, k + 1 < g.nz};
        const double sc[3] = {SIG_P, SIG_S, sig_x(flag[c])};
        double rinv[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            double m = 0.0;
#pragma unroll
            for (int v = 0; v < 3; ++v) m = fmax(m, fabs(A[(size_t)(3 * e + v) * n + c]) * sc[v]);
            rinv[e] = m > 0.0 ? 1.0 / m : 0.0;
        }
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            const double sx = has[b] ? (double)sig_x(flag[nbc[b]]) : 0.0;
            const double sn[3] = {SIG_P, SIG_S, sx};
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const double a =
                        has[b] ? A[(size_t)(b * 9 + 3 * e + v) * n + c] * sn[v] * rinv[e] : 0.0;
                    const size_t q = (size_t)c * 64 + b * 9 + 3 * e + v;
                    fbf[q] = __double2bfloat16(a);
                    if (ff) ff[q] = (float)a;
                }
        }
        fbf[(size_t)c * 64 + 63] = __float2bfloat16(0.f);
        if (ff) ff[(size_t)c * 64 + 63] = 0.f;
        cell[c] = make_float4((float)rinv[0], (float)rinv[1], (float)rinv[2], sig_x(flag[c]));
    }
}

// ---------------------------------------------------------------------------
// The network on the tensor cores (once per factorisation)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    unsigned u;
    memcpy(&u, &v, 4);
    return u;
}

__device__ __forceinline__ unsigned ld_u32(const __nv_bfloat16* p) {
    return *reinterpret_cast<const unsigned*>(p);
}

// W[q][c] = N(f_c)[q], q < 9, for every cell.
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4):
//   A regs {X[g][2t..], X[g+8][2t..], X[g][2t+8..], X[g+8][2t+8..]}
//   B regs {W[n=g][k=2t..], W[g][2t+8..]}   (W stored n-major: B = W^T)
//   C regs {C[g][2t], C[g][2t+1], C[g+8][2t], C[g+8][2t+1]}
__global__ void __launch_bounds__(32 * INF_WARPS)
k_ml_net(int n, const __nv_bfloat16* __restrict__ feat, const __nv_bfloat16* __restrict__ wbf,
         const float* __restrict__ theta, float* __restrict__ Wc) {
    extern __shared__ __align__(16) unsigned char ml_smem[];
    __nv_bfloat16* W1s = reinterpret_cast<__nv_bfloat16*>(ml_smem);
    __nv_bfloat16* W2s = W1s + W1S;
    __nv_bfloat16* W3s = W2s + W2S;
    __nv_bfloat16* Xall = W3s + W3S;
    float* bias = reinterpret_cast<float*>(Xall + INF_WARPS * XS);   // b1[128], b2[128], b3[16]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {   // weights: 16-byte copies of the prepared image
        const uint4* src = reinterpret_cast<const uint4*>(wbf);
        uint4* dst = reinterpret_cast<uint4*>(W1s);
        for (int q = tid; q < WBF_ELEMS / 8; q += blockDim.x) dst[q] = src[q];
        for (int q = tid; q < 2 * MLH + N3; q += blockDim.x)
            bias[q] = q < MLH ? theta[OFF_B1 + q]
                              : (q < 2 * MLH ? theta[OFF_B2 + q - MLH]
                                             : (q - 2 * MLH < MLO ? theta[OFF_B3 + q - 2 * MLH] : 0.f));
    }
    __syncthreads();
    const int gq = lane >> 2, tq = lane & 3;
    __nv_bfloat16* X = Xall + warp * XS;
    const int stride = gridDim.x * INF_WARPS * 16;
    for (int base = (blockIdx.x * INF_WARPS + warp) * 16; base < n; base += stride) {
        // stage 16 cells x 64 features (entry 63 is zero)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = lane + 32 * q, row = idx >> 3, ch = idx & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (base + row < n)
                v = *reinterpret_cast<const uint4*>(feat + (size_t)(base + row) * 64 + ch * 8);
            *reinterpret_cast<uint4*>(X + row * K1P + ch * 8) = v;
        }
        __syncwarp();
        // layer 1: K = 64
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const float b0 = bias[8 * nt + 2 * tq], b1v = bias[8 * nt + 2 * tq + 1];
            acc[nt][0] = b0; acc[nt][1] = b1v; acc[nt][2] = b0; acc[nt][3] = b1v;
        }
#pragma unroll
        for (int s = 0; s < K1 / 16; ++s) {
            unsigned a[4];
            a[0] = ld_u32(X + gq * K1P + 16 * s + 2 * tq);
            a[1] = ld_u32(X + (gq + 8) * K1P + 16 * s + 2 * tq);
            a[2] = ld_u32(X + gq * K1P + 16 * s + 8 + 2 * tq);
            a[3] = ld_u32(X + (gq + 8) * K1P + 16 * s + 8 + 2 * tq);
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const __nv_bfloat16* w = W1s + (8 * nt + gq) * K1P + 16 * s + 2 * tq;
                mma_bf16(acc[nt], a, ld_u32(w), ld_u32(w + 8));
            }
        }
        // ReLU, BF16: the accumulators of n-tiles 2s, 2s+1 are the A operand of k-step s
        unsigned h[8][4];
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            h[s][0] = pack_bf16(fmaxf(acc[2 * s][0], 0.f), fmaxf(acc[2 * s][1], 0.f));
            h[s][1] = pack_bf16(fmaxf(acc[2 * s][2], 0.f), fmaxf(acc[2 * s][3], 0.f));
            h[s][2] = pack_bf16(fmaxf(acc[2 * s + 1][0], 0.f), fmaxf(acc[2 * s + 1][1], 0.f));
            h[s][3] = pack_bf16(fmaxf(acc[2 * s + 1][2], 0.f), fmaxf(acc[2 * s + 1][3], 0.f));
        }
        // layer 2: K = 128
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const float b0 = bias[MLH + 8 * nt + 2 * tq], b1v = bias[MLH + 8 * nt + 2 * tq + 1];
            acc[nt][0] = b0; acc[nt][1] = b1v; acc[nt][2] = b0; acc[nt][3] = b1v;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const __nv_bfloat16* w = W2s + (8 * nt + gq) * K2P + 16 * s + 2 * tq;
                mma_bf16(acc[nt], h[s], ld_u32(w), ld_u32(w + 8));
            }
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            h[s][0] = pack_bf16(fmaxf(acc[2 * s][0], 0.f), fmaxf(acc[2 * s][1], 0.f));
            h[s][1] = pack_bf16(fmaxf(acc[2 * s][2], 0.f), fmaxf(acc[2 * s][3], 0.f));
            h[s][2] = pack_bf16(fmaxf(acc[2 * s + 1][0], 0.f), fmaxf(acc[2 * s + 1][1], 0.f));
            h[s][3] = pack_bf16(fmaxf(acc[2 * s + 1][2], 0.f), fmaxf(acc[2 * s + 1][3], 0.f));
        }
        // layer 3: two n-tiles of 8 outputs (rows 9..15 of W3 are zero)
        float o[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float b0 = bias[2 * MLH + 8 * nt + 2 * tq], b1v = bias[2 * MLH + 8 * nt + 2 * tq + 1];
            o[nt][0] = b0; o[nt][1] = b1v; o[nt][2] = b0; o[nt][3] = b1v;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const __nv_bfloat16* w = W3s + (8 * nt + gq) * K2P + 16 * s + 2 * tq;
                mma_bf16(o[nt], h[s], ld_u32(w), ld_u32(w + 8));
            }
        // outputs q = 8 nt + 2 t (+1) of rows g and g + 8
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int c = base + gq + 8 * half;
                const int q0 = 8 * nt + 2 * tq;
                if (c < n) {
                    if (q0 < MLO) Wc[(size_t)q0 * n + c] = o[nt][2 * half];
                    if (q0 + 1 < MLO) Wc[(size_t)(q0 + 1) * n + c] = o[nt][2 * half + 1];
                }
            }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// The same network on the fifth-generation tensor cores (tcgen05).  A CTA
// takes 128 cells at a time (the MMA's M = 128); each layer is one chain of
// tcgen05.mma kind::f16 -- BF16 operands in shared memory, FP32 accumulators
// in tensor memory -- issued by one thread and completed on an mbarrier; the
// layer's epilogue reads the accumulator rows back with tcgen05.ld (thread t
// of warp w holds row 32 w + t), adds the bias, applies ReLU, rounds to BF16
// and writes the next layer's operand tile.  Tensor memory: 256 columns,
// layer 1 in columns 0..127, layer 2 in 128..255, layer 3 in 0..15.
//
// Operand tiles are K-major without swizzling, in 8-row x 16-byte core
// matrices: row r, column k of a tile with K columns sits at byte
// (r / 8) SBO + (k / 8) 128 + (r % 8) 16 + (k % 8) 2, SBO = (K / 8) 128, so
// the leading (K-direction) core-matrix offset is 128 and one MMA (K = 16,
// two core matrices) advances the start address by 256 bytes.
// ---------------------------------------------------------------------------
constexpr int TC_BS = 128;   // four warps: one per 32 accumulator lanes
constexpr int TC_W1 = 0, TC_W2 = TC_W1 + 128 * 64 * 2, TC_W3 = TC_W2 + 128 * 128 * 2,
              TC_X = TC_W3 + 16 * 128 * 2, TC_H = TC_X + 128 * 64 * 2,
              TC_BIAS = TC_H + 128 * 128 * 2, TC_MBAR = TC_BIAS + (2 * MLH + N3) * 4,
              TC_TADDR = TC_MBAR + 8, TC_FLAG = TC_TADDR + 4, TC_SMEM = TC_FLAG + 4;
constexpr uint32_t TC_COLS = 256;
constexpr long long TC_WAIT_LIMIT = 1LL << 24;   // polls of a layer's completion

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start, leading and stride byte offsets
// (each >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_proxy_fence() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ bool tc_mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
// byte offset of (row r, column k) in a K-major no-swizzle tile of K columns
__device__ __forceinline__ uint32_t tc_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
// copy rows x K of a row-major BF16 matrix (row stride ld elements, 16-byte
// aligned rows) into a tile; rows >= valid are zero
__device__ __forceinline__ void tc_fill(unsigned char* tile, const __nv_bfloat16* src, int rows,
                                        int K, int ld, int valid) {
    const int chunks = K / 8;
    for (int q = threadIdx.x; q < rows * chunks; q += blockDim.x) {
        const int r = q / chunks, kc = q % chunks;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < valid) v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + kc * 8);
        *reinterpret_cast<uint4*>(tile + tc_off(r, kc * 8, K)) = v;
    }
}

// Thread 0 waits (bounded) for the layer's MMAs; the outcome reaches every
// thread through shared memory, so all threads take the same path.
__device__ __forceinline__ bool tc_layer_done(uint32_t mbar, uint32_t parity, int* flag) {
    if (threadIdx.x == 0) {
        long long q = 0;
        while (!tc_mbar_try(mbar, parity) && ++q < TC_WAIT_LIMIT) {
        }
        *flag = q < TC_WAIT_LIMIT ? 1 : 0;
    }
    __syncthreads();
    const bool ok = *reinterpret_cast<volatile int*>(flag) != 0;
    tc_fence_after();
    return ok;
}

// accumulator columns [col, col + ncols) of this thread's row + bias, ReLU,
// BF16 into the hidden tile (K = 128)
__device__ __forceinline__ void tc_hidden(uint32_t taddr, int col, const float* bias,
                                          unsigned char* H) {
    const int warp = threadIdx.x >> 5, row = threadIdx.x;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
#pragma unroll 1
    for (int cb = 0; cb < 8; ++cb) {
        float v[16];
        tc_ld16(taddr + lane_base + (uint32_t)(col + 16 * cb), v);
        unsigned u[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            u[k] = pack_bf16(fmaxf(v[2 * k] + bias[16 * cb + 2 * k], 0.f),
                             fmaxf(v[2 * k + 1] + bias[16 * cb + 2 * k + 1], 0.f));
        *reinterpret_cast<uint4*>(H + tc_off(row, 16 * cb, 128)) = make_uint4(u[0], u[1], u[2], u[3]);
        *reinterpret_cast<uint4*>(H + tc_off(row, 16 * cb + 8, 128)) = make_uint4(u[4], u[5], u[6], u[7]);
    }
}

// W[q][c] = N(f_c)[q], q < 9, for every cell; *bad is set if a layer's MMAs
// did not complete within the wait limit.
__global__ void __launch_bounds__(TC_BS)
k_ml_net_tc(int n, const __nv_bfloat16* __restrict__ feat, const __nv_bfloat16* __restrict__ wbf,
            const float* __restrict__ theta, float* __restrict__ Wc, int* __restrict__ bad) {
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    unsigned char* W1 = tc_sm + TC_W1;
    unsigned char* W2 = tc_sm + TC_W2;
    unsigned char* W3 = tc_sm + TC_W3;
    unsigned char* X = tc_sm + TC_X;
    unsigned char* H = tc_sm + TC_H;
    float* bias = reinterpret_cast<float*>(tc_sm + TC_BIAS);   // b1[128], b2[128], b3[16]
    const uint32_t mbar = tc_smem(tc_sm + TC_MBAR);
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(tc_sm + TC_TADDR);
    int* flag = reinterpret_cast<int*>(tc_sm + TC_FLAG);
    const int warp = threadIdx.x >> 5;
    // weights into the tile layout, biases
    tc_fill(W1, wbf, 128, 64, K1P, 128);
    tc_fill(W2, wbf + W1S, 128, 128, K2P, 128);
    tc_fill(W3, wbf + W1S + W2S, 16, 128, K2P, 16);
    for (int q = threadIdx.x; q < 2 * MLH + N3; q += blockDim.x)
        bias[q] = q < MLH ? theta[OFF_B1 + q]
                          : (q < 2 * MLH ? theta[OFF_B2 + q - MLH]
                                         : (q - 2 * MLH < MLO ? theta[OFF_B3 + q - 2 * MLH] : 0.f));
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(taddr_slot)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *taddr_slot;
    constexpr uint32_t ID1 = tc_idesc(128, 128), ID3 = tc_idesc(128, 16);
    uint32_t parity = 0;
    bool ok = true;
    for (int base = blockIdx.x * 128; base < n && ok; base += gridDim.x * 128) {
        // stage 128 cells x 64 features
        tc_fill(X, feat + (size_t)base * 64, 128, 64, 64, min(128, n - base));
        tc_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {   // layer 1: K = 64 -> accumulator columns 0..127
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < 4; ++s)
                tc_mma(taddr, tc_desc(tc_smem(X) + 256 * s, 128, 1024),
                       tc_desc(tc_smem(W1) + 256 * s, 128, 1024), ID1, s > 0);
            tc_commit(mbar);
        }
        ok = tc_layer_done(mbar, parity, flag);
        parity ^= 1u;
        if (!ok) break;
        tc_hidden(taddr, 0, bias, H);
        tc_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {   // layer 2: K = 128 -> columns 128..255
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < 8; ++s)
                tc_mma(taddr + 128, tc_desc(tc_smem(H) + 256 * s, 128, 2048),
                       tc_desc(tc_smem(W2) + 256 * s, 128, 2048), ID1, s > 0);
            tc_commit(mbar);
        }
        ok = tc_layer_done(mbar, parity, flag);
        parity ^= 1u;
        if (!ok) break;
        tc_hidden(taddr, 128, bias + MLH, H);   // H is free: layer 2 has read it
        tc_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {   // layer 3: N = 16 -> columns 0..15
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < 8; ++s)
                tc_mma(taddr, tc_desc(tc_smem(H) + 256 * s, 128, 2048),
                       tc_desc(tc_smem(W3) + 256 * s, 128, 2048), ID3, s > 0);
            tc_commit(mbar);
        }
        ok = tc_layer_done(mbar, parity, flag);
        parity ^= 1u;
        if (!ok) break;
        float v[16];
        tc_ld16(taddr + ((uint32_t)(32 * warp) << 16), v);
        const int c = base + threadIdx.x;
        if (c < n)
#pragma unroll
            for (int q = 0; q < MLO; ++q) Wc[(size_t)q * n + c] = v[q] + bias[2 * MLH + q];
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(bad, 1);
            long long q = 0;   // the layer still in flight: a second bounded wait
            while (!tc_mbar_try(mbar, parity ^ 1u) && ++q < TC_WAIT_LIMIT) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TC_COLS)
                     : "memory");
    }
}

// z += delta(r): delta_c[v] = sigma_v sum_e W_c[3 v + e] r_c[e] / rho_c[e]
// (ks: skip when the solve has finished).  FP32 products, FP64 accumulation
// into z.
__global__ void __launch_bounds__(ML_BS)
k_ml_apply(int n, const float* __restrict__ Wc, const float4* __restrict__ cell,
           const double* __restrict__ r, double* __restrict__ z, const KrylovScalars* __restrict__ ks) {
    if (ks != nullptr && ks->state != KS_RUN) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const float4 q = cell[c];
        const float rh[3] = {(float)r[c] * q.x, (float)r[(size_t)n + c] * q.y,
                             (float)r[2 * (size_t)n + c] * q.z};
        const float sg[3] = {SIG_P, SIG_S, q.w};
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            float o = Wc[(size_t)(3 * v) * n + c] * rh[0];
            o = fmaf(Wc[(size_t)(3 * v + 1) * n + c], rh[1], o);
            o = fmaf(Wc[(size_t)(3 * v + 2) * n + c], rh[2], o);
            z[(size_t)v * n + c] += (double)(sg[v] * o);
        }
    }
}

// FP32 parameters -> BF16 shared-memory image (zero padding included).
__global__ void k_ml_pack(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < WBF_ELEMS; q += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (q < W1S) {
            const int nn = q / K1P, k = q % K1P;
            if (k < MLF) v = theta[OFF_W1 + nn * MLF + k];
        } else if (q < W1S + W2S) {
            const int p = q - W1S, nn = p / K2P, k = p % K2P;
            if (k < MLH) v = theta[OFF_W2 + nn * MLH + k];
        } else {
            const int p = q - W1S - W2S, nn = p / K2P, k = p % K2P;
            if (nn < MLO && k < MLH) v = theta[OFF_W3 + nn * MLH + k];
        }
        wbf[q] = __float2bfloat16(v);
    }
}

// ---------------------------------------------------------------------------
// Training in FP32 on the CUDA cores
// ---------------------------------------------------------------------------
constexpr int TR_CH = 32;        // cells per chunk
constexpr int TR_BS = 256;
constexpr int TR_GRID = 152;     // one persistent CTA per SM
// shared memory: the FP32 weights with padded rows, W1 [128][65], b1,
// W2 [128][129], b2, W3 [9][128], b3 (odd row strides make both W[j][k] over
// consecutive j and W[q][j] over consecutive j conflict-free), then the
// chunk tiles F [32][63], H1 [32][128], H2 [32][128], dH2, dH1, O / dO [32][9]
constexpr int S1 = MLF + 2, S2 = MLH + 1;
constexpr int SW1 = 0, SB1 = SW1 + MLH * S1, SW2 = SB1 + MLH, SB2 = SW2 + MLH * S2,
              SW3 = SB2 + MLH, SB3 = SW3 + MLO * MLH;
constexpr int TR_WFLOATS = (SB3 + MLO + 3) / 4 * 4;
constexpr int TR_TILE = TR_CH * MLF + 4 * TR_CH * MLH + TR_CH * MLO;
constexpr size_t TR_SMEM = (size_t)(TR_WFLOATS + TR_TILE + 8) * 4;

__device__ __forceinline__ void load_weights_f32(const float* __restrict__ theta, float* W) {
    for (int q = threadIdx.x; q < NPARAM; q += blockDim.x) {
        int d;
        if (q < OFF_B1) d = SW1 + (q / MLF) * S1 + q % MLF;
        else if (q < OFF_W2) d = SB1 + q - OFF_B1;
        else if (q < OFF_B2) d = SW2 + ((q - OFF_W2) / MLH) * S2 + (q - OFF_W2) % MLH;
        else if (q < OFF_W3) d = SB2 + q - OFF_B2;
        else if (q < OFF_B3) d = SW3 + q - OFF_W3;
        else d = SB3 + q - OFF_B3;
        W[d] = theta[q];
    }
    __syncthreads();
}

// Forward pass of the chunk [base, base + TR_CH): F, H1, H2 and the outputs
// O [32][9] in shared memory.  Thread t owns column j = t % 128 of the hidden
// layers for the cells c0 + 2m (c0 = t / 128, m < 16).
__device__ __forceinline__ void tr_forward(int n, int base, const float* __restrict__ ff,
                                           const float* W, float* F, float* H1, float* H2,
                                           float* O) {
    const int tid = threadIdx.x;
    for (int q = tid; q < TR_CH * MLF; q += TR_BS) {
        const int cc = q / MLF, k = q % MLF, c = base + cc;
        F[q] = c < n ? ff[(size_t)c * 64 + k] : 0.f;
    }
    __syncthreads();
    const int j = tid & (MLH - 1), c0 = tid >> 7;
    {
        float a[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) a[m] = W[SB1 + j];
        for (int k = 0; k < MLF; ++k) {
            const float w = W[SW1 + j * S1 + k];
#pragma unroll
            for (int m = 0; m < 16; ++m) a[m] = fmaf(w, F[(c0 + 2 * m) * MLF + k], a[m]);
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) H1[(c0 + 2 * m) * MLH + j] = fmaxf(a[m], 0.f);
    }
    __syncthreads();
    {
        float a[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) a[m] = W[SB2 + j];
        for (int k = 0; k < MLH; ++k) {
            const float w = W[SW2 + j * S2 + k];
#pragma unroll
            for (int m = 0; m < 16; ++m) a[m] = fmaf(w, H1[(c0 + 2 * m) * MLH + k], a[m]);
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) H2[(c0 + 2 * m) * MLH + j] = fmaxf(a[m], 0.f);
    }
    __syncthreads();
    for (int q = tid; q < TR_CH * MLO; q += TR_BS) {
        const int cc = q / MLO, v = q % MLO;
        float a = W[SB3 + v];
        for (int k = 0; k < MLH; ++k) a = fmaf(W[SW3 + v * MLH + k], H2[cc * MLH + k], a);
        O[q] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ float rhat_of(int n, int c, int e, const double* __restrict__ r,
                                         const float4& q) {
    const float ri = e == 0 ? q.x : (e == 1 ? q.y : q.z);
    return (float)r[(size_t)e * n + c] * ri;
}

// delta = sigma (N(f) rhat) for every cell (FP32 network, FP64 output).
__global__ void __launch_bounds__(TR_BS)
k_ml_fwd_f32(int n, const float* __restrict__ ff, const float4* __restrict__ cell,
             const double* __restrict__ r, const float* __restrict__ theta,
             double* __restrict__ delta) {
    extern __shared__ __align__(16) float tr_smem[];
    float* W = tr_smem;
    float* F = W + TR_WFLOATS;
    float* H1 = F + TR_CH * MLF;
    float* H2 = H1 + TR_CH * MLH;
    float* O = H2 + 3 * TR_CH * MLH;   // after the two gradient tiles of the backward kernel
    load_weights_f32(theta, W);
    for (int base = blockIdx.x * TR_CH; base < n; base += gridDim.x * TR_CH) {
        tr_forward(n, base, ff, W, F, H1, H2, O);
        const int tid = threadIdx.x;
        if (tid < TR_CH * 3) {
            const int cc = tid / 3, v = tid % 3, c = base + cc;
            if (c < n) {
                const float4 q = cell[c];
                float a = 0.f;
#pragma unroll
                for (int e = 0; e < 3; ++e) a = fmaf(O[cc * MLO + 3 * v + e], rhat_of(n, c, e, r, q), a);
                const float sg = v == 0 ? SIG_P : (v == 1 ? SIG_S : q.w);
                delta[(size_t)v * n + c] = (double)(sg * a);
            }
        }
        __syncthreads();
    }
}

// Weight gradients for dL/ddelta = dd (FP64 [3][n]); the forward pass is
// recomputed per chunk.  Each thread accumulates its share of dW1, dW2, dW3
// in registers over all its chunks, then adds it to grad once.
__global__ void __launch_bounds__(TR_BS, 1)
k_ml_bwd_f32(int n, const float* __restrict__ ff, const float4* __restrict__ cell,
             const double* __restrict__ r, const float* __restrict__ theta,
             const double* __restrict__ dd, float* __restrict__ grad) {
    extern __shared__ __align__(16) float tr_smem[];
    float* W = tr_smem;
    float* F = W + TR_WFLOATS;
    float* H1 = F + TR_CH * MLF;
    float* H2 = H1 + TR_CH * MLH;
    float* dH2 = H2 + TR_CH * MLH;
    float* dH1 = dH2 + TR_CH * MLH;
    float* O = dH1 + TR_CH * MLH;      // forward outputs, then their gradient dO
    load_weights_f32(theta, W);
    const int tid = threadIdx.x;
    // ownership: dW2 row jr = tid / 2, columns [64 kh, 64 kh + 64);
    //            dW1 row jr, columns kh + 2 m (m < 32, k < 63), kh = tid % 2;
    //            dW3 entries tid + 256 h (h < 5, < 1152)
    const int jr = tid >> 1, kh = tid & 1;
    float gW2[64], gW1[32], gW3[5];
#pragma unroll
    for (int q = 0; q < 64; ++q) gW2[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 32; ++q) gW1[q] = 0.f;
#pragma unroll
    for (int q = 0; q < 5; ++q) gW3[q] = 0.f;
    float gB1 = 0.f, gB2 = 0.f, gB3 = 0.f;
    const int j = tid & (MLH - 1), c0 = tid >> 7;
    for (int base = blockIdx.x * TR_CH; base < n; base += gridDim.x * TR_CH) {
        tr_forward(n, base, ff, W, F, H1, H2, O);
        // dO[cc][3 v + e] = sigma_v dd_v rhat_e
        for (int q = tid; q < TR_CH * MLO; q += TR_BS) {
            const int cc = q / MLO, ve = q % MLO, v = ve / 3, e = ve % 3, c = base + cc;
            float d = 0.f;
            if (c < n) {
                const float4 cq = cell[c];
                const float sg = v == 0 ? SIG_P : (v == 1 ? SIG_S : cq.w);
                d = sg * (float)dd[(size_t)v * n + c] * rhat_of(n, c, e, r, cq);
            }
            O[q] = d;
        }
        __syncthreads();
        // dH2 = (dO W3) * [H2 > 0]
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int cc = c0 + 2 * m;
            float a = 0.f;
#pragma unroll
            for (int v = 0; v < MLO; ++v) a = fmaf(O[cc * MLO + v], W[SW3 + v * MLH + j], a);
            dH2[cc * MLH + j] = H2[cc * MLH + j] > 0.f ? a : 0.f;
        }
        __syncthreads();
        // dH1 = (dH2 W2) * [H1 > 0]: column j of dH1 needs column j of W2
        {
            float a[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) a[m] = 0.f;
            for (int q = 0; q < MLH; ++q) {
                const float w = W[SW2 + q * S2 + j];
#pragma unroll
                for (int m = 0; m < 16; ++m) a[m] = fmaf(dH2[(c0 + 2 * m) * MLH + q], w, a[m]);
            }
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int cc = c0 + 2 * m;
                dH1[cc * MLH + j] = H1[cc * MLH + j] > 0.f ? a[m] : 0.f;
            }
        }
        __syncthreads();
        // weight gradients over the chunk's cells
        for (int cc = 0; cc < TR_CH; ++cc) {
            const float d2 = dH2[cc * MLH + jr];
            const float d1 = dH1[cc * MLH + jr];
#pragma unroll
            for (int q = 0; q < 64; ++q) gW2[q] = fmaf(d2, H1[cc * MLH + 64 * kh + q], gW2[q]);
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (kh + 2 * q < MLF) gW1[q] = fmaf(d1, F[cc * MLF + kh + 2 * q], gW1[q]);
            if (kh == 0) {
                gB1 += d1;
                gB2 += d2;
            }
        }
#pragma unroll
        for (int h = 0; h < 5; ++h) {
            const int q = tid + TR_BS * h;
            if (q < MLO * MLH) {
                const int v = q / MLH, k = q % MLH;
                float a = 0.f;
                for (int cc = 0; cc < TR_CH; ++cc) a = fmaf(O[cc * MLO + v], H2[cc * MLH + k], a);
                gW3[h] += a;
            }
        }
        if (tid < MLO)
            for (int cc = 0; cc < TR_CH; ++cc) gB3 += O[cc * MLO + tid];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 64; ++q) atomicAdd(&grad[OFF_W2 + jr * MLH + 64 * kh + q], gW2[q]);
#pragma unroll
    for (int q = 0; q < 32; ++q)
        if (kh + 2 * q < MLF) atomicAdd(&grad[OFF_W1 + jr * MLF + kh + 2 * q], gW1[q]);
    if (kh == 0) {
        atomicAdd(&grad[OFF_B1 + jr], gB1);
        atomicAdd(&grad[OFF_B2 + jr], gB2);
    }
#pragma unroll
    for (int h = 0; h < 5; ++h) {
        const int q = tid + TR_BS * h;
        if (q < MLO * MLH) atomicAdd(&grad[OFF_W3 + q], gW3[h]);
    }
    if (tid < MLO) atomicAdd(&grad[OFF_B3 + tid], gB3);
}

// ---------------------------------------------------------------------------
// Plain Jacobian operator (no well term), its transpose, reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ void nb7(const Geom& g, int c, int (&nb)[7], bool (&has)[7]) {
    const int plane = g.nx * g.ny, i = c % g.nx, j = (c / g.nx) % g.ny, k = c / plane;
    nb[0] = c; nb[1] = c - 1; nb[2] = c + 1; nb[3] = c - g.nx; nb[4] = c + g.nx;
    nb[5] = c - plane; nb[6] = c + plane;
    has[0] = true; has[1] = i > 0; has[2] = i + 1 < g.nx; has[3] = j > 0; has[4] = j + 1 < g.ny;
    has[5] = k > 0; has[6] = k + 1 < g.nz;
}

__device__ __forceinline__ void block_sum_to(double acc, double* __restrict__ part) {
    __shared__ double sh[ML_BS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < ML_BS / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// y = o - A x; part (may be null) [blockIdx] = ||y||^2 partial
__global__ void __launch_bounds__(ML_BS)
k_ml_resid(Geom g, const double* __restrict__ A, const double* __restrict__ x,
           const double* __restrict__ o, double* __restrict__ y, double* __restrict__ part) {
    const int n = g.n;
    double acc2 = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int nb[7];
        bool has[7];
        nb7(g, c, nb, has);
        double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            if (!has[b]) continue;
            const double x0 = x[nb[b]], x1 = x[(size_t)n + nb[b]], x2 = x[2 * (size_t)n + nb[b]];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const double* a = A + (size_t)(b * 9 + 3 * e) * n + c;
                s[e] = fma(a[0], x0, fma(a[n], x1, fma(a[2 * (size_t)n], x2, s[e])));
            }
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const double v = o[(size_t)e * n + c] - s[e];
            y[(size_t)e * n + c] = v;
            acc2 += v * v;
        }
    }
    if (part) block_sum_to(acc2, part);
}

// y = A^T x: row c gathers block (nb, opposite direction)^T x_nb.
__global__ void __launch_bounds__(ML_BS)
k_ml_AT(Geom g, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
    const int n = g.n;
    const int opp[7] = {0, 2, 1, 4, 3, 6, 5};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int nb[7];
        bool has[7];
        nb7(g, c, nb, has);
        double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int b = 0; b < 7; ++b) {
            if (!has[b]) continue;
            const int m = nb[b], ob = opp[b];
            const double x0 = x[m], x1 = x[(size_t)n + m], x2 = x[2 * (size_t)n + m];
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                // column v of block (m, ob): entries 3e + v
                const double* a = A + (size_t)(ob * 9 + v) * n + m;
                s[v] = fma(a[0], x0, fma(a[3 * (size_t)n], x1, fma(a[6 * (size_t)n], x2, s[v])));
            }
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) y[(size_t)v * n + c] = s[v];
    }
}

// Partial sums of a . b (fixed grid).
__global__ void __launch_bounds__(ML_BS)
k_ml_dot(int N, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
    double acc = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) acc += a[q] * b[q];
    block_sum_to(acc, part);
}

__global__ void k_ml_sum(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    if (threadIdx.x >= 32) return;
    double s = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32) s += part[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

// v *= -2 / rr (dL/ddelta = -2 A^T u / ||r||^2), rr read from the device
__global__ void k_ml_scale_vec(int N, double* __restrict__ v, const double* __restrict__ rr) {
    const double f = *rr > 0.0 ? -2.0 / *rr : 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) v[q] *= f;
}

// Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// theta -= lr * (m / c1) / (sqrt(v / c2) + eps); the gradient is cleared.
__global__ void k_ml_adam(int np, float* __restrict__ theta, float* __restrict__ grad,
                          float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                          float b2, float eps, float c1, float c2) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
        const float gq = grad[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        grad[q] = 0.f;
    }
}

// Sample store: slot = ks->it - 1 (the iteration that produced r), while it
// is below the store's capacity.
__global__ void k_ml_collect(int N, const double* __restrict__ r, double* __restrict__ store,
                             int cap, int* __restrict__ count, const KrylovScalars* __restrict__ ks) {
    if (ks->state != KS_RUN) return;
    const int slot = ks->it - 1;
    if (slot < 0 || slot >= cap) return;
    double* dst = store + (size_t)slot * N;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) dst[q] = r[q];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(count, slot + 1);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <class T>
static void ml_alloc(T** p, size_t count) {
    if (*p == nullptr)
        BO_CUDA(cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1)));
}

void learn_setup(bo_sim* s) {
    const size_t n = s->geo.n;
    ml_alloc(&s->d_ml_theta, NPARAM);
    ml_alloc(&s->d_ml_grad, NPARAM);
    ml_alloc(&s->d_ml_m, NPARAM);
    ml_alloc(&s->d_ml_v, NPARAM);
    if (s->d_ml_wbf == nullptr) BO_CUDA(cudaMalloc(&s->d_ml_wbf, sizeof(__nv_bfloat16) * WBF_ELEMS));
    if (s->d_ml_feat == nullptr) BO_CUDA(cudaMalloc(&s->d_ml_feat, sizeof(__nv_bfloat16) * 64 * n));
    ml_alloc(&s->d_ml_cell, n);
    ml_alloc(&s->d_ml_W, 9 * n);
    ml_alloc(&s->d_ml_part, 2 * ML_GRID + 8);
    BO_CUDA(cudaMemsetAsync(s->d_ml_grad, 0, sizeof(float) * NPARAM, s->stream));
    BO_CUDA(cudaFuncSetAttribute(k_ml_net, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INF_SMEM));
    BO_CUDA(cudaFuncSetAttribute(k_ml_net_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
    BO_CUDA(cudaFuncSetAttribute(k_ml_fwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM));
    BO_CUDA(cudaFuncSetAttribute(k_ml_bwd_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM));
}

void learn_setup_training(bo_sim* s) {
    const size_t n = s->geo.n, N = 3 * n;
    ml_alloc(&s->d_ml_featf, 64 * n);
    for (double** v : {&s->d_ml_delta, &s->d_ml_u, &s->d_ml_z0, &s->d_ml_e, &s->d_ml_dd})
        ml_alloc(v, N);
    ml_alloc(&s->d_ml_scal, 8);
    ml_alloc(&s->d_ml_count, 1);
}

void learn_set_params(bo_sim* s, const float* host) {
    BO_CUDA(cudaMemcpyAsync(s->d_ml_theta, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice,
                            s->stream));
    k_ml_pack<<<64, 256, 0, s->stream>>>(s->d_ml_theta, wbf_of(s));
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("k_ml_pack");
    BO_CUDA(cudaMemsetAsync(s->d_ml_m, 0, sizeof(float) * NPARAM, s->stream));
    BO_CUDA(cudaMemsetAsync(s->d_ml_v, 0, sizeof(float) * NPARAM, s->stream));
    s->ml_adam_t = 0;
    BO_CUDA(cudaStreamSynchronize(s->stream));
}

void learn_get_params(bo_sim* s, float* host) {
    BO_CUDA(cudaMemcpyAsync(host, s->d_ml_theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
}

void learn_get_grad(bo_sim* s, float* host) {
    BO_CUDA(cudaMemcpyAsync(host, s->d_ml_grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost,
                            s->stream));
    BO_CUDA(cudaStreamSynchronize(s->stream));
}

void learn_clear_grad(bo_sim* s) {
    BO_CUDA(cudaMemsetAsync(s->d_ml_grad, 0, sizeof(float) * NPARAM, s->stream));
}

// Features of the last assembly and, with parameters set, the per-cell
// matrices W_c of the network (tensor cores).
void enqueue_learn_features(bo_sim* s, cudaStream_t st) {
    const int n = s->geo.n;
    k_ml_feat<<<ML_GRID, ML_BS, 0, st>>>(s->geo, s->d_A, s->d_flag, feat_of(s), s->d_ml_featf,
                                        s->d_ml_cell);
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_ml_feat");
    if (s->ml_engine == BO_LEARN_ENGINE_TCGEN05) {
        // 128 cells per CTA, two CTAs per SM (103.5 KB of shared memory and
        // 256 tensor-memory columns each)
        const int grid = std::max(1, std::min(152 * 2, (n + 127) / 128));
        k_ml_net_tc<<<grid, TC_BS, TC_SMEM, st>>>(n, feat_of(s), wbf_of(s), s->d_ml_theta, s->d_ml_W,
                                                  reinterpret_cast<int*>(&s->d_ns->pad));
        count_launch(s, st);
        BO_LAUNCH_CHECK("k_ml_net_tc");
    } else {
        const int grid = std::max(1, std::min(152 * 2, (n + 16 * INF_WARPS - 1) / (16 * INF_WARPS)));
        k_ml_net<<<grid, 32 * INF_WARPS, INF_SMEM, st>>>(n, feat_of(s), wbf_of(s), s->d_ml_theta,
                                                         s->d_ml_W);
        count_launch(s, st);
        BO_LAUNCH_CHECK("k_ml_net");
    }
}

// z += delta(r) (inside the BiCGStab graph when ks is given)
void enqueue_learn_apply(bo_sim* s, cudaStream_t st, const double* r, double* z,
                         const KrylovScalars* ks) {
    k_ml_apply<<<ML_GRID, ML_BS, 0, st>>>(s->geo.n, s->d_ml_W, s->d_ml_cell, r, z, ks);
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_ml_apply");
}

void enqueue_learn_collect(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks) {
    const int N = 3 * s->geo.n;
    k_ml_collect<<<ML_GRID, ML_BS, 0, st>>>(N, r, s->d_ml_samples, s->ml_cap, s->d_ml_count, ks);
    count_launch(s, st);
    BO_LAUNCH_CHECK("k_ml_collect");
}

// One training sample r (device, [3][n]): z0 = M^-1 r (current factors),
// e = r - A z0, delta, u = e - A delta, L = ||u||^2/||r||^2, and the
// gradient of L added to d_ml_grad.  Returns L (synchronises).
double learn_loss_grad(bo_sim* s, const double* r) {
    cudaStream_t st = s->stream;
    const Geom g = s->geo;
    const int n = g.n, N = 3 * n;
    double* part2 = s->d_ml_part + ML_GRID;
    launch_precond(s, r, s->d_ml_z0);
    k_ml_resid<<<ML_GRID, ML_BS, 0, st>>>(g, s->d_A, s->d_ml_z0, r, s->d_ml_e, nullptr);
    count_launch(s, st);
    k_ml_fwd_f32<<<TR_GRID, TR_BS, TR_SMEM, st>>>(n, s->d_ml_featf, s->d_ml_cell, r, s->d_ml_theta,
                                                  s->d_ml_delta);
    count_launch(s, st);
    k_ml_resid<<<ML_GRID, ML_BS, 0, st>>>(g, s->d_A, s->d_ml_delta, s->d_ml_e, s->d_ml_u, part2);
    count_launch(s, st);
    k_ml_sum<<<1, 32, 0, st>>>(part2, ML_GRID, s->d_ml_scal);          // ||u||^2
    count_launch(s, st);
    k_ml_dot<<<ML_GRID, ML_BS, 0, st>>>(N, r, r, part2);
    count_launch(s, st);
    k_ml_sum<<<1, 32, 0, st>>>(part2, ML_GRID, s->d_ml_scal + 1);      // ||r||^2
    count_launch(s, st);
    k_ml_AT<<<ML_GRID, ML_BS, 0, st>>>(g, s->d_A, s->d_ml_u, s->d_ml_dd);
    count_launch(s, st);
    k_ml_scale_vec<<<ML_GRID, ML_BS, 0, st>>>(N, s->d_ml_dd, s->d_ml_scal + 1);
    count_launch(s, st);
    k_ml_bwd_f32<<<TR_GRID, TR_BS, TR_SMEM, st>>>(n, s->d_ml_featf, s->d_ml_cell, r, s->d_ml_theta,
                                                  s->d_ml_dd, s->d_ml_grad);
    count_launch(s, st);
    BO_LAUNCH_CHECK("learn_loss_grad");
    double h[2];
    BO_CUDA(cudaMemcpyAsync(h, s->d_ml_scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    BO_CUDA(cudaStreamSynchronize(st));
    return h[1] > 0.0 ? h[0] / h[1] : 0.0;
}

void learn_adam(bo_sim* s, double lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    s->ml_adam_t += 1;
    const float c1 = 1.f - powf(b1, (float)s->ml_adam_t);
    const float c2 = 1.f - powf(b2, (float)s->ml_adam_t);
    k_ml_adam<<<64, 256, 0, s->stream>>>(NPARAM, s->d_ml_theta, s->d_ml_grad, s->d_ml_m, s->d_ml_v,
                                         (float)lr, b1, b2, eps, c1, c2);
    count_launch(s, s->stream);
    k_ml_pack<<<64, 256, 0, s->stream>>>(s->d_ml_theta, wbf_of(s));
    count_launch(s, s->stream);
    BO_LAUNCH_CHECK("learn_adam");
}

}  // namespace bo
