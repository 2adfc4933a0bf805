// Tile schedule shared by the wavefront kernels (ILU(0) factorisation, the
// FP64 sweeps and the FP32 sweeps): tile geometry, face slots, the sentinel
// protocol of the face buffers and relaxed global accesses.
#pragma once
#include "common.cuh"

namespace bo {

constexpr int TJ = 8, TK = 4;          // tile of x-lines per warp (lane = jj + TJ kk)
constexpr unsigned long long SENTINEL_BITS = 0x7FF4DEADBEEF0001ull;  // a NaN no arithmetic yields
// bounded waits: with the back-off below, 2^20 polls take about one second
constexpr long long POLL_LIMIT = 1LL << 20;
#ifndef BO_POLL_SLEEP_NS
#define BO_POLL_SLEEP_NS 32
#endif
constexpr unsigned FULL = 0xffffffffu;

// ILU(0) data in tile order: slot s = t NL + l (tile t, level l) holds NPE
// entries x 32 lanes contiguously, P[(s NPE + q) 32 + lane]; q = 9 b + e with
// b 0: D^-1, 1..3: D^-1 A_{c,-x/-y/-z}, 4..6: D^-1 A_{c,+x/+y/+z}.  Entries
// 0..35 of a slot are the forward sweep's data, 36..62 the backward sweep's.
constexpr int NPE = 63;
__host__ __device__ __forceinline__ size_t pidx(size_t slot, int q, int lane) {
    return (slot * NPE + q) * 32 + lane;
}

struct TileArgs {
    Geom g;
    int NJ, NK, T, NL;
    size_t NP;
    int* err;
    int ysub;   // block-Jacobi slabs of ysub cell rows in y (a multiple of TJ), 0: no cut in y
    int zsub;   // and of zsub cell layers in z (a multiple of TK), 0: no cut in z
};

// j is the first cell row of a block-Jacobi slab (not the first of the grid):
// the -y coupling of row j and the +y coupling of row j - 1 are left out of
// the factors, and no face crosses the cut.  Cuts fall on tile boundaries.
__device__ __forceinline__ bool ycut(const TileArgs& a, int j) {
    return a.ysub > 0 && j > 0 && j % a.ysub == 0;
}
// The same in z: layer k starts a slab, the -z coupling of layer k and the +z
// coupling of layer k - 1 are left out.
__device__ __forceinline__ bool zcut(const TileArgs& a, int k) {
    return a.zsub > 0 && k > 0 && k % a.zsub == 0;
}

__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool is_sentinel(double v) {
    return (unsigned long long)__double_as_longlong(v) == SENTINEL_BITS;
}
// FP32 faces of the mixed-precision sweeps: a NaN payload no arithmetic yields
constexpr unsigned SENTINEL_BITS32 = 0x7FA5DEADu;
__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
__device__ __forceinline__ bool is_sentinel(float v) {
    return (unsigned)__float_as_uint(v) == SENTINEL_BITS32;
}

// Face slots: j-face of tile t for lane row kk at x index i; k-face for jj.
__device__ __forceinline__ size_t jslot(const TileArgs& a, int t, int i, int kk, int K) {
    return (((size_t)t * a.g.nx + i) * TK + kk) * K;
}
__device__ __forceinline__ size_t kslot(const TileArgs& a, int t, int i, int jj, int K) {
    return (((size_t)t * a.g.nx + i) * TJ + jj) * K;
}

__device__ __forceinline__ bool ks_skip_t(const KrylovScalars* ks) {
    return ks != nullptr && ks->state != KS_RUN;
}

// Host side: tile geometry of a model, face buffers, cooperative launches.
TileArgs tile_args(const bo_sim* s);
double* faceJ3(bo_sim* s);   // 3-value face buffers of the sweeps
double* faceK3(bo_sim* s);

template <class... Args>
void launch_coop(cudaStream_t st, int grid, int block, void (*kern)(Args...), Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BO_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

template <class... Args>
void launch_coop_smem(cudaStream_t st, int grid, int block, size_t smem, void (*kern)(Args...),
                      Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BO_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
}

// FP64 sweeps (sweep64.cu)
void setup_sweeps64(bo_sim* s);                              // attributes, residency, tile lists
void enqueue_fwd64(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks);
void enqueue_bwd64(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks);
int sweep_ctas(const bo_sim* s);

// FP32 sweeps of the mixed-precision solver (ilu_sweep32.cu)
void setup_sweeps32(bo_sim* s);                              // attributes, residency check
void convert_factors32(bo_sim* s, cudaStream_t st);          // d_P -> FP32 sweep layout
void enqueue_fwd32(bo_sim* s, cudaStream_t st, const double* r, const KrylovScalars* ks);
void enqueue_bwd32(bo_sim* s, cudaStream_t st, double* z, const KrylovScalars* ks);
void reset_faces32(bo_sim* s, cudaStream_t st);

}  // namespace bo
