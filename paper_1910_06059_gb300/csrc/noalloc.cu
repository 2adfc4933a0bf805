// Residual convergence measures computed without allocating anything.
//
// Some callers cannot call cudaMalloc: code running inside a memory budget
// that is fixed up front (a plugin or host application that owns all device
// memory and hands out only its own buffers), code that must not
// synchronise the device the way an allocation can, or code that wants to
// run right after a failure to allocate.  bo_residual_norms_noalloc serves
// them: the caller passes the residual, pore volumes and shrinkage factors
// in its own device buffers and a device buffer for the result; the
// per-block partial sums live in a fixed array of this file, so the call
// allocates no memory at all.
//
// The partial-sum array is a file-scope device variable of NA_MAX_BLOCKS x
// NA_SLOTS doubles (320 KB).  Host code cannot pass the variable's name to a
// kernel (in host code it is only a stand-in for the device symbol), so the
// call looks up its device address with cudaGetSymbolAddress.  A symbol's
// address belongs to a CUDA context, so the lookup is made once per context
// -- keyed on the context's unique ID, which is never reused: a caller's own
// driver-API context, or the primary context re-created after
// cudaDeviceReset, gets its own lookup -- and kept for later calls in that
// context.  CUDA loads a library's device code lazily by default: the first
// call in a context loads this module and places the array in device memory
// (an allocation made by the driver), and it is that call which looks the
// address up.  Make that first call once at start-up, before the memory
// budget is fixed and before any stream capture; from then on a call
// allocates nothing.  (With CUDA_MODULE_LOADING=EAGER the module is loaded
// when the context is created.)  All calls share the one array: each call
// overwrites the partials of the blocks it uses before reading them, so
// nothing has to start at zero, but calls that overlap on the GPU (on
// different streams, or from different threads) race on it and must be
// serialised by the caller.
#include <cuda.h>   // CUcontext / CUresult types only; the functions come from the runtime

#include <mutex>
#include <string>

#include "common.cuh"

namespace bo {

constexpr int NA_BS = 256;                              // threads per block
constexpr int NA_CELLS_PER_THREAD = 8;
constexpr int NA_CELLS_PER_BLOCK = NA_BS * NA_CELLS_PER_THREAD;   // 2048
constexpr int NA_MAX_BLOCKS = 4096;
constexpr long long NA_MAX_CELLS = (long long)NA_MAX_BLOCKS * NA_CELLS_PER_BLOCK;  // 8,388,608
// per block: sum R_a (3), max |R_a| / pv (3), sum pv (1), sum 1/b_a (3)
constexpr int NA_SLOTS = 10;
constexpr int NA_MAX_CONTEXTS = 64;   // contexts whose lookup is kept

static __device__ __align__(256) double g_norm_scratch[NA_MAX_BLOCKS * NA_SLOTS];

// Maximum that propagates NaN (fmax drops it): a NaN residual entry makes the
// CNV measure NaN, as it makes the MB sum NaN.
__device__ __forceinline__ double nan_max(double a, double b) {
    return (a > b || a != a) ? a : b;
}

// One block per NA_CELLS_PER_BLOCK cells; fixed-order reductions.
__global__ void __launch_bounds__(NA_BS)
k_na_partials(const double* __restrict__ R, const double* __restrict__ pv,
              const double* __restrict__ b, int n, double* __restrict__ scratch) {
    double v[NA_SLOTS];
#pragma unroll
    for (int q = 0; q < NA_SLOTS; ++q) v[q] = 0.0;
    const int base = blockIdx.x * NA_CELLS_PER_BLOCK;
#pragma unroll
    for (int k = 0; k < NA_CELLS_PER_THREAD; ++k) {
        const int c = base + k * NA_BS + threadIdx.x;
        if (c >= n) break;
        const double p = pv[c];
        v[6] += p;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double r = R[(size_t)a * n + c];
            v[a] += r;
            v[3 + a] = nan_max(v[3 + a], fabs(r) / p);
            v[7 + a] += 1.0 / b[(size_t)a * n + c];
        }
    }
    __shared__ double sh[NA_SLOTS][NA_BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NA_SLOTS; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = (q >= 3 && q < 6) ? nan_max(x, y) : x + y;
        }
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_SLOTS) {
        const int q = threadIdx.x;
        double x = sh[q][0];
        for (int w = 1; w < NA_BS / 32; ++w) x = (q >= 3 && q < 6) ? nan_max(x, sh[q][w]) : x + sh[q][w];
        scratch[blockIdx.x * NA_SLOTS + q] = x;
    }
}

// One block of NA_SLOTS x 32 threads: slot q reduced by warp q in fixed order.
__global__ void k_na_final(const double* __restrict__ scratch, int nblocks, int n, double dt,
                           double* __restrict__ out6) {
    __shared__ double acc[NA_SLOTS];
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double x = 0.0;  // sums start at 0; the maxima of |R|/pv are >= 0
    for (int blk = lane; blk < nblocks; blk += 32) {
        const double y = scratch[blk * NA_SLOTS + q];
        x = (q >= 3 && q < 6) ? nan_max(x, y) : x + y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, x, o);
        x = (q >= 3 && q < 6) ? nan_max(x, y) : x + y;
    }
    if (lane == 0) acc[q] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            const double bavg = acc[7 + a] / n;
            out6[a] = dt * bavg * fabs(acc[a]) / acc[6];
            out6[3 + a] = dt * bavg * acc[3 + a];
        }
    }
}

// The current context and its unique ID, through the driver entry points the
// runtime hands out (no link against the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

static bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

struct ScratchEntry {
    unsigned long long ctx_id;
    double* addr;
};
static std::mutex g_na_mutex;
static ScratchEntry g_na_cache[NA_MAX_CONTEXTS];
static int g_na_used = 0, g_na_next = 0;

// Device address of the scratch array in the current context.  The first
// call in a context looks it up (loading the module there if it is not
// loaded yet); later calls in the same context reuse it.  Without the
// context ID (driver entry points unavailable) every call looks it up.
static double* scratch_address() {
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (keyed)
        for (int q = 0; q < g_na_used; ++q)
            if (g_na_cache[q].ctx_id == id) return g_na_cache[q].addr;
    double* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_norm_scratch);
    check_cuda(e, "cudaGetSymbolAddress(g_norm_scratch)", __FILE__, __LINE__);
    // the lookup may have made the device's primary context current
    if (current_context_id(&id)) {
        g_na_cache[g_na_next] = {id, ptr};
        g_na_next = (g_na_next + 1) % NA_MAX_CONTEXTS;
        if (g_na_used < NA_MAX_CONTEXTS) ++g_na_used;
    }
    return ptr;
}

void residual_norms_noalloc(const double* R, const double* pv, const double* b, int n, double dt,
                            double* out6, cudaStream_t stream) {
    if (R == nullptr || pv == nullptr || b == nullptr || out6 == nullptr)
        fail(BO_ERR_INVALID_ARG, "bo_residual_norms_noalloc: NULL device pointer");
    if (n < 1) fail(BO_ERR_INVALID_ARG, "bo_residual_norms_noalloc: n must be >= 1");
    if ((long long)n > NA_MAX_CELLS)
        fail(BO_ERR_INVALID_ARG, "bo_residual_norms_noalloc: n = " + std::to_string(n) +
                                     " exceeds the maximum of " + std::to_string(NA_MAX_CELLS) +
                                     " cells of its fixed scratch array");
    if (!(dt > 0.0)) fail(BO_ERR_INVALID_ARG, "bo_residual_norms_noalloc: dt must be > 0");
    double* scratch = scratch_address();
    const int nblocks = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    k_na_partials<<<nblocks, NA_BS, 0, stream>>>(R, pv, b, n, scratch);
    BO_LAUNCH_CHECK("k_na_partials");
    k_na_final<<<1, 32 * NA_SLOTS, 0, stream>>>(scratch, nblocks, n, dt, out6);
    BO_LAUNCH_CHECK("k_na_final");
}

}  // namespace bo
