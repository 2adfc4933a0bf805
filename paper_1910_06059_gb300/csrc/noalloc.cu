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
// NA_SLOTS doubles (320 KB).  Every GPU that loads the library holds it
// until the process exits.  Host code cannot pass the variable's name to a
// kernel (in host code it is only a stand-in for the device symbol), so the
// first call on each device looks up its device address with
// cudaGetSymbolAddress while that device is current and keeps it; make that
// first call before any stream capture.  All calls share the one array:
// each call overwrites the partials of the blocks it uses before reading
// them, so nothing has to start at zero, but calls that overlap on the GPU
// (on different streams, or from different threads) race on it and must be
// serialised by the caller.
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
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_norm_scratch[NA_MAX_BLOCKS * NA_SLOTS];

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
            v[3 + a] = fmax(v[3 + a], fabs(r) / p);
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
            x = (q >= 3 && q < 6) ? fmax(x, y) : x + y;
        }
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_SLOTS) {
        const int q = threadIdx.x;
        double x = sh[q][0];
        for (int w = 1; w < NA_BS / 32; ++w) x = (q >= 3 && q < 6) ? fmax(x, sh[q][w]) : x + sh[q][w];
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
        x = (q >= 3 && q < 6) ? fmax(x, y) : x + y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, x, o);
        x = (q >= 3 && q < 6) ? fmax(x, y) : x + y;
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

static std::mutex g_na_mutex;
static double* g_na_addr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
static double* scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (g_na_addr[dev] == nullptr) {
        double* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_norm_scratch);
        check_cuda(e, "cudaGetSymbolAddress(g_norm_scratch)", __FILE__, __LINE__);
        g_na_addr[dev] = ptr;
    }
    return g_na_addr[dev];
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
    int dev = 0;
    BO_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        fail(BO_ERR_INVALID_ARG, "bo_residual_norms_noalloc: device ordinal out of range");
    double* scratch = scratch_address(dev);
    const int nblocks = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    k_na_partials<<<nblocks, NA_BS, 0, stream>>>(R, pv, b, n, scratch);
    BO_LAUNCH_CHECK("k_na_partials");
    k_na_final<<<1, 32 * NA_SLOTS, 0, stream>>>(scratch, nblocks, n, dt, out6);
    BO_LAUNCH_CHECK("k_na_final");
}

}  // namespace bo
