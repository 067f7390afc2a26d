// Residual norm of the pressure equation without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// number: a control loop running under a fixed memory budget, or a host
// process that has handed all device memory to another allocator and may not
// call cudaMalloc itself.  For them, wec_residual_norm_noalloc computes
// ||b - A x||_2 with the solver's own per-cell operator (poisson_op.cuh), and
// its scratch (the per-block partial sums and a completion counter) lives in
// one file-scope device array instead of memory the caller or the library
// allocates.
//
// The array holds kNoAllocBlocks partial sums and the counter (about 4.9 KB);
// every GPU that loads the library holds it until the process exits.  Grids of
// up to kNoAllocMaxCells cells are accepted (the kernel's 32-bit face indexing).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"
#include "poisson_op.cuh"

namespace wec {
namespace {

constexpr long long kNoAllocMaxCells = 1LL << 28;          // largest nx * ny accepted
constexpr int kNoAllocBlocks = 608;                        // partial sums (4 x 152 SMs)
constexpr int kNoAllocDoubles = kNoAllocBlocks + 32;
constexpr int kNoAllocMaxDevices = 64;

// [0, kNoAllocBlocks): partial sums; then the completion counter (an unsigned
// int in the first slot of the tail).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

__device__ double nd_block_sum(double v, double *sh8)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh8[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) r += sh8[w];
    __syncthreads();
    return r;
}

// ||b - A x||^2 per block into the scratch partials; the block that finishes
// last adds the partials in block order and writes sqrt of the total to *out.
// 256 threads per block.
__global__ void __launch_bounds__(256) k_residual_norm_static(int nx, int ny, const double *__restrict__ bu,
                                                                const double *__restrict__ bv,
                                                                const double *__restrict__ x,
                                                                const double *__restrict__ b, double *out)
{
    __shared__ double sh[8];
    __shared__ int s_last;
    double *part = g_noalloc_scratch;
    unsigned int *cnt = reinterpret_cast<unsigned int *>(g_noalloc_scratch + kNoAllocBlocks);
    const long long n = (long long)nx * ny;
    double a = 0.0;
    for (long long c = blockIdx.x * 256LL + threadIdx.x; c < n; c += (long long)gridDim.x * 256) {
        const int i = (int)(c % nx), j = (int)(c / nx);
        const double d = diag_at<double>(bu, bv, nx, ny, i, j);
        const double rc = b[c] - (d * x[c] - offsum_at<double, double>(bu, bv, x, nx, ny, i, j));
        a += rc * rc;
    }
    a = nd_block_sum(a, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        __threadfence();
        s_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    double s = 0.0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += 256) s += __ldcg(part + q);
    s = nd_block_sum(s, sh);
    if (threadIdx.x == 0) {
        *out = sqrt(s);
        *cnt = 0u;
    }
}

}  // namespace
}  // namespace wec

using namespace wec;

extern "C" int wec_residual_norm_noalloc(int nx, int ny, const double *beta_u, const double *beta_v,
                                         const double *x, const double *b, double *norm_out, void *cuda_stream)
{
    if (!beta_u || !beta_v || !x || !b || !norm_out) return fail(WEC_ERR_INVALID, "residual_norm_noalloc: NULL argument");
    if (nx < 1 || ny < 1) return fail(WEC_ERR_INVALID, "residual_norm_noalloc: nx, ny must be >= 1");
    if ((long long)nx * ny > kNoAllocMaxCells)
        return fail(WEC_ERR_INVALID, "residual_norm_noalloc: nx * ny = " + std::to_string((long long)nx * ny) +
                                         " exceeds the maximum of " + std::to_string(kNoAllocMaxCells) + " cells");
    int dev = 0;
    WEC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(WEC_ERR_INVALID, "residual_norm_noalloc: device index too large");
    double *base = nullptr;
    {
        // Once per device, with that device current: the scratch array's device
        // address (its host-side name is only a stand-in).  The first call on a
        // device does this, so it should come before any stream capture; the
        // address is kept for the process, so calls after a cudaDeviceReset are
        // not supported.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_noalloc_ptr[dev] = static_cast<double *>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the completion counter must start at zero (a call that failed midway could have left it set)
    WEC_CK(cudaMemsetAsync(base + kNoAllocBlocks, 0, sizeof(unsigned int), st));
    const long long n = (long long)nx * ny;
    const int grid = (int)std::min<long long>((n + 255) / 256, kNoAllocBlocks);
    WEC_PROF("residual_norm_noalloc", -1, 8.0 * (3.0 * n + (nx + 1.0) * ny + nx * (ny + 1.0)), st);
    prof::count_launch();
    k_residual_norm_static<<<grid, 256, 0, st>>>(nx, ny, beta_u, beta_v, x, b, norm_out);
    WEC_CK(cudaGetLastError());
    return WEC_OK;
}
