// noalloc.cu -- moment sums of a caller-owned population field without any allocation.
//
// Some callers cannot let a library allocate device memory: code that runs while a
// memory pool owns every byte of the device, real-time loops that forbid allocation after
// start-up, or code about to be captured into a CUDA graph, where cudaMalloc is not
// allowed.  This entry point therefore needs no context and allocates nothing: the
// caller passes the populations, the flags and the output, all in device memory, and
// the per-block partial sums go to a fixed scratch array compiled into this library.
//
// The scratch is a file-scope __device__ array of kNoAllocMaxBlocks slots (4 doubles
// each, 256 KiB in total).  Every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address; the address is
// looked up once per device (cudaGetSymbolAddress, with that device current) by the first
// call on that device, which should therefore happen before any stream capture.  The
// address is kept per device ordinal until the process exits; a cudaDeviceReset unloads the
// module, so after one the kept address is stale and this entry point must not be called
// on that device again.  All calls share the array: a call only reads slots that it wrote
// itself earlier in the same call, so nothing has to start at zero, but two calls that
// overlap on the GPU (on different streams without ordering) race on it.
#include <mutex>

#include "batch.h"

namespace lbm {
namespace {

constexpr int kNoAllocMaxBlocks = 8192;      // scratch slots: 8192 * 4 doubles = 256 KiB
constexpr int kNoAllocThreads = 256;
constexpr long long kNoAllocCellsPerBlock = 32768;  // fixed cells per block: 128 per thread
constexpr long long kNoAllocMaxCells = (long long)kNoAllocMaxBlocks * kNoAllocCellsPerBlock;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * 4];

// Block b sums cells [b * kNoAllocCellsPerBlock, ...) of the fluid cells: threads stride
// over the range in a fixed order, then a fixed tree; partial -> partials[b].
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_partials_kernel(const double *__restrict__ f,
                                                                          const uint8_t *__restrict__ solid,
                                                                          long long n, double rho0,
                                                                          double *__restrict__ partials)
{
    __shared__ double sm[kNoAllocThreads][4];
    const long long c0 = (long long)blockIdx.x * kNoAllocCellsPerBlock;
    const long long c1 = c0 + kNoAllocCellsPerBlock < n ? c0 + kNoAllocCellsPerBlock : n;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long c = c0 + threadIdx.x; c < c1; c += kNoAllocThreads) {
        if (solid && solid[c]) continue;
        double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const double v = f[(long long)k * n + c];
            rho += v;
            jx += ex(k) * v;
            jy += ey(k) * v;
            jz += ez(k) * v;
        }
        a[0] += rho - rho0;
        a[1] += jx / rho0;
        a[2] += jy / rho0;
        a[3] += jz / rho0;
    }
    for (int d = 0; d < 4; ++d) sm[threadIdx.x][d] = a[d];
    __syncthreads();
    for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 4; ++d) sm[threadIdx.x][d] += sm[threadIdx.x + w][d];
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[(long long)blockIdx.x * 4 + threadIdx.x] = sm[0][threadIdx.x];
}

// One block: out[d] = sum over blocks of partials[b][d], in a fixed order.
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_final_kernel(const double *__restrict__ partials,
                                                                       int nblocks, double *__restrict__ out)
{
    __shared__ double sm[kNoAllocThreads][4];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kNoAllocThreads)
        for (int d = 0; d < 4; ++d) a[d] += partials[(long long)b * 4 + d];
    for (int d = 0; d < 4; ++d) sm[threadIdx.x][d] = a[d];
    __syncthreads();
    for (int w = kNoAllocThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int d = 0; d < 4; ++d) sm[threadIdx.x][d] += sm[threadIdx.x + w][d];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = sm[0][threadIdx.x];
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kMaxDevices] = {};

lbm_status noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_ARG, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_moment_sums_f64_noalloc(const double *f_dev, const uint8_t *solid_dev, int64_t n_cells,
                                                  double rho0, double *sums_dev, void *cuda_stream)
{
    if (!f_dev || !sums_dev) return fail(LBM_ERR_ARG, "f_dev and sums_dev must be device pointers");
    if (n_cells < 1) return fail(LBM_ERR_ARG, "n_cells must be >= 1");
    if (n_cells > kNoAllocMaxCells)
        return fail(LBM_ERR_ARG, "n_cells exceeds the no-allocation limit of " + std::to_string(kNoAllocMaxCells) +
                                     " cells (the fixed scratch holds " + std::to_string(kNoAllocMaxBlocks) +
                                     " block sums)");
    if (!(rho0 > 0.0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
    if ((reinterpret_cast<uintptr_t>(f_dev) | reinterpret_cast<uintptr_t>(sums_dev)) & 7u)
        return fail(LBM_ERR_ARG, "f_dev and sums_dev must be 8-byte aligned");
    double *scratch = nullptr;
    lbm_status st = noalloc_scratch(&scratch);
    if (st != LBM_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((n_cells + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
    noalloc_partials_kernel<<<nblocks, kNoAllocThreads, 0, s>>>(f_dev, solid_dev, (long long)n_cells, rho0, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation moment sums (partials)");
    noalloc_final_kernel<<<1, kNoAllocThreads, 0, s>>>(scratch, nblocks, sums_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation moment sums (final)");
    return LBM_OK;
}
