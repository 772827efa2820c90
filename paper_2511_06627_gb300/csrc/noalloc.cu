// Handle-free FP64 inner product whose scratch is a file-scope device array, for
// callers that cannot allocate device memory (see mpi_ffl_dot_f64_noalloc in
// include/mpi_ffl.h). The paper has no counterpart to this call.
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerBlock = 1024;  // elements reduced by one block
static_assert((int64_t)kPerBlock * MPI_FFL_NOALLOC_MAX_PARTIALS == MPI_FFL_NOALLOC_MAX_N, "limit mismatch");

// One partial sum per block of the last call on this device (512 KiB).
static __device__ __align__(256) double g_partials[MPI_FFL_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

__device__ __forceinline__ double block_total(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
    return t;
}

// Block b sums a_i b_i over i in [b*1024, min(n, (b+1)*1024)) into partials[b].
__global__ void __launch_bounds__(kThreads) k_dot_blocks(const float *__restrict__ a, const float *__restrict__ b,
                                                         int64_t n, double *__restrict__ partials) {
    __shared__ double sh[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kPerBlock;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kPerBlock / kThreads; ++k) {
        const int64_t i = base + k * kThreads + threadIdx.x;
        if (i < n) acc += (double)a[i] * (double)b[i];
    }
    const double t = block_total(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// One block adds partials[0..nblk) in index order.
__global__ void __launch_bounds__(kThreads) k_dot_total(const double *__restrict__ partials, int nblk,
                                                        double *__restrict__ out) {
    __shared__ double sh[kThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) acc += partials[i];
    const double t = block_total(acc, sh);
    if (threadIdx.x == 0) *out = t;
}

// Device address of g_partials on the current device, looked up once per device and
// kept for the life of the process (a cudaDeviceReset of that device makes it stale).
int partials_address(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        mpiffl::set_thread_error(std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
        return MPI_FFL_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_partials);
        if (e != cudaSuccess || !p) {
            mpiffl::set_thread_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return MPI_FFL_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MPI_FFL_OK;
}

}  // namespace

extern "C" int mpi_ffl_dot_f64_noalloc(const float *d_a, const float *d_b, int64_t n, double *d_out, void *stream) {
    if (!d_out || n < 0 || (n > 0 && (!d_a || !d_b))) {
        mpiffl::set_thread_error("mpi_ffl_dot_f64_noalloc: NULL pointer or negative n");
        return MPI_FFL_ERR_INVALID_ARG;
    }
    if (n > MPI_FFL_NOALLOC_MAX_N) {
        mpiffl::set_thread_error("mpi_ffl_dot_f64_noalloc: n = " + std::to_string(n) +
                                 " exceeds the maximum of " + std::to_string((long long)MPI_FFL_NOALLOC_MAX_N) +
                                 " elements (scratch holds " + std::to_string(MPI_FFL_NOALLOC_MAX_PARTIALS) +
                                 " partial sums of 1024 elements)");
        return MPI_FFL_ERR_INVALID_ARG;
    }
    double *partials = nullptr;
    int rc = partials_address(&partials);
    if (rc != MPI_FFL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = n > 0 ? (int)((n + kPerBlock - 1) / kPerBlock) : 1;
    // An error left pending by an earlier runtime call of the caller's is neither
    // reported as this call's nor cleared: only a launch error that replaced it (or
    // appeared where none was pending) is this call's, and only that one is consumed.
    const cudaError_t before = cudaPeekAtLastError();
    k_dot_blocks<<<nblk, kThreads, 0, st>>>(d_a, d_b, n, partials);
    k_dot_total<<<1, kThreads, 0, st>>>(partials, nblk, d_out);
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess && e != before) {
        (void)cudaGetLastError();
        mpiffl::set_thread_error(std::string("mpi_ffl_dot_f64_noalloc launch: ") + cudaGetErrorString(e));
        return MPI_FFL_ERR_CUDA;
    }
    return MPI_FFL_OK;
}
