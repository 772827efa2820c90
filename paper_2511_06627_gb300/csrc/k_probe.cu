// Shared-memory bandwidth probe: the measured peak that the projector pair's on-chip
// roofline is held against. The paper has no counterpart to this file.
//
// Every block fills 32 KB of shared memory, then each thread reads 16-byte words in a
// conflict-free pattern (the 8 lanes of a quarter warp read 8 consecutive words, so
// every phase of a 128-bit load takes one 128-byte wavefront) for a fixed number of
// rounds, and adds them into a register so that no load is dead. The grid holds
// several blocks per SM on every SM. Bytes moved = blocks x threads x rounds x 16.
#include "internal.h"

namespace mpiffl {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeWords = 2048;  // float4 words per block (32 KB)
constexpr int kProbeRounds = 4096;

__global__ void __launch_bounds__(kProbeThreads) k_smem_probe(float *__restrict__ out, float seed) {
    __shared__ float4 buf[kProbeWords];
    for (int i = threadIdx.x; i < kProbeWords; i += kProbeThreads)
        buf[i] = make_float4(seed * i, seed + i, seed - i, seed * 0.5f * i);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll 16
    for (int r = 0; r < kProbeRounds; ++r) {
        // a volatile load: neither the compiler nor the assembler may merge the
        // addresses that repeat every few rounds, or drop a load
        float4 v;
        asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                     : "r"(base + 16u * (uint32_t)idx));
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
        idx = (idx + kProbeThreads) & (kProbeWords - 1);
    }
    out[blockIdx.x * kProbeThreads + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

}  // namespace
}  // namespace mpiffl

extern "C" int mpi_ffl_probe_smem_bandwidth(double *gbs, void *stream) {
    using namespace mpiffl;
    if (!gbs) {
        set_thread_error("mpi_ffl_probe_smem_bandwidth: gbs is NULL");
        return MPI_FFL_ERR_INVALID_ARG;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smem_probe, kProbeThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        set_thread_error("mpi_ffl_probe_smem_bandwidth: device query failed");
        return MPI_FFL_ERR_CUDA;
    }
    const int blocks = n_sm * per_sm * 4;  // four full waves
    float *out = nullptr;
    if (dev_malloc((void **)&out, sizeof(float) * blocks * kProbeThreads) != cudaSuccess) {
        set_thread_error("mpi_ffl_probe_smem_bandwidth: device allocation failed");
        return MPI_FFL_ERR_OOM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = MPI_FFL_OK;
    float best = 0.f;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = MPI_FFL_ERR_CUDA;
    for (int rep = 0; rep < 6 && rc == MPI_FFL_OK; ++rep) {  // the first is a warm-up
        cudaEventRecord(a, st);
        k_smem_probe<<<blocks, kProbeThreads, 0, st>>>(out, 1.0f + rep);
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            rc = MPI_FFL_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (rc == MPI_FFL_OK && cudaGetLastError() != cudaSuccess) rc = MPI_FFL_ERR_CUDA;
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    dev_free(out);
    if (rc != MPI_FFL_OK) {
        set_thread_error("mpi_ffl_probe_smem_bandwidth: launch failed");
        return rc;
    }
    const double bytes = (double)blocks * kProbeThreads * kProbeRounds * 16.0;
    *gbs = bytes / (best * 1e-3) / 1e9;
    return MPI_FFL_OK;
}
