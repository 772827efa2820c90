// Device allocations of the library, routed through one place: a registry of the live
// allocations (count and bytes, for leak checks) and a test hook that makes the n-th
// allocation from now fail the way cudaMalloc fails on a full device. The paper has no
// counterpart to this file.
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace mpiffl {

namespace {

std::mutex g_mu;
std::unordered_map<void *, size_t> g_live;
int64_t g_live_bytes = 0;
int64_t g_countdown = 0;  // > 0: the allocation that brings it to zero fails

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_countdown > 0 && --g_countdown == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_live[*p] = bytes;
        g_live_bytes += (int64_t)bytes;
    }
    return e;
}

cudaError_t dev_free(void *p) {
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            g_live_bytes -= (int64_t)it->second;
            g_live.erase(it);
        }
    }
    return cudaFree(p);
}

}  // namespace mpiffl

extern "C" int mpi_ffl_test_fail_alloc(int32_t nth) {
    if (nth < 0) {
        mpiffl::set_thread_error("mpi_ffl_test_fail_alloc: nth must be >= 0");
        return MPI_FFL_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(mpiffl::g_mu);
    mpiffl::g_countdown = nth;
    return MPI_FFL_OK;
}

extern "C" int mpi_ffl_test_live_allocs(int64_t *count, int64_t *bytes) {
    std::lock_guard<std::mutex> lock(mpiffl::g_mu);
    if (count) *count = (int64_t)mpiffl::g_live.size();
    if (bytes) *bytes = mpiffl::g_live_bytes;
    return MPI_FFL_OK;
}
