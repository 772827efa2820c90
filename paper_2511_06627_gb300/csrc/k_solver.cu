// Solver kernels for Eq. (26) (Sec. 3.3) and the FP64 reductions it needs.
//
// Reductions are deterministic: each block writes one FP64 partial sum in a fixed
// order and a single block adds the partials in index order.
// The stop test leaves its verdict in a device flag; the host reads it only when
// an early stop was requested. The optional `done` flag of the per-iteration
// kernels turns them into no-ops once it is set.
#include <algorithm>

#include "internal.h"

namespace mpiffl {

constexpr int kRedThreads = 256;

int reduce_blocks(int64_t n) {
    int64_t b = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void k_momentum(const float *__restrict__ x, const float *__restrict__ xp,
                           float *__restrict__ y, float beta, int64_t n, const int *done) {
    if (done && *done) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float xi = x[i];
        y[i] = fmaf(beta, xi - xp[i], xi);
    }
}

void launch_momentum(const float *x, const float *xp, float *y, double beta_num, int k,
                     int64_t n, const int *done, cudaStream_t st) {
    (void)k;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_momentum<<<blocks, 256, 0, st>>>(x, xp, y, (float)beta_num, n, done);
}

// r <- r - b, partial sums of r^2 (FP64)
__global__ void __launch_bounds__(kRedThreads) k_sub_norm(float *__restrict__ r, const float *__restrict__ b,
                                                          int64_t n, double *partials, const int *done) {
    if (done && *done) return;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = r[i] - b[i];
        r[i] = v;
        acc += (double)v * (double)v;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

void launch_sub_norm(float *r, const float *b, int64_t n, double *partials, int nblk,
                     const int *done, cudaStream_t st) {
    k_sub_norm<<<nblk, kRedThreads, 0, st>>>(r, b, n, partials, done);
}

__global__ void __launch_bounds__(kRedThreads) k_dot(const float *__restrict__ a, const float *__restrict__ b,
                                                     int64_t n, double *partials) {
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

void launch_dot(const float *a, const float *b, int64_t n, double *partials, int nblk, cudaStream_t st) {
    k_dot<<<nblk, kRedThreads, 0, st>>>(a, b, n, partials);
}

__global__ void __launch_bounds__(kRedThreads) k_finalize(const double *partials, int nblk, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += partials[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) *out = t;
}

void launch_finalize(const double *partials, int nblk, double *out, cudaStream_t st) {
    k_finalize<<<1, kRedThreads, 0, st>>>(partials, nblk, out);
}

__global__ void __launch_bounds__(kRedThreads) k_finalize_f(const double *partials, int nblk, float *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += partials[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) *out = (float)t;
}

void launch_finalize_to_float(const double *partials, int nblk, float *out, cudaStream_t st) {
    k_finalize_f<<<1, kRedThreads, 0, st>>>(partials, nblk, out);
}

// Per-angle dot products: blockIdx.y = angle, per_angle contiguous floats each.
__global__ void __launch_bounds__(kRedThreads) k_angle_dots(const float *__restrict__ a, const float *__restrict__ b,
                                                            int64_t per_angle, double *partials) {
    const float *pa = a + (size_t)blockIdx.y * per_angle;
    const float *pb = b + (size_t)blockIdx.y * per_angle;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per_angle; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)pa[i] * (double)pb[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

void launch_angle_dots(const float *a, const float *b, int M, int64_t per_angle, double *partials,
                       int nblk_per_angle, cudaStream_t st) {
    dim3 grid(nblk_per_angle, M);
    k_angle_dots<<<grid, kRedThreads, 0, st>>>(a, b, per_angle, partials);
}

__global__ void __launch_bounds__(kRedThreads) k_angle_finalize(const double *partials, int nblk, float *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += partials[(size_t)blockIdx.x * nblk + i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = (float)t;
}

void launch_angle_finalize(const double *partials, int M, int nblk_per_angle, float *out, cudaStream_t st) {
    k_angle_finalize<<<M, kRedThreads, 0, st>>>(partials, nblk_per_angle, out);
}

// T^T T x with forward differences and no wrap (Neumann): 7-point stencil with the
// face-reduced diagonal.
__device__ __forceinline__ float ttt_at(const float *__restrict__ x, int N, int Nz, int z, int y, int xx) {
    const size_t i = ((size_t)z * N + y) * N + xx;
    const float c = x[i];
    float s = 0.f;
    if (xx > 0) s += c - x[i - 1];
    if (xx < N - 1) s += c - x[i + 1];
    if (y > 0) s += c - x[i - N];
    if (y < N - 1) s += c - x[i + N];
    if (z > 0) s += c - x[i - (size_t)N * N];
    if (z < Nz - 1) s += c - x[i + (size_t)N * N];
    return s;
}

__global__ void k_ttt(const float *__restrict__ x, float *__restrict__ out, int N, int Nz) {
    const int xx = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (xx >= N) return;
    out[((size_t)z * N + y) * N + xx] = ttt_at(x, N, Nz, z, y, xx);
}

void launch_ttt(const float *x, float *out, int N, int Nz, cudaStream_t st) {
    dim3 grid((N + 127) / 128, N, Nz);
    k_ttt<<<grid, 128, 0, st>>>(x, out, N, Nz);
}

// x_out = P(y - tau (g + lam T^T T y)), P = max(0, .) when nonneg. Once *done is set
// the solve is frozen: x_out = xcur (the current iterate), so that the buffer swap of
// the next iteration keeps the final iterate.
__global__ void k_update(const float *__restrict__ y, const float *__restrict__ g, float *__restrict__ xo,
                         float tau, float lam, int nonneg, int N, int Nz, const int *done,
                         const float *__restrict__ xcur) {
    const int xx = blockIdx.x * blockDim.x + threadIdx.x;
    const int yy = blockIdx.y, z = blockIdx.z;
    if (xx >= N) return;
    const size_t i = ((size_t)z * N + yy) * N + xx;
    if (done && *done) {
        if (xcur) xo[i] = xcur[i];
        return;
    }
    const float grad = fmaf(lam, ttt_at(y, N, Nz, z, yy, xx), g[i]);
    float v = fmaf(-tau, grad, y[i]);
    if (nonneg) v = fmaxf(v, 0.f);
    xo[i] = v;
}

void launch_update(const float *y, const float *g, float *xout, float tau, float lam, int nonneg,
                   int N, int Nz, const int *done, cudaStream_t st, const float *xcur) {
    dim3 grid((N + 127) / 128, N, Nz);
    k_update<<<grid, 128, 0, st>>>(y, g, xout, tau, lam, nonneg, N, Nz, done, xcur);
}

// Per kept bin q: sum over segments of |b[seg][q]|^2 in FP64, segments in order.
__global__ void k_bin_energy(const float2 *__restrict__ data, int nseg, int nb, double *__restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nb) return;
    double acc = 0.0;
    for (int sgi = 0; sgi < nseg; ++sgi) {
        const float2 v = data[(size_t)sgi * nb + q];
        acc = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, acc));
    }
    out[q] = acc;
}

void launch_bin_energy(const float *data, int nseg, int nb, double *out, cudaStream_t st) {
    k_bin_energy<<<(nb + 127) / 128, 128, 0, st>>>(reinterpret_cast<const float2 *>(data), nseg, nb, out);
}

// frozen = stop (after the update of the stopping iteration)
__global__ void k_freeze(const int *stop, int *frozen) {
    if (*stop) *frozen = 1;
}

void launch_freeze(const int *stop, int *frozen, cudaStream_t st) { k_freeze<<<1, 1, 0, st>>>(stop, frozen); }

// SplitMix64 (Steele, Lea, Flood 2014) evaluated at counter i + 1: u in [-1, 1).
__global__ void k_splitmix_fill(float *v, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = (float)((double)(z >> 11) * 0x1.0p-52 - 1.0);
    }
}

void launch_splitmix_fill(float *v, int64_t n, uint64_t seed, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_splitmix_fill<<<blocks, 256, 0, st>>>(v, n, seed);
}

__global__ void k_scale_by_rsqrt(const float *__restrict__ in, float *__restrict__ out, int64_t n, const double *n2) {
    const double nn = *n2;
    const float s = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * s;
}

void launch_scale_by_rsqrt(const float *in, float *out, int64_t n, const double *n2, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_scale_by_rsqrt<<<blocks, 256, 0, st>>>(in, out, n, n2);
}

// hist[k] holds ||r_k||^2 on entry; replaces it by ||r_k|| and sets *done when the
// relative change from hist[k-1] is at most stop_rel (or the norm is not finite).
__global__ void k_stop_check(double *hist, int k, double stop_rel, int *done, int *iters_done) {
    if (*done) return;
    const double r = sqrt(hist[k]);
    hist[k] = r;
    *iters_done = k + 1;
    if (!(r == r) || r > 1e300) {
        *done = 2;
        return;
    }
    if (stop_rel > 0.0 && k > 0) {
        const double prev = hist[k - 1];
        if (fabs(prev - r) <= stop_rel * prev) *done = 1;
    }
}

void launch_stop_check(double *hist, int k, double stop_rel, int *done, int *iters_done, cudaStream_t st) {
    k_stop_check<<<1, 1, 0, st>>>(hist, k, stop_rel, done, iters_done);
}

// ---------------------------------------------------------------------- batches
__device__ __forceinline__ int batch_find_s(const int *__restrict__ offs, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int kVecPerBlock = 256 * 8;  // elements per block of the batched element-wise kernels

// The batched kernels are persistent: a grid of at most as many blocks as the GPU holds
// at once loops over the work items (item b belongs to the job j with offs[j] <= b <
// offs[j + 1]), so one launch per kind serves every job whatever their count and sizes.
// An item's arithmetic does not depend on the block that runs it.
__global__ void __launch_bounds__(256) k_momentum_batch(const MomentumJob *__restrict__ jobs,
                                                        const int *__restrict__ offs, int n, int total) {
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find_s(offs, n, bi);
        const MomentumJob J = jobs[j];
        if (J.done && *J.done) continue;
        const int64_t base = (int64_t)(bi - offs[j]) * kVecPerBlock;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = base + u * 256 + threadIdx.x;
            if (i < J.n) {
                const float xi = J.x[i];
                J.y[i] = fmaf(J.beta, xi - J.xp[i], xi);
            }
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) k_residual_batch(const ResidualJob *__restrict__ jobs,
                                                                const int *__restrict__ offs, int n, int total) {
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find_s(offs, n, bi);
        const ResidualJob J = jobs[j];
        if (J.done && *J.done) continue;  // uniform over the block
        const int b = bi - offs[j];
        double acc = 0.0;
        for (int64_t i = (int64_t)b * blockDim.x + threadIdx.x; i < J.n; i += (int64_t)J.nblk * blockDim.x) {
            const float v = J.r[i] - J.b[i];
            J.r[i] = v;
            acc += (double)v * (double)v;
        }
        const double t = block_sum(acc);
        if (threadIdx.x == 0) J.partials[b] = t;
        __syncthreads();  // block_sum's shared words are reused by the next item
    }
}

// one block per problem: partial sums in index order, then the stop test
__global__ void __launch_bounds__(kRedThreads) k_stop_batch(const StopJob *__restrict__ jobs, int n) {
    for (int bi = blockIdx.x; bi < n; bi += gridDim.x) {
        const StopJob J = jobs[bi];
        if (*J.done) continue;
        double acc = 0.0;
        for (int i = threadIdx.x; i < J.nblk; i += blockDim.x) acc += J.partials[i];
        const double t = block_sum(acc);
        if (threadIdx.x == 0) {
            const double r = sqrt(t);
            J.hist[J.k] = r;
            J.flags[1] = J.k + 1;
            if (!(r == r) || r > 1e300) {
                J.flags[0] = 2;
            } else if (J.stop_rel > 0.0 && J.k > 0) {
                const double prev = J.hist[J.k - 1];
                if (fabs(prev - r) <= J.stop_rel * prev) J.flags[0] = 1;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(128) k_update_batch(const UpdateJob *__restrict__ jobs, const int *__restrict__ offs,
                                                      int n, int total) {
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find_s(offs, n, bi);
        const UpdateJob J = jobs[j];
        const int b = bi - offs[j];
        const int gx = (J.N + 127) / 128;
        const int xx = (b % gx) * 128 + threadIdx.x;
        const int yy = (b / gx) % J.N, z = b / (gx * J.N);
        if (xx >= J.N) continue;
        const size_t i = ((size_t)z * J.N + yy) * J.N + xx;
        if (J.done && *J.done) {  // frozen: keep the final iterate in the buffer that becomes x
            J.xo[i] = J.xcur[i];
            continue;
        }
        const float grad = fmaf(J.lam, ttt_at(J.y, J.N, J.Nz, z, yy, xx), J.g[i]);
        float v = fmaf(-J.tau, grad, J.y[i]);
        if (J.nonneg) v = fmaxf(v, 0.f);
        J.xo[i] = v;
    }
}

int update_blocks(int N, int Nz) { return ((N + 127) / 128) * N * Nz; }

__global__ void k_freeze_batch(const StopJob *__restrict__ jobs, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && jobs[j].flags[0] != 0) *jobs[j].done = 1;
}

void launch_freeze_batch(const StopJob *jobs, int n, cudaStream_t st) {
    k_freeze_batch<<<(n + 127) / 128, 128, 0, st>>>(jobs, n);
}

// Blocks of a persistent batched launch: what the GPU holds at once, at most one per item.
template <class K>
int persistent_grid(K kernel, int threads, size_t smem, int total) {
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();  // a failed query is not the caller's error
        per = 1;
    }
    return std::max(1, std::min(total, per * n_sm));
}

void launch_momentum_batch(const MomentumJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    if (total <= 0) return;
    k_momentum_batch<<<persistent_grid(k_momentum_batch, 256, 0, total), 256, 0, st>>>(jobs, offs, n, total);
}
void launch_residual_batch(const ResidualJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    if (total <= 0) return;
    k_residual_batch<<<persistent_grid(k_residual_batch, kRedThreads, 0, total), kRedThreads, 0, st>>>(jobs, offs, n,
                                                                                                       total);
}
void launch_stop_batch(const StopJob *jobs, int n, cudaStream_t st) {
    if (n <= 0) return;
    k_stop_batch<<<persistent_grid(k_stop_batch, kRedThreads, 0, n), kRedThreads, 0, st>>>(jobs, n);
}
void launch_update_batch(const UpdateJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    if (total <= 0) return;
    k_update_batch<<<persistent_grid(k_update_batch, 128, 0, total), 128, 0, st>>>(jobs, offs, n, total);
}

}  // namespace mpiffl
