// Parallel-beam projector P_theta and its gather-form transpose
// (Sec. 2.2, Eqs. (16)-(19); Joseph interpolation, see AngleParam).
//
// Both directions process kZc z slices per thread: every slice shares the ray
// geometry, so the interpolation weights are computed once per kZc samples.
// Column-marched angles read a transposed copy of the volume, so that every
// staged voxel line is contiguous.
#include "internal.h"
#include "tc_ptx.cuh"

namespace mpiffl {

__device__ __forceinline__ void transpose_body(const float *__restrict__ vol, float *__restrict__ volT, int N,
                                               int bx, int by, int bz) {
    __shared__ float tile[32][33];
    const size_t zoff = (size_t)bz * N * N;
    int x = bx * 32 + threadIdx.x;
    int y0 = by * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int y = y0 + k;
        if (x < N && y < N) tile[k][threadIdx.x] = vol[zoff + (size_t)y * N + x];
    }
    __syncthreads();
    int yo = by * 32 + threadIdx.x;
    int x0 = bx * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int xo = x0 + k;
        if (xo < N && yo < N) volT[zoff + (size_t)xo * N + yo] = tile[threadIdx.x][k];
    }
}

__global__ void k_transpose_xy(const float *__restrict__ vol, float *__restrict__ volT, int N) {
    transpose_body(vol, volT, N, blockIdx.x, blockIdx.y, blockIdx.z);
}

void launch_transpose_xy(const float *vol, float *volT, int N, int Nz, cudaStream_t st) {
    dim3 grid((N + 31) / 32, (N + 31) / 32, Nz), block(32, 8);
    k_transpose_xy<<<grid, block, 0, st>>>(vol, volT, N);
}

// Forward: a block owns kProjAnglesPerBlock angles of one orientation and kZc slices. At
// march step s the block stages voxel line s of its kZc slices in shared memory
// (double-buffered, loads for step s+1 in flight while step s is summed); each
// thread is one ray (angle, bin i) and adds its interpolated sample for all kZc
// slices at once, so the interpolation weights are computed once per kZc samples.
constexpr int kZc = 8;
constexpr int kMaxLd = 8;  // staged floats per thread and step

__global__ void __launch_bounds__(1024) k_project(const float *__restrict__ vol, const float *__restrict__ volT,
                                                  const AngleParam *__restrict__ ang,
                                                  const int *__restrict__ agroups, float *__restrict__ proj,
                                                  int N, int Nz, int rays_per_angle) {
    extern __shared__ float sm[];  // 2 x kZc x N
    const int z0 = blockIdx.y * kZc;
    const int nz = min(kZc, Nz - z0);
    const int slot = threadIdx.x / rays_per_angle;
    const int i = threadIdx.x % rays_per_angle;
    const int m = agroups[blockIdx.x * kProjAnglesPerBlock + slot];
    const bool active = (m >= 0) && (i < N);
    const AngleParam ap = ang[m >= 0 ? m : agroups[blockIdx.x * kProjAnglesPerBlock]];
    const float *src = ap.row_major ? vol : volT;  // one orientation per block
    const float c = 0.5f * (float)(N - 1);
    const float fi = fmaf(ap.inv_c, (float)i - c, c);
    const int nld = kZc * N;
    float acc[kZc];
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] = 0.f;
    float reg[kMaxLd];
    auto fetch = [&](int s) {
#pragma unroll
        for (int u = 0; u < kMaxLd; ++u) {
            const int t = threadIdx.x + u * blockDim.x;
            const int zz = t / N, x = t - zz * N;
            reg[u] = (t < nld && zz < nz) ? __ldg(src + ((size_t)(z0 + zz) * N + s) * N + x) : 0.f;
        }
    };
    auto stash = [&](float *dst) {
#pragma unroll
        for (int u = 0; u < kMaxLd; ++u) {
            const int t = threadIdx.x + u * blockDim.x;
            if (t < nld) dst[t] = reg[u];
        }
    };
    fetch(0);
    stash(sm);
    __syncthreads();
    for (int s = 0; s < N; ++s) {
        const float *cur = sm + (s & 1) * nld;
        if (s + 1 < N) fetch(s + 1);
        if (active) {
            const float f = fmaf(ap.slope, (float)s - c, fi);
            const float fl = floorf(f);
            const int k = (int)fl;
            const float t = f - fl;
            const float w0 = (k >= 0 && k < N) ? 1.f - t : 0.f;
            const float w1 = (k + 1 >= 0 && k + 1 < N) ? t : 0.f;
            const int k0 = min(max(k, 0), N - 1);
            const int k1 = min(max(k + 1, 0), N - 1);
#pragma unroll
            for (int zz = 0; zz < kZc; ++zz) acc[zz] = fmaf(w0, cur[zz * N + k0], fmaf(w1, cur[zz * N + k1], acc[zz]));
        }
        if (s + 1 < N) stash(sm + ((s + 1) & 1) * nld);
        __syncthreads();
    }
    if (active) {
#pragma unroll
        for (int zz = 0; zz < kZc; ++zz)
            if (zz < nz) proj[((size_t)m * Nz + z0 + zz) * N + i] = acc[zz] * ap.scale;
    }
}

// Pipelined variant (N % 4 == 0): an extra producer warp streams voxel line s of the
// block's kZc slices into a ring of kPStages shared-memory stages with bulk copies
// that complete on full[stage]; every consumer warp signals empty[stage] when it has
// used a stage, so no block-wide barrier sits in the march loop.
constexpr int kPStages = 8;

__device__ __forceinline__ void project_pipe_body(const float *__restrict__ vol, const float *__restrict__ volT,
                                                  const AngleParam *__restrict__ ang,
                                                  const int *__restrict__ agroups, float *__restrict__ proj,
                                                  int N, int Nz, int rays_per_angle, int *err, int bx, int by,
                                                  float *psm) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(psm + kPStages * kZc * N);  // full[K], empty[K]
    const int nthreads_c = rays_per_angle * kProjAnglesPerBlock;  // consumers
    const int ncw = nthreads_c / 32;
    const int z0 = by * kZc;
    const int nz = min(kZc, Nz - z0);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < kPStages; ++k) {
            ptx::mbar_init(&bars[k], 1);
            ptx::mbar_init(&bars[kPStages + k], ncw);
        }
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const AngleParam a0 = ang[agroups[bx * kProjAnglesPerBlock]];
    const float *src = a0.row_major ? vol : volT;  // one orientation per block
    const uint32_t row_bytes = (uint32_t)N * 4u;
    if (tid >= nthreads_c) {
        // ---------------------------------------------------------------- producer warp
        if (tid == nthreads_c) {
            for (int s = 0; s < N; ++s) {
                const int k = s % kPStages;
                if (s >= kPStages && !ptx::mbar_wait_bounded(&bars[kPStages + k], ((s / kPStages) - 1) & 1, 1u << 24)) {
                    atomicExch(err, 1);
                    break;
                }
                float *dst = psm + k * kZc * N;
                ptx::mbar_arrive_expect_tx(&bars[k], row_bytes * nz);
                for (int zz = 0; zz < nz; ++zz)
                    ptx::bulk_g2s(dst + zz * N, src + ((size_t)(z0 + zz) * N + s) * N, row_bytes, &bars[k]);
            }
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    const int slot = tid / rays_per_angle;
    const int i = tid % rays_per_angle;
    const int m = agroups[bx * kProjAnglesPerBlock + slot];
    const bool active = (m >= 0) && (i < N);
    const AngleParam ap = ang[m >= 0 ? m : agroups[bx * kProjAnglesPerBlock]];
    const float c = 0.5f * (float)(N - 1);
    const float fi = fmaf(ap.inv_c, (float)i - c, c);
    float acc[kZc];
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] = 0.f;
    bool good = true;
    for (int s = 0; s < N; ++s) {
        const int k = s % kPStages;
        if (!ptx::mbar_wait_bounded(&bars[k], (s / kPStages) & 1, 1u << 24)) {
            good = false;
            break;
        }
        const float *cur = psm + k * kZc * N;
        if (active) {
            const float f = fmaf(ap.slope, (float)s - c, fi);
            const float fl = floorf(f);
            const int kk = (int)fl;
            const float t = f - fl;
            const float w0 = (kk >= 0 && kk < N) ? 1.f - t : 0.f;
            const float w1 = (kk + 1 >= 0 && kk + 1 < N) ? t : 0.f;
            const int k0 = min(max(kk, 0), N - 1);
            const int k1 = min(max(kk + 1, 0), N - 1);
#pragma unroll
            for (int zz = 0; zz < kZc; ++zz)
                if (zz < nz) acc[zz] = fmaf(w0, cur[zz * N + k0], fmaf(w1, cur[zz * N + k1], acc[zz]));
        }
        __syncwarp();
        if ((tid & 31) == 0) ptx::mbar_arrive(&bars[kPStages + k]);
    }
    if (!good) {
        if ((tid & 31) == 0) atomicExch(err, 1);
        return;
    }
    if (active) {
#pragma unroll
        for (int zz = 0; zz < kZc; ++zz)
            if (zz < nz) proj[((size_t)m * Nz + z0 + zz) * N + i] = acc[zz] * ap.scale;
    }
}

__global__ void __launch_bounds__(1024 + 32) k_project_pipe(const float *__restrict__ vol,
                                                            const float *__restrict__ volT,
                                                            const AngleParam *__restrict__ ang,
                                                            const int *__restrict__ agroups,
                                                            float *__restrict__ proj, int N, int Nz,
                                                            int rays_per_angle, int *err) {
    extern __shared__ __align__(128) float psm[];  // kPStages x kZc x N
    project_pipe_body(vol, volT, ang, agroups, proj, N, Nz, rays_per_angle, err, blockIdx.x, blockIdx.y, psm);
}

void launch_project(const float *vol, const float *volT, const AngleParam *ang, const int *agroups,
                    int n_agroups, float *proj, int N, int Nz, cudaStream_t st, int *err) {
    const int rays = (N + 31) / 32 * 32;
    if (N % 4 == 0 && err) {
        const size_t smem = sizeof(float) * kPStages * kZc * N + 16 * kPStages;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_project_pipe, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        dim3 grid(n_agroups, (Nz + kZc - 1) / kZc);
        k_project_pipe<<<grid, rays * kProjAnglesPerBlock + 32, smem, st>>>(vol, volT, ang, agroups, proj, N, Nz,
                                                                            rays, err);
        return;
    }
    const int threads = rays * kProjAnglesPerBlock;
    const size_t smem = sizeof(float) * 2 * kZc * N;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    dim3 grid(n_agroups, (Nz + kZc - 1) / kZc);
    k_project<<<grid, threads, smem, st>>>(vol, volT, ang, agroups, proj, N, Nz, rays);
}

// Transpose: a thread owns one voxel column (x, y) and kZc slices. For every angle
// the rays whose interpolation touches the voxel are among i1-1, i1, i1+1 (i1 the
// nearest ray); ray i's sample position f_i is recomputed with the forward's exact
// arithmetic and its weight max(0, 1 - |f_i - q|) equals the forward's (1-t or t)
// bit for bit. The kZc projection values of each ray are gathered. No atomics.
__device__ __forceinline__ void backproject_body(const float *__restrict__ proj, const AngleParam *__restrict__ ang,
                                                 float *__restrict__ vol, int N, int Nz, int M, int bx, int by,
                                                 int bz) {
    const int x = bx * 32 + threadIdx.x;
    const int y = by * 8 + threadIdx.y;
    const int z0 = bz * kZc;
    const int nz = min(kZc, Nz - z0);
    if (x >= N || y >= N) return;
    const float c = 0.5f * (float)(N - 1);
    float acc[kZc];
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] = 0.f;
    for (int m = 0; m < M; ++m) {
        const AngleParam a = ang[m];
        const int s = a.row_major ? y : x;             // march step holding this voxel
        const float q = (float)(a.row_major ? x : y);  // its index along the step's line
        const float sm = (float)s - c;
        // nearest ray: inv_c (i - c) + slope (s - c) + c = q
        const int i1 = __float2int_rn(fmaf(q - fmaf(a.slope, sm, c), a.inv_c_rcp, c));
        float w[3];
        int ii[3];
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const int i = i1 - 1 + u;
            const float f = fmaf(a.slope, sm, fmaf(a.inv_c, (float)i - c, c));  // the forward's f
            const bool in = (i >= 0) && (i < N);
            w[u] = in ? fmaxf(0.f, 1.f - fabsf(f - q)) * a.scale : 0.f;
            ii[u] = in ? i : 0;
        }
        // at most two consecutive rays carry weight: (i1-1, i1) or (i1, i1+1)
        const bool lo = w[0] != 0.f;
        const float wA = lo ? w[0] : w[1], wB = lo ? w[1] : w[2];
        const int iA = lo ? ii[0] : ii[1], iB = lo ? ii[1] : ii[2];
        const float *pm = proj + ((size_t)m * Nz + z0) * N;
#pragma unroll
        for (int zz = 0; zz < kZc; ++zz)
            if (zz < nz) acc[zz] = fmaf(wA, __ldg(pm + zz * N + iA), fmaf(wB, __ldg(pm + zz * N + iB), acc[zz]));
    }
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz)
        if (zz < nz) vol[((size_t)(z0 + zz) * N + y) * N + x] = acc[zz];
}

__global__ void __launch_bounds__(256) k_backproject(const float *__restrict__ proj,
                                                     const AngleParam *__restrict__ ang,
                                                     float *__restrict__ vol, int N, int Nz, int M) {
    backproject_body(proj, ang, vol, N, Nz, M, blockIdx.x, blockIdx.y, blockIdx.z);
}

void launch_backproject(const float *proj, const AngleParam *ang, float *vol, int N, int Nz,
                        int M, cudaStream_t st) {
    dim3 grid((N + 31) / 32, (N + 7) / 8, (Nz + kZc - 1) / kZc), block(32, 8);
    k_backproject<<<grid, block, 0, st>>>(proj, ang, vol, N, Nz, M);
}

// ---------------------------------------------------------------------- batches
// One launch serves several problems: block b belongs to the problem j with
// offs[j] <= b < offs[j + 1]; its local block index is b - offs[j].
__device__ __forceinline__ int batch_find(const int *__restrict__ offs, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_transpose_batch(const TransposeJob *__restrict__ jobs, const int *__restrict__ offs, int n) {
    const int j = batch_find(offs, n, blockIdx.x);
    const TransposeJob J = jobs[j];
    if (J.done && *J.done) return;
    int b = blockIdx.x - offs[j];
    const int gx = (J.N + 31) / 32;
    const int bx = b % gx, by = (b / gx) % gx, bz = b / (gx * gx);
    transpose_body(J.vol, J.volT, J.N, bx, by, bz);
}

__global__ void __launch_bounds__(1024 + 32) k_project_batch(const ProjectJob *__restrict__ jobs,
                                                             const int *__restrict__ offs, int n, int *err) {
    extern __shared__ __align__(128) float psm[];
    const int j = batch_find(offs, n, blockIdx.x);
    const ProjectJob J = jobs[j];
    if (J.done && *J.done) return;
    const int b = blockIdx.x - offs[j];
    const int rays = (J.N + 31) / 32 * 32;
    if ((int)threadIdx.x >= rays * kProjAnglesPerBlock + 32) {
        // threads beyond this problem's block shape take no part (barrier counts use its shape)
        __syncthreads();
        return;
    }
    project_pipe_body(J.vol, J.volT, J.ang, J.agroups, J.proj, J.N, J.Nz, rays, err, b % J.n_agroups,
                      b / J.n_agroups, psm);
}

__global__ void __launch_bounds__(256) k_backproject_batch(const BackprojectJob *__restrict__ jobs,
                                                           const int *__restrict__ offs, int n) {
    const int j = batch_find(offs, n, blockIdx.x);
    const BackprojectJob J = jobs[j];
    if (J.done && *J.done) return;
    const int b = blockIdx.x - offs[j];
    const int gx = (J.N + 31) / 32, gy = (J.N + 7) / 8;
    backproject_body(J.proj, J.ang, J.vol, J.N, J.Nz, J.M, b % gx, (b / gx) % gy, b / (gx * gy));
}

int transpose_blocks(int N, int Nz) { return ((N + 31) / 32) * ((N + 31) / 32) * Nz; }
int project_blocks(int n_agroups, int Nz) { return n_agroups * ((Nz + kZc - 1) / kZc); }
int backproject_blocks(int N, int Nz) { return ((N + 31) / 32) * ((N + 7) / 8) * ((Nz + kZc - 1) / kZc); }

void launch_transpose_batch(const TransposeJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    k_transpose_batch<<<total, dim3(32, 8), 0, st>>>(jobs, offs, n);
}

void launch_project_batch(const ProjectJob *jobs, const int *offs, int n, int total, int maxN, int *err,
                          cudaStream_t st) {
    const int rays = (maxN + 31) / 32 * 32;
    const size_t smem = sizeof(float) * kPStages * kZc * maxN + 16 * kPStages;
    cudaFuncSetAttribute(k_project_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_project_batch<<<total, rays * kProjAnglesPerBlock + 32, smem, st>>>(jobs, offs, n, err);
}

void launch_backproject_batch(const BackprojectJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    k_backproject_batch<<<total, dim3(32, 8), 0, st>>>(jobs, offs, n);
}

}  // namespace mpiffl
