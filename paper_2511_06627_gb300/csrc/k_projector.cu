// Parallel-beam projector P_theta and its gather-form transpose
// (Sec. 2.2, Eqs. (16)-(19); Joseph interpolation, see AngleParam).
//
// Both directions process kZc z slices per thread: every slice shares the ray
// geometry, so the interpolation weights are computed once per kZc samples.
// Column-marched angles read a transposed copy of the volume, so that every
// staged voxel line is contiguous.
#include <algorithm>

#include "internal.h"
#include "split_operands.cuh"
#include "tc_ptx.cuh"

namespace mpiffl {

// Cell and fraction of a Q32.32 position: floor and f - floor, the fraction cut to
// its top 23 bits. The float is assembled from the bits, 1 + m 2^-23 with m the
// fraction's top 23 bits, minus 1: exact, in [0, 1), and on the integer and FMA pipes
// rather than the conversion unit.
__device__ __forceinline__ void fx_split(long long f, int &k, float &t) {
    k = (int)(f >> 32);
    t = __uint_as_float(0x3f800000u | ((unsigned)f >> 9)) - 1.0f;
}

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

// Vector form (N % 4 == 0, 16-byte aligned): a block of 8 x 32 threads moves one 32 x 32
// tile of two slices; thread (tx, ty) reads 4 consecutive x of row ty of both slices
// (two 16-byte loads in flight) and writes 4 consecutive y of output row ty. The
// column reads of the padded tiles hit 32 distinct banks per warp.
__global__ void __launch_bounds__(256) k_transpose_xy4(const float *__restrict__ vol, float *__restrict__ volT,
                                                       int N, int Nz) {
    __shared__ float tile[2][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int z0 = 2 * blockIdx.z;
    const size_t slice = (size_t)N * N;
    float4 v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (z0 + u < Nz && y0 + ty < N && x0 + 4 * tx < N)
            v[u] = __ldg(reinterpret_cast<const float4 *>(vol + (z0 + u) * slice + (y0 + ty) * N + x0 + 4 * tx));
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        tile[u][ty][4 * tx] = v[u].x;
        tile[u][ty][4 * tx + 1] = v[u].y;
        tile[u][ty][4 * tx + 2] = v[u].z;
        tile[u][ty][4 * tx + 3] = v[u].w;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (z0 + u < Nz && x0 + ty < N && y0 + 4 * tx < N)
            *reinterpret_cast<float4 *>(volT + (z0 + u) * slice + (x0 + ty) * N + y0 + 4 * tx) =
                make_float4(tile[u][4 * tx][ty], tile[u][4 * tx + 1][ty], tile[u][4 * tx + 2][ty],
                            tile[u][4 * tx + 3][ty]);
}

void launch_transpose_xy(const float *vol, float *volT, int N, int Nz, cudaStream_t st) {
    if (N % 4 == 0 && ((reinterpret_cast<uintptr_t>(vol) | reinterpret_cast<uintptr_t>(volT)) & 15) == 0) {
        dim3 grid((N + 31) / 32, (N + 31) / 32, (Nz + 1) / 2), block(8, 32);
        k_transpose_xy4<<<grid, block, 0, st>>>(vol, volT, N, Nz);
        return;
    }
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
    const long long f0 = ap.fx_a + (long long)i * ap.fx_d;
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
            int k;
            float t;
            fx_split(f0 + (long long)s * ap.fx_b, k, t);
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

// Pipelined variant (N % 4 == 0, N <= 512): an extra producer warp streams voxel line
// s of the block's kZc slices into a ring of kPStages shared-memory stages with bulk
// copies that complete on full[stage]; every consumer warp signals empty[stage] when
// it has used a stage, so no block-wide barrier sits in the march loop. Each staged
// line sits between kPad zeros on the left and at least 4 on the right (row stride
// LD >= N + 8, a compile-time constant), so a tap index clamped to [-2, N] reads a
// zero outside the grid: the taps need no range checks, the slice offsets are
// immediates, and the sums equal those of the checked form (a zero tap adds nothing).
constexpr int kPStages = 12;
constexpr int kPad = 4;
// the interleaved projector's stages go in groups of kPGroup march steps, one pair of
// barriers per group (fewer waits and arrivals per step)
constexpr int kPGroup = 4, kPSlots = kPStages / kPGroup;

template <int LD>
__device__ __forceinline__ void project_pipe_body(const float *__restrict__ vol, const float *__restrict__ volT,
                                                  const AngleParam *__restrict__ ang,
                                                  const int *__restrict__ agroups, float *__restrict__ proj,
                                                  int N, int Nz, int rays_per_angle, int *err, int bx, int by,
                                                  float *psm) {
    uint64_t *bars = reinterpret_cast<uint64_t *>(psm + kPStages * kZc * LD);  // full[K], empty[K]
    const int nthreads_c = rays_per_angle * kProjAnglesPerBlock;  // consumers
    const int ncw = nthreads_c / 32;
    const int z0 = by * kZc;
    const int nz = min(kZc, Nz - z0);
    const int tid = threadIdx.x;
    // zero the pads of every staged line: [0, kPad) and [kPad + N, LD). The stride is
    // this problem's thread count: in a batch launch, threads past it have left.
    const int padw = LD - N;
    for (int t = tid; t < kPStages * kZc * padw; t += nthreads_c + 32) {
        const int row = t / padw, cpos = t - row * padw;
        psm[row * LD + (cpos < kPad ? cpos : N + cpos)] = 0.f;
    }
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
        // lane 0 announces the stage's bytes, then lane zz copies slice zz: the nz
        // copies of a step are issued side by side, not one after another
        const int lane = tid - nthreads_c;
        for (int s = 0; s < N; ++s) {
            const int k = s % kPStages;
            int ok = 1;  // lane 0 waits for the stage to be free; the warp leaves together
            if (s >= kPStages && lane == 0)
                ok = ptx::mbar_wait_bounded(&bars[kPStages + k], ((s / kPStages) - 1) & 1, 1u << 24);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            float *dst = psm + k * kZc * LD + kPad;
            if (lane == 0) ptx::mbar_arrive_expect_tx(&bars[k], row_bytes * nz);
            __syncwarp();
            if (lane < nz) {
                // the consumers read the stage with ordinary loads (generic proxy) and
                // the bulk copy writes it through the async proxy: the empty barrier
                // orders the two only with this fence between them
                ptx::fence_proxy_async_smem();
                ptx::bulk_g2s(dst + lane * LD, src + ((size_t)(z0 + lane) * N + s) * N, row_bytes, &bars[k]);
            }
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    // The warps of an inactive slot (a block with one angle) only wait and arrive, as do
    // the warps all of whose rays lie off the grid at a step (both taps on the zero pads:
    // nothing to add). Threads beyond the last ray run the loop on clamped, in-bounds
    // taps and store nothing; slices past nz hold stale data, never stored.
    const int slot = tid / rays_per_angle;
    const int i = tid % rays_per_angle;
    const int m = agroups[bx * kProjAnglesPerBlock + slot];
    const bool active = (m >= 0) && (i < N);
    const AngleParam ap = ang[m >= 0 ? m : agroups[bx * kProjAnglesPerBlock]];
    long long fs = ap.fx_a + (long long)i * ap.fx_d;  // position of ray i at march step s
    float acc[kZc];
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] = 0.f;
    bool good = true;
    for (int s = 0; s < N; ++s, fs += ap.fx_b) {
        const int k = s % kPStages;
        // the warp gives up as one, so that its vote below sees all lanes
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&bars[k], (s / kPStages) & 1, 1u << 24))) {
            good = false;
            break;
        }
        int cell;
        float t;
        fx_split(fs, cell, t);
        if (m >= 0 && __any_sync(0xffffffffu, cell >= -1 && cell <= N - 1)) {  // m: uniform per warp
            const int kk = min(max(cell, -2), N);
            const float *p = psm + k * kZc * LD + kPad + kk;
#pragma unroll
            for (int zz = 0; zz < kZc; ++zz) acc[zz] = fmaf(1.f - t, p[zz * LD], fmaf(t, p[zz * LD + 1], acc[zz]));
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

template <int LD>
__global__ void __launch_bounds__(1024 + 32) k_project_pipe(const float *__restrict__ vol,
                                                            const float *__restrict__ volT,
                                                            const AngleParam *__restrict__ ang,
                                                            const int *__restrict__ agroups,
                                                            float *__restrict__ proj, int N, int Nz,
                                                            int rays_per_angle, int *err) {
    extern __shared__ __align__(128) float psm[];  // kPStages x kZc x LD
    project_pipe_body<LD>(vol, volT, ang, agroups, proj, N, Nz, rays_per_angle, err, blockIdx.x, blockIdx.y, psm);
}

// Smallest compiled row stride that holds N + 8 floats; 0 if N is above 512.
int pipe_ld(int N) {
    for (int ld : {40, 72, 136, 200, 264, 392, 520})
        if (N + 8 <= ld) return ld;
    return 0;
}

size_t pipe_smem(int ld) { return sizeof(float) * kPStages * kZc * ld + 16 * kPStages; }

// The pipelined and interleaved projectors run kProjAnglesPerBlock angles of
// (N + 31) / 32 * 32 rays each plus a producer warp in one block: at most 1024 threads,
// so N <= 496; wider detectors take the plain projector.
bool pipe_threads_ok(int N) { return (N + 31) / 32 * 32 * kProjAnglesPerBlock + 32 <= 1024; }

bool pipe_ok(const float *vol, const float *volT, int N) {
    return N % 4 == 0 && pipe_ld(N) > 0 && pipe_threads_ok(N) && (reinterpret_cast<uintptr_t>(vol) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(volT) & 15) == 0;
}

template <int LD>
void launch_pipe(dim3 grid, int threads, cudaStream_t st, const float *vol, const float *volT, const AngleParam *ang,
                 const int *agroups, float *proj, int N, int Nz, int rays, int *err) {
    cudaFuncSetAttribute(k_project_pipe<LD>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_project_pipe<LD><<<grid, threads, pipe_smem(LD), st>>>(vol, volT, ang, agroups, proj, N, Nz, rays, err);
}

void launch_project(const float *vol, const float *volT, const AngleParam *ang, const int *agroups,
                    int n_agroups, float *proj, int N, int Nz, cudaStream_t st, int *err) {
    const int rays = (N + 31) / 32 * 32;
    if (err && pipe_ok(vol, volT, N)) {
        dim3 grid(n_agroups, (Nz + kZc - 1) / kZc);
        const int threads = rays * kProjAnglesPerBlock + 32;
        switch (pipe_ld(N)) {
        case 40: launch_pipe<40>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        case 72: launch_pipe<72>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        case 136: launch_pipe<136>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        case 200: launch_pipe<200>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        case 264: launch_pipe<264>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        case 392: launch_pipe<392>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        default: launch_pipe<520>(grid, threads, st, vol, volT, ang, agroups, proj, N, Nz, rays, err); break;
        }
        return;
    }
    const int threads = rays * kProjAnglesPerBlock;
    const size_t smem = sizeof(float) * 2 * kZc * N;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    dim3 grid(n_agroups, (Nz + kZc - 1) / kZc);
    k_project<<<grid, threads, smem, st>>>(vol, volT, ang, agroups, proj, N, Nz, rays);
}

// Interleaved variant (same shapes as the pipelined one). The volume is copied once with
// each line's kZc slices innermost, volI[z block][y][x][kZc]. A march step is one tensor
// copy of the step's line: a row of volI for row-marched angles, a column (32-byte
// pieces N rows apart) for column-marched ones. The copy writes shared memory with the
// 32-byte swizzle, which swaps the two 16-byte halves of staged position p when bit 2
// of p is set (stage bases are 256-byte aligned). A ray reads its two taps for all kZc
// slices with four 16-byte loads. Eight rays whose positions differ mod 8 read eight
// distinct 16-byte bank groups: position p puts slices 0-3 in group
// 2p + ((p >> 2) & 1) mod 8. The sums are those of the pipelined variant, slice by slice.
__host__ __device__ __forceinline__ int il_swap(int cs) { return (cs >> 2) & 1; }

// Shared-memory wavefronts one angle costs the interleaved projector for one slice
// block: per active warp-step, its four 16-byte tap loads, each quarter warp taking one
// wavefront per distinct 16-byte address in its most used bank group (a model that
// matches the measured bank conflicts), over 8 march steps spread over the N (the
// angles rank as with all steps). The host uses it to give the projector blocks equal
// work; at 256 bins and 36 angles it costs about 2 ms at handle creation.
double project_il_cost(const AngleParam &a, int N) {
    const int rays = (N + 31) / 32 * 32;
    const int stride = std::max(1, N / 8);
    double total = 0.0;
    int cs[32];
    for (int s = stride / 2; s < N; s += stride) {
        for (int w = 0; w < rays; w += 32) {
            bool any = false;
            for (int l = 0; l < 32; ++l) {
                const long long f = a.fx_a + (long long)(w + l) * a.fx_d + (long long)s * a.fx_b;
                const int cell = (int)(f >> 32);
                any |= cell >= -1 && cell <= N - 1;
                cs[l] = std::min(std::max(cell, -2), N) + kPad;
            }
            if (!any) continue;
            for (int ld = 0; ld < 4; ++ld) {
                const int dp = ld >> 1, h = ld & 1;
                for (int q = 0; q < 4; ++q) {
                    int addr[8], per_group[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    int worst = 0;
                    for (int j = 0; j < 8; ++j) {
                        const int p = cs[8 * q + j] + dp;
                        addr[j] = 2 * p + (h ^ il_swap(p));
                        bool seen = false;
                        for (int k = 0; k < j; ++k) seen |= addr[k] == addr[j];
                        if (!seen) worst = std::max(worst, ++per_group[addr[j] & 7]);
                    }
                    total += worst;
                }
            }
        }
    }
    return total;
}

size_t il_len(int N, int Nz) { return (size_t)((Nz + kZc - 1) / kZc) * kZc * N * N; }

// volI[zb][y][x][e] = vol[kZc zb + e][y][x] (zero past Nz). A block of 8 x 32 threads
// moves a 32 x 32 tile of one slice block:
// thread (tx, ty) loads 4 consecutive x of row ty of every slice (eight 16-byte loads;
// N % 4 == 0) and forms each position's two halves in registers. The tile goes through
// shared memory as 16-byte halves: half h of tile row r, column c sits at 16-byte slot
// 64 r + 8 (c >> 2) + ((2 (c & 3) + h) ^ sw), sw = (c >> 2) ^ 2 (r & 3). The rows are
// then written from the tile, 32 consecutive 16-byte units of one output row per warp
// (full 128-byte lines). Every 8-lane phase takes 8 distinct bank groups: the tile
// stores (c = 4 tx + q, tx over the lanes) and the row reads (four aligned positions,
// both halves).
__device__ __forceinline__ int il_tile_slot(int r, int c, int h) {
    return 64 * r + 8 * (c >> 2) + ((2 * (c & 3) + h) ^ (((c >> 2) ^ (2 * (r & 3))) & 7));
}

__global__ void __launch_bounds__(256) k_interleave(const float *__restrict__ vol, float *__restrict__ volI, int N,
                                                    int Nz) {
    __shared__ float4 tile[32 * 64];  // 32 rows x 32 columns x 2 halves
    const int tx = threadIdx.x, ty = threadIdx.y;  // 8 x 32
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, zb = blockIdx.z;
    const int y = y0 + ty, xs = x0 + 4 * tx;
    ptx::grid_dep_wait();  // the volume comes from the previous kernel
    ptx::grid_dep_launch();
    float4 v[kZc];
#pragma unroll
    for (int e = 0; e < kZc; ++e) {
        const int z = zb * kZc + e;
        v[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (z < Nz && y < N && xs < N) v[e] = __ldg(reinterpret_cast<const float4 *>(vol + ((size_t)z * N + y) * N + xs));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float f0 = q == 0 ? v[0].x : q == 1 ? v[0].y : q == 2 ? v[0].z : v[0].w;
        const float f1 = q == 0 ? v[1].x : q == 1 ? v[1].y : q == 2 ? v[1].z : v[1].w;
        const float f2 = q == 0 ? v[2].x : q == 1 ? v[2].y : q == 2 ? v[2].z : v[2].w;
        const float f3 = q == 0 ? v[3].x : q == 1 ? v[3].y : q == 2 ? v[3].z : v[3].w;
        const float f4 = q == 0 ? v[4].x : q == 1 ? v[4].y : q == 2 ? v[4].z : v[4].w;
        const float f5 = q == 0 ? v[5].x : q == 1 ? v[5].y : q == 2 ? v[5].z : v[5].w;
        const float f6 = q == 0 ? v[6].x : q == 1 ? v[6].y : q == 2 ? v[6].z : v[6].w;
        const float f7 = q == 0 ? v[7].x : q == 1 ? v[7].y : q == 2 ? v[7].z : v[7].w;
        const int c = 4 * tx + q;
        tile[il_tile_slot(ty, c, 0)] = make_float4(f0, f1, f2, f3);
        tile[il_tile_slot(ty, c, 1)] = make_float4(f4, f5, f6, f7);
    }
    __syncthreads();
    // thread t writes 16-byte unit j = t mod 64 (position j / 2, half j mod 2) of tile
    // rows 4 i + t / 64
    const int t = ty * 8 + tx, j = t & 63, c = j >> 1, m = j & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = 4 * i + (t >> 6);
        const int yy = y0 + r, x = x0 + c;  // volI: row yy, position x
        if (yy < N && x < N)
            reinterpret_cast<float4 *>(volI + (((size_t)zb * N + yy) * N + x) * kZc)[m] = tile[il_tile_slot(r, c, m)];
    }
}

void launch_interleave(const float *vol, float *volI, int N, int Nz, cudaStream_t st) {
    dim3 grid((N + 31) / 32, (N + 31) / 32, (Nz + kZc - 1) / kZc), block(8, 32);
    launch_dependent(k_interleave, grid, block, 0, st, vol, volI, N, Nz);
}

// Tensor maps of volI as a 4-D array (kZc floats, x, y, z block): boxes of one row
// (kZc x box x 1 x 1) and of one column (kZc x 1 x box x 1), 32-byte swizzle, zero fill
// past the volume's edge.
bool make_il_maps(const float *volI, int N, int Nz, IlMaps *maps) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    // looked up once, thread-safely (handles may be created from several threads)
    static const Encode encode = []() -> Encode {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<Encode>(fn);
    }();
    if (!encode) return false;
    const int nbox = (N + 255) / 256;
    const int box = ((N + nbox - 1) / nbox + 3) / 4 * 4;
    if (kPad + nbox * box > pipe_ld(N)) return false;  // the boxes' zero fill stays inside the stage
    const cuuint64_t dims[4] = {(cuuint64_t)kZc, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)((Nz + kZc - 1) / kZc)};
    const cuuint64_t strides[3] = {(cuuint64_t)kZc * 4, (cuuint64_t)kZc * 4 * N, (cuuint64_t)kZc * 4 * N * N};
    const cuuint32_t elem[4] = {1, 1, 1, 1};
    const cuuint32_t brow[4] = {(cuuint32_t)kZc, (cuuint32_t)box, 1, 1};
    const cuuint32_t bcol[4] = {(cuuint32_t)kZc, 1, (cuuint32_t)box, 1};
    void *base = const_cast<float *>(volI);
    if (encode(&maps->row, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, brow, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        encode(&maps->col, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, bcol, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    maps->nbox = nbox;
    maps->box = box;
    return true;
}

// One tensor copy of box positions from volI into shared memory (4-D coordinates:
// slice 0, x, y, z block), completing its bytes on *bar.
__device__ __forceinline__ void il_copy(float *dst, const CUtensorMap *map, int x, int y, int zb, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(ptx::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(zb), "r"(ptx::smem_u32(bar))
        : "memory");
}

template <int LDC>
__global__ void __launch_bounds__(1024 + 32) k_project_il(const __grid_constant__ CUtensorMap map_row,
                                                          const __grid_constant__ CUtensorMap map_col, int nbox,
                                                          int box, const AngleParam *__restrict__ ang,
                                                          const int *__restrict__ agroups, float *__restrict__ proj,
                                                          int N, int Nz, int rays_per_angle, int *err,
                                                          uint32_t inject, ProjPack pack) {
    extern __shared__ __align__(128) float psm[];  // kPStages x LDC positions x kZc
    // kPGroup consecutive march steps share one pair of barriers: full[kPSlots], empty[kPSlots]
    uint64_t *bars = reinterpret_cast<uint64_t *>(psm + kPStages * LDC * kZc);
    const int bx = blockIdx.x, zb = blockIdx.y;
    const int nthreads_c = rays_per_angle * kProjAnglesPerBlock;  // consumers
    const int ncw = nthreads_c / 32;
    const int z0 = zb * kZc;
    const int nz = min(kZc, Nz - z0);
    const int tid = threadIdx.x;
    // the 32-byte swizzle is a function of the shared address: the stages must start on
    // 256-byte boundaries for it to swap the halves of staged positions as il_swap says
    if (ptx::smem_u32(psm) & 255u) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    // zero the pad positions [0, kPad) and [kPad + N, LDC) of every stage
    const int padp = LDC - N;
    for (int t = tid; t < kPStages * padp * kZc; t += nthreads_c + 32) {
        const int stg = t / (padp * kZc), r = t - stg * padp * kZc;
        const int pp = r / kZc, e = r - pp * kZc;
        psm[((size_t)stg * LDC + (pp < kPad ? pp : N + pp)) * kZc + e] = 0.f;
    }
    if (tid == 0) {
        for (int u = 0; u < kPSlots; ++u) {
            ptx::mbar_init(&bars[u], 1);
            ptx::mbar_init(&bars[kPSlots + u], ncw);
        }
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (inject > 0) {
        // failure-detection test hook: before any copy is issued, every thread waits on
        // the first empty barrier, which only the consumers (all waiting here) would
        // complete; the bounded waits run out, the block records a timeout and returns
        if (!ptx::mbar_wait_bounded(&bars[kPSlots], 0, inject) && tid == 0) atomicExch(err, 1);
        return;
    }
    ptx::grid_dep_wait();  // the interleaved volume comes from the previous kernel
    const AngleParam a0 = ang[agroups[bx * kProjAnglesPerBlock]];
    const bool rows = a0.row_major != 0;  // one orientation per block
    const CUtensorMap *map = rows ? &map_row : &map_col;
    const uint32_t step_bytes = (uint32_t)(nbox * box) * kZc * 4u;  // zero fill past N included
    if (tid >= nthreads_c) {
        // ---------------------------------------------------------------- producer
        if (tid == nthreads_c) {
            for (int s0 = 0; s0 < N; s0 += kPGroup) {
                const int gi = s0 / kPGroup, u = gi % kPSlots;
                if (gi >= kPSlots &&
                    !ptx::mbar_wait_bounded(&bars[kPSlots + u], ((gi / kPSlots) - 1) & 1, 1u << 24)) {
                    atomicExch(err, 1);
                    break;
                }
                // generic-proxy reads of the stages, then their async-proxy refill: without
                // this fence some consumers read the next step's data (the sums then
                // changed from run to run)
                ptx::fence_proxy_async_smem();
                const int ns = min(kPGroup, N - s0);
                ptx::mbar_arrive_expect_tx(&bars[u], (uint32_t)ns * step_bytes);
                for (int e = 0; e < ns; ++e) {
                    const int s = s0 + e, k = u * kPGroup + e;
                    for (int b = 0; b < nbox; ++b) {
                        float *dst = psm + ((size_t)k * LDC + kPad + b * box) * kZc;
                        if (rows) il_copy(dst, map, b * box, s, zb, &bars[u]);  // row y = s
                        else il_copy(dst, map, s, b * box, zb, &bars[u]);       // column x = s
                    }
                }
            }
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    // The warps of an inactive slot (a block with one angle) only wait and arrive.
    // Threads beyond the last ray run the loop on clamped, in-bounds taps and store
    // nothing; slices past nz hold zeros, never stored.
    const int slot = tid / rays_per_angle;
    const int i = tid % rays_per_angle;
    const int m = agroups[bx * kProjAnglesPerBlock + slot];
    const bool active = (m >= 0) && (i < N);
    const AngleParam ap = ang[m >= 0 ? m : agroups[bx * kProjAnglesPerBlock]];
    long long fs = ap.fx_a + (long long)i * ap.fx_d;  // position of ray i at march step s
    float acc[kZc];
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] = 0.f;
    bool good = true;
    for (int s0 = 0; s0 < N; s0 += kPGroup) {
        const int gi = s0 / kPGroup, u = gi % kPSlots;
        // the warp gives up as one, so that its later votes and shuffles see all lanes
        if (!__all_sync(0xffffffffu, ptx::mbar_wait_bounded(&bars[u], (gi / kPSlots) & 1, 1u << 24))) {
            good = false;
            break;
        }
#pragma unroll
        for (int e = 0; e < kPGroup; ++e) {
            if (s0 + e >= N) break;  // uniform over the block
            const int k = u * kPGroup + e;
            int cell;
            float t;
            fx_split(fs, cell, t);
            fs += ap.fx_b;
            // A ray whose left tap is below -1 or above N - 1 has both taps on the zero pads
            // and adds nothing at this step; a warp all of whose rays are there (oblique
            // rays near the detector's edges, about a tenth of the warp-steps) skips the loads.
            if (m >= 0 && __any_sync(0xffffffffu, cell >= -1 && cell <= N - 1)) {  // m: uniform per warp
                const int cs = min(max(cell, -2), N) + kPad;  // staged position of the left tap
                const float *b0 = psm + ((size_t)k * LDC + cs) * kZc;
                const int w0 = 4 * il_swap(cs), w1 = 4 * il_swap(cs + 1);
                const float4 l0 = *reinterpret_cast<const float4 *>(b0 + w0);
                const float4 l1 = *reinterpret_cast<const float4 *>(b0 + 4 - w0);
                const float4 r0 = *reinterpret_cast<const float4 *>(b0 + kZc + w1);
                const float4 r1 = *reinterpret_cast<const float4 *>(b0 + kZc + 4 - w1);
                const float v0[kZc] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
                const float v1[kZc] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
                for (int zz = 0; zz < kZc; ++zz) acc[zz] = fmaf(1.f - t, v0[zz], fmaf(t, v1[zz], acc[zz]));
            }
        }
        __syncwarp();
        if ((tid & 31) == 0) ptx::mbar_arrive(&bars[kPSlots + u]);
    }
    ptx::grid_dep_launch();
    if (!good) {
        if ((tid & 31) == 0) atomicExch(err, 1);
        return;
    }
#pragma unroll
    for (int zz = 0; zz < kZc; ++zz) acc[zz] *= ap.scale;
    if (active && proj) {
#pragma unroll
        for (int zz = 0; zz < kZc; ++zz)
            if (zz < nz) proj[((size_t)m * Nz + z0 + zz) * N + i] = acc[zz];
    }
    if (pack.out[0]) {
        // The eight lanes of rays 8u..8u+7 hold 8 slices each; a butterfly of shuffles
        // transposes the 8 x 8 block, so that lane 8u + v holds slice v of those rays:
        // eight consecutive K values of line (m, z0 + v): one 16-byte unit of the GEMM's
        // A rows in bf16 or two in tf32, split to hi and lo exactly as the packing pass
        // splits them.
        const int lane = tid & 31, v = lane & 7;
        float a[kZc];
#pragma unroll
        for (int zz = 0; zz < kZc; ++zz) a[zz] = acc[zz];
#pragma unroll
        for (int stage = 0; stage < 3; ++stage) {
            const int sh = 4 >> stage;
            const bool hi = (lane & sh) != 0;
#pragma unroll
            for (int jj = 0; jj < kZc; ++jj) {
                if (jj & sh) continue;  // j runs over the lower index of each exchanged pair
                const float send = hi ? a[jj] : a[jj + sh];
                const float recv = __shfl_xor_sync(0xffffffffu, send, sh);
                if (hi) a[jj] = recv;
                else a[jj + sh] = recv;
            }
        }
        const int i0 = i - v;  // first ray of the unit
        const int z = z0 + v;
        if (m >= 0 && i0 < N && v < nz) {
            const int par = pack.n_par > 1 ? (z & 1) : 0;
            // selects, not indexing, so that the parameter block stays out of local memory
            const int r = m * (par ? pack.nrow[1] : pack.nrow[0]) + (pack.n_par > 1 ? z >> 1 : z);
            const int G = par ? pack.G[1] : pack.G[0];
            uint8_t *row = (par ? pack.out[1] : pack.out[0]) + (size_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 16u;
            auto put = [&](int c, int kg, const uint4 &hv, const uint4 &lv) {
                uint8_t *base = row + (uint32_t)kg * 128u;
                *reinterpret_cast<uint4 *>(base + (size_t)(2 * c) * G * 1024u) = hv;
                *reinterpret_cast<uint4 *>(base + (size_t)(2 * c + 1) * G * 1024u) = lv;
            };
            uint4 hv, lv;
            if (pack.tf32) {  // 32 K values per chunk, two units of four
                const float f0[4] = {a[0], a[1], a[2], a[3]}, f1[4] = {a[4], a[5], a[6], a[7]};
                split4_tf32(f0, hv, lv);
                put(i0 >> 5, (i0 & 31) >> 2, hv, lv);
                split4_tf32(f1, hv, lv);
                put(i0 >> 5, ((i0 & 31) >> 2) + 1, hv, lv);
            } else {  // 64 K values per chunk, one unit of eight
                split8_bf16(a, hv, lv);
                put(i0 >> 6, (i0 & 63) >> 3, hv, lv);
            }
        }
    }
}

template <int LDC>
void launch_il(dim3 grid, int threads, cudaStream_t st, const IlMaps &maps, const AngleParam *ang,
               const int *agroups, float *proj, int N, int Nz, int rays, int *err, uint32_t inject, ProjPack pack) {
    const size_t smem = pipe_smem(LDC);  // kPStages x kZc x LDC floats, as the pipelined variant
    cudaFuncSetAttribute(k_project_il<LDC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    launch_dependent(k_project_il<LDC>, grid, dim3(threads), smem, st, maps.row, maps.col, maps.nbox, maps.box, ang,
                     agroups, proj, N, Nz, rays, err, inject, pack);
}

bool project_il_ok(int N) { return N % 4 == 0 && pipe_ld(N) > 0 && pipe_threads_ok(N); }

void launch_project_il(const IlMaps &maps, const AngleParam *ang, const int *agroups,
                       int n_agroups, float *proj, int N, int Nz, cudaStream_t st, int *err, uint32_t inject,
                       ProjPack pack) {
    const int rays = (N + 31) / 32 * 32;
    dim3 grid(n_agroups, (Nz + kZc - 1) / kZc);
    const int threads = rays * kProjAnglesPerBlock + 32;
    switch (pipe_ld(N)) {
    case 40: launch_il<40>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    case 72: launch_il<72>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    case 136: launch_il<136>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    case 200: launch_il<200>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    case 264: launch_il<264>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    case 392: launch_il<392>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    default: launch_il<520>(grid, threads, st, maps, ang, agroups, proj, N, Nz, rays, err, inject, pack); break;
    }
}

// Transpose: a block owns a tile of kBpTX x kBpTY voxel columns and kBpZ slices; a
// thread owns one column (x, y) and its kBpZ slices. For every angle the rays whose
// interpolation touches the voxel are among i1-1, i1, i1+1 (i1 the nearest ray); ray
// i's sample position f_i is recomputed with the forward's exact arithmetic and its
// weight max(0, 1 - |f_i - q|) equals the forward's (1-t or t), so at most two
// consecutive rays carry weight. No atomics. The rays a tile can touch for one angle
// form a window of at most kBpSeg consecutive rays that starts one before the
// smallest nearest ray of the tile's corners (the nearest-ray map is monotone in
// both coordinates, so the corners bound it). Angles are taken kBpChunk at a time:
// the chunk's windows of proj x scale (zero outside the detector) are staged in
// shared memory, then every thread gathers its two rays per slice from there.
constexpr int kBpTX = 32, kBpTY = 16, kBpZ = 16, kBpSeg = 40, kBpChunk = 12;
// A staged ray holds its kBpZ slices innermost in a row of kBpRow floats: a voxel reads
// its two rays' taps for all slices with eight 16-byte loads. kBpRow = 20 is an odd
// number of 16-byte groups, so eight consecutive rays start in distinct bank groups.
// (32 slices per thread, sharing each angle's weights over more samples, measured
// slower: 186 against 125 us at 256^2 x 128, 36 angles.)
constexpr int kBpRow = 20;
static_assert(kBpRow >= kBpZ && kBpRow % 4 == 0 && (kBpRow / 4) % 2 == 1, "row of 16-byte groups, odd count");
static_assert(kBpChunk * kBpSeg <= kBpTX * kBpTY, "one staging thread per (angle, ray) of a chunk");

// What the gather loop reads per angle (one 16-byte load): the ray spacing fx_d, the
// nearest-ray estimate's 1/inv_c, and the window's first ray ilo with the orientation
// in bit 0 (2 ilo + row_major).
struct __align__(16) BpAngle {
    long long fx_d;
    float inv_c_rcp;
    int ilo_rm;
};
// Per angle and march step s = (row-major ? y_lo : x_lo) + ds of the tile (one 16-byte
// load): the step's Q32.32 base position fx_a + s fx_b, and slope (s - c) + c of the
// nearest-ray estimate, the same operations the thread would do for its own step.
struct __align__(16) BpStep {
    long long gs;
    float bs;
    float pad_;
};

struct __align__(16) BpShared {
    float seg[kBpChunk][kBpSeg][kBpRow];
    AngleParam ang[kBpChunk];
    int ilo[kBpChunk];
    BpAngle pa[kBpChunk];
    BpStep st[kBpChunk][kBpTX];
};
static_assert(kBpTX >= kBpTY, "the per-step tables hold the tile's longer side");

__device__ __forceinline__ int nearest_ray(const AngleParam &a, int s, int q, float c) {
    const float sm = (float)s - c;
    return __float2int_rn(fmaf((float)q - fmaf(a.slope, sm, c), a.inv_c_rcp, c));
}

__device__ __forceinline__ void backproject_body(const float *__restrict__ proj, const AngleParam *__restrict__ ang,
                                                 float *__restrict__ vol, int N, int Nz, int M, int bx, int by,
                                                 int bz, BpShared &S) {
    const int tid = threadIdx.y * kBpTX + threadIdx.x;
    const int x = bx * kBpTX + threadIdx.x;
    const int y = by * kBpTY + threadIdx.y;
    const int z0 = bz * kBpZ;
    const int nz = min(kBpZ, Nz - z0);
    const float c = 0.5f * (float)(N - 1);
    const int xlo = bx * kBpTX, xhi = min(xlo + kBpTX, N) - 1;
    const int ylo = by * kBpTY, yhi = min(ylo + kBpTY, N) - 1;
    // threads past the grid edge follow the loop on the edge voxel and store nothing
    const int ix = min(x, N - 1), iy = min(y, N - 1);
    // the voxel's march step within the tile and its index along the step's line, for
    // row-marched (R) and column-marched (C) angles
    const int dsR = iy - ylo, dsC = ix - xlo;
    const float fqR = (float)ix, fqC = (float)iy;
    float acc[kBpZ];
#pragma unroll
    for (int zz = 0; zz < kBpZ; ++zz) acc[zz] = 0.f;
    for (int m0 = 0; m0 < M; m0 += kBpChunk) {
        const int na = min(kBpChunk, M - m0);
        __syncthreads();  // the previous chunk has been used
        if (tid < na) {
            const AngleParam a = ang[m0 + tid];
            S.ang[tid] = a;
            const int s0 = a.row_major ? ylo : xlo, s1 = a.row_major ? yhi : xhi;
            const int q0 = a.row_major ? xlo : ylo, q1 = a.row_major ? xhi : yhi;
            const int lo = min(min(nearest_ray(a, s0, q0, c), nearest_ray(a, s0, q1, c)),
                               min(nearest_ray(a, s1, q0, c), nearest_ray(a, s1, q1, c)));
            S.ilo[tid] = lo - 1;
            S.pa[tid] = BpAngle{a.fx_d, a.inv_c_rcp, 2 * (lo - 1) + (a.row_major ? 1 : 0)};
        }
        __syncthreads();
        // thread (a, j) stages ray ilo[a] + j of angle m0 + a: its kBpZ slices, read with
        // the rays of the angle side by side (coalesced), stored as one row of 16-byte units
        if (tid < na * kBpSeg) {
            const int a = tid / kBpSeg, j = tid - a * kBpSeg;
            const int i = S.ilo[a] + j;
            const float sc = S.ang[a].scale;
            const bool in = i >= 0 && i < N;
            const float *src = proj + ((size_t)(m0 + a) * Nz + z0) * N + (in ? i : 0);
            float v[kBpZ];
#pragma unroll
            for (int zz = 0; zz < kBpZ; ++zz) v[zz] = (in && zz < nz) ? __ldg(src + (size_t)zz * N) * sc : 0.f;
            float4 *dst = reinterpret_cast<float4 *>(&S.seg[a][j][0]);
#pragma unroll
            for (int g4 = 0; g4 < kBpZ / 4; ++g4)
                dst[g4] = make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
        }
        for (int t = tid; t < na * kBpTX; t += kBpTX * kBpTY) {
            const int a = t / kBpTX, ds = t - a * kBpTX;
            const AngleParam A = S.ang[a];
            const int s = (A.row_major ? ylo : xlo) + ds;
            S.st[a][ds] = BpStep{A.fx_a + (long long)s * A.fx_b, fmaf(A.slope, (float)s - c, c), 0.f};
        }
        __syncthreads();
        for (int a = 0; a < na; ++a) {
            const BpAngle an = S.pa[a];
            const bool rm = (an.ilo_rm & 1) != 0;
            const int ds = rm ? dsR : dsC;  // march step holding this voxel, within the tile
            const int q = rm ? ix : iy;     // its index along the step's line
            const long long fxd = an.fx_d;
            const BpStep sp = S.st[a][ds];
            // nearest ray (estimate): inv_c (i - c) + slope (s - c) + c = q
            const int i1 = __float2int_rn(fmaf((rm ? fqR : fqC) - sp.bs, an.inv_c_rcp, c));
            // The forward's fixed-point positions of rays i1-1, i1, i1+1 at step s give cell
            // q the weight 1 - t from a ray in cell q and t from one in cell q-1; two
            // consecutive rays carry it. Ray i1-1 does (and the pair is (i1-1, i1)) when it
            // lies in cell q, or in cell q-1 with a nonzero fraction (t = 0 when the
            // fraction's top 23 bits are zero); else the pair is (i1, i1+1). Only the two
            // rays of the pair are evaluated.
            const long long g0 = sp.gs + (long long)(i1 - 1) * fxd;
            const int k0 = (int)(g0 >> 32);
            const bool lo = k0 == q || (k0 == q - 1 && (unsigned)g0 >= 512u);
            const long long gA = lo ? g0 : g0 + fxd;
            auto weight = [q](long long g) {
                int k;
                float t;
                fx_split(g, k, t);
                return k == q ? 1.f - t : (k == q - 1 ? t : 0.f);
            };
            const float wA = weight(gA), wB = weight(gA + fxd);
            const int j = min(max(i1 - (lo ? 1 : 0) - (an.ilo_rm >> 1), 0), kBpSeg - 2);
            const float4 *pa = reinterpret_cast<const float4 *>(&S.seg[a][j][0]);
            const float4 *pb = reinterpret_cast<const float4 *>(&S.seg[a][j + 1][0]);
#pragma unroll
            for (int g4 = 0; g4 < kBpZ / 4; ++g4) {
                const float4 va = pa[g4], vb = pb[g4];
                acc[4 * g4] = fmaf(wA, va.x, fmaf(wB, vb.x, acc[4 * g4]));
                acc[4 * g4 + 1] = fmaf(wA, va.y, fmaf(wB, vb.y, acc[4 * g4 + 1]));
                acc[4 * g4 + 2] = fmaf(wA, va.z, fmaf(wB, vb.z, acc[4 * g4 + 2]));
                acc[4 * g4 + 3] = fmaf(wA, va.w, fmaf(wB, vb.w, acc[4 * g4 + 3]));
            }
        }
    }
    if (x < N && y < N) {
#pragma unroll
        for (int zz = 0; zz < kBpZ; ++zz)
            if (zz < nz) vol[((size_t)(z0 + zz) * N + y) * N + x] = acc[zz];
    }
}

__global__ void __launch_bounds__(kBpTX * kBpTY, 2) k_backproject(const float *__restrict__ proj,
                                                              const AngleParam *__restrict__ ang,
                                                              float *__restrict__ vol, int N, int Nz, int M) {
    __shared__ BpShared S;
    ptx::grid_dep_wait();  // the projections come from the previous kernel
    ptx::grid_dep_launch();
    backproject_body(proj, ang, vol, N, Nz, M, blockIdx.x, blockIdx.y, blockIdx.z, S);
}

void launch_backproject(const float *proj, const AngleParam *ang, float *vol, int N, int Nz,
                        int M, cudaStream_t st) {
    dim3 grid((N + kBpTX - 1) / kBpTX, (N + kBpTY - 1) / kBpTY, (Nz + kBpZ - 1) / kBpZ), block(kBpTX, kBpTY);
    launch_dependent(k_backproject, grid, block, 0, st, proj, ang, vol, N, Nz, M);
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

// The batched kernels are persistent: a grid of at most as many blocks as the GPU holds
// at once loops over the work items of every job (see batch_find). An item's arithmetic
// does not depend on the block that runs it, so a job gives the same bits alone and in
// any mix.
__global__ void k_transpose_batch(const TransposeJob *__restrict__ jobs, const int *__restrict__ offs, int n,
                                  int total) {
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find(offs, n, bi);
        const TransposeJob J = jobs[j];
        if (J.done && *J.done) continue;
        int b = bi - offs[j];
        const int gx = (J.N + 31) / 32;
        const int bx = b % gx, by = (b / gx) % gx, bz = b / (gx * gx);
        __syncthreads();  // the tile of the previous item has been read
        transpose_body(J.vol, J.volT, J.N, bx, by, bz);
    }
}

template <int LD>
__global__ void __launch_bounds__(1024 + 32) k_project_batch(const ProjectJob *__restrict__ jobs,
                                                             const int *__restrict__ offs, int n, int total,
                                                             int *err) {
    extern __shared__ __align__(128) float psm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(psm + kPStages * kZc * LD);
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find(offs, n, bi);
        const ProjectJob J = jobs[j];
        if (J.done && *J.done) continue;  // uniform over the block
        const int b = bi - offs[j];
        const int rays = (J.N + 31) / 32 * 32;
        if ((int)threadIdx.x < rays * kProjAnglesPerBlock + 32)
            project_pipe_body<LD>(J.vol, J.volT, J.ang, J.agroups, J.proj, J.N, J.Nz, rays, err, b % J.n_agroups,
                                  b / J.n_agroups, psm);
        else
            __syncthreads();  // threads beyond this problem's block shape meet the body's one barrier
        // every thread has left the item: its barriers are idle and are set up anew
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < 2 * kPStages; ++k) ptx::mbar_inval(&bars[k]);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBpTX * kBpTY, 2) k_backproject_batch(const BackprojectJob *__restrict__ jobs,
                                                                    const int *__restrict__ offs, int n, int total) {
    __shared__ BpShared S;
    for (int bi = blockIdx.x; bi < total; bi += gridDim.x) {
        const int j = batch_find(offs, n, bi);
        const BackprojectJob J = jobs[j];
        if (J.done && *J.done) continue;  // uniform over the block
        const int b = bi - offs[j];
        const int gx = (J.N + kBpTX - 1) / kBpTX, gy = (J.N + kBpTY - 1) / kBpTY;
        // the body starts each chunk of angles with a barrier, so the previous item's
        // staging is no longer read when this one overwrites it
        backproject_body(J.proj, J.ang, J.vol, J.N, J.Nz, J.M, b % gx, (b / gx) % gy, b / (gx * gy), S);
    }
}

int transpose_blocks(int N, int Nz) { return ((N + 31) / 32) * ((N + 31) / 32) * Nz; }
int project_blocks(int n_agroups, int Nz) { return n_agroups * ((Nz + kZc - 1) / kZc); }
int backproject_blocks(int N, int Nz) {
    return ((N + kBpTX - 1) / kBpTX) * ((N + kBpTY - 1) / kBpTY) * ((Nz + kBpZ - 1) / kBpZ);
}

// Blocks of a persistent batched launch: what the GPU holds at once, at most one per item.
template <class K>
int persistent_grid_p(K kernel, int threads, size_t smem, int total) {
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

void launch_transpose_batch(const TransposeJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    if (total <= 0) return;
    k_transpose_batch<<<persistent_grid_p(k_transpose_batch, 256, 0, total), dim3(32, 8), 0, st>>>(jobs, offs, n,
                                                                                                   total);
}

bool project_batch_ok(int N) { return N % 4 == 0 && pipe_ld(N) > 0 && pipe_threads_ok(N); }

template <int LD>
void launch_pbatch(const ProjectJob *jobs, const int *offs, int n, int total, int threads, int *err,
                   cudaStream_t st) {
    cudaFuncSetAttribute(k_project_batch<LD>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    const int grid = persistent_grid_p(k_project_batch<LD>, threads, pipe_smem(LD), total);
    k_project_batch<LD><<<grid, threads, pipe_smem(LD), st>>>(jobs, offs, n, total, err);
}

// Every problem in the batch has N % 4 == 0 and N <= 512 (project_batch_ok); the ring
// stride is the one of the largest N.
void launch_project_batch(const ProjectJob *jobs, const int *offs, int n, int total, int maxN, int *err,
                          cudaStream_t st) {
    const int threads = (maxN + 31) / 32 * 32 * kProjAnglesPerBlock + 32;
    switch (pipe_ld(maxN)) {
    case 40: launch_pbatch<40>(jobs, offs, n, total, threads, err, st); break;
    case 72: launch_pbatch<72>(jobs, offs, n, total, threads, err, st); break;
    case 136: launch_pbatch<136>(jobs, offs, n, total, threads, err, st); break;
    case 200: launch_pbatch<200>(jobs, offs, n, total, threads, err, st); break;
    case 264: launch_pbatch<264>(jobs, offs, n, total, threads, err, st); break;
    case 392: launch_pbatch<392>(jobs, offs, n, total, threads, err, st); break;
    default: launch_pbatch<520>(jobs, offs, n, total, threads, err, st); break;
    }
}

void launch_backproject_batch(const BackprojectJob *jobs, const int *offs, int n, int total, cudaStream_t st) {
    if (total <= 0) return;
    const int grid = persistent_grid_p(k_backproject_batch, kBpTX * kBpTY, 0, total);
    k_backproject_batch<<<grid, dim3(kBpTX, kBpTY), 0, st>>>(jobs, offs, n, total);
}

}  // namespace mpiffl
