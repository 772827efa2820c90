// Parallel-beam projector P_theta and its gather-form transpose
// (Sec. 2.2, Eqs. (16)-(19); Joseph interpolation, see AngleParam).
//
// Forward: one thread per ray (angle m, slice z, detector bin i) marches the
// N steps of its ray; rays of one warp are adjacent bins, so at every step they
// read neighbouring addresses of one voxel line. Column-marched angles read a
// transposed copy of the volume so that their voxel lines are contiguous too.
// Transpose: one thread per voxel gathers, for every angle, the (at most two)
// rays whose interpolation touches it, with the forward's exact weights. No
// atomics.
#include "internal.h"

namespace mpiffl {

__global__ void k_transpose_xy(const float *__restrict__ vol, float *__restrict__ volT, int N) {
    __shared__ float tile[32][33];
    const size_t zoff = (size_t)blockIdx.z * N * N;
    int x = blockIdx.x * 32 + threadIdx.x;
    int y0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int y = y0 + k;
        if (x < N && y < N) tile[k][threadIdx.x] = vol[zoff + (size_t)y * N + x];
    }
    __syncthreads();
    int yo = blockIdx.y * 32 + threadIdx.x;
    int x0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int xo = x0 + k;
        if (xo < N && yo < N) volT[zoff + (size_t)xo * N + yo] = tile[threadIdx.x][k];
    }
}

void launch_transpose_xy(const float *vol, float *volT, int N, int Nz, cudaStream_t st) {
    dim3 grid((N + 31) / 32, (N + 31) / 32, Nz), block(32, 8);
    k_transpose_xy<<<grid, block, 0, st>>>(vol, volT, N);
}

__global__ void __launch_bounds__(128) k_project(const float *__restrict__ vol, const float *__restrict__ volT,
                                                 const AngleParam *__restrict__ ang,
                                                 float *__restrict__ proj, int N, int Nz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const int m = blockIdx.z;
    if (i >= N) return;
    const AngleParam a = ang[m];
    const float *base = (a.row_major ? vol : volT) + (size_t)z * N * N;
    const float c = 0.5f * (float)(N - 1);
    const float fi = fmaf(a.inv_c, (float)i - c, c);
    float acc = 0.f;
    for (int s = 0; s < N; ++s) {
        const float f = fmaf(a.slope, (float)s - c, fi);
        const float fl = floorf(f);
        const int k = (int)fl;
        const float t = f - fl;
        const float *line = base + (size_t)s * N;
        const float v0 = (k >= 0 && k < N) ? __ldg(line + k) : 0.f;
        const float v1 = (k + 1 >= 0 && k + 1 < N) ? __ldg(line + k + 1) : 0.f;
        acc = fmaf(1.f - t, v0, fmaf(t, v1, acc));
    }
    proj[((size_t)m * Nz + z) * N + i] = acc * a.scale;
}

void launch_project(const float *vol, const float *volT, const AngleParam *ang, float *proj,
                    int N, int Nz, int M, cudaStream_t st) {
    dim3 grid((N + 127) / 128, Nz, M);
    k_project<<<grid, 128, 0, st>>>(vol, volT, ang, proj, N, Nz);
}

__global__ void __launch_bounds__(128) k_backproject(const float *__restrict__ proj,
                                                     const AngleParam *__restrict__ ang,
                                                     float *__restrict__ vol, int N, int Nz, int M) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= N) return;
    const float c = 0.5f * (float)(N - 1);
    float acc = 0.f;
    for (int m = 0; m < M; ++m) {
        const AngleParam a = ang[m];
        const int s = a.row_major ? y : x;          // march step holding this voxel
        const float q = (float)(a.row_major ? x : y);  // its position along the step's line
        const float off = a.slope * ((float)s - c);
        // ray i samples f_i = inv_c (i - c) + off + c; voxel q gets weight 1 - |f_i - q|
        const float ir = (q - off - c) / a.inv_c + c;
        const int i0 = (int)floorf(ir);
        const float *pr = proj + ((size_t)m * Nz + z) * N;
        float sum = 0.f;
#pragma unroll
        for (int di = -1; di <= 2; ++di) {
            const int i = i0 + di;
            if (i < 0 || i >= N) continue;
            const float f = fmaf(a.slope, (float)s - c, fmaf(a.inv_c, (float)i - c, c));
            const float fl = floorf(f);
            const int k = (int)fl;
            const float t = f - fl;
            // identical weights to the forward: (1-t) on k, t on k+1
            float w = 0.f;
            if (k == (int)q) w = 1.f - t;
            else if (k + 1 == (int)q) w = t;
            if (w != 0.f) sum = fmaf(w, __ldg(pr + i), sum);
        }
        acc = fmaf(sum, a.scale, acc);
    }
    vol[((size_t)z * N + y) * N + x] = acc;
}

void launch_backproject(const float *proj, const AngleParam *ang, float *vol, int N, int Nz,
                        int M, cudaStream_t st) {
    dim3 grid((N + 127) / 128, N, Nz);
    k_backproject<<<grid, 128, 0, st>>>(proj, ang, vol, N, Nz, M);
}

}  // namespace mpiffl
