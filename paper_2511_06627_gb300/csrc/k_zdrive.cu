// The z-drive scan of the dual-drive acquisition (Sec. 3.1): the drive and the
// Langevin-derivative PSF act along z while the raster is the x-drive one. Sample j
// of line l reads the z-convolved projection cz[m][u][e] bilinearly at
// (u = c_j, z = l + A sin(2 pi j / S + phi0)): between detector columns u0_j and
// u0_j + 1 (weight a_j), and on the fine z grid at n = Q l + n0_r (fraction f0_r),
// where r = j mod S (the drive phase sets the z offset; the slow raster sets u).
//
// Forward:  s[m][l][j] = g_m v_r bilinear(cz[m], u0_j, a_j, Q l + n0_r, f0_r)
// Transpose, in two gathers (no atomics):
//   t[m][l][u][r]  = g_m v_r sum over the periods p whose sample pS + r reads column u
//                    (u0 = u with weight 1 - a, u0 = u - 1 with weight a) of s[m][l][pS+r]
//   cz[m][u][e]    = sum over the taps (r, e_off, w) of the phase table with
//                    e - e_off = Q l, 0 <= l < N_z, of w t[m][l][u][r]
// The tap table lists, for every residue of e modulo Q, the phases r whose two
// z-taps (n0_r with weight 1 - f0_r, n0_r + 1 with f0_r) fall on that residue.
#include "internal.h"

namespace mpiffl {

// out[b][c][r] = in[b][r][c] for rows x cols matrices (batched, padded tile).
__global__ void __launch_bounds__(256) k_transpose_2d(const float *__restrict__ in, float *__restrict__ out, int rows,
                                                      int cols) {
    __shared__ float tile[32][33];
    const size_t mat = (size_t)rows * cols;
    const float *src = in + blockIdx.z * mat;
    float *dst = out + blockIdx.z * mat;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

void launch_transpose_2d(const float *in, float *out, int batch, int rows, int cols, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, batch), block(32, 8);
    k_transpose_2d<<<grid, block, 0, st>>>(in, out, rows, cols);
}

// A block per line (m, l), a thread per drive phase r looping over the periods p:
// the z cell, its fraction and the velocity are the thread's constants, and the
// samples p S + r of a warp's phases are contiguous (coalesced table reads and stores).
__global__ void __launch_bounds__(128) k_resample_z_fwd(const float *__restrict__ cz, const ZTables T,
                                                        const float *__restrict__ gain, float *__restrict__ sig,
                                                        int N, int Nz, int L, int S, int P, int Q, int Nez,
                                                        int zigzag) {
    const int seg = blockIdx.x;
    const int m = seg / Nz, l = seg - m * Nz;
    const int par = zigzag ? (l & 1) : 0;
    const float2 *tua = T.ua + (size_t)par * L;
    const float *czm = cz + (size_t)m * N * Nez;
    float *out = sig + (size_t)seg * L;
    const float g = __ldg(gain + m);
    for (int r = threadIdx.x; r < S; r += blockDim.x) {
        int n = Q * l + __ldg(T.n0 + r);
        float f = __ldg(T.f0 + r);
        if (n > Nez - 2) {  // the grid's last cell, reached with f = 1
            f += (float)(n - (Nez - 2));
            n = Nez - 2;
        }
        const float gv = g * __ldg(T.v + r);
        // the z-interpolated values of the two columns a sample reads change only when
        // its column does (every few periods): keep them in registers
        int ucur = -1;
        float v0 = 0.f, v1 = 0.f;
        for (int p = 0, j = r; p < P; ++p, j += S) {
            const float2 ua = __ldg(tua + j);
            const int u0 = __float_as_int(ua.x);
            if (u0 != ucur) {
                const float *c0 = czm + (size_t)u0 * Nez + n;
                v0 = fmaf(f, __ldg(c0 + 1), (1.f - f) * __ldg(c0));
                v1 = u0 + 1 < N ? fmaf(f, __ldg(c0 + Nez + 1), (1.f - f) * __ldg(c0 + Nez)) : 0.f;
                ucur = u0;
            }
            out[j] = gv * fmaf(ua.y, v1, (1.f - ua.y) * v0);
        }
    }
}

void launch_resample_z_fwd(const float *cz, const ZTables &T, const float *gain, float *sig, const Dims &d,
                           int zigzag, cudaStream_t st) {
    k_resample_z_fwd<<<d.M * d.Nz, 128, 0, st>>>(cz, T, gain, sig, d.N, d.Nz, d.L, d.S, d.P, d.Q, d.Nez, zigzag);
}

// t[m][l][u][r]: a block per line (m, l), a thread per phase r. The thread visits the
// samples p S + r of its phase in the order of increasing detector column (periods
// ascending on lines swept left to right, descending on the reversed ones), keeps the
// sums of the two columns the current sample reads, and writes a column when no later
// sample can reach it. Every sample is read once; the reads are coalesced over r.
__global__ void __launch_bounds__(128) k_resample_z_adj_u(const float *__restrict__ sig, const ZTables T,
                                                          const float *__restrict__ gain, float *__restrict__ tz,
                                                          int N, int Nz, int L, int S, int P, int zigzag) {
    const int seg = blockIdx.x;
    const int m = seg / Nz, l = seg - m * Nz;
    const int par = zigzag ? (l & 1) : 0;
    const float g = __ldg(gain + m);
    const float *s = sig + (size_t)seg * L;
    const float2 *tua = T.ua + (size_t)par * L;
    float *out = tz + (size_t)seg * N * S;
    for (int r = threadIdx.x; r < S; r += blockDim.x) {
        const float gv = g * __ldg(T.v + r);
        int u = 0;  // the columns u and u + 1 are open
        float acc0 = 0.f, acc1 = 0.f;
        for (int q = 0; q < P; ++q) {
            const int j = (par ? P - 1 - q : q) * S + r;
            const float2 ua = __ldg(tua + j);
            const int u0 = __float_as_int(ua.x);
            const float a = ua.y;
            const float sv = __ldg(s + j);
            while (u < u0) {  // column u is complete
                out[(size_t)u * S + r] = gv * acc0;
                acc0 = acc1;
                acc1 = 0.f;
                ++u;
            }
            acc0 = fmaf(1.f - a, sv, acc0);
            acc1 = fmaf(a, sv, acc1);
        }
        for (; u < N; ++u) {
            out[(size_t)u * S + r] = gv * acc0;
            acc0 = acc1;
            acc1 = 0.f;
        }
    }
}

// cz[m][u][e]: a block per column (m, u) stages t[m][.][u][.] in shared memory as
// [r][l] rows padded to N_z + 1 (consecutive lines of a phase in distinct banks). A warp
// takes one residue rho of e modulo Q at a time, its lanes the cells e = Q q + rho of
// consecutive q: the warp walks one tap list (uniform loads), and each tap reads the
// lines q - (e_off - rho)/Q of consecutive lanes, conflict-free. Q = 2^lq.
__global__ void __launch_bounds__(256) k_resample_z_adj_z(const float *__restrict__ tz, const ZTables T,
                                                          float *__restrict__ cz, int N, int Nz, int S, int lq,
                                                          int Nez) {
    extern __shared__ float st[];  // [S][Nz + 1]
    const int col = blockIdx.x;
    const int m = col / N, u = col - m * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ld = Nz + 1;
    for (int l = warp; l < Nz; l += nwarps) {
        const float *src = tz + (((size_t)m * Nz + l) * N + u) * S;
        for (int r = lane; r < S; r += 32) st[r * ld + l] = src[r];
    }
    __syncthreads();
    float *out = cz + (size_t)col * Nez;
    const int Q = 1 << lq;
    const int nq = (Nez + Q - 1) >> lq;  // cells per residue (upper bound)
    const int nchunk = (nq + 31) >> 5;
    for (int item = warp; item < Q * nchunk; item += nwarps) {
        const int rho = item & (Q - 1), qc = item >> lq;
        const int q = (qc << 5) + lane;
        const int e = (q << lq) + rho;
        float acc = 0.f;
        const int k1 = __ldg(T.tap_ptr + rho + 1);
        for (int k = __ldg(T.tap_ptr + rho); k < k1; ++k) {
            const int4 tp = __ldg(T.taps + k);  // (r, e_off, w bits, 0), e_off = rho (mod Q)
            const int ll = q - ((tp.y - rho) >> lq);
            if (ll >= 0 && ll < Nz) acc = fmaf(__int_as_float(tp.z), st[tp.x * ld + ll], acc);
        }
        if (e < Nez) out[e] = acc;
    }
}

void launch_resample_z_adj(const float *sig, const ZTables &T, const float *gain, float *tz, float *cz,
                           const Dims &d, int zigzag, cudaStream_t st) {
    k_resample_z_adj_u<<<d.M * d.Nz, 128, 0, st>>>(sig, T, gain, tz, d.N, d.Nz, d.L, d.S, d.P, zigzag);
    const size_t smem = sizeof(float) * (size_t)(d.Nz + 1) * d.S;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_resample_z_adj_z, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    int lq = 0;
    while ((1 << lq) < d.Q) ++lq;
    k_resample_z_adj_z<<<d.M * d.N, 256, smem, st>>>(tz, T, cz, d.N, d.Nz, d.S, lq, d.Nez);
}

}  // namespace mpiffl
