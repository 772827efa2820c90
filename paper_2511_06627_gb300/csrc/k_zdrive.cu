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

#include <algorithm>

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

// ------------------------------------------------------------------ fused with S D F
// The band DFT factorised over j = p S + r (k_line.cu) runs one thread per phase r
// over the periods p, the same loop as the z resampling. Fused, the forward builds
// each sample from cz and adds it to the 2w+1 period sums, and the adjoint
// synthesises the samples from the per-phase coefficients and gathers them straight
// into the fine z grid: the time signal is never stored.
//
// Both walk a line's periods in the order of increasing detector column. The slow
// position is kept in exact integers: on a line swept left to right, sample
// j = p S + r sits at c = (N-1) j / (L-1) = u0 + rem / (L-1); a reversed line walked
// in increasing column order (q = P-1-p) is the same with the phase S-1-r. Each step
// of one period adds (N-1) S to the numerator.
//
// Twiddle rows are padded to WP = 4 ceil(W/4) floats in shared memory and read as
// float4 (the period index is uniform across a warp: broadcasts).

// Lines per forward thread. Lines 2i apart share the trajectory (the same parity), so
// their samples have the same column, fraction and twiddle row: one position update and
// one set of twiddle loads serve kZLines samples.
constexpr int kZLines = 4;
// Lines per synthesis pass of the adjoint (same parity, 2 apart).
constexpr int kZSynLines = 4;
// Detector columns per adjoint block.
constexpr int kZSynCols = 8;

// c = (N-1) j0 / (L-1) as (u0, rem)
__device__ __forceinline__ void slow_start(int N1, int Lm1, int j0, int &u0, int &rem) {
    const long long num = (long long)N1 * j0;
    u0 = (int)(num / Lm1);
    rem = (int)(num - (long long)u0 * Lm1);
}

template <int WP>
__device__ __forceinline__ void load_twiddles(const float *tp, float (&t)[WP]) {
#pragma unroll
    for (int i = 0; i < WP / 4; ++i) {
        const float4 x = reinterpret_cast<const float4 *>(tp)[i];
        t[4 * i] = x.x;
        t[4 * i + 1] = x.y;
        t[4 * i + 2] = x.z;
        t[4 * i + 3] = x.w;
    }
}

template <int HW>
__device__ __forceinline__ void stage_twiddles(float *stw, const float *__restrict__ tw1, int P) {
    constexpr int W = 2 * HW + 1, WP = (W + 3) & ~3;
    for (int i = threadIdx.x; i < P * WP; i += blockDim.x) {
        const int p = i / WP, k = i - p * WP;
        stw[i] = k < W ? __ldg(tw1 + p * W + k) : 0.f;
    }
}

// Columns per forward chunk: at least 16, and more than the largest column spread of
// 32 consecutive phases at one period, so that every lane's two columns fit.
static int zdft_chunk(const Dims &d) {
    const long long spread = (long long)(d.N - 1) * 31 / (d.L - 1) + 1;
    return (int)std::max(16LL, spread + 1);
}

static int twiddle_row(const Dims &d) { return (2 * d.hw + 1 + 3) & ~3; }

size_t zdft_fwd_smem(const Dims &d) {
    const size_t bd = 128, W = 2 * d.hw + 1;
    const size_t sv = (size_t)kZLines * (zdft_chunk(d) + 1) * bd, sT = (size_t)kZLines * d.S * W * 2;
    return sizeof(float) * ((size_t)d.P * twiddle_row(d) + ((size_t)d.S <= bd ? std::max(sv, sT) : sv + sT));
}

// ring cells per column: a power of two covering the live window 2 (R - 1) Q + no
int zsyn_ring(const Dims &d, int no) {
    int rb = 1;
    while (rb < 2 * (kZSynLines - 1) * d.Q + no) rb <<= 1;
    return rb;
}

size_t zsyn_smem(const Dims &d, int no) {
    return sizeof(float) * ((size_t)d.P * twiddle_row(d) + (size_t)kZSynLines * kZSynCols * (d.S + 1) +
                            (size_t)kZSynCols * (zsyn_ring(d, no) + 1) + ((no + 2) & ~1) + 4 * (size_t)d.S);
}

// Forward. A block takes kZLines lines of one angle and one parity (l0 + 2i). The
// columns a lane reads are z-interpolated once per line into the lane's own slots of a
// shared chunk [line][uc + 1][blockDim] (a batch of independent loads); the chunk's
// periods then run from shared memory. Chunks are warp-uniform: they start at the
// warp's smallest column, and uc is sized so that every lane's two columns fit.
template <int HW>
__global__ void __launch_bounds__(128) k_zdft_fwd(const float *__restrict__ cz, const ZTables T,
                                                  const float *__restrict__ gain, const float *__restrict__ tw1,
                                                  const float2 *__restrict__ tw2_ro,
                                                  const float2 *__restrict__ dgam, float *__restrict__ data,
                                                  Dims d, int zigzag, int uc, float inv_sqrt_l) {
    constexpr int W = 2 * HW + 1, WP = (W + 3) & ~3, R = kZLines;
    extern __shared__ float4 sm4[];
    const int bd = blockDim.x;
    float *stw = reinterpret_cast<float *>(sm4);  // P * WP
    float *sV = stw + d.P * WP;                   // [R][uc + 1][bd]
    // [R][S][W] period sums; they take the place of sV once a single pass covers S
    float2 *sT = reinterpret_cast<float2 *>(d.S <= bd ? sV : sV + R * (uc + 1) * bd);
    const int nband = (d.Nz + 2 * R - 1) / (2 * R);
    const int m = blockIdx.x / (2 * nband), bg = blockIdx.x - m * 2 * nband;
    const int l0 = (bg >> 1) * 2 * R + (bg & 1);
    if (l0 >= d.Nz) return;  // the whole block
    const int par = zigzag ? (l0 & 1) : 0;
    stage_twiddles<HW>(stw, tw1, d.P);
    __syncthreads();
    const int N1 = d.N - 1, Lm1 = d.L - 1;
    const int du = N1 * d.S / Lm1, drem = N1 * d.S - du * Lm1;
    const float inv = 1.f / (float)Lm1;
    const float *czm = cz + (size_t)m * d.N * d.Nez;
    const float g = __ldg(gain + m);
    const size_t lstride = (size_t)(uc + 1) * bd;
    for (int r0 = 0; r0 < d.S; r0 += bd) {  // uniform trip count
        const int r = r0 + threadIdx.x, re = min(r, d.S - 1);
        const int n0 = __ldg(T.n0 + re);
        const float f0 = __ldg(T.f0 + re);
        const float *cb[R];
        float fr[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            // a line past the last reads a valid one; its sums are not written
            const int l = min(l0 + 2 * i, d.Nz - 1);
            int n = d.Q * l + n0;
            float f = f0;
            if (n > d.Nez - 2) {  // the grid's last cell, reached with f = 1
                f += (float)(n - (d.Nez - 2));
                n = d.Nez - 2;
            }
            cb[i] = czm + n;
            fr[i] = f;
        }
        const float gv = g * __ldg(T.v + re);
        const int j0 = par ? d.S - 1 - re : re;
        int u0, rem;
        slow_start(N1, Lm1, j0, u0, rem);
        float ac[R][HW + 1], as[R][HW + 1];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
            for (int k = 0; k <= HW; ++k) ac[i][k] = as[i][k] = 0.f;
        const float *tp = stw + (par ? d.P - 1 : 0) * WP;
        const int dtp = par ? -WP : WP;
        float *sv = sV + threadIdx.x;
        int q = 0;
        while (q < d.P) {
            const int ub = __reduce_min_sync(0xffffffffu, u0);
            // the first period at which this lane's column reaches ub + uc
            int qe = d.P;
            if (N1 > 0) {
                const long long need = (long long)(ub + uc) * Lm1 - (long long)N1 * j0;
                const long long step = (long long)N1 * d.S;
                qe = (int)min((long long)d.P, (need + step - 1) / step);
            }
            qe = __reduce_min_sync(0xffffffffu, qe);
            // columns past the detector read the last one and store 0 (no branch: the
            // loads of several columns are in flight together)
#pragma unroll 4
            for (int k = 0; k <= uc; ++k) {
                const int u = ub + k;
                const float keep = u < d.N ? 1.f : 0.f;
                const size_t cu = (size_t)min(u, d.N - 1) * d.Nez;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float *c0 = cb[i] + cu;
                    sv[i * lstride + k * bd] = keep * fmaf(fr[i], __ldg(c0 + 1), (1.f - fr[i]) * __ldg(c0));
                }
            }
            for (; q < qe; ++q) {
                const float a = (float)rem * inv;
                const float *vk = sv + (u0 - ub) * bd;
                float t[WP];
                load_twiddles<WP>(tp, t);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const float v = gv * fmaf(a, vk[i * lstride + bd], (1.f - a) * vk[i * lstride]);
#pragma unroll
                    for (int k = 0; k <= HW; ++k) ac[i][k] = fmaf(v, t[k], ac[i][k]);
#pragma unroll
                    for (int k = 1; k <= HW; ++k) as[i][k] = fmaf(v, t[HW + k], as[i][k]);
                }
                tp += dtp;
                u0 += du;
                rem += drem;
                if (rem >= Lm1) {
                    rem -= Lm1;
                    ++u0;
                }
            }
        }
        if (d.S <= bd) __syncthreads();  // sT overwrites sV
        if (r < d.S) {
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int k = -HW; k <= HW; ++k) {
                    const int ka = k < 0 ? -k : k;
                    sT[((size_t)i * d.S + r) * W + (k + HW)] = make_float2(ac[i][ka], k < 0 ? -as[i][ka] : as[i][ka]);
                }
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < d.nb; o += bd) {
        const int di = o % W;
        float xr[R], xi[R];
#pragma unroll
        for (int i = 0; i < R; ++i) xr[i] = xi[i] = 0.f;
        for (int r = 0; r < d.S; ++r) {
            const float2 w = __ldg(tw2_ro + (size_t)r * d.nb + o);
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const float2 t = sT[((size_t)i * d.S + r) * W + di];
                xr[i] = fmaf(t.x, w.x, fmaf(-t.y, w.y, xr[i]));
                xi[i] = fmaf(t.x, w.y, fmaf(t.y, w.x, xi[i]));
            }
        }
        const float2 gm = dgam[o];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int l = l0 + 2 * i;
            if (l >= d.Nz) break;
            const float re = xr[i] * inv_sqrt_l, im = xi[i] * inv_sqrt_l;
            float2 *out = reinterpret_cast<float2 *>(data) + ((size_t)m * d.Nz + l) * d.nb + o;
            *out = make_float2(gm.x * re - gm.y * im, gm.x * im + gm.y * re);
        }
    }
}

// Adjoint, first step: per line (m, l) and phase r the synthesis coefficients
// U[d] = sum_k y'[k,d] e^{-2 pi i (kP+d) r / L}, y' = conj(D_Gamma) y / sqrt(L), folded
// into s[pS+r] = sum_{d>=0} A_d cos(2 pi d p / P) + sum_{d>0} B_d sin(2 pi d p / P) and
// scaled by g_m v_r: coef[m][l][0..W)[r] = g_m v_r (A_0..A_w, B_1..B_w).
template <int HW>
__global__ void __launch_bounds__(128) k_zsyn_coef(const float *__restrict__ data,
                                                   const float2 *__restrict__ tw2_qr,
                                                   const float2 *__restrict__ dgam, const ZTables T,
                                                   const float *__restrict__ gain, float *__restrict__ coef, Dims d,
                                                   float inv_sqrt_l) {
    constexpr int W = 2 * HW + 1;
    extern __shared__ float4 sm4[];
    float2 *sy = reinterpret_cast<float2 *>(sm4);  // nb
    const int seg = blockIdx.x;
    const int m = seg / d.Nz;
    for (int o = threadIdx.x; o < d.nb; o += blockDim.x) {
        const float2 y = reinterpret_cast<const float2 *>(data)[(size_t)seg * d.nb + o];
        const float2 gm = dgam[o];
        sy[o] = make_float2((gm.x * y.x + gm.y * y.y) * inv_sqrt_l, (gm.x * y.y - gm.y * y.x) * inv_sqrt_l);
    }
    __syncthreads();
    const float g = __ldg(gain + m);
    for (int r = threadIdx.x; r < d.S; r += blockDim.x) {
        float ur[W], ui[W];
#pragma unroll
        for (int k = 0; k < W; ++k) ur[k] = ui[k] = 0.f;
        for (int k = 0; k < d.K; ++k) {
#pragma unroll
            for (int di = 0; di < W; ++di) {
                const int o = k * W + di;
                const float2 y = sy[o];
                const float2 w = __ldg(tw2_qr + (size_t)o * d.S + r);
                ur[di] = fmaf(y.x, w.x, fmaf(y.y, w.y, ur[di]));
                ui[di] = fmaf(y.y, w.x, fmaf(-y.x, w.y, ui[di]));
            }
        }
        const float gv = g * __ldg(T.v + r);
        float *c = coef + (size_t)seg * W * d.S + r;
        c[0] = gv * ur[HW];
#pragma unroll
        for (int k = 1; k <= HW; ++k) {
            c[(size_t)k * d.S] = gv * (ur[HW + k] + ur[HW - k]);
            c[(size_t)(HW + k) * d.S] = gv * (ui[HW + k] - ui[HW - k]);
        }
    }
}

// Adjoint, second step: cz[m][u][e] for a chunk of kZSynCols detector columns, from
// the coefficients of every line. Lines are taken kZSynLines at a time (one parity, 2
// apart: l0 + 2i), in bands of 2 kZSynLines, even group then odd.
//  synthesis  the thread of phase r generates the samples of its phase that read a
//             column of the chunk (periods in increasing column order) and sums them
//             into t[i][u][r] (weights 1 - a and a, columns written once complete);
//  z gather   cell e = Q l + o of line l collects the taps of offset o, the phases with
//             n0_r = o (weight 1 - f0_r) or n0_r + 1 = o (weight f0_r). A warp takes one
//             offset at a time with its lanes on (column, line): one tap list per warp.
//             Cells of two lines coincide only for offsets 2Q apart, and each warp keeps
//             to one class of offsets modulo 2Q, so no two warps add to the same cell;
//  flush      cells below Q times the lowest line not yet taken are final: they are
//             written to cz and their ring slots cleared.
// Every cell is a sum in a fixed order: the result does not depend on scheduling.
static_assert(kZSynLines * kZSynCols == 32, "the z gather puts (column, line) on the lanes of a warp");

// The period range of a warp that reaches columns [ub - 1, ub + UC) on parity par, and
// the lane's position at its start.
__device__ __forceinline__ void zsyn_range(int par, int re, int ub, int UC, const Dims &d, int N1, int Lm1,
                                           int &qlo, int &qhi, int &u0, int &rem) {
    const int j0 = par ? d.S - 1 - re : re;
    int qa = 0, qb = d.P;
    if (N1 > 0) {
        const long long step = (long long)N1 * d.S;
        const long long na = (long long)(ub - 1) * Lm1 - (long long)N1 * j0;
        const long long nb_ = (long long)(ub + UC) * Lm1 - (long long)N1 * j0;
        qa = na <= 0 ? 0 : (int)min((long long)d.P, (na + step - 1) / step);
        qb = nb_ <= 0 ? 0 : (int)min((long long)d.P, (nb_ + step - 1) / step);
    }
    qlo = __reduce_min_sync(0xffffffffu, qa);
    qhi = __reduce_max_sync(0xffffffffu, qb);
    slow_start(N1, Lm1, qlo * d.S + j0, u0, rem);
}

template <int HW>
__global__ void __launch_bounds__(128) k_zsyn_gather(const float *__restrict__ coef, const float *__restrict__ tw1,
                                                     const ZTables T, float *__restrict__ cz, Dims d, int zigzag,
                                                     int rb) {
    constexpr int W = 2 * HW + 1, WP = (W + 3) & ~3, R = kZSynLines, UC = kZSynCols;
    extern __shared__ float4 sm4[];
    const int bd = blockDim.x;
    const int no = T.no;
    const int SP = d.S + 1;                       // padded t rows: lanes on (column, line) hit distinct banks
    float *stw = reinterpret_cast<float *>(sm4);  // P * WP
    float *tl = stw + d.P * WP;                   // [R][UC][SP]
    const int RS = rb + 1;                        // padded ring rows: the 8 columns of a line in distinct banks
    float *ring = tl + R * UC * SP;               // [UC][RS]
    int *optr = reinterpret_cast<int *>(ring + UC * RS);  // no + 1 (UC RS is even: otap stays 8-byte aligned)
    int2 *otap = reinterpret_cast<int2 *>(optr + ((no + 2) & ~1));  // (r, weight bits)
    const int nchunk = (d.N + UC - 1) / UC;
    const int m = blockIdx.x / nchunk, ub = (blockIdx.x - m * nchunk) * UC;
    stage_twiddles<HW>(stw, tw1, d.P);
    for (int i = threadIdx.x; i <= no; i += bd) optr[i] = __ldg(T.optr + i);
    for (int i = threadIdx.x; i < 2 * d.S; i += bd) otap[i] = __ldg(T.otap + i);
    for (int i = threadIdx.x; i < UC * RS; i += bd) ring[i] = 0.f;
    const int N1 = d.N - 1, Lm1 = d.L - 1;
    const int du = N1 * d.S / Lm1, drem = N1 * d.S - du * Lm1;
    const float inv = 1.f / (float)Lm1;
    const bool one_pass = d.S <= bd;
    // positions of both parities, kept when one pass covers S
    int cq0[2], cq1[2], cu[2], cr[2];
    if (one_pass) {
        const int re = min((int)threadIdx.x, d.S - 1);
        zsyn_range(0, re, ub, UC, d, N1, Lm1, cq0[0], cq1[0], cu[0], cr[0]);
        zsyn_range(1, re, ub, UC, d, N1, Lm1, cq0[1], cq1[1], cu[1], cr[1]);
    }
    __syncthreads();
    const float *ctm = coef + (size_t)m * d.Nz * W * d.S;
    float *czm = cz + (size_t)m * d.N * d.Nez;
    const int ngroups = 2 * ((d.Nz + 2 * R - 1) / (2 * R));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = bd >> 5;
    const int gl = lane / UC, gu = lane - gl * UC;  // gather lane: line gl, column gu
    int flushed = 0;  // cells below are written
    for (int gi = 0; gi <= ngroups; ++gi) {
        // cells below Q times the lowest line not yet taken are final
        const int lim = gi == ngroups ? d.Nez : min(d.Nez, d.Q * ((gi >> 1) * 2 * R + (gi & 1)));
        if (lim > flushed) {
            const int cnt = lim - flushed;
            for (int c = threadIdx.x; c < UC * cnt; c += bd) {
                const int ul = c / cnt, e = flushed + (c - ul * cnt);
                float *slot = ring + ul * RS + (e & (rb - 1));
                if (ub + ul < d.N) czm[(size_t)(ub + ul) * d.Nez + e] = *slot;
                *slot = 0.f;
            }
            flushed = lim;
        }
        if (gi == ngroups) break;
        const int l0 = (gi >> 1) * 2 * R + (gi & 1);
        if (l0 >= d.Nz) continue;  // uniform: an empty odd group
        const int par = zigzag ? (gi & 1) : 0;
        // synthesis
        for (int r0 = 0; r0 < d.S; r0 += bd) {
            const int r = r0 + threadIdx.x, re = min(r, d.S - 1);
            const bool live = r < d.S;
            float cf[R][W];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int l = l0 + 2 * i;
#pragma unroll
                for (int k = 0; k < W; ++k) cf[i][k] = l < d.Nz ? __ldg(ctm + ((size_t)l * W + k) * d.S + re) : 0.f;
            }
            int q, qend, u0, rem;
            if (one_pass) {  // (selects, not a dynamic index: the pairs stay in registers)
                q = par ? cq0[1] : cq0[0];
                qend = par ? cq1[1] : cq1[0];
                u0 = par ? cu[1] : cu[0];
                rem = par ? cr[1] : cr[0];
            } else {
                zsyn_range(par, re, ub, UC, d, N1, Lm1, q, qend, u0, rem);
            }
            const int dtp = par ? -WP : WP;
            int u = ub - 1;  // the columns u and u + 1 are open
            float acc0[R], acc1[R];
#pragma unroll
            for (int i = 0; i < R; ++i) acc0[i] = acc1[i] = 0.f;
            if (q < qend) {
                const float *tp = stw + (par ? d.P - 1 - q : q) * WP;
                for (; q < qend; ++q) {
                    float t[WP];
                    load_twiddles<WP>(tp, t);
                    float v[R];
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        float x = 0.f;
#pragma unroll
                        for (int k = 0; k <= HW; ++k) x = fmaf(cf[i][k], t[k], x);
#pragma unroll
                        for (int k = 1; k <= HW; ++k) x = fmaf(cf[i][HW + k], t[HW + k], x);
                        v[i] = x;
                    }
                    const float a = (float)rem * inv;
                    if (u0 >= ub - 1 && u0 < ub + UC) {
                        while (u < u0) {  // column u is complete
                            if (u >= ub && live) {
#pragma unroll
                                for (int i = 0; i < R; ++i) tl[(i * UC + (u - ub)) * SP + r] = acc0[i];
                            }
#pragma unroll
                            for (int i = 0; i < R; ++i) {
                                acc0[i] = acc1[i];
                                acc1[i] = 0.f;
                            }
                            ++u;
                        }
#pragma unroll
                        for (int i = 0; i < R; ++i) {
                            acc0[i] = fmaf(1.f - a, v[i], acc0[i]);
                            acc1[i] = fmaf(a, v[i], acc1[i]);
                        }
                    }
                    tp += dtp;
                    u0 += du;
                    rem += drem;
                    if (rem >= Lm1) {
                        rem -= Lm1;
                        ++u0;
                    }
                }
            }
            for (; u < ub + UC; ++u) {
                if (u >= ub && live) {
#pragma unroll
                    for (int i = 0; i < R; ++i) tl[(i * UC + (u - ub)) * SP + r] = acc0[i];
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    acc0[i] = acc1[i];
                    acc1[i] = 0.f;
                }
            }
        }
        __syncthreads();
        // z gather into the ring: warp w takes the offsets of classes w, w + nwarps, ...
        // modulo 2Q, each class in increasing offset order
        const int l = l0 + 2 * gl;
        const bool lv = l < d.Nz;
        const float *ti = tl + (gl * UC + gu) * SP;
        float *rr = ring + gu * RS;
        for (int cls = warp; cls < 2 * d.Q; cls += nwarps) {
            for (int o = cls; o < no; o += 2 * d.Q) {
                float sum = 0.f;
                for (int k = optr[o]; k < optr[o + 1]; ++k) {
                    const int2 tap = otap[k];
                    sum = fmaf(__int_as_float(tap.y), ti[tap.x], sum);
                }
                const int e = d.Q * l + o;
                if (lv && e < d.Nez) rr[e & (rb - 1)] += sum;
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

template <int HW>
static void zdft_fwd_hw(const float *cz, const ZTables &T, const float *gain, const float *tw1, const float2 *tw2_ro,
                        const float2 *dgam, float *data, const Dims &d, int zigzag, cudaStream_t st) {
    const int uc = zdft_chunk(d);
    const size_t smem = zdft_fwd_smem(d);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_zdft_fwd<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    const int nband = (d.Nz + 2 * kZLines - 1) / (2 * kZLines);
    k_zdft_fwd<HW><<<d.M * 2 * nband, 128, smem, st>>>(cz, T, gain, tw1, tw2_ro, dgam, data, d, zigzag, uc,
                                                        (float)(1.0 / sqrt((double)d.L)));
}

template <int HW>
static void zdft_adj_hw(const float *data, const float *tw1, const float2 *tw2_qr, const float2 *dgam,
                        const ZTables &T, const float *gain, float *coef, float *cz, const Dims &d, int zigzag,
                        cudaStream_t st) {
    const float inv_sqrt_l = (float)(1.0 / sqrt((double)d.L));
    k_zsyn_coef<HW><<<d.nseg, 128, sizeof(float2) * d.nb, st>>>(data, tw2_qr, dgam, T, gain, coef, d, inv_sqrt_l);
    const int rb = zsyn_ring(d, T.no);
    const size_t smem = zsyn_smem(d, T.no);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_zsyn_gather<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    const int nchunk = (d.N + kZSynCols - 1) / kZSynCols;
    k_zsyn_gather<HW><<<d.M * nchunk, 128, smem, st>>>(coef, tw1, T, cz, d, zigzag, rb);
}

#define MPIFFL_ZHW_DISPATCH(FN, ...)                \
    switch (d.hw) {                                 \
        case 0: FN<0>(__VA_ARGS__); break;          \
        case 1: FN<1>(__VA_ARGS__); break;          \
        case 2: FN<2>(__VA_ARGS__); break;          \
        case 3: FN<3>(__VA_ARGS__); break;          \
        case 4: FN<4>(__VA_ARGS__); break;          \
        case 5: FN<5>(__VA_ARGS__); break;          \
        case 6: FN<6>(__VA_ARGS__); break;          \
        case 7: FN<7>(__VA_ARGS__); break;          \
        default: FN<8>(__VA_ARGS__); break;         \
    }

// E_z V_z B fused with S D_Gamma F
void launch_zdft_fwd(const float *cz, const ZTables &T, const float *gain, const float *tw1, const float2 *tw2_ro,
                     const float2 *dgam, float *data, const Dims &d, int zigzag, cudaStream_t st) {
    MPIFFL_ZHW_DISPATCH(zdft_fwd_hw, cz, T, gain, tw1, tw2_ro, dgam, data, d, zigzag, st);
}

// (S D F)^T fused with the transpose of E_z V_z B: coefficients, then cz
void launch_zdft_adj(const float *data, const float *tw1, const float2 *tw2_qr, const float2 *dgam,
                     const ZTables &T, const float *gain, float *coef, float *cz, const Dims &d, int zigzag,
                     cudaStream_t st) {
    MPIFFL_ZHW_DISPATCH(zdft_adj_hw, data, tw1, tw2_qr, dgam, T, gain, coef, cz, d, zigzag, st);
}

}  // namespace mpiffl
