// Staged per-line kernels of A_DC = S D_Gamma F V E H B (Sec. 2.1, Eq. (13)) and of
// its transpose, in FP32 on CUDA cores. A "segment" is one raster line (z slice)
// of one angle: proj[seg][N] -> fine[seg][N_e] -> sig[seg][L] -> data[seg][nb].
//
// H   : full-support polyphase convolution on the fine grid. Output e has phase
//       (e - D) mod Q; a thread owns kPsfT outputs of one phase and slides a
//       register window over the tap table, so each tap load feeds kPsfT FMAs.
// EVB : velocity-weighted linear interpolation at the FFL positions; the
//       trajectory table is read once per group of kGroup lines that share it.
//       The transpose gathers through a per-trajectory CSR (fine cell <- samples).
// F   : the band DFT factorised over the period structure j = p S + r:
//       b[k, d] = L^-1/2 sum_r e^{2 pi i (kP+d) r / L} sum_p s[pS+r] e^{2 pi i d p / P},
//       exactly equal to Eq. (27) on the kept bins. The inner sum over periods
//       costs 2w+1 FMAs per sample (the signal is real); the outer one is small.
#include "internal.h"

namespace mpiffl {

// ----------------------------------------------------------------------------- H

__global__ void __launch_bounds__(256) k_psf_fwd(const float *__restrict__ proj,
                                                 const float *__restrict__ htab,
                                                 float *__restrict__ fine, Dims d) {
    extern __shared__ float sm[];
    float *sp = sm;            // N
    float *sh = sm + d.N;      // htab_len
    const int seg = blockIdx.x;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) sp[i] = proj[(size_t)seg * d.N + i];
    for (int i = threadIdx.x; i < d.htab_len; i += blockDim.x) sh[i] = htab[i];
    __syncthreads();
    const int Q = d.Q;
    const int n_a = (d.Ne + Q - 1) / Q;               // fine points per phase (upper bound)
    const int n_ab = (n_a + kPsfT - 1) / kPsfT;       // register blocks per phase
    for (int task = threadIdx.x; task < Q * n_ab; task += blockDim.x) {
        const int q = task % Q;
        const int ab = task / Q;
        const int base = q - d.D + d.htab_off + Q * ab * kPsfT;
        float w[kPsfT], acc[kPsfT];
#pragma unroll
        for (int t = 0; t < kPsfT; ++t) {
            w[t] = sh[base + Q * t];
            acc[t] = 0.f;
        }
        for (int i = 0; i < d.N; ++i) {
            const float pi = sp[i];
#pragma unroll
            for (int t = 0; t < kPsfT; ++t) acc[t] = fmaf(pi, w[t], acc[t]);
#pragma unroll
            for (int t = kPsfT - 1; t > 0; --t) w[t] = w[t - 1];
            w[0] = sh[base - Q * (i + 1)];
        }
        float *out = fine + (size_t)seg * d.Ne;
#pragma unroll
        for (int t = 0; t < kPsfT; ++t) {
            const int e = q + Q * (ab * kPsfT + t);
            if (e < d.Ne) out[e] = acc[t];
        }
    }
}

void launch_psf_fwd(const float *proj, const float *htab, float *fine, const Dims &d, cudaStream_t st) {
    const size_t smem = sizeof(float) * (d.N + d.htab_len);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_psf_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_psf_fwd<<<d.nseg, 256, smem, st>>>(proj, htab, fine, d);
}

// H^T: proj[i] = sum_e fine[e] h((e - D)/Q - i). Lanes of a warp are
// (segment s = lane / Q, phase q = lane % Q): each owns kPsfT outputs i0..i0+T-1 of its
// segment and sums the fine points of its phase with a sliding tap window; the Q
// phase partials are then added with shuffles. Rows sit kPsfRowPad floats apart
// modulo 32 so that the lanes' row reads fall in distinct banks, and the tap
// reads of different segments coincide (broadcast).
constexpr int kPsfAdjThreads = 256;

__global__ void __launch_bounds__(kPsfAdjThreads) k_psf_adj(const float *__restrict__ fine,
                                                            const float *__restrict__ htab,
                                                            float *__restrict__ proj, Dims d, int row_stride,
                                                            int segs_per_block) {
    extern __shared__ float sm[];
    float *sh = sm;                      // htab_len
    float *sf = sm + d.htab_len;         // segs_per_block rows of row_stride floats
    const int seg0 = blockIdx.x * segs_per_block;
    const int nsg = min(segs_per_block, d.nseg - seg0);
    for (int i = threadIdx.x; i < d.htab_len; i += blockDim.x) sh[i] = htab[i];
    for (int sl = 0; sl < nsg; ++sl)
        for (int e = threadIdx.x; e < d.Ne; e += blockDim.x)
            sf[sl * row_stride + e] = fine[(size_t)(seg0 + sl) * d.Ne + e];
    __syncthreads();
    const int Q = d.Q;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int q = lane % Q;
    const int sl = lane / Q;               // segment within the block handled by this lane
    const int n_ib = (d.N + kPsfT - 1) / kPsfT;
    const bool active_seg = sl < nsg;
    const float *row = sf + (active_seg ? sl : 0) * row_stride;
    for (int ib = warp; ib < n_ib; ib += nwarps) {
        const int i0 = ib * kPsfT;
        float acc[kPsfT];
#pragma unroll
        for (int t = 0; t < kPsfT; ++t) acc[t] = 0.f;
        const int baseq = q - d.D - Q * i0 + d.htab_off;
        float w[kPsfT];
#pragma unroll
        for (int t = 0; t < kPsfT; ++t) w[t] = sh[baseq - Q * t];
        for (int a = 0, e = q; e < d.Ne; ++a, e += Q) {
            const float c = row[e];
#pragma unroll
            for (int t = 0; t < kPsfT; ++t) acc[t] = fmaf(c, w[t], acc[t]);
#pragma unroll
            for (int t = kPsfT - 1; t > 0; --t) w[t] = w[t - 1];
            w[0] = sh[baseq + Q * (a + 1)];
        }
        // add the Q phase partials (lanes sl*Q .. sl*Q+Q-1)
#pragma unroll
        for (int t = 0; t < kPsfT; ++t)
            for (int o = 1; o < Q; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        if (active_seg && q == 0) {
            float *out = proj + (size_t)(seg0 + sl) * d.N;
#pragma unroll
            for (int t = 0; t < kPsfT; ++t)
                if (i0 + t < d.N) out[i0 + t] = acc[t];
        }
    }
}

void launch_psf_adj(const float *fine, const float *htab, float *proj, const Dims &d, cudaStream_t st) {
    // lanes = (segment, phase); Q must be a power of two dividing 32 for the shuffle tree
    const int segs = 32 / d.Q;
    const int stride = d.Ne + (((d.Q - d.Ne) % 32) + 32) % 32;  // stride = Q (mod 32)
    const size_t smem = sizeof(float) * (d.htab_len + (size_t)segs * stride);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_psf_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_psf_adj<<<(d.nseg + segs - 1) / segs, kPsfAdjThreads, smem, st>>>(fine, htab, proj, d, stride, segs);
}

// ----------------------------------------------------------------------------- E V B

__global__ void __launch_bounds__(256) k_resample_fwd(const float *__restrict__ fine,
                                                      const TrajEntry *__restrict__ traj,
                                                      const float *__restrict__ gain,
                                                      const SegGroup *__restrict__ groups,
                                                      float *__restrict__ sig, Dims d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.L) return;
    const SegGroup g = groups[blockIdx.y];
    const TrajEntry te = traj[(size_t)g.parity * d.L + j];
    const float gm = gain[g.m];
    for (int l = 0; l < g.count; ++l) {
        const int seg = g.m * d.Nz + g.z0 + l * g.zstride;
        const float *row = fine + (size_t)seg * d.Ne;
        const float v = fmaf(te.w0, __ldg(row + te.n), te.w1 * __ldg(row + te.n + 1));
        sig[(size_t)seg * d.L + j] = gm * v;
    }
}

void launch_resample_fwd(const float *fine, const TrajEntry *traj, const float *gain,
                         const SegGroup *groups, int n_groups, float *sig, const Dims &d,
                         cudaStream_t st) {
    dim3 grid((d.L + 255) / 256, n_groups);
    k_resample_fwd<<<grid, 256, 0, st>>>(fine, traj, gain, groups, sig, d);
}

__global__ void __launch_bounds__(128) k_resample_adj(const float *__restrict__ sig,
                                                      const int *__restrict__ csr_ptr,
                                                      const CsrEntry *__restrict__ csr,
                                                      const float *__restrict__ gain,
                                                      const SegGroup *__restrict__ groups,
                                                      float *__restrict__ fine, Dims d) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.Ne) return;
    const SegGroup g = groups[blockIdx.y];
    const int *ptr = csr_ptr + (size_t)g.parity * (d.Ne + 1);
    const CsrEntry *ent = csr + (size_t)g.parity * 2 * d.L;
    float acc[kGroup];
#pragma unroll
    for (int l = 0; l < kGroup; ++l) acc[l] = 0.f;
    const size_t seg0 = (size_t)g.m * d.Nz + g.z0;
    const size_t stride = (size_t)g.zstride * d.L;
    const float *s0 = sig + seg0 * d.L;
    for (int k = ptr[e]; k < ptr[e + 1]; ++k) {
        const CsrEntry c = ent[k];
#pragma unroll
        for (int l = 0; l < kGroup; ++l)
            if (l < g.count) acc[l] = fmaf(c.w, __ldg(s0 + l * stride + c.j), acc[l]);
    }
    const float gm = gain[g.m];
#pragma unroll
    for (int l = 0; l < kGroup; ++l)
        if (l < g.count) fine[(seg0 + (size_t)l * g.zstride) * d.Ne + e] = gm * acc[l];
}

void launch_resample_adj(const float *sig, const int *csr_ptr, const CsrEntry *csr,
                         const float *gain, const SegGroup *groups, int n_groups, float *fine,
                         const Dims &d, cudaStream_t st) {
    dim3 grid((d.Ne + 127) / 128, n_groups);
    k_resample_adj<<<grid, 128, 0, st>>>(sig, csr_ptr, csr, gain, groups, fine, d);
}

// ----------------------------------------------------------------------------- S D F

// Twiddle table tw1[p][0..W): cos(2 pi d p / P) for d = 0..hw, then sin(2 pi d p / P)
// for d = 1..hw.
template <int HW>
__global__ void __launch_bounds__(128) k_dft_fwd(const float *__restrict__ sig,
                                                 const float *__restrict__ tw1,
                                                 const float2 *__restrict__ tw2_ro,
                                                 const float2 *__restrict__ dgam,
                                                 float *__restrict__ data, Dims d, float inv_sqrt_l) {
    extern __shared__ float sm[];
    const int W = 2 * HW + 1;
    float *stw = sm;                               // P * W
    float2 *sT = (float2 *)(sm + d.P * W);         // S * W
    const int seg = blockIdx.x;
    for (int i = threadIdx.x; i < d.P * W; i += blockDim.x) stw[i] = tw1[i];
    __syncthreads();
    const float *s = sig + (size_t)seg * d.L;
    for (int r = threadIdx.x; r < d.S; r += blockDim.x) {
        float ac[HW + 1], as[HW + 1];
#pragma unroll
        for (int k = 0; k <= HW; ++k) ac[k] = as[k] = 0.f;
        for (int p = 0; p < d.P; ++p) {
            const float v = __ldg(s + (size_t)p * d.S + r);
            const float *t = stw + p * W;
#pragma unroll
            for (int k = 0; k <= HW; ++k) ac[k] = fmaf(v, t[k], ac[k]);
#pragma unroll
            for (int k = 1; k <= HW; ++k) as[k] = fmaf(v, t[HW + k], as[k]);
        }
#pragma unroll
        for (int k = -HW; k <= HW; ++k) {
            const int a = k < 0 ? -k : k;
            sT[r * W + (k + HW)] = make_float2(ac[a], k < 0 ? -as[a] : as[a]);
        }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < d.nb; o += blockDim.x) {
        const int di = o % W;
        float re = 0.f, im = 0.f;
        for (int r = 0; r < d.S; ++r) {
            const float2 t = sT[r * W + di];
            const float2 w = __ldg(tw2_ro + (size_t)r * d.nb + o);
            re = fmaf(t.x, w.x, fmaf(-t.y, w.y, re));
            im = fmaf(t.x, w.y, fmaf(t.y, w.x, im));
        }
        const float2 g = dgam[o];
        re *= inv_sqrt_l;
        im *= inv_sqrt_l;
        float2 *out = (float2 *)data + (size_t)seg * d.nb + o;
        *out = make_float2(g.x * re - g.y * im, g.x * im + g.y * re);
    }
}

template <int HW>
__global__ void __launch_bounds__(128) k_dft_adj(const float *__restrict__ data,
                                                 const float *__restrict__ tw1,
                                                 const float2 *__restrict__ tw2_qr,
                                                 const float2 *__restrict__ dgam,
                                                 float *__restrict__ sig, Dims d, float inv_sqrt_l) {
    extern __shared__ float sm[];
    const int W = 2 * HW + 1;
    float *stw = sm;                               // P * W
    float2 *sy = (float2 *)(sm + d.P * W);         // nb: conj(D) y / sqrt(L)
    const int seg = blockIdx.x;
    for (int i = threadIdx.x; i < d.P * W; i += blockDim.x) stw[i] = tw1[i];
    for (int o = threadIdx.x; o < d.nb; o += blockDim.x) {
        const float2 y = ((const float2 *)data)[(size_t)seg * d.nb + o];
        const float2 g = dgam[o];
        sy[o] = make_float2((g.x * y.x + g.y * y.y) * inv_sqrt_l, (g.x * y.y - g.y * y.x) * inv_sqrt_l);
    }
    __syncthreads();
    float *s = sig + (size_t)seg * d.L;
    for (int r = threadIdx.x; r < d.S; r += blockDim.x) {
        // U[d] = sum_k y'[k,d] exp(-2 pi i (kP+d) r / L)
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
        // s[pS+r] = sum_d Re(U[d] e^{-2 pi i d p / P}) = sum_{d>=0} A_d cos + sum_{d>0} B_d sin
        float A[HW + 1], B[HW + 1];
        A[0] = ur[HW];
        B[0] = 0.f;
#pragma unroll
        for (int k = 1; k <= HW; ++k) {
            A[k] = ur[HW + k] + ur[HW - k];
            B[k] = ui[HW + k] - ui[HW - k];
        }
        for (int p = 0; p < d.P; ++p) {
            const float *t = stw + p * W;
            float v = 0.f;
#pragma unroll
            for (int k = 0; k <= HW; ++k) v = fmaf(A[k], t[k], v);
#pragma unroll
            for (int k = 1; k <= HW; ++k) v = fmaf(B[k], t[HW + k], v);
            s[(size_t)p * d.S + r] = v;
        }
    }
}

template <int HW>
static void dft_fwd_hw(const float *sig, const float *tw1, const float2 *tw2_ro, const float2 *dgam,
                       float *data, const Dims &d, cudaStream_t st) {
    const int W = 2 * HW + 1;
    const size_t smem = sizeof(float) * d.P * W + sizeof(float2) * d.S * W;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_dft_fwd<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_dft_fwd<HW><<<d.nseg, 128, smem, st>>>(sig, tw1, tw2_ro, dgam, data, d, (float)(1.0 / sqrt((double)d.L)));
}

template <int HW>
static void dft_adj_hw(const float *data, const float *tw1, const float2 *tw2_qr, const float2 *dgam,
                       float *sig, const Dims &d, cudaStream_t st) {
    const int W = 2 * HW + 1;
    const size_t smem = sizeof(float) * d.P * W + sizeof(float2) * d.nb;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_dft_adj<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_dft_adj<HW><<<d.nseg, 128, smem, st>>>(data, tw1, tw2_qr, dgam, sig, d, (float)(1.0 / sqrt((double)d.L)));
}

#define MPIFFL_HW_DISPATCH(FN, ...)                 \
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

void launch_dft_fwd(const float *sig, const float *tw1, const float2 *tw2_ro, const float2 *dgam,
                    float *data, const Dims &d, cudaStream_t st) {
    MPIFFL_HW_DISPATCH(dft_fwd_hw, sig, tw1, tw2_ro, dgam, data, d, st);
}

void launch_dft_adj(const float *data, const float *tw1, const float2 *tw2_qr, const float2 *dgam,
                    float *sig, const Dims &d, cudaStream_t st) {
    MPIFFL_HW_DISPATCH(dft_adj_hw, data, tw1, tw2_qr, dgam, sig, d, st);
}

}  // namespace mpiffl
