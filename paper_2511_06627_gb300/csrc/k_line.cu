// Staged per-line kernels of A_DC = S D_Gamma F V E H B (Sec. 2.1, Eq. (13)) and of
// its transpose, in FP32 on CUDA cores. A "segment" is one raster line (z slice)
// of one angle: proj[seg][N] -> fine[seg][N_e] -> sig[seg][L] -> data[seg][nb].
//
// H   : full-support polyphase convolution on the fine grid. Output e has phase
//       (e - D) mod Q; a thread owns kPsfTF outputs of one phase and slides a
//       register window over the tap table, so each tap load feeds kPsfTF FMAs.
// EVB : velocity-weighted linear interpolation at the FFL positions; the
//       trajectory table is read once per group of kGroup lines that share it.
//       The transpose gathers through a per-trajectory CSR (fine cell <- samples).
// F   : the band DFT factorised over the period structure j = p S + r:
//       b[k, d] = L^-1/2 sum_r e^{2 pi i (kP+d) r / L} sum_p s[pS+r] e^{2 pi i d p / P},
//       exactly equal to Eq. (27) on the kept bins. The inner sum over periods
//       costs 2w+1 FMAs per sample (the signal is real); the outer one is small.
#include "internal.h"
#include "tc_ptx.cuh"

namespace mpiffl {

// ----------------------------------------------------------------------------- H

// Nine outputs per thread: at Q = 8 the 30 register blocks of the 8 phases of a
// 256-bin line fill one round of 256 threads, and lanes of different blocks read taps
// 9 Q words apart, in distinct banks (with eight, 34 blocks took two rounds and four
// lanes shared each bank).
constexpr int kPsfTF = 9;
// sixteen outputs per lane in the transpose: 16 FMAs per pair of shared loads
constexpr int kPsfTA = 16;
static_assert(kPsfTF <= kPsfT && kPsfTA <= kPsfT, "the tap table is padded for the windows");

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
    const int n_ab = (n_a + kPsfTF - 1) / kPsfTF;       // register blocks per phase
    for (int task = threadIdx.x; task < Q * n_ab; task += blockDim.x) {
        const int q = task % Q;
        const int ab = task / Q;
        const int base = q - d.D + d.htab_off + Q * ab * kPsfTF;
        float w[kPsfTF], acc[kPsfTF];
#pragma unroll
        for (int t = 0; t < kPsfTF; ++t) {
            w[t] = sh[base + Q * t];
            acc[t] = 0.f;
        }
        // unrolled by the window length, so that the window's shift is a renaming of
        // registers rather than moves
#pragma unroll kPsfTF
        for (int i = 0; i < d.N; ++i) {
            const float pi = sp[i];
#pragma unroll
            for (int t = 0; t < kPsfTF; ++t) acc[t] = fmaf(pi, w[t], acc[t]);
#pragma unroll
            for (int t = kPsfTF - 1; t > 0; --t) w[t] = w[t - 1];
            w[0] = sh[base - Q * (i + 1)];
        }
        float *out = fine + (size_t)seg * d.Ne;
#pragma unroll
        for (int t = 0; t < kPsfTF; ++t) {
            const int e = q + Q * (ab * kPsfTF + t);
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
// (segment s = lane / Q, phase q = lane % Q): each owns kPsfTA outputs i0..i0+T-1 of its
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
    const int n_ib = (d.N + kPsfTA - 1) / kPsfTA;
    const bool active_seg = sl < nsg;
    const float *row = sf + (active_seg ? sl : 0) * row_stride;
    for (int ib = warp; ib < n_ib; ib += nwarps) {
        const int i0 = ib * kPsfTA;
        float acc[kPsfTA];
#pragma unroll
        for (int t = 0; t < kPsfTA; ++t) acc[t] = 0.f;
        const int baseq = q - d.D - Q * i0 + d.htab_off;
        float w[kPsfTA];
#pragma unroll
        for (int t = 0; t < kPsfTA; ++t) w[t] = sh[baseq - Q * t];
#pragma unroll kPsfTA
        for (int a = 0, e = q; e < d.Ne; ++a, e += Q) {
            const float c = row[e];
#pragma unroll
            for (int t = 0; t < kPsfTA; ++t) acc[t] = fmaf(c, w[t], acc[t]);
#pragma unroll
            for (int t = kPsfTA - 1; t > 0; --t) w[t] = w[t - 1];
            w[0] = sh[baseq + Q * (a + 1)];
        }
        // add the Q phase partials (lanes sl*Q .. sl*Q+Q-1)
#pragma unroll
        for (int t = 0; t < kPsfTA; ++t)
            for (int o = 1; o < Q; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
        if (active_seg && q == 0) {
            float *out = proj + (size_t)(seg0 + sl) * d.N;
#pragma unroll
            for (int t = 0; t < kPsfTA; ++t)
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

// Four samples per thread, each of the group's lines: the signal s = g_m v_j lerp of the
// fine row at the FFL position (one product per tap, the same for every line).
__global__ void __launch_bounds__(256) k_resample_fwd4(const float *__restrict__ fine,
                                                       const TrajEntry *__restrict__ traj,
                                                       const float *__restrict__ gain,
                                                       const SegGroup *__restrict__ groups,
                                                       float *__restrict__ sig, Dims d) {
    // A warp takes 128 consecutive samples, lane l the samples l, l + 32, l + 64, l + 96:
    // the lanes of one gather read neighbouring fine cells (a few sectors per load,
    // where four consecutive samples per lane spread a load over a sector per lane),
    // and each store is one 128-byte line of the signal, stored with the streaming hint
    // (written once, read once by the band DFT).
    const int lane = threadIdx.x & 31;
    const int jw = 4 * (blockIdx.x * blockDim.x + (threadIdx.x & ~31));
    const SegGroup g = groups[blockIdx.y];
    TrajEntry te[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int j = jw + lane + 32 * u;
        te[u] = j < d.L ? traj[(size_t)g.parity * d.L + j] : TrajEntry{0, 0.f, 0.f};
    }
    const float gm = gain[g.m];
#pragma unroll
    for (int l = 0; l < kGroup; ++l) {
        if (l >= g.count) break;
        const int seg = g.m * d.Nz + g.z0 + l * g.zstride;
        const float *row = fine + (size_t)seg * d.Ne;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = jw + lane + 32 * u;
            const float v = gm * fmaf(te[u].w0, __ldg(row + te[u].n), te[u].w1 * __ldg(row + te[u].n + 1));
            if (j < d.L) __stcs(sig + (size_t)seg * d.L + j, v);
        }
    }
}

void launch_resample_fwd(const float *fine, const TrajEntry *traj, const float *gain,
                         const SegGroup *groups, int n_groups, float *sig, const Dims &d,
                         cudaStream_t st) {
    dim3 grid((d.L + 1023) / 1024, n_groups);
    k_resample_fwd4<<<grid, 256, 0, st>>>(fine, traj, gain, groups, sig, d);
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

// Tiled transpose of E V B. A block owns a tile of kRaCells fine cells of one angle and
// trajectory parity and runs over a chunk of that parity's lines. The CSR entries of its
// cells (sample j, weight w; ascending j per cell) are line-independent: each thread
// keeps its share of them in registers, with j relative to the tile's sample window
// [j_lo, j_lo + len), which covers every sample that touches a cell of the tile. Per
// line, one thread bulk-copies that window into shared memory (two buffers, the next
// line's copy in flight while this one is summed), and each cell sums its entries from
// there: the signal is read from HBM once per tile, in full 16-byte-aligned runs.
// Entry k of a cell belongs to half k & 1 of the block (threads c and c + kRaCells); the
// halves are added in that order. Padding entries point at a zero word past the window.
constexpr int kRaCells = kRaTileCells;
constexpr int kRaHalf = kRaMaxEntries / 2;
static_assert(kRaHalf % 2 == 0, "two 16-bit sample offsets per register");

__global__ void __launch_bounds__(2 * kRaCells, 1) k_resample_adj_tiled(
    const float *__restrict__ sig, const int4 *__restrict__ tiles, const uint16_t *__restrict__ tj,
    const float *__restrict__ tw, const float *__restrict__ gain, float *__restrict__ fine, Dims d, int ntile,
    int cap, int lines_per_block, int *err) {
    extern __shared__ __align__(128) float ra_sm[];  // 2 windows of cap + 4 floats, 2 x kRaCells partials
    float *win0 = ra_sm, *win1 = ra_sm + (cap + 4);
    float *part = ra_sm + 2 * (cap + 4);  // [2][kRaCells]
    uint64_t *full = reinterpret_cast<uint64_t *>(part + 2 * kRaCells);
    const int tid = threadIdx.x, c = tid % kRaCells, half = tid / kRaCells;
    // block -> (angle, parity, tile, chunk of lines)
    const int nl_par = (d.Nz + d.n_par - 1) / d.n_par;  // lines of one parity (upper bound)
    const int nchunk = (nl_par + lines_per_block - 1) / lines_per_block;
    int b = blockIdx.x;
    const int chunk = b % nchunk;
    b /= nchunk;
    const int tile = b % ntile;
    b /= ntile;
    const int par = b % d.n_par;
    const int m = b / d.n_par;
    const int4 T = tiles[par * ntile + tile];  // (j_lo, len, e0, ncell)
    // this thread's entries, j relative to the window (cap = the zero word)
    uint32_t jr[kRaHalf / 2];
    float w[kRaHalf];
    {
        const size_t base = (size_t)(par * ntile + tile) * kRaMaxEntries * kRaCells;
#pragma unroll
        for (int q = 0; q < kRaHalf; ++q) {
            const size_t at = base + (size_t)(2 * q + half) * kRaCells + c;
            w[q] = __ldg(tw + at);
            const uint32_t jv = __ldg(tj + at);
            if (q & 1) jr[q >> 1] |= jv << 16;
            else jr[q >> 1] = jv;
        }
    }
    if (tid == 0) {
        ptx::mbar_init(&full[0], 1);
        ptx::mbar_init(&full[1], 1);
        ptx::fence_mbar_init();
    }
    if (tid < 2) (tid ? win1 : win0)[cap] = 0.f;  // the padding entries' zero word
    __syncthreads();
    // lines of this parity: z = par + n_par * q; this block takes q in [q0, q1)
    const int q0 = chunk * lines_per_block;
    const int nz_par = (d.Nz - par + d.n_par - 1) / d.n_par;
    const int q1 = min(q0 + lines_per_block, nz_par);
    const uint32_t bytes = (uint32_t)T.y * 4u;
    auto issue = [&](int q, float *dst, uint64_t *bar) {
        const int z = par + d.n_par * q;
        ptx::mbar_arrive_expect_tx(bar, bytes);
        ptx::bulk_g2s(dst, sig + ((size_t)m * d.Nz + z) * d.L + T.x, bytes, bar);
    };
    if (tid == 0) {
        if (q0 < q1) issue(q0, win0, &full[0]);
        if (q0 + 1 < q1) issue(q0 + 1, win1, &full[1]);
    }
    const float gm = __ldg(gain + m);
    for (int q = q0; q < q1; ++q) {
        const int k = q - q0, bufi = k & 1;
        float *wn = bufi ? win1 : win0;
        const bool got = ptx::mbar_wait_bounded(&full[bufi], (k >> 1) & 1, 1u << 24);
        if (!__syncthreads_and(got)) {  // one decision for the whole block
            if (tid == 0) {
                atomicExch(err, 1);
                // the other buffer's copy, if one was issued, lands before the block leaves
                if (q + 1 < q1) ptx::mbar_wait_bounded(&full[bufi ^ 1], ((k + 1) >> 1) & 1, 1u << 24);
            }
            __syncthreads();
            break;
        }
        float acc = 0.f;
#pragma unroll
        for (int e = 0; e < kRaHalf; ++e) {
            const uint32_t jj = (jr[e >> 1] >> ((e & 1) * 16)) & 0xffffu;
            acc = fmaf(w[e], wn[jj], acc);
        }
        float *pt = part + bufi * kRaCells;
        if (half) pt[c] = acc;
        __syncthreads();  // window k read by all, partials written
        if (!half && c < T.w) {
            const int z = par + d.n_par * q;
            fine[((size_t)m * d.Nz + z) * d.Ne + T.z + c] = gm * (acc + pt[c]);
        }
        if (tid == 0 && q + 2 < q1) {
            ptx::fence_proxy_async_smem();  // the generic reads of the window, then its refill
            issue(q + 2, wn, &full[bufi]);
        }
    }
}

void launch_resample_adj_tiled(const float *sig, const int4 *tiles, const uint16_t *tj, const float *tw,
                               const float *gain, float *fine, const Dims &d, int ntile, int cap, int *err,
                               cudaStream_t st) {
    const int lines_per_block = 32;
    const int nl_par = (d.Nz + d.n_par - 1) / d.n_par;
    const int nchunk = (nl_par + lines_per_block - 1) / lines_per_block;
    const size_t smem = sizeof(float) * (2 * (size_t)(cap + 4) + 2 * kRaCells) + 2 * sizeof(uint64_t);
    cudaFuncSetAttribute(k_resample_adj_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    const int blocks = d.M * d.n_par * ntile * nchunk;
    k_resample_adj_tiled<<<blocks, 2 * kRaCells, smem, st>>>(sig, tiles, tj, tw, gain, fine, d, ntile, cap,
                                                             lines_per_block, err);
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

// Streaming form (S % 4 == 0, S <= 128): a warp owns one segment. Lane 0 bulk-copies the
// segment's signal through a ring of kDfStages chunks of kDfChunk periods (the warp's own
// mbarriers), and lane l sums the four phases 4l..4l+3 with one 16-byte load per period.
// The period twiddles e^{2 pi i k p / P} come from one table of e^{2 pi i q / P} at
// q = k p mod P, the same values as the per-(p, k) table. The phase sums are the same
// FMAs in the same order as the one-phase-per-thread form; the synthesis over phases
// then runs as there, in the warp's own ring memory.
constexpr int kDfWarps = 8;
constexpr int kDfChunk = 8;
constexpr int kDfStages = 3;

template <int HW>
__global__ void __launch_bounds__(32 * kDfWarps) k_dft_fwd_stream(const float *__restrict__ sig,
                                                                  const float2 *__restrict__ twp,
                                                                  const float2 *__restrict__ tw2_ro,
                                                                  const float2 *__restrict__ dgam,
                                                                  float *__restrict__ data, Dims d,
                                                                  float inv_sqrt_l, int *err) {
    constexpr int W = 2 * HW + 1;
    extern __shared__ __align__(128) float df_sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ring_f = kDfStages * kDfChunk * d.S;  // floats per warp
    float *ring = df_sm + (size_t)warp * ring_f;
    float2 *stp = reinterpret_cast<float2 *>(df_sm + (size_t)kDfWarps * ring_f);  // [P] e^{2 pi i q / P}
    uint64_t *bars = reinterpret_cast<uint64_t *>(stp + d.P) + warp * kDfStages;
    for (int i = threadIdx.x; i < d.P; i += blockDim.x) stp[i] = twp[i];
    if (lane == 0) {
        for (int k = 0; k < kDfStages; ++k) ptx::mbar_init(&bars[k], 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const int seg = blockIdx.x * kDfWarps + warp;
    if (seg >= d.nseg) return;
    const float *src = sig + (size_t)seg * d.L;
    const int nchunk = (d.P + kDfChunk - 1) / kDfChunk;
    auto issue = [&](int c) {
        const int per = min(kDfChunk, d.P - c * kDfChunk);
        const uint32_t bytes = (uint32_t)per * d.S * 4u;
        uint64_t *bar = &bars[c % kDfStages];
        ptx::mbar_arrive_expect_tx(bar, bytes);
        ptx::bulk_g2s(ring + (size_t)(c % kDfStages) * kDfChunk * d.S, src + (size_t)c * kDfChunk * d.S, bytes, bar);
    };
    if (lane == 0)
        for (int c = 0; c < kDfStages && c < nchunk; ++c) issue(c);
    const int nq = d.S / 4;
    const bool act = lane < nq;
    float ac[4][HW + 1], as[4][HW + 1];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k <= HW; ++k) ac[i][k] = as[i][k] = 0.f;
    int idx[HW + 1];  // k p mod P
#pragma unroll
    for (int k = 0; k <= HW; ++k) idx[k] = 0;
    bool good = true;
    for (int c = 0; c < nchunk; ++c) {
        const bool got = ptx::mbar_wait_bounded(&bars[c % kDfStages], (c / kDfStages) & 1, 1u << 24);
        if (!__all_sync(0xffffffffu, got)) {
            good = false;
            break;
        }
        const float *stage = ring + (size_t)(c % kDfStages) * kDfChunk * d.S;
        const int per = min(kDfChunk, d.P - c * kDfChunk);
        for (int pl = 0; pl < per; ++pl) {
            float2 t[HW + 1];
#pragma unroll
            for (int k = 0; k <= HW; ++k) t[k] = stp[idx[k]];
            if (act) {
                const float4 v4 = reinterpret_cast<const float4 *>(stage + (size_t)pl * d.S)[lane];
                const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int k = 0; k <= HW; ++k) ac[i][k] = fmaf(v[i], t[k].x, ac[i][k]);
#pragma unroll
                    for (int k = 1; k <= HW; ++k) as[i][k] = fmaf(v[i], t[k].y, as[i][k]);
                }
            }
#pragma unroll
            for (int k = 1; k <= HW; ++k) {
                idx[k] += k;
                if (idx[k] >= d.P) idx[k] -= d.P;
            }
        }
        __syncwarp();
        if (lane == 0 && c + kDfStages < nchunk) {
            ptx::fence_proxy_async_smem();  // the warp's reads of the stage, then its refill
            issue(c + kDfStages);
        }
    }
    if (!good) {
        if (lane == 0) atomicExch(err, 1);
        return;
    }
    __syncwarp();
    // the warp's ring now holds sT[r][W] (complex), then the synthesis over phases
    float2 *sT = reinterpret_cast<float2 *>(ring);
    if (act) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * lane + i;
#pragma unroll
            for (int k = -HW; k <= HW; ++k) {
                const int a = k < 0 ? -k : k;
                sT[r * W + (k + HW)] = make_float2(ac[i][a], k < 0 ? -as[i][a] : as[i][a]);
            }
        }
    }
    __syncwarp();
    for (int o = lane; o < d.nb; o += 32) {
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

size_t dft_stream_smem(const Dims &d) {
    return sizeof(float) * (size_t)kDfWarps * kDfStages * kDfChunk * d.S + sizeof(float2) * d.P +
           sizeof(uint64_t) * kDfWarps * kDfStages;
}

// The streaming form takes S % 4 == 0, S <= 128, a signal whose segments start on 16
// bytes, and a ring that can hold the S x W synthesis inputs afterwards.
bool dft_stream_ok(const Dims &d, const float *sig) {
    return d.S % 4 == 0 && d.S <= 128 && d.L % 4 == 0 && (reinterpret_cast<uintptr_t>(sig) & 15) == 0 &&
           (size_t)d.S * d.W * 2 <= (size_t)kDfStages * kDfChunk * d.S && dft_stream_smem(d) <= 227 * 1024;
}

template <int HW>
static void dft_fwd_stream_hw(const float *sig, const float2 *twp, const float2 *tw2_ro, const float2 *dgam,
                              float *data, const Dims &d, int *err, cudaStream_t st) {
    const size_t smem = dft_stream_smem(d);
    cudaFuncSetAttribute(k_dft_fwd_stream<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_dft_fwd_stream<HW><<<(d.nseg + kDfWarps - 1) / kDfWarps, 32 * kDfWarps, smem, st>>>(
        sig, twp, tw2_ro, dgam, data, d, (float)(1.0 / sqrt((double)d.L)), err);
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

// Streaming transpose (S % 4 == 0, S <= 128): a warp owns one segment and lane l the
// phases 4l..4l+3. Each lane forms its phases' coefficients A_d, B_d as the
// one-phase-per-thread form does, then writes the segment period by period with one
// 16-byte store (four phases) per lane: 512 contiguous bytes per warp and period. The
// period twiddles come from the e^{2 pi i q / P} table at q = d p mod P (the same values).
template <int HW>
__global__ void __launch_bounds__(32 * kDfWarps) k_dft_adj_stream(const float *__restrict__ data,
                                                                  const float2 *__restrict__ twp,
                                                                  const float2 *__restrict__ tw2_qr,
                                                                  const float2 *__restrict__ dgam,
                                                                  float *__restrict__ sig, Dims d,
                                                                  float inv_sqrt_l) {
    constexpr int W = 2 * HW + 1;
    extern __shared__ __align__(16) float da_sm[];
    float2 *stp = reinterpret_cast<float2 *>(da_sm);  // [P]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *sy = stp + d.P + (size_t)warp * d.nb;     // this warp's conj(D) y / sqrt(L)
    for (int i = threadIdx.x; i < d.P; i += blockDim.x) stp[i] = twp[i];
    const int seg = blockIdx.x * kDfWarps + warp;
    if (seg < d.nseg)
        for (int o = lane; o < d.nb; o += 32) {
            const float2 y = ((const float2 *)data)[(size_t)seg * d.nb + o];
            const float2 g = dgam[o];
            sy[o] = make_float2((g.x * y.x + g.y * y.y) * inv_sqrt_l, (g.x * y.y - g.y * y.x) * inv_sqrt_l);
        }
    __syncthreads();
    if (seg >= d.nseg || lane >= d.S / 4) return;
    float A[4][HW + 1], B[4][HW + 1];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 4 * lane + i;
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
        A[i][0] = ur[HW];
        B[i][0] = 0.f;
#pragma unroll
        for (int k = 1; k <= HW; ++k) {
            A[i][k] = ur[HW + k] + ur[HW - k];
            B[i][k] = ui[HW + k] - ui[HW - k];
        }
    }
    float4 *out = reinterpret_cast<float4 *>(sig + (size_t)seg * d.L) + lane;
    int idx[HW + 1];  // d p mod P
#pragma unroll
    for (int k = 0; k <= HW; ++k) idx[k] = 0;
    const int q4 = d.S / 4;
    for (int p = 0; p < d.P; ++p) {
        float2 t[HW + 1];
#pragma unroll
        for (int k = 0; k <= HW; ++k) t[k] = stp[idx[k]];
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= HW; ++k) acc = fmaf(A[i][k], t[k].x, acc);
#pragma unroll
            for (int k = 1; k <= HW; ++k) acc = fmaf(B[i][k], t[k].y, acc);
            v[i] = acc;
        }
        __stcs(out + (size_t)p * q4, make_float4(v[0], v[1], v[2], v[3]));  // written once, read once
#pragma unroll
        for (int k = 1; k <= HW; ++k) {
            idx[k] += k;
            if (idx[k] >= d.P) idx[k] -= d.P;
        }
    }
}

template <int HW>
static void dft_adj_stream_hw(const float *data, const float2 *twp, const float2 *tw2_qr, const float2 *dgam,
                              float *sig, const Dims &d, cudaStream_t st) {
    const size_t smem = sizeof(float2) * ((size_t)d.P + (size_t)kDfWarps * d.nb);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_dft_adj_stream<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    k_dft_adj_stream<HW><<<(d.nseg + kDfWarps - 1) / kDfWarps, 32 * kDfWarps, smem, st>>>(
        data, twp, tw2_qr, dgam, sig, d, (float)(1.0 / sqrt((double)d.L)));
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

void launch_dft_fwd(const float *sig, const float *tw1, const float2 *twp, const float2 *tw2_ro, const float2 *dgam,
                    float *data, const Dims &d, int *err, cudaStream_t st) {
    if (twp && err && dft_stream_ok(d, sig)) {
        MPIFFL_HW_DISPATCH(dft_fwd_stream_hw, sig, twp, tw2_ro, dgam, data, d, err, st);
        return;
    }
    MPIFFL_HW_DISPATCH(dft_fwd_hw, sig, tw1, tw2_ro, dgam, data, d, st);
}

void launch_dft_adj(const float *data, const float *tw1, const float2 *twp, const float2 *tw2_qr, const float2 *dgam,
                    float *sig, const Dims &d, cudaStream_t st) {
    if (twp && d.S % 4 == 0 && d.S <= 128 && d.L % 4 == 0 && (reinterpret_cast<uintptr_t>(sig) & 15) == 0 &&
        sizeof(float2) * ((size_t)d.P + (size_t)kDfWarps * d.nb) <= 200 * 1024) {
        MPIFFL_HW_DISPATCH(dft_adj_stream_hw, data, twp, tw2_qr, dgam, sig, d, st);
        return;
    }
    MPIFFL_HW_DISPATCH(dft_adj_hw, data, tw1, tw2_qr, dgam, sig, d, st);
}

}  // namespace mpiffl
