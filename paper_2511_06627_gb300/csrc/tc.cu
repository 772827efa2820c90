// Tensor-core path of the line stages (tcgen05, sm_103a).
//
// Forward, one block per job of up to kTcMaxSeg raster lines that share a
// trajectory: E V B is evaluated on the fly from the lines' PSF-convolved rows
// (held in shared memory) and fed straight into the band DFT, so the 4-byte-per-
// sample time signal never reaches HBM. The DFT is factorised over the period
// structure j = p S + r (Eq. (27) on the kept bins, unchanged):
//     T[r, c] = sum_p s[p S + r] Tw[p, c]          (tensor cores, K = P)
//     b[k, d] = L^-1/2 D_kd sum_r T[r, d] e^{2 pi i (kP+d) r / L}   (CUDA cores)
// where column c of Tw is cos(2 pi d p / P) (c = d = 0..w) or sin(2 pi d p / P)
// (c = w + d, d = 1..w). A row of the MMA is one (line, r) pair (128 / S lines per
// 128-row tile); A = samples (K-major, periods along K), B = Tw.
//
// Adjoint: the transposed chain. Per line, U[r, d] = sum_k conj(D) y e^{-2 pi i (kP+d) r/L}
// (CUDA cores) folds into W real coefficients per r; the time signal of a chunk of
// 128 periods is then one MMA, s[p, (line, r)] = sum_c Tw[p, c] C[(line, r), c],
// read back from TMEM and scattered into the lines' fine rows (shared-memory
// float atomics), which are finally scaled by the gain and written out.
//
// Products are split into bf16 hi + lo parts and accumulated in FP32 as
// hi*hi + hi*lo + lo*hi (PREC_BF16X3), or taken once in TF32 (PREC_TF32).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc.h"
#include "tc_ptx.cuh"

namespace mpiffl {

namespace {

constexpr int kTcMaxSeg = 8;       // lines per job
constexpr int kFwdThreads = 512;   // 4 threads per MMA row
constexpr int kAdjThreads = 512;   // 4 TMEM lane quadrants x 4 period groups
constexpr int kAdjChunk = 128;     // periods per adjoint MMA (M)
constexpr uint32_t kWaitLimit = 1u << 24;

struct TcJob {
    int parity;
    int nseg;
    int seg[kTcMaxSeg];
};

struct TcCfg {
    int G;          // 128-row tiles per forward job
    int spt;        // lines per tile (128 / S)
    int Kc;         // periods per forward pipeline stage
    int ne_pad;     // fine-row stride (floats) in the forward
    int ne_adj;     // padded fine-row length in the adjoint (one pad word per 32)
    int nseg_adj;   // lines per adjoint job
    int ncols_adj;  // MMA N of the adjoint = nseg_adj * S
    uint32_t tmem_fwd, tmem_adj;
    // forward shared-memory carve-up (bytes)
    uint32_t f_fine, f_B, f_A, f_tw, f_T, f_bar, f_total;
    // adjoint carve-up
    uint32_t a_fine, a_A, a_B, a_tw, a_y, a_coef, a_win, a_bar, a_total;
    int win_len;    // floats per warp window in the adjoint
    int wide_step;  // cells of one r move by >= 2 per period: n and n+1 updates never collide
    uint32_t a_vr;
    int prec;
};

struct TcState {
    TcCfg cfg{};
    TcJob *jobs_fwd = nullptr, *jobs_adj = nullptr;
    int n_fwd = 0, n_adj = 0;
    uint8_t *twB = nullptr;   // forward B operand (hi, lo)
    uint8_t *twA = nullptr;   // adjoint A operand (hi, lo)
    float2 *tw2 = nullptr;    // [S] e^{2 pi i m / S}, then [W][S] e^{2 pi i d r / L}
    int *err = nullptr;
    int *wbase = nullptr;   // adjoint window base cell per (trajectory, 32-period block)
    int n_sm = 1;
    bool ok = false;
    bool oom = false;  // the shape is supported but a device allocation failed
};

__host__ __device__ inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// byte offset of element (row, k) of a bf16 K-major canonical tile
__host__ __device__ inline uint32_t canon_off(uint32_t row, uint32_t k, uint32_t sbo) {
    return (row / 8) * sbo + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ TrajEntry load_te(const TrajEntry *p) {
    TrajEntry t;
    t.n = __ldg(&p->n);
    t.w0 = __ldg(&p->w0);
    t.w1 = __ldg(&p->w1);
    return t;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    float h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        h[u] = __bfloat162float(__float2bfloat16_rn(v[u]));
        l[u] = v[u] - h[u];
    }
    hi = make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
    lo = make_uint4(pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]), pack_bf16(l[4], l[5]), pack_bf16(l[6], l[7]));
}

// ============================================================================ forward

// bf16 hi/lo split of 8 floats, two at a time: hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void split8x2(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h2 = __float22bfloat162_rn(make_float2(v[2 * i], v[2 * i + 1]));
        const uint32_t hb = *reinterpret_cast<uint32_t *>(&h2);
        const float h0 = __uint_as_float(hb << 16), h1 = __uint_as_float(hb & 0xFFFF0000u);
        __nv_bfloat162 l2 = __float22bfloat162_rn(make_float2(v[2 * i] - h0, v[2 * i + 1] - h1));
        h[i] = hb;
        l[i] = *reinterpret_cast<uint32_t *>(&l2);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Persistent: each block loops over jobs. Warps 0..15 produce the A operand (row =
// tid % 128 of the MMA tile, part = tid / 128 selects the 8-period groups of a stage)
// and run the epilogue; warp 16 only issues the MMAs. Stage handoff uses mbarriers:
// full[st] (one arrival per producer warp) and empty[st] (MMA completion), so
// producers never wait for the MMA issue. Fine rows are staged as c[n] and
// c[n+1] - c[n], so a sample is s = g v (c[n] + f (c[n+1] - c[n])).
__global__ void __launch_bounds__(kFwdThreads + 32, 1)
    k_tc_fwd(const float *__restrict__ fine, const int2 *__restrict__ tnf, const float *__restrict__ vr,
             const float *__restrict__ gain, const TcJob *__restrict__ jobs, int njobs,
             const uint8_t *__restrict__ twB, const float2 *__restrict__ tw2, const float2 *__restrict__ dgam,
             float *__restrict__ data, Dims d, TcCfg c, int *err) {
    extern __shared__ __align__(128) uint8_t sm[];
    float *sf0 = reinterpret_cast<float *>(sm + c.f_fine);
    float *sf1 = sf0 + c.G * c.spt * c.ne_pad;
    uint8_t *sB = sm + c.f_B;
    uint8_t *sA = sm + c.f_A;
    float2 *stw = reinterpret_cast<float2 *>(sm + c.f_tw);
    float *sT = reinterpret_cast<float *>(sm + c.f_T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + c.f_bar);  // full[2], empty[2], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + c.f_bar + 48);
    int *sflag = reinterpret_cast<int *>(sm + c.f_bar + 52);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = d.S;
    const int nsegc = c.G * c.spt;
    const int nprod_warps = kFwdThreads / 32;
    const bool mma_warp = warp == nprod_warps;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(&bars[i], nprod_warps);  // full
            ptx::mbar_init(&bars[2 + i], 1);        // empty
        }
        ptx::mbar_init(&bars[4], 1);                // done
        ptx::fence_mbar_init();
        *sflag = 0;
    }
    if (warp == 0) {
        ptx::tmem_alloc(tslot, c.tmem_fwd);
        ptx::tmem_relinquish();
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(twB);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        const int n16 = (64 * d.P) / 16;
        for (int i = tid; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
        for (int i = tid; i < S + d.W * S; i += blockDim.x) stw[i] = __ldg(tw2 + i);
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;
    const int nchunks = d.P / c.Kc;
    const uint32_t tileA = 128u * c.Kc * 2u;
    const uint32_t stageA = tileA * 2u * c.G;
    const uint32_t sboA = (c.Kc / 8) * 128u;

    if (mma_warp) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t sboB = (d.P / 8) * 128u;
            const uint32_t halfB = 32u * d.P;
            const uint32_t idesc = ptx::instr_desc(1, 128, 16);
            uint32_t it = 0;
            bool ok = true;
            for (int jb = blockIdx.x; jb < njobs && ok; jb += gridDim.x) {
                for (int q = 0; q < nchunks; ++q, ++it) {
                    const int st = it & 1;
                    if (!ptx::mbar_wait_bounded(&bars[st], (it >> 1) & 1, kWaitLimit)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint8_t *A = sA + st * stageA;
                    for (int g = 0; g < c.G; ++g) {
                        const uint32_t ahi = ptx::smem_u32(A + (2 * g) * tileA);
                        const uint32_t alo = ptx::smem_u32(A + (2 * g + 1) * tileA);
                        for (int ks = 0; ks < c.Kc / 16; ++ks) {
                            const uint32_t kg = q * c.Kc + ks * 16;
                            const uint64_t dAh = ptx::smem_desc(ahi + ks * 256, 128, sboA);
                            const uint64_t dAl = ptx::smem_desc(alo + ks * 256, 128, sboA);
                            const uint64_t dBh = ptx::smem_desc(ptx::smem_u32(sB) + (kg / 8) * 128, 128, sboB);
                            const uint64_t dBl = ptx::smem_desc(ptx::smem_u32(sB) + halfB + (kg / 8) * 128, 128, sboB);
                            const uint32_t dt = tmem + g * 16;
                            ptx::mma_bf16(dt, dAh, dBh, idesc, (q > 0 || ks > 0) ? 1u : 0u);
                            if (c.prec == MPI_FFL_PREC_BF16X3) {
                                ptx::mma_bf16(dt, dAh, dBl, idesc, 1u);
                                ptx::mma_bf16(dt, dAl, dBh, idesc, 1u);
                            }
                        }
                    }
                    ptx::mma_commit(&bars[2 + st]);
                    if (q == nchunks - 1) ptx::mma_commit(&bars[4]);
                }
            }
            if (!ok) atomicExch(sflag, 1);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- producers + epilogue
        const int row = tid & 127, part = tid >> 7, nparts = kFwdThreads / 128;
        const int sg = row / S, r = row % S;
        const float inv_sqrt_l = rsqrtf((float)d.L);
        uint32_t it = 0, njob_done = 0;
        bool good = true;
        for (int jb = blockIdx.x; jb < njobs && good; jb += gridDim.x, ++njob_done) {
            const TcJob job = jobs[jb];
            for (int sl = 0; sl < nsegc; ++sl) {
                float *d0 = sf0 + sl * c.ne_pad, *d1 = sf1 + sl * c.ne_pad;
                if (sl < job.nseg) {
                    const float *src = fine + (size_t)job.seg[sl] * d.Ne;
                    for (int e = tid; e < d.Ne - 1; e += kFwdThreads) {
                        const float c0 = __ldg(src + e), c1 = __ldg(src + e + 1);
                        d0[e] = c0;
                        d1[e] = c1 - c0;
                    }
                } else {
                    for (int e = tid; e < d.Ne - 1; e += kFwdThreads) d0[e] = d1[e] = 0.f;
                }
            }
            ptx::named_sync(1, kFwdThreads);
            const int2 *tr = tnf + (size_t)job.parity * d.L;
            const float vrow = __ldg(vr + job.parity * S + r);
            int foff[2];
            float gl[2];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const int sl = g * c.spt + sg;
                foff[g] = (g < c.G ? sl : 0) * c.ne_pad;
                gl[g] = (g < c.G && sl < job.nseg) ? __ldg(gain + job.seg[sl] / d.Nz) * vrow : 0.f;
            }
            for (int q = 0; q < nchunks; ++q, ++it) {
                const int st = it & 1;
                if (it >= 2 && !ptx::mbar_wait_bounded(&bars[2 + st], ((it - 2) >> 1) & 1, kWaitLimit)) {
                    good = false;
                    break;
                }
                uint8_t *A = sA + st * stageA;
                for (int p8 = part; p8 < c.Kc / 8; p8 += nparts) {
                    int n8[8];
                    float f8[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int2 e = __ldg(tr + (size_t)(q * c.Kc + p8 * 8 + u) * S + r);
                        n8[u] = e.x;
                        f8[u] = __int_as_float(e.y);
                    }
                    const uint32_t off = (row / 8) * sboA + p8 * 128 + (row % 8) * 16;
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        if (g >= c.G) break;
                        float v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int ix = foff[g] + n8[u];
                            v[u] = gl[g] * fmaf(f8[u], sf1[ix], sf0[ix]);
                        }
                        uint4 hi, lo;
                        split8x2(v, hi, lo);
                        *reinterpret_cast<uint4 *>(A + (2 * g) * tileA + off) = hi;
                        *reinterpret_cast<uint4 *>(A + (2 * g + 1) * tileA + off) = lo;
                    }
                }
                ptx::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&bars[st]);
            }
            if (!good) break;
            if (!ptx::mbar_wait_bounded(&bars[4], njob_done & 1, kWaitLimit)) {
                good = false;
                break;
            }
            ptx::tc_fence_after();
            if (warp < 4) {
                for (int g = 0; g < c.G; ++g) {
                    float v[16];
                    ptx::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + g * 16, v);
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc)
                        if (cc < d.W) sT[(g * 128 + tid) * d.W + cc] = v[cc];
                }
            }
            ptx::tc_fence_before();
            ptx::named_sync(1, kFwdThreads);
            // b[k, d] = D L^-1/2 sum_r T[r, d] e^{2 pi i k r / S} e^{2 pi i d r / L}; the sum over
            // r is split over the 4 adjacent lanes of a task and added with shuffles
            const int quarter = tid & 3, rq = S / 4;
            const int ntask = job.nseg * d.nb;
            for (int t0 = 0; t0 < ntask; t0 += kFwdThreads / 4) {
                const int task = t0 + (tid >> 2);
                const bool act = task < ntask;
                const int tk = act ? task : 0;
                const int sl = tk / d.nb, o = tk % d.nb;
                const int di = o % d.W, dl = di - d.hw, ad = dl < 0 ? -dl : dl;
                const int kmod = (d.kmin + o / d.W) % S;
                const float sgn = dl < 0 ? -1.f : 1.f;
                const float *rowT = sT + ((sl / c.spt) * 128 + (sl % c.spt) * S) * d.W;
                const float2 *twd = stw + S + di * S;
                float re = 0.f, im = 0.f;
                const int r0 = quarter * rq;
                int idx = (kmod * r0) % S;
                for (int rr = r0; rr < r0 + rq; ++rr) {
                    const float tre = rowT[rr * d.W + ad];
                    const float tim = ad == 0 ? 0.f : sgn * rowT[rr * d.W + d.hw + ad];
                    const float2 a = stw[idx], b = twd[rr];
                    const float wr = a.x * b.x - a.y * b.y, wi = a.x * b.y + a.y * b.x;
                    re = fmaf(tre, wr, fmaf(-tim, wi, re));
                    im = fmaf(tre, wi, fmaf(tim, wr, im));
                    idx += kmod;
                    if (idx >= S) idx -= S;
                }
                re += __shfl_xor_sync(0xffffffffu, re, 1);
                im += __shfl_xor_sync(0xffffffffu, im, 1);
                re += __shfl_xor_sync(0xffffffffu, re, 2);
                im += __shfl_xor_sync(0xffffffffu, im, 2);
                if (act && quarter == 0) {
                    re *= inv_sqrt_l;
                    im *= inv_sqrt_l;
                    const float2 gd = __ldg(dgam + o);
                    reinterpret_cast<float2 *>(data)[(size_t)job.seg[sl] * d.nb + o] =
                        make_float2(gd.x * re - gd.y * im, gd.x * im + gd.y * re);
                }
            }
            ptx::named_sync(1, kFwdThreads);  // sT and the fine rows are reused by the next job
        }
        if (!good) atomicExch(sflag, 1);
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *sflag) atomicExch(err, 1);
    if (warp == 0) ptx::tmem_dealloc(tmem, c.tmem_fwd);
}

// ============================================================================ adjoint

// Persistent. The MMA gives D[p][(line, r)] for a chunk of 128 periods, TMEM lane = p.
// Warp w reads lanes 32 (w % 4)..+31 (32 consecutive periods) and 64 columns
// (64 r of one line). At a fixed r the fine-grid cell of a sample is strictly
// monotone in p (checked on the host), so the 32 lanes of one update touch 32
// distinct cells: every warp accumulates into its own window of the fine row with
// plain shared-memory read-modify-writes, and the windows are then added into the
// line accumulators by cell, in a fixed order (no atomics, deterministic).
__global__ void __launch_bounds__(kAdjThreads, 1)
    k_tc_adj(const float *__restrict__ data, const int2 *__restrict__ tnf, const float *__restrict__ vr,
             const float *__restrict__ gain, const TcJob *__restrict__ jobs, int njobs,
             const uint8_t *__restrict__ twA, const float2 *__restrict__ tw2, const float2 *__restrict__ dgam,
             const int *__restrict__ wbase, float *__restrict__ fine, Dims d, TcCfg c, int *err) {
    extern __shared__ __align__(128) uint8_t sm[];
    float *sacc = reinterpret_cast<float *>(sm + c.a_fine);
    uint8_t *sTw = sm + c.a_A;   // Tw: rows p, K = 16 (hi, lo) -- the MMA's A operand
    uint8_t *sC = sm + c.a_B;    // coefficients: rows (line, r), K = 16 (hi, lo) -- the B operand
    float2 *stw = reinterpret_cast<float2 *>(sm + c.a_tw);
    float2 *sy = reinterpret_cast<float2 *>(sm + c.a_y);
    float *scoef = reinterpret_cast<float *>(sm + c.a_coef);
    float *swin = reinterpret_cast<float *>(sm + c.a_win);
    float *svr = reinterpret_cast<float *>(sm + c.a_vr);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + c.a_bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + c.a_bar + 16);
    int *sbase = reinterpret_cast<int *>(sm + c.a_bar + 32);  // window bases of the current chunk
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = d.S;
    const int nsegc = c.nseg_adj;
    const int ncols = nsegc * S;  // 256
    const int quad = warp & 3, cgrp = warp >> 2;  // period quadrant, 64-column group
    const int col0 = cgrp * 64;
    const int wline = col0 / S;                   // line of this warp's columns
    const int wstride = c.win_len + (c.win_len >> 5);  // windows are stored with one pad word per 32
    float *win = swin + warp * wstride;
    const int nwin_per_line = 4 * (S / 64);       // warps sharing a line

    if (tid == 0) {
        ptx::mbar_init(&bars[0], 1);
        ptx::mbar_init(&bars[1], 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(tslot, c.tmem_adj);
        ptx::tmem_relinquish();
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(twA);
        uint4 *dst = reinterpret_cast<uint4 *>(sTw);
        const int n16 = (64 * d.P) / 16;
        for (int i = tid; i < n16; i += kAdjThreads) dst[i] = __ldg(src + i);
        for (int i = tid; i < S + d.W * S; i += kAdjThreads) stw[i] = __ldg(tw2 + i);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = ptx::instr_desc(1, 128, (uint32_t)ncols);
    const uint32_t halfTw = 32u * d.P;
    const uint32_t halfC = (uint32_t)ncols * 32u;
    const int nchunks = d.P / kAdjChunk;
    const float inv_sqrt_l = rsqrtf((float)d.L);
    uint32_t it = 0;  // MMA batches committed by this block
    bool good = true;

    auto issue = [&](int q, int buf) {  // D[buf] = Tw(chunk q) x C^T
        ptx::tc_fence_after();
        const uint32_t a0 = ptx::smem_u32(sTw) + q * (kAdjChunk * 16 * 2);
        const uint64_t dAh = ptx::smem_desc(a0, 128, 256);
        const uint64_t dAl = ptx::smem_desc(a0 + halfTw, 128, 256);
        const uint64_t dBh = ptx::smem_desc(ptx::smem_u32(sC), 128, 256);
        const uint64_t dBl = ptx::smem_desc(ptx::smem_u32(sC) + halfC, 128, 256);
        const uint32_t dt = tmem + (uint32_t)(buf * ncols);
        ptx::mma_bf16(dt, dAh, dBh, idesc, 0u);
        if (c.prec == MPI_FFL_PREC_BF16X3) {
            ptx::mma_bf16(dt, dAh, dBl, idesc, 1u);
            ptx::mma_bf16(dt, dAl, dBh, idesc, 1u);
        }
        ptx::mma_commit(&bars[buf]);
    };

    for (int jb = blockIdx.x; jb < njobs && good; jb += gridDim.x) {
        const TcJob job = jobs[jb];
        for (int i = tid; i < nsegc * d.Ne; i += kAdjThreads) sacc[i] = 0.f;
        for (int i = tid; i < nsegc * d.nb; i += kAdjThreads) {
            const int sl = i / d.nb, o = i % d.nb;
            float2 y = make_float2(0.f, 0.f);
            if (sl < job.nseg) {
                const float2 v = reinterpret_cast<const float2 *>(data)[(size_t)job.seg[sl] * d.nb + o];
                const float2 g = __ldg(dgam + o);
                y = make_float2((g.x * v.x + g.y * v.y) * inv_sqrt_l, (g.x * v.y - g.y * v.x) * inv_sqrt_l);
            }
            sy[i] = y;
        }
        __syncthreads();
        // coefficients of column (line, r): U[d] = sum_k y'[k,d] e^{-2 pi i (kP+d) r / L};
        // c_0 = Re U[0], c_d = Re U[d] + Re U[-d], c_{w+d} = Im U[d] - Im U[-d]
        for (int n = tid; n < ncols; n += kAdjThreads) {
            const int sl = n / S, rr = n % S;
            float *cf = scoef + n * 16;
            for (int cc = 0; cc < 16; ++cc) cf[cc] = 0.f;
            const float2 *yl = sy + sl * d.nb;
            for (int a = 0; a <= d.hw; ++a) {
                float ur_p = 0.f, ui_p = 0.f, ur_m = 0.f, ui_m = 0.f;
                const float2 bp = stw[S + (d.hw + a) * S + rr], bm = stw[S + (d.hw - a) * S + rr];
                for (int k = 0; k < d.K; ++k) {
                    const float2 e = stw[((d.kmin + k) % S) * rr % S];
                    const float wpr = e.x * bp.x - e.y * bp.y, wpi = e.x * bp.y + e.y * bp.x;
                    const float wmr = e.x * bm.x - e.y * bm.y, wmi = e.x * bm.y + e.y * bm.x;
                    const float2 yp = yl[k * d.W + d.hw + a], ym = yl[k * d.W + d.hw - a];
                    ur_p = fmaf(yp.x, wpr, fmaf(yp.y, wpi, ur_p));
                    ui_p = fmaf(yp.y, wpr, fmaf(-yp.x, wpi, ui_p));
                    ur_m = fmaf(ym.x, wmr, fmaf(ym.y, wmi, ur_m));
                    ui_m = fmaf(ym.y, wmr, fmaf(-ym.x, wmi, ui_m));
                }
                if (a == 0) {
                    cf[0] = ur_p;
                } else {
                    cf[a] = ur_p + ur_m;
                    cf[d.hw + a] = ui_p - ui_m;
                }
            }
            for (int h = 0; h < 2; ++h) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = cf[h * 8 + u];
                uint4 hi4, lo4;
                split8x2(v, hi4, lo4);
                const uint32_t off = canon_off(n, h * 8, 256);
                *reinterpret_cast<uint4 *>(sC + off) = hi4;
                *reinterpret_cast<uint4 *>(sC + halfC + off) = lo4;
            }
        }
        ptx::fence_proxy_async_smem();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            issue(0, it & 1);
            if (nchunks > 1) issue(1, (it + 1) & 1);
        }
        const int2 *tr = tnf + (size_t)job.parity * d.L;
        const int *wb = wbase + job.parity * (d.P / 32);
        for (int i = tid; i < S; i += kAdjThreads) svr[i] = __ldg(vr + job.parity * S + i);
        for (int q = 0; q < nchunks; ++q) {
            const uint32_t b = (it + q) & 1;
            for (int i = lane; i < wstride; i += 32) win[i] = 0.f;
            if (tid < 4) sbase[tid] = __ldg(wb + q * 4 + tid);
            const int p = q * kAdjChunk + quad * 32 + lane;  // this lane's period
            const int base = __ldg(wb + q * 4 + quad);
            const bool w = ptx::mbar_wait_bounded(&bars[b], ((it + q) >> 1) & 1, kWaitLimit);
            good = __syncthreads_and(w);
            if (!good) break;
            ptx::tc_fence_after();
            for (int cb = 0; cb < 64; cb += 16) {
                const int rr0 = (col0 + cb) % S;
                const int4 *te = reinterpret_cast<const int4 *>(tr + (size_t)p * S + rr0);
                int n16[16];
                float f16[16];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int4 e = __ldg(te + u);
                    n16[2 * u] = e.x - base;
                    f16[2 * u] = __int_as_float(e.y);
                    n16[2 * u + 1] = e.z - base;
                    f16[2 * u + 1] = __int_as_float(e.w);
                }
                float v[16];
                ptx::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * ncols + col0 + cb), v);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float vs = svr[rr0 + u] * v[u];
                    const float hv = f16[u] * vs;  // f v s -> cell n + 1
                    const int i0 = n16[u] + (n16[u] >> 5), i1 = (n16[u] + 1) + ((n16[u] + 1) >> 5);
                    win[i0] += vs - hv;            // (1 - f) v s -> cell n
                    if (!c.wide_step) __syncwarp();
                    win[i1] += hv;
                    __syncwarp();
                }
            }
            ptx::tc_fence_before();
            __syncthreads();
            if (tid == 0 && q + 2 < nchunks) issue(q + 2, b);
            // add the windows into the line accumulators, cell by cell, warps in order
            for (int i = tid; i < nsegc * d.Ne; i += kAdjThreads) {
                const int sl = i / d.Ne, e = i % d.Ne;
                float add = 0.f;
                for (int k = 0; k < nwin_per_line; ++k) {
                    // warps of line sl: column groups cg with cg*64/S == sl, all 4 quadrants
                    const int cg = sl * (S / 64) + k / 4, qd = k % 4;
                    const int off = e - sbase[qd];
                    if (off >= 0 && off < c.win_len) add += swin[(cg * 4 + qd) * wstride + off + (off >> 5)];
                }
                sacc[i] += add;
            }
            __syncthreads();
        }
        if (!good) break;
        it += nchunks;
        for (int sl = 0; sl < job.nseg; ++sl) {
            const float g = __ldg(gain + job.seg[sl] / d.Nz);
            float *dst = fine + (size_t)job.seg[sl] * d.Ne;
            const float *acc = sacc + sl * d.Ne;
            for (int e = tid; e < d.Ne; e += kAdjThreads) dst[e] = g * acc[e];
        }
        __syncthreads();
    }
    if (!good && tid == 0) atomicExch(err, 1);
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, c.tmem_adj);
}

// ============================================================================ host

TcState *state(const mpi_ffl_handle *h) { return reinterpret_cast<TcState *>(h->tc_state); }

uint32_t pow2_cols(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

bool plan(const Dims &d, TcCfg &c, int win_len) {
    if (d.S > 128 || 128 % d.S != 0 || d.S % 64 != 0) return false;  // S in {64, 128}
    if (d.W > 16) return false;                                      // twiddle columns fit N = 16
    if (d.P % kAdjChunk != 0) return false;                          // adjoint period chunks
    c.spt = 128 / d.S;
    c.Kc = 64;
    c.G = 2;  // 128-row tiles per forward job
    if (c.spt * c.G > kTcMaxSeg) return false;
    c.ne_pad = (d.Ne + 3) / 4 * 4;
    c.tmem_fwd = pow2_cols(c.G * 16);
    uint32_t o = 0;
    c.f_fine = o;
    o = align_up(o + 8u * c.ne_pad * c.G * c.spt, 128);  // c[n] and c[n+1]-c[n] arrays
    c.f_B = o;
    o = align_up(o + 64u * d.P, 128);
    c.f_A = o;
    o = align_up(o + 2u * 2u * c.G * 128u * c.Kc * 2u, 128);
    c.f_tw = o;
    o = align_up(o + 8u * (d.S + d.W * d.S), 128);
    c.f_T = o;
    o = align_up(o + 4u * c.G * 128u * d.W, 128);
    c.f_bar = o;
    c.f_total = o + 64;
    // adjoint: 256 MMA columns (line, r), two D buffers
    c.nseg_adj = 256 / d.S;
    c.ncols_adj = c.nseg_adj * d.S;
    c.tmem_adj = pow2_cols(2 * c.ncols_adj);
    if (c.tmem_adj > 512) return false;
    c.win_len = win_len;
    o = 0;
    c.a_fine = o;
    o = align_up(o + 4u * d.Ne * c.nseg_adj, 128);
    c.a_A = o;
    o = align_up(o + 64u * d.P, 128);
    c.a_B = o;
    o = align_up(o + 64u * c.ncols_adj, 128);
    c.a_tw = o;
    o = align_up(o + 8u * (d.S + d.W * d.S), 128);
    c.a_y = o;
    o = align_up(o + 8u * c.nseg_adj * d.nb, 128);
    c.a_coef = o;
    o = align_up(o + 4u * 16u * c.ncols_adj, 128);
    c.a_win = o;
    o = align_up(o + 4u * (uint32_t)(win_len + (win_len >> 5)) * (kAdjThreads / 32), 128);
    c.a_vr = o;
    o = align_up(o + 4u * d.S, 128);
    c.a_bar = o;
    c.a_total = o + 64;
    return c.f_total <= 227 * 1024 && c.a_total <= 227 * 1024;
}

template <class T>
void upload_vec(T **p, const std::vector<T> &v) {
    if (dev_malloc((void **)p, v.size() * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        return;
    }
    cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

uint16_t bf16_bits(float f) {
    // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + rounding) >> 16);
}
float bf16_to_float(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

bool tc_supported(const mpi_ffl_handle *h) {
    const TcState *s = state(h);
    return s && s->ok;
}

void tc_init(mpi_ffl_handle *h) {
    TcState *s = new TcState();
    h->tc_state = s;
    const Dims &d = h->d;
    // adjoint windows: per trajectory and block of 32 periods, the smallest fine cell
    // touched (any r); the window must hold every cell of the block, and the cell of
    // a fixed r must move strictly monotonically with the period (distinct lanes)
    const std::vector<int> &tn = h->traj_n;
    if ((int64_t)tn.size() != (int64_t)d.n_par * d.L || d.P % 32 != 0) return;
    std::vector<int> wb((size_t)d.n_par * (d.P / 32));
    int span = 0, min_step = 1 << 30;
    bool monotone = true;
    for (int par = 0; par < d.n_par; ++par) {
        const int *n = tn.data() + (size_t)par * d.L;
        for (int b = 0; b < d.P / 32; ++b) {
            int lo = 1 << 30, hi = -1;
            for (int p = 32 * b; p < 32 * b + 32; ++p)
                for (int r = 0; r < d.S; ++r) {
                    lo = std::min(lo, n[(size_t)p * d.S + r]);
                    hi = std::max(hi, n[(size_t)p * d.S + r]);
                }
            wb[(size_t)par * (d.P / 32) + b] = lo;
            span = std::max(span, hi + 2 - lo);
        }
        for (int r = 0; r < d.S && monotone; ++r) {
            const int dir = n[(size_t)d.S + r] - n[r];
            for (int p = 0; p + 1 < d.P; ++p) {
                const int st = n[(size_t)(p + 1) * d.S + r] - n[(size_t)p * d.S + r];
                min_step = std::min(min_step, st < 0 ? -st : st);
                if (st == 0 || (st > 0) != (dir > 0)) {
                    monotone = false;
                    break;
                }
            }
        }
    }
    const int win_len = (span + 31) / 32 * 32;
    if (!monotone || win_len > 2048) return;
    if (!plan(d, s->cfg, win_len)) return;
    TcCfg &c = s->cfg;
    c.wide_step = min_step >= 2 ? 1 : 0;
    upload_vec(&s->wbase, wb);
    const double kPi = 3.14159265358979323846;
    // twiddle columns: c = d (cos, d = 0..w) and c = w + d (sin, d = 1..w)
    auto tw = [&](int p, int col) -> double {
        if (col >= d.W) return 0.0;
        const int dd = col <= d.hw ? col : col - d.hw;
        const double ang = 2.0 * kPi * (double)(((int64_t)dd * p) % d.P) / d.P;
        return col <= d.hw ? std::cos(ang) : std::sin(ang);
    };
    // forward B operand: rows n = col (16), K = p; adjoint A operand: rows p, K = col (16)
    std::vector<uint8_t> fb(64u * d.P, 0), aa(64u * d.P, 0);
    const uint32_t sboB = (d.P / 8) * 128u;
    for (int p = 0; p < d.P; ++p) {
        for (int col = 0; col < 16; ++col) {
            const float v = (float)tw(p, col);
            const uint16_t hb = bf16_bits(v);
            const uint16_t lb = bf16_bits(v - bf16_to_float(hb));
            const uint32_t ob = canon_off(col, p, sboB);
            std::memcpy(&fb[ob], &hb, 2);
            std::memcpy(&fb[32u * d.P + ob], &lb, 2);
            const int q = p / kAdjChunk, pl = p % kAdjChunk;
            const uint32_t oa = q * (kAdjChunk * 16 * 2) + canon_off(pl, col, 256);
            std::memcpy(&aa[oa], &hb, 2);
            std::memcpy(&aa[32u * d.P + oa], &lb, 2);
        }
    }
    upload_vec(&s->twB, fb);
    upload_vec(&s->twA, aa);
    std::vector<float2> t2(d.S + d.W * d.S);
    for (int m = 0; m < d.S; ++m) {
        const double ang = 2.0 * kPi * m / d.S;
        t2[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    for (int di = 0; di < d.W; ++di)
        for (int r = 0; r < d.S; ++r) {
            const int64_t dl = di - d.hw;
            const int64_t num = ((dl * r) % d.L + d.L) % d.L;
            const double ang = 2.0 * kPi * (double)num / d.L;
            t2[d.S + di * d.S + r] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
    upload_vec(&s->tw2, t2);
    // jobs: lines of one trajectory (parity), all angles, in groups
    std::vector<TcJob> jf, ja;
    for (int par = 0; par < d.n_par; ++par) {
        std::vector<int> segs;
        for (int m = 0; m < d.M; ++m)
            for (int z = 0; z < d.Nz; ++z)
                if ((d.n_par == 1 ? 0 : (z & 1)) == par) segs.push_back(m * d.Nz + z);
        const int gf = c.G * c.spt, ga = c.nseg_adj;
        for (size_t k = 0; k < segs.size(); k += gf) {
            TcJob j{};
            j.parity = par;
            j.nseg = (int)std::min<size_t>(gf, segs.size() - k);
            for (int u = 0; u < j.nseg; ++u) j.seg[u] = segs[k + u];
            jf.push_back(j);
        }
        for (size_t k = 0; k < segs.size(); k += ga) {
            TcJob j{};
            j.parity = par;
            j.nseg = (int)std::min<size_t>(ga, segs.size() - k);
            for (int u = 0; u < j.nseg; ++u) j.seg[u] = segs[k + u];
            ja.push_back(j);
        }
    }
    s->n_fwd = (int)jf.size();
    s->n_adj = (int)ja.size();
    upload_vec(&s->jobs_fwd, jf);
    upload_vec(&s->jobs_adj, ja);
    dev_malloc((void **)&s->err, sizeof(int));
    if (s->err) cudaMemset(s->err, 0, sizeof(int));
    if (!s->twB || !s->twA || !s->tw2 || !s->jobs_fwd || !s->jobs_adj || !s->err || !s->wbase) {
        s->oom = true;
        return;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
    // the attribute is global to the kernel: allow the largest carve-up any handle may use
    cudaFuncSetAttribute(k_tc_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_tc_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaGetLastError();
    s->ok = true;
}

bool tc_init_oom(const mpi_ffl_handle *h) {
    const TcState *s = state(h);
    return s && s->oom;
}

void tc_release(mpi_ffl_handle *h) {
    TcState *s = state(h);
    if (!s) return;
    void *ptrs[] = {s->jobs_fwd, s->jobs_adj, s->twB, s->twA, s->tw2, s->err, s->wbase};
    for (void *p : ptrs)
        if (p) dev_free(p);
    delete s;
    h->tc_state = nullptr;
}

void tc_tables_changed(mpi_ffl_handle *) {}

void tc_forward_line(mpi_ffl_handle *h, const float *fine, const float *gain, float *data, cudaStream_t st) {
    TcState *s = state(h);
    s->cfg.prec = h->precision;
    const int grid = std::min(s->n_fwd, s->n_sm);
    k_tc_fwd<<<grid, kFwdThreads + 32, s->cfg.f_total, st>>>(fine, h->t_tnf, h->t_vr, gain, s->jobs_fwd, s->n_fwd, s->twB,
                                                        s->tw2, h->t_dgam, data, h->d, s->cfg, s->err);
}

void tc_adjoint_line(mpi_ffl_handle *h, const float *data, const float *gain, float *fine, cudaStream_t st) {
    TcState *s = state(h);
    s->cfg.prec = h->precision;
    const int grid = std::min(s->n_adj, s->n_sm);
    k_tc_adj<<<grid, kAdjThreads, s->cfg.a_total, st>>>(data, h->t_tnf, h->t_vr, gain, s->jobs_adj, s->n_adj, s->twA,
                                                        s->tw2, h->t_dgam, s->wbase, fine, h->d, s->cfg, s->err);
}

int tc_take_error(mpi_ffl_handle *h) {
    TcState *s = state(h);
    if (!s || !s->err) return 0;
    int v = 0;
    cudaMemcpy(&v, s->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (v) cudaMemset(s->err, 0, sizeof(int));
    return v;
}

}  // namespace mpiffl
