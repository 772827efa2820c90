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
constexpr int kFwdThreads = 128;   // one thread per MMA row
constexpr int kAdjThreads = 256;
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
    uint32_t f_fine, f_B, f_A, f_tw, f_bar, f_total;
    // adjoint carve-up
    uint32_t a_fine, a_A, a_B, a_tw, a_y, a_bar, a_total;
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
    bool ok = false;
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

__global__ void __launch_bounds__(kFwdThreads, 1)
    k_tc_fwd(const float *__restrict__ fine, const TrajEntry *__restrict__ traj, const float *__restrict__ gain,
             const TcJob *__restrict__ jobs, const uint8_t *__restrict__ twB, const float2 *__restrict__ tw2,
             const float2 *__restrict__ dgam, float *__restrict__ data, Dims d, TcCfg c, int *err) {
    extern __shared__ __align__(128) uint8_t sm[];
    const TcJob job = jobs[blockIdx.x];
    float *sfine = reinterpret_cast<float *>(sm + c.f_fine);
    uint8_t *sB = sm + c.f_B;
    uint8_t *sA = sm + c.f_A;
    float2 *stw = reinterpret_cast<float2 *>(sm + c.f_tw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + c.f_bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + c.f_bar + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int S = d.S;
    const int nsegc = c.G * c.spt;

    if (tid == 0) {
        ptx::mbar_init(&bars[0], 1);
        ptx::mbar_init(&bars[1], 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(tslot, c.tmem_fwd);
        ptx::tmem_relinquish();
    }
    // stage the jobs' fine rows (zero rows for empty slots), the twiddle operand and tables
    for (int sl = 0; sl < nsegc; ++sl) {
        float *dst = sfine + sl * c.ne_pad;
        if (sl < job.nseg) {
            const float *src = fine + (size_t)job.seg[sl] * d.Ne;
            for (int e = tid; e < d.Ne; e += kFwdThreads) dst[e] = __ldg(src + e);
        } else {
            for (int e = tid; e < d.Ne; e += kFwdThreads) dst[e] = 0.f;
        }
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(twB);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        const int n16 = (64 * d.P) / 16;
        for (int i = tid; i < n16; i += kFwdThreads) dst[i] = __ldg(src + i);
        for (int i = tid; i < S + d.W * S; i += kFwdThreads) stw[i] = __ldg(tw2 + i);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;

    const int sg = tid / S, r = tid % S;
    const TrajEntry *tr = traj + (size_t)job.parity * d.L;
    const float *frow[2];
    float gl[2];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const int sl = g * c.spt + sg;
        frow[g] = sfine + (g < c.G ? sl : 0) * c.ne_pad;
        gl[g] = (g < c.G && sl < job.nseg) ? __ldg(gain + job.seg[sl] / d.Nz) : 0.f;
    }
    const int nchunks = d.P / c.Kc;
    const uint32_t tileA = 128u * c.Kc * 2u;  // bytes of one (tile, hi|lo) A buffer
    const uint32_t stageA = tileA * 2u * c.G;
    const uint32_t sboA = (c.Kc / 8) * 128u;
    const uint32_t sboB = (d.P / 8) * 128u;
    const uint32_t halfB = 32u * d.P;
    const uint32_t idesc = ptx::instr_desc(1, 128, 16);
    bool good = true;
    for (int q = 0; q < nchunks && good; ++q) {
        const int st = q & 1;
        if (q >= 2) {
            const bool w = ptx::mbar_wait_bounded(&bars[st], ((q - 2) >> 1) & 1, kWaitLimit);
            good = __syncthreads_and(w);
            if (!good) break;
        }
        uint8_t *A = sA + st * stageA;
        for (int p8 = 0; p8 < c.Kc / 8; ++p8) {
            TrajEntry te[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) te[u] = load_te(tr + (size_t)(q * c.Kc + p8 * 8 + u) * S + r);
            const uint32_t off = (tid / 8) * sboA + p8 * 128 + (tid % 8) * 16;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                if (g >= c.G) break;
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = gl[g] * fmaf(te[u].w0, frow[g][te[u].n], te[u].w1 * frow[g][te[u].n + 1]);
                uint4 hi, lo;
                split8(v, hi, lo);
                *reinterpret_cast<uint4 *>(A + (2 * g) * tileA + off) = hi;
                *reinterpret_cast<uint4 *>(A + (2 * g + 1) * tileA + off) = lo;
            }
        }
        ptx::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
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
            ptx::mma_commit(&bars[st]);
        }
    }
    if (good) {
        const int ql = nchunks - 1;
        const bool w = ptx::mbar_wait_bounded(&bars[ql & 1], (ql >> 1) & 1, kWaitLimit);
        good = __syncthreads_and(w);
    }
    ptx::tc_fence_after();
    if (good) {
        // T[row][c] from TMEM into shared memory (reusing the A buffers)
        float *sT = reinterpret_cast<float *>(sA);
        for (int g = 0; g < c.G; ++g) {
            float v[16];
            ptx::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + g * 16, v);
#pragma unroll
            for (int cc = 0; cc < 16; ++cc)
                if (cc < d.W) sT[(g * 128 + tid) * d.W + cc] = v[cc];
        }
        ptx::tc_fence_before();
        __syncthreads();
        const float inv_sqrt_l = rsqrtf((float)d.L);
        for (int task = tid; task < job.nseg * d.nb; task += kFwdThreads) {
            const int sl = task / d.nb, o = task % d.nb;
            const int di = o % d.W, dl = di - d.hw, ad = dl < 0 ? -dl : dl;
            const int kmod = (d.kmin + o / d.W) % S;
            const float sgn = dl < 0 ? -1.f : 1.f;
            const float *rowT = sT + ((sl / c.spt) * 128 + (sl % c.spt) * S) * d.W;
            const float2 *twd = stw + S + di * S;
            float re = 0.f, im = 0.f;
            int idx = 0;
            for (int rr = 0; rr < S; ++rr) {
                const float tre = rowT[rr * d.W + ad];
                const float tim = ad == 0 ? 0.f : sgn * rowT[rr * d.W + d.hw + ad];
                const float2 a = stw[idx], b = twd[rr];
                const float wr = a.x * b.x - a.y * b.y, wi = a.x * b.y + a.y * b.x;
                re = fmaf(tre, wr, fmaf(-tim, wi, re));
                im = fmaf(tre, wi, fmaf(tim, wr, im));
                idx += kmod;
                if (idx >= S) idx -= S;
            }
            re *= inv_sqrt_l;
            im *= inv_sqrt_l;
            const float2 gd = __ldg(dgam + o);
            reinterpret_cast<float2 *>(data)[(size_t)job.seg[sl] * d.nb + o] =
                make_float2(gd.x * re - gd.y * im, gd.x * im + gd.y * re);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, c.tmem_fwd);
}

// ============================================================================ adjoint

__device__ __forceinline__ int padx(int e) { return e + (e >> 5); }

__global__ void __launch_bounds__(kAdjThreads, 1)
    k_tc_adj(const float *__restrict__ data, const TrajEntry *__restrict__ traj, const float *__restrict__ gain,
             const TcJob *__restrict__ jobs, const uint8_t *__restrict__ twA, const float2 *__restrict__ tw2,
             const float2 *__restrict__ dgam, float *__restrict__ fine, Dims d, TcCfg c, int *err) {
    extern __shared__ __align__(128) uint8_t sm[];
    const TcJob job = jobs[blockIdx.x];
    float *sacc = reinterpret_cast<float *>(sm + c.a_fine);
    uint8_t *sA = sm + c.a_A;
    uint8_t *sB = sm + c.a_B;
    float2 *stw = reinterpret_cast<float2 *>(sm + c.a_tw);
    float2 *sy = reinterpret_cast<float2 *>(sm + c.a_y);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + c.a_bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + c.a_bar + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = d.S;
    const int nsegc = c.nseg_adj;
    const int ncols = c.ncols_adj;

    if (tid == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(tslot, c.tmem_adj);
        ptx::tmem_relinquish();
    }
    for (int i = tid; i < nsegc * c.ne_adj; i += kAdjThreads) sacc[i] = 0.f;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(twA);
        uint4 *dst = reinterpret_cast<uint4 *>(sA);
        const int n16 = (64 * d.P) / 16;
        for (int i = tid; i < n16; i += kAdjThreads) dst[i] = __ldg(src + i);
        for (int i = tid; i < S + d.W * S; i += kAdjThreads) stw[i] = __ldg(tw2 + i);
    }
    const float inv_sqrt_l = rsqrtf((float)d.L);
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
    // per column n = (line, r): U[d] = sum_k y'[k, d] conj(e^{2 pi i k r/S} e^{2 pi i d r/L}),
    // coefficients A_0 = Re U[0], A_d = Re U[d] + Re U[-d], B_d = Im U[d] - Im U[-d]
    for (int n = tid; n < ncols; n += kAdjThreads) {
        const int sl = n / S, rr = n % S;
        float ur[2 * kMaxHw + 1], ui[2 * kMaxHw + 1];
#pragma unroll
        for (int di = 0; di < 2 * kMaxHw + 1; ++di) ur[di] = ui[di] = 0.f;
        for (int k = 0; k < d.K; ++k) {
            const float2 a = stw[((d.kmin + k) % S) * rr % S];
#pragma unroll
            for (int di = 0; di < 2 * kMaxHw + 1; ++di) {
                if (di >= d.W) break;
                const float2 b = stw[S + di * S + rr];
                const float wr = a.x * b.x - a.y * b.y, wi = a.x * b.y + a.y * b.x;  // e^{+i phi}
                const float2 y = sy[sl * d.nb + k * d.W + di];
                // y * e^{-i phi}
                ur[di] = fmaf(y.x, wr, fmaf(y.y, wi, ur[di]));
                ui[di] = fmaf(y.y, wr, fmaf(-y.x, wi, ui[di]));
            }
        }
        float coef[16];
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) coef[cc] = 0.f;
        coef[0] = ur[d.hw];
        for (int a = 1; a <= d.hw; ++a) {
            coef[a] = ur[d.hw + a] + ur[d.hw - a];
            coef[d.hw + a] = ui[d.hw + a] - ui[d.hw - a];
        }
        for (int h = 0; h < 2; ++h) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = coef[h * 8 + u];
            uint4 hi4, lo4;
            split8(v, hi4, lo4);
            const uint32_t off = canon_off(n, h * 8, 256);
            *reinterpret_cast<uint4 *>(sB + off) = hi4;
            *reinterpret_cast<uint4 *>(sB + (uint32_t)ncols * 32u + off) = lo4;
        }
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;
    const TrajEntry *tr = traj + (size_t)job.parity * d.L;
    const uint32_t idesc = ptx::instr_desc(1, 128, (uint32_t)ncols);
    const uint32_t halfA = 32u * d.P;
    const uint32_t halfB = (uint32_t)ncols * 32u;
    const int nchunks = d.P / kAdjChunk;
    const int quad = warp & 3, colhalf = warp >> 2;
    const int seg_lo = colhalf * (nsegc / 2), seg_hi = (colhalf + 1) * (nsegc / 2);
    bool good = true;
    for (int q = 0; q < nchunks; ++q) {
        if (tid == 0) {
            ptx::tc_fence_after();
            const uint32_t a0 = ptx::smem_u32(sA) + q * (kAdjChunk * 16 * 2);
            const uint64_t dAh = ptx::smem_desc(a0, 128, 256);
            const uint64_t dAl = ptx::smem_desc(a0 + halfA, 128, 256);
            const uint64_t dBh = ptx::smem_desc(ptx::smem_u32(sB), 128, 256);
            const uint64_t dBl = ptx::smem_desc(ptx::smem_u32(sB) + halfB, 128, 256);
            ptx::mma_bf16(tmem, dAh, dBh, idesc, 0u);
            if (c.prec == MPI_FFL_PREC_BF16X3) {
                ptx::mma_bf16(tmem, dAh, dBl, idesc, 1u);
                ptx::mma_bf16(tmem, dAl, dBh, idesc, 1u);
            }
            ptx::mma_commit(bar);
        }
        const bool w = ptx::mbar_wait_bounded(bar, q & 1, kWaitLimit);
        good = __syncthreads_and(w);
        if (!good) break;
        ptx::tc_fence_after();
        const int p = q * kAdjChunk + quad * 32 + lane;  // this thread's period
        for (int rb = 0; rb < S; rb += 16) {
            TrajEntry te[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) te[u] = load_te(tr + (size_t)p * S + rb + u);
            for (int sl = seg_lo; sl < seg_hi; ++sl) {
                float v[16];
                ptx::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(sl * S + rb), v);
                float *acc = sacc + sl * c.ne_adj;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    atomicAdd(acc + padx(te[u].n), te[u].w0 * v[u]);
                    atomicAdd(acc + padx(te[u].n + 1), te[u].w1 * v[u]);
                }
            }
        }
        ptx::tc_fence_before();
        __syncthreads();
    }
    if (good) {
        for (int sl = 0; sl < job.nseg; ++sl) {
            const float g = __ldg(gain + job.seg[sl] / d.Nz);
            float *dst = fine + (size_t)job.seg[sl] * d.Ne;
            const float *acc = sacc + sl * c.ne_adj;
            for (int e = tid; e < d.Ne; e += kAdjThreads) dst[e] = g * acc[padx(e)];
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
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

bool plan(const Dims &d, TcCfg &c) {
    if (d.S > 128 || 128 % d.S != 0 || d.S % 16 != 0) return false;  // lines tile 128 MMA rows
    if (d.W > 16) return false;                                      // twiddle columns fit N = 16
    if (d.P % kAdjChunk != 0) return false;                          // adjoint period chunks
    c.spt = 128 / d.S;
    c.Kc = (d.P % 64 == 0) ? 64 : 32;
    c.G = c.spt >= 2 ? 1 : 2;  // two lines per forward job either way
    if (c.spt * c.G > kTcMaxSeg) return false;
    c.ne_pad = (d.Ne + 3) / 4 * 4;
    c.tmem_fwd = pow2_cols(c.G * 16);
    uint32_t o = 0;
    c.f_fine = o;
    o = align_up(o + 4u * c.ne_pad * c.G * c.spt, 128);
    c.f_B = o;
    o = align_up(o + 64u * d.P, 128);
    c.f_A = o;
    o = align_up(o + 2u * 2u * c.G * 128u * c.Kc * 2u, 128);
    c.f_tw = o;
    o = align_up(o + 8u * (d.S + d.W * d.S), 128);
    c.f_bar = o;
    c.f_total = o + 64;
    // adjoint: 256 MMA columns of (line, r)
    c.nseg_adj = 256 / d.S;
    if (c.nseg_adj > kTcMaxSeg || c.nseg_adj < 2) return false;
    c.ncols_adj = c.nseg_adj * d.S;
    c.tmem_adj = pow2_cols(c.ncols_adj);
    c.ne_adj = d.Ne + (d.Ne >> 5) + 2;
    o = 0;
    c.a_fine = o;
    o = align_up(o + 4u * c.ne_adj * c.nseg_adj, 128);
    c.a_A = o;
    o = align_up(o + 64u * d.P, 128);
    c.a_B = o;
    o = align_up(o + 64u * c.ncols_adj, 128);
    c.a_tw = o;
    o = align_up(o + 8u * (d.S + d.W * d.S), 128);
    c.a_y = o;
    o = align_up(o + 8u * c.nseg_adj * d.nb, 128);
    c.a_bar = o;
    // at least 80 KiB so that at most two blocks (2 x 256 TMEM columns) share an SM
    c.a_total = std::max<uint32_t>(o + 64, 80u * 1024u);
    return c.f_total <= 227 * 1024 && c.a_total <= 227 * 1024;
}

template <class T>
void upload_vec(T **p, const std::vector<T> &v) {
    if (cudaMalloc((void **)p, v.size() * sizeof(T)) != cudaSuccess) {
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
    if (!plan(d, s->cfg)) return;
    TcCfg &c = s->cfg;
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
    cudaMalloc((void **)&s->err, sizeof(int));
    if (s->err) cudaMemset(s->err, 0, sizeof(int));
    if (!s->twB || !s->twA || !s->tw2 || !s->jobs_fwd || !s->jobs_adj || !s->err) return;
    cudaFuncSetAttribute(k_tc_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.f_total);
    cudaFuncSetAttribute(k_tc_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.a_total);
    cudaGetLastError();
    s->ok = true;
}

void tc_release(mpi_ffl_handle *h) {
    TcState *s = state(h);
    if (!s) return;
    void *ptrs[] = {s->jobs_fwd, s->jobs_adj, s->twB, s->twA, s->tw2, s->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete s;
    h->tc_state = nullptr;
}

void tc_tables_changed(mpi_ffl_handle *) {}

void tc_forward_line(mpi_ffl_handle *h, const float *fine, const float *gain, float *data, cudaStream_t st) {
    TcState *s = state(h);
    s->cfg.prec = h->precision;
    k_tc_fwd<<<s->n_fwd, kFwdThreads, s->cfg.f_total, st>>>(fine, h->t_traj, gain, s->jobs_fwd, s->twB, s->tw2,
                                                           h->t_dgam, data, h->d, s->cfg, s->err);
}

void tc_adjoint_line(mpi_ffl_handle *h, const float *data, const float *gain, float *fine, cudaStream_t st) {
    TcState *s = state(h);
    s->cfg.prec = h->precision;
    k_tc_adj<<<s->n_adj, kAdjThreads, s->cfg.a_total, st>>>(data, h->t_traj, gain, s->jobs_adj, s->twA, s->tw2,
                                                           h->t_dgam, fine, h->d, s->cfg, s->err);
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
