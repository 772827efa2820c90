// Collapsed line operator on tensor cores.
//
// Every raster line of one trajectory (line parity) sees the same E, V and the
// same band DFT, so S D_Gamma F V E (Sec. 2.1, Eq. (13), without the per-angle
// gain) is one fixed complex matrix W of n_bins x N_e per trajectory -- the same
// reassociation of the operator chain that lets the paper apply one FFT instead of
// three. W is built once on the host in double precision from the trajectory
// (W[o][e] = D_o L^-1/2 sum_j e^{2 pi i w_o j / L} (w0_j [n_j = e] + w1_j [n_j + 1 = e])),
// and optionally folded with H into W H (n_bins x N). A line stage then is
//     data[line] = g_m W fine[line]          (forward)
//     fine[line] = g_m Re(W^H data[line])    (adjoint, real inner product)
// i.e. one dense GEMM per trajectory, with W stored as a real matrix whose rows
// alternate Re and Im, so the data stay in their interleaved complex layout.
//
// GEMM kernel: C[row] = scale[row] * sum_k A[row][k] B[n][k] on tcgen05 with the
// FP32 operands split into bf16 or tf32 hi + lo (hi*hi + hi*lo + lo*hi, FP32
// accumulate): bf16 parts keep 16 mantissa bits of each operand, tf32 parts 22.
// Warps 0-3 convert A rows (gathered by an index list) into the canonical K-major
// shared-memory layout and run the epilogue; warp 4 issues the MMAs; warp 5 streams
// the pre-split B operand with bulk copies. Stages are handed over with mbarriers.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "collapsed.h"
#include "split_operands.cuh"
#include "tc_ptx.cuh"

namespace mpiffl {

namespace {

constexpr int kBM = 128;     // rows per tile (MMA M)
constexpr int kBK = 64;      // K per pipeline stage
constexpr int kProd = 128;   // producer threads (one per row)
constexpr uint32_t kWait = 1u << 24;
constexpr uint32_t kWaitSleep = 1u << 22;  // polls of mbar_wait_sleep_bounded: over a second

struct GemmArgs {
    const float *A;
    int64_t lda;
    const int *arow;     // M row indices into A
    int M, Ka;           // rows, valid K
    const uint8_t *B;    // per N tile, per K chunk: hi then lo blocks of BN x kBK bf16 (canonical)
    int BN, nkc;         // N tile width, K chunks
    float *C;
    int64_t ldc;
    const int *crow;     // M row indices into C
    int Nc;              // valid N
    const float *rscale; // per-row scale: scale[arow / rdiv]
    int rdiv;
    int prec;
    int stages;
    uint32_t tmem_cols;
    int *err;
    const int *done;     // nonzero: the problem is finished, its blocks do nothing
    int tf32;            // 1: tf32 hi + lo operands (32 K elements per stage), 0: bf16 (64)
    int nacc;            // accumulators in TMEM: K chunk kc adds into accumulator kc % nacc
    int acc_stride;      // TMEM columns between accumulators (a multiple of 32, >= BN)
    int b_tstride;       // K chunks per N tile in B's storage (0: nkc); B may be a K window of a table
    // A pre-split in its canonical layout (NULL: the producer warps split g.A). 1 KB blocks
    // (group of 8 rows, K chunk) ordered [chunk][hi, lo][group]; tile row group
    // j * apk_gper + g (g < apk_gper, j < apk_jg) takes the blocks of group g at chunk
    // apk_cbase + j * apk_cstep + kc, so each j is one contiguous copy per half.
    const uint8_t *apk;
    int apk_jg, apk_gper, apk_cbase, apk_cstep;
    // failure-detection test hook: > 0 makes every block wait this many polls on the
    // final-MMA barrier before any copy or MMA is issued (so nothing ever arrives
    // there), record a timeout and free its TMEM (mpi_ffl_test_inject_timeout)
    uint32_t inject;
};

// The tensor-core accumulation into TMEM is not round-to-nearest FP32, so its error
// grows with the number of MMAs chained into one accumulator. K chunks are spread
// over nacc accumulators (as many as fit per_sm blocks per SM into the 512 TMEM
// columns, at most 4), which the epilogue adds in FP32.
void set_accumulators(GemmArgs &g, int per_sm = 2) {
    g.acc_stride = (g.BN + 31) / 32 * 32;
    g.nacc = std::max(1, std::min({4, 512 / per_sm / g.acc_stride, g.nkc}));
    const int cols = g.nacc * g.acc_stride;
    g.tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
}

__device__ __forceinline__ void split8(const float (&v)[8], uint4 &hi, uint4 &lo) { split8_bf16(v, hi, lo); }

constexpr int kProdWarps = 8;                     // A producers (and epilogue)
constexpr int kGemmThreads = (kProdWarps + 2) * 32;  // + MMA issuer + B loader

// One K chunk of the A tile for one producer thread: 4 units of (row, core-matrix
// row kg), 8 bf16 or 4 tf32 values each, as float4s (bf16: 2 per unit).
struct AChunk {
    float4 v[8];
};

// MODE 0: bf16 operands, 1: tf32, 2: as g.tf32 says (batches that may mix both).
// One output tile. With tslot_ext NULL the block allocates (and at the end frees) its own
// TMEM columns; a persistent block passes the slot of columns it holds for all its tiles.
// PRE: every problem of the launch has A pre-split (g.apk), and the producer warps' split
// is compiled out (a smaller kernel: the forward's blocks live a few microseconds, and
// instruction fetch is among their stalls).
template <int MODE, bool PRE = false>
__device__ __forceinline__ void gemm_tile(const GemmArgs &g, int mt, int nt, uint8_t *sm, const uint32_t *tslot_ext) {
    const bool tf32 = MODE == 2 ? g.tf32 != 0 : MODE == 1;
    const uint32_t bytesA = kBM * kBK * 2;          // one of hi | lo
    const uint32_t bytesB = (uint32_t)g.BN * kBK * 2;
    const uint32_t stage = 2 * bytesA + 2 * bytesB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + g.stages * stage);  // full[S], empty[S], done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * g.stages + 1);
    int *flag = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < g.stages; ++s) {
            // producer warps + the B copy, or the loader alone when A comes pre-split
            ptx::mbar_init(&bars[s], g.apk ? 1 : kProdWarps + 1);
            ptx::mbar_init(&bars[g.stages + s], 1);
        }
        ptx::mbar_init(&bars[2 * g.stages], 1);
        ptx::fence_mbar_init();
        *flag = 0;
    }
    if (!tslot_ext && warp == 0) {
        ptx::tmem_alloc(tslot, g.tmem_cols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot_ext ? *tslot_ext : *tslot;
    ptx::grid_dep_wait();  // A (and the output rows) belong to earlier kernels of the stream
    ptx::grid_dep_launch();

    if (g.inject > 0) {
        // test hook: no role runs, so the final-MMA barrier never completes and every
        // thread's bounded wait on it runs out; the block then records a timeout and
        // frees its TMEM below like a block whose pipeline stalled
        if (!ptx::mbar_wait_bounded(&bars[2 * g.stages], 0, g.inject) && lane == 0) atomicExch(flag, 1);
    } else if (warp < kProdWarps) {
        // ------------------------------------------------------------ A producers
        // Warp w fills row groups 2w and 2w+1 (rows 16w..16w+15). In one pass a lane
        // takes row 8rg + (lane & 7) and 16-byte core-matrix row kg = 4kh + (lane >> 3)
        // (8 bf16 or 4 tf32 values): 8 rows x 4 consecutive core-matrix rows per warp
        // store, 512 contiguous shared-memory bytes, conflict-free; the global reads
        // are 8 row segments of 128 (bf16) or 64 (tf32) bytes. The loads of chunk
        // kc + 1 are issued before chunk kc is split and stored.
        const int r7 = lane & 7, kq = lane >> 3;
        const float *rp[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gmr = mt * kBM + 8 * (2 * warp + q) + r7;
            const int arr = gmr < g.M ? __ldg(g.arow + gmr) : -1;
            rp[q] = arr >= 0 ? g.A + (size_t)arr * g.lda : nullptr;
        }
        const bool vec = (g.lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.A) & 15) == 0);
        auto load = [&](int kc, AChunk &c) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = u >> 1, kg = 4 * (u & 1) + kq;
                const float *p = rp[q];
                if (tf32) {
                    const int k = kc * (kBK / 2) + kg * 4;
                    if (p && vec && k + 4 <= g.Ka) {
                        c.v[u] = __ldg(reinterpret_cast<const float4 *>(p + k));
                    } else {
                        c.v[u].x = (p && k + 0 < g.Ka) ? __ldg(p + k + 0) : 0.f;
                        c.v[u].y = (p && k + 1 < g.Ka) ? __ldg(p + k + 1) : 0.f;
                        c.v[u].z = (p && k + 2 < g.Ka) ? __ldg(p + k + 2) : 0.f;
                        c.v[u].w = (p && k + 3 < g.Ka) ? __ldg(p + k + 3) : 0.f;
                    }
                } else {
                    const int k = kc * kBK + kg * 8;
                    if (p && vec && k + 8 <= g.Ka) {
                        c.v[2 * u] = __ldg(reinterpret_cast<const float4 *>(p + k));
                        c.v[2 * u + 1] = __ldg(reinterpret_cast<const float4 *>(p + k + 4));
                    } else {
                        float t[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) t[e] = (p && k + e < g.Ka) ? __ldg(p + k + e) : 0.f;
                        c.v[2 * u] = make_float4(t[0], t[1], t[2], t[3]);
                        c.v[2 * u + 1] = make_float4(t[4], t[5], t[6], t[7]);
                    }
                }
            }
        };
        // split and store chunk kc into its stage; false if the stage never came free
        auto produce = [&](int kc, const AChunk &c) -> bool {
            const int s = kc % g.stages;
            if (kc >= g.stages) {
                // one lane per warp polls; __syncwarp orders the warp's stores after its acquire
                int fr = 1;
                if (lane == 0) fr = ptx::mbar_wait_bounded(&bars[g.stages + s], ((kc / g.stages) - 1) & 1, kWait);
                fr = __shfl_sync(0xffffffffu, fr, 0);
                __syncwarp();
                if (!fr) return false;
            }
            uint8_t *sa = sm + s * stage;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = u >> 1, kg = 4 * (u & 1) + kq;
                uint4 hi, lo;
                if (tf32) {
                    const float f[4] = {c.v[u].x, c.v[u].y, c.v[u].z, c.v[u].w};
                    split4_tf32(f, hi, lo);
                } else {
                    const float f[8] = {c.v[2 * u].x,     c.v[2 * u].y,     c.v[2 * u].z,     c.v[2 * u].w,
                                        c.v[2 * u + 1].x, c.v[2 * u + 1].y, c.v[2 * u + 1].z, c.v[2 * u + 1].w};
                    split8(f, hi, lo);
                }
                const uint32_t off = (2 * warp + q) * 1024u + kg * 128u + r7 * 16u;
                *reinterpret_cast<uint4 *>(sa + off) = hi;
                *reinterpret_cast<uint4 *>(sa + bytesA + off) = lo;
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars[s]);
            return true;
        };
        bool ok = true;
        if constexpr (!PRE) {
            AChunk ca, cb;
            if (!g.apk) load(0, ca);
            for (int kc = 0; kc < g.nkc && ok && !g.apk; kc += 2) {
                if (kc + 1 < g.nkc) load(kc + 1, cb);
                ok = produce(kc, ca);
                if (!ok || kc + 1 >= g.nkc) break;
                if (kc + 2 < g.nkc) load(kc + 2, ca);
                ok = produce(kc + 1, cb);
            }
        }
        // ------------------------------------------------------------ epilogue
        // TMEM lane quadrant w % 4 = tile rows 32 (w % 4) .. +31; warps w and w + 4
        // take alternate 16-column groups. The scaled tile goes through shared memory
        // (the stages are free once the last MMA is done; rows padded by 16 bytes, so a
        // quarter warp's 16-byte stores take distinct bank groups) and leaves as one
        // bulk copy per row, whole sectors instead of a row per lane per store.
        const int row = 32 * (warp & 3) + lane;
        const int gm = mt * kBM + row;
        // the row's output index and scale are read while the MMAs run
        const int ar = gm < g.M ? __ldg(g.arow + gm) : -1;
        const int cr = gm < g.M ? __ldg(g.crow + gm) : -1;
        const float sc = (cr >= 0 && g.rscale) ? __ldg(g.rscale + ar / g.rdiv) : 1.f;
        int done = 0;
        if (ok && lane == 0) done = ptx::mbar_wait_sleep_bounded(&bars[2 * g.stages], 0, kWaitSleep);
        done = __shfl_sync(0xffffffffu, done, 0);
        __syncwarp();
        // the producer warps go on together only if every one of them saw the last MMA
        if (ptx::bar_and(1, kProdWarps * 32, ok && done)) {
            ptx::tc_fence_after();
            float *crow = cr >= 0 ? g.C + (size_t)cr * g.ldc : nullptr;
            const bool vecc = (g.ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(g.C) & 15) == 0);
            const bool staged = vecc && g.Nc % 4 == 0;  // whole 16-byte units per row
            float *ct = reinterpret_cast<float *>(sm);
            const int ldt = g.BN + 4;
            const int nacc = min(g.nacc, g.nkc);
            const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            for (int c0 = 16 * (warp >> 2); c0 < g.BN; c0 += 32) {
                float v[16];
                ptx::tmem_ld16(tl + c0, v);
                for (int a = 1; a < nacc; ++a) {
                    float w[16];
                    ptx::tmem_ld16(tl + (uint32_t)(a * g.acc_stride + c0), w);
#pragma unroll
                    for (int u = 0; u < 16; ++u) v[u] += w[u];
                }
                const int n0 = nt * g.BN + c0;
                if (staged) {
                    float4 *dst = reinterpret_cast<float4 *>(ct + row * ldt + c0);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        dst[u] = make_float4(sc * v[4 * u], sc * v[4 * u + 1], sc * v[4 * u + 2], sc * v[4 * u + 3]);
                } else if (crow) {
                    if (vecc && n0 + 16 <= g.Nc) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            *reinterpret_cast<float4 *>(crow + n0 + 4 * u) =
                                make_float4(sc * v[4 * u], sc * v[4 * u + 1], sc * v[4 * u + 2], sc * v[4 * u + 3]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (n0 + u < g.Nc) crow[n0 + u] = sc * v[u];
                    }
                }
            }
            if (staged) {
                ptx::fence_proxy_async_smem();  // the tile's generic stores, then the async-proxy reads
                ptx::named_sync(1, kProdWarps * 32);
                const int n0 = nt * g.BN, ncols = min(g.BN, g.Nc - n0);
                if (warp < 4 && crow && ncols > 0) {
                    ptx::bulk_s2g(crow + n0, ct + row * ldt, 4u * (uint32_t)ncols);
                    ptx::bulk_commit();
                    ptx::bulk_wait_all();
                }
            }
        } else if (lane == 0) {
            atomicExch(flag, 1);
        }
    } else if (warp == kProdWarps) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = ptx::instr_desc(tf32 ? 2 : 1, kBM, (uint32_t)g.BN);
            bool ok = true;
            for (int kc = 0; kc < g.nkc && ok; ++kc) {
                const int s = kc % g.stages;
                if (!ptx::mbar_wait_bounded(&bars[s], (kc / g.stages) & 1, kWait)) {
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t a0 = ptx::smem_u32(sm + s * stage);
                const uint32_t b0 = a0 + 2 * bytesA;
                const uint32_t tacc = tmem + (uint32_t)((kc % g.nacc) * g.acc_stride);
                const bool first = kc < g.nacc;  // the first chunk of its accumulator
                for (int ks = 0; ks < kBK / 16; ++ks) {
                    const uint64_t dAh = ptx::smem_desc(a0 + ks * 256, 128, 1024);
                    const uint64_t dAl = ptx::smem_desc(a0 + bytesA + ks * 256, 128, 1024);
                    const uint64_t dBh = ptx::smem_desc(b0 + ks * 256, 128, 1024);
                    const uint64_t dBl = ptx::smem_desc(b0 + bytesB + ks * 256, 128, 1024);
                    // 4 MMA K-steps of 256 bytes per stage: K = 16 bf16 or K = 8 tf32 elements
                    const uint32_t acc = (!first || ks > 0) ? 1u : 0u;
                    if (tf32) {
                        ptx::mma_tf32(tacc, dAh, dBh, idesc, acc);
                        ptx::mma_tf32(tacc, dAh, dBl, idesc, 1u);
                        ptx::mma_tf32(tacc, dAl, dBh, idesc, 1u);
                    } else {
                        ptx::mma_bf16(tacc, dAh, dBh, idesc, acc);
                        ptx::mma_bf16(tacc, dAh, dBl, idesc, 1u);
                        ptx::mma_bf16(tacc, dAl, dBh, idesc, 1u);
                    }
                }
                ptx::mma_commit(&bars[g.stages + s]);
            }
            if (ok) ptx::mma_commit(&bars[2 * g.stages]);
            else atomicExch(flag, 1);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ B loader
        if (lane == 0) {
            const uint8_t *bt = g.B + (size_t)nt * (g.b_tstride ? g.b_tstride : g.nkc) * 2 * bytesB;
            // pre-split A: the row groups of this m tile that hold rows
            const int rg0 = mt * (kBM / 8);
            const int nrg = g.apk ? max(0, min(kBM / 8, g.apk_jg * g.apk_gper - rg0)) : 0;
            for (int kc = 0; kc < g.nkc; ++kc) {
                const int s = kc % g.stages;
                if (kc >= g.stages && !ptx::mbar_wait_bounded(&bars[g.stages + s], ((kc / g.stages) - 1) & 1, kWait)) {
                    atomicExch(flag, 1);
                    break;
                }
                uint8_t *sa = sm + s * stage;
                uint8_t *sb = sa + 2 * bytesA;
                ptx::mbar_arrive_expect_tx(&bars[s], 2 * bytesB + 2048u * (uint32_t)nrg);
                ptx::bulk_g2s(sb, bt + (size_t)kc * 2 * bytesB, 2 * bytesB, &bars[s]);
                for (int r = 0; r < nrg;) {  // one copy per half for each run of one j
                    const int rg = rg0 + r, j = rg / g.apk_gper, gg = rg - j * g.apk_gper;
                    const int len = min(g.apk_gper - gg, nrg - r);
                    const size_t c2 = 2 * (size_t)(g.apk_cbase + j * g.apk_cstep + kc);
                    const uint8_t *hi = g.apk + (c2 * g.apk_gper + gg) * 1024u;
                    const uint8_t *lo = g.apk + ((c2 + 1) * g.apk_gper + gg) * 1024u;
                    ptx::bulk_g2s(sa + r * 1024u, hi, 1024u * len, &bars[s]);
                    ptx::bulk_g2s(sa + bytesA + r * 1024u, lo, 1024u * len, &bars[s]);
                    r += len;
                }
            }
        }
        __syncwarp();
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *flag) atomicExch(g.err, 1);
    if (!tslot_ext && warp == 0) ptx::tmem_dealloc(tmem, g.tmem_cols);
}

template <int MODE, bool PRE = false>
__device__ __forceinline__ void gemm_body(const GemmArgs &g, int mt, int nt, uint8_t *sm) {
    gemm_tile<MODE, PRE>(g, mt, nt, sm, nullptr);
}

template <int MODE>
__global__ void __launch_bounds__(kGemmThreads, 2) k_gemm_split(GemmArgs g) {
    extern __shared__ __align__(128) uint8_t sm[];
    gemm_body<MODE>(g, blockIdx.x, blockIdx.y, sm);
}

// Both trajectories of a line stage in one launch: blocks [0, n0) belong to g0 (m
// tile b / nt0, n tile b % nt0, so the n tiles of an m tile run side by side and
// share its A rows in L2), the rest to g1.
template <int MODE, bool PRE = false>
__global__ void __launch_bounds__(kGemmThreads, 2) k_gemm_pair(GemmArgs g0, GemmArgs g1, int nt0, int n0, int nt1) {
    extern __shared__ __align__(128) uint8_t sm[];
    const int b = blockIdx.x;
    if (b < n0) gemm_body<MODE, PRE>(g0, b / nt0, b % nt0, sm);
    else gemm_body<MODE, PRE>(g1, (b - n0) / nt1, (b - n0) % nt1, sm);
}

// One persistent launch for several GEMM problems: items[i] = (problem, m tile, n tile).
// A block holds `cols` TMEM columns (the largest problem's need, at most 256, so two
// blocks share an SM) for all its items; each item sets up its own barriers, which are
// invalidated once the item is done.
__global__ void __launch_bounds__(kGemmThreads, 2) k_gemm_batch(const GemmArgs *__restrict__ args,
                                                       const int4 *__restrict__ items, int n_items,
                                                       uint32_t cols, uint32_t slot_off) {
    extern __shared__ __align__(128) uint8_t sm[];
    // the TMEM address lives past every item's layout (slot_off = the largest item's bytes)
    uint32_t &tslot = *reinterpret_cast<uint32_t *>(sm + slot_off);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        ptx::tmem_alloc(&tslot, cols);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
        const int4 it = items[i];
        const GemmArgs g = args[it.x];
        if (g.done && *g.done) continue;  // uniform over the block
        gemm_tile<2>(g, it.y, it.z, sm, &tslot);
        if (threadIdx.x == 0) {
            const uint32_t stage = 2u * kBM * kBK * 2 + 2u * (uint32_t)g.BN * kBK * 2;
            uint64_t *bars = reinterpret_cast<uint64_t *>(sm + g.stages * stage);
            for (int k = 0; k < 2 * g.stages + 1; ++k) ptx::mbar_inval(&bars[k]);
        }
        __syncthreads();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tslot, cols);
}

uint16_t bf16_bits(double x) {
    const float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t rounding = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + rounding) >> 16);
}
double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

uint32_t tf32_bits(double x) {
    const float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u + 0x1000u) & 0xFFFFE000u;  // round to nearest (ties away), 10-bit mantissa
}
double tf32_value(uint32_t b) {
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

// Pre-split B operand for k_gemm_split: Bm is Nv x Kv (row-major, double); padded to
// ntile*BN x nkc*(K per chunk); blocks [tile][chunk][hi, lo] of BN rows x 128 bytes per
// row in the canonical layout (64 bf16 or 32 tf32 elements per row and chunk).
std::vector<uint8_t> pack_b(const std::vector<double> &Bm, int Nv, int Kv, int BN, int &ntile, int &nkc, bool tf32) {
    ntile = (Nv + BN - 1) / BN;
    const int kpc = tf32 ? kBK / 2 : kBK;
    nkc = (Kv + kpc - 1) / kpc;
    const size_t blk = (size_t)BN * kBK * 2;
    std::vector<uint8_t> out((size_t)ntile * nkc * 2 * blk, 0);
    for (int t = 0; t < ntile; ++t)
        for (int kc = 0; kc < nkc; ++kc) {
            uint8_t *hi = out.data() + ((size_t)t * nkc + kc) * 2 * blk;
            uint8_t *lo = hi + blk;
            for (int nl = 0; nl < BN; ++nl) {
                const int n = t * BN + nl;
                for (int kl = 0; kl < kpc; ++kl) {
                    const int k = kc * kpc + kl;
                    const double v = (n < Nv && k < Kv) ? Bm[(size_t)n * Kv + k] : 0.0;
                    if (tf32) {
                        const uint32_t hb = tf32_bits(v);
                        const uint32_t lb = tf32_bits(v - tf32_value(hb));
                        const size_t off = (size_t)(nl / 8) * 1024 + (kl / 4) * 128 + (nl % 8) * 16 + (kl % 4) * 4;
                        std::memcpy(hi + off, &hb, 4);
                        std::memcpy(lo + off, &lb, 4);
                    } else {
                        const uint16_t hb = bf16_bits(v);
                        const uint16_t lb = bf16_bits(v - bf16_value(hb));
                        const size_t off = (size_t)(nl / 8) * 1024 + (kl / 8) * 128 + (nl % 8) * 16 + (kl % 8) * 2;
                        std::memcpy(hi + off, &hb, 2);
                        std::memcpy(lo + off, &lb, 2);
                    }
                }
            }
        }
    return out;
}

struct Packed {
    uint8_t *dev = nullptr;
    int BN = 0, ntile = 0, nkc = 0;
    int per_sm = 2;  // blocks per SM the tiling was chosen for (1: deeper pipeline, all TMEM)
};

struct ColState {
    bool ok = false;
    // per operand format (0 bf16, 1 tf32) and trajectory: forward / adjoint operands of
    // W (line) and W H (full)
    Packed evf_f[2][2], evf_a[2][2], full_f[2][2], full_a[2][2];
    std::vector<double> W[2];           // S D_Gamma F V E per trajectory (2 n_b x N_e, double)
    struct TensorState *ten = nullptr;  // slice-coupled operator of the tensor PSF
    int *rows[2] = {nullptr, nullptr};  // line indices of each trajectory
    int nrows[2] = {0, 0};
    int *err = nullptr;
    int n_par = 1;
    // A of the full line stage split once per call (forward: projections, adjoint: data),
    // per direction and trajectory, sized for the tf32 chunk count
    uint8_t *apk[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    bool oom = false;  // the shape is supported but a device allocation failed
    bool psf_stale = false;  // W H was built for another PSF width (W itself holds no PSF)
};

ColState *cs(const mpi_ffl_handle *h) { return reinterpret_cast<ColState *>(h->col_state); }

// Rows of one trajectory's full line stage for k_pack_lines.
struct PackLines {
    const int *arow;  // line index of each row
    int M;            // rows
    uint8_t *out;     // 1 KB blocks [chunk][hi, lo][group of 8 rows]
};

// A rows of the full line stage, split once per call into the canonical layout the
// producer warps would write, as k_pack_rows does for the tensor PSF: row r of
// trajectory blockIdx.y is line arow[r] of in (stride lda, Ka valid values, zero past
// Ka and past the last row). One thread per 16-byte row of a block (8 bf16 or 4 tf32
// values), split exactly as the producers split.
__global__ void __launch_bounds__(256) k_pack_lines(const float *__restrict__ in, int64_t lda, int Ka, int nkc,
                                                    int tf32, PackLines p0, PackLines p1) {
    const PackLines p = blockIdx.y ? p1 : p0;
    ptx::grid_dep_wait();  // the rows come from the previous kernel
    ptx::grid_dep_launch();
    const int kpc = tf32 ? kBK / 2 : kBK, epk = tf32 ? 4 : 8;
    const int G = (p.M + 7) / 8;
    const long long total = (long long)G * nkc * 64;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int kg = (int)(t & 7), r7 = (int)((t >> 3) & 7);
        const long long gc = t >> 6;  // block: (row group, chunk), row group fastest
        const int gq = (int)(gc % G), c = (int)(gc / G);
        const int r = 8 * gq + r7;
        const int line = r < p.M ? __ldg(p.arow + r) : -1;
        const float *src = line >= 0 ? in + (size_t)line * lda : nullptr;
        const int k0 = c * kpc + kg * epk;
        float v[8];
        if (src && epk == 8 && k0 + 8 <= Ka && (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(src + k0));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(src + k0 + 4));
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (src && e < epk && k0 + e < Ka) ? __ldg(src + k0 + e) : 0.f;
        }
        uint4 hi, lo;
        if (tf32) {
            const float f[4] = {v[0], v[1], v[2], v[3]};
            split4_tf32(f, hi, lo);
        } else {
            split8(v, hi, lo);
        }
        const uint32_t off = (uint32_t)kg * 128u + (uint32_t)r7 * 16u;
        *reinterpret_cast<uint4 *>(p.out + ((2 * (size_t)c) * G + gq) * 1024u + off) = hi;
        *reinterpret_cast<uint4 *>(p.out + ((2 * (size_t)c + 1) * G + gq) * 1024u + off) = lo;
    }
}

bool upload_packed(Packed &p, const std::vector<uint8_t> &v) {
    if (dev_malloc((void **)&p.dev, v.size()) != cudaSuccess) {
        p.dev = nullptr;
        return false;
    }
    return cudaMemcpy(p.dev, v.data(), v.size(), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Pipeline depth: for two blocks per SM, as many stages (2..4) as leave room for both,
// so that a grid of up to two blocks per SM runs in one wave; for one block per SM, up
// to 4 stages in the whole shared memory (all K chunks of a 256-deep K in flight).
size_t smem_for(int BN, int &stages, int per_sm = 2) {
    const size_t stage = 2u * kBM * kBK * 2 + 2u * BN * kBK * 2;
    const size_t two_per_sm = (113u * 1024u - 256u) / stage;
    const size_t cap = (220u * 1024u - 256u) / stage;
    stages = (int)std::min<size_t>(cap, std::max<size_t>(2, std::min<size_t>(4, per_sm == 1 ? cap : two_per_sm)));
    return stages * stage + 256;
}

GemmArgs make_args(const mpi_ffl_handle *h, const float *A, int64_t lda, int Ka, const int *arow, int M,
                   const Packed &B, float *C, int64_t ldc, const int *crow, int Nc, const float *rscale, int rdiv) {
    GemmArgs g{};
    g.A = A;
    g.lda = lda;
    g.arow = arow;
    g.M = M;
    g.Ka = Ka;
    g.B = B.dev;
    g.BN = B.BN;
    g.nkc = B.nkc;
    g.C = C;
    g.ldc = ldc;
    g.crow = crow;
    g.Nc = Nc;
    g.rscale = rscale;
    g.rdiv = rdiv;
    g.prec = h->precision;
    g.tf32 = h->precision == MPI_FFL_PREC_TF32 ? 1 : 0;
    smem_for(B.BN, g.stages, B.per_sm);
    set_accumulators(g, B.per_sm);
    g.err = cs(h)->err;
    g.done = nullptr;
    g.inject = h->inject_polls;
    return g;
}

// One GEMM problem per trajectory, all in one launch.
void launch_problems(const GemmArgs *g, const Packed *const *B, int n, cudaStream_t st) {
    int stages = 0;
    size_t smem = 0;
    for (int i = 0; i < n; ++i) smem = std::max(smem, smem_for(B[i]->BN, stages, B[i]->per_sm));
    const int mt0 = (g[0].M + kBM - 1) / kBM;
    const bool tf32 = g[0].tf32 != 0;
    if (n == 1) {
        if (tf32) k_gemm_split<1><<<dim3(mt0, B[0]->ntile), kGemmThreads, smem, st>>>(g[0]);
        else k_gemm_split<0><<<dim3(mt0, B[0]->ntile), kGemmThreads, smem, st>>>(g[0]);
        return;
    }
    const int n0 = mt0 * B[0]->ntile;
    const int n1 = (g[1].M + kBM - 1) / kBM * B[1]->ntile;
    const bool pre = g[0].apk && g[1].apk;  // both trajectories' A pre-split
    auto kern = tf32 ? (pre ? k_gemm_pair<1, true> : k_gemm_pair<1>) : (pre ? k_gemm_pair<0, true> : k_gemm_pair<0>);
    launch_dependent(kern, dim3(n0 + n1), dim3(kGemmThreads), smem, st, g[0], g[1], B[0]->ntile, n0, B[1]->ntile);
}

}  // namespace

// Arguments of the GEMM problems of one line stage of handle h (one per trajectory).
int gemm_problems(const mpi_ffl_handle *h, bool adjoint, const float *in, float *out, const int *done,
                  GemmArgs *args, int4 *items, int item_cap, int &n_items) {
    ColState *s = cs(h);
    const Dims &d = h->d;
    int np = 0;
    for (int par = 0; par < s->n_par; ++par) {
        const int f = h->precision == MPI_FFL_PREC_TF32 ? 1 : 0;
        const Packed &B = adjoint ? s->full_a[f][par] : s->full_f[f][par];
        GemmArgs &g = args[np];
        g = GemmArgs{};
        g.A = in;
        g.lda = adjoint ? 2 * d.nb : d.N;
        g.Ka = (int)g.lda;
        g.arow = s->rows[par];
        g.M = s->nrows[par];
        g.B = B.dev;
        g.BN = B.BN;
        g.nkc = B.nkc;
        g.C = out;
        g.ldc = adjoint ? d.N : 2 * d.nb;
        g.crow = s->rows[par];
        g.Nc = (int)g.ldc;
        g.rscale = h->t_gain;
        g.rdiv = d.Nz;
        g.prec = h->precision;
        g.tf32 = f;
        smem_for(B.BN, g.stages, B.per_sm);
        set_accumulators(g, B.per_sm);
        g.err = s->err;
        g.done = done;
        for (int mt = 0; mt < (g.M + kBM - 1) / kBM; ++mt)
            for (int nt = 0; nt < B.ntile; ++nt) {
                if (n_items >= item_cap) return -1;
                items[n_items++] = make_int4(np, mt, nt, 0);
            }
        ++np;
    }
    return np;
}

bool col_supported(const mpi_ffl_handle *h) {
    const ColState *s = cs(h);
    return s && s->ok;
}

// W per trajectory (real rows: Re then Im of each kept bin), from the double-precision
// trajectory; then W H with the PSF taps h(u_lo + e/Q - i).
void col_init(mpi_ffl_handle *h) {
    ColState *s = new ColState();
    h->col_state = s;
    const Dims &d = h->d;
    if ((size_t)d.N * 2 * d.nb * 8 > (size_t)1 << 31) return;
    s->n_par = d.n_par;
    const double kPi = 3.14159265358979323846;
    const int R = 2 * d.nb;
    // PSF matrix H[e][i] in double
    const double a = h->fwhm / (2.0 * langevin_half_point_host());
    std::vector<double> Hm((size_t)d.Ne * d.N);
    for (int e = 0; e < d.Ne; ++e)
        for (int i = 0; i < d.N; ++i) {
            const double u = (double)(e - d.D) / d.Q - i;
            Hm[(size_t)e * d.N + i] = 3.0 * langevin_d1_host(u / a);
        }
    // e^{2 pi i k r / S} and e^{2 pi i delta j / L}
    std::vector<double> ckr(d.S), skr(d.S);
    for (int m = 0; m < d.S; ++m) {
        ckr[m] = std::cos(2.0 * kPi * m / d.S);
        skr[m] = std::sin(2.0 * kPi * m / d.S);
    }
    const double isl = 1.0 / std::sqrt((double)d.L);
    for (int par = 0; par < d.n_par; ++par) {
        std::vector<double> Wr((size_t)R * d.Ne, 0.0);
        for (int j = 0; j < d.L; ++j) {
            int n;
            double f, v;
            traj_point_host(h, par, j, n, f, v);
            const int r = j % d.S;
            for (int di = 0; di < d.W; ++di) {
                const int64_t dl = di - d.hw;
                const int64_t num = ((dl * j) % d.L + d.L) % d.L;
                const double ang = 2.0 * kPi * (double)num / d.L;
                const double cd = std::cos(ang), sd = std::sin(ang);
                for (int k = 0; k < d.K; ++k) {
                    const int o = k * d.W + di;
                    const int m = (int)(((int64_t)(d.kmin + k) * r) % d.S);
                    // e^{2 pi i (kP + delta) j / L} = e^{2 pi i k r / S} e^{2 pi i delta j / L}
                    const double er = ckr[m] * cd - skr[m] * sd, ei = ckr[m] * sd + skr[m] * cd;
                    const double gr = h->dgamma[2 * o], gi = h->dgamma[2 * o + 1];
                    const double wr = (gr * er - gi * ei) * isl, wi = (gr * ei + gi * er) * isl;
                    const double w0 = (1.0 - f) * v, w1 = f * v;
                    Wr[(size_t)(2 * o) * d.Ne + n] += w0 * wr;
                    Wr[(size_t)(2 * o + 1) * d.Ne + n] += w0 * wi;
                    Wr[(size_t)(2 * o) * d.Ne + n + 1] += w1 * wr;
                    Wr[(size_t)(2 * o + 1) * d.Ne + n + 1] += w1 * wi;
                }
            }
        }
        // transposed W (Ne x R), W H (R x N) and its transpose (N x R)
        std::vector<double> Wt((size_t)d.Ne * R), WH((size_t)R * d.N, 0.0), WHt((size_t)d.N * R);
        for (int o = 0; o < R; ++o)
            for (int e = 0; e < d.Ne; ++e) Wt[(size_t)e * R + o] = Wr[(size_t)o * d.Ne + e];
        {
            // rows of W H on the host's cores (each row is independent)
            const int nt = std::max(1, std::min<int>(R, (int)std::thread::hardware_concurrency()));
            std::vector<std::thread> pool;
            for (int t = 0; t < nt; ++t)
                pool.emplace_back([&, t]() {
                    for (int o = t; o < R; o += nt) {
                        double *out = WH.data() + (size_t)o * d.N;
                        const double *wrow = Wr.data() + (size_t)o * d.Ne;
                        for (int e = 0; e < d.Ne; ++e) {
                            const double w = wrow[e];
                            if (w == 0.0) continue;
                            const double *hrow = Hm.data() + (size_t)e * d.N;
                            for (int i = 0; i < d.N; ++i) out[i] += w * hrow[i];
                        }
                    }
                });
            for (auto &th : pool) th.join();
        }
        for (int o = 0; o < R; ++o)
            for (int i = 0; i < d.N; ++i) WHt[(size_t)i * R + o] = WH[(size_t)o * d.N + i];
        auto mk1 = [&](Packed &p, const std::vector<double> &m, int Nv, int Kv, int BN, int per_sm, bool tf) {
            p.BN = BN;
            p.per_sm = per_sm;
            return upload_packed(p, pack_b(m, Nv, Kv, BN, p.ntile, p.nkc, tf));
        };
        auto mk = [&](Packed (&p)[2][2], const std::vector<double> &m, int Nv, int Kv, int BN, int per_sm) {
            return mk1(p[0][par], m, Nv, Kv, BN, per_sm, false) && mk1(p[1][par], m, Nv, Kv, BN, per_sm, true);
        };
        // N tile: about two blocks per SM over both trajectories' M tiles
        int n_sm = 152, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const int mtiles = std::max(1, d.n_par * ((d.nseg / d.n_par + kBM - 1) / kBM));
        // N tile: one block per SM over the m tiles of both trajectories when tiles of at
        // most 256 columns fit in one wave that way (then a block keeps all K chunks in
        // flight and owns the TMEM); else at most two blocks per SM, still one wave
        auto pick_bn = [&](int Nv, int &per_sm) {
            auto round = [](int bn) { return std::max(32, std::min(256, (bn + 15) / 16 * 16)); };
            const int one = n_sm / mtiles;
            if (one >= 1) {
                const int bn = round((Nv + one - 1) / one);
                if ((Nv + bn - 1) / bn * mtiles <= n_sm) {
                    per_sm = 1;
                    return bn;
                }
            }
            per_sm = 2;
            const int want_tiles = std::max(1, (2 * n_sm) / mtiles);
            return round((Nv + want_tiles - 1) / want_tiles);
        };
        int ps[4];
        const int bn_ef = pick_bn(R, ps[0]), bn_ea = pick_bn(d.Ne, ps[1]);
        const int bn_ff = pick_bn(R, ps[2]), bn_fa = pick_bn(d.N, ps[3]);
        if (!mk(s->evf_f, Wr, R, d.Ne, bn_ef, ps[0]) || !mk(s->evf_a, Wt, d.Ne, R, bn_ea, ps[1]) ||
            !mk(s->full_f, WH, R, d.N, bn_ff, ps[2]) || !mk(s->full_a, WHt, d.N, R, bn_fa, ps[3])) {
            s->oom = true;
            return;
        }
        s->W[par] = std::move(Wr);
        // lines of this trajectory
        std::vector<int> rows;
        for (int m = 0; m < d.M; ++m)
            for (int z = 0; z < d.Nz; ++z)
                if ((d.n_par == 1 ? 0 : (z & 1)) == par) rows.push_back(m * d.Nz + z);
        s->nrows[par] = (int)rows.size();
        if (dev_malloc((void **)&s->rows[par], rows.size() * sizeof(int)) != cudaSuccess) {
            s->oom = true;
            return;
        }
        for (int dir = 0; dir < 2; ++dir) {  // K = N (forward) or 2 n_b (adjoint), tf32 chunks of 32
            const int kmax = dir ? 2 * d.nb : d.N;
            const size_t bytes = (size_t)((kmax + kBK / 2 - 1) / (kBK / 2)) * 2 * ((rows.size() + 7) / 8) * 1024;
            if (dev_malloc((void **)&s->apk[dir][par], std::max<size_t>(bytes, 1024)) != cudaSuccess) {
                s->oom = true;
                return;
            }
            // the rows past the last of a group stay zero when the projector writes A
            cudaMemset(s->apk[dir][par], 0, std::max<size_t>(bytes, 1024));
        }
        cudaMemcpy(s->rows[par], rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (dev_malloc((void **)&s->err, sizeof(int)) != cudaSuccess) {
        s->oom = true;
        return;
    }
    cudaMemset(s->err, 0, sizeof(int));
    for (const void *k : {(const void *)k_gemm_split<0>, (const void *)k_gemm_split<1>, (const void *)k_gemm_pair<0>,
                          (const void *)k_gemm_pair<1>, (const void *)k_gemm_pair<0, true>,
                          (const void *)k_gemm_pair<1, true>})
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaGetLastError();
    s->ok = true;
}

void ten_release(ColState *s);

void col_release(mpi_ffl_handle *h) {
    ColState *s = cs(h);
    if (!s) return;
    ten_release(s);
    for (int p = 0; p < 2; ++p) {
        for (int f = 0; f < 2; ++f)
            for (Packed *pk : {&s->evf_f[f][p], &s->evf_a[f][p], &s->full_f[f][p], &s->full_a[f][p]})
                if (pk->dev) dev_free(pk->dev);
        if (s->rows[p]) dev_free(s->rows[p]);
        for (int dir = 0; dir < 2; ++dir)
            if (s->apk[dir][p]) dev_free(s->apk[dir][p]);
    }
    if (s->err) dev_free(s->err);
    delete s;
    h->col_state = nullptr;
}

void col_mark_psf_stale(mpi_ffl_handle *h) {
    if (ColState *s = cs(h)) s->psf_stale = true;
}

bool col_psf_stale(const mpi_ffl_handle *h) {
    const ColState *s = cs(h);
    return s && s->psf_stale;
}

bool col_init_oom(const mpi_ffl_handle *h) {
    const ColState *s = cs(h);
    return s && s->oom;
}

int col_take_error(mpi_ffl_handle *h) {
    ColState *s = cs(h);
    if (!s || !s->err) return 0;
    int v = 0;
    cudaMemcpy(&v, s->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (v) cudaMemset(s->err, 0, sizeof(int));
    return v;
}

// Splits the A rows of the full line stage once (k_pack_lines, one launch for both
// trajectories) and points the problems at them: the loader warp then stages A with one
// bulk copy per half next to B's, and the producer warps only run the epilogue (the
// launch then takes the GEMM without the producers' split, a smaller kernel).

static void pack_full(mpi_ffl_handle *h, int dir, const float *in, GemmArgs *g, cudaStream_t st,
                      bool prepacked = false) {
    ColState *s = cs(h);
    PackLines pl[2] = {};
    for (int par = 0; par < s->n_par; ++par) {
        pl[par] = PackLines{g[par].arow, g[par].M, s->apk[dir][par]};
        g[par].apk = s->apk[dir][par];
        g[par].apk_jg = 1;
        g[par].apk_gper = (g[par].M + 7) / 8;
        g[par].apk_cbase = 0;
        g[par].apk_cstep = 0;
    }
    if (prepacked) return;
    const int G = (std::max(g[0].M, s->n_par > 1 ? g[1].M : 0) + 7) / 8;
    const long long work = (long long)G * g[0].nkc * 64;
    const int blocks = (int)std::min<long long>(4 * 152, (work + 255) / 256);
    launch_dependent(k_pack_lines, dim3(std::max(1, blocks), s->n_par), dim3(256), 0, st, in, g[0].lda, g[0].Ka,
                     g[0].nkc, g[0].tf32, pl[0], pl[1]);
    h->launches++;  // a second kernel inside the caller's timed GEMM stage
}

// fine -> data (W) or proj -> data (W H), gain per line
bool col_prepack_targets(const mpi_ffl_handle *h, ProjPack *p) {
    const ColState *s = cs(h);
    const bool tf32 = h->precision == MPI_FFL_PREC_TF32;
    if (!s || !s->ok || s->psf_stale || h->d.N % (tf32 ? kBK / 2 : kBK) != 0) return false;
    *p = ProjPack{};
    p->n_par = s->n_par;
    p->tf32 = tf32 ? 1 : 0;
    for (int par = 0; par < s->n_par; ++par) {
        p->out[par] = s->apk[0][par];
        p->G[par] = (s->nrows[par] + 7) / 8;
        p->nrow[par] = s->nrows[par] / h->d.M;
    }
    return true;
}

void col_forward(mpi_ffl_handle *h, const float *in, bool full, const float *gain, float *data, cudaStream_t st,
                 bool prepacked) {
    ColState *s = cs(h);
    const Dims &d = h->d;
    GemmArgs g[2];
    const Packed *B[2];
    const int f = h->precision == MPI_FFL_PREC_TF32 ? 1 : 0;
    for (int par = 0; par < s->n_par; ++par) {
        B[par] = full ? &s->full_f[f][par] : &s->evf_f[f][par];
        g[par] = make_args(h, in, full ? d.N : d.Ne, full ? d.N : d.Ne, s->rows[par], s->nrows[par], *B[par], data,
                           2 * d.nb, s->rows[par], 2 * d.nb, gain, d.Nz);
    }
    if (full) pack_full(h, 0, in, g, st, prepacked);
    launch_problems(g, B, s->n_par, st);
}

// data -> fine (W^T) or data -> proj ((W H)^T), gain per line
void col_adjoint(mpi_ffl_handle *h, const float *data, bool full, const float *gain, float *out, cudaStream_t st) {
    ColState *s = cs(h);
    const Dims &d = h->d;
    GemmArgs g[2];
    const Packed *B[2];
    const int f = h->precision == MPI_FFL_PREC_TF32 ? 1 : 0;
    const int nout = full ? d.N : d.Ne;
    for (int par = 0; par < s->n_par; ++par) {
        B[par] = full ? &s->full_a[f][par] : &s->evf_a[f][par];
        g[par] = make_args(h, data, 2 * d.nb, 2 * d.nb, s->rows[par], s->nrows[par], *B[par], out, nout, s->rows[par],
                           nout, gain, d.Nz);
    }
    if (full) pack_full(h, 1, data, g, st);
    launch_problems(g, B, s->n_par, st);
}

size_t gemm_args_size() { return sizeof(GemmArgs); }

// Full-GEMM line stage (W H or its transpose) of several handles in one launch.
// args/items are host staging arrays; dargs/ditems their device copies (same
// layout), already uploaded by the caller before this launch runs.
int col_batch_prepare(mpi_ffl_handle *const *hs, const float *const *in, float *const *out, const int *const *done,
                      int n, bool adjoint, void *args, int4 *items, int arg_cap, int item_cap, int &n_items,
                      size_t &smem, uint32_t &tmem_cols) {
    GemmArgs *a = reinterpret_cast<GemmArgs *>(args);
    int np = 0;
    n_items = 0;
    smem = 0;
    tmem_cols = 32;
    for (int j = 0; j < n; ++j) {
        if (np + 2 > arg_cap) return -1;
        const int base_items = n_items;
        const int k = gemm_problems(hs[j], adjoint, in[j], out[j], done[j], a + np, items, item_cap, n_items);
        if (k < 0) return -1;
        for (int i = base_items; i < n_items; ++i) items[i].x += np;
        for (int i = 0; i < k; ++i) {
            smem = std::max(smem, (size_t)a[np + i].stages * (2u * kBM * kBK * 2 + 2u * a[np + i].BN * kBK * 2) + 256);
            tmem_cols = std::max(tmem_cols, a[np + i].tmem_cols);
        }
        np += k;
    }
    return np;
}

void col_batch_launch(const void *dargs, const int4 *ditems, int n_items, size_t smem, uint32_t tmem_cols,
                      cudaStream_t st) {
    if (n_items <= 0) return;
    static int n_sm = 0;
    if (!n_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gemm_batch, kGemmThreads, smem + 16) != cudaSuccess ||
        per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    per = std::min(per, (int)(512 / std::max(32u, tmem_cols)));  // the TMEM columns of an SM
    const int grid = std::max(1, std::min(n_items, per * n_sm));
    k_gemm_batch<<<grid, kGemmThreads, smem + 16, st>>>(reinterpret_cast<const GemmArgs *>(dargs), ditems, n_items,
                                                        tmem_cols, (uint32_t)smem);
}

void col_batch_init() {
    cudaFuncSetAttribute(k_gemm_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

// ============================================================ tensor PSF (slices coupled)
// With the in-plane tensor PSF (Appendix B, Eq. (31): an x drive read by a collinear
// coil takes h_uu(u, z) = 3 [L'(xi) u^2/rho^2 + (L(xi)/xi) z^2/rho^2], xi = rho / a) the
// PSF-convolved projection of line l mixes every slice z': c_l = sum_z' H_{l-z'} b.p_z',
// with H_d[e][i] = h_uu(u_lo + e/Q - i, d). Folded with the line operator W_par of the
// line's trajectory, line l's data are
//     data[m][l] = g_m sum_z' W_{par(l), l-z'} (b . p)[m][z'],    W_{par,d} = W_par H_d,
// one 2 n_b x N matrix per trajectory and slice offset (H_d is even in d). Stacked by
// offset, T_par[t] = W_{par, Nz-1-t} (t = 0 .. 2 Nz - 2), line l is one GEMM whose K
// runs over all slices (z', i) and whose B is the window t = Nz-1-l .. 2Nz-2-l of
// T_par; its rows are the angles. The transpose is one GEMM per slice z' whose K runs
// over all lines (l, o): B is the window t = Nz-1-z' .. 2Nz-2-z' of Tadj_s[t] =
// W_{par(l), t-(Nz-1)}^T, where line l = z' + t - (Nz-1) has parity (s + t - Nz + 1) & 1
// for slices of parity s.
//
// The rows of one such GEMM are the M angles only, so J = 128 / M lines of one
// trajectory share a problem: line l + step j (step = 2 with zig-zag, else 1) reads the
// window of line l shifted by step j slices, which is the same window applied to the
// projection shifted by step j slices. Row (j, m) of the problem whose last line is
// l_J reads the coil-weighted projection, padded with step (J - 1) zero slices in
// front, from slice step (j + J - J_g) on; the window starts at t = Nz - 1 - l_J and
// spans Nz + step (J - 1) slices. The tables carry step (J - 1) zero slices at both
// ends so that a partial group keeps the same extent (its missing rows write
// nothing). The transpose groups slices the same way.
namespace {

constexpr int kTenSplitK = 4096; // K per problem at most (64 bf16 chunks: 32 per accumulator)

// N tile: the fewest tiles of at most 256 columns (one MMA), rounded up to 16. Fewer
// tiles fetch the A rows fewer times; one block per SM holds up to 512 TMEM columns, two
// accumulators of 256 or three of 160.
int ten_bn(int Nv) {
    const int tiles = (Nv + 255) / 256;
    return std::min(256, ((Nv + tiles - 1) / tiles + 15) / 16 * 16);
}

struct TensorState {
    int fmt = -1;              // operand format of the packed tables (0 bf16, 1 tf32)
    Packed fwd[2], adj[2];     // T per trajectory (forward), Tadj per slice parity (adjoint)
    int Np = 0, Op = 0;        // K per slice (forward) and per line (adjoint), multiples of 64
    int step = 1, J = 1;       // line step of one trajectory; lines per problem
    int Zp = 0, P0 = 0;        // padded slices per angle (a multiple of step), leading zeros
    int Tpre = 0;              // zero offsets in front of and behind each table (step (J - 1))
    double *Wd = nullptr;      // [n_par][Nz][2 n_b][N], offsets d >= 0
    int M8 = 0;                // angles rounded up to a multiple of 8 (rows of a shift j)
    uint8_t *apk_f = nullptr;  // split A of the forward: coil-weighted projections, padded
    uint8_t *apk_a = nullptr;  // split A of the adjoint: data rows, padded
    int cm[2] = {0, 0};        // K chunks per angle row of apk_f / apk_a (current format)
    int nsplit[2] = {1, 1};    // K splits of the forward and adjoint problems
    int ksplit[2] = {0, 0};    // K per split (a multiple of 64)
    float *c_fwd = nullptr;    // [nsplit][M][Nz][2 n_b] partial sums
    float *c_adj = nullptr;    // [nsplit][M][Nz][N] partial sums
    int *idx = nullptr;        // per problem group: M8 J A rows, then M8 J C rows
    GemmArgs *dargs = nullptr; // forward problems, then adjoint problems
    int n_prob_f = 0;
    int4 *ditems = nullptr;    // forward items, then adjoint items
    int n_items_f = 0, n_items_a = 0;
    size_t smem[2] = {0, 0};   // dynamic shared memory of the forward and adjoint launches
    uint32_t cols[2] = {32, 32};  // TMEM columns a block of the forward and adjoint launches holds
};

// W_{par,d}[o][i] = sum_e W_par[o][e] g_d[e - D - Q i - kmin] in FP64 (g_d[k - kmin] =
// h_uu(k / Q, d)). A block takes 8 rows o, 128 columns i, one offset and trajectory;
// e runs in tiles of 256 staged in shared memory with the g values they meet.
constexpr int kWdRows = 8, kWdCols = 128, kWdTile = 256;

__global__ void __launch_bounds__(kWdCols) k_tensor_wd(const double *__restrict__ W, const double *__restrict__ g,
                                                       double *__restrict__ Wd, int R, int Ne, int N, int Nz, int D,
                                                       int Q, int kmin, int Lk) {
    __shared__ double sw[kWdRows][kWdTile];
    extern __shared__ double sg[];  // kWdTile + Q (kWdCols - 1) values of g_d
    const int ncb = (N + kWdCols - 1) / kWdCols;
    const int o0 = (blockIdx.x / ncb) * kWdRows, i0 = (blockIdx.x % ncb) * kWdCols;
    const int d = blockIdx.y, par = blockIdx.z;
    const int il = threadIdx.x, i = i0 + il;
    const double *Wp = W + (size_t)par * R * Ne;
    const double *gd = g + (size_t)d * Lk;
    const int span = kWdTile + Q * (kWdCols - 1);
    double acc[kWdRows];
#pragma unroll
    for (int r = 0; r < kWdRows; ++r) acc[r] = 0.0;
    for (int e0 = 0; e0 < Ne; e0 += kWdTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kWdRows * kWdTile; t += blockDim.x) {
            const int r = t / kWdTile, e = e0 + t % kWdTile;
            sw[r][t % kWdTile] = (o0 + r < R && e < Ne) ? Wp[(size_t)(o0 + r) * Ne + e] : 0.0;
        }
        // k = e - D - Q i runs from kb (e = e0, i = i0 + kWdCols - 1) upwards
        const int kb = e0 - D - Q * (i0 + kWdCols - 1) - kmin;
        for (int t = threadIdx.x; t < span; t += blockDim.x) {
            const int k = kb + t;
            sg[t] = (k >= 0 && k < Lk) ? gd[k] : 0.0;
        }
        __syncthreads();
        const double *gl = sg + Q * (kWdCols - 1 - il);
        for (int e = 0; e < kWdTile; ++e) {
            const double gv = gl[e];
#pragma unroll
            for (int r = 0; r < kWdRows; ++r) acc[r] = fma(sw[r][e], gv, acc[r]);
        }
    }
    if (i < N)
        for (int r = 0; r < kWdRows; ++r)
            if (o0 + r < R) Wd[(((size_t)par * Nz + d) * R + o0 + r) * N + i] = acc[r];
}

// Forward table value T_par[n = o][k = (t + Tpre) Np + i] and adjoint table value
// Tadj_s[n = i][k = (t + Tpre) Op + o], read from W_{par,|d|} (zero past |d| = Nz - 1).
struct TenFwdSrc {
    const double *Wd;
    int par, Nz, R, N, Np, Tpre;
    __device__ double operator()(int n, long long k) const {
        const int ts = (int)(k / Np), i = (int)(k - (long long)ts * Np);
        const int d = abs(Nz - 1 - (ts - Tpre));
        if (i >= N || d > Nz - 1) return 0.0;
        return Wd[(((size_t)par * Nz + d) * R + n) * N + i];
    }
};
struct TenAdjSrc {
    const double *Wd;
    int s, n_par, Nz, R, N, Op, Tpre;
    __device__ double operator()(int n, long long k) const {
        const int ts = (int)(k / Op), o = (int)(k - (long long)ts * Op);
        const int dd = ts - Tpre - (Nz - 1);
        if (o >= R || abs(dd) > Nz - 1) return 0.0;
        const int par = n_par == 1 ? 0 : ((dd + s) & 1);
        return Wd[(((size_t)par * Nz + abs(dd)) * R + o) * N + n];
    }
};

__device__ __forceinline__ uint16_t bf16_bits_dev(double x) {
    const uint32_t u = __float_as_uint((float)x);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ uint32_t tf32_bits_dev(double x) {
    return (__float_as_uint((float)x) + 0x1000u) & 0xFFFFE000u;
}

// pack_b on the device: one thread per (tile, chunk, row, K element) of the canonical
// layout; hi = round(v), lo = round(v - hi), in bf16 or tf32.
template <class Src>
__global__ void k_pack_b(Src src, int Nv, long long Kv, int BN, int ntile, int nkc, int tf32, uint8_t *out) {
    const int kpc = tf32 ? kBK / 2 : kBK;
    const size_t blk = (size_t)BN * kBK * 2;
    const size_t total = (size_t)ntile * nkc * BN * kpc;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int kl = (int)(idx % kpc);
        size_t r = idx / kpc;
        const int nl = (int)(r % BN);
        r /= BN;
        const int kc = (int)(r % nkc), t = (int)(r / nkc);
        const int n = t * BN + nl;
        const long long k = (long long)kc * kpc + kl;
        const double v = (n < Nv && k < Kv) ? src(n, k) : 0.0;
        uint8_t *hi = out + ((size_t)t * nkc + kc) * 2 * blk;
        uint8_t *lo = hi + blk;
        if (tf32) {
            const uint32_t hb = tf32_bits_dev(v);
            const uint32_t lb = tf32_bits_dev(v - (double)__uint_as_float(hb));
            const size_t off = (size_t)(nl / 8) * 1024 + (kl / 4) * 128 + (nl % 8) * 16 + (kl % 4) * 4;
            *reinterpret_cast<uint32_t *>(hi + off) = hb;
            *reinterpret_cast<uint32_t *>(lo + off) = lb;
        } else {
            const uint16_t hb = bf16_bits_dev(v);
            const uint16_t lb = bf16_bits_dev(v - (double)__uint_as_float((uint32_t)hb << 16));
            const size_t off = (size_t)(nl / 8) * 1024 + (kl / 8) * 128 + (nl % 8) * 16 + (kl % 8) * 2;
            *reinterpret_cast<uint16_t *>(hi + off) = hb;
            *reinterpret_cast<uint16_t *>(lo + off) = lb;
        }
    }
}

// A operand of the tensor-PSF GEMMs, split once per call: row m (angle) of the padded
// block holds K = Zp * per values, value (zp, c) = b[z][c] in[(m Nz + z) ncols + c] for
// z = zp - P0 in [0, Nz) and c < ncols, else 0 (b NULL: 1). 1 KB blocks per (group of 8
// angles, K chunk, half), ordered [chunk][hi, lo][group], each in the canonical layout
// the producer warps write: core-matrix column kg at kg * 128, row r7 at r7 * 16. One
// thread per 16-byte row of a block (8 bf16 or 4 tf32 values), split as the producers
// split.
__global__ void __launch_bounds__(256) k_pack_rows(const float *__restrict__ in, const float *__restrict__ coil,
                                                   int M, int Nz, int ncols, int per, int P0, int Zp, int cm,
                                                   int tf32, uint8_t *__restrict__ out) {
    const int kpc = tf32 ? kBK / 2 : kBK, epk = tf32 ? 4 : 8;
    const long long total = (long long)((M + 7) / 8) * cm * 64;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int kg = (int)(t & 7), r7 = (int)((t >> 3) & 7);
        const long long gc = t >> 6;  // block: (angle group, chunk)
        const int c = (int)(gc % cm), gq = (int)(gc / cm);
        const int m = 8 * gq + r7;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            v[e] = 0.f;
            if (e < epk && m < M) {
                const long long k = (long long)c * kpc + kg * epk + e;
                const int zp = (int)(k / per), col = (int)(k - (long long)zp * per);
                const int z = zp - P0;
                if (z >= 0 && z < Nz && col < ncols) {
                    v[e] = __ldg(in + ((size_t)m * Nz + z) * ncols + col);
                    if (coil) v[e] *= __ldg(coil + (size_t)z * ncols + col);
                }
            }
        }
        uint4 hi, lo;
        if (tf32) {
            const float f[4] = {v[0], v[1], v[2], v[3]};
            split4_tf32(f, hi, lo);
        } else {
            split8(v, hi, lo);
        }
        const int G = (M + 7) / 8;
        const uint32_t off = (uint32_t)kg * 128u + (uint32_t)r7 * 16u;
        *reinterpret_cast<uint4 *>(out + ((2 * (size_t)c) * G + gq) * 1024u + off) = hi;
        *reinterpret_cast<uint4 *>(out + ((2 * (size_t)c + 1) * G + gq) * 1024u + off) = lo;
    }
}

template <class Src>
bool pack_dev(Packed &p, Src src, int Nv, long long Kv, int BN, int tf32) {
    const int kpc = tf32 ? kBK / 2 : kBK;
    p.BN = BN;
    p.ntile = (Nv + BN - 1) / BN;
    p.nkc = (int)((Kv + kpc - 1) / kpc);
    const size_t bytes = (size_t)p.ntile * p.nkc * 2 * BN * kBK * 2;
    if (p.dev) dev_free(p.dev);
    p.dev = nullptr;
    if (dev_malloc((void **)&p.dev, bytes) != cudaSuccess) {
        p.dev = nullptr;
        cudaGetLastError();
        return false;
    }
    k_pack_b<Src><<<4 * 152 * 8, 256>>>(src, Nv, Kv, BN, p.ntile, p.nkc, tf32, p.dev);
    return cudaGetLastError() == cudaSuccess;
}

// h_uu at in-plane offset (u, z) voxels; a = FWHM / (2 x_h)
double h_uu_host(double u, double z, double a) {
    const double rho2 = u * u + z * z;
    if (rho2 == 0.0) return 1.0;
    const double xi = std::sqrt(rho2) / a;
    double lx;  // L(xi) / xi
    if (xi < 0.05) {
        const double x2 = xi * xi;
        lx = 1.0 / 3.0 - x2 / 45.0 + 2.0 * x2 * x2 / 945.0 - x2 * x2 * x2 / 4725.0;
    } else {
        lx = (1.0 / std::tanh(xi) - 1.0 / xi) / xi;
    }
    return 3.0 * (langevin_d1_host(xi) * u * u / rho2 + lx * z * z / rho2);
}

template <class T>
bool talloc(T **p, size_t n) {
    if (dev_malloc((void **)p, std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return false;
    }
    return true;
}

// W_{par,d} for d = 0 .. Nz-1 from W_par and the tensor PSF (FP64, on the device).
bool ten_build_wd(const mpi_ffl_handle *h, ColState *s, TensorState *t) {
    const Dims &d = h->d;
    const int R = 2 * d.nb;
    const int kmin = -d.D - d.Q * (d.N - 1), Lk = d.Ne + d.Q * (d.N - 1);
    const double a = h->fwhm / (2.0 * langevin_half_point_host());
    std::vector<double> g((size_t)d.Nz * Lk);
    for (int dz = 0; dz < d.Nz; ++dz)
        for (int k = 0; k < Lk; ++k) g[(size_t)dz * Lk + k] = h_uu_host((double)(k + kmin) / d.Q, dz, a);
    double *dW = nullptr, *dg = nullptr;
    bool ok = talloc(&dW, (size_t)s->n_par * R * d.Ne) && talloc(&dg, g.size());
    if (ok && !t->Wd) ok = talloc(&t->Wd, (size_t)s->n_par * d.Nz * R * d.N);
    if (ok) {
        for (int par = 0; par < s->n_par; ++par)
            cudaMemcpy(dW + (size_t)par * R * d.Ne, s->W[par].data(), (size_t)R * d.Ne * sizeof(double),
                       cudaMemcpyHostToDevice);
        cudaMemcpy(dg, g.data(), g.size() * sizeof(double), cudaMemcpyHostToDevice);
        const int ncb = (d.N + kWdCols - 1) / kWdCols;
        const size_t smem = sizeof(double) * (kWdTile + d.Q * (kWdCols - 1));
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_tensor_wd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tensor_wd<<<dim3(((R + kWdRows - 1) / kWdRows) * ncb, d.Nz, s->n_par), kWdCols, smem>>>(
            dW, dg, t->Wd, R, d.Ne, d.N, d.Nz, d.D, d.Q, kmin, Lk);
        ok = cudaDeviceSynchronize() == cudaSuccess;
    }
    if (dW) dev_free(dW);
    if (dg) dev_free(dg);
    cudaGetLastError();
    return ok;
}

// Line (slice) groups of one trajectory (slice parity): first line and count.
std::vector<int2> ten_groups(const Dims &d, int step, int J) {
    std::vector<int2> g;
    for (int p = 0; p < step; ++p)
        for (int l = p; l < d.Nz; l += step * J) g.push_back(make_int2(l, std::min(J, (d.Nz - 1 - l) / step + 1)));
    return g;
}

// Packed tables, problems and items for operand format fmt.
bool ten_prepare(const mpi_ffl_handle *h, ColState *s, TensorState *t, int fmt) {
    const Dims &d = h->d;
    const int R = 2 * d.nb;
    const int kpc = fmt ? kBK / 2 : kBK;
    const long long tslices = 2LL * d.Nz - 1 + 2LL * t->Tpre;  // zero offsets at both ends
    for (int par = 0; par < s->n_par; ++par)
        if (!pack_dev(t->fwd[par], TenFwdSrc{t->Wd, par, d.Nz, R, d.N, t->Np, t->Tpre}, R, tslices * t->Np,
                      ten_bn(R), fmt))
            return false;
    for (int sp = 0; sp < s->n_par; ++sp)
        if (!pack_dev(t->adj[sp], TenAdjSrc{t->Wd, sp, s->n_par, d.Nz, R, d.N, t->Op, t->Tpre}, d.N,
                      tslices * t->Op, ten_bn(d.N), fmt))
            return false;
    if (cudaDeviceSynchronize() != cudaSuccess) return false;
    const std::vector<int2> groups = ten_groups(d, t->step, t->J);
    const int rows = t->M8 * t->J;  // tile rows (j, m), m padded to M8
    t->cm[0] = t->Zp * t->Np / kpc;
    t->cm[1] = t->Zp * t->Op / kpc;
    std::vector<int> idx(groups.size() * 2 * 2 * rows);
    std::vector<GemmArgs> args;
    std::vector<int4> items[2];
    const int mtiles = (rows + kBM - 1) / kBM;
    const int span = d.Nz + t->step * (t->J - 1);  // window slices (lines)
    // one block per SM (it measured faster than two for these long-K problems), so the
    // pipeline takes as many stages as fit: A and B both arrive by bulk copies
    auto deep = [](int BN, int &stages) {
        const size_t stage = 2u * kBM * kBK * 2 + 2u * BN * kBK * 2;
        stages = (int)std::max<size_t>(2, std::min<size_t>(4, (220u * 1024u - 256u) / stage));
        return stages * stage + 256;
    };
    int st_dir[2] = {0, 0};
    t->smem[0] = t->smem[1] = std::max(deep(t->fwd[0].BN, st_dir[0]), deep(t->adj[0].BN, st_dir[1]));
    for (int dir = 0; dir < 2; ++dir) {
        const int per = dir ? t->Op : t->Np;  // K per line (adjoint) or per slice (forward)
        const int BN = dir ? t->adj[0].BN : t->fwd[0].BN;
        const size_t blk = (size_t)BN * kBK * 2;
        const int stages = st_dir[dir];
        const int base = (int)args.size();
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            const int l0 = groups[gi].x, Jg = groups[gi].y;
            const int llast = l0 + t->step * (Jg - 1);
            int *ar = idx.data() + ((size_t)dir * groups.size() + gi) * 2 * rows;
            int *cr = ar + rows;
            for (int j = 0; j < t->J; ++j)
                for (int m = 0; m < t->M8; ++m) {
                    // row (j, m): angle m's padded block from slice step (j + J - Jg); the
                    // A row list only gives the gain (A comes pre-split)
                    ar[j * t->M8 + m] = m < d.M ? m : 0;
                    cr[j * t->M8 + m] = (j < Jg && m < d.M) ? m * d.Nz + l0 + t->step * j : -1;
                }
            const int *dar = t->idx + (ar - idx.data());
            const int *dcr = t->idx + (cr - idx.data());
            // the window starts at t = Nz - 1 - llast (table slice + Tpre)
            const long long kwin = (long long)(d.Nz - 1 - llast + t->Tpre) * per;
            const Packed &B = dir ? t->adj[s->n_par == 1 ? 0 : (l0 & 1)] : t->fwd[s->n_par == 1 ? 0 : (l0 & 1)];
            for (int ks = 0; ks < t->nsplit[dir]; ++ks) {
                const int k0 = ks * t->ksplit[dir];
                const int kn = std::min(t->ksplit[dir], span * per - k0);
                GemmArgs g{};
                g.A = nullptr;
                g.lda = 0;
                g.Ka = kn;
                g.arow = dar;
                g.M = rows;
                g.apk = dir ? t->apk_a : t->apk_f;
                g.apk_jg = Jg;
                g.apk_gper = t->M8 / 8;
                g.apk_cbase = (t->step * (t->J - Jg) * per + k0) / kpc;
                g.apk_cstep = t->step * per / kpc;
                g.B = B.dev + (size_t)((kwin + k0) / kpc) * 2 * blk;
                g.BN = BN;
                g.nkc = kn / kpc;
                g.b_tstride = B.nkc;
                g.C = (dir ? t->c_adj : t->c_fwd) + (size_t)ks * d.M * d.Nz * (dir ? d.N : R);
                g.ldc = dir ? d.N : R;
                g.crow = dcr;
                g.Nc = dir ? d.N : R;
                g.rscale = h->t_gain;
                g.rdiv = 1;  // A row list = angle
                g.prec = h->precision;
                g.tf32 = fmt;
                g.stages = stages;
                // one block per SM: up to 512 TMEM columns, at most 4 accumulators
                g.acc_stride = (g.BN + 31) / 32 * 32;
                g.nacc = std::max(1, std::min({4, 512 / g.acc_stride, g.nkc}));
                {
                    const int cols = g.nacc * g.acc_stride;
                    g.tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
                }
                g.err = s->err;
                g.done = nullptr;
                t->cols[dir] = std::max(t->cols[dir], g.tmem_cols);
                const int pi = (int)args.size() - base;
                args.push_back(g);
                for (int mt = 0; mt < mtiles; ++mt)
                    for (int nt = 0; nt < B.ntile; ++nt) items[dir].push_back(make_int4(pi, mt, nt, 0));
            }
        }
        if (dir == 0) t->n_prob_f = (int)args.size();
    }
    if (cudaMemcpy(t->idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return false;
    // the adjoint items index their problems from the adjoint part of the arguments
    t->n_items_f = (int)items[0].size();
    t->n_items_a = (int)items[1].size();
    items[0].insert(items[0].end(), items[1].begin(), items[1].end());
    if (t->dargs) dev_free(t->dargs);
    if (t->ditems) dev_free(t->ditems);
    t->dargs = nullptr;
    t->ditems = nullptr;
    if (!talloc(&t->dargs, args.size()) || !talloc(&t->ditems, items[0].size())) return false;
    cudaMemcpy(t->dargs, args.data(), args.size() * sizeof(GemmArgs), cudaMemcpyHostToDevice);
    cudaMemcpy(t->ditems, items[0].data(), items[0].size() * sizeof(int4), cudaMemcpyHostToDevice);
    t->fmt = fmt;
    return cudaGetLastError() == cudaSuccess;
}

}  // namespace

void ten_release(ColState *s) {
    TensorState *t = s->ten;
    if (!t) return;
    for (int p = 0; p < 2; ++p)
        for (Packed *pk : {&t->fwd[p], &t->adj[p]})
            if (pk->dev) dev_free(pk->dev);
    for (void *p : {(void *)t->Wd, (void *)t->apk_f, (void *)t->apk_a, (void *)t->c_fwd, (void *)t->c_adj,
                    (void *)t->idx, (void *)t->dargs, (void *)t->ditems})
        if (p) dev_free(p);
    delete t;
    s->ten = nullptr;
}

int ten_init(mpi_ffl_handle *h) {
    ColState *s = cs(h);
    if (!s || !s->ok || s->W[0].empty()) return MPI_FFL_ERR_UNSUPPORTED;
    const Dims &d = h->d;
    const int R = 2 * d.nb;
    ten_release(s);
    TensorState *t = new TensorState();
    s->ten = t;
    t->Np = (d.N + kBK - 1) / kBK * kBK;
    t->Op = (R + kBK - 1) / kBK * kBK;
    t->step = s->n_par;
    t->M8 = (d.M + 7) / 8 * 8;
    t->J = std::max(1, std::min(kBM / t->M8, (d.Nz + t->step - 1) / t->step));
    t->P0 = t->step * (t->J - 1);
    t->Tpre = t->step * (t->J - 1);
    t->Zp = (d.Nz + 2 * t->P0 + t->step - 1) / t->step * t->step;
    // the accumulation in TMEM is not round-to-nearest, so its error grows with the MMAs
    // chained into one accumulator: K is split into parts of at most kTenSplitK, summed
    // in FP32 afterwards (in a fixed order)
    const int span = d.Nz + t->step * (t->J - 1);
    for (int dir = 0; dir < 2; ++dir) {
        const int K = span * (dir ? t->Op : t->Np);
        t->nsplit[dir] = (K + kTenSplitK - 1) / kTenSplitK;
        t->ksplit[dir] = ((K + t->nsplit[dir] - 1) / t->nsplit[dir] + kBK - 1) / kBK * kBK;
        t->nsplit[dir] = (K + t->ksplit[dir] - 1) / t->ksplit[dir];
    }
    const size_t ng = ten_groups(d, t->step, t->J).size();
    // split A: 2 KB per (8 angles, K chunk); a tf32 chunk holds 32 values, a bf16 one 64
    const size_t blocks_f = (size_t)(t->M8 / 8) * (t->Zp * t->Np / (kBK / 2));
    const size_t blocks_a = (size_t)(t->M8 / 8) * (t->Zp * t->Op / (kBK / 2));
    bool ok = talloc(&t->apk_f, blocks_f * 2048) && talloc(&t->apk_a, blocks_a * 2048) &&
              talloc(&t->c_fwd, (size_t)t->nsplit[0] * d.M * d.Nz * R) &&
              talloc(&t->c_adj, (size_t)t->nsplit[1] * d.M * d.Nz * d.N) &&
              talloc(&t->idx, ng * 2 * 2 * (size_t)t->M8 * t->J);
    ok = ok && ten_build_wd(h, s, t) && ten_prepare(h, s, t, h->precision == MPI_FFL_PREC_TF32 ? 1 : 0);
    if (!ok) {
        ten_release(s);
        cudaGetLastError();
        return MPI_FFL_ERR_OOM;
    }
    cudaFuncSetAttribute(k_gemm_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return MPI_FFL_OK;
}

bool ten_ready(const mpi_ffl_handle *h) {
    const ColState *s = cs(h);
    return s && s->ten;
}

int ten_refresh(mpi_ffl_handle *h, bool psf_changed) {
    ColState *s = cs(h);
    if (!s || !s->ten) return MPI_FFL_OK;
    TensorState *t = s->ten;
    const int fmt = h->precision == MPI_FFL_PREC_TF32 ? 1 : 0;
    if (psf_changed) {
        if (!ten_build_wd(h, s, t)) return MPI_FFL_ERR_CUDA;
        t->fmt = -1;
    }
    if (t->fmt != fmt && !ten_prepare(h, s, t, fmt)) return MPI_FFL_ERR_OOM;
    return MPI_FFL_OK;
}

void ten_pack(TensorState *t, const float *in, const float *coil, int M, int Nz, int ncols, int per, int dir,
              cudaStream_t st) {
    const long long total = (long long)(t->M8 / 8) * t->cm[dir] * 64;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    k_pack_rows<<<std::max(1, blocks), 256, 0, st>>>(in, coil, M, Nz, ncols, per, t->P0, t->Zp, t->cm[dir], t->fmt,
                                                    dir ? t->apk_a : t->apk_f);
}

// proj -> data: coil-weighted, padded A rows split once; the GEMM problems; sum of the K splits
void ten_forward(mpi_ffl_handle *h, const float *proj, const float *coil, float *data, cudaStream_t st) {
    ColState *s = cs(h);
    TensorState *t = s->ten;
    const Dims &d = h->d;
    const long long rows = (long long)d.M * d.Nz;
    ten_pack(t, proj, coil, d.M, d.Nz, d.N, t->Np, 0, st);
    // one block per item (each holds up to 512 TMEM columns, one block per SM)
    k_gemm_batch<<<t->n_items_f, kGemmThreads, t->smem[0] + 16, st>>>(t->dargs, t->ditems, t->n_items_f, t->cols[0],
                                                                      (uint32_t)t->smem[0]);
    launch_coil_pad(t->c_fwd, nullptr, data, rows, d.Nz, 2 * d.nb, 2 * d.nb, st, t->nsplit[0], rows * 2 * d.nb);
}

// data -> proj: padded data rows; the GEMM problems; sum of the K splits, coil weighting
void ten_adjoint(mpi_ffl_handle *h, const float *data, const float *coil, float *proj, cudaStream_t st) {
    ColState *s = cs(h);
    TensorState *t = s->ten;
    const Dims &d = h->d;
    const long long rows = (long long)d.M * d.Nz;
    ten_pack(t, data, nullptr, d.M, d.Nz, 2 * d.nb, t->Op, 1, st);
    k_gemm_batch<<<t->n_items_a, kGemmThreads, t->smem[1] + 16, st>>>(t->dargs + t->n_prob_f, t->ditems + t->n_items_f,
                                                                      t->n_items_a, t->cols[1], (uint32_t)t->smem[1]);
    launch_coil_pad(t->c_adj, coil, proj, rows, d.Nz, d.N, d.N, st, t->nsplit[1], rows * d.N);
}

}  // namespace mpiffl
