// Collapsed line operator (collapsed.cu): S D_Gamma F V E (and optionally H) as one
// precomputed matrix per trajectory, applied with a split-bf16 (or split-tf32) tcgen05 GEMM.
#pragma once

#include "internal.h"

namespace mpiffl {

void col_init(mpi_ffl_handle *h);        // builds W and W H in double precision and uploads them
void col_release(mpi_ffl_handle *h);
bool col_supported(const mpi_ffl_handle *h);
bool col_init_oom(const mpi_ffl_handle *h);  // col_init failed on a device allocation
void col_mark_psf_stale(mpi_ffl_handle *h);  // the PSF changed: W H must be rebuilt before use
bool col_psf_stale(const mpi_ffl_handle *h);
int col_take_error(mpi_ffl_handle *h);   // 1 if a GEMM gave up on a bounded wait (clears it)
// full = false: fine -> data with W; full = true: proj -> data with W H (per-line gain).
// prepacked: the projector already wrote the full stage's A operand (col_prepack_targets).
void col_forward(mpi_ffl_handle *h, const float *in, bool full, const float *gain, float *data, cudaStream_t st,
                 bool prepacked = false);
// Where the projector may write the forward full stage's A operand (bf16 or tf32 hi +
// lo), or false when that stage does not take it (N not a multiple of the K chunk: 64
// bins in bf16, 32 in tf32).
bool col_prepack_targets(const mpi_ffl_handle *h, ProjPack *p);
void col_adjoint(mpi_ffl_handle *h, const float *data, bool full, const float *gain, float *out, cudaStream_t st);

// Batched full-GEMM line stages (continuous batching): fill host staging arrays of
// GEMM problems and (problem, m tile, n tile) items for handles hs[0..n); returns the
// number of problems or -1 when the capacities are too small, and in smem the dynamic
// shared memory the launch needs.
size_t gemm_args_size();
int col_batch_prepare(mpi_ffl_handle *const *hs, const float *const *in, float *const *out, const int *const *done,
                      int n, bool adjoint, void *args, int4 *items, int arg_cap, int item_cap, int &n_items,
                      size_t &smem, uint32_t &tmem_cols);
void col_batch_launch(const void *dargs, const int4 *ditems, int n_items, size_t smem, uint32_t tmem_cols,
                      cudaStream_t st);
void col_batch_init();

// Slice-coupled operator of the tensor PSF (Appendix B, Eq. (31)): per-offset folded
// line operators W_par H_d stacked by offset, one GEMM per line (forward) or per slice
// (adjoint). ten_init builds the tables (FP64 fold, then split operands for the
// handle's precision); ten_refresh rebuilds them after a PSF or precision change.
int ten_init(mpi_ffl_handle *h);
bool ten_ready(const mpi_ffl_handle *h);
int ten_refresh(mpi_ffl_handle *h, bool psf_changed);
void ten_forward(mpi_ffl_handle *h, const float *proj, const float *coil, float *data, cudaStream_t st);
void ten_adjoint(mpi_ffl_handle *h, const float *data, const float *coil, float *proj, cudaStream_t st);

// host-side model pieces shared with the table builders (api.cu)
double langevin_d1_host(double x);
double langevin_half_point_host();
void traj_point_host(const mpi_ffl_handle *h, int parity, int j, int &n, double &f, double &v);

}  // namespace mpiffl
