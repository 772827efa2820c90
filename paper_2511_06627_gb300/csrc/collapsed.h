// Collapsed line operator (collapsed.cu): S D_Gamma F V E (and optionally H) as one
// precomputed matrix per trajectory, applied with a split-bf16 tcgen05 GEMM.
#pragma once

#include "internal.h"

namespace mpiffl {

void col_init(mpi_ffl_handle *h);        // builds W and W H in double precision and uploads them
void col_release(mpi_ffl_handle *h);
bool col_supported(const mpi_ffl_handle *h);
int col_take_error(mpi_ffl_handle *h);   // 1 if a GEMM gave up on a bounded wait (clears it)
// full = false: fine -> data with W; full = true: proj -> data with W H (per-line gain)
void col_forward(mpi_ffl_handle *h, const float *in, bool full, const float *gain, float *data, cudaStream_t st);
void col_adjoint(mpi_ffl_handle *h, const float *data, bool full, const float *gain, float *out, cudaStream_t st);

// host-side model pieces shared with the table builders (api.cu)
double langevin_d1_host(double x);
double langevin_half_point_host();
void traj_point_host(const mpi_ffl_handle *h, int parity, int j, int &n, double &f, double &v);

}  // namespace mpiffl
