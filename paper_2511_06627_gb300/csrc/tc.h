// Tensor-core (tcgen05) path of the line stages: E V B fused with the band DFT
// (forward) and the band synthesis fused with the transposed resampling (adjoint).
#pragma once

#include "internal.h"

namespace mpiffl {

void tc_init(mpi_ffl_handle *h);                 // builds the operand tables
void tc_release(mpi_ffl_handle *h);
void tc_tables_changed(mpi_ffl_handle *h);      // PSF or gain tables were replaced
bool tc_supported(const mpi_ffl_handle *h);     // shapes the kernels accept
bool tc_init_oom(const mpi_ffl_handle *h);      // tc_init failed on a device allocation
void tc_forward_line(mpi_ffl_handle *h, const float *fine, const float *gain, float *data, cudaStream_t st);
int tc_take_error(mpi_ffl_handle *h);        // 1 if a tensor-core kernel timed out (clears it)
void tc_adjoint_line(mpi_ffl_handle *h, const float *data, const float *gain, float *fine, cudaStream_t st);

}  // namespace mpiffl
