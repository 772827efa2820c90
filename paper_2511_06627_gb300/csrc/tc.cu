// Tensor-core path of the line stages (not yet enabled for any shape).
#include "tc.h"

namespace mpiffl {

void tc_init(mpi_ffl_handle *) {}
void tc_release(mpi_ffl_handle *) {}
void tc_tables_changed(mpi_ffl_handle *) {}
bool tc_supported(const mpi_ffl_handle *) { return false; }
void tc_forward_line(mpi_ffl_handle *, const float *, const float *, float *, cudaStream_t) {}
void tc_adjoint_line(mpi_ffl_handle *, const float *, const float *, float *, cudaStream_t) {}

}  // namespace mpiffl
