// Inputs of the solve (Section 2.1): X and Y in the element types of cggm_dtype, brought
// into the solver's transposed double layout; int8 genotype columns standardised.
#pragma once

#include "common.cuh"

namespace cggm {

// Bytes per element of a cggm_dtype (0 for an unknown type).
size_t dtype_size(int dt);

// rows x cols row-major matrix src (device) of element type dt -> dst (device, double,
// cols x rows).  CGGM_I8_GENO: column k is standardised with its mean and population
// standard deviation over the rows, (x - mean_k) / sd_k, in double; a constant column
// becomes zero.  stats: device scratch of 2 cols doubles (I8_GENO only).
cggm_status load_input_transposed(const void *src, int dt, int64_t rows, int64_t cols,
                                  double *dst, double *stats, cudaStream_t st);

}  // namespace cggm
