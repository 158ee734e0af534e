// Coordinate-list (COO) conversion of the parameters at the C boundary.
#pragma once

#include "common.cuh"

namespace cggm {

// A (rows x cols, row-major double, zeroed by the caller) += the listed entries; with `sym`
// the list is one triangle (row <= col) of a symmetric matrix and both A[r][c] and A[c][r]
// receive each off-diagonal value.  A bad index sets *err to DEV_BADINDEX, a non-finite
// value to DEV_NONFINITE.
void coo_scatter(int64_t nnz, const int32_t *row, const int32_t *col, const double *val,
                 int64_t rows, int64_t cols, bool sym, double *A, int *err, cudaStream_t st);

// val[e] = A[row[e]][col[e]].
void coo_gather(int64_t nnz, const int32_t *row, const int32_t *col, const double *A,
                int64_t cols, double *val, cudaStream_t st);

}  // namespace cggm
