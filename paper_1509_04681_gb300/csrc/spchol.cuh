// Numeric sparse Cholesky in double precision (see spchol.cu).
#pragma once

#include "common.cuh"

namespace cggm {

struct SpCholPlan;

// Symbolic analysis (host, symbolic.cpp) of the q x q pattern row_ptr/col and the device
// structures of the numeric factorisation; device memory on `device`.
cggm_status spchol_analyse(int device, int64_t q, const int64_t *row_ptr, const int32_t *col,
                           int ordering, const int32_t *perm_in, SpCholPlan **out);
void spchol_free(SpCholPlan *p);

// Factor the matrix whose CSR values (in the analysed entry order; host or device) are val;
// waits for the result.  CGGM_ENOTPD when a pivot is not positive.
cggm_status spchol_factor(SpCholPlan *p, const double *val, double *logdet_out, cudaStream_t st);

// Enqueue the factorisation of device values d_vals (no wait, no status read).
cggm_status spchol_factor_device(SpCholPlan *p, const double *d_vals, cudaStream_t st);

// X = A^-1 B (q x k row-major, host or device; B NULL: identity columns c0 .. c0 + k - 1).
cggm_status spchol_solve(SpCholPlan *p, int64_t k, const double *B, int64_t c0, double *X,
                         cudaStream_t st);

cggm_status spchol_export(SpCholPlan *p, int64_t *nsuper_out, int64_t *nblock_out,
                          int64_t *nnz_L_out, int32_t *perm_out, int64_t *super_start_out,
                          int64_t *rows_ptr_out, int32_t *rows_out, int64_t *block_ptr_out,
                          double *blocks_out, cudaStream_t st);

}  // namespace cggm
