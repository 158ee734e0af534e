// Double-precision Cholesky family (see chol.cu).
#pragma once

#include "common.cuh"

namespace cggm {

// In-place recursive blocked Cholesky of the n x n matrix A (row-major, lda): the lower
// triangle becomes L, the strict upper triangle is zeroed, logd[i] = log L_ii.
// Sets *err = DEV_NOTPD when a pivot is not positive.
void cholesky_inplace(int64_t n, double *A, int64_t lda, double *logd, int *err,
                      cudaStream_t st);

// *out = 2 sum_i logd[i]  (= log|Lambda|)
void logdet_from_logd(int64_t n, const double *logd, double *out, cudaStream_t st);

// B[0:n, 0:ncols] <- L^-1 B (recursive blocked forward substitution).  With
// lower_tri_rhs the right-hand side (and solution) is lower triangular.
void trsm_lower_inplace(int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                        int64_t ncols, bool lower_tri_rhs, cudaStream_t st);

// Sigma = L^-T L^-1 (full symmetric n x n).  work: n x n scratch.
void inverse_from_cholesky(int64_t n, const double *L, double *Sigma, double *work,
                           cudaStream_t st);

}  // namespace cggm
