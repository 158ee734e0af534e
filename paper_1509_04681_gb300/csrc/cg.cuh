// Sparse symmetric positive definite solves by conjugate gradient (the block regime of
// Section 4: columns of Sigma = Lambda^-1, and P = R Sigma as Lambda P^T = R^T); see cg.cu.
#pragma once

#include "common.cuh"

namespace cggm {

// Device scratch of pcg_solve for q rows and k right-hand sides (sizes in doubles):
// R, Z, P, AP: q k each; dinv: q; col: 6 k (per-column scalars); part: 2 kChunks k.
struct CgWork {
    double *R, *Z, *P, *AP, *dinv, *col, *part;
    int *err;
};
constexpr int kCgChunks = 64;
size_t cg_work_doubles(int64_t q, int64_t k);
CgWork cg_work_at(double *base, int *err, int64_t q, int64_t k);

// Validates a CSR matrix on the device (row pointers non-decreasing from 0 to nnz, columns
// in [0, q)); returns CGGM_EINVAL otherwise.
cggm_status csr_check(int64_t q, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                      int *err, cudaStream_t st);

// Solves A X = B (all device pointers; A q x q CSR, symmetric positive definite; B q x k
// row-major, or nullptr for the identity columns c0 .. c0 + k - 1; X q x k row-major).
// Jacobi-preconditioned CG in double on the k columns at once, until every column's
// residual norm is <= tol times its right-hand side's norm (CGGM_OK) or max_iter
// iterations (CGGM_EMAXITER).  A non-positive curvature p^T A p (A not positive definite)
// or a non-positive diagonal gives CGGM_ENOTPD.
cggm_status pcg_solve(int64_t q, const int64_t *row_ptr, const int32_t *col, const double *val,
                      int64_t k, const double *B, int64_t c0, double tol, int max_iter,
                      double *X, CgWork w, int *iters, double *resid, cudaStream_t st);

}  // namespace cggm
