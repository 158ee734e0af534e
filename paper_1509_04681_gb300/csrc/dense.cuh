// Dense building blocks (SIMT GEMM, elementwise maps, double reductions).
#pragma once

#include "common.cuh"

namespace cggm {

// C[M x N] = alpha * op(A) op(B) + beta * C, all row-major.
//  op(A) = A (M x K, lda) or A^T (A stored K x M, lda) when transA;
//  op(B) = B (K x N, ldb) or B^T (B stored N x K, ldb) when transB.
//  tri: 0 = full C; 1 = only tiles meeting the lower triangle (i >= j) of C are computed
//  (others untouched).  kdiag = 1 declares op(A)(m, k) = 0 for k < m and op(B)(k, n) = 0
//  for k < n (W^T W with W lower triangular), so a tile at rows i0.., cols j0.. starts
//  its k loop at max(i0, j0).
template <typename T>
void gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, T alpha, const T *A,
          int64_t lda, const T *B, int64_t ldb, T beta, T *C, int64_t ldc,
          cudaStream_t st, int tri = 0, int kdiag = 0);

// y = a*x + b*y elementwise over len
template <typename T>
void axpby(int64_t len, T a, const T *x, T b, T *y, cudaStream_t st);

void convert_d2f(int64_t len, const double *x, float *y, cudaStream_t st);
// out = a x + z  (x, out double; z float)
void axpy_f2d(int64_t len, double a, const double *x, const float *z, double *out, cudaStream_t st);
void convert_f2d(int64_t len, const float *x, double *y, cudaStream_t st);

// out (cols x rows) = in^T (rows x cols), element type converted
template <typename Tin, typename Tout>
void transpose(int64_t rows, int64_t cols, const Tin *in, Tout *out, cudaStream_t st);

// R^T = Theta^T X^T for a sparse Theta held densely (p x q, row-major) and X^T (p x n,
// row-major), into R^T (q x n, row-major): R = X Theta costs O(n m_Theta) with Theta's
// nonzeros (Section 3.2) instead of the O(n p q) of a dense product.  Row j of R^T sums
// Theta_ij X^T_i over the nonzero Theta_ij in ascending i, one fused multiply-add at a
// time, so the result does not depend on the launch.
void theta_t_xt(int64_t p, int64_t q, int64_t n, const double *Th, const double *Xt, double *Rt,
                cudaStream_t st);

// Mirror the lower triangle of a square matrix into the upper one.
template <typename T>
void symmetrize_lower(int64_t n, T *A, cudaStream_t st);

// Copy the diagonal of A (n x n) into d (double).
template <typename T>
void diag_to_double(int64_t n, const T *A, double *d, cudaStream_t st);

// Double-precision reductions; results accumulate into *out (device), which the
// caller zeroes.  Deterministic order (fixed grid, block tree, ordered final pass).
struct Reducer {
    double *partial = nullptr;  // [kMaxBlocks]
    static const int kMaxBlocks = 1024;
};

// sum_i x_i * y_i
template <typename T>
void dot_d(int64_t len, const T *x, const T *y, double *partial, double *out, cudaStream_t st);
// sum |x_i| (skip the diagonal of an n x n matrix when n > 0)
template <typename T>
void l1_d(int64_t len, const T *x, int64_t n_diag_skip, double *partial, double *out,
          cudaStream_t st);

}  // namespace cggm
