// Double-precision dense Cholesky, log determinant, triangular solves and the inverse
// Sigma = Lambda^-1 = L^-T L^-1 (Section 2.3: Sigma is initialised through a Cholesky
// factorisation of Lambda; the Armijo test of Algorithm 1 needs log|Lambda + alpha D|
// and the positive-definiteness that the factorisation certifies).
#include "chol.cuh"
#include "dense.cuh"

namespace cggm {

namespace {
constexpr int NB = 64;

// Factor the diagonal block A[k0:k0+nb, k0:k0+nb] (lower) in place.  Writes log L_ii
// into logd[k0 + i].  A pivot that is not > 0 (or not finite) sets *err = DEV_NOTPD.
__global__ void __launch_bounds__(256)
potrf_diag_kernel(double *A, int64_t lda, int64_t k0, int nb, double *logd, int *err) {
    __shared__ double T[NB][NB + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        T[i][c] = (c <= i) ? A[(k0 + i) * lda + k0 + c] : 0.0;
    }
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (tid == 0) {
            const double d = T[j][j];
            if (!(d > 0.0) || !isfinite(d)) {
                s_bad = 1;
                T[j][j] = 1.0;  // keep the rest finite; the result is discarded
            } else {
                T[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        const double piv = T[j][j];
        for (int i = j + 1 + tid; i < nb; i += blockDim.x) T[i][j] /= piv;
        __syncthreads();
        const int m = nb - j - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int ii = j + 1 + e / m, cc = j + 1 + e % m;
            if (cc <= ii) T[ii][cc] -= T[ii][j] * T[cc][j];
        }
        __syncthreads();
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        if (c <= i) A[(k0 + i) * lda + k0 + c] = T[i][c];
    }
    for (int i = tid; i < nb; i += blockDim.x) logd[k0 + i] = log(T[i][i]);
    if (tid == 0 && s_bad) atomicCAS(err, 0, (int)DEV_NOTPD);
}

// Rows r >= r0 of the panel A[:, k0:k0+nb] <- A[r, k0:k0+nb] L_kk^-T  (solve L x = a per row)
__global__ void __launch_bounds__(128)
trsm_panel_kernel(int64_t n, double *A, int64_t lda, int64_t k0, int nb, int64_t r0) {
    __shared__ double L[NB][NB + 1];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e % nb;
        L[i][c] = (c <= i) ? A[(k0 + i) * lda + k0 + c] : 0.0;
    }
    __syncthreads();
    const int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double *row = A + r * lda + k0;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
        if (j < nb) {
            double v = row[j];
#pragma unroll
            for (int m = 0; m < NB; m++)
                if (m < j) v -= L[j][m] * x[m];
            x[j] = v / L[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < nb) row[j] = x[j];
}

// Forward substitution on one row block: B[i0:i0+rb, c] <- L_ii^-1 B[i0:i0+rb, c] for
// columns c < ncols (thread per column).
__global__ void __launch_bounds__(128)
trsv_block_kernel(const double *Lm, int64_t ldl, int64_t i0, int rb, double *B, int64_t ldb,
                  int64_t ncols) {
    __shared__ double L[NB][NB + 1];
    for (int e = threadIdx.x; e < rb * rb; e += blockDim.x) {
        const int i = e / rb, c = e % rb;
        L[i][c] = (c <= i) ? Lm[(i0 + i) * ldl + i0 + c] : 0.0;
    }
    __syncthreads();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    double x[NB];
#pragma unroll
    for (int j = 0; j < NB; j++) {
        if (j < rb) {
            double v = B[(i0 + j) * ldb + c];
#pragma unroll
            for (int m = 0; m < NB; m++)
                if (m < j) v -= L[j][m] * x[m];
            x[j] = v / L[j][j];
        }
    }
#pragma unroll
    for (int j = 0; j < NB; j++)
        if (j < rb) B[(i0 + j) * ldb + c] = x[j];
}

__global__ void zero_upper_kernel(int64_t n, double *A, int64_t lda) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        if (j > i) A[i * lda + j] = 0.0;
    }
}

__global__ void set_identity_kernel(int64_t n, double *A, int64_t lda) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        A[i * lda + j] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void sum_kernel(int64_t len, const double *x, double scale, double *out) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) s += x[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = scale * s;
}

inline unsigned grid_cap(int64_t len) {
    int64_t g = (len + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
}  // namespace

void cholesky_inplace(int64_t n, double *A, int64_t lda, double *logd, int *err,
                      cudaStream_t st) {
    for (int64_t k0 = 0; k0 < n; k0 += NB) {
        const int nb = (int)((n - k0) < NB ? (n - k0) : NB);
        note_launch();
        potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, nb, logd, err);
        const int64_t k1 = k0 + nb;
        if (k1 < n) {
            note_launch();
            trsm_panel_kernel<<<ceil_div(n - k1, 128), 128, 0, st>>>(n, A, lda, k0, nb, k1);
            // trailing lower update A[k1:, k1:] -= P P^T with P = A[k1:, k0:k1]
            gemm<double>(false, true, n - k1, n - k1, nb, -1.0, A + k1 * lda + k0, lda,
                         A + k1 * lda + k0, lda, 1.0, A + k1 * lda + k1, lda, st, /*tri=*/1);
        }
    }
    note_launch();
    zero_upper_kernel<<<grid_cap(n * n), 256, 0, st>>>(n, A, lda);
}

void logdet_from_logd(int64_t n, const double *logd, double *out, cudaStream_t st) {
    note_launch();
    sum_kernel<<<1, 1024, 0, st>>>(n, logd, 2.0, out);
}

void trsm_lower_inplace(int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                        int64_t ncols, bool lower_tri_rhs, cudaStream_t st) {
    for (int64_t i0 = 0; i0 < n; i0 += NB) {
        const int rb = (int)((n - i0) < NB ? (n - i0) : NB);
        // columns that can be nonzero in this row block of the solution: when the
        // right-hand side is lower triangular (inverse), only c < i0 + rb
        const int64_t nc = lower_tri_rhs ? ((i0 + rb) < ncols ? (i0 + rb) : ncols) : ncols;
        if (i0 > 0)
            gemm<double>(false, false, rb, nc, i0, -1.0, L + i0 * ldl, ldl, B, ldb, 1.0,
                         B + i0 * ldb, ldb, st);
        note_launch();
        trsv_block_kernel<<<ceil_div(nc, 128), 128, 0, st>>>(L, ldl, i0, rb, B, ldb, nc);
    }
}

void inverse_from_cholesky(int64_t n, const double *L, double *Sigma, double *work,
                           cudaStream_t st) {
    note_launch();
    set_identity_kernel<<<grid_cap(n * n), 256, 0, st>>>(n, work, n);
    trsm_lower_inplace(n, L, n, work, n, n, true, st);  // work = L^-1 (lower)
    // Sigma = W^T W, lower triangle, then mirror
    gemm<double>(true, false, n, n, n, 1.0, work, n, work, n, 0.0, Sigma, n, st, /*tri=*/1,
                 /*kdiag=*/1);
    symmetrize_lower<double>(n, Sigma, st);
}

}  // namespace cggm
