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

// Rows r0 <= r < n of the panel A[:, k0:k0+nb] <- A[r, k0:k0+nb] L_kk^-T (solve L x = a per row)
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

// Recursive forms: every level halves the problem (at a multiple of NB) and does the
// off-diagonal work as one GEMM, so that most of the flops run in a few large GEMMs rather
// than in n / NB thin ones (a 64-row GEMM fills a fraction of the GPU).
namespace {
int64_t split_at(int64_t n) {
    const int64_t h = (n / 2 / NB) * NB;
    return h < NB ? NB : h;
}

// X L^T = A[r0:r1, c0:c0+w] in place, with L = A[c0:c0+w, c0:c0+w] (lower, factored).
void trsm_right_rec(int64_t r0, int64_t r1, int64_t c0, int64_t w, double *A, int64_t lda,
                    cudaStream_t st) {
    if (r1 <= r0) return;
    if (w <= NB) {
        note_launch();
        trsm_panel_kernel<<<ceil_div(r1 - r0, 128), 128, 0, st>>>(r1, A, lda, c0, (int)w, r0);
        return;
    }
    const int64_t w1 = split_at(w);
    trsm_right_rec(r0, r1, c0, w1, A, lda, st);
    // A[r0:r1, c0+w1 : c0+w] -= X1 L21^T
    gemm<double>(false, true, r1 - r0, w - w1, w1, -1.0, A + r0 * lda + c0, lda,
                 A + (c0 + w1) * lda + c0, lda, 1.0, A + r0 * lda + c0 + w1, lda, st);
    trsm_right_rec(r0, r1, c0 + w1, w - w1, A, lda, st);
}

// Factor A[k0:k0+n, k0:k0+n] (updates from the columns before k0 already applied).
void chol_rec(int64_t k0, int64_t n, double *A, int64_t lda, double *logd, int *err,
              cudaStream_t st) {
    if (n <= NB) {
        note_launch();
        potrf_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, (int)n, logd, err);
        return;
    }
    const int64_t n1 = split_at(n), k1 = k0 + n1, k2 = k0 + n;
    chol_rec(k0, n1, A, lda, logd, err, st);
    trsm_right_rec(k1, k2, k0, n1, A, lda, st);  // L21 = A21 L11^-T
    // A22 -= L21 L21^T (lower triangle)
    gemm<double>(false, true, k2 - k1, k2 - k1, n1, -1.0, A + k1 * lda + k0, lda,
                 A + k1 * lda + k0, lda, 1.0, A + k1 * lda + k1, lda, st, /*tri=*/1);
    chol_rec(k1, n - n1, A, lda, logd, err, st);
}

// Rows [r0, r0 + n) of B <- L^-1 B, the rows before r0 solved and applied.  With tri the
// right-hand side (and solution) is lower triangular: row i has no nonzero beyond column i.
void trsm_left_rec(int64_t r0, int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                   int64_t ncols, bool tri, cudaStream_t st) {
    const int64_t nc = tri ? ((r0 + n) < ncols ? (r0 + n) : ncols) : ncols;
    if (n <= NB) {
        note_launch();
        trsv_block_kernel<<<ceil_div(nc, 128), 128, 0, st>>>(L, ldl, r0, (int)n, B, ldb, nc);
        return;
    }
    const int64_t n1 = split_at(n);
    trsm_left_rec(r0, n1, L, ldl, B, ldb, ncols, tri, st);
    const int64_t nc1 = tri ? ((r0 + n1) < ncols ? (r0 + n1) : ncols) : ncols;
    // B[r0+n1 : r0+n] -= L[r0+n1 : r0+n, r0 : r0+n1] X[r0 : r0+n1]
    gemm<double>(false, false, n - n1, nc1, n1, -1.0, L + (r0 + n1) * ldl + r0, ldl,
                 B + r0 * ldb, ldb, 1.0, B + (r0 + n1) * ldb, ldb, st);
    trsm_left_rec(r0 + n1, n - n1, L, ldl, B, ldb, ncols, tri, st);
}
}  // namespace

void cholesky_inplace(int64_t n, double *A, int64_t lda, double *logd, int *err,
                      cudaStream_t st) {
    if (n <= 0) return;
    chol_rec(0, n, A, lda, logd, err, st);
    note_launch();
    zero_upper_kernel<<<grid_cap(n * n), 256, 0, st>>>(n, A, lda);
}

void logdet_from_logd(int64_t n, const double *logd, double *out, cudaStream_t st) {
    note_launch();
    sum_kernel<<<1, 1024, 0, st>>>(n, logd, 2.0, out);
}

void trsm_lower_inplace(int64_t n, const double *L, int64_t ldl, double *B, int64_t ldb,
                        int64_t ncols, bool lower_tri_rhs, cudaStream_t st) {
    if (n <= 0 || ncols <= 0) return;
    trsm_left_rec(0, n, L, ldl, B, ldb, ncols, lower_tri_rhs, st);
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
