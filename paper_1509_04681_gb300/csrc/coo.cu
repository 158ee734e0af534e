// Sparse (coordinate-list) exchange of Lambda and Theta at the C boundary: the paper keeps
// both parameters in sparse form (Section 5), Lambda by symmetry as one triangle.  The
// solver works on dense device copies; these kernels convert between the two.
#include "coo.cuh"

#include "dense.cuh"

namespace cggm {

namespace {

// A[r][c] += v for every listed entry (and A[c][r] += v when `sym` and r != c).  Rows and
// columns are checked against the matrix (and r <= c when `sym`), values for finiteness;
// a bad entry sets the status word and is skipped.  Repeated entries add up.
__global__ void coo_scatter_kernel(int64_t nnz, const int32_t *__restrict__ row,
                                   const int32_t *__restrict__ col,
                                   const double *__restrict__ val, int64_t rows, int64_t cols,
                                   bool sym, double *A, int *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = row[e], c = col[e];
        const double v = val[e];
        if (r < 0 || r >= rows || c < 0 || c >= cols || (sym && r > c)) {
            atomicCAS(err, 0, (int)DEV_BADINDEX);
            continue;
        }
        if (!isfinite(v)) {
            atomicCAS(err, 0, (int)DEV_NONFINITE);
            continue;
        }
        atomicAdd(A + r * cols + c, v);
        if (sym && r != c) atomicAdd(A + c * cols + r, v);
    }
}

__global__ void coo_gather_kernel(int64_t nnz, const int32_t *__restrict__ row,
                                  const int32_t *__restrict__ col, const double *__restrict__ A,
                                  int64_t cols, double *val) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        val[e] = A[(int64_t)row[e] * cols + col[e]];
}

unsigned grid_for(int64_t len) {
    const int64_t g = (len + 255) / 256, cap = (int64_t)sm_count() * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void coo_scatter(int64_t nnz, const int32_t *row, const int32_t *col, const double *val,
                 int64_t rows, int64_t cols, bool sym, double *A, int *err, cudaStream_t st) {
    if (nnz <= 0) return;
    note_launch();
    coo_scatter_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, row, col, val, rows, cols, sym, A,
                                                      err);
}

void coo_gather(int64_t nnz, const int32_t *row, const int32_t *col, const double *A,
                int64_t cols, double *val, cudaStream_t st) {
    if (nnz <= 0) return;
    note_launch();
    coo_gather_kernel<<<grid_for(nnz), 256, 0, st>>>(nnz, row, col, A, cols, val);
}

}  // namespace cggm
