// SIMT dense kernels: tiled GEMM (double or float), maps and deterministic reductions.
#include "dense.cuh"

#include <mutex>

namespace cggm {

int64_t &launch_counter() {
    static int64_t n = 0;
    return n;
}

int sm_count() {
    // cached per device (contexts on different devices may share the process)
    constexpr int kMaxDev = 64;
    static int counts[kMaxDev] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    if (dev < 0 || dev >= kMaxDev) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (counts[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        counts[dev] = n > 0 ? n : 1;
    }
    return counts[dev];
}

// ---------------------------------------------------------------------------------
// GEMM: 64x64 output tile per 256-thread block, 4x4 per thread, BK = 16.
// ---------------------------------------------------------------------------------
namespace {
constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256)
gemm_kernel(int64_t M, int64_t N, int64_t K, T alpha, const T *__restrict__ A, int64_t lda,
            const T *__restrict__ B, int64_t ldb, T beta, T *__restrict__ C, int64_t ldc,
            int tri, int kdiag) {
    const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
    if (tri == 1 && j0 > i0 + BM - 1) return;  // tile entirely above the diagonal
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tr = tid / 16, tc = tid % 16;  // thread's 4x4 sub-tile at rows tr*4, cols tc*4
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; a++)
#pragma unroll
        for (int b = 0; b < TN; b++) acc[a][b] = T(0);
    int64_t kbeg = 0;
    if (kdiag == 1) kbeg = (i0 > j0 ? i0 : j0);  // op(A)(m,k) = 0 for k < m, op(B)(k,n) = 0 for k < n
    for (int64_t k0 = kbeg; k0 < K; k0 += BK) {
        // load A tile: BM x BK elements, 256 threads, 4 each
#pragma unroll
        for (int r = 0; r < (BM * BK) / 256; r++) {
            const int e = tid + r * 256;
            int mm, kk;
            if (!TA) { mm = e / BK; kk = e % BK; }  // k contiguous in memory
            else { kk = e / BM; mm = e % BM; }     // m contiguous in memory
            const int64_t gm = i0 + mm, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < K) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int r = 0; r < (BN * BK) / 256; r++) {
            const int e = tid + r * 256;
            int nn, kk;
            if (TB) { nn = e / BK; kk = e % BK; }  // k contiguous
            else { kk = e / BN; nn = e % BN; }     // n contiguous
            const int64_t gn = j0 + nn, gk = k0 + kk;
            T v = T(0);
            if (gn < N && gk < K) v = TB ? B[gn * ldb + gk] : B[gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            T a[TM], b[TN];
#pragma unroll
            for (int x = 0; x < TM; x++) a[x] = As[kk][tr * TM + x];
#pragma unroll
            for (int y = 0; y < TN; y++) b[y] = Bs[kk][tc * TN + y];
#pragma unroll
            for (int x = 0; x < TM; x++)
#pragma unroll
                for (int y = 0; y < TN; y++) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < TM; x++) {
        const int64_t gm = i0 + tr * TM + x;
        if (gm >= M) continue;
#pragma unroll
        for (int y = 0; y < TN; y++) {
            const int64_t gn = j0 + tc * TN + y;
            if (gn >= N) continue;
            if (tri == 1 && gn > gm) continue;
            T *c = C + gm * ldc + gn;
            *c = (beta == T(0)) ? alpha * acc[x][y] : alpha * acc[x][y] + beta * *c;
        }
    }
}
}  // namespace

template <typename T>
void gemm(bool transA, bool transB, int64_t M, int64_t N, int64_t K, T alpha, const T *A,
          int64_t lda, const T *B, int64_t ldb, T beta, T *C, int64_t ldc, cudaStream_t st,
          int tri, int kdiag) {
    if (M <= 0 || N <= 0) return;
    dim3 grid(ceil_div(N, BN), ceil_div(M, BM));
    dim3 block(256);
    note_launch();
    if (!transA && !transB)
        gemm_kernel<T, false, false><<<grid, block, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, kdiag);
    else if (!transA && transB)
        gemm_kernel<T, false, true><<<grid, block, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, kdiag);
    else if (transA && !transB)
        gemm_kernel<T, true, false><<<grid, block, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, kdiag);
    else
        gemm_kernel<T, true, true><<<grid, block, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri, kdiag);
}
template void gemm<double>(bool, bool, int64_t, int64_t, int64_t, double, const double *, int64_t,
                           const double *, int64_t, double, double *, int64_t, cudaStream_t, int, int);
template void gemm<float>(bool, bool, int64_t, int64_t, int64_t, float, const float *, int64_t,
                          const float *, int64_t, float, float *, int64_t, cudaStream_t, int, int);

// ---------------------------------------------------------------------------------
// maps
// ---------------------------------------------------------------------------------
namespace {
template <typename T>
__global__ void axpby_kernel(int64_t len, T a, const T *x, T b, T *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
__global__ void axpy_f2d_kernel(int64_t len, double a, const double *x, const float *z,
                                double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * x[i] + (double)z[i];
}
__global__ void d2f_kernel(int64_t len, const double *x, float *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
__global__ void f2d_kernel(int64_t len, const float *x, double *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}
template <typename Tin, typename Tout>
__global__ void transpose_kernel(int64_t rows, int64_t cols, const Tin *in, Tout *out) {
    __shared__ Tout tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = (Tout)in[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][k];
    }
}
template <typename T>
__global__ void symmetrize_kernel(int64_t n, T *A) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n, j = e % n;
        if (j > i) A[e] = A[j * n + i];
    }
}
template <typename T>
__global__ void diag_kernel(int64_t n, const T *A, double *d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = (double)A[i * n + i];
}
// R^T = Theta^T X^T with a sparse Theta (see theta_t_xt).  One CTA per column j of Theta:
// the column is scanned in chunks of kSpThreads rows; each chunk's nonzeros are compacted
// into shared memory in ascending row order (a ballot per warp, an exclusive prefix over
// the warps), then every thread adds them, in that order, into its entries of row j of
// R^T, kSpPerThread entries a thread per pass over n.
constexpr int kSpThreads = 256;
constexpr int kSpPerThread = 4;
__global__ void __launch_bounds__(kSpThreads)
theta_t_xt_kernel(int64_t p, int64_t q, int64_t n, const double *__restrict__ Th,
                  const double *__restrict__ Xt, double *__restrict__ Rt) {
    __shared__ int s_off[kSpThreads];
    __shared__ double s_val[kSpThreads];
    __shared__ int s_count[kSpThreads / 32];
    const int64_t j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t span = (int64_t)kSpThreads * kSpPerThread;
    for (int64_t t0 = 0; t0 < n; t0 += span) {
        double acc[kSpPerThread];
#pragma unroll
        for (int k = 0; k < kSpPerThread; k++) acc[k] = 0.0;
        for (int64_t i0 = 0; i0 < p; i0 += kSpThreads) {
            const int64_t i = i0 + tid;
            const double v = i < p ? Th[i * q + j] : 0.0;
            const unsigned mask = __ballot_sync(0xffffffffu, v != 0.0);
            if (lane == 0) s_count[warp] = __popc(mask);
            __syncthreads();
            int base = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kSpThreads / 32; w++) {
                base += w < warp ? s_count[w] : 0;
                total += s_count[w];
            }
            if (v != 0.0) {
                const int pos = base + __popc(mask & ((1u << lane) - 1u));
                s_off[pos] = tid;
                s_val[pos] = v;
            }
            __syncthreads();
            for (int e = 0; e < total; e++) {
                const double th = s_val[e];
                const double *x = Xt + (i0 + s_off[e]) * n + t0;
#pragma unroll
                for (int k = 0; k < kSpPerThread; k++) {
                    const int64_t t = tid + (int64_t)k * kSpThreads;
                    if (t0 + t < n) acc[k] = fma(th, x[t], acc[k]);
                }
            }
            __syncthreads();  // the next chunk rewrites s_count, s_off, s_val
        }
#pragma unroll
        for (int k = 0; k < kSpPerThread; k++) {
            const int64_t t = t0 + tid + (int64_t)k * kSpThreads;
            if (t < n) Rt[j * n + t] = acc[k];
        }
    }
}

inline unsigned grid_for(int64_t len) {
    int64_t g = (len + 255) / 256;
    int64_t cap = (int64_t)sm_count() * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
}  // namespace

template <typename T>
void axpby(int64_t len, T a, const T *x, T b, T *y, cudaStream_t st) {
    if (len > 0) {
        note_launch();
        axpby_kernel<<<grid_for(len), 256, 0, st>>>(len, a, x, b, y);
    }
}
template void axpby<double>(int64_t, double, const double *, double, double *, cudaStream_t);
template void axpby<float>(int64_t, float, const float *, float, float *, cudaStream_t);

void axpy_f2d(int64_t len, double a, const double *x, const float *z, double *out,
              cudaStream_t st) {
    if (len > 0) {
        note_launch();
        axpy_f2d_kernel<<<grid_for(len), 256, 0, st>>>(len, a, x, z, out);
    }
}

void convert_d2f(int64_t len, const double *x, float *y, cudaStream_t st) {
    if (len > 0) {
        note_launch();
        d2f_kernel<<<grid_for(len), 256, 0, st>>>(len, x, y);
    }
}
void convert_f2d(int64_t len, const float *x, double *y, cudaStream_t st) {
    if (len > 0) {
        note_launch();
        f2d_kernel<<<grid_for(len), 256, 0, st>>>(len, x, y);
    }
}

template <typename Tin, typename Tout>
void transpose(int64_t rows, int64_t cols, const Tin *in, Tout *out, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid(ceil_div(cols, 32), ceil_div(rows, 32)), block(32, 8);
    note_launch();
    transpose_kernel<Tin, Tout><<<grid, block, 0, st>>>(rows, cols, in, out);
}
template void transpose<double, double>(int64_t, int64_t, const double *, double *, cudaStream_t);
template void transpose<double, float>(int64_t, int64_t, const double *, float *, cudaStream_t);
template void transpose<float, float>(int64_t, int64_t, const float *, float *, cudaStream_t);
template void transpose<float, double>(int64_t, int64_t, const float *, double *, cudaStream_t);

void theta_t_xt(int64_t p, int64_t q, int64_t n, const double *Th, const double *Xt, double *Rt,
                cudaStream_t st) {
    if (q > 0 && n > 0) {
        note_launch();
        theta_t_xt_kernel<<<(unsigned)q, kSpThreads, 0, st>>>(p, q, n, Th, Xt, Rt);
    }
}

template <typename T>
void symmetrize_lower(int64_t n, T *A, cudaStream_t st) {
    if (n > 0) {
        note_launch();
        symmetrize_kernel<<<grid_for(n * n), 256, 0, st>>>(n, A);
    }
}
template void symmetrize_lower<double>(int64_t, double *, cudaStream_t);
template void symmetrize_lower<float>(int64_t, float *, cudaStream_t);

template <typename T>
void diag_to_double(int64_t n, const T *A, double *d, cudaStream_t st) {
    if (n > 0) {
        note_launch();
        diag_kernel<<<grid_for(n), 256, 0, st>>>(n, A, d);
    }
}
template void diag_to_double<double>(int64_t, const double *, double *, cudaStream_t);
template void diag_to_double<float>(int64_t, const float *, double *, cudaStream_t);

// ---------------------------------------------------------------------------------
// deterministic double reductions: fixed 512-block grid -> partials -> one ordered block
// ---------------------------------------------------------------------------------
namespace {
constexpr int RED_BLOCKS = 512;

template <typename T>
__global__ void dot_partial_kernel(int64_t len, const T *x, const T *y, double *partial) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
template <typename T>
__global__ void l1_partial_kernel(int64_t len, const T *x, int64_t nd, double *partial) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (nd > 0 && (i / nd) == (i % nd)) continue;
        s += fabs((double)x[i]);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
}  // namespace

__global__ void finish_sum_kernel(int nparts, const double *partial, double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out += s;
}

template <typename T>
void dot_d(int64_t len, const T *x, const T *y, double *partial, double *out, cudaStream_t st) {
    note_launch();
    dot_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(len, x, y, partial);
    note_launch();
    finish_sum_kernel<<<1, 512, 0, st>>>(RED_BLOCKS, partial, out);
}
template void dot_d<double>(int64_t, const double *, const double *, double *, double *, cudaStream_t);
template void dot_d<float>(int64_t, const float *, const float *, double *, double *, cudaStream_t);

template <typename T>
void l1_d(int64_t len, const T *x, int64_t nd, double *partial, double *out, cudaStream_t st) {
    note_launch();
    l1_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(len, x, nd, partial);
    note_launch();
    finish_sum_kernel<<<1, 512, 0, st>>>(RED_BLOCKS, partial, out);
}
template void l1_d<double>(int64_t, const double *, int64_t, double *, double *, cudaStream_t);
template void l1_d<float>(int64_t, const float *, int64_t, double *, double *, cudaStream_t);

}  // namespace cggm
