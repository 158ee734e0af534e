// Gradient of Lambda, stopping quantity and active sets (Eq. 3, Section 2.2, Section 5.1).
#include "iter.cuh"

#include "dense.cuh"

namespace cggm {

namespace {
template <typename TP>
__global__ void grad_lambda_kernel(int64_t len, const double *Syy, const double *Sigma,
                                   const TP *Psi, double *G) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x)
        G[e] = Syy[e] - Sigma[e] - (double)Psi[e];
}

constexpr int RED_BLOCKS = 512;

__global__ void subgrad_partial_kernel(int64_t r, int64_t c, const double *G, const double *P,
                                       double lam, double diag_lam, double *partial) {
    double s0 = 0.0, s1 = 0.0;
    const int64_t len = r * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / c, j = e % c;
        const double l = (diag_lam >= 0.0 && i == j) ? diag_lam : lam;
        const double g = G[e], x = P[e];
        double gs;
        if (x != 0.0) gs = g + (x > 0.0 ? l : -l);
        else gs = (g > l) ? g - l : (g < -l ? g + l : 0.0);
        s0 += fabs(gs);
        s1 += fabs(x);
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0;
        partial[2 * blockIdx.x + 1] = s1;
    }
}

__global__ void subgrad_finish_kernel(int nparts, const double *partial, double *out) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        s0 += partial[2 * i];
        s1 += partial[2 * i + 1];
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
        out[0] += s0;
        out[1] += s1;
    }
}

__device__ __forceinline__ bool is_active(double g, double x, double thr) {
    return fabs(g) > thr || x != 0.0;
}

// one block per row: count active entries
__global__ void active_count_kernel(int64_t c, const double *G, const double *P, double thr,
                                    double thr_diag, bool upper, int64_t *rowcnt) {
    const int64_t i = blockIdx.x;
    const int64_t j0 = upper ? i : 0;
    double cnt = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < c; j += blockDim.x) {
        const double t = (i == j) ? thr_diag : thr;
        cnt += is_active(G[i * c + j], P[i * c + j], t) ? 1.0 : 0.0;
    }
    cnt = block_sum(cnt);
    if (threadIdx.x == 0) rowcnt[i] = (int64_t)cnt;
}

// exclusive scan of r row counts (single block), total into rowcnt[r] and *count
__global__ void scan_rows_kernel(int64_t r, int64_t *rowcnt, int64_t *count) {
    __shared__ int64_t s_part[1024];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < r; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = (i < r) ? rowcnt[i] : 0;
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int64_t add = (threadIdx.x >= (unsigned)o) ? s_part[threadIdx.x - o] : 0;
            __syncthreads();
            s_part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < r) rowcnt[i] = s_carry + s_part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rowcnt[r] = s_carry;
        *count = s_carry;
    }
}

// one block per row: write active (i, j) in ascending j
__global__ void active_write_kernel(int64_t c, const double *G, const double *P, double thr,
                                    double thr_diag, bool upper, const int64_t *rowoff,
                                    int32_t *ii, int32_t *jj) {
    __shared__ int s_scan[1024];
    __shared__ int64_t s_base;
    const int64_t i = blockIdx.x;
    const int64_t j0 = upper ? i : 0;
    if (threadIdx.x == 0) s_base = rowoff[i];
    __syncthreads();
    for (int64_t jb = j0; jb < c; jb += blockDim.x) {
        const int64_t j = jb + threadIdx.x;
        int f = 0;
        if (j < c) {
            const double t = (i == j) ? thr_diag : thr;
            f = is_active(G[i * c + j], P[i * c + j], t) ? 1 : 0;
        }
        s_scan[threadIdx.x] = f;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int add = (threadIdx.x >= (unsigned)o) ? s_scan[threadIdx.x - o] : 0;
            __syncthreads();
            s_scan[threadIdx.x] += add;
            __syncthreads();
        }
        if (f) {
            const int64_t pos = s_base + s_scan[threadIdx.x] - 1;
            ii[pos] = (int32_t)i;
            jj[pos] = (int32_t)j;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += s_scan[threadIdx.x];
        __syncthreads();
    }
}

inline unsigned grid_cap(int64_t len) {
    int64_t g = (len + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}
}  // namespace

template <typename TP>
void grad_lambda(int64_t q, const double *Syy, const double *Sigma, const TP *Psi, double *G,
                 cudaStream_t st) {
    note_launch();
    grad_lambda_kernel<<<grid_cap(q * q), 256, 0, st>>>(q * q, Syy, Sigma, Psi, G);
}
template void grad_lambda<double>(int64_t, const double *, const double *, const double *,
                                  double *, cudaStream_t);
template void grad_lambda<float>(int64_t, const double *, const double *, const float *,
                                 double *, cudaStream_t);

void subgrad_sums(int64_t r, int64_t c, const double *G, const double *P, double lam,
                  double diag_lam, double *partial, double *out, cudaStream_t st) {
    note_launch();
    subgrad_partial_kernel<<<RED_BLOCKS, 256, 0, st>>>(r, c, G, P, lam, diag_lam, partial);
    note_launch();
    subgrad_finish_kernel<<<1, 512, 0, st>>>(RED_BLOCKS, partial, out);
}

void active_compact(int64_t r, int64_t c, const double *G, const double *P, double thr,
                    double thr_diag, bool upper, int64_t *rowcnt, int32_t *ii, int32_t *jj,
                    int64_t *count, cudaStream_t st) {
    if (r <= 0) return;
    note_launch();
    active_count_kernel<<<(unsigned)r, 256, 0, st>>>(c, G, P, thr, thr_diag, upper, rowcnt);
    note_launch();
    scan_rows_kernel<<<1, 1024, 0, st>>>(r, rowcnt, count);
    note_launch();
    active_write_kernel<<<(unsigned)r, 256, 0, st>>>(c, G, P, thr, thr_diag, upper, rowcnt, ii,
                                                     jj);
}

}  // namespace cggm
