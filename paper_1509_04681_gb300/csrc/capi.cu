// C ABI of the CGGM solver (include/cggm.h): context, the Newton-iteration driver of
// Algorithm 1, and the step-level entry points.  Host code only issues kernels; every
// arithmetic step of the solve runs on the device.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "cg.cuh"
#include "chol.cuh"
#include "coo.cuh"

#include <map>
#include <mutex>
#include <tuple>
#include "common.cuh"
#include "dense.cuh"
#include "gemm_tc.cuh"
#include "iter.cuh"
#include "load.cuh"
#include "spchol.cuh"
#include "sweeps.cuh"

using namespace cggm;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

cggm_status ensure(Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return CGGM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e == cudaErrorMemoryAllocation ? CGGM_ENOMEM : CGGM_ECUDA;
    }
    b.bytes = bytes;
    return CGGM_OK;
}

template <typename T>
T *P(Buf &b) { return reinterpret_cast<T *>(b.p); }

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------------
// Batch-size tuner of the coordinate passes.  The batch size B is the tile shape of the
// sweep kernels: larger batches amortise the per-batch barriers over more coordinates but
// lengthen the serial phase and the coefficient work.  For opts.sweep_batch = -1, the first
// Newton iteration of a size class (precision, q and the Lambda active-set size, each rounded
// up to a power of two) times the Lambda pass at every candidate B and keeps the fastest for
// the process; later solves of the class reuse it.
// ---------------------------------------------------------------------------------
namespace {
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tuned;

int log2_ceil(int64_t v) {
    int r = 0;
    while (((int64_t)1 << r) < v) r++;
    return r;
}
std::tuple<int, int, int> tune_key(int precision, int64_t q, int64_t m) {
    return std::make_tuple(precision, log2_ceil(q < 1 ? 1 : q), log2_ceil(m < 1 ? 1 : m));
}
int tuned_lookup(int precision, int64_t q, int64_t m) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    const auto it = g_tuned.find(tune_key(precision, q, m));
    return it == g_tuned.end() ? 0 : it->second;
}
void tuned_store(int precision, int64_t q, int64_t m, int B) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_tuned[tune_key(precision, q, m)] = B;
}
}  // namespace

struct cggm_ctx {
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    // data
    Buf stage, Xt, Yt, Xt_f, Syy, Sxy, Sxx, Xd, colstats;
    // sparse solves (cggm_spd_solve)
    Buf cg_rp, cg_ci, cg_v, cg_b, cg_x, cg_w;
    // block gradients (cggm_grad_lambda_block)
    Buf bk_th, bk_rt, bk_pt, bk_sig, bk_psi, bk_g;
    // parameters and factorisations
    Buf Lam, Th, Lch, logd, Sig, Sig_f, Sd, Lam_a, Lch_a, logd_a, work;
    // products and gradients
    Buf Rt, Pt, Z, Psi, Pd, GL, GT, W;
    // coordinate passes
    Buf D, U, dV, li, lj, ti, tj, rowcnt;
    // scalars
    Buf scal, cnt, err;
    Buf tcA_hi, tcA_lo, tcB_hi, tcB_lo;  // split operands of the tensor-core contraction
    // mixed path: float operands of the tensor-core products and their TF32 hi/lo splits
    Buf Xt_hi, Xt_lo, Sig_hi, Sig_lo, R_f, R_hi, R_lo, Pt_f, Pt_hi, Pt_lo, Zf, tcerr;
    Buf partial;
    // sparse exchange at the boundary (cggm_solve): the caller's coordinate lists
    Buf coo_r, coo_c, coo_v;
    SweepScratch scr;
    cudaEvent_t ev[8];
    bool events = false;
};

namespace {

// scalar slots in ctx->scal (double)
enum {
    S_LOGDET = 0, S_SYYL, S_SXYT, S_TRACE, S_L1L, S_L1T, S_SUBL, S_NRML, S_SUBT, S_NRMT,
    S_GD, S_L1LD, S_LOGDET_A, S_TRACE_A, S_SYYL_A, S_L1L_A, S_COUNT
};

cggm_status sync_err(cggm_ctx *c) {
    CGGM_CUDA_TRY(cudaStreamSynchronize(c->st));
    CGGM_CUDA_TRY(cudaGetLastError());
    return CGGM_OK;
}

cggm_status read_dev_err(cggm_ctx *c, int *out) {
    CGGM_CUDA_TRY(cudaMemcpyAsync(out, c->err.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(c->st));
    return CGGM_OK;
}

// Copy a row-major rows x cols matrix of dtype dt (host or device) into a device double
// matrix transposed (cols x rows).  Also optionally a float copy.
// X may be any cggm_dtype; Y any but the genotype type (it is not standardised).
bool dtypes_ok(int xdt, int ydt) {
    const bool x = xdt == CGGM_F32 || xdt == CGGM_F64 || xdt == CGGM_BF16 || xdt == CGGM_I8_GENO;
    const bool y = ydt == CGGM_F32 || ydt == CGGM_F64 || ydt == CGGM_BF16;
    return x && y;
}

cggm_status load_transposed(cggm_ctx *c, const void *src, int dt, int64_t rows, int64_t cols,
                            Buf &dst, Buf *dst_f) {
    const size_t esz = dtype_size(dt);
    if (esz == 0) return CGGM_EINVAL;
    const size_t bytes = esz * (size_t)rows * (size_t)cols;
    const void *dsrc = src;
    if (!is_device_ptr(src)) {
        CGGM_TRY(ensure(c->stage, bytes));
        CGGM_CUDA_TRY(cudaMemcpyAsync(c->stage.p, src, bytes, cudaMemcpyHostToDevice, c->st));
        dsrc = c->stage.p;
    }
    CGGM_TRY(ensure(dst, 8 * (size_t)rows * cols));
    if (dt == CGGM_F64) {
        transpose<double, double>(rows, cols, (const double *)dsrc, P<double>(dst), c->st);
    } else if (dt == CGGM_F32) {
        transpose<float, double>(rows, cols, (const float *)dsrc, P<double>(dst), c->st);
    } else {
        CGGM_TRY(ensure(c->colstats, 16 * (size_t)cols));
        CGGM_TRY(load_input_transposed(dsrc, dt, rows, cols, P<double>(dst), P<double>(c->colstats),
                                       c->st));
    }
    if (dst_f) {
        CGGM_TRY(ensure(*dst_f, 4 * (size_t)rows * cols));
        convert_d2f(rows * cols, P<double>(dst), P<float>(*dst_f), c->st);
    }
    CGGM_CUDA_TRY(cudaGetLastError());
    return CGGM_OK;
}

cggm_status load_double(cggm_ctx *c, const double *src, size_t count, Buf &dst) {
    CGGM_TRY(ensure(dst, 8 * count));
    CGGM_CUDA_TRY(cudaMemcpyAsync(dst.p, src, 8 * count, cudaMemcpyDefault, c->st));
    return CGGM_OK;
}

cggm_status store_double(cggm_ctx *c, double *dst, const void *src, size_t count) {
    CGGM_CUDA_TRY(cudaMemcpyAsync(dst, src, 8 * count, cudaMemcpyDefault, c->st));
    return CGGM_OK;
}

__global__ void set_identity(int64_t n, double *A) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        A[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// diag of (1/n) M M^T for M rows x n (row-major), double
template <typename T>
__global__ void rowsq_kernel(int64_t rows, int64_t n, const T *M, double inv_n, double *d) {
    const int64_t r = blockIdx.x;
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double v = (double)M[r * n + k];
        s += v * v;
    }
    s = block_sum(s);
    if (threadIdx.x == 0) d[r] = s * inv_n;
}

__global__ void finite_check_kernel(int64_t len, const double *x, int *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[e])) { atomicCAS(err, 0, (int)DEV_NONFINITE); return; }
}

unsigned gcap(int64_t len) {
    int64_t g = (len + 255) / 256, cap = (int64_t)sm_count() * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

struct Sizes {
    int64_t n, p, q;
};

// ---------------------------------------------------------------------------------
// The solver, templated on the storage type of the large caches and products
// (double for CGGM_FP64, float for CGGM_MIXED).
// ---------------------------------------------------------------------------------
template <typename T>
struct Solver {
    cggm_ctx *c;
    Sizes z;
    cudaStream_t st;
    double lamL, lamT, lamLd;  // lamLd: penalty on the diagonal
    cggm_opts o;
    // the starting Lambda / Theta were already written into c->Lam / c->Th (sparse warm
    // starts); otherwise run() starts from its warm-start pointers or from I and 0
    bool lam_ready = false, th_ready = false;
    // rows of S_xx held at once (all p when they fit in kSxxChunkBytes: then S_xx is formed
    // once per solve), and the host copy of the Theta active list's row offsets, by which
    // the Theta pass is cut into chunks of rows otherwise
    int64_t sxx_rows = 0;
    std::vector<int64_t> th_rowoff;

    double *scal() { return P<double>(c->scal); }

    cggm_status alloc() {
        const int64_t n = z.n, p = z.p, q = z.q;
        const size_t qq = (size_t)q * q, pq = (size_t)p * q;
        CGGM_TRY(ensure(c->Syy, 8 * qq));
        CGGM_TRY(ensure(c->Sxy, 8 * pq));
        sxx_rows = sxx_chunk_rows(p, (int64_t)sizeof(T));
        if (o.sxx_rows > 0 && o.sxx_rows < sxx_rows) sxx_rows = o.sxx_rows;
        CGGM_TRY(ensure(c->Sxx, sizeof(T) * (size_t)sxx_rows * p));
        CGGM_TRY(ensure(c->Xd, 8 * (size_t)p));
        CGGM_TRY(ensure(c->Lam, 8 * qq));
        CGGM_TRY(ensure(c->Th, 8 * pq));
        CGGM_TRY(ensure(c->Lch, 8 * qq));
        CGGM_TRY(ensure(c->logd, 8 * (size_t)q));
        CGGM_TRY(ensure(c->Sig, 8 * qq));
        CGGM_TRY(ensure(c->Sig_f, sizeof(T) * qq));
        CGGM_TRY(ensure(c->Sd, 8 * (size_t)q));
        CGGM_TRY(ensure(c->Lam_a, 8 * qq));
        CGGM_TRY(ensure(c->Lch_a, 8 * qq));
        CGGM_TRY(ensure(c->logd_a, 8 * (size_t)q));
        CGGM_TRY(ensure(c->work, 8 * qq));
        CGGM_TRY(ensure(c->Rt, 8 * (size_t)q * n));
        CGGM_TRY(ensure(c->Pt, 8 * (size_t)q * n));
        CGGM_TRY(ensure(c->Z, 8 * (size_t)q * n));
        CGGM_TRY(ensure(c->Psi, sizeof(T) * qq));
        CGGM_TRY(ensure(c->Pd, 8 * (size_t)q));
        CGGM_TRY(ensure(c->GL, 8 * qq));
        CGGM_TRY(ensure(c->GT, 8 * pq));
        CGGM_TRY(ensure(c->W, 8 * pq));
        CGGM_TRY(ensure(c->D, 8 * qq));
        CGGM_TRY(ensure(c->U, sizeof(T) * qq));
        CGGM_TRY(ensure(c->dV, sizeof(T) * pq));
        CGGM_TRY(ensure(c->li, 4 * (qq / 2 + q + 1)));
        CGGM_TRY(ensure(c->lj, 4 * (qq / 2 + q + 1)));
        CGGM_TRY(ensure(c->ti, 4 * pq));
        CGGM_TRY(ensure(c->tj, 4 * pq));
        CGGM_TRY(ensure(c->rowcnt, 8 * (size_t)((p > q ? p : q) + 1)));
        CGGM_TRY(ensure(c->scal, 8 * S_COUNT));
        CGGM_TRY(ensure(c->cnt, 8 * 4));
        CGGM_TRY(ensure(c->err, sizeof(int)));
        CGGM_TRY(ensure(c->partial, 8 * 4096));
        return CGGM_OK;
    }

    // The mixed path runs the products from X on the tensor cores (3xTF32) when every
    // contracted dimension gives 16-byte rows (multiples of 4 floats).
    bool tc() const { return sizeof(T) == 4 && z.n % 4 == 0 && z.p % 4 == 0 && z.q % 4 == 0; }

    cggm_status tc_alloc() {
        const int64_t n = z.n, p = z.p, q = z.q;
        Buf *pn[] = {&c->Xt_hi, &c->Xt_lo};
        for (Buf *b : pn) CGGM_TRY(ensure(*b, 4 * (size_t)p * n));
        Buf *qq[] = {&c->Sig_hi, &c->Sig_lo};
        for (Buf *b : qq) CGGM_TRY(ensure(*b, 4 * (size_t)q * q));
        Buf *nq[] = {&c->R_f, &c->R_hi, &c->R_lo, &c->Pt_f, &c->Pt_hi, &c->Pt_lo};
        for (Buf *b : nq) CGGM_TRY(ensure(*b, 4 * (size_t)n * q));
        CGGM_TRY(ensure(c->Zf, 4 * (size_t)p * q));
        CGGM_TRY(ensure(c->tcerr, sizeof(int)));
        return CGGM_OK;
    }

    // Pt_f = Sigma R^T (q x n) on the tensor cores from the current splits of Sigma and R,
    // then its own split.
    cggm_status tc_P() {
        const int64_t n = z.n, q = z.q;
        CGGM_TRY(gemm_tc_nt(q, n, q, 1.0f, P<float>(c->Sig_hi), q, P<float>(c->R_hi), q, 0.0f,
                            P<float>(c->Pt_f), n, true, P<float>(c->Sig_lo), P<float>(c->R_lo),
                            P<int>(c->tcerr), st));
        split_tf32(q, n, n, P<float>(c->Pt_f), P<float>(c->Pt_hi), P<float>(c->Pt_lo), st);
        return CGGM_OK;
    }

    // out = a S_xy + scale X^T P_f^T... : Zf = scale Xt Pt_f^T (p x q), out = a S_xy + Zf
    cggm_status tc_XtP(double scale, double a, double *out) {
        const int64_t n = z.n, p = z.p, q = z.q;
        CGGM_TRY(gemm_tc_nt(p, q, n, (float)scale, P<float>(c->Xt_hi), n, P<float>(c->Pt_hi), n,
                            0.0f, P<float>(c->Zf), q, true, P<float>(c->Xt_lo), P<float>(c->Pt_lo),
                            P<int>(c->tcerr), st));
        axpy_f2d(p * q, a, P<double>(c->Sxy), P<float>(c->Zf), out, st);
        return CGGM_OK;
    }

    cggm_status tc_check() {
        if (!tc()) return CGGM_OK;
        int h = 0;
        CGGM_CUDA_TRY(cudaMemcpyAsync(&h, c->tcerr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CGGM_CUDA_TRY(cudaStreamSynchronize(st));
        if (h == DEV_TIMEOUT) return CGGM_ETIMEDOUT;
        if (h != 0) return CGGM_ECUDA;
        return CGGM_OK;
    }

    // Rows r0 .. r1 - 1 of S_xx = X^T X / n (Section 2.1) into the chunk buffer c->Sxx,
    // from X: on the tensor cores (3xTF32) in the mixed path, SIMT double in the FP64 path.
    cggm_status form_sxx(int64_t r0, int64_t r1) {
        const int64_t n = z.n, p = z.p, rows = r1 - r0;
        const double inv = 1.0 / (double)n;
        if (sizeof(T) == 8) {
            const double *Xt = P<double>(c->Xt);
            gemm<double>(false, true, rows, p, n, inv, Xt + r0 * n, n, Xt, n, 0.0,
                         (double *)c->Sxx.p, p, st);
        } else if (tc()) {
            CGGM_TRY(gemm_tc_nt(rows, p, n, (float)inv, P<float>(c->Xt_hi) + r0 * n, n,
                                P<float>(c->Xt_hi), n, 0.0f, (float *)c->Sxx.p, p, true,
                                P<float>(c->Xt_lo) + r0 * n, P<float>(c->Xt_lo),
                                P<int>(c->tcerr), st));
        } else {
            gemm<float>(false, true, rows, p, n, (float)inv, P<float>(c->Xt_f) + r0 * n, n,
                        P<float>(c->Xt_f), n, 0.0f, (float *)c->Sxx.p, p, st);
        }
        return CGGM_OK;
    }

    // S_yy, S_xy (Section 2.1) from Xt (p x n) and Yt (q x n), double; S_xx whole when it
    // fits in one chunk (otherwise the Theta pass forms its rows chunk by chunk)
    cggm_status covariances() {
        const int64_t n = z.n, p = z.p, q = z.q;
        const double inv = 1.0 / (double)n;
        const double *Xt = P<double>(c->Xt), *Yt = P<double>(c->Yt);
        gemm<double>(false, true, q, q, n, inv, Yt, n, Yt, n, 0.0, P<double>(c->Syy), q, st);
        gemm<double>(false, true, p, q, n, inv, Xt, n, Yt, n, 0.0, P<double>(c->Sxy), q, st);
        if (sizeof(T) == 4) {
            CGGM_TRY(ensure(c->Xt_f, 4 * (size_t)p * n));
            convert_d2f(p * n, Xt, P<float>(c->Xt_f), st);
            if (tc()) {
                CGGM_TRY(tc_alloc());
                CGGM_CUDA_TRY(cudaMemsetAsync(c->tcerr.p, 0, sizeof(int), st));
                split_tf32(p, n, n, P<float>(c->Xt_f), P<float>(c->Xt_hi), P<float>(c->Xt_lo), st);
            }
        }
        if (sxx_rows == p) CGGM_TRY(form_sxx(0, p));
        note_launch();
        rowsq_kernel<double><<<(unsigned)p, 256, 0, st>>>(p, n, Xt, inv, P<double>(c->Xd));
        CGGM_CUDA_TRY(cudaGetLastError());
        return CGGM_OK;
    }

    // Cholesky of Lambda into Lch, logdet into scal[S_LOGDET]; returns ENOTPD if not PD
    cggm_status factor(Buf &Lam, Buf &Lch, Buf &logd, int slot) {
        const int64_t q = z.q;
        CGGM_CUDA_TRY(cudaMemcpyAsync(Lch.p, Lam.p, 8 * (size_t)q * q, cudaMemcpyDeviceToDevice, st));
        CGGM_CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), st));
        cholesky_inplace(q, P<double>(Lch), q, P<double>(logd), P<int>(c->err), st);
        logdet_from_logd(q, P<double>(logd), scal() + slot, st);
        int h = 0;
        CGGM_TRY(read_dev_err(c, &h));
        if (h == DEV_NOTPD) return CGGM_ENOTPD;
        if (h != 0) return CGGM_ECUDA;
        return CGGM_OK;
    }

    // Sigma (double and T copies) and its double diagonal from Lch
    void sigma_from_factor() {
        const int64_t q = z.q;
        inverse_from_cholesky(q, P<double>(c->Lch), P<double>(c->Sig), P<double>(c->work), st);
        if (sizeof(T) == 4) convert_d2f(q * q, P<double>(c->Sig), (float *)c->Sig_f.p, st);
        if (tc()) split_tf32(q, q, q, (const float *)c->Sig_f.p, P<float>(c->Sig_hi),
                             P<float>(c->Sig_lo), st);
        diag_to_double<double>(q, P<double>(c->Sig), P<double>(c->Sd), st);
    }
    const T *SigT() {
        return sizeof(T) == 8 ? (const T *)c->Sig.p : (const T *)c->Sig_f.p;
    }

    // Rt = Theta^T X^T (q x n) in double (it enters the double-precision objective), over
    // Theta's nonzeros only; Pt = Sigma Rt: double, or float on the tensor cores in the
    // mixed path
    cggm_status products_R_P() {
        const int64_t n = z.n, p = z.p, q = z.q;
        theta_t_xt(p, q, n, P<double>(c->Th), P<double>(c->Xt), P<double>(c->Rt), st);
        if (tc()) {
            transpose<double, float>(q, n, P<double>(c->Rt), P<float>(c->R_f), st);
            split_tf32(n, q, q, P<float>(c->R_f), P<float>(c->R_hi), P<float>(c->R_lo), st);
            return tc_P();
        }
        gemm<double>(false, false, q, n, q, 1.0, P<double>(c->Sig), q, P<double>(c->Rt), n, 0.0,
                     P<double>(c->Pt), n, st);
        return CGGM_OK;
    }

    // Psi = Pt Pt^T / n (T), its double diagonal
    cggm_status product_Psi() {
        const int64_t n = z.n, q = z.q;
        const double inv = 1.0 / (double)n;
        if (tc()) {
            CGGM_TRY(gemm_tc_nt(q, q, n, (float)inv, P<float>(c->Pt_hi), n, P<float>(c->Pt_hi), n,
                                0.0f, (float *)c->Psi.p, q, true, P<float>(c->Pt_lo),
                                P<float>(c->Pt_lo), P<int>(c->tcerr), st));
            note_launch();
            rowsq_kernel<float><<<(unsigned)q, 256, 0, st>>>(q, n, P<float>(c->Pt_f), inv,
                                                              P<double>(c->Pd));
            return CGGM_OK;
        }
        if (sizeof(T) == 8) {
            gemm<double>(false, true, q, q, n, inv, P<double>(c->Pt), n, P<double>(c->Pt), n, 0.0,
                         (double *)c->Psi.p, q, st);
        } else {
            float *Ptf = P<float>(c->Z);  // scratch
            convert_d2f(q * n, P<double>(c->Pt), Ptf, st);
            gemm<float>(false, true, q, q, n, (float)inv, Ptf, n, Ptf, n, 0.0f, (float *)c->Psi.p, q, st);
        }
        note_launch();
        rowsq_kernel<double><<<(unsigned)q, 256, 0, st>>>(q, n, P<double>(c->Pt), inv, P<double>(c->Pd));
        return CGGM_OK;
    }

    // Theta-only pieces of f at the current Theta: 2 tr(S_xy^T Theta) and ||Theta||_1
    void theta_pieces() {
        const int64_t p = z.p, q = z.q;
        double *s = scal();
        double *part = P<double>(c->partial);
        cudaMemsetAsync(s + S_SXYT, 0, 8, st);
        cudaMemsetAsync(s + S_L1T, 0, 8, st);
        dot_d<double>(p * q, P<double>(c->Sxy), P<double>(c->Th), part, s + S_SXYT, st);
        l1_d<double>(p * q, P<double>(c->Th), 0, part, s + S_L1T, st);
    }

    // f(Lam, Theta) of Eq. 1 with Lch = chol(Lam) and log|Lam| in scal[ld_slot]; the
    // trace term is tr(Lam^-1 R^T R) / n = ||Lch^-1 R^T||_F^2 / n with R = X Theta (Rt
    // current).  The start-of-iteration value and every Armijo trial go through this one
    // function, so that equal arguments give bit-equal values.
    cggm_status eval_f(Buf &Lam, Buf &Lch, int ld_slot, double *f_out) {
        const int64_t n = z.n, q = z.q;
        double *s = scal();
        double *part = P<double>(c->partial);
        CGGM_CUDA_TRY(cudaMemcpyAsync(c->Z.p, c->Rt.p, 8 * (size_t)q * n, cudaMemcpyDeviceToDevice, st));
        trsm_lower_inplace(q, P<double>(Lch), q, P<double>(c->Z), n, n, false, st);
        CGGM_CUDA_TRY(cudaMemsetAsync(s + S_TRACE_A, 0, 24, st));
        dot_d<double>(q * n, P<double>(c->Z), P<double>(c->Z), part, s + S_TRACE_A, st);
        dot_d<double>(q * q, P<double>(c->Syy), P<double>(Lam), part, s + S_SYYL_A, st);
        l1_d<double>(q * q, P<double>(Lam), o.penalize_diag ? 0 : q, part, s + S_L1L_A, st);
        double h[S_COUNT];
        CGGM_CUDA_TRY(cudaMemcpyAsync(h, s, 8 * S_COUNT, cudaMemcpyDeviceToHost, st));
        CGGM_TRY(sync_err(c));
        *f_out = -h[ld_slot] + h[S_SYYL_A] + 2.0 * h[S_SXYT] + h[S_TRACE_A] / (double)n +
                 lamL * h[S_L1L_A] + lamT * h[S_L1T];
        return CGGM_OK;
    }

    // One Theta pass (Section 3.2) over the m active coordinates, S_xx rows from the chunk
    // buffer: with all of S_xx held, one launch; otherwise, for each chunk of rows that
    // holds active coordinates, its rows of S_xx are formed and the pass continues over
    // that chunk's part of the (row-major) list.
    cggm_status theta_pass(int64_t m, int B) {
        const int64_t p = z.p, q = z.q;
        const int32_t *ti = P<int32_t>(c->ti), *tj = P<int32_t>(c->tj);
        if (sxx_rows == p)
            return theta_sweep<T>(p, q, (const T *)c->Sxx.p, 0, P<double>(c->Xd), SigT(),
                                  P<double>(c->Sd), P<double>(c->W), P<double>(c->Th), m, ti,
                                  tj, lamT, (T *)c->dV.p, B, c->scr, st);
        for (int64_t r0 = 0; r0 < p; r0 += sxx_rows) {
            const int64_t r1 = r0 + sxx_rows < p ? r0 + sxx_rows : p;
            const int64_t k0 = th_rowoff[r0], k1 = th_rowoff[r1];
            if (k1 <= k0) continue;
            CGGM_TRY(form_sxx(r0, r1));
            CGGM_TRY(theta_sweep<T>(p, q, (const T *)c->Sxx.p, r0, P<double>(c->Xd), SigT(),
                                    P<double>(c->Sd), P<double>(c->W), P<double>(c->Th),
                                    k1 - k0, ti + k0, tj + k0, lamT, (T *)c->dV.p, B, c->scr,
                                    st));
        }
        return CGGM_OK;
    }

    double f_from(const double *h) const {
        return -h[S_LOGDET] + h[S_SYYL] + 2.0 * h[S_SXYT] + h[S_TRACE] / (double)z.n +
               lamL * h[S_L1L] + lamT * h[S_L1T];
    }

    cggm_status run(const double *warmL, const double *warmT, cggm_info *info, int *iters_out,
                    bool *conv_out) {
        const int64_t n = z.n, p = z.p, q = z.q;
        const size_t qq = (size_t)q * q, pq = (size_t)p * q;
        CGGM_TRY(alloc());
        CGGM_TRY(covariances());
        // initial point (Algorithm 1: Theta <- 0, Lambda <- I, or the warm start)
        if (warmL) {
            CGGM_TRY(load_double(c, warmL, qq, c->Lam));
        } else if (!lam_ready) {
            note_launch();
            set_identity<<<gcap(q * q), 256, 0, st>>>(q, P<double>(c->Lam));
        }
        if (warmT) {
            CGGM_TRY(load_double(c, warmT, pq, c->Th));
        } else if (!th_ready) {
            CGGM_CUDA_TRY(cudaMemsetAsync(c->Th.p, 0, 8 * pq, st));
        }
        CGGM_CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), st));
        note_launch();
        finite_check_kernel<<<gcap(n * p), 256, 0, st>>>(n * p, P<double>(c->Xt), P<int>(c->err));
        note_launch();
        finite_check_kernel<<<gcap(n * q), 256, 0, st>>>(n * q, P<double>(c->Yt), P<int>(c->err));
        note_launch();
        finite_check_kernel<<<gcap(q * q), 256, 0, st>>>(q * q, P<double>(c->Lam), P<int>(c->err));
        note_launch();
        finite_check_kernel<<<gcap(p * q), 256, 0, st>>>(p * q, P<double>(c->Th), P<int>(c->err));
        {
            int h = 0;
            CGGM_TRY(read_dev_err(c, &h));
            if (h) return CGGM_ENONFINITE;
        }
        CGGM_TRY(factor(c->Lam, c->Lch, c->logd, S_LOGDET));
        sigma_from_factor();

        const int B_default = sizeof(T) == 8 ? 128 : 256;
        int B = o.sweep_batch > 0 ? o.sweep_batch : B_default;
        const bool autotune = o.sweep_batch == CGGM_SWEEP_BATCH_AUTO;
        const int prec_key = sizeof(T) == 8 ? CGGM_FP64 : CGGM_MIXED;
        double h[S_COUNT];
        int64_t hc[2];
        bool converged = false;
        int it = 0;
        double f = 0.0, subgrad = 0.0, nrm = 0.0;
        int ls_total = 0;
        int64_t coords_l = 0, coords_t = 0;
        cudaEvent_t *ev = c->ev;
        double t_prod = 0, t_fac = 0, t_act = 0, t_swl = 0, t_ls = 0, t_swt = 0;
        cudaEventRecord(ev[7], st);
        for (it = 0; it < o.max_iter; it++) {
            cudaEventRecord(ev[0], st);
            // ---- products (R, P, Psi) and the gradients (Eq. 3) ----
            CGGM_TRY(products_R_P());
            CGGM_TRY(product_Psi());
            theta_pieces();
            double f_start = 0.0;
            CGGM_TRY(eval_f(c->Lam, c->Lch, S_LOGDET, &f_start));
            grad_lambda<T>(q, P<double>(c->Syy), P<double>(c->Sig), (const T *)c->Psi.p,
                           P<double>(c->GL), st);
            // G_Theta = 2 S_xy + (2/n) X^T P
            if (tc()) {
                CGGM_TRY(tc_XtP(2.0 / (double)n, 2.0, P<double>(c->GT)));
            } else {
                axpby<double>(pq, 2.0, P<double>(c->Sxy), 0.0, P<double>(c->GT), st);
                gemm<double>(false, true, p, q, n, 2.0 / (double)n, P<double>(c->Xt), n,
                             P<double>(c->Pt), n, 1.0, P<double>(c->GT), q, st);
            }
            cudaEventRecord(ev[1], st);
            // ---- stopping quantity (Section 5.1) and active sets (Section 2.2) ----
            double *s = scal();
            CGGM_CUDA_TRY(cudaMemsetAsync(s + S_SUBL, 0, 8 * 4, st));
            subgrad_sums(q, q, P<double>(c->GL), P<double>(c->Lam), lamL, lamLd,
                         P<double>(c->partial), s + S_SUBL, st);
            subgrad_sums(p, q, P<double>(c->GT), P<double>(c->Th), lamT, -1.0,
                         P<double>(c->partial), s + S_SUBT, st);
            const double thrd = o.penalize_diag ? lamL : -1.0;
            active_compact(q, q, P<double>(c->GL), P<double>(c->Lam), lamL, thrd, true,
                           P<int64_t>(c->rowcnt), P<int32_t>(c->li), P<int32_t>(c->lj),
                           P<int64_t>(c->cnt), st);
            active_compact(p, q, P<double>(c->GT), P<double>(c->Th), lamT, lamT, false,
                           P<int64_t>(c->rowcnt), P<int32_t>(c->ti), P<int32_t>(c->tj),
                           P<int64_t>(c->cnt) + 1, st);
            if (sxx_rows < p) {  // row offsets of the Theta list (read after the sync below)
                th_rowoff.resize((size_t)p + 1);
                CGGM_CUDA_TRY(cudaMemcpyAsync(th_rowoff.data(), c->rowcnt.p, 8 * (size_t)(p + 1),
                                              cudaMemcpyDeviceToHost, st));
            }
            cudaEventRecord(ev[2], st);
            CGGM_CUDA_TRY(cudaMemcpyAsync(h, s, 8 * S_COUNT, cudaMemcpyDeviceToHost, st));
            CGGM_CUDA_TRY(cudaMemcpyAsync(hc, c->cnt.p, 16, cudaMemcpyDeviceToHost, st));
            CGGM_TRY(sync_err(c));
            f = f_start;
            subgrad = h[S_SUBL] + h[S_SUBT];
            nrm = h[S_NRML] + h[S_NRMT];
            {
                float a, b;
                cudaEventElapsedTime(&a, ev[0], ev[1]);
                cudaEventElapsedTime(&b, ev[1], ev[2]);
                t_prod += a * 1e-3;
                t_act += b * 1e-3;
            }
            if (info) {
                info->m_lambda = hc[0];
                info->m_theta = hc[1];
            }
            if (!std::isfinite(f)) return CGGM_ENONFINITE;
            if (o.verbose)
                fprintf(stderr, "cggm it %d f %.15g ratio %.3e mL %lld mT %lld\n", it, f,
                        subgrad / (nrm > 0 ? nrm : 1.0), (long long)hc[0], (long long)hc[1]);
            if (subgrad < o.tol * nrm || f <= o.target_f) {
                converged = true;
                break;
            }
            // ---- Lambda direction (Section 3.1) ----
            coords_l += hc[0];
            coords_t += hc[1];
            auto lambda_pass = [&](int Bp) -> cggm_status {
                CGGM_CUDA_TRY(cudaMemsetAsync(c->D.p, 0, 8 * qq, st));
                CGGM_CUDA_TRY(cudaMemsetAsync(c->U.p, 0, sizeof(T) * qq, st));
                return lambda_sweep<T>(q, SigT(), (const T *)c->Psi.p, P<double>(c->Sd),
                                       P<double>(c->Pd), P<double>(c->GL), P<double>(c->Lam),
                                       hc[0], P<int32_t>(c->li), P<int32_t>(c->lj), lamL, lamLd,
                                       P<double>(c->D), (T *)c->U.p, Bp, c->scr, st);
            };
            if (autotune) {
                const int tb = tuned_lookup(prec_key, q, hc[0]);
                if (tb > 0) {
                    B = tb;
                } else if (hc[0] > 0) {
                    // time the pass at each candidate (each run recomputes D from zero)
                    const int cands_f[] = {64, 128, 256, 512}, cands_d[] = {32, 64, 128};
                    const int *cands = sizeof(T) == 8 ? cands_d : cands_f;
                    const int nc = sizeof(T) == 8 ? 3 : 4;
                    float best = -1.0f;
                    for (int ci = 0; ci < nc; ci++) {
                        cudaEventRecord(ev[3], st);
                        CGGM_TRY(lambda_pass(cands[ci]));
                        cudaEventRecord(ev[4], st);
                        CGGM_CUDA_TRY(cudaEventSynchronize(ev[4]));
                        float ms = 0.0f;
                        cudaEventElapsedTime(&ms, ev[3], ev[4]);
                        if (best < 0.0f || ms < best) {
                            best = ms;
                            B = cands[ci];
                        }
                    }
                    tuned_store(prec_key, q, hc[0], B);
                }
            }
            cudaEventRecord(ev[3], st);
            CGGM_TRY(lambda_pass(B));
            cudaEventRecord(ev[4], st);
            // ---- Armijo (Algorithm 1) ----
            // delta = tr(G D) + lamL (||Lam + D||_1 - ||Lam||_1)
            double *part = P<double>(c->partial);
            CGGM_CUDA_TRY(cudaMemsetAsync(s + S_GD, 0, 16, st));
            CGGM_CUDA_TRY(cudaMemsetAsync(s + S_L1L, 0, 8, st));
            dot_d<double>(q * q, P<double>(c->GL), P<double>(c->D), part, s + S_GD, st);
            l1_d<double>(q * q, P<double>(c->Lam), o.penalize_diag ? 0 : q, part, s + S_L1L, st);
            CGGM_CUDA_TRY(cudaMemcpyAsync(c->Lam_a.p, c->Lam.p, 8 * qq, cudaMemcpyDeviceToDevice, st));
            axpby<double>(qq, 1.0, P<double>(c->D), 1.0, P<double>(c->Lam_a), st);
            l1_d<double>(q * q, P<double>(c->Lam_a), o.penalize_diag ? 0 : q, part, s + S_L1LD, st);
            CGGM_CUDA_TRY(cudaMemcpyAsync(h, s, 8 * S_COUNT, cudaMemcpyDeviceToHost, st));
            CGGM_TRY(sync_err(c));
            const double delta = h[S_GD] + lamL * (h[S_L1LD] - h[S_L1L]);
            double alpha = 1.0;
            bool accepted = false;
            int trials = 0;
            for (trials = 1; trials <= o.ls_max_trials; trials++) {
                CGGM_CUDA_TRY(cudaMemcpyAsync(c->Lam_a.p, c->Lam.p, 8 * qq, cudaMemcpyDeviceToDevice, st));
                axpby<double>(qq, alpha, P<double>(c->D), 1.0, P<double>(c->Lam_a), st);
                cggm_status fs = factor(c->Lam_a, c->Lch_a, c->logd_a, S_LOGDET_A);
                if (fs == CGGM_OK) {
                    double fa = 0.0;
                    CGGM_TRY(eval_f(c->Lam_a, c->Lch_a, S_LOGDET_A, &fa));
                    if (std::isfinite(fa) && fa <= f + o.ls_sigma * alpha * delta) {
                        accepted = true;
                        break;
                    }
                } else if (fs != CGGM_ENOTPD) {
                    return fs;
                }
                alpha *= o.ls_beta;
            }
            ls_total += trials;
            if (!accepted) return CGGM_ELINESEARCH;
            std::swap(c->Lam, c->Lam_a);
            std::swap(c->Lch, c->Lch_a);
            std::swap(c->logd, c->logd_a);
            CGGM_CUDA_TRY(cudaMemcpyAsync(s + S_LOGDET, s + S_LOGDET_A, 8, cudaMemcpyDeviceToDevice, st));
            cudaEventRecord(ev[5], st);
            sigma_from_factor();
            // ---- Theta pass (Section 3.2) with the new Sigma ----
            // W = S_xy + S_xx Theta Sigma = S_xy + (1/n) X^T (X Theta Sigma)
            if (tc()) {
                CGGM_TRY(tc_P());
                CGGM_TRY(tc_XtP(1.0 / (double)n, 1.0, P<double>(c->W)));
            } else {
                gemm<double>(false, false, q, n, q, 1.0, P<double>(c->Sig), q, P<double>(c->Rt), n,
                             0.0, P<double>(c->Pt), n, st);
                CGGM_CUDA_TRY(cudaMemcpyAsync(c->W.p, c->Sxy.p, 8 * pq, cudaMemcpyDeviceToDevice, st));
                gemm<double>(false, true, p, q, n, 1.0 / (double)n, P<double>(c->Xt), n,
                             P<double>(c->Pt), n, 1.0, P<double>(c->W), q, st);
            }
            cudaEventRecord(ev[2], st);  // Sigma and W formed
            CGGM_CUDA_TRY(cudaMemsetAsync(c->dV.p, 0, sizeof(T) * pq, st));
            CGGM_TRY(theta_pass(hc[1], B));
            cudaEventRecord(ev[6], st);
            CGGM_TRY(sync_err(c));
            CGGM_TRY(tc_check());
            {
                float a, b, d1, d2;
                cudaEventElapsedTime(&a, ev[3], ev[4]);
                cudaEventElapsedTime(&b, ev[4], ev[5]);
                cudaEventElapsedTime(&d1, ev[5], ev[2]);
                cudaEventElapsedTime(&d2, ev[2], ev[6]);
                t_swl += a * 1e-3;
                t_ls += b * 1e-3;
                t_fac += d1 * 1e-3;
                t_swt += d2 * 1e-3;
            }
        }
        cudaEventRecord(ev[6], st);
        CGGM_TRY(sync_err(c));
        if (info) {
            float tot = 0;
            cudaEventElapsedTime(&tot, ev[7], ev[6]);
            info->iterations = it + (converged ? 1 : 0);
            info->converged = converged ? 1 : 0;
            info->f = f;
            info->subgrad = subgrad;
            info->l1norm = nrm;
            info->ls_trials = ls_total;
            info->seconds = tot * 1e-3;
            info->sec_products = t_prod;
            info->sec_factor = t_fac;
            info->sec_active = t_act;
            info->sec_sweep_lambda = t_swl;
            info->sec_linesearch = t_ls;
            info->sec_sweep_theta = t_swt;
            info->coords_lambda = coords_l;
            info->coords_theta = coords_t;
        }
        *iters_out = it;
        *conv_out = converged;
        return CGGM_OK;
    }
};

cggm_status check_sizes(int64_t n, int64_t p, int64_t q) {
    if (n <= 0 || p <= 0 || q <= 0) return CGGM_EINVAL;
    if (q > 2147483647LL || p > 2147483647LL) return CGGM_EINVAL;
    return CGGM_OK;
}

cggm_status set_device(cggm_ctx *c) {
    CGGM_CUDA_TRY(cudaSetDevice(c->device));
    return CGGM_OK;
}

// A caller's coordinate list (host or device arrays) into the dense device matrix dst
// (rows x cols), which it overwrites; `sym`: one triangle (row <= col) of a symmetric
// matrix.  Bad indices give CGGM_EINVAL, non-finite values CGGM_ENONFINITE.
cggm_status coo_in(cggm_ctx *c, const cggm_coo *a, int64_t rows, int64_t cols, bool sym,
                   double *dst) {
    const int64_t nnz = a->nnz;
    if (nnz < 0 || nnz > rows * cols || (nnz > 0 && (!a->row || !a->col || !a->val)))
        return CGGM_EINVAL;
    cudaStream_t st = c->st;
    CGGM_CUDA_TRY(cudaMemsetAsync(dst, 0, 8 * (size_t)rows * cols, st));
    if (nnz == 0) return CGGM_OK;
    CGGM_TRY(ensure(c->coo_r, 4 * (size_t)nnz));
    CGGM_TRY(ensure(c->coo_c, 4 * (size_t)nnz));
    CGGM_TRY(ensure(c->coo_v, 8 * (size_t)nnz));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->coo_r.p, a->row, 4 * (size_t)nnz, cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->coo_c.p, a->col, 4 * (size_t)nnz, cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->coo_v.p, a->val, 8 * (size_t)nnz, cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), st));
    coo_scatter(nnz, P<int32_t>(c->coo_r), P<int32_t>(c->coo_c), P<double>(c->coo_v), rows,
                cols, sym, dst, P<int>(c->err), st);
    CGGM_CUDA_TRY(cudaGetLastError());
    int h = 0;
    CGGM_TRY(read_dev_err(c, &h));
    if (h == DEV_NONFINITE) return CGGM_ENONFINITE;
    if (h != 0) return CGGM_EINVAL;
    return CGGM_OK;
}

// The nonzero entries of the dense device matrix A (rows x cols; with `upper` only j >= i)
// as a coordinate list in row-major order, in arrays allocated on the host with malloc
// (released by cggm_free_coo).  ii, jj: index scratch of the size of the list's worst
// case; vv: value scratch as large.
cggm_status coo_out(cggm_ctx *c, const double *A, int64_t rows, int64_t cols, bool upper,
                    Buf &ii, Buf &jj, Buf &vv, cggm_coo *out) {
    cudaStream_t st = c->st;
    int64_t *cnt = P<int64_t>(c->cnt) + 2;
    active_compact(rows, cols, A, A, INFINITY, INFINITY, upper, P<int64_t>(c->rowcnt),
                   P<int32_t>(ii), P<int32_t>(jj), cnt, st);
    int64_t nnz = 0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&nnz, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CGGM_TRY(sync_err(c));
    coo_gather(nnz, P<int32_t>(ii), P<int32_t>(jj), A, cols, P<double>(vv), st);
    const size_t k = nnz > 0 ? (size_t)nnz : 1;
    int32_t *r = (int32_t *)malloc(4 * k), *cl = (int32_t *)malloc(4 * k);
    double *v = (double *)malloc(8 * k);
    if (!r || !cl || !v) {
        free(r); free(cl); free(v);
        return CGGM_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    if (nnz > 0) {
        e = cudaMemcpyAsync(r, ii.p, 4 * (size_t)nnz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cl, jj.p, 4 * (size_t)nnz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(v, vv.p, 8 * (size_t)nnz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free(r); free(cl); free(v);
        return CGGM_ECUDA;
    }
    out->nnz = nnz;
    out->row = r;
    out->col = cl;
    out->val = v;
    return CGGM_OK;
}

template <typename T>
cggm_status solve_t(cggm_ctx *c, Sizes z, double lamL, double lamT, double lamLd,
                    const cggm_opts &o, const double *wL, const double *wT, const cggm_coo *cL,
                    const cggm_coo *cT, cggm_info *info, bool *conv) {
    Solver<T> S{c, z, c->st, lamL, lamT, lamLd, o};
    CGGM_TRY(S.alloc());
    if (cL) {
        CGGM_TRY(coo_in(c, cL, z.q, z.q, true, P<double>(c->Lam)));
        S.lam_ready = true;
    }
    if (cT) {
        CGGM_TRY(coo_in(c, cT, z.p, z.q, false, P<double>(c->Th)));
        S.th_ready = true;
    }
    int iters = 0;
    return S.run(wL, wT, info, &iters, conv);
}

// Argument checks, input upload and the solve of cggm_solve and cggm_solve_dense; the
// result is left in c->Lam and c->Th.  Warm starts: dense (wL, wT) or sparse (cL, cT).
cggm_status solve_common(cggm_ctx *c, const void *X, int xdtype, const void *Y, int ydtype,
                         int64_t n, int64_t p, int64_t q, double lam_L, double lam_T,
                         double tol, const double *wL, const double *wT, const cggm_coo *cL,
                         const cggm_coo *cT, const cggm_opts *opts, cggm_info *info,
                         bool *conv) {
    if (!c || !X || !Y) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    if (!(lam_L >= 0.0) || !(lam_T >= 0.0)) return CGGM_EINVAL;
    if (!dtypes_ok(xdtype, ydtype)) return CGGM_EINVAL;
    cggm_opts o;
    if (opts) o = *opts; else cggm_opts_default(&o);
    if (tol > 0.0) o.tol = tol;
    if (!(o.tol > 0.0) || o.max_iter < 0 || o.ls_max_trials < 1 || !(o.ls_beta > 0.0 && o.ls_beta < 1.0))
        return CGGM_EINVAL;
    if (o.sweep_batch != 0 && o.sweep_batch != CGGM_SWEEP_BATCH_AUTO && o.sweep_batch != 32 &&
        o.sweep_batch != 64 && o.sweep_batch != 128 &&
        !((o.sweep_batch == 256 || o.sweep_batch == 512) && o.precision == CGGM_MIXED))
        return CGGM_EINVAL;
    if (o.precision != CGGM_FP64 && o.precision != CGGM_MIXED) return CGGM_EINVAL;
    if (o.sxx_rows < 0) return CGGM_EINVAL;
    if (info) memset(info, 0, sizeof(*info));
    CGGM_TRY(set_device(c));
    CGGM_TRY(ensure(c->err, sizeof(int)));
    CGGM_TRY(load_transposed(c, X, xdtype, n, p, c->Xt, nullptr));
    CGGM_TRY(load_transposed(c, Y, ydtype, n, q, c->Yt, nullptr));
    const double lamLd = o.penalize_diag ? lam_L : 0.0;
    const Sizes z{n, p, q};
    if (o.precision == CGGM_FP64)
        return solve_t<double>(c, z, lam_L, lam_T, lamLd, o, wL, wT, cL, cT, info, conv);
    return solve_t<float>(c, z, lam_L, lam_T, lamLd, o, wL, wT, cL, cT, info, conv);
}

}  // namespace

namespace cggm {
void ctx_set_batcher(cggm_ctx *c, PassBatcher *b) {
    if (c) c->scr.batcher = b;
}
}  // namespace cggm

extern "C" {

void cggm_opts_default(cggm_opts *o) {
    if (!o) return;
    o->tol = 0.01;
    o->max_iter = 1000;
    o->precision = CGGM_MIXED;
    o->ls_sigma = 1e-3;
    o->ls_beta = 0.5;
    o->ls_max_trials = 50;
    o->penalize_diag = 1;
    o->sweep_batch = 0;
    o->target_f = -INFINITY;
    o->verbose = 0;
    o->sxx_rows = 0;
}

const char *cggm_status_string(int s) {
    switch (s) {
        case CGGM_OK: return "ok";
        case CGGM_EINVAL: return "invalid argument";
        case CGGM_ENOTPD: return "matrix not positive definite";
        case CGGM_ENOMEM: return "out of device memory";
        case CGGM_EMAXITER: return "iteration limit reached";
        case CGGM_ELINESEARCH: return "line search failed";
        case CGGM_ECUDA: return "CUDA error";
        case CGGM_ETIMEDOUT: return "device wait timed out";
        case CGGM_ENONFINITE: return "non-finite value";
        case CGGM_ECANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

cggm_status cggm_create(cggm_ctx **out, int device, void *stream) {
    if (!out) return CGGM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CGGM_EINVAL;
    }
    cggm_ctx *c = new cggm_ctx();
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return CGGM_ECUDA;
    }
    if (stream) {
        c->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return CGGM_ECUDA;
        }
        c->own_stream = true;
    }
    for (int i = 0; i < 8; i++) cudaEventCreate(&c->ev[i]);
    c->events = true;
    *out = c;
    return CGGM_OK;
}

void cggm_destroy(cggm_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    Buf *bufs[] = {&c->stage, &c->Xt, &c->Yt, &c->Xt_f, &c->Syy, &c->Sxy, &c->Sxx, &c->Xd,
                   &c->Lam, &c->Th, &c->Lch, &c->logd, &c->Sig, &c->Sig_f, &c->Sd, &c->Lam_a,
                   &c->Lch_a, &c->logd_a, &c->work, &c->Rt, &c->Pt, &c->Z, &c->Psi, &c->Pd,
                   &c->GL, &c->GT, &c->W, &c->D, &c->U, &c->dV, &c->li, &c->lj, &c->ti,
                   &c->tj, &c->rowcnt, &c->scal, &c->cnt, &c->err, &c->partial, &c->colstats, &c->cg_rp, &c->cg_ci, &c->cg_v, &c->cg_b, &c->cg_x, &c->cg_w, &c->bk_th, &c->bk_rt, &c->bk_pt, &c->bk_sig, &c->bk_psi, &c->bk_g,
                   &c->tcA_hi, &c->tcA_lo, &c->tcB_hi, &c->tcB_lo, &c->Xt_hi, &c->Xt_lo,
                   &c->Sig_hi, &c->Sig_lo, &c->R_f, &c->R_hi, &c->R_lo, &c->Pt_f, &c->Pt_hi,
                   &c->Pt_lo, &c->Zf, &c->tcerr, &c->coo_r, &c->coo_c, &c->coo_v};
    for (Buf *b : bufs) if (b->p) cudaFree(b->p);
    scratch_free(c->scr);
    if (c->events) for (int i = 0; i < 8; i++) cudaEventDestroy(c->ev[i]);
    if (c->own_stream) cudaStreamDestroy(c->st);
    delete c;
}

cggm_status cggm_solve_dense(cggm_ctx *c, const void *X, int xdtype, const void *Y,
                             int ydtype, int64_t n, int64_t p, int64_t q, double lam_L,
                             double lam_T, double tol, const double *warm_Lambda,
                             const double *warm_Theta, const cggm_opts *opts,
                             double *Lambda_out, double *Theta_out, cggm_info *info) {
    const int64_t launches0 = launch_counter();
    bool conv = false;
    CGGM_TRY(solve_common(c, X, xdtype, Y, ydtype, n, p, q, lam_L, lam_T, tol, warm_Lambda,
                          warm_Theta, nullptr, nullptr, opts, info, &conv));
    if (Lambda_out) CGGM_TRY(store_double(c, Lambda_out, c->Lam.p, (size_t)q * q));
    if (Theta_out) CGGM_TRY(store_double(c, Theta_out, c->Th.p, (size_t)p * q));
    CGGM_CUDA_TRY(cudaStreamSynchronize(c->st));
    if (info) info->launches = launch_counter() - launches0;
    return conv ? CGGM_OK : CGGM_EMAXITER;
}

void cggm_free_coo(cggm_coo *a) {
    if (!a) return;
    free(a->row);
    free(a->col);
    free(a->val);
    a->nnz = 0;
    a->row = nullptr;
    a->col = nullptr;
    a->val = nullptr;
}

cggm_status cggm_solve(cggm_ctx *c, const void *X, int xdtype, const void *Y, int ydtype,
                       int64_t n, int64_t p, int64_t q, double lam_L, double lam_T, double tol,
                       const cggm_coo *warm_Lambda, const cggm_coo *warm_Theta,
                       const cggm_opts *opts, cggm_coo *Lambda_out, cggm_coo *Theta_out,
                       cggm_info *info) {
    const cggm_coo empty = {0, nullptr, nullptr, nullptr};
    if (Lambda_out) *Lambda_out = empty;
    if (Theta_out) *Theta_out = empty;
    const int64_t launches0 = launch_counter();
    bool conv = false;
    CGGM_TRY(solve_common(c, X, xdtype, Y, ydtype, n, p, q, lam_L, lam_T, tol, nullptr,
                          nullptr, warm_Lambda, warm_Theta, opts, info, &conv));
    if (Lambda_out)
        CGGM_TRY(coo_out(c, P<double>(c->Lam), q, q, true, c->li, c->lj, c->GL, Lambda_out));
    if (Theta_out) {
        const cggm_status s = coo_out(c, P<double>(c->Th), p, q, false, c->ti, c->tj, c->GT,
                                      Theta_out);
        if (s != CGGM_OK) {
            cggm_free_coo(Lambda_out);
            return s;
        }
    }
    if (info) info->launches = launch_counter() - launches0;
    return conv ? CGGM_OK : CGGM_EMAXITER;
}

cggm_status cggm_predict(cggm_ctx *c, const void *X, int xdtype, int64_t n, int64_t p,
                         int64_t q, const cggm_coo *Lambda, const cggm_coo *Theta,
                         double *Yhat_out, double *B_out) {
    if (!c || !X || !Lambda || !Theta || (!Yhat_out && !B_out)) return CGGM_EINVAL;
    if (!dtypes_ok(xdtype, CGGM_F64)) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    CGGM_TRY(set_device(c));
    const size_t qq = (size_t)q * q, pq = (size_t)p * q, qn = (size_t)q * n;
    CGGM_TRY(ensure(c->err, sizeof(int)));
    CGGM_TRY(ensure(c->scal, 8 * S_COUNT));
    CGGM_TRY(ensure(c->Lam, 8 * qq));
    CGGM_TRY(ensure(c->Lch, 8 * qq));
    CGGM_TRY(ensure(c->logd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->Sig, 8 * qq));
    CGGM_TRY(ensure(c->work, 8 * qq));
    CGGM_TRY(ensure(c->Th, 8 * pq));
    CGGM_TRY(coo_in(c, Lambda, q, q, true, P<double>(c->Lam)));
    CGGM_TRY(coo_in(c, Theta, p, q, false, P<double>(c->Th)));
    cggm_opts o;
    cggm_opts_default(&o);
    Solver<double> S{c, {n, p, q}, c->st, 0.0, 0.0, 0.0, o};
    CGGM_TRY(S.factor(c->Lam, c->Lch, c->logd, S_LOGDET));  // CGGM_ENOTPD if not PD
    inverse_from_cholesky(q, P<double>(c->Lch), P<double>(c->Sig), P<double>(c->work), c->st);
    if (B_out) {  // B = -Theta Sigma (p x q)
        CGGM_TRY(ensure(c->W, 8 * pq));
        gemm<double>(false, false, p, q, q, -1.0, P<double>(c->Th), q, P<double>(c->Sig), q, 0.0,
                     P<double>(c->W), q, c->st);
        CGGM_TRY(store_double(c, B_out, c->W.p, pq));
    }
    if (Yhat_out) {  // Yhat^T = -Sigma Theta^T X^T (q x n), R^T over Theta's nonzeros
        CGGM_TRY(load_transposed(c, X, xdtype, n, p, c->Xt, nullptr));
        CGGM_TRY(ensure(c->Rt, 8 * qn));
        CGGM_TRY(ensure(c->Pt, 8 * qn));
        CGGM_TRY(ensure(c->Z, 8 * qn));
        theta_t_xt(p, q, n, P<double>(c->Th), P<double>(c->Xt), P<double>(c->Rt), c->st);
        gemm<double>(false, false, q, n, q, -1.0, P<double>(c->Sig), q, P<double>(c->Rt), n, 0.0,
                     P<double>(c->Pt), n, c->st);
        transpose<double, double>(q, n, P<double>(c->Pt), P<double>(c->Z), c->st);
        CGGM_TRY(store_double(c, Yhat_out, c->Z.p, qn));
    }
    return sync_err(c);
}

cggm_status cggm_objective(cggm_ctx *c, const void *X, int xdtype, const void *Y, int ydtype,
                           int64_t n, int64_t p, int64_t q, const double *Lambda,
                           const double *Theta, double lam_L, double lam_T, int penalize_diag,
                           double *f_out) {
    if (!c || !X || !Y || !Lambda || !Theta || !f_out) return CGGM_EINVAL;
    if (!dtypes_ok(xdtype, ydtype)) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    CGGM_TRY(set_device(c));
    CGGM_TRY(load_transposed(c, X, xdtype, n, p, c->Xt, nullptr));
    CGGM_TRY(load_transposed(c, Y, ydtype, n, q, c->Yt, nullptr));
    cggm_opts o;
    cggm_opts_default(&o);
    o.penalize_diag = penalize_diag;
    Solver<double> S{c, {n, p, q}, c->st, lam_L, lam_T, penalize_diag ? lam_L : 0.0, o};
    CGGM_TRY(S.alloc());
    const size_t qq = (size_t)q * q, pq = (size_t)p * q;
    const double inv = 1.0 / (double)n;
    gemm<double>(false, true, q, q, n, inv, P<double>(c->Yt), n, P<double>(c->Yt), n, 0.0,
                 P<double>(c->Syy), q, c->st);
    gemm<double>(false, true, p, q, n, inv, P<double>(c->Xt), n, P<double>(c->Yt), n, 0.0,
                 P<double>(c->Sxy), q, c->st);
    CGGM_TRY(load_double(c, Lambda, qq, c->Lam));
    CGGM_TRY(load_double(c, Theta, pq, c->Th));
    CGGM_TRY(S.factor(c->Lam, c->Lch, c->logd, S_LOGDET));
    // trace tr(Lambda^-1 Theta^T S_xx Theta) = ||L^-1 (X Theta)^T||_F^2 / n
    theta_t_xt(p, q, n, P<double>(c->Th), P<double>(c->Xt), P<double>(c->Rt), c->st);
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->Z.p, c->Rt.p, 8 * (size_t)q * n, cudaMemcpyDeviceToDevice, c->st));
    trsm_lower_inplace(q, P<double>(c->Lch), q, P<double>(c->Z), n, n, false, c->st);
    double *s = P<double>(c->scal);
    double *part = P<double>(c->partial);
    CGGM_CUDA_TRY(cudaMemsetAsync(s + S_SYYL, 0, 8 * (S_L1T - S_SYYL + 1), c->st));
    dot_d<double>(q * q, P<double>(c->Syy), P<double>(c->Lam), part, s + S_SYYL, c->st);
    dot_d<double>(p * q, P<double>(c->Sxy), P<double>(c->Th), part, s + S_SXYT, c->st);
    dot_d<double>(q * n, P<double>(c->Z), P<double>(c->Z), part, s + S_TRACE, c->st);
    l1_d<double>(q * q, P<double>(c->Lam), penalize_diag ? 0 : q, part, s + S_L1L, c->st);
    l1_d<double>(p * q, P<double>(c->Th), 0, part, s + S_L1T, c->st);
    double h[S_COUNT];
    CGGM_CUDA_TRY(cudaMemcpyAsync(h, s, 8 * S_COUNT, cudaMemcpyDeviceToHost, c->st));
    CGGM_TRY(sync_err(c));
    *f_out = S.f_from(h);
    return CGGM_OK;
}

cggm_status cggm_grad(cggm_ctx *c, const void *X, int xdtype, const void *Y, int ydtype,
                      int64_t n, int64_t p, int64_t q, const double *Lambda, const double *Theta,
                      double *G_Lambda, double *G_Theta) {
    if (!c || !X || !Y || !Lambda || !Theta) return CGGM_EINVAL;
    if (!dtypes_ok(xdtype, ydtype)) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    CGGM_TRY(set_device(c));
    CGGM_TRY(load_transposed(c, X, xdtype, n, p, c->Xt, nullptr));
    CGGM_TRY(load_transposed(c, Y, ydtype, n, q, c->Yt, nullptr));
    cggm_opts o;
    cggm_opts_default(&o);
    Solver<double> S{c, {n, p, q}, c->st, 0.0, 0.0, 0.0, o};
    CGGM_TRY(S.alloc());
    const size_t qq = (size_t)q * q, pq = (size_t)p * q;
    const double inv = 1.0 / (double)n;
    gemm<double>(false, true, q, q, n, inv, P<double>(c->Yt), n, P<double>(c->Yt), n, 0.0,
                 P<double>(c->Syy), q, c->st);
    gemm<double>(false, true, p, q, n, inv, P<double>(c->Xt), n, P<double>(c->Yt), n, 0.0,
                 P<double>(c->Sxy), q, c->st);
    CGGM_TRY(load_double(c, Lambda, qq, c->Lam));
    CGGM_TRY(load_double(c, Theta, pq, c->Th));
    CGGM_TRY(S.factor(c->Lam, c->Lch, c->logd, S_LOGDET));
    S.sigma_from_factor();
    CGGM_TRY(S.products_R_P());
    CGGM_TRY(S.product_Psi());
    grad_lambda<double>(q, P<double>(c->Syy), P<double>(c->Sig), P<double>(c->Psi),
                        P<double>(c->GL), c->st);
    axpby<double>(pq, 2.0, P<double>(c->Sxy), 0.0, P<double>(c->GT), c->st);
    gemm<double>(false, true, p, q, n, 2.0 * inv, P<double>(c->Xt), n, P<double>(c->Pt), n, 1.0,
                 P<double>(c->GT), q, c->st);
    if (G_Lambda) CGGM_TRY(store_double(c, G_Lambda, c->GL.p, qq));
    if (G_Theta) CGGM_TRY(store_double(c, G_Theta, c->GT.p, pq));
    return sync_err(c);
}

cggm_status cggm_cholesky(cggm_ctx *c, int64_t q, const double *Lambda, double *L_out,
                          double *logdet_out, double *Sigma_out, int precision) {
    (void)precision;
    if (!c || !Lambda || q <= 0) return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    cggm_opts o;
    cggm_opts_default(&o);
    Solver<double> S{c, {1, 1, q}, c->st, 0.0, 0.0, 0.0, o};
    const size_t qq = (size_t)q * q;
    CGGM_TRY(ensure(c->Lam, 8 * qq));
    CGGM_TRY(ensure(c->Lch, 8 * qq));
    CGGM_TRY(ensure(c->logd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->Sig, 8 * qq));
    CGGM_TRY(ensure(c->Sd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->work, 8 * qq));
    CGGM_TRY(ensure(c->scal, 8 * S_COUNT));
    CGGM_TRY(ensure(c->err, sizeof(int)));
    CGGM_TRY(load_double(c, Lambda, qq, c->Lam));
    CGGM_TRY(S.factor(c->Lam, c->Lch, c->logd, S_LOGDET));
    if (Sigma_out) {
        inverse_from_cholesky(q, P<double>(c->Lch), P<double>(c->Sig), P<double>(c->work), c->st);
        CGGM_TRY(store_double(c, Sigma_out, c->Sig.p, qq));
    }
    if (L_out) CGGM_TRY(store_double(c, L_out, c->Lch.p, qq));
    if (logdet_out) {
        double h;
        CGGM_CUDA_TRY(cudaMemcpyAsync(&h, P<double>(c->scal) + S_LOGDET, 8, cudaMemcpyDeviceToHost, c->st));
        CGGM_TRY(sync_err(c));
        *logdet_out = h;
    }
    return sync_err(c);
}

// Caller-given coordinate lists (host or device memory) are checked on the host before
// any kernel reads them: 0 <= a[k] < rows, 0 <= b[k] < cols, and a[k] <= b[k] when
// `upper`.  The coordinate passes index their matrices with these values unchecked.
static cggm_status check_pairs(cggm_ctx *c, const int32_t *a, const int32_t *b, int64_t m,
                               int64_t rows, int64_t cols, bool upper) {
    if (m <= 0) return CGGM_OK;
    std::vector<int32_t> ha, hb;
    if (is_device_ptr(a) || is_device_ptr(b)) {
        ha.resize((size_t)m);
        hb.resize((size_t)m);
        CGGM_CUDA_TRY(cudaMemcpyAsync(ha.data(), a, 4 * (size_t)m, cudaMemcpyDefault, c->st));
        CGGM_CUDA_TRY(cudaMemcpyAsync(hb.data(), b, 4 * (size_t)m, cudaMemcpyDefault, c->st));
        CGGM_CUDA_TRY(cudaStreamSynchronize(c->st));
        a = ha.data();
        b = hb.data();
    }
    for (int64_t k = 0; k < m; k++)
        if (a[k] < 0 || a[k] >= rows || b[k] < 0 || b[k] >= cols || (upper && a[k] > b[k]))
            return CGGM_EINVAL;
    return CGGM_OK;
}

static cggm_status load_index(cggm_ctx *c, const int32_t *src, int64_t m, Buf &dst) {
    CGGM_TRY(ensure(dst, 4 * (size_t)(m > 0 ? m : 1)));
    if (m > 0) CGGM_CUDA_TRY(cudaMemcpyAsync(dst.p, src, 4 * (size_t)m, cudaMemcpyDefault, c->st));
    return CGGM_OK;
}

cggm_status cggm_lambda_sweep(cggm_ctx *c, int64_t q, const double *Sigma, const double *Psi,
                              const double *Syy, const double *Lambda, int64_t m,
                              const int32_t *ai, const int32_t *aj, double lam_L,
                              int penalize_diag, int precision, double *D_out) {
    if (!c || q <= 0 || m < 0 || !Sigma || !Psi || !Syy || !Lambda || !D_out) return CGGM_EINVAL;
    if (m > 0 && (!ai || !aj)) return CGGM_EINVAL;
    if (precision != CGGM_FP64 && precision != CGGM_MIXED) return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    CGGM_TRY(check_pairs(c, ai, aj, m, q, q, true));
    const size_t qq = (size_t)q * q;
    CGGM_TRY(load_double(c, Sigma, qq, c->Sig));
    CGGM_TRY(load_double(c, Psi, qq, c->work));
    CGGM_TRY(load_double(c, Syy, qq, c->Syy));
    CGGM_TRY(load_double(c, Lambda, qq, c->Lam));
    CGGM_TRY(load_index(c, ai, m, c->li));
    CGGM_TRY(load_index(c, aj, m, c->lj));
    CGGM_TRY(ensure(c->Sd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->Pd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->GL, 8 * qq));
    CGGM_TRY(ensure(c->D, 8 * qq));
    diag_to_double<double>(q, P<double>(c->Sig), P<double>(c->Sd), c->st);
    diag_to_double<double>(q, P<double>(c->work), P<double>(c->Pd), c->st);
    grad_lambda<double>(q, P<double>(c->Syy), P<double>(c->Sig), P<double>(c->work),
                        P<double>(c->GL), c->st);
    CGGM_CUDA_TRY(cudaMemsetAsync(c->D.p, 0, 8 * qq, c->st));
    const double lamd = penalize_diag ? lam_L : 0.0;
    if (precision == CGGM_FP64) {
        CGGM_TRY(ensure(c->U, 8 * qq));
        CGGM_CUDA_TRY(cudaMemsetAsync(c->U.p, 0, 8 * qq, c->st));
        CGGM_TRY(lambda_sweep<double>(q, P<double>(c->Sig), P<double>(c->work), P<double>(c->Sd),
                                      P<double>(c->Pd), P<double>(c->GL), P<double>(c->Lam), m,
                                      P<int32_t>(c->li), P<int32_t>(c->lj), lam_L, lamd,
                                      P<double>(c->D), P<double>(c->U), 128, c->scr, c->st));
    } else {
        CGGM_TRY(ensure(c->U, 4 * qq));
        CGGM_TRY(ensure(c->Sig_f, 4 * qq));
        CGGM_TRY(ensure(c->Psi, 4 * qq));
        convert_d2f(q * q, P<double>(c->Sig), P<float>(c->Sig_f), c->st);
        convert_d2f(q * q, P<double>(c->work), P<float>(c->Psi), c->st);
        CGGM_CUDA_TRY(cudaMemsetAsync(c->U.p, 0, 4 * qq, c->st));
        CGGM_TRY(lambda_sweep<float>(q, P<float>(c->Sig_f), P<float>(c->Psi), P<double>(c->Sd),
                                     P<double>(c->Pd), P<double>(c->GL), P<double>(c->Lam), m,
                                     P<int32_t>(c->li), P<int32_t>(c->lj), lam_L, lamd,
                                     P<double>(c->D), P<float>(c->U), 256, c->scr, c->st));
    }
    CGGM_TRY(store_double(c, D_out, c->D.p, qq));
    return sync_err(c);
}

cggm_status cggm_theta_sweep(cggm_ctx *c, int64_t n, int64_t p, int64_t q, const double *X,
                             const double *Sxy, const double *Sigma, const double *Theta_in,
                             int64_t m, const int32_t *ti, const int32_t *tj, double lam_T,
                             int precision, double *Theta_out) {
    if (!c || !X || !Sxy || !Sigma || !Theta_in || !Theta_out || m < 0) return CGGM_EINVAL;
    if (m > 0 && (!ti || !tj)) return CGGM_EINVAL;
    if (precision != CGGM_FP64 && precision != CGGM_MIXED) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    CGGM_TRY(set_device(c));
    CGGM_TRY(check_pairs(c, ti, tj, m, p, q, false));
    // the rows of the list on the host, to cut it into runs whose rows fit one S_xx chunk
    std::vector<int32_t> rows_h((size_t)m);
    if (m > 0)
        CGGM_CUDA_TRY(cudaMemcpy(rows_h.data(), ti, 4 * (size_t)m, cudaMemcpyDefault));
    const size_t qq = (size_t)q * q, pq = (size_t)p * q;
    const int64_t esz = precision == CGGM_FP64 ? 8 : 4;
    const int64_t R = sxx_chunk_rows(p, esz);
    const bool sorted = std::is_sorted(rows_h.begin(), rows_h.end());
    CGGM_TRY(load_transposed(c, X, CGGM_F64, n, p, c->Xt, nullptr));
    CGGM_TRY(ensure(c->Sxx, (size_t)esz * (size_t)R * p));
    CGGM_TRY(ensure(c->Xd, 8 * (size_t)p));
    CGGM_TRY(load_double(c, Sxy, pq, c->Sxy));
    CGGM_TRY(load_double(c, Sigma, qq, c->Sig));
    CGGM_TRY(load_double(c, Theta_in, pq, c->Th));
    CGGM_TRY(load_index(c, ti, m, c->ti));
    CGGM_TRY(load_index(c, tj, m, c->tj));
    CGGM_TRY(ensure(c->Sd, 8 * (size_t)q));
    CGGM_TRY(ensure(c->Rt, 8 * (size_t)q * n));
    CGGM_TRY(ensure(c->Pt, 8 * (size_t)q * n));
    CGGM_TRY(ensure(c->W, 8 * pq));
    const double inv = 1.0 / (double)n;
    const double *Xt = P<double>(c->Xt);
    note_launch();
    rowsq_kernel<double><<<(unsigned)p, 256, 0, c->st>>>(p, n, Xt, inv, P<double>(c->Xd));
    diag_to_double<double>(q, P<double>(c->Sig), P<double>(c->Sd), c->st);
    // W = S_xy + S_xx Theta Sigma
    theta_t_xt(p, q, n, P<double>(c->Th), Xt, P<double>(c->Rt), c->st);
    gemm<double>(false, false, q, n, q, 1.0, P<double>(c->Sig), q, P<double>(c->Rt), n, 0.0,
                 P<double>(c->Pt), n, c->st);
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->W.p, c->Sxy.p, 8 * pq, cudaMemcpyDeviceToDevice, c->st));
    gemm<double>(false, true, p, q, n, inv, Xt, n, P<double>(c->Pt), n, 1.0, P<double>(c->W), q, c->st);
    if (precision == CGGM_MIXED) {
        CGGM_TRY(ensure(c->Xt_f, 4 * (size_t)p * n));
        CGGM_TRY(ensure(c->Sig_f, 4 * qq));
        convert_d2f(p * n, Xt, P<float>(c->Xt_f), c->st);
        convert_d2f(q * q, P<double>(c->Sig), P<float>(c->Sig_f), c->st);
    }
    CGGM_TRY(ensure(c->dV, (size_t)esz * pq));
    CGGM_CUDA_TRY(cudaMemsetAsync(c->dV.p, 0, (size_t)esz * pq, c->st));
    // runs of the list whose rows lie within R consecutive rows: S_xx rows lo .. lo + R - 1
    // formed from X, then the pass continues over the run
    for (int64_t k0 = 0; k0 < m;) {
        int64_t lo = rows_h[k0], hi = lo, k1 = k0 + 1;
        while (k1 < m) {
            const int64_t r = rows_h[k1];
            const int64_t nlo = r < lo ? r : lo, nhi = r > hi ? r : hi;
            if (nhi - nlo + 1 > R) break;
            lo = nlo;
            hi = nhi;
            k1++;
        }
        const int64_t x0 = (lo + R <= p) ? lo : p - R;  // the chunk's first row
        const int64_t rows = R;
        const int32_t *ri = P<int32_t>(c->ti) + k0, *rj = P<int32_t>(c->tj) + k0;
        if (precision == CGGM_FP64) {
            gemm<double>(false, true, rows, p, n, inv, Xt + x0 * n, n, Xt, n, 0.0,
                         P<double>(c->Sxx), p, c->st);
            CGGM_TRY(theta_sweep<double>(p, q, P<double>(c->Sxx), x0, P<double>(c->Xd),
                                         P<double>(c->Sig), P<double>(c->Sd), P<double>(c->W),
                                         P<double>(c->Th), k1 - k0, ri, rj, lam_T,
                                         P<double>(c->dV), 128, c->scr, c->st, sorted));
        } else {
            gemm<float>(false, true, rows, p, n, (float)inv, P<float>(c->Xt_f) + x0 * n, n,
                        P<float>(c->Xt_f), n, 0.0f, P<float>(c->Sxx), p, c->st);
            CGGM_TRY(theta_sweep<float>(p, q, P<float>(c->Sxx), x0, P<double>(c->Xd),
                                        P<float>(c->Sig_f), P<double>(c->Sd), P<double>(c->W),
                                        P<double>(c->Th), k1 - k0, ri, rj, lam_T,
                                        P<float>(c->dV), 256, c->scr, c->st, sorted));
        }
        k0 = k1;
    }
    CGGM_TRY(store_double(c, Theta_out, c->Th.p, pq));
    return sync_err(c);
}

cggm_status cggm_active_sets(cggm_ctx *c, int64_t p, int64_t q, const double *G_Lambda,
                             const double *G_Theta, const double *Lambda, const double *Theta,
                             double lam_L, double lam_T, int penalize_diag, int32_t *li,
                             int32_t *lj, int64_t *m_lambda, int32_t *ti, int32_t *tj,
                             int64_t *m_theta) {
    if (!c || p <= 0 || q <= 0 || !G_Lambda || !G_Theta || !Lambda || !Theta || !li || !lj ||
        !ti || !tj || !m_lambda || !m_theta)
        return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    const size_t qq = (size_t)q * q, pq = (size_t)p * q;
    CGGM_TRY(load_double(c, G_Lambda, qq, c->GL));
    CGGM_TRY(load_double(c, G_Theta, pq, c->GT));
    CGGM_TRY(load_double(c, Lambda, qq, c->Lam));
    CGGM_TRY(load_double(c, Theta, pq, c->Th));
    CGGM_TRY(ensure(c->li, 4 * (qq / 2 + q + 1)));
    CGGM_TRY(ensure(c->lj, 4 * (qq / 2 + q + 1)));
    CGGM_TRY(ensure(c->ti, 4 * pq));
    CGGM_TRY(ensure(c->tj, 4 * pq));
    CGGM_TRY(ensure(c->rowcnt, 8 * (size_t)((p > q ? p : q) + 1)));
    CGGM_TRY(ensure(c->cnt, 32));
    const double thrd = penalize_diag ? lam_L : -1.0;
    active_compact(q, q, P<double>(c->GL), P<double>(c->Lam), lam_L, thrd, true,
                   P<int64_t>(c->rowcnt), P<int32_t>(c->li), P<int32_t>(c->lj), P<int64_t>(c->cnt), c->st);
    active_compact(p, q, P<double>(c->GT), P<double>(c->Th), lam_T, lam_T, false,
                   P<int64_t>(c->rowcnt), P<int32_t>(c->ti), P<int32_t>(c->tj),
                   P<int64_t>(c->cnt) + 1, c->st);
    int64_t hc[2];
    CGGM_CUDA_TRY(cudaMemcpyAsync(hc, c->cnt.p, 16, cudaMemcpyDeviceToHost, c->st));
    CGGM_TRY(sync_err(c));
    *m_lambda = hc[0];
    *m_theta = hc[1];
    CGGM_CUDA_TRY(cudaMemcpyAsync(li, c->li.p, 4 * (size_t)hc[0], cudaMemcpyDefault, c->st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(lj, c->lj.p, 4 * (size_t)hc[0], cudaMemcpyDefault, c->st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(ti, c->ti.p, 4 * (size_t)hc[1], cudaMemcpyDefault, c->st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(tj, c->tj.p, 4 * (size_t)hc[1], cudaMemcpyDefault, c->st));
    return sync_err(c);
}

// Copies a CSR matrix (host or device) into the context and validates it on the device.
cggm_status upload_csr(cggm_ctx *c, int64_t q, const int64_t *row_ptr, const int32_t *col,
                       const double *val, int64_t *nnz_out) {
    cudaStream_t st = c->st;
    int64_t nnz = 0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + q, sizeof(int64_t), cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    if (nnz < 1 || nnz > q * q || !col || !val) return CGGM_EINVAL;
    CGGM_TRY(ensure(c->cg_rp, 8 * (size_t)(q + 1)));
    CGGM_TRY(ensure(c->cg_ci, 4 * (size_t)nnz));
    CGGM_TRY(ensure(c->cg_v, 8 * (size_t)nnz));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->cg_rp.p, row_ptr, 8 * (size_t)(q + 1), cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->cg_ci.p, col, 4 * (size_t)nnz, cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(c->cg_v.p, val, 8 * (size_t)nnz, cudaMemcpyDefault, st));
    CGGM_TRY(ensure(c->err, sizeof(int)));
    CGGM_TRY(csr_check(q, nnz, P<int64_t>(c->cg_rp), P<int32_t>(c->cg_ci), P<int>(c->err), st));
    *nnz_out = nnz;
    return CGGM_OK;
}

cggm_status cggm_spd_solve(cggm_ctx *c, int64_t q, const int64_t *row_ptr, const int32_t *col,
                           const double *val, int64_t k, const double *B, int64_t c0, double tol,
                           int max_iter, double *X, int *iters_out, double *resid_out) {
    if (!c || q < 1 || k < 1 || !row_ptr || !X || !(tol > 0.0) || max_iter < 1) return CGGM_EINVAL;
    if (!B && (c0 < 0 || c0 + k > q)) return CGGM_EINVAL;
    CGGM_CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t st = c->st;
    int64_t nnz = 0;
    CGGM_TRY(upload_csr(c, q, row_ptr, col, val, &nnz));
    const size_t qk = (size_t)q * k;
    const double *dB = nullptr;
    if (B) {
        CGGM_TRY(ensure(c->cg_b, 8 * qk));
        CGGM_CUDA_TRY(cudaMemcpyAsync(c->cg_b.p, B, 8 * qk, cudaMemcpyDefault, st));
        dB = P<double>(c->cg_b);
    }
    double *dX = X;
    if (!is_device_ptr(X)) {
        CGGM_TRY(ensure(c->cg_x, 8 * qk));
        dX = P<double>(c->cg_x);
    }
    CGGM_TRY(ensure(c->cg_w, 8 * cg_work_doubles(q, k)));
    const CgWork w = cg_work_at(P<double>(c->cg_w), P<int>(c->err), q, k);
    const cggm_status s = pcg_solve(q, P<int64_t>(c->cg_rp), P<int32_t>(c->cg_ci),
                                    P<double>(c->cg_v), k, dB, c0, tol, max_iter, dX, w,
                                    iters_out, resid_out, st);
    if (s != CGGM_OK && s != CGGM_EMAXITER) return s;
    if (dX != X) CGGM_CUDA_TRY(cudaMemcpyAsync(X, dX, 8 * qk, cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

cggm_status cggm_grad_lambda_block(cggm_ctx *c, const void *X, int xdtype, const void *Y,
                                   int ydtype, int64_t n, int64_t p, int64_t q,
                                   const int64_t *row_ptr, const int32_t *col, const double *val,
                                   const double *Theta, int64_t c0, int64_t k, double tol,
                                   int max_iter, double *G_out, int *iters_out) {
    if (!c || !X || !Y || !row_ptr || !Theta || !G_out || k < 1 || c0 < 0 || !(tol > 0.0) ||
        max_iter < 1)
        return CGGM_EINVAL;
    if (!dtypes_ok(xdtype, ydtype)) return CGGM_EINVAL;
    CGGM_TRY(check_sizes(n, p, q));
    if (c0 + k > q) return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    cudaStream_t st = c->st;
    int64_t nnz = 0;
    CGGM_TRY(upload_csr(c, q, row_ptr, col, val, &nnz));
    CGGM_TRY(load_transposed(c, X, xdtype, n, p, c->Xt, nullptr));
    CGGM_TRY(load_transposed(c, Y, ydtype, n, q, c->Yt, nullptr));
    const size_t pq = (size_t)p * q, qn = (size_t)q * n, qk = (size_t)q * k;
    CGGM_TRY(load_double(c, Theta, pq, c->bk_th));
    CGGM_TRY(ensure(c->bk_rt, 8 * qn));
    CGGM_TRY(ensure(c->bk_pt, 8 * qn));
    CGGM_TRY(ensure(c->bk_sig, 8 * qk));
    CGGM_TRY(ensure(c->bk_psi, 8 * qk));
    CGGM_TRY(ensure(c->bk_g, 8 * qk));
    const int64_t kmax = n > k ? n : k;
    CGGM_TRY(ensure(c->cg_w, 8 * cg_work_doubles(q, kmax)));
    const CgWork w = cg_work_at(P<double>(c->cg_w), P<int>(c->err), q, kmax);
    const int64_t *rp = P<int64_t>(c->cg_rp);
    const int32_t *ci = P<int32_t>(c->cg_ci);
    const double *va = P<double>(c->cg_v);
    const double inv = 1.0 / (double)n;
    // R^T = Theta^T X^T (q x n); P^T = Sigma R^T from Lambda P^T = R^T; Sigma[:, C]
    theta_t_xt(p, q, n, P<double>(c->bk_th), P<double>(c->Xt), P<double>(c->bk_rt), st);
    int it1 = 0, it2 = 0;
    double res = 0.0;
    cggm_status s = pcg_solve(q, rp, ci, va, n, P<double>(c->bk_rt), 0, tol, max_iter,
                              P<double>(c->bk_pt), w, &it1, &res, st);
    if (s != CGGM_OK) return s;
    s = pcg_solve(q, rp, ci, va, k, nullptr, c0, tol, max_iter, P<double>(c->bk_sig), w, &it2,
                  &res, st);
    if (s != CGGM_OK) return s;
    // Psi[:, C] = P^T P_C / n and S_yy[:, C] = Y^T Y_C / n (both q x k), then
    // G_Lambda[:, C] = S_yy[:, C] - Sigma[:, C] - Psi[:, C]  (Eq. 3)
    gemm<double>(false, true, q, k, n, inv, P<double>(c->bk_pt), n, P<double>(c->bk_pt) + c0 * n,
                 n, 0.0, P<double>(c->bk_psi), k, st);
    gemm<double>(false, true, q, k, n, inv, P<double>(c->Yt), n, P<double>(c->Yt) + c0 * n, n,
                 0.0, P<double>(c->bk_g), k, st);
    axpby<double>((int64_t)qk, -1.0, P<double>(c->bk_sig), 1.0, P<double>(c->bk_g), st);
    axpby<double>((int64_t)qk, -1.0, P<double>(c->bk_psi), 1.0, P<double>(c->bk_g), st);
    CGGM_TRY(store_double(c, G_out, c->bk_g.p, qk));
    if (iters_out) *iters_out = it1 > it2 ? it1 : it2;
    return sync_err(c);
}

int cggm_tuned_batch(int64_t q, int64_t m, int precision) {
    if (q < 1 || m < 0 || (precision != CGGM_FP64 && precision != CGGM_MIXED)) return -1;
    return tuned_lookup(precision, q, m);
}

// The tuner's table as text: a comment line, then one line per size class,
// "precision log2_q log2_m batch".
cggm_status cggm_tuner_save(const char *path, int64_t *count_out) {
    if (!path) return CGGM_EINVAL;
    std::vector<std::pair<std::tuple<int, int, int>, int>> rows;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        rows.assign(g_tuned.begin(), g_tuned.end());
    }
    FILE *f = std::fopen(path, "w");
    if (!f) return CGGM_EINVAL;
    bool ok = std::fprintf(f, "# cggm batch-size tuner table: precision log2_q log2_m batch\n") > 0;
    for (const auto &r : rows)
        ok = ok && std::fprintf(f, "%d %d %d %d\n", std::get<0>(r.first), std::get<1>(r.first),
                                std::get<2>(r.first), r.second) > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return CGGM_EINVAL;
    if (count_out) *count_out = (int64_t)rows.size();
    return CGGM_OK;
}

cggm_status cggm_tuner_load(const char *path, int64_t *count_out) {
    if (!path) return CGGM_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return CGGM_EINVAL;
    std::vector<std::pair<std::tuple<int, int, int>, int>> rows;
    char line[256];
    bool ok = true;
    while (ok && std::fgets(line, sizeof line, f)) {
        const char *c = line;
        while (*c == ' ' || *c == '\t') c++;
        if (*c == '#' || *c == '\n' || *c == '\r' || *c == 0) continue;
        int prec = -1, lq = -1, lm = -1, B = 0, used = 0;
        if (std::sscanf(c, "%d %d %d %d %n", &prec, &lq, &lm, &B, &used) != 4 || c[used] != 0) {
            ok = false;
            break;
        }
        const bool batch_ok = B == 32 || B == 64 || B == 128 ||
                              (prec == CGGM_MIXED && (B == 256 || B == 512));
        if ((prec != CGGM_FP64 && prec != CGGM_MIXED) || lq < 0 || lq > 62 || lm < 0 ||
            lm > 62 || !batch_ok)
            ok = false;
        else
            rows.push_back({std::make_tuple(prec, lq, lm), B});
    }
    std::fclose(f);
    if (!ok) return CGGM_EINVAL;  // nothing merged from a malformed file
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        for (const auto &r : rows) g_tuned[r.first] = r.second;
    }
    if (count_out) *count_out = (int64_t)rows.size();
    return CGGM_OK;
}

cggm_status cggm_contract(cggm_ctx *c, int64_t M, int64_t N, int64_t K, float alpha,
                          const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
                          float *C, int64_t ldc, int mode) {
    if (!c || !A || !B || !C || M < 0 || N < 0 || K <= 0 || ldc < N) return CGGM_EINVAL;
    if ((mode != 0 && mode != 1) || lda < K || ldb < K) return CGGM_EINVAL;
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    CGGM_TRY(ensure(c->err, sizeof(int)));
    CGGM_CUDA_TRY(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->st));
    if (mode == 0) {
        CGGM_TRY(gemm_tc_nt(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, false, nullptr, nullptr,
                            P<int>(c->err), c->st));
    } else {
        CGGM_TRY(ensure(c->tcA_hi, 4 * (size_t)M * lda));
        CGGM_TRY(ensure(c->tcA_lo, 4 * (size_t)M * lda));
        CGGM_TRY(ensure(c->tcB_hi, 4 * (size_t)N * ldb));
        CGGM_TRY(ensure(c->tcB_lo, 4 * (size_t)N * ldb));
        split_tf32(M, K, lda, A, P<float>(c->tcA_hi), P<float>(c->tcA_lo), c->st);
        split_tf32(N, K, ldb, B, P<float>(c->tcB_hi), P<float>(c->tcB_lo), c->st);
        CGGM_TRY(gemm_tc_nt(M, N, K, alpha, P<float>(c->tcA_hi), lda, P<float>(c->tcB_hi), ldb,
                            beta, C, ldc, true, P<float>(c->tcA_lo), P<float>(c->tcB_lo),
                            P<int>(c->err), c->st));
    }
    int h = 0;
    CGGM_TRY(read_dev_err(c, &h));
    if (h == DEV_TIMEOUT) return CGGM_ETIMEDOUT;
    if (h != 0) return CGGM_ECUDA;
    return CGGM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Numeric sparse Cholesky (spchol.cu): a plan bound to a context's device and stream.
// ---------------------------------------------------------------------------------
struct cggm_spchol {
    cggm_ctx *ctx;
    SpCholPlan *plan;
};

extern "C" cggm_status cggm_spchol_create(cggm_ctx *c, int64_t q, const int64_t *row_ptr,
                                          const int32_t *col, int ordering,
                                          const int32_t *perm_in, cggm_spchol **out) {
    if (!out) return CGGM_EINVAL;
    *out = nullptr;
    if (!c) return CGGM_EINVAL;
    CGGM_TRY(set_device(c));
    SpCholPlan *p = nullptr;
    CGGM_TRY(spchol_analyse(c->device, q, row_ptr, col, ordering, perm_in, &p));
    *out = new cggm_spchol{c, p};
    return CGGM_OK;
}

extern "C" cggm_status cggm_spchol_factor(cggm_spchol *f, const double *val,
                                          double *logdet_out) {
    if (!f) return CGGM_EINVAL;
    CGGM_TRY(set_device(f->ctx));
    return spchol_factor(f->plan, val, logdet_out, f->ctx->st);
}

extern "C" cggm_status cggm_spchol_solve(cggm_spchol *f, int64_t k, const double *B,
                                         int64_t c0, double *X) {
    if (!f) return CGGM_EINVAL;
    CGGM_TRY(set_device(f->ctx));
    return spchol_solve(f->plan, k, B, c0, X, f->ctx->st);
}

extern "C" cggm_status cggm_spchol_export(cggm_spchol *f, int64_t *nsuper_out,
                                          int64_t *nblock_out, int64_t *nnz_L_out,
                                          int32_t *perm_out, int64_t *super_start_out,
                                          int64_t *rows_ptr_out, int32_t *rows_out,
                                          int64_t *block_ptr_out, double *blocks_out) {
    if (!f) return CGGM_EINVAL;
    return spchol_export(f->plan, nsuper_out, nblock_out, nnz_L_out, perm_out, super_start_out,
                         rows_ptr_out, rows_out, block_ptr_out, blocks_out, f->ctx->st);
}

extern "C" cggm_status cggm_spchol_destroy(cggm_spchol *f) {
    if (!f) return CGGM_OK;
    spchol_free(f->plan);
    delete f;
    return CGGM_OK;
}
