// Numeric sparse Cholesky in double precision (Section 4: the block regime of Algorithm 2
// keeps Lambda sparse, and the Armijo rule of Algorithm 1 needs log det(Lambda + alpha D)
// and the positive definiteness that a factorisation certifies; Section 2.3 takes both from
// a Cholesky factor.  Columns of Sigma = Lambda^-1 follow from two triangular solves with
// the same factor).
//
// The symbolic half (pivot order, elimination tree, column counts, fundamental supernodes
// and their row structure) is host code in symbolic.cpp.  This file adds:
//   - the plan: device copies of that structure; the slot in L of every lower-triangle
//     entry of the input; and for each supernode t the increasing list of the supernodes
//     whose rows meet t's columns, which are exactly the ones whose columns update t;
//   - the factorisation, one persistent kernel: each CTA takes supernodes in increasing
//     order from a counter.  A supernode waits until its children in the supernodal tree
//     have finished (then all its descendants have), subtracts the updates of the
//     supernodes in its list in list order (left-looking: the result does not depend on
//     which CTA ran what, or when), factors its dense block of columns and counts itself
//     off its parent.  Supernodes are numbered so that children come before their parent,
//     so a CTA only ever waits for supernodes that running CTAs have already taken;
//   - log det = 2 sum_k log L_kk, summed in a fixed order;
//   - the solve A X = B through P A P^T = L L^T (forward, then backward substitution over
//     the supernodes), one thread per right-hand side column.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "chol.cuh"
#include "common.cuh"
#include "spchol.cuh"

namespace cggm {

namespace {

constexpr int kFactorThreads = 256;
constexpr int kMapChunk = 1024;             // rows of an updating supernode mapped at a time
constexpr uint64_t kWaitNs = 10000000000ull;  // a supernode's wait for its children

struct SpDev {
    int32_t nsuper;
    const int32_t *sstart;   // nsuper + 1: columns of supernode s are sstart[s] .. sstart[s+1]-1
    const int64_t *rptr;     // nsuper + 1: its rows are rows[rptr[s] .. rptr[s+1]), sorted
    const int32_t *rows;
    const int64_t *loff;     // its dense block of L: nr x nc row-major at L + loff[s]
    const int32_t *sparent;  // parent supernode, -1 for a root
    const int64_t *uptr;     // nsuper + 1
    const int32_t *ulist;    // the supernodes updating s, increasing
    double *L;
    double *logd;            // q: log L_kk
    int *pending;            // nsuper: children not yet finished
    unsigned *next;          // the next supernode to take
    int *err;
};

__device__ __forceinline__ int lower_pos(const int32_t *r, int n, int32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (r[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kFactorThreads) spchol_factor_kernel(SpDev d) {
    __shared__ int s_task;
    __shared__ int s_map[kMapChunk];
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_task = (int)atomicAdd(d.next, 1u);
        __syncthreads();
        const int t = s_task;
        if (t >= d.nsuper) return;
        if (tid == 0) {
            const uint64_t t0 = global_ns();
            while (ld_acquire_int(d.pending + t) > 0) {
                // after one wait has given up, the others leave at once
                if (ld_acquire_int(d.err) == (int)DEV_TIMEOUT) break;
                if (global_ns() - t0 > kWaitNs) {
                    atomicCAS(d.err, 0, (int)DEV_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
            __threadfence();
        }
        __syncthreads();

        const int f = d.sstart[t], nc = d.sstart[t + 1] - f;
        const int64_t r0 = d.rptr[t];
        const int nr = (int)(d.rptr[t + 1] - r0);
        const int32_t *rt = d.rows + r0;
        double *B = d.L + d.loff[t];

        // 1. updates from the supernodes whose rows meet columns f .. f + nc - 1
        for (int64_t u = d.uptr[t]; u < d.uptr[t + 1]; u++) {
            const int s = d.ulist[u];
            const int ncs = d.sstart[s + 1] - d.sstart[s];
            const int64_t rs0 = d.rptr[s];
            const int nrs = (int)(d.rptr[s + 1] - rs0);
            const int32_t *rs = d.rows + rs0;
            const double *Ls = d.L + d.loff[s];
            // rows of s at positions [p0, p1) are columns of t; those from p0 on lie in t's
            // structure (the structure of a column contains that of its descendants' below it)
            const int p0 = ncs + lower_pos(rs + ncs, nrs - ncs, f);
            const int p1 = p0 + lower_pos(rs + p0, nrs - p0, f + nc);
            const int nb = p1 - p0;
            if (nb <= 0) continue;
            for (int a0 = p0; a0 < nrs; a0 += kMapChunk) {
                const int na = min(kMapChunk, nrs - a0);
                for (int a = tid; a < na; a += kFactorThreads) {
                    const int32_t key = rs[a0 + a];
                    const int pos = lower_pos(rt, nr, key);
                    s_map[a] = (pos < nr && rt[pos] == key) ? pos : -1;
                }
                __syncthreads();
                const int64_t npairs = (int64_t)na * nb;
                for (int64_t e = tid; e < npairs; e += kFactorThreads) {
                    const int a = a0 + (int)(e / nb), b = p0 + (int)(e % nb);
                    if (a < b) continue;  // upper triangle of the diagonal block
                    const int pa = s_map[a - a0];
                    if (pa < 0) {
                        atomicCAS(d.err, 0, (int)DEV_BADINDEX);
                        continue;
                    }
                    const double *la = Ls + (int64_t)a * ncs, *lb = Ls + (int64_t)b * ncs;
                    double v = 0.0;
                    for (int k = 0; k < ncs; k++) v = fma(la[k], lb[k], v);
                    B[(int64_t)pa * nc + (rs[b] - f)] -= v;
                }
                __syncthreads();
            }
        }

        // 2. dense factorisation of the supernode's columns (right-looking inside the block)
        for (int j = 0; j < nc; j++) {
            if (tid == 0) {
                double dj = B[(int64_t)j * nc + j];
                if (!(dj > 0.0) || !isfinite(dj)) {
                    atomicCAS(d.err, 0, (int)DEV_NOTPD);
                    dj = 1.0;  // keep the rest finite; the result is discarded
                }
                dj = sqrt(dj);
                B[(int64_t)j * nc + j] = dj;
                d.logd[f + j] = log(dj);
            }
            __syncthreads();
            const double piv = B[(int64_t)j * nc + j];
            for (int i = j + 1 + tid; i < nr; i += kFactorThreads) B[(int64_t)i * nc + j] /= piv;
            __syncthreads();
            const int w = nc - j - 1;
            if (w > 0) {
                const int64_t h = nr - j - 1, total = h * w;
                for (int64_t e = tid; e < total; e += kFactorThreads) {
                    const int i = j + 1 + (int)(e / w), k = j + 1 + (int)(e % w);
                    if (k > i) continue;
                    B[(int64_t)i * nc + k] -= B[(int64_t)i * nc + j] * B[(int64_t)k * nc + j];
                }
                __syncthreads();
            }
        }

        // 3. count this supernode off its parent (its writes ordered before by the fence)
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const int par = d.sparent[t];
            if (par >= 0) atomicSub(d.pending + par, 1);
        }
    }
}

// L's slots from the input's lower-triangle entries: slot u receives the sum, in input
// order, of the entries uent[uptr[u] .. uptr[u+1]) (repeated entries add up); every other
// slot of L is zero.
__global__ void spchol_assemble_kernel(int64_t nu, const int64_t *__restrict__ uslot,
                                       const int64_t *__restrict__ uptr,
                                       const int64_t *__restrict__ uent,
                                       const double *__restrict__ val, double *L, int *err) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t t = uptr[u]; t < uptr[u + 1]; t++) {
            const double v = val[uent[t]];
            if (!isfinite(v)) atomicCAS(err, 0, (int)DEV_NONFINITE);
            s += v;
        }
        L[uslot[u]] = s;
    }
}

// X = A^-1 B for the factored A (P A P^T = L L^T), one thread per column c < k of B
// (q x k row-major; NULL for the identity columns c0 .. c0 + k - 1).  W: q x k scratch.
__global__ void __launch_bounds__(128)
spchol_solve_kernel(SpDev d, int64_t q, int64_t k, const int32_t *__restrict__ perm,
                    const double *__restrict__ Bin, int64_t c0, double *W, double *X) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= k) return;
    for (int64_t r = 0; r < q; r++)
        W[r * k + c] = Bin ? Bin[(int64_t)perm[r] * k + c] : (perm[r] == c0 + c ? 1.0 : 0.0);
    // L y = P b
    for (int s = 0; s < d.nsuper; s++) {
        const int f = d.sstart[s], nc = d.sstart[s + 1] - f;
        const int64_t r0 = d.rptr[s];
        const int nr = (int)(d.rptr[s + 1] - r0);
        const int32_t *rw = d.rows + r0;
        const double *Bk = d.L + d.loff[s];
        for (int j = 0; j < nc; j++) {
            const double y = W[(int64_t)(f + j) * k + c] / Bk[(int64_t)j * nc + j];
            W[(int64_t)(f + j) * k + c] = y;
            for (int i = j + 1; i < nr; i++) W[(int64_t)rw[i] * k + c] -= Bk[(int64_t)i * nc + j] * y;
        }
    }
    // L^T z = y
    for (int s = d.nsuper - 1; s >= 0; s--) {
        const int f = d.sstart[s], nc = d.sstart[s + 1] - f;
        const int64_t r0 = d.rptr[s];
        const int nr = (int)(d.rptr[s + 1] - r0);
        const int32_t *rw = d.rows + r0;
        const double *Bk = d.L + d.loff[s];
        for (int j = nc - 1; j >= 0; j--) {
            double v = W[(int64_t)(f + j) * k + c];
            for (int i = j + 1; i < nr; i++) v -= Bk[(int64_t)i * nc + j] * W[(int64_t)rw[i] * k + c];
            W[(int64_t)(f + j) * k + c] = v / Bk[(int64_t)j * nc + j];
        }
    }
    for (int64_t r = 0; r < q; r++) X[(int64_t)perm[r] * k + c] = W[r * k + c];
}

template <typename T>
cggm_status upload(std::vector<void *> &owned, T **dst, const std::vector<T> &src) {
    const size_t bytes = std::max<size_t>(sizeof(T) * src.size(), 16);
    void *p = nullptr;
    CGGM_CUDA_TRY(cudaMalloc(&p, bytes));
    owned.push_back(p);
    if (!src.empty()) CGGM_CUDA_TRY(cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    *dst = static_cast<T *>(p);
    return CGGM_OK;
}

cggm_status alloc(std::vector<void *> &owned, void **dst, size_t bytes) {
    void *p = nullptr;
    CGGM_CUDA_TRY(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
    owned.push_back(p);
    *dst = p;
    return CGGM_OK;
}

}  // namespace

struct SpCholPlan {
    int device = 0;
    int64_t q = 0, nnz_in = 0, nsuper = 0, nblock = 0, nnz_L = 0, nu = 0;
    std::vector<int32_t> perm;
    std::vector<int64_t> super_start, rows_ptr, loff;
    std::vector<int32_t> rows;
    std::vector<int32_t> kids;  // children per supernode (the pending counts' reset value)
    std::vector<void *> owned;  // device allocations
    int32_t *d_sstart = nullptr, *d_rows = nullptr, *d_sparent = nullptr, *d_ulist = nullptr,
            *d_perm = nullptr, *d_kids = nullptr, *d_pending = nullptr;
    int64_t *d_rptr = nullptr, *d_loff = nullptr, *d_uptr = nullptr, *d_uslot = nullptr,
            *d_uvptr = nullptr, *d_uent = nullptr;
    double *d_L = nullptr, *d_logd = nullptr, *d_val = nullptr, *d_scal = nullptr;
    unsigned *d_next = nullptr;
    int *d_err = nullptr;
    void *d_W = nullptr, *d_B = nullptr, *d_X = nullptr;
    size_t solve_bytes = 0;
    bool factored = false;

    SpDev dev() const {
        SpDev d;
        d.nsuper = (int32_t)nsuper;
        d.sstart = d_sstart;
        d.rptr = d_rptr;
        d.rows = d_rows;
        d.loff = d_loff;
        d.sparent = d_sparent;
        d.uptr = d_uptr;
        d.ulist = d_ulist;
        d.L = d_L;
        d.logd = d_logd;
        d.pending = d_pending;
        d.next = d_next;
        d.err = d_err;
        return d;
    }
};

cggm_status spchol_analyse(int device, int64_t q, const int64_t *row_ptr, const int32_t *col,
                           int ordering, const int32_t *perm_in, SpCholPlan **out) {
    if (!out) return CGGM_EINVAL;
    *out = nullptr;
    if (q < 1 || q > INT32_MAX || !row_ptr || !col) return CGGM_EINVAL;
    std::vector<int32_t> perm(q), parent(q);
    std::vector<int64_t> colcount(q);
    int64_t nnz_L = 0;
    CGGM_TRY(cggm_chol_symbolic(q, row_ptr, col, ordering, perm_in, perm.data(), parent.data(),
                                colcount.data(), &nnz_L));
    std::vector<int64_t> start(q + 1);
    int64_t ns = 0;
    CGGM_TRY(cggm_chol_supernodes(q, parent.data(), colcount.data(), start.data(), &ns));
    start.resize(ns + 1);
    std::vector<int64_t> rptr(ns + 1);
    CGGM_TRY(cggm_chol_structure(q, row_ptr, col, perm.data(), parent.data(), colcount.data(), ns,
                                 start.data(), rptr.data(), nullptr));
    std::vector<int32_t> rows(rptr[ns]);
    CGGM_TRY(cggm_chol_structure(q, row_ptr, col, perm.data(), parent.data(), colcount.data(), ns,
                                 start.data(), rptr.data(), rows.data()));

    std::vector<int32_t> snode(q), iperm(q), sstart(ns + 1), sparent(ns, -1), kids(ns, 0);
    std::vector<int64_t> loff(ns + 1, 0);
    for (int64_t k = 0; k < q; k++) iperm[perm[k]] = (int32_t)k;
    for (int64_t s = 0; s < ns; s++) {
        sstart[s] = (int32_t)start[s];
        const int64_t nc = start[s + 1] - start[s], nr = rptr[s + 1] - rptr[s];
        if (nr * nc > INT32_MAX) return CGGM_ENOMEM;  // one supernode's block beyond int range
        loff[s + 1] = loff[s] + nr * nc;
        for (int64_t k = start[s]; k < start[s + 1]; k++) snode[k] = (int32_t)s;
    }
    sstart[ns] = (int32_t)q;
    for (int64_t s = 0; s < ns; s++) {
        const int32_t par = parent[start[s + 1] - 1];
        if (par >= 0) {
            sparent[s] = snode[par];
            kids[snode[par]]++;
        }
    }
    // update lists: s updates t when a row of s below its own columns is a column of t
    std::vector<int64_t> uptr(ns + 1, 0);
    std::vector<int32_t> mark(ns, -1);
    for (int64_t s = 0; s < ns; s++) {
        const int64_t nc = start[s + 1] - start[s];
        for (int64_t e = rptr[s] + nc; e < rptr[s + 1]; e++) {
            const int32_t t = snode[rows[e]];
            if (mark[t] != s) {
                mark[t] = (int32_t)s;
                uptr[t + 1]++;
            }
        }
    }
    for (int64_t t = 0; t < ns; t++) uptr[t + 1] += uptr[t];
    std::vector<int32_t> ulist(uptr[ns]);
    {
        std::vector<int64_t> fill(uptr.begin(), uptr.end() - 1);
        std::fill(mark.begin(), mark.end(), -1);
        for (int64_t s = 0; s < ns; s++) {  // increasing s: each list comes out increasing
            const int64_t nc = start[s + 1] - start[s];
            for (int64_t e = rptr[s] + nc; e < rptr[s + 1]; e++) {
                const int32_t t = snode[rows[e]];
                if (mark[t] != s) {
                    mark[t] = (int32_t)s;
                    ulist[fill[t]++] = (int32_t)s;
                }
            }
        }
    }
    // slots of the input's lower-triangle entries (row >= col, original numbering)
    const int64_t nnz_in = row_ptr[q];
    std::vector<std::pair<int64_t, int64_t>> se;  // (slot, entry)
    se.reserve(nnz_in);
    for (int64_t i = 0; i < q; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            const int64_t j = col[e];
            if (j > i) continue;
            const int32_t I = iperm[i], J = iperm[j];
            const int32_t R = std::max(I, J), C = std::min(I, J);
            const int32_t s = snode[C];
            const int32_t *rb = rows.data() + rptr[s], *re = rows.data() + rptr[s + 1];
            const int32_t *hit = std::lower_bound(rb, re, R);
            if (hit == re || *hit != R) return CGGM_EINVAL;  // not from one analysis
            const int64_t nc = start[s + 1] - start[s];
            se.emplace_back(loff[s] + (int64_t)(hit - rb) * nc + (C - start[s]), e);
        }
    std::stable_sort(se.begin(), se.end(),
                     [](const std::pair<int64_t, int64_t> &a, const std::pair<int64_t, int64_t> &b) {
                         return a.first < b.first;
                     });
    std::vector<int64_t> uslot, uvptr(1, 0), uent(se.size());
    for (size_t e = 0; e < se.size(); e++) {
        if (e == 0 || se[e].first != se[e - 1].first) {
            if (e > 0) uvptr.push_back((int64_t)e);
            uslot.push_back(se[e].first);
        }
        uent[e] = se[e].second;
    }
    uvptr.push_back((int64_t)se.size());
    if (se.empty()) uvptr.assign(1, 0);

    SpCholPlan *P = new SpCholPlan;
    P->device = device;
    P->q = q;
    P->nnz_in = nnz_in;
    P->nsuper = ns;
    P->nblock = loff[ns];
    P->nnz_L = nnz_L;
    P->nu = (int64_t)uslot.size();
    P->perm = perm;
    P->super_start = start;
    P->rows_ptr = rptr;
    P->rows = rows;
    P->loff = loff;
    P->kids = kids;
    auto fail = [&](cggm_status st) {
        spchol_free(P);
        return st;
    };
    cggm_status st;
#define SP_UP(dst, src)                                         \
    if ((st = upload(P->owned, &P->dst, src)) != CGGM_OK) return fail(st)
    SP_UP(d_sstart, sstart);
    SP_UP(d_rows, rows);
    SP_UP(d_sparent, sparent);
    SP_UP(d_ulist, ulist);
    SP_UP(d_perm, perm);
    SP_UP(d_kids, kids);
    SP_UP(d_pending, kids);
    SP_UP(d_rptr, rptr);
    SP_UP(d_loff, loff);
    SP_UP(d_uptr, uptr);
    SP_UP(d_uslot, uslot);
    SP_UP(d_uvptr, uvptr);
    SP_UP(d_uent, uent);
#undef SP_UP
    void *p = nullptr;
    if ((st = alloc(P->owned, &p, 8 * (size_t)P->nblock)) != CGGM_OK) return fail(st);
    P->d_L = static_cast<double *>(p);
    if ((st = alloc(P->owned, &p, 8 * (size_t)q)) != CGGM_OK) return fail(st);
    P->d_logd = static_cast<double *>(p);
    if ((st = alloc(P->owned, &p, 8 * (size_t)nnz_in)) != CGGM_OK) return fail(st);
    P->d_val = static_cast<double *>(p);
    if ((st = alloc(P->owned, &p, 8)) != CGGM_OK) return fail(st);
    P->d_scal = static_cast<double *>(p);
    if ((st = alloc(P->owned, &p, sizeof(unsigned))) != CGGM_OK) return fail(st);
    P->d_next = static_cast<unsigned *>(p);
    if ((st = alloc(P->owned, &p, sizeof(int))) != CGGM_OK) return fail(st);
    P->d_err = static_cast<int *>(p);
    *out = P;
    return CGGM_OK;
}

void spchol_free(SpCholPlan *P) {
    if (!P) return;
    cudaSetDevice(P->device);
    for (void *p : P->owned) cudaFree(p);
    if (P->d_W) cudaFree(P->d_W);
    if (P->d_B) cudaFree(P->d_B);
    if (P->d_X) cudaFree(P->d_X);
    delete P;
}

namespace {
cggm_status read_status(SpCholPlan *P, cudaStream_t st) {
    int e = 0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&e, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    CGGM_CUDA_TRY(cudaGetLastError());
    switch (e) {
        case DEV_OK: return CGGM_OK;
        case DEV_NOTPD: return CGGM_ENOTPD;
        case DEV_NONFINITE: return CGGM_ENONFINITE;
        case DEV_TIMEOUT: return CGGM_ETIMEDOUT;
        default: return CGGM_ECUDA;
    }
}
}  // namespace

cggm_status spchol_factor_device(SpCholPlan *P, const double *d_vals, cudaStream_t st) {
    P->factored = false;
    CGGM_CUDA_TRY(cudaMemsetAsync(P->d_err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(P->d_next, 0, sizeof(unsigned), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(P->d_L, 0, 8 * (size_t)P->nblock, st));
    CGGM_CUDA_TRY(cudaMemcpyAsync(P->d_pending, P->d_kids, 4 * (size_t)P->nsuper,
                                  cudaMemcpyDeviceToDevice, st));
    if (P->nu > 0) {
        const int64_t g = std::min<int64_t>((P->nu + 255) / 256, (int64_t)sm_count() * 8);
        note_launch();
        spchol_assemble_kernel<<<(unsigned)std::max<int64_t>(g, 1), 256, 0, st>>>(
            P->nu, P->d_uslot, P->d_uvptr, P->d_uent, d_vals, P->d_L, P->d_err);
    }
    // every CTA takes supernodes until none is left; a few per SM keep independent
    // subtrees going side by side
    const int64_t grid = std::min<int64_t>(P->nsuper, (int64_t)sm_count() * 4);
    note_launch();
    spchol_factor_kernel<<<(unsigned)grid, kFactorThreads, 0, st>>>(P->dev());
    logdet_from_logd(P->q, P->d_logd, P->d_scal, st);
    CGGM_CUDA_TRY(cudaGetLastError());
    return CGGM_OK;
}

cggm_status spchol_factor(SpCholPlan *P, const double *val, double *logdet_out,
                          cudaStream_t st) {
    if (!P || (!val && P->nnz_in > 0)) return CGGM_EINVAL;
    CGGM_CUDA_TRY(cudaSetDevice(P->device));
    if (P->nnz_in > 0)
        CGGM_CUDA_TRY(cudaMemcpyAsync(P->d_val, val, 8 * (size_t)P->nnz_in, cudaMemcpyDefault, st));
    CGGM_TRY(spchol_factor_device(P, P->d_val, st));
    double h = 0.0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&h, P->d_scal, 8, cudaMemcpyDeviceToHost, st));
    const cggm_status s = read_status(P, st);
    if (s != CGGM_OK) return s;
    P->factored = true;
    if (logdet_out) *logdet_out = h;
    return CGGM_OK;
}

cggm_status spchol_solve(SpCholPlan *P, int64_t k, const double *B, int64_t c0, double *X,
                         cudaStream_t st) {
    if (!P || k < 1 || !X) return CGGM_EINVAL;
    if (!B && (c0 < 0 || c0 + k > P->q)) return CGGM_EINVAL;
    if (!P->factored) return CGGM_EINVAL;
    CGGM_CUDA_TRY(cudaSetDevice(P->device));
    const size_t bytes = 8 * (size_t)P->q * (size_t)k;
    if (P->solve_bytes < bytes) {
        if (P->d_W) cudaFree(P->d_W);
        if (P->d_B) cudaFree(P->d_B);
        if (P->d_X) cudaFree(P->d_X);
        P->d_W = P->d_B = P->d_X = nullptr;
        P->solve_bytes = 0;
        CGGM_CUDA_TRY(cudaMalloc(&P->d_W, bytes));
        CGGM_CUDA_TRY(cudaMalloc(&P->d_B, bytes));
        CGGM_CUDA_TRY(cudaMalloc(&P->d_X, bytes));
        P->solve_bytes = bytes;
    }
    const double *dB = nullptr;
    if (B) {
        CGGM_CUDA_TRY(cudaMemcpyAsync(P->d_B, B, bytes, cudaMemcpyDefault, st));
        dB = static_cast<const double *>(P->d_B);
    }
    note_launch();
    spchol_solve_kernel<<<ceil_div(k, 128), 128, 0, st>>>(P->dev(), P->q, k, P->d_perm, dB, c0,
                                                          static_cast<double *>(P->d_W),
                                                          static_cast<double *>(P->d_X));
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_CUDA_TRY(cudaMemcpyAsync(X, P->d_X, bytes, cudaMemcpyDefault, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    return CGGM_OK;
}

cggm_status spchol_export(SpCholPlan *P, int64_t *nsuper_out, int64_t *nblock_out,
                          int64_t *nnz_L_out, int32_t *perm_out, int64_t *super_start_out,
                          int64_t *rows_ptr_out, int32_t *rows_out, int64_t *block_ptr_out,
                          double *blocks_out, cudaStream_t st) {
    if (!P) return CGGM_EINVAL;
    if (nsuper_out) *nsuper_out = P->nsuper;
    if (nblock_out) *nblock_out = P->nblock;
    if (nnz_L_out) *nnz_L_out = P->nnz_L;
    if (perm_out) std::memcpy(perm_out, P->perm.data(), 4 * (size_t)P->q);
    if (super_start_out) std::memcpy(super_start_out, P->super_start.data(), 8 * (size_t)(P->nsuper + 1));
    if (rows_ptr_out) std::memcpy(rows_ptr_out, P->rows_ptr.data(), 8 * (size_t)(P->nsuper + 1));
    if (rows_out) std::memcpy(rows_out, P->rows.data(), 4 * P->rows.size());
    if (block_ptr_out) std::memcpy(block_ptr_out, P->loff.data(), 8 * (size_t)(P->nsuper + 1));
    if (blocks_out) {
        if (!P->factored) return CGGM_EINVAL;
        CGGM_CUDA_TRY(cudaSetDevice(P->device));
        CGGM_CUDA_TRY(cudaMemcpyAsync(blocks_out, P->d_L, 8 * (size_t)P->nblock,
                                      cudaMemcpyDeviceToHost, st));
        CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return CGGM_OK;
}

}  // namespace cggm
