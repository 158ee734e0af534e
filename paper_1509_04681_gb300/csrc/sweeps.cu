// Coordinate-descent passes of the alternating Newton method, as blocked exact
// Gauss-Seidel on the GPU.
//
// The pass visits the active coordinates in order, and each step depends on all the
// steps before it through the cache (U = D Sigma for Lambda, Section 3.1; Delta V =
// Delta Theta Sigma for Theta, Section 3.2).  The GPU form keeps that order and that
// arithmetic exactly, up to the order of floating-point sums, by cutting the list into
// batches of B consecutive coordinates:
//   phase A (all CTAs): for every coordinate of the batch, the dot products against the
//           cache as it stands at the start of the batch; the cache is read row by row
//           (row t at the batch's column indices), so each CTA owns a band of rows and
//           produces partial sums.  The same phase gathers the small submatrices of
//           Sigma / Psi / S_xx on the batch's indices.
//   phase B (the last CTA to finish A): sums the partials in a fixed order, then one
//           warp runs the B coordinate steps in order.  A step's dot products differ
//           from their batch-start values only by the updates of the earlier steps of
//           the same batch, and those corrections are bilinear in entries of the
//           gathered submatrices, so the warp applies them exactly (forward
//           substitution with a soft-threshold at every step).
//   phase C (all CTAs): applies the batch's B updates to the cache rows.
// A grid barrier separates C from the next batch's A, and B from C.
#include "sweeps.cuh"

#include <cooperative_groups.h>

namespace cggm {

namespace {
constexpr int kThreads = 256;

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// ---------------------------------------------------------------------------------
// batch plans
// ---------------------------------------------------------------------------------
// Bitonic sort of K (power of two) ints in shared memory, ascending.
__device__ void bitonic_sort(int *key, int K) {
    for (int size = 2; size <= K; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int t = threadIdx.x; t < K / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const int a = key[lo], b = key[hi];
                if ((a > b) == up) { key[lo] = b; key[hi] = a; }
            }
        }
    }
    __syncthreads();
}

// Sort, deduplicate; returns count, writes the distinct values to out[0..count).
__device__ int sort_unique(int *key, int K, int32_t *out, int *s_cnt) {
    bitonic_sort(key, K);
    if (threadIdx.x == 0) {
        int c = 0;
        for (int k = 0; k < K; k++) {
            const int v = key[k];
            if (v == INT_MAX) break;
            if (c == 0 || out[c - 1] != v) out[c++] = v;
        }
        *s_cnt = c;
    }
    __syncthreads();
    return *s_cnt;
}

__device__ int lower_bound(const int32_t *a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Lambda plan: one index set (both coordinates of (a, b) index q); lists per distinct
// index u: every coordinate with a == u (partner b) and with b == u != a (partner a).
__global__ void lambda_plan_kernel(int64_t m, const int32_t *ai, const int32_t *aj, int B,
                                   BatchPlan plan) {
    extern __shared__ int smem_i[];
    const int K = 2 * B;
    int *key = smem_i;              // K
    int32_t *sidx = key + K;        // K
    int *cnt = sidx + K;            // K + 1
    __shared__ int s_cnt;
    const int64_t b = blockIdx.x;
    const int64_t s = b * B;
    const int nb = (int)((m - s) < B ? (m - s) : B);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int l = k >> 1;
        key[k] = (l < nb) ? ((k & 1) ? aj[s + l] : ai[s + l]) : INT_MAX;
    }
    const int nidx = sort_unique(key, K, sidx, &s_cnt);
    int32_t *idx = plan.idx + b * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) idx[k] = (k < nidx) ? sidx[k] : 0;
    for (int l = threadIdx.x; l < B; l += blockDim.x) {
        int pa = 0, pb = 0;
        if (l < nb) {
            pa = lower_bound(sidx, nidx, ai[s + l]);
            pb = lower_bound(sidx, nidx, aj[s + l]);
        }
        plan.pa[b * B + l] = pa;
        plan.pb[b * B + l] = pb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        plan.nidx[b] = nidx;
        for (int k = 0; k <= K; k++) cnt[k] = 0;
        for (int l = 0; l < nb; l++) {
            const int pa = plan.pa[b * B + l], pb = plan.pb[b * B + l];
            cnt[pa + 1]++;
            if (pa != pb) cnt[pb + 1]++;
        }
        for (int k = 0; k < K; k++) cnt[k + 1] += cnt[k];
        int32_t *lptr = plan.lptr + b * (K + 1);
        for (int k = 0; k <= K; k++) lptr[k] = cnt[k];
        int32_t *lent = plan.lent + b * K;
        for (int l = 0; l < nb; l++) {
            const int pa = plan.pa[b * B + l], pb = plan.pb[b * B + l];
            lent[cnt[pa]++] = (l << 16) | pb;
            if (pa != pb) lent[cnt[pb]++] = (l << 16) | pa;
        }
    }
}

// Theta plan: distinct i (idx) and distinct j (idx2); lists per distinct i: every
// coordinate of that row (partner = position of its j in idx2).
__global__ void theta_plan_kernel(int64_t m, const int32_t *ti, const int32_t *tj, int B,
                                  BatchPlan plan) {
    extern __shared__ int smem_i[];
    const int K = 2 * B;
    int *key = smem_i;            // K
    int32_t *sI = key + K;        // K
    int32_t *sJ = sI + K;         // K
    int *cnt = sJ + K;            // K + 1
    __shared__ int s_cnt;
    const int64_t b = blockIdx.x;
    const int64_t s = b * B;
    const int nb = (int)((m - s) < B ? (m - s) : B);
    for (int k = threadIdx.x; k < K; k += blockDim.x) key[k] = (k < nb) ? ti[s + k] : INT_MAX;
    const int nI = sort_unique(key, K, sI, &s_cnt);
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) key[k] = (k < nb) ? tj[s + k] : INT_MAX;
    const int nJ = sort_unique(key, K, sJ, &s_cnt);
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        plan.idx[b * K + k] = (k < nI) ? sI[k] : 0;
        plan.idx2[b * K + k] = (k < nJ) ? sJ[k] : 0;
    }
    for (int l = threadIdx.x; l < B; l += blockDim.x) {
        int pa = 0, pb = 0;
        if (l < nb) {
            pa = lower_bound(sI, nI, ti[s + l]);
            pb = lower_bound(sJ, nJ, tj[s + l]);
        }
        plan.pa[b * B + l] = pa;
        plan.pb[b * B + l] = pb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        plan.nidx[b] = nI;
        plan.nidx2[b] = nJ;
        for (int k = 0; k <= K; k++) cnt[k] = 0;
        for (int l = 0; l < nb; l++) cnt[plan.pa[b * B + l] + 1]++;
        for (int k = 0; k < K; k++) cnt[k + 1] += cnt[k];
        int32_t *lptr = plan.lptr + b * (K + 1);
        for (int k = 0; k <= K; k++) lptr[k] = cnt[k];
        int32_t *lent = plan.lent + b * K;
        for (int l = 0; l < nb; l++) {
            const int pa = plan.pa[b * B + l], pb = plan.pb[b * B + l];
            lent[cnt[pa]++] = (l << 16) | pb;
        }
    }
}

// ---------------------------------------------------------------------------------
// shared pieces of the sweep kernels
// ---------------------------------------------------------------------------------
// Per-coordinate step constants, formed in double in phase A and stored in the cache
// type T (hi + lo pairs where the value carries the result):
//   u = c - base/a, r = lam/a, vp = u - r - c, vm = u + r - c, ai = 1/a, mc = -c.
// With acc = the in-batch correction sum, w = u - acc/a and the step is vp - acc/a
// (w > r), vm - acc/a (w < -r), -c otherwise (zero curvature: always -c).
enum { PRE_UH, PRE_UL, PRE_VPH, PRE_VPL, PRE_VMH, PRE_VML, PRE_AI, PRE_R, PRE_MC, PRE_N };

template <typename T>
__device__ __forceinline__ void split(double v, T *hi, T *lo) {
    *hi = (T)v;
    *lo = (T)(v - (double)*hi);
}

template <typename T>
__device__ void step_constants(double base, double a, double c, double lam, T *pre, int B, int l) {
    T *o = pre;
    if (a > 0.0 && isfinite(a)) {
        const double ai = 1.0 / a;
        const double u = c - base * ai, r = lam * ai;
        split<T>(u, o + PRE_UH * B + l, o + PRE_UL * B + l);
        split<T>(u - r - c, o + PRE_VPH * B + l, o + PRE_VPL * B + l);
        split<T>(u + r - c, o + PRE_VMH * B + l, o + PRE_VML * B + l);
        o[PRE_AI * B + l] = (T)ai;
        o[PRE_R * B + l] = (T)r;
    } else {  // zero curvature: w = 0 inside [-1, 1] selects -c
        o[PRE_UH * B + l] = T(0); o[PRE_UL * B + l] = T(0);
        split<T>(-c, o + PRE_VPH * B + l, o + PRE_VPL * B + l);
        split<T>(-c, o + PRE_VMH * B + l, o + PRE_VML * B + l);
        o[PRE_AI * B + l] = T(0);
        o[PRE_R * B + l] = T(1);
    }
    o[PRE_MC * B + l] = (T)(-c);
}

__device__ __forceinline__ void decode_pair(int e, int &l, int &l1) {
    // e = l (l - 1) / 2 + l1, 0 <= l1 < l
    l = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
    while (l * (l - 1) / 2 > e) l--;
    while ((l + 1) * l / 2 <= e) l++;
    l1 = e - l * (l - 1) / 2;
}

// In-batch coefficients are stored column by column: the entries coef(l2, l) for all
// later l2 > l are contiguous, at colbase(l) + (l2 - l - 1), so that at step l the lanes
// of the warp read consecutive words.
__host__ __device__ __forceinline__ int colbase(int l, int B) { return l * (2 * B - l - 1) / 2; }
// shared-memory slots for the coefficients (16-byte multiple with copy slack)
__host__ __device__ __forceinline__ int coef_slots(int B) { return ((B * (B - 1) / 2 + 8) + 3) & ~3; }

constexpr int kRowsC = 16;  // rows of the band staged per round in phase C

struct SmemLayout {
    size_t meta;  // idx[K], idx2[K], pa[B], pb[B], lptr[K+1], lent[K] (ints)
    size_t work;  // union: phase B coef[B(B-1)/2] (T);
                  //        phase C mu[B], Sigma rows [kRowsC][K], cache rows [kRowsC][K] (T)
    size_t total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int B) {
    const int K = 2 * B;
    SmemLayout s;
    s.meta = 0;
    size_t off = (size_t)(2 * K + 2 * B + (K + 1) + K) * sizeof(int32_t);
    off = (off + 15) & ~size_t(15);
    s.work = off;
    const size_t phb = ((size_t)coef_slots(B) + PRE_N * B + 8) * sizeof(T);
    const size_t phc = (size_t)(B + 4) * sizeof(T) + (size_t)kRowsC * (K + 4) * sizeof(T) * 2;
    s.total = off + (phb > phc ? phb : phc);
    return s;
}

// Forward substitution of one batch on warp 0: for l = 0..nb-1,
//   b_l = base_l + sum_{l' < l} coef(l, l') mu_l',  mu_l = -c_l + S_{lam_l/a_l}(c_l - b_l/a_l)
// (exact minimiser of (a/2) mu^2 + b mu + lam |c + mu|, Appendix A.1), written with the
// step constants above.  coef is the strictly lower triangle, row-major packed, in shared
// memory (column-packed, see colbase).  Lane k owns coordinates 32 s + k; at step l every lane forms the candidate
// step of its own coordinate of the current panel and the owner's candidate is broadcast,
// so the dependent chain per coordinate is a few T operations and one warp shuffle.
template <typename T, int NS>
__device__ void forward_substitution(int nb, int B, const T *__restrict__ pre,
                                     const T *coef, double *mu_out, int *err) {
    // pre[] holds, for padding coordinates l >= nb, constants that give mu = 0 whatever
    // the correction sum (ai = 0, u = 0, r = 1, mc = 0), so panels run all 32 steps
    // without branches.
    const int lane = threadIdx.x & 31;
    T acc[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = T(0);
    bool bad = false;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s * 32 >= nb) break;
        const int lo = s * 32 + lane;
        const T uh = pre[PRE_UH * B + lo], ul = pre[PRE_UL * B + lo];
        const T vph = pre[PRE_VPH * B + lo], vpl = pre[PRE_VPL * B + lo];
        const T vmh = pre[PRE_VMH * B + lo], vml = pre[PRE_VML * B + lo];
        const T ai = pre[PRE_AI * B + lo], r = pre[PRE_R * B + lo], mc = pre[PRE_MC * B + lo];
        // this panel's own coefficients coef(lo, 32 s + o) for o < lane, in registers
        T cw[32];
#pragma unroll
        for (int o = 0; o < 32; o++) {
            const int l = s * 32 + o;
            cw[o] = (lane > o) ? coef[colbase(l, B) + (lo - l - 1)] : T(0);
        }
        T mymu = T(0);
#pragma unroll
        for (int o = 0; o < 32; o++) {
            const int l = s * 32 + o;
            const T w = fma(-acc[s], ai, uh) + ul;
            const T mp = fma(-acc[s], ai, vph) + vpl;
            const T mm = fma(-acc[s], ai, vmh) + vml;
            const T cand = (w > r) ? mp : ((w < -r) ? mm : mc);
            const T mu = __shfl_sync(0xffffffffu, cand, o);
            mymu = (lane == o) ? cand : mymu;
            acc[s] = fma(cw[o], mu, acc[s]);
#pragma unroll
            for (int s2 = s + 1; s2 < NS; s2++) {
                const int l2 = s2 * 32 + lane;
                acc[s2] = fma(coef[colbase(l, B) + (l2 - l - 1)], mu, acc[s2]);
            }
        }
        if (lo < nb) {
            double m = (double)mymu;
            if (!isfinite(m)) { bad = true; m = 0.0; }
            mu_out[lo] = m;
        }
    }
    if (bad) set_err(err, DEV_NONFINITE);
}

// Ticket: returns true in the last CTA to arrive (all CTAs' prior global writes visible).
__device__ __forceinline__ bool last_cta(unsigned *ticket, unsigned nblocks) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == nblocks - 1);
        if (s_last) {
            *ticket = 0;
            __threadfence();
        }
    }
    __syncthreads();
    return s_last != 0;
}

// Three dot products of length len over contiguous rows by the whole CTA:
//   r0 = x0 . y0, r1 = x1 . y0, r2 = x2 . y1   (y rows read through L2); valid in thread 0
template <typename T>
__device__ void cta_dot3(int64_t len, const T *x0, const T *x1, const T *x2, const T *y0,
                         const T *y1, double *r) {
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) {
        const T u0 = __ldcg(y0 + t), u1 = __ldcg(y1 + t);
        a0 = fma(x0[t], u0, a0);
        a1 = fma(x1[t], u0, a1);
        a2 = fma(x2[t], u1, a2);
    }
    r[0] = block_sum((double)a0);
    r[1] = block_sum((double)a1);
    r[2] = block_sum((double)a2);
}

template <typename T>
__device__ double cta_dot1(int64_t len, const T *x0, const T *y0) {
    T a0 = T(0);
    for (int64_t t = threadIdx.x; t < len; t += blockDim.x) a0 = fma(x0[t], __ldcg(y0 + t), a0);
    return block_sum((double)a0);
}

// Load the batch metadata of batch b into shared memory.
__device__ void load_meta(const BatchPlan &plan, int64_t b, int B, bool theta, int32_t *sidx,
                          int32_t *sidx2, int32_t *spa, int32_t *spb, int32_t *slptr,
                          int32_t *slent) {
    const int K = 2 * B;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        sidx[k] = plan.idx[b * K + k];
        if (theta) sidx2[k] = plan.idx2[b * K + k];
        slent[k] = plan.lent[b * K + k];
    }
    for (int k = threadIdx.x; k <= K; k += blockDim.x) slptr[k] = plan.lptr[b * (K + 1) + k];
    for (int l = threadIdx.x; l < B; l += blockDim.x) {
        spa[l] = plan.pa[b * B + l];
        spb[l] = plan.pb[b * B + l];
    }
    __syncthreads();
}

// Copy n elements global -> shared (both 16-byte aligned, n rounded up to 16 bytes; the
// buffers have that slack) with 16-byte loads, eight in flight per thread.
template <typename T>
__device__ void copy_to_smem(const T *g, T *sm, int n) {
    const int nv = (int)((n * sizeof(T) + 15) / 16);
    const int4 *gv = reinterpret_cast<const int4 *>(g);
    int4 *sv = reinterpret_cast<int4 *>(sm);
    for (int base = threadIdx.x; base < nv; base += 8 * blockDim.x) {
        int4 v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = base + u * blockDim.x;
            if (k < nv) v[u] = __ldcg(gv + k);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = base + u * blockDim.x;
            if (k < nv) sv[k] = v[u];
        }
    }
}

// Phase B body shared by both passes: stage the coefficients and step constants, run
// the substitution.
template <typename T, int NS>
__device__ void phase_b(int nb, int B, const T *gcoef, const T *gpre, T *scoef, T *spre,
                        double *mu, int *err) {
    const int ncoef = colbase(nb - 1, B) + 1;  // through column nb - 2 (all entries used)
    copy_to_smem<T>(gcoef, scoef, ncoef);
    copy_to_smem<T>(gpre, spre, PRE_N * B);
    __syncthreads();
    for (int l = nb + threadIdx.x; l < B; l += blockDim.x) {  // padding: mu = 0
        for (int k = 0; k < PRE_N; k++) spre[k * B + l] = T(0);
        spre[PRE_R * B + l] = T(1);
    }
    const int nc = colbase(nb - 1, B) + 1, ncb = B * (B - 1) / 2;
    for (int e = nc + threadIdx.x; e < ncb; e += blockDim.x) scoef[e] = T(0);
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) forward_substitution<T, NS>(nb, B, spre, scoef, mu, err);
    __syncthreads();
}

// Phase C body shared by both passes.  For every row t of this CTA's band and every
// distinct target index k: cache[t][tgt[k]] += sum over the list of k of
// mu_l Sigma[t][partner[e]].  Rows are processed kRowsC at a time: the Sigma values at
// the partner columns and the cache values at the target columns are first staged in
// shared memory by all threads (independent loads), then combined, then written back.
template <typename T>
__device__ void phase_c(int nb, int ntgt, const int32_t *tgt, const int32_t *part,
                        const int32_t *lptr, const int32_t *lent, const T *__restrict__ Sig,
                        int64_t q, T *cache, int64_t ld, int64_t r0, int64_t r1, T *work,
                        const double *mu) {
    const int nent = lptr[ntgt];
    T *smu = work;
    T *sS = smu + ((nb + 3) & ~3);
    for (int l = threadIdx.x; l < nb; l += blockDim.x) smu[l] = (T)__ldcg(mu + l);
    const int npart = nent;  // one staged Sigma value per entry
    T *sC = sS + (size_t)kRowsC * ((npart + 3) & ~3);
    const int lds = (npart + 3) & ~3, ldc = (ntgt + 3) & ~3;
    for (int64_t t0 = r0; t0 < r1; t0 += kRowsC) {
        const int nr = (int)((r1 - t0) < kRowsC ? (r1 - t0) : kRowsC);
        __syncthreads();
        const int tot_s = nr * npart, tot_c = nr * ntgt;
        for (int base = threadIdx.x; base < tot_s; base += 8 * blockDim.x) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int x = base + u * blockDim.x;
                if (x < tot_s) {
                    const int rr = x / npart, e = x - rr * npart;
                    v[u] = Sig[(t0 + rr) * q + part[lent[e] & 0xffff]];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int x = base + u * blockDim.x;
                if (x < tot_s) {
                    const int rr = x / npart, e = x - rr * npart;
                    sS[(size_t)rr * lds + e] = v[u];
                }
            }
        }
        for (int base = threadIdx.x; base < tot_c; base += 8 * blockDim.x) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int x = base + u * blockDim.x;
                if (x < tot_c) {
                    const int rr = x / ntgt, k = x - rr * ntgt;
                    v[u] = __ldcg(cache + (t0 + rr) * ld + tgt[k]);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int x = base + u * blockDim.x;
                if (x < tot_c) {
                    const int rr = x / ntgt, k = x - rr * ntgt;
                    sC[(size_t)rr * ldc + k] = v[u];
                }
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < tot_c; x += blockDim.x) {
            const int rr = x / ntgt, k = x - rr * ntgt;
            const T *srow = sS + (size_t)rr * lds;
            T acc = T(0);
            for (int e = lptr[k]; e < lptr[k + 1]; e++) acc = fma(smu[lent[e] >> 16], srow[e], acc);
            cache[(t0 + rr) * ld + tgt[k]] = sC[(size_t)rr * ldc + k] + acc;
        }
    }
}

// ---------------------------------------------------------------------------------
// Lambda sweep kernel.  Cache: Ut = U^T (q x q), Ut[r][t] = U[t][r] = (D Sigma)[t][r].
// ---------------------------------------------------------------------------------
template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
lambda_sweep_kernel(int64_t q, const T *__restrict__ Sig, const T *__restrict__ Psi,
                    const double *__restrict__ Sd, const double *__restrict__ Pd,
                    const double *__restrict__ G, const double *__restrict__ Lam, int64_t m,
                    const int32_t *__restrict__ ai, const int32_t *__restrict__ aj,
                    double lam_off, double lam_diag, double *D, T *Ut, int B, BatchPlan plan,
                    SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout<T>(B);
    const int K = 2 * B;
    int32_t *sidx = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *spa = sidx + 2 * K;
    int32_t *spb = spa + B;
    int32_t *slptr = spb + B;
    int32_t *slent = slptr + K + 1;
    unsigned char *work = smem + L.work;
    const unsigned nblk = gridDim.x;
    T *pre = reinterpret_cast<T *>(scr.sub1);   // [PRE_N][B]
    T *gcoef = reinterpret_cast<T *>(scr.sub2); // [B(B-1)/2]
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nblk * blockDim.x;

    for (int64_t b = 0; b < plan.nbatch; b++) {
        const int64_t s = b * B;
        const int nb = (int)((m - s) < B ? (m - s) : B);
        const int nidx = plan.nidx[b];
        load_meta(plan, b, B, false, sidx, nullptr, spa, spb, slptr, slent);

        // ---- phase A: dots and step constants (two coordinates per CTA in one pass) ----
        for (int l = blockIdx.x; l < nb; l += 2 * nblk) {
            const int lb = l + (int)nblk;
            const bool two = lb < nb;
            const int64_t i0 = ai[s + l], j0 = aj[s + l];
            const int64_t i1 = two ? ai[s + lb] : i0, j1 = two ? aj[s + lb] : j0;
            // (Sigma D Sigma)_ij = Sigma_i . U_{:,j}, (Psi D Sigma)_ij = Psi_i . U_{:,j},
            // (Psi D Sigma)_ji = Psi_j . U_{:,i}
            const T *x0 = Sig + i0 * q, *x1 = Psi + i0 * q, *x2 = Psi + j0 * q;
            const T *y0 = Ut + j0 * q, *y1 = Ut + i0 * q;
            const T *z0 = Sig + i1 * q, *z1 = Psi + i1 * q, *z2 = Psi + j1 * q;
            const T *w0 = Ut + j1 * q, *w1 = Ut + i1 * q;
            T a0 = T(0), a1 = T(0), a2 = T(0), b0 = T(0), b1 = T(0), b2 = T(0);
            for (int64_t t = threadIdx.x; t < q; t += blockDim.x) {
                const T u0 = __ldcg(y0 + t), u1 = __ldcg(y1 + t);
                a0 = fma(x0[t], u0, a0);
                a1 = fma(x1[t], u0, a1);
                a2 = fma(x2[t], u1, a2);
                if (two) {
                    const T v0 = __ldcg(w0 + t), v1 = __ldcg(w1 + t);
                    b0 = fma(z0[t], v0, b0);
                    b1 = fma(z1[t], v0, b1);
                    b2 = fma(z2[t], v1, b2);
                }
            }
            double d[6];
            d[0] = block_sum((double)a0);
            d[1] = block_sum((double)a1);
            d[2] = block_sum((double)a2);
            d[3] = block_sum((double)b0);
            d[4] = block_sum((double)b1);
            d[5] = block_sum((double)b2);
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            if (which >= 0) {
                const int lw = which ? lb : l;
                const int64_t i = which ? i1 : i0, j = which ? j1 : j0;
                const double *dd = d + 3 * which;
                double a, bb, lam;
                if (i != j) {
                    const double sij = (double)Sig[i * q + j], pij = (double)Psi[i * q + j];
                    a = sij * sij + Sd[i] * Sd[j] + Sd[i] * Pd[j] + Sd[j] * Pd[i] + 2.0 * sij * pij;
                    bb = G[i * q + j] + dd[0] + dd[1] + dd[2];
                    lam = lam_off;
                } else {
                    a = Sd[i] * Sd[i] + 2.0 * Sd[i] * Pd[i];
                    bb = G[i * q + i] + dd[0] + 2.0 * dd[1];
                    lam = lam_diag;
                }
                step_constants<T>(bb, a, Lam[i * q + j], lam, pre, B, lw);
            }
        }
        {
            // coefficient of the correction of coordinate l = (i, j) by the earlier step of
            // l1 = (a, b):  (Sigma dD Sigma)_ij + (Psi dD Sigma)_ij + (Psi dD Sigma)_ji per unit
            // step, dD = E_ab + E_ba (one term when a == b); doubled middle term on the diagonal
            const int ncoef = nb * (nb - 1) / 2;
            for (int64_t e = gtid; e < ncoef; e += gthreads) {
                int l, l1;
                decode_pair((int)e, l, l1);
                const int64_t pi = sidx[spa[l]], pj = sidx[spb[l]];
                const int64_t pa = sidx[spa[l1]], pb = sidx[spb[l1]];
                auto S = [&](int64_t x, int64_t y) -> T { return Sig[x * q + y]; };
                auto P = [&](int64_t x, int64_t y) -> T { return Psi[x * q + y]; };
                T c1, c2, c3;
                if (pa != pb) {
                    c1 = S(pi, pa) * S(pb, pj) + S(pi, pb) * S(pa, pj);
                    c2 = P(pi, pa) * S(pb, pj) + P(pi, pb) * S(pa, pj);
                    c3 = P(pj, pa) * S(pb, pi) + P(pj, pb) * S(pa, pi);
                } else {
                    c1 = S(pi, pa) * S(pa, pj);
                    c2 = P(pi, pa) * S(pa, pj);
                    c3 = P(pj, pa) * S(pa, pi);
                }
                gcoef[colbase(l1, B) + (l - l1 - 1)] = (pi != pj) ? (c1 + c2 + c3) : (c1 + T(2) * c2);
            }
        }

        // ---- phase B: last CTA runs the coordinate steps in order ----
        if (last_cta(scr.ticket, nblk)) {
            phase_b<T, NS>(nb, B, gcoef, pre, reinterpret_cast<T *>(work),
                           reinterpret_cast<T *>(work) + coef_slots(B), scr.mu, scr.err);
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ai[s + l], j = aj[s + l];
                const double mu = scr.mu[l];
                D[i * q + j] = mu;
                if (i != j) D[j * q + i] = mu;
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: Ut[t][u] += sum mu Sigma[t][partner] over this CTA's rows t ----
        phase_c<T>(nb, nidx, sidx, sidx, slptr, slent, Sig, q, Ut, q, r0, r1,
                   reinterpret_cast<T *>(work), scr.mu);
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
    }
}

// ---------------------------------------------------------------------------------
// Theta sweep kernel.  Cache: dVt = (Delta V)^T (q x p), dVt[j][t] = (Delta Theta Sigma)[t][j].
// ---------------------------------------------------------------------------------
template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
theta_sweep_kernel(int64_t p, int64_t q, const T *__restrict__ Sxx, const double *__restrict__ Xd,
                   const T *__restrict__ Sig, const double *__restrict__ Sd,
                   const double *__restrict__ W, double *Theta, int64_t m,
                   const int32_t *__restrict__ ti, const int32_t *__restrict__ tj, double lam,
                   T *dVt, int B, BatchPlan plan, SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout<T>(B);
    const int K = 2 * B;
    int32_t *sI = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *sJ = sI + K;
    int32_t *spa = sJ + K;
    int32_t *spb = spa + B;
    int32_t *slptr = spb + B;
    int32_t *slent = slptr + K + 1;
    unsigned char *work = smem + L.work;
    const unsigned nblk = gridDim.x;
    T *pre = reinterpret_cast<T *>(scr.sub1);
    T *gcoef = reinterpret_cast<T *>(scr.sub2);
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nblk * blockDim.x;

    for (int64_t b = 0; b < plan.nbatch; b++) {
        const int64_t s = b * B;
        const int nb = (int)((m - s) < B ? (m - s) : B);
        const int nI = plan.nidx[b];
        load_meta(plan, b, B, true, sI, sJ, spa, spb, slptr, slent);
        // rows of Delta V that can be nonzero: those at or before the batch's first row
        const int64_t tmax = (int64_t)ti[s] + 1;

        // ---- phase A (two coordinates per CTA in one pass) ----
        for (int l = blockIdx.x; l < nb; l += 2 * nblk) {
            const int lb = l + (int)nblk;
            const bool two = lb < nb;
            const int64_t i0 = ti[s + l], j0 = tj[s + l];
            const int64_t i1 = two ? ti[s + lb] : i0, j1 = two ? tj[s + lb] : j0;
            // (S_xx Delta V)_ij = (S_xx)_i . Delta V_{:,j}
            const T *x0 = Sxx + i0 * p, *y0 = dVt + j0 * p, *x1 = Sxx + i1 * p, *y1 = dVt + j1 * p;
            T a0 = T(0), a1 = T(0);
            for (int64_t t = threadIdx.x; t < tmax; t += blockDim.x) {
                a0 = fma(x0[t], __ldcg(y0 + t), a0);
                if (two) a1 = fma(x1[t], __ldcg(y1 + t), a1);
            }
            const double d0 = block_sum((double)a0);
            const double d1 = block_sum((double)a1);
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            if (which >= 0) {
                const int lw = which ? lb : l;
                const int64_t i = which ? i1 : i0, j = which ? j1 : j0;
                const double xii = Xd[i];
                const double a = (xii != 0.0) ? 2.0 * Sd[j] * xii : 0.0;
                step_constants<T>(2.0 * W[i * q + j] + 2.0 * (which ? d1 : d0), a,
                                  __ldcg(Theta + i * q + j), lam, pre, B, lw);
            }
        }
        {
            // 2 (S_xx)_{i a} Sigma_{b j}: coordinate l = (i, j), earlier l1 = (a, b)
            const int ncoef = nb * (nb - 1) / 2;
            for (int64_t e = gtid; e < ncoef; e += gthreads) {
                int l, l1;
                decode_pair((int)e, l, l1);
                const int64_t i = sI[spa[l]], j = sJ[spb[l]];
                const int64_t a = sI[spa[l1]], bq = sJ[spb[l1]];
                gcoef[colbase(l1, B) + (l - l1 - 1)] = T(2) * Sxx[i * p + a] * Sig[bq * q + j];
            }
        }

        // ---- phase B ----
        if (last_cta(scr.ticket, nblk)) {
            phase_b<T, NS>(nb, B, gcoef, pre, reinterpret_cast<T *>(work),
                           reinterpret_cast<T *>(work) + coef_slots(B), scr.mu, scr.err);
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ti[s + l], j = tj[s + l];
                Theta[i * q + j] = __ldcg(Theta + i * q + j) + scr.mu[l];
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: dVt[t][i] += sum mu Sigma[t][j] over this CTA's rows t ----
        phase_c<T>(nb, nI, sI, sJ, slptr, slent, Sig, q, dVt, p, r0, r1,
                   reinterpret_cast<T *>(work), scr.mu);
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
    }
}

template <typename T>
cggm_status launch_coop(const void *fn, void **args, size_t smem, cudaStream_t st) {
    CGGM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const int grid = sweep_grid();
    note_launch();
    CGGM_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, smem, st));
    return CGGM_OK;
}

cggm_status read_err(int *err, cudaStream_t st) {
    int h = 0;
    CGGM_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CGGM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h == DEV_TIMEOUT) return CGGM_ETIMEDOUT;
    if (h == DEV_NONFINITE) return CGGM_ENONFINITE;
    if (h != 0) return CGGM_ECUDA;
    return CGGM_OK;
}
}  // namespace

int sweep_grid() { return sm_count(); }

cggm_status plan_reserve(BatchPlan &plan, int B, int64_t nbatch, bool theta) {
    const int K = 2 * B;
    const bool grow = !plan.idx || plan.B != B || nbatch > plan.cap ||
                      (theta && !plan.idx2);
    if (grow) {
        plan_free(plan);
        const int64_t nb = nbatch < 1 ? 1 : nbatch;
        CGGM_CUDA_TRY(cudaMalloc(&plan.nidx, sizeof(int32_t) * nb));
        CGGM_CUDA_TRY(cudaMalloc(&plan.nidx2, sizeof(int32_t) * nb));
        CGGM_CUDA_TRY(cudaMalloc(&plan.idx, sizeof(int32_t) * nb * K));
        CGGM_CUDA_TRY(cudaMalloc(&plan.idx2, sizeof(int32_t) * nb * K));
        CGGM_CUDA_TRY(cudaMalloc(&plan.pa, sizeof(int32_t) * nb * B));
        CGGM_CUDA_TRY(cudaMalloc(&plan.pb, sizeof(int32_t) * nb * B));
        CGGM_CUDA_TRY(cudaMalloc(&plan.lptr, sizeof(int32_t) * nb * (K + 1)));
        CGGM_CUDA_TRY(cudaMalloc(&plan.lent, sizeof(int32_t) * nb * K));
        plan.B = B;
        plan.K = K;
        plan.nbatch = nb;
        plan.cap = nb;
    }
    return CGGM_OK;
}

void plan_free(BatchPlan &plan) {
    cudaFree(plan.nidx); cudaFree(plan.nidx2); cudaFree(plan.idx); cudaFree(plan.idx2);
    cudaFree(plan.pa); cudaFree(plan.pb); cudaFree(plan.lptr); cudaFree(plan.lent);
    plan = BatchPlan();
}

cggm_status scratch_reserve(SweepScratch &scr, int B, int grid) {
    if (scr.partial) return CGGM_OK;
    const int Bmax = 256, K = 2 * Bmax;
    (void)B;
    CGGM_CUDA_TRY(cudaMalloc(&scr.partial, sizeof(double) * (size_t)grid * Bmax * 3));
    CGGM_CUDA_TRY(cudaMalloc(&scr.mu, sizeof(double) * Bmax));
    CGGM_CUDA_TRY(cudaMalloc(&scr.sub1, sizeof(double) * (size_t)K * K));
    CGGM_CUDA_TRY(cudaMalloc(&scr.sub2, sizeof(double) * (size_t)K * K));
    CGGM_CUDA_TRY(cudaMalloc(&scr.bar, sizeof(GridBarrier)));
    CGGM_CUDA_TRY(cudaMalloc(&scr.ticket, sizeof(unsigned)));
    CGGM_CUDA_TRY(cudaMalloc(&scr.err, sizeof(int)));
    CGGM_CUDA_TRY(cudaMemset(scr.bar, 0, sizeof(GridBarrier)));
    CGGM_CUDA_TRY(cudaMemset(scr.ticket, 0, sizeof(unsigned)));
    CGGM_CUDA_TRY(cudaMemset(scr.err, 0, sizeof(int)));
    return CGGM_OK;
}

void scratch_free(SweepScratch &scr) {
    cudaFree(scr.partial); cudaFree(scr.mu); cudaFree(scr.sub1); cudaFree(scr.sub2);
    cudaFree(scr.bar); cudaFree(scr.ticket); cudaFree(scr.err);
    scr = SweepScratch();
}

template <typename T>
cggm_status lambda_sweep(int64_t q, const T *Sigma, const T *Psi, const double *Sd,
                         const double *Pd, const double *G, const double *Lambda, int64_t m,
                         const int32_t *ai, const int32_t *aj, double lam_off, double lam_diag,
                         double *D, T *U, int B, BatchPlan &plan, SweepScratch &scr,
                         cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > (sizeof(T) == 4 ? 256 : 128) || (B & (B - 1))) return CGGM_EINVAL;
    const int64_t nbatch = (m + B - 1) / B;
    CGGM_TRY(plan_reserve(plan, B, nbatch, false));
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    plan.nbatch = nbatch;
    const int K = 2 * B;
    note_launch();
    lambda_plan_kernel<<<(unsigned)nbatch, 256, (size_t)(3 * K + 1) * sizeof(int), st>>>(
        m, ai, aj, B, plan);
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<T>(B).total;
    void *args[] = {(void *)&q, (void *)&Sigma, (void *)&Psi, (void *)&Sd, (void *)&Pd,
                    (void *)&G, (void *)&Lambda, (void *)&m, (void *)&ai, (void *)&aj,
                    (void *)&lam_off, (void *)&lam_diag, (void *)&D, (void *)&U, (void *)&B,
                    (void *)&plan, (void *)&scr};
    const void *fn;
    switch (B) {
        case 32: fn = (const void *)lambda_sweep_kernel<T, 1>; break;
        case 64: fn = (const void *)lambda_sweep_kernel<T, 2>; break;
        case 128: fn = (const void *)lambda_sweep_kernel<T, 4>; break;
        case 256: fn = (const void *)lambda_sweep_kernel<T, 8>; break;
        default: return CGGM_EINVAL;
    }
    CGGM_TRY(launch_coop<T>(fn, args, smem, st));
    return read_err(scr.err, st);
}

// Same pass as lambda_sweep on plan and scratch buffers that the caller has already laid
// out (pointers set, capacity for ceil(m / B) batches); allocates nothing.
cggm_status lambda_sweep_preplanned_f64(int64_t q, const double *Sigma, const double *Psi,
                                        const double *Sd, const double *Pd, const double *G,
                                        const double *Lambda, int64_t m, const int32_t *ai,
                                        const int32_t *aj, double lam_off, double lam_diag,
                                        double *D, double *U, int B, BatchPlan plan,
                                        SweepScratch scr, cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B != 32 && B != 64 && B != 128) return CGGM_EINVAL;
    const int64_t nbatch = (m + B - 1) / B;
    if (nbatch > plan.cap) return CGGM_EINVAL;
    plan.B = B;
    plan.K = 2 * B;
    plan.nbatch = nbatch;
    const int K = 2 * B;
    note_launch();
    lambda_plan_kernel<<<(unsigned)nbatch, 256, (size_t)(3 * K + 1) * sizeof(int), st>>>(
        m, ai, aj, B, plan);
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<double>(B).total;
    void *args[] = {(void *)&q, (void *)&Sigma, (void *)&Psi, (void *)&Sd, (void *)&Pd,
                    (void *)&G, (void *)&Lambda, (void *)&m, (void *)&ai, (void *)&aj,
                    (void *)&lam_off, (void *)&lam_diag, (void *)&D, (void *)&U, (void *)&B,
                    (void *)&plan, (void *)&scr};
    const void *fn = B == 32 ? (const void *)lambda_sweep_kernel<double, 1>
                   : B == 64 ? (const void *)lambda_sweep_kernel<double, 2>
                             : (const void *)lambda_sweep_kernel<double, 4>;
    CGGM_TRY(launch_coop<double>(fn, args, smem, st));
    return read_err(scr.err, st);
}

template <typename T>
cggm_status theta_sweep(int64_t p, int64_t q, const T *Sxx, const double *Xd, const T *Sigma,
                        const double *Sd, const double *W, double *Theta, int64_t m,
                        const int32_t *ti, const int32_t *tj, double lam, T *dV, int B,
                        BatchPlan &plan, SweepScratch &scr, cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > (sizeof(T) == 4 ? 256 : 128) || (B & (B - 1))) return CGGM_EINVAL;
    const int64_t nbatch = (m + B - 1) / B;
    CGGM_TRY(plan_reserve(plan, B, nbatch, true));
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    plan.nbatch = nbatch;
    const int K = 2 * B;
    note_launch();
    theta_plan_kernel<<<(unsigned)nbatch, 256, (size_t)(4 * K + 1) * sizeof(int), st>>>(
        m, ti, tj, B, plan);
    CGGM_CUDA_TRY(cudaGetLastError());
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<T>(B).total;
    void *args[] = {(void *)&p, (void *)&q, (void *)&Sxx, (void *)&Xd, (void *)&Sigma,
                    (void *)&Sd, (void *)&W, (void *)&Theta, (void *)&m, (void *)&ti,
                    (void *)&tj, (void *)&lam, (void *)&dV, (void *)&B, (void *)&plan,
                    (void *)&scr};
    const void *fn;
    switch (B) {
        case 32: fn = (const void *)theta_sweep_kernel<T, 1>; break;
        case 64: fn = (const void *)theta_sweep_kernel<T, 2>; break;
        case 128: fn = (const void *)theta_sweep_kernel<T, 4>; break;
        case 256: fn = (const void *)theta_sweep_kernel<T, 8>; break;
        default: return CGGM_EINVAL;
    }
    CGGM_TRY(launch_coop<T>(fn, args, smem, st));
    return read_err(scr.err, st);
}

template cggm_status lambda_sweep<double>(int64_t, const double *, const double *, const double *,
                                          const double *, const double *, const double *, int64_t,
                                          const int32_t *, const int32_t *, double, double, double *,
                                          double *, int, BatchPlan &, SweepScratch &, cudaStream_t);
template cggm_status lambda_sweep<float>(int64_t, const float *, const float *, const double *,
                                         const double *, const double *, const double *, int64_t,
                                         const int32_t *, const int32_t *, double, double, double *,
                                         float *, int, BatchPlan &, SweepScratch &, cudaStream_t);
template cggm_status theta_sweep<double>(int64_t, int64_t, const double *, const double *,
                                         const double *, const double *, const double *, double *,
                                         int64_t, const int32_t *, const int32_t *, double, double *,
                                         int, BatchPlan &, SweepScratch &, cudaStream_t);
template cggm_status theta_sweep<float>(int64_t, int64_t, const float *, const double *,
                                        const float *, const double *, const double *, double *,
                                        int64_t, const int32_t *, const int32_t *, double, float *,
                                        int, BatchPlan &, SweepScratch &, cudaStream_t);

}  // namespace cggm
