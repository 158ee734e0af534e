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
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

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
struct SmemLayout {
    // per-warp staging of gathered row segments: kWarps * 3 * K values of T
    // reduction buffer: kWarps * B * 3 doubles
    // batch metadata: idx[K], idx2[K], pa[B], pb[B]
    // phase B: base[B], ainv[B], c[B], lam[B], coef[B*(B-1)/2] doubles
    size_t stage, red, meta, phb;
    size_t total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int B) {
    const int K = 2 * B;
    SmemLayout s;
    s.stage = 0;
    size_t off = (size_t)kWarps * 3 * K * sizeof(T);
    off = (off + 15) & ~size_t(15);
    s.red = off;
    off += (size_t)kWarps * B * 3 * sizeof(double);
    s.meta = off;
    off += (size_t)(2 * K + 2 * B) * sizeof(int32_t);
    off = (off + 15) & ~size_t(15);
    s.phb = off;
    off += (size_t)(4 * B + (size_t)B * (B - 1) / 2) * sizeof(double);
    s.total = off;
    return s;
}

// Forward substitution of one batch on warp 0.  For l = 0..nb-1:
//   b_l = base_l + sum_{l' < l} coef(l, l') mu_l',  mu_l = -c_l + S_{lam_l/a_l}(c_l - b_l/a_l)
// (exact minimiser of (a/2) mu^2 + b mu + lam |c + mu|, Appendix A.1).  ainv_l = 0 marks a
// coordinate whose curvature is zero (its minimiser is mu = -c).  coef is the strictly
// lower triangle, row-major packed: coef(l, l') at l (l - 1) / 2 + l'.
template <int NS>
__device__ void forward_substitution(int nb, const double *base, const double *ainv,
                                     const double *cc, const double *lam, const double *coef,
                                     double *mu_out, int *err) {
    const int lane = threadIdx.x & 31;
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = 0.0;
    for (int l = 0; l < nb; l++) {
        const int owner = l & 31, slot = l >> 5;
        double mu = 0.0;
        if (lane == owner) {
            double mine = 0.0;
#pragma unroll
            for (int s = 0; s < NS; s++)
                if (s == slot) mine = acc[s];
            const double c = cc[l], ai = ainv[l];
            if (ai == 0.0) {
                mu = -c;
            } else {
                const double b = base[l] + mine;
                mu = -c + soft_threshold(c - b * ai, lam[l] * ai);
            }
            if (!isfinite(mu)) {
                set_err(err, DEV_NONFINITE);
                mu = 0.0;
            }
            mu_out[l] = mu;
        }
        mu = __shfl_sync(0xffffffffu, mu, owner);
        if (mu != 0.0) {
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const int l2 = s * 32 + lane;
                if (l2 > l && l2 < nb) acc[s] = fma(coef[(size_t)l2 * (l2 - 1) / 2 + l], mu, acc[s]);
            }
        }
    }
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

template <typename T>
__device__ __forceinline__ double ldg_cg(const T *p) {
    return (double)__ldcg(p);
}

// ---------------------------------------------------------------------------------
// Lambda sweep kernel
// ---------------------------------------------------------------------------------
template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
lambda_sweep_kernel(int64_t q, const T *__restrict__ Sig, const T *__restrict__ Psi,
                    const double *__restrict__ Sd, const double *__restrict__ Pd,
                    const double *__restrict__ G, const double *__restrict__ Lam, int64_t m,
                    const int32_t *__restrict__ ai, const int32_t *__restrict__ aj,
                    double lam_off, double lam_diag, double *D, T *U, int B, BatchPlan plan,
                    SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout<T>(B);
    const int K = 2 * B;
    T *stage = reinterpret_cast<T *>(smem + L.stage);
    double *red = reinterpret_cast<double *>(smem + L.red);
    int32_t *sidx = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *spa = sidx + 2 * K;
    int32_t *spb = spa + B;
    double *sbase = reinterpret_cast<double *>(smem + L.phb);
    double *sainv = sbase + B, *sc = sainv + B, *slam = sc + B, *scoef = slam + B;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nblk = gridDim.x;
    T *sub1 = reinterpret_cast<T *>(scr.sub1);  // Sigma[I, I]
    T *sub2 = reinterpret_cast<T *>(scr.sub2);  // Psi[I, I]

    // rows of U / Sigma / Psi owned by this CTA in phase A
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;

    for (int64_t b = 0; b < plan.nbatch; b++) {
        const int64_t s = b * B;
        const int nb = (int)((m - s) < B ? (m - s) : B);
        const int nidx = plan.nidx[b];
        for (int k = threadIdx.x; k < K; k += blockDim.x) sidx[k] = plan.idx[b * K + k];
        for (int l = threadIdx.x; l < B; l += blockDim.x) {
            spa[l] = plan.pa[b * B + l];
            spb[l] = plan.pb[b * B + l];
        }
        __syncthreads();

        // ---------------- phase A: partial dots over this CTA's rows ----------------
        double p1[NS], p2[NS], p3[NS];
#pragma unroll
        for (int s2 = 0; s2 < NS; s2++) p1[s2] = p2[s2] = p3[s2] = 0.0;
        T *sU = stage + (size_t)warp * 3 * K;
        T *sP = sU + K;
        T *sS = sP + K;
        for (int64_t t = r0 + warp; t < r1; t += kWarps) {
            const T *Ur = U + t * q, *Pr = Psi + t * q, *Sr = Sig + t * q;
            for (int k = lane; k < nidx; k += 32) {
                const int64_t c = sidx[k];
                sU[k] = __ldcg(Ur + c);
                sP[k] = Pr[c];
                sS[k] = Sr[c];
            }
            __syncwarp();
#pragma unroll
            for (int s2 = 0; s2 < NS; s2++) {
                const int l = s2 * 32 + lane;
                if (l < nb) {
                    const int pa = spa[l], pb = spb[l];
                    const double ub = (double)sU[pb];
                    p1[s2] = fma((double)sS[pa], ub, p1[s2]);  // Sigma_{t a} U_{t b}
                    p2[s2] = fma((double)sP[pa], ub, p2[s2]);  // Psi_{t a} U_{t b}
                    p3[s2] = fma((double)sP[pb], (double)sU[pa], p3[s2]);  // Psi_{t b} U_{t a}
                }
            }
            __syncwarp();
        }
        // gathered submatrices Sigma[I, I], Psi[I, I] (rows split over CTAs)
        for (int k = blockIdx.x; k < nidx; k += nblk) {
            const int64_t r = sidx[k];
            for (int k2 = threadIdx.x; k2 < nidx; k2 += blockDim.x) {
                sub1[(size_t)k * K + k2] = Sig[r * q + sidx[k2]];
                sub2[(size_t)k * K + k2] = Psi[r * q + sidx[k2]];
            }
        }
        // CTA reduction of the per-warp partials (fixed order)
#pragma unroll
        for (int s2 = 0; s2 < NS; s2++) {
            const int l = s2 * 32 + lane;
            if (l < B) {
                red[((size_t)warp * B + l) * 3 + 0] = p1[s2];
                red[((size_t)warp * B + l) * 3 + 1] = p2[s2];
                red[((size_t)warp * B + l) * 3 + 2] = p3[s2];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nb * 3; e += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < kWarps; w++) acc += red[(size_t)w * B * 3 + e];
            scr.partial[(size_t)blockIdx.x * B * 3 + e] = acc;
        }

        // ---------------- phase B: last CTA ----------------
        if (last_cta(scr.ticket, nblk)) {
            for (int e = threadIdx.x; e < nb * 3; e += blockDim.x) {
                double acc = 0.0;
                for (unsigned c = 0; c < nblk; c++) acc += __ldcg(scr.partial + (size_t)c * B * 3 + e);
                red[e] = acc;  // reuse: red[l*3 + k]
            }
            __syncthreads();
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ai[s + l], j = aj[s + l];
                const double s1 = red[l * 3 + 0], s2v = red[l * 3 + 1], s3 = red[l * 3 + 2];
                double a, bb;
                if (i != j) {
                    const double sij = ldg_cg(Sig + i * q + j), pij = ldg_cg(Psi + i * q + j);
                    a = sij * sij + Sd[i] * Sd[j] + Sd[i] * Pd[j] + Sd[j] * Pd[i] + 2.0 * sij * pij;
                    bb = G[i * q + j] + s1 + s2v + s3;
                    slam[l] = lam_off;
                } else {
                    a = Sd[i] * Sd[i] + 2.0 * Sd[i] * Pd[i];
                    bb = G[i * q + i] + s1 + 2.0 * s2v;
                    slam[l] = lam_diag;
                }
                sbase[l] = bb;
                sainv[l] = (a > 0.0) ? 1.0 / a : 0.0;
                sc[l] = Lam[i * q + j];
            }
            // coefficients of the in-batch corrections (packed strict lower triangle)
            const size_t ncoef = (size_t)nb * (nb - 1) / 2;
            for (size_t e = threadIdx.x; e < ncoef; e += blockDim.x) {
                // invert e = l (l - 1) / 2 + l'
                int l = (int)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
                while ((size_t)l * (l - 1) / 2 > e) l--;
                while ((size_t)(l + 1) * l / 2 <= e) l++;
                const int l1 = (int)(e - (size_t)l * (l - 1) / 2);
                const int pi = spa[l], pj = spb[l];   // coordinate l = (i, j)
                const int pa = spa[l1], pb = spb[l1]; // earlier coordinate l1 = (a, b)
                auto S = [&](int x, int y) { return ldg_cg(sub1 + (size_t)x * K + y); };
                auto P = [&](int x, int y) { return ldg_cg(sub2 + (size_t)x * K + y); };
                double c1, c2, c3;
                if (pa != pb) {
                    c1 = S(pi, pa) * S(pb, pj) + S(pi, pb) * S(pa, pj);
                    c2 = P(pi, pa) * S(pb, pj) + P(pi, pb) * S(pa, pj);
                    c3 = P(pj, pa) * S(pb, pi) + P(pj, pb) * S(pa, pi);
                } else {
                    c1 = S(pi, pa) * S(pa, pj);
                    c2 = P(pi, pa) * S(pa, pj);
                    c3 = P(pj, pa) * S(pa, pi);
                }
                scoef[e] = (pi != pj) ? (c1 + c2 + c3) : (c1 + 2.0 * c2);
            }
            __syncthreads();
            if (warp == 0)
                forward_substitution<NS>(nb, sbase, sainv, sc, slam, scoef, scr.mu, scr.err);
            __syncthreads();
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ai[s + l], j = aj[s + l];
                const double mu = scr.mu[l];
                D[i * q + j] = mu;
                if (i != j) D[j * q + i] = mu;
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---------------- phase C: U rows += mu Sigma rows ----------------
        {
            const int32_t *lptr = plan.lptr + b * (K + 1);
            const int32_t *lent = plan.lent + b * K;
            const int64_t nchunk = (q + 31) / 32;
            const int64_t items = (int64_t)nidx * nchunk;
            for (int64_t it = (int64_t)blockIdx.x * kWarps + warp; it < items;
                 it += (int64_t)nblk * kWarps) {
                const int k = (int)(it / nchunk);
                const int64_t t = (it % nchunk) * 32 + lane;
                if (t >= q) continue;
                const int64_t u = sidx[k];
                double acc = 0.0;
                for (int e = lptr[k]; e < lptr[k + 1]; e++) {
                    const int ent = lent[e];
                    const int l = ent >> 16, pp = ent & 0xffff;
                    acc = fma(__ldcg(scr.mu + l), (double)Sig[(int64_t)sidx[pp] * q + t], acc);
                }
                U[u * q + t] = (T)((double)__ldcg(U + u * q + t) + acc);
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
    }
}

// ---------------------------------------------------------------------------------
// Theta sweep kernel
// ---------------------------------------------------------------------------------
template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
theta_sweep_kernel(int64_t p, int64_t q, const T *__restrict__ Sxx, const double *__restrict__ Xd,
                   const T *__restrict__ Sig, const double *__restrict__ Sd,
                   const double *__restrict__ W, double *Theta, int64_t m,
                   const int32_t *__restrict__ ti, const int32_t *__restrict__ tj, double lam,
                   T *dV, int B, BatchPlan plan, SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout L = smem_layout<T>(B);
    const int K = 2 * B;
    T *stage = reinterpret_cast<T *>(smem + L.stage);
    double *red = reinterpret_cast<double *>(smem + L.red);
    int32_t *sI = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *sJ = sI + K;
    int32_t *spa = sJ + K;
    int32_t *spb = spa + B;
    double *sbase = reinterpret_cast<double *>(smem + L.phb);
    double *sainv = sbase + B, *sc = sainv + B, *slam = sc + B, *scoef = slam + B;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned nblk = gridDim.x;
    T *sub1 = reinterpret_cast<T *>(scr.sub1);  // Sxx[I, I]
    T *sub2 = reinterpret_cast<T *>(scr.sub2);  // Sigma[J, J]

    for (int64_t b = 0; b < plan.nbatch; b++) {
        const int64_t s = b * B;
        const int nb = (int)((m - s) < B ? (m - s) : B);
        const int nI = plan.nidx[b], nJ = plan.nidx2[b];
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            sI[k] = plan.idx[b * K + k];
            sJ[k] = plan.idx2[b * K + k];
        }
        for (int l = threadIdx.x; l < B; l += blockDim.x) {
            spa[l] = plan.pa[b * B + l];
            spb[l] = plan.pb[b * B + l];
        }
        __syncthreads();
        // rows of dV that can be nonzero: those at or before the batch's first row
        const int64_t tmax = (int64_t)ti[s] + 1;
        const int64_t rows_per = (tmax + nblk - 1) / nblk;
        const int64_t r0 = (int64_t)blockIdx.x * rows_per;
        const int64_t r1 = (r0 + rows_per) < tmax ? (r0 + rows_per) : tmax;

        // ---------------- phase A ----------------
        double p1[NS];
#pragma unroll
        for (int s2 = 0; s2 < NS; s2++) p1[s2] = 0.0;
        T *sV = stage + (size_t)warp * 3 * K;
        T *sX = sV + K;
        for (int64_t t = r0 + warp; t < r1; t += kWarps) {
            const T *Vr = dV + t * q, *Xr = Sxx + t * p;
            for (int k = lane; k < nJ; k += 32) sV[k] = __ldcg(Vr + sJ[k]);
            for (int k = lane; k < nI; k += 32) sX[k] = Xr[sI[k]];
            __syncwarp();
#pragma unroll
            for (int s2 = 0; s2 < NS; s2++) {
                const int l = s2 * 32 + lane;
                if (l < nb) p1[s2] = fma((double)sX[spa[l]], (double)sV[spb[l]], p1[s2]);
            }
            __syncwarp();
        }
        for (int k = blockIdx.x; k < nI; k += nblk) {
            const int64_t r = sI[k];
            for (int k2 = threadIdx.x; k2 < nI; k2 += blockDim.x)
                sub1[(size_t)k * K + k2] = Sxx[r * p + sI[k2]];
        }
        for (int k = blockIdx.x; k < nJ; k += nblk) {
            const int64_t r = sJ[k];
            for (int k2 = threadIdx.x; k2 < nJ; k2 += blockDim.x)
                sub2[(size_t)k * K + k2] = Sig[r * q + sJ[k2]];
        }
#pragma unroll
        for (int s2 = 0; s2 < NS; s2++) {
            const int l = s2 * 32 + lane;
            if (l < B) red[(size_t)warp * B + l] = p1[s2];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nb; e += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < kWarps; w++) acc += red[(size_t)w * B + e];
            scr.partial[(size_t)blockIdx.x * B + e] = acc;
        }

        // ---------------- phase B ----------------
        if (last_cta(scr.ticket, nblk)) {
            for (int e = threadIdx.x; e < nb; e += blockDim.x) {
                double acc = 0.0;
                for (unsigned c = 0; c < nblk; c++) acc += __ldcg(scr.partial + (size_t)c * B + e);
                red[e] = acc;
            }
            __syncthreads();
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ti[s + l], j = tj[s + l];
                const double xii = Xd[i];
                const double a = 2.0 * Sd[j] * xii;
                sbase[l] = 2.0 * W[i * q + j] + 2.0 * red[l];
                sainv[l] = (xii != 0.0 && a > 0.0) ? 1.0 / a : 0.0;
                sc[l] = __ldcg(Theta + i * q + j);
                slam[l] = lam;
            }
            const size_t ncoef = (size_t)nb * (nb - 1) / 2;
            for (size_t e = threadIdx.x; e < ncoef; e += blockDim.x) {
                int l = (int)((1.0 + sqrt(1.0 + 8.0 * (double)e)) * 0.5);
                while ((size_t)l * (l - 1) / 2 > e) l--;
                while ((size_t)(l + 1) * l / 2 <= e) l++;
                const int l1 = (int)(e - (size_t)l * (l - 1) / 2);
                // 2 (S_xx)_{i a} Sigma_{b j}: coordinate l = (i, j), earlier l1 = (a, b)
                scoef[e] = 2.0 * ldg_cg(sub1 + (size_t)spa[l] * K + spa[l1]) *
                           ldg_cg(sub2 + (size_t)spb[l1] * K + spb[l]);
            }
            __syncthreads();
            if (warp == 0)
                forward_substitution<NS>(nb, sbase, sainv, sc, slam, scoef, scr.mu, scr.err);
            __syncthreads();
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = ti[s + l], j = tj[s + l];
                Theta[i * q + j] = sc[l] + scr.mu[l];
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---------------- phase C: dV rows += mu Sigma rows ----------------
        {
            const int32_t *lptr = plan.lptr + b * (K + 1);
            const int32_t *lent = plan.lent + b * K;
            const int64_t nchunk = (q + 31) / 32;
            const int64_t items = (int64_t)nI * nchunk;
            for (int64_t it = (int64_t)blockIdx.x * kWarps + warp; it < items;
                 it += (int64_t)nblk * kWarps) {
                const int k = (int)(it / nchunk);
                const int64_t t = (it % nchunk) * 32 + lane;
                if (t >= q) continue;
                const int64_t u = sI[k];
                double acc = 0.0;
                for (int e = lptr[k]; e < lptr[k + 1]; e++) {
                    const int ent = lent[e];
                    const int l = ent >> 16, pp = ent & 0xffff;
                    acc = fma(__ldcg(scr.mu + l), (double)Sig[(int64_t)sJ[pp] * q + t], acc);
                }
                dV[u * q + t] = (T)((double)__ldcg(dV + u * q + t) + acc);
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
    }
}

template <typename T>
cggm_status launch_coop(const void *fn, void **args, size_t smem, cudaStream_t st) {
    CGGM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const int grid = sweep_grid();
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
    const int Bmax = 128, K = 2 * Bmax;
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
    if (B < 32 || B > 128 || (B & (B - 1))) return CGGM_EINVAL;
    const int64_t nbatch = (m + B - 1) / B;
    CGGM_TRY(plan_reserve(plan, B, nbatch, false));
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    plan.nbatch = nbatch;
    const int K = 2 * B;
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
        default: return CGGM_EINVAL;
    }
    CGGM_TRY(launch_coop<T>(fn, args, smem, st));
    return read_err(scr.err, st);
}

template <typename T>
cggm_status theta_sweep(int64_t p, int64_t q, const T *Sxx, const double *Xd, const T *Sigma,
                        const double *Sd, const double *W, double *Theta, int64_t m,
                        const int32_t *ti, const int32_t *tj, double lam, T *dV, int B,
                        BatchPlan &plan, SweepScratch &scr, cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > 128 || (B & (B - 1))) return CGGM_EINVAL;
    const int64_t nbatch = (m + B - 1) / B;
    CGGM_TRY(plan_reserve(plan, B, nbatch, true));
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    plan.nbatch = nbatch;
    const int K = 2 * B;
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
