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
#include <mutex>

namespace cggm {

namespace {
constexpr int kThreads = 256;

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

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


struct SmemLayout {
    size_t meta;  // sa[B], sb[B] (batch coordinates), sseg[B + 1] (segment starts), nseg (ints)
    size_t work;  // union: phase B coef[coef_slots(B)] + step constants [PRE_N][B] (T);
                  //        phase C mu[B] (T)
    size_t total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int B) {
    SmemLayout s;
    s.meta = 0;
    size_t off = (size_t)(2 * B + (B + 1) + 1) * sizeof(int32_t);
    off = (off + 15) & ~size_t(15);
    s.work = off;
    const size_t phb = ((size_t)coef_slots(B) + PRE_N * B + 8) * sizeof(T);
    const size_t phc = (size_t)(B + 4) * sizeof(T);
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

// 16-byte vector of the cache type
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static const int n = 4; };
template <> struct V16<double> { using type = double2; static const int n = 2; };

__device__ __forceinline__ float vget(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2 &v, int k) { return k == 0 ? v.x : v.y; }

// Sum of NV per-thread values over the CTA, in double, in a fixed order; results in r[]
// (valid in every thread).  red: shared scratch of kThreads / 32 * NV doubles.
template <int NV>
__device__ void cta_sums(double *v, double *red, double *r) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) red[warp * NV + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += red[w * NV + k];
        r[k] = s;
    }
    __syncthreads();
}

// Load the coordinates of the batch [s, s + nb) into shared memory and find its segments
// (maximal runs of coordinates with the same first index; the lists are row-major, so a
// segment is the part of one row of the active set that falls in the batch).
__device__ void load_batch(const int32_t *__restrict__ ai, const int32_t *__restrict__ aj,
                           int64_t s, int nb, int32_t *sa, int32_t *sb, int32_t *sseg,
                           int32_t *snseg) {
    for (int l = threadIdx.x; l < nb; l += blockDim.x) {
        sa[l] = ai[s + l];
        sb[l] = aj[s + l];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int base = 0;
        for (int l0 = 0; l0 < nb; l0 += 32) {
            const int l = l0 + lane;
            const bool f = l < nb && (l == 0 || sa[l] != sa[l - 1]);
            const unsigned m = __ballot_sync(0xffffffffu, f);
            if (f) sseg[base + __popc(m & ((1u << lane) - 1u))] = l;
            base += __popc(m);
        }
        if (lane == 0) {
            sseg[base] = nb;
            *snseg = base;
        }
    }
    __syncthreads();
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
                    double lam_off, double lam_diag, double *D, T *Ut, int B,
                    SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[(kThreads / 32) * 6];
    const SmemLayout L = smem_layout<T>(B);
    int32_t *sa = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *sb = sa + B;
    int32_t *sseg = sb + B;
    int32_t *snseg = sseg + B + 1;
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x;
    T *pre = reinterpret_cast<T *>(scr.sub1);    // [PRE_N][B]
    T *gcoef = reinterpret_cast<T *>(scr.sub2);  // column-packed coefficients
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nblk * blockDim.x;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    const bool vec = (q % VN) == 0;

    for (int64_t s = 0; s < m; s += B) {
        const int nb = (int)((m - s) < B ? (m - s) : B);
        load_batch(ai, aj, s, nb, sa, sb, sseg, snseg);

        // ---- phase A: dot products and step constants, two coordinates per CTA ----
        for (int l = blockIdx.x; l < nb; l += 2 * nblk) {
            const int lb = l + (int)nblk;
            const bool two = lb < nb;
            const int64_t i0 = sa[l], j0 = sb[l];
            const int64_t i1 = two ? sa[lb] : i0, j1 = two ? sb[lb] : j0;
            // (Sigma D Sigma)_ij = Sigma_i . U_{:,j}, (Psi D Sigma)_ij = Psi_i . U_{:,j},
            // (Psi D Sigma)_ji = Psi_j . U_{:,i}
            const T *x0 = Sig + i0 * q, *x1 = Psi + i0 * q, *x2 = Psi + j0 * q;
            const T *y0 = Ut + j0 * q, *y1 = Ut + i0 * q;
            const T *z0 = Sig + i1 * q, *z1 = Psi + i1 * q, *z2 = Psi + j1 * q;
            const T *w0 = Ut + j1 * q, *w1 = Ut + i1 * q;
            T a0 = T(0), a1 = T(0), a2 = T(0), b0 = T(0), b1 = T(0), b2 = T(0);
            if (vec) {
                const int64_t nv = q / VN;
#pragma unroll 4
                for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
                    const VT X0 = reinterpret_cast<const VT *>(x0)[v];
                    const VT X1 = reinterpret_cast<const VT *>(x1)[v];
                    const VT X2 = reinterpret_cast<const VT *>(x2)[v];
                    const VT Y0 = __ldcg(reinterpret_cast<const VT *>(y0) + v);
                    const VT Y1 = __ldcg(reinterpret_cast<const VT *>(y1) + v);
#pragma unroll
                    for (int k = 0; k < VN; k++) {
                        a0 = fma(vget(X0, k), vget(Y0, k), a0);
                        a1 = fma(vget(X1, k), vget(Y0, k), a1);
                        a2 = fma(vget(X2, k), vget(Y1, k), a2);
                    }
                    if (two) {
                        const VT Z0 = reinterpret_cast<const VT *>(z0)[v];
                        const VT Z1 = reinterpret_cast<const VT *>(z1)[v];
                        const VT Z2 = reinterpret_cast<const VT *>(z2)[v];
                        const VT W0 = __ldcg(reinterpret_cast<const VT *>(w0) + v);
                        const VT W1 = __ldcg(reinterpret_cast<const VT *>(w1) + v);
#pragma unroll
                        for (int k = 0; k < VN; k++) {
                            b0 = fma(vget(Z0, k), vget(W0, k), b0);
                            b1 = fma(vget(Z1, k), vget(W0, k), b1);
                            b2 = fma(vget(Z2, k), vget(W1, k), b2);
                        }
                    }
                }
            } else {
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
            }
            double v6[6] = {(double)a0, (double)a1, (double)a2, (double)b0, (double)b1, (double)b2};
            double d[6];
            cta_sums<6>(v6, s_red, d);
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            if (which >= 0) {
                const int lw = which ? lb : l;
                const int64_t i = which ? i1 : i0, j = which ? j1 : j0;
                const double d0 = which ? d[3] : d[0], d1 = which ? d[4] : d[1],
                             d2 = which ? d[5] : d[2];
                double a, bb, lam;
                if (i != j) {
                    const double sij = (double)Sig[i * q + j], pij = (double)Psi[i * q + j];
                    a = sij * sij + Sd[i] * Sd[j] + Sd[i] * Pd[j] + Sd[j] * Pd[i] + 2.0 * sij * pij;
                    bb = G[i * q + j] + d0 + d1 + d2;
                    lam = lam_off;
                } else {
                    a = Sd[i] * Sd[i] + 2.0 * Sd[i] * Pd[i];
                    bb = G[i * q + i] + d0 + 2.0 * d1;
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
                const int64_t pi = sa[l], pj = sb[l];
                const int64_t pa = sa[l1], pb = sb[l1];
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
                const int64_t i = sa[l], j = sb[l];
                const double mu = scr.mu[l];
                D[i * q + j] = mu;
                if (i != j) D[j * q + i] = mu;
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: rows t of this CTA's band, segment by segment ----
        // coordinate (a, b) of a segment with row a: U_a += mu Sigma_b, U_b += mu Sigma_a
        // (b != a); transposed: Ut[t][a] += sum mu Sigma[t][b], Ut[t][b] += mu Sigma[t][a]
        {
            T *smu = reinterpret_cast<T *>(work);
            for (int l = threadIdx.x; l < nb; l += blockDim.x) smu[l] = (T)__ldcg(scr.mu + l);
            __syncthreads();
            const int nseg = *snseg;
            for (int64_t t = r0 + warp; t < r1; t += (kThreads / 32)) {
                const T *Sr = Sig + t * q;
                T *Ur = Ut + t * q;
                for (int g = 0; g < nseg; g++) {
                    const int l0 = sseg[g], l1 = sseg[g + 1];
                    const int64_t a = sa[l0];
                    // issue every load of this lane first (up to NS coordinates per lane)
                    T sv[NS], uv[NS], mv[NS];
                    int64_t bv[NS];
                    const T sta = Sr[a];
#pragma unroll
                    for (int k = 0; k < NS; k++) {
                        const int l = l0 + lane + 32 * k;
                        bv[k] = -1;
                        if (l < l1) {
                            bv[k] = sb[l];
                            mv[k] = smu[l];
                            sv[k] = Sr[bv[k]];
                            uv[k] = (bv[k] != a) ? __ldcg(Ur + bv[k]) : T(0);
                        }
                    }
                    T dot = T(0);
#pragma unroll
                    for (int k = 0; k < NS; k++) {
                        if (bv[k] >= 0) {
                            dot = fma(mv[k], sv[k], dot);
                            if (bv[k] != a) Ur[bv[k]] = uv[k] + mv[k] * sta;
                        }
                    }
                    dot = warp_sum(dot);
                    __syncwarp();
                    if (lane == 0) Ur[a] = __ldcg(Ur + a) + dot;
                    __syncwarp();
                }
            }
        }
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
                   T *dVt, int B, SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[(kThreads / 32) * 2];
    const SmemLayout L = smem_layout<T>(B);
    int32_t *sa = reinterpret_cast<int32_t *>(smem + L.meta);
    int32_t *sb = sa + B;
    int32_t *sseg = sb + B;
    int32_t *snseg = sseg + B + 1;
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x;
    T *pre = reinterpret_cast<T *>(scr.sub1);
    T *gcoef = reinterpret_cast<T *>(scr.sub2);
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)nblk * blockDim.x;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;

    for (int64_t s = 0; s < m; s += B) {
        const int nb = (int)((m - s) < B ? (m - s) : B);
        load_batch(ti, tj, s, nb, sa, sb, sseg, snseg);
        // rows of Delta V that can be nonzero: those at or before the batch's first row
        const int64_t tmax = (int64_t)sa[0] + 1;

        // ---- phase A (two coordinates per CTA in one pass) ----
        for (int l = blockIdx.x; l < nb; l += 2 * nblk) {
            const int lb = l + (int)nblk;
            const bool two = lb < nb;
            const int64_t i0 = sa[l], j0 = sb[l];
            const int64_t i1 = two ? sa[lb] : i0, j1 = two ? sb[lb] : j0;
            // (S_xx Delta V)_ij = (S_xx)_i . Delta V_{:,j}
            const T *x0 = Sxx + i0 * p, *y0 = dVt + j0 * p, *x1 = Sxx + i1 * p, *y1 = dVt + j1 * p;
            T a0 = T(0), a1 = T(0);
            int64_t tv = 0;
            if ((p % VN) == 0) {
                const int64_t nv = tmax / VN;
#pragma unroll 4
                for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
                    const VT X0 = reinterpret_cast<const VT *>(x0)[v];
                    const VT Y0 = __ldcg(reinterpret_cast<const VT *>(y0) + v);
#pragma unroll
                    for (int k = 0; k < VN; k++) a0 = fma(vget(X0, k), vget(Y0, k), a0);
                    if (two) {
                        const VT X1 = reinterpret_cast<const VT *>(x1)[v];
                        const VT Y1 = __ldcg(reinterpret_cast<const VT *>(y1) + v);
#pragma unroll
                        for (int k = 0; k < VN; k++) a1 = fma(vget(X1, k), vget(Y1, k), a1);
                    }
                }
                tv = nv * VN;
            }
            for (int64_t t = tv + threadIdx.x; t < tmax; t += blockDim.x) {
                a0 = fma(x0[t], __ldcg(y0 + t), a0);
                if (two) a1 = fma(x1[t], __ldcg(y1 + t), a1);
            }
            double v2[2] = {(double)a0, (double)a1};
            double d[2];
            cta_sums<2>(v2, s_red, d);
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            if (which >= 0) {
                const int lw = which ? lb : l;
                const int64_t i = which ? i1 : i0, j = which ? j1 : j0;
                const double xii = Xd[i];
                const double a = (xii != 0.0) ? 2.0 * Sd[j] * xii : 0.0;
                step_constants<T>(2.0 * W[i * q + j] + 2.0 * d[which], a,
                                  __ldcg(Theta + i * q + j), lam, pre, B, lw);
            }
        }
        {
            // 2 (S_xx)_{i a} Sigma_{b j}: coordinate l = (i, j), earlier l1 = (a, b)
            const int ncoef = nb * (nb - 1) / 2;
            for (int64_t e = gtid; e < ncoef; e += gthreads) {
                int l, l1;
                decode_pair((int)e, l, l1);
                const int64_t i = sa[l], j = sb[l];
                const int64_t a = sa[l1], bq = sb[l1];
                gcoef[colbase(l1, B) + (l - l1 - 1)] = T(2) * Sxx[i * p + a] * Sig[bq * q + j];
            }
        }

        // ---- phase B ----
        if (last_cta(scr.ticket, nblk)) {
            phase_b<T, NS>(nb, B, gcoef, pre, reinterpret_cast<T *>(work),
                           reinterpret_cast<T *>(work) + coef_slots(B), scr.mu, scr.err);
            for (int l = threadIdx.x; l < nb; l += blockDim.x) {
                const int64_t i = sa[l], j = sb[l];
                Theta[i * q + j] = __ldcg(Theta + i * q + j) + scr.mu[l];
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: dVt[t][i] += sum over the segment of row i of mu Sigma[t][j] ----
        {
            T *smu = reinterpret_cast<T *>(work);
            for (int l = threadIdx.x; l < nb; l += blockDim.x) smu[l] = (T)__ldcg(scr.mu + l);
            __syncthreads();
            const int nseg = *snseg;
            for (int64_t t = r0 + warp; t < r1; t += (kThreads / 32)) {
                const T *Sr = Sig + t * q;
                T *Vr = dVt + t * p;
                for (int g = 0; g < nseg; g++) {
                    const int l0 = sseg[g], l1 = sseg[g + 1];
                    T sv[NS], mv[NS];
#pragma unroll
                    for (int k = 0; k < NS; k++) {
                        const int l = l0 + lane + 32 * k;
                        sv[k] = T(0);
                        mv[k] = T(0);
                        if (l < l1) {
                            mv[k] = smu[l];
                            sv[k] = Sr[sb[l]];
                        }
                    }
                    T dot = T(0);
#pragma unroll
                    for (int k = 0; k < NS; k++) dot = fma(mv[k], sv[k], dot);
                    dot = warp_sum(dot);
                    if (lane == 0) {
                        const int64_t i = sa[l0];
                        Vr[i] = __ldcg(Vr + i) + dot;
                    }
                }
            }
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
    }
}

// A persistent pass needs every SM at once; two of them issued from different host threads
// (concurrent solves) could each hold part of the GPU while waiting at a grid barrier for
// the rest.  One process-wide lock covers a pass from its launch to its completion check, so
// passes of concurrent solves run one after another while other kernels still overlap.
std::mutex &coop_mutex() {
    static std::mutex m;
    return m;
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
    (void)plan;
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<T>(B).total;
    void *args[] = {(void *)&q, (void *)&Sigma, (void *)&Psi, (void *)&Sd, (void *)&Pd,
                    (void *)&G, (void *)&Lambda, (void *)&m, (void *)&ai, (void *)&aj,
                    (void *)&lam_off, (void *)&lam_diag, (void *)&D, (void *)&U, (void *)&B,
                    (void *)&scr};
    const void *fn;
    switch (B) {
        case 32: fn = (const void *)lambda_sweep_kernel<T, 1>; break;
        case 64: fn = (const void *)lambda_sweep_kernel<T, 2>; break;
        case 128: fn = (const void *)lambda_sweep_kernel<T, 4>; break;
        case 256: fn = (const void *)lambda_sweep_kernel<T, 8>; break;
        default: return CGGM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(coop_mutex());
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
    (void)plan;
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<double>(B).total;
    void *args[] = {(void *)&q, (void *)&Sigma, (void *)&Psi, (void *)&Sd, (void *)&Pd,
                    (void *)&G, (void *)&Lambda, (void *)&m, (void *)&ai, (void *)&aj,
                    (void *)&lam_off, (void *)&lam_diag, (void *)&D, (void *)&U, (void *)&B,
                    (void *)&scr};
    const void *fn = B == 32 ? (const void *)lambda_sweep_kernel<double, 1>
                   : B == 64 ? (const void *)lambda_sweep_kernel<double, 2>
                             : (const void *)lambda_sweep_kernel<double, 4>;
    std::lock_guard<std::mutex> lock(coop_mutex());
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
    (void)plan;
    CGGM_TRY(scratch_reserve(scr, B, sweep_grid()));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.ticket, 0, sizeof(unsigned), st));
    const size_t smem = smem_layout<T>(B).total;
    void *args[] = {(void *)&p, (void *)&q, (void *)&Sxx, (void *)&Xd, (void *)&Sigma,
                    (void *)&Sd, (void *)&W, (void *)&Theta, (void *)&m, (void *)&ti,
                    (void *)&tj, (void *)&lam, (void *)&dV, (void *)&B, (void *)&scr};
    const void *fn;
    switch (B) {
        case 32: fn = (const void *)theta_sweep_kernel<T, 1>; break;
        case 64: fn = (const void *)theta_sweep_kernel<T, 2>; break;
        case 128: fn = (const void *)theta_sweep_kernel<T, 4>; break;
        case 256: fn = (const void *)theta_sweep_kernel<T, 8>; break;
        default: return CGGM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(coop_mutex());
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
