// Coordinate-descent passes of the alternating Newton method, as blocked exact
// Gauss-Seidel on the GPU.
//
// The pass visits the active coordinates in order, and each step depends on all the
// steps before it through the cache (U = D Sigma for Lambda, Section 3.1; Delta V =
// Delta Theta Sigma for Theta, Section 3.2).  The GPU form keeps that order and that
// arithmetic exactly, up to the order of floating-point sums, by cutting the list into
// batches of B consecutive coordinates:
//   phase A: for every coordinate of the batch, its dot products against the cache as
//           it stands at the start of the batch, two coordinates per CTA, and from them
//           the step constants; also the coefficients by which each step of the batch
//           changes the dot products of the later ones (entries of Sigma, Psi, S_xx).
//   phase B (one warp of CTA 0): the B steps in order.  A step's dot products differ
//           from their batch-start values only by the updates of the earlier steps of
//           the same batch, and those corrections are bilinear in the coefficients, so
//           the warp applies them exactly (forward substitution with a soft-threshold
//           at every step).
//   phase C (all CTAs): applies the batch's B updates to the cache rows.
// Phase A of batch k+1 runs on CTAs 1.. while CTA 0 runs phase B of batch k; the cache it
// reads then lacks batch k's update, and the missing part of each dot product is
// sum_l X(k+1, k)[., l] mu_l over batch k's steps mu, with coefficients X of the same form
// as the in-batch ones.  Phase C forms that sum once mu is known, and phase B of batch k+1
// starts its correction sums from it.  Grid barriers separate B from C and C from the
// next B.
#include "sweeps.cuh"
#include "mbar.cuh"

#include <cooperative_groups.h>
#include <mutex>

namespace cggm {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Phase C: each warp updates this many cache rows at once, their loads all issued before
// the first use, so that the L2 round trips of different rows overlap.
constexpr int kRowsInFlight = 4;

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// ---------------------------------------------------------------------------------
// shared pieces of the sweep kernels
// ---------------------------------------------------------------------------------
// Per-coordinate step constants, formed in double in phase A and stored in the cache
// type T (hi + lo pairs where the value carries the result).  The exact minimiser of
// (a/2) mu^2 + b mu + lam |c + mu| (Appendix A.1) is mu = -c + S_{lam/a}(c - b/a); written
// with  vp = -(b + lam)/a  (the step when the soft-threshold takes its upper branch),
// vm = (lam - b)/a  (lower branch) and mc = -c  (the entry goes to zero), and since vp <= vm,
//   mu = median(vp, mc, vm) = max(vp, min(vm, mc)):
// the upper branch is taken exactly when vp > -c, the lower one when vm < -c.  A correction
// sum acc added to b shifts both vp and vm by -acc/a, so they are kept as
// vp - ai acc, vm - ai acc with ai = 1/a.  Zero curvature (a = 0): vp = vm = -c, ai = 0.
enum { PRE_VPH, PRE_VPL, PRE_VMH, PRE_VML, PRE_AI, PRE_MC, PRE_N };
static_assert(PRE_N == kStepConstants, "step constant count");

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
        split<T>(-(base + lam) * ai, o + PRE_VPH * B + l, o + PRE_VPL * B + l);
        split<T>((lam - base) * ai, o + PRE_VMH * B + l, o + PRE_VML * B + l);
        o[PRE_AI * B + l] = (T)ai;
    } else {  // zero curvature: the entry goes to zero
        split<T>(-c, o + PRE_VPH * B + l, o + PRE_VPL * B + l);
        split<T>(-c, o + PRE_VMH * B + l, o + PRE_VML * B + l);
        o[PRE_AI * B + l] = T(0);
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


struct SmemLayout {
    size_t meta;  // twice (current and next batch): sa[B], sb[B], sseg[B + 1], nseg (ints)
    size_t work;  // union: phase B coef[coef_slots(B)], step constants [PRE_N][B], corr[B] (T);
                  //        phase C mu[B] (T)
    size_t total;
};

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int B) {
    SmemLayout s;
    s.meta = 0;
    size_t off = (size_t)2 * (3 * B + 2) * sizeof(int32_t);  // two batches' metadata
    off = (off + 15) & ~size_t(15);
    s.work = off;
    const size_t phb = ((size_t)coef_slots(B) + PRE_N * B + B + 8) * sizeof(T);
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
__device__ void forward_substitution(int nb, const T *__restrict__ pre, const T *acc0,
                                     const T *coef, uint64_t *mb, uint32_t &phase,
                                     double *mu_out, int *err) {
    // pre[] holds zeros for padding coordinates l >= nb, which give mu = 0 whatever the
    // correction sum (also a non-finite one: fmin / fmax return the other operand), so
    // panels run all 32 steps without branches.  B is a compile-time constant, so that every coefficient address
    // below is the lane index plus an immediate offset.
    constexpr int B = NS * 32;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    int lost = -1;  // first panel whose data did not arrive (NS: the step constants)
    if (!mbar_wait(&mb[NS], (phase >> NS) & 1u, err)) {
        lost = 0;
        for (int s = 0; s * 32 < nb && s < NS; s++)
            if (mbar_wait(&mb[s], (phase >> s) & 1u, err, false)) phase ^= 1u << s;
        if (mbar_wait(&mb[NS], (phase >> NS) & 1u, err, false)) phase ^= 1u << NS;
        return;
    }
    phase ^= 1u << NS;
    T acc[NS];  // correction sums, starting from the corrections carried from the previous batch
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = acc0[s * 32 + lane];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s * 32 >= nb) break;
        // the coefficients of panel s (columns 32 s .. 32 s + 31) land on mb[s]
        if (!mbar_wait(&mb[s], (phase >> s) & 1u, err)) {
            lost = s;
            break;
        }
        phase ^= 1u << s;
        const int lo = s * 32 + lane;
        const T vph = pre[PRE_VPH * B + lo], vpl = pre[PRE_VPL * B + lo];
        const T vmh = pre[PRE_VMH * B + lo], vml = pre[PRE_VML * B + lo];
        const T ai = pre[PRE_AI * B + lo], mc = pre[PRE_MC * B + lo];
        // the two branch values of this lane's coordinate with the corrections so far
        T xp = fma(-acc[s], ai, vph) + vpl;
        T xm = fma(-acc[s], ai, vmh) + vml;
        T mymu = T(0);
        // Steps are unrolled by four only: fully unrolled, the batch is tens of kilobytes of
        // straight-line code that the instruction cache has to bring back for every batch.
        // col points at column l of the packed coefficients, col[l2] = coef(l2, l), l2 > l.
        const T *col = coef + colbase(32 * s, B) - 32 * s - 1;
#pragma unroll 4
        for (int o = 0; o < 32; o++) {
            const int l = s * 32 + o;
            const T y = (lane > o) ? ai * col[lane > o ? lo : l + 1] : T(0);
            const T cand = fmax(xp, fmin(xm, mc));
            const T mu = __shfl_sync(0xffffffffu, cand, o);
            mymu = (lane == o) ? cand : mymu;
            xp = fma(-y, mu, xp);
            xm = fma(-y, mu, xm);
#pragma unroll
            for (int s2 = s + 1; s2 < NS; s2++) acc[s2] = fma(col[s2 * 32 + lane], mu, acc[s2]);
            col += B - l - 2;  // colbase(l + 1) - (l + 1) - 1 = colbase(l) - l - 1 + (B - l - 2)
        }
        if (lo < nb) {
            double m = (double)mymu;
            if (!isfinite(m)) { bad = true; m = 0.0; }
            mu_out[lo] = m;
        }
    }
    if (lost >= 0) {  // the pass is abandoned; wait (bounded) for the copies still in flight
        for (int s = lost; s * 32 < nb && s < NS; s++)
            if (mbar_wait(&mb[s], (phase >> s) & 1u, err, false)) phase ^= 1u << s;
    }
    if (bad) set_err(err, DEV_NONFINITE);
}

// Phase B body shared by both passes: one thread starts bulk copies of the step constants
// and carried corrections (completing on mb[NS]) and of each panel's coefficient columns
// (panel s on mb[s]) into shared memory; warp 0 runs the substitution, starting each panel
// as soon as its coefficients have landed.  The step constants of padding coordinates
// (l >= nb) and their corrections were written in global memory with the batch, so the
// copies bring whole arrays.  Coefficient slots of padding coordinates are never used by a
// real coordinate: they only reach the correction sums of padding coordinates.
template <typename T, int NS>
__device__ void phase_b(int nb, const T *gcoef, const T *gpre, const T *gcorr, T *scoef, T *spre,
                        uint64_t *mb, uint32_t &phase, double *mu, int *err) {
    constexpr int B = NS * 32;
    T *scorr = spre + PRE_N * B;
    if ((threadIdx.x >> 5) == 0) {
        if (threadIdx.x == 0) {
            // the sources were written by other CTAs (ordered before this point by the grid
            // barrier) and the destination was last used through the generic proxy
            fence_proxy_async();
            mbar_expect_tx(&mb[NS], (uint32_t)((PRE_N * B + B) * sizeof(T)));
            bulk_load(spre, gpre, (uint32_t)(PRE_N * B * sizeof(T)), &mb[NS]);
            bulk_load(scorr, gcorr, (uint32_t)(B * sizeof(T)), &mb[NS]);
            for (int s = 0; s * 32 < nb; s++) {
                const int c0 = colbase(32 * s, B), c1 = colbase(32 * s + 32, B);
                const uint32_t bytes = (uint32_t)((size_t)(c1 - c0) * sizeof(T));
                mbar_expect_tx(&mb[s], bytes);
                bulk_load(scoef + c0, gcoef + c0, bytes, &mb[s]);
            }
        }
        __syncwarp();
        forward_substitution<T, NS>(nb, spre, scorr, scoef, mb, phase, mu, err);
    }
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
//
// Batches are pipelined one deep: while CTA 0 runs the steps of batch k (phase B), the
// other CTAs compute the dot products of batch k+1 against the cache as it stands before
// batch k's update, together with the coefficients X(k+1, k) that give the change of those
// dot products per unit step of each coordinate of batch k.  After the barrier, phase C
// applies batch k's update to the cache and forms corr(k+1) = X(k+1, k) mu(k), which
// phase B of batch k+1 takes as the initial correction sums.  The result is the same
// sequential pass, with phase A of one batch overlapping phase B of the previous one.
// ---------------------------------------------------------------------------------
struct BatchMeta {
    int32_t *sa, *sb, *sseg, *snseg;
};

__device__ __forceinline__ BatchMeta meta_at(unsigned char *base, int B, int which) {
    int32_t *p = reinterpret_cast<int32_t *>(base) + which * (3 * B + 2);
    return BatchMeta{p, p + B, p + 2 * B, p + 3 * B + 1};
}

// corr[l] = sum_{l'} X[l][l'] mu[l'] for l < nbn (one warp per coordinate over the grid)
template <typename T>
__device__ void cross_corrections(int nbn, int nbk, int B, const T *X, const double *mu,
                                  T *corr) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int l = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); l < nbn; l += warps) {
        T acc = T(0);
        for (int l1 = lane; l1 < nbk; l1 += 32)
            acc = fma(__ldcg(X + (size_t)l * B + l1), (T)__ldcg(mu + l1), acc);
        acc = warp_sum(acc);
        if (lane == 0) corr[l] = acc;
    }
    if (blockIdx.x == gridDim.x - 1)  // padding coordinates of the next batch
        for (int l = nbn + threadIdx.x; l < B; l += blockDim.x) corr[l] = T(0);
}

template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
lambda_sweep_kernel(int64_t q, const T *__restrict__ Sig, const T *__restrict__ Psi,
                    const double *__restrict__ Sd, const double *__restrict__ Pd,
                    const double *__restrict__ G, const double *__restrict__ Lam, int64_t m,
                    const int32_t *__restrict__ ai, const int32_t *__restrict__ aj,
                    double lam_off, double lam_diag, double *D, T *Ut, int B_arg,
                    SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[(kThreads / 32) * 6];
    __shared__ uint64_t s_mb[NS + 1];  // phase B (CTA 0): panels, then step constants
    uint32_t mb_phase = 0;
    constexpr int B = NS * 32;
    if (B_arg != B) return;  // the host launches the instance of its batch size
    const SmemLayout L = smem_layout<T>(B);
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x;
    T *preb = reinterpret_cast<T *>(scr.sub1);                // [2][PRE_N][B]
    T *coefb = reinterpret_cast<T *>(scr.sub2);               // [2][coef_slots(B)]
    T *gX = coefb + 2 * (size_t)coef_slots(B);                // [B][B]
    T *gcorr = gX + (size_t)B * B;                            // [B]
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    const bool vec = (q % VN) == 0;
    const int64_t nbatch = (m + B - 1) / B;
    if (nbatch == 0) return;

    auto S = [&](int64_t x, int64_t y) -> T { return Sig[x * q + y]; };
    auto P = [&](int64_t x, int64_t y) -> T { return Psi[x * q + y]; };
    // change of the three dot products of coordinate (pi, pj) per unit step of (pa, pb):
    // (Sigma E Sigma)_ij + (Psi E Sigma)_ij + (Psi E Sigma)_ji with E = E_ab + E_ba (E_aa on
    // the diagonal), the middle term doubled when i == j.  Sigma and Psi are symmetric, and
    // every entry that involves pb (the index that varies fastest across threads) is read
    // along a row, so that neighbouring threads read neighbouring words.
    auto coefficient = [&](int64_t pi, int64_t pj, int64_t pa, int64_t pb) -> T {
        const T s_ia = S(pi, pa), s_ib = S(pi, pb), s_aj = S(pa, pj), s_jb = S(pj, pb);
        const T p_ia = P(pi, pa), p_ib = P(pi, pb), p_ja = P(pj, pa), p_jb = P(pj, pb);
        T c1, c2, c3;
        if (pa != pb) {
            c1 = s_ia * s_jb + s_ib * s_aj;
            c2 = p_ia * s_jb + p_ib * s_aj;
            c3 = p_ja * s_ib + p_jb * s_ia;
        } else {
            c1 = s_ia * s_aj;
            c2 = p_ia * s_aj;
            c3 = p_ja * s_ia;
        }
        return (pi != pj) ? (c1 + c2 + c3) : (c1 + T(2) * c2);
    };

    // Phase A of the batch held in `bm` (nb coordinates) by the CTAs rank0 .. nblk-1:
    // dot products against the cache, step constants -> pre, in-batch coefficients -> coef,
    // and, when prev is given, the cross coefficients against the previous batch -> gX.
    auto phase_a = [&](const BatchMeta &bm, int nb, T *pre, T *coef, const BatchMeta *prev,
                       int nbp, int rank0) {
        const int nA = (int)nblk - rank0, rank = (int)blockIdx.x - rank0;
        for (int l = rank; l < nb; l += 2 * nA) {
            const int lb = l + nA;
            const bool two = lb < nb;
            const int64_t i0 = bm.sa[l], j0 = bm.sb[l];
            const int64_t i1 = two ? bm.sa[lb] : i0, j1 = two ? bm.sb[lb] : j0;
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
        const int64_t t0 = (int64_t)rank * blockDim.x + threadIdx.x;
        const int64_t nt = (int64_t)nA * blockDim.x;
        for (int64_t e = t0; e < (int64_t)(B - nb) * PRE_N; e += nt) {  // padding coordinates
            const int k = (int)(e / (B - nb)), l = nb + (int)(e % (B - nb));
            pre[k * B + l] = T(0);
        }
        const int ncoef = nb * (nb - 1) / 2;
        for (int64_t e = t0; e < ncoef; e += nt) {
            int l, l1;
            decode_pair((int)e, l, l1);
            coef[colbase(l1, B) + (l - l1 - 1)] = coefficient(bm.sa[l], bm.sb[l], bm.sa[l1], bm.sb[l1]);
        }
        if (prev) {
            const int64_t ncross = (int64_t)nb * nbp;
            for (int64_t e = t0; e < ncross; e += nt) {
                const int l = (int)(e / nbp), l1 = (int)(e % nbp);
                gX[(size_t)l * B + l1] = coefficient(bm.sa[l], bm.sb[l], prev->sa[l1], prev->sb[l1]);
            }
        }
    };

    // prologue: phase A of batch 0 by every CTA; no correction from an earlier batch
    BatchMeta cur = meta_at(smem + L.meta, B, 0), nxt = meta_at(smem + L.meta, B, 1);
    int nbk = (int)(m < B ? m : B);
    load_batch(ai, aj, 0, nbk, cur.sa, cur.sb, cur.sseg, cur.snseg);
    phase_a(cur, nbk, preb, coefb, nullptr, 0, 0);
    if (blockIdx.x == 0) {
        for (int l = threadIdx.x; l < B; l += blockDim.x) gcorr[l] = T(0);
        if (threadIdx.x == 0) {
            for (int k = 0; k <= NS; k++) mbar_init(&s_mb[k], 1);
            mbar_init_fence();
        }
    }
    if (!grid_sync(scr.bar, scr.err, nblk)) return;

    for (int64_t k = 0; k < nbatch; k++) {
        const int64_t sk = k * B, sn = sk + B;
        const int nbn = (int)(sn < m ? ((m - sn) < B ? (m - sn) : B) : 0);
        T *pre_k = preb + (size_t)(k & 1) * PRE_N * B, *coef_k = coefb + (size_t)(k & 1) * coef_slots(B);
        T *pre_n = preb + (size_t)((k + 1) & 1) * PRE_N * B;
        T *coef_n = coefb + (size_t)((k + 1) & 1) * coef_slots(B);
        if (nbn > 0) load_batch(ai, aj, sn, nbn, nxt.sa, nxt.sb, nxt.sseg, nxt.snseg);

        // ---- phase B of batch k on CTA 0, phase A of batch k+1 on the others ----
        if (blockIdx.x == 0) {
            phase_b<T, NS>(nbk, coef_k, pre_k, gcorr, reinterpret_cast<T *>(work),
                           reinterpret_cast<T *>(work) + coef_slots(B), s_mb, mb_phase, scr.mu,
                           scr.err);
        } else if (nbn > 0) {
            phase_a(nxt, nbn, pre_n, coef_n, &cur, nbk, 1);
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: batch k's update on this CTA's rows; corrections for batch k+1 ----
        // coordinate (a, b) of a segment with row a: U_a += mu Sigma_b, U_b += mu Sigma_a
        // (b != a); transposed: Ut[t][a] += sum mu Sigma[t][b], Ut[t][b] += mu Sigma[t][a]
        {
            T *smu = reinterpret_cast<T *>(work);
            for (int l = threadIdx.x; l < nbk; l += blockDim.x) {
                const double mu = __ldcg(scr.mu + l);
                smu[l] = (T)mu;
                if (blockIdx.x == nblk - 1) {  // the direction itself
                    const int64_t i = cur.sa[l], j = cur.sb[l];
                    D[i * q + j] = mu;
                    if (i != j) D[j * q + i] = mu;
                }
            }
            __syncthreads();
            const int nseg = *cur.snseg;
            constexpr int R = kRowsInFlight;
            for (int g = 0; g < nseg; g++) {
                const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
                const int a = cur.sa[l0];
                int bv[NS];
                T mv[NS];
#pragma unroll
                for (int kk = 0; kk < NS; kk++) {
                    const int l = l0 + lane + 32 * kk;
                    bv[kk] = (l < l1) ? cur.sb[l] : -1;
                    mv[kk] = (l < l1) ? smu[l] : T(0);
                }
                for (int64_t tb = r0 + warp; tb < r1; tb += kWarps * R) {
                    T sta[R], sv[R][NS], uv[R][NS];
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int64_t t = tb + (int64_t)kWarps * r;
                        sta[r] = T(0);
#pragma unroll
                        for (int kk = 0; kk < NS; kk++) sv[r][kk] = uv[r][kk] = T(0);
                        if (t < r1) {
                            const T *Sr = Sig + t * q;
                            const T *Ur = Ut + t * q;
                            sta[r] = Sr[a];
#pragma unroll
                            for (int kk = 0; kk < NS; kk++) {
                                if (bv[kk] >= 0) {
                                    sv[r][kk] = Sr[bv[kk]];
                                    if (bv[kk] != a) uv[r][kk] = __ldcg(Ur + bv[kk]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int64_t t = tb + (int64_t)kWarps * r;
                        if (t >= r1) break;  // warp-uniform
                        T *Ur = Ut + t * q;
                        T dot = T(0);
#pragma unroll
                        for (int kk = 0; kk < NS; kk++) {
                            if (bv[kk] >= 0) {
                                dot = fma(mv[kk], sv[r][kk], dot);
                                if (bv[kk] != a) Ur[bv[kk]] = uv[r][kk] + mv[kk] * sta[r];
                            }
                        }
                        dot = warp_sum(dot);
                        if (lane == 0) Ur[a] = __ldcg(Ur + a) + dot;
                    }
                }
                __syncwarp();  // this segment's writes before the next segment's reads
            }
            if (nbn > 0) cross_corrections<T>(nbn, nbk, B, gX, scr.mu, gcorr);
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
        BatchMeta tmp = cur;
        cur = nxt;
        nxt = tmp;
        nbk = nbn;
    }
}

// ---------------------------------------------------------------------------------
// Theta sweep kernel.  Cache: dVt = (Delta V)^T (q x p), dVt[j][t] = (Delta Theta Sigma)[t][j].
// Pipelined like the Lambda pass.
// ---------------------------------------------------------------------------------
template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
theta_sweep_kernel(int64_t p, int64_t q, const T *__restrict__ Sxx, const double *__restrict__ Xd,
                   const T *__restrict__ Sig, const double *__restrict__ Sd,
                   const double *__restrict__ W, double *Theta, int64_t m,
                   const int32_t *__restrict__ ti, const int32_t *__restrict__ tj, double lam,
                   T *dVt, int B_arg, SweepScratch scr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[(kThreads / 32) * 2];
    __shared__ uint64_t s_mb[NS + 1];  // phase B (CTA 0): panels, then step constants
    uint32_t mb_phase = 0;
    constexpr int B = NS * 32;
    if (B_arg != B) return;  // the host launches the instance of its batch size
    const SmemLayout L = smem_layout<T>(B);
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nblk = gridDim.x;
    T *preb = reinterpret_cast<T *>(scr.sub1);
    T *coefb = reinterpret_cast<T *>(scr.sub2);
    T *gX = coefb + 2 * (size_t)coef_slots(B);
    T *gcorr = gX + (size_t)B * B;
    const int64_t rows_per = (q + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = (r0 + rows_per) < q ? (r0 + rows_per) : q;
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    const int64_t nbatch = (m + B - 1) / B;
    if (nbatch == 0) return;

    // change of (S_xx Delta V)_ij per unit step of Theta_ab, times 2: 2 (S_xx)_{i a} Sigma_{j b}
    // (Sigma symmetric; read along row j, b varying fastest across threads)
    auto coefficient = [&](int64_t i, int64_t j, int64_t a, int64_t b) -> T {
        return T(2) * Sxx[i * p + a] * Sig[j * q + b];
    };

    auto phase_a = [&](const BatchMeta &bm, int nb, T *pre, T *coef, const BatchMeta *prev,
                       int nbp, int rank0) {
        const int nA = (int)nblk - rank0, rank = (int)blockIdx.x - rank0;
        // rows of Delta V that can be nonzero: those at or before this batch's first row
        const int64_t tmax = (int64_t)bm.sa[0] + 1;
        for (int l = rank; l < nb; l += 2 * nA) {
            const int lb = l + nA;
            const bool two = lb < nb;
            const int64_t i0 = bm.sa[l], j0 = bm.sb[l];
            const int64_t i1 = two ? bm.sa[lb] : i0, j1 = two ? bm.sb[lb] : j0;
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
        const int64_t t0 = (int64_t)rank * blockDim.x + threadIdx.x;
        const int64_t nt = (int64_t)nA * blockDim.x;
        for (int64_t e = t0; e < (int64_t)(B - nb) * PRE_N; e += nt) {  // padding coordinates
            const int k = (int)(e / (B - nb)), l = nb + (int)(e % (B - nb));
            pre[k * B + l] = T(0);
        }
        const int ncoef = nb * (nb - 1) / 2;
        for (int64_t e = t0; e < ncoef; e += nt) {
            int l, l1;
            decode_pair((int)e, l, l1);
            coef[colbase(l1, B) + (l - l1 - 1)] = coefficient(bm.sa[l], bm.sb[l], bm.sa[l1], bm.sb[l1]);
        }
        if (prev) {
            const int64_t ncross = (int64_t)nb * nbp;
            for (int64_t e = t0; e < ncross; e += nt) {
                const int l = (int)(e / nbp), l1 = (int)(e % nbp);
                gX[(size_t)l * B + l1] = coefficient(bm.sa[l], bm.sb[l], prev->sa[l1], prev->sb[l1]);
            }
        }
    };

    BatchMeta cur = meta_at(smem + L.meta, B, 0), nxt = meta_at(smem + L.meta, B, 1);
    int nbk = (int)(m < B ? m : B);
    load_batch(ti, tj, 0, nbk, cur.sa, cur.sb, cur.sseg, cur.snseg);
    phase_a(cur, nbk, preb, coefb, nullptr, 0, 0);
    if (blockIdx.x == 0) {
        for (int l = threadIdx.x; l < B; l += blockDim.x) gcorr[l] = T(0);
        if (threadIdx.x == 0) {
            for (int k = 0; k <= NS; k++) mbar_init(&s_mb[k], 1);
            mbar_init_fence();
        }
    }
    if (!grid_sync(scr.bar, scr.err, nblk)) return;

    for (int64_t k = 0; k < nbatch; k++) {
        const int64_t sk = k * B, sn = sk + B;
        const int nbn = (int)(sn < m ? ((m - sn) < B ? (m - sn) : B) : 0);
        T *pre_k = preb + (size_t)(k & 1) * PRE_N * B, *coef_k = coefb + (size_t)(k & 1) * coef_slots(B);
        T *pre_n = preb + (size_t)((k + 1) & 1) * PRE_N * B;
        T *coef_n = coefb + (size_t)((k + 1) & 1) * coef_slots(B);
        if (nbn > 0) load_batch(ti, tj, sn, nbn, nxt.sa, nxt.sb, nxt.sseg, nxt.snseg);

        if (blockIdx.x == 0) {
            phase_b<T, NS>(nbk, coef_k, pre_k, gcorr, reinterpret_cast<T *>(work),
                           reinterpret_cast<T *>(work) + coef_slots(B), s_mb, mb_phase, scr.mu,
                           scr.err);
        } else if (nbn > 0) {
            phase_a(nxt, nbn, pre_n, coef_n, &cur, nbk, 1);
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;

        // ---- phase C: dVt[t][i] += sum over the segment of row i of mu Sigma[t][j] ----
        {
            T *smu = reinterpret_cast<T *>(work);
            for (int l = threadIdx.x; l < nbk; l += blockDim.x) {
                const double mu = __ldcg(scr.mu + l);
                smu[l] = (T)mu;
                if (blockIdx.x == nblk - 1) {  // Theta itself
                    const int64_t i = cur.sa[l], j = cur.sb[l];
                    Theta[i * q + j] = __ldcg(Theta + i * q + j) + mu;
                }
            }
            __syncthreads();
            const int nseg = *cur.snseg;
            constexpr int R = kRowsInFlight;
            for (int g = 0; g < nseg; g++) {
                const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
                const int i = cur.sa[l0];
                int jv[NS];
                T mv[NS];
#pragma unroll
                for (int kk = 0; kk < NS; kk++) {
                    const int l = l0 + lane + 32 * kk;
                    jv[kk] = (l < l1) ? cur.sb[l] : -1;
                    mv[kk] = (l < l1) ? smu[l] : T(0);
                }
                for (int64_t tb = r0 + warp; tb < r1; tb += kWarps * R) {
                    T sv[R][NS];
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int64_t t = tb + (int64_t)kWarps * r;
#pragma unroll
                        for (int kk = 0; kk < NS; kk++)
                            sv[r][kk] = (t < r1 && jv[kk] >= 0) ? Sig[t * q + jv[kk]] : T(0);
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int64_t t = tb + (int64_t)kWarps * r;
                        if (t >= r1) break;  // warp-uniform
                        T dot = T(0);
#pragma unroll
                        for (int kk = 0; kk < NS; kk++) dot = fma(mv[kk], sv[r][kk], dot);
                        dot = warp_sum(dot);
                        if (lane == 0) {
                            T *Vr = dVt + t * p;
                            Vr[i] = __ldcg(Vr + i) + dot;
                        }
                    }
                }
            }
            if (nbn > 0) cross_corrections<T>(nbn, nbk, B, gX, scr.mu, gcorr);
        }
        if (!grid_sync(scr.bar, scr.err, nblk)) return;
        BatchMeta tmp = cur;
        cur = nxt;
        nxt = tmp;
        nbk = nbn;
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
    if (grid < 2) return CGGM_ECUDA;  // phase B runs beside phase A: needs two CTAs at least
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

cggm_status scratch_reserve(SweepScratch &scr) {
    if (scr.mu) return CGGM_OK;
    const int Bmax = 256;  // float; double batches are at most 128 and take less
    CGGM_CUDA_TRY(cudaMalloc(&scr.mu, sizeof(double) * Bmax));
    CGGM_CUDA_TRY(cudaMalloc(&scr.sub1, scratch_sub1_bytes(Bmax, sizeof(float))));
    CGGM_CUDA_TRY(cudaMalloc(&scr.sub2, scratch_sub2_bytes(Bmax, sizeof(float))));
    CGGM_CUDA_TRY(cudaMalloc(&scr.bar, sizeof(GridBarrier)));
    CGGM_CUDA_TRY(cudaMalloc(&scr.err, sizeof(int)));
    CGGM_CUDA_TRY(cudaMemset(scr.bar, 0, sizeof(GridBarrier)));
    CGGM_CUDA_TRY(cudaMemset(scr.err, 0, sizeof(int)));
    return CGGM_OK;
}

void scratch_free(SweepScratch &scr) {
    cudaFree(scr.mu); cudaFree(scr.sub1); cudaFree(scr.sub2);
    cudaFree(scr.bar); cudaFree(scr.err);
    scr = SweepScratch();
}

template <typename T>
cggm_status lambda_sweep(int64_t q, const T *Sigma, const T *Psi, const double *Sd,
                         const double *Pd, const double *G, const double *Lambda, int64_t m,
                         const int32_t *ai, const int32_t *aj, double lam_off, double lam_diag,
                         double *D, T *U, int B, SweepScratch &scr,
                         cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > (sizeof(T) == 4 ? 256 : 128) || (B & (B - 1))) return CGGM_EINVAL;
    CGGM_TRY(scratch_reserve(scr));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
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

// Same pass as lambda_sweep on scratch buffers that the caller has already laid out;
// allocates nothing.
cggm_status lambda_sweep_preplanned_f64(int64_t q, const double *Sigma, const double *Psi,
                                        const double *Sd, const double *Pd, const double *G,
                                        const double *Lambda, int64_t m, const int32_t *ai,
                                        const int32_t *aj, double lam_off, double lam_diag,
                                        double *D, double *U, int B, SweepScratch scr,
                                        cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B != 32 && B != 64 && B != 128) return CGGM_EINVAL;
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
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
                        SweepScratch &scr, cudaStream_t st) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > (sizeof(T) == 4 ? 256 : 128) || (B & (B - 1))) return CGGM_EINVAL;
    CGGM_TRY(scratch_reserve(scr));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
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
                                          double *, int, SweepScratch &, cudaStream_t);
template cggm_status lambda_sweep<float>(int64_t, const float *, const float *, const double *,
                                         const double *, const double *, const double *, int64_t,
                                         const int32_t *, const int32_t *, double, double, double *,
                                         float *, int, SweepScratch &, cudaStream_t);
template cggm_status theta_sweep<double>(int64_t, int64_t, const double *, const double *,
                                         const double *, const double *, const double *, double *,
                                         int64_t, const int32_t *, const int32_t *, double, double *,
                                         int, SweepScratch &, cudaStream_t);
template cggm_status theta_sweep<float>(int64_t, int64_t, const float *, const double *,
                                        const float *, const double *, const double *, double *,
                                        int64_t, const int32_t *, const int32_t *, double, float *,
                                        int, SweepScratch &, cudaStream_t);

}  // namespace cggm
