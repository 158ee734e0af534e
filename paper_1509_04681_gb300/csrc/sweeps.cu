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
//   phase C (CTAs 1..): applies the batch's B updates to the cache rows.
// The phases are pipelined two deep: CTA 0 runs phase B of batch k while the other CTAs
// apply batch k - 1 to the cache (phase C) and then run phase A of batch k + 1 against the
// cache as it stands after batch k - 1.  The missing part of each of batch k + 1's dot
// products is sum_l X(k+1, k)[., l] mu_l over batch k's steps mu, with coefficients X of the
// same form as the in-batch ones; CTA 0's other warps form it during phase B of batch k + 1,
// panel by panel ahead of the steps.  CTA 0 and the other CTAs are ordered by counters, not
// by grid barriers: CTA 0 waits only for the phase A of the batch it runs next.
#include "sweeps.cuh"
#include "mbar.cuh"

#include <chrono>
#include <condition_variable>
#include <cooperative_groups.h>
#include <deque>
#include <mutex>
#include <vector>

namespace cggm {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Phase C: each warp updates this many cache rows at once, their loads all issued before
// the first use, so that the L2 round trips of different rows overlap.
constexpr int kRowsInFlight = 5;
// Phase A: rows per CTA held at once, chunks in flight, bytes per row and chunk.
constexpr int kRingRows = 10;
constexpr int kChunkBytes = 8192;
// The ring holds as many stages of the plan's rows as fit in kRingBytes, up to kMaxStages
// (two stages of ten rows, three of seven; more of fewer rows).  Measured on the 5000 x 5000
// workload: 8 KB chunks in 168 KB took 0.66 s per Lambda pass against 0.72 s with 4 KB in
// 120 KB (fewer, larger copies) and 0.70 s with 16 KB chunks; a larger ring costs L1 cache,
// which the coefficient gathers use (the Theta pass, 0.61 s, barely moves).
constexpr int kMaxStages = 16;
// Phase A: warps 0 .. kDotWarps - 1 compute the dot products (through the ring) while the
// other warps form the coefficients; the dot warps synchronise among themselves on named
// barrier kBarDots.
constexpr int kDotWarps = 4;
constexpr int kDotThreads = kDotWarps * 32;
constexpr int kCoefThreads = kThreads - kDotThreads;
constexpr int kBarDots = 1;
// Phase B on CTA 0: warps 1 .. kWarps - 2 (the carried corrections) on named barrier kBarCorr.
constexpr int kBarCorr = 2;

__device__ __forceinline__ void bar_sync_n(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// barrier `id` over n threads that also reduces p by AND
__device__ __forceinline__ bool bar_and_n(int id, int n, bool p) {
    int r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.s32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, %2, %3, pi;\n\tselp.s32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((int)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}
constexpr size_t kRingBytes = (size_t)168 << 10;

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

// Step constants in two parts.  The part that depends on scalars only (G_ij or W_ij, the
// curvature a from the Sigma/Psi or S_xx diagonals, lambda, c) is formed in double before
// the dot products: vp0 = -(g + lam) / a and vm0 = (lam - g) / a, split into hi + lo
// words of T.  The dot products' part enters afterwards in T: their sum d shifts both by
// -d / a, which is folded into the lo words (d carries the cache type's accuracy anyway),
// so that only a few T operations follow the dot products.  curv: a > 0 (otherwise the
// entry goes to zero: vp = vm = -c, 1/a = 0).
template <typename T>
struct StepHead {
    T vph, vpl, vmh, vml, ai, mc;
};

template <typename T>
__device__ StepHead<T> step_head(double g, double a, double lam, double c) {
    StepHead<T> h;
    if (a > 0.0 && isfinite(a)) {
        const double ai = 1.0 / a;
        split<T>(-(g + lam) * ai, &h.vph, &h.vpl);
        split<T>((lam - g) * ai, &h.vmh, &h.vml);
        h.ai = (T)ai;
    } else {  // zero curvature: the entry goes to zero
        split<T>(-c, &h.vph, &h.vpl);
        split<T>(-c, &h.vmh, &h.vml);
        h.ai = T(0);
    }
    h.mc = (T)(-c);
    return h;
}

// Stores coordinate l's constants with the dot products' sum d applied.
template <typename T>
__device__ void step_constants(const StepHead<T> &h, T d, T *pre, int B, int l) {
    const T corr = d * h.ai;  // zero when the curvature is zero
    pre[PRE_VPH * B + l] = h.vph;
    pre[PRE_VPL * B + l] = h.vpl - corr;
    pre[PRE_VMH * B + l] = h.vmh;
    pre[PRE_VML * B + l] = h.vml - corr;
    pre[PRE_AI * B + l] = h.ai;
    pre[PRE_MC * B + l] = h.mc;
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

// Phase B keeps every panel's coefficients in shared memory up to B = 256; above, they do not
// fit (B = 512: 523 KB in float) and two panel buffers take turns.  Panel s (columns 32 s ..
// 32 s + 31) holds colbase(32 s + 32) - colbase(32 s) = 32 (B - 1) - 1024 s - 496 entries,
// the largest for s = 0.
__host__ __device__ constexpr int panel_bufs(int B) { return B <= 256 ? B / 32 : 2; }
__host__ __device__ constexpr int panel_max(int B) { return ((32 * B - 528) + 3) & ~3; }
__host__ __device__ constexpr int coef_area(int B) {
    return panel_bufs(B) == B / 32 ? coef_slots(B) : panel_bufs(B) * panel_max(B);
}
// offset of panel s's buffer in the coefficient area
__host__ __device__ __forceinline__ int panel_off(int s, int B) {
    return panel_bufs(B) == B / 32 ? colbase(32 * s, B) : (s % panel_bufs(B)) * panel_max(B);
}
// shared-memory slots for the coefficients (16-byte multiple with copy slack)


struct SmemLayout {
    size_t meta;  // three batches (k, k + 1, k + 2): sa[B], sb[B], sseg[B + 1], nseg (ints)
    size_t work;  // union: phase A ring of row chunks (kRingBytes, all stages);
                  //        phase B (CTA 0) coefficient panels [coef_area(B)], step constants
                  //          [2][PRE_N][B], carried corrections [B] (T), steps [2][B]
                  //          (double);
                  //        phase C (the other CTAs) mu[B] (T) at work + phc
    size_t phc;   // offset of phase C's area within the work area
    size_t total;
};

// Phase B's shared memory on CTA 0: coefficient panels, two batches' step constants and the
// carried corrections (T, with copy slack), then two batches' steps (double) at this offset.
template <typename T>
__host__ __device__ constexpr size_t phase_b_steps_offset(int B) {
    return (((size_t)coef_area(B) + 2 * PRE_N * B + B + 8) * sizeof(T) + 15) & ~size_t(15);
}

template <typename T>
__host__ __device__ inline SmemLayout smem_layout(int B) {
    SmemLayout s;
    s.meta = 0;
    size_t off = (size_t)3 * (3 * B + 2) * sizeof(int32_t);  // three batches' metadata
    off = (off + 15) & ~size_t(15);
    s.work = off;
    const size_t phb = phase_b_steps_offset<T>(B) + 2 * (size_t)B * sizeof(double);
    const size_t phc = (size_t)(B + 4) * sizeof(T);
    s.phc = phb;
    size_t w = phb + phc;
    w = w > kRingBytes ? w : kRingBytes;
    s.total = off + w;
    return s;
}

// Issues the bulk copy of panel s's coefficient columns into its buffer (one thread).
template <typename T, int NS>
__device__ __forceinline__ void issue_panel(int s, const T *gcoef, T *scoef, uint64_t *mb) {
    constexpr int B = NS * 32;
    const int c0 = colbase(32 * s, B), c1 = colbase(32 * s + 32, B);
    const uint32_t bytes = (uint32_t)((size_t)(c1 - c0) * sizeof(T));
    uint64_t *bar = &mb[s % panel_bufs(B)];
    mbar_expect_tx(bar, bytes);
    bulk_load(scoef + panel_off(s, B), gcoef + c0, bytes, bar);
}

// Shared-memory flags between the warps of CTA 0 (release / acquire at CTA scope).
__device__ __forceinline__ int ld_acquire_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// Waits (bounded) until the flag reaches target; returns the value seen, or -1 at the
// deadline (DEV_TIMEOUT recorded) or when another thread has recorded an error.  The flags
// are raised by other warps of the same CTA.
__device__ int wait_flag(const int *flag, int target, int *err, unsigned sleep_ns) {
    int v = ld_acquire_cta(flag);
    if (v >= target) return v;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; it++) {
        if (sleep_ns) __nanosleep(sleep_ns);
        v = ld_acquire_cta(flag);
        if (v >= target) return v;
        if ((it & 63u) == 0) {
            if (*(volatile int *)err != 0) return -1;
            if (global_ns() - t0 > 2000000000ull) {
                set_err(err, DEV_TIMEOUT);
                return -1;
            }
        }
    }
}

// One thread: waits (bounded) until the device-wide counter reaches target (acquire).
__device__ bool wait_counter(const unsigned long long *c, unsigned long long target, int *err) {
    if (ld_acquire_u64(c) >= target) return true;
    const uint64_t t0 = global_ns();
    for (unsigned it = 1;; it++) {
        if (ld_acquire_u64(c) >= target) return true;
        if ((it & 63u) == 0) {
            if (ld_acquire_int(err) != 0) return false;
            if (global_ns() - t0 > 2000000000ull) {
                set_err(err, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// CTA 0's part of a pass: phase B of every batch, by three groups of warps that meet only
// through shared-memory flags and mbarriers, so that the serial chain never waits for a
// copy, a correction or a device-wide counter that could have been ready earlier.
//   warp 0 (the chain): for each batch in turn, the forward substitution
//     b_l = base_l + sum_{l' < l} coef(l, l') mu_l',  mu_l = -c_l + S_{lam_l/a_l}(c_l - b_l/a_l)
//     (the exact minimiser of (a/2) mu^2 + b mu + lam |c + mu|, Appendix A.1, written with
//     the step constants), panel by panel: lane k owns coordinates 32 s + k; at step l every
//     lane forms the candidate step of its own coordinate and the owner's candidate is
//     broadcast, so the dependent chain per coordinate is a few T operations and one warp
//     shuffle.  coef is the strictly lower triangle, column-packed (colbase), in shared
//     memory.  After each panel it stores the panel's steps (device memory for the other
//     CTAs, shared memory for warps 1..6) and raises `prog` (panels done, counted over the
//     pass: batch k's panel s is number k NS + s).
//   warp 7, lane 0 (the feeder): for each batch k, once the other CTAs' phase A of batch k
//     is complete (a_done), the bulk copies of its step constants into one of two buffers and
//     of each coefficient panel into its buffer as soon as the chain has finished the
//     panel that last occupied it; and, as soon as the chain has finished a batch, also
//     while it waits, publishes that batch's steps to the other CTAs (mu_ready).
//   warps 1..6 (the corrections): for each batch k > 0, the part that batch k - 1 carries
//     into it, corr[l] = sum_{l'} X(k, k-1)[l][l'] mu_{l'} (phase A of batch k ran against the
//     cache without batch k - 1's steps), panel by panel, raising `corr_prog` (same
//     numbering as prog); the rows of panel 0 are loaded ahead, while batch k - 1 still runs.
// Shared memory (the work area): coefficient panels [coef_area(B)], step constants [2][PRE_N][B]
// and corrections [B] (T), then the steps of two batches [2][B] (double).
template <typename T, int NS>
__device__ void phase_b_cta0(int64_t nbatch, int64_t m, const T *preb, const T *coefb,
                             const T *gX, unsigned long long nA, unsigned char *work,
                             uint64_t *mb, uint64_t *mbpre, int *prog, int *corr_prog,
                             SweepScratch scr) {
    constexpr int B = NS * 32;
    constexpr int NBUF = panel_bufs(B);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *scoef = reinterpret_cast<T *>(work);
    T *spre = scoef + coef_area(B);  // [2][PRE_N][B]
    T *scorr = spre + 2 * PRE_N * B;
    double *smu = reinterpret_cast<double *>(work + phase_b_steps_offset<T>(B));
    int *err = scr.err;
    auto nb_of = [&](int64_t k) -> int {
        const int64_t s0 = k * B;
        return s0 < m ? (int)((m - s0) < B ? (m - s0) : B) : 0;
    };

    if (warp == 0) {  // ---- the chain ----
        uint32_t phase = 0, pphase = 0;
        for (int64_t k = 0; k < nbatch; k++) {
            const int nb = nb_of(k);
            const int pb = (int)(k & 1);
            const T *pre = spre + (size_t)pb * PRE_N * B;
            double *mu_g = scr.mu + (size_t)pb * B;
            double *mu_s = smu + (size_t)pb * B;
            if (!mbar_wait(&mbpre[pb], (pphase >> pb) & 1u, err)) return;
            pphase ^= 1u << pb;
            // pre[] holds zeros for padding coordinates l >= nb, which give mu = 0 whatever
            // the correction sum (also a non-finite one: fmin / fmax return the other
            // operand), so panels run all 32 steps without branches
            T acc[NS];  // correction sums: the in-batch steps of earlier panels, then the
                        // carried part, added when the panel starts
#pragma unroll
            for (int s = 0; s < NS; s++) acc[s] = T(0);
            bool bad = false;
#pragma unroll
            for (int s = 0; s < NS; s++) {
                if (s * 32 >= nb) break;
                const int bi = s % NBUF;
                if (!mbar_wait(&mb[bi], (phase >> bi) & 1u, err)) return;
                phase ^= 1u << bi;
                if (k > 0) {
                    if (wait_flag(corr_prog, (int)(k * NS) + s + 1, err, 0) < 0) return;
                    acc[s] += scorr[s * 32 + lane];
                }
                const int lo = s * 32 + lane;
                const T vph = pre[PRE_VPH * B + lo], vpl = pre[PRE_VPL * B + lo];
                const T vmh = pre[PRE_VMH * B + lo], vml = pre[PRE_VML * B + lo];
                const T ai = pre[PRE_AI * B + lo], mc = pre[PRE_MC * B + lo];
                // the two branch values of this lane's coordinate with the corrections so far
                T xp = fma(-acc[s], ai, vph) + vpl;
                T xm = fma(-acc[s], ai, vmh) + vml;
                T mymu = T(0);
                // Steps are unrolled by four only: fully unrolled, the batch is tens of
                // kilobytes of straight-line code that the instruction cache has to bring back
                // for every batch.  col points at column l of the packed coefficients,
                // col[l2] = coef(l2, l), l2 > l.
                const T *col = scoef + panel_off(s, B) - 32 * s - 1;
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
                    for (int s2 = s + 1; s2 < NS; s2++)
                        acc[s2] = fma(col[s2 * 32 + lane], mu, acc[s2]);
                    col += B - l - 2;  // colbase(l + 1) - (l + 1) - 1 = colbase(l) - l - 1 + (B - l - 2)
                }
                if (lo < nb) {
                    double mv = (double)mymu;
                    if (!isfinite(mv)) {
                        bad = true;
                        mv = 0.0;
                    }
                    mu_g[lo] = mv;
                    mu_s[lo] = mv;
                }
                __syncwarp();  // the panel's steps stored and its buffer read
                if (lane == 0) st_release_cta(prog, (int)(k * NS) + s + 1);
            }
            if (bad) set_err(err, DEV_NONFINITE);
        }
        return;
    }

    if (warp == kWarps - 1) {  // ---- the feeder ----
        if (lane != 0) return;
        int nuse[NBUF > 2 ? NBUF : 2] = {};  // copies issued into each panel buffer
        int npre[2] = {0, 0};
        bool ok = true;
        int64_t published = 0;  // batches whose steps are published
        auto publish_upto = [&](int64_t done) {  // batches 0 .. done - 1 are complete
            if (done > published) {
                __threadfence();
                red_release_add(&scr.bar->mu_ready, (unsigned long long)(done - published));
                published = done;
            }
        };
        for (int64_t k = 0; k < nbatch && ok; k++) {
            const int nb = nb_of(k), npan = (nb + 31) / 32;
            const int pb = (int)(k & 1);
            if (k > 0) {  // batch k's phase A; batches the chain completes meanwhile are published
                const uint64_t t0 = global_ns();
                for (unsigned it = 1; ld_acquire_u64(&scr.bar->a_done) < (unsigned long long)k * nA;
                     it++) {
                    publish_upto(ld_acquire_cta(prog) / NS);
                    if ((it & 63u) == 0) {
                        if (ld_acquire_int(err) != 0) {
                            ok = false;
                            break;
                        }
                        if (global_ns() - t0 > 2000000000ull) {
                            set_err(err, DEV_TIMEOUT);
                            ok = false;
                            break;
                        }
                    }
                }
                if (!ok) break;
            }
            // the step constants' buffer was last read by batch k - 2
            if (k >= 2) {
                const int v = wait_flag(prog, (int)((k - 1) * NS), err, 64);
                if (v < 0) break;
                publish_upto(v / NS);
            }
            fence_proxy_async();
            mbar_expect_tx(&mbpre[pb], (uint32_t)(PRE_N * B * sizeof(T)));
            bulk_load(spre + (size_t)pb * PRE_N * B, preb + (size_t)pb * PRE_N * B,
                      (uint32_t)(PRE_N * B * sizeof(T)), &mbpre[pb]);
            npre[pb]++;
            const T *gcoef = coefb + (size_t)pb * coef_slots(B);
            for (int s = 0; s < npan; s++) {
                // the panel that last occupied this buffer: number k NS + s - NBUF
                const int64_t prev = k * NS + s - NBUF;
                if (prev >= 0) {
                    const int v = wait_flag(prog, (int)prev + 1, err, 64);
                    if (v < 0) {
                        ok = false;
                        break;
                    }
                    publish_upto(v / NS);
                }
                fence_proxy_async();
                issue_panel<T, NS>(s, gcoef, scoef, mb);
                nuse[s % NBUF]++;
            }
            if (ok && k >= 1) {  // batch k - 1 (whose last panels a short batch k skips)
                const int v = wait_flag(prog, (int)(k * NS), err, 64);
                if (v < 0) break;
                publish_upto(v / NS);
            }
        }
        if (ok) {  // the last batch's steps
            const int last = (int)((nbatch - 1) * NS) + (nb_of(nbatch - 1) + 31) / 32;
            if (wait_flag(prog, last, err, 64) >= 0) publish_upto(nbatch);
        }
        // the copies still in flight land before the CTA may leave (bounded)
        for (int b = 0; b < NBUF; b++)
            if (nuse[b] > 0) mbar_wait(&mb[b], (uint32_t)(nuse[b] - 1) & 1u, err, false);
        for (int b = 0; b < 2; b++)
            if (npre[b] > 0) mbar_wait(&mbpre[b], (uint32_t)(npre[b] - 1) & 1u, err, false);
        return;
    }

    // ---- the corrections: warps 1 .. kWarps - 2 ----
    constexpr int NW = kWarps - 2;
    constexpr int RW = (32 + NW - 1) / NW;  // rows of a panel per warp
    const int w = warp - 1;
    __shared__ int s_ok1, s_ok2;
    for (int64_t k = 1; k < nbatch; k++) {
        const int nb = nb_of(k), nbp = nb_of(k - 1);
        const T *X = gX + (size_t)(k & 1) * B * B;
        // X(k, k-1) is complete with the other CTAs' phase A of batch k
        if (threadIdx.x == 32) s_ok1 = wait_counter(&scr.bar->a_done, (unsigned long long)k * nA, err);
        bar_sync_n(kBarCorr, NW * 32);
        if (!s_ok1) return;
        T x[RW][NS];
        auto load_panel = [&](int s) {
#pragma unroll
            for (int r = 0; r < RW; r++) {
                const int l = s * 32 + w + NW * r;
#pragma unroll
                for (int kk = 0; kk < NS; kk++) {
                    const int l1 = lane + 32 * kk;
                    x[r][kk] = (w + NW * r < 32 && l < nb && l1 < nbp)
                                   ? __ldcg(X + (size_t)l * B + l1) : T(0);
                }
            }
        };
        load_panel(0);
        // batch k - 1's steps are all in shared memory
        if (threadIdx.x == 32) s_ok2 = wait_flag(prog, (int)(k * NS), err, 32) >= 0;
        bar_sync_n(kBarCorr, NW * 32);
        if (!s_ok2) return;
        T muv[NS];
        const double *mu_s = smu + (size_t)((k - 1) & 1) * B;
#pragma unroll
        for (int kk = 0; kk < NS; kk++) {
            const int l1 = lane + 32 * kk;
            muv[kk] = l1 < nbp ? (T)mu_s[l1] : T(0);
        }
        for (int s = 0; s * 32 < nb; s++) {
            if (s > 0) load_panel(s);
#pragma unroll
            for (int r = 0; r < RW; r++) {
                const int l = s * 32 + w + NW * r;
                T a = T(0);
#pragma unroll
                for (int kk = 0; kk < NS; kk++) a = fma(x[r][kk], muv[kk], a);
                a = warp_sum(a);
                if (lane == 0 && w + NW * r < 32) scorr[l] = a;
            }
            bar_sync_n(kBarCorr, NW * 32);  // the panel's rows are all written
            if (threadIdx.x == 32) st_release_cta(corr_prog, (int)(k * NS) + s + 1);
        }
    }
}

// 16-byte vector of the cache type
template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static const int n = 4; };
template <> struct V16<double> { using type = double2; static const int n = 2; };

__device__ __forceinline__ float vget(const float4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2 &v, int k) { return k == 0 ? v.x : v.y; }

// Per-warp sums of ND per-thread values of the dot warps, written to red[warp][d] (shared);
// after their barrier, cta_total(red, d) adds the warps' sums in the cache type, in a fixed
// order.
template <typename T, int ND>
__device__ __forceinline__ void warp_partials(const T (&v)[ND], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; d++) {
        const T w = warp_sum(v[d]);
        if (lane == 0) red[warp * ND + d] = (double)w;
    }
}

template <typename T, int ND>
__device__ __forceinline__ T cta_total(const double *red, int d) {
    T s[kDotWarps];
#pragma unroll
    for (int w = 0; w < kDotWarps; w++) s[w] = (T)red[w * ND + d];
#pragma unroll
    for (int h = kDotWarps / 2; h > 0; h /= 2)  // pairwise
#pragma unroll
        for (int w = 0; w < h; w++) s[w] += s[w + h];
    return s[0];
}

// ---------------------------------------------------------------------------------
// Phase A dot products from shared memory.  The rows that one CTA's dot products read
// (kRingRows at most) are brought into shared memory in column chunks by bulk copies, as
// many chunks ahead as the ring holds (120 KB in flight per SM), rather than the few loads
// per thread its warps would have outstanding.
// ---------------------------------------------------------------------------------

template <typename T, int ND>
struct DotPlan {
    const T *rows[kRingRows];  // row bases, 16-byte aligned (read by thread 0)
    int nrows;
    int ia[ND], ib[ND];        // dot product d = rows[ia[d]] . rows[ib[d]]
};

// Per-thread partial sums acc[d] of the plan's dot products over columns [0, len), with
// len * sizeof(T) a multiple of 16.  The kDotThreads threads of the dot warps call it.  A
// copy that does not land within the wait limit makes them all give up (false, err set),
// after thread 0 has waited, again with a limit, for the copies it still has in flight.
template <typename T, int ND>
__device__ bool ring_dots(const DotPlan<T, ND> &pl, int64_t len, T (&acc)[ND],
                          unsigned char *ring, uint64_t *mb, uint32_t &phase, int *err) {
    constexpr int CW = kChunkBytes / (int)sizeof(T);
    using VT = typename V16<T>::type;
    constexpr int VN = V16<T>::n;
    const int64_t nch = (len + CW - 1) / CW;
    // stages of pl.nrows chunks that the ring holds
    int nst = (int)(kRingBytes / ((size_t)pl.nrows * kChunkBytes));
    nst = nst > kMaxStages ? kMaxStages : nst;
    const size_t stage_bytes = (size_t)pl.nrows * kChunkBytes;
    int64_t issued = 0;  // chunks issued (thread 0)
    auto issue = [&](int64_t c) {
        const int st = (int)(c % nst);
        const int64_t c0 = c * CW;
        const int64_t n = (len - c0) < CW ? (len - c0) : CW;
        const uint32_t bytes = (uint32_t)(n * (int64_t)sizeof(T));
        T *dst = reinterpret_cast<T *>(ring + (size_t)st * stage_bytes);
        mbar_expect_tx(&mb[st], bytes * (uint32_t)pl.nrows);
        for (int r = 0; r < pl.nrows; r++)
            bulk_load(dst + (size_t)r * CW, pl.rows[r] + c0, bytes, &mb[st]);
    };
    int oa[ND], ob[ND];  // the operands' offsets in a stage, in 16-byte words
#pragma unroll
    for (int d = 0; d < ND; d++) {
        acc[d] = T(0);
        oa[d] = pl.ia[d] * (CW / VN);
        ob[d] = pl.ib[d] * (CW / VN);
    }
    if (threadIdx.x == 0) {
        // the ring was last read (and the rows possibly written) through the generic proxy
        fence_proxy_async();
        for (; issued < nch && issued < nst; issued++) issue(issued);
    }
    for (int64_t c = 0; c < nch; c++) {
        const int st = (int)(c % nst);
        const bool ok = mbar_wait(&mb[st], (phase >> st) & 1u, err);
        if (ok) {
            phase ^= 1u << st;
            const VT *src = reinterpret_cast<const VT *>(ring + (size_t)st * stage_bytes);
            const int64_t c0 = c * CW;
            const int nv = (int)(((len - c0) < CW ? (len - c0) : CW) / VN);
            for (int v = threadIdx.x; v < nv; v += kDotThreads) {
#pragma unroll
                for (int d = 0; d < ND; d++) {
                    const VT x = src[oa[d] + v];
                    const VT y = src[ob[d] + v];
#pragma unroll
                    for (int k = 0; k < VN; k++) acc[d] = fma(vget(x, k), vget(y, k), acc[d]);
                }
            }
        }
        if (!bar_and_n(kBarDots, kDotThreads, ok)) {
            if (threadIdx.x == 0)
                for (int64_t c2 = ok ? c + 1 : c; c2 < issued; c2++) {
                    const int s2 = (int)(c2 % nst);
                    if (!mbar_wait(&mb[s2], (phase >> s2) & 1u, err, false)) break;
                    phase ^= 1u << s2;
                }
            bar_sync_n(kBarDots, kDotThreads);
            return false;
        }
        if (threadIdx.x == 0 && issued < nch) {  // stage st is free again
            fence_proxy_async();
            issue(issued);
            issued++;
        }
    }
    return true;
}

template <typename T>
__device__ __forceinline__ bool aligned16(const T *p) {
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// The coordinates of a batch [s, s + nb) in registers (at most two per thread: B <= 512),
// fetched ahead of the point where they are stored, so that the load latency overlaps other
// work (the wait of a grid barrier).
struct BatchRegs {
    int32_t a[2], b[2];
};
static_assert(2 * kThreads >= 512, "BatchRegs holds two coordinates per thread");

__device__ __forceinline__ void fetch_batch(const int32_t *__restrict__ ai,
                                            const int32_t *__restrict__ aj, int64_t s, int nb,
                                            BatchRegs &r) {
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int l = threadIdx.x + u * kThreads;
        r.a[u] = l < nb ? __ldg(ai + s + l) : 0;
        r.b[u] = l < nb ? __ldg(aj + s + l) : 0;
    }
}

// Store a fetched batch into shared memory and find its segments (maximal runs of
// coordinates with the same first index; the lists are row-major, so a segment is the part
// of one row of the active set that falls in the batch).
__device__ void store_batch(const BatchRegs &r, int nb, int32_t *sa, int32_t *sb, int32_t *sseg,
                            int32_t *snseg) {
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int l = threadIdx.x + u * kThreads;
        if (l < nb) {
            sa[l] = r.a[u];
            sb[l] = r.b[u];
        }
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
struct BatchMeta {
    int32_t *sa, *sb, *sseg, *snseg;
};

__device__ __forceinline__ BatchMeta meta_at(unsigned char *base, int B, int which) {
    int32_t *p = reinterpret_cast<int32_t *>(base) + which * (3 * B + 2);
    return BatchMeta{p, p + B, p + 2 * B, p + 3 * B + 1};
}

// The pass on a group of nblk CTAs of a cooperative launch, this CTA being number bid of
// the group (the whole grid for a single pass; a part of it when several passes share one
// launch).  Every reduction is done by one CTA or one warp in a fixed order, so the result
// does not depend on nblk.
template <typename T, int NS>
__device__ __forceinline__ void
lambda_pass(int64_t q, const T *__restrict__ Sig, const T *__restrict__ Psi,
            const double *__restrict__ Sd, const double *__restrict__ Pd,
            const double *__restrict__ G, const double *__restrict__ Lam, int64_t m,
            const int32_t *__restrict__ ai, const int32_t *__restrict__ aj, double lam_off,
            double lam_diag, double *D, T *Ut, int B_arg, SweepScratch scr, unsigned bid,
            unsigned nblk) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[kWarps * 6];
    __shared__ StepHead<T> s_head[2];  // the scalar part of the two coordinates' constants
    __shared__ uint64_t s_mb[NS + 2];  // phase B (CTA 0): panel buffers, two step-constant buffers
    __shared__ uint64_t s_ring[kMaxStages];  // phase A ring
    uint32_t ring_phase = 0;
    unsigned bar_round = 0;  // grid barriers passed (every CTA of the group passes the same)
    constexpr int B = NS * 32;
    if (B_arg != B) return;  // the host launches the instance of its batch size
    const SmemLayout L = smem_layout<T>(B);
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *preb = reinterpret_cast<T *>(scr.sub1);                // [2][PRE_N][B]
    T *coefb = reinterpret_cast<T *>(scr.sub2);               // [2][coef_slots(B)]
    T *gX = coefb + 2 * (size_t)coef_slots(B);                // [2][B][B] cross coefficients
    // phase C: CTAs 1 .. nblk - 1 share the q rows of the cache; CTA 0 holds none
    const int64_t nC = (int64_t)nblk - 1;
    const int64_t rows_per = (q + nC - 1) / nC;
    const int64_t r0 = bid >= 1 ? (int64_t)(bid - 1) * rows_per : 0;
    const int64_t r1 = bid >= 1 ? ((r0 + rows_per) < q ? (r0 + rows_per) : q) : 0;
    // phase A reads rows through the ring when bulk copies can address them
    const bool use_ring = ((q * (int64_t)sizeof(T)) % 16) == 0 && aligned16(Sig) &&
                          aligned16(Psi) && aligned16(Ut);
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
                       int nbp, T *Xo, int rank0) {
        const int nA = (int)nblk - rank0, rank = (int)bid - rank0;
        // the coefficient warps' thread index and count over the group's phase-A CTAs
        const int64_t t0 = (int64_t)rank * kCoefThreads + ((int)threadIdx.x - kDotThreads);
        const int64_t nt = (int64_t)nA * kCoefThreads;
        // The coefficients depend on entries of Sigma and Psi only, not on the dot products:
        // the coefficient warps form them while the dot warps compute the dot products.
        auto coef_work = [&]() {
            for (int64_t e = t0; e < (int64_t)(B - nb) * PRE_N; e += nt) {  // padding coordinates
                const int k = (int)(e / (B - nb)), l = nb + (int)(e % (B - nb));
                pre[k * B + l] = T(0);
            }
            const int ncoef = nb * (nb - 1) / 2;
#pragma unroll 2
            for (int64_t e = t0; e < ncoef; e += nt) {
                int l, l1;
                decode_pair((int)e, l, l1);
                coef[colbase(l1, B) + (l - l1 - 1)] =
                    coefficient(bm.sa[l], bm.sb[l], bm.sa[l1], bm.sb[l1]);
            }
            if (prev) {
                const int64_t ncross = (int64_t)nb * nbp;
#pragma unroll 4
                for (int64_t e = t0; e < ncross; e += nt) {
                    const int l = (int)(e / nbp), l1 = (int)(e % nbp);
                    Xo[(size_t)l * B + l1] =
                        coefficient(bm.sa[l], bm.sb[l], prev->sa[l1], prev->sb[l1]);
                }
            }
        };
        if (threadIdx.x >= kDotThreads) {
            coef_work();
            return;
        }
        for (int l = rank; l < nb; l += 2 * nA) {
            const int lb = l + nA;
            const bool two = lb < nb;
            const int64_t i0 = bm.sa[l], j0 = bm.sb[l];
            const int64_t i1 = two ? bm.sa[lb] : i0, j1 = two ? bm.sb[lb] : j0;
            // thread 0 finishes coordinate l, thread 32 coordinate lb; the scalars they need
            // are loaded first, so that their latency hides behind the dot products
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            const int64_t ii = which == 1 ? i1 : i0, jj = which == 1 ? j1 : j0;
            if (which >= 0) {
                const double sij = (double)Sig[ii * q + jj], pij = (double)Psi[ii * q + jj];
                const double sdi = Sd[ii], sdj = Sd[jj], pdi = Pd[ii], pdj = Pd[jj];
                // curvature of the exact quadratic model along the coordinate (Appendix A.1
                // with the E1/E5 readings) and the constants' scalar part, ahead of the dots
                const double a = (ii != jj)
                                     ? sij * sij + sdi * sdj + sdi * pdj + sdj * pdi + 2.0 * sij * pij
                                     : sdi * sdi + 2.0 * sdi * pdi;
                // stored before the dot products (the ring's waits order it): the double
                // operations then run while the data is in flight, not after it
                s_head[which] = step_head<T>(G[ii * q + jj], a, (ii != jj) ? lam_off : lam_diag,
                                             Lam[ii * q + jj]);
            }
            // (Sigma D Sigma)_ij = Sigma_i . U_{:,j}, (Psi D Sigma)_ij = Psi_i . U_{:,j},
            // (Psi D Sigma)_ji = Psi_j . U_{:,i}; rows 0..4 serve coordinate l, and the
            // second coordinate shares rows 0..2 when it lies in the same row of Lambda
            DotPlan<T, 6> pl;
            pl.rows[0] = Sig + i0 * q;
            pl.rows[1] = Psi + i0 * q;
            pl.rows[2] = Ut + i0 * q;
            pl.rows[3] = Psi + j0 * q;
            pl.rows[4] = Ut + j0 * q;
            pl.ia[0] = 0; pl.ib[0] = 4;
            pl.ia[1] = 1; pl.ib[1] = 4;
            pl.ia[2] = 3; pl.ib[2] = 2;
            if (!two) {
                pl.nrows = 5;
                pl.ia[3] = 0; pl.ib[3] = 4;
                pl.ia[4] = 1; pl.ib[4] = 4;
                pl.ia[5] = 3; pl.ib[5] = 2;
            } else if (i1 == i0) {
                pl.nrows = 7;
                pl.rows[5] = Psi + j1 * q;
                pl.rows[6] = Ut + j1 * q;
                pl.ia[3] = 0; pl.ib[3] = 6;
                pl.ia[4] = 1; pl.ib[4] = 6;
                pl.ia[5] = 5; pl.ib[5] = 2;
            } else {
                pl.nrows = 10;
                pl.rows[5] = Sig + i1 * q;
                pl.rows[6] = Psi + i1 * q;
                pl.rows[7] = Ut + i1 * q;
                pl.rows[8] = Psi + j1 * q;
                pl.rows[9] = Ut + j1 * q;
                pl.ia[3] = 5; pl.ib[3] = 9;
                pl.ia[4] = 6; pl.ib[4] = 9;
                pl.ia[5] = 8; pl.ib[5] = 7;
            }
            T acc[6];
            if (use_ring) {
                if (!ring_dots<T, 6>(pl, q, acc, work, s_ring, ring_phase, scr.err)) return;
            } else {
#pragma unroll
                for (int d = 0; d < 6; d++) acc[d] = T(0);
                for (int64_t t = threadIdx.x; t < q; t += kDotThreads) {
                    T x[kRingRows];
                    for (int r = 0; r < pl.nrows; r++) x[r] = __ldcg(pl.rows[r] + t);
#pragma unroll
                    for (int d = 0; d < 6; d++) acc[d] = fma(x[pl.ia[d]], x[pl.ib[d]], acc[d]);
                }
            }
            warp_partials<T, 6>(acc, s_red);
            bar_sync_n(kBarDots, kDotThreads);
            if (which >= 0) {
                const int lw = which ? lb : l;
                const T d0 = cta_total<T, 6>(s_red, 3 * which);
                const T d1 = cta_total<T, 6>(s_red, 3 * which + 1);
                const T d2 = cta_total<T, 6>(s_red, 3 * which + 2);
                step_constants<T>(s_head[which], (ii != jj) ? d0 + (d1 + d2) : d0 + T(2) * d1,
                                  pre, B, lw);
            }
            bar_sync_n(kBarDots, kDotThreads);  // s_red read before the next pair writes it
        }
    };

    // Batches are pipelined two deep.  CTA 0 runs the steps (phase B) of batch k while CTAs
    // 1 .. nblk - 1 apply batch k - 1's steps to the cache (phase C) and then compute the dot
    // products and coefficients of batch k + 1 (phase A) against the cache as it stands
    // after batch k - 1: their missing part, batch k's own steps, is carried into batch k + 1
    // by the cross coefficients X(k + 1, k), which CTA 0's other warps apply during phase B of
    // batch k + 1.  Counters order the two sides: CTA 0 publishes each batch's steps
    // (mu_ready) and waits for the phase A of the batch it is about to run (a_done); the
    // other CTAs wait for a batch's steps and for the end of every CTA's phase A of the next
    // batch (which reads the cache rows phase C writes) before phase C, and for the end of
    // every CTA's phase C (c_done) before the next phase A.
    auto nb_of = [&](int64_t k) -> int {
        const int64_t s0 = k * B;
        return s0 < m ? (int)((m - s0) < B ? (m - s0) : B) : 0;
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < kMaxStages; k++) mbar_init(&s_ring[k], 1);
        mbar_init_fence();
    }
    auto slot = [&](int64_t k) -> BatchMeta { return meta_at(smem + L.meta, B, (int)(k % 3)); };
    const int nb0 = nb_of(0);
    BatchRegs breg;  // indices of a batch, fetched ahead of storing them
    fetch_batch(ai, aj, 0, nb0, breg);
    const BatchMeta s0m = slot(0);
    store_batch(breg, nb0, s0m.sa, s0m.sb, s0m.sseg, s0m.snseg);
    // prologue: phase A of batch 0 by every CTA; nothing carried into it
    phase_a(s0m, nb0, preb, coefb, nullptr, 0, gX, 0);
    __shared__ int s_prog, s_corr_prog;  // CTA 0: phase B's progress flags
    if (bid == 0 && threadIdx.x == 0) {
        for (int k = 0; k < NS + 2; k++) mbar_init(&s_mb[k], 1);
        mbar_init_fence();
        s_prog = 0;
        s_corr_prog = 0;
    }
    if (!grid_sync(scr.bar, scr.err, nblk, bar_round)) return;
    const unsigned long long nA = nblk - 1;

    if (bid == 0) {  // ---- phase B of every batch ----
        phase_b_cta0<T, NS>(nbatch, m, preb, coefb, gX, nA, work, s_mb, s_mb + NS, &s_prog,
                            &s_corr_prog, scr);
        return;
    }

    // ---- CTAs 1 .. nblk - 1: phase C of batch k, then phase A of batch k + 2 ----
    if (nbatch > 1) {
        const int nb1 = nb_of(1);
        fetch_batch(ai, aj, B, nb1, breg);
        const BatchMeta s1m = slot(1);
        store_batch(breg, nb1, s1m.sa, s1m.sb, s1m.sseg, s1m.snseg);
        phase_a(s1m, nb1, preb + PRE_N * B, coefb + coef_slots(B), &s0m, nb0,
                gX + (size_t)B * B, 1);
        __syncthreads();
        cta_count(&scr.bar->a_done);
    }
    for (int64_t k = 0; k < nbatch; k++) {
        const int nbk = nb_of(k), nbn = nb_of(k + 1), nb2 = nb_of(k + 2);
        const BatchMeta cur = slot(k);
        // Phase C's first reads (segment 0, this warp's first R rows) do not depend on the
        // steps: they are issued before the wait for them, so that their latency overlaps it.
        constexpr int R = NS <= 8 ? kRowsInFlight : 2;  // registers: R x NS values per lane
        T sta[R], sv[R][NS], uv[R][NS], ua[R];
        int bv[NS];
        auto seg_columns = [&](int g) {
            const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
#pragma unroll
            for (int kk = 0; kk < NS; kk++) {
                const int l = l0 + lane + 32 * kk;
                bv[kk] = (l < l1) ? cur.sb[l] : -1;
            }
        };
        auto load_rows = [&](int a, int64_t tb) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int64_t t = tb + (int64_t)kWarps * r;
                sta[r] = T(0);
                ua[r] = T(0);
#pragma unroll
                for (int kk = 0; kk < NS; kk++) sv[r][kk] = uv[r][kk] = T(0);
                if (t < r1) {
                    const T *Sr = Sig + t * q;
                    const T *Ur = Ut + t * q;
                    sta[r] = Sr[a];
                    // U^T[t][a] is written at the end of this row's update only (the segment's
                    // other columns b != a), so it is read here with the rest
                    if (lane == 0) ua[r] = __ldcg(Ur + a);
#pragma unroll
                    for (int kk = 0; kk < NS; kk++) {
                        if (bv[kk] >= 0) {
                            sv[r][kk] = Sr[bv[kk]];
                            if (bv[kk] != a) uv[r][kk] = __ldcg(Ur + bv[kk]);
                        }
                    }
                }
            }
        };
        seg_columns(0);
        load_rows(cur.sa[cur.sseg[0]], r0 + warp);
        // batch k's steps, and every CTA's phase A of batch k + 1 (it reads the cache rows
        // this phase C writes)
        if (!cta_wait_counts(&scr.bar->mu_ready, (unsigned long long)k + 1,
                             nbn > 0 ? &scr.bar->a_done : nullptr,
                             (unsigned long long)(k + 1) * nA, scr.err))
            return;

        // ---- phase C: batch k's update on this CTA's rows ----
        // coordinate (a, b) of a segment with row a: U_a += mu Sigma_b, U_b += mu Sigma_a
        // (b != a); transposed: Ut[t][a] += sum mu Sigma[t][b], Ut[t][b] += mu Sigma[t][a]
        {
            T *smu = reinterpret_cast<T *>(work + L.phc);
            const double *muk = scr.mu + (size_t)(k & 1) * B;
            for (int l = threadIdx.x; l < nbk; l += blockDim.x) {
                const double mu = __ldcg(muk + l);
                smu[l] = (T)mu;
                if (bid == nblk - 1) {  // the direction itself
                    const int64_t i = cur.sa[l], j = cur.sb[l];
                    D[i * q + j] = mu;
                    if (i != j) D[j * q + i] = mu;
                }
            }
            __syncthreads();
            const int nseg = *cur.snseg;
            for (int g = 0; g < nseg; g++) {
                const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
                const int a = cur.sa[l0];
                if (g > 0) seg_columns(g);
                T mv[NS];
#pragma unroll
                for (int kk = 0; kk < NS; kk++) {
                    const int l = l0 + lane + 32 * kk;
                    mv[kk] = (l < l1) ? smu[l] : T(0);
                }
                for (int64_t tb = r0 + warp; tb < r1; tb += kWarps * R) {
                    if (g > 0 || tb != r0 + warp) load_rows(a, tb);  // else: loaded before the wait
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
                        if (lane == 0) Ur[a] = ua[r] + dot;
                    }
                }
                __syncwarp();  // this segment's writes before the next segment's reads
            }
        }
        __syncthreads();
        cta_count(&scr.bar->c_done);
        // the indices of batch k + 2 are fetched while the other CTAs finish their phase C
        if (nb2 > 0) {
            const BatchMeta s2 = slot(k + 2);
            fetch_batch(ai, aj, (k + 2) * B, nb2, breg);
            store_batch(breg, nb2, s2.sa, s2.sb, s2.sseg, s2.snseg);
        }
        if (!cta_wait_counts(&scr.bar->c_done, (unsigned long long)(k + 1) * nA, nullptr, 0,
                             scr.err))
            return;
        if (nb2 > 0) {  // ---- phase A of batch k + 2 ----
            const size_t par = (size_t)((k + 2) & 1);
            const BatchMeta prv = slot(k + 1);
            phase_a(slot(k + 2), nb2, preb + par * PRE_N * B, coefb + par * coef_slots(B), &prv,
                    nbn, gX + par * B * B, 1);
            __syncthreads();
            cta_count(&scr.bar->a_done);
        }
    }
}

// ---------------------------------------------------------------------------------
// Theta sweep kernel.  Cache: dVt = (Delta V)^T (q x p), dVt[j][t] = (Delta Theta Sigma)[t][j].
// Pipelined like the Lambda pass.
// ---------------------------------------------------------------------------------
// The pass on a group of nblk CTAs (see lambda_pass).
template <typename T, int NS>
__device__ __forceinline__ void
theta_pass(int64_t p, int64_t q, const T *__restrict__ Sxx, int64_t x0,
           const double *__restrict__ Xd, const T *__restrict__ Sig,
           const double *__restrict__ Sd, const double *__restrict__ W, double *Theta, int64_t m,
           const int32_t *__restrict__ ti, const int32_t *__restrict__ tj, double lam, T *dVt,
           int B_arg, SweepScratch scr, bool rows_sorted, unsigned bid, unsigned nblk) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_red[kWarps * 2];
    __shared__ StepHead<T> s_head[2];
    __shared__ uint64_t s_mb[NS + 2];  // phase B (CTA 0): panel buffers, two step-constant buffers
    __shared__ uint64_t s_ring[kMaxStages];  // phase A ring
    uint32_t ring_phase = 0;
    unsigned bar_round = 0;  // grid barriers passed (every CTA of the group passes the same)
    constexpr int B = NS * 32;
    if (B_arg != B) return;  // the host launches the instance of its batch size
    const SmemLayout L = smem_layout<T>(B);
    unsigned char *work = smem + L.work;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *preb = reinterpret_cast<T *>(scr.sub1);
    T *coefb = reinterpret_cast<T *>(scr.sub2);
    T *gX = coefb + 2 * (size_t)coef_slots(B);  // [2][B][B] cross coefficients
    // phase C: CTAs 1 .. nblk - 1 share the q rows of the cache; CTA 0 holds none
    const int64_t nC = (int64_t)nblk - 1;
    const int64_t rows_per = (q + nC - 1) / nC;
    const int64_t r0 = bid >= 1 ? (int64_t)(bid - 1) * rows_per : 0;
    const int64_t r1 = bid >= 1 ? ((r0 + rows_per) < q ? (r0 + rows_per) : q) : 0;
    constexpr int VN = V16<T>::n;
    const int64_t nbatch = (m + B - 1) / B;
    if (nbatch == 0) return;
    const bool use_ring = ((p * (int64_t)sizeof(T)) % 16) == 0 && aligned16(Sxx) && aligned16(dVt);

    // change of (S_xx Delta V)_ij per unit step of Theta_ab, times 2: 2 (S_xx)_{i a} Sigma_{j b}
    // (Sigma symmetric; read along row j, b varying fastest across threads).  Sxx holds the
    // rows x0, x0 + 1, ... of S_xx that this launch's coordinates lie in.
    auto coefficient = [&](int64_t i, int64_t j, int64_t a, int64_t b) -> T {
        return T(2) * Sxx[(i - x0) * p + a] * Sig[j * q + b];
    };

    auto phase_a = [&](const BatchMeta &bm, int nb, T *pre, T *coef, const BatchMeta *prev,
                       int nbp, T *Xo, int rank0) {
        const int nA = (int)nblk - rank0, rank = (int)bid - rank0;
        // rows of Delta V that can be nonzero: with the list in ascending rows, those at or
        // before this batch's first row (the ring copies whole 16-byte words: entries beyond
        // tmax are zero); all p rows otherwise
        const int64_t tmax = rows_sorted ? (int64_t)bm.sa[0] + 1 : p;
        const int64_t tlen = ((tmax + VN - 1) / VN) * VN < p ? ((tmax + VN - 1) / VN) * VN : p;
        // the coefficient warps' thread index and count over the group's phase-A CTAs
        const int64_t t0 = (int64_t)rank * kCoefThreads + ((int)threadIdx.x - kDotThreads);
        const int64_t nt = (int64_t)nA * kCoefThreads;
        // the coefficients (entries of S_xx and Sigma only) are formed by the coefficient
        // warps while the dot warps compute the dot products
        auto coef_work = [&]() {
            for (int64_t e = t0; e < (int64_t)(B - nb) * PRE_N; e += nt) {  // padding coordinates
                const int k = (int)(e / (B - nb)), l = nb + (int)(e % (B - nb));
                pre[k * B + l] = T(0);
            }
            const int ncoef = nb * (nb - 1) / 2;
#pragma unroll 2
            for (int64_t e = t0; e < ncoef; e += nt) {
                int l, l1;
                decode_pair((int)e, l, l1);
                coef[colbase(l1, B) + (l - l1 - 1)] =
                    coefficient(bm.sa[l], bm.sb[l], bm.sa[l1], bm.sb[l1]);
            }
            if (prev) {
                const int64_t ncross = (int64_t)nb * nbp;
#pragma unroll 4
                for (int64_t e = t0; e < ncross; e += nt) {
                    const int l = (int)(e / nbp), l1 = (int)(e % nbp);
                    Xo[(size_t)l * B + l1] =
                        coefficient(bm.sa[l], bm.sb[l], prev->sa[l1], prev->sb[l1]);
                }
            }
        };
        if (threadIdx.x >= kDotThreads) {
            coef_work();
            return;
        }
        for (int l = rank; l < nb; l += 2 * nA) {
            const int lb = l + nA;
            const bool two = lb < nb;
            const int64_t i0 = bm.sa[l], j0 = bm.sb[l];
            const int64_t i1 = two ? bm.sa[lb] : i0, j1 = two ? bm.sb[lb] : j0;
            // thread 0 finishes coordinate l, thread 32 coordinate lb; their scalars first
            const int which = threadIdx.x == 0 ? 0 : (threadIdx.x == 32 && two ? 1 : -1);
            const int64_t ii = which == 1 ? i1 : i0, jj = which == 1 ? j1 : j0;
            if (which >= 0) {
                const double xii = Xd[ii], sdj = Sd[jj];
                // curvature 2 Sigma_jj (S_xx)_ii (Appendix A.1 with the E2 reading), zero for a
                // constant input column, and the constants' scalar part ahead of the dots
                const double a = (xii != 0.0) ? 2.0 * sdj * xii : 0.0;
                s_head[which] = step_head<T>(2.0 * W[ii * q + jj], a, lam,
                                             __ldcg(Theta + ii * q + jj));
            }
            // (S_xx Delta V)_ij = (S_xx)_i . Delta V_{:,j}
            DotPlan<T, 2> pl;
            pl.rows[0] = Sxx + (i0 - x0) * p;
            pl.rows[1] = dVt + j0 * p;
            pl.ia[0] = 0; pl.ib[0] = 1;
            if (!two) {
                pl.nrows = 2;
                pl.ia[1] = 0; pl.ib[1] = 1;
            } else if (i1 == i0) {
                pl.nrows = 3;
                pl.rows[2] = dVt + j1 * p;
                pl.ia[1] = 0; pl.ib[1] = 2;
            } else {
                pl.nrows = 4;
                pl.rows[2] = Sxx + (i1 - x0) * p;
                pl.rows[3] = dVt + j1 * p;
                pl.ia[1] = 2; pl.ib[1] = 3;
            }
            T acc[2];
            if (use_ring) {
                if (!ring_dots<T, 2>(pl, tlen, acc, work, s_ring, ring_phase, scr.err)) return;
            } else {
                acc[0] = acc[1] = T(0);
                for (int64_t t = threadIdx.x; t < tmax; t += kDotThreads) {
                    T x[4];
                    for (int r = 0; r < pl.nrows; r++) x[r] = __ldcg(pl.rows[r] + t);
                    acc[0] = fma(x[pl.ia[0]], x[pl.ib[0]], acc[0]);
                    acc[1] = fma(x[pl.ia[1]], x[pl.ib[1]], acc[1]);
                }
            }
            warp_partials<T, 2>(acc, s_red);
            bar_sync_n(kBarDots, kDotThreads);
            if (which >= 0) {
                const int lw = which ? lb : l;
                step_constants<T>(s_head[which], T(2) * cta_total<T, 2>(s_red, which), pre, B,
                                  lw);
            }
            bar_sync_n(kBarDots, kDotThreads);  // s_red read before the next pair writes it
        }
    };

    // pipelined as the Lambda pass (see there)
    auto nb_of = [&](int64_t k) -> int {
        const int64_t s0 = k * B;
        return s0 < m ? (int)((m - s0) < B ? (m - s0) : B) : 0;
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < kMaxStages; k++) mbar_init(&s_ring[k], 1);
        mbar_init_fence();
    }
    auto slot = [&](int64_t k) -> BatchMeta { return meta_at(smem + L.meta, B, (int)(k % 3)); };
    const int nb0 = nb_of(0);
    BatchRegs breg;  // indices of a batch, fetched ahead of storing them
    fetch_batch(ti, tj, 0, nb0, breg);
    const BatchMeta s0m = slot(0);
    store_batch(breg, nb0, s0m.sa, s0m.sb, s0m.sseg, s0m.snseg);
    phase_a(s0m, nb0, preb, coefb, nullptr, 0, gX, 0);
    __shared__ int s_prog, s_corr_prog;  // CTA 0: phase B's progress flags
    if (bid == 0 && threadIdx.x == 0) {
        for (int k = 0; k < NS + 2; k++) mbar_init(&s_mb[k], 1);
        mbar_init_fence();
        s_prog = 0;
        s_corr_prog = 0;
    }
    if (!grid_sync(scr.bar, scr.err, nblk, bar_round)) return;
    const unsigned long long nA = nblk - 1;

    if (bid == 0) {  // ---- phase B of every batch ----
        phase_b_cta0<T, NS>(nbatch, m, preb, coefb, gX, nA, work, s_mb, s_mb + NS, &s_prog,
                            &s_corr_prog, scr);
        return;
    }

    // ---- CTAs 1 .. nblk - 1: phase C of batch k, then phase A of batch k + 2 ----
    if (nbatch > 1) {
        const int nb1 = nb_of(1);
        fetch_batch(ti, tj, B, nb1, breg);
        const BatchMeta s1m = slot(1);
        store_batch(breg, nb1, s1m.sa, s1m.sb, s1m.sseg, s1m.snseg);
        phase_a(s1m, nb1, preb + PRE_N * B, coefb + coef_slots(B), &s0m, nb0,
                gX + (size_t)B * B, 1);
        __syncthreads();
        cta_count(&scr.bar->a_done);
    }
    for (int64_t k = 0; k < nbatch; k++) {
        const int nbk = nb_of(k), nbn = nb_of(k + 1), nb2 = nb_of(k + 2);
        const BatchMeta cur = slot(k);
        // Phase C's first reads (segment 0, this warp's first R rows of Sigma) do not depend
        // on the steps: they are issued before the wait for them.
        constexpr int R = NS <= 8 ? kRowsInFlight : 2;  // registers: R x NS values per lane
        T sv[R][NS], va[R];
        int jv[NS];
        auto seg_columns = [&](int g) {
            const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
#pragma unroll
            for (int kk = 0; kk < NS; kk++) {
                const int l = l0 + lane + 32 * kk;
                jv[kk] = (l < l1) ? cur.sb[l] : -1;
            }
        };
        // Delta V^T[t][i] (the entry this segment adds to in row t) is read with the Sigma
        // entries, by the lane that writes it
        auto load_rows = [&](int64_t i, int64_t tb) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int64_t t = tb + (int64_t)kWarps * r;
#pragma unroll
                for (int kk = 0; kk < NS; kk++)
                    sv[r][kk] = (t < r1 && jv[kk] >= 0) ? Sig[t * q + jv[kk]] : T(0);
                va[r] = (t < r1 && lane == 0) ? __ldcg(dVt + t * p + i) : T(0);
            }
        };
        seg_columns(0);
        load_rows(cur.sa[cur.sseg[0]], r0 + warp);
        if (!cta_wait_counts(&scr.bar->mu_ready, (unsigned long long)k + 1,
                             nbn > 0 ? &scr.bar->a_done : nullptr,
                             (unsigned long long)(k + 1) * nA, scr.err))
            return;

        // ---- phase C: dVt[t][i] += sum over the segment of row i of mu Sigma[t][j] ----
        {
            T *smu = reinterpret_cast<T *>(work + L.phc);
            const double *muk = scr.mu + (size_t)(k & 1) * B;
            for (int l = threadIdx.x; l < nbk; l += blockDim.x) {
                const double mu = __ldcg(muk + l);
                smu[l] = (T)mu;
                if (bid == nblk - 1) {  // Theta itself
                    const int64_t i = cur.sa[l], j = cur.sb[l];
                    Theta[i * q + j] = __ldcg(Theta + i * q + j) + mu;
                }
            }
            __syncthreads();
            const int nseg = *cur.snseg;
            for (int g = 0; g < nseg; g++) {
                const int l0 = cur.sseg[g], l1 = cur.sseg[g + 1];
                const int i = cur.sa[l0];
                if (g > 0) seg_columns(g);
                T mv[NS];
#pragma unroll
                for (int kk = 0; kk < NS; kk++) {
                    const int l = l0 + lane + 32 * kk;
                    mv[kk] = (l < l1) ? smu[l] : T(0);
                }
                for (int64_t tb = r0 + warp; tb < r1; tb += kWarps * R) {
                    if (g > 0 || tb != r0 + warp) load_rows(i, tb);  // else: before the wait
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int64_t t = tb + (int64_t)kWarps * r;
                        if (t >= r1) break;  // warp-uniform
                        T dot = T(0);
#pragma unroll
                        for (int kk = 0; kk < NS; kk++) dot = fma(mv[kk], sv[r][kk], dot);
                        dot = warp_sum(dot);
                        if (lane == 0) dVt[t * p + i] = va[r] + dot;
                    }
                }
            }
        }
        __syncthreads();
        cta_count(&scr.bar->c_done);
        if (nb2 > 0) {  // fetched while the other CTAs finish their phase C
            const BatchMeta s2 = slot(k + 2);
            fetch_batch(ti, tj, (k + 2) * B, nb2, breg);
            store_batch(breg, nb2, s2.sa, s2.sb, s2.sseg, s2.snseg);
        }
        if (!cta_wait_counts(&scr.bar->c_done, (unsigned long long)(k + 1) * nA, nullptr, 0,
                             scr.err))
            return;
        if (nb2 > 0) {  // ---- phase A of batch k + 2 ----
            const size_t par = (size_t)((k + 2) & 1);
            const BatchMeta prv = slot(k + 1);
            phase_a(slot(k + 2), nb2, preb + par * PRE_N * B, coefb + par * coef_slots(B), &prv,
                    nbn, gX + par * B * B, 1);
            __syncthreads();
            cta_count(&scr.bar->a_done);
        }
    }
}

template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
lambda_sweep_kernel(int64_t q, const T *__restrict__ Sig, const T *__restrict__ Psi,
                    const double *__restrict__ Sd, const double *__restrict__ Pd,
                    const double *__restrict__ G, const double *__restrict__ Lam, int64_t m,
                    const int32_t *__restrict__ ai, const int32_t *__restrict__ aj,
                    double lam_off, double lam_diag, double *D, T *Ut, int B_arg,
                    SweepScratch scr) {
    lambda_pass<T, NS>(q, Sig, Psi, Sd, Pd, G, Lam, m, ai, aj, lam_off, lam_diag, D, Ut, B_arg,
                       scr, blockIdx.x, gridDim.x);
}

template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
theta_sweep_kernel(int64_t p, int64_t q, const T *__restrict__ Sxx, int64_t x0,
                   const double *__restrict__ Xd, const T *__restrict__ Sig,
                   const double *__restrict__ Sd, const double *__restrict__ W, double *Theta,
                   int64_t m, const int32_t *__restrict__ ti, const int32_t *__restrict__ tj,
                   double lam, T *dVt, int B_arg, SweepScratch scr, int rows_sorted) {
    theta_pass<T, NS>(p, q, Sxx, x0, Xd, Sig, Sd, W, Theta, m, ti, tj, lam, dVt, B_arg, scr,
                      rows_sorted != 0, blockIdx.x, gridDim.x);
}

// One pass of a multi-pass launch: its kind, its group of CTAs and its arguments.
template <typename T>
struct PassDesc {
    int kind;  // 0: Lambda pass, 1: Theta pass
    int rows_sorted;  // Theta pass: the list is in ascending rows
    unsigned cta0, ncta;
    int64_t p, q, m, x0;
    const T *Sig, *Psi, *Sxx;
    const double *Sd, *Pd, *G, *Lam, *Xd, *W;
    const int32_t *ia, *ja;
    double lam_off, lam_diag;  // Theta pass: lam_off is its lambda
    double *out;               // Lambda pass: D; Theta pass: Theta
    T *cache;                  // Lambda pass: U^T; Theta pass: Delta V^T
    SweepScratch scr;
};
constexpr int kMaxPassGroups = 8;
template <typename T>
struct MultiPass {
    int n;
    PassDesc<T> d[kMaxPassGroups];
};

template <typename T, int NS>
__global__ void __launch_bounds__(kThreads, 1)
multi_pass_kernel(const __grid_constant__ MultiPass<T> mp) {
    int g = 0;
    while (g + 1 < mp.n && blockIdx.x >= mp.d[g + 1].cta0) g++;
    const PassDesc<T> &d = mp.d[g];
    const unsigned bid = blockIdx.x - d.cta0;
    if (d.kind == 0)
        lambda_pass<T, NS>(d.q, d.Sig, d.Psi, d.Sd, d.Pd, d.G, d.Lam, d.m, d.ia, d.ja, d.lam_off,
                           d.lam_diag, d.out, d.cache, NS * 32, d.scr, bid, d.ncta);
    else
        theta_pass<T, NS>(d.p, d.q, d.Sxx, d.x0, d.Xd, d.Sig, d.Sd, d.W, d.out, d.m, d.ia, d.ja,
                          d.lam_off, d.cache, NS * 32, d.scr, d.rows_sorted != 0, bid, d.ncta);
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
    if (h == DEV_BADINDEX) return CGGM_EINVAL;
    if (h != 0) return CGGM_ECUDA;
    return CGGM_OK;
}
}  // namespace

int sweep_grid() { return sm_count(); }

// ---------------------------------------------------------------------------------
// Pass batcher: the coordinate passes of concurrent solves in one cooperative launch.
// ---------------------------------------------------------------------------------
struct PassBatcher {
    struct Entry {
        bool f32;
        int B;
        PassDesc<float> df;
        PassDesc<double> dd;
        cudaStream_t st;
        cudaEvent_t ready;  // the submitting stream's work before the pass
        cggm_status status = CGGM_OK;
        bool done = false;
    };
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Entry *> pending;
    bool leader = false;
    int busy = 0;
    int device = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    int64_t n_launch = 0, n_pass = 0, n_shared = 0;
};

PassBatcher *batcher_create() { return new PassBatcher(); }

void batcher_destroy(PassBatcher *b) {
    if (!b) return;
    if (b->stream) {
        cudaSetDevice(b->device);
        cudaStreamSynchronize(b->stream);
        cudaEventDestroy(b->done_ev);
        cudaStreamDestroy(b->stream);
    }
    delete b;
}

void batcher_add_busy(PassBatcher *b, int delta) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->busy += delta;
    b->cv.notify_all();
}

void batcher_counts(PassBatcher *b, int64_t *launches, int64_t *passes, int64_t *shared) {
    std::lock_guard<std::mutex> lk(b->mu);
    if (launches) *launches = b->n_launch;
    if (passes) *passes = b->n_pass;
    if (shared) *shared = b->n_shared;
}

namespace {

template <typename T, int NS>
cggm_status launch_multi(PassBatcher &b, std::vector<PassBatcher::Entry *> &batch) {
    MultiPass<T> mp;
    mp.n = (int)batch.size();
    const int grid = sweep_grid();
    const int per = grid / mp.n, rem = grid % mp.n;
    if (per < 2) return CGGM_ECUDA;  // each pass needs two CTAs at least
    unsigned c0 = 0;
    for (int g = 0; g < mp.n; g++) {
        PassDesc<T> d;
        if constexpr (sizeof(T) == 4) d = batch[g]->df;
        else d = batch[g]->dd;
        d.cta0 = c0;
        d.ncta = (unsigned)(per + (g < rem ? 1 : 0));
        c0 += d.ncta;
        mp.d[g] = d;
    }
    const size_t smem = smem_layout<T>(NS * 32).total;
    const void *fn = (const void *)multi_pass_kernel<T, NS>;
    CGGM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    void *args[] = {(void *)&mp};
    for (PassBatcher::Entry *e : batch) CGGM_CUDA_TRY(cudaStreamWaitEvent(b.stream, e->ready, 0));
    {
        std::lock_guard<std::mutex> lock(coop_mutex());
        note_launch();
        CGGM_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(c0), dim3(kThreads), args, smem,
                                                  b.stream));
        CGGM_CUDA_TRY(cudaEventRecord(b.done_ev, b.stream));
        CGGM_CUDA_TRY(cudaEventSynchronize(b.done_ev));
    }
    for (PassBatcher::Entry *e : batch) CGGM_CUDA_TRY(cudaStreamWaitEvent(e->st, b.done_ev, 0));
    return CGGM_OK;
}

cggm_status launch_batch(PassBatcher &b, std::vector<PassBatcher::Entry *> &batch) {
    if (!b.stream) {
        CGGM_CUDA_TRY(cudaGetDevice(&b.device));
        CGGM_CUDA_TRY(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
        CGGM_CUDA_TRY(cudaEventCreateWithFlags(&b.done_ev, cudaEventDisableTiming));
    }
    const bool f32 = batch[0]->f32;
    switch (batch[0]->B) {
        case 32: return f32 ? launch_multi<float, 1>(b, batch) : launch_multi<double, 1>(b, batch);
        case 64: return f32 ? launch_multi<float, 2>(b, batch) : launch_multi<double, 2>(b, batch);
        case 128: return f32 ? launch_multi<float, 4>(b, batch) : launch_multi<double, 4>(b, batch);
        case 256: return f32 ? launch_multi<float, 8>(b, batch) : CGGM_EINVAL;
        case 512: return f32 ? launch_multi<float, 16>(b, batch) : CGGM_EINVAL;
        default: return CGGM_EINVAL;
    }
}

// Hand one pass to the batcher and return once it has run (its error word is then read by
// the caller).  The first thread to find no launch being prepared gathers: it waits until
// every busy solve has a pass waiting or 200 us have passed, takes the oldest pass and up to
// seven more of the same precision and batch size, and launches them together.
cggm_status run_batched(PassBatcher &b, PassBatcher::Entry &e) {
    CGGM_CUDA_TRY(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
    cudaError_t re = cudaEventRecord(e.ready, e.st);
    if (re != cudaSuccess) {
        cudaEventDestroy(e.ready);
        CGGM_CUDA_TRY(re);
    }
    std::unique_lock<std::mutex> lk(b.mu);
    b.pending.push_back(&e);
    b.cv.notify_all();
    while (!e.done) {
        if (b.leader) {
            b.cv.wait(lk);
            continue;
        }
        b.leader = true;
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(200);
        while ((int)b.pending.size() < b.busy && std::chrono::steady_clock::now() < deadline)
            b.cv.wait_until(lk, deadline);
        std::vector<PassBatcher::Entry *> batch;
        const PassBatcher::Entry *first = b.pending.front();
        for (auto it = b.pending.begin(); it != b.pending.end() && (int)batch.size() < kMaxPassGroups;) {
            if ((*it)->f32 == first->f32 && (*it)->B == first->B) {
                batch.push_back(*it);
                it = b.pending.erase(it);
            } else {
                ++it;
            }
        }
        lk.unlock();
        const cggm_status st = launch_batch(b, batch);
        lk.lock();
        b.n_launch++;
        b.n_pass += (int64_t)batch.size();
        if (batch.size() > 1) b.n_shared++;
        for (PassBatcher::Entry *x : batch) {
            x->status = st;
            x->done = true;
        }
        b.leader = false;
        b.cv.notify_all();
    }
    lk.unlock();
    cudaEventDestroy(e.ready);
    return e.status;
}

template <typename T>
PassDesc<T> &desc_of(PassBatcher::Entry &e);
template <>
PassDesc<float> &desc_of<float>(PassBatcher::Entry &e) { return e.df; }
template <>
PassDesc<double> &desc_of<double>(PassBatcher::Entry &e) { return e.dd; }

}  // namespace

cggm_status scratch_reserve(SweepScratch &scr) {
    if (scr.mu) return CGGM_OK;
    const int Bmax = 512;  // float; double batches are at most 128 and take less
    CGGM_CUDA_TRY(cudaMalloc(&scr.mu, sizeof(double) * 2 * Bmax));
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
    if (B < 32 || B > (sizeof(T) == 4 ? 512 : 128) || (B & (B - 1))) return CGGM_EINVAL;
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
        case 512: fn = (const void *)lambda_sweep_kernel<float, 16>; break;
        default: return CGGM_EINVAL;
    }
    if (scr.batcher) {
        PassBatcher::Entry e;
        e.f32 = sizeof(T) == 4;
        e.B = B;
        e.st = st;
        PassDesc<T> &d = desc_of<T>(e);
        d = PassDesc<T>{};
        d.kind = 0;
        d.q = q; d.m = m;
        d.Sig = Sigma; d.Psi = Psi; d.Sd = Sd; d.Pd = Pd; d.G = G; d.Lam = Lambda;
        d.ia = ai; d.ja = aj; d.lam_off = lam_off; d.lam_diag = lam_diag;
        d.out = D; d.cache = U; d.scr = scr;
        CGGM_TRY(run_batched(*scr.batcher, e));
        return read_err(scr.err, st);
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
cggm_status theta_sweep(int64_t p, int64_t q, const T *Sxx, int64_t x0, const double *Xd,
                        const T *Sigma, const double *Sd, const double *W, double *Theta,
                        int64_t m, const int32_t *ti, const int32_t *tj, double lam, T *dV,
                        int B, SweepScratch &scr, cudaStream_t st, bool rows_sorted) {
    if (m <= 0) return CGGM_OK;
    if (B < 32 || B > (sizeof(T) == 4 ? 512 : 128) || (B & (B - 1))) return CGGM_EINVAL;
    CGGM_TRY(scratch_reserve(scr));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.err, 0, sizeof(int), st));
    CGGM_CUDA_TRY(cudaMemsetAsync(scr.bar, 0, sizeof(GridBarrier), st));
    const size_t smem = smem_layout<T>(B).total;
    int sorted_arg = rows_sorted ? 1 : 0;
    void *args[] = {(void *)&p, (void *)&q, (void *)&Sxx, (void *)&x0, (void *)&Xd, (void *)&Sigma,
                    (void *)&Sd, (void *)&W, (void *)&Theta, (void *)&m, (void *)&ti,
                    (void *)&tj, (void *)&lam, (void *)&dV, (void *)&B, (void *)&scr,
                    (void *)&sorted_arg};
    const void *fn;
    switch (B) {
        case 32: fn = (const void *)theta_sweep_kernel<T, 1>; break;
        case 64: fn = (const void *)theta_sweep_kernel<T, 2>; break;
        case 128: fn = (const void *)theta_sweep_kernel<T, 4>; break;
        case 256: fn = (const void *)theta_sweep_kernel<T, 8>; break;
        case 512: fn = (const void *)theta_sweep_kernel<float, 16>; break;
        default: return CGGM_EINVAL;
    }
    if (scr.batcher) {
        PassBatcher::Entry e;
        e.f32 = sizeof(T) == 4;
        e.B = B;
        e.st = st;
        PassDesc<T> &d = desc_of<T>(e);
        d = PassDesc<T>{};
        d.kind = 1;
        d.rows_sorted = rows_sorted ? 1 : 0;
        d.p = p; d.q = q; d.m = m; d.x0 = x0;
        d.Sxx = Sxx; d.Xd = Xd; d.Sig = Sigma; d.Sd = Sd; d.W = W;
        d.ia = ti; d.ja = tj; d.lam_off = lam;
        d.out = Theta; d.cache = dV; d.scr = scr;
        CGGM_TRY(run_batched(*scr.batcher, e));
        return read_err(scr.err, st);
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
template cggm_status theta_sweep<double>(int64_t, int64_t, const double *, int64_t,
                                         const double *, const double *, const double *,
                                         const double *, double *, int64_t, const int32_t *,
                                         const int32_t *, double, double *, int, SweepScratch &,
                                         cudaStream_t, bool);
template cggm_status theta_sweep<float>(int64_t, int64_t, const float *, int64_t, const double *,
                                        const float *, const double *, const double *, double *,
                                        int64_t, const int32_t *, const int32_t *, double, float *,
                                        int, SweepScratch &, cudaStream_t, bool);

}  // namespace cggm
