// Coordinate-descent passes of the alternating Newton method (Sections 3.1 and 3.2).
#pragma once

#include "common.cuh"

namespace cggm {

struct PassBatcher;

// Device scratch shared by the sweep kernels (sized for the largest B).
struct SweepScratch {
    double *mu = nullptr;  // [2][B] the steps of two consecutive batches
    void *sub1 = nullptr;  // [2][PRE_N][B] step constants of two batches (T)
    void *sub2 = nullptr;  // [2][coef_slots(B)] in-batch coefficients of two batches,
                           // [2][B][B] their cross coefficients against the batch before (T)
    GridBarrier *bar = nullptr;
    int *err = nullptr;
    // host: when set, the passes of this context are handed to the batcher, which runs the
    // passes of concurrent solves together in one cooperative launch
    PassBatcher *batcher = nullptr;
};

// Several coordinate passes of concurrent solves in one cooperative launch: the grid is cut
// into groups of CTAs, one per pass, each running its pass on its own scratch and barrier
// (results do not depend on the group's size).  Passes handed over by
// lambda_sweep/theta_sweep of contexts that share a batcher are collected for a short
// window - until every solve the batcher serves has one waiting, or 200 us - and launched
// together (passes of one precision and batch size per launch, at most 8).
PassBatcher *batcher_create();
void batcher_destroy(PassBatcher *b);
// solves in progress that may hand over passes (the gathering window ends early once as
// many passes wait)
void batcher_add_busy(PassBatcher *b, int delta);
// launches, passes launched, and launches that held more than one pass (statistics)
void batcher_counts(PassBatcher *b, int64_t *launches, int64_t *passes, int64_t *shared);
// route the passes of a context's solves through a batcher (nullptr: launch them alone)
void ctx_set_batcher(cggm_ctx *c, PassBatcher *b);

// Lambda direction: one pass over (ai, aj), ai <= aj.  Sigma, Psi (q x q, T) with
// double diagonals Sd, Pd; G = S_yy - Sigma - Psi (double); Lambda (double).
// D (double, q x q) and U (T, q x q) must be zero on entry; D receives the direction.
template <typename T>
cggm_status lambda_sweep(int64_t q, const T *Sigma, const T *Psi, const double *Sd,
                         const double *Pd, const double *G, const double *Lambda, int64_t m,
                         const int32_t *ai, const int32_t *aj, double lam_off, double lam_diag,
                         double *D, T *U, int B, SweepScratch &scr,
                         cudaStream_t st);

// Theta pass: coordinates (ti, tj) in visiting order; rows_sorted: they are in ascending
// rows (the active sets are), so that the dot products stop at the rows Delta V can hold
// yet.  Sxx: rows x0 .. x0 + k - 1 of S_xx (k x p,
// T), holding every row i that the coordinates name; Xd the double diagonal of S_xx;
// Sigma (q x q, T) with double diagonal Sd, W = S_xy + S_xx Theta Sigma at entry
// (double p x q), Theta (double p x q) updated in place.  dV (T, p x q): Delta V of the
// pass so far (zero at the start of the pass; a pass may be split into launches over
// consecutive parts of its list, each with the S_xx rows of its part).
template <typename T>
cggm_status theta_sweep(int64_t p, int64_t q, const T *Sxx, int64_t x0, const double *Xd,
                        const T *Sigma, const double *Sd, const double *W, double *Theta,
                        int64_t m, const int32_t *ti, const int32_t *tj, double lam, T *dV,
                        int B, SweepScratch &scr, cudaStream_t st, bool rows_sorted = true);

// Rows of S_xx (p x p, element size esz) that the Theta pass holds at once: all p when they
// fit in 256 MiB, otherwise as many as fit (at least one).  S_xx is formed from X in chunks
// of this many rows and never stored whole beyond that size.
constexpr int64_t kSxxChunkBytes = (int64_t)256 << 20;
inline int64_t sxx_chunk_rows(int64_t p, int64_t esz) {
    const int64_t r = kSxxChunkBytes / (p * esz);
    return r >= p ? p : (r < 1 ? 1 : r);
}

// lambda_sweep in double on scratch buffers laid out by the caller (mu: 2 B doubles, sub1:
// scratch_sub1_bytes(B, 8), sub2: scratch_sub2_bytes(B, 8), bar, err); allocates nothing.
// B in {32, 64, 128}.
cggm_status lambda_sweep_preplanned_f64(int64_t q, const double *Sigma, const double *Psi,
                                        const double *Sd, const double *Pd, const double *G,
                                        const double *Lambda, int64_t m, const int32_t *ai,
                                        const int32_t *aj, double lam_off, double lam_diag,
                                        double *D, double *U, int B, SweepScratch scr,
                                        cudaStream_t st);

// Per-coordinate step constants kept for phase B, and the slots of a batch's in-batch
// coefficients (B (B - 1) / 2 of them, padded).
constexpr int kStepConstants = 6;
__host__ __device__ constexpr int coef_slots(int B) { return ((B * (B - 1) / 2 + 8) + 3) & ~3; }

// Scratch sizes for batch size B and element size esz.
constexpr size_t scratch_sub1_bytes(int B, size_t esz) {
    return esz * 2 * kStepConstants * (size_t)B;
}
constexpr size_t scratch_sub2_bytes(int B, size_t esz) {
    return esz * (2 * (size_t)coef_slots(B) + 2 * (size_t)B * B);
}

// Allocates the scratch once, for B 256 in float (which also covers B <= 128 in double).
cggm_status scratch_reserve(SweepScratch &scr);
void scratch_free(SweepScratch &scr);

int sweep_grid();  // CTAs of the persistent sweep kernels (one per SM)

}  // namespace cggm
