// Coordinate-descent passes of the alternating Newton method (Sections 3.1 and 3.2).
#pragma once

#include "common.cuh"

namespace cggm {

// Batch plan: the active list cut into batches of B consecutive coordinates, with the
// sorted distinct indices each batch touches, every coordinate's positions in them,
// and, per distinct index, the list of (coordinate, partner position) pairs whose
// update lands on that index's row of the cache (U or Delta V).
struct BatchPlan {
    int B = 0;           // coordinates per batch (32, 64 or 128)
    int K = 0;           // 2B
    int64_t nbatch = 0;
    int64_t cap = 0;     // batches the buffers hold
    int32_t *nidx = nullptr;   // [nbatch]      distinct first indices (Theta: distinct i)
    int32_t *nidx2 = nullptr;  // [nbatch]      Theta only: distinct j
    int32_t *idx = nullptr;    // [nbatch][K]
    int32_t *idx2 = nullptr;   // [nbatch][K]   Theta only
    int32_t *pa = nullptr;     // [nbatch][B]
    int32_t *pb = nullptr;     // [nbatch][B]
    int32_t *lptr = nullptr;   // [nbatch][K+1]
    int32_t *lent = nullptr;   // [nbatch][K]   (l << 16) | partner position
};

// Device scratch shared by the sweep kernels (sized for the largest B and grid).
struct SweepScratch {
    double *partial = nullptr;  // [grid][B][3]
    double *mu = nullptr;       // [B]
    void *sub1 = nullptr;       // [K][K] gathered submatrix (T)
    void *sub2 = nullptr;       // [K][K]
    GridBarrier *bar = nullptr;
    unsigned *ticket = nullptr;
    int *err = nullptr;
};

// Lambda direction: one pass over (ai, aj), ai <= aj.  Sigma, Psi (q x q, T) with
// double diagonals Sd, Pd; G = S_yy - Sigma - Psi (double); Lambda (double).
// D (double, q x q) and U (T, q x q) must be zero on entry; D receives the direction.
template <typename T>
cggm_status lambda_sweep(int64_t q, const T *Sigma, const T *Psi, const double *Sd,
                         const double *Pd, const double *G, const double *Lambda, int64_t m,
                         const int32_t *ai, const int32_t *aj, double lam_off, double lam_diag,
                         double *D, T *U, int B, BatchPlan &plan, SweepScratch &scr,
                         cudaStream_t st);

// Theta pass: coordinates (ti, tj) row-major.  Sxx (p x p, T) with double diagonal Xd,
// Sigma (q x q, T) with double diagonal Sd, W = S_xy + S_xx Theta Sigma at entry
// (double p x q), Theta (double p x q) updated in place.  dV (T, p x q) must be zero.
template <typename T>
cggm_status theta_sweep(int64_t p, int64_t q, const T *Sxx, const double *Xd, const T *Sigma,
                        const double *Sd, const double *W, double *Theta, int64_t m,
                        const int32_t *ti, const int32_t *tj, double lam, T *dV, int B,
                        BatchPlan &plan, SweepScratch &scr, cudaStream_t st);

// lambda_sweep in double on plan and scratch buffers laid out by the caller (their
// pointers set, plan.cap >= ceil(m / B)); allocates nothing.  B in {32, 64, 128}.
cggm_status lambda_sweep_preplanned_f64(int64_t q, const double *Sigma, const double *Psi,
                                        const double *Sd, const double *Pd, const double *G,
                                        const double *Lambda, int64_t m, const int32_t *ai,
                                        const int32_t *aj, double lam_off, double lam_diag,
                                        double *D, double *U, int B, BatchPlan plan,
                                        SweepScratch scr, cudaStream_t st);

// Plan storage helpers (allocate on demand, grow only).
cggm_status plan_reserve(BatchPlan &plan, int B, int64_t nbatch, bool theta);
void plan_free(BatchPlan &plan);
cggm_status scratch_reserve(SweepScratch &scr, int B, int grid);
void scratch_free(SweepScratch &scr);

int sweep_grid();  // CTAs of the persistent sweep kernels (one per SM)

}  // namespace cggm
