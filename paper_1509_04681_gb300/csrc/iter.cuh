// Per-iteration maps and reductions of Algorithm 1 that are neither contractions nor
// coordinate passes: the Lambda gradient, the stopping quantity and the active sets.
#pragma once

#include "common.cuh"

namespace cggm {

// G = S_yy - Sigma - Psi (Eq. 3), all q x q.
template <typename TP>
void grad_lambda(int64_t q, const double *Syy, const double *Sigma, const TP *Psi, double *G,
                 cudaStream_t st);

// Accumulates into out[0..1] (zeroed by the caller):
//   out[0] += sum |grad^S|  (minimum-norm subgradient of Section 5.1, entry-wise:
//             G + lam sign(P) where P != 0, sign(G) max(|G| - lam, 0) where P == 0)
//   out[1] += sum |P|
// over an r x c matrix; when diag_lam >= 0 the diagonal (r == c) uses diag_lam.
void subgrad_sums(int64_t r, int64_t c, const double *G, const double *P, double lam,
                  double diag_lam, double *partial, double *out, cudaStream_t st);

// Active set (Section 2.2): entries with |G| > thr or P != 0, row-major; when `upper`,
// only j >= i.  thr_diag applies on the diagonal.  Writes (ii, jj) and *count (device).
// rowcnt: scratch of r + 1 int64.
void active_compact(int64_t r, int64_t c, const double *G, const double *P, double thr,
                    double thr_diag, bool upper, int64_t *rowcnt, int32_t *ii, int32_t *jj,
                    int64_t *count, cudaStream_t st);

}  // namespace cggm
