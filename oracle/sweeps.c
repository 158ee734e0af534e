/*
 * CPU oracle: the two coordinate-descent passes of the alternating Newton CD method,
 * in plain C, double precision, single thread, written for reading rather than speed.
 *
 * TEST INFRASTRUCTURE.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark use this file; the CUDA solver never links, calls or includes it.
 *
 * Conventions: every dense matrix is row-major, q x q (Sigma, Psi, S_yy, Lambda, D) or
 * p x q (S_xy, Theta) or p x p (S_xx).  Active sets are lists of (i, j) pairs visited in
 * the order given (row-major ascending).  One coordinate step minimises
 *     (a/2) mu^2 + b mu + lam |c + mu|
 * exactly:  mu = -c + S_{lam/a}(c - b/a),  S_r(w) = sign(w) max(|w| - r, 0)   (Appendix A.1).
 *
 * Build macro ORACLE_MUTANT_PRINTED_CURVATURE (tests only) swaps in the curvatures as
 * the Appendix prints them, a_Lambda = S_ij^2 + S_ii S_jj + S_ii P_jj + 2 S_ij P_ii and
 * a_Theta = S_jj (S_xx)_ii, so that a test can show the 1-D pins reject them.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Soft-thresholding operator S_r(w) (Appendix A.1); zero when |w| <= r. */
static double soft_threshold(double w, double r)
{
    if (w > r) return w - r;
    if (w < -r) return w + r;
    return 0.0;
}

static double dot(const double *x, const double *y, int64_t len)
{
    double s = 0.0;
    for (int64_t t = 0; t < len; t++) s += x[t] * y[t];
    return s;
}

/*
 * One coordinate-descent pass for the Newton direction D of Lambda (Section 3.1, Eq. 7).
 *
 * The quadratic model of g_Theta around Lambda is
 *     gbar(D) = tr(G D) + 1/2 tr(Sigma D Sigma D) + tr(Psi D Sigma D),
 * G = S_yy - Sigma - Psi (Eq. 3), whose Hessian on symmetric D is
 * Sigma(x)Sigma + Sigma(x)Psi + Psi(x)Sigma (Eq. 4).  Along the symmetric direction
 * E_ij + E_ji (i != j) the exact one-dimensional problem, divided by two, has
 *     a = S_ij^2 + S_ii S_jj + S_ii P_jj + S_jj P_ii + 2 S_ij P_ij
 *     b = G_ij + (Sigma D Sigma)_ij + (Psi D Sigma)_ij + (Psi D Sigma)_ji
 *     c = Lambda_ij + D_ij
 * and along E_ii
 *     a = S_ii^2 + 2 S_ii P_ii,  b = G_ii + (Sigma D Sigma)_ii + 2 (Psi D Sigma)_ii.
 * (S = Sigma, P = Psi.)  U = D Sigma is kept up to date (Section 2.2): after D_ij and
 * D_ji grow by mu, row i of U grows by mu Sigma_j and row j by mu Sigma_i.
 *
 * U is stored transposed (Ut = U^T, row t of Ut is column t of U) so that the dot
 * products (Sigma D Sigma)_ij = Sigma_i . U_{:,j} read contiguous memory.
 *
 * D (q x q) and Ut (q x q) are outputs; they are zeroed here.  lam_off applies to
 * off-diagonal coordinates, lam_diag to diagonal ones.
 */
void oracle_lambda_sweep(int64_t q, const double *Sigma, const double *Psi,
                         const double *Syy, const double *Lambda,
                         int64_t m, const int32_t *ai, const int32_t *aj,
                         double lam_off, double lam_diag, double *D, double *Ut)
{
    memset(D, 0, sizeof(double) * (size_t)(q * q));
    memset(Ut, 0, sizeof(double) * (size_t)(q * q));
    for (int64_t l = 0; l < m; l++) {
        const int64_t i = ai[l], j = aj[l];
        const double *Si = Sigma + i * q, *Sj = Sigma + j * q;
        const double *Pi = Psi + i * q, *Pj = Psi + j * q;
        const double *Ucol_i = Ut + i * q, *Ucol_j = Ut + j * q;
        const double s_ii = Si[i], s_jj = Sj[j], s_ij = Si[j];
        const double p_ii = Pi[i], p_jj = Pj[j], p_ij = Pi[j];
        const double sds_ij = dot(Si, Ucol_j, q);   /* (Sigma D Sigma)_ij */
        const double pds_ij = dot(Pi, Ucol_j, q);   /* (Psi D Sigma)_ij   */
        double a, b, lam;
        if (i != j) {
            const double pds_ji = dot(Pj, Ucol_i, q); /* (Psi D Sigma)_ji */
#ifdef ORACLE_MUTANT_PRINTED_CURVATURE
            a = s_ij * s_ij + s_ii * s_jj + s_ii * p_jj + 2.0 * s_ij * p_ii;
#else
            a = s_ij * s_ij + s_ii * s_jj + s_ii * p_jj + s_jj * p_ii + 2.0 * s_ij * p_ij;
#endif
            b = Syy[i * q + j] - s_ij - p_ij + sds_ij + pds_ij + pds_ji;
            lam = lam_off;
        } else {
            a = s_ii * s_ii + 2.0 * s_ii * p_ii;
            b = Syy[i * q + i] - s_ii - p_ii + sds_ij + 2.0 * pds_ij;
            lam = lam_diag;
        }
        const double c = Lambda[i * q + j] + D[i * q + j];
        const double mu = -c + soft_threshold(c - b / a, lam / a);
        if (mu == 0.0) continue;
        D[i * q + j] += mu;
        if (i != j) D[j * q + i] += mu;
        /* U_i += mu Sigma_j ; U_j += mu Sigma_i   (column i / j of Ut) */
        for (int64_t t = 0; t < q; t++) Ut[t * q + i] += mu * Sj[t];
        if (i != j)
            for (int64_t t = 0; t < q; t++) Ut[t * q + j] += mu * Si[t];
    }
}

/*
 * One coordinate-descent pass over the active entries of Theta with Lambda fixed
 * (Section 3.2, Eq. 8).  g_Lambda(Theta) = tr(2 S_xy^T Theta + Sigma Theta^T S_xx Theta)
 * is quadratic; along E_ij its exact one-dimensional problem has
 *     a = 2 Sigma_jj (S_xx)_ii,  b = 2 (S_xy)_ij + 2 (S_xx Theta Sigma)_ij,  c = Theta_ij.
 * V = Theta Sigma (p x q) is kept up to date: after Theta_ij grows by mu, row i of V
 * grows by mu Sigma_j.  V is stored transposed (Vt = V^T, q x p) so that
 * (S_xx V)_ij = (S_xx)_i . V_{:,j} reads contiguous memory.
 *
 * A coordinate whose input column is identically zero ((S_xx)_ii = 0) does not enter
 * g; its exact minimiser under the l1 term is 0.
 *
 * Theta (p x q) is updated in place; Vt must hold (Theta Sigma)^T on entry.
 */
void oracle_theta_sweep(int64_t p, int64_t q, const double *Sxx, const double *Sxy,
                        const double *Sigma, int64_t m, const int32_t *ai,
                        const int32_t *aj, double lam, double *Theta, double *Vt)
{
    for (int64_t l = 0; l < m; l++) {
        const int64_t i = ai[l], j = aj[l];
        const double sxx_ii = Sxx[i * p + i];
        const double c = Theta[i * q + j];
        double mu;
        if (sxx_ii == 0.0) {
            mu = -c;
        } else {
#ifdef ORACLE_MUTANT_PRINTED_CURVATURE
            const double a = Sigma[j * q + j] * sxx_ii;
#else
            const double a = 2.0 * Sigma[j * q + j] * sxx_ii;
#endif
            const double b = 2.0 * Sxy[i * q + j] + 2.0 * dot(Sxx + i * p, Vt + j * p, p);
            mu = -c + soft_threshold(c - b / a, lam / a);
        }
        if (mu == 0.0) continue;
        Theta[i * q + j] += mu;
        const double *Sj = Sigma + j * q;
        for (int64_t t = 0; t < q; t++) Vt[t * p + i] += mu * Sj[t];
    }
}
