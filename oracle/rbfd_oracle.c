/*
 * rbfd_oracle.c -- plain, slow, FP64 CPU oracle of multi-level greedy
 * compact-support RBF mesh deformation with volume point reduction
 * (Morelli, Bellosta, Guardone, "Efficient Radial Basis Function Mesh
 * Deformation Methods for Aircraft Icing", Sections 2-4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or helper with the CUDA library; nothing here is tuned.
 *
 * Every step is written the way the paper states it:
 *   - basis functions: Table 1 / Eq. 2 (Wendland C0, C2, C4, C6), eta = |r - r_i| / R;
 *   - interpolant and solve: Eq. 1 and Eq. 9 on the control set, Phi_cc alpha = dS_c,
 *     solved with a dense row-oriented Cholesky (Cholesky-Banachiewicz) and
 *     forward / back substitution;
 *   - greedy selection (Section 3): first control is surface point 0, the
 *     error vector is Eq. 12, E = dS - Phi_sc alpha, the next control is the
 *     point of largest error, stop once the normalised largest error is below
 *     the tolerance;
 *   - multi-level subspace (Section 3): dS_{l+1} = E at the end of level l;
 *   - volume point reduction (Section 4, Eq. 19 and Eq. 23): volume points
 *     move by sum_l psi(d / D_l) Phi_vc^(l) alpha^(l), with
 *     psi(xi) = 1 - xi on [0, 1) and 0 beyond, D_l = k * max |dS_l|.
 *
 * Readings where the paper is silent or ambiguous (all of them are options or
 * fixed choices below):
 *   - the stop test divides the largest error norm |E_i|_2 by the largest
 *     ORIGINAL displacement norm S0 = max_i |dS_i|_2;
 *   - level l stops at tau_l = eps^((l+1)/L) so that L levels reach eps
 *     with an equal reduction per level (the paper's "reduction of 10^-1 per
 *     level");
 *   - the first control of EVERY level is surface point 0 (first_rule = 0);
 *     first_rule = 1 starts each level at the point of largest |dS_l|;
 *   - points already selected are excluded from the argmax; ties go to the
 *     lowest surface index; the comparison key is Ex*Ex + Ey*Ey (+ Ez*Ez);
 *   - psi applies at every level; if k > 0, D_l = k * max_i |dS_l,i|, capped
 *     at D when D > 0; if k == 0, D_l = D; a D_l of 0 leaves points fixed;
 *     d < 0 is clamped to 0;
 *   - wall distance d (Section 4, taken as given by the paper): the distance
 *     to the nearest surface point;
 *   - mesh quality (Section 5, "orthogonality angle"): per cell of a
 *     structured grid, the smallest angle between two grid lines meeting at
 *     a corner, folded into [0, 90] degrees (90 = orthogonal); a cell whose
 *     corners disagree in orientation is counted as tangled.
 *
 * Compiled with -O2 -ffp-contract=off so that every product and sum is a
 * separately rounded IEEE double operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ESINGULAR 3
#define ORC_ENOTCONV 4

/* ------------------------------------------------------------------ basis */

/* Wendland compact basis functions of Table 1; Eq. 2 is the C2 row.
 * eta >= 1 gives exactly 0 (compact support). */
double orc_phi(int basis, double eta)
{
    if (eta >= 1.0) return 0.0;
    double t = 1.0 - eta;
    double t2 = t * t;
    switch (basis) {
    case 0: /* C0: (1 - eta)^2 */
        return t2;
    case 2: /* C2: (1 - eta)^4 (4 eta + 1) */
        return (t2 * t2) * (4.0 * eta + 1.0);
    case 4: { /* C4: (1 - eta)^6 (35/3 eta^2 + 6 eta + 1) */
        double t6 = (t2 * t2) * t2;
        return t6 * ((35.0 / 3.0) * eta * eta + 6.0 * eta + 1.0);
    }
    case 6: { /* C6: (1 - eta)^8 (32 eta^3 + 25 eta^2 + 8 eta + 1) */
        double t4 = t2 * t2;
        double t8 = t4 * t4;
        return t8 * (32.0 * eta * eta * eta + 25.0 * eta * eta + 8.0 * eta + 1.0);
    }
    default:
        return NAN;
    }
}

/* Wall-distance function psi(xi) of Section 4: 1 - xi on [0, 1), 0 beyond. */
double orc_psi(double xi)
{
    if (xi < 0.0) xi = 0.0;
    if (xi >= 1.0) return 0.0;
    return 1.0 - xi;
}

static double dist(const double *a, const double *b, int dim)
{
    double s = 0.0;
    for (int k = 0; k < dim; ++k) {
        double d = a[k] - b[k];
        s = s + d * d;
    }
    return sqrt(s);
}

static double norm2sq(const double *v, int dim)
{
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s = s + v[k] * v[k];
    return s;
}

/* ------------------------------------------------------ dense linear algebra */

/* Row-oriented (Cholesky-Banachiewicz) factorisation of row i of A = L L^T,
 * given rows 0..i-1 of L.  a_row[j] = A_ij for j <= i.  Writes L_i0..L_ii
 * into Lrow.  Returns -1 if the pivot A_ii - sum_k L_ik^2 is not positive. */
static int chol_row(const double *L, int64_t ld, int64_t i, const double *a_row, double *Lrow)
{
    for (int64_t j = 0; j < i; ++j) {
        double s = a_row[j];
        const double *Lj = L + j * ld;
        for (int64_t k = 0; k < j; ++k) s = s - Lrow[k] * Lj[k];
        Lrow[j] = s / Lj[j];
    }
    double s = a_row[i];
    for (int64_t k = 0; k < i; ++k) s = s - Lrow[k] * Lrow[k];
    if (!(s > 0.0)) return -1;
    Lrow[i] = sqrt(s);
    return 0;
}

/* Full factorisation A = L L^T of an n x n SPD matrix (lower part of A used),
 * row by row.  L and A may not alias.  Returns 0 or -1 (not positive definite). */
int orc_cholesky(int64_t n, const double *A, int64_t lda, double *L, int64_t ldl)
{
    for (int64_t i = 0; i < n; ++i) {
        memset(L + i * ldl, 0, sizeof(double) * (size_t)n);
        if (chol_row(L, ldl, i, A + i * lda, L + i * ldl) != 0) return -1;
    }
    return 0;
}

/* Solve L L^T X = B for nrhs right-hand sides stored as B[i*nrhs + r]:
 * forward substitution L W = B, then back substitution L^T X = W. */
void orc_chol_solve(int64_t n, const double *L, int64_t ld, int nrhs, const double *B, double *X)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)(n * nrhs + 1));
    for (int r = 0; r < nrhs; ++r) {
        for (int64_t i = 0; i < n; ++i) {
            double s = B[i * nrhs + r];
            for (int64_t k = 0; k < i; ++k) s = s - L[i * ld + k] * W[k * nrhs + r];
            W[i * nrhs + r] = s / L[i * ld + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = W[i * nrhs + r];
            for (int64_t k = i + 1; k < n; ++k) s = s - L[k * ld + i] * X[k * nrhs + r];
            X[i * nrhs + r] = s / L[i * ld + i];
        }
    }
    free(W);
}

/* ------------------------------------------------------------- evaluation */

/* f(r) = sum_j alpha_j phi(|r - r_cj| / R) (Eq. 1 with the /R form of
 * Section 2) at n_p points, summed in control order j = 0..n_c-1. */
void orc_eval(int dim, int basis, double R, int64_t n_c, const double *xyz_c, const double *alpha,
              int64_t n_p, const double *xyz_p, double *f, int n_threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int64_t i = 0; i < n_p; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        const double *xi = xyz_p + i * dim;
        for (int64_t j = 0; j < n_c; ++j) {
            double p = orc_phi(basis, dist(xi, xyz_c + j * dim, dim) / R);
            for (int k = 0; k < dim; ++k) acc[k] = acc[k] + alpha[j * dim + k] * p;
        }
        for (int k = 0; k < dim; ++k) f[i * dim + k] = acc[k];
    }
    (void)n_threads;
}

/* ----------------------------------------------------------------- greedy */

/*
 * Multi-level greedy surface point selection (Section 3).
 *
 * Inputs: n_s surface points xyz_s[n_s*dim], displacements dS[n_s*dim],
 * n_levels support radii R[], final tolerance eps, basis id, control cap per
 * level, first-point rule, solve mode (0: append one Cholesky row per added
 * control; 1: refactorise Phi_cc from scratch after every addition).
 *
 * Outputs per level l: nc_out[l] controls, idx_out[l*nc_cap + j] their surface
 * indices in selection order, alpha_out[(l*nc_cap + j)*dim + k] the weights,
 * smax_out[l] = max_i |dS_l,i|, emax_out[l] = max_i |E_i| / S0 after the level,
 * gap_out[l] (optional) the smallest relative gap (key1 - key2) / key1 between
 * the two largest keys over all argmax steps of the level.  E_out (optional)
 * receives the final error E after the last level.  step_gap_out (optional,
 * [n_levels * nc_cap]) receives, at [l*nc_cap + k], the relative gap between
 * the two largest keys of the step that selected control k (k >= 1) and, at
 * [l*nc_cap], the gap of the level's final (stopping) sweep.
 *
 * A level that reaches nc_cap controls ends there, and the next level takes
 * its error.  Returns ORC_OK, ORC_ENOTCONV (the last level's error is not
 * below eps; outputs valid), ORC_ESINGULAR or ORC_EINVAL / ORC_ENOMEM.
 */
int orc_greedy(int dim, int64_t n_s, const double *xyz_s, const double *dS, int n_levels,
               const double *R, double eps, int basis, int64_t nc_cap, int first_rule,
               int solve_mode, int n_threads, int64_t *nc_out, int64_t *idx_out,
               double *alpha_out, double *smax_out, double *emax_out, double *E_out,
               double *gap_out, double *step_gap_out)
{
    if ((dim != 2 && dim != 3) || n_s < 1 || n_levels < 1 || !(eps > 0.0) || nc_cap < 1 ||
        !xyz_s || !dS || !R || !nc_out || !idx_out || !alpha_out || !smax_out || !emax_out)
        return ORC_EINVAL;
    for (int l = 0; l < n_levels; ++l)
        if (!(R[l] > 0.0)) return ORC_EINVAL;
    if (nc_cap > n_s) nc_cap = n_s;

    int status = ORC_OK;
    double S0 = 0.0;
    for (int64_t i = 0; i < n_s; ++i) {
        double v = norm2sq(dS + i * dim, dim);
        if (v > S0) S0 = v;
    }
    S0 = sqrt(S0);
    for (int l = 0; l < n_levels; ++l) {
        nc_out[l] = 0;
        smax_out[l] = 0.0;
        emax_out[l] = 0.0;
        if (gap_out) gap_out[l] = 1.0;
    }
    if (E_out) memset(E_out, 0, sizeof(double) * (size_t)(n_s * dim));
    if (S0 == 0.0) return ORC_OK; /* nothing moves: zero levels */

    double *cur = (double *)malloc(sizeof(double) * (size_t)(n_s * dim));
    double *E = (double *)malloc(sizeof(double) * (size_t)(n_s * dim));
    double *key = (double *)malloc(sizeof(double) * (size_t)n_s);
    unsigned char *sel = (unsigned char *)malloc((size_t)n_s);
    double *L = (double *)malloc(sizeof(double) * (size_t)(nc_cap * nc_cap));
    double *A = (solve_mode == 1) ? (double *)malloc(sizeof(double) * (size_t)(nc_cap * nc_cap)) : NULL;
    double *arow = (double *)malloc(sizeof(double) * (size_t)(nc_cap + 1));
    double *b = (double *)malloc(sizeof(double) * (size_t)(nc_cap * dim));
    double *xc = (double *)malloc(sizeof(double) * (size_t)(nc_cap * dim));
    if (!cur || !E || !key || !sel || !L || (solve_mode == 1 && !A) || !arow || !b || !xc) {
        status = ORC_ENOMEM;
        goto done;
    }
    memcpy(cur, dS, sizeof(double) * (size_t)(n_s * dim));

    for (int l = 0; l < n_levels; ++l) {
        const double Rl = R[l];
        const double tau = pow(eps, (double)(l + 1) / (double)n_levels);
        double smax = 0.0;
        int64_t first = 0;
        for (int64_t i = 0; i < n_s; ++i) {
            double v = norm2sq(cur + i * dim, dim);
            if (v > smax) {
                smax = v;
                if (first_rule == 1) first = i;
            }
        }
        smax_out[l] = sqrt(smax);
        memset(sel, 0, (size_t)n_s);
        int64_t *idx = idx_out + (int64_t)l * nc_cap;
        double *alpha = alpha_out + (int64_t)l * nc_cap * dim;
        int64_t n = 1;
        idx[0] = first;
        sel[first] = 1;
        memcpy(xc, xyz_s + first * dim, sizeof(double) * (size_t)dim);
        /* Phi_cc = [phi(0)], L = [sqrt(phi(0))] */
        arow[0] = orc_phi(basis, 0.0);
        if (solve_mode == 1) A[0] = arow[0];
        if (chol_row(L, nc_cap, 0, arow, L) != 0) {
            status = ORC_ESINGULAR;
            goto done;
        }
        double gap_min = 1.0;
        for (;;) {
            /* Eq. 9 on the control set: Phi_cc alpha = dS_l(C) */
            for (int64_t j = 0; j < n; ++j)
                for (int k = 0; k < dim; ++k) b[j * dim + k] = cur[idx[j] * dim + k];
            orc_chol_solve(n, L, nc_cap, dim, b, alpha);
            /* Eq. 12: E = dS_l - Phi_sc alpha, by brute force over all controls */
            orc_eval(dim, basis, Rl, n, xc, alpha, n_s, xyz_s, E, n_threads);
            for (int64_t i = 0; i < n_s * dim; ++i) E[i] = cur[i] - E[i];
            /* largest error among points not yet selected; lowest index on ties */
            int64_t best = -1;
            double bestv = -1.0, second = -1.0;
            for (int64_t i = 0; i < n_s; ++i) {
                double v = norm2sq(E + i * dim, dim);
                key[i] = v;
                if (sel[i]) continue;
                if (v > bestv) {
                    second = bestv;
                    bestv = v;
                    best = i;
                } else if (v > second) {
                    second = v;
                }
            }
            double g = 1.0;
            if (best >= 0 && bestv > 0.0 && second >= 0.0) {
                g = (bestv - second) / bestv;
                if (g < gap_min) gap_min = g;
            }
            if (step_gap_out) step_gap_out[(int64_t)l * nc_cap + (n < nc_cap ? n : 0)] = g;
            if (best < 0 || sqrt(bestv) / S0 < tau) break;
            if (n == nc_cap) break; /* cap reached: the level ends unconverged */
            /* append the new control: row n of Phi_cc and of its Cholesky factor */
            const double *xb = xyz_s + best * dim;
            for (int64_t j = 0; j < n; ++j) arow[j] = orc_phi(basis, dist(xb, xc + j * dim, dim) / Rl);
            arow[n] = orc_phi(basis, 0.0);
            idx[n] = best;
            sel[best] = 1;
            memcpy(xc + n * dim, xb, sizeof(double) * (size_t)dim);
            if (solve_mode == 1) {
                for (int64_t j = 0; j <= n; ++j) {
                    A[n * nc_cap + j] = arow[j];
                    A[j * nc_cap + n] = arow[j];
                }
                ++n;
                if (orc_cholesky(n, A, nc_cap, L, nc_cap) != 0) {
                    status = ORC_ESINGULAR;
                    goto done;
                }
            } else {
                if (chol_row(L, nc_cap, n, arow, L + n * nc_cap) != 0) {
                    status = ORC_ESINGULAR;
                    goto done;
                }
                ++n;
            }
        }
        nc_out[l] = n;
        double emax = 0.0;
        for (int64_t i = 0; i < n_s; ++i)
            if (key[i] > emax) emax = key[i];
        emax_out[l] = sqrt(emax) / S0;
        if (gap_out) gap_out[l] = gap_min;
        /* multi-level subspace: the next level interpolates this level's error */
        memcpy(cur, E, sizeof(double) * (size_t)(n_s * dim));
    }
    if (!(emax_out[n_levels - 1] < eps)) status = ORC_ENOTCONV; /* final target missed */
    if (E_out) memcpy(E_out, cur, sizeof(double) * (size_t)(n_s * dim));
done:
    free(cur);
    free(E);
    free(key);
    free(sel);
    free(L);
    free(A);
    free(arow);
    free(b);
    free(xc);
    return status;
}

/*
 * Replay of a given control sequence through the greedy of Section 3, as a
 * check of another implementation's choices (test infrastructure).
 *
 * Level by level, the controls are given[l*nc_cap + j] for j < given_nc[l]
 * (the first one included) instead of being chosen here; everything else is
 * orc_greedy's arithmetic: Eq. 9 solved on the controls so far, Eq. 12 by
 * brute force, keys |E_i|^2, and the next level's target is the replayed
 * level's error.  Before appending given control k (k >= 1), and once more
 * after the last one (slot k = given_nc[l]), the step is recorded at
 * [l*(nc_cap+1) + k]:
 *   best_key   the largest key over the points not yet selected (the point
 *              this oracle would pick);
 *   pick_key   the key of the given control k (of the best point at the last
 *              slot, where nothing is picked);
 *   best_scale, pick_scale   the rounding scale of E at those two points,
 *              |dS_l,i|_2 + sum_j |alpha_j|_2 phi_ij: two evaluations of
 *              Eq. 12 that sum in different orders differ by a few n u times it.
 * alpha_out[(l*nc_cap + j)*dim + k] receives the weights of the replayed
 * levels, smax_out[l] the max |dS_l|.  Returns ORC_OK, ORC_EINVAL (a given
 * index out of range or repeated in a level), ORC_ESINGULAR or ORC_ENOMEM.
 */
int orc_replay(int dim, int64_t n_s, const double *xyz_s, const double *dS, int n_levels,
               const double *R, int basis, int64_t nc_cap, const int64_t *given_nc, const int64_t *given,
               int n_threads, double *alpha_out, double *smax_out, double *best_key, double *pick_key,
               double *best_scale, double *pick_scale)
{
    if ((dim != 2 && dim != 3) || n_s < 1 || n_levels < 1 || nc_cap < 1 || !xyz_s || !dS || !R || !given_nc ||
        !given || !alpha_out || !smax_out || !best_key || !pick_key || !best_scale || !pick_scale)
        return ORC_EINVAL;
    for (int l = 0; l < n_levels; ++l) {
        if (!(R[l] > 0.0) || given_nc[l] < 1 || given_nc[l] > nc_cap) return ORC_EINVAL;
        for (int64_t j = 0; j < given_nc[l]; ++j)
            if (given[l * nc_cap + j] < 0 || given[l * nc_cap + j] >= n_s) return ORC_EINVAL;
    }
    int status = ORC_OK;
    double *cur = (double *)malloc(sizeof(double) * (size_t)(n_s * dim));
    double *E = (double *)malloc(sizeof(double) * (size_t)(n_s * dim));
    unsigned char *sel = (unsigned char *)malloc((size_t)n_s);
    double *L = (double *)malloc(sizeof(double) * (size_t)(nc_cap * nc_cap));
    double *arow = (double *)malloc(sizeof(double) * (size_t)(nc_cap + 1));
    double *b = (double *)malloc(sizeof(double) * (size_t)(nc_cap * dim));
    double *xc = (double *)malloc(sizeof(double) * (size_t)(nc_cap * dim));
    if (!cur || !E || !sel || !L || !arow || !b || !xc) {
        status = ORC_ENOMEM;
        goto done;
    }
    memcpy(cur, dS, sizeof(double) * (size_t)(n_s * dim));
    for (int l = 0; l < n_levels; ++l) {
        const double Rl = R[l];
        const int64_t nl = given_nc[l];
        const int64_t *gl = given + l * nc_cap;
        double *alpha = alpha_out + l * nc_cap * dim;
        double smax = 0.0;
        for (int64_t i = 0; i < n_s; ++i) {
            double v = norm2sq(cur + i * dim, dim);
            if (v > smax) smax = v;
        }
        smax_out[l] = sqrt(smax);
        memset(sel, 0, (size_t)n_s);
        int64_t n = 1;
        sel[gl[0]] = 1;
        memcpy(xc, xyz_s + gl[0] * dim, sizeof(double) * (size_t)dim);
        arow[0] = orc_phi(basis, 0.0);
        if (chol_row(L, nc_cap, 0, arow, L) != 0) {
            status = ORC_ESINGULAR;
            goto done;
        }
        for (;;) {
            for (int64_t j = 0; j < n; ++j)
                for (int k = 0; k < dim; ++k) b[j * dim + k] = cur[gl[j] * dim + k];
            orc_chol_solve(n, L, nc_cap, dim, b, alpha);
            orc_eval(dim, basis, Rl, n, xc, alpha, n_s, xyz_s, E, n_threads);
            for (int64_t i = 0; i < n_s * dim; ++i) E[i] = cur[i] - E[i];
            int64_t best = -1;
            double bestv = -1.0;
            for (int64_t i = 0; i < n_s; ++i) {
                if (sel[i]) continue;
                double v = norm2sq(E + i * dim, dim);
                if (v > bestv) {
                    bestv = v;
                    best = i;
                }
            }
            const int64_t pick = n < nl ? gl[n] : best;
            const int64_t slot = l * (nc_cap + 1) + n;
            best_key[slot] = bestv;
            pick_key[slot] = pick >= 0 ? norm2sq(E + pick * dim, dim) : -1.0;
            for (int which = 0; which < 2; ++which) {
                const int64_t i = which == 0 ? best : pick;
                double sc = 0.0;
                if (i >= 0) {
                    sc = sqrt(norm2sq(cur + i * dim, dim));
                    for (int64_t j = 0; j < n; ++j)
                        sc = sc + sqrt(norm2sq(alpha + j * dim, dim)) *
                                      orc_phi(basis, dist(xyz_s + i * dim, xc + j * dim, dim) / Rl);
                }
                if (which == 0) best_scale[slot] = sc;
                else pick_scale[slot] = sc;
            }
            if (n == nl) break;
            if (sel[pick]) {
                status = ORC_EINVAL; /* a control given twice in one level */
                goto done;
            }
            const double *xb = xyz_s + pick * dim;
            for (int64_t j = 0; j < n; ++j) arow[j] = orc_phi(basis, dist(xb, xc + j * dim, dim) / Rl);
            arow[n] = orc_phi(basis, 0.0);
            sel[pick] = 1;
            memcpy(xc + n * dim, xb, sizeof(double) * (size_t)dim);
            if (chol_row(L, nc_cap, n, arow, L + n * nc_cap) != 0) {
                status = ORC_ESINGULAR;
                goto done;
            }
            ++n;
        }
        memcpy(cur, E, sizeof(double) * (size_t)(n_s * dim));
    }
done:
    free(cur);
    free(E);
    free(sel);
    free(L);
    free(arow);
    free(b);
    free(xc);
    return status;
}

/* ----------------------------------------------------------- volume update */

/* Support distance per level (Section 4): D_l = k * max_i |dS_l,i| (capped at
 * D when D > 0) if k > 0, else D_l = D. */
void orc_support_distances(int n_levels, const double *smax, double k, double D, double *Dl)
{
    for (int l = 0; l < n_levels; ++l) {
        double v = (k > 0.0) ? k * smax[l] : D;
        if (k > 0.0 && D > 0.0 && v > D) v = D;
        Dl[l] = v;
    }
}

/*
 * Volume update of Eq. 19 with the blending of Eq. 23:
 *   dV(r) = sum_l psi(d(r) / D_l) sum_{j < nc[l]} alpha_j^(l) phi(|r - r_cj^(l)| / R_l)
 * by brute force over every control of every level, for volume points with
 * d < D_l (all others get psi = 0 for that level).
 *
 * idx[l*nc_cap + j] and alpha[(l*nc_cap + j)*dim + k] as written by orc_greedy.
 * xyz_v[n_v*dim] and d_v[n_v] are the volume points and wall distances;
 * out[n_v*dim] receives dV.
 */
int orc_deform(int dim, int basis, int n_levels, const double *R, const double *Dl,
               const int64_t *nc, const int64_t *idx, const double *alpha, int64_t nc_cap,
               const double *xyz_s, int64_t n_v, const double *xyz_v, const double *d_v,
               double *out, int n_threads)
{
    if ((dim != 2 && dim != 3) || n_levels < 0 || n_v < 0 || !out) return ORC_EINVAL;
    int64_t ncmax = 1;
    for (int l = 0; l < n_levels; ++l)
        if (nc[l] > ncmax) ncmax = nc[l];
    double *xc = (double *)malloc(sizeof(double) * (size_t)(ncmax * dim));
    if (!xc) return ORC_ENOMEM;
    memset(out, 0, sizeof(double) * (size_t)(n_v * dim));
    for (int l = 0; l < n_levels; ++l) {
        if (nc[l] == 0 || !(Dl[l] > 0.0)) continue;
        for (int64_t j = 0; j < nc[l]; ++j)
            memcpy(xc + j * dim, xyz_s + idx[(int64_t)l * nc_cap + j] * dim, sizeof(double) * (size_t)dim);
        const double *al = alpha + (int64_t)l * nc_cap * dim;
        const double Rl = R[l], D = Dl[l];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1)
#endif
        for (int64_t v = 0; v < n_v; ++v) {
            double dv = d_v[v];
            if (dv < 0.0) dv = 0.0;
            if (!(dv < D)) continue; /* volume point reduction: psi = 0 */
            double w = orc_psi(dv / D);
            const double *xv = xyz_v + v * dim;
            double acc[3] = {0.0, 0.0, 0.0};
            for (int64_t j = 0; j < nc[l]; ++j) {
                double p = orc_phi(basis, dist(xv, xc + j * dim, dim) / Rl);
                for (int k = 0; k < dim; ++k) acc[k] = acc[k] + al[j * dim + k] * p;
            }
            for (int k = 0; k < dim; ++k) out[v * dim + k] = out[v * dim + k] + w * acc[k];
        }
    }
    free(xc);
    (void)n_threads;
    return ORC_OK;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ wall distance */

/* d(r) of Section 4 for each volume point: the distance to the nearest surface
 * point (the paper takes d as given; this is its plainest definition on a
 * point cloud), by brute force over every surface point. */
void orc_wall_distance(int dim, int64_t n_s, const double *xyz_s, int64_t n_v, const double *xyz_v, double *d,
                       int n_threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads > 0 ? n_threads : 1)
#endif
    for (int64_t v = 0; v < n_v; ++v) {
        double best = INFINITY;
        for (int64_t i = 0; i < n_s; ++i) {
            double r = dist(xyz_v + v * dim, xyz_s + i * dim, dim);
            if (r < best) best = r;
        }
        d[v] = best;
    }
    (void)n_threads;
}

/* ------------------------------------------------------------ mesh quality */

/* Node (i, k, j) of a structured grid grown off the surface: layer j = 0 is
 * the wall (surface point (k, i) moved by its displacement), layers j >= 1 are
 * volume points (k, i, j - 1) moved by theirs.  Every coordinate is the FP64
 * sum of the stored value and its displacement. */
typedef struct {
    int dim;
    int64_t n_i, n_k, n_layers;
    const double *wall, *wall_disp;
    const float *vol, *vol_disp;
} orc_grid;

static void grid_node(const orc_grid *g, int64_t i, int64_t k, int64_t j, double *p)
{
    for (int c = 0; c < 3; ++c) p[c] = 0.0;
    for (int c = 0; c < g->dim; ++c) {
        if (j == 0) {
            int64_t q = (k * g->n_i + i) * g->dim + c;
            p[c] = g->wall[q] + (g->wall_disp ? g->wall_disp[q] : 0.0);
        } else {
            int64_t q = ((k * g->n_i + i) * g->n_layers + (j - 1)) * g->dim + c;
            p[c] = (double)g->vol[q] + (g->vol_disp ? (double)g->vol_disp[q] : 0.0);
        }
    }
}

/* Angle between the grid lines a and b at a corner, folded into [0, 90]
 * degrees: atan2(|a x b|, |a . b|). */
static double folded_angle_deg(const double *a, const double *b, int dim)
{
    double dot = a[0] * b[0] + a[1] * b[1] + (dim == 3 ? a[2] * b[2] : 0.0);
    double cr;
    if (dim == 2) {
        cr = fabs(a[0] * b[1] - a[1] * b[0]);
    } else {
        double c0 = a[1] * b[2] - a[2] * b[1];
        double c1 = a[2] * b[0] - a[0] * b[2];
        double c2 = a[0] * b[1] - a[1] * b[0];
        cr = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    return atan2(cr, fabs(dot)) * (180.0 / 3.14159265358979323846);
}

static void sub3(const double *a, const double *b, double *out)
{
    for (int c = 0; c < 3; ++c) out[c] = a[c] - b[c];
}

/* Orthogonality angle of every cell of the grid and a summary.
 *   2D: cells (i, j) between wall-normal lines i, i+1 and layers j, j+1;
 *       theta index i * n_layers + j.
 *   3D: cells (k, i, j) with the span direction k; index (k * n_ci + i) * n_layers + j.
 * n_ci = n_i if the i direction closes on itself (periodic), else n_i - 1.
 * Orientation at a corner: 2D, the cross product of the edges to the next and
 * the previous corner going round the cell; 3D, the triple product of the
 * three edges leaving the corner, sign-corrected by the corner's parity.  A
 * cell with both positive and negative orientations is tangled.
 * summary: [0] min angle, [1] mean angle, [2] argmin (lowest index on ties),
 *          [3] cells, [4] tangled cells, [5..13] cells per 10-degree bin. */
int orc_orthogonality(int dim, int64_t n_i, int64_t n_k, int64_t n_layers, int periodic_i, const double *wall,
                      const double *wall_disp, const float *vol, const float *vol_disp, double *theta,
                      double *summary)
{
    if ((dim != 2 && dim != 3) || n_i < 2 || n_layers < 1 || (dim == 3 && n_k < 2) || !wall || !vol)
        return ORC_EINVAL;
    if (dim == 2) n_k = 1;
    orc_grid g = {dim, n_i, n_k, n_layers, wall, wall_disp, vol, vol_disp};
    int64_t n_ci = periodic_i ? n_i : n_i - 1;
    int64_t n_ck = dim == 3 ? n_k - 1 : 1;
    int64_t cells = n_ck * n_ci * n_layers;
    double mn = INFINITY, sum = 0.0;
    int64_t argmin = -1, tangled = 0, hist[9] = {0};
    for (int64_t k = 0; k < n_ck; ++k)
        for (int64_t i = 0; i < n_ci; ++i)
            for (int64_t j = 0; j < n_layers; ++j) {
                int64_t i1 = (i + 1) % n_i;
                double th = INFINITY;
                int pos = 0, neg = 0;
                if (dim == 2) {
                    /* corners in order round the cell */
                    double P[4][3], e0[3], e1[3];
                    grid_node(&g, i, 0, j, P[0]);
                    grid_node(&g, i1, 0, j, P[1]);
                    grid_node(&g, i1, 0, j + 1, P[2]);
                    grid_node(&g, i, 0, j + 1, P[3]);
                    for (int q = 0; q < 4; ++q) {
                        sub3(P[(q + 1) % 4], P[q], e0);
                        sub3(P[(q + 3) % 4], P[q], e1);
                        double a = folded_angle_deg(e0, e1, 2);
                        if (a < th) th = a;
                        double o = e0[0] * e1[1] - e0[1] * e1[0];
                        pos |= o > 0.0;
                        neg |= o < 0.0;
                    }
                } else {
                    double P[2][2][2][3]; /* [di][dk][dj] */
                    for (int di = 0; di < 2; ++di)
                        for (int dk = 0; dk < 2; ++dk)
                            for (int dj = 0; dj < 2; ++dj)
                                grid_node(&g, di ? i1 : i, k + dk, j + dj, P[di][dk][dj]);
                    for (int di = 0; di < 2; ++di)
                        for (int dk = 0; dk < 2; ++dk)
                            for (int dj = 0; dj < 2; ++dj) {
                                double ei[3], ek[3], ej[3];
                                const double *c = P[di][dk][dj];
                                sub3(P[1 - di][dk][dj], c, ei);
                                sub3(P[di][1 - dk][dj], c, ek);
                                sub3(P[di][dk][1 - dj], c, ej);
                                double a = folded_angle_deg(ei, ek, 3);
                                if (a < th) th = a;
                                a = folded_angle_deg(ei, ej, 3);
                                if (a < th) th = a;
                                a = folded_angle_deg(ek, ej, 3);
                                if (a < th) th = a;
                                /* ei . (ek x ej), times -1 for odd corners */
                                double x0 = ek[1] * ej[2] - ek[2] * ej[1];
                                double x1 = ek[2] * ej[0] - ek[0] * ej[2];
                                double x2 = ek[0] * ej[1] - ek[1] * ej[0];
                                double o = ei[0] * x0 + ei[1] * x1 + ei[2] * x2;
                                if ((di + dk + dj) & 1) o = -o;
                                pos |= o > 0.0;
                                neg |= o < 0.0;
                            }
                }
                int64_t idx = (k * n_ci + i) * n_layers + j;
                if (theta) theta[idx] = th;
                if (th < mn) {
                    mn = th;
                    argmin = idx;
                }
                sum += th;
                tangled += (pos && neg);
                int b = (int)(th / 10.0);
                hist[b < 0 ? 0 : (b > 8 ? 8 : b)]++;
            }
    summary[0] = mn;
    summary[1] = cells ? sum / (double)cells : 0.0;
    summary[2] = (double)argmin;
    summary[3] = (double)cells;
    summary[4] = (double)tangled;
    for (int b = 0; b < 9; ++b) summary[5 + b] = (double)hist[b];
    return ORC_OK;
}
