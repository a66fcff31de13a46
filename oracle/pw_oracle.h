/*
 * pw_oracle.h -- plain FP64 CPU oracle for Piacsek-Williams (PW) advection.
 *
 * TEST INFRASTRUCTURE ONLY. This is the slow, obviously-correct statement of
 * what the GPU library computes. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it. It shares no code, header,
 * table or helper with the CUDA library, and the library never calls it.
 *
 * Indexing follows the paper's notation with C storage: a field f of an
 * nx x ny x nz domain is stored as f[k*sz + j*sy + i] with x fastest,
 *   i = 0 .. nx+1  (0 and nx+1 are the one-cell halo),
 *   j = 0 .. ny+1  (0 and ny+1 are the halo),
 *   k = 0 .. nz-1  (paper level k+1; no halo in the vertical).
 * sy >= nx+2 and sz >= sy*(ny+2) are element strides.
 */
#ifndef PW_ORACLE_H
#define PW_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Vertical and horizontal coefficients (Listing 1 uses tcx, tcy, tzc1(k),
 * tzc2(k); the paper never defines them, see pw_oracle.c for the reading).
 * dz[k] (k >= 1) is the thickness of cell k, i.e. z[k] - z[k-1] with z[0] = 0.
 * rho[k] is the reference density at w-level z[k], rhon[k] at the u-level
 * zn[k]; either may be NULL, meaning 1 everywhere.
 * Returns 0, or -1 on bad arguments (nz < 1, dx/dy/dz <= 0). */
int pwo_coeffs(int nz, double dx, double dy, const double *dz,
               const double *rho, const double *rhon,
               double *tcx, double *tcy,
               double *tzc1, double *tzc2, double *tzd1, double *tzd2);

/* Source terms su, sv, sw of Listing 1 (su) and its two companions (sv, sw).
 * Writes the interior i=1..nx, j=1..ny, every k; halo cells are untouched.
 * If asu/asv/asw are non-NULL they receive, per point, the sum of the
 * absolute values of the products the formula adds up: each face term
 * c*q*(a+b) contributes |c||q||a+b|. This is the scale against which the
 * rounding error of an FP64 evaluation is measured.
 * nthreads <= 0 means one thread. */
void pwo_advect(int nx, int ny, int nz, long long sy, long long sz,
                const double *u, const double *v, const double *w,
                double tcx, double tcy,
                const double *tzc1, const double *tzc2,
                const double *tzd1, const double *tzd2,
                double *su, double *sv, double *sw,
                double *asu, double *asv, double *asw, int nthreads);

/* The monomial error scale: per point, each face term c*q*(a+b) counted as
 * its two monomials, |c||q|(|a|+|b|). It is >= the scale of pwo_advect and
 * differs from it only where the two velocity samples of a face nearly
 * cancel. It is the scale for evaluations that round the inputs a and b
 * before adding them (each rounding is relative to |a| or |b|, not to
 * |a+b|). Interior only; halo cells are untouched. */
void pwo_monomial_scale(int nx, int ny, int nz, long long sy, long long sz,
                        const double *u, const double *v, const double *w,
                        double tcx, double tcy,
                        const double *tzc1, const double *tzc2,
                        const double *tzd1, const double *tzd2,
                        double *msu, double *msv, double *msw, int nthreads);

/* Mass weights of the discrete energy budget: wu[k] = dz(k) rhon(k) for the
 * u and v cells, ww[k] = dzn(k) rho(k) for the w cells (dzn as in
 * pwo_coeffs), 0 at the levels nothing is computed on (wu at level 1, ww at
 * levels 1 and nz). rho/rhon may be NULL (1). Returns 0 or -1. */
int pwo_energy_weights(int nz, const double *dz, const double *rho, const double *rhon,
                       double *wu, double *ww);

/* out[0..2] = sum over the interior of wu(k)*u*su, wu(k)*v*sv, ww(k)*w*sw;
 * out[3..5] = the sums of the absolute values of the same summands. Fixed
 * order (levels, rows, columns); each sum compensated (Neumaier), so its
 * error does not grow with the number of summands. */
void pwo_energy_budget(int nx, int ny, int nz, long long sy, long long sz,
                       const double *u, const double *v, const double *w,
                       const double *su, const double *sv, const double *sw,
                       const double *wu, const double *ww, double *out);

/* Transpose of the Jacobian of (u,v,w) -> (su,sv,sw) at (u,v,w), applied to
 * cotangents (gsu,gsv,gsw) given on the interior; result ADDED into
 * (gu,gv,gw) over every cell that the forward map reads, halo included.
 * Scatter form: walks the forward loops and, for each product term, adds its
 * two partial derivatives times the cotangent to the cells it read. */
void pwo_advect_adjoint(int nx, int ny, int nz, long long sy, long long sz,
                        const double *u, const double *v, const double *w,
                        double tcx, double tcy,
                        const double *tzc1, const double *tzc2,
                        const double *tzd1, const double *tzd2,
                        const double *gsu, const double *gsv, const double *gsw,
                        double *gu, double *gv, double *gw);

/* Operation count of one column of nz levels as the paper accounts it:
 * 21 per field per level, dropping the upper vertical flux (4 operations)
 * of su and sv at the column top; level 1 is not computed. */
long long pwo_flops_per_column(int nz);

#ifdef __cplusplus
}
#endif
#endif
