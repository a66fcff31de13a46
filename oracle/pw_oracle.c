/*
 * pw_oracle.c -- plain FP64 CPU oracle for Piacsek-Williams (PW) advection.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library. Compiled with
 * -O2 -ffp-contract=off so every multiply and add rounds separately, in the
 * order written here.
 *
 * What it follows (paper: N. Brown, "Accelerating advection for atmospheric
 * modelling on Xilinx and Intel FPGAs", arXiv:2107.13500):
 *   - su: Listing 1 of Sec. II-A, term by term and in its evaluation order,
 *     over k = 2..nz with the upper vertical flux dropped at k = nz.
 *   - sv, sw: Sec. II-A says the scheme loops over U, V and W and returns the
 *     three source terms, 21 operations each (Sec. III), but prints only su.
 *     sv is su with the roles of x and y (u and v, tcx and tcy) exchanged;
 *     sw applies the same flux form to w on its own (w-level) grid. Both are
 *     readings, pinned by the tests (transpose identity, energy conservation,
 *     second-order convergence, closed forms).
 *   - Staggering (Arakawa C): u at (i+1/2, j, zn_k), v at (i, j+1/2, zn_k),
 *     w at (i, j, z_k), the top face of cell k.
 *   - Level 1 is not computed (Listing 1 starts at k = 2): outputs there are
 *     0. sw is computed for k = 2..nz-1 and is 0 at k = nz (rigid lid,
 *     w(nz) = 0), so no vertical halo is ever read.
 *
 * Storage is C order f[k*sz + j*sy + i], x fastest; index k here is the
 * paper's level k+1.
 */
#include "pw_oracle.h"

#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(f, k, j, i) (f)[(size_t)(k) * (size_t)sz + (size_t)(j) * (size_t)sy + (size_t)(i)]

static double absd(double x) { return x < 0.0 ? -x : x; }

/*
 * Coefficients. The paper uses tcx, tcy, tzc1(k), tzc2(k) in Listing 1 but
 * never defines them. Reading (flux form on a stretched, density-weighted
 * vertical grid; 0.25 = the two 1/2 averaging factors of a centred flux):
 *   tcx = 0.25/dx, tcy = 0.25/dy
 *   z(1) = 0, z(k) = z(k-1) + dz(k)              (w levels, top of cell k)
 *   zn(k) = (z(k-1) + z(k))/2 for k >= 2,  zn(1) = -zn(2)   (u/v levels)
 *   dzn(k) = zn(k+1) - zn(k)                     (spacing around w level k)
 *   tzc1(k) = 0.25 rho(k-1) / (rhon(k) dz(k))     lower face of u/v cell k
 *   tzc2(k) = 0.25 rho(k)   / (rhon(k) dz(k))     upper face of u/v cell k
 *   tzd1(k) = 0.25 rhon(k)   / (rho(k) dzn(k))    lower face of w cell k
 *   tzd2(k) = 0.25 rhon(k+1) / (rho(k) dzn(k))    upper face of w cell k
 * Entries a level never uses (tzc at level 1, tzd at levels 1 and nz) are 0.
 */
int pwo_coeffs(int nz, double dx, double dy, const double *dz,
               const double *rho, const double *rhon,
               double *tcx, double *tcy,
               double *tzc1, double *tzc2, double *tzd1, double *tzd2)
{
    if (nz < 1 || !(dx > 0.0) || !(dy > 0.0) || dz == NULL) return -1;
    for (int k = 1; k < nz; ++k)
        if (!(dz[k] > 0.0)) return -1;

    *tcx = 0.25 / dx;
    *tcy = 0.25 / dy;

    /* Level heights, written out one by one. */
    double *z = (double *)malloc(sizeof(double) * (size_t)nz);
    double *zn = (double *)malloc(sizeof(double) * (size_t)nz);
    if (!z || !zn) { free(z); free(zn); return -1; }
    z[0] = 0.0;
    for (int k = 1; k < nz; ++k) z[k] = z[k - 1] + dz[k];
    for (int k = 1; k < nz; ++k) zn[k] = 0.5 * (z[k - 1] + z[k]);
    zn[0] = (nz > 1) ? -zn[1] : 0.0;

    for (int k = 0; k < nz; ++k) {
        tzc1[k] = tzc2[k] = tzd1[k] = tzd2[k] = 0.0;
    }
    for (int k = 1; k < nz; ++k) {
        double rho_lo = rho ? rho[k - 1] : 1.0;
        double rho_hi = rho ? rho[k] : 1.0;
        double rn = rhon ? rhon[k] : 1.0;
        tzc1[k] = 0.25 * rho_lo / (rn * dz[k]);
        tzc2[k] = 0.25 * rho_hi / (rn * dz[k]);
    }
    for (int k = 1; k < nz - 1; ++k) {
        double dzn = zn[k + 1] - zn[k];
        double rn_lo = rhon ? rhon[k] : 1.0;
        double rn_hi = rhon ? rhon[k + 1] : 1.0;
        double rw = rho ? rho[k] : 1.0;
        tzd1[k] = 0.25 * rn_lo / (rw * dzn);
        tzd2[k] = 0.25 * rn_hi / (rw * dzn);
    }
    free(z);
    free(zn);
    return 0;
}

void pwo_advect(int nx, int ny, int nz, long long sy, long long sz,
                const double *u, const double *v, const double *w,
                double tcx, double tcy,
                const double *tzc1, const double *tzc2,
                const double *tzd1, const double *tzd2,
                double *su, double *sv, double *sw,
                double *asu, double *asv, double *asw, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1) return;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int i = 1; i <= nx; ++i) {
        for (int j = 1; j <= ny; ++j) {
            /* Level 1 (k = 0 here) is not computed. */
            AT(su, 0, j, i) = 0.0;
            AT(sv, 0, j, i) = 0.0;
            AT(sw, 0, j, i) = 0.0;
            if (asu) { AT(asu, 0, j, i) = 0.0; AT(asv, 0, j, i) = 0.0; AT(asw, 0, j, i) = 0.0; }

            for (int k = 1; k < nz; ++k) {
                const int top = (k == nz - 1);
                double s, a;

                /* su: Listing 1. x self term, y cross term with v, z cross term with w. */
                s = tcx * (AT(u, k, j, i - 1) * (AT(u, k, j, i) + AT(u, k, j, i - 1))
                           - AT(u, k, j, i + 1) * (AT(u, k, j, i) + AT(u, k, j, i + 1)));
                s = s + tcy * (AT(u, k, j - 1, i) * (AT(v, k, j - 1, i) + AT(v, k, j - 1, i + 1))
                               - AT(u, k, j + 1, i) * (AT(v, k, j, i) + AT(v, k, j, i + 1)));
                if (!top) {
                    s = s + tzc1[k] * AT(u, k - 1, j, i) * (AT(w, k - 1, j, i) + AT(w, k - 1, j, i + 1))
                          - tzc2[k] * AT(u, k + 1, j, i) * (AT(w, k, j, i) + AT(w, k, j, i + 1));
                } else {
                    s = s + tzc1[k] * AT(u, k - 1, j, i) * (AT(w, k - 1, j, i) + AT(w, k - 1, j, i + 1));
                }
                AT(su, k, j, i) = s;
                if (asu) {
                    a = absd(tcx) * (absd(AT(u, k, j, i - 1)) * (absd(AT(u, k, j, i)) + absd(AT(u, k, j, i - 1)))
                                     + absd(AT(u, k, j, i + 1)) * (absd(AT(u, k, j, i)) + absd(AT(u, k, j, i + 1))));
                    a += absd(tcy) * (absd(AT(u, k, j - 1, i)) * (absd(AT(v, k, j - 1, i)) + absd(AT(v, k, j - 1, i + 1)))
                                      + absd(AT(u, k, j + 1, i)) * (absd(AT(v, k, j, i)) + absd(AT(v, k, j, i + 1))));
                    a += absd(tzc1[k]) * absd(AT(u, k - 1, j, i)) * (absd(AT(w, k - 1, j, i)) + absd(AT(w, k - 1, j, i + 1)));
                    if (!top)
                        a += absd(tzc2[k]) * absd(AT(u, k + 1, j, i)) * (absd(AT(w, k, j, i)) + absd(AT(w, k, j, i + 1)));
                    AT(asu, k, j, i) = a;
                }

                /* sv: su with x and y exchanged (u <-> v, tcx <-> tcy). */
                s = tcy * (AT(v, k, j - 1, i) * (AT(v, k, j, i) + AT(v, k, j - 1, i))
                           - AT(v, k, j + 1, i) * (AT(v, k, j, i) + AT(v, k, j + 1, i)));
                s = s + tcx * (AT(v, k, j, i - 1) * (AT(u, k, j, i - 1) + AT(u, k, j + 1, i - 1))
                               - AT(v, k, j, i + 1) * (AT(u, k, j, i) + AT(u, k, j + 1, i)));
                if (!top) {
                    s = s + tzc1[k] * AT(v, k - 1, j, i) * (AT(w, k - 1, j, i) + AT(w, k - 1, j + 1, i))
                          - tzc2[k] * AT(v, k + 1, j, i) * (AT(w, k, j, i) + AT(w, k, j + 1, i));
                } else {
                    s = s + tzc1[k] * AT(v, k - 1, j, i) * (AT(w, k - 1, j, i) + AT(w, k - 1, j + 1, i));
                }
                AT(sv, k, j, i) = s;
                if (asv) {
                    a = absd(tcy) * (absd(AT(v, k, j - 1, i)) * (absd(AT(v, k, j, i)) + absd(AT(v, k, j - 1, i)))
                                     + absd(AT(v, k, j + 1, i)) * (absd(AT(v, k, j, i)) + absd(AT(v, k, j + 1, i))));
                    a += absd(tcx) * (absd(AT(v, k, j, i - 1)) * (absd(AT(u, k, j, i - 1)) + absd(AT(u, k, j + 1, i - 1)))
                                      + absd(AT(v, k, j, i + 1)) * (absd(AT(u, k, j, i)) + absd(AT(u, k, j + 1, i))));
                    a += absd(tzc1[k]) * absd(AT(v, k - 1, j, i)) * (absd(AT(w, k - 1, j, i)) + absd(AT(w, k - 1, j + 1, i)));
                    if (!top)
                        a += absd(tzc2[k]) * absd(AT(v, k + 1, j, i)) * (absd(AT(w, k, j, i)) + absd(AT(w, k, j + 1, i)));
                    AT(asv, k, j, i) = a;
                }

                /* sw: same flux form on the w grid. Horizontal advecting
                 * velocities are the sums of u (v) at the two u-levels k and
                 * k+1 around w-level k. Rigid lid: sw(nz) = 0. */
                if (!top) {
                    s = tcx * (AT(w, k, j, i - 1) * (AT(u, k, j, i - 1) + AT(u, k + 1, j, i - 1))
                               - AT(w, k, j, i + 1) * (AT(u, k, j, i) + AT(u, k + 1, j, i)));
                    s = s + tcy * (AT(w, k, j - 1, i) * (AT(v, k, j - 1, i) + AT(v, k + 1, j - 1, i))
                                   - AT(w, k, j + 1, i) * (AT(v, k, j, i) + AT(v, k + 1, j, i)));
                    s = s + tzd1[k] * AT(w, k - 1, j, i) * (AT(w, k, j, i) + AT(w, k - 1, j, i))
                          - tzd2[k] * AT(w, k + 1, j, i) * (AT(w, k, j, i) + AT(w, k + 1, j, i));
                    AT(sw, k, j, i) = s;
                    if (asw) {
                        a = absd(tcx) * (absd(AT(w, k, j, i - 1)) * (absd(AT(u, k, j, i - 1)) + absd(AT(u, k + 1, j, i - 1)))
                                         + absd(AT(w, k, j, i + 1)) * (absd(AT(u, k, j, i)) + absd(AT(u, k + 1, j, i))));
                        a += absd(tcy) * (absd(AT(w, k, j - 1, i)) * (absd(AT(v, k, j - 1, i)) + absd(AT(v, k + 1, j - 1, i)))
                                          + absd(AT(w, k, j + 1, i)) * (absd(AT(v, k, j, i)) + absd(AT(v, k + 1, j, i))));
                        a += absd(tzd1[k]) * absd(AT(w, k - 1, j, i)) * (absd(AT(w, k, j, i)) + absd(AT(w, k - 1, j, i)));
                        a += absd(tzd2[k]) * absd(AT(w, k + 1, j, i)) * (absd(AT(w, k, j, i)) + absd(AT(w, k + 1, j, i)));
                        AT(asw, k, j, i) = a;
                    }
                } else {
                    AT(sw, k, j, i) = 0.0;
                    if (asw) AT(asw, k, j, i) = 0.0;
                }
            }
        }
    }
}

/*
 * Adjoint, scatter form. Every product term of the forward map has the shape
 *   c * p * (q + r)
 * with c a coefficient and p, q, r field values; its partial derivatives are
 * c*(q+r) with respect to p and c*p with respect to q and to r. For each
 * output point and each term we add (sign * derivative * cotangent) to the
 * three cells it read. Single-threaded on purpose (scatter writes collide).
 */
static void term_adj(double g, double c, double *gp, double p, double *gq, double q,
                     double *gr, double r)
{
    double cg = c * g;
    *gp += cg * (q + r);
    *gq += cg * p;
    *gr += cg * p;
}

void pwo_advect_adjoint(int nx, int ny, int nz, long long sy, long long sz,
                        const double *u, const double *v, const double *w,
                        double tcx, double tcy,
                        const double *tzc1, const double *tzc2,
                        const double *tzd1, const double *tzd2,
                        const double *gsu, const double *gsv, const double *gsw,
                        double *gu, double *gv, double *gw)
{
    if (nx < 1 || ny < 1 || nz < 1) return;
#define G(f, k, j, i) (&AT(f, k, j, i))
    for (int i = 1; i <= nx; ++i) {
        for (int j = 1; j <= ny; ++j) {
            for (int k = 1; k < nz; ++k) {
                const int top = (k == nz - 1);
                double g;

                /* su */
                g = AT(gsu, k, j, i);
                term_adj(g, tcx, G(gu, k, j, i - 1), AT(u, k, j, i - 1),
                         G(gu, k, j, i), AT(u, k, j, i), G(gu, k, j, i - 1), AT(u, k, j, i - 1));
                term_adj(-g, tcx, G(gu, k, j, i + 1), AT(u, k, j, i + 1),
                         G(gu, k, j, i), AT(u, k, j, i), G(gu, k, j, i + 1), AT(u, k, j, i + 1));
                term_adj(g, tcy, G(gu, k, j - 1, i), AT(u, k, j - 1, i),
                         G(gv, k, j - 1, i), AT(v, k, j - 1, i), G(gv, k, j - 1, i + 1), AT(v, k, j - 1, i + 1));
                term_adj(-g, tcy, G(gu, k, j + 1, i), AT(u, k, j + 1, i),
                         G(gv, k, j, i), AT(v, k, j, i), G(gv, k, j, i + 1), AT(v, k, j, i + 1));
                term_adj(g, tzc1[k], G(gu, k - 1, j, i), AT(u, k - 1, j, i),
                         G(gw, k - 1, j, i), AT(w, k - 1, j, i), G(gw, k - 1, j, i + 1), AT(w, k - 1, j, i + 1));
                if (!top)
                    term_adj(-g, tzc2[k], G(gu, k + 1, j, i), AT(u, k + 1, j, i),
                             G(gw, k, j, i), AT(w, k, j, i), G(gw, k, j, i + 1), AT(w, k, j, i + 1));

                /* sv */
                g = AT(gsv, k, j, i);
                term_adj(g, tcy, G(gv, k, j - 1, i), AT(v, k, j - 1, i),
                         G(gv, k, j, i), AT(v, k, j, i), G(gv, k, j - 1, i), AT(v, k, j - 1, i));
                term_adj(-g, tcy, G(gv, k, j + 1, i), AT(v, k, j + 1, i),
                         G(gv, k, j, i), AT(v, k, j, i), G(gv, k, j + 1, i), AT(v, k, j + 1, i));
                term_adj(g, tcx, G(gv, k, j, i - 1), AT(v, k, j, i - 1),
                         G(gu, k, j, i - 1), AT(u, k, j, i - 1), G(gu, k, j + 1, i - 1), AT(u, k, j + 1, i - 1));
                term_adj(-g, tcx, G(gv, k, j, i + 1), AT(v, k, j, i + 1),
                         G(gu, k, j, i), AT(u, k, j, i), G(gu, k, j + 1, i), AT(u, k, j + 1, i));
                term_adj(g, tzc1[k], G(gv, k - 1, j, i), AT(v, k - 1, j, i),
                         G(gw, k - 1, j, i), AT(w, k - 1, j, i), G(gw, k - 1, j + 1, i), AT(w, k - 1, j + 1, i));
                if (!top)
                    term_adj(-g, tzc2[k], G(gv, k + 1, j, i), AT(v, k + 1, j, i),
                             G(gw, k, j, i), AT(w, k, j, i), G(gw, k, j + 1, i), AT(w, k, j + 1, i));

                /* sw */
                if (!top) {
                    g = AT(gsw, k, j, i);
                    term_adj(g, tcx, G(gw, k, j, i - 1), AT(w, k, j, i - 1),
                             G(gu, k, j, i - 1), AT(u, k, j, i - 1), G(gu, k + 1, j, i - 1), AT(u, k + 1, j, i - 1));
                    term_adj(-g, tcx, G(gw, k, j, i + 1), AT(w, k, j, i + 1),
                             G(gu, k, j, i), AT(u, k, j, i), G(gu, k + 1, j, i), AT(u, k + 1, j, i));
                    term_adj(g, tcy, G(gw, k, j - 1, i), AT(w, k, j - 1, i),
                             G(gv, k, j - 1, i), AT(v, k, j - 1, i), G(gv, k + 1, j - 1, i), AT(v, k + 1, j - 1, i));
                    term_adj(-g, tcy, G(gw, k, j + 1, i), AT(w, k, j + 1, i),
                             G(gv, k, j, i), AT(v, k, j, i), G(gv, k + 1, j, i), AT(v, k + 1, j, i));
                    term_adj(g, tzd1[k], G(gw, k - 1, j, i), AT(w, k - 1, j, i),
                             G(gw, k, j, i), AT(w, k, j, i), G(gw, k - 1, j, i), AT(w, k - 1, j, i));
                    term_adj(-g, tzd2[k], G(gw, k + 1, j, i), AT(w, k + 1, j, i),
                             G(gw, k, j, i), AT(w, k, j, i), G(gw, k + 1, j, i), AT(w, k + 1, j, i));
                }
            }
        }
    }
#undef G
}

long long pwo_flops_per_column(int nz)
{
    /* Sec. III: 21 operations per field and level, 63 per cell, 55 at the
     * column top; Listing 1 computes levels 2..nz. */
    if (nz < 2) return 0;
    return (long long)(nz - 2) * 63 + 55;
}
