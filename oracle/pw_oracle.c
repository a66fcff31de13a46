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
 *   - Sec. II-A: the PW scheme returns the source terms su, sv, sw of the
 *     three wind fields in flux form; Listing 1 prints su. Each term is
 *     computed here per direction as inflow through the lower face minus
 *     outflow through the upper face, a flux being the neighbour's value
 *     times the sum of the two velocity samples at the face, weighted by
 *     tcx, tcy or the vertical coefficients (see `gather` below), over
 *     k = 2..nz with the upper vertical face dropped at k = nz.
 *   - sv, sw: Sec. II-A says the scheme returns all three source terms, 21
 *     operations each (Sec. III), but prints only su. sv is su with the
 *     roles of x and y (u and v, tcx and tcy) exchanged; sw applies the same
 *     flux form to w on its own (w-level) grid. Both are readings, pinned by
 *     the tests (transpose identity, energy conservation, second-order
 *     convergence, closed forms).
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

/*
 * Forward map, written per face. Sec. II-A computes each source term in the
 * flux form of the Piacsek-Williams scheme: for every direction, what enters
 * through the lower face minus what leaves through the upper face. The
 * "flux" through a face is the advected field's value at the neighbour
 * across that face, q, times the sum a + b of the two velocity samples that
 * straddle the face (twice the advecting velocity there), weighted by the
 * direction's coefficient. Listing 1 prints this for su; sv is the same with
 * x and y exchanged, and sw applies it on the w grid (horizontal advecting
 * velocities are the sums of u or v at the two u-levels around w level k).
 */
typedef struct {
    double q, a, b;  /* neighbour value; the two velocity samples at the face */
} face;

typedef struct {
    face lo, hi;        /* lower (inflow) and upper (outflow) face */
    double c_lo, c_hi;  /* their coefficients */
    int horizontal;     /* one coefficient for both faces (tcx or tcy) */
    int hi_on;          /* 0 where the scheme drops the upper face */
} direction;

static double flux(face f) { return f.q * (f.a + f.b); }

/* The value of one direction: c (F_lo - F_hi) horizontally, as Listing 1
 * groups it; c_lo F_lo - c_hi F_hi vertically. */
static double dir_value(const direction *d)
{
    if (d->horizontal) return d->c_lo * (flux(d->lo) - flux(d->hi));
    if (d->hi_on) return d->c_lo * flux(d->lo) - d->c_hi * flux(d->hi);
    return d->c_lo * flux(d->lo);
}

/* Error scales of one direction. strict: |c| |q| |a + b| per face, the sum
 * of the absolute values of the products the formula adds up. monomial:
 * |c| |q| (|a| + |b|) per face, the same with each product expanded into
 * its two monomials c q a and c q b. */
static double dir_scale(const direction *d, int monomial)
{
    double lo = monomial ? absd(d->lo.a) + absd(d->lo.b) : absd(d->lo.a + d->lo.b);
    double hi = monomial ? absd(d->hi.a) + absd(d->hi.b) : absd(d->hi.a + d->hi.b);
    double s = absd(d->c_lo) * absd(d->lo.q) * lo;
    if (d->hi_on) s += absd(d->c_hi) * absd(d->hi.q) * hi;
    return s;
}

static face mkface(double q, double a, double b)
{
    face f;
    f.q = q;
    f.a = a;
    f.b = b;
    return f;
}

static direction mkdir(face lo, face hi, double c_lo, double c_hi, int horizontal, int hi_on)
{
    direction d;
    d.lo = lo;
    d.hi = hi;
    d.c_lo = c_lo;
    d.c_hi = c_hi;
    d.horizontal = horizontal;
    d.hi_on = hi_on;
    return d;
}

/* The three directions of su, sv and sw at (k, j, i), k = 1 .. nz-1 (sw:
 * k = 1 .. nz-2). dirs[0] is the output's own direction (x for su and sw, y
 * for sv), so that sv is evaluated in the mirror order of su. */
enum { OUT_SU = 0, OUT_SV = 1, OUT_SW = 2 };

static void gather(int out, int k, int j, int i, int nz, long long sy, long long sz,
                   const double *u, const double *v, const double *w,
                   double tcx, double tcy, const double *tzc1, const double *tzc2,
                   const double *tzd1, const double *tzd2, direction dirs[3])
{
    const int top = (k == nz - 1);
    if (out == OUT_SU) {
        /* x: u advected by u; y: u advected by v at the two faces j-1/2,
         * j+1/2 of the u point; z: u advected by w at the faces below and
         * above (dropped at the top level). */
        dirs[0] = mkdir(mkface(AT(u, k, j, i - 1), AT(u, k, j, i - 1), AT(u, k, j, i)),
                        mkface(AT(u, k, j, i + 1), AT(u, k, j, i), AT(u, k, j, i + 1)), tcx, tcx, 1, 1);
        dirs[1] = mkdir(mkface(AT(u, k, j - 1, i), AT(v, k, j - 1, i), AT(v, k, j - 1, i + 1)),
                        mkface(AT(u, k, j + 1, i), AT(v, k, j, i), AT(v, k, j, i + 1)), tcy, tcy, 1, 1);
        dirs[2] = mkdir(mkface(AT(u, k - 1, j, i), AT(w, k - 1, j, i), AT(w, k - 1, j, i + 1)),
                        mkface(top ? 0.0 : AT(u, k + 1, j, i), AT(w, k, j, i), AT(w, k, j, i + 1)),
                        tzc1[k], tzc2[k], 0, !top);
    } else if (out == OUT_SV) {
        dirs[0] = mkdir(mkface(AT(v, k, j - 1, i), AT(v, k, j - 1, i), AT(v, k, j, i)),
                        mkface(AT(v, k, j + 1, i), AT(v, k, j, i), AT(v, k, j + 1, i)), tcy, tcy, 1, 1);
        dirs[1] = mkdir(mkface(AT(v, k, j, i - 1), AT(u, k, j, i - 1), AT(u, k, j + 1, i - 1)),
                        mkface(AT(v, k, j, i + 1), AT(u, k, j, i), AT(u, k, j + 1, i)), tcx, tcx, 1, 1);
        dirs[2] = mkdir(mkface(AT(v, k - 1, j, i), AT(w, k - 1, j, i), AT(w, k - 1, j + 1, i)),
                        mkface(top ? 0.0 : AT(v, k + 1, j, i), AT(w, k, j, i), AT(w, k, j + 1, i)),
                        tzc1[k], tzc2[k], 0, !top);
    } else {
        dirs[0] = mkdir(mkface(AT(w, k, j, i - 1), AT(u, k, j, i - 1), AT(u, k + 1, j, i - 1)),
                        mkface(AT(w, k, j, i + 1), AT(u, k, j, i), AT(u, k + 1, j, i)), tcx, tcx, 1, 1);
        dirs[1] = mkdir(mkface(AT(w, k, j - 1, i), AT(v, k, j - 1, i), AT(v, k + 1, j - 1, i)),
                        mkface(AT(w, k, j + 1, i), AT(v, k, j, i), AT(v, k + 1, j, i)), tcy, tcy, 1, 1);
        dirs[2] = mkdir(mkface(AT(w, k - 1, j, i), AT(w, k - 1, j, i), AT(w, k, j, i)),
                        mkface(AT(w, k + 1, j, i), AT(w, k, j, i), AT(w, k + 1, j, i)),
                        tzd1[k], tzd2[k], 0, 1);
    }
}

/* Walk every interior point; per output: value (s != NULL) and error scale
 * (a != NULL; monomial selects the scale). Level 1 and sw at level nz are 0. */
static void walk(int nx, int ny, int nz, long long sy, long long sz,
                 const double *u, const double *v, const double *w,
                 double tcx, double tcy, const double *tzc1, const double *tzc2,
                 const double *tzd1, const double *tzd2,
                 double *const s[3], double *const a[3], int monomial, int nthreads)
{
    if (nx < 1 || ny < 1 || nz < 1) return;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int i = 1; i <= nx; ++i) {
        for (int j = 1; j <= ny; ++j) {
            for (int o = 0; o < 3; ++o) {
                if (s[o]) AT(s[o], 0, j, i) = 0.0;
                if (a[o]) AT(a[o], 0, j, i) = 0.0;
            }
            for (int k = 1; k < nz; ++k) {
                for (int o = 0; o < 3; ++o) {
                    if (!s[o] && !a[o]) continue;
                    if (o == OUT_SW && k == nz - 1) { /* rigid lid */
                        if (s[o]) AT(s[o], k, j, i) = 0.0;
                        if (a[o]) AT(a[o], k, j, i) = 0.0;
                        continue;
                    }
                    direction d[3];
                    gather(o, k, j, i, nz, sy, sz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, d);
                    if (s[o]) {
                        double t = dir_value(&d[0]);
                        t = t + dir_value(&d[1]);
                        t = t + dir_value(&d[2]);
                        AT(s[o], k, j, i) = t;
                    }
                    if (a[o]) AT(a[o], k, j, i) = dir_scale(&d[0], monomial) + dir_scale(&d[1], monomial)
                                                  + dir_scale(&d[2], monomial);
                }
            }
        }
    }
}

void pwo_advect(int nx, int ny, int nz, long long sy, long long sz,
                const double *u, const double *v, const double *w,
                double tcx, double tcy,
                const double *tzc1, const double *tzc2,
                const double *tzd1, const double *tzd2,
                double *su, double *sv, double *sw,
                double *asu, double *asv, double *asw, int nthreads)
{
    double *const s[3] = {su, sv, sw};
    double *const a[3] = {asu, asv, asw};
    walk(nx, ny, nz, sy, sz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, s, a, 0, nthreads);
}

void pwo_monomial_scale(int nx, int ny, int nz, long long sy, long long sz,
                        const double *u, const double *v, const double *w,
                        double tcx, double tcy,
                        const double *tzc1, const double *tzc2,
                        const double *tzd1, const double *tzd2,
                        double *msu, double *msv, double *msw, int nthreads)
{
    double *const s[3] = {NULL, NULL, NULL};
    double *const a[3] = {msu, msv, msw};
    walk(nx, ny, nz, sy, sz, u, v, w, tcx, tcy, tzc1, tzc2, tzd1, tzd2, s, a, 1, nthreads);
}

/*
 * Energy weights. The flux form conserves the discrete kinetic energy of
 * each wind component when the domain is periodic in x and y and w = 0 on
 * the ground and at the lid: the fluxes through a face enter the budgets of
 * the two cells that share it with opposite signs, once each cell's
 * tendency is weighted by its mass, so the weighted sums telescope to 0.
 * Mass of a u or v cell at level k: dz(k) rhon(k); of a w cell: dzn(k)
 * rho(k), with dzn(k) = zn(k+1) - zn(k) as in pwo_coeffs (0 at levels 1
 * and nz, where nothing is computed).
 */
int pwo_energy_weights(int nz, const double *dz, const double *rho, const double *rhon,
                       double *wu, double *ww)
{
    if (nz < 1 || dz == NULL || wu == NULL || ww == NULL) return -1;
    double *z = (double *)malloc(sizeof(double) * (size_t)nz);
    double *zn = (double *)malloc(sizeof(double) * (size_t)nz);
    if (!z || !zn) { free(z); free(zn); return -1; }
    z[0] = 0.0;
    for (int k = 1; k < nz; ++k) z[k] = z[k - 1] + dz[k];
    for (int k = 1; k < nz; ++k) zn[k] = 0.5 * (z[k - 1] + z[k]);
    zn[0] = (nz > 1) ? -zn[1] : 0.0;
    for (int k = 0; k < nz; ++k) {
        wu[k] = 0.0;
        ww[k] = 0.0;
    }
    for (int k = 1; k < nz; ++k) wu[k] = dz[k] * (rhon ? rhon[k] : 1.0);
    for (int k = 1; k < nz - 1; ++k) ww[k] = (zn[k + 1] - zn[k]) * (rho ? rho[k] : 1.0);
    free(z);
    free(zn);
    return 0;
}

/*
 * Energy budget: out[0..2] = sum over the interior of wu(k) u su, wu(k) v sv
 * and ww(k) w sw; out[3..5] = the same sums of absolute values. Levels in
 * order, rows in order, columns in order. Each sum is accumulated with
 * Neumaier's compensated summation (Kahan's method with the Babuska /
 * Neumaier branch on magnitudes), so its error stays near one rounding of
 * the result whatever the number of summands.
 */
typedef struct {
    double s, c;  /* running sum and its compensation */
} csum;

static void csum_add(csum *a, double x)
{
    const double t = a->s + x;
    if (absd(a->s) >= absd(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

void pwo_energy_budget(int nx, int ny, int nz, long long sy, long long sz,
                       const double *u, const double *v, const double *w,
                       const double *su, const double *sv, const double *sw,
                       const double *wu, const double *ww, double *out)
{
    csum acc[6];
    for (int n = 0; n < 6; ++n) {
        acc[n].s = 0.0;
        acc[n].c = 0.0;
    }
    for (int k = 0; k < nz; ++k) {
        for (int j = 1; j <= ny; ++j) {
            for (int i = 1; i <= nx; ++i) {
                const double eu = wu[k] * AT(u, k, j, i) * AT(su, k, j, i);
                const double ev = wu[k] * AT(v, k, j, i) * AT(sv, k, j, i);
                const double ew = ww[k] * AT(w, k, j, i) * AT(sw, k, j, i);
                csum_add(&acc[0], eu);
                csum_add(&acc[1], ev);
                csum_add(&acc[2], ew);
                csum_add(&acc[3], absd(eu));
                csum_add(&acc[4], absd(ev));
                csum_add(&acc[5], absd(ew));
            }
        }
    }
    for (int n = 0; n < 6; ++n) out[n] = acc[n].s + acc[n].c;
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
