/*
 * pw.h -- C ABI of the GB300 Piacsek-Williams (PW) advection library.
 *
 * The library computes the PW advection source terms (su, sv, sw) of the
 * staggered Arakawa-C winds (u, v, w) on sm_103a GPUs. Paper: N. Brown,
 * "Accelerating advection for atmospheric modelling on Xilinx and Intel
 * FPGAs", arXiv:2107.13500; the su stencil is its Listing 1 (Sec. II-A),
 * the operation count its Sec. III.
 *
 * Conventions for every entry point:
 *  - Layout. A field of an nx x ny x nz domain is stored x fastest as
 *    f[k*sz + j*sy + i] with i = 0..nx+1, j = 0..ny+1 (0 and n+1 are a
 *    one-cell halo) and k = 0..nz-1 (the paper's level k+1; no vertical
 *    halo). sy >= nx+2 and sz >= sy*(ny+2) are element strides that must
 *    be multiples of 16 bytes (TMA tile loads); rows padded to 32 bytes
 *    satisfy this. Device buffers must be aligned to their element size, and
 *    u, v, w must have the same address modulo 16 bytes. When the interior
 *    cell i = 1 of all six fields starts on a 16-byte boundary (base address
 *    = 16n - element size) the kernels use 16-byte vector accesses; any
 *    other element-aligned layout takes an equivalent scalar path.
 *  - Ownership. The caller owns every buffer. The library allocates no
 *    device memory on any compute path.
 *  - Asynchrony. Compute calls enqueue work on `stream` (a cudaStream_t;
 *    NULL = the legacy default stream) and return before it finishes.
 *  - Outputs. Only interior cells (i = 1..nx, j = 1..ny, all k) are written;
 *    output halo cells are never touched. Outputs may not overlap inputs or
 *    each other.
 *  - Inputs. Halo cells of inputs must hold valid values (periodic copies
 *    from pw_fill_periodic_halo, or boundary data the caller supplies).
 *  - Errors. Every call returns PW_OK (0) or a negative PW_E* code, and
 *    pw_last_error() returns a message for the last failure in the calling
 *    thread. A failed validation enqueues nothing.
 */
#ifndef PW_H
#define PW_H

#ifdef __cplusplus
extern "C" {
#endif

#define PW_OK 0
#define PW_EINVAL (-1)        /* bad size, halo, stride, alignment or option */
#define PW_ENULL (-2)         /* a required pointer is NULL */
#define PW_EALIAS (-3)        /* an output overlaps an input or another output */
#define PW_EUNSUPPORTED (-4)  /* dtype/operation combination not provided */
#define PW_ECUDA (-5)         /* a CUDA runtime or driver call failed */
#define PW_ETIMEOUT (-6)      /* a kernel's bounded wait expired (see pw_device_status) */

typedef enum {
    PW_F64 = 0,        /* double in, double out, native FP64 arithmetic */
    PW_F32_SPLIT = 1,  /* float perturbations about per-level means, FP32 arithmetic */
    PW_F64_PAIRED = 2, /* double in, double out, paired-FP32 (double-float) arithmetic */
    PW_F32 = 3         /* float in, float out, FP32 arithmetic on the full fields */
} pw_dtype;

/* Domain shape and strides (elements). halo must be 1. */
typedef struct {
    int nx, ny, nz, halo;
    long long sy, sz;
} pw_dims;

/* Stencil coefficients of Listing 1 and its companions: tcx, tcy (host
 * scalars) and four DEVICE arrays of length nz (level k at index k-1):
 * tzc1/tzc2 weight the lower/upper vertical flux of su and sv, tzd1/tzd2
 * those of sw. pw_make_coeffs fills them on the host. */
typedef struct {
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
} pw_coeffs;

/* Number of floats per level in the PW_F32_SPLIT table (see pw_make_split_table). */
#define PW_SPLIT_NCOEF 32

/*
 * pw_make_coeffs -- host FP64 coefficients (no GPU work).
 *   tc2_host[0] = tcx = 0.25/dx, tc2_host[1] = tcy = 0.25/dy.
 *   tz4_host (4*nz doubles) = tzc1 | tzc2 | tzd1 | tzd2, each nz long:
 *     z(1) = 0, z(k) = z(k-1) + dz(k); zn(k) = (z(k-1)+z(k))/2, zn(1) = -zn(2);
 *     dzn(k) = zn(k+1) - zn(k);
 *     tzc1(k) = 0.25 rho(k-1)/(rhon(k) dz(k)),  tzc2(k) = 0.25 rho(k)/(rhon(k) dz(k));
 *     tzd1(k) = 0.25 rhon(k)/(rho(k) dzn(k)),   tzd2(k) = 0.25 rhon(k+1)/(rho(k) dzn(k));
 *   unused entries (tzc at level 1, tzd at levels 1 and nz) are 0.
 * The paper uses these coefficients in Listing 1 without defining them;
 * this is the flux-form reading on a stretched, density-weighted grid.
 * dz: host, nz entries (dz[0] unused). rho (w levels) and rhon (u levels):
 * host, nz entries, or NULL for 1. Errors: PW_ENULL, PW_EINVAL (nz < 1,
 * dx, dy or dz(k>=2) not > 0).
 */
int pw_make_coeffs(int nz, double dx, double dy, const double *dz, const double *rho,
                   const double *rhon, double *tc2_host, double *tz4_host);

/*
 * pw_fill_periodic_halo -- make a field periodic in x and y on the device:
 * copies column nx into column 0 and column 1 into column nx+1 (every row),
 * then row ny into row 0 and row 1 into row ny+1 (every column, so corners
 * follow). dtype selects the element size (PW_F32_SPLIT = float, else
 * double). Errors: PW_ENULL, PW_EINVAL, PW_ECUDA.
 */
int pw_fill_periodic_halo(pw_dtype dtype, void *field, const pw_dims *dims, void *stream);

/*
 * pw_advect -- the source terms of Listing 1 (su) and its two companions.
 * For every interior column (i, j):
 *   level 1: su = sv = sw = 0 (Listing 1 starts at k = 2);
 *   k = 2..nz:
 *     su = tcx[u(i-1)(u(i)+u(i-1)) - u(i+1)(u(i)+u(i+1))]
 *        + tcy[u(j-1)(v(j-1,i)+v(j-1,i+1)) - u(j+1)(v(j,i)+v(j,i+1))]
 *        + tzc1(k) u(k-1)(w(k-1,i)+w(k-1,i+1)) - [k<nz] tzc2(k) u(k+1)(w(k,i)+w(k,i+1))
 *     sv = the same with x and y exchanged (u<->v, tcx<->tcy, i<->j);
 *   k = 2..nz-1:
 *     sw = tcx[w(i-1)(u(k,i-1)+u(k+1,i-1)) - w(i+1)(u(k,i)+u(k+1,i))]
 *        + tcy[w(j-1)(v(k,j-1)+v(k+1,j-1)) - w(j+1)(v(k,j)+v(k+1,j))]
 *        + tzd1(k) w(k-1)(w(k)+w(k-1)) - tzd2(k) w(k+1)(w(k)+w(k+1));
 *   k = nz: sw = 0 (rigid lid).
 * Unlisted indices are (k, j, i). All of u, v, w, su, sv, sw share `dims`.
 *
 * dtype PW_F64 / PW_F64_PAIRED: u, v, w, su, sv, sw are double; split must
 *   be NULL. Error scales at a point: A = sum over the face terms c*q*(a+b)
 *   of |c||q||a+b| (the absolute values of the products the formula adds);
 *   M = the same with |a|+|b| in place of |a+b| (M >= A).
 *   PW_F64 computes in FP64, each operation rounded once (u and v are scaled
 *   by tcx and tcy once per cell, then every face sum is formed once and
 *   shared); its error is a few units of 2^-53 of M, within 1e-13 of A.
 *   PW_F64_PAIRED carries every value as an unevaluated sum of two floats
 *   (about 48 significant bits); each double is split into a pair before
 *   a + b is formed, so its error is bounded by M: within 1e-13 of M at
 *   every point and 1e-13 of max|su| normwise. Float pairs have FP32's
 *   exponent range: the bound holds while every input lies in
 *   [2^-74, 2^120] (or is 0) and every product c*q*a of the formula in
 *   [2^-100, 2^120] (tested with the winds scaled by 2^-40 and 2^40).
 * dtype PW_F32_SPLIT: u, v, w are float perturbations u' = u - U(k) about
 *   per-level means, su, sv, sw are float, and `split` is a DEVICE table of
 *   PW_SPLIT_NCOEF*nz floats built by pw_make_split_table (the coefficient
 *   arrays in `c` are then not read, but c must still be non-NULL).
 * dtype PW_F32: u, v, w, su, sv, sw are float full fields; `split` is the
 *   table of pw_make_split_table built with all means 0 (it then carries
 *   only the coefficients, rounded to float).
 * Errors: PW_ENULL, PW_EINVAL, PW_EALIAS, PW_EUNSUPPORTED, PW_ECUDA.
 */
int pw_advect(pw_dtype dtype, const void *u, const void *v, const void *w, const pw_coeffs *c,
              const pw_dims *dims, const void *split, void *su, void *sv, void *sw, void *stream);

/*
 * pw_make_split_table -- host FP64 set-up for PW_F32_SPLIT (no GPU work).
 * Given tcx, tcy, tz4_host (as from pw_make_coeffs) and the per-level means
 * ubar, vbar, wbar (host, nz doubles each), writes table_host
 * (PW_SPLIT_NCOEF*nz floats, level-major: entry m of level k at k*NCOEF+m).
 * Writing u = U(k) + u' (likewise v, w), every mean x mean product of a
 * horizontal flux difference cancels exactly, and each vertical flux
 * difference leaves a per-level constant that is formed here in FP64 and
 * rounded to float once; the remaining terms are linear or quadratic in the
 * perturbations. Errors: PW_ENULL, PW_EINVAL.
 */
int pw_make_split_table(int nz, double tcx, double tcy, const double *tz4_host,
                        const double *ubar, const double *vbar, const double *wbar,
                        float *table_host);

/*
 * pw_split_field -- per-level mean and float perturbation of a double field
 * on the device: mean[k] = average of f over the interior of level k, and
 * fp = float(f - mean[k]) on every cell of the level including the halo
 * (the FP64 difference rounded to nearest even, bit for bit the hardware's
 * conversion). The means are summed in a fixed order, so they repeat from
 * call to call: in bands of 16 rows, part of each band in FP64 and the rest
 * in paired FP32 (about 48 significant bits; error at most a few hundred
 * units of 2^-48 of the mean magnitude), when the pair-summed values and the
 * FP64 parts are 0 or lie in [2^-60, 2^100); else the level in FP64. The
 * band sums pass through cells of fp before fp is written. Any value near the
 * average serves the split, since pw_make_split_table and the
 * perturbations use the same stored mean. f uses dims_f (double), fp uses
 * dims_p (float; same nx, ny, nz). mean is a DEVICE array of nz doubles.
 * Errors: PW_ENULL, PW_EINVAL, PW_EALIAS, PW_ECUDA.
 */
int pw_split_field(const double *f, const pw_dims *dims_f, float *fp, const pw_dims *dims_p,
                   double *mean, void *stream);

/*
 * pw_advect_adjoint -- transpose of the Jacobian of pw_advect at (u, v, w)
 * applied to cotangents (gsu, gsv, gsw): the gradient a scalar J(su, sv, sw)
 * passes back to the winds, as used in variational data assimilation. The
 * forward map is quadratic (Listing 1 and its companions are sums of
 * c*p*(q+r)), so d/dp = c*(q+r) and d/dq = d/dr = c*p; each cell gathers
 * those derivatives times the cotangents of every output point that read it
 * (no atomics). Only the computed cotangents count: the halo cells of gsu,
 * gsv, gsw, their level 1, and level nz of gsw are ignored (read as 0).
 * Results cover every cell the forward map reads, halo included
 * (i = 0..nx+1, j = 0..ny+1, all k); accumulate != 0 adds them to gu, gv, gw,
 * otherwise they overwrite. Cells beyond i = nx+1 (row padding) are not
 * touched. dtype PW_F64 (double, native FP64), PW_F64_PAIRED (double,
 * paired-FP32 arithmetic as in pw_advect, within 1e-13 of native FP64) or
 * PW_F32 (float). All nine
 * fields share `dims`; u, v, w, gsu, gsv, gsw must have the same address
 * modulo 16 bytes. Errors: PW_ENULL, PW_EINVAL, PW_EALIAS, PW_EUNSUPPORTED,
 * PW_ECUDA.
 */
int pw_advect_adjoint(pw_dtype dtype, const void *u, const void *v, const void *w, const pw_coeffs *c,
                      const pw_dims *dims, const void *gsu, const void *gsv, const void *gsw, void *gu, void *gv,
                      void *gw, int accumulate, void *stream);

/*
 * pw_fold_periodic_halo -- transpose of pw_fill_periodic_halo: adds row 0
 * into row ny and row ny+1 into row 1 (every column), then column 0 into
 * column nx and column nx+1 into column 1 (rows 1..ny), zeroing the halo.
 * Turns a gradient over all cells of a periodic field into the gradient over
 * its interior. dtype selects the element size (PW_F32_SPLIT and PW_F32 =
 * float, else double). Errors: PW_ENULL, PW_EINVAL, PW_ECUDA.
 */
int pw_fold_periodic_halo(pw_dtype dtype, void *field, const pw_dims *dims, void *stream);

/*
 * pw_advect_host_chunked -- pw_advect on fields that live in (pinned) host
 * memory, with the transfers overlapped with the computation (the paper's
 * Sec. IV chunking of host<->device traffic, here in slabs of levels). The
 * levels are cut into nchunks slabs; for each slab, in order, its level
 * planes of u, v, w go host->device on stream_h2d (one contiguous copy per
 * field), its levels are computed on stream_compute (once the next slab,
 * which holds their upper neighbour level, has landed), and rows 1..ny of
 * its output levels go device->host on stream_d2h (one 2-D copy per field,
 * a row of ny*sy elements per level). Host and device fields share `dims`
 * (same strides); u_d..sw_d are caller-owned device buffers of the full
 * size. dtype and split as for pw_advect. Returns after enqueueing; the
 * outputs are in host memory once stream_d2h reaches its end. The host
 * outputs' halo rows 0 and ny+1 are not written; their halo columns in rows
 * 1..ny receive what the device outputs hold there (pw_advect never writes
 * them). nchunks is clamped to [1, nz]. Errors: as pw_advect, plus
 * PW_ECUDA from copies and events.
 */
int pw_advect_host_chunked(pw_dtype dtype, const void *u_h, const void *v_h, const void *w_h, void *su_h,
                           void *sv_h, void *sw_h, void *u_d, void *v_d, void *w_d, void *su_d, void *sv_d,
                           void *sw_d, const pw_coeffs *c, const pw_dims *dims, const void *split, int nchunks,
                           void *stream_h2d, void *stream_compute, void *stream_d2h);

/*
 * Batched evaluation: many independent domains of uneven sizes in ONE
 * persistent launch. Every CTA of the launch takes work items (one tile of
 * one domain) from an atomic counter until none are left, so small and
 * large domains share the GPU without a tail per domain.
 */
typedef struct {
    const void *u, *v, *w;  /* inputs (device) */
    void *su, *sv, *sw;     /* outputs (device) */
    pw_dims dims;
    pw_coeffs coeffs;       /* device coefficient arrays of this domain */
    const void *split;      /* PW_F32 / PW_F32_SPLIT: this domain's device table; else NULL */
} pw_domain;

/* Bytes of a batch plan for n domains (host and device copies alike). */
size_t pw_batch_plan_bytes(int n);

/* Number of kernel variants (tile shape x pipeline depth) for dtype; variant
 * indices 0 .. count-1 are accepted by pw_make_batch_plan, 0 is the default.
 * PW_F32 / PW_F32_SPLIT (points per CTA, TMA ring depth): 0 = 128x4, 4 levels;
 * 1 = 64x4; 2 = 32x8; 3 = 64x8; 4 = 32x16; 5 = 128x2 (all 4 levels);
 * 6 = 64x4, 3 levels; 7 = 64x4, 6 levels.
 * PW_F64_PAIRED: 0 = 32x8, 2 levels; 1 = 32x4; 2 = 32x16 (2 levels);
 * 3 = 32x8, 3 levels. PW_F64: 0 = 32x16, 1 = 32x8 (4-level rings). */
int pw_variant_count(pw_dtype dtype);

/*
 * pw_make_batch_plan -- host-only set-up of a batch (no GPU work, no
 * allocation): validates every domain as pw_advect would, encodes its TMA
 * descriptors and lays out the plan in plan_host (plan_bytes >=
 * pw_batch_plan_bytes(n)). Domains are ordered tallest first. *n_items
 * receives the number of work items. The caller copies the plan to a device
 * buffer (64-byte aligned) and passes it to pw_advect_batched; the device
 * buffer is also the kernel's work-queue scratch. Any dtype. Errors:
 * PW_ENULL, PW_EINVAL, PW_EALIAS, PW_EUNSUPPORTED, PW_ECUDA (descriptor
 * encoding).
 */
int pw_make_batch_plan(pw_dtype dtype, int n, const pw_domain *doms, int variant, void *plan_host,
                       size_t plan_bytes, long long *n_items);

/*
 * pw_advect_batched -- evaluate every domain of a plan: resets the plan's
 * work counter on `stream`, then launches one persistent kernel (CTAs = SMs x
 * resident CTAs per SM, at most n_items). dtype and variant must be those the
 * plan was built with (a mismatch is reported by pw_device_status as
 * PW_EINVAL, outputs unspecified). Launches on the same plan must not overlap
 * on the GPU (they share its counter). Capturable in a CUDA graph (the
 * counter reset is a memset node). Any dtype.
 * Errors: PW_ENULL, PW_EINVAL, PW_EUNSUPPORTED, PW_ECUDA.
 */
int pw_advect_batched(pw_dtype dtype, int variant, void *plan_dev, long long n_items, void *stream);

/*
 * pw_advect_batched_noalloc -- pw_advect_batched for callers that cannot
 * allocate device memory. (The paper has no counterpart: this is a property
 * of the library, not of the method.) pw_advect_batched needs the batch plan
 * in a device buffer the caller allocates. Some callers cannot make one:
 * real-time loops that must not call cudaMalloc (it can synchronise the
 * device and its latency is unbounded), plug-ins that run inside a host
 * program which owns every device allocation, and programs whose device
 * memory is wholly reserved by another allocator. This entry point takes the
 * HOST plan from pw_make_batch_plan instead and copies it, on `stream`, into
 * a fixed device array inside the library (room for PW_NOALLOC_MAX_DOMAINS
 * domains, about 150 KB, which every GPU that loads the library holds until
 * the process exits), zeroes the work counter there and launches the same
 * persistent kernel. It calls no cudaMalloc, cudaFree or allocating library
 * routine. The first call on a device looks up the array's address on that
 * device, with the device current; make that first call before any stream
 * capture. plan_host may be pageable (the copy is staged before the call
 * returns) or pinned (then it must stay unchanged until the copy has run on
 * `stream`). Every call on a device shares the one array: calls whose work
 * overlaps on the GPU race and produce unspecified results, so order them
 * (same stream, or events). Plans with more than PW_NOALLOC_MAX_DOMAINS
 * domains are rejected with PW_EINVAL. dtype PW_F64_PAIRED, PW_F32 or
 * PW_F32_SPLIT. Its own errors are reported through pw_noalloc_last_error.
 * Errors: PW_ENULL, PW_EINVAL, PW_EUNSUPPORTED, PW_ECUDA.
 */
#define PW_NOALLOC_MAX_DOMAINS 256
int pw_advect_batched_noalloc(pw_dtype dtype, int variant, const void *plan_host, size_t plan_bytes,
                              long long n_items, void *stream);

/* Message for the last failure of pw_advect_batched_noalloc in this thread. */
const char *pw_noalloc_last_error(void);

/*
 * pw_make_energy_weights -- host masses of the energy budget (no GPU work).
 * wu_host[k] = dz(k) rhon(k), the mass of the u and v cells of level k;
 * ww_host[k] = dzn(k) rho(k), the mass of the w cell around w level k, with
 * dzn as in pw_make_coeffs; 0 at the levels nothing is computed on (wu at
 * level 1, ww at levels 1 and nz). dz, rho, rhon as for pw_make_coeffs.
 * Errors: PW_ENULL, PW_EINVAL.
 */
int pw_make_energy_weights(int nz, const double *dz, const double *rho, const double *rhon, double *wu_host,
                           double *ww_host);

/*
 * pw_energy_budget -- FP64 conservation diagnostic of a set of source
 * terms. The paper accelerates the Piacsek-Williams scheme (Sec. I) in the
 * flux form of Listing 1: on a domain periodic in x and y with w = 0 on the
 * ground and at the lid, the flux through each face enters the two cells
 * that share it with opposite signs, so the mass-weighted energy tendencies
 *   sum wu(k) u su,  sum wu(k) v sv,  sum ww(k) w sw   (over the interior)
 * vanish in exact arithmetic. This call measures how far a path's rounding
 * moves them from 0. level_sums (DEVICE, 6*nz doubles) receives per level k
 * the interior sums [u su, v sv, w sw, |u su|, |v sv|, |w sw|] (unweighted);
 * totals (DEVICE, 6 doubles) the same weighted by wu (u, v) and ww (w) and
 * added over the levels in order. All arithmetic is FP64 in a fixed order,
 * so the result is repeatable. Winds (u, v, w; layout dims_wind) and
 * tendencies (su, sv, sw; layout dims_tend, same nx, ny, nz) are each float
 * or double (elem_bytes 4 or 8), e.g. the FP64 winds and the float source
 * terms of the PW_F32_SPLIT path. wu, ww: DEVICE arrays of nz doubles (from
 * pw_make_energy_weights). Asynchronous on `stream`; nz <= 65535.
 * Errors: PW_ENULL, PW_EINVAL, PW_EALIAS, PW_ECUDA.
 */
int pw_energy_budget(const void *u, const void *v, const void *w, int wind_elem_bytes, const pw_dims *dims_wind,
                     const void *su, const void *sv, const void *sw, int tend_elem_bytes, const pw_dims *dims_tend,
                     const double *wu, const double *ww, double *level_sums, double *totals, void *stream);

/*
 * pw_device_status -- read and clear the library's device error word on the
 * current device (synchronises `stream`). *status receives 0, PW_ETIMEOUT if
 * a kernel gave up on a bounded wait since the last call, or PW_EINVAL if a
 * batched launch met a plan built for another dtype or variant (outputs of
 * those launches are unspecified). Errors: PW_ENULL, PW_ECUDA.
 */
int pw_device_status(int *status, void *stream);

/*
 * pw_selftest_bounded_wait -- exercises the failure path of the bounded
 * waits every kernel of the library uses: one thread waits on a barrier
 * that nothing ever completes and must give up after limit_us microseconds
 * (1..100000), record a timeout and return, leaving the device usable.
 * Clears the status word first, then stores in *status what
 * pw_device_status reports afterwards (PW_ETIMEOUT when the bound works).
 * Synchronises `stream`. Errors: PW_ENULL, PW_EINVAL, PW_ECUDA.
 */
int pw_selftest_bounded_wait(unsigned int limit_us, int *status, void *stream);

/* Message for the last failing call in this thread ("" if none). */
const char *pw_last_error(void);

/* Library version string. */
const char *pw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PW_H */
