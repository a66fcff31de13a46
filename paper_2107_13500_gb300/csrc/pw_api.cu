// pw_api.cu -- the C ABI declared in include/pw.h: argument validation, TMA
// descriptor set-up, dispatch to the kernels, host-side coefficient tables.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "pw.h"
#include "pw_internal.h"

namespace {

thread_local std::string t_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(PW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- TMA maps

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn(cudaError_t* err) {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        status = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (status == cudaSuccess && q != cudaDriverEntryPointSuccess) status = cudaErrorSymbolNotFound;
        fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    *err = status;
    return fn;
}

// The descriptor starts at the 16-byte boundary at or below the field's base
// pointer; x coordinates of the tensor are i + xoff, xoff = elements between.
int make_field_map(CUtensorMap* map, const void* base, int elem_bytes, const pw_dims& d, int box_x, int box_y) {
    cudaError_t e;
    EncodeTiledFn enc = get_encode_fn(&e);
    if (!enc) return cuda_fail(e, "cuTensorMapEncodeTiled lookup");
    const int xoff = (int)(((uintptr_t)base % 16) / elem_bytes);
    base = static_cast<const char*>(base) - (size_t)xoff * elem_bytes;
    cuuint64_t gdim[3] = {(cuuint64_t)(d.nx + 2 + xoff), (cuuint64_t)(d.ny + 2), (cuuint64_t)d.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)d.sy * elem_bytes, (cuuint64_t)d.sz * elem_bytes};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
    cuuint32_t estride[3] = {1u, 1u, 1u};
    CUresult r = enc(map, elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     const_cast<void*>(base), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PW_ECUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return PW_OK;
}

// ---------------------------------------------------------------- validation

int check_dims(const pw_dims* d, int elem_bytes, const char* who) {
    if (!d) return fail(PW_ENULL, "%s: dims is NULL", who);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return fail(PW_EINVAL, "%s: nx, ny, nz must be >= 1 (got %d, %d, %d)", who, d->nx, d->ny, d->nz);
    if (d->halo != 1) return fail(PW_EINVAL, "%s: halo must be 1 (got %d)", who, d->halo);
    if (d->nx > (1 << 30) || d->ny > (1 << 30) || d->nz > (1 << 30))
        return fail(PW_EINVAL, "%s: extent too large", who);
    if (d->sy < (long long)d->nx + 2)
        return fail(PW_EINVAL, "%s: sy (%lld) must be >= nx + 2 (%d)", who, d->sy, d->nx + 2);
    if (d->sz < d->sy * (long long)(d->ny + 2))
        return fail(PW_EINVAL, "%s: sz (%lld) must be >= sy * (ny + 2) (%lld)", who, d->sz,
                    d->sy * (long long)(d->ny + 2));
    if ((d->sy * elem_bytes) % 16 != 0 || (d->sz * elem_bytes) % 16 != 0)
        return fail(PW_EINVAL, "%s: sy and sz must be multiples of 16 bytes (sy=%lld, sz=%lld elements of %d bytes)",
                    who, d->sy, d->sz, elem_bytes);
    if (d->sz > (1ll << 40) / elem_bytes || (long long)d->nz * d->sz > (1ll << 46) / elem_bytes)
        return fail(PW_EINVAL, "%s: strides too large", who);
    return PW_OK;
}

// Bytes from a field's base to one past its last addressable element.
long long field_extent_bytes(const pw_dims& d, int elem_bytes) {
    return ((long long)(d.nz - 1) * d.sz + (long long)(d.ny + 1) * d.sy + d.nx + 2) * elem_bytes;
}

bool overlap(const void* a, long long na, const void* b, long long nb) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + (uintptr_t)nb && pb < pa + (uintptr_t)na;
}

int check_ptr(const void* p, int elem_bytes, const char* name, const char* who) {
    if (!p) return fail(PW_ENULL, "%s: %s is NULL", who, name);
    if (((uintptr_t)p) % elem_bytes != 0)
        return fail(PW_EINVAL, "%s: %s is not aligned to its %d-byte element", who, name, elem_bytes);
    return PW_OK;
}

int elem_size(pw_dtype d) { return (d == PW_F32_SPLIT || d == PW_F32) ? 4 : 8; }

bool known_dtype(pw_dtype d) { return d == PW_F64 || d == PW_F32_SPLIT || d == PW_F64_PAIRED || d == PW_F32; }

}  // namespace

// ============================================================================

extern "C" const char* pw_last_error(void) { return t_last_error.c_str(); }

extern "C" const char* pw_version(void) { return "pw-gb300 0.2 (sm_103a)"; }

extern "C" int pw_make_coeffs(int nz, double dx, double dy, const double* dz, const double* rho,
                              const double* rhon, double* tc2_host, double* tz4_host) {
    const char* who = "pw_make_coeffs";
    if (!dz || !tc2_host || !tz4_host) return fail(PW_ENULL, "%s: dz, tc2_host and tz4_host are required", who);
    if (nz < 1) return fail(PW_EINVAL, "%s: nz must be >= 1", who);
    if (!(dx > 0.0) || !(dy > 0.0)) return fail(PW_EINVAL, "%s: dx and dy must be > 0", who);
    for (int k = 1; k < nz; ++k)
        if (!(dz[k] > 0.0)) return fail(PW_EINVAL, "%s: dz[%d] must be > 0", who, k);
    tc2_host[0] = 0.25 / dx;
    tc2_host[1] = 0.25 / dy;
    double* tzc1 = tz4_host;
    double* tzc2 = tz4_host + nz;
    double* tzd1 = tz4_host + 2 * (size_t)nz;
    double* tzd2 = tz4_host + 3 * (size_t)nz;
    for (int k = 0; k < nz; ++k) tzc1[k] = tzc2[k] = tzd1[k] = tzd2[k] = 0.0;
    auto r_w = [&](int k) { return rho ? rho[k] : 1.0; };    // density on w levels
    auto r_n = [&](int k) { return rhon ? rhon[k] : 1.0; };  // density on u levels
    // w-level height below and above u-level k, and the u-level heights
    std::vector<double> zw(nz), zu(nz);
    double top = 0.0;
    zw[0] = 0.0;
    for (int k = 1; k < nz; ++k) {
        top += dz[k];
        zw[k] = top;
        zu[k] = 0.5 * (zw[k - 1] + zw[k]);
    }
    zu[0] = nz > 1 ? -zu[1] : 0.0;
    for (int k = 1; k < nz; ++k) {
        const double inv = 1.0 / (r_n(k) * dz[k]);
        tzc1[k] = 0.25 * r_w(k - 1) * inv;
        tzc2[k] = 0.25 * r_w(k) * inv;
    }
    for (int k = 1; k + 1 < nz; ++k) {
        const double inv = 1.0 / (r_w(k) * (zu[k + 1] - zu[k]));
        tzd1[k] = 0.25 * r_n(k) * inv;
        tzd2[k] = 0.25 * r_n(k + 1) * inv;
    }
    return PW_OK;
}

extern "C" int pw_make_split_table(int nz, double tcx, double tcy, const double* tz4_host, const double* ubar,
                                   const double* vbar, const double* wbar, float* table_host) {
    const char* who = "pw_make_split_table";
    if (!tz4_host || !ubar || !vbar || !wbar || !table_host)
        return fail(PW_ENULL, "%s: every pointer argument is required", who);
    if (nz < 1) return fail(PW_EINVAL, "%s: nz must be >= 1", who);
    const double* tzc1 = tz4_host;
    const double* tzc2 = tz4_host + nz;
    const double* tzd1 = tz4_host + 2 * (size_t)nz;
    const double* tzd2 = tz4_host + 3 * (size_t)nz;
    for (size_t n = 0; n < (size_t)PW_SPLIT_NCOEF * nz; ++n) table_host[n] = 0.0f;
    for (int k = 0; k < nz; ++k) {
        float* t = table_host + (size_t)k * PW_SPLIT_NCOEF;
        t[26] = (float)tcx;
        t[27] = (float)tcy;
        if (k == 0) continue;  // level 1 is not computed
        const bool up = (k + 1 < nz);  // upper vertical flux present (not the top level)
        const double U0 = ubar[k], V0 = vbar[k], W0 = wbar[k];
        const double Um = ubar[k - 1], Vm = vbar[k - 1], Wm = wbar[k - 1];
        const double Up = up ? ubar[k + 1] : 0.0, Vp = up ? vbar[k + 1] : 0.0, Wp = up ? wbar[k + 1] : 0.0;
        const double g2 = up ? tzc2[k] : 0.0;
        // su
        t[0] = (float)(3.0 * U0);
        t[1] = (float)(2.0 * V0);
        t[2] = (float)U0;
        t[3] = (float)(2.0 * (tzc1[k] * Um * Wm - g2 * Up * W0));
        t[4] = (float)tzc1[k];
        t[5] = (float)Um;
        t[6] = (float)(2.0 * Wm);
        t[7] = (float)g2;
        t[8] = (float)Up;
        t[9] = (float)(2.0 * W0);
        // sv
        t[10] = (float)(3.0 * V0);
        t[11] = (float)(2.0 * U0);
        t[12] = (float)V0;
        t[13] = (float)(2.0 * (tzc1[k] * Vm * Wm - g2 * Vp * W0));
        t[14] = (float)Vm;
        t[15] = (float)Vp;
        // sw (levels 2..nz-1)
        if (up) {
            t[16] = (float)W0;
            t[17] = (float)(U0 + Up);
            t[18] = (float)(V0 + Vp);
            t[19] = (float)(tzd1[k] * Wm * (W0 + Wm) - tzd2[k] * Wp * (W0 + Wp));
            t[20] = (float)tzd1[k];
            t[21] = (float)Wm;
            t[22] = (float)(W0 + Wm);
            t[23] = (float)tzd2[k];
            t[24] = (float)Wp;
            t[25] = (float)(W0 + Wp);
        }
    }
    return PW_OK;
}

extern "C" int pw_fill_periodic_halo(pw_dtype dtype, void* field, const pw_dims* dims, void* stream) {
    const char* who = "pw_fill_periodic_halo";
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = elem_size(dtype);
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!field) return fail(PW_ENULL, "%s: field is NULL", who);
    if (((uintptr_t)field) % es != 0) return fail(PW_EINVAL, "%s: field is misaligned", who);
    cudaError_t e = pw::launch_fill_halo(field, es, dims->nx, dims->ny, dims->nz, dims->sy, dims->sz,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

// pw_advect restricted to output levels k0..k1-1 (0 <= k0 < k1 <= nz) of the
// full-depth domain `dims`: level k0-1 and level k1 (where they exist) are
// read as neighbours, and the paper's bottom and top levels keep their
// treatment. Validation as pw_advect.
static int advect_levels(pw_dtype dtype, const void* u, const void* v, const void* w, const pw_coeffs* c,
                         const pw_dims* dims, const void* split, void* su, void* sv, void* sw, void* stream, int k0,
                         int k1, const char* who) {
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = elem_size(dtype);
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!c) return fail(PW_ENULL, "%s: coeffs is NULL", who);
    const void* ptrs[6] = {u, v, w, su, sv, sw};
    const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int n = 0; n < 6; ++n)
        if ((rc = check_ptr(ptrs[n], es, names[n], who))) return rc;
    // u, v, w share one set of box coordinates, so they must sit at the same
    // offset from a 16-byte boundary
    if ((uintptr_t)v % 16 != (uintptr_t)u % 16 || (uintptr_t)w % 16 != (uintptr_t)u % 16)
        return fail(PW_EINVAL, "%s: u, v and w must have the same address modulo 16 bytes", who);
    if (dtype == PW_F32_SPLIT || dtype == PW_F32) {
        if (!split) return fail(PW_ENULL, "%s: PW_F32_SPLIT and PW_F32 need the split table", who);
        if (((uintptr_t)split) % 16 != 0) return fail(PW_EINVAL, "%s: split table is not 16-byte aligned", who);
    } else {
        if (split) return fail(PW_EINVAL, "%s: split must be NULL for FP64 dtypes", who);
        if (!c->tzc1 || !c->tzc2 || !c->tzd1 || !c->tzd2)
            return fail(PW_ENULL, "%s: coefficient arrays are required", who);
    }
    const long long ext = field_extent_bytes(*dims, es);
    for (int o = 3; o < 6; ++o) {
        for (int n = 0; n < 3; ++n)
            if (overlap(ptrs[o], ext, ptrs[n], ext))
                return fail(PW_EALIAS, "%s: output %s overlaps input %s", who, names[o], names[n]);
        for (int n = 3; n < o; ++n)
            if (overlap(ptrs[o], ext, ptrs[n], ext))
                return fail(PW_EALIAS, "%s: output %s overlaps output %s", who, names[o], names[n]);
    }

    pw::TileShape shp;
    switch (dtype) {
        case PW_F64: shp = pw::fwd_f64_shape(); break;
        case PW_F64_PAIRED: shp = pw::fwd_paired_shape(); break;
        default: shp = pw::fwd_split_shape(); break;
    }
    CUtensorMap mu, mv, mw;
    if ((rc = make_field_map(&mu, u, es, *dims, shp.box_x, shp.box_y))) return rc;
    if ((rc = make_field_map(&mv, v, es, *dims, shp.box_x, shp.box_y))) return rc;
    if ((rc = make_field_map(&mw, w, es, *dims, shp.box_x, shp.box_y))) return rc;

    pw::FwdArgs a;
    a.xoff = (int)(((uintptr_t)u % 16) / es);
    // vector loads/stores need i = 1 of every field on a 16-byte boundary
    a.vec = 1;
    for (int n = 0; n < 6; ++n)
        if (((uintptr_t)ptrs[n] + es) % 16 != 0) a.vec = 0;
    a.nx = dims->nx;
    a.ny = dims->ny;
    a.nz = dims->nz;
    if (k0 < 0 || k1 > dims->nz || k0 >= k1)
        return fail(PW_EINVAL, "%s: level range [%d, %d) outside [0, %d)", who, k0, k1, dims->nz);
    a.kbeg = k0;
    a.kend = k1;
    a.sy = dims->sy;
    a.sz = dims->sz;
    a.tcx = c->tcx;
    a.tcy = c->tcy;
    a.tzc1 = c->tzc1;
    a.tzc2 = c->tzc2;
    a.tzd1 = c->tzd1;
    a.tzd2 = c->tzd2;
    a.split = static_cast<const float*>(split);
    a.su = su;
    a.sv = sv;
    a.sw = sw;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (dtype) {
        case PW_F64: e = pw::launch_fwd_f64(mu, mv, mw, a, st); break;
        case PW_F64_PAIRED: e = pw::launch_fwd_paired(mu, mv, mw, a, st); break;
        default: e = pw::launch_fwd_split(mu, mv, mw, a, st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

extern "C" int pw_advect(pw_dtype dtype, const void* u, const void* v, const void* w, const pw_coeffs* c,
                         const pw_dims* dims, const void* split, void* su, void* sv, void* sw, void* stream) {
    if (!dims) return fail(PW_ENULL, "pw_advect: dims is NULL");
    return advect_levels(dtype, u, v, w, c, dims, split, su, sv, sw, stream, 0, dims->nz, "pw_advect");
}

extern "C" int pw_split_field(const double* f, const pw_dims* dims_f, float* fp, const pw_dims* dims_p,
                              double* mean, void* stream) {
    const char* who = "pw_split_field";
    int rc = check_dims(dims_f, 8, who);
    if (rc) return rc;
    if ((rc = check_dims(dims_p, 4, who))) return rc;
    if (dims_f->nx != dims_p->nx || dims_f->ny != dims_p->ny || dims_f->nz != dims_p->nz)
        return fail(PW_EINVAL, "%s: dims_f and dims_p describe different domains", who);
    if (!f || !fp || !mean) return fail(PW_ENULL, "%s: f, fp and mean are required", who);
    if (((uintptr_t)f) % 8 || ((uintptr_t)fp) % 4 || ((uintptr_t)mean) % 8)
        return fail(PW_EINVAL, "%s: misaligned pointer", who);
    const long long ef = field_extent_bytes(*dims_f, 8), ep = field_extent_bytes(*dims_p, 4);
    if (overlap(f, ef, fp, ep) || overlap(mean, 8ll * dims_f->nz, f, ef) || overlap(mean, 8ll * dims_f->nz, fp, ep))
        return fail(PW_EALIAS, "%s: outputs overlap", who);
    cudaError_t e = pw::launch_split_field(f, dims_f->sy, dims_f->sz, fp, dims_p->sy, dims_p->sz, dims_f->nx,
                                           dims_f->ny, dims_f->nz, mean, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

extern "C" int pw_make_energy_weights(int nz, const double* dz, const double* rho, const double* rhon,
                                      double* wu_host, double* ww_host) {
    const char* who = "pw_make_energy_weights";
    if (!dz || !wu_host || !ww_host) return fail(PW_ENULL, "%s: dz, wu_host and ww_host are required", who);
    if (nz < 1) return fail(PW_EINVAL, "%s: nz must be >= 1", who);
    for (int k = 1; k < nz; ++k)
        if (!(dz[k] > 0.0)) return fail(PW_EINVAL, "%s: dz[%d] must be > 0", who, k);
    // u-level heights (as pw_make_coeffs): zu(k) midway between w levels k-1, k
    std::vector<double> zw(nz), zu(nz);
    double top = 0.0;
    zw[0] = 0.0;
    for (int k = 1; k < nz; ++k) {
        top += dz[k];
        zw[k] = top;
        zu[k] = 0.5 * (zw[k - 1] + zw[k]);
    }
    zu[0] = nz > 1 ? -zu[1] : 0.0;
    for (int k = 0; k < nz; ++k) wu_host[k] = ww_host[k] = 0.0;
    for (int k = 1; k < nz; ++k) wu_host[k] = dz[k] * (rhon ? rhon[k] : 1.0);
    for (int k = 1; k + 1 < nz; ++k) ww_host[k] = (zu[k + 1] - zu[k]) * (rho ? rho[k] : 1.0);
    return PW_OK;
}

extern "C" int pw_energy_budget(const void* u, const void* v, const void* w, int wind_elem_bytes,
                                const pw_dims* dims_wind, const void* su, const void* sv, const void* sw,
                                int tend_elem_bytes, const pw_dims* dims_tend, const double* wu, const double* ww,
                                double* level_sums, double* totals, void* stream) {
    const char* who = "pw_energy_budget";
    if ((wind_elem_bytes != 4 && wind_elem_bytes != 8) || (tend_elem_bytes != 4 && tend_elem_bytes != 8))
        return fail(PW_EINVAL, "%s: element sizes must be 4 or 8 bytes", who);
    int rc = check_dims(dims_wind, wind_elem_bytes, who);
    if (rc) return rc;
    if ((rc = check_dims(dims_tend, tend_elem_bytes, who))) return rc;
    if (dims_wind->nx != dims_tend->nx || dims_wind->ny != dims_tend->ny || dims_wind->nz != dims_tend->nz)
        return fail(PW_EINVAL, "%s: the winds and the tendencies describe different domains", who);
    if (dims_wind->nz > 65535) return fail(PW_EINVAL, "%s: nz above 65535", who);
    const void* wp[3] = {u, v, w};
    const void* sp[3] = {su, sv, sw};
    const char* wn[3] = {"u", "v", "w"};
    const char* sn[3] = {"su", "sv", "sw"};
    for (int n = 0; n < 3; ++n) {
        if ((rc = check_ptr(wp[n], wind_elem_bytes, wn[n], who))) return rc;
        if ((rc = check_ptr(sp[n], tend_elem_bytes, sn[n], who))) return rc;
    }
    if (!wu || !ww || !level_sums || !totals) return fail(PW_ENULL, "%s: wu, ww, level_sums and totals are required", who);
    if (((uintptr_t)wu | (uintptr_t)ww | (uintptr_t)level_sums | (uintptr_t)totals) % 8)
        return fail(PW_EINVAL, "%s: misaligned weight or result array", who);
    const long long nz = dims_wind->nz;
    if (overlap(level_sums, 48 * nz, totals, 48)) return fail(PW_EALIAS, "%s: level_sums overlaps totals", who);
    cudaError_t e = pw::launch_energy_budget(u, v, w, wind_elem_bytes, dims_wind->sy, dims_wind->sz, su, sv, sw,
                                             tend_elem_bytes, dims_tend->sy, dims_tend->sz, dims_wind->nx,
                                             dims_wind->ny, dims_wind->nz, wu, ww, level_sums, totals,
                                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

extern "C" int pw_selftest_bounded_wait(unsigned int limit_us, int* status, void* stream) {
    const char* who = "pw_selftest_bounded_wait";
    if (!status) return fail(PW_ENULL, "%s: status is NULL", who);
    if (limit_us < 1 || limit_us > 100000) return fail(PW_EINVAL, "%s: limit_us must be in 1..100000", who);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned int before = 0;
    cudaError_t e = pw::read_and_clear_status(&before, st);  // start from a clear word
    if (e == cudaSuccess) e = pw::launch_selftest_wait(1000ull * limit_us, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return pw_device_status(status, stream);
}

extern "C" int pw_device_status(int* status, void* stream) {
    if (!status) return fail(PW_ENULL, "pw_device_status: status is NULL");
    unsigned int s = 0;
    cudaError_t e = pw::read_and_clear_status(&s, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "pw_device_status");
    *status = (s & 1u) ? PW_ETIMEOUT : (s & 2u) ? PW_EINVAL : PW_OK;
    return PW_OK;
}

extern "C" int pw_advect_adjoint(pw_dtype dtype, const void* u, const void* v, const void* w, const pw_coeffs* c,
                                 const pw_dims* dims, const void* gsu, const void* gsv, const void* gsw, void* gu,
                                 void* gv, void* gw, int accumulate, void* stream) {
    const char* who = "pw_advect_adjoint";
    if (dtype != PW_F64 && dtype != PW_F32 && dtype != PW_F64_PAIRED)
        return fail(known_dtype(dtype) ? PW_EUNSUPPORTED : PW_EINVAL,
                    "%s: dtype must be PW_F64, PW_F64_PAIRED or PW_F32", who);
    const int es = elem_size(dtype);
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!c) return fail(PW_ENULL, "%s: coeffs is NULL", who);
    if (!c->tzc1 || !c->tzc2 || !c->tzd1 || !c->tzd2)
        return fail(PW_ENULL, "%s: coefficient arrays are required", who);
    const void* ptrs[9] = {u, v, w, gsu, gsv, gsw, gu, gv, gw};
    const char* names[9] = {"u", "v", "w", "gsu", "gsv", "gsw", "gu", "gv", "gw"};
    for (int n = 0; n < 9; ++n)
        if ((rc = check_ptr(ptrs[n], es, names[n], who))) return rc;
    for (int n = 1; n < 6; ++n)
        if ((uintptr_t)ptrs[n] % 16 != (uintptr_t)u % 16)
            return fail(PW_EINVAL, "%s: u, v, w, gsu, gsv, gsw must have the same address modulo 16 bytes", who);
    const long long ext = field_extent_bytes(*dims, es);
    for (int o = 6; o < 9; ++o) {
        for (int n = 0; n < o; ++n)
            if (overlap(ptrs[o], ext, ptrs[n], ext))
                return fail(PW_EALIAS, "%s: output %s overlaps %s", who, names[o], names[n]);
    }
    const pw::TileShape shp = dtype == PW_F64 ? pw::adjoint_f64_shape() : pw::adjoint_shape(es);
    CUtensorMap maps[6];
    for (int n = 0; n < 6; ++n)
        if ((rc = make_field_map(&maps[n], ptrs[n], es, *dims, shp.box_x, shp.box_y))) return rc;
    pw::AdjArgs a;
    a.nx = dims->nx;
    a.ny = dims->ny;
    a.nz = dims->nz;
    a.sy = dims->sy;
    a.sz = dims->sz;
    a.xoff = (int)(((uintptr_t)u % 16) / es);
    a.tcx = c->tcx;
    a.tcy = c->tcy;
    a.tzc1 = c->tzc1;
    a.tzc2 = c->tzc2;
    a.tzd1 = c->tzd1;
    a.tzd2 = c->tzd2;
    a.u = u;
    a.v = v;
    a.w = w;
    a.gsu = gsu;
    a.gsv = gsv;
    a.gsw = gsw;
    a.gu = gu;
    a.gv = gv;
    a.gw = gw;
    a.accumulate = accumulate ? 1 : 0;
    a.vec = ((uintptr_t)gu % 16 == (uintptr_t)u % 16 && (uintptr_t)gv % 16 == (uintptr_t)u % 16 &&
             (uintptr_t)gw % 16 == (uintptr_t)u % 16)
                ? 1
                : 0;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = dtype == PW_F64          ? pw::launch_adjoint_f64(maps, a, st)
                    : dtype == PW_F64_PAIRED ? pw::launch_adjoint_paired(maps, a, st)
                                             : pw::launch_adjoint(maps, a, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

extern "C" int pw_fold_periodic_halo(pw_dtype dtype, void* field, const pw_dims* dims, void* stream) {
    const char* who = "pw_fold_periodic_halo";
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = elem_size(dtype);
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!field) return fail(PW_ENULL, "%s: field is NULL", who);
    if (((uintptr_t)field) % es != 0) return fail(PW_EINVAL, "%s: field is misaligned", who);
    cudaError_t e = pw::launch_fold_halo(field, es, dims->nx, dims->ny, dims->nz, dims->sy, dims->sz,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

// ---------------------------------------------------------------- batches

extern "C" size_t pw_batch_plan_bytes(int n) { return pw::batch_plan_bytes(n); }

extern "C" int pw_variant_count(pw_dtype dtype) {
    switch (dtype) {
        case PW_F32:
        case PW_F32_SPLIT: return pw::split_variant_count();
        case PW_F64_PAIRED: return pw::paired_variant_count();
        case PW_F64: return pw::f64_variant_count();
        default: return 0;
    }
}

extern "C" int pw_make_batch_plan(pw_dtype dtype, int n, const pw_domain* doms, int variant, void* plan_host,
                                  size_t plan_bytes, long long* n_items) {
    const char* who = "pw_make_batch_plan";
    if (!doms || !plan_host || !n_items) return fail(PW_ENULL, "%s: doms, plan_host and n_items are required", who);
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    if (n < 1) return fail(PW_EINVAL, "%s: n must be >= 1", who);
    if (variant < 0 || variant >= pw_variant_count(dtype))
        return fail(PW_EINVAL, "%s: variant %d out of range for this dtype", who, variant);
    if (plan_bytes < pw::batch_plan_bytes(n))
        return fail(PW_EINVAL, "%s: plan_bytes %zu < %zu", who, plan_bytes, pw::batch_plan_bytes(n));
    if (((uintptr_t)plan_host) % 64 != 0) return fail(PW_EINVAL, "%s: plan_host must be 64-byte aligned", who);
    const int es = elem_size(dtype);
    const pw::TileShape shp = dtype == PW_F64_PAIRED ? pw::fwd_paired_shape_variant(variant)
                              : dtype == PW_F64    ? pw::fwd_f64_shape_variant(variant)
                                                   : pw::fwd_split_shape_variant(variant);
    // tallest domains first: their tiles take longest, so they start first
    std::vector<int> order(n);
    for (int d = 0; d < n; ++d) order[d] = d;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return doms[a].dims.nz > doms[b].dims.nz; });
    pw::BatchPlan* plan = static_cast<pw::BatchPlan*>(plan_host);
    memset(plan_host, 0, pw::batch_plan_bytes(n));
    long long items = 0;
    for (int q = 0; q < n; ++q) {
        const int d = order[q];
        const pw_domain& dm = doms[d];
        char tag[64];
        snprintf(tag, sizeof(tag), "%s: domain %d", who, d);
        int rc = check_dims(&dm.dims, es, tag);
        if (rc) return rc;
        const void* ptrs[6] = {dm.u, dm.v, dm.w, dm.su, dm.sv, dm.sw};
        const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
        for (int k = 0; k < 6; ++k)
            if ((rc = check_ptr(ptrs[k], es, names[k], tag))) return rc;
        if ((uintptr_t)dm.v % 16 != (uintptr_t)dm.u % 16 || (uintptr_t)dm.w % 16 != (uintptr_t)dm.u % 16)
            return fail(PW_EINVAL, "%s: u, v and w must have the same address modulo 16 bytes", tag);
        const bool f32 = (dtype == PW_F32 || dtype == PW_F32_SPLIT);
        if (f32 && !dm.split) return fail(PW_ENULL, "%s: the split table is required", tag);
        if (f32 && ((uintptr_t)dm.split) % 16 != 0) return fail(PW_EINVAL, "%s: split table not 16-byte aligned", tag);
        if (!f32 && (!dm.coeffs.tzc1 || !dm.coeffs.tzc2 || !dm.coeffs.tzd1 || !dm.coeffs.tzd2))
            return fail(PW_ENULL, "%s: coefficient arrays are required", tag);
        const long long ext = field_extent_bytes(dm.dims, es);
        for (int o = 3; o < 6; ++o)
            for (int k = 0; k < o; ++k)
                if (overlap(ptrs[o], ext, ptrs[k], ext))
                    return fail(PW_EALIAS, "%s: output %s overlaps %s", tag, names[o], names[k]);
        pw::BatchDomain& bd = plan->dom[q];
        if ((rc = make_field_map(&bd.mu, dm.u, es, dm.dims, shp.box_x, shp.box_y))) return rc;
        if ((rc = make_field_map(&bd.mv, dm.v, es, dm.dims, shp.box_x, shp.box_y))) return rc;
        if ((rc = make_field_map(&bd.mw, dm.w, es, dm.dims, shp.box_x, shp.box_y))) return rc;
        pw::FwdArgs& a = bd.args;
        a.nx = dm.dims.nx;
        a.ny = dm.dims.ny;
        a.nz = dm.dims.nz;
        a.kbeg = 0;
        a.kend = dm.dims.nz;
        a.sy = dm.dims.sy;
        a.sz = dm.dims.sz;
        a.xoff = (int)(((uintptr_t)dm.u % 16) / es);
        a.vec = 1;
        for (int k = 0; k < 6; ++k)
            if (((uintptr_t)ptrs[k] + es) % 16 != 0) a.vec = 0;
        a.tcx = dm.coeffs.tcx;
        a.tcy = dm.coeffs.tcy;
        a.tzc1 = dm.coeffs.tzc1;
        a.tzc2 = dm.coeffs.tzc2;
        a.tzd1 = dm.coeffs.tzd1;
        a.tzd2 = dm.coeffs.tzd2;
        a.split = static_cast<const float*>(dm.split);
        a.su = dm.su;
        a.sv = dm.sv;
        a.sw = dm.sw;
        bd.tiles_x = (dm.dims.nx + shp.tx - 1) / shp.tx;
        bd.tiles_y = (dm.dims.ny + shp.ty - 1) / shp.ty;
        bd.kchunks = 1;  // batches bring enough tiles; each item is a full column
        bd.first_item = items;
        items += (long long)bd.tiles_x * bd.tiles_y * bd.kchunks;
    }
    plan->counter = 0;
    plan->n_items = items;
    plan->n_domains = n;
    plan->dtype = (int)dtype;
    plan->variant = variant;
    plan->all_vec = 1;
    for (int q = 0; q < n; ++q)
        if (!plan->dom[q].args.vec) plan->all_vec = 0;
    *n_items = items;
    return PW_OK;
}

extern "C" int pw_advect_batched(pw_dtype dtype, int variant, void* plan_dev, long long n_items, void* stream) {
    const char* who = "pw_advect_batched";
    if (!plan_dev) return fail(PW_ENULL, "%s: plan_dev is NULL", who);
    if (((uintptr_t)plan_dev) % 64 != 0) return fail(PW_EINVAL, "%s: plan_dev must be 64-byte aligned", who);
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    if (variant < 0 || variant >= pw_variant_count(dtype)) return fail(PW_EINVAL, "%s: bad variant", who);
    if (n_items < 1) return fail(PW_EINVAL, "%s: n_items must be >= 1", who);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pw::BatchPlan* plan = static_cast<pw::BatchPlan*>(plan_dev);
    cudaError_t e = cudaMemsetAsync(&plan->counter, 0, sizeof(plan->counter), st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    e = dtype == PW_F64_PAIRED ? pw::launch_paired_batched(variant, plan, n_items, st)
        : dtype == PW_F64      ? pw::launch_f64_batched(variant, plan, n_items, st)
                               : pw::launch_split_batched(variant, plan, n_items, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

// ---------------------------------------------------------------- host overlap

extern "C" int pw_advect_host_chunked(pw_dtype dtype, const void* u_h, const void* v_h, const void* w_h, void* su_h,
                                      void* sv_h, void* sw_h, void* u_d, void* v_d, void* w_d, void* su_d,
                                      void* sv_d, void* sw_d, const pw_coeffs* c, const pw_dims* dims,
                                      const void* split, int nchunks, void* stream_h2d, void* stream_compute,
                                      void* stream_d2h) {
    const char* who = "pw_advect_host_chunked";
    if (!known_dtype(dtype)) return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = elem_size(dtype);
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    const void* hp[6] = {u_h, v_h, w_h, su_h, sv_h, sw_h};
    for (int n = 0; n < 6; ++n)
        if (!hp[n]) return fail(PW_ENULL, "%s: host field %d is NULL", who, n);
    const int ny = dims->ny, nz = dims->nz;
    if (nchunks < 1) nchunks = 1;
    if (nchunks > nz) nchunks = nz;
    cudaStream_t sh = static_cast<cudaStream_t>(stream_h2d);
    cudaStream_t sc = static_cast<cudaStream_t>(stream_compute);
    cudaStream_t sd = static_cast<cudaStream_t>(stream_d2h);
    const size_t row = (size_t)dims->sy * es, plane = (size_t)dims->sz * es;
    const size_t extent = (size_t)field_extent_bytes(*dims, es);
    // levels [k0, k1) of chunk q
    auto levels_of = [&](int q, int* k0, int* k1) {
        *k0 = (int)((long long)nz * q / nchunks);
        *k1 = (int)((long long)nz * (q + 1) / nchunks);
    };
    std::vector<cudaEvent_t> h2d(nchunks), done(nchunks);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < nchunks && e == cudaSuccess; ++q) {
        e = cudaEventCreateWithFlags(&h2d[q], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[q], cudaEventDisableTiming);
    }
    const void* in_h[3] = {u_h, v_h, w_h};
    void* in_d[3] = {u_d, v_d, w_d};
    void* out_h[3] = {su_h, sv_h, sw_h};
    const void* out_d[3] = {su_d, sv_d, sw_d};
    // inputs of chunk q: its whole level planes, one contiguous copy per field
    // (the last chunk ends at the field's extent)
    for (int q = 0; q < nchunks && e == cudaSuccess; ++q) {
        int k0, k1;
        levels_of(q, &k0, &k1);
        const size_t b0 = (size_t)k0 * plane, b1 = (q == nchunks - 1) ? extent : (size_t)k1 * plane;
        for (int f = 0; f < 3 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(static_cast<char*>(in_d[f]) + b0, static_cast<const char*>(in_h[f]) + b0, b1 - b0,
                                cudaMemcpyHostToDevice, sh);
        if (e == cudaSuccess) e = cudaEventRecord(h2d[q], sh);
    }
    // compute chunk q's levels once chunk q+1 (holding level k1, their upper
    // neighbour) has landed; then its output rows 1..ny of each level go back
    for (int q = 0; q < nchunks && e == cudaSuccess; ++q) {
        int k0, k1;
        levels_of(q, &k0, &k1);
        e = cudaStreamWaitEvent(sc, h2d[q + 1 < nchunks ? q + 1 : q], 0);
        if (e != cudaSuccess) break;
        rc = advect_levels(dtype, u_d, v_d, w_d, c, dims, split, su_d, sv_d, sw_d, sc, k0, k1, who);
        if (rc != PW_OK) break;
        e = cudaEventRecord(done[q], sc);
        if (e != cudaSuccess) break;
        e = cudaStreamWaitEvent(sd, done[q], 0);
        const size_t off = (size_t)k0 * plane + row;
        for (int f = 0; f < 3 && e == cudaSuccess; ++f)
            e = cudaMemcpy2DAsync(static_cast<char*>(out_h[f]) + off, plane, static_cast<const char*>(out_d[f]) + off,
                                  plane, (size_t)ny * row, (size_t)(k1 - k0), cudaMemcpyDeviceToHost, sd);
    }
    for (int q = 0; q < nchunks; ++q) {
        if (h2d[q]) cudaEventDestroy(h2d[q]);
        if (done[q]) cudaEventDestroy(done[q]);
    }
    if (rc != PW_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}
