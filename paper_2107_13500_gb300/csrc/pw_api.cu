// pw_api.cu -- the C ABI declared in include/pw.h: argument validation, TMA
// descriptor set-up, dispatch to the kernels, host-side coefficient tables.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
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

int make_field_map(CUtensorMap* map, const void* base, int elem_bytes, const pw_dims& d, int box_x, int box_y) {
    cudaError_t e;
    EncodeTiledFn enc = get_encode_fn(&e);
    if (!enc) return cuda_fail(e, "cuTensorMapEncodeTiled lookup");
    cuuint64_t gdim[3] = {(cuuint64_t)(d.nx + 2), (cuuint64_t)(d.ny + 2), (cuuint64_t)d.nz};
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

int check_ptr(const void* p, const char* name, const char* who) {
    if (!p) return fail(PW_ENULL, "%s: %s is NULL", who, name);
    if (((uintptr_t)p) % 16 != 0) return fail(PW_EINVAL, "%s: %s is not 16-byte aligned", who, name);
    return PW_OK;
}

}  // namespace

// ============================================================================

extern "C" const char* pw_last_error(void) { return t_last_error.c_str(); }

extern "C" const char* pw_version(void) { return "pw-gb300 0.1 (sm_103a)"; }

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
    if (dtype != PW_F64 && dtype != PW_F32_SPLIT && dtype != PW_F64_PAIRED)
        return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = dtype == PW_F32_SPLIT ? 4 : 8;
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!field) return fail(PW_ENULL, "%s: field is NULL", who);
    if (((uintptr_t)field) % es != 0) return fail(PW_EINVAL, "%s: field is misaligned", who);
    cudaError_t e = pw::launch_fill_halo(field, es, dims->nx, dims->ny, dims->nz, dims->sy, dims->sz,
                                         static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, who);
    return PW_OK;
}

extern "C" int pw_advect(pw_dtype dtype, const void* u, const void* v, const void* w, const pw_coeffs* c,
                         const pw_dims* dims, const void* split, void* su, void* sv, void* sw, void* stream) {
    const char* who = "pw_advect";
    if (dtype != PW_F64 && dtype != PW_F32_SPLIT && dtype != PW_F64_PAIRED)
        return fail(PW_EINVAL, "%s: unknown dtype %d", who, (int)dtype);
    const int es = dtype == PW_F32_SPLIT ? 4 : 8;
    int rc = check_dims(dims, es, who);
    if (rc) return rc;
    if (!c) return fail(PW_ENULL, "%s: coeffs is NULL", who);
    const void* ptrs[6] = {u, v, w, su, sv, sw};
    const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
    for (int n = 0; n < 6; ++n)
        if ((rc = check_ptr(ptrs[n], names[n], who))) return rc;
    if (dtype == PW_F32_SPLIT) {
        if (!split) return fail(PW_ENULL, "%s: PW_F32_SPLIT needs the split table", who);
        if (((uintptr_t)split) % 16 != 0) return fail(PW_EINVAL, "%s: split table is not 16-byte aligned", who);
    } else {
        if (split) return fail(PW_EINVAL, "%s: split must be NULL unless dtype is PW_F32_SPLIT", who);
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
    a.nx = dims->nx;
    a.ny = dims->ny;
    a.nz = dims->nz;
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

extern "C" int pw_device_status(int* status, void* stream) {
    if (!status) return fail(PW_ENULL, "pw_device_status: status is NULL");
    unsigned int s = 0;
    cudaError_t e = pw::read_and_clear_status(&s, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "pw_device_status");
    *status = (s & 1u) ? PW_ETIMEOUT : PW_OK;
    return PW_OK;
}
