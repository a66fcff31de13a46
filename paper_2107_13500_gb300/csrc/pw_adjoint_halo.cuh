// pw_adjoint_halo.cuh -- the adjoint's halo cells (i = 0, nx+1 or j = 0,
// ny+1), gathered cell by cell on plain loads: the part of the FP64 adjoint
// that its interior-aligned tiles leave out.
//
// Each halo cell receives, like every cell, the derivative of every face
// term c * p * (q + r) that reads it times the cotangent of the output point
// that term belongs to: c * (q + r) where it is the advected value p, c * p
// where it is in the face sum. Only the interior output points next to the
// halo read it, so most of those cotangents are zero (read as such below);
// the evaluation is the full cell-by-cell sum all the same, the
// T1..T6 / S1..S6 / W1..W6 terms of include/pw.h's formulas, one thread per
// cell and level.
#pragma once

#include <cuda_runtime.h>

#include "pw_internal.h"

namespace pw {

namespace {

// Level coefficient `lev` (0 outside the column).
__device__ __forceinline__ double coef_at(const double* c, int lev, int nz) {
    return (lev >= 0 && lev < nz) ? __ldg(c + lev) : 0.0;
}
// tzc2 of an su/sv output level; the top level has no upper flux.
__device__ __forceinline__ double tzc2_at(const double* c, int lev, int nz) {
    return (lev >= 0 && lev <= nz - 2) ? __ldg(c + lev) : 0.0;
}

// Field value at (ii, jj, kk); 0 outside the array.
template <typename T>
__device__ __forceinline__ T halo_f(const void* p, const AdjArgs& a, int ii, int jj, int kk) {
    if (ii < 0 || ii > a.nx + 1 || jj < 0 || jj > a.ny + 1 || kk < 0 || kk >= a.nz) return T(0);
    return __ldg(static_cast<const T*>(p) + (size_t)kk * (size_t)a.sz + (size_t)jj * (size_t)a.sy + ii);
}
// Cotangent at (ii, jj, kk); 0 unless it is a computed output point (sw:
// levels 1..nz-2, su and sv: 1..nz-1).
template <typename T>
__device__ __forceinline__ T halo_g(const void* p, const AdjArgs& a, int ii, int jj, int kk, bool sw) {
    if (ii < 1 || ii > a.nx || jj < 1 || jj > a.ny || kk < 1 || kk > a.nz - (sw ? 2 : 1)) return T(0);
    return __ldg(static_cast<const T*>(p) + (size_t)kk * (size_t)a.sz + (size_t)jj * (size_t)a.sy + ii);
}

// Halo cell number t of the domain (level-major: t = k * nh + h, h running
// over the west column, the east column, the south row and the north row);
// nothing for t beyond the last.
template <typename T>
__device__ __noinline__ void adjoint_halo_cell(const AdjArgs& a, long long t) {
    const int nh = 2 * (a.ny + 2) + 2 * a.nx;  // halo cells per level
    if (t >= (long long)nh * a.nz) return;
    const int k = (int)(t / nh), h = (int)(t - (long long)k * nh);
    int i, j;
    if (h < a.ny + 2) {
        i = 0;
        j = h;
    } else if (h < 2 * (a.ny + 2)) {
        i = a.nx + 1;
        j = h - (a.ny + 2);
    } else if (h < 2 * (a.ny + 2) + a.nx) {
        i = 1 + h - 2 * (a.ny + 2);
        j = 0;
    } else {
        i = 1 + h - 2 * (a.ny + 2) - a.nx;
        j = a.ny + 1;
    }
    auto F = [&](const void* p, int di, int dj, int dk) { return halo_f<T>(p, a, i + di, j + dj, k + dk); };
    auto G = [&](const void* p, int di, int dj, int dk, bool sw) {
        return halo_g<T>(p, a, i + di, j + dj, k + dk, sw);
    };
    const int nz = a.nz;
    const T tcx = (T)a.tcx, tcy = (T)a.tcy;
    const T tz1p = (T)coef_at(a.tzc1, k + 1, nz), tz2m = (T)coef_at(a.tzc2, k - 1, nz);
    const T tz20 = (T)tzc2_at(a.tzc2, k, nz);
    const T td1p = (T)coef_at(a.tzd1, k + 1, nz), td10 = (T)coef_at(a.tzd1, k, nz);
    const T td2m = (T)coef_at(a.tzd2, k - 1, nz), td20 = (T)coef_at(a.tzd2, k, nz);

    const T su_c = G(a.gsu, 0, 0, 0, false), su_e = G(a.gsu, 1, 0, 0, false), su_w = G(a.gsu, -1, 0, 0, false);
    const T su_n = G(a.gsu, 0, 1, 0, false), su_s = G(a.gsu, 0, -1, 0, false), su_nw = G(a.gsu, -1, 1, 0, false);
    const T su_km = G(a.gsu, 0, 0, -1, false), su_kp = G(a.gsu, 0, 0, 1, false);
    const T su_kp_w = G(a.gsu, -1, 0, 1, false);
    const T sv_c = G(a.gsv, 0, 0, 0, false), sv_e = G(a.gsv, 1, 0, 0, false), sv_w = G(a.gsv, -1, 0, 0, false);
    const T sv_n = G(a.gsv, 0, 1, 0, false), sv_s = G(a.gsv, 0, -1, 0, false), sv_se = G(a.gsv, 1, -1, 0, false);
    const T sv_km = G(a.gsv, 0, 0, -1, false), sv_kp = G(a.gsv, 0, 0, 1, false);
    const T sv_kp_s = G(a.gsv, 0, -1, 1, false);
    const T sw_c = G(a.gsw, 0, 0, 0, true), sw_e = G(a.gsw, 1, 0, 0, true), sw_w = G(a.gsw, -1, 0, 0, true);
    const T sw_n = G(a.gsw, 0, 1, 0, true), sw_s = G(a.gsw, 0, -1, 0, true);
    const T sw_km = G(a.gsw, 0, 0, -1, true), sw_km_e = G(a.gsw, 1, 0, -1, true);
    const T sw_km_n = G(a.gsw, 0, 1, -1, true), sw_kp = G(a.gsw, 0, 0, 1, true);

    const T u_c = F(a.u, 0, 0, 0), u_e = F(a.u, 1, 0, 0), u_w = F(a.u, -1, 0, 0);
    const T u_n = F(a.u, 0, 1, 0), u_nw = F(a.u, -1, 1, 0);
    const T u_kp = F(a.u, 0, 0, 1), u_kp_w = F(a.u, -1, 0, 1);
    const T v_c = F(a.v, 0, 0, 0), v_e = F(a.v, 1, 0, 0), v_n = F(a.v, 0, 1, 0);
    const T v_s = F(a.v, 0, -1, 0), v_se = F(a.v, 1, -1, 0);
    const T v_kp = F(a.v, 0, 0, 1), v_kp_s = F(a.v, 0, -1, 1);
    const T w_c = F(a.w, 0, 0, 0), w_e = F(a.w, 1, 0, 0), w_n = F(a.w, 0, 1, 0);
    const T w_kmc = F(a.w, 0, 0, -1), w_kme = F(a.w, 1, 0, -1), w_kmn = F(a.w, 0, 1, -1);
    const T w_kp = F(a.w, 0, 0, 1);

    // gu(C): su-x (P = C+x, C, C-x), su-y (P = C+y, C-y), su-z (P = C+z, C-z),
    // sv-x (P = C+x, C+x-y, C, C-y), sw-x (P = C+x, C+x-z, C, C-z)
    T r_u = tcx * ((u_e + u_c + u_c) * su_e + u_w * su_c - (u_w + u_c + u_c) * su_w - u_e * su_c);
    r_u += tcy * ((v_c + v_e) * su_n - (v_s + v_se) * su_s);
    r_u += tz1p * (w_c + w_e) * su_kp - tz2m * (w_kmc + w_kme) * su_km;
    r_u += tcx * (v_c * sv_e + v_s * sv_se - v_e * sv_c - v_se * sv_s);
    r_u += tcx * (w_c * sw_e + w_kmc * sw_km_e - w_e * sw_c - w_kme * sw_km);
    // gv(C): the mirror
    T r_v = tcy * ((v_n + v_c + v_c) * sv_n + v_s * sv_c - (v_s + v_c + v_c) * sv_s - v_n * sv_c);
    r_v += tcx * ((u_c + u_n) * sv_e - (u_w + u_nw) * sv_w);
    r_v += tz1p * (w_c + w_n) * sv_kp - tz2m * (w_kmc + w_kmn) * sv_km;
    r_v += tcy * (u_c * su_n + u_w * su_nw - u_n * su_c - u_nw * su_w);
    r_v += tcy * (w_c * sw_n + w_kmc * sw_km_n - w_n * sw_c - w_kmn * sw_km);
    // gw(C): su-z, sv-z (P = C+z, C+z-x / C+z-y, C, C-x / C-y), sw-x, sw-y, sw-z
    T r_w = tz1p * (u_c * su_kp + u_w * su_kp_w) - tz20 * (u_kp * su_c + u_kp_w * su_w);
    r_w += tz1p * (v_c * sv_kp + v_s * sv_kp_s) - tz20 * (v_kp * sv_c + v_kp_s * sv_s);
    r_w += tcx * ((u_c + u_kp) * sw_e - (u_w + u_kp_w) * sw_w);
    r_w += tcy * ((v_c + v_kp) * sw_n - (v_s + v_kp_s) * sw_s);
    r_w += td1p * (w_kp + w_c + w_c) * sw_kp + td10 * w_kmc * sw_c;
    r_w -= td2m * (w_kmc + w_c + w_c) * sw_km + td20 * w_kp * sw_c;

    const size_t o = (size_t)k * (size_t)a.sz + (size_t)j * (size_t)a.sy + i;
    T* gu = static_cast<T*>(a.gu) + o;
    T* gv = static_cast<T*>(a.gv) + o;
    T* gw = static_cast<T*>(a.gw) + o;
    if (a.accumulate) {
        *gu += r_u;
        *gv += r_v;
        *gw += r_w;
    } else {
        *gu = r_u;
        *gv = r_v;
        *gw = r_w;
    }
}

}  // namespace

}  // namespace pw
