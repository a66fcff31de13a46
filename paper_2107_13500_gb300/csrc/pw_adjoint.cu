// pw_adjoint.cu -- transpose of the PW advection Jacobian (gather form), and
// the transpose of the periodic halo fill.
//
// The forward map is a quadratic form: every term is c * p * (q + r) with c a
// coefficient and p, q, r field values, so its partial derivatives are
// c * (q + r) (by p) and c * p (by q and by r). For a cell C the adjoint
// gathers, from every output point P that read C, the cotangent at P times
// that derivative. Writing each forward term out (su: T1..T6, sv: S1..S6,
// sw: W1..W6, the order of the formulas in include/pw.h), a u cell is read by
// 16 (P, term) pairs, a v cell by 16, a w cell by 16; they are listed at the
// three gather blocks below. Cotangents outside the computed points (halo
// columns and rows, level 1, and level nz for sw) count as zero, so output
// cells include the halo: gu, gv, gw are defined on every cell the forward
// map reads. Each thread owns one cell column and marches k with a TMA ring
// of the six fields (u, v, w, gsu, gsv, gsw) -- no atomics, one write per cell.
// A launch splits the columns into k-chunks (blockIdx.z) so that small
// domains still fill the GPU; a chunk of output levels kb..ke-1 reads levels
// kb-1..ke.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace {

constexpr int kTX = 32, kTY = 8, kS = 4, kFields = 6;

// v where b holds, else 0 (a select, so garbage in unused halo cotangents,
// NaN included, never reaches a result)
template <typename T>
__device__ __forceinline__ T gate(bool b, T v) {
    return b ? v : T(0);
}

template <typename T>
struct AdjShape {
    static constexpr int NT = kTX * kTY;
    static constexpr int XOFF_MAX = 16 / (int)sizeof(T) - 1;
    static constexpr int UNIT = 16 / (int)sizeof(T);  // box x start granularity (elements)
    // box x start = x0 - UNIT (x0 = tile origin), covering cells x0-1 .. x0+kTX
    static constexpr int BX = round_up(kTX + 2 + UNIT + XOFF_MAX, UNIT);
    static constexpr int BY = kTY + 2;
    static constexpr int BOX_BYTES = BX * BY * (int)sizeof(T);
    static constexpr int BOX_STRIDE = round_up(BOX_BYTES, 128);
    static constexpr int STAGE_BYTES = kFields * BOX_STRIDE;
    static constexpr int SMEM_BYTES = kS * STAGE_BYTES + 64 + 128;
    static_assert(BX <= 256, "TMA box limit");
};

struct AdjMaps {
    CUtensorMap m[kFields];  // u, v, w, gsu, gsv, gsw
};

template <typename T>
struct AdjRing {
    using Sh = AdjShape<T>;
    unsigned char* base;
    uint64_t* full;
    __device__ __forceinline__ void setup(unsigned char* raw) {
        base = raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
        full = reinterpret_cast<uint64_t*>(base + kS * Sh::STAGE_BYTES);
    }
    __device__ __forceinline__ const T* box(int slot, int f) const {
        return reinterpret_cast<const T*>(base + slot * Sh::STAGE_BYTES + f * Sh::BOX_STRIDE);
    }
    // wait for load number `seq` (stage seq % kS, phase seq / kS)
    __device__ __forceinline__ bool wait(int seq) {
        return mbar_wait_bounded(&full[seq % kS], (uint32_t)((seq / kS) & 1));
    }
};

// Load number `seq` of a chunk brings level `lev` (may be -1 or nz: the TMA
// zero-fills out-of-range levels) into stage seq % kS.
template <typename T>
__device__ __forceinline__ void adj_issue(AdjRing<T>& r, const AdjMaps& maps, int seq, int lev, int x, int y) {
    using Sh = AdjShape<T>;
    const int s = seq % kS;
    uint64_t* bar = &r.full[s];
    unsigned char* dst = r.base + s * Sh::STAGE_BYTES;
    mbar_arrive_expect_tx(bar, kFields * Sh::BOX_BYTES);
    for (int f = 0; f < kFields; ++f) tma_load_3d(dst + f * Sh::BOX_STRIDE, &maps.m[f], bar, x, y, lev);
}

// The seven vertical coefficients step k uses (zero where the paper's level
// has no such flux), in T. One thread each loads and converts them once per
// level; the CTA barrier of the step before publishes them. (A per-thread
// double->float conversion would run on the FP64 pipe and bound the FP32
// kernel.)
template <typename T>
__device__ __forceinline__ void level_coefs(const AdjArgs& a, int k, int tid, T* dst) {
    if (tid >= 7) return;
    const int nz = a.nz;
    double c = 0.0;
    switch (tid) {
        case 0: c = (k + 1 <= nz - 1) ? __ldg(a.tzc1 + k + 1) : 0.0; break;  // tz1p
        case 1: c = (k >= 1) ? __ldg(a.tzc2 + k - 1) : 0.0; break;           // tz2m
        case 2: c = __ldg(a.tzc2 + k); break;                                // tz20
        case 3: c = (k + 1 <= nz - 1) ? __ldg(a.tzd1 + k + 1) : 0.0; break;  // td1p
        case 4: c = __ldg(a.tzd1 + k); break;                                // td10
        case 5: c = (k >= 1) ? __ldg(a.tzd2 + k - 1) : 0.0; break;           // td2m
        default: c = __ldg(a.tzd2 + k); break;                               // td20
    }
    dst[tid] = (T)c;
}

template <typename T>
__global__ void __launch_bounds__(kTX* kTY) adjoint_kernel(const __grid_constant__ AdjMaps maps, const AdjArgs a) {
    using Sh = AdjShape<T>;
    constexpr int BX = Sh::BX;
    extern __shared__ unsigned char smem_raw[];
    __shared__ T coef_s[2][8];  // level coefficients, two levels in flight
    AdjRing<T> ring;
    ring.setup(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid % kTX, ty = tid / kTX;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int i = x0 + tx, j = y0 + ty;  // output cell, halo included (0..nx+1, 0..ny+1)
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool act = (i <= nx + 1) && (j <= ny + 1);
    const int bxs = x0 - Sh::UNIT;  // box x start (tensor coordinate), aligned
    const int bys = y0 - 1;
    const int kb = (int)((long long)nz * blockIdx.z / gridDim.z);
    const int ke = (int)((long long)nz * (blockIdx.z + 1) / gridDim.z);
    const int nseq = ke - kb + 2;   // loads: levels kb-1 .. ke

    if (tid == 0) {
        for (int f = 0; f < kFields; ++f) prefetch_tensormap(&maps.m[f]);
        for (int s = 0; s < kS; ++s) mbar_init(&ring.full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < kS && issued < nseq; ++issued) adj_issue(ring, maps, issued, kb - 1 + issued, bxs, bys);

    // shared index of cell (i, j): tensor x = i + xoff, box starts at bxs
    const int c0 = (ty + 1) * BX + (tx + Sh::UNIT + a.xoff);
    // interior masks of the neighbouring output points
    const bool mxm = (i - 1 >= 1 && i - 1 <= nx);
    const bool mx0 = (i >= 1 && i <= nx);
    const bool mxp = (i + 1 >= 1 && i + 1 <= nx);
    const bool mym = (j - 1 >= 1 && j - 1 <= ny);
    const bool my0 = (j >= 1 && j <= ny);
    const bool myp = (j + 1 >= 1 && j + 1 <= ny);
    const T tcx = (T)a.tcx, tcy = (T)a.tcy;
    T* __restrict__ gu = static_cast<T*>(a.gu);
    T* __restrict__ gv = static_cast<T*>(a.gv);
    T* __restrict__ gw = static_cast<T*>(a.gw);
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)kb * (size_t)a.sz;

    bool bad = false;
    for (int s = 0; s < 3 && s < nseq; ++s) bad |= !ring.wait(s);  // levels kb-1, kb, kb+1
    level_coefs<T>(a, kb, tid, coef_s[0]);
    bool abort = __syncthreads_or(bad);

    for (int k = kb; k < ke && !abort; ++k) {
        const int r = k - kb;
        if (r > 0) bad |= !ring.wait(r + 2);  // level k+1 (load r+2)
        // stages of levels k-1, k, k+1
        const int sm = r % kS, s0 = (r + 1) % kS, sp = (r + 2) % kS;
        const T* Um = ring.box(sm, 0);
        const T* U0 = ring.box(s0, 0);
        const T* Up = ring.box(sp, 0);
        const T* Vm = ring.box(sm, 1);
        const T* V0 = ring.box(s0, 1);
        const T* Vp = ring.box(sp, 1);
        const T* Wm = ring.box(sm, 2);
        const T* W0 = ring.box(s0, 2);
        const T* Wp = ring.box(sp, 2);
        const T* GUm = ring.box(sm, 3);
        const T* GU0 = ring.box(s0, 3);
        const T* GUp = ring.box(sp, 3);
        const T* GVm = ring.box(sm, 4);
        const T* GV0 = ring.box(s0, 4);
        const T* GVp = ring.box(sp, 4);
        const T* GWm = ring.box(sm, 5);
        const T* GW0 = ring.box(s0, 5);
        const T* GWp = ring.box(sp, 5);
        // level masks: su, sv computed on levels 1..nz-1; sw on 1..nz-2
        const bool l_m = (k - 1 >= 1);
        const bool l_0 = (k >= 1);
        const bool l_p = (k + 1 <= nz - 1);
        const bool w_m = (k - 1 >= 1 && k - 1 <= nz - 2);
        const bool w_0 = (k >= 1 && k <= nz - 2);
        const bool w_p = (k + 1 <= nz - 2);
        const bool up0 = (k <= nz - 2);  // level k has an upper flux
        const T* cs = coef_s[r & 1];
        const T tz1p = cs[0], tz2m = cs[1], tz20 = cs[2], td1p = cs[3], td10 = cs[4], td2m = cs[5], td20 = cs[6];
        constexpr int E = 1, N = BX;

        // masked cotangents (index: P = C + offset)
        const T su_c = gate(mx0 && my0 && l_0, GU0[c0]);
        const T su_e = gate(mxp && my0 && l_0, GU0[c0 + E]);
        const T su_w = gate(mxm && my0 && l_0, GU0[c0 - E]);
        const T su_n = gate(mx0 && myp && l_0, GU0[c0 + N]);
        const T su_s = gate(mx0 && mym && l_0, GU0[c0 - N]);
        const T su_nw = gate(mxm && myp && l_0, GU0[c0 + N - E]);
        const T su_w_up = gate(mxm && my0 && l_0 && up0, GU0[c0 - E]);
        const T su_c_up = gate(up0, su_c);
        const T su_km = gate(mx0 && my0 && l_m, GUm[c0]);
        const T su_kp = gate(mx0 && my0 && l_p, GUp[c0]);
        const T su_kp_w = gate(mxm && my0 && l_p, GUp[c0 - E]);
        const T sv_c = gate(mx0 && my0 && l_0, GV0[c0]);
        const T sv_e = gate(mxp && my0 && l_0, GV0[c0 + E]);
        const T sv_w = gate(mxm && my0 && l_0, GV0[c0 - E]);
        const T sv_n = gate(mx0 && myp && l_0, GV0[c0 + N]);
        const T sv_s = gate(mx0 && mym && l_0, GV0[c0 - N]);
        const T sv_se = gate(mxp && mym && l_0, GV0[c0 - N + E]);
        const T sv_s_up = gate(up0, sv_s);
        const T sv_c_up = gate(up0, sv_c);
        const T sv_km = gate(mx0 && my0 && l_m, GVm[c0]);
        const T sv_kp = gate(mx0 && my0 && l_p, GVp[c0]);
        const T sv_kp_s = gate(mx0 && mym && l_p, GVp[c0 - N]);
        const T sw_c = gate(mx0 && my0 && w_0, GW0[c0]);
        const T sw_e = gate(mxp && my0 && w_0, GW0[c0 + E]);
        const T sw_w = gate(mxm && my0 && w_0, GW0[c0 - E]);
        const T sw_n = gate(mx0 && myp && w_0, GW0[c0 + N]);
        const T sw_s = gate(mx0 && mym && w_0, GW0[c0 - N]);
        const T sw_km = gate(mx0 && my0 && w_m, GWm[c0]);
        const T sw_km_e = gate(mxp && my0 && w_m, GWm[c0 + E]);
        const T sw_km_n = gate(mx0 && myp && w_m, GWm[c0 + N]);
        const T sw_kp = gate(mx0 && my0 && w_p, GWp[c0]);

        // fields around C
        const T u_c = U0[c0], u_e = U0[c0 + E], u_w = U0[c0 - E], u_n = U0[c0 + N], u_nw = U0[c0 + N - E];
        const T u_kp = Up[c0], u_kp_w = Up[c0 - E];
        const T v_c = V0[c0], v_e = V0[c0 + E], v_n = V0[c0 + N], v_s = V0[c0 - N], v_se = V0[c0 - N + E];
        const T v_kp = Vp[c0], v_kp_s = Vp[c0 - N];
        const T w_c = W0[c0], w_e = W0[c0 + E], w_n = W0[c0 + N];
        const T w_kmc = Wm[c0], w_kme = Wm[c0 + E], w_kmn = Wm[c0 + N];
        const T w_kp = Wp[c0];

        // gu(C): T1 (P=C+x, P=C), T2 (P=C-x, P=C), T3 (P=C+y), T4 (P=C-y),
        // T5 (P=C+z), T6 (P=C-z), S3 (P=C+x, P=C+x-y), S4 (P=C, P=C-y),
        // W1 (P=C+x, P=C+x-z), W2 (P=C, P=C-z)
        T r_u = tcx * ((u_e + u_c + u_c) * su_e + u_w * su_c - (u_w + u_c + u_c) * su_w - u_e * su_c);
        r_u += tcy * ((v_c + v_e) * su_n - (v_s + v_se) * su_s);
        r_u += tz1p * (w_c + w_e) * su_kp - tz2m * (w_kmc + w_kme) * su_km;
        r_u += tcx * (v_c * sv_e + v_s * sv_se - v_e * sv_c - v_se * sv_s);
        r_u += tcx * (w_c * sw_e + w_kmc * sw_km_e - w_e * sw_c - w_kme * sw_km);
        // gv(C): mirror of the first four lines; T3 (P=C+y, P=C+y-x), T4 (P=C, P=C-x);
        // W3 (P=C+y, P=C+y-z), W4 (P=C, P=C-z)
        T r_v = tcy * ((v_n + v_c + v_c) * sv_n + v_s * sv_c - (v_s + v_c + v_c) * sv_s - v_n * sv_c);
        r_v += tcx * ((u_c + u_n) * sv_e - (u_w + u_nw) * sv_w);
        r_v += tz1p * (w_c + w_n) * sv_kp - tz2m * (w_kmc + w_kmn) * sv_km;
        r_v += tcy * (u_c * su_n + u_w * su_nw - u_n * su_c - u_nw * su_w);
        r_v += tcy * (w_c * sw_n + w_kmc * sw_km_n - w_n * sw_c - w_kmn * sw_km);
        // gw(C): T5 (P=C+z, P=C+z-x), T6 (P=C, P=C-x), S5 (P=C+z, P=C+z-y),
        // S6 (P=C, P=C-y), W1 (P=C+x), W2 (P=C-x), W3 (P=C+y), W4 (P=C-y),
        // W5 (P=C+z, P=C), W6 (P=C-z, P=C)
        T r_w = tz1p * (u_c * su_kp + u_w * su_kp_w) - tz20 * (u_kp * su_c_up + u_kp_w * su_w_up);
        r_w += tz1p * (v_c * sv_kp + v_s * sv_kp_s) - tz20 * (v_kp * sv_c_up + v_kp_s * sv_s_up);
        r_w += tcx * ((u_c + u_kp) * sw_e - (u_w + u_kp_w) * sw_w);
        r_w += tcy * ((v_c + v_kp) * sw_n - (v_s + v_kp_s) * sw_s);
        r_w += td1p * (w_kp + w_c + w_c) * sw_kp + td10 * w_kmc * sw_c;
        r_w -= td2m * (w_kmc + w_c + w_c) * sw_km + td20 * w_kp * sw_c;

        if (act) {
            if (a.accumulate) {
                gu[g] += r_u;
                gv[g] += r_v;
                gw[g] += r_w;
            } else {
                gu[g] = r_u;
                gv[g] = r_v;
                gw[g] = r_w;
            }
        }
        g += (size_t)a.sz;
        if (k + 1 < ke) level_coefs<T>(a, k + 1, tid, coef_s[(r + 1) & 1]);
        abort = __syncthreads_or(bad);  // level k-1's stage is free
        if (!abort && tid == 0 && issued < nseq) {
            fence_proxy_async_smem();
            adj_issue(ring, maps, issued, kb - 1 + issued, bxs, bys);
            ++issued;
        }
    }
    if (abort && tid == 0) {
        atomicOr(&tu_status, kStatusTimeout);
        for (int s = (issued > kS ? issued - kS : 0); s < issued; ++s) (void)ring.wait(s);
    }
}

// Transpose of the periodic halo fill: halo rows are added into the rows
// they were copied from and cleared, then halo columns likewise (the fill
// copied columns first, then full rows).
template <typename T>
__global__ void fold_halo_y_kernel(T* f, int nx, int ny, long long sy, long long sz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i > nx + 1) return;
    T* lev = f + (size_t)k * (size_t)sz;
    T* r0 = lev + i;
    T* r1 = lev + (size_t)sy + i;
    T* rn = lev + (size_t)ny * (size_t)sy + i;
    T* rn1 = lev + (size_t)(ny + 1) * (size_t)sy + i;
    const T g0 = *r0, gn1 = *rn1;
    *r0 = T(0);
    *rn1 = T(0);
    *rn += g0;
    *r1 += gn1;
}

template <typename T>
__global__ void fold_halo_x_kernel(T* f, int nx, int ny, int nz, long long sy, long long sz) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)nz * ny) return;
    const int k = (int)(r / ny), j = 1 + (int)(r % ny);
    T* row = f + (size_t)k * (size_t)sz + (size_t)j * (size_t)sy;
    const T g0 = row[0], gn1 = row[nx + 1];
    row[0] = T(0);
    row[nx + 1] = T(0);
    row[nx] += g0;
    row[1] += gn1;
}

}  // namespace

TileShape adjoint_shape(int elem_bytes) {
    if (elem_bytes == 8)
        return TileShape{kTX, kTY, AdjShape<double>::BX, AdjShape<double>::BY, AdjShape<double>::SMEM_BYTES,
                         AdjShape<double>::NT};
    return TileShape{kTX, kTY, AdjShape<float>::BX, AdjShape<float>::BY, AdjShape<float>::SMEM_BYTES,
                     AdjShape<float>::NT};
}

cudaError_t launch_adjoint(const CUtensorMap* maps6, int elem_bytes, const AdjArgs& a, cudaStream_t st) {
    AdjMaps m;
    for (int f = 0; f < kFields; ++f) m.m[f] = maps6[f];
    const int tx = (a.nx + 2 + kTX - 1) / kTX, ty = (a.ny + 2 + kTY - 1) / kTY;
    const long long tiles = (long long)tx * ty;
    cudaError_t e;
    int chunks = 1;
    if (elem_bytes == 8) {
        e = cudaFuncSetAttribute(adjoint_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 AdjShape<double>::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if ((e = choose_kchunks(adjoint_kernel<double>, kTX * kTY, AdjShape<double>::SMEM_BYTES, tiles, a.nz,
                                &chunks)) != cudaSuccess)
            return e;
        adjoint_kernel<double><<<dim3(tx, ty, chunks), kTX * kTY, AdjShape<double>::SMEM_BYTES, st>>>(m, a);
    } else {
        e = cudaFuncSetAttribute(adjoint_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 AdjShape<float>::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        if ((e = choose_kchunks(adjoint_kernel<float>, kTX * kTY, AdjShape<float>::SMEM_BYTES, tiles, a.nz,
                                &chunks)) != cudaSuccess)
            return e;
        adjoint_kernel<float><<<dim3(tx, ty, chunks), kTX * kTY, AdjShape<float>::SMEM_BYTES, st>>>(m, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_fold_halo(void* field, int elem_bytes, int nx, int ny, int nz, long long sy, long long sz,
                             cudaStream_t st) {
    dim3 gy((nx + 2 + 255) / 256, nz);
    const long long rows = (long long)nz * ny;
    const unsigned gx = (unsigned)((rows + 255) / 256);
    if (elem_bytes == 8) {
        fold_halo_y_kernel<double><<<gy, 256, 0, st>>>(static_cast<double*>(field), nx, ny, sy, sz);
        fold_halo_x_kernel<double><<<gx, 256, 0, st>>>(static_cast<double*>(field), nx, ny, nz, sy, sz);
    } else {
        fold_halo_y_kernel<float><<<gy, 256, 0, st>>>(static_cast<float*>(field), nx, ny, sy, sz);
        fold_halo_x_kernel<float><<<gx, 256, 0, st>>>(static_cast<float*>(field), nx, ny, nz, sy, sz);
    }
    return cudaGetLastError();
}

cudaError_t read_and_clear_status_adjoint(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

}  // namespace pw
