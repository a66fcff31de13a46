// pw_split.cu -- PW advection in FP32 on perturbations about per-level FP64
// means (PW_F32_SPLIT).
//
// Writing u = U(k) + u' (likewise v, w) with U(k) the level mean, the mean x
// mean parts of every horizontal flux difference cancel exactly, and each
// vertical flux difference leaves a per-level constant; pw_make_split_table
// forms those constants in FP64 and rounds them to float once. What remains
// is computed here in FP32 on the perturbations, so the difference-of-
// products fluxes cancel only perturbation-sized quantities. The k-march is
// the native kernel's (float TMA ring); each level's 32-float table row
// travels on the same mbarrier as the level's three field boxes.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw.h"
#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace {

constexpr int kTX = 32, kTY = 8, kS = 4;
using Shape = RingShape<float, kTX, kTY, kS>;
constexpr int kRowBytes = PW_SPLIT_NCOEF * 4;
// ring stages | ring barriers (padded to 64 B) | S table rows | alignment slack
constexpr int kRowOffset = Shape::S * Shape::STAGE_BYTES + 64;
constexpr int kSmemBytes = kRowOffset + kS * kRowBytes + 128;

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct SplitRing : Ring<Shape> {
    float* rows;  // [S][PW_SPLIT_NCOEF]
    __device__ __forceinline__ void issue_level(int lev, const CUtensorMap* mu, const CUtensorMap* mv,
                                                const CUtensorMap* mw, const float* table, int x0, int y0) {
        const int s = lev % Shape::S;
        uint64_t* bar = &full[s];
        unsigned char* dst = base + s * Shape::STAGE_BYTES;
        mbar_arrive_expect_tx(bar, 3 * Shape::BOX_BYTES + kRowBytes);
        tma_load_3d(dst, mu, bar, x0, y0, lev);
        tma_load_3d(dst + Shape::BOX_STRIDE, mv, bar, x0, y0, lev);
        tma_load_3d(dst + 2 * Shape::BOX_STRIDE, mw, bar, x0, y0, lev);
        bulk_load(rows + s * PW_SPLIT_NCOEF, table + (size_t)lev * PW_SPLIT_NCOEF, kRowBytes, bar);
    }
    __device__ __forceinline__ const float* row(int lev) const { return rows + (lev % Shape::S) * PW_SPLIT_NCOEF; }
};

__global__ void __launch_bounds__(Shape::NT) fwd_split_kernel(const __grid_constant__ CUtensorMap mu,
                                                              const __grid_constant__ CUtensorMap mv,
                                                              const __grid_constant__ CUtensorMap mw,
                                                              const FwdArgs a) {
    constexpr int TX = Shape::TX, TY = Shape::TY, S = Shape::S, BX = Shape::BX;
    extern __shared__ unsigned char smem_raw[];
    SplitRing ring;
    ring.setup(smem_raw);
    ring.rows = reinterpret_cast<float*>(ring.base + kRowOffset);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;
    const bool act = (i <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
    const float* table = a.split;

    if (tid == 0) {
        prefetch_tensormap(&mu);
        prefetch_tensormap(&mv);
        prefetch_tensormap(&mw);
        ring.init_barriers();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0) {
        for (; issued < S && issued < nz; ++issued) ring.issue_level(issued, &mu, &mv, &mw, table, x0, y0);
    }

    const int c0 = (ty + 1) * BX + (tx + 1);
    float* __restrict__ su = static_cast<float*>(a.su);
    float* __restrict__ sv = static_cast<float*>(a.sv);
    float* __restrict__ sw = static_cast<float*>(a.sw);
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i;
    const size_t gsz = (size_t)a.sz;

    bool bad = !ring.wait(0);
    if (nz > 1) bad |= !ring.wait(1);
    float uo_m, vo_m, wo_m, wx_m, wy_m, wz_m;
    {
        const float* U = ring.template box<float>(0, 0);
        const float* V = ring.template box<float>(0, 1);
        const float* W = ring.template box<float>(0, 2);
        uo_m = U[c0];
        vo_m = V[c0];
        wo_m = W[c0];
        wx_m = W[c0] + W[c0 + 1];
        wy_m = W[c0] + W[c0 + BX];
        wz_m = nz > 1 ? wo_m + ring.template box<float>(1, 2)[c0] : 0.0f;
    }
    if (act) {
        su[g] = 0.0f;
        sv[g] = 0.0f;
        sw[g] = 0.0f;
    }
    bool abort = __syncthreads_or(bad);
    if (!abort && tid == 0 && issued < nz) {
        fence_proxy_async_smem();
        ring.issue_level(issued, &mu, &mv, &mw, table, x0, y0);
        ++issued;
    }

    for (int k = 1; k < nz && !abort; ++k) {
        g += gsz;
        const bool top = (k == nz - 1);
        if (!top) bad |= !ring.wait(k + 1);
        const float* U = ring.template box<float>(k, 0);
        const float* V = ring.template box<float>(k, 1);
        const float* W = ring.template box<float>(k, 2);
        const float4* T4 = reinterpret_cast<const float4*>(ring.row(k));
        const float4 t0 = T4[0], t1 = T4[1], t2 = T4[2], t3 = T4[3];
        const float4 t4 = T4[4], t5 = T4[5], t6 = T4[6];
        const float tcx = t6.z, tcy = t6.w;

        const float uc = U[c0], uw = U[c0 - 1], ue = U[c0 + 1], us = U[c0 - BX], un = U[c0 + BX];
        const float unw = U[c0 + BX - 1];
        const float vc = V[c0], vw = V[c0 - 1], ve = V[c0 + 1], vs = V[c0 - BX], vn = V[c0 + BX];
        const float vse = V[c0 - BX + 1];
        const float wc = W[c0], ww = W[c0 - 1], we = W[c0 + 1], ws = W[c0 - BX], wn = W[c0 + BX];

        // su: self term, y cross term, lower vertical flux (table entries 0..6)
        float p = vs + vse, q = vc + ve;
        float r_su = tcx * (uw - ue) * (t0.x + uw + uc + ue);
        r_su += tcy * (t0.y * (us - un) + t0.z * (p - q) + us * p - un * q);
        r_su += t0.w + t1.x * (t1.y * wx_m + t1.z * uo_m + uo_m * wx_m);
        // sv: mirror (entries 10..15, shared vertical entries 4, 6, 7, 9)
        p = uw + unw;
        q = uc + un;
        float r_sv = tcy * (vs - vn) * (t2.z + vs + vc + vn);
        r_sv += tcx * (t2.w * (vw - ve) + t3.x * (p - q) + vw * p - ve * q);
        r_sv += t3.y + t1.x * (t3.z * wy_m + t1.z * vo_m + vo_m * wy_m);
        const float wx = wc + we, wy = wc + wn;
        float r_sw = 0.0f, wz = 0.0f;
        if (!top) {
            const float* Uu = ring.template box<float>(k + 1, 0);
            const float* Vu = ring.template box<float>(k + 1, 1);
            const float* Wu = ring.template box<float>(k + 1, 2);
            const float uu = Uu[c0], uuw = Uu[c0 - 1];
            const float vu = Vu[c0], vus = Vu[c0 - BX];
            const float wu = Wu[c0];
            // upper vertical fluxes of su and sv (entries 7, 8, 9, 15)
            r_su -= t1.w * (t2.x * wx + t2.y * uu + uu * wx);
            r_sv -= t1.w * (t3.w * wy + t2.y * vu + vu * wy);
            // sw (entries 16..25)
            wz = wc + wu;
            p = uw + uuw;
            q = uc + uu;
            r_sw = tcx * (t4.x * (p - q) + t4.y * (ww - we) + ww * p - we * q);
            p = vs + vus;
            q = vc + vu;
            r_sw += tcy * (t4.x * (p - q) + t4.z * (ws - wn) + ws * p - wn * q);
            r_sw += t4.w + t5.x * (wz_m * (t5.y + wo_m) + t5.z * wo_m);
            r_sw -= t5.w * (wz * (t6.x + wu) + t6.y * wu);
        }
        if (act) {
            su[g] = r_su;
            sv[g] = r_sv;
            sw[g] = r_sw;
        }
        uo_m = uc;
        vo_m = vc;
        wo_m = wc;
        wx_m = wx;
        wy_m = wy;
        wz_m = wz;

        abort = __syncthreads_or(bad);  // releases level k's stage
        if (!abort && tid == 0 && issued < nz) {
            fence_proxy_async_smem();
            ring.issue_level(issued, &mu, &mv, &mw, table, x0, y0);
            ++issued;
        }
    }
    if (abort && tid == 0) {
        atomicOr(&tu_status, kStatusTimeout);
        for (int lev = (issued > S ? issued - S : 0); lev < issued; ++lev) (void)ring.wait(lev);
    }
}

}  // namespace

cudaError_t read_and_clear_status_split(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

TileShape fwd_split_shape() { return TileShape{kTX, kTY, Shape::BX, Shape::BY, kSmemBytes, Shape::NT}; }

cudaError_t launch_fwd_split(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                             const FwdArgs& a, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(fwd_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kTX - 1) / kTX, (a.ny + kTY - 1) / kTY);
    fwd_split_kernel<<<grid, Shape::NT, kSmemBytes, st>>>(mu, mv, mw, a);
    return cudaGetLastError();
}

}  // namespace pw
