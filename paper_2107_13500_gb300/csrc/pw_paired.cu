// pw_paired.cu -- PW advection with FP64 inputs and outputs and paired-FP32
// arithmetic (PW_F64_PAIRED).
//
// Same k-march as the native kernel: a 4-stage TMA ring brings each level
// of u, v, w (tile + halo, doubles) into shared memory. Each level is then
// split once, cooperatively, into (hi, lo) float pairs in a second, two-level
// shared buffer, so neighbouring points do not split the same value again.
// Step k computes level k from the pairs of levels k and k+1 plus pairs of
// level k-1 carried in registers (own-column values and face sums of w).
// Per level: wait(k+1) -> split(k+1) -> barrier -> compute(k) -> barrier.
// Loads are numbered per CTA (`seq`), so the persistent form can run many
// tiles of many domains through one ring (see pw_ring.cuh).
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw.h"
#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_pair.cuh"
#include "pw_ring.cuh"

namespace pw {

namespace {

constexpr int kTX = 32, kTY = 8, kS = 4;
using Shape = RingShape<double, kTX, kTY, kS>;
constexpr int kBoxElems = Shape::BX * Shape::BY;
// pair buffers: [2 levels][3 fields][box] float2, then [2 levels][4] coefficient pairs
constexpr int kPairBytes = 2 * 3 * kBoxElems * 8;
constexpr int kCoefBytes = 2 * 4 * 8;
// ring stages | ring barriers (S x 8 B, padded to 64 B) | pairs | coefficient
// pairs | work-item slot, plus 128 B of slack for aligning the ring base
constexpr int kPairOffset = Shape::S * Shape::STAGE_BYTES + 64;
constexpr int kItemOffset = kPairOffset + kPairBytes + kCoefBytes;
constexpr int kSmemBytes = kItemOffset + 16 + 128;
static_assert(Shape::S * 8 <= 64, "ring barriers must fit before the pair buffers");

struct PairSmem {
    float2* pairs;    // [2][3][kBoxElems]
    float2* coef;     // [2][4]: tzc1, tzc2, tzd1, tzd2 of a level
    long long* item;  // work item handed from thread 0 to the CTA
    __device__ __forceinline__ const pf* field(int lev, int f) const {
        return reinterpret_cast<const pf*>(pairs + ((lev & 1) * 3 + f) * kBoxElems);
    }
    __device__ __forceinline__ pf cf(int lev, int n) const {
        const float2 c = coef[(lev & 1) * 4 + n];
        return {c.x, c.y};
    }
};

// Split load `seq` (= level `lev`) into pairs; threads 0..3 also split the
// level's four vertical coefficients.
__device__ __forceinline__ void convert_level(const Ring<Shape>& ring, const PairSmem& ps, long long seq, int lev,
                                              const FwdArgs& a, int tid) {
    float2* dst = ps.pairs + (lev & 1) * 3 * kBoxElems;
    for (int f = 0; f < 3; ++f) {
        const double* src = ring.template box<double>(seq, f);
        for (int e = tid; e < kBoxElems; e += Shape::NT) {
            const pf p = split_double(src[e]);
            dst[f * kBoxElems + e] = make_float2(p.h, p.l);
        }
    }
    if (tid < 4) {
        const double* arr = tid == 0 ? a.tzc1 : tid == 1 ? a.tzc2 : tid == 2 ? a.tzd1 : a.tzd2;
        const pf p = split_double(__ldg(arr + lev));
        ps.coef[(lev & 1) * 4 + tid] = make_float2(p.h, p.l);
    }
}

__device__ __forceinline__ pf ld(const pf* b, int idx) {
    const float2 v = reinterpret_cast<const float2*>(b)[idx];
    return {v.x, v.y};
}

// One tile (bx, by) of domain `a`; `seq` is the CTA's running load count.
// Returns false if a bounded wait expired (status set, copies drained).
__device__ bool paired_tile(Ring<Shape>& ring, const PairSmem& ps, const CUtensorMap* mu, const CUtensorMap* mv,
                            const CUtensorMap* mw, const FwdArgs& a, int bx, int by, long long& seq, int tid) {
    constexpr int TX = Shape::TX, S = Shape::S, BX = Shape::BX;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX, y0 = by * Shape::TY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;
    const bool act = (i <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
    const long long s0 = seq;

    int issued = 0;
    if (tid == 0) {
        fence_proxy_async_smem();
        for (; issued < S && issued < nz; ++issued) ring.issue(s0 + issued, issued, mu, mv, mw, x0, y0);
    }

    const pf tcx = split_double(a.tcx), tcy = split_double(a.tcy);
    const int c0 = (ty + 1) * BX + (tx + 1) + a.xoff;
    double* __restrict__ su = static_cast<double*>(a.su);
    double* __restrict__ sv = static_cast<double*>(a.sv);
    double* __restrict__ sw = static_cast<double*>(a.sw);
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i;
    const size_t gsz = (size_t)a.sz;

    // Levels 0 and 1 are split up front; later steps split level k+1.
    const int pre = nz > 1 ? 2 : 1;
    bool bad = false;
    for (int lev = 0; lev < pre; ++lev) {
        bad |= !ring.wait(s0 + lev);
        convert_level(ring, ps, s0 + lev, lev, a, tid);
    }
    bool abort = __syncthreads_or(bad);
    if (!abort && tid == 0) {
        fence_proxy_async_smem();
        for (int n = 0; n < pre && issued < nz; ++n, ++issued) ring.issue(s0 + issued, issued, mu, mv, mw, x0, y0);
    }

    pf uo_m, vo_m, wo_m, wx_m, wy_m, wz_m;
    {
        const pf* U = ps.field(0, 0);
        const pf* V = ps.field(0, 1);
        const pf* W = ps.field(0, 2);
        uo_m = ld(U, c0);
        vo_m = ld(V, c0);
        wo_m = ld(W, c0);
        wx_m = padd(wo_m, ld(W, c0 + 1));
        wy_m = padd(wo_m, ld(W, c0 + BX));
        wz_m = nz > 1 ? padd(ld(ps.field(1, 2), c0), wo_m) : pf{0.f, 0.f};
    }
    __syncthreads();  // level 0's pair slot is rewritten by the first step
    if (act) {
        su[g] = 0.0;
        sv[g] = 0.0;
        sw[g] = 0.0;
    }

    for (int k = 1; k < nz && !abort; ++k) {
        g += gsz;
        const bool top = (k == nz - 1);
        if (!top) {
            // split level k+1 (its pair slot held level k-1, consumed last step)
            bad |= !ring.wait(s0 + k + 1);
            convert_level(ring, ps, s0 + k + 1, k + 1, a, tid);
            abort = __syncthreads_or(bad);
            if (abort) break;
            if (tid == 0 && issued < nz) {
                fence_proxy_async_smem();
                ring.issue(s0 + issued, issued, mu, mv, mw, x0, y0);
                ++issued;
            }
        }
        const pf* U = ps.field(k, 0);
        const pf* V = ps.field(k, 1);
        const pf* W = ps.field(k, 2);
        const pf uc = ld(U, c0), uw = ld(U, c0 - 1), ue = ld(U, c0 + 1), us = ld(U, c0 - BX), un = ld(U, c0 + BX);
        const pf unw = ld(U, c0 + BX - 1);
        const pf vc = ld(V, c0), vw = ld(V, c0 - 1), ve = ld(V, c0 + 1), vs = ld(V, c0 - BX), vn = ld(V, c0 + BX);
        const pf vse = ld(V, c0 - BX + 1);
        const pf wc = ld(W, c0), ww = ld(W, c0 - 1), we = ld(W, c0 + 1), ws = ld(W, c0 - BX), wn = ld(W, c0 + BX);
        const pf tz1 = ps.cf(k, 0), tz2 = ps.cf(k, 1);

        // su: tcx (a-c)(a+b+c) + tcy [u(j-1) V(j-1) - u(j+1) V(j)] + tzc1 u(k-1) W(k-1) - tzc2 u(k+1) W(k)
        pf r_su = pmul(tcx, pmul(psub(uw, ue), padd(padd(uw, uc), ue)));
        r_su = padd(r_su, pmul(tcy, psub(pmul(us, padd(vs, vse)), pmul(un, padd(vc, ve)))));
        r_su = padd(r_su, pmul(tz1, pmul(uo_m, wx_m)));
        // sv: mirror of su in x and y
        pf r_sv = pmul(tcy, pmul(psub(vs, vn), padd(padd(vs, vc), vn)));
        r_sv = padd(r_sv, pmul(tcx, psub(pmul(vw, padd(uw, unw)), pmul(ve, padd(uc, un)))));
        r_sv = padd(r_sv, pmul(tz1, pmul(vo_m, wy_m)));
        const pf wx = padd(wc, we), wy = padd(wc, wn);
        double d_sw = 0.0;
        pf wz = {0.f, 0.f};
        if (!top) {
            const pf* Uu = ps.field(k + 1, 0);
            const pf* Vu = ps.field(k + 1, 1);
            const pf* Wu = ps.field(k + 1, 2);
            const pf uu = ld(Uu, c0), uuw = ld(Uu, c0 - 1);
            const pf vu = ld(Vu, c0), vus = ld(Vu, c0 - BX);
            const pf wu = ld(Wu, c0);
            const pf td1 = ps.cf(k, 2), td2 = ps.cf(k, 3);
            r_su = psub(r_su, pmul(tz2, pmul(uu, wx)));
            r_sv = psub(r_sv, pmul(tz2, pmul(vu, wy)));
            wz = padd(wc, wu);
            pf r_sw = pmul(tcx, psub(pmul(ww, padd(uw, uuw)), pmul(we, padd(uc, uu))));
            r_sw = padd(r_sw, pmul(tcy, psub(pmul(ws, padd(vs, vus)), pmul(wn, padd(vc, vu)))));
            r_sw = padd(r_sw, psub(pmul(td1, pmul(wo_m, wz_m)), pmul(td2, pmul(wu, wz))));
            d_sw = pair_to_double(r_sw);
        }
        if (act) {
            su[g] = pair_to_double(r_su);
            sv[g] = pair_to_double(r_sv);
            sw[g] = d_sw;
        }
        uo_m = uc;
        vo_m = vc;
        wo_m = wc;
        wx_m = wx;
        wy_m = wy;
        wz_m = wz;
        abort = __syncthreads_or(bad);  // level k's pairs are free after this
    }
    if (abort) {
        if (tid == 0) {
            atomicOr(&tu_status, kStatusTimeout);
            for (int lev = (issued > S ? issued - S : 0); lev < issued; ++lev) (void)ring.wait(s0 + lev);
        }
        return false;
    }
    seq = s0 + nz;
    return true;
}

__device__ __forceinline__ void setup_smem(unsigned char* raw, Ring<Shape>& ring, PairSmem& ps) {
    ring.setup(raw);
    ps.pairs = reinterpret_cast<float2*>(ring.base + kPairOffset);
    ps.coef = ps.pairs + 2 * 3 * kBoxElems;
    ps.item = reinterpret_cast<long long*>(ring.base + kItemOffset);
}

__global__ void __launch_bounds__(Shape::NT) fwd_paired_kernel(const __grid_constant__ CUtensorMap mu,
                                                               const __grid_constant__ CUtensorMap mv,
                                                               const __grid_constant__ CUtensorMap mw,
                                                               const FwdArgs a) {
    extern __shared__ unsigned char smem_raw[];
    Ring<Shape> ring;
    PairSmem ps;
    setup_smem(smem_raw, ring, ps);
    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_tensormap(&mu);
        prefetch_tensormap(&mv);
        prefetch_tensormap(&mw);
        ring.init_barriers();
    }
    __syncthreads();
    long long seq = 0;
    (void)paired_tile(ring, ps, &mu, &mv, &mw, a, blockIdx.x, blockIdx.y, seq, tid);
}

// Persistent form over a batch plan: work items (one tile of one domain)
// come from the plan's counter, at most n_items iterations.
__global__ void __launch_bounds__(Shape::NT) fwd_paired_batched(BatchPlan* plan) {
    extern __shared__ unsigned char smem_raw[];
    Ring<Shape> ring;
    PairSmem ps;
    setup_smem(smem_raw, ring, ps);
    const int tid = threadIdx.x;
    if (plan->variant != 0 || plan->dtype != PW_F64_PAIRED) {
        if (tid == 0) atomicOr(&tu_status, kStatusBadPlan);
        return;
    }
    if (tid == 0) ring.init_barriers();
    __syncthreads();
    const long long n_items = plan->n_items;
    long long seq = 0;
    for (long long it = 0; it < n_items; ++it) {
        if (tid == 0) *ps.item = (long long)atomicAdd(&plan->counter, 1ull);
        __syncthreads();
        const long long item = *ps.item;
        __syncthreads();  // every thread has read the slot before thread 0 rewrites it
        if (item >= n_items) break;
        const BatchDomain& d = plan->dom[find_domain(plan, item)];
        const long long t = item - d.first_item;
        if (!paired_tile(ring, ps, &d.mu, &d.mv, &d.mw, d.args, (int)(t % d.tiles_x), (int)(t / d.tiles_x), seq,
                         tid))
            break;
    }
}

}  // namespace

cudaError_t read_and_clear_status_paired(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

TileShape fwd_paired_shape() { return TileShape{kTX, kTY, Shape::BX, Shape::BY, kSmemBytes, Shape::NT}; }

cudaError_t launch_fwd_paired(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                              const FwdArgs& a, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(fwd_paired_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + kTX - 1) / kTX, (a.ny + kTY - 1) / kTY);
    fwd_paired_kernel<<<grid, Shape::NT, kSmemBytes, st>>>(mu, mv, mw, a);
    return cudaGetLastError();
}

cudaError_t launch_paired_batched(BatchPlan* plan, long long n_items, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(fwd_paired_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    long long grid = 0;
    if ((e = persistent_grid(fwd_paired_batched, Shape::NT, kSmemBytes, n_items, &grid)) != cudaSuccess) return e;
    if (grid < 1) return cudaSuccess;
    fwd_paired_batched<<<(unsigned)grid, Shape::NT, kSmemBytes, st>>>(plan);
    return cudaGetLastError();
}

}  // namespace pw
