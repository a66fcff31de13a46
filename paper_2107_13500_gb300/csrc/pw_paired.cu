// pw_paired.cu -- PW advection with FP64 inputs and outputs and paired-FP32
// arithmetic (PW_F64_PAIRED).
//
// Same k-march as the native kernel: a 3-stage TMA ring brings each level
// of u, v, w (tile + halo, doubles) into shared memory. Each level is then
// split once, cooperatively, into (hi, lo) float pairs in a second,
// three-level shared ring, so neighbouring points do not split the same
// value again. Step k computes level k from the pairs of levels k and k+1
// plus pairs of level k-1 carried in registers (own-column values and face
// sums of w), and splits level k+2 for the next step; one CTA barrier per
// level both publishes level k+2's pairs and frees level k's slot.
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

constexpr int kTX = 32, kTY = 8, kS = 3, kPL = 3;  // TMA stages, pair-ring levels
using Shape = RingShape<double, kTX, kTY, kS>;
constexpr int kBoxElems = Shape::BX * Shape::BY;
static_assert(kBoxElems % 2 == 0, "the split pass moves two doubles at a time");
// pair ring: [kPL levels][3 fields][box] float2, then [kPL levels][4] coefficient pairs
constexpr int kPairBytes = kPL * 3 * kBoxElems * 8;
constexpr int kCoefBytes = kPL * 4 * 8;
// ring stages | ring barriers (S x 8 B, padded to 64 B) | pairs | coefficient
// pairs | work-item slot, plus 128 B of slack for aligning the ring base
constexpr int kPairOffset = Shape::S * Shape::STAGE_BYTES + 64;
constexpr int kItemOffset = kPairOffset + kPairBytes + kCoefBytes;
constexpr int kSmemBytes = kItemOffset + 16 + 128;
static_assert(Shape::S * 8 <= 64, "ring barriers must fit before the pair buffers");

struct PairSmem {
    float2* pairs;    // [kPL][3][kBoxElems]
    float2* coef;     // [kPL][4]: tzc1, tzc2, tzd1, tzd2 of a level
    long long* item;  // work item handed from thread 0 to the CTA
    __device__ __forceinline__ const pf* field(int lev, int f) const {
        return reinterpret_cast<const pf*>(pairs + ((lev % kPL) * 3 + f) * kBoxElems);
    }
    __device__ __forceinline__ pf cf(int lev, int n) const {
        const float2 c = coef[(lev % kPL) * 4 + n];
        return {c.x, c.y};
    }
};

// Split load `seq` (level `lev`) into pair slot `slot`, two doubles per
// 16-byte shared read and two pairs per 16-byte write; threads 0..3 also
// split the level's four vertical coefficients into the same slot.
__device__ __forceinline__ void convert_level(const Ring<Shape>& ring, const PairSmem& ps, long long seq, int lev,
                                              int slot, const FwdArgs& a, int tid) {
    float4* dst = reinterpret_cast<float4*>(ps.pairs + (slot % kPL) * 3 * kBoxElems);
    for (int f = 0; f < 3; ++f) {
        const double2* src = reinterpret_cast<const double2*>(ring.template box<double>(seq, f));
        for (int e = tid; e < kBoxElems / 2; e += Shape::NT) {
            const double2 d = src[e];
            const pf p0 = split_double(d.x), p1 = split_double(d.y);
            dst[f * (kBoxElems / 2) + e] = make_float4(p0.h, p0.l, p1.h, p1.l);
        }
    }
    if (tid < 4) {
        const double* arr = tid == 0 ? a.tzc1 : tid == 1 ? a.tzc2 : tid == 2 ? a.tzd1 : a.tzd2;
        const pf p = split_double(__ldg(arr + lev));
        ps.coef[(slot % kPL) * 4 + tid] = make_float2(p.h, p.l);
    }
}

__device__ __forceinline__ pf ld(const pf* b, int idx) {
    const float2 v = reinterpret_cast<const float2*>(b)[idx];
    return {v.x, v.y};
}

// One tile (bx, by) of domain `a`, output levels kb..ke-1 (a k-chunk; the
// chunk reads one level below and one above). `seq` is the CTA's running
// load count. Loads, pair slots and coefficient slots are numbered relative
// to the lowest level read, lo. Returns false if a bounded wait expired
// (status set, copies drained).
__device__ bool paired_tile(Ring<Shape>& ring, const PairSmem& ps, const CUtensorMap* mu, const CUtensorMap* mv,
                            const CUtensorMap* mw, const FwdArgs& a, int bx, int by, int kb, int ke,
                            long long& seq, int tid) {
    constexpr int TX = Shape::TX, S = Shape::S, BX = Shape::BX;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX, y0 = by * Shape::TY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;
    const bool act = (i <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
    const int lo = kb > 0 ? kb - 1 : 0, hi = ke < nz ? ke : nz - 1;
    const int nl = hi - lo + 1;  // levels read
    const long long s0 = seq;

    int issued = 0;  // relative loads issued (thread 0)
    if (tid == 0) {
        fence_proxy_async_smem();
        for (; issued < S && issued < nl; ++issued) ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
    }

    const pf tcx = split_double(a.tcx), tcy = split_double(a.tcy);
    const int c0 = (ty + 1) * BX + (tx + 1) + a.xoff;
    double* __restrict__ su = static_cast<double*>(a.su);
    double* __restrict__ sv = static_cast<double*>(a.sv);
    double* __restrict__ sw = static_cast<double*>(a.sw);
    const size_t gsz = (size_t)a.sz;
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)lo * gsz;

    // Relative levels 0..2 are split up front; the step at relative level r
    // splits r+2.
    const int pre = nl < kPL ? nl : kPL;
    bool bad = false;
    for (int r = 0; r < pre; ++r) {
        bad |= !ring.wait(s0 + r);
        convert_level(ring, ps, s0 + r, lo + r, r, a, tid);
    }
    bool abort = __syncthreads_or(bad);
    if (!abort && tid == 0) {
        fence_proxy_async_smem();
        for (int n = 0; n < pre && issued < nl; ++n, ++issued) ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
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
        wz_m = nl > 1 ? padd(ld(ps.field(1, 2), c0), wo_m) : pf{0.f, 0.f};
    }
    if (act && kb == 0) {  // level 1 of the paper is not computed
        su[g] = 0.0;
        sv[g] = 0.0;
        sw[g] = 0.0;
    }
    abort = __syncthreads_or(bad);  // relative slot 0 is rewritten by the first step

    for (int k = (kb > 1 ? kb : 1); k < ke && !abort; ++k) {
        const int r = k - lo;
        g += gsz;
        const bool top = (k == nz - 1);
        if (r + 2 < nl) {
            // split relative level r+2 into the slot of r-1 (freed by the last barrier)
            bad |= !ring.wait(s0 + r + 2);
            convert_level(ring, ps, s0 + r + 2, k + 2, r + 2, a, tid);
        }
        const pf* U = ps.field(r, 0);
        const pf* V = ps.field(r, 1);
        const pf* W = ps.field(r, 2);
        const pf uc = ld(U, c0), uw = ld(U, c0 - 1), ue = ld(U, c0 + 1), us = ld(U, c0 - BX), un = ld(U, c0 + BX);
        const pf unw = ld(U, c0 + BX - 1);
        const pf vc = ld(V, c0), vw = ld(V, c0 - 1), ve = ld(V, c0 + 1), vs = ld(V, c0 - BX), vn = ld(V, c0 + BX);
        const pf vse = ld(V, c0 - BX + 1);
        const pf wc = ld(W, c0), ww = ld(W, c0 - 1), we = ld(W, c0 + 1), ws = ld(W, c0 - BX), wn = ld(W, c0 + BX);
        const pf tz1 = ps.cf(r, 0), tz2 = ps.cf(r, 1);

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
            const pf* Uu = ps.field(r + 1, 0);
            const pf* Vu = ps.field(r + 1, 1);
            const pf* Wu = ps.field(r + 1, 2);
            const pf uu = ld(Uu, c0), uuw = ld(Uu, c0 - 1);
            const pf vu = ld(Vu, c0), vus = ld(Vu, c0 - BX);
            const pf wu = ld(Wu, c0);
            const pf td1 = ps.cf(r, 2), td2 = ps.cf(r, 3);
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
        // publishes r+2's pairs, frees r's slot and r+2's TMA stage
        abort = __syncthreads_or(bad);
        if (!abort && tid == 0 && issued < nl) {
            fence_proxy_async_smem();
            ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
            ++issued;
        }
    }
    if (abort) {
        if (tid == 0) {
            atomicOr(&tu_status, kStatusTimeout);
            for (int q = (issued > S ? issued - S : 0); q < issued; ++q) (void)ring.wait(s0 + q);
        }
        return false;
    }
    seq = s0 + nl;
    return true;
}

__device__ __forceinline__ void setup_smem(unsigned char* raw, Ring<Shape>& ring, PairSmem& ps) {
    ring.setup(raw);
    ps.pairs = reinterpret_cast<float2*>(ring.base + kPairOffset);
    ps.coef = ps.pairs + kPL * 3 * kBoxElems;
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
    const int kb = (int)((long long)a.nz * blockIdx.z / gridDim.z);
    const int ke = (int)((long long)a.nz * (blockIdx.z + 1) / gridDim.z);
    (void)paired_tile(ring, ps, &mu, &mv, &mw, a, blockIdx.x, blockIdx.y, kb, ke, seq, tid);
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
        // private copy (see the FP32 batched kernel)
        const FwdArgs args = d.args;
        const long long t = item - d.first_item;
        const int tiles_x = d.tiles_x, kchunks = d.kchunks;
        const long long tiles = (long long)tiles_x * d.tiles_y;
        const int ch = (int)(t / tiles), tt = (int)(t % tiles);
        const int kb = (int)((long long)args.nz * ch / kchunks);
        const int ke = (int)((long long)args.nz * (ch + 1) / kchunks);
        if (!paired_tile(ring, ps, &d.mu, &d.mv, &d.mw, args, tt % tiles_x, tt / tiles_x, kb, ke, seq, tid)) break;
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
    const long long tiles = (long long)((a.nx + kTX - 1) / kTX) * ((a.ny + kTY - 1) / kTY);
    int chunks = 1;
    if ((e = choose_kchunks(fwd_paired_kernel, Shape::NT, kSmemBytes, tiles, a.nz, &chunks)) != cudaSuccess) return e;
    dim3 grid((a.nx + kTX - 1) / kTX, (a.ny + kTY - 1) / kTY, chunks);
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
