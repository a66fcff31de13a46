// pw_paired.cu -- PW advection with FP64 inputs and outputs and paired-FP32
// arithmetic (PW_F64_PAIRED).
//
// Same k-march as the native kernel: a 2-stage TMA ring brings each level
// of u, v, w (tile + halo, doubles) into shared memory. Each level is then
// split once, cooperatively, into (hi, lo) float pairs in a second,
// three-level shared ring, so neighbouring points do not split the same
// value again; a TMA stage is free again as soon as its level is split.
// Two stages keep the shared memory at five CTAs per SM. Step k computes level k from the pairs of levels k and k+1
// plus pairs of level k-1 carried in registers (own-column values and face
// sums of w), and splits level k+2 for the next step; one CTA barrier per
// level both publishes level k+2's pairs and frees level k's slot.
//
// Each thread evaluates two points of one tile row, A = (x0+1+t, j) and
// B = A + TX/2 in x, on packed FP32 lanes (pw_pair.cuh: f32x2 add/mul/fma,
// the same rounding per lane as the scalar form). Because A and B sit at
// the same offset in the two halves of the tile, every stencil neighbour of
// the pair is the same offset in both halves: the pair ring interleaves the
// halves, so one 16-byte read {hA, hB, lA, lB} gives a neighbour of both
// points already in lane order.
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

// Tile height and TMA stages of a variant (the tile is 32 points wide: the
// two lanes of a thread are 16 apart).
template <int TY_, int S_>
struct PairedCfg {
    static constexpr int kTX = 32, kTY = TY_, kS = S_, kPL = 3;  // TMA stages, pair-ring levels
    using Shape = RingShape<double, kTX, kTY, kS>;
    static constexpr int kHalf = kTX / 2;          // x distance from A to B; threads per tile row
    static constexpr int kNT = kHalf * kTY;
    static constexpr int kHX = kHalf + 2;          // pair-box row: columns x' = 0..kHalf+1 of both halves
    static constexpr int kBoxItems = Shape::BY * kHX;  // float4 {hA, hB, lA, lB} per field and level
    // pair ring: [kPL levels][3 fields][kBoxItems] float4, then [kPL levels][4]
    // coefficients as float4 {h, h, l, l}
    static constexpr int kPairBytes = kPL * 3 * kBoxItems * 16;
    static constexpr int kCoefBytes = kPL * 4 * 16;
    // ring stages | ring barriers (S x 8 B, padded to 64 B) | pairs | coefficient
    // pairs | work-item slot, plus 128 B of slack for aligning the ring base
    static constexpr int kPairOffset = Shape::S * Shape::STAGE_BYTES + 64;
    static constexpr int kItemOffset = kPairOffset + kPairBytes + kCoefBytes;
    static constexpr int kSmemBytes = kItemOffset + 16 + 128;
    // CTAs per SM the shared memory allows (1 KB per CTA is reserved by the
    // hardware); the register budget follows from it.
    static constexpr int kMinBlocks = (227 * 1024) / (kSmemBytes + 1024);
    // split work per thread and level (see ConvPlan)
    static constexpr int kConvIters = (3 * kBoxItems + kNT - 1) / kNT;
    // Per-level extra work is spread over warps: thread 0 issues the TMA
    // loads, warp kCoefWarp splits the four vertical coefficients, and the
    // split items are rotated by one warp so the partial last round of items
    // falls on the last warp.
    static constexpr int kCoefWarp = kNT >= 96 ? 2 : 0;
    static_assert((kHX - 1) + kHalf + Shape::XOFF_MAX < Shape::BX,
                  "both halves' columns must lie inside the TMA box row");
    static_assert(Shape::S * 8 <= 64, "ring barriers must fit before the pair buffers");
    // A stage is reissued once its level is split, so two stages keep one load
    // in flight while the other level is split.
    static_assert(kS >= 2, "the TMA ring needs a load in flight behind the one being split");
    static_assert(Shape::BOX_STRIDE % 8 == 0, "box stride in doubles");
};

// The batched variants (the autotuner's search space); variant 0 also serves
// pw_advect.
using PV0 = PairedCfg<8, 2>;
using PV1 = PairedCfg<4, 2>;
using PV2 = PairedCfg<16, 2>;
using PV3 = PairedCfg<8, 3>;

// The device code of one variant: constants of C in scope.
template <class C>
struct PairedK : C {
    using typename C::Shape;
    using C::kTX;
    using C::kTY;
    using C::kPL;
    using C::kHalf;
    using C::kNT;
    using C::kHX;
    using C::kBoxItems;
    using C::kPairOffset;
    using C::kItemOffset;
    using C::kConvIters;
    using C::kCoefWarp;

struct PairSmem {
    float4* pairs;    // [kPL][3][kBoxItems]
    float4* coef;     // [kPL][4]: tzc1, tzc2, tzd1, tzd2 of a level
    long long* item;  // work item handed from thread 0 to the CTA
    __device__ __forceinline__ const float4* field(int lev, int f) const {
        return pairs + ((lev % kPL) * 3 + f) * kBoxItems;
    }
    __device__ __forceinline__ pf2 cf(int lev, int n) const {
        const float4 c = coef[(lev % kPL) * 4 + n];
        return {make_float2(c.x, c.y), make_float2(c.z, c.w)};
    }
};

// The split pass gives thread t the items t', t' + kNT, ... of a level, with
// t' = (t + 32) mod kNT (item n = (field, row, x') of the pair slot). Which
// doubles of a stage those are does not depend on the level or the tile, so
// each thread works out their offsets once.
struct ConvPlan {
    int off[kConvIters];  // offset (doubles) in a stage of lane A's value of item tid + q*kNT, xoff = 0
};

static __device__ __forceinline__ int conv_item(int tid, int q) { return (tid + 32) % kNT + q * kNT; }

static __device__ __forceinline__ ConvPlan make_conv_plan(int tid) {
    ConvPlan cp;
#pragma unroll
    for (int q = 0; q < kConvIters; ++q) {
        const int n = conv_item(tid, q);
        const int f = n / kBoxItems, e = n - f * kBoxItems;
        const int row = e / kHX, xp = e - row * kHX;
        cp.off[q] = f * (Shape::BOX_STRIDE / 8) + row * Shape::BX + xp;
    }
    return cp;
}

// Vertical coefficient n (tzc1, tzc2, tzd1, tzd2) of level lev for lane n =
// 0..3 of warp kCoefWarp, 0 elsewhere.
static __device__ __forceinline__ double coef_for(const FwdArgs& a, int lev, int tid) {
    const int n = tid - 32 * kCoefWarp;
    if ((unsigned)n >= 4u) return 0.0;
    const double* arr = n == 0 ? a.tzc1 : n == 1 ? a.tzc2 : n == 2 ? a.tzd1 : a.tzd2;
    return __ldg(arr + lev);
}

// Split load `seq` (level `lev`) into pair slot `slot`: item (row, x') of a
// field takes the doubles of columns x0 + x' (lane A) and x0 + x' + kHalf
// (lane B) of its box. Lanes 0..3 of warp kCoefWarp also split the level's
// four vertical coefficients, given in `coef` (loaded one conversion
// earlier), into the same slot.
static __device__ __forceinline__ void convert_level(const Ring<Shape>& ring, const PairSmem& ps, long long seq, int lev,
                                              int slot, const FwdArgs& a, int tid, const ConvPlan& cp, double coef) {
    float4* dst = ps.pairs + (slot % kPL) * 3 * kBoxItems;
    const double* base = ring.template box<double>(seq, 0) + a.xoff;
#pragma unroll
    for (int q = 0; q < kConvIters; ++q) {
        const int n = conv_item(tid, q);
        if ((q + 1) * kNT <= 3 * kBoxItems || n < 3 * kBoxItems) {
            const double* src = base + cp.off[q];
            const pf p0 = split_double(src[0]), p1 = split_double(src[kHalf]);
            dst[n] = make_float4(p0.h, p1.h, p0.l, p1.l);
        }
    }
    const int cn = tid - 32 * kCoefWarp;
    if ((unsigned)cn < 4u) {
        const pf p = split_double(coef);
        ps.coef[(slot % kPL) * 4 + cn] = make_float4(p.h, p.h, p.l, p.l);
    }
}

static __device__ __forceinline__ pf2 ld(const float4* b, int idx) {
    const float4 v = b[idx];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

static __device__ __forceinline__ double join_a(const pf2& p) { return pair_to_double(pf{p.h.x, p.l.x}); }
static __device__ __forceinline__ double join_b(const pf2& p) { return pair_to_double(pf{p.h.y, p.l.y}); }

// One tile (bx, by) of domain `a`, output levels kb..ke-1 (a k-chunk; the
// chunk reads one level below and one above). `seq` is the CTA's running
// load count. Loads, pair slots and coefficient slots are numbered relative
// to the lowest level read, lo. Returns false if a bounded wait expired
// (status set, copies drained).
static __device__ bool paired_tile(Ring<Shape>& ring, const PairSmem& ps, const CUtensorMap* mu, const CUtensorMap* mv,
                            const CUtensorMap* mw, const FwdArgs& a, int bx, int by, int kb, int ke,
                            long long& seq, int tid, const ConvPlan& cp) {
    constexpr int S = Shape::S;
    const int tx = tid % kHalf, ty = tid / kHalf;
    const int x0 = bx * kTX, y0 = by * kTY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;  // point A; B is i + kHalf
    const bool act_a = (i <= a.nx) && (j <= a.ny);
    const bool act_b = (i + kHalf <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
    const int lo = kb > 0 ? kb - 1 : 0, hi = ke < nz ? ke : nz - 1;
    const int nl = hi - lo + 1;  // levels read
    const long long s0 = seq;

    int issued = 0;  // relative loads issued (thread 0)
    if (tid == 0) {
        fence_proxy_async_smem();
        for (; issued < S && issued < nl; ++issued) ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
    }

    const pf2 tcx = dup2(split_double(a.tcx)), tcy = dup2(split_double(a.tcy));
    const int c = (ty + 1) * kHX + (tx + 1);  // pair item of (A, B)
    double* __restrict__ su = static_cast<double*>(a.su);
    double* __restrict__ sv = static_cast<double*>(a.sv);
    double* __restrict__ sw = static_cast<double*>(a.sw);
    const size_t gsz = (size_t)a.sz;
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)lo * gsz;

    // Relative levels 0..2 are split up front, each stage reissued as soon
    // as its level is split; the step at relative level r splits r+2.
    const int pre = nl < kPL ? nl : kPL;
    bool bad = false, abort = false;
    double c_pre = coef_for(a, lo, tid);  // next level's coefficient, one conversion ahead
    for (int r = 0; r < pre && !abort; ++r) {
        bad |= !ring.wait(s0 + r);
        convert_level(ring, ps, s0 + r, lo + r, r, a, tid, cp, c_pre);
        c_pre = (lo + r + 1 <= hi) ? coef_for(a, lo + r + 1, tid) : 0.0;
        abort = __syncthreads_or(bad);  // load r's stage is free again
        if (!abort && tid == 0 && issued < nl) {
            fence_proxy_async_smem();
            ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
            ++issued;
        }
    }

    pf2 uo_m, vo_m, wo_m, wx_m, wy_m, wz_m;
    {
        const float4* U = ps.field(0, 0);
        const float4* V = ps.field(0, 1);
        const float4* W = ps.field(0, 2);
        uo_m = ld(U, c);
        vo_m = ld(V, c);
        wo_m = ld(W, c);
        wx_m = padd2(wo_m, ld(W, c + 1));
        wy_m = padd2(wo_m, ld(W, c + kHX));
        wz_m = nl > 1 ? padd2(ld(ps.field(1, 2), c), wo_m) : pf2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
    if (kb == 0) {  // level 1 of the paper is not computed
        if (act_a) {
            su[g] = 0.0;
            sv[g] = 0.0;
            sw[g] = 0.0;
        }
        if (act_b) {
            su[g + kHalf] = 0.0;
            sv[g + kHalf] = 0.0;
            sw[g + kHalf] = 0.0;
        }
    }
    abort = __syncthreads_or(bad);  // relative slot 0 is rewritten by the first step

    // two levels per unrolled iteration: the level-(k-1) carries swap
    // registers instead of being copied
#pragma unroll 2
    for (int k = (kb > 1 ? kb : 1); k < ke && !abort; ++k) {
        const int r = k - lo;
        g += gsz;
        const bool top = (k == nz - 1);
        if (r + 2 < nl) {
            // split relative level r+2 into the slot of r-1 (freed by the last barrier)
            bad |= !ring.wait(s0 + r + 2);
            convert_level(ring, ps, s0 + r + 2, k + 2, r + 2, a, tid, cp, c_pre);
            c_pre = (k + 3 <= hi) ? coef_for(a, k + 3, tid) : 0.0;
        }
        const float4* U = ps.field(r, 0);
        const float4* V = ps.field(r, 1);
        const float4* W = ps.field(r, 2);
        const pf2 uc = ld(U, c), uw = ld(U, c - 1), ue = ld(U, c + 1), us = ld(U, c - kHX), un = ld(U, c + kHX);
        const pf2 unw = ld(U, c + kHX - 1);
        const pf2 vc = ld(V, c), vw = ld(V, c - 1), ve = ld(V, c + 1), vs = ld(V, c - kHX), vn = ld(V, c + kHX);
        const pf2 vse = ld(V, c - kHX + 1);
        const pf2 wc = ld(W, c), ww = ld(W, c - 1), we = ld(W, c + 1), ws = ld(W, c - kHX), wn = ld(W, c + kHX);
        const pf2 tz1 = ps.cf(r, 0), tz2 = ps.cf(r, 1);

        // su: tcx (a-c)(a+b+c) + tcy [u(j-1) V(j-1) - u(j+1) V(j)] + tzc1 u(k-1) W(k-1) - tzc2 u(k+1) W(k)
        pf2 r_su = pmul2(tcx, pmul2(psub2(uw, ue), padd2(padd2(uw, uc), ue)));
        r_su = padd2(r_su, pmul2(tcy, psub2(pmul2(us, padd2(vs, vse)), pmul2(un, padd2(vc, ve)))));
        r_su = padd2(r_su, pmul2(tz1, pmul2(uo_m, wx_m)));
        // sv: mirror of su in x and y
        pf2 r_sv = pmul2(tcy, pmul2(psub2(vs, vn), padd2(padd2(vs, vc), vn)));
        r_sv = padd2(r_sv, pmul2(tcx, psub2(pmul2(vw, padd2(uw, unw)), pmul2(ve, padd2(uc, un)))));
        r_sv = padd2(r_sv, pmul2(tz1, pmul2(vo_m, wy_m)));
        const pf2 wx = padd2(wc, we), wy = padd2(wc, wn);
        double sw_a = 0.0, sw_b = 0.0;
        pf2 wz = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (!top) {
            const float4* Uu = ps.field(r + 1, 0);
            const float4* Vu = ps.field(r + 1, 1);
            const float4* Wu = ps.field(r + 1, 2);
            const pf2 uu = ld(Uu, c), uuw = ld(Uu, c - 1);
            const pf2 vu = ld(Vu, c), vus = ld(Vu, c - kHX);
            const pf2 wu = ld(Wu, c);
            const pf2 td1 = ps.cf(r, 2), td2 = ps.cf(r, 3);
            r_su = psub2(r_su, pmul2(tz2, pmul2(uu, wx)));
            r_sv = psub2(r_sv, pmul2(tz2, pmul2(vu, wy)));
            wz = padd2(wc, wu);
            pf2 r_sw = pmul2(tcx, psub2(pmul2(ww, padd2(uw, uuw)), pmul2(we, padd2(uc, uu))));
            r_sw = padd2(r_sw, pmul2(tcy, psub2(pmul2(ws, padd2(vs, vus)), pmul2(wn, padd2(vc, vu)))));
            r_sw = padd2(r_sw, psub2(pmul2(td1, pmul2(wo_m, wz_m)), pmul2(td2, pmul2(wu, wz))));
            sw_a = join_a(r_sw);
            sw_b = join_b(r_sw);
        }
        if (act_a) {
            su[g] = join_a(r_su);
            sv[g] = join_a(r_sv);
            sw[g] = sw_a;
        }
        if (act_b) {
            su[g + kHalf] = join_b(r_su);
            sv[g + kHalf] = join_b(r_sv);
            sw[g + kHalf] = sw_b;
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

static __device__ __forceinline__ void setup_smem(unsigned char* raw, Ring<Shape>& ring, PairSmem& ps) {
    ring.setup(raw);
    ps.pairs = reinterpret_cast<float4*>(ring.base + kPairOffset);
    ps.coef = ps.pairs + kPL * 3 * kBoxItems;
    ps.item = reinterpret_cast<long long*>(ring.base + kItemOffset);
}
};

template <class C>
__global__ void __launch_bounds__(C::kNT, C::kMinBlocks) fwd_paired_kernel(const __grid_constant__ CUtensorMap mu,
                                                                           const __grid_constant__ CUtensorMap mv,
                                                                           const __grid_constant__ CUtensorMap mw,
                                                                           const FwdArgs a, const ItemSched sched) {
    using K = PairedK<C>;
    extern __shared__ unsigned char smem_raw[];
    Ring<typename C::Shape> ring;
    typename K::PairSmem ps;
    K::setup_smem(smem_raw, ring, ps);
    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_tensormap(&mu);
        prefetch_tensormap(&mv);
        prefetch_tensormap(&mw);
        ring.init_barriers();
    }
    __syncthreads();
    long long seq = 0;
    int bx, by, k0, k1;
    sched_item(sched, a.kend - a.kbeg, blockIdx.x, &bx, &by, &k0, &k1);
    const typename K::ConvPlan cp = K::make_conv_plan(tid);
    (void)K::paired_tile(ring, ps, &mu, &mv, &mw, a, bx, by, a.kbeg + k0, a.kbeg + k1, seq, tid, cp);
}

// Persistent form over a batch plan: work items (one tile of one domain)
// come from the plan's counter, at most n_items iterations.
template <class C>
__global__ void __launch_bounds__(C::kNT, C::kMinBlocks) fwd_paired_batched(BatchPlan* plan, int variant) {
    using K = PairedK<C>;
    extern __shared__ unsigned char smem_raw[];
    Ring<typename C::Shape> ring;
    typename K::PairSmem ps;
    K::setup_smem(smem_raw, ring, ps);
    const int tid = threadIdx.x;
    if (plan->variant != variant || plan->dtype != PW_F64_PAIRED) {
        if (tid == 0) atomicOr(&tu_status, kStatusBadPlan);
        return;
    }
    if (tid == 0) ring.init_barriers();
    __syncthreads();
    const long long n_items = plan->n_items;
    const typename K::ConvPlan cp = K::make_conv_plan(tid);
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
        if (!K::paired_tile(ring, ps, &d.mu, &d.mv, &d.mw, args, tt % tiles_x, tt / tiles_x, kb, ke, seq, tid, cp))
            break;
    }
}

template <class C>
TileShape paired_shape_of() {
    return TileShape{C::kTX, C::kTY, C::Shape::BX, C::Shape::BY, C::kSmemBytes, C::kNT};
}

template <class C>
cudaError_t launch_one(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw, const FwdArgs& a,
                       cudaStream_t st) {
    auto kern = fwd_paired_kernel<C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    ItemSched sched;
    if ((e = choose_sched(kern, C::kNT, C::kSmemBytes, (a.nx + C::kTX - 1) / C::kTX, (a.ny + C::kTY - 1) / C::kTY,
                          a.kend - a.kbeg, &sched)) != cudaSuccess)
        return e;
    kern<<<(unsigned)sched.items, C::kNT, C::kSmemBytes, st>>>(mu, mv, mw, a, sched);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_batched_cfg(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    auto kern = fwd_paired_batched<C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
    if (e != cudaSuccess) return e;
    long long grid = 0;
    if ((e = persistent_grid(kern, C::kNT, C::kSmemBytes, n_items, &grid)) != cudaSuccess) return e;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, C::kNT, C::kSmemBytes, st>>>(plan, v);
    return cudaGetLastError();
}

}  // namespace

cudaError_t read_and_clear_status_paired(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

int paired_variant_count() { return 4; }

TileShape fwd_paired_shape_variant(int v) {
    switch (v) {
        case 1: return paired_shape_of<PV1>();
        case 2: return paired_shape_of<PV2>();
        case 3: return paired_shape_of<PV3>();
        default: return paired_shape_of<PV0>();
    }
}

TileShape fwd_paired_shape() { return fwd_paired_shape_variant(0); }

cudaError_t launch_fwd_paired(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                              const FwdArgs& a, cudaStream_t st) {
    return launch_one<PV0>(mu, mv, mw, a, st);
}

cudaError_t launch_paired_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    switch (v) {
        case 1: return launch_batched_cfg<PV1>(1, plan, n_items, st);
        case 2: return launch_batched_cfg<PV2>(2, plan, n_items, st);
        case 3: return launch_batched_cfg<PV3>(3, plan, n_items, st);
        default: return launch_batched_cfg<PV0>(0, plan, n_items, st);
    }
}

}  // namespace pw
