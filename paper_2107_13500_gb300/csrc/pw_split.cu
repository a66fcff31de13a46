// pw_split.cu -- PW advection in FP32 on perturbations about per-level FP64
// means (PW_F32_SPLIT), and on full float fields (PW_F32 = the same kernel
// with every mean 0).
//
// Writing u = U(k) + u' (likewise v, w) with U(k) the level mean, the mean x
// mean parts of every horizontal flux difference cancel exactly, and each
// vertical flux difference leaves a per-level constant; pw_make_split_table
// forms those constants in FP64 and rounds them to float once. What remains
// is computed here in FP32 on the perturbations, so the difference-of-
// products fluxes cancel only perturbation-sized quantities.
//
// k-march: a CTA owns TXP x TY interior points, each thread a strip of four
// consecutive points along x (float4 shared-memory reads, 16-byte stores
// when every field's interior starts on a 16-byte boundary). One thread
// keeps an S-stage TMA ring of levels (three field boxes plus the level's
// 32-float table row on one mbarrier) S-1 levels ahead. Loads are numbered
// per CTA (`seq`), so a persistent CTA can run many tiles, of many domains,
// through one ring: load n uses stage n % S and barrier phase n / S.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw.h"
#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace {

constexpr int kStrip = 4;
constexpr int kRowBytes = PW_SPLIT_NCOEF * 4;

// Resident warps per SM the one-shot and the persistent kernels are
// compiled for, whatever the CTA size (the register budget follows).
constexpr int kWarpsOneShot = 20, kWarpsBatched = 16;

template <int TXP_, int TY_, int S_>
struct SplitCfg {
    static constexpr int TXP = TXP_, TY = TY_, S = S_;
    static constexpr int NT = (TXP / kStrip) * TY;
    static constexpr int MIN_BLOCKS = kWarpsOneShot * 32 / NT;
    static constexpr int MIN_BLOCKS_BATCHED = kWarpsBatched * 32 / NT;
    static_assert(NT % 32 == 0, "whole warps per CTA");
    using Shape = RingShape<float, TXP, TY, S>;
    static constexpr int BX = Shape::BX;
    static constexpr int STAGE_BYTES = Shape::STAGE_BYTES;
    // ring stages | ring barriers (padded to 64 B) | S table rows | item slot | alignment slack
    static constexpr int ROW_OFFSET = S * STAGE_BYTES + 64;
    static constexpr int SMEM_BYTES = ROW_OFFSET + S * kRowBytes + 16 + 128;
    static_assert(S * 8 <= 64, "barriers must fit before the table rows");
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// kLowBits: stage and phase from the low 32 bits of the load count (needs a
// power-of-two S). The one-shot kernel takes it (two registers fewer); in
// the persistent kernel it made the compiler spill, so that one keeps the
// 64-bit form.
template <class Cfg, bool kLowBits = false>
struct SplitRing {
    unsigned char* base;
    uint64_t* full;
    float* rows;      // [S][PW_SPLIT_NCOEF]
    long long* item;  // work item handed from thread 0 to the CTA (persistent kernel)

    __device__ __forceinline__ void setup(unsigned char* raw) {
        base = raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
        full = reinterpret_cast<uint64_t*>(base + Cfg::S * Cfg::STAGE_BYTES);
        rows = reinterpret_cast<float*>(base + Cfg::ROW_OFFSET);
        item = reinterpret_cast<long long*>(base + Cfg::ROW_OFFSET + Cfg::S * kRowBytes);
    }
    __device__ __forceinline__ void init_barriers() {
        for (int s = 0; s < Cfg::S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    // Stage (n % S) and phase ((n / S) & 1) of load n. With a power-of-two
    // S both follow from the low 32 bits of n, so no 64-bit arithmetic is
    // needed for them.
    static constexpr bool kPow2 = kLowBits && (Cfg::S & (Cfg::S - 1)) == 0;
    static __device__ __forceinline__ int stage_of(long long seq) {
        if constexpr (kPow2) return (int)((unsigned)seq & (unsigned)(Cfg::S - 1));
        else return (int)(seq % Cfg::S);
    }
    static __device__ __forceinline__ uint32_t phase_of(long long seq) {
        if constexpr (kPow2) return ((unsigned)seq / (unsigned)Cfg::S) & 1u;
        else return (uint32_t)((seq / Cfg::S) & 1);
    }
    __device__ __forceinline__ const float* box(long long seq, int f) const {
        return reinterpret_cast<const float*>(base + stage_of(seq) * Cfg::STAGE_BYTES + f * Cfg::Shape::BOX_STRIDE);
    }
    __device__ __forceinline__ const float* row(long long seq) const {
        return rows + stage_of(seq) * PW_SPLIT_NCOEF;
    }
    // load number `seq` = level `lev` of the tile at (x0, y0)
    __device__ __forceinline__ void issue(long long seq, int lev, const CUtensorMap* mu, const CUtensorMap* mv,
                                          const CUtensorMap* mw, const float* table, int x0, int y0) {
        const int s = stage_of(seq);
        uint64_t* bar = &full[s];
        unsigned char* dst = base + s * Cfg::STAGE_BYTES;
        mbar_arrive_expect_tx(bar, 3 * Cfg::Shape::BOX_BYTES + kRowBytes);
        tma_load_3d(dst, mu, bar, x0, y0, lev);
        tma_load_3d(dst + Cfg::Shape::BOX_STRIDE, mv, bar, x0, y0, lev);
        tma_load_3d(dst + 2 * Cfg::Shape::BOX_STRIDE, mw, bar, x0, y0, lev);
        bulk_load(rows + s * PW_SPLIT_NCOEF, table + (size_t)lev * PW_SPLIT_NCOEF, kRowBytes, bar);
    }
    __device__ __forceinline__ bool wait(long long seq) {
        return mbar_wait_bounded(&full[stage_of(seq)], phase_of(seq));
    }
};

// Four consecutive floats starting at p (one LDS.128 when p is 16-byte aligned).
template <bool kVec>
__device__ __forceinline__ void ld4(const float* p, float* d) {
    if constexpr (kVec) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        d[0] = t.x;
        d[1] = t.y;
        d[2] = t.z;
        d[3] = t.w;
    } else {
        d[0] = p[0];
        d[1] = p[1];
        d[2] = p[2];
        d[3] = p[3];
    }
}

template <bool kVec>
__device__ __forceinline__ void st4(float* g, const float* v, int n) {
    if (kVec && n == 4) {
        *reinterpret_cast<float4*>(g) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m < n) g[m] = v[m];
    }
}

// One tile: output levels kb..ke-1 of the TXP x TY columns at tile (bx, by)
// (a k-chunk; it reads one level below and one above). `seq` is the CTA's
// running load count (CTA-uniform); loads are numbered relative to the
// lowest level read, lo. Returns false if a bounded wait expired (status
// set, in-flight loads drained).
template <class Cfg, bool kVec, bool kLowBits>
__device__ bool split_tile(SplitRing<Cfg, kLowBits>& ring, const CUtensorMap* mu, const CUtensorMap* mv,
                           const CUtensorMap* mw, const FwdArgs& a, int bx, int by, int kb, int ke, long long& seq,
                           int tid) {
    constexpr int S = Cfg::S, BX = Cfg::BX, TXP = Cfg::TXP, TY = Cfg::TY;
    const int sx = tid % (TXP / kStrip), ry = tid / (TXP / kStrip);
    const int x0 = bx * TXP, y0 = by * TY;
    const int i0 = x0 + 1 + kStrip * sx, j = y0 + 1 + ry;
    const int nval = (j <= a.ny) ? max(0, min(kStrip, a.nx - i0 + 1)) : 0;
    const int nz = a.nz;
    const int lo = kb > 0 ? kb - 1 : 0, hi = ke < nz ? ke : nz - 1;
    const int nl = hi - lo + 1;  // levels read
    const float* table = a.split;
    const long long s0 = seq;

    int issued = 0;  // relative loads issued (thread 0)
    if (tid == 0) {
        fence_proxy_async_smem();
        for (; issued < S && issued < nl; ++issued) ring.issue(s0 + issued, lo + issued, mu, mv, mw, table, x0, y0);
    }

    const int cb = (ry + 1) * BX + 1 + a.xoff + kStrip * sx;
    float* __restrict__ su = static_cast<float*>(a.su);
    float* __restrict__ sv = static_cast<float*>(a.sv);
    float* __restrict__ sw = static_cast<float*>(a.sw);
    const size_t gsz = (size_t)a.sz;
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i0 + (size_t)lo * gsz;

    bool bad = !ring.wait(s0);
    if (nl > 1) bad |= !ring.wait(s0 + 1);
    float uo_m[4], vo_m[4], wo_m[4], wx_m[4], wy_m[4], wz_m[4];
    {
        const float* U = ring.box(s0, 0) + cb;
        const float* V = ring.box(s0, 1) + cb;
        const float* W = ring.box(s0, 2) + cb;
        float w5[5];
        ld4<kVec>(U, uo_m);
        ld4<kVec>(V, vo_m);
        ld4<kVec>(W, w5);
        w5[4] = W[4];
        float wn[4], wu[4] = {0.f, 0.f, 0.f, 0.f};
        ld4<kVec>(W + BX, wn);
        if (nl > 1) ld4<kVec>(ring.box(s0 + 1, 2) + cb, wu);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            wo_m[m] = w5[m];
            wx_m[m] = w5[m] + w5[m + 1];
            wy_m[m] = w5[m] + wn[m];
            wz_m[m] = nl > 1 ? w5[m] + wu[m] : 0.0f;
        }
    }
    if (nval > 0 && kb == 0) {  // level 1 of the paper is not computed
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
        st4<kVec>(su + g, z, nval);
        st4<kVec>(sv + g, z, nval);
        st4<kVec>(sw + g, z, nval);
    }
    bool abort = __syncthreads_or(bad);
    if (!abort && tid == 0 && issued < nl) {
        fence_proxy_async_smem();
        ring.issue(s0 + issued, lo + issued, mu, mv, mw, table, x0, y0);
        ++issued;
    }

    for (int k = (kb > 1 ? kb : 1); k < ke && !abort; ++k) {
        const int r = k - lo;
        g += gsz;
        const bool top = (k == nz - 1);
        if (!top) bad |= !ring.wait(s0 + r + 1);
        const float* U = ring.box(s0 + r, 0) + cb;
        const float* V = ring.box(s0 + r, 1) + cb;
        const float* W = ring.box(s0 + r, 2) + cb;
        const float4* T4 = reinterpret_cast<const float4*>(ring.row(s0 + r));

        // neighbourhoods of the strip: index m+1 is point m, 0 and 5 the x halo
        float uj[6], us[4], un[5], vj[6], vs[5], vn[4], wj[6], ws[4], wn[4];
        uj[0] = U[-1];
        ld4<kVec>(U, uj + 1);
        uj[5] = U[4];
        ld4<kVec>(U - BX, us);
        un[0] = U[BX - 1];
        ld4<kVec>(U + BX, un + 1);
        vj[0] = V[-1];
        ld4<kVec>(V, vj + 1);
        vj[5] = V[4];
        ld4<kVec>(V - BX, vs);
        vs[4] = V[4 - BX];
        ld4<kVec>(V + BX, vn);
        wj[0] = W[-1];
        ld4<kVec>(W, wj + 1);
        wj[5] = W[4];
        ld4<kVec>(W - BX, ws);
        ld4<kVec>(W + BX, wn);
        float uu[5], vu[4], vus[4], wu[4];
        if (!top) {
            const float* Uu = ring.box(s0 + r + 1, 0) + cb;
            const float* Vu = ring.box(s0 + r + 1, 1) + cb;
            const float* Wu = ring.box(s0 + r + 1, 2) + cb;
            uu[0] = Uu[-1];
            ld4<kVec>(Uu, uu + 1);
            ld4<kVec>(Vu, vu);
            ld4<kVec>(Vu - BX, vus);
            ld4<kVec>(Wu, wu);
        }
        const float4 t0 = T4[0], t1 = T4[1], t2 = T4[2], t3 = T4[3];
        const float tcx = T4[6].z, tcy = T4[6].w;
        float r_su[4], r_sv[4], r_sw[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float uw = uj[m], uc = uj[m + 1], ue = uj[m + 2];
            const float vw = vj[m], vc = vj[m + 1], ve = vj[m + 2];
            const float wc = wj[m + 1], ww = wj[m], we = wj[m + 2];
            // su: self term, y cross term, lower vertical flux (table entries 0..6)
            float p = vs[m] + vs[m + 1], q = vc + ve;
            float s = tcx * (uw - ue) * (t0.x + uw + uc + ue);
            s += tcy * (t0.y * (us[m] - un[m + 1]) + t0.z * (p - q) + us[m] * p - un[m + 1] * q);
            s += t0.w + t1.x * (t1.y * wx_m[m] + t1.z * uo_m[m] + uo_m[m] * wx_m[m]);
            r_su[m] = s;
            // sv: mirror (entries 10..15, shared vertical entries 4, 6, 7, 9)
            p = uw + un[m];
            q = uc + un[m + 1];
            s = tcy * (vs[m] - vn[m]) * (t2.z + vs[m] + vc + vn[m]);
            s += tcx * (t2.w * (vw - ve) + t3.x * (p - q) + vw * p - ve * q);
            s += t3.y + t1.x * (t3.z * wy_m[m] + t1.z * vo_m[m] + vo_m[m] * wy_m[m]);
            r_sv[m] = s;
            const float wx = wc + we, wy = wc + wn[m];
            float wz = 0.0f;
            r_sw[m] = 0.0f;
            if (!top) {
                const float4 t4 = T4[4], t5 = T4[5], t6 = T4[6];
                // upper vertical fluxes of su and sv (entries 7, 8, 9, 15)
                r_su[m] -= t1.w * (t2.x * wx + t2.y * uu[m + 1] + uu[m + 1] * wx);
                r_sv[m] -= t1.w * (t3.w * wy + t2.y * vu[m] + vu[m] * wy);
                // sw (entries 16..25)
                wz = wc + wu[m];
                p = uw + uu[m];
                q = uc + uu[m + 1];
                s = tcx * (t4.x * (p - q) + t4.y * (ww - we) + ww * p - we * q);
                p = vs[m] + vus[m];
                q = vc + vu[m];
                s += tcy * (t4.x * (p - q) + t4.z * (ws[m] - wn[m]) + ws[m] * p - wn[m] * q);
                s += t4.w + t5.x * (wz_m[m] * (t5.y + wo_m[m]) + t5.z * wo_m[m]);
                s -= t5.w * (wz * (t6.x + wu[m]) + t6.y * wu[m]);
                r_sw[m] = s;
            }
            uo_m[m] = uc;
            vo_m[m] = vc;
            wo_m[m] = wc;
            wx_m[m] = wx;
            wy_m[m] = wy;
            wz_m[m] = wz;
        }
        if (nval > 0) {
            st4<kVec>(su + g, r_su, nval);
            st4<kVec>(sv + g, r_sv, nval);
            st4<kVec>(sw + g, r_sw, nval);
        }
        abort = __syncthreads_or(bad);  // releases relative level r's stage
        if (!abort && tid == 0 && issued < nl) {
            fence_proxy_async_smem();
            ring.issue(s0 + issued, lo + issued, mu, mv, mw, table, x0, y0);
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

template <class Cfg, bool kVec>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MIN_BLOCKS) fwd_split_kernel(const __grid_constant__ CUtensorMap mu,
                                                            const __grid_constant__ CUtensorMap mv,
                                                            const __grid_constant__ CUtensorMap mw,
                                                            const FwdArgs a, const ItemSched sched) {
    extern __shared__ unsigned char smem_raw[];
    SplitRing<Cfg, true> ring;
    ring.setup(smem_raw);
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
    (void)split_tile<Cfg, kVec, true>(ring, &mu, &mv, &mw, a, bx, by, a.kbeg + k0, a.kbeg + k1, seq, tid);
}

// Persistent form: the CTA takes work items (one k-chunk of one tile of one
// domain) from the plan's counter until none are left; at most n_items
// iterations. Items are ordered by the plan builder (taller columns first).
template <class Cfg, bool kVec>
__device__ __forceinline__ void run_items(BatchPlan* plan, SplitRing<Cfg>& ring, int tid) {
    const long long n_items = plan->n_items;
    long long seq = 0;
    for (long long it = 0; it < n_items; ++it) {
        if (tid == 0) *ring.item = (long long)atomicAdd(&plan->counter, 1ull);
        __syncthreads();
        const long long item = *ring.item;
        __syncthreads();  // every thread has read the slot before thread 0 rewrites it
        if (item >= n_items) break;
        const BatchDomain& d = plan->dom[find_domain(plan, item)];
        // private copy: the plan is global memory the compiler cannot prove
        // free of the output stores, so fields read from it would be reloaded
        const FwdArgs args = d.args;
        const long long t = item - d.first_item;
        const int tiles_x = d.tiles_x, kchunks = d.kchunks;
        const long long tiles = (long long)tiles_x * d.tiles_y;
        const int ch = (int)(t / tiles), tt = (int)(t % tiles);
        const int kb = (int)((long long)args.nz * ch / kchunks);
        const int ke = (int)((long long)args.nz * (ch + 1) / kchunks);
        if (!split_tile<Cfg, kVec, false>(ring, &d.mu, &d.mv, &d.mw, args, tt % tiles_x, tt / tiles_x, kb, ke, seq, tid))
            break;
    }
}

template <class Cfg>
__global__ void __launch_bounds__(Cfg::NT, Cfg::MIN_BLOCKS_BATCHED) fwd_split_batched(BatchPlan* plan, int variant) {
    extern __shared__ unsigned char smem_raw[];
    SplitRing<Cfg> ring;
    ring.setup(smem_raw);
    const int tid = threadIdx.x;
    if (plan->variant != variant || (plan->dtype != PW_F32 && plan->dtype != PW_F32_SPLIT)) {
        if (tid == 0) atomicOr(&tu_status, kStatusBadPlan);
        return;
    }
    if (tid == 0) ring.init_barriers();
    __syncthreads();
    // one whole item loop per path, chosen once, so each gets the registers to itself
    if (plan->all_vec) run_items<Cfg, true>(plan, ring, tid);
    else run_items<Cfg, false>(plan, ring, tid);
}

// Tile-shape / pipeline-depth variants (the autotuner's search space).
using V0 = SplitCfg<128, 4, 4>;
using V1 = SplitCfg<64, 4, 4>;
using V2 = SplitCfg<32, 8, 4>;
using V3 = SplitCfg<64, 8, 4>;
using V4 = SplitCfg<32, 16, 4>;
using V5 = SplitCfg<128, 2, 4>;
using V6 = SplitCfg<64, 4, 3>;
using V7 = SplitCfg<64, 4, 6>;

template <class Cfg>
TileShape shape_of() {
    return TileShape{Cfg::TXP, Cfg::TY, Cfg::BX, Cfg::Shape::BY, Cfg::SMEM_BYTES, Cfg::NT};
}

template <class Cfg>
cudaError_t launch_one(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw, const FwdArgs& a,
                       cudaStream_t st) {
    auto kern = a.vec ? fwd_split_kernel<Cfg, true> : fwd_split_kernel<Cfg, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    ItemSched sched;
    if ((e = choose_sched(kern, Cfg::NT, Cfg::SMEM_BYTES, (a.nx + Cfg::TXP - 1) / Cfg::TXP, (a.ny + Cfg::TY - 1) / Cfg::TY,
                          a.kend - a.kbeg, &sched)) != cudaSuccess)
        return e;
    kern<<<(unsigned)sched.items, Cfg::NT, Cfg::SMEM_BYTES, st>>>(mu, mv, mw, a, sched);
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_batched_cfg(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    auto kern = fwd_split_batched<Cfg>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    long long grid = 0;
    if ((e = persistent_grid(kern, Cfg::NT, Cfg::SMEM_BYTES, n_items, &grid)) != cudaSuccess) return e;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, Cfg::NT, Cfg::SMEM_BYTES, st>>>(plan, v);
    return cudaGetLastError();
}

}  // namespace

cudaError_t read_and_clear_status_split(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

int split_variant_count() { return 8; }

TileShape fwd_split_shape_variant(int v) {
    switch (v) {
        case 1: return shape_of<V1>();
        case 2: return shape_of<V2>();
        case 3: return shape_of<V3>();
        case 4: return shape_of<V4>();
        case 5: return shape_of<V5>();
        case 6: return shape_of<V6>();
        case 7: return shape_of<V7>();
        default: return shape_of<V0>();
    }
}

TileShape fwd_split_shape() { return fwd_split_shape_variant(0); }

cudaError_t launch_fwd_split_variant(int v, const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                                     const FwdArgs& a, cudaStream_t st) {
    switch (v) {
        case 1: return launch_one<V1>(mu, mv, mw, a, st);
        case 2: return launch_one<V2>(mu, mv, mw, a, st);
        case 3: return launch_one<V3>(mu, mv, mw, a, st);
        case 4: return launch_one<V4>(mu, mv, mw, a, st);
        case 5: return launch_one<V5>(mu, mv, mw, a, st);
        case 6: return launch_one<V6>(mu, mv, mw, a, st);
        case 7: return launch_one<V7>(mu, mv, mw, a, st);
        default: return launch_one<V0>(mu, mv, mw, a, st);
    }
}

cudaError_t launch_fwd_split(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                             const FwdArgs& a, cudaStream_t st) {
    return launch_fwd_split_variant(0, mu, mv, mw, a, st);
}

cudaError_t launch_split_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    switch (v) {
        case 1: return launch_batched_cfg<V1>(1, plan, n_items, st);
        case 2: return launch_batched_cfg<V2>(2, plan, n_items, st);
        case 3: return launch_batched_cfg<V3>(3, plan, n_items, st);
        case 4: return launch_batched_cfg<V4>(4, plan, n_items, st);
        case 5: return launch_batched_cfg<V5>(5, plan, n_items, st);
        case 6: return launch_batched_cfg<V6>(6, plan, n_items, st);
        case 7: return launch_batched_cfg<V7>(7, plan, n_items, st);
        default: return launch_batched_cfg<V0>(0, plan, n_items, st);
    }
}

}  // namespace pw
