// pw_adjoint.cu -- transpose of the PW advection Jacobian in paired FP32
// (PW_F64_PAIRED) and FP32 (PW_F32), cell by cell (gather form), and the
// transpose of the periodic halo fill. (Native FP64 is in pw_adjoint_f64.cu,
// regrouped by faces.)
//
// The forward map is a quadratic form: every term is c * p * (q + r) with c a
// coefficient and p, q, r field values, so its partial derivatives are
// c * (q + r) (by p) and c * p (by q and by r). For a cell C the adjoint
// gathers, from every output point P that read C, the cotangent at P times
// that derivative. Writing each forward term out (su: T1..T6, sv: S1..S6,
// sw: W1..W6, the order of the formulas in include/pw.h), a u cell is read by
// 16 (P, term) pairs, a v cell by 16, a w cell by 16; they are listed at the
// gather blocks below. Cotangents outside the computed points (halo
// columns and rows, level 1, and level nz for sw) count as zero, so output
// cells include the halo: gu, gv, gw are defined on every cell the forward
// map reads. Threads own cells (the paired kernel two, the FP32 kernel a
// strip of two or four) and march k with a TMA ring of the six fields (u, v,
// w, gsu, gsv, gsw) -- no atomics, one write per cell. A launch splits the
// columns into k-chunks so that small domains still fill the GPU (the FP32
// kernel hands small domains out as equal runs of tile levels instead); a
// chunk of output levels kb..ke-1 reads levels kb-1..ke.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_pair.cuh"
#include "pw_ring.cuh"
#include "pw_strip_sched.h"

namespace pw {

namespace {

constexpr int kTX = 32, kTY = 8, kS = 4, kFields = 6;

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

// The seven vertical coefficients step k uses (zero where the paper's level
// has no such flux), in T. One thread each loads and converts them once per
// level; the CTA barrier of the step before publishes them. (A per-thread
// double->float conversion would run on the FP64 pipe and bound the FP32
// kernel.)
__device__ __forceinline__ double level_coef(const AdjArgs& a, int k, int n) {
    const int nz = a.nz;
    switch (n) {
        case 0: return (k + 1 <= nz - 1) ? __ldg(a.tzc1 + k + 1) : 0.0;  // tz1p
        case 1: return (k >= 1) ? __ldg(a.tzc2 + k - 1) : 0.0;           // tz2m
        case 2: return (k <= nz - 2) ? __ldg(a.tzc2 + k) : 0.0;         // tz20 (level k has an upper flux)
        case 3: return (k + 1 <= nz - 1) ? __ldg(a.tzd1 + k + 1) : 0.0;  // td1p
        case 4: return __ldg(a.tzd1 + k);                                // td10
        case 5: return (k >= 1) ? __ldg(a.tzd2 + k - 1) : 0.0;           // td2m
        default: return __ldg(a.tzd2 + k);                               // td20
    }
}

template <typename T>
__device__ __forceinline__ void level_coefs(const AdjArgs& a, int k, int tid, T* dst) {
    if (tid < 7) dst[tid] = (T)level_coef(a, k, tid);
}

// ---------------------------------------------------------------------------
// Paired-FP32 adjoint (PW_F64_PAIRED): doubles in and out, the same gather on
// (hi, lo) float pairs (pw_pair.cuh). A one-level TMA stage brings the six
// fields of a level as doubles (reissued as soon as the level is split, a
// full step ahead of its use; one stage keeps three CTAs per SM); each level is split once into a three-level
// pair ring, and a thread evaluates cells A = (x0+t, j) and B = A + 16 on
// packed lanes, reading every neighbour of both as one 16-byte item of the
// interleaved halves (as in the paired forward kernel). Level k-1's values
// the gather needs are carried in registers.
//
// Cotangents that the forward map never produces (halo cells, level 1, and
// the top level of sw) are set to zero while they are split, so the gather
// needs no per-cell masks; only the upper vertical fluxes of su and sv, absent
// at the top level, are skipped by a level-uniform test.

constexpr int kPS = 1, kPPL = 3;                    // TMA stages, pair-ring levels
constexpr int kPHalf = kTX / 2;                    // x distance from A to B; threads per tile row
constexpr int kPNT = kPHalf * kTY;
constexpr int kPHX = kPHalf + 2;                   // pair-box row: x' = 0..kPHalf+1 of both halves
using PSh = AdjShape<double>;
constexpr int kPItems = PSh::BY * kPHX;            // float4 {hA, hB, lA, lB} per field and level
constexpr int kPPairOffset = kPS * PSh::STAGE_BYTES + 64;
constexpr int kPPairBytes = kPPL * kFields * kPItems * 16;
constexpr int kPCoefOffset = kPPairOffset + kPPairBytes;
constexpr int kPCoefBytes = kPPL * 8 * 16;
constexpr int kPSmemBytes = kPCoefOffset + kPCoefBytes + 128;
constexpr int kPConvIters = (kFields * kPItems + kPNT - 1) / kPNT;
static_assert(PSh::BOX_STRIDE % 8 == 0, "box stride in doubles");
// lane A of item x' is box column x' + 1 + xoff (the box starts one 16-byte
// unit left of the tile), lane B kPHalf further
static_assert((kPHX - 1) + 1 + PSh::XOFF_MAX + kPHalf < PSh::BX, "both halves must lie inside the box row");

// Per-thread split work: item t' + q*kPNT of a level is (field, row, x'),
// with t' = (tid + 64) mod kPNT, so the partial last round of items falls on
// warps 2 and 3 while thread 0 issues the TMA loads and warp 1 splits the
// level coefficients. Offsets and positions depend on neither the level nor
// the tile.
__device__ __forceinline__ int adj_conv_item(int tid, int q) { return (tid + 64) % kPNT + q * kPNT; }
constexpr int kPCoefWarp = 1;
static_assert(kPNT >= 128, "the split work is spread over four warps");

struct AdjConvPlan {
    int off[kPConvIters];   // lane A's double offset in a stage (xoff = 0)
    int info[kPConvIters];  // field | row << 8 | x' << 16
};

__device__ __forceinline__ AdjConvPlan make_adj_conv_plan(int tid) {
    AdjConvPlan cp;
#pragma unroll
    for (int q = 0; q < kPConvIters; ++q) {
        const int n = adj_conv_item(tid, q);
        const int f = n / kPItems, e = n - f * kPItems;
        const int row = e / kPHX, xp = e - row * kPHX;
        cp.off[q] = f * (PSh::BOX_STRIDE / 8) + row * PSh::BX + xp + 1;
        cp.info[q] = f | (row << 8) | (xp << 16);
    }
    return cp;
}

// Coefficient n of level lev for lane n = 0..6 of warp kPCoefWarp (0
// elsewhere and for levels outside the domain).
__device__ __forceinline__ double adj_coef_for(const AdjArgs& a, int lev, int tid) {
    const int n = tid - 32 * kPCoefWarp;
    return ((unsigned)n < 7u && lev >= 0 && lev < a.nz) ? level_coef(a, lev, n) : 0.0;
}

// Split the level `lev` held in `stage` into pair slot `dst`; cotangent cells
// outside the computed output points become (0, 0). Lanes 0..6 of warp
// kPCoefWarp also store the level's seven coefficients (as for the FP64 kernel), given in `coef`
// (loaded one conversion earlier), as pairs {h, h, l, l}.
__device__ __forceinline__ void adj_convert(const unsigned char* stage, float4* dst, float4* cdst, int lev,
                                            int x0, int y0, const AdjArgs& a, int tid, const AdjConvPlan& cp,
                                            double coef) {
    const double* base = reinterpret_cast<const double*>(stage) + a.xoff;
    const bool s_ok = lev >= 1;                    // su, sv: levels 1..nz-1 (level nz reads as 0)
    const bool w_ok = lev >= 1 && lev <= a.nz - 2; // sw: levels 1..nz-2
#pragma unroll
    for (int q = 0; q < kPConvIters; ++q) {
        const int n = adj_conv_item(tid, q);
        if ((q + 1) * kPNT <= kFields * kPItems || n < kFields * kPItems) {
            const double* src = base + cp.off[q];
            double da = src[0], db = src[kPHalf];
            const int f = cp.info[q] & 0xff;
            if (f >= 3) {
                const int row = (cp.info[q] >> 8) & 0xff, xp = cp.info[q] >> 16;
                const int ia = x0 - 1 + xp, j = y0 - 1 + row;
                const bool lv = (f == 5) ? w_ok : s_ok;
                const bool jy = lv && j >= 1 && j <= a.ny;
                da = (jy && ia >= 1 && ia <= a.nx) ? da : 0.0;
                db = (jy && ia + kPHalf >= 1 && ia + kPHalf <= a.nx) ? db : 0.0;
            }
            const pf p0 = split_double(da), p1 = split_double(db);
            dst[n] = make_float4(p0.h, p1.h, p0.l, p1.l);
        }
    }
    const int cn = tid - 32 * kPCoefWarp;
    if ((unsigned)cn < 7u && lev >= 0 && lev < a.nz) {
        const pf p = split_double(coef);
        cdst[cn] = make_float4(p.h, p.h, p.l, p.l);
    }
}

__device__ __forceinline__ pf2 ldp(const float4* b, int idx) {
    const float4 v = b[idx];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

__device__ __forceinline__ pf2 cf2(const float4* c, int n) {
    const float4 v = c[n];
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

__device__ __forceinline__ void adj_issue_p(unsigned char* base, uint64_t* full, const AdjMaps& maps, int seq, int lev,
                                            int x, int y) {
    const int s = seq % kPS;
    uint64_t* bar = &full[s];
    unsigned char* dst = base + s * PSh::STAGE_BYTES;
    mbar_arrive_expect_tx(bar, kFields * PSh::BOX_BYTES);
    for (int f = 0; f < kFields; ++f) tma_load_3d(dst + f * PSh::BOX_STRIDE, &maps.m[f], bar, x, y, lev);
}

__global__ void __launch_bounds__(kPNT, 3) adjoint_paired_kernel(const __grid_constant__ AdjMaps maps,
                                                                 const AdjArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kPS * PSh::STAGE_BYTES);
    float4* pairs = reinterpret_cast<float4*>(base + kPPairOffset);
    float4* coefs = reinterpret_cast<float4*>(base + kPCoefOffset);
    auto slot = [&](int rel) { return pairs + (rel % kPPL) * kFields * kPItems; };
    auto cslot = [&](int rel) { return coefs + (rel % kPPL) * 8; };
    auto wait = [&](int seq) { return mbar_wait_bounded(&full[seq % kPS], (uint32_t)((seq / kPS) & 1)); };

    const int tid = threadIdx.x;
    const int tx = tid % kPHalf, ty = tid / kPHalf;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int ia = x0 + tx, j = y0 + ty;  // cell A; B is ia + kPHalf
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool act_a = (ia <= nx + 1) && (j <= ny + 1);
    const bool act_b = (ia + kPHalf <= nx + 1) && (j <= ny + 1);
    const int bxs = x0 - PSh::UNIT, bys = y0 - 1;
    const int kb = (int)((long long)nz * blockIdx.z / gridDim.z);
    const int ke = (int)((long long)nz * (blockIdx.z + 1) / gridDim.z);
    const int nl = ke - kb + 2;  // loads: levels kb-1 .. ke (relative 0 .. nl-1)
    const AdjConvPlan cp = make_adj_conv_plan(tid);

    if (tid == 0) {
        for (int f = 0; f < kFields; ++f) prefetch_tensormap(&maps.m[f]);
        for (int s = 0; s < kPS; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < kPS && issued < nl; ++issued) adj_issue_p(base, full, maps, issued, kb - 1 + issued, bxs, bys);

    // relative levels 0..2 split up front, each stage reissued once split;
    // c_pre is the next level's coefficient, loaded one conversion ahead
    bool bad = false, abort = false;
    double c_pre = adj_coef_for(a, kb - 1, tid);
    for (int r = 0; r < kPPL && r < nl && !abort; ++r) {
        bad |= !wait(r);
        adj_convert(base + (r % kPS) * PSh::STAGE_BYTES, slot(r), cslot(r), kb - 1 + r, x0, y0, a, tid, cp, c_pre);
        c_pre = adj_coef_for(a, kb + r, tid);
        abort = __syncthreads_or(bad);
        if (!abort && tid == 0 && issued < nl) {
            fence_proxy_async_smem();
            adj_issue_p(base, full, maps, issued, kb - 1 + issued, bxs, bys);
            ++issued;
        }
    }

    const int c = (ty + 1) * kPHX + (tx + 1);
    constexpr int E = 1, N = kPHX;
    const pf2 tcx = dup2(split_double(a.tcx)), tcy = dup2(split_double(a.tcy));
    // level k-1 carries: w at C, C+x, C+y; su, sv at C; sw at C, C+x, C+y
    pf2 w_kmc, w_kme, w_kmn, su_km, sv_km, sw_km, sw_km_e, sw_km_n;
    {
        const float4* L = slot(0);
        w_kmc = ldp(L + 2 * kPItems, c);
        w_kme = ldp(L + 2 * kPItems, c + E);
        w_kmn = ldp(L + 2 * kPItems, c + N);
        su_km = ldp(L + 3 * kPItems, c);
        sv_km = ldp(L + 4 * kPItems, c);
        sw_km = ldp(L + 5 * kPItems, c);
        sw_km_e = ldp(L + 5 * kPItems, c + E);
        sw_km_n = ldp(L + 5 * kPItems, c + N);
    }
    double* __restrict__ gu = static_cast<double*>(a.gu);
    double* __restrict__ gv = static_cast<double*>(a.gv);
    double* __restrict__ gw = static_cast<double*>(a.gw);
    size_t g = (size_t)j * (size_t)a.sy + (size_t)ia + (size_t)kb * (size_t)a.sz;
    abort = __syncthreads_or(bad);  // relative slot 0 is rewritten by the first step

    for (int k = kb; k < ke && !abort; ++k) {
        const int rc = k - kb + 1;  // relative level of k
        if (rc + 2 < nl) {
            bad |= !wait(rc + 2);
            adj_convert(base + ((rc + 2) % kPS) * PSh::STAGE_BYTES, slot(rc + 2), cslot(rc + 2), k + 2, x0, y0, a,
                        tid, cp, c_pre);
            c_pre = adj_coef_for(a, k + 3, tid);
            // the staged level is split: reissue its stage now, so that the
            // copy of the next level overlaps this step's gather
            abort = __syncthreads_or(bad);
            if (abort) break;
            if (tid == 0 && issued < nl) {
                fence_proxy_async_smem();
                adj_issue_p(base, full, maps, issued, kb - 1 + issued, bxs, bys);
                ++issued;
            }
        }
        const float4* L0 = slot(rc);
        const float4* Lp = slot(rc + 1);
        const float4* U0 = L0;
        const float4* V0 = L0 + kPItems;
        const float4* W0 = L0 + 2 * kPItems;
        const float4* GU0 = L0 + 3 * kPItems;
        const float4* GV0 = L0 + 4 * kPItems;
        const float4* GW0 = L0 + 5 * kPItems;
        const float4* Up = Lp;
        const float4* Vp = Lp + kPItems;
        const float4* Wp = Lp + 2 * kPItems;
        const float4* GUp = Lp + 3 * kPItems;
        const float4* GVp = Lp + 4 * kPItems;
        const float4* GWp = Lp + 5 * kPItems;
        const float4* C0 = cslot(rc);
        const bool up0 = (k <= nz - 2);  // level k has an upper flux

        const pf2 su_c = ldp(GU0, c), su_e = ldp(GU0, c + E), su_w = ldp(GU0, c - E), su_n = ldp(GU0, c + N);
        const pf2 su_s = ldp(GU0, c - N), su_nw = ldp(GU0, c + N - E);
        const pf2 su_kp = ldp(GUp, c), su_kp_w = ldp(GUp, c - E);
        const pf2 sv_c = ldp(GV0, c), sv_e = ldp(GV0, c + E), sv_w = ldp(GV0, c - E), sv_n = ldp(GV0, c + N);
        const pf2 sv_s = ldp(GV0, c - N), sv_se = ldp(GV0, c - N + E);
        const pf2 sv_kp = ldp(GVp, c), sv_kp_s = ldp(GVp, c - N);
        const pf2 sw_c = ldp(GW0, c), sw_e = ldp(GW0, c + E), sw_w = ldp(GW0, c - E), sw_n = ldp(GW0, c + N);
        const pf2 sw_s = ldp(GW0, c - N), sw_kp = ldp(GWp, c);
        const pf2 u_c = ldp(U0, c), u_e = ldp(U0, c + E), u_w = ldp(U0, c - E), u_n = ldp(U0, c + N);
        const pf2 u_nw = ldp(U0, c + N - E), u_kp = ldp(Up, c), u_kp_w = ldp(Up, c - E);
        const pf2 v_c = ldp(V0, c), v_e = ldp(V0, c + E), v_n = ldp(V0, c + N), v_s = ldp(V0, c - N);
        const pf2 v_se = ldp(V0, c - N + E), v_kp = ldp(Vp, c), v_kp_s = ldp(Vp, c - N);
        const pf2 w_c = ldp(W0, c), w_e = ldp(W0, c + E), w_n = ldp(W0, c + N), w_kp = ldp(Wp, c);
        const pf2 tz1p = cf2(C0, 0), tz2m = cf2(C0, 1), tz20 = cf2(C0, 2), td1p = cf2(C0, 3), td10 = cf2(C0, 4);
        const pf2 td2m = cf2(C0, 5), td20 = cf2(C0, 6);

        // gu(C) (same terms and order as the FP64 kernel)
        pf2 r_u = pmul2(tcx, psub2(psub2(padd2(pmul2(padd2(padd2(u_e, u_c), u_c), su_e), pmul2(u_w, su_c)),
                                         pmul2(padd2(padd2(u_w, u_c), u_c), su_w)),
                                   pmul2(u_e, su_c)));
        r_u = padd2(r_u, pmul2(tcy, psub2(pmul2(padd2(v_c, v_e), su_n), pmul2(padd2(v_s, v_se), su_s))));
        r_u = padd2(r_u, psub2(pmul2(pmul2(tz1p, padd2(w_c, w_e)), su_kp), pmul2(pmul2(tz2m, padd2(w_kmc, w_kme)), su_km)));
        r_u = padd2(r_u, pmul2(tcx, psub2(psub2(padd2(pmul2(v_c, sv_e), pmul2(v_s, sv_se)), pmul2(v_e, sv_c)),
                                         pmul2(v_se, sv_s))));
        r_u = padd2(r_u, pmul2(tcx, psub2(psub2(padd2(pmul2(w_c, sw_e), pmul2(w_kmc, sw_km_e)), pmul2(w_e, sw_c)),
                                         pmul2(w_kme, sw_km))));
        // gv(C)
        pf2 r_v = pmul2(tcy, psub2(psub2(padd2(pmul2(padd2(padd2(v_n, v_c), v_c), sv_n), pmul2(v_s, sv_c)),
                                         pmul2(padd2(padd2(v_s, v_c), v_c), sv_s)),
                                   pmul2(v_n, sv_c)));
        r_v = padd2(r_v, pmul2(tcx, psub2(pmul2(padd2(u_c, u_n), sv_e), pmul2(padd2(u_w, u_nw), sv_w))));
        r_v = padd2(r_v, psub2(pmul2(pmul2(tz1p, padd2(w_c, w_n)), sv_kp), pmul2(pmul2(tz2m, padd2(w_kmc, w_kmn)), sv_km)));
        r_v = padd2(r_v, pmul2(tcy, psub2(psub2(padd2(pmul2(u_c, su_n), pmul2(u_w, su_nw)), pmul2(u_n, su_c)),
                                         pmul2(u_nw, su_w))));
        r_v = padd2(r_v, pmul2(tcy, psub2(psub2(padd2(pmul2(w_c, sw_n), pmul2(w_kmc, sw_km_n)), pmul2(w_n, sw_c)),
                                         pmul2(w_kmn, sw_km))));
        // gw(C)
        pf2 r_w = pmul2(tz1p, padd2(pmul2(u_c, su_kp), pmul2(u_w, su_kp_w)));
        pf2 r_w2 = pmul2(tz1p, padd2(pmul2(v_c, sv_kp), pmul2(v_s, sv_kp_s)));
        if (up0) {  // the upper fluxes of su and sv at level k
            r_w = psub2(r_w, pmul2(tz20, padd2(pmul2(u_kp, su_c), pmul2(u_kp_w, su_w))));
            r_w2 = psub2(r_w2, pmul2(tz20, padd2(pmul2(v_kp, sv_c), pmul2(v_kp_s, sv_s))));
        }
        r_w = padd2(r_w, r_w2);
        r_w = padd2(r_w, pmul2(tcx, psub2(pmul2(padd2(u_c, u_kp), sw_e), pmul2(padd2(u_w, u_kp_w), sw_w))));
        r_w = padd2(r_w, pmul2(tcy, psub2(pmul2(padd2(v_c, v_kp), sw_n), pmul2(padd2(v_s, v_kp_s), sw_s))));
        r_w = padd2(r_w, padd2(pmul2(pmul2(td1p, padd2(padd2(w_kp, w_c), w_c)), sw_kp), pmul2(pmul2(td10, w_kmc), sw_c)));
        r_w = psub2(r_w, padd2(pmul2(pmul2(td2m, padd2(padd2(w_kmc, w_c), w_c)), sw_km), pmul2(pmul2(td20, w_kp), sw_c)));

        const double ua = pair_to_double(pf{r_u.h.x, r_u.l.x}), ub = pair_to_double(pf{r_u.h.y, r_u.l.y});
        const double va = pair_to_double(pf{r_v.h.x, r_v.l.x}), vb = pair_to_double(pf{r_v.h.y, r_v.l.y});
        const double wa = pair_to_double(pf{r_w.h.x, r_w.l.x}), wb = pair_to_double(pf{r_w.h.y, r_w.l.y});
        if (a.accumulate) {
            if (act_a) {
                gu[g] += ua;
                gv[g] += va;
                gw[g] += wa;
            }
            if (act_b) {
                gu[g + kPHalf] += ub;
                gv[g + kPHalf] += vb;
                gw[g + kPHalf] += wb;
            }
        } else {
            if (act_a) {
                gu[g] = ua;
                gv[g] = va;
                gw[g] = wa;
            }
            if (act_b) {
                gu[g + kPHalf] = ub;
                gv[g + kPHalf] = vb;
                gw[g + kPHalf] = wb;
            }
        }
        g += (size_t)a.sz;
        w_kmc = w_c;
        w_kme = w_e;
        w_kmn = w_n;
        su_km = su_c;
        sv_km = sv_c;
        sw_km = sw_c;
        sw_km_e = sw_e;
        sw_km_n = sw_n;
        abort = __syncthreads_or(bad);  // publishes rc+2's pairs, frees rc's slot
    }
    if (abort && tid == 0) {
        atomicOr(&tu_status, kStatusTimeout);
        for (int q = (issued > kPS ? issued - kPS : 0); q < issued; ++q) (void)wait(q);
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

// ---------------------------------------------------------------------------
// FP32 adjoint on strips (PW_F32): the cell-by-cell gather, with each
// thread owning kStripCells (two or four) consecutive cells along x. Tiles
// are laid out in the TMA tensor's x coordinate X = i + xoff (the descriptor
// starts at the 16-byte boundary at or below i = 0), so a strip's first cell
// sits at a multiple of the strip's width both in the staged box and in
// global memory: a strip of four reads the six columns i-1 .. i+4 of a
// neighbour row with three 16-byte loads and stores each gradient with one
// 16-byte store; a strip of two reads i-1 .. i+2 with one 8-byte and two
// 4-byte loads and stores 8 bytes. Two cells per thread (the default) give
// 256-thread CTAs on the same staged boxes: twice the warps per SM to hide
// the level march's latency, for about a fifth more instructions per cell.

#ifndef PW_ADJ_STRIP_TY
#define PW_ADJ_STRIP_TY 12
#endif
#ifndef PW_ADJ_STRIP_STAGES
#define PW_ADJ_STRIP_STAGES 4
#endif
#ifndef PW_ADJ_STRIP_TX
#define PW_ADJ_STRIP_TX 32
#endif
#ifndef PW_ADJ_STRIP_CELLS
#define PW_ADJ_STRIP_CELLS 2
#endif
constexpr int kSTX = PW_ADJ_STRIP_TX, kSTY = PW_ADJ_STRIP_TY, kSS = PW_ADJ_STRIP_STAGES;  // cells per tile row, rows, TMA stages
// Cells of a row per thread (a strip): 4 or 2. Two cells per thread double
// the threads of a CTA on the same staged boxes (more warps to hide latency)
// at the cost of more shared loads per cell.
constexpr int kStripCells = PW_ADJ_STRIP_CELLS;
template <int kCells>
struct StripThreads {
    static_assert(kCells == 4 || kCells == 2, "strips of 4 or 2 cells");
    static constexpr int NT = (kSTX / kCells) * kSTY;
};
constexpr int kSNT = StripThreads<kStripCells>::NT;  // threads
constexpr int kSMinBlocks = (227 * 1024) / (kSS * kFields * (((kSTX + 8) * (kSTY + 2) * 4 + 127) / 128 * 128) + 1280);
struct StripShape {
    static constexpr int BX = kSTX + 8;  // tensor x from X0 - 4 to X0 + kSTX + 3
    static constexpr int BY = kSTY + 2;
    static constexpr int BOX_BYTES = BX * BY * 4;
    static constexpr int BOX_STRIDE = round_up(BOX_BYTES, 128);
    static constexpr int STAGE_BYTES = kFields * BOX_STRIDE;
    static constexpr int SMEM_BYTES = kSS * STAGE_BYTES + 64 + 128;
    static_assert(BX % 4 == 0 && BOX_STRIDE % 16 == 0, "16-byte rows");
    static_assert(kSS >= 4, "step k reads levels k-1..k+1 and waits for k+2, which needs a fourth stage");
    static_assert(kSTX % 32 == 0 || kSTX == 16, "tile width in whole 16-byte units");
};

// Zero the cotangent cells of a staged level that are not computed output
// points (the paired kernel does the same while it splits a level).
template <int NT>
__device__ __forceinline__ void zero_outside_strip(unsigned char* stage, int lev, const AdjArgs& a, int X0, int y0,
                                                   int tid) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool lev_s = lev >= 1 && lev <= nz - 1;
    const bool lev_w = lev >= 1 && lev <= nz - 2;
    const int i0 = X0 - 4 - a.xoff, j0 = y0 - 1;  // cell of box column 0, row 0
    const bool edge = i0 < 1 || i0 + StripShape::BX - 1 > nx || j0 < 1 || j0 + StripShape::BY - 1 > ny;
    if (!edge && lev_s && lev_w) return;  // CTA-uniform
    bool wrote = false;
    for (int f = 3; f < kFields; ++f) {
        const bool lv = (f == 5) ? lev_w : lev_s;
        if (lv && !edge) continue;
        float* box = reinterpret_cast<float*>(stage + f * StripShape::BOX_STRIDE);
        for (int n = tid; n < StripShape::BX * StripShape::BY; n += NT) {
            const int r = n / StripShape::BX, b = n - r * StripShape::BX;
            const int i = i0 + b, j = j0 + r;
            if (!lv || i < 1 || i > nx || j < 1 || j > ny) {
                box[n] = 0.0f;
                wrote = true;
            }
        }
    }
    if (wrote) fence_proxy_async_smem();
}

// Columns cc-1 .. cc+kCells of a box row (cc aligned to the strip's width
// in bytes): v[0] = west of the strip's first cell, v[1..kCells] = the
// strip, v[kCells+1] = east of its last cell. Only the loads whose columns
// are used are issued.
template <int kCells, bool kW, bool kE>
__device__ __forceinline__ void row_strip(const float* p, float* v) {
    if constexpr (kCells == 4) {
        const float4 b = *reinterpret_cast<const float4*>(p);
        v[1] = b.x;
        v[2] = b.y;
        v[3] = b.z;
        v[4] = b.w;
        if constexpr (kW) v[0] = reinterpret_cast<const float4*>(p)[-1].w;
        else v[0] = 0.0f;
        if constexpr (kE) v[5] = reinterpret_cast<const float4*>(p)[1].x;
        else v[5] = 0.0f;
    } else {
        const float2 b = *reinterpret_cast<const float2*>(p);
        v[1] = b.x;
        v[2] = b.y;
        if constexpr (kW) v[0] = p[-1];
        else v[0] = 0.0f;
        if constexpr (kE) v[3] = p[2];
        else v[3] = 0.0f;
    }
}


template <int kCells>
__global__ void __launch_bounds__(StripThreads<kCells>::NT, kSMinBlocks)
    adjoint_strip_kernel(const __grid_constant__ AdjMaps maps, const AdjArgs a, const StripSched sch) {
    constexpr int NT = StripThreads<kCells>::NT;
    constexpr int BX = StripShape::BX;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float coef_s[2][8];  // level coefficients, two levels in flight
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + kSS * StripShape::STAGE_BYTES);

    const int tid = threadIdx.x;
    const int tq = tid % (kSTX / kCells), ty = tid / (kSTX / kCells);
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    // loads are numbered per CTA across its tiles: load n uses stage n % kSS
    // and barrier phase n / kSS
    auto stage_abs = [&](int n) { return base + (n % kSS) * StripShape::STAGE_BYTES; };
    auto wait_abs = [&](int n) { return mbar_wait_bounded(&full[n % kSS], (uint32_t)((n / kSS) & 1)); };

    if (tid == 0) {
        for (int f = 0; f < kFields; ++f) prefetch_tensormap(&maps.m[f]);
        for (int q = 0; q < kSS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int seq0 = 0;  // loads of this CTA's earlier tiles (all issued and consumed)
    long long unit, unit_end;
    strip_units(sch, nz, blockIdx.x, &unit, &unit_end);
    while (unit < unit_end) {
        long long t;
        int kb, ke;
        unit = strip_segment(unit, unit_end, nz, &t, &kb, &ke);
        const int X0 = (int)(t % sch.tiles_x) * kSTX, y0 = (int)(t / sch.tiles_x) * kSTY;
        const int i0 = X0 + kCells * tq - a.xoff;  // the strip's first cell (halo included: 0..nx+1)
        const int j = y0 + ty;
        const bool row_act = j <= ny + 1;
        int nact = 0;  // cells of the strip inside 0..nx+1 (a prefix or suffix of the strip)
        for (int m = 0; m < kCells; ++m) nact += (i0 + m >= 0 && i0 + m <= nx + 1) ? 1 : 0;
        const bool full_strip = row_act && nact == kCells && a.vec;
        const int bxs = X0 - 4, bys = y0 - 1;  // box start (tensor coordinates), x 16-byte aligned
        const int nseq = ke - kb + 2;  // loads: levels kb-1 .. ke

        // load r of this tile (levels kb-1+r) is the CTA's load seq0 + r
        auto stage_of = [&](int r) { return stage_abs(seq0 + r); };
        auto wait = [&](int r) { return wait_abs(seq0 + r); };
        auto issue = [&](int r, int lev) {
            uint64_t* bar = &full[(seq0 + r) % kSS];
            unsigned char* dst = stage_of(r);
            mbar_arrive_expect_tx(bar, kFields * StripShape::BOX_BYTES);
            for (int f = 0; f < kFields; ++f) tma_load_3d(dst + f * StripShape::BOX_STRIDE, &maps.m[f], bar, bxs, bys, lev);
        };

        int issued = 0;
        if (tid == 0)
            for (; issued < kSS && issued < nseq; ++issued) issue(issued, kb - 1 + issued);

        const int cc = (ty + 1) * BX + 4 + kCells * tq;  // box index of the strip's first cell
        const float tcx = (float)a.tcx, tcy = (float)a.tcy;
        float* __restrict__ gu = static_cast<float*>(a.gu);
        float* __restrict__ gv = static_cast<float*>(a.gv);
        float* __restrict__ gw = static_cast<float*>(a.gw);
        size_t g = (size_t)j * (size_t)a.sy + (size_t)(long long)i0 + (size_t)kb * (size_t)a.sz;

        bool bad = false;
        for (int q = 0; q < 3 && q < nseq; ++q) {
            const bool ok = wait(q);
            bad |= !ok;
            if (ok) zero_outside_strip<NT>(stage_of(q), kb - 1 + q, a, X0, y0, tid);
        }
        level_coefs<float>(a, kb, tid, coef_s[0]);
        bool abort = __syncthreads_or(bad);

        for (int k = kb; k < ke && !abort; ++k) {
            const int r = k - kb;
            const double c_next = (tid < 7 && k + 1 < ke) ? level_coef(a, k + 1, tid) : 0.0;
            const unsigned char* Sm = stage_of(r);      // level k-1
            const unsigned char* S0 = stage_of(r + 1);  // level k
            const unsigned char* Sp = stage_of(r + 2);  // level k+1
            auto fld = [&](const unsigned char* st, int f) {
                return reinterpret_cast<const float*>(st + f * StripShape::BOX_STRIDE) + cc;
            };
            const float* cs = coef_s[r & 1];
            const float tz1p = cs[0], tz2m = cs[1], tz20 = cs[2], td1p = cs[3], td10 = cs[4], td2m = cs[5], td20 = cs[6];

            // rows: 0 = the strip's row, N = +1, S = -1; index m+1 = cell m,
            // m = its west neighbour, m+2 = its east neighbour
            float gu0[kCells + 2], guN[kCells + 2], guS[kCells + 2], gum[kCells + 2], gup[kCells + 2];
            float gv0[kCells + 2], gvN[kCells + 2], gvS[kCells + 2], gvm[kCells + 2], gvp[kCells + 2], gvpS[kCells + 2];
            float gw0[kCells + 2], gwN[kCells + 2], gwS[kCells + 2], gwm[kCells + 2], gwmN[kCells + 2], gwp[kCells + 2];
            float u0[kCells + 2], uN[kCells + 2], up[kCells + 2], v0[kCells + 2], vN[kCells + 2], vS[kCells + 2];
            float vp[kCells + 2], vpS[kCells + 2], w0[kCells + 2], wN[kCells + 2], wm[kCells + 2], wmN[kCells + 2];
            float wp[kCells + 2];
            row_strip<kCells, true, true>(fld(S0, 3), gu0);
            row_strip<kCells, true, false>(fld(S0, 3) + BX, guN);
            row_strip<kCells, false, false>(fld(S0, 3) - BX, guS);
            row_strip<kCells, false, false>(fld(Sm, 3), gum);
            row_strip<kCells, true, false>(fld(Sp, 3), gup);
            row_strip<kCells, true, true>(fld(S0, 4), gv0);
            row_strip<kCells, false, false>(fld(S0, 4) + BX, gvN);
            row_strip<kCells, false, true>(fld(S0, 4) - BX, gvS);
            row_strip<kCells, false, false>(fld(Sm, 4), gvm);
            row_strip<kCells, false, false>(fld(Sp, 4), gvp);
            row_strip<kCells, false, false>(fld(Sp, 4) - BX, gvpS);
            row_strip<kCells, true, true>(fld(S0, 5), gw0);
            row_strip<kCells, false, false>(fld(S0, 5) + BX, gwN);
            row_strip<kCells, false, false>(fld(S0, 5) - BX, gwS);
            row_strip<kCells, false, true>(fld(Sm, 5), gwm);
            row_strip<kCells, false, false>(fld(Sm, 5) + BX, gwmN);
            row_strip<kCells, false, false>(fld(Sp, 5), gwp);
            row_strip<kCells, true, true>(fld(S0, 0), u0);
            row_strip<kCells, true, false>(fld(S0, 0) + BX, uN);
            row_strip<kCells, true, false>(fld(Sp, 0), up);
            row_strip<kCells, false, true>(fld(S0, 1), v0);
            row_strip<kCells, false, false>(fld(S0, 1) + BX, vN);
            row_strip<kCells, false, true>(fld(S0, 1) - BX, vS);
            row_strip<kCells, false, false>(fld(Sp, 1), vp);
            row_strip<kCells, false, false>(fld(Sp, 1) - BX, vpS);
            row_strip<kCells, false, true>(fld(S0, 2), w0);
            row_strip<kCells, false, false>(fld(S0, 2) + BX, wN);
            row_strip<kCells, false, true>(fld(Sm, 2), wm);
            row_strip<kCells, false, false>(fld(Sm, 2) + BX, wmN);
            row_strip<kCells, false, false>(fld(Sp, 2), wp);

            float ru[kCells], rv[kCells], rw[kCells];
    #pragma unroll
            for (int m = 0; m < kCells; ++m) {
                const int C = m + 1, W = m, E = m + 2;
                const float su_c = gu0[C], su_e = gu0[E], su_w = gu0[W], su_n = guN[C], su_s = guS[C], su_nw = guN[W];
                const float su_km = gum[C], su_kp = gup[C], su_kp_w = gup[W];
                const float sv_c = gv0[C], sv_e = gv0[E], sv_w = gv0[W], sv_n = gvN[C], sv_s = gvS[C], sv_se = gvS[E];
                const float sv_km = gvm[C], sv_kp = gvp[C], sv_kp_s = gvpS[C];
                const float sw_c = gw0[C], sw_e = gw0[E], sw_w = gw0[W], sw_n = gwN[C], sw_s = gwS[C];
                const float sw_km = gwm[C], sw_km_e = gwm[E], sw_km_n = gwmN[C], sw_kp = gwp[C];
                const float u_c = u0[C], u_e = u0[E], u_w = u0[W], u_n = uN[C], u_nw = uN[W];
                const float u_kp = up[C], u_kp_w = up[W];
                const float v_c = v0[C], v_e = v0[E], v_n = vN[C], v_s = vS[C], v_se = vS[E];
                const float v_kp = vp[C], v_kp_s = vpS[C];
                const float w_c = w0[C], w_e = w0[E], w_n = wN[C];
                const float w_kmc = wm[C], w_kme = wm[E], w_kmn = wmN[C], w_kp = wp[C];
                float r_u = tcx * ((u_e + u_c + u_c) * su_e + u_w * su_c - (u_w + u_c + u_c) * su_w - u_e * su_c);
                r_u += tcy * ((v_c + v_e) * su_n - (v_s + v_se) * su_s);
                r_u += tz1p * (w_c + w_e) * su_kp - tz2m * (w_kmc + w_kme) * su_km;
                r_u += tcx * (v_c * sv_e + v_s * sv_se - v_e * sv_c - v_se * sv_s);
                r_u += tcx * (w_c * sw_e + w_kmc * sw_km_e - w_e * sw_c - w_kme * sw_km);
                float r_v = tcy * ((v_n + v_c + v_c) * sv_n + v_s * sv_c - (v_s + v_c + v_c) * sv_s - v_n * sv_c);
                r_v += tcx * ((u_c + u_n) * sv_e - (u_w + u_nw) * sv_w);
                r_v += tz1p * (w_c + w_n) * sv_kp - tz2m * (w_kmc + w_kmn) * sv_km;
                r_v += tcy * (u_c * su_n + u_w * su_nw - u_n * su_c - u_nw * su_w);
                r_v += tcy * (w_c * sw_n + w_kmc * sw_km_n - w_n * sw_c - w_kmn * sw_km);
                float r_w = tz1p * (u_c * su_kp + u_w * su_kp_w) - tz20 * (u_kp * su_c + u_kp_w * su_w);
                r_w += tz1p * (v_c * sv_kp + v_s * sv_kp_s) - tz20 * (v_kp * sv_c + v_kp_s * sv_s);
                r_w += tcx * ((u_c + u_kp) * sw_e - (u_w + u_kp_w) * sw_w);
                r_w += tcy * ((v_c + v_kp) * sw_n - (v_s + v_kp_s) * sw_s);
                r_w += td1p * (w_kp + w_c + w_c) * sw_kp + td10 * w_kmc * sw_c;
                r_w -= td2m * (w_kmc + w_c + w_c) * sw_km + td20 * w_kp * sw_c;
                ru[m] = r_u;
                rv[m] = r_v;
                rw[m] = r_w;
            }
            if (full_strip && kCells == 4) {
                float4* pu = reinterpret_cast<float4*>(gu + g);
                float4* pv = reinterpret_cast<float4*>(gv + g);
                float4* pw_ = reinterpret_cast<float4*>(gw + g);
                float4 nu = make_float4(ru[0], ru[1], ru[kCells - 2], ru[kCells - 1]);
                float4 nv = make_float4(rv[0], rv[1], rv[kCells - 2], rv[kCells - 1]);
                float4 nw = make_float4(rw[0], rw[1], rw[kCells - 2], rw[kCells - 1]);
                if (a.accumulate) {
                    const float4 ou = *pu, ov = *pv, ow = *pw_;
                    nu = make_float4(ou.x + nu.x, ou.y + nu.y, ou.z + nu.z, ou.w + nu.w);
                    nv = make_float4(ov.x + nv.x, ov.y + nv.y, ov.z + nv.z, ov.w + nv.w);
                    nw = make_float4(ow.x + nw.x, ow.y + nw.y, ow.z + nw.z, ow.w + nw.w);
                }
                *pu = nu;
                *pv = nv;
                *pw_ = nw;
            } else if (full_strip) {
                float2* pu = reinterpret_cast<float2*>(gu + g);
                float2* pv = reinterpret_cast<float2*>(gv + g);
                float2* pw_ = reinterpret_cast<float2*>(gw + g);
                float2 nu = make_float2(ru[0], ru[kCells - 1]);
                float2 nv = make_float2(rv[0], rv[kCells - 1]);
                float2 nw = make_float2(rw[0], rw[kCells - 1]);
                if (a.accumulate) {
                    const float2 ou = *pu, ov = *pv, ow = *pw_;
                    nu = make_float2(ou.x + nu.x, ou.y + nu.y);
                    nv = make_float2(ov.x + nv.x, ov.y + nv.y);
                    nw = make_float2(ow.x + nw.x, ow.y + nw.y);
                }
                *pu = nu;
                *pv = nv;
                *pw_ = nw;
            } else if (row_act) {
    #pragma unroll
                for (int m = 0; m < kCells; ++m) {
                    if (i0 + m < 0 || i0 + m > nx + 1) continue;
                    const size_t gm = g + (size_t)m;
                    if (a.accumulate) {
                        gu[gm] += ru[m];
                        gv[gm] += rv[m];
                        gw[gm] += rw[m];
                    } else {
                        gu[gm] = ru[m];
                        gv[gm] = rv[m];
                        gw[gm] = rw[m];
                    }
                }
            }
            g += (size_t)a.sz;
            if (tid < 7 && k + 1 < ke) coef_s[(r + 1) & 1][tid] = (float)c_next;
            // level k+2, the next step's upper level: waited for here, after
            // this step's work, so that its copy (issued at the end of the
            // previous step) has had the whole step to arrive
            if (r + 3 < nseq) {
                const bool ok = wait(r + 3);
                bad |= !ok;
                if (ok) zero_outside_strip<NT>(stage_of(r + 3), k + 2, a, X0, y0, tid);
            }
            abort = __syncthreads_or(bad);  // level k-1's stage is free
            if (!abort && tid == 0 && issued < nseq) {
                fence_proxy_async_smem();
                issue(issued, kb - 1 + issued);
                ++issued;
            }
        }
        if (abort) {
            if (tid == 0) {
                atomicOr(&tu_status, kStatusTimeout);
                for (int q = (issued > kSS ? issued - kSS : 0); q < issued; ++q) (void)wait(q);
            }
            return;
        }
        seq0 += nseq;
    }
}

}  // namespace

TileShape adjoint_shape(int elem_bytes) {
    if (elem_bytes == 8)
        return TileShape{kTX, kTY, AdjShape<double>::BX, AdjShape<double>::BY, AdjShape<double>::SMEM_BYTES,
                         AdjShape<double>::NT};
    return TileShape{kSTX, kSTY, StripShape::BX, StripShape::BY, StripShape::SMEM_BYTES, kSNT};
}

cudaError_t launch_adjoint(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st) {
    AdjMaps m;
    for (int f = 0; f < kFields; ++f) m.m[f] = maps6[f];
    // strips of kStripCells cells, tiles laid out in tensor x = i + xoff
    const int sx = (a.nx + 2 + a.xoff + kSTX - 1) / kSTX, sy = (a.ny + 2 + kSTY - 1) / kSTY;
    auto kern = adjoint_strip_kernel<kStripCells>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, StripShape::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)sx * sy;
    long long slots = 0;
    if ((e = persistent_grid(kern, kSNT, StripShape::SMEM_BYTES, 1ll << 40, &slots)) != cudaSuccess) return e;
    int chunks = 1;  // chunk-major items when the tiles fill the slots, as many chunks as fill the waves best
    if (tiles >= slots &&
        (e = choose_kchunks(kern, kSNT, StripShape::SMEM_BYTES, tiles, a.nz, &chunks)) != cudaSuccess)
        return e;
    const StripSched sch = make_strip_sched(sx, tiles, a.nz, slots, chunks);
    kern<<<(unsigned)sch.grid, kSNT, StripShape::SMEM_BYTES, st>>>(m, a, sch);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_paired(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st) {
    AdjMaps m;
    for (int f = 0; f < kFields; ++f) m.m[f] = maps6[f];
    const int tx = (a.nx + 2 + kTX - 1) / kTX, ty = (a.ny + 2 + kTY - 1) / kTY;
    cudaError_t e = cudaFuncSetAttribute(adjoint_paired_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmemBytes);
    if (e != cudaSuccess) return e;
    int chunks = 1;
    if ((e = choose_kchunks(adjoint_paired_kernel, kPNT, kPSmemBytes, (long long)tx * ty, a.nz, &chunks)) !=
        cudaSuccess)
        return e;
    adjoint_paired_kernel<<<dim3(tx, ty, chunks), kPNT, kPSmemBytes, st>>>(m, a);
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
