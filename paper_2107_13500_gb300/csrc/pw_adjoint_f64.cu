// pw_adjoint_f64.cu -- transpose of the PW advection Jacobian in native FP64
// (PW_F64), arranged so that every product shared by two cells is formed
// once.
//
// GB300 retires about two FP64 lane operations per clock per SM, so this
// kernel is bound by its FP64 operation count. The forward map is a sum of
// face terms: for each of the nine (output, direction) families -- su, sv,
// sw advected along x, y, z -- output P has a lower term c_lo(P) q(P-e) F(P-e/2)
// and an upper term -c_hi(P) q(P+e) F(P+e/2), with q the advected field and
// F = a + b the face sum of the advecting one (Sec. II-A, Listing 1 and its
// two companions). The scalar J = sum_P lam(P) s(P) then regroups by face:
// J = sum_f F(f) Phi(f), Phi(P+e/2) = c_lo(P+e) lam(P+e) q(P) - c_hi(P) lam(P) q(P+e),
// so that
//   dJ/dq(C) = c_lo(C+e) lam(C+e) F(C+e/2) - c_hi(C-e) lam(C-e) F(C-e/2)
//   dJ/da(C) = Phi of each face whose sum F contains cell C (two faces).
// For the three families that advect a field by itself (su along x, sv
// along y, sw along z) the two roles merge; with a constant coefficient
// (x and y) D(P+e/2) = lam(P+e) - lam(P) and E = D F give
//   dJ/dq(C) = E(C+e/2) + E(C-e/2) + q(C) (lam(C+e) - lam(C-e)).
// The constant coefficients tcx and tcy are applied once per output
// (gu = tcx Xu + tcy Yu + Zu), and the level coefficients are folded into
// the cotangents once per cell (a = c_lo lam, b = c_hi lam).
//
// A CTA owns a TX x TY tile of interior cells and marches up the column.
// Per level it runs three phases, as the FP64 forward kernel does:
//   scale   a = tzc1 lam and b = tzc2 lam of u and v cotangents, for the
//           level two above, into a two-level shared ring;
//   items   the quantities a cell shares with its x neighbour (E of su-x,
//           F of sv-x and sw-x, Phi of su-y and su-z) and with its y
//           neighbour (E of sv-y, F of su-y and sw-y, Phi of sv-x and sv-z),
//           each once per position, into shared arrays;
//   points  one thread per cell: the rest, with the vertical face terms
//           carried in registers to the next level.
// FP64 operations per cell (32 x 8 tile): about 50 in the point phase, 20 in
// items and 4.5 in scale, against about 100 for the cell-by-cell gather.
// The halo cells (i = 0, nx+1 or j = 0, ny+1), which only the few output
// points next to them read, are gathered cell by cell by the launch's
// trailing CTAs, so that the tiles stay aligned with the interior.
//
// Levels arrive through a four-stage TMA ring of the six fields (u, v, w,
// gsu, gsv, gsw; tile plus a one-cell halo); a level's cotangent cells that
// are not computed output points are cleared in the stage one step before
// their first read. All waits are bounded.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw.h"
#include "pw_adjoint_halo.cuh"
#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace {

constexpr int kTX = 32, kTY = 8, kS = 4, kFields = 6;
constexpr int kNT = kTX * kTY;

struct AF {
    // box: tensor x from the tile origin x0 (cells x0 - xoff .. x0 - xoff + BX - 1), rows y0 .. y0 + TY + 1
    static constexpr int BX = round_up(kTX + 2 + 1, 2);
    static constexpr int BY = kTY + 2;
    static constexpr int BOX_BYTES = BX * BY * 8;
    static constexpr int BOX_STRIDE = round_up(BOX_BYTES, 128);
    static constexpr int STAGE_BYTES = kFields * BOX_STRIDE;
    // x-shared positions P = (x0 + c, y0 + 1 + r): TY rows x (TX + 1) columns
    static constexpr int XW = kTX + 1, NXP = kTY * XW;
    // y-shared positions P = (x0 + 1 + c, y0 + r): (TY + 1) rows x TX columns
    static constexpr int YW = kTX, NYP = (kTY + 1) * YW;
    // one flat work list per phase: x positions in slots [0, NXP), y positions
    // from the next warp boundary, so that no warp mixes the two
    static constexpr int YSLOT0 = round_up(NXP, 32);
    static constexpr int NSLOT = YSLOT0 + NYP;
    static constexpr int ITERS = (NSLOT + kNT - 1) / kNT;
    // per level: a3 | b3 (x positions) | a6 | b6 (y positions)
    static constexpr int NSCALE = 2 * NXP + 2 * NYP;
    // ring | barriers (64 B) | scale [2][NSCALE] | x items [5][NXP] | y items [5][NYP] | alignment slack
    static constexpr int SC_OFFSET = kS * STAGE_BYTES + 64;
    static constexpr int IX_OFFSET = SC_OFFSET + 2 * NSCALE * 8;
    static constexpr int IY_OFFSET = IX_OFFSET + 5 * NXP * 8;
    static constexpr int SMEM_BYTES = IY_OFFSET + 5 * NYP * 8 + 128;
    static_assert(BX <= 256 && BY <= 256, "TMA box limit");
    static_assert(kS * 8 <= 64, "ring barriers must fit before the scale ring");
    static_assert(kS >= 4, "step k reads levels k, k+1, scales k+2 and cleans k+3");
    static_assert(SMEM_BYTES <= 113 * 1024, "two CTAs per SM");
};

// x items: E1 (su-x), F4 (sv-x), F7 (sw-x), P2 (su-y), P3 (su-z)
enum { kE1 = 0, kF4, kF7, kP2, kP3 };
// y items: E5 (sv-y), F2 (su-y), F8 (sw-y), P4 (sv-x), P6 (sv-z)
enum { kE5 = 0, kF2, kF8, kP4, kP6 };

struct AdjF64Maps {
    CUtensorMap m[kFields];  // u, v, w, gsu, gsv, gsw
};

// Clear, in a landed stage (level lev), every cotangent cell that is not a
// computed output point: cells outside i = 1..nx, j = 1..ny, and whole boxes
// of levels where the field is not computed (su, sv: levels 1..nz-1; sw:
// 1..nz-2). Only tiles at the domain edge and the bottom and top levels
// have such cells. The writes are ordered before the stage's next TMA load.
__device__ __forceinline__ void clean_stage(unsigned char* stage, int lev, const AdjArgs& a, int x0, int y0,
                                            int tid) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool lev_s = lev >= 1 && lev <= nz - 1;
    const bool lev_w = lev >= 1 && lev <= nz - 2;
    const int i0 = x0 - a.xoff, j0 = y0;  // cell of box column 0, row 0
    const bool edge = i0 < 1 || i0 + AF::BX - 1 > nx || j0 < 1 || j0 + AF::BY - 1 > ny;
    if (!edge && lev_s && lev_w) return;  // CTA-uniform
    bool wrote = false;
    for (int f = 3; f < kFields; ++f) {
        const bool lv = (f == 5) ? lev_w : lev_s;
        if (lv && !edge) continue;
        double* box = reinterpret_cast<double*>(stage + f * AF::BOX_STRIDE);
        for (int n = tid; n < AF::BX * AF::BY; n += kNT) {
            const int r = n / AF::BX, b = n - r * AF::BX;
            const int i = i0 + b, j = j0 + r;
            if (!lv || i < 1 || i > nx || j < 1 || j > ny) {
                box[n] = 0.0;
                wrote = true;
            }
        }
    }
    if (wrote) fence_proxy_async_smem();
}

struct Smem {
    unsigned char* base;  // ring stages, 128-byte aligned
    uint64_t* full;
    double* scl;  // [slot = level & 1][NSCALE]
    double* ix;   // [5][NXP]
    double* iy;   // [5][NYP]

    __device__ __forceinline__ void setup(unsigned char* raw) {
        base = raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
        full = reinterpret_cast<uint64_t*>(base + kS * AF::STAGE_BYTES);
        scl = reinterpret_cast<double*>(base + AF::SC_OFFSET);
        ix = reinterpret_cast<double*>(base + AF::IX_OFFSET);
        iy = reinterpret_cast<double*>(base + AF::IY_OFFSET);
    }
    __device__ __forceinline__ unsigned char* stage(int seq) const { return base + (seq % kS) * AF::STAGE_BYTES; }
    __device__ __forceinline__ const double* box(int seq, int f) const {
        return reinterpret_cast<const double*>(stage(seq) + f * AF::BOX_STRIDE);
    }
    __device__ __forceinline__ bool wait(int seq) {
        return mbar_wait_bounded(&full[seq % kS], (uint32_t)((seq / kS) & 1));
    }
};

// Offsets of b3 and b6 in a level's scale slot: with equal coefficients
// they are a3 and a6. (At the top level, where b is 0 and a is not, every use
// of b multiplies a value of the level above the domain, which reads as 0.)
template <bool kEq>
__device__ __forceinline__ constexpr int b3_off() { return kEq ? 0 : AF::NXP; }
template <bool kEq>
__device__ __forceinline__ constexpr int b6_off() { return kEq ? 2 * AF::NXP : 2 * AF::NXP + AF::NYP; }

// True when every level's two vertical coefficients are the same number
// (tzc1(k) = tzc2(k) and tzd1(k) = tzd2(k) on levels 1..nz-2: a grid without
// density stratification); the same answer for every tile of a domain.
// Compared as 32-bit words (a comparison of doubles issues on the FP64 pipe).
__device__ __forceinline__ bool vertical_pairs_equal(const AdjArgs& a, int tid) {
    auto same = [](double x, double y) {
        return __double2hiint(x) == __double2hiint(y) && __double2loint(x) == __double2loint(y);
    };
    bool eq = true;
    for (int k = 1 + tid; k <= a.nz - 2; k += kNT)
        eq &= same(__ldg(a.tzc1 + k), __ldg(a.tzc2 + k)) && same(__ldg(a.tzd1 + k), __ldg(a.tzd2 + k));
    return __syncthreads_and(eq) != 0;
}

// a3 = tzc1 gsu, b3 = tzc2 gsu at the x positions, a6, b6 of gsv at the y
// positions, of level lev (load seq) into slot lev & 1. kEq: the level's two
// coefficients are equal, so only a3 and a6 are formed and stand for b3 and
// b6 too (see b_off).
template <bool kEq>
__device__ __forceinline__ void scale_level(const Smem& sm, int seq, int lev, const AdjArgs& a, int tid) {
    const double* LU = sm.box(seq, 3) + a.xoff;
    const double* LV = sm.box(seq, 4) + a.xoff;
    const double c1 = coef_at(a.tzc1, lev, a.nz), c2 = tzc2_at(a.tzc2, lev, a.nz);
    double* s = sm.scl + (lev & 1) * AF::NSCALE;
#pragma unroll
    for (int q = 0; q < AF::ITERS; ++q) {
        const int n = tid + q * kNT;
        if (n < AF::NXP) {
            const int r = n / AF::XW, c = n - r * AF::XW;
            const double lu = LU[(r + 1) * AF::BX + c];
            s[n] = __dmul_rn(c1, lu);
            if (!kEq) s[AF::NXP + n] = __dmul_rn(c2, lu);
        } else if (n >= AF::YSLOT0 && n < AF::NSLOT) {
            const int m = n - AF::YSLOT0;
            const int r = m / AF::YW, c = m - r * AF::YW;
            const double lv = LV[r * AF::BX + c + 1];
            s[2 * AF::NXP + m] = __dmul_rn(c1, lv);
            if (!kEq) s[2 * AF::NXP + AF::NYP + m] = __dmul_rn(c2, lv);
        }
    }
}

// The shared items of level lev (load seq; the level above is load seq + 1).
template <bool kEq>
__device__ __forceinline__ void items_level(const Smem& sm, int seq, int lev, const AdjArgs& a, int tid) {
    const int xo = a.xoff;
    const double* U = sm.box(seq, 0) + xo;
    const double* V = sm.box(seq, 1) + xo;
    const double* LU = sm.box(seq, 3) + xo;
    const double* LV = sm.box(seq, 4) + xo;
    const double* U1 = sm.box(seq + 1, 0) + xo;
    const double* V1 = sm.box(seq + 1, 1) + xo;
    const double* sb = sm.scl + (lev & 1) * AF::NSCALE;        // b of this level
    const double* sa = sm.scl + ((lev + 1) & 1) * AF::NSCALE;  // a of the level above
#pragma unroll
    for (int q = 0; q < AF::ITERS; ++q) {
        const int n = tid + q * kNT;
        if (n < AF::NXP) {
            const int r = n / AF::XW, c = n - r * AF::XW;
            const int p = (r + 1) * AF::BX + c;
            const double u0 = U[p], ue = U[p + 1], un = U[p + AF::BX], uk = U1[p];
            const double l0 = LU[p], le = LU[p + 1], ln = LU[p + AF::BX];
            double* ix = sm.ix + n;
            ix[kE1 * AF::NXP] = __dmul_rn(__dsub_rn(le, l0), __dadd_rn(u0, ue));
            ix[kF4 * AF::NXP] = __dadd_rn(u0, un);
            ix[kF7 * AF::NXP] = __dadd_rn(u0, uk);
            ix[kP2 * AF::NXP] = __fma_rn(ln, u0, -__dmul_rn(l0, un));
            ix[kP3 * AF::NXP] = __fma_rn(sa[n], u0, -__dmul_rn(sb[b3_off<kEq>() + n], uk));
        } else if (n >= AF::YSLOT0 && n < AF::NSLOT) {
            const int m = n - AF::YSLOT0;
            const int r = m / AF::YW, c = m - r * AF::YW;
            const int p = r * AF::BX + c + 1;
            const double v0 = V[p], vn = V[p + AF::BX], ve = V[p + 1], vk = V1[p];
            const double l0 = LV[p], ln = LV[p + AF::BX], le = LV[p + 1];
            double* iy = sm.iy + m;
            iy[kE5 * AF::NYP] = __dmul_rn(__dsub_rn(ln, l0), __dadd_rn(v0, vn));
            iy[kF2 * AF::NYP] = __dadd_rn(v0, ve);
            iy[kF8 * AF::NYP] = __dadd_rn(v0, vk);
            iy[kP4 * AF::NYP] = __fma_rn(le, v0, -__dmul_rn(l0, ve));
            iy[kP6 * AF::NYP] = __fma_rn(sa[2 * AF::NXP + m], v0, -__dmul_rn(sb[b6_off<kEq>() + m], vk));
        }
    }
}

// One work item: output levels kb..ke-1 of the tile (bx, by). kEq: every
// level's two vertical coefficients are equal; kSameT: tcx = tcy. Each lets
// a product be shared (the b cotangents are the a ones; sw's per-level
// scaled cotangent serves both its faces; x and y parts of an output take
// one coefficient product).
template <bool kEq, bool kSameT>
__device__ __forceinline__ void adjoint_tile(const AdjF64Maps& maps, const AdjArgs& a, Smem& sm, int bx, int by,
                                             int kb, int ke, int tid) {
    const int tx = tid % kTX, ty = tid / kTX;
    const int x0 = bx * kTX, y0 = by * kTY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;  // interior cell
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool act = (i <= nx) && (j <= ny);
    const int nseq = ke - kb + 2;  // loads: levels kb-1 .. ke (out-of-range levels read as 0)

    auto issue = [&](int seq) {
        const int s = seq % kS;
        uint64_t* bar = &sm.full[s];
        unsigned char* dst = sm.base + s * AF::STAGE_BYTES;
        mbar_arrive_expect_tx(bar, kFields * AF::BOX_BYTES);
        for (int f = 0; f < kFields; ++f)
            tma_load_3d(dst + f * AF::BOX_STRIDE, &maps.m[f], bar, x0, y0, kb - 1 + seq);
    };

    if (tid == 0) {
        for (int f = 0; f < kFields; ++f) prefetch_tensormap(&maps.m[f]);
        for (int s = 0; s < kS; ++s) mbar_init(&sm.full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < kS && issued < nseq; ++issued) issue(issued);

    const int c0 = (ty + 1) * AF::BX + a.xoff + tx + 1;  // the cell in a box
    const int xi = ty * AF::XW + tx + 1;                  // its x position; the west neighbour's is xi - 1
    const int yi = (ty + 1) * AF::YW + tx;                // its y position; the south neighbour's is yi - YW
    const double tcx = a.tcx, tcy = a.tcy;

    bool bad = false;
    int cleaned = 0;
    for (; cleaned < kS && cleaned < nseq; ++cleaned) {
        const bool ok = sm.wait(cleaned);
        bad |= !ok;
        if (ok) clean_stage(sm.stage(cleaned), kb - 1 + cleaned, a, x0, y0, tid);
    }
    bool abort = __syncthreads_or(bad);

    // values of level k-1 carried up the column (k = kb first): the two
    // vertical-family Phi of sw-x and sw-y at the cell, the vertical face
    // sums and Phi of su-z, sv-z, sw-z below the cell's level, and the b
    // cotangents of the level below
    double p7m = 0.0, p8m = 0.0, f3m = 0.0, f6m = 0.0, f9m = 0.0, p9m = 0.0;
    double b3m = 0.0, b6m = 0.0, b9m = 0.0, b3c = 0.0, b6c = 0.0;
    double a9c = 0.0;  // kEq: tzd1(k) gsw(k), which is also sw's b cotangent of level k
    if (!abort) {
        const double* W = sm.box(0, 2);
        const double* LW = sm.box(0, 5);
        const double wc = W[c0], we = W[c0 + 1], wn = W[c0 + AF::BX];
        const double lc = LW[c0], le = LW[c0 + 1], ln = LW[c0 + AF::BX];
        const double wk = sm.box(1, 2)[c0];
        p7m = __fma_rn(le, wc, -__dmul_rn(lc, we));
        p8m = __fma_rn(ln, wc, -__dmul_rn(lc, wn));
        f3m = __dadd_rn(wc, we);
        f6m = __dadd_rn(wc, wn);
        f9m = __dadd_rn(wc, wk);
        const double c2 = tzc2_at(a.tzc2, kb - 1, nz);
        b3m = __dmul_rn(c2, sm.box(0, 3)[c0]);
        b6m = __dmul_rn(c2, sm.box(0, 4)[c0]);
        b9m = __dmul_rn(coef_at(a.tzd2, kb - 1, nz), lc);
        const double a9 = __dmul_rn(coef_at(a.tzd1, kb, nz), sm.box(1, 5)[c0]);
        p9m = __fma_rn(a9, wc, -__dmul_rn(b9m, wk));
        a9c = a9;
        scale_level<kEq>(sm, 1, kb, a, tid);
        scale_level<kEq>(sm, 2, kb + 1, a, tid);
    }
    abort = __syncthreads_or(bad);  // load 0 is free
    if (!abort && tid == 0 && issued < nseq) {
        fence_proxy_async_smem();
        issue(issued);
        ++issued;
    }
    if (!abort) {
        items_level<kEq>(sm, 1, kb, a, tid);
        const double* s = sm.scl + (kb & 1) * AF::NSCALE;
        b3c = s[b3_off<kEq>() + xi];
        b6c = s[b6_off<kEq>() + yi];
    }
    abort = __syncthreads_or(bad);

    double* __restrict__ gu = static_cast<double*>(a.gu);
    double* __restrict__ gv = static_cast<double*>(a.gv);
    double* __restrict__ gw = static_cast<double*>(a.gw);
    const size_t gsz = (size_t)a.sz;
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)kb * gsz;
    const double* ix = sm.ix;
    const double* iy = sm.iy;

    for (int k = kb; k < ke && !abort; ++k, g += gsz) {
        const int r = k - kb;
        // ---- points (level k = load r+1, level k+1 = load r+2)
        const double* U = sm.box(r + 1, 0);
        const double* V = sm.box(r + 1, 1);
        const double* W = sm.box(r + 1, 2);
        const double* LU = sm.box(r + 1, 3);
        const double* LV = sm.box(r + 1, 4);
        const double* LW = sm.box(r + 1, 5);
        const double wk = sm.box(r + 2, 2)[c0];
        const double lwk = sm.box(r + 2, 5)[c0];
        const double* sa = sm.scl + ((k + 1) & 1) * AF::NSCALE;
        const double uc = U[c0], vc = V[c0], wc = W[c0], we = W[c0 + 1], wn = W[c0 + AF::BX];
        const double lwc = LW[c0], lwe = LW[c0 + 1], lww = LW[c0 - 1], lwn = LW[c0 + AF::BX], lws = LW[c0 - AF::BX];

        // gu: x (su-x, F of sv-x and sw-x), y (su-y), z (su-z)
        double xu = __dadd_rn(ix[kE1 * AF::NXP + xi], ix[kE1 * AF::NXP + xi - 1]);
        xu = __fma_rn(uc, __dsub_rn(LU[c0 + 1], LU[c0 - 1]), xu);
        xu = __dadd_rn(xu, iy[kP4 * AF::NYP + yi]);
        xu = __dadd_rn(xu, iy[kP4 * AF::NYP + yi - AF::YW]);
        const double p7 = __fma_rn(lwe, wc, -__dmul_rn(lwc, we));
        xu = __dadd_rn(xu, p7);
        xu = __dadd_rn(xu, p7m);
        double yu = 0.0;
        if (kSameT) {  // one coefficient for the x and y parts
            xu = __fma_rn(LU[c0 + AF::BX], iy[kF2 * AF::NYP + yi], xu);
            xu = __fma_rn(-LU[c0 - AF::BX], iy[kF2 * AF::NYP + yi - AF::YW], xu);
        } else {
            yu = __fma_rn(LU[c0 + AF::BX], iy[kF2 * AF::NYP + yi],
                          -__dmul_rn(LU[c0 - AF::BX], iy[kF2 * AF::NYP + yi - AF::YW]));
        }
        const double f3 = __dadd_rn(wc, we);
        const double zu = __fma_rn(sa[xi], f3, -__dmul_rn(b3m, f3m));

        // gv: y (sv-y, F of su-y and sw-y), x (sv-x), z (sv-z)
        double yv = __dadd_rn(iy[kE5 * AF::NYP + yi], iy[kE5 * AF::NYP + yi - AF::YW]);
        yv = __fma_rn(vc, __dsub_rn(LV[c0 + AF::BX], LV[c0 - AF::BX]), yv);
        yv = __dadd_rn(yv, ix[kP2 * AF::NXP + xi]);
        yv = __dadd_rn(yv, ix[kP2 * AF::NXP + xi - 1]);
        const double p8 = __fma_rn(lwn, wc, -__dmul_rn(lwc, wn));
        yv = __dadd_rn(yv, p8);
        yv = __dadd_rn(yv, p8m);
        double xv = 0.0;
        if (kSameT) {
            yv = __fma_rn(LV[c0 + 1], ix[kF4 * AF::NXP + xi], yv);
            yv = __fma_rn(-LV[c0 - 1], ix[kF4 * AF::NXP + xi - 1], yv);
        } else {
            xv = __fma_rn(LV[c0 + 1], ix[kF4 * AF::NXP + xi], -__dmul_rn(LV[c0 - 1], ix[kF4 * AF::NXP + xi - 1]));
        }
        const double f6 = __dadd_rn(wc, wn);
        const double zv = __fma_rn(sa[2 * AF::NXP + yi], f6, -__dmul_rn(b6m, f6m));

        // gw: x (sw-x), y (sw-y), z (sw-z, F of su-z and sv-z)
        double xw = __fma_rn(lwe, ix[kF7 * AF::NXP + xi], -__dmul_rn(lww, ix[kF7 * AF::NXP + xi - 1]));
        double yw = 0.0;
        if (kSameT) {
            xw = __fma_rn(lwn, iy[kF8 * AF::NYP + yi], xw);
            xw = __fma_rn(-lws, iy[kF8 * AF::NYP + yi - AF::YW], xw);
        } else {
            yw = __fma_rn(lwn, iy[kF8 * AF::NYP + yi], -__dmul_rn(lws, iy[kF8 * AF::NYP + yi - AF::YW]));
        }
        const double a9 = __dmul_rn(coef_at(a.tzd1, k + 1, nz), lwk);
        // kEq: tzd2(k) gsw(k) = tzd1(k) gsw(k), formed one step earlier
        const double b9 = kEq ? a9c : __dmul_rn(coef_at(a.tzd2, k, nz), lwc);
        const double f9 = __dadd_rn(wc, wk);
        const double p9 = __fma_rn(a9, wc, -__dmul_rn(b9, wk));
        double zw = __dadd_rn(ix[kP3 * AF::NXP + xi], ix[kP3 * AF::NXP + xi - 1]);
        zw = __dadd_rn(zw, iy[kP6 * AF::NYP + yi]);
        zw = __dadd_rn(zw, iy[kP6 * AF::NYP + yi - AF::YW]);
        zw = __fma_rn(a9, f9, zw);
        zw = __fma_rn(-b9m, f9m, zw);
        zw = __dadd_rn(zw, p9);
        zw = __dadd_rn(zw, p9m);

        double ru, rv, rw;
        if (kSameT) {
            ru = __fma_rn(tcx, xu, zu);
            rv = __fma_rn(tcx, yv, zv);
            rw = __fma_rn(tcx, xw, zw);
        } else {
            ru = __fma_rn(tcx, xu, __fma_rn(tcy, yu, zu));
            rv = __fma_rn(tcx, xv, __fma_rn(tcy, yv, zv));
            rw = __fma_rn(tcx, xw, __fma_rn(tcy, yw, zw));
        }
        if (act) {
            if (a.accumulate) {
                gu[g] += ru;
                gv[g] += rv;
                gw[g] += rw;
            } else {
                gu[g] = ru;
                gv[g] = rv;
                gw[g] = rw;
            }
        }
        p7m = p7;
        p8m = p8;
        f3m = f3;
        f6m = f6;
        f9m = f9;
        p9m = p9;
        b9m = b9;
        a9c = a9;
        b3m = b3c;
        b6m = b6c;

        if (k + 1 < ke) {
            // ---- scale level k+2 (load r+3) into the slot level k used
            scale_level<kEq>(sm, r + 3, k + 2, a, tid);
            abort = __syncthreads_or(bad);  // load r+1 (level k) is free
            if (!abort && tid == 0 && issued < nseq) {
                fence_proxy_async_smem();
                issue(issued);
                ++issued;
            }
            // ---- items of level k+1 (loads r+2, r+3)
            if (!abort) {
                items_level<kEq>(sm, r + 2, k + 1, a, tid);
                const double* s = sm.scl + ((k + 1) & 1) * AF::NSCALE;
                b3c = s[b3_off<kEq>() + xi];
                b6c = s[b6_off<kEq>() + yi];
            }
            // level k+3, first read by the next step's scale phase: waited for
            // after the items phase, so that its copy (issued above) overlaps it
            if (!abort && cleaned < nseq) {
                const bool ok = sm.wait(cleaned);
                bad |= !ok;
                if (ok) clean_stage(sm.stage(cleaned), kb - 1 + cleaned, a, x0, y0, tid);
                ++cleaned;
            }
            abort = __syncthreads_or(bad);
        }
    }
    if (abort && tid == 0) {
        atomicOr(&tu_status, kStatusTimeout);
        for (int s = (issued > kS ? issued - kS : 0); s < issued; ++s) (void)sm.wait(s);
    }
}

// One launch: CTAs [0, sched.items) each take one work item (a level chunk
// of one tile, in the order of the one-shot schedule); the CTAs after them
// gather the halo cells, one per thread, filling the schedule's last wave.
// kSameT (tcx = tcy) is chosen on the host, equal vertical coefficients per
// CTA from the coefficient arrays.
template <bool kSameT>
__global__ void __launch_bounds__(kNT, 2) adjoint_f64_kernel(const __grid_constant__ AdjF64Maps maps, const AdjArgs a,
                                                             const ItemSched sched) {
    extern __shared__ unsigned char smem_raw[];
    const int tid = threadIdx.x;
    if ((long long)blockIdx.x >= sched.items) {  // CTA-uniform
        adjoint_halo_cell<double>(a, ((long long)blockIdx.x - sched.items) * kNT + tid);
        return;
    }
    Smem sm;
    sm.setup(smem_raw);
    int bx, by, kb, ke;
    sched_item(sched, a.nz, blockIdx.x, &bx, &by, &kb, &ke);
    if (vertical_pairs_equal(a, tid)) adjoint_tile<true, kSameT>(maps, a, sm, bx, by, kb, ke, tid);
    else adjoint_tile<false, kSameT>(maps, a, sm, bx, by, kb, ke, tid);
}

template <bool kSameT>
cudaError_t launch_adjoint_f64_t(const AdjF64Maps& m, const AdjArgs& a, cudaStream_t st) {
    auto kern = adjoint_f64_kernel<kSameT>;
    const int tx = (a.nx + kTX - 1) / kTX, ty = (a.ny + kTY - 1) / kTY;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, AF::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    ItemSched sched;
    if ((e = choose_sched(kern, kNT, AF::SMEM_BYTES, tx, ty, a.nz, &sched)) != cudaSuccess) return e;
    const long long halo = (long long)(2 * (a.ny + 2) + 2 * a.nx) * a.nz;
    const long long grid = sched.items + (halo + kNT - 1) / kNT;
    kern<<<(unsigned)grid, kNT, AF::SMEM_BYTES, st>>>(m, a, sched);
    return cudaGetLastError();
}

}  // namespace

TileShape adjoint_f64_shape() { return TileShape{kTX, kTY, AF::BX, AF::BY, AF::SMEM_BYTES, kNT}; }

cudaError_t launch_adjoint_f64(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st) {
    AdjF64Maps m;
    for (int f = 0; f < kFields; ++f) m.m[f] = maps6[f];
    return a.tcx == a.tcy ? launch_adjoint_f64_t<true>(m, a, st) : launch_adjoint_f64_t<false>(m, a, st);
}

cudaError_t read_and_clear_status_adjoint_f64(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

}  // namespace pw
