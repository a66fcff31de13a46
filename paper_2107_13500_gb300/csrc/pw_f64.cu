// pw_f64.cu -- PW advection in native FP64 arithmetic (PW_F64): the one-shot
// forward kernel and its persistent form over a batch plan.
//
// GB300 retires about two FP64 lane operations per clock per SM, so this
// kernel is bound by its FP64 instruction count, not by HBM; the design
// minimises FP64 operations per point. Every source term is a sum of six
// face terms c * q * (a + b) (Listing 1 and its two companions): q the
// advected value at the neighbour across a face, a + b twice the advecting
// velocity on that face. Two facts cut the work:
//   * every x-direction face of every output is advected by u with
//     coefficient tcx, every y-direction face by v with tcy. Scaling u and v
//     once per cell (u~ = tcx u, v~ = tcy v) turns each horizontal face sum
//     into a + b of scaled velocities, so no product needs its coefficient;
//   * each horizontal face sum is shared by the two points on either side
//     of the face, and each vertical one by the two levels around it.
// Per level, a CTA owning a TX x TY tile therefore runs three phases:
//   scale   tcx u and tcy v of the level above (all the cells the tile's
//           faces read) into a two-level shared ring;
//   faces   the six horizontal face-sum types of the level, each face once,
//           into shared arrays (a flat list of items over all threads);
//   points  one thread per point: the three vertical face sums (carried to
//           the next level in registers), then each output from its six
//           face products.
// A level's two vertical face terms carry the coefficients tzc1(k) and
// tzc2(k) (tzd1, tzd2 for sw), which differ only with density
// stratification. Where they are equal on every level (checked per domain on
// the device, bit for bit), the two terms share one product:
// c(k) (q(k-1) F(k-1/2) - q(k+1) F(k+1/2)); otherwise each face sum is
// scaled by its own coefficient.
// FP64 operations per point (32 x 16 tile): about 2.3 scaling, 6.3 face
// sums, 3 vertical sums, 18 face products, and 3 vertical coefficient
// products (6 with density): about 32.6 (35.6), against about 48 for the
// term-by-term evaluation.
//
// Levels arrive through the TMA ring of pw_ring.cuh (u, v, w boxes of the
// tile plus its one-cell halo). Step k reads boxes k and k+1 and scales
// k+2, so four stages keep the load of level k+3 in flight.
#include <cuda.h>
#include <cuda_runtime.h>

#include "pw.h"
#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace {

template <int TY_, int S_, int MINB_>
struct F64Cfg {
    static constexpr int TX = 32, TY = TY_, S = S_, MINB = MINB_;
    using Shape = RingShape<double, TX, TY, S>;
    static constexpr int NT = TX * TY;
    static constexpr int BX = Shape::BX;
    // scaled velocities: columns x0 .. x0+TX+1, rows y0 .. y0+TY+1
    static constexpr int SCW = TX + 2, SCH = TY + 2, SC_ELEMS = SCW * SCH;
    static constexpr int NSU = (TY + 1) * (TX + 2);  // tcx u: rows 1..TY+1, columns 0..TX+1
    static constexpr int NSV = (TY + 2) * (TX + 1);  // tcy v: rows 0..TY+1, columns 1..TX+1
    static constexpr int SCALE_ITERS = (NSU + NSV + NT - 1) / NT;
    // x faces of a type: TY rows x (TX+1) columns; y faces: (TY+1) rows x TX columns
    static constexpr int FXW = TX + 1, NFX = TY * FXW;
    static constexpr int FYW = TX, NFY = (TY + 1) * FYW;
    static constexpr int NFACE = 3 * NFX + 3 * NFY;
    static constexpr int FACE_ITERS = (NFACE + NT - 1) / NT;
    // ring stages | ring barriers (64 B) | scaled [2 slots][2 fields] | fx [3] | fy [3] | item | slack
    static constexpr int SC_OFFSET = S * Shape::STAGE_BYTES + 64;
    static constexpr int FX_OFFSET = SC_OFFSET + 4 * SC_ELEMS * 8;
    static constexpr int FY_OFFSET = FX_OFFSET + 3 * NFX * 8;
    static constexpr int ITEM_OFFSET = FY_OFFSET + 3 * NFY * 8;
    static constexpr int SMEM_BYTES = ITEM_OFFSET + 16 + 128;
    static_assert(S * 8 <= 64, "ring barriers must fit before the scaled velocities");
    static_assert(S >= 4, "step k reads boxes k, k+1 and scales k+2 while k+3 loads");
    static_assert(Shape::BOX_STRIDE % 8 == 0, "box stride in doubles");
};

// Variants: 0 = 32 x 16 tile, two CTAs per SM; 1 = 32 x 8 tile, three.
using FV0 = F64Cfg<16, 4, 2>;
using FV1 = F64Cfg<8, 4, 3>;

template <class C>
struct F64K {
    using Shape = typename C::Shape;

    struct Smem {
        double* sc;       // [slot = level & 1][0: tcx u, 1: tcy v][SC_ELEMS]
        double* fx;       // [3][NFX]: A (tcx u summed along x), Uy (along y), Uz (along z)
        double* fy;       // [3][NFY]: Vx (tcy v summed along x), By (along y), Vz (along z)
        long long* item;  // work item handed from thread 0 to the CTA
    };

    static __device__ __forceinline__ void setup(unsigned char* raw, Ring<Shape>& ring, Smem& sm) {
        ring.setup(raw);
        sm.sc = reinterpret_cast<double*>(ring.base + C::SC_OFFSET);
        sm.fx = reinterpret_cast<double*>(ring.base + C::FX_OFFSET);
        sm.fy = reinterpret_cast<double*>(ring.base + C::FY_OFFSET);
        sm.item = reinterpret_cast<long long*>(ring.base + C::ITEM_OFFSET);
    }

    // tcx u and tcy v of load `seq` (level lev) into slot lev & 1.
    static __device__ __forceinline__ void scale_level(const Ring<Shape>& ring, const Smem& sm, long long seq, int lev,
                                                       int xoff, double tcx, double tcy, int tid) {
        const double* U = ring.template box<double>(seq, 0) + xoff;
        const double* V = ring.template box<double>(seq, 1) + xoff;
        double* su = sm.sc + (lev & 1) * 2 * C::SC_ELEMS;
        double* sv = su + C::SC_ELEMS;
#pragma unroll
        for (int q = 0; q < C::SCALE_ITERS; ++q) {
            const int n = tid + q * C::NT;
            if (n < C::NSU) {
                const int r = 1 + n / (C::TX + 2), c = n % (C::TX + 2);
                su[r * C::SCW + c] = __dmul_rn(tcx, U[r * C::BX + c]);
            } else if (n < C::NSU + C::NSV) {
                const int m = n - C::NSU;
                const int r = m / (C::TX + 1), c = 1 + m % (C::TX + 1);
                sv[r * C::SCW + c] = __dmul_rn(tcy, V[r * C::BX + c]);
            }
        }
    }

    // The six horizontal face-sum types of level lev (scaled velocities of
    // lev in slot lev & 1, of lev+1 in the other slot). Face (r, c) of an
    // x type lies between columns x0+c and x0+c+1 on row y0+1+r; of a y type
    // between rows y0+r and y0+r+1 on column x0+1+c.
    static __device__ __forceinline__ void faces_level(const Smem& sm, int lev, int tid) {
        const double* sc = sm.sc;
        const int k0 = (lev & 1) * 2 * C::SC_ELEMS;         // tcx u of lev; tcy v follows
        const int dk = (((lev + 1) & 1) * 2 * C::SC_ELEMS) - k0;  // to the same cell at lev+1
#pragma unroll
        for (int q = 0; q < C::FACE_ITERS; ++q) {
            const int n = tid + q * C::NT;
            if (n < 3 * C::NFX) {
                const int t = n / C::NFX, e = n - t * C::NFX;
                const int r = e / C::FXW, c = e - r * C::FXW;
                const int a = k0 + (r + 1) * C::SCW + c;
                const int b = a + (t == 0 ? 1 : t == 1 ? C::SCW : dk);
                sm.fx[n] = __dadd_rn(sc[a], sc[b]);
            } else if (n < C::NFACE) {
                const int m = n - 3 * C::NFX;
                const int t = m / C::NFY, e = m - t * C::NFY;
                const int r = e / C::FYW, c = e - r * C::FYW;
                const int a = k0 + C::SC_ELEMS + r * C::SCW + c + 1;
                const int b = a + (t == 0 ? 1 : t == 1 ? C::SCW : dk);
                sm.fy[m] = __dadd_rn(sc[a], sc[b]);
            }
        }
    }

    // True when every level's two vertical coefficients are the same number:
    // tzc1(k) = tzc2(k) wherever su and sv have an upper flux, tzd1(k) =
    // tzd2(k) wherever sw is computed (a grid without density stratification).
    // The answer depends on the domain only, so every tile of it, one-shot or
    // batched, takes the same arithmetic. Compared as 32-bit words: a
    // comparison of doubles issues on the FP64 pipe.
    static __device__ bool vertical_pairs_equal(const FwdArgs& a, int tid) {
        auto same = [](double x, double y) {
            return __double2hiint(x) == __double2hiint(y) && __double2loint(x) == __double2loint(y);
        };
        bool eq = true;
        for (int k = 1 + tid; k <= a.nz - 2; k += C::NT)
            eq &= same(__ldg(a.tzc1 + k), __ldg(a.tzc2 + k)) && same(__ldg(a.tzd1 + k), __ldg(a.tzd2 + k));
        return __syncthreads_and(eq) != 0;
    }

    // One tile (bx, by) of domain `a`, output levels kb..ke-1 (a chunk of the
    // column; it reads one level below and one above). `seq` is the CTA's
    // running load count; loads are numbered relative to the lowest level
    // read, lo. Returns false if a bounded wait expired (status set, copies
    // drained).
    static __device__ bool tile(Ring<Shape>& ring, const Smem& sm, const CUtensorMap* mu, const CUtensorMap* mv,
                                const CUtensorMap* mw, const FwdArgs& a, int bx, int by, int kb, int ke, long long& seq,
                                int tid) {
        if (vertical_pairs_equal(a, tid))
            return tile_impl<true>(ring, sm, mu, mv, mw, a, bx, by, kb, ke, seq, tid);
        return tile_impl<false>(ring, sm, mu, mv, mw, a, bx, by, kb, ke, seq, tid);
    }

    // kEq: the level's vertical face terms share one coefficient product,
    // c(k) (q(k-1) F(k-1/2) - q(k+1) F(k+1/2)) with c = tzc1 = tzc2 (tzd1 =
    // tzd2 for sw): one FP64 operation less per output than scaling each face
    // sum by its own coefficient.
    template <bool kEq>
    static __device__ bool tile_impl(Ring<Shape>& ring, const Smem& sm, const CUtensorMap* mu, const CUtensorMap* mv,
                                     const CUtensorMap* mw, const FwdArgs& a, int bx, int by, int kb, int ke,
                                     long long& seq, int tid) {
        constexpr int S = C::S, BX = C::BX, TX = C::TX;
        const int tx = tid % TX, ty = tid / TX;
        const int x0 = bx * TX, y0 = by * C::TY;
        const int i = x0 + 1 + tx, j = y0 + 1 + ty;
        const bool act = (i <= a.nx) && (j <= a.ny);
        const int nz = a.nz;
        const int lo = kb > 0 ? kb - 1 : 0, hi = ke < nz ? ke : nz - 1;
        const int nl = hi - lo + 1;  // levels read
        const long long s0 = seq;
        const int xoff = a.xoff;
        const double tcx = a.tcx, tcy = a.tcy;

        int issued = 0;  // relative loads issued (thread 0)
        if (tid == 0) {
            fence_proxy_async_smem();
            for (; issued < S && issued < nl; ++issued) ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
        }
        double* __restrict__ su = static_cast<double*>(a.su);
        double* __restrict__ sv = static_cast<double*>(a.sv);
        double* __restrict__ sw = static_cast<double*>(a.sw);
        const size_t gsz = (size_t)a.sz;
        size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)lo * gsz;
        if (kb == 0 && act) {  // level 1 of the paper is not computed
            su[g] = 0.0;
            sv[g] = 0.0;
            sw[g] = 0.0;
        }

        const int c0 = (ty + 1) * BX + xoff + tx + 1;  // the point in a box
        const int fxw = ty * C::FXW + tx;                // its west x face; east = fxw + 1
        const int fys = ty * C::FYW + tx;                // its south y face; north = fys + FYW
        const int k1 = kb > 1 ? kb : 1;                  // first computed level (lo = k1 - 1)
        bool bad = false, abort = false;
        // level-(k-1) values carried up the column: the point's own u, v, w,
        // and its three vertical face sums, scaled by level k's lower
        // coefficients (tzc1(k) for su and sv, tzd1(k) for sw) unless kEq
        double uo = 0.0, vo = 0.0, wo = 0.0, w1x = 0.0, w1y = 0.0, c1 = 0.0;

        if (k1 < ke) {
            bad |= !ring.wait(s0);
            bad |= !ring.wait(s0 + 1);
            const bool top1 = (k1 == nz - 1);
            if (!top1) bad |= !ring.wait(s0 + 2);
            {
                const double* W0 = ring.template box<double>(s0, 2);
                const double* W1 = ring.template box<double>(s0 + 1, 2);
                uo = ring.template box<double>(s0, 0)[c0];
                vo = ring.template box<double>(s0, 1)[c0];
                wo = W0[c0];
                w1x = __dadd_rn(wo, W0[c0 + 1]);
                w1y = __dadd_rn(wo, W0[c0 + BX]);
                c1 = __dadd_rn(wo, W1[c0]);
                if (!kEq) {
                    const double t1 = __ldg(a.tzc1 + k1), d1 = __ldg(a.tzd1 + k1);
                    w1x = __dmul_rn(t1, w1x);
                    w1y = __dmul_rn(t1, w1y);
                    c1 = __dmul_rn(d1, c1);
                }
            }
            scale_level(ring, sm, s0 + 1, k1, xoff, tcx, tcy, tid);
            if (!top1) scale_level(ring, sm, s0 + 2, k1 + 1, xoff, tcx, tcy, tid);
            abort = __syncthreads_or(bad);  // box lo is free again
            if (!abort && tid == 0 && issued < nl) {
                fence_proxy_async_smem();
                ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
                ++issued;
            }
            if (!abort) faces_level(sm, k1, tid);
            abort = __syncthreads_or(bad);
        }

        const double* fx0 = sm.fx;
        const double* fx1 = sm.fx + C::NFX;
        const double* fx2 = sm.fx + 2 * C::NFX;
        const double* fy0 = sm.fy;
        const double* fy1 = sm.fy + C::NFY;
        const double* fy2 = sm.fy + 2 * C::NFY;
        g += (size_t)(k1 - lo) * gsz;
        for (int k = k1; k < ke && !abort; ++k, g += gsz) {
            const int r = k - lo;
            const bool top = (k == nz - 1);
            const double* U = ring.template box<double>(s0 + r, 0);
            const double* V = ring.template box<double>(s0 + r, 1);
            const double* W = ring.template box<double>(s0 + r, 2);
            const double uc = U[c0], vc = V[c0], wc = W[c0];
            const double wxk = __dadd_rn(wc, W[c0 + 1]);   // w face sum of su's upper face
            const double wyk = __dadd_rn(wc, W[c0 + BX]);  // of sv's upper face
            // su: x (u advected by tcx u), y (by tcy v), z (by w)
            double ru = __dmul_rn(U[c0 - 1], fx0[fxw]);
            ru = __fma_rn(-U[c0 + 1], fx0[fxw + 1], ru);
            ru = __fma_rn(U[c0 - BX], fy0[fys], ru);
            ru = __fma_rn(-U[c0 + BX], fy0[fys + C::FYW], ru);
            // sv: y first (its own direction), then x, then z
            double rv = __dmul_rn(V[c0 - BX], fy1[fys]);
            rv = __fma_rn(-V[c0 + BX], fy1[fys + C::FYW], rv);
            rv = __fma_rn(V[c0 - 1], fx1[fxw], rv);
            rv = __fma_rn(-V[c0 + 1], fx1[fxw + 1], rv);
            // the lower vertical terms (their coefficient is applied below if kEq)
            double zu = 0.0, zv = 0.0;
            if (kEq) {
                zu = __dmul_rn(uo, w1x);
                zv = __dmul_rn(vo, w1y);
            } else {
                ru = __fma_rn(uo, w1x, ru);
                rv = __fma_rn(vo, w1y, rv);
            }
            double rw = 0.0;
            if (!top) {
                const double* U1 = ring.template box<double>(s0 + r + 1, 0);
                const double* V1 = ring.template box<double>(s0 + r + 1, 1);
                const double* W1 = ring.template box<double>(s0 + r + 1, 2);
                const double wu = W1[c0];
                const double ck = __dadd_rn(wc, wu);  // w face sum of sw's upper face
                // sw: x (w advected by tcx (u(k) + u(k+1))), y, z (by w)
                rw = __dmul_rn(W[c0 - 1], fx2[fxw]);
                rw = __fma_rn(-W[c0 + 1], fx2[fxw + 1], rw);
                rw = __fma_rn(W[c0 - BX], fy2[fys], rw);
                rw = __fma_rn(-W[c0 + BX], fy2[fys + C::FYW], rw);
                if (kEq) {
                    zu = __fma_rn(-U1[c0], wxk, zu);
                    zv = __fma_rn(-V1[c0], wyk, zv);
                    const double zw = __fma_rn(-wu, ck, __dmul_rn(wo, c1));
                    rw = __fma_rn(__ldg(a.tzd1 + k), zw, rw);
                    w1x = wxk;
                    w1y = wyk;
                    c1 = ck;
                } else {
                    const double tz2 = __ldg(a.tzc2 + k), td2 = __ldg(a.tzd2 + k);
                    const double tn1 = __ldg(a.tzc1 + k + 1), dn1 = __ldg(a.tzd1 + k + 1);
                    ru = __fma_rn(-U1[c0], __dmul_rn(tz2, wxk), ru);
                    rv = __fma_rn(-V1[c0], __dmul_rn(tz2, wyk), rv);
                    rw = __fma_rn(wo, c1, rw);
                    rw = __fma_rn(-wu, __dmul_rn(td2, ck), rw);
                    w1x = __dmul_rn(tn1, wxk);
                    w1y = __dmul_rn(tn1, wyk);
                    c1 = __dmul_rn(dn1, ck);
                }
            }
            if (kEq) {
                const double ck1 = __ldg(a.tzc1 + k);
                ru = __fma_rn(ck1, zu, ru);
                rv = __fma_rn(ck1, zv, rv);
            }
            if (act) {
                su[g] = ru;
                sv[g] = rv;
                sw[g] = rw;
            }
            uo = uc;
            vo = vc;
            wo = wc;
            if (k + 1 < ke) {
                // next level's scaled velocities, then its faces
                if (k + 1 < nz - 1) {
                    bad |= !ring.wait(s0 + r + 2);
                    scale_level(ring, sm, s0 + r + 2, k + 2, xoff, tcx, tcy, tid);
                }
                abort = __syncthreads_or(bad);  // box r (level k) is free again
                if (!abort && tid == 0 && issued < nl) {
                    fence_proxy_async_smem();
                    ring.issue(s0 + issued, lo + issued, mu, mv, mw, x0, y0);
                    ++issued;
                }
                if (!abort) faces_level(sm, k + 1, tid);
                abort = __syncthreads_or(bad);
            }
        }
        if (k1 >= ke) {
            // nothing computed (only level 1 in this chunk): let the loads land
            if (tid == 0)
                for (int q = 0; q < issued; ++q) bad |= !ring.wait(s0 + q);
            abort = __syncthreads_or(bad);
        }
        if (abort) {
            if (tid == 0) {
                atomicOr(&tu_status, kStatusTimeout);
                for (int q = (issued > S ? issued - S : 0); q < issued; ++q) (void)ring.wait(s0 + q);
            }
            return false;
        }
        __syncthreads();  // every read of this tile's stages is done before the next tile's loads
        seq = s0 + nl;
        return true;
    }
};

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB) fwd_f64_kernel(const __grid_constant__ CUtensorMap mu,
                                                                 const __grid_constant__ CUtensorMap mv,
                                                                 const __grid_constant__ CUtensorMap mw,
                                                                 const FwdArgs a, const ItemSched sched) {
    using K = F64K<C>;
    extern __shared__ unsigned char smem_raw[];
    Ring<typename C::Shape> ring;
    typename K::Smem sm;
    K::setup(smem_raw, ring, sm);
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
    (void)K::tile(ring, sm, &mu, &mv, &mw, a, bx, by, a.kbeg + k0, a.kbeg + k1, seq, tid);
}

// Persistent form over a batch plan: work items (one tile column of one
// domain) come from the plan's counter, at most n_items iterations.
template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB) fwd_f64_batched(BatchPlan* plan, int variant) {
    using K = F64K<C>;
    extern __shared__ unsigned char smem_raw[];
    Ring<typename C::Shape> ring;
    typename K::Smem sm;
    K::setup(smem_raw, ring, sm);
    const int tid = threadIdx.x;
    if (plan->variant != variant || plan->dtype != PW_F64) {
        if (tid == 0) atomicOr(&tu_status, kStatusBadPlan);
        return;
    }
    if (tid == 0) ring.init_barriers();
    __syncthreads();
    const long long n_items = plan->n_items;
    long long seq = 0;
    for (long long it = 0; it < n_items; ++it) {
        if (tid == 0) *sm.item = (long long)atomicAdd(&plan->counter, 1ull);
        __syncthreads();
        const long long item = *sm.item;
        __syncthreads();  // every thread has read the slot before thread 0 rewrites it
        if (item >= n_items) break;
        const BatchDomain& d = plan->dom[find_domain(plan, item)];
        // private copy: the plan is global memory the compiler cannot prove
        // free of the output stores
        const FwdArgs args = d.args;
        const long long t = item - d.first_item;
        const int tiles_x = d.tiles_x, kchunks = d.kchunks;
        const long long tiles = (long long)tiles_x * d.tiles_y;
        const int ch = (int)(t / tiles), tt = (int)(t % tiles);
        const int kb = (int)((long long)args.nz * ch / kchunks);
        const int ke = (int)((long long)args.nz * (ch + 1) / kchunks);
        if (!K::tile(ring, sm, &d.mu, &d.mv, &d.mw, args, tt % tiles_x, tt / tiles_x, kb, ke, seq, tid)) break;
    }
}

template <class C>
TileShape f64_shape_of() {
    return TileShape{C::TX, C::TY, C::Shape::BX, C::Shape::BY, C::SMEM_BYTES, C::NT};
}

template <class C>
cudaError_t launch_one(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw, const FwdArgs& a,
                       cudaStream_t st) {
    auto kern = fwd_f64_kernel<C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    ItemSched sched;
    if ((e = choose_sched(kern, C::NT, C::SMEM_BYTES, (a.nx + C::TX - 1) / C::TX, (a.ny + C::TY - 1) / C::TY,
                          a.kend - a.kbeg, &sched)) != cudaSuccess)
        return e;
    kern<<<(unsigned)sched.items, C::NT, C::SMEM_BYTES, st>>>(mu, mv, mw, a, sched);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_batched_cfg(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    auto kern = fwd_f64_batched<C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    long long grid = 0;
    if ((e = persistent_grid(kern, C::NT, C::SMEM_BYTES, n_items, &grid)) != cudaSuccess) return e;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, C::NT, C::SMEM_BYTES, st>>>(plan, v);
    return cudaGetLastError();
}

}  // namespace

cudaError_t read_and_clear_status_f64(unsigned int* status, cudaStream_t st) {
    return read_and_clear_tu_status(status, st);
}

int f64_variant_count() { return 2; }

TileShape fwd_f64_shape_variant(int v) { return v == 1 ? f64_shape_of<FV1>() : f64_shape_of<FV0>(); }

// Tile of the one-shot launch (pw_advect): variant 0 (32 x 16) unless built otherwise.
#ifndef PW_F64_ONESHOT_VARIANT
#define PW_F64_ONESHOT_VARIANT 0
#endif

TileShape fwd_f64_shape() { return fwd_f64_shape_variant(PW_F64_ONESHOT_VARIANT); }

cudaError_t launch_fwd_f64(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw, const FwdArgs& a,
                           cudaStream_t st) {
    return PW_F64_ONESHOT_VARIANT == 1 ? launch_one<FV1>(mu, mv, mw, a, st) : launch_one<FV0>(mu, mv, mw, a, st);
}

cudaError_t launch_f64_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st) {
    return v == 1 ? launch_batched_cfg<FV1>(1, plan, n_items, st) : launch_batched_cfg<FV0>(0, plan, n_items, st);
}

}  // namespace pw
