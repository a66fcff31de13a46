// pw_ring.cuh -- the k-march tile pipeline shared by the forward kernels.
//
// A CTA owns a TX x TY tile of interior columns and walks it up the column
// (k = 0..nz-1). Each level of u, v, w for the tile plus its one-cell halo
// is one TMA box (BX x BY x 1) landing in a ring of S shared-memory stages;
// one elected thread keeps the ring full S-1 levels ahead, so each input
// element crosses HBM once (halo re-reads of neighbouring tiles hit L2).
// Level k's stage is released after the level-k step, because every value
// a later level needs from level k (own-column values, face sums of w) is
// carried in registers.
#pragma once

#include "pw_common.cuh"

namespace pw {

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

template <typename T, int TX_, int TY_, int S_>
struct RingShape {
    static constexpr int TX = TX_, TY = TY_, S = S_;
    static constexpr int NT = TX * TY;
    // Element offset of the halo column i = 0 from the 16-byte boundary the
    // TMA descriptor starts at: 0 .. XOFF_MAX (the caller's base pointer
    // need only be element-aligned). The box covers the tile, its halo and
    // that offset, and its inner extent is a whole number of 16-byte units.
    static constexpr int XOFF_MAX = 16 / (int)sizeof(T) - 1;
    static constexpr int BX = round_up(TX + 2 + XOFF_MAX, 16 / (int)sizeof(T));
    static constexpr int BY = TY + 2;
    static constexpr int BOX_BYTES = BX * BY * (int)sizeof(T);
    static constexpr int BOX_STRIDE = round_up(BOX_BYTES, 128);
    static constexpr int STAGE_BYTES = 3 * BOX_STRIDE;
    static constexpr int SMEM_BYTES = S * STAGE_BYTES + S * 8 + 128;  // + barriers + alignment slack
    static_assert(BX <= 256 && BY <= 256, "TMA box dimension limit");
    static_assert((TX * (int)sizeof(T)) % 16 == 0, "tile x origin must stay 16-byte aligned");
};

// Shared-memory ring addressed by load number: the CTA numbers its level
// loads 0, 1, 2, ... across every tile it processes; load `seq` lives in
// stage seq % S and completes barrier phase seq / S, so the parity to wait
// for is (seq / S) & 1. A one-shot kernel simply starts at seq = 0.
template <typename Shape>
struct Ring {
    unsigned char* base;  // 128-byte aligned
    uint64_t* full;       // S barriers

    // `raw` must be the kernel's extern __shared__ array: the base is found by
    // pointer arithmetic on it (not through an integer), so the compiler keeps
    // every derived access in the shared address space (LDS, not generic LD).
    __device__ __forceinline__ void setup(unsigned char* raw) {
        base = raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
        full = reinterpret_cast<uint64_t*>(base + Shape::S * Shape::STAGE_BYTES);
    }
    template <typename T>
    __device__ __forceinline__ const T* box(long long seq, int field) const {
        return reinterpret_cast<const T*>(base + (int)(seq % Shape::S) * Shape::STAGE_BYTES +
                                          field * Shape::BOX_STRIDE);
    }
    __device__ __forceinline__ void init_barriers() {
        for (int s = 0; s < Shape::S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    // Issue the three box loads of level `lev` as load number `seq` (one thread).
    __device__ __forceinline__ void issue(long long seq, int lev, const CUtensorMap* mu, const CUtensorMap* mv,
                                          const CUtensorMap* mw, int x0, int y0) {
        const int s = (int)(seq % Shape::S);
        uint64_t* bar = &full[s];
        unsigned char* dst = base + s * Shape::STAGE_BYTES;
        mbar_arrive_expect_tx(bar, 3 * Shape::BOX_BYTES);
        tma_load_3d(dst, mu, bar, x0, y0, lev);
        tma_load_3d(dst + Shape::BOX_STRIDE, mv, bar, x0, y0, lev);
        tma_load_3d(dst + 2 * Shape::BOX_STRIDE, mw, bar, x0, y0, lev);
    }
    __device__ __forceinline__ bool wait(long long seq) {
        return mbar_wait_bounded(&full[(int)(seq % Shape::S)], (uint32_t)((seq / Shape::S) & 1));
    }
};

}  // namespace pw
