// pw_strip_sched.h -- work schedule of the FP32 adjoint strip kernel
// (pw_adjoint.cu), as host/device functions so that a host test can check
// that it covers every (tile, level) exactly once.
#pragma once

#include <cuda_runtime.h>

namespace pw {

// ------------------------------------------------ strip adjoint schedule
// The work of a launch as (tile, level) units, tile-major (tile t's levels
// 0..nz-1 are units t*nz .. t*nz+nz-1), handed to CTAs in one of two ways:
//   chunks > 0: CTA b takes level chunk b / tiles of tile b % tiles (the
//     column cut into `chunks` equal chunks, every tile's first chunk first),
//     so the CTAs in flight read the same levels of neighbouring tiles and
//     share their halo rows in L2 -- for domains with at least as many tiles
//     as resident CTAs;
//   chunks == 0: CTA b takes the run of `len` units from b * len, the end of
//     one tile's column and the start of the next (or several whole
//     columns), so that one wave of resident CTAs does equal work however
//     few the tiles -- for small domains, where uniform chunks leave a
//     partial second wave.
struct StripSched {
    int tiles_x;      // tiles per row of the tile grid
    int chunks;       // level chunks per tile, or 0 for runs
    long long total;  // tiles * nz
    long long len;    // units per CTA (runs)
    long long grid;   // CTAs of the launch
};

// The schedule of `tiles` tiles of nz levels on `slots` resident CTA slots;
// `chunks` is the level-chunk count to use when the tiles fill the slots.
inline StripSched make_strip_sched(int tiles_x, long long tiles, int nz, long long slots, int chunks) {
    StripSched s;
    s.tiles_x = tiles_x;
    s.total = tiles * nz;
    if (tiles >= slots) {
        s.chunks = chunks < 1 ? 1 : chunks > nz ? nz : chunks;  // no empty chunk
        s.len = 0;
        s.grid = tiles * s.chunks;
    } else {
        s.chunks = 0;
        s.len = (s.total + slots - 1) / slots;
        s.grid = (s.total + s.len - 1) / s.len;
    }
    return s;
}

// Units [*u0, *u1) of CTA b.
__host__ __device__ __forceinline__ void strip_units(const StripSched& s, int nz, long long b, long long* u0,
                                                     long long* u1) {
    if (s.chunks > 0) {
        const long long tiles = s.total / nz;
        const long long c = b / tiles, t = b - c * tiles;
        *u0 = t * nz + (long long)nz * c / s.chunks;
        *u1 = t * nz + (long long)nz * (c + 1) / s.chunks;
    } else {
        *u0 = b * s.len;
        *u1 = *u0 + s.len < s.total ? *u0 + s.len : s.total;
    }
}

// The next segment of a CTA's units from `unit` (< u1): tile *t, levels
// [*kb, *ke); returns the unit after it.
__host__ __device__ __forceinline__ long long strip_segment(long long unit, long long u1, int nz, long long* t,
                                                            int* kb, int* ke) {
    *t = unit / nz;
    *kb = (int)(unit - *t * nz);
    *ke = (int)(u1 - *t * nz < nz ? u1 - *t * nz : nz);
    return *t * nz + *ke;
}

}  // namespace pw
