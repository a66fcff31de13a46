// pw_internal.h -- launchers shared between the C ABI (pw_api.cu) and the
// kernel translation units. Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <map>
#include <mutex>
#include <tuple>

namespace pw {

struct FwdArgs {
    int nx, ny, nz;
    int kbeg, kend;            // levels kbeg..kend-1 are computed (0 <= kbeg < kend <= nz)
    long long sy, sz;          // element strides of every field
    int xoff;                  // elements from the descriptors' 16-byte base to i = 0
    int vec;                   // 1: every field's interior i = 1 starts on 16 bytes
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
    const float* split;        // PW_F32_SPLIT table, else nullptr
    void *su, *sv, *sw;
};

// Tile shape of each forward kernel (the host builds TMA boxes to match).
struct TileShape {
    int tx, ty;       // interior columns per CTA
    int box_x, box_y; // TMA box (tile + halo, x rounded to 16 bytes)
    int smem_bytes;   // dynamic shared memory per CTA
    int threads;
};

TileShape fwd_f64_shape();
TileShape fwd_paired_shape();
TileShape fwd_split_shape();

// ---------------------------------------------------------------- batches
// One domain of a batch: its three TMA descriptors (in device memory, so the
// persistent kernel can switch domains per work item), its launch arguments,
// its tile grid and the index of its first work item.
struct BatchDomain {
    CUtensorMap mu, mv, mw;
    FwdArgs args;
    int tiles_x, tiles_y;
    int kchunks;      // items per tile: the column is cut into kchunks level ranges
    int reserved;
    long long first_item;
};

// A batch plan as laid out in device memory: header, then n_domains entries.
// `counter` is the persistent kernel's work queue (scratch: reset to 0 before
// every launch).
struct BatchPlan {
    unsigned long long counter;
    long long n_items;
    int n_domains;
    int dtype;
    int variant;
    int all_vec;  // every domain takes the 16-byte vector path
    BatchDomain dom[1];
};

inline size_t batch_plan_bytes(int n) {
    return offsetof(BatchPlan, dom) + (size_t)(n > 0 ? n : 1) * sizeof(BatchDomain);
}

// Domain holding work item `item` (domains are stored in item order).
__device__ __forceinline__ int find_domain(const BatchPlan* plan, long long item) {
    int lo = 0, hi = plan->n_domains - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (plan->dom[mid].first_item <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Grid of a persistent kernel: resident CTAs on every SM, at most n_items.
template <typename Kern>
cudaError_t persistent_grid(Kern kern, int threads, int smem, long long n_items, long long* grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
    long long g = (long long)sms * (per_sm > 0 ? per_sm : 1);
    *grid = g < n_items ? g : n_items;
    return cudaSuccess;
}

// Level chunks per tile column so that tiles * chunks work units fill the
// GPU's resident CTA slots in nearly whole waves. Each chunk re-reads one
// level below and one above, so chunks stay at least 8 levels tall -- unless
// the domain has so few tiles that even 8 chunks each leave most slots idle
// (a small domain): then up to 64 chunks of at least 2 levels, since a
// CTA's time is mostly the latency of its serial level march.
inline int pick_kchunks(long long tiles, int nz, long long slots) {
    const bool small = tiles * 8 < slots;
    const int max_chunks = small ? 64 : 8, min_levels = small ? 2 : 8;
    int best = 1;
    double best_cost = 1e300;
    for (int c = 1; c <= max_chunks; ++c) {
        if (c > 1 && nz / c < min_levels) break;
        const double units = (double)tiles * c;
        const double waves = units / (double)slots;
        const double used = waves / (double)((long long)(waves + 0.999999));  // fraction of the last-wave-rounded time
        const double extra = (double)(nz + 2 * (c - 1)) / (double)nz;       // re-read and re-split levels
        const double cost = extra / used;
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

template <typename Kern>
cudaError_t choose_kchunks(Kern kern, int threads, int smem, long long tiles, int nz, int* chunks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
    *chunks = pick_kchunks(tiles, nz, (long long)sms * (per_sm > 0 ? per_sm : 1));
    return cudaSuccess;
}

// ------------------------------------------------------- one-shot schedule
// Work items of a one-shot forward launch (a 1-D grid, one CTA per item). A
// tile column is one tile of the x-y grid over the computed levels
// kbeg..kend-1. Tiles [0, ta) are cut into ca level chunks and come first;
// tiles [ta, tiles) are cut into cb chunks. Chunks re-read one level below
// and one above, so whole columns are cheapest; chunks make enough small
// items for the last wave of CTAs. The block scheduler starts CTAs in
// index order, so the short items of the second group fill the tail.
// Within a group items run chunk by chunk (every tile's first chunk, then
// every tile's second, ...), so CTAs in flight together read the same
// levels of neighbouring tiles.
struct ItemSched {
    int tiles_x;         // tiles per row of the tile grid
    int ta, ca, cb;      // tiles of the first group; chunks per tile in each group
    long long items_a;   // ta * ca
    long long items;     // all items (grid size)
};

// Tile and relative level range [k0, k1) (0 <= k0 < k1 <= nlev) of item b.
__host__ __device__ __forceinline__ void sched_item(const ItemSched& s, int nlev, long long b, int* bx, int* by,
                                                    int* k0, int* k1) {
    long long t;
    int ch, c;
    if (b < s.items_a) {
        ch = (int)(b / s.ta);
        t = b - (long long)ch * s.ta;
        c = s.ca;
    } else {
        const long long r = b - s.items_a;
        const long long nb = (s.items - s.items_a) / s.cb;  // tiles of the second group (>= 1 here)
        ch = (int)(r / nb);
        t = s.ta + (r - (long long)ch * nb);
        c = s.cb;
    }
    *bx = (int)(t % s.tiles_x);
    *by = (int)(t / s.tiles_x);
    *k0 = (int)((long long)nlev * ch / c);
    *k1 = (int)((long long)nlev * (ch + 1) / c);
}

// Makespan of greedy list scheduling (each item to the least-loaded slot, in
// order) of na items of length la, then nb items of length lb, on `slots`
// equal slots. Slots with equal loads are kept as one entry with a count.
inline double greedy_makespan(long long na, double la, long long nb, double lb, long long slots) {
    std::map<double, long long> load;
    load[0.0] = slots;
    auto place = [&load](long long n, double len) {
        while (n > 0) {
            auto it = load.begin();
            const double l = it->first;
            const long long k = it->second < n ? it->second : n;
            if (k == it->second) load.erase(it);
            else it->second -= k;
            load[l + len] += k;
            n -= k;
        }
    };
    place(na, la);
    place(nb, lb);
    return load.rbegin()->first;
}

// Items of one launch: a uniform cut (every tile in c chunks, as
// pick_kchunks allows) or whole waves of tiles in ca = 1 or 2 chunks followed
// by the remaining tiles in finer chunks (at least 4 levels each), whichever
// the greedy model finishes first. An item of L levels costs L + kItemCost
// level-times (its two re-read levels and its pipeline start); 1, 2 and 4
// were measured, and 1 was fastest by about 0.5 % on every kernel.
inline ItemSched pick_sched(long long tiles, int tiles_x, int nlev, long long slots) {
#ifndef PW_ITEM_COST
#define PW_ITEM_COST 1.0
#endif
    constexpr double kItemCost = PW_ITEM_COST;
    const bool small = tiles * 8 < slots;
    const int max_chunks = small ? 64 : 8, min_levels = small ? 2 : 8;
    ItemSched best{tiles_x, (int)tiles, 1, 1, tiles, tiles};
    double best_t = greedy_makespan(tiles, nlev + kItemCost, 0, 0.0, slots);
    for (int c = 2; c <= max_chunks && nlev / c >= min_levels; ++c) {
        const double t = greedy_makespan(tiles * c, (double)nlev / c + kItemCost, 0, 0.0, slots);
        if (t < best_t - 1e-9) {
            best_t = t;
            best = ItemSched{tiles_x, (int)tiles, c, 1, tiles * c, tiles * c};
        }
    }
    if (!small) {
        for (int ca = 1; ca <= 2 && (ca == 1 || nlev / ca >= min_levels); ++ca) {
            const long long waves = tiles * ca / slots;
            if (waves < 1) continue;
            const long long ta = waves * slots / ca;
            if (ta >= tiles) continue;
            for (int cb = ca + 1; cb <= 64 && nlev / cb >= 4; ++cb) {
                const double t = greedy_makespan(ta * ca, (double)nlev / ca + kItemCost, (tiles - ta) * cb,
                                                 (double)nlev / cb + kItemCost, slots);
                if (t < best_t - 1e-9) {
                    best_t = t;
                    best = ItemSched{tiles_x, (int)ta, ca, cb, ta * ca, ta * ca + (tiles - ta) * cb};
                }
            }
        }
    }
    return best;
}

// The schedule of a one-shot launch of `kern`, cached per shape (the search
// runs once per tile count, level count and occupancy).
template <typename Kern>
cudaError_t choose_sched(Kern kern, int threads, int smem, int tiles_x, int tiles_y, int nlev, ItemSched* out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, long long>, ItemSched> cache;
    const auto key = std::make_tuple(tiles_x, tiles_y, nlev, slots);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        if (cache.size() > 4096) cache.clear();
        it = cache.emplace(key, pick_sched((long long)tiles_x * tiles_y, tiles_x, nlev, slots)).first;
    }
    *out = it->second;
    return cudaSuccess;
}

int f64_variant_count();
TileShape fwd_f64_shape_variant(int v);
cudaError_t launch_f64_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st);
int split_variant_count();
TileShape fwd_split_shape_variant(int v);
cudaError_t launch_fwd_split_variant(int v, const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                                     const FwdArgs& a, cudaStream_t st);
cudaError_t launch_split_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st);
int paired_variant_count();
TileShape fwd_paired_shape_variant(int v);
cudaError_t launch_paired_batched(int v, BatchPlan* plan, long long n_items, cudaStream_t st);

cudaError_t launch_fwd_f64(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                           const FwdArgs& a, cudaStream_t st);
cudaError_t launch_fwd_paired(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                              const FwdArgs& a, cudaStream_t st);
cudaError_t launch_fwd_split(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                             const FwdArgs& a, cudaStream_t st);

struct AdjArgs {
    int nx, ny, nz;
    long long sy, sz;
    int xoff;                  // elements from the descriptors' 16-byte base to i = 0
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
    const void *u, *v, *w;        // the fields and cotangents, for kernels that read them
    const void *gsu, *gsv, *gsw;  // with plain loads (the FP64 halo cells)
    void *gu, *gv, *gw;
    int accumulate;
    int vec;                   // gu, gv, gw have u's address modulo 16 bytes (16-byte stores of strips)
};

// PW_F32 (elem_bytes 4, strips) and PW_F64_PAIRED (elem_bytes 8)
TileShape adjoint_shape(int elem_bytes);
// maps6: u, v, w, gsu, gsv, gsw; PW_F32
cudaError_t launch_adjoint(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st);
// PW_F64: the face-form kernel and its halo-cell kernel
TileShape adjoint_f64_shape();
cudaError_t launch_adjoint_f64(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st);
// PW_F64_PAIRED: double fields, the box of adjoint_shape(8)
cudaError_t launch_adjoint_paired(const CUtensorMap* maps6, const AdjArgs& a, cudaStream_t st);
cudaError_t launch_fold_halo(void* field, int elem_bytes, int nx, int ny, int nz, long long sy, long long sz,
                             cudaStream_t st);

cudaError_t launch_fill_halo(void* field, int elem_bytes, int nx, int ny, int nz, long long sy, long long sz,
                             cudaStream_t st);

cudaError_t launch_split_field(const double* f, long long fsy, long long fsz, float* fp, long long psy,
                               long long psz, int nx, int ny, int nz, double* mean, cudaStream_t st);

cudaError_t launch_selftest_wait(unsigned long long limit_ns, cudaStream_t st);

cudaError_t launch_energy_budget(const void* u, const void* v, const void* w, int wind_bytes, long long wsy,
                                 long long wsz, const void* su, const void* sv, const void* sw, int tend_bytes,
                                 long long ssy, long long ssz, int nx, int ny, int nz, const double* wu,
                                 const double* ww, double* level_sums, double* totals, cudaStream_t st);

// Read and clear the device status words of every kernel unit (synchronises st).
cudaError_t read_and_clear_status(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_paired(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_split(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_adjoint(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_f64(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_adjoint_f64(unsigned int* status, cudaStream_t st);

}  // namespace pw
