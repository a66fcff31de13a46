// Host check of the launch schedules (pw_internal.h, pw_strip_sched.h): for many tile grids,
// level counts and slot counts, every (tile, level) of a one-shot launch is
// computed by exactly one work item, and every item has a valid tile and a
// non-empty level range; the grouped greedy model (greedy_makespan) equals a
// direct simulation that places items one at a time on a priority queue of
// slot loads; and the strip adjoint's schedule (equal runs of tile levels,
// or chunk-major level chunks) covers every (tile, level) exactly once with
// non-empty segments, runs taking one wave (at most `slots` CTAs, each at
// most ceil(units / slots) units). Prints "cases N bad M".
#include <cmath>
#include <cstdio>
#include <functional>
#include <queue>
#include <vector>

#include "pw_internal.h"
#include "pw_strip_sched.h"

int main() {
    long long bad = 0, cases = 0;
    for (int tx : {1, 2, 3, 5, 8, 16, 32})
        for (int ty : {1, 2, 7, 33, 64, 128, 256})
            for (int nlev : {1, 2, 3, 5, 8, 16, 37, 64, 128, 300})
                for (long long slots : {152LL, 608LL, 760LL, 1520LL}) {
                    const pw::ItemSched s = pw::pick_sched((long long)tx * ty, tx, nlev, slots);
                    std::vector<int> cover((size_t)tx * ty * nlev, 0);
                    for (long long b = 0; b < s.items; ++b) {
                        int bx, by, k0, k1;
                        pw::sched_item(s, nlev, b, &bx, &by, &k0, &k1);
                        if (bx < 0 || bx >= tx || by < 0 || by >= ty || k0 < 0 || k1 > nlev || k0 >= k1) {
                            ++bad;
                            continue;
                        }
                        for (int k = k0; k < k1; ++k) cover[((size_t)by * tx + bx) * nlev + k]++;
                    }
                    for (int c : cover)
                        if (c != 1) ++bad;
                    ++cases;
                }
    // the grouped model against item-by-item list scheduling
    unsigned long long x = 88172645463325252ull;
    auto rnd = [&x](long long n) { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return (long long)(x % (unsigned long long)n); };
    for (int t = 0; t < 400; ++t) {
        const long long slots = 1 + rnd(200), na = rnd(2000), nb = rnd(2000);
        const double la = 1.0 + (double)rnd(64) / 4.0, lb = 1.0 + (double)rnd(64) / 4.0;
        std::priority_queue<double, std::vector<double>, std::greater<double>> q;
        for (long long i = 0; i < slots; ++i) q.push(0.0);
        double top = 0.0;
        for (long long i = 0; i < na + nb; ++i) {
            const double l = q.top() + (i < na ? la : lb);
            q.pop();
            q.push(l);
            top = l > top ? l : top;
        }
        if (std::fabs(pw::greedy_makespan(na, la, nb, lb, slots) - top) > 1e-9) ++bad;
        ++cases;
    }
    // the strip adjoint's schedule
    for (int tx : {1, 2, 9, 17, 33})
        for (int ty : {1, 3, 17, 65})
            for (int nz : {1, 2, 5, 37, 64, 128})
                for (long long slots : {1LL, 7LL, 456LL, 912LL})
                    for (int chunks : {1, 3, 5}) {
                        const long long tiles = (long long)tx * ty;
                        const pw::StripSched s = pw::make_strip_sched(tx, tiles, nz, slots, chunks);
                        std::vector<int> cover((size_t)tiles * nz, 0);
                        if (s.chunks == 0 && (s.grid > slots || s.len > (s.total + slots - 1) / slots)) ++bad;
                        for (long long b = 0; b < s.grid; ++b) {
                            long long u, u1;
                            pw::strip_units(s, nz, b, &u, &u1);
                            if (u >= u1) ++bad;  // every CTA has work
                            while (u < u1) {
                                long long t;
                                int kb, ke;
                                const long long next = pw::strip_segment(u, u1, nz, &t, &kb, &ke);
                                if (t < 0 || t >= tiles || kb < 0 || ke > nz || kb >= ke || next <= u) {
                                    ++bad;
                                    break;
                                }
                                for (int k = kb; k < ke; ++k) cover[(size_t)t * nz + k]++;
                                u = next;
                            }
                        }
                        for (int c : cover)
                            if (c != 1) ++bad;
                        ++cases;
                    }
    std::printf("cases %lld bad %lld\n", cases, bad);
    return bad != 0;
}
