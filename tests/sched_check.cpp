// Host check of the one-shot launch schedule (pw_internal.h): for many tile
// grids, level counts and slot counts, every (tile, level) of the launch is
// computed by exactly one work item, and every item has a valid tile and a
// non-empty level range; and the grouped greedy model (greedy_makespan)
// equals a direct simulation that places items one at a time on a priority
// queue of slot loads. Prints "cases N bad M".
#include <cmath>
#include <cstdio>
#include <functional>
#include <queue>
#include <vector>

#include "pw_internal.h"

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
    std::printf("cases %lld bad %lld\n", cases, bad);
    return bad != 0;
}
