// Host check of the one-shot launch schedule (pw_internal.h): for many tile
// grids, level counts and slot counts, every (tile, level) of the launch is
// computed by exactly one work item, and every item has a valid tile and a
// non-empty level range. Prints "cases N bad M".
#include <cstdio>
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
    std::printf("cases %lld bad %lld\n", cases, bad);
    return bad != 0;
}
