// Reads runs from stdin and prints 1 or 0 per run: latk::runner_maps_ok, the
// host check of the runner's tile maps before every launch.  One run:
//   n K threads
//   n lines "items tile_items ntiles"
//   n + 1 values htp, K + 1 values hpb, K values hact
#include <cstdio>
#include <cstdint>
#include <vector>

#include "runner_bounds.h"

struct Desc {
    uint32_t items, tile_items, ntiles;
};

int main()
{
    unsigned n, K, threads;
    while (std::scanf("%u %u %u", &n, &K, &threads) == 3) {
        std::vector<Desc> d(n);
        for (auto& x : d)
            if (std::scanf("%u %u %u", &x.items, &x.tile_items, &x.ntiles) != 3) return 1;
        std::vector<uint32_t> htp(n + 1), hact(K);
        std::vector<unsigned long long> hpb(K + 1);
        for (auto& v : htp)
            if (std::scanf("%u", &v) != 1) return 1;
        for (auto& v : hpb)
            if (std::scanf("%llu", &v) != 1) return 1;
        for (auto& v : hact)
            if (std::scanf("%u", &v) != 1) return 1;
        std::printf("%d\n", latk::runner_maps_ok(d.data(), htp.data(), hpb.data(), hact.data(), n, K, threads) ? 1 : 0);
    }
    return 0;
}
