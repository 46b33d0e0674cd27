// Reads lines "base nsweeps ntiles" (decimal) from stdin and prints 1 or 0
// per line: latk::runner_counts_fit(base, nsweeps, ntiles), the host bound
// the runner applies to its 64-bit tile counters before every launch.
#include <cstdio>
#include <cstdint>

#include "runner_bounds.h"

int main()
{
    unsigned long long base, ns, nt;
    while (std::scanf("%llu %llu %llu", &base, &ns, &nt) == 3)
        std::printf("%d\n", latk::runner_counts_fit(base, ns, nt) ? 1 : 0);
    return 0;
}
