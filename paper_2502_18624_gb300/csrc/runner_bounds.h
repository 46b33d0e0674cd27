// runner_bounds.h -- host-side bound on the runner's per-lattice tile
// counters (lat_multi.cu), kept in a header of its own so that it can be
// compiled and tested without a GPU.
//
// In one run, done[r] of a lattice starts at `base` and is incremented once
// per finished tile: it ends at base + 2 * nsweeps * ntiles (two colour
// phases per sweep), and phase k waits until done[r] >= base + k * ntiles.
// Every such value must fit the 64-bit counter and stay below the wait target
// of a stalled lattice (UINT64_MAX, never reached).
#pragma once
#include <cstdint>

namespace latk {

constexpr uint64_t kRunnerStallTarget = ~0ull;

// True iff base + 2 * nsweeps * ntiles < kRunnerStallTarget, evaluated
// without overflow.
inline bool runner_counts_fit(uint64_t base, uint64_t nsweeps, uint64_t ntiles)
{
    if (base >= kRunnerStallTarget) return false;
    if (nsweeps == 0 || ntiles == 0) return true;
    const uint64_t room = kRunnerStallTarget - 1 - base;  // largest admissible 2 * nsweeps * ntiles
    if (ntiles > room / 2) return false;
    return nsweeps <= room / (2 * ntiles);
}

}  // namespace latk
