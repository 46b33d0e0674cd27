// runner_bounds.h -- host-side checks of the runner's launch data
// (lat_multi.cu), kept in a header of their own so that they can be
// compiled and tested without a GPU: the bound on the per-lattice tile
// counters, and the consistency of the tile maps the kernel indexes.
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

// The tile maps of one run, checked before it is launched (the persistent
// kernel indexes them without checks of its own).  n lattices, ordered by
// descending sweep count, each with `items` work items per colour phase cut
// into `ntiles` tiles of `tile_items` items (a multiple of the block size
// `threads`); K phases.
//   htp[s]  tiles of lattices 0..s-1 (htp[0] = 0, htp[s+1] = htp[s] + ntiles)
//   hact[k] lattices active in phase k (a non-increasing prefix count, >= 1)
//   hpb[k]  tiles of phases 0..k-1 (hpb[0] = 0, hpb[k+1] = hpb[k] + htp[hact[k]])
// Then a tile number below hpb[K] maps to one phase k, one lattice r <
// hact[k] and one tile t < ntiles[r], and every tile covers items inside its
// lattice: tiles cover the items, and the last tile is not empty.
template <typename Desc>
inline bool runner_maps_ok(const Desc* hd, const uint32_t* htp, const unsigned long long* hpb,
                           const uint32_t* hact, uint32_t n, uint32_t K, uint32_t threads)
{
    if (htp[0] != 0) return false;
    for (uint32_t s = 0; s < n; ++s) {
        const Desc& d = hd[s];
        if (d.tile_items == 0 || d.tile_items % threads != 0 || d.ntiles == 0) return false;
        if ((uint64_t)d.ntiles * d.tile_items < d.items || (uint64_t)(d.ntiles - 1) * d.tile_items >= d.items)
            return false;
        if ((uint64_t)htp[s + 1] != (uint64_t)htp[s] + d.ntiles) return false;
    }
    if (hpb[0] != 0) return false;
    for (uint32_t k = 0; k < K; ++k) {
        if (hact[k] == 0 || hact[k] > n || (k > 0 && hact[k] > hact[k - 1])) return false;
        if (hpb[k + 1] != hpb[k] + htp[hact[k]]) return false;
    }
    return true;
}

}  // namespace latk
