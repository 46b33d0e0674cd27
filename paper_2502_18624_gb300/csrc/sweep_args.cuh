// sweep_args.cuh -- the arguments of the colour-phase sweep kernels and the
// constants their code depends on (acceptance modes, observable record
// layout).  Kept apart from the other declarations so that the sweep kernels'
// sources are exactly k_sweep.cu, sweep_item.cuh, philox.cuh and this file.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"

namespace latk {

constexpr uint64_t kAlways = 1ull << 32;
constexpr uint32_t LAT_RNG_TABLE_MODE = 1;  // lat_params.rng value of the lookup-table mode

// Per-class acceptance mode of an integer threshold t in [0, 2^32]:
// t == 2^32 accepts without drawing, t == 0 rejects without drawing, any
// other value draws word 0 and accepts iff word 0 < t.  Skipping the draw
// does not change any result: the stream is counter-based.
enum ClassMode : uint32_t { kNever = 0, kAlwaysAccept = 1, kDraw = 2 };

inline uint32_t class_mode(uint64_t t)
{
    return t >= kAlways ? kAlwaysAccept : (t == 0 ? kNever : kDraw);
}

// Layout of the per-sweep observable record on the device (int64 each).
constexpr int kObsM = 0, kObsB = 1, kObsQ = 2, kObsDraws = 3, kObsWords = 4;

struct IsingPhaseArgs {
    uint64_t* spins;   // L rows of W words
    uint32_t L, W;
    uint32_t sweep, colour;
    uint32_t thr4, thr8;    // thresholds for s*h = 2 and s*h = 4
    uint32_t mode4, mode8;  // ClassMode of the two uphill classes
    long long* obs;         // colour-1 phase: record to accumulate (M, B, Q); else null
    long long* draws;       // counter of Philox draws to accumulate, or null
    long long* sd;          // 9 counters of the fused Schwinger-Dyson histogram of the active sites, or null
    uint32_t rng;           // LAT_RNG_SITE or LAT_RNG_TABLE
    uint32_t lut[16];       // LAT_RNG_TABLE lookup table
    RoundKeys rk;
};

struct BcPhaseArgs {
    ulonglong2* spins;  // L rows of W (n, g) word pairs
    uint32_t L, W;
    uint32_t sweep, colour;
    long long* obs;
    long long* draws;
    long long* sd;      // as in IsingPhaseArgs
    RoundKeys rk;
    unsigned long long thr[54];  // acceptance table (2^32 = always)
};

}  // namespace latk
