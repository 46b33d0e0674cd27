// lat_internal.cuh -- declarations shared by the kernel files and the C ABI.
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
    RoundKeys rk;
    unsigned long long thr[54];  // acceptance table (2^32 = always)
};

struct LaunchShape {
    int sms;          // multiprocessors on the device
    int ising_bpsm;   // resident blocks per SM of the sweep kernels
    int bc_bpsm;
};

// Sweep phases (k_sweep.cu).
cudaError_t launch_ising_phase(const IsingPhaseArgs& a, const LaunchShape& ls, cudaStream_t st);
cudaError_t launch_bc_phase(const BcPhaseArgs& a, const LaunchShape& ls, cudaStream_t st);
cudaError_t query_sweep_occupancy(LaunchShape& ls);

// Initial quench and lattice utilities (k_lattice.cu).
cudaError_t launch_init(int model, void* spins, uint32_t L, uint32_t W, const RoundKeys& rk, int sms,
                        cudaStream_t st);
cudaError_t launch_measure(int model, const void* spins, uint32_t L, uint32_t W, long long* out3, int sms,
                           cudaStream_t st);
cudaError_t launch_spin_counts(int model, const void* spins, uint32_t L, uint32_t W, long long* out4, int sms,
                               cudaStream_t st);
cudaError_t launch_sd_hist(int model, const void* spins, uint32_t L, uint32_t W, long long* hist9, int sms,
                           cudaStream_t st);
cudaError_t launch_hash(int model, const void* spins, uint32_t L, uint32_t W, unsigned long long* out, int sms,
                        cudaStream_t st);
cudaError_t launch_unpack_rows(int model, const void* spins, uint32_t L, uint32_t W, uint32_t y0,
                               uint32_t nrows, int8_t* out, cudaStream_t st);
cudaError_t launch_pack_rows(int model, void* spins, uint32_t L, uint32_t W, uint32_t y0, uint32_t nrows,
                             const int8_t* in, unsigned int* bad, cudaStream_t st);

// Correlation (k_corr.cu).
cudaError_t launch_correlation(int model, const void* spins, uint32_t L, uint32_t W, uint32_t rmax,
                               long long* cx, long long* cy, cudaStream_t st);
// Correlation from downsampled sources (k_corr_ds.cu): one source per R x R
// square, for a list of nr distances.  R >= kDsMinScratchR uses the compact
// source-column copy in escratch (ds_scratch_words(model, L) words).
constexpr uint32_t kDsChunk = 2048;       // distances per launch
constexpr uint32_t kDsMinScratchR = 16;
size_t ds_scratch_words(int model, uint32_t L);
cudaError_t launch_correlation_sampled(int model, const void* spins, uint32_t L, uint32_t W, uint32_t R,
                                       const uint32_t* rlist, uint32_t nr, long long* cx, long long* cy,
                                       uint64_t* escratch, int sms, cudaStream_t st);

}  // namespace latk
