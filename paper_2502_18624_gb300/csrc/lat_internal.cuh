// lat_internal.cuh -- declarations shared by the kernel files and the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"
#include "sweep_args.cuh"

namespace latk {

struct LaunchShape {
    int sms;          // multiprocessors on the device
    int ising_bpsm;   // resident blocks per SM of the sweep kernels
    int bc_bpsm;
    int lut_bpsm;     // ... and of the lookup-table Ising kernel
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
// Adds (no clearing) the histogram of the sites of the colours in the mask
// `colours` (1: colour 0, 2: colour 1, 3: both) to hist9.
cudaError_t launch_sd_hist_add(int model, const void* spins, uint32_t L, uint32_t W, long long* hist9,
                               uint32_t colours, int sms, cudaStream_t st);
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
