// k_sweep.cu -- one checkerboard colour phase of a Metropolis sweep on one
// lattice (section 3.1: spins of one colour are updated in parallel, two
// phases per step), for the Ising model (1 bit per spin, section 3.2) and
// the Blume-Capel model (2 bits per spin in two bit planes).
//
// The per-item update lives in sweep_item.cuh (shared with the persistent
// multi-lattice kernel).  Here a grid of SMs x resident blocks walks the
// items of the phase with a grid stride; every grid-stride iteration keeps
// whole warps either active or inactive, because the item count
// (L * W / CW, or L * W) is a multiple of 32.  The fused E/M/Q reduction
// (colour-1 phase) and the draw count are reduced per warp and added with
// one atomic per warp.
#include "lat_internal.cuh"
#include "sweep_item.cuh"

namespace latk {
namespace {

constexpr int kSweepThreads = 256;

template <int CW, bool OBS, bool SD = false>
__global__ void __launch_bounds__(kSweepThreads, 3) k_ising_phase(const __grid_constant__ IsingPhaseArgs a)
{
    const IsingPhase ph{a.spins, a.L, a.W, a.sweep, a.colour, a.thr4, a.thr8, a.mode4, a.mode8};
    const uint64_t nitems = (uint64_t)a.L * (a.W / CW);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    PhaseAcc acc;
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nitems; item += stride)
        ising_item<CW, OBS, false, SD>(ph, a.rk, item, lane, acc);
    flush_acc(OBS ? a.obs : nullptr, a.draws, acc);
    if constexpr (SD) flush_sd(a.sd, acc);
}

template <int CW, bool OBS, bool SD = false>
__global__ void __launch_bounds__(kSweepThreads, 3) k_ising_phase_lut(const __grid_constant__ IsingPhaseArgs a)
{
    __shared__ uint32_t s_lut[kLutSlots];
    __shared__ uint8_t s_lutb[kLutBuckets];
    if (threadIdx.x < kLutSlots) s_lut[threadIdx.x] = lut_slot(a.lut, threadIdx.x);
    __syncthreads();
    lut_buckets(s_lut, s_lutb);
    __syncthreads();
    const IsingPhase ph{a.spins, a.L, a.W, a.sweep, a.colour, a.thr4, a.thr8, a.mode4, a.mode8};
    const uint64_t nitems = (uint64_t)a.L * (a.W / CW);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    PhaseAcc acc;
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nitems; item += stride)
        ising_item_lut<CW, OBS, false, SD, true>(ph, a.rk, s_lut, s_lutb, item, lane, acc);
    flush_acc(OBS ? a.obs : nullptr, a.draws, acc);
    if constexpr (SD) flush_sd(a.sd, acc);
}

template <bool OBS, bool SD = false>
__global__ void __launch_bounds__(kSweepThreads, 3) k_bc_phase(const __grid_constant__ BcPhaseArgs a)
{
    __shared__ uint2 s_thr[kBcTable];
    bc_table128(a.thr, s_thr);
    __syncthreads();
    const BcPhase ph{a.spins, a.L, a.W, a.sweep, a.colour};
    const uint64_t nitems = (uint64_t)a.L * a.W;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    PhaseAcc acc;
    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nitems; item += stride)
        bc_item<OBS, false, SD>(ph, a.rk, s_thr, item, lane, acc);
    flush_acc(OBS ? a.obs : nullptr, a.draws, acc);
    if constexpr (SD) flush_sd(a.sd, acc);
}

int blocks_for(uint64_t nitems, int sms, int bpsm)
{
    const uint64_t need = (nitems + kSweepThreads - 1) / kSweepThreads;
    const uint64_t cap = (uint64_t)sms * (uint64_t)bpsm;
    return (int)(need < cap ? need : cap);
}

}  // namespace

cudaError_t query_sweep_occupancy(LaunchShape& ls)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&ls.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ls.ising_bpsm, k_ising_phase<2, true>, kSweepThreads, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ls.bc_bpsm, k_bc_phase<true>, kSweepThreads, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ls.lut_bpsm, k_ising_phase_lut<2, true>, kSweepThreads, 0);
    if (ls.ising_bpsm < 1) ls.ising_bpsm = 1;
    if (ls.bc_bpsm < 1) ls.bc_bpsm = 1;
    if (ls.lut_bpsm < 1) ls.lut_bpsm = 1;
    return e;
}

// The kernel instance for (words per item, fused observables, fused
// Schwinger-Dyson histogram).
template <int CW>
cudaError_t ising_launch(const IsingPhaseArgs& a, int grid, cudaStream_t st)
{
    const bool obs = a.obs != nullptr, sd = a.sd != nullptr;
    if (a.rng == LAT_RNG_TABLE_MODE) {
        if (sd) {
            if (obs) k_ising_phase_lut<CW, true, true><<<grid, kSweepThreads, 0, st>>>(a);
            else k_ising_phase_lut<CW, false, true><<<grid, kSweepThreads, 0, st>>>(a);
        } else {
            if (obs) k_ising_phase_lut<CW, true><<<grid, kSweepThreads, 0, st>>>(a);
            else k_ising_phase_lut<CW, false><<<grid, kSweepThreads, 0, st>>>(a);
        }
    } else if (sd) {
        if (obs) k_ising_phase<CW, true, true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_ising_phase<CW, false, true><<<grid, kSweepThreads, 0, st>>>(a);
    } else {
        if (obs) k_ising_phase<CW, true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_ising_phase<CW, false><<<grid, kSweepThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_ising_phase(const IsingPhaseArgs& a, const LaunchShape& ls, cudaStream_t st)
{
    const bool even_words = (a.W % 2) == 0;
    const uint64_t nitems = (uint64_t)a.L * (even_words ? a.W / 2 : a.W);
    const int grid = blocks_for(nitems, ls.sms, a.rng == LAT_RNG_TABLE_MODE ? ls.lut_bpsm : ls.ising_bpsm);
    return even_words ? ising_launch<2>(a, grid, st) : ising_launch<1>(a, grid, st);
}

cudaError_t launch_bc_phase(const BcPhaseArgs& a, const LaunchShape& ls, cudaStream_t st)
{
    const uint64_t nitems = (uint64_t)a.L * a.W;
    const int grid = blocks_for(nitems, ls.sms, ls.bc_bpsm);
    if (a.sd) {
        if (a.obs) k_bc_phase<true, true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_bc_phase<false, true><<<grid, kSweepThreads, 0, st>>>(a);
    } else {
        if (a.obs) k_bc_phase<true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_bc_phase<false><<<grid, kSweepThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace latk
