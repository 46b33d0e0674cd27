// lat_multi.cu -- many independent lattices advanced together in one
// persistent launch (the "runner" of include/lat.h).
//
// Work decomposition.  Every colour phase k of every lattice r is split into
// tiles of `tile_items` items (sweep_item.cuh).  Tiles are numbered
// phase-major: all tiles of phase 0 of every lattice, then phase 1, ...;
// within a phase, lattices in descending order of their sweep counts, so the
// lattices still active at phase k are a prefix of that order.  A global
// atomic counter hands tiles out in this order.  Before a block works on a
// tile of (r, k > 0) it waits until every tile of (r, k-1) is done, counted
// by done[r]; after the tile it publishes its stores (fence) and increments
// done[r].  done[r] is a 64-bit count that starts at a per-run base (0 unless
// a test sets it): it reaches base + 2 * nsweeps * ntiles, which a 32-bit
// count would not hold for large lattices with small tiles, and the host
// checks that it fits before launching (runner_bounds.h).
//
// Progress.  A block waits only for tiles with smaller numbers, which were
// taken by blocks that were already running, and those wait only for tiles
// with still smaller numbers, so every wait ends without any co-residency
// guarantee.  Each wait is still bounded by a %globaltimer limit; a block
// that gives up records the failure in the control word and every block
// then leaves at its next tile, and the host returns LAT_ETIMEDOUT.
//
// Coherence.  One launch runs many phases, so a block may read a row that
// it cached in L1 during an earlier phase; all lattice loads therefore go
// through L2 (ld.global.cg), which is coherent across the GPU.
//
// Results.  Tiles of one lattice run exactly the per-item code of the
// one-lattice kernels with the same counters (site, sweep index, colour), so
// every lattice ends bit-identical to its one-lattice run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

#include "lat_handle.h"
#include "runner_bounds.h"
#include "sweep_item.cuh"

using namespace latk;

namespace {

constexpr int kMultiThreads = 256;
constexpr uint32_t kDefaultTile = 4096;  // items per tile when no schedule entry applies
constexpr uint32_t kTilesPerBlock = 4;   // a phase with few lattices left still has this many tiles per block

uint32_t items_of(const lat* h)
{
    const uint32_t cw = (h->p.model == LAT_ISING && h->W % 2 == 0) ? 2 : 1;
    return (uint32_t)((uint64_t)h->p.L * (h->p.model == LAT_ISING ? h->W / cw : h->W));
}

struct MultiDesc {
    void* spins;
    long long* obs;                     // record of this lattice's first sweep in the run
    const unsigned long long* bc_thr;   // 54-entry table (Blume-Capel)
    uint32_t model, L, W, cw;
    uint32_t items, tile_items, ntiles, sweep0;
    uint32_t thr4, thr8, mode4, mode8;
    uint32_t rng, pad[3];
    uint32_t lut[16];
    RoundKeys rk;
};

struct MultiCtl {
    unsigned long long next;     // next tile number
    unsigned long long total;    // number of tiles
    unsigned long long timeout_ns;
    unsigned long long done_base;  // value every done[] counter starts the run at
    unsigned int nphases;        // phases of the longest lattice
    unsigned int error;          // 0 ok, 1 a wait timed out
    unsigned int err_lattice, err_phase;
    unsigned int stall_lattice;  // failure-path testing: waits of this lattice (run order) never complete
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <bool OBS>
__device__ __forceinline__ void ising_tile(const MultiDesc& d, const uint32_t* s_lut, uint32_t sweep,
                                           uint32_t colour, uint64_t i0, uint64_t i1, PhaseAcc& acc)
{
    const IsingPhase ph{static_cast<uint64_t*>(d.spins), d.L, d.W, sweep, colour, d.thr4, d.thr8, d.mode4, d.mode8};
    const RoundKeys rk = d.rk;
    const int lane = threadIdx.x & 31;
    if (d.rng == LAT_RNG_TABLE_MODE) {
        if (d.cw == 2) {
            for (uint64_t it = i0 + threadIdx.x; it < i1; it += blockDim.x)
                ising_item_lut<2, OBS, true>(ph, rk, s_lut, nullptr, it, lane, acc);
        } else {
            for (uint64_t it = i0 + threadIdx.x; it < i1; it += blockDim.x)
                ising_item_lut<1, OBS, true>(ph, rk, s_lut, nullptr, it, lane, acc);
        }
        return;
    }
    if (d.cw == 2) {
        for (uint64_t it = i0 + threadIdx.x; it < i1; it += blockDim.x) ising_item<2, OBS, true>(ph, rk, it, lane, acc);
    } else {
        for (uint64_t it = i0 + threadIdx.x; it < i1; it += blockDim.x) ising_item<1, OBS, true>(ph, rk, it, lane, acc);
    }
}

template <bool OBS>
__device__ __forceinline__ void bc_tile(const MultiDesc& d, const uint2* s_thr, uint32_t sweep,
                                        uint32_t colour, uint64_t i0, uint64_t i1, PhaseAcc& acc)
{
    const BcPhase ph{static_cast<ulonglong2*>(d.spins), d.L, d.W, sweep, colour};
    const RoundKeys rk = d.rk;
    const int lane = threadIdx.x & 31;
    for (uint64_t it = i0 + threadIdx.x; it < i1; it += blockDim.x) bc_item<OBS, true>(ph, rk, s_thr, it, lane, acc);
}

template <int MINB>
__global__ void __launch_bounds__(kMultiThreads, MINB)
    k_multi(const MultiDesc* __restrict__ desc, const uint32_t* __restrict__ tile_prefix,
            const unsigned long long* __restrict__ phase_base, const uint32_t* __restrict__ active,
            unsigned long long* done, MultiCtl* ctl)
{
    __shared__ unsigned long long s_g;
    __shared__ int s_stop;
    __shared__ uint2 s_thr[kBcTable];
    __shared__ uint32_t s_lut[kLutSlots];
    const unsigned long long total = ctl->total;
    const uint32_t K = ctl->nphases;
    for (;;) {
        if (threadIdx.x == 0) s_g = atomicAdd(&ctl->next, 1ull);
        __syncthreads();
        const unsigned long long g = s_g;
        if (g >= total) break;
        // phase k: the last k with phase_base[k] <= g
        uint32_t lo = 0, hi = K;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (phase_base[mid] <= g) lo = mid;
            else hi = mid;
        }
        const uint32_t k = lo;
        const uint32_t rem = (uint32_t)(g - phase_base[k]);
        // lattice r among the first active[k]: the last r with tile_prefix[r] <= rem
        uint32_t rlo = 0, rhi = active[k];
        while (rhi - rlo > 1) {
            const uint32_t mid = (rlo + rhi) >> 1;
            if (tile_prefix[mid] <= rem) rlo = mid;
            else rhi = mid;
        }
        const uint32_t r = rlo;
        const uint32_t t = rem - tile_prefix[r];
        const MultiDesc& d = desc[r];
        if (threadIdx.x == 0) {
            int stop = 0;
            if (k > 0) {
                const unsigned long long target = r == ctl->stall_lattice
                    ? kRunnerStallTarget : ctl->done_base + (unsigned long long)k * d.ntiles;
                const unsigned long long t0 = global_ns();
                while (load_acquire(&done[r]) < target) {
                    if (*(volatile unsigned int*)&ctl->error) {
                        stop = 1;
                        break;
                    }
                    if (global_ns() - t0 > ctl->timeout_ns) {
                        if (atomicCAS(&ctl->error, 0u, 1u) == 0u) {
                            ctl->err_lattice = r;
                            ctl->err_phase = k;
                        }
                        stop = 1;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            if (*(volatile unsigned int*)&ctl->error) stop = 1;
            s_stop = stop;
        }
        if (d.model == 1) bc_table128(d.bc_thr, s_thr);
        else if (d.rng == LAT_RNG_TABLE_MODE && threadIdx.x < kLutSlots) s_lut[threadIdx.x] = lut_slot(d.lut, threadIdx.x);
        __syncthreads();
        if (s_stop) break;

        const uint32_t colour = k & 1u, sweep = d.sweep0 + (k >> 1);
        const uint64_t i0 = (uint64_t)t * d.tile_items;
        const uint64_t i1 = min(i0 + d.tile_items, (uint64_t)d.items);
        long long* rec = d.obs ? d.obs + (size_t)(k >> 1) * kObsWords : nullptr;
        PhaseAcc acc;
        if (d.model == 0) {
            if (colour) ising_tile<true>(d, s_lut, sweep, colour, i0, i1, acc);
            else ising_tile<false>(d, s_lut, sweep, colour, i0, i1, acc);
        } else {
            if (colour) bc_tile<true>(d, s_thr, sweep, colour, i0, i1, acc);
            else bc_tile<false>(d, s_thr, sweep, colour, i0, i1, acc);
        }
        flush_acc(colour ? rec : nullptr, rec ? rec + kObsDraws : nullptr, acc);
        __threadfence();  // this thread's lattice stores before the tile is published
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&done[r], 1ull);
    }
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct RunnerLayout {
    size_t desc, tile_prefix, phase_base, active, done, ctl, obs, bcthr, total;
};

RunnerLayout runner_layout(uint32_t cap, uint32_t max_sweeps)
{
    RunnerLayout l;
    size_t off = 0;
    l.desc = off;
    off = align_up(off + (size_t)cap * sizeof(MultiDesc));
    l.tile_prefix = off;
    off = align_up(off + ((size_t)cap + 1) * sizeof(uint32_t));
    l.phase_base = off;
    off = align_up(off + (2 * (size_t)max_sweeps + 1) * sizeof(unsigned long long));
    l.active = off;
    off = align_up(off + 2 * (size_t)max_sweeps * sizeof(uint32_t));
    l.done = off;
    off = align_up(off + (size_t)cap * sizeof(unsigned long long));
    l.ctl = off;
    off = align_up(off + sizeof(MultiCtl));
    l.obs = off;
    off = align_up(off + (size_t)cap * max_sweeps * kObsWords * sizeof(long long));
    l.bcthr = off;
    off = align_up(off + (size_t)cap * 54 * sizeof(unsigned long long));
    l.total = off;
    return l;
}

}  // namespace

struct lat_runner {
    uint32_t cap, max_sweeps;
    RunnerLayout lay;
    char* buf;
    bool owns;
    cudaStream_t stream;
    int grid;
    int minb;  // resident blocks per SM the persistent kernel is built for (2 or 3)
    unsigned long long timeout_ns;
    uint32_t stall;  // input index whose waits never complete (failure-path tests), or ~0
    unsigned long long done_base;  // start value of the tile counters (0; tests move it near 2^32)
    std::map<std::pair<int, uint32_t>, uint32_t> tile_of;  // (model, L) -> items per tile
    // pinned host staging
    char* host;
    size_t host_bytes;
    cudaGraphExec_t graph;
    bool have_graph;
    // a run submitted and not yet collected
    bool pending = false;
    std::vector<lat_t*> pend_lat;
    std::vector<uint32_t> pend_ns;
    long long* pend_hobs = nullptr;
    MultiCtl* pend_hctl = nullptr;
    cudaEvent_t dep_event = nullptr;  // orders the runner's stream after work on a handle's other stream

    MultiDesc* d_desc() const { return reinterpret_cast<MultiDesc*>(buf + lay.desc); }
    uint32_t* d_tile_prefix() const { return reinterpret_cast<uint32_t*>(buf + lay.tile_prefix); }
    unsigned long long* d_phase_base() const { return reinterpret_cast<unsigned long long*>(buf + lay.phase_base); }
    uint32_t* d_active() const { return reinterpret_cast<uint32_t*>(buf + lay.active); }
    unsigned long long* d_done() const { return reinterpret_cast<unsigned long long*>(buf + lay.done); }
    MultiCtl* d_ctl() const { return reinterpret_cast<MultiCtl*>(buf + lay.ctl); }
    long long* d_obs() const { return reinterpret_cast<long long*>(buf + lay.obs); }
    unsigned long long* d_bcthr() const { return reinterpret_cast<unsigned long long*>(buf + lay.bcthr); }
};

namespace {

// Host staging layout (pinned): descriptors, tile prefix, phase base, active
// counts, control, tables, start values of the tile counters, records.
size_t host_bytes_for(uint32_t cap, uint32_t max_sweeps)
{
    return (size_t)cap * sizeof(MultiDesc) + ((size_t)cap + 1) * sizeof(uint32_t) +
           (size_t)cap * sizeof(unsigned long long) +
           (2 * (size_t)max_sweeps + 1) * sizeof(unsigned long long) + 2 * (size_t)max_sweeps * sizeof(uint32_t) +
           sizeof(MultiCtl) + (size_t)cap * 54 * sizeof(unsigned long long) + 64 + 256 +
           (size_t)cap * max_sweeps * kObsWords * sizeof(long long);
}

// The persistent launch itself (the tile counters are set by each run's uploads).
cudaError_t enqueue_run(lat_runner* R, cudaStream_t st)
{
    if (R->minb == 3)
        k_multi<3><<<R->grid, kMultiThreads, 0, st>>>(R->d_desc(), R->d_tile_prefix(), R->d_phase_base(),
                                                      R->d_active(), R->d_done(), R->d_ctl());
    else
        k_multi<2><<<R->grid, kMultiThreads, 0, st>>>(R->d_desc(), R->d_tile_prefix(), R->d_phase_base(),
                                                      R->d_active(), R->d_done(), R->d_ctl());
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t lat_runner_footprint(uint32_t max_lattices, uint32_t max_sweeps)
{
    if (max_lattices == 0 || max_sweeps == 0 || max_sweeps > (1u << 20) || max_lattices > (1u << 20)) return 0;
    return runner_layout(max_lattices, max_sweeps).total;
}

int lat_runner_create(uint32_t max_lattices, uint32_t max_sweeps, void* dev_buf, size_t bytes, void* stream,
                      lat_runner_t** out)
{
    if (!out || lat_runner_footprint(max_lattices, max_sweeps) == 0) return LAT_EINVAL;
    *out = nullptr;
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) % kAlign) != 0) return LAT_EINVAL;
    int dev = 0, sms = 0, bpsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LAT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LAT_ECUDA;
    // Two resident blocks per SM give the kernel the registers it needs
    // without spilling, which measured faster than three blocks with spills
    // on the mixed 512-lattice workload; LAT_MULTI_BLOCKS=3 selects the other.
    const char* env = std::getenv("LAT_MULTI_BLOCKS");
    const int minb = (env && env[0] == '3') ? 3 : 2;
    const cudaError_t oe = minb == 3
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_multi<3>, kMultiThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_multi<2>, kMultiThreads, 0);
    if (oe != cudaSuccess) return LAT_ECUDA;
    lat_runner* R = new (std::nothrow) lat_runner();
    if (!R) return LAT_ENOMEM;
    R->cap = max_lattices;
    R->max_sweeps = max_sweeps;
    R->lay = runner_layout(max_lattices, max_sweeps);
    R->stream = static_cast<cudaStream_t>(stream);
    R->grid = sms * (bpsm < 1 ? 1 : bpsm);
    R->minb = minb;
    R->timeout_ns = 10ull * 1000 * 1000 * 1000;  // 10 s per wait
    R->stall = 0xFFFFFFFFu;
    R->done_base = 0;
    R->have_graph = false;
    if (dev_buf) {
        if (bytes < R->lay.total) {
            delete R;
            return LAT_ENOMEM;
        }
        R->buf = static_cast<char*>(dev_buf);
        R->owns = false;
    } else {
        if (cudaMalloc(&R->buf, R->lay.total) != cudaSuccess) {
            cudaGetLastError();
            delete R;
            return LAT_ENOMEM;
        }
        R->owns = true;
    }
    R->host_bytes = host_bytes_for(max_lattices, max_sweeps);
    if (cudaMallocHost(&R->host, R->host_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (R->owns) cudaFree(R->buf);
        delete R;
        return LAT_ENOMEM;
    }
    // Capture the launch (counter reset + persistent kernel) once; every run
    // replays it after uploading that run's descriptors.
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e1 = enqueue_run(R, cs);
            const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&R->graph, g, 0) == cudaSuccess)
                R->have_graph = true;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
    }
    *out = R;
    return LAT_OK;
}

int lat_runner_set_tile(lat_runner_t* R, int32_t model, uint32_t L, uint32_t tile_items)
{
    if (!R || (model != LAT_ISING && model != LAT_BLUME_CAPEL) || L < 64 || L % 64 != 0) return LAT_EINVAL;
    if (tile_items != 0 && tile_items % kMultiThreads != 0) return LAT_EINVAL;
    if (tile_items == 0) R->tile_of.erase({model, L});
    else R->tile_of[{model, L}] = tile_items;
    return LAT_OK;
}

int lat_runner_set_timeout(lat_runner_t* R, uint64_t ns)
{
    if (!R || ns == 0) return LAT_EINVAL;
    R->timeout_ns = ns;
    return LAT_OK;
}

int lat_runner_inject_stall(lat_runner_t* R, uint32_t index)
{
    if (!R) return LAT_EINVAL;
    R->stall = index;
    return LAT_OK;
}

int lat_runner_set_counter_base(lat_runner_t* R, uint64_t base)
{
    if (!R || base >= kRunnerStallTarget) return LAT_EINVAL;
    R->done_base = base;
    return LAT_OK;
}

int lat_runner_submit(lat_runner_t* R, lat_t* const* lattices, uint32_t n, const uint32_t* nsweeps)
{
    const NvtxRange range("lat_runner_submit");
    if (!R || !lattices || !nsweeps || n == 0 || n > R->cap) return LAT_EINVAL;
    if (R->pending) return LAT_ESTATE;
    for (uint32_t i = 0; i < n; ++i) {
        if (!lattices[i] || nsweeps[i] > R->max_sweeps) return LAT_EINVAL;
        if (lattices[i]->p.L > (1u << 19)) return LAT_EINVAL;  // items of one phase must fit in 31 bits
        if (lattices[i]->next_sweep + nsweeps[i] > 0xFFFFFFFFull) return LAT_EINVAL;
        for (uint32_t j = 0; j < i; ++j)
            if (lattices[j] == lattices[i]) return LAT_EINVAL;  // a lattice may appear once per run
    }
    // every handle's earlier work must be complete before the runner's stream
    // touches it: stream order covers handles on the runner's own stream; the
    // runner's stream waits (on the device) for the last work of any other
    if (!R->dep_event &&
        cudaEventCreateWithFlags(&R->dep_event, cudaEventDisableTiming) != cudaSuccess) {
        R->dep_event = nullptr;
        return LAT_ECUDA;
    }
    for (uint32_t i = 0; i < n; ++i) {
        cudaStream_t hs = lattices[i]->stream;
        if (hs == R->stream) continue;
        bool seen = false;
        for (uint32_t j = 0; j < i && !seen; ++j) seen = lattices[j]->stream == hs;
        if (seen) continue;
        if (cudaEventRecord(R->dep_event, hs) != cudaSuccess ||
            cudaStreamWaitEvent(R->stream, R->dep_event, 0) != cudaSuccess)
            return LAT_ECUDA;
    }

    // order: descending sweep count (stable), so active lattices of a phase are a prefix
    std::vector<uint32_t> order(n);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return nsweeps[a] > nsweeps[b]; });

    char* hp = R->host;
    MultiDesc* hd = reinterpret_cast<MultiDesc*>(hp);
    hp += (size_t)R->cap * sizeof(MultiDesc);
    uint32_t* htp = reinterpret_cast<uint32_t*>(hp);
    hp += ((size_t)R->cap + 1) * sizeof(uint32_t);
    unsigned long long* hpb = reinterpret_cast<unsigned long long*>(hp);
    hp += (2 * (size_t)R->max_sweeps + 1) * sizeof(unsigned long long);
    uint32_t* hact = reinterpret_cast<uint32_t*>(hp);
    hp += 2 * (size_t)R->max_sweeps * sizeof(uint32_t);
    MultiCtl* hctl = reinterpret_cast<MultiCtl*>(hp);
    hp += sizeof(MultiCtl);
    unsigned long long* hthr = reinterpret_cast<unsigned long long*>(hp);
    hp += (size_t)R->cap * 54 * sizeof(unsigned long long);
    unsigned long long* hdone = reinterpret_cast<unsigned long long*>(hp);
    hp += (size_t)R->cap * sizeof(unsigned long long);
    long long* hobs = reinterpret_cast<long long*>(R->host + (((size_t)(hp - R->host) + 255) / 256 * 256));

    // The sparsest phase of lattice order[s] is its last one, where only the
    // lattices with at least as many sweeps are active: their items are
    // busy[s].  A tile of that lattice is capped at busy[s] / (kTilesPerBlock *
    // grid), so that a lattice left almost alone at the end of a run still
    // spreads over every block (a schedule tuned for a full batch would not).
    std::vector<uint64_t> busy(n);
    {
        uint64_t acc = 0;
        uint32_t s = 0;
        while (s < n) {
            uint32_t e2 = s;
            while (e2 < n && nsweeps[order[e2]] == nsweeps[order[s]]) acc += items_of(lattices[order[e2++]]);
            for (; s < e2; ++s) busy[s] = acc;
        }
    }
    uint32_t maxs = 0;
    uint64_t tiles_acc = 0;
    for (uint32_t s = 0; s < n; ++s) {
        const uint32_t i = order[s];
        const lat* h = lattices[i];
        MultiDesc& d = hd[s];
        std::memset(&d, 0, sizeof(d));
        d.spins = h->spins();
        d.obs = R->d_obs() + (size_t)i * R->max_sweeps * kObsWords;
        d.model = (uint32_t)h->p.model;
        d.L = h->p.L;
        d.W = h->W;
        d.cw = (h->p.model == LAT_ISING && h->W % 2 == 0) ? 2 : 1;
        d.items = items_of(h);
        auto it = R->tile_of.find({h->p.model, h->p.L});
        uint32_t tile = it != R->tile_of.end() ? it->second : kDefaultTile;
        const uint64_t cap = busy[s] / ((uint64_t)kTilesPerBlock * (uint64_t)R->grid) / kMultiThreads * kMultiThreads;
        if (tile > cap) tile = (uint32_t)std::max<uint64_t>(cap, kMultiThreads);
        if (tile > d.items) tile = (d.items + kMultiThreads - 1) / kMultiThreads * kMultiThreads;
        d.tile_items = tile;
        d.ntiles = (d.items + tile - 1) / tile;
        if (!runner_counts_fit(R->done_base, nsweeps[i], d.ntiles)) return LAT_EINVAL;
        d.sweep0 = (uint32_t)h->next_sweep;
        d.rk = h->rk;
        if (h->p.model == LAT_ISING) {
            d.thr4 = (uint32_t)(h->thr[3] >= kAlways ? 0 : h->thr[3]);
            d.thr8 = (uint32_t)(h->thr[4] >= kAlways ? 0 : h->thr[4]);
            d.mode4 = class_mode(h->thr[3]);
            d.mode8 = class_mode(h->thr[4]);
            d.rng = (uint32_t)h->p.rng;
            std::memcpy(d.lut, h->lut, sizeof(d.lut));
        } else {
            std::memcpy(hthr + (size_t)s * 54, h->thr, 54 * sizeof(uint64_t));
            d.bc_thr = R->d_bcthr() + (size_t)s * 54;
        }
        htp[s] = (uint32_t)tiles_acc;
        tiles_acc += d.ntiles;
        if (tiles_acc > 0xFFFFFFFFull) return LAT_EINVAL;
        maxs = std::max(maxs, nsweeps[i]);
    }
    htp[n] = (uint32_t)tiles_acc;
    const uint32_t K = 2 * maxs;
    uint64_t base = 0;
    uint32_t act = n;
    for (uint32_t k = 0; k < K; ++k) {
        while (act > 0 && 2 * nsweeps[order[act - 1]] <= k) --act;
        hact[k] = act;
        hpb[k] = base;
        base += htp[act];
    }
    hpb[K] = base;
    if (!runner_maps_ok(hd, htp, hpb, hact, n, K, (uint32_t)kMultiThreads)) return LAT_ESTATE;
    std::memset(hctl, 0, sizeof(MultiCtl));
    hctl->total = base;
    hctl->nphases = K;
    hctl->timeout_ns = R->timeout_ns;
    hctl->stall_lattice = 0xFFFFFFFFu;
    hctl->done_base = R->done_base;
    for (uint32_t s = 0; s < n; ++s) hdone[s] = R->done_base;
    for (uint32_t s = 0; s < n; ++s)
        if (order[s] == R->stall) hctl->stall_lattice = s;

    cudaStream_t st = R->stream;
    cudaError_t e = cudaSuccess;
    auto up = [&](size_t doff, const void* src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(R->buf + doff, src, bytes, cudaMemcpyHostToDevice, st);
    };
    up(R->lay.desc, hd, (size_t)n * sizeof(MultiDesc));
    up(R->lay.tile_prefix, htp, ((size_t)n + 1) * sizeof(uint32_t));
    up(R->lay.phase_base, hpb, ((size_t)K + 1) * sizeof(unsigned long long));
    up(R->lay.active, hact, (size_t)K * sizeof(uint32_t));
    up(R->lay.ctl, hctl, sizeof(MultiCtl));
    up(R->lay.bcthr, hthr, (size_t)n * 54 * sizeof(unsigned long long));
    up(R->lay.done, hdone, (size_t)n * sizeof(unsigned long long));
    // per-sweep records of the lattices in this run start at zero (one contiguous region)
    const size_t obs_words = (size_t)n * R->max_sweeps * kObsWords;
    if (e == cudaSuccess && maxs > 0) e = cudaMemsetAsync(R->d_obs(), 0, obs_words * sizeof(long long), st);
    if (e == cudaSuccess && K > 0) e = R->have_graph ? cudaGraphLaunch(R->graph, st) : enqueue_run(R, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hctl, R->d_ctl(), sizeof(MultiCtl), cudaMemcpyDeviceToHost, st);
    // one copy of the whole record region into pinned staging
    if (e == cudaSuccess && maxs > 0)
        e = cudaMemcpyAsync(hobs, R->d_obs(), obs_words * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return LAT_ECUDA;
    R->pending = true;
    R->pend_lat.assign(lattices, lattices + n);
    R->pend_ns.assign(nsweeps, nsweeps + n);
    R->pend_hobs = hobs;
    R->pend_hctl = hctl;
    return LAT_OK;
}

int lat_runner_collect(lat_runner_t* R, lat_obs* const* per_sweep)
{
    const NvtxRange range("lat_runner_collect");
    if (!R) return LAT_EINVAL;
    if (!R->pending) return LAT_ESTATE;
    R->pending = false;
    if (cudaStreamSynchronize(R->stream) != cudaSuccess) return LAT_ECUDA;
    if (R->pend_hctl->error) return LAT_ETIMEDOUT;
    const uint32_t n = (uint32_t)R->pend_lat.size();
    for (uint32_t i = 0; i < n; ++i) {
        if (!per_sweep || !per_sweep[i] || R->pend_ns[i] == 0) continue;
        const long long* r = R->pend_hobs + (size_t)i * R->max_sweeps * kObsWords;
        for (uint32_t s = 0; s < R->pend_ns[i]; ++s) {
            lat_obs& o = per_sweep[i][s];
            o.M = r[(size_t)s * kObsWords + kObsM];
            o.B = r[(size_t)s * kObsWords + kObsB];
            o.Q = r[(size_t)s * kObsWords + kObsQ];
            o.draws = (uint64_t)r[(size_t)s * kObsWords + kObsDraws];
            o.sweep = R->pend_lat[i]->next_sweep + s + 1;
        }
    }
    for (uint32_t i = 0; i < n; ++i) R->pend_lat[i]->next_sweep += R->pend_ns[i];
    return LAT_OK;
}

int lat_runner_run(lat_runner_t* R, lat_t* const* lattices, uint32_t n, const uint32_t* nsweeps,
                   lat_obs* const* per_sweep)
{
    const NvtxRange range("lat_runner_run");
    const int rc = lat_runner_submit(R, lattices, n, nsweeps);
    if (rc != LAT_OK) return rc;
    return lat_runner_collect(R, per_sweep);
}

int lat_runner_destroy(lat_runner_t* R)
{
    if (!R) return LAT_OK;
    cudaError_t e = cudaStreamSynchronize(R->stream);
    if (R->dep_event) cudaEventDestroy(R->dep_event);
    if (R->have_graph) cudaGraphExecDestroy(R->graph);
    if (R->host) cudaFreeHost(R->host);
    if (R->owns) {
        const cudaError_t f = cudaFree(R->buf);
        if (e == cudaSuccess) e = f;
    }
    delete R;
    return e == cudaSuccess ? LAT_OK : LAT_ECUDA;
}

}  // extern "C"
