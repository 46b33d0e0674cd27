// lat_handle.h -- the private state behind a lat_t handle, shared by the
// C ABI translation units (lat_api.cu, lat_multi.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lat.h"
#include "lat_internal.cuh"

struct Layout {
    size_t spins, obs, sd, corr, misc, stage, ds, rlist, total, stage_bytes;
};

struct lat {
    lat_params p;
    uint32_t W;
    uint64_t thr[54];
    size_t nthr;
    uint32_t lut[16];  // LAT_RNG_TABLE lookup table
    Layout lay;
    char* buf;
    bool owns;
    cudaStream_t stream;
    uint64_t next_sweep;
    latk::LaunchShape ls;
    latk::RoundKeys rk;
    std::vector<long long> host_obs;
    std::vector<long long> host_sd;

    void* spins() const { return buf + lay.spins; }
    long long* obs() const { return reinterpret_cast<long long*>(buf + lay.obs); }
    long long* sd() const { return reinterpret_cast<long long*>(buf + lay.sd); }
    long long* corr() const { return reinterpret_cast<long long*>(buf + lay.corr); }
    long long* misc() const { return reinterpret_cast<long long*>(buf + lay.misc); }
    int8_t* stage() const { return reinterpret_cast<int8_t*>(buf + lay.stage); }
    uint64_t* ds_scratch() const { return reinterpret_cast<uint64_t*>(buf + lay.ds); }
    uint32_t* rlist() const { return reinterpret_cast<uint32_t*>(buf + lay.rlist); }
};

// A named NVTX range over one entry point, so that profiler timelines show
// the library's calls around their kernels (header-only NVTX3: no cost
// beyond a pointer test when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
