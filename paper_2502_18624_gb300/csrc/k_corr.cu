// k_corr.cu -- spin-spin correlation from every site along both lattice
// axes (section 3.3, first item of the protocol, here for every distance
// r = 0..rmax): cx[r] = sum s(x,y) s(x+r,y), cy[r] = sum s(x,y) s(x,y+r),
// periodic, exact int64.
//
// On the packed words a product of two Ising spins is 1 - 2 (a XOR b), so a
// 64-site word pair contributes 64 - 2 popc(a ^ b).  For Blume-Capel
// (planes n: s != 0, g: s = -1) a pair contributes
// popc(na & nb) - 2 popc(na & nb & (ga ^ gb)).
//
// x: a block stages one row at a time in shared memory; thread r compares the
//    row with itself rotated by r bits (word offset r/64, funnel shift r%64).
// y: a block stages a strip of TW words x (HY + HY + RC - 1) rows in shared
//    memory (pitch TW+1 words, so the 32 lanes of a warp, which read 32
//    different rows, hit distinct banks); thread r compares row y with row
//    y + r for the block's HY rows.
#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr int kCorrThreads = 256;
constexpr uint32_t kRowsX = 64;    // rows per x block
constexpr uint32_t kTW = 8;        // words per y strip
constexpr uint32_t kHY = 64;       // rows per y block
constexpr uint32_t kRC = kCorrThreads;  // distances per y block

__device__ __forceinline__ uint64_t rot_word(uint64_t cur, uint64_t nxt, uint32_t sh)
{
    // bits sh..63 of cur, then bits 0..sh-1 of nxt; well defined for sh = 0.
    return (cur >> sh) | ((nxt << 1) << (63 - sh));
}

template <int MODEL>
__global__ void __launch_bounds__(kCorrThreads) k_corr_x(const void* spins, uint32_t L, uint32_t W, uint32_t rmax,
                                                        long long* cx)
{
    extern __shared__ uint64_t srow[];  // W words (Ising) or n[W], g[W] (Blume-Capel)
    const uint32_t r = blockIdx.y * blockDim.x + threadIdx.x;
    const bool active = r <= rmax;
    const uint32_t q = r >> 6, sh = r & 63u;
    const uint32_t y0 = blockIdx.x * kRowsX;
    long long total = 0;
    for (uint32_t y = y0; y < y0 + kRowsX && y < L; ++y) {
        __syncthreads();
        if constexpr (MODEL == 0) {
            const uint64_t* row = static_cast<const uint64_t*>(spins) + (uint64_t)y * W;
            for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) srow[i] = row[i];
        } else {
            const ulonglong2* row = static_cast<const ulonglong2*>(spins) + (uint64_t)y * W;
            for (uint32_t i = threadIdx.x; i < W; i += blockDim.x) {
                const ulonglong2 v = row[i];
                srow[i] = v.x;
                srow[W + i] = v.y;
            }
        }
        __syncthreads();
        if (!active) continue;
        uint32_t j = q % W;
        long long acc = 0;
        if constexpr (MODEL == 0) {
            uint64_t cur = srow[j];
            for (uint32_t i = 0; i < W; ++i) {
                uint32_t j1 = j + 1;
                if (j1 >= W) j1 -= W;
                const uint64_t nxt = srow[j1];
                acc += __popcll(srow[i] ^ rot_word(cur, nxt, sh));
                cur = nxt;
                j = j1;
            }
            total += (long long)L - 2 * acc;
        } else {
            uint64_t curn = srow[j], curg = srow[W + j];
            for (uint32_t i = 0; i < W; ++i) {
                uint32_t j1 = j + 1;
                if (j1 >= W) j1 -= W;
                const uint64_t nxn = srow[j1], nxg = srow[W + j1];
                const uint64_t both = srow[i] & rot_word(curn, nxn, sh);
                acc += __popcll(both) - 2 * __popcll(both & (srow[W + i] ^ rot_word(curg, nxg, sh)));
                curn = nxn;
                curg = nxg;
                j = j1;
            }
            total += acc;
        }
    }
    if (active) atomicAdd(reinterpret_cast<unsigned long long*>(cx + r), (unsigned long long)total);
}

template <int MODEL>
__global__ void __launch_bounds__(kCorrThreads) k_corr_y(const void* spins, uint32_t L, uint32_t W, uint32_t rmax,
                                                        long long* cy)
{
    extern __shared__ uint64_t sm[];
    constexpr uint32_t P = kTW + 1;  // padded pitch in words
    constexpr uint32_t NB = kHY + kRC - 1;
    uint64_t* A = sm;                       // kHY rows
    uint64_t* B = sm + kHY * P;             // NB rows
    uint64_t* Ag = B + NB * P;              // Blume-Capel sign planes
    uint64_t* Bg = Ag + kHY * P;
    const uint32_t j0 = blockIdx.x * kTW;
    const uint32_t tw = min(kTW, W - j0);
    const uint32_t y0 = blockIdx.y * kHY;
    const uint32_t r0 = blockIdx.z * kRC;

    auto load = [&](uint64_t* dst, uint64_t* dstg, uint32_t ybase, uint32_t nrows) {
        for (uint32_t t = threadIdx.x; t < nrows * kTW; t += blockDim.x) {
            const uint32_t rr = t / kTW, i = t - rr * kTW;
            if (i >= tw) continue;
            const uint64_t y = ((uint64_t)ybase + rr) % L;
            if constexpr (MODEL == 0) {
                dst[rr * P + i] = static_cast<const uint64_t*>(spins)[y * W + j0 + i];
            } else {
                const ulonglong2 v = static_cast<const ulonglong2*>(spins)[y * W + j0 + i];
                dst[rr * P + i] = v.x;
                dstg[rr * P + i] = v.y;
            }
        }
    };
    load(A, Ag, y0, kHY);
    load(B, Bg, (uint32_t)(((uint64_t)y0 + r0) % L), NB);
    __syncthreads();

    const uint32_t r = r0 + threadIdx.x;
    if (r > rmax) return;
    long long acc = 0;
    for (uint32_t y = 0; y < kHY; ++y) {
        const uint64_t* a = A + y * P;
        const uint64_t* b = B + (y + threadIdx.x) * P;
        if constexpr (MODEL == 0) {
            for (uint32_t i = 0; i < tw; ++i) acc += __popcll(a[i] ^ b[i]);
        } else {
            const uint64_t* ag = Ag + y * P;
            const uint64_t* bg = Bg + (y + threadIdx.x) * P;
            for (uint32_t i = 0; i < tw; ++i) {
                const uint64_t both = a[i] & b[i];
                acc += __popcll(both) - 2 * __popcll(both & (ag[i] ^ bg[i]));
            }
        }
    }
    const long long total = MODEL == 0 ? (long long)kHY * 64 * tw - 2 * acc : acc;
    atomicAdd(reinterpret_cast<unsigned long long*>(cy + r), (unsigned long long)total);
}

}  // namespace

cudaError_t launch_correlation(int model, const void* spins, uint32_t L, uint32_t W, uint32_t rmax, long long* cx,
                               long long* cy, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cx, 0, (rmax + 1) * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cy, 0, (rmax + 1) * sizeof(long long), st);
    if (e != cudaSuccess) return e;

    const uint32_t rchunks = (rmax + kCorrThreads) / kCorrThreads;
    const size_t smx = (size_t)W * (model == 0 ? 1 : 2) * sizeof(uint64_t);
    const dim3 gx((L + kRowsX - 1) / kRowsX, rchunks);
    const size_t smy = (size_t)(kHY + kHY + kRC - 1) * (kTW + 1) * sizeof(uint64_t) * (model == 0 ? 1 : 2);
    const dim3 gy((W + kTW - 1) / kTW, L / kHY, rchunks);
    if (model == 0) {
        e = cudaFuncSetAttribute(k_corr_x<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_corr_y<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy);
        if (e != cudaSuccess) return e;
        k_corr_x<0><<<gx, kCorrThreads, smx, st>>>(spins, L, W, rmax, cx);
        k_corr_y<0><<<gy, kCorrThreads, smy, st>>>(spins, L, W, rmax, cy);
    } else {
        e = cudaFuncSetAttribute(k_corr_x<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_corr_y<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy);
        if (e != cudaSuccess) return e;
        k_corr_x<1><<<gx, kCorrThreads, smx, st>>>(spins, L, W, rmax, cx);
        k_corr_y<1><<<gy, kCorrThreads, smy, st>>>(spins, L, W, rmax, cy);
    }
    return cudaGetLastError();
}

}  // namespace latk
