// k_corr.cu -- spin-spin correlation from every site along both lattice
// axes (section 3.3, first item of the protocol, here for every distance
// r = 0..rmax): cx[r] = sum s(x,y) s(x+r,y), cy[r] = sum s(x,y) s(x,y+r),
// periodic, exact int64.
//
// On packed words a product of two Ising spins is 1 - 2 (a XOR b), so a
// 32-site word pair contributes 32 - 2 popc(a ^ b); for Blume-Capel (planes
// n: s != 0, g: s = -1) it contributes popc(na & nb) - 2 popc(na & nb &
// (ga ^ gb)).  The work is one population count per 32-bit word pair and
// distance (two for Blume-Capel), and POPC is the binding unit, so both
// kernels are built so that a word pair costs only XOR + POPC + add:
//
// x: lane s of a warp owns bit shift s and a window of NQ consecutive word
//    offsets q0..q0+NQ-1, i.e. distances r = 32 q + s.  The row (in shared
//    memory, 32-bit words) rotated by 32 (q0+k) + s is produced one word at
//    a time with a funnel shift and kept in a register window that slides
//    along the row; each rotated word meets NQ row words.
// y: lane j owns column word j of a 32-word strip; warp g owns NQ
//    consecutive distances.  Rows y0..y0+HY-1 and the rows they pair with are
//    staged in shared memory; a register window of NQ rows slides down the
//    strip.
// In both, the window's slots rotate by full unrolling (slot (i+k) % NQ
// holds the element at offset k), so no register moves are needed.
#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kXWarpsMax = 4;     // rows in flight per x block (one per warp)
constexpr uint32_t kXRows = 64;   // rows per warp in the x kernel
constexpr int kYWarps = 8;        // distance groups per y block
constexpr uint32_t kHY = 64;      // rows per y block

template <int MODEL>
struct Planes {
    static constexpr int n = MODEL == 0 ? 1 : 2;
};

// Load row y as 32-bit words: Ising plane at dst[0..W32); Blume-Capel n
// plane at dst[0..W32) and g plane at dst[W32..2 W32).
template <int MODEL>
__device__ __forceinline__ void load_row32(const void* spins, uint32_t W, uint64_t y, uint32_t* dst, int lane,
                                           int nlanes)
{
    const uint32_t W32 = 2 * W;
    if constexpr (MODEL == 0) {
        const uint2* src = static_cast<const uint2*>(spins) + y * W;
        for (uint32_t j = lane; j < W; j += nlanes) {
            const uint2 v = src[j];
            dst[2 * j] = v.x;
            dst[2 * j + 1] = v.y;
        }
    } else {
        const uint4* src = static_cast<const uint4*>(spins) + y * W;
        for (uint32_t j = lane; j < W; j += nlanes) {
            const uint4 v = src[j];  // n lo, n hi, g lo, g hi
            dst[2 * j] = v.x;
            dst[2 * j + 1] = v.y;
            dst[W32 + 2 * j] = v.z;
            dst[W32 + 2 * j + 1] = v.w;
        }
    }
}

// Word j0 (0 <= j0 < W32) of the row rotated right by s bits: bits s..31 of
// word j0 followed by bits 0..s-1 of the next word (periodic).
__device__ __forceinline__ uint32_t rot_word(const uint32_t* row, uint32_t W32, uint32_t j0, uint32_t s)
{
    const uint32_t j1 = j0 + 1 == W32 ? 0 : j0 + 1;
    return __funnelshift_r(row[j0], row[j1], s);
}

template <int MODEL, int NQ>
__global__ void __launch_bounds__(kXWarpsMax * 32) k_corr_x(const void* spins, uint32_t L, uint32_t rmax,
                                                           long long* cx)
{
    extern __shared__ uint32_t sm[];
    const uint32_t W = L / 64, W32 = L / 32;
    const int warp = threadIdx.x >> 5, s = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const uint32_t q0 = blockIdx.y * NQ;
    uint32_t* row = sm + (size_t)warp * W32 * Planes<MODEL>::n;
    int acc[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = 0;
    const uint32_t ybeg = (blockIdx.x * nwarps + warp) * kXRows;
    const uint32_t yend = min(ybeg + kXRows, L);
    for (uint32_t y = ybeg; y < yend; ++y) {
        __syncwarp();
        load_row32<MODEL>(spins, W, y, row, s, 32);
        __syncwarp();
        uint32_t win[NQ], wing[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const uint32_t j = (q0 + k) % W32;
            win[k] = rot_word(row, W32, j, s);
            if constexpr (MODEL == 1) wing[k] = rot_word(row + W32, W32, j, s);
        }
        uint32_t jn = (q0 + NQ) % W32;  // (i + q0 + NQ) mod W32: the word entering the window
        for (uint32_t ib = 0; ib < W32; ib += NQ) {
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const uint32_t i = ib + u;
                if (i < W32) {
                    const uint32_t a = row[i];
                    if constexpr (MODEL == 0) {
#pragma unroll
                        for (int k = 0; k < NQ; ++k) acc[k] += __popc(a ^ win[(u + k) % NQ]);
                        win[u] = rot_word(row, W32, jn, s);
                    } else {
                        const uint32_t ag = row[W32 + i];
#pragma unroll
                        for (int k = 0; k < NQ; ++k) {
                            const uint32_t both = a & win[(u + k) % NQ];
                            acc[k] += __popc(both) - 2 * __popc(both & (ag ^ wing[(u + k) % NQ]));
                        }
                        win[u] = rot_word(row, W32, jn, s);
                        wing[u] = rot_word(row + W32, W32, jn, s);
                    }
                    jn = jn + 1 == W32 ? 0 : jn + 1;
                }
            }
        }
    }
    const long long rows = yend > ybeg ? (long long)(yend - ybeg) : 0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const uint32_t r = 32u * (q0 + k) + s;
        if (r <= rmax && rows) {
            const long long v = MODEL == 0 ? rows * (long long)L - 2ll * acc[k] : (long long)acc[k];
            atomicAdd(reinterpret_cast<unsigned long long*>(cx + r), (unsigned long long)v);
        }
    }
}

template <int MODEL, int NQ>
__global__ void __launch_bounds__(kYWarps * 32) k_corr_y(const void* spins, uint32_t L, uint32_t rmax,
                                                        long long* cy)
{
    extern __shared__ uint32_t sm[];
    constexpr int P = Planes<MODEL>::n;
    constexpr uint32_t NB = kHY + kYWarps * NQ - 1;  // B rows per block
    const uint32_t W = L / 64, W32 = L / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t j0 = blockIdx.x * 32;             // first column word of the strip
    const uint32_t tw = min(32u, W32 - j0);          // strip width in words
    const uint32_t y0 = blockIdx.y * kHY;
    const uint32_t r0 = blockIdx.z * (kYWarps * NQ);
    uint32_t* A = sm;                      // kHY x 32 words per plane
    uint32_t* B = sm + kHY * 32 * P;       // NB x 32 words per plane

    // stage A rows y0.. and B rows y0 + r0 .. (mod L), plane-major per row block
    for (uint32_t t = threadIdx.x; t < (kHY + NB) * 32; t += blockDim.x) {
        const uint32_t rr = t / 32, c = t % 32;
        const bool isA = rr < kHY;
        const uint32_t rloc = isA ? rr : rr - kHY;
        const uint64_t y = ((uint64_t)(isA ? y0 : y0 + r0) + rloc) % L;
        uint32_t vn = 0, vg = 0;
        if (c < tw) {
            const uint32_t j = j0 + c;  // 32-bit column word
            if constexpr (MODEL == 0) {
                vn = static_cast<const uint32_t*>(spins)[y * W32 + j];
            } else {
                const uint32_t* p = static_cast<const uint32_t*>(spins) + y * 2 * W32;
                vn = p[4 * (j / 2) + (j & 1)];
                vg = p[4 * (j / 2) + 2 + (j & 1)];
            }
        }
        uint32_t* base = isA ? A : B;
        const uint32_t nrows = isA ? kHY : NB;
        base[rloc * 32 + c] = vn;
        if constexpr (MODEL == 1) base[nrows * 32 + rloc * 32 + c] = vg;
    }
    __syncthreads();

    const uint32_t g0 = (uint32_t)warp * NQ;  // this warp's first distance offset within the block
    int acc[NQ];
    uint32_t win[NQ], wing[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        acc[k] = 0;
        win[k] = B[(g0 + k) * 32 + lane];
        if constexpr (MODEL == 1) wing[k] = B[NB * 32 + (g0 + k) * 32 + lane];
    }
    for (uint32_t yb = 0; yb < kHY; yb += NQ) {
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            const uint32_t y = yb + u;
            if (y < kHY) {
                const uint32_t a = A[y * 32 + lane];
                if constexpr (MODEL == 0) {
#pragma unroll
                    for (int k = 0; k < NQ; ++k) acc[k] += __popc(a ^ win[(u + k) % NQ]);
                } else {
                    const uint32_t ag = A[kHY * 32 + y * 32 + lane];
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        const uint32_t both = a & win[(u + k) % NQ];
                        acc[k] += __popc(both) - 2 * __popc(both & (ag ^ wing[(u + k) % NQ]));
                    }
                }
                const uint32_t nb = y + g0 + NQ;  // next B row for this slot (< NB except past the end)
                if (nb < NB) {
                    win[u] = B[nb * 32 + lane];
                    if constexpr (MODEL == 1) wing[u] = B[NB * 32 + nb * 32 + lane];
                }
            }
        }
    }
    const bool valid = lane < tw;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        int v = valid ? acc[k] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        const uint32_t r = r0 + g0 + k;
        if (lane == 0 && r <= rmax) {
            const long long t = MODEL == 0 ? (long long)kHY * 32 * tw - 2ll * v : (long long)v;
            atomicAdd(reinterpret_cast<unsigned long long*>(cy + r), (unsigned long long)t);
        }
    }
}

// Window sizes instantiated; the launcher picks the one that wastes the
// fewest distance slots.
constexpr int kNQ[] = {4, 8, 11, 13, 16};

int pick_nq(uint32_t count, uint32_t per_group_mult)
{
    int best = kNQ[0];
    uint64_t best_slots = ~0ull;
    for (int nq : kNQ) {
        const uint64_t chunk = (uint64_t)nq * per_group_mult;
        const uint64_t slots = (count + chunk - 1) / chunk * chunk;
        if (slots < best_slots || (slots == best_slots && nq > best)) {
            best = nq;
            best_slots = slots;
        }
    }
    return best;
}

template <int MODEL, int NQ>
cudaError_t launch_x(const void* spins, uint32_t L, uint32_t rmax, long long* cx, cudaStream_t st)
{
    const uint32_t W32 = L / 32;
    const size_t per_warp = (size_t)W32 * Planes<MODEL>::n * sizeof(uint32_t);
    int nwarps = (int)(160u * 1024u / per_warp);
    nwarps = nwarps < 1 ? 1 : (nwarps > kXWarpsMax ? kXWarpsMax : nwarps);
    const size_t smem = per_warp * nwarps;
    cudaError_t e = cudaFuncSetAttribute(k_corr_x<MODEL, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t qtot = rmax / 32 + 1;
    const dim3 grid((L + nwarps * kXRows - 1) / (nwarps * kXRows), (qtot + NQ - 1) / NQ);
    k_corr_x<MODEL, NQ><<<grid, nwarps * 32, smem, st>>>(spins, L, rmax, cx);
    return cudaGetLastError();
}

template <int MODEL, int NQ>
cudaError_t launch_y(const void* spins, uint32_t L, uint32_t rmax, long long* cy, cudaStream_t st)
{
    const uint32_t W32 = L / 32;
    const size_t smem = (size_t)(kHY + kHY + kYWarps * NQ - 1) * 32 * Planes<MODEL>::n * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_corr_y<MODEL, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t per_block = kYWarps * NQ;
    const dim3 grid((W32 + 31) / 32, L / kHY, (rmax + per_block) / per_block);
    k_corr_y<MODEL, NQ><<<grid, kYWarps * 32, smem, st>>>(spins, L, rmax, cy);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_xy(const void* spins, uint32_t L, uint32_t rmax, long long* cx, long long* cy, cudaStream_t st)
{
    cudaError_t e;
    switch (pick_nq(rmax / 32 + 1, 1)) {
        case 4: e = launch_x<MODEL, 4>(spins, L, rmax, cx, st); break;
        case 8: e = launch_x<MODEL, 8>(spins, L, rmax, cx, st); break;
        case 11: e = launch_x<MODEL, 11>(spins, L, rmax, cx, st); break;
        case 13: e = launch_x<MODEL, 13>(spins, L, rmax, cx, st); break;
        default: e = launch_x<MODEL, 16>(spins, L, rmax, cx, st); break;
    }
    if (e != cudaSuccess) return e;
    switch (pick_nq(rmax + 1, kYWarps)) {
        case 4: return launch_y<MODEL, 4>(spins, L, rmax, cy, st);
        case 8: return launch_y<MODEL, 8>(spins, L, rmax, cy, st);
        case 11: return launch_y<MODEL, 11>(spins, L, rmax, cy, st);
        case 13: return launch_y<MODEL, 13>(spins, L, rmax, cy, st);
        default: return launch_y<MODEL, 16>(spins, L, rmax, cy, st);
    }
}

}  // namespace

cudaError_t launch_correlation(int model, const void* spins, uint32_t L, uint32_t W, uint32_t rmax, long long* cx,
                               long long* cy, cudaStream_t st)
{
    (void)W;
    cudaError_t e = cudaMemsetAsync(cx, 0, (rmax + 1) * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cy, 0, (rmax + 1) * sizeof(long long), st);
    if (e != cudaSuccess) return e;
    return model == 0 ? launch_xy<0>(spins, L, rmax, cx, cy, st) : launch_xy<1>(spins, L, rmax, cx, cy, st);
}

}  // namespace latk
