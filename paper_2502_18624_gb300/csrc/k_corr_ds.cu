// k_corr_ds.cu -- spin-spin correlation from downsampled sources (section
// 3.3, second and third items of the protocol): the sources are one site per
// R x R square, its top-left corner (x % R == 0, y % R == 0), and the
// distances are an arbitrary list of r <= L/2:
//   cx[i] = sum_{sources} s(x,y) s(x + r_i, y),
//   cy[i] = sum_{sources} s(x,y) s(x, y + r_i),       periodic, exact int64.
// R is a power of two, 1 <= R <= 64, so the source columns of one packed
// word are a fixed bit mask and every row holds nd = L/R sources.
//
// x: the targets of source row y at distance r = q R + p are the sites
//    (k R + p + q R, y), i.e. the phase-p subsequence of the row rotated by
//    q.  A block takes one source row, splits it in shared memory into its R
//    phase subsequences D_p (bit k of D_p = s(k R + p, y), zero padded), and
//    then each warp takes distances: sum_k D_0[k] * D_p[(k + q) mod nd],
//    64 sources per word operation.
// y: the targets of source row y at distance r are row y + r at the source
//    columns.  With R >= 16 the source columns of every row are first
//    gathered into a compact copy E (L rows of nd bits, zero padded, one
//    lattice read), so a (row, distance) pair costs nd / 64 word operations
//    instead of L / 64; with R < 16 the kernel reads the lattice rows with
//    the source-column mask.
// Products of packed spins: Ising 1 - 2 (a XOR b), so a row contributes
// nd - 2 popc(xor); Blume-Capel (planes n: s != 0, g: s = -1) contributes
// popc(na & nb) - 2 popc(na & nb & (ga ^ gb)).
//
// Accumulation: inside a block each distance has exactly one owning warp,
// which adds its row sums to a shared accumulator without atomics; at the
// end every block adds its accumulators to the global sums (one atomic per
// distance and block).
#include <algorithm>

#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr int kDsThreads = 256;
constexpr int kDsWarps = kDsThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ long long warp_total(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Bits at positions p, p+R, p+2R, ... of w, packed into the low 64/R bits.
__device__ __forceinline__ uint64_t every_rth(uint64_t w, uint32_t R, uint32_t p)
{
    w >>= p;
    if (R == 1) return w;
    uint64_t out = 0;
    const uint32_t n = 64u / R;
    for (uint32_t b = 0; b < n; ++b) out |= ((w >> (b * R)) & 1ull) << b;
    return out;
}

// Word m of the phase-p subsequence of a row (bits k = 64m .. 64m+63 with
// k < nd, zero beyond): lattice words m R .. m R + R - 1 each give 64/R bits.
template <int PL>
__device__ __forceinline__ uint64_t gather_word(const uint64_t* row, uint32_t W, uint32_t R, uint32_t p, uint32_t m)
{
    const uint32_t per = 64u / R;
    uint64_t out = 0;
    const uint32_t j0 = m * R;
    for (uint32_t i = 0; i < R && j0 + i < W; ++i) {
        const uint64_t w = __ldg(row + (size_t)(j0 + i) * PL);
        out |= every_rth(w, R, p) << (i * per);
    }
    return out;
}

// 64 consecutive bits of a cyclic sequence of nd bits stored in words d[]
// (zero beyond bit nd, plus one zero word), starting at bit pos < nd.  Bits
// of the result at index >= nd are unspecified and must be masked.
__device__ __forceinline__ uint64_t window64(const uint64_t* d, uint32_t pos, uint32_t nd)
{
    const uint32_t wi = pos >> 6, sh = pos & 63;
    uint64_t v = sh ? (d[wi] >> sh) | (d[wi + 1] << (64 - sh)) : d[wi];
    if (pos + 64 > nd) v |= d[0] << (nd - pos);
    return v;
}

template <int MODEL>
__global__ void __launch_bounds__(kDsThreads) k_ds_x(const uint64_t* __restrict__ spins, uint32_t L, uint32_t W,
                                                     uint32_t R, const uint32_t* __restrict__ rlist, uint32_t nr,
                                                     long long* __restrict__ acc)
{
    constexpr int PL = MODEL == 0 ? 1 : 2;
    extern __shared__ __align__(16) unsigned char ds_smem[];
    const uint32_t nd = L / R;
    const uint32_t nwd = (nd + 63) / 64;
    const uint32_t stride = nwd + 1;  // one zero word after each subsequence
    uint64_t* D = reinterpret_cast<uint64_t*>(ds_smem);  // [plane][p][stride]
    long long* s_acc = reinterpret_cast<long long*>(D + (size_t)PL * R * stride);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t wfirst = blockIdx.y * kDsWarps + warp;
    const uint32_t wstep = gridDim.y * kDsWarps;
    for (uint32_t i = wfirst; i < nr; i += wstep)
        if (lane == 0) s_acc[i] = 0;

    const uint32_t nrows = L / R;
    for (uint32_t row_i = blockIdx.x; row_i < nrows; row_i += gridDim.x) {
        const uint64_t* row = spins + (size_t)row_i * R * W * PL;
        __syncthreads();  // the previous row's subsequences are no longer read
        for (uint32_t t = threadIdx.x; t < (uint32_t)PL * R * stride; t += kDsThreads) {
            const uint32_t pl = t / (R * stride), rem = t % (R * stride);
            const uint32_t p = rem / stride, m = rem % stride;
            D[t] = m < nwd ? gather_word<PL>(row + pl, W, R, p, m) : 0ull;
        }
        __syncthreads();
        const uint64_t lastmask = (nd & 63) ? (1ull << (nd & 63)) - 1 : ~0ull;
        for (uint32_t i = wfirst; i < nr; i += wstep) {
            const uint32_t r = rlist[i];
            const uint32_t p = r % R;
            const uint32_t q = (r / R) % nd;
            long long sum = 0;
            for (uint32_t m = lane; m < nwd; m += 32) {
                const uint64_t vm = m == nwd - 1 ? lastmask : ~0ull;
                uint32_t pos = 64 * m + q;
                if (pos >= nd) pos -= nd;
                if (MODEL == 0) {
                    const uint64_t a = D[m];
                    const uint64_t b = window64(D + (size_t)p * stride, pos, nd);
                    sum += __popcll((a ^ b) & vm);
                } else {
                    const uint64_t na = D[m], ga = D[(size_t)R * stride + m];
                    const uint64_t nb = window64(D + (size_t)p * stride, pos, nd);
                    const uint64_t gb = window64(D + (size_t)(R + p) * stride, pos, nd);
                    const uint64_t nn = na & nb & vm;
                    sum += __popcll(nn) - 2 * __popcll(nn & (ga ^ gb));
                }
            }
            sum = warp_total(sum);
            // Ising: the row sum is nd - 2 (number of unequal pairs)
            if (lane == 0) s_acc[i] += MODEL == 0 ? (long long)nd - 2 * sum : sum;
        }
    }
    __syncwarp();
    for (uint32_t i = wfirst; i < nr; i += wstep)
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc + i), (unsigned long long)s_acc[i]);
}

// E[y][m] = word m of the phase-0 subsequence of row y (the source columns).
template <int MODEL>
__global__ void __launch_bounds__(kDsThreads) k_ds_build_e(const uint64_t* __restrict__ spins, uint32_t L, uint32_t W,
                                                           uint32_t R, uint32_t nwe, uint64_t* __restrict__ E)
{
    constexpr int PL = MODEL == 0 ? 1 : 2;
    const uint64_t n = (uint64_t)L * nwe;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t y = t / nwe;
        const uint32_t m = (uint32_t)(t % nwe);
        const uint64_t* row = spins + y * W * PL;
#pragma unroll
        for (int pl = 0; pl < PL; ++pl) E[t * PL + pl] = gather_word<PL>(row + pl, W, R, 0, m);
    }
}

// rows: L rows of `pitch` words per plane (planes interleaved as in the
// lattice); mask selects the source bits of a word (all ones for E, whose
// padding is zero).
template <int MODEL>
__global__ void __launch_bounds__(kDsThreads) k_ds_y(const uint64_t* __restrict__ rows, uint32_t L, uint32_t pitch,
                                                     uint32_t R, uint64_t mask, const uint32_t* __restrict__ rlist,
                                                     uint32_t nr, long long* __restrict__ acc)
{
    constexpr int PL = MODEL == 0 ? 1 : 2;
    extern __shared__ __align__(16) unsigned char ds_smem[];
    long long* s_acc = reinterpret_cast<long long*>(ds_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t wfirst = blockIdx.y * kDsWarps + warp;
    const uint32_t wstep = gridDim.y * kDsWarps;
    for (uint32_t i = wfirst; i < nr; i += wstep)
        if (lane == 0) s_acc[i] = 0;
    const uint32_t nrows = L / R, nd = L / R;
    for (uint32_t row_i = blockIdx.x; row_i < nrows; row_i += gridDim.x) {
        const uint64_t y = (uint64_t)row_i * R;
        const uint64_t* a = rows + y * pitch * PL;
        for (uint32_t i = wfirst; i < nr; i += wstep) {
            uint64_t yt = y + rlist[i];
            if (yt >= L) yt -= L;
            const uint64_t* b = rows + yt * pitch * PL;
            long long sum = 0;
            for (uint32_t m = lane; m < pitch; m += 32) {
                if (MODEL == 0) {
                    sum += __popcll((__ldg(a + m) ^ __ldg(b + m)) & mask);
                } else {
                    const ulonglong2 va = __ldg(reinterpret_cast<const ulonglong2*>(a) + m);
                    const ulonglong2 vb = __ldg(reinterpret_cast<const ulonglong2*>(b) + m);
                    const uint64_t nn = va.x & vb.x & mask;
                    sum += __popcll(nn) - 2 * __popcll(nn & (va.y ^ vb.y));
                }
            }
            sum = warp_total(sum);
            if (lane == 0) s_acc[i] += MODEL == 0 ? (long long)nd - 2 * sum : sum;
        }
    }
    __syncwarp();
    for (uint32_t i = wfirst; i < nr; i += wstep)
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc + i), (unsigned long long)s_acc[i]);
}

uint64_t source_mask(uint32_t R)
{
    uint64_t m = 0;
    for (uint32_t b = 0; b < 64; b += R) m |= 1ull << b;
    return m;
}

// Grid: gx blocks over source rows, gy slices of the distance list, about
// `waves` x (resident blocks) in total.
void ds_grid(uint32_t nrows, uint32_t nr, int sms, int resident, dim3& g)
{
    const uint64_t want = (uint64_t)sms * (uint64_t)(resident < 1 ? 1 : resident) * 2;
    const uint32_t gx = (uint32_t)std::min<uint64_t>(nrows, want);
    uint64_t gy = (want + gx - 1) / gx;
    const uint64_t gymax = (nr + kDsWarps - 1) / kDsWarps;
    if (gy > gymax) gy = gymax;
    if (gy < 1) gy = 1;
    if (gy > 65535) gy = 65535;
    g = dim3(gx, (uint32_t)gy, 1);
}

template <int MODEL>
cudaError_t launch_ds_model(const void* spins, uint32_t L, uint32_t W, uint32_t R, const uint32_t* rlist,
                            uint32_t nr, long long* cx, long long* cy, uint64_t* escratch, int sms, cudaStream_t st)
{
    constexpr int PL = MODEL == 0 ? 1 : 2;
    const uint64_t* sp = static_cast<const uint64_t*>(spins);
    const uint32_t nd = L / R, nwd = (nd + 63) / 64;
    const uint32_t nrows = L / R;
    // x
    const size_t smem_x = (size_t)PL * R * (nwd + 1) * sizeof(uint64_t) + (size_t)kDsChunk * sizeof(long long);
    cudaError_t e = cudaFuncSetAttribute(k_ds_x<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x);
    if (e != cudaSuccess) return e;
    int resident = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_ds_x<MODEL>, kDsThreads, smem_x);
    if (e != cudaSuccess) return e;
    for (uint32_t c0 = 0; c0 < nr; c0 += kDsChunk) {
        const uint32_t n = std::min(kDsChunk, nr - c0);
        dim3 g;
        ds_grid(nrows, n, sms, resident, g);
        k_ds_x<MODEL><<<g, kDsThreads, smem_x, st>>>(sp, L, W, R, rlist + c0, n, cx + c0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // y
    const uint64_t* rows = sp;
    uint32_t pitch = W;
    uint64_t mask = source_mask(R);
    if (escratch) {
        const uint64_t n = (uint64_t)L * nwd;
        const int gb = (int)std::min<uint64_t>((n + kDsThreads - 1) / kDsThreads, (uint64_t)sms * 8);
        k_ds_build_e<MODEL><<<gb, kDsThreads, 0, st>>>(sp, L, W, R, nwd, escratch);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        rows = escratch;
        pitch = nwd;
        mask = ~0ull;
    }
    const size_t smem_y = (size_t)kDsChunk * sizeof(long long);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_ds_y<MODEL>, kDsThreads, smem_y);
    if (e != cudaSuccess) return e;
    for (uint32_t c0 = 0; c0 < nr; c0 += kDsChunk) {
        const uint32_t n = std::min(kDsChunk, nr - c0);
        dim3 g;
        ds_grid(nrows, n, sms, resident, g);
        k_ds_y<MODEL><<<g, kDsThreads, smem_y, st>>>(rows, L, pitch, R, mask, rlist + c0, n, cy + c0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t ds_scratch_words(int model, uint32_t L)
{
    // E for R >= kDsMinScratchR: L rows of ceil(L / R / 64) words per plane
    const uint32_t nd = L / kDsMinScratchR;
    return (size_t)L * ((nd + 63) / 64) * (model == 0 ? 1 : 2);
}

cudaError_t launch_correlation_sampled(int model, const void* spins, uint32_t L, uint32_t W, uint32_t R,
                                       const uint32_t* rlist, uint32_t nr, long long* cx, long long* cy,
                                       uint64_t* escratch, int sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cx, 0, (size_t)nr * sizeof(long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cy, 0, (size_t)nr * sizeof(long long), st);
    if (e != cudaSuccess || nr == 0) return e;
    uint64_t* es = R >= kDsMinScratchR ? escratch : nullptr;
    return model == 0 ? launch_ds_model<0>(spins, L, W, R, rlist, nr, cx, cy, es, sms, st)
                      : launch_ds_model<1>(spins, L, W, R, rlist, nr, cx, cy, es, sms, st);
}

}  // namespace latk
