// k_lattice.cu -- initial quench, whole-lattice reductions, canonical hash
// and int8 row transfers for the packed lattices of k_sweep.cu.
//
// All kernels here are HBM-bound passes over the packed lattice (or
// Philox-bound for the quench); each thread owns one 64-site word (Ising) or
// one 64-site (n, g) word pair (Blume-Capel).
#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr int kThreads = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

int grid_for(uint64_t n, int sms, int per_sm)
{
    const uint64_t need = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)sms * (uint64_t)per_sm;
    return (int)(need < cap ? (need == 0 ? 1 : need) : cap);
}

// Infinite-temperature quench (section 1: the system starts at high
// temperature).  Counter (site, quench sweep index, colour 0); Ising spin +1
// iff bit 31 of word 0; Blume-Capel value floor(3 w0 / 2^32) - 1.
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_init(void* spins, uint32_t L, uint32_t W, const __grid_constant__ RoundKeys rk)
{
    const uint64_t nwords = (uint64_t)L * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t y = (uint32_t)(i / W), j = (uint32_t)(i - (uint64_t)y * W);
        const uint64_t base = (uint64_t)y * L + 64ull * j;
        const PhiloxChunk pc = philox_chunk((uint32_t)(base >> 32), kQuenchSweep, 0u, rk);
        const uint32_t base_lo = (uint32_t)base;
        if constexpr (MODEL == 0) {
            uint64_t w = 0;
            for (uint32_t b = 0; b < 64; ++b) w |= (uint64_t)(philox_site_w0(base_lo + b, pc, rk) >> 31) << b;
            static_cast<uint64_t*>(spins)[i] = w;
        } else {
            uint64_t n = 0, g = 0;
            for (uint32_t b = 0; b < 64; ++b) {
                const uint32_t v = (uint32_t)(((uint64_t)philox_site_w0(base_lo + b, pc, rk) * 3ull) >> 32);
                n |= (uint64_t)(v != 1u) << b;
                g |= (uint64_t)(v == 0u) << b;
            }
            static_cast<ulonglong2*>(spins)[i] = make_ulonglong2(n, g);
        }
    }
}

// (M, B, Q) of Eqs. (1)-(2): bonds to the east and south neighbours of every
// site, each bond once.
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_measure(const void* spins, uint32_t L, uint32_t W, long long* out)
{
    long long m = 0, b = 0, q = 0;
    const uint64_t nwords = (uint64_t)L * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t y = (uint32_t)(i / W), j = (uint32_t)(i - (uint64_t)y * W);
        const uint64_t ir = (uint64_t)y * W + (j + 1 == W ? 0 : j + 1);
        const uint64_t id = (uint64_t)(y + 1 == L ? 0 : y + 1) * W + j;
        if constexpr (MODEL == 0) {
            const uint64_t* s = static_cast<const uint64_t*>(spins);
            const uint64_t c = s[i], e = (c >> 1) | (s[ir] << 63), d = s[id];
            b += 128 - 2 * (__popcll(c ^ e) + __popcll(c ^ d));
            m += 2 * __popcll(c) - 64;
            q += 64;
        } else {
            const ulonglong2* s = static_cast<const ulonglong2*>(spins);
            const ulonglong2 c = s[i], r = s[ir], d = s[id];
            const uint64_t ne = (c.x >> 1) | (r.x << 63), ge = (c.y >> 1) | (r.y << 63);
            const uint64_t be = c.x & ne, bd = c.x & d.x;
            b += __popcll(be) - 2 * __popcll(be & (c.y ^ ge)) + __popcll(bd) - 2 * __popcll(bd & (c.y ^ d.y));
            m += __popcll(c.x & ~c.y) - __popcll(c.x & c.y);
            q += __popcll(c.x);
        }
    }
    m = warp_sum(m); b = warp_sum(b); q = warp_sum(q);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 0), (unsigned long long)m);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)b);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 2), (unsigned long long)q);
    }
}

// Number of sites holding each spin value (the consistency check of the
// paper's runs: the counts of -1, 0 and +1 add up to L^2), and the number of
// Blume-Capel words' 2-bit codes that are not a spin (g set without n).
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_spin_counts(const void* spins, uint32_t L, uint32_t W, long long* out)
{
    long long neg = 0, zero = 0, pos = 0, bad = 0;
    const uint64_t nwords = (uint64_t)L * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if constexpr (MODEL == 0) {
            const int up = __popcll(static_cast<const uint64_t*>(spins)[i]);
            pos += up;
            neg += 64 - up;
        } else {
            const ulonglong2 c = static_cast<const ulonglong2*>(spins)[i];
            pos += __popcll(c.x & ~c.y);
            neg += __popcll(c.x & c.y);
            zero += __popcll(~c.x & ~c.y);
            bad += __popcll(~c.x & c.y);
        }
    }
    neg = warp_sum(neg); zero = warp_sum(zero); pos = warp_sum(pos); bad = warp_sum(bad);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 0), (unsigned long long)neg);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 1), (unsigned long long)zero);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 2), (unsigned long long)pos);
        atomicAdd(reinterpret_cast<unsigned long long*>(out + 3), (unsigned long long)bad);
    }
}

// Histogram of s_x * h_x (Eq. (3)), bins v = -4..4 at v + 4, added to hist,
// over the sites of the colours in the bit mask `colours` (1: x+y even,
// 2: x+y odd, 3: every site).
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_sd_hist(const void* spins, uint32_t L, uint32_t W, long long* hist,
                                                     uint32_t colours)
{
    long long hcount[9];
#pragma unroll
    for (int v = 0; v < 9; ++v) hcount[v] = 0;
    const uint64_t nwords = (uint64_t)L * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t y = (uint32_t)(i / W), j = (uint32_t)(i - (uint64_t)y * W);
        // sites of colour c in row y sit at the bit positions b with (b + y) % 2 == c
        const uint64_t cm = colours == 3u ? ~0ull : 0x5555555555555555ull << ((y + (colours == 2u ? 1u : 0u)) & 1u);
        const uint64_t il = (uint64_t)y * W + (j == 0 ? W - 1 : j - 1);
        const uint64_t ir = (uint64_t)y * W + (j + 1 == W ? 0 : j + 1);
        const uint64_t iu = (uint64_t)(y == 0 ? L - 1 : y - 1) * W + j;
        const uint64_t id = (uint64_t)(y + 1 == L ? 0 : y + 1) * W + j;
        if constexpr (MODEL == 0) {
            const uint64_t* s = static_cast<const uint64_t*>(spins);
            const uint64_t c = s[i];
            const uint64_t dw = c ^ ((c << 1) | (s[il] >> 63)), de = c ^ ((c >> 1) | (s[ir] << 63));
            const uint64_t dn = c ^ s[iu], ds = c ^ s[id];
            // number of disagreeing neighbours d = 0..4, and s*h = 4 - 2d
            const uint64_t s1 = dn ^ ds, c1 = dn & ds, s2 = dw ^ de, c2 = dw & de;
            const uint64_t d0 = s1 ^ s2, c3 = s1 & s2;
            const uint64_t d1 = c1 ^ c2 ^ c3, d2 = (c1 & c2) | (c1 & c3) | (c2 & c3);
            hcount[8] += __popcll(~(d0 | d1 | d2) & cm);
            hcount[6] += __popcll(d0 & ~d1 & ~d2 & cm);
            hcount[4] += __popcll(~d0 & d1 & ~d2 & cm);
            hcount[2] += __popcll(d0 & d1 & ~d2 & cm);
            hcount[0] += __popcll(d2 & cm);
        } else {
            const ulonglong2* s = static_cast<const ulonglong2*>(spins);
            const ulonglong2 c = s[i], l = s[il], r = s[ir], u = s[iu], d = s[id];
            const uint64_t nw = (c.x << 1) | (l.x >> 63), gw = (c.y << 1) | (l.y >> 63);
            const uint64_t ne = (c.x >> 1) | (r.x << 63), ge = (c.y >> 1) | (r.y << 63);
            for (int bpos = 0; bpos < 64; ++bpos) {
                if (!((cm >> bpos) & 1)) continue;
                const int sv = ((c.x >> bpos) & 1) ? (((c.y >> bpos) & 1) ? -1 : 1) : 0;
                if (sv == 0) {
                    hcount[4] += 1;
                    continue;
                }
                int h = 0;
                const uint64_t nb[4] = {u.x, d.x, nw, ne}, gb[4] = {u.y, d.y, gw, ge};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((nb[k] >> bpos) & 1) h += ((gb[k] >> bpos) & 1) ? -1 : 1;
                hcount[sv * h + 4] += 1;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 9; ++v) {
        const long long t = warp_sum(hcount[v]);
        if ((threadIdx.x & 31) == 0 && t) atomicAdd(reinterpret_cast<unsigned long long*>(hist + v), (unsigned long long)t);
    }
}

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_hash(const void* spins, uint32_t L, uint32_t W, unsigned long long* out)
{
    uint64_t h = 0;
    const uint64_t nwords = (uint64_t)L * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if constexpr (MODEL == 0) {
            h += mix64(i ^ static_cast<const uint64_t*>(spins)[i]);
        } else {
            const ulonglong2 v = static_cast<const ulonglong2*>(spins)[i];
            h += mix64(i ^ v.x) + mix64((nwords + i) ^ v.y);
        }
    }
    h = warp_sum(h);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)h);
}

// Rows y0 .. y0+nrows-1 (mod L) to int8 values, one thread per word.
template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_unpack_rows(const void* spins, uint32_t L, uint32_t W, uint32_t y0,
                                                          uint32_t nrows, int8_t* out)
{
    const uint64_t n = (uint64_t)nrows * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(i / W), j = (uint32_t)(i - (uint64_t)r * W);
        const uint32_t y = (uint32_t)(((uint64_t)y0 + r) % L);
        uint64_t nw, gw;
        if constexpr (MODEL == 0) {
            nw = static_cast<const uint64_t*>(spins)[(uint64_t)y * W + j];
        } else {
            const ulonglong2 v = static_cast<const ulonglong2*>(spins)[(uint64_t)y * W + j];
            nw = v.x;
            gw = v.y;
        }
        uint64_t* dst = reinterpret_cast<uint64_t*>(out + (uint64_t)r * L + 64ull * j);
        for (int k = 0; k < 8; ++k) {
            uint64_t bytes = 0;
            for (int t = 0; t < 8; ++t) {
                const int b = 8 * k + t;
                int v;
                if constexpr (MODEL == 0) v = ((nw >> b) & 1) ? 1 : -1;
                else v = ((nw >> b) & 1) ? (((gw >> b) & 1) ? -1 : 1) : 0;
                bytes |= (uint64_t)(uint8_t)(int8_t)v << (8 * t);
            }
            dst[k] = bytes;
        }
    }
}

template <int MODEL>
__global__ void __launch_bounds__(kThreads) k_pack_rows(void* spins, uint32_t L, uint32_t W, uint32_t y0,
                                                        uint32_t nrows, const int8_t* in, unsigned int* bad)
{
    const uint64_t n = (uint64_t)nrows * W;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(i / W), j = (uint32_t)(i - (uint64_t)r * W);
        const uint32_t y = (uint32_t)(((uint64_t)y0 + r) % L);
        const int8_t* src = in + (uint64_t)r * L + 64ull * j;
        uint64_t nw = 0, gw = 0;
        bool ok = true;
        for (int b = 0; b < 64; ++b) {
            const int v = src[b];
            if constexpr (MODEL == 0) {
                ok &= (v == 1 || v == -1);
                nw |= (uint64_t)(v == 1) << b;
            } else {
                ok &= (v >= -1 && v <= 1);
                nw |= (uint64_t)(v != 0) << b;
                gw |= (uint64_t)(v == -1) << b;
            }
        }
        if (!ok) atomicOr(bad, 1u);
        if constexpr (MODEL == 0) static_cast<uint64_t*>(spins)[(uint64_t)y * W + j] = nw;
        else static_cast<ulonglong2*>(spins)[(uint64_t)y * W + j] = make_ulonglong2(nw, gw);
    }
}

}  // namespace

cudaError_t launch_init(int model, void* spins, uint32_t L, uint32_t W, const RoundKeys& rk, int sms, cudaStream_t st)
{
    const int grid = grid_for((uint64_t)L * W, sms, 8);
    if (model == 0) k_init<0><<<grid, kThreads, 0, st>>>(spins, L, W, rk);
    else k_init<1><<<grid, kThreads, 0, st>>>(spins, L, W, rk);
    return cudaGetLastError();
}

cudaError_t launch_measure(int model, const void* spins, uint32_t L, uint32_t W, long long* out3, int sms,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out3, 0, 3 * sizeof(long long), st);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((uint64_t)L * W, sms, 8);
    if (model == 0) k_measure<0><<<grid, kThreads, 0, st>>>(spins, L, W, out3);
    else k_measure<1><<<grid, kThreads, 0, st>>>(spins, L, W, out3);
    return cudaGetLastError();
}

cudaError_t launch_spin_counts(int model, const void* spins, uint32_t L, uint32_t W, long long* out4, int sms,
                               cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out4, 0, 4 * sizeof(long long), st);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((uint64_t)L * W, sms, 8);
    if (model == 0) k_spin_counts<0><<<grid, kThreads, 0, st>>>(spins, L, W, out4);
    else k_spin_counts<1><<<grid, kThreads, 0, st>>>(spins, L, W, out4);
    return cudaGetLastError();
}

cudaError_t launch_sd_hist_add(int model, const void* spins, uint32_t L, uint32_t W, long long* hist9,
                               uint32_t colours, int sms, cudaStream_t st)
{
    const int grid = grid_for((uint64_t)L * W, sms, 8);
    if (model == 0) k_sd_hist<0><<<grid, kThreads, 0, st>>>(spins, L, W, hist9, colours);
    else k_sd_hist<1><<<grid, kThreads, 0, st>>>(spins, L, W, hist9, colours);
    return cudaGetLastError();
}

cudaError_t launch_sd_hist(int model, const void* spins, uint32_t L, uint32_t W, long long* hist9, int sms,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist9, 0, 9 * sizeof(long long), st);
    if (e != cudaSuccess) return e;
    return launch_sd_hist_add(model, spins, L, W, hist9, 3u, sms, st);
}

cudaError_t launch_hash(int model, const void* spins, uint32_t L, uint32_t W, unsigned long long* out, int sms,
                        cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((uint64_t)L * W, sms, 8);
    if (model == 0) k_hash<0><<<grid, kThreads, 0, st>>>(spins, L, W, out);
    else k_hash<1><<<grid, kThreads, 0, st>>>(spins, L, W, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_rows(int model, const void* spins, uint32_t L, uint32_t W, uint32_t y0, uint32_t nrows,
                               int8_t* out, cudaStream_t st)
{
    const int grid = grid_for((uint64_t)nrows * W, 152, 8);
    if (model == 0) k_unpack_rows<0><<<grid, kThreads, 0, st>>>(spins, L, W, y0, nrows, out);
    else k_unpack_rows<1><<<grid, kThreads, 0, st>>>(spins, L, W, y0, nrows, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_rows(int model, void* spins, uint32_t L, uint32_t W, uint32_t y0, uint32_t nrows,
                             const int8_t* in, unsigned int* bad, cudaStream_t st)
{
    const int grid = grid_for((uint64_t)nrows * W, 152, 8);
    if (model == 0) k_pack_rows<0><<<grid, kThreads, 0, st>>>(spins, L, W, y0, nrows, in, bad);
    else k_pack_rows<1><<<grid, kThreads, 0, st>>>(spins, L, W, y0, nrows, in, bad);
    return cudaGetLastError();
}

}  // namespace latk
