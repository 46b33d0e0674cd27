// k_sweep.cu -- one checkerboard colour phase of a Metropolis sweep
// (section 3.1: spins of one colour are updated in parallel, two phases per
// step), for the Ising model (1 bit per spin, section 3.2) and the
// Blume-Capel model (2 bits per spin in two bit planes).
//
// Layout: row-major, W = L/64 words per row; bit b of word (y, j) is site
// x = 64 j + b.  Colour-c sites of row y sit at bit positions b with
// (b + y) % 2 == c, i.e. every other bit, so one phase reads whole words and
// rewrites only the active half of their bits.
//
// Work item: one chunk of CW words (CW = 2: a 128-bit load/store, 128 sites,
// 64 of them active; CW = 1 when L/64 is odd).  Consecutive lanes hold
// consecutive chunks of a row; the west/east edge words come from the
// neighbouring lanes by warp shuffles and from memory only at warp or row
// edges.  North/south words are plain loads of the rows above and below
// (served from L1/L2).  Every grid-stride iteration keeps whole warps either
// active or inactive, because the item count L * W / CW is a multiple of 32.
//
// Ising decision (section 3.2): a site with all four neighbours equal to it
// (dE = 8J) or exactly three (dE = 4J) is uphill; every other site flips
// unconditionally.  The classes come from a bit-sliced count of the four
// disagreement words (two half adders: "exactly one disagreement" and
// "none"), the same eq3/eq4 masks the paper builds with its compare-exchange
// network.  Uphill sites of a class whose threshold is neither 0 nor 2^32
// need a draw; the draw loop itself runs over every active site of the chunk
// in a fixed order (see the comment there), two independent Philox chains per
// iteration, and the per-site class is applied bit-parallel afterwards.
//
// Fused observables (colour-1 phase only): every bond has exactly one
// colour-1 end, and a colour-1 site's four neighbours are colour 0 and
// already final, so B = sum over colour-1 sites of s * h after the update;
// M and Q are summed over whole words, which are final after this phase.
#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr int kSweepThreads = 256;
constexpr uint64_t kEven = 0x5555555555555555ull;
constexpr unsigned kFull = 0xFFFFFFFFu;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void flush_obs(long long* obs, long long m, long long b, long long q)
{
    m = warp_sum(m);
    b = warp_sum(b);
    q = warp_sum(q);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsM), (unsigned long long)m);
        atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsB), (unsigned long long)b);
        atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsQ), (unsigned long long)q);
    }
}

__device__ __forceinline__ void flush_count(long long* counter, long long v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) atomicAdd(reinterpret_cast<unsigned long long*>(counter), (unsigned long long)v);
}

template <int CW, bool OBS>
__global__ void __launch_bounds__(kSweepThreads, 4) k_ising_phase(const __grid_constant__ IsingPhaseArgs a)
{
    const uint32_t cpr = a.W / CW;  // chunks per row
    const uint64_t nitems = (uint64_t)a.L * cpr;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const uint64_t all8 = a.mode8 == kAlwaysAccept ? ~0ull : 0ull;
    const uint64_t all4 = a.mode4 == kAlwaysAccept ? ~0ull : 0ull;
    const uint64_t drw8 = a.mode8 == kDraw ? ~0ull : 0ull;
    const uint64_t drw4 = a.mode4 == kDraw ? ~0ull : 0ull;
    long long accM = 0, accB = 0, accQ = 0, accD = 0;

    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nitems; item += stride) {
        const uint32_t y = (uint32_t)(item / cpr);
        const uint32_t ch = (uint32_t)(item - (uint64_t)y * cpr);
        const uint32_t yn = y == 0 ? a.L - 1 : y - 1;
        const uint32_t ys = y + 1 == a.L ? 0 : y + 1;
        uint64_t* row = a.spins + (uint64_t)y * a.W;
        const uint64_t* rown = a.spins + (uint64_t)yn * a.W;
        const uint64_t* rows = a.spins + (uint64_t)ys * a.W;

        uint64_t c[CW], n[CW], s[CW];
        if constexpr (CW == 2) {
            const ulonglong2 vc = reinterpret_cast<const ulonglong2*>(row)[ch];
            const ulonglong2 vn = reinterpret_cast<const ulonglong2*>(rown)[ch];
            const ulonglong2 vs = reinterpret_cast<const ulonglong2*>(rows)[ch];
            c[0] = vc.x; c[1] = vc.y; n[0] = vn.x; n[1] = vn.y; s[0] = vs.x; s[1] = vs.y;
        } else {
            c[0] = row[ch]; n[0] = rown[ch]; s[0] = rows[ch];
        }
        uint64_t left = __shfl_up_sync(kFull, c[CW - 1], 1);
        uint64_t right = __shfl_down_sync(kFull, c[0], 1);
        if (lane == 0 || ch == 0) left = row[ch == 0 ? a.W - 1 : ch * CW - 1];
        if (lane == 31 || ch + 1 == cpr) right = row[ch + 1 == cpr ? 0 : (ch + 1) * CW];

        uint64_t w[CW], e[CW];
        if constexpr (CW == 2) {
            w[0] = (c[0] << 1) | (left >> 63);
            w[1] = (c[1] << 1) | (c[0] >> 63);
            e[0] = (c[0] >> 1) | (c[1] << 63);
            e[1] = (c[1] >> 1) | (right << 63);
        } else {
            w[0] = (c[0] << 1) | (left >> 63);
            e[0] = (c[0] >> 1) | (right << 63);
        }

        const uint32_t p = (y + a.colour) & 1u;
        const uint64_t amask = kEven << p;
        uint64_t flip[CW], u8[CW], need[CW];
        int dpre = 0;  // disagreeing bonds of active sites after the flips decided without a draw
#pragma unroll
        for (int k = 0; k < CW; ++k) {
            const uint64_t dn = c[k] ^ n[k], ds = c[k] ^ s[k], dw = c[k] ^ w[k], de = c[k] ^ e[k];
            const uint64_t x1 = dn ^ ds, a1 = dn & ds;
            const uint64_t x2 = dw ^ de, a2 = dw & de;
            const uint64_t eq3 = (x1 ^ x2) & ~(a1 | a2);  // exactly one neighbour differs
            const uint64_t eq4 = ~(dn | ds | dw | de);    // none differs
            u8[k] = eq4 & amask;
            const uint64_t u4 = eq3 & amask;
            flip[k] = (amask & ~(eq4 | eq3)) | (u8[k] & all8) | (u4 & all4);
            need[k] = (u8[k] & drw8) | (u4 & drw4);
            if constexpr (OBS) {
                const uint64_t f = flip[k];
                dpre += __popcll((dn ^ f) & amask) + __popcll((ds ^ f) & amask) + __popcll((dw ^ f) & amask) +
                        __popcll((de ^ f) & amask);
            }
        }

        // Draws.  In SIMT a warp instruction costs its issue slot whatever its
        // active mask, and across 32 chunks some lane almost always needs any
        // given site position, so skipping individual sites saves nothing: every
        // active site of the chunk draws, in a fixed order with no per-site
        // bookkeeping, and is compared with both uphill thresholds.  The class
        // and mode of each site are applied afterwards, 64 sites at a time.
        accD += __popcll(need[0]) + (CW == 2 ? __popcll(need[CW - 1]) : 0);
        if (__any_sync(kFull, (need[0] | need[CW - 1]) != 0)) {
            const uint64_t base = (uint64_t)y * a.L + (uint64_t)ch * (64u * CW);
            const uint32_t site0 = (uint32_t)base + p;  // chunks never straddle 2^32 (64*CW | 2^32)
            const PhiloxChunk pc = philox_chunk((uint32_t)(base >> 32), a.sweep, a.colour, a.rk);
            uint32_t r4[CW][2], r8[CW][2];  // [word][32-bit half]: u < thr4, u < thr8
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t acc4[CW], acc8[CW];
#pragma unroll
                for (int k = 0; k < CW; ++k) acc4[k] = acc8[k] = 0;
                uint32_t bit = 1u << p;
#pragma unroll 2
                for (uint32_t j = 0; j < 16; ++j) {
                    const uint32_t off = 32u * half + 2u * j;
#pragma unroll
                    for (int k = 0; k < CW; ++k) {
                        const uint32_t u = philox_site_w0(site0 + 64u * k + off, pc, a.rk);
                        acc4[k] |= u < a.thr4 ? bit : 0u;
                        acc8[k] |= u < a.thr8 ? bit : 0u;
                    }
                    bit <<= 2;
                }
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    r4[k][half] = acc4[k];
                    r8[k][half] = acc8[k];
                }
            }
#pragma unroll
            for (int k = 0; k < CW; ++k) {
                const uint64_t R4 = ((uint64_t)r4[k][1] << 32) | r4[k][0];
                const uint64_t R8 = ((uint64_t)r8[k][1] << 32) | r8[k][0];
                const uint64_t acc8 = need[k] & u8[k] & R8, acc4 = need[k] & ~u8[k] & R4;
                flip[k] |= acc8 | acc4;
                // an accepted 3-agree site goes from 1 to 3 disagreeing bonds, a 4-agree site from 0 to 4
                if constexpr (OBS) dpre += 2 * __popcll(acc4) + 4 * __popcll(acc8);
            }
        }

        uint64_t cn[CW];
#pragma unroll
        for (int k = 0; k < CW; ++k) cn[k] = c[k] ^ flip[k];
        if constexpr (CW == 2) {
            reinterpret_cast<ulonglong2*>(row)[ch] = make_ulonglong2(cn[0], cn[1]);
        } else {
            row[ch] = cn[0];
        }

        if constexpr (OBS) {
            accB += 128 * CW - 2 * dpre;  // 32 active sites x 4 bonds per word
#pragma unroll
            for (int k = 0; k < CW; ++k) accM += 2 * __popcll(cn[k]) - 64;
            accQ += 64 * CW;
        }
    }
    if constexpr (OBS) flush_obs(a.obs, accM, accB, accQ);
    if (a.draws) flush_count(a.draws, accD);
}

// Three-bit sum of four one-bit words (bit-sliced): returns b0 + 2 b1 + 4 b2.
__device__ __forceinline__ void add4(uint64_t a, uint64_t b, uint64_t c, uint64_t d, uint64_t& b0,
                                     uint64_t& b1, uint64_t& b2)
{
    const uint64_t s1 = a ^ b, c1 = a & b;
    const uint64_t s2 = c ^ d, c2 = c & d;
    b0 = s1 ^ s2;
    const uint64_t c3 = s1 & s2;
    b1 = c1 ^ c2 ^ c3;
    b2 = (c1 & c2) | (c1 & c3) | (c2 & c3);
}

// New (n, g) code after accepting the proposal: index (s+1)*2 + b, two bits
// (n | g << 1) per entry.  s=-1: {0, +1}; s=0: {-1, +1}; s=+1: {-1, 0}.
constexpr uint32_t kBcNewCode = (0u << 0) | (1u << 2) | (3u << 4) | (1u << 6) | (3u << 8) | (0u << 10);

template <bool OBS>
__global__ void __launch_bounds__(kSweepThreads) k_bc_phase(const __grid_constant__ BcPhaseArgs a)
{
    __shared__ unsigned long long s_thr[54];
    for (int i = threadIdx.x; i < 54; i += blockDim.x) s_thr[i] = a.thr[i];
    __syncthreads();

    const uint64_t nitems = (uint64_t)a.L * a.W;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    long long accM = 0, accB = 0, accQ = 0;

    for (uint64_t item = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; item < nitems; item += stride) {
        const uint32_t y = (uint32_t)(item / a.W);
        const uint32_t j = (uint32_t)(item - (uint64_t)y * a.W);
        const uint32_t yn = y == 0 ? a.L - 1 : y - 1;
        const uint32_t ys = y + 1 == a.L ? 0 : y + 1;
        ulonglong2* row = a.spins + (uint64_t)y * a.W;
        const ulonglong2 c = row[j];
        const ulonglong2 vn = a.spins[(uint64_t)yn * a.W + j];
        const ulonglong2 vs = a.spins[(uint64_t)ys * a.W + j];
        ulonglong2 left, right;
        left.x = __shfl_up_sync(kFull, c.x, 1);
        left.y = __shfl_up_sync(kFull, c.y, 1);
        right.x = __shfl_down_sync(kFull, c.x, 1);
        right.y = __shfl_down_sync(kFull, c.y, 1);
        if (lane == 0 || j == 0) left = row[j == 0 ? a.W - 1 : j - 1];
        if (lane == 31 || j + 1 == a.W) right = row[j + 1 == a.W ? 0 : j + 1];

        // Neighbour planes: n (nonzero) and g (negative).
        const uint64_t nw = (c.x << 1) | (left.x >> 63), gw = (c.y << 1) | (left.y >> 63);
        const uint64_t ne = (c.x >> 1) | (right.x << 63), ge = (c.y >> 1) | (right.y << 63);
        uint64_t p0, p1, p2, q0, q1, q2;
        add4(vn.x & ~vn.y, vs.x & ~vs.y, nw & ~gw, ne & ~ge, p0, p1, p2);  // +1 neighbours
        add4(vn.x & vn.y, vs.x & vs.y, nw & gw, ne & ge, q0, q1, q2);      // -1 neighbours

        const uint32_t p = (y + a.colour) & 1u;
        const uint64_t base = (uint64_t)y * a.L + (uint64_t)j * 64u;
        const uint32_t base_lo = (uint32_t)base;
        const PhiloxChunk pc = philox_chunk((uint32_t)(base >> 32), a.sweep, a.colour, a.rk);
        uint64_t nn = c.x, gg = c.y;
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const uint32_t b = 2u * k + p;
            const uint32_t sn = (uint32_t)(c.x >> b) & 1u, sg = (uint32_t)(c.y >> b) & 1u;
            const uint32_t sidx = sn ? (sg ? 0u : 2u) : 1u;  // s + 1
            const uint32_t P = ((uint32_t)(p0 >> b) & 1u) | (((uint32_t)(p1 >> b) & 1u) << 1) |
                               (((uint32_t)(p2 >> b) & 1u) << 2);
            const uint32_t Nn = ((uint32_t)(q0 >> b) & 1u) | (((uint32_t)(q1 >> b) & 1u) << 1) |
                                (((uint32_t)(q2 >> b) & 1u) << 2);
            const uint32_t h4 = 4u + P - Nn;
            const uint2 r = philox_site_w01(base_lo + b, pc, a.rk);
            const uint32_t bp = r.y & 1u;
            const uint32_t mv = sidx * 2u + bp;
            if ((unsigned long long)r.x < s_thr[mv * 9u + h4]) {
                const uint32_t code = (kBcNewCode >> (2u * mv)) & 3u;
                const uint64_t bit = 1ull << b;
                nn = (nn & ~bit) | ((uint64_t)(code & 1u) << b);
                gg = (gg & ~bit) | ((uint64_t)(code >> 1) << b);
            }
        }
        row[j] = make_ulonglong2(nn, gg);

        if constexpr (OBS) {
            const uint64_t amask = kEven << p;
            const uint64_t na = nn & amask;
            const uint64_t nbn[4] = {vn.x, vs.x, nw, ne}, nbg[4] = {vn.y, vs.y, gw, ge};
            long long b = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const uint64_t both = na & nbn[d];
                b += __popcll(both) - 2 * __popcll(both & (gg ^ nbg[d]));
            }
            accB += b;
            accM += __popcll(nn & ~gg) - __popcll(nn & gg);
            accQ += __popcll(nn);
        }
    }
    if constexpr (OBS) flush_obs(a.obs, accM, accB, accQ);
    if (a.draws) {
        const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const long long mine = first < nitems ? (long long)((nitems - 1 - first) / stride + 1) * 32 : 0;
        flush_count(a.draws, mine);
    }
}

template <typename K>
int blocks_for(K kernel, uint64_t nitems, int sms, int bpsm)
{
    (void)kernel;
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
    if (ls.ising_bpsm < 1) ls.ising_bpsm = 1;
    if (ls.bc_bpsm < 1) ls.bc_bpsm = 1;
    return e;
}

cudaError_t launch_ising_phase(const IsingPhaseArgs& a, const LaunchShape& ls, cudaStream_t st)
{
    const bool even_words = (a.W % 2) == 0;
    const uint64_t nitems = (uint64_t)a.L * (even_words ? a.W / 2 : a.W);
    const int grid = blocks_for(0, nitems, ls.sms, ls.ising_bpsm);
    if (even_words) {
        if (a.obs) k_ising_phase<2, true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_ising_phase<2, false><<<grid, kSweepThreads, 0, st>>>(a);
    } else {
        if (a.obs) k_ising_phase<1, true><<<grid, kSweepThreads, 0, st>>>(a);
        else k_ising_phase<1, false><<<grid, kSweepThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_bc_phase(const BcPhaseArgs& a, const LaunchShape& ls, cudaStream_t st)
{
    const uint64_t nitems = (uint64_t)a.L * a.W;
    const int grid = blocks_for(0, nitems, ls.sms, ls.bc_bpsm);
    if (a.obs) k_bc_phase<true><<<grid, kSweepThreads, 0, st>>>(a);
    else k_bc_phase<false><<<grid, kSweepThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace latk
