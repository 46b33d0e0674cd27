// sweep_item.cuh -- the update of one work item of a checkerboard colour
// phase (section 3.1), shared by the one-lattice kernels (k_sweep.cu) and the
// persistent multi-lattice kernel (k_multi in lat_multi.cu), so that both produce the same
// bits from the same counters.
//
// Layout: row-major, W = L/64 words per row; bit b of word (y, j) is site
// x = 64 j + b.  Colour-c sites of row y sit at bit positions b with
// (b + y) % 2 == c.  An Ising item is a chunk of CW words (CW = 2: one 128-bit
// access, 128 sites of which 64 are active; CW = 1 when L/64 is odd); a
// Blume-Capel item is one (n, g) word pair (64 sites, 32 active).
//
// Consecutive lanes of a warp must hold consecutive items of the same phase,
// and a warp's lanes must be all active or all inactive: the west/east edge
// words are exchanged by warp shuffles.
//
// CG selects L2-coherent loads (ld.global.cg).  The one-lattice kernels
// read a lattice that no other block of the same launch writes between
// their kernel boundaries, so plain loads are safe; the persistent kernel
// runs many phases in one launch, and a block may read a row it cached in
// L1 during an earlier phase, so it bypasses L1.
#pragma once
#include "sweep_args.cuh"

namespace latk {

constexpr uint64_t kEvenBits = 0x5555555555555555ull;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFullMask, v, o);
    return v;
}

template <bool CG, typename T>
__device__ __forceinline__ T ld(const T* p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Per-thread partial sums of one phase: (M, B, Q) of the fused reduction
// and the number of Philox draws the phase needed; with the fused
// Schwinger-Dyson histogram, the counts of the phase's active sites by
// s_x * h_x (bin v + 4, v = -4..4).  Per thread these stay far below 2^31
// (a grid-stride thread visits at most a few million sites).
struct PhaseAcc {
    long long M = 0, B = 0, Q = 0, D = 0;
    int sd[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

// Add one thread's histogram to the 9 device counters hist (one atomic per
// bin and warp).
__device__ __forceinline__ void flush_sd(long long* hist, const PhaseAcc& a)
{
#pragma unroll
    for (int v = 0; v < 9; ++v) {
        const long long c = warp_sum((long long)a.sd[v]);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(reinterpret_cast<unsigned long long*>(hist + v), (unsigned long long)c);
    }
}

__device__ __forceinline__ void flush_acc(long long* obs, long long* draws, PhaseAcc a)
{
    if (obs) {
        const long long m = warp_sum(a.M), b = warp_sum(a.B), q = warp_sum(a.Q);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsM), (unsigned long long)m);
            atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsB), (unsigned long long)b);
            atomicAdd(reinterpret_cast<unsigned long long*>(obs + kObsQ), (unsigned long long)q);
        }
    }
    if (draws) {
        const long long d = warp_sum(a.D);
        if ((threadIdx.x & 31) == 0) atomicAdd(reinterpret_cast<unsigned long long*>(draws), (unsigned long long)d);
    }
}

// Parameters of one Ising colour phase.
struct IsingPhase {
    uint64_t* spins;
    uint32_t L, W;
    uint32_t sweep, colour;
    uint32_t thr4, thr8;    // thresholds for s*h = 2 and s*h = 4
    uint32_t mode4, mode8;  // ClassMode of the two uphill classes
};

// Ising decision (section 3.2): a site with all four neighbours equal to it
// (dE = 8J) or exactly three (dE = 4J) is uphill; every other site flips
// unconditionally.  The classes come from a bit-sliced count of the four
// disagreement words (two half adders: "exactly one disagreement" and
// "none"), the same eq3/eq4 masks the paper builds with its compare-exchange
// network.  Uphill sites of a class whose threshold is neither 0 nor 2^32
// need a draw.  In SIMT a warp instruction costs its issue slot whatever its
// active mask, and across 32 chunks some lane almost always needs any given
// site position, so skipping individual sites saves nothing: every active
// site of the chunk draws, in a fixed order with no per-site bookkeeping
// (two independent Philox chains per iteration), and is compared with both
// uphill thresholds; the class and mode of each site are applied afterwards,
// 64 sites at a time.
//
// Fused observables (colour-1 phase, OBS): every bond has exactly one
// colour-1 end, and a colour-1 site's four neighbours are colour 0 and
// already final, so B = sum over colour-1 sites of s * h after the update;
// M and Q are summed over whole words, which are final after this phase.
// Loads, neighbour words and uphill classes of one Ising item, shared by
// both random-number modes.
template <int CW>
struct IsingItem {
    uint64_t* row;
    uint32_t y, ch, p;
    uint64_t amask;
    uint64_t c[CW], flip[CW], u8[CW], u4[CW];
    int dpre;  // disagreeing bonds of active sites after the flips decided so far
    int n2, n3, n4;  // SD: active sites with 2, 3, 4 disagreeing neighbours (they flip whatever is drawn)
};

template <int CW, bool OBS, bool CG, bool SD = false>
__device__ __forceinline__ void ising_classify(const IsingPhase& a, uint64_t item, int lane, bool modes,
                                               IsingItem<CW>& it)
{
    const uint32_t cpr = a.W / CW;  // chunks per row
    const uint64_t all8 = modes && a.mode8 == kAlwaysAccept ? ~0ull : 0ull;
    const uint64_t all4 = modes && a.mode4 == kAlwaysAccept ? ~0ull : 0ull;
    it.y = (uint32_t)(item / cpr);
    it.ch = (uint32_t)(item - (uint64_t)it.y * cpr);
    const uint32_t y = it.y, ch = it.ch;
    const uint32_t yn = y == 0 ? a.L - 1 : y - 1;
    const uint32_t ys = y + 1 == a.L ? 0 : y + 1;
    uint64_t* row = a.spins + (uint64_t)y * a.W;
    it.row = row;
    const uint64_t* rown = a.spins + (uint64_t)yn * a.W;
    const uint64_t* rows = a.spins + (uint64_t)ys * a.W;

    uint64_t n[CW], s[CW];
    uint64_t* c = it.c;
    if constexpr (CW == 2) {
        const ulonglong2 vc = ld<CG>(reinterpret_cast<const ulonglong2*>(row) + ch);
        const ulonglong2 vn = ld<CG>(reinterpret_cast<const ulonglong2*>(rown) + ch);
        const ulonglong2 vs = ld<CG>(reinterpret_cast<const ulonglong2*>(rows) + ch);
        c[0] = vc.x; c[1] = vc.y; n[0] = vn.x; n[1] = vn.y; s[0] = vs.x; s[1] = vs.y;
    } else {
        c[0] = ld<CG>(row + ch); n[0] = ld<CG>(rown + ch); s[0] = ld<CG>(rows + ch);
    }
    uint64_t left = __shfl_up_sync(kFullMask, c[CW - 1], 1);
    uint64_t right = __shfl_down_sync(kFullMask, c[0], 1);
    if (lane == 0 || ch == 0) left = ld<CG>(row + (ch == 0 ? a.W - 1 : ch * CW - 1));
    if (lane == 31 || ch + 1 == cpr) right = ld<CG>(row + (ch + 1 == cpr ? 0 : (ch + 1) * CW));

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

    it.p = (y + a.colour) & 1u;
    const uint64_t amask = kEvenBits << it.p;
    it.amask = amask;
    it.dpre = 0;
    it.n2 = it.n3 = it.n4 = 0;
#pragma unroll
    for (int k = 0; k < CW; ++k) {
        const uint64_t dn = c[k] ^ n[k], ds = c[k] ^ s[k], dw = c[k] ^ w[k], de = c[k] ^ e[k];
        const uint64_t x1 = dn ^ ds, a1 = dn & ds;
        const uint64_t x2 = dw ^ de, a2 = dw & de;
        if constexpr (SD) {
            // disagreements d = (x1 + 2 a1) + (x2 + 2 a2): d = 4, 3, 2
            it.n4 += __popcll(a1 & a2 & amask);
            it.n3 += __popcll(((a1 & x2) | (a2 & x1)) & amask);
            it.n2 += __popcll(((x1 & x2) | (a1 & ~(x2 | a2)) | (a2 & ~(x1 | a1))) & amask);
        }
        const uint64_t eq3 = (x1 ^ x2) & ~(a1 | a2);  // exactly one neighbour differs
        const uint64_t eq4 = ~(dn | ds | dw | de);    // none differs
        it.u8[k] = eq4 & amask;
        it.u4[k] = eq3 & amask;
        it.flip[k] = (amask & ~(eq4 | eq3)) | (it.u8[k] & all8) | (it.u4[k] & all4);
        if constexpr (OBS) {
            const uint64_t f = it.flip[k];
            it.dpre += __popcll((dn ^ f) & amask) + __popcll((ds ^ f) & amask) + __popcll((dw ^ f) & amask) +
                       __popcll((de ^ f) & amask);
        }
    }
}

// Store the new words and add the fused observables.  SD: the histogram
// of s h = 4 - 2 d over the item's active sites, d the number of
// disagreeing neighbours: before the update (post = false: colour 0, whose
// neighbours are final at the end of the previous sweep) or after it (post:
// colour 1, whose neighbours are final).  A site with d >= 2 always flips
// (d -> 4 - d); one with d = 0 or 1 flips as drawn (d -> 4 or 3).
template <int CW, bool OBS, bool SD = false>
__device__ __forceinline__ void ising_finish(IsingItem<CW>& it, PhaseAcc& acc, bool post = false)
{
    if constexpr (SD) {
        int f8 = 0, f4 = 0, u8 = 0, u4 = 0;  // flipped / all sites of the two drawn classes
#pragma unroll
        for (int k = 0; k < CW; ++k) {
            u8 += __popcll(it.u8[k]);
            u4 += __popcll(it.u4[k]);
            f8 += __popcll(it.u8[k] & it.flip[k]);
            f4 += __popcll(it.u4[k] & it.flip[k]);
        }
        if (post) {
            acc.sd[8] += it.n4 + u8 - f8;  // d' = 0
            acc.sd[6] += it.n3 + u4 - f4;  // d' = 1
            acc.sd[4] += it.n2;            // d' = 2
            acc.sd[2] += f4;               // d' = 3
            acc.sd[0] += f8;               // d' = 4
        } else {
            acc.sd[8] += u8;
            acc.sd[6] += u4;
            acc.sd[4] += it.n2;
            acc.sd[2] += it.n3;
            acc.sd[0] += it.n4;
        }
    }
    uint64_t cn[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) cn[k] = it.c[k] ^ it.flip[k];
    if constexpr (CW == 2) {
        reinterpret_cast<ulonglong2*>(it.row)[it.ch] = make_ulonglong2(cn[0], cn[1]);
    } else {
        it.row[it.ch] = cn[0];
    }
    if constexpr (OBS) {
        acc.B += 128 * CW - 2 * it.dpre;  // 32 active sites x 4 bonds per word
#pragma unroll
        for (int k = 0; k < CW; ++k) acc.M += 2 * __popcll(cn[k]) - 64;
        acc.Q += 64 * CW;
    }
}

template <int CW, bool OBS, bool CG, bool SD = false>
__device__ __forceinline__ void ising_item(const IsingPhase& a, const RoundKeys& rk, uint64_t item, int lane,
                                           PhaseAcc& acc)
{
    IsingItem<CW> it;
    ising_classify<CW, OBS, CG, SD>(a, item, lane, true, it);
    const uint64_t drw8 = a.mode8 == kDraw ? ~0ull : 0ull;
    const uint64_t drw4 = a.mode4 == kDraw ? ~0ull : 0ull;
    uint64_t need[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) need[k] = (it.u8[k] & drw8) | (it.u4[k] & drw4);

    acc.D += __popcll(need[0]) + (CW == 2 ? __popcll(need[CW - 1]) : 0);
    if (__any_sync(kFullMask, (need[0] | need[CW - 1]) != 0)) {
        const uint64_t base = (uint64_t)it.y * a.L + (uint64_t)it.ch * (64u * CW);
        const uint32_t site0 = (uint32_t)base + it.p;  // chunks never straddle 2^32 (64*CW | 2^32)
        const PhiloxChunk pc = philox_chunk((uint32_t)(base >> 32), a.sweep, a.colour, rk);
        uint32_t r4[CW][2], r8[CW][2];  // [word][32-bit half]: u < thr4, u < thr8
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t acc4[CW], acc8[CW];
#pragma unroll
            for (int k = 0; k < CW; ++k) acc4[k] = acc8[k] = 0;
            uint32_t bit = 1u << it.p;
#pragma unroll 2
            for (uint32_t j = 0; j < 16; ++j) {
                const uint32_t off = 32u * half + 2u * j;
#pragma unroll
                for (int k = 0; k < CW; ++k) {
                    const uint32_t u = philox_site_w0(site0 + 64u * k + off, pc, rk);
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
            const uint64_t acc8 = need[k] & it.u8[k] & R8, acc4 = need[k] & ~it.u8[k] & R4;
            it.flip[k] |= acc8 | acc4;
            // an accepted 3-agree site goes from 1 to 3 disagreeing bonds, a 4-agree site from 0 to 4
            if constexpr (OBS) it.dpre += 2 * __popcll(acc4) + 4 * __popcll(acc8);
        }
    }
    ising_finish<CW, OBS, SD>(it, acc, a.colour == 1);
}

// The 16-entry table is searched in "spread" form: entry j sits at slot
// spread4(j) (bit k of j moved to bit 2k) of an 86-slot shared array, so the
// binary search yields the four random bits already at the even positions
// of a byte, where the word's active sites take them (no later spreading).
constexpr int kLutSlots = 86;  // spread4(15) + 1

__host__ __device__ __forceinline__ constexpr uint32_t spread4(uint32_t j)
{
    return (j & 1u) | ((j & 2u) << 1) | ((j & 4u) << 2) | ((j & 8u) << 3);
}

// Slot i of the spread table built from the 16 entries t16 (0 where i is
// not spread4 of any index).
__device__ __forceinline__ uint32_t lut_slot(const uint32_t* t16, uint32_t i)
{
    if (i & 0xAAu) return 0u;
    return t16[(i & 1u) | ((i >> 1) & 2u) | ((i >> 2) & 4u) | ((i >> 3) & 8u)];
}

// spread4 of the largest index j with t[j] <= u (t[0] = 0): a four-step
// binary search over the spread table.
__device__ __forceinline__ uint32_t lut_find_spread(const uint32_t* ts, uint32_t u)
{
    uint32_t js = u >= ts[spread4(8)] ? spread4(8) : 0u;
    js += u >= ts[js + spread4(4)] ? spread4(4) : 0u;
    js += u >= ts[js + spread4(2)] ? spread4(2) : 0u;
    js += u >= ts[js + spread4(1)] ? spread4(1) : 0u;
    return js;
}

// One-lookup form of the same search for kernels that hold a 32 KiB shared
// table: the top 15 bits of a uniform pick a bucket of 2^17 values.  The
// table is non-decreasing, so where the index is the same at both ends of a
// bucket it is the same throughout, and the bucket's byte is its spread4; a
// bucket that holds a step of the index gets the marker 0xAA (bits that no
// spread index sets), and a uniform that meets it takes the four-step search.
// At most 15 of the 2^15 buckets hold a step.
constexpr int kLutBucketShift = 17;
constexpr int kLutBuckets = 1 << (32 - kLutBucketShift);
constexpr uint32_t kLutMarker = 0xAAu;

// Fill the bucket table tb from the spread table ts (all threads of the
// block; ts must be complete, and tb is complete after the next barrier).
__device__ __forceinline__ void lut_buckets(const uint32_t* ts, uint8_t* tb)
{
    for (int b = threadIdx.x; b < kLutBuckets; b += blockDim.x) {
        const uint32_t u0 = (uint32_t)b << kLutBucketShift, u1 = u0 | ((1u << kLutBucketShift) - 1u);
        const uint32_t j0 = lut_find_spread(ts, u0);
        tb[b] = (uint8_t)(j0 == lut_find_spread(ts, u1) ? j0 : kLutMarker);
    }
}

// The spread indices of the four uniforms of one Philox block, in bytes 0..3.
template <bool BUCKETS>
__device__ __forceinline__ uint32_t lut_bits4(const uint32_t* ts, const uint8_t* tb, const uint4& r)
{
    if constexpr (BUCKETS) {
        const uint32_t xy = __byte_perm(tb[r.x >> kLutBucketShift], tb[r.y >> kLutBucketShift], 0x40u);
        const uint32_t zw = __byte_perm(tb[r.z >> kLutBucketShift], tb[r.w >> kLutBucketShift], 0x40u);
        const uint32_t b4 = __byte_perm(xy, zw, 0x5410u);
        if (!(b4 & (kLutMarker * 0x01010101u))) return b4;
    }
    return lut_find_spread(ts, r.x) | (lut_find_spread(ts, r.y) << 8) | (lut_find_spread(ts, r.z) << 16) |
           (lut_find_spread(ts, r.w) << 24);
}

// The paper's lookup-table random bits (section 3.2, LAT_RNG_TABLE): per
// 64-bit word, four Philox blocks (counters 4w+q, sweep, colour+2) give 16
// uniforms; each is located in the table s_lut (spread form, kLutSlots
// slots), and the index is four random bits.  Uniforms 0..7 build word e0,
// 8..15 word e1: uniform i gives the bits of the word's active sites 4i ..
// 4i+3, which sit at bits 8i + 2b (+ the row's colour parity).  A 3-agree
// site flips iff its e0 bit is set, a 4-agree site iff its e0 and e1 bits
// are.  BUCKETS: the uniforms are first looked up in the bucket table
// s_lutb (lut_buckets).
template <int CW, bool OBS, bool CG, bool SD = false, bool BUCKETS = false>
__device__ __forceinline__ void ising_item_lut(const IsingPhase& a, const RoundKeys& rk, const uint32_t* s_lut,
                                               const uint8_t* s_lutb, uint64_t item, int lane, PhaseAcc& acc)
{
    IsingItem<CW> it;
    ising_classify<CW, OBS, CG, SD>(a, item, lane, false, it);
    acc.D += 4 * CW;
#pragma unroll
    for (int k = 0; k < CW; ++k) {
        const uint64_t w = (uint64_t)it.y * a.W + (uint64_t)it.ch * CW + k;  // word index
        const uint64_t ctr = 4ull * w;                                      // 4w+q never carries into the high word
        const PhiloxChunk pc = philox_chunk((uint32_t)(ctr >> 32), a.sweep, a.colour + 2u, rk);
        uint64_t e0 = 0, e1 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 r = philox_site_w4((uint32_t)ctr + (uint32_t)q, pc, rk);
            const uint32_t b4 = lut_bits4<BUCKETS>(s_lut, s_lutb, r);
            if (q < 2) e0 |= (uint64_t)b4 << (32 * q);  // uniforms 4q .. 4q+3
            else e1 |= (uint64_t)b4 << (32 * (q - 2));
        }
        const uint64_t x0 = e0 << it.p, x1 = e1 << it.p;
        const uint64_t acc4 = it.u4[k] & x0, acc8 = it.u8[k] & x0 & x1;
        it.flip[k] |= acc4 | acc8;
        if constexpr (OBS) it.dpre += 2 * __popcll(acc4) + 4 * __popcll(acc8);
    }
    ising_finish<CW, OBS, SD>(it, acc, a.colour == 1);
}

// Three-bit sum of four one-bit words (bit-sliced): returns b0 + 2 b1 + 4 b2.
template <typename U>
__device__ __forceinline__ void add4(U a, U b, U c, U d, U& b0, U& b1, U& b2)
{
    const U s1 = a ^ b, c1 = a & b;
    const U s2 = c ^ d, c2 = c & d;
    b0 = s1 ^ s2;
    const U c3 = s1 & s2;
    b1 = c1 ^ c2 ^ c3;
    b2 = (c1 & c2) | (c1 & c3) | (c2 & c3);
}

// A Blume-Capel spin's 2-bit code is n | g << 1 (n: s != 0, g: s = -1):
// 0 for s = 0, 1 for s = +1, 3 for s = -1 (2 never occurs).  kBcNext gives
// the code of the proposed value, the b-th of the two other values in
// ascending order, at index code*2 + b (2 bits each): s=0 -> {-1, +1},
// s=+1 -> {-1, 0}, s=-1 -> {0, +1}.
constexpr uint32_t kBcNext = (3u << 0) | (1u << 2) | (3u << 4) | (0u << 6) | (0u << 8) | (0u << 10) |
                             (0u << 12) | (1u << 14);

// Value of a 2-bit spin code: 0, +1 or -1.
__host__ __device__ __forceinline__ int bc_value(uint32_t code)
{
    return (int)(code & 1u) * (1 - (int)(code & 2u));
}

// The kernels' Blume-Capel table, 128 entries indexed by
//   code | (h+4) << 2 | b << 6
// (spin code, neighbour sum h = -4..4 as h+4 in 4 bits, proposal bit b).
// An entry is (bound, xm): the move is accepted iff word 0 <= bound, and an
// accepted move XORs the site's code with xm = code ^ (code of the proposed
// value).  From the 54-entry table's t: bound = 2^32 - 1 when t = 2^32
// (always), t - 1 when 0 < t < 2^32 (u < t iff u <= t - 1); a move that is
// never accepted (t = 0) and unused indices (code 2, h+4 > 8) get xm = 0, so
// whatever the comparison gives, the site keeps its code.
constexpr int kBcTable = 128;

// Sites of one half-item per unrolled step of the Blume-Capel site loop.
#ifndef LAT_BC_UNROLL
#define LAT_BC_UNROLL 2
#endif
constexpr int kBcUnroll = LAT_BC_UNROLL;

__device__ __forceinline__ void bc_table128(const unsigned long long* thr54, uint2* t)
{
    for (int i = threadIdx.x; i < kBcTable; i += blockDim.x) {
        const uint32_t code = i & 3u, h4 = (i >> 2) & 15u, b = (uint32_t)i >> 6;
        uint2 e = make_uint2(0u, 0u);
        if (code != 2u && h4 <= 8u) {
            const int sv = bc_value(code);
            const unsigned long long th = thr54[((sv + 1) * 2 + (int)b) * 9 + (int)h4];
            const uint32_t next = (kBcNext >> (2u * (code * 2u + b))) & 3u;
            if (th >= kAlways) e = make_uint2(0xFFFFFFFFu, code ^ next);
            else if (th > 0) e = make_uint2((uint32_t)th - 1u, code ^ next);
        }
        t[i] = e;
    }
}

struct BcPhase {
    ulonglong2* spins;  // L rows of W (n, g) word pairs
    uint32_t L, W;
    uint32_t sweep, colour;
};

// Blume-Capel decision (Eq. (2)): every active site draws; the low bit of
// word 1 picks the proposal among the two other values, and the move is
// accepted iff the table entry for (s, proposal, h) is 2^32 or word 0 is
// below it.  The update is branch-free.
//
// Every plane is first shifted right by the row's colour parity, so the 32
// active sites sit at the even bit positions.  A site's table index is
// built once per item, bit-sliced for all 64 positions: h + 4 = 2 P + Z,
// with P (Z) the number of +1 (zero) neighbours, so h+4 needs no
// subtraction.  Two planes share one word (one at the even, one at the odd
// positions), so three shifts give a site's code and h+4.  Per site the
// loop only compares word 0 with the entry's bound and adds the entry's
// code mask at the site's position; the new planes are the old ones XOR
// those masks.  The fused bond sum (colour 1) is then taken bit-sliced over
// the item: sum over active sites of s' h = sum over new +1 sites of
// (h+4) - 4 minus the same over new -1 sites, h the final neighbour sum (its
// four neighbours are colour 0 and already final).
template <bool OBS, bool CG, bool SD = false>
__device__ __forceinline__ void bc_item(const BcPhase& a, const RoundKeys& rk, const uint2* s_tab, uint64_t item,
                                        int lane, PhaseAcc& acc)
{
    const uint32_t y = (uint32_t)(item / a.W);
    const uint32_t j = (uint32_t)(item - (uint64_t)y * a.W);
    const uint32_t yn = y == 0 ? a.L - 1 : y - 1;
    const uint32_t ys = y + 1 == a.L ? 0 : y + 1;
    ulonglong2* row = a.spins + (uint64_t)y * a.W;
    const ulonglong2 c = ld<CG>(row + j);
    const ulonglong2 vn = ld<CG>(a.spins + (uint64_t)yn * a.W + j);
    const ulonglong2 vs = ld<CG>(a.spins + (uint64_t)ys * a.W + j);
    ulonglong2 left, right;
    left.x = __shfl_up_sync(kFullMask, c.x, 1);
    left.y = __shfl_up_sync(kFullMask, c.y, 1);
    right.x = __shfl_down_sync(kFullMask, c.x, 1);
    right.y = __shfl_down_sync(kFullMask, c.y, 1);
    if (lane == 0 || j == 0) left = ld<CG>(row + (j == 0 ? a.W - 1 : j - 1));
    if (lane == 31 || j + 1 == a.W) right = ld<CG>(row + (j + 1 == a.W ? 0 : j + 1));

    const uint32_t p = (y + a.colour) & 1u;
    constexpr uint64_t E = kEvenBits;
    // Planes in the shifted frame (active sites at even positions).
    uint64_t wcode, wh01, wh23;  // code; h+4 bits 0,1; h+4 bits 2,3 (even/odd positions)
    uint64_t H0, H1, H2, H3;     // h+4, bit-sliced (bits 0..3)
    {
        const uint64_t nn_ = vn.x >> p, ng_ = vn.y >> p, sn_ = vs.x >> p, sg_ = vs.y >> p;
        const uint64_t wn_ = ((c.x << 1) | (left.x >> 63)) >> p, wg_ = ((c.y << 1) | (left.y >> 63)) >> p;
        const uint64_t en_ = ((c.x >> 1) | (right.x << 63)) >> p, eg_ = ((c.y >> 1) | (right.y << 63)) >> p;
        uint64_t P0, P1, P2, Z0, Z1, Z2;
        add4<uint64_t>(nn_ & ~ng_, sn_ & ~sg_, wn_ & ~wg_, en_ & ~eg_, P0, P1, P2);
        add4<uint64_t>(~nn_, ~sn_, ~wn_, ~en_, Z0, Z1, Z2);
        // h+4 = Z + 2P, bit-sliced (at most 8: no carry out of bit 3)
        const uint64_t s1 = Z1 ^ P0, c1 = Z1 & P0;
        const uint64_t s2 = Z2 ^ P1 ^ c1, c2 = (Z2 & P1) | (Z2 & c1) | (P1 & c1);
        const uint64_t s3 = P2 ^ c2;
        H0 = Z0, H1 = s1, H2 = s2, H3 = s3;
        wcode = ((c.x >> p) & E) | (((c.y >> p) & E) << 1);
        wh01 = (Z0 & E) | ((s1 & E) << 1);
        wh23 = (s2 & E) | ((s3 & E) << 1);
    }

    const uint64_t base = (uint64_t)y * a.L + (uint64_t)j * 64u;
    const uint32_t site0 = (uint32_t)base + p;  // site of shifted position 0
    const PhiloxChunk pc = philox_chunk((uint32_t)(base >> 32), a.sweep, a.colour, rk);
    uint64_t fm = 0;  // code masks of the accepted moves (2 bits per active site)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int hs = 32 * half;
        const uint32_t x0 = (uint32_t)(wcode >> hs), x1 = (uint32_t)(wh01 >> hs), x2 = (uint32_t)(wh23 >> hs);
        uint32_t m = 0;
#pragma unroll kBcUnroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t b = 2u * k;
            const uint2 r = philox_site_w01(site0 + (uint32_t)hs + b, pc, rk);
            const uint32_t idx = ((x0 >> b) & 3u) | (((x1 >> b) & 3u) << 2) | (((x2 >> b) & 3u) << 4) |
                                 ((r.y & 1u) << 6);
            const uint2 e = s_tab[idx];
            m += (r.x <= e.x ? e.y : 0u) << b;
        }
        fm |= (uint64_t)m << hs;
    }
    const uint64_t nn = c.x ^ ((fm & E) << p), gg = c.y ^ (((fm >> 1) & E) << p);
    row[j] = make_ulonglong2(nn, gg);
    acc.D += 32;
    if constexpr (OBS) {
        acc.M += __popcll(nn & ~gg) - __popcll(nn & gg);
        acc.Q += __popcll(nn);
        // bond sum: new +1 and -1 active sites in the shifted frame
        const uint64_t n1 = (nn >> p) & E, g1 = (gg >> p) & E;
        const uint64_t up = n1 & ~g1, dn = n1 & g1;
        const int hu = __popcll(up & H0) + 2 * __popcll(up & H1) + 4 * __popcll(up & H2) + 8 * __popcll(up & H3);
        const int hd = __popcll(dn & H0) + 2 * __popcll(dn & H1) + 4 * __popcll(dn & H2) + 8 * __popcll(dn & H3);
        acc.B += (hu - 4 * __popcll(up)) - (hd - 4 * __popcll(dn));
    }
    if constexpr (SD) {
        // Histogram of s h over the active sites: before the update in the
        // colour-0 phase, after it in the colour-1 phase (h is final in both,
        // the neighbours being of the other colour).  s = 0 (code n clear)
        // gives bin 4; s = +1 bin h + 4 = H; s = -1 bin 4 - h = 8 - H.
        const bool post = a.colour == 1;
        const uint64_t sn = ((post ? nn : c.x) >> p) & E, sg = ((post ? gg : c.y) >> p) & E;
        const uint64_t up = sn & ~sg, dn = sn & sg;
        acc.sd[4] += 32 - __popcll(sn);
#pragma unroll
        for (int k = 0; k <= 8; ++k) {
            const uint64_t m = ((k & 1) ? H0 : ~H0) & ((k & 2) ? H1 : ~H1) & ((k & 4) ? H2 : ~H2) &
                               ((k & 8) ? H3 : ~H3);
            acc.sd[k] += __popcll(up & m);
            acc.sd[8 - k] += __popcll(dn & m);
        }
    }
}

}  // namespace latk
