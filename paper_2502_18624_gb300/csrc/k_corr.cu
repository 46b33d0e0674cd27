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
#include <type_traits>

#include "lat_internal.cuh"

namespace latk {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kXGroupsMax = 8;    // word-offset groups per x block
constexpr int kXWarpsMax = 16;    // warps per x block: groups x row parts
constexpr int kYWarps = 8;        // distance groups per y block

template <int MODEL>
struct Planes {
    static constexpr int n = MODEL == 0 ? 1 : 2;
};

// acc + v on the multiply-add pipe.  `one` is a kernel argument equal to 1,
// so the multiply cannot be folded away and the sum stays an IMAD, off the
// ALU pipe that the XORs and carry-save logic of the pairs already fill.
__device__ __forceinline__ int mad_acc(int acc, uint32_t v, uint32_t one)
{
    int r;
    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(r) : "r"(v), "r"(one), "r"(acc));
    return r;
}

// One carry-save step of the running sum (ones, carries) with two new words:
// the new sum bit is ones ^ x1 ^ x2 and the carry is their majority, each
// one 3-input logic operation.
__device__ __forceinline__ uint32_t csa_sum(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t csa_carry(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Asynchronous 4-byte copy global -> shared (zero-filled when !ok; src must
// still be a valid address), and the group fences that order them.
__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src, bool ok)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Word j0 of the row rotated right by s bits: bits s..31 of word j0
// followed by bits 0..s-1 of the next word.  The staged row is extended
// periodically past its end (row[W32 + i] = row[i]), so no wrap is needed.
__device__ __forceinline__ uint32_t rot_word(const uint32_t* row, uint32_t j0, uint32_t s)
{
    return __funnelshift_r(row[j0], row[j0 + 1], s);
}

// Stage row y as 32-bit words extended periodically to n >= W32 words
// (asynchronous copies): word j of the staged row is word j mod W32 of the
// lattice row.  Ising plane at dst[0..n); Blume-Capel n plane at dst[0..n)
// and g plane at dst[n..2n).
template <int MODEL>
__device__ __forceinline__ void stage_row32_ext(const void* spins, uint32_t W32, uint64_t y, uint32_t n,
                                                uint32_t* dst, int lane, int nlanes)
{
    const uint32_t* src = static_cast<const uint32_t*>(spins) + y * W32 * (MODEL == 0 ? 1 : 2);
    for (uint32_t j = lane; j < n; j += nlanes) {
        const uint32_t w = j < W32 ? j : j - W32 * (j / W32);
        if constexpr (MODEL == 0) {
            cp_async4(dst + j, src + w, true);
        } else {  // words (n lo, n hi, g lo, g hi) per 64 sites
            cp_async4(dst + j, src + 4 * (w / 2) + (w & 1), true);
            cp_async4(dst + n + j, src + 4 * (w / 2) + 2 + (w & 1), true);
        }
    }
}

template <int MODEL, int NQ>
__global__ void __launch_bounds__(kXWarpsMax * 32) k_corr_x(const void* spins, uint32_t L, uint32_t rmax,
                                                           uint32_t rows_per_block, long long* cx, uint32_t ext,
                                                           uint32_t nbuf, uint32_t gpb, uint32_t span, uint32_t one)
{
    // One row at a time is worked on by the whole block, extended
    // periodically to `ext` words (enough for the largest offset any warp of
    // the grid reads), while the next row is copied into the other of two
    // buffers (nbuf = 2; with nbuf = 1, for rows too long for two buffers, the
    // next row is copied after the block is done with this one).  The block
    // has gpb offset groups times (warps / gpb) row parts: warp w owns word
    // offsets q0 = (blockIdx.y * gpb + w % gpb) * NQ .. + NQ - 1 for the row
    // words [i0, i1) of part w / gpb (span words each), so that several
    // warps share one staged row even when rmax needs few offset groups.
    extern __shared__ uint32_t sm[];
    const uint32_t W32 = L / 32;
    const int warp = threadIdx.x >> 5, s = threadIdx.x & 31;
    const uint32_t q0 = (blockIdx.y * gpb + (uint32_t)warp % gpb) * NQ;
    const uint32_t i0 = min(W32, ((uint32_t)warp / gpb) * span), i1 = min(W32, i0 + span);
    constexpr int P = Planes<MODEL>::n;
    const uint32_t m2 = 0u - 2u * one;  // -2, for the Blume-Capel opposite-sign pairs
    int acc[NQ];        // Ising: carries of the carry-save sums; Blume-Capel: the sums themselves
    uint32_t ones[NQ];  // Ising: carry-save sum bits
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = 0, ones[k] = 0;
    const uint32_t ybeg = blockIdx.x * rows_per_block;
    const uint32_t yend = min(ybeg + rows_per_block, L);
    if (ybeg < yend) stage_row32_ext<MODEL>(spins, W32, ybeg, ext, sm, threadIdx.x, blockDim.x);
    cp_async_commit();
    for (uint32_t y = ybeg; y < yend; ++y) {
        const uint32_t* row = sm + (nbuf == 2 ? ((y - ybeg) & 1u) * ext * P : 0u);
        if (nbuf == 2 && y + 1 < yend)   // the next row, into the other buffer
            stage_row32_ext<MODEL>(spins, W32, y + 1, ext, sm + ((y + 1 - ybeg) & 1u) * ext * P, threadIdx.x,
                                   blockDim.x);
        cp_async_commit();
        cp_async_wait1();   // this row's copies have landed
        __syncthreads();
        uint32_t win[NQ], wing[NQ];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            win[k] = rot_word(row, q0 + i0 + k, s);
            if constexpr (MODEL == 1) wing[k] = rot_word(row + ext, q0 + i0 + k, s);
        }
        uint32_t jn = q0 + NQ + i0;  // i + q0 + NQ: the word entering the window (< ext - 1)
        if constexpr (MODEL == 0) {
            // Words i and i+1 (W32 is even) go through one carry-save step per
            // distance: sum bits stay in ones[k], the carries are counted.
            // A group covers words ib .. ib + 2 NQ - 1 (FULL: all below W32);
            // the entering word of word i is row[q0 + NQ + i].
            auto group = [&](auto full, uint32_t ib) {
                constexpr bool FULL = decltype(full)::value;
                const uint32_t* rw = row + ib;           // row word i = rw[u]
                const uint32_t* en = row + q0 + NQ + ib; // entering word of word i = en[u]
#pragma unroll
                for (int u = 0; u < 2 * NQ; u += 2) {
                    if (FULL || ib + u < i1) {
                        const uint32_t a1 = rw[u], a2 = rw[u + 1];
                        uint32_t x1[NQ];
#pragma unroll
                        for (int k = 0; k < NQ; ++k) x1[k] = a1 ^ win[(u + k) % NQ];
                        win[u % NQ] = __funnelshift_r(en[u], en[u + 1], s);
#pragma unroll
                        for (int k = 0; k < NQ; ++k) {
                            const uint32_t x2 = a2 ^ win[(u + 1 + k) % NQ];
                            acc[k] = mad_acc(acc[k], __popc(csa_carry(ones[k], x1[k], x2)), one);
                            ones[k] = csa_sum(ones[k], x1[k], x2);
                        }
                        win[(u + 1) % NQ] = __funnelshift_r(en[u + 1], en[u + 2], s);
                    }
                }
            };
            uint32_t ib = i0;
            for (; ib + 2 * NQ <= i1; ib += 2 * NQ) group(std::integral_constant<bool, true>{}, ib);
            if (ib < i1) group(std::integral_constant<bool, false>{}, ib);
        } else {
            for (uint32_t ib = i0; ib < i1; ib += NQ) {
#pragma unroll
                for (int u = 0; u < NQ; ++u) {
                    const uint32_t i = ib + u;
                    if (i < i1) {
                        const uint32_t a = row[i];
                        {
                            const uint32_t ag = row[ext + i];
#pragma unroll
                            for (int k = 0; k < NQ; ++k) {
                                const uint32_t both = a & win[(u + k) % NQ];
                                acc[k] = mad_acc(acc[k], __popc(both), one);
                                acc[k] = mad_acc(acc[k], __popc(both & (ag ^ wing[(u + k) % NQ])), m2);
                            }
                            win[u] = rot_word(row, jn, s);
                            wing[u] = rot_word(row + ext, jn, s);
                        }
                        ++jn;
                    }
                }
            }
        }
        __syncthreads();  // every warp is done with this buffer before it is refilled
        if (nbuf == 1 && y + 1 < yend) stage_row32_ext<MODEL>(spins, W32, y + 1, ext, sm, threadIdx.x, blockDim.x);
    }
    const long long rows = yend > ybeg ? (long long)(yend - ybeg) : 0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        const uint32_t r = 32u * (q0 + k) + s;
        if (r <= rmax && rows && i1 > i0) {
            const long long mism = 2ll * acc[k] + __popc(ones[k]);  // Ising: disagreeing pairs
            // Ising: this warp's pairs are rows x 32 (i1 - i0) sites, each 1 - 2 [unequal]
            const long long v = MODEL == 0 ? rows * 32ll * (i1 - i0) - 2ll * mism : (long long)acc[k];
            atomicAdd(reinterpret_cast<unsigned long long*>(cx + r), (unsigned long long)v);
        }
    }
}

// y: a block owns a 32-word column strip, a segment of rows [y0, y0+H) and
// the distances r0 .. r0 + kYWarps*NQ - 1.  The rows y0 + r0 + t (t >= 0)
// that row y0 + y pairs with stream through a shared-memory ring of
// YRing<NQ>::rows rows; each step stages 2 NQ new A rows and 2 NQ new ring
// rows, so the register window's slot rotation restarts at every step and
// stays a compile-time pattern, and (Ising) rows y and y+1 share one
// carry-save step per distance.
template <int NQ>
struct YRing {
    static constexpr uint32_t step = 2 * NQ;  // rows staged per step
    // A step reads ring entries [ys, ys + D + step) while the next step's
    // entries [ys + D + step, ys + D + 2 step) are copied in: with D + 2 step
    // slots (entry t in slot t mod entries) the two never share a slot.
    static constexpr uint32_t entries = kYWarps * NQ + 2 * step;
    // In a step a warp reads the NQ + step consecutive entries from ys + g0.
    // Slots below `mirror` are stored a second time after the last slot, so
    // that such a run sits at consecutive addresses whatever slot it starts at.
    static constexpr uint32_t mirror = NQ + step;
    static constexpr uint32_t rows = entries + mirror;  // physical rows per plane
};

// Asynchronous copy of word j of row y into shared memory: Ising to dn;
// Blume-Capel n plane to dn and g plane to dg.  Zero when !ok (then no
// address in the lattice is formed).
template <int MODEL>
__device__ __forceinline__ void stage_strip_word(const void* spins, uint32_t W32, uint64_t y, uint32_t j, bool ok,
                                                 uint32_t* dn, uint32_t* dg)
{
    const uint32_t* base = static_cast<const uint32_t*>(spins);
    if constexpr (MODEL == 0) {
        cp_async4(dn, ok ? base + y * W32 + j : base, ok);
    } else {
        const uint32_t* p = base + y * 2 * W32 + 4 * (j / 2) + (j & 1);
        cp_async4(dn, ok ? p : base, ok);
        cp_async4(dg, ok ? p + 2 : base, ok);
    }
}

template <int MODEL>
__device__ __forceinline__ void load_strip_word(const void* spins, uint32_t W32, uint64_t y, uint32_t j, bool ok,
                                                uint32_t& vn, uint32_t& vg)
{
    vn = 0;
    vg = 0;
    if (!ok) return;
    if constexpr (MODEL == 0) {
        vn = static_cast<const uint32_t*>(spins)[y * W32 + j];
    } else {
        const uint32_t* p = static_cast<const uint32_t*>(spins) + y * 2 * W32;
        vn = p[4 * (j / 2) + (j & 1)];
        vg = p[4 * (j / 2) + 2 + (j & 1)];
    }
}

template <int MODEL, int NQ>
__global__ void __launch_bounds__(kYWarps * 32) k_corr_y(const void* spins, uint32_t L, uint32_t rmax,
                                                        uint32_t rows_per_block, long long* cy, uint32_t chunks,
                                                        uint32_t strips, uint32_t one)
{
    extern __shared__ uint32_t sm[];
    constexpr int P = Planes<MODEL>::n;
    constexpr uint32_t RN = YRing<NQ>::entries, RM = YRing<NQ>::mirror, RP = YRing<NQ>::rows;
    constexpr uint32_t D = kYWarps * NQ;  // distances per block
    constexpr uint32_t S = YRing<NQ>::step;
    const uint32_t W32 = L / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Block b covers distance chunk b % chunks of strip (b / chunks) % strips
    // and row segment b / (chunks * strips): the blocks of one strip and
    // segment are consecutive, so they run together and read their shared
    // rows through L2 once.
    const uint32_t bid = blockIdx.x;
    const uint32_t chunk = bid % chunks, strip = (bid / chunks) % strips, seg = bid / (chunks * strips);
    const uint32_t j0 = strip * 32;
    const uint32_t tw = min(32u, W32 - j0);
    const uint32_t y0 = seg * rows_per_block;
    const uint32_t H = min(rows_per_block, L - y0);  // even: L and rows_per_block are even
    const uint32_t r0 = chunk * D;
    const uint32_t m2 = 0u - 2u * one;
    uint32_t* ring = sm;                // RP x 32 words per plane
    uint32_t* arow = sm + RP * 32 * P;  // two buffers of S x 32 words per plane

    // Lattice row of ring entry t is (y0 + r0 + t) mod L (staging only, so a
    // plain modulo is cheap next to the pair work).
    const uint32_t rb = (uint32_t)(((uint64_t)y0 + r0) % L);
    auto brow = [L, rb](uint32_t t) { return (uint32_t)(((uint64_t)rb + t) % L); };
    // Column c of ring entry t: slot t mod RN, and again at RN + slot when
    // the slot is below RM.
    auto stage_ring = [&](uint32_t t, uint32_t c) {
        const uint32_t slot = t % RN, yb = brow(t);
        stage_strip_word<MODEL>(spins, W32, yb, j0 + c, c < tw, ring + slot * 32 + c,
                                ring + RP * 32 + slot * 32 + c);
        if (slot < RM)
            stage_strip_word<MODEL>(spins, W32, yb, j0 + c, c < tw, ring + (RN + slot) * 32 + c,
                                    ring + RP * 32 + (RN + slot) * 32 + c);
    };
    // Copies for the step at ys: A rows ys .. ys+S-1 into buffer b, ring
    // entries D+ys .. D+ys+S-1.
    auto stage_step = [&](uint32_t ys, uint32_t b) {
        uint32_t* ab = arow + b * S * 32 * P;
        for (uint32_t t = threadIdx.x; t < 2 * S * 32; t += blockDim.x) {
            const uint32_t rr = (t / 32) % S, c = t % 32;
            if (t < S * 32) {
                const uint32_t ya = (uint32_t)(((uint64_t)y0 + ys + rr) % L);
                stage_strip_word<MODEL>(spins, W32, ya, j0 + c, c < tw && ys + rr < H, ab + rr * 32 + c,
                                        ab + S * 32 + rr * 32 + c);
            } else {
                stage_ring(D + ys + rr, c);
            }
        }
    };
    for (uint32_t t = threadIdx.x; t < D * 32; t += blockDim.x) stage_ring(t / 32, t % 32);  // entries 0 .. D-1
    stage_step(0, 0);
    cp_async_commit();

    const uint32_t g0 = (uint32_t)warp * NQ;
    int acc[NQ];        // Ising: carries of the carry-save sums; Blume-Capel: the sums themselves
    uint32_t ones[NQ];  // Ising: carry-save sum bits
    uint32_t win[NQ], wing[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = 0, ones[k] = 0;
    // One step of S rows: window slot k holds entry ys + g0 + k at its start,
    // and entry ys + g0 + j sits at rp[j * 32] (rp[RP * 32 + j * 32] for the g
    // plane).  FULL: all S rows of the step are in the segment.
    auto run_step = [&](auto full, uint32_t ys, const uint32_t* ab, const uint32_t* rp) {
        constexpr bool FULL = decltype(full)::value;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            win[k] = rp[k * 32];
            if constexpr (P == 2) wing[k] = rp[RP * 32 + k * 32];
        }
        if constexpr (MODEL == 0) {
#pragma unroll
            for (int u = 0; u < (int)S; u += 2) {
                if (FULL || ys + u < H) {  // then ys + u + 1 < H too (H is even)
                    const uint32_t a1 = ab[u * 32 + lane], a2 = ab[(u + 1) * 32 + lane];
                    uint32_t x1[NQ];
#pragma unroll
                    for (int k = 0; k < NQ; ++k) x1[k] = a1 ^ win[(u + k) % NQ];
                    win[u % NQ] = rp[(NQ + u) * 32];  // the entry entering this warp's window
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        const uint32_t x2 = a2 ^ win[(u + 1 + k) % NQ];
                        acc[k] = mad_acc(acc[k], __popc(csa_carry(ones[k], x1[k], x2)), one);
                        ones[k] = csa_sum(ones[k], x1[k], x2);
                    }
                    win[(u + 1) % NQ] = rp[(NQ + u + 1) * 32];
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < (int)S; ++u) {
                if (FULL || ys + u < H) {
                    const uint32_t a = ab[u * 32 + lane];
                    const uint32_t ag = ab[S * 32 + u * 32 + lane];
#pragma unroll
                    for (int k = 0; k < NQ; ++k) {
                        const uint32_t both = a & win[(u + k) % NQ];
                        acc[k] = mad_acc(acc[k], __popc(both), one);
                        acc[k] = mad_acc(acc[k], __popc(both & (ag ^ wing[(u + k) % NQ])), m2);
                    }
                    win[u % NQ] = rp[(NQ + u) * 32];
                    wing[u % NQ] = rp[RP * 32 + (NQ + u) * 32];
                }
            }
        }
    };
    for (uint32_t ys = 0, it = 0; ys < H; ys += S, ++it) {
        const uint32_t* ab = arow + (it & 1u) * S * 32 * P;
        if (ys + S < H) stage_step(ys + S, (it & 1u) ^ 1u);  // the next step, while this one runs
        cp_async_commit();
        cp_async_wait1();  // this step's copies have landed
        __syncthreads();
        const uint32_t* rp = ring + ((ys + g0) % RN) * 32 + lane;
        if (ys + S <= H) run_step(std::integral_constant<bool, true>{}, ys, ab, rp);
        else run_step(std::integral_constant<bool, false>{}, ys, ab, rp);
        __syncthreads();  // every warp is done with this A buffer before it is refilled
    }
    const bool colok = (uint32_t)lane < tw;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        int v = colok ? (MODEL == 0 ? 2 * acc[k] + __popc(ones[k]) : acc[k]) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        const uint32_t r = r0 + g0 + k;
        if (lane == 0 && r <= rmax) {
            const long long t = MODEL == 0 ? (long long)H * 32 * tw - 2ll * v : (long long)v;
            atomicAdd(reinterpret_cast<unsigned long long*>(cy + r), (unsigned long long)t);
        }
    }
}

// Near distances, r <= kNear = 32, both axes in one kernel (the all-sites
// part of the section 3.3 protocol asks for r <= 2R = 32).  A block owns a
// strip of 32 column words and kNearRows rows; it stages those rows, the
// kNear rows below them and the word right of the strip in shared memory.
// Warps 0..3 take the x distances 8k+1 .. 8k+8 (k = warp), warps 4..7 the y
// distances 8k+1 .. 8k+8 (k = warp - 4); every warp walks all rows of the
// block, lane = column word, and rows u and u+1 share one carry-save step per
// distance.  Distance 0 is counted by warp 0 (Ising: every site; Blume-Capel:
// the non-zero sites).
constexpr uint32_t kNear = 32;
constexpr uint32_t kNearRows = 64;
constexpr uint32_t kNearStride = 33;  // 32 strip words + the next word

// One warp's share of the near kernel: distances RB .. RB+7 (compile-time)
// along x (X) or y, over all staged rows; m masks the lanes beyond the strip.
template <int MODEL, bool X, int RB>
__device__ __forceinline__ void near_rows(const uint32_t (*Sn)[kNearStride], const uint32_t (*Sg)[kNearStride],
                                          int lane, uint32_t m, uint32_t one, long long* v)
{
    int acc[8], acc2[8];          // carries of the carry-save sums (Blume-Capel: two chains)
    uint32_t ones[8], ones2[8];   // sum bits
#pragma unroll
    for (int d = 0; d < 8; ++d) acc[d] = acc2[d] = 0, ones[d] = ones2[d] = 0;
#pragma unroll(MODEL == 0 ? 2 : 1)
    for (uint32_t u = 0; u < kNearRows; u += 2) {
        uint32_t a[2], an[2], ag[2], agn[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            a[h] = Sn[u + h][lane];
            if (X) an[h] = Sn[u + h][lane + 1];
            if (MODEL == 1) {
                ag[h] = Sg[u + h][lane];
                if (X) agn[h] = Sg[u + h][lane + 1];
            }
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int r = RB + d;
            uint32_t b[2], bg[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (X) {
                    b[h] = r < 32 ? __funnelshift_r(a[h], an[h], r) : an[h];
                    if (MODEL == 1) bg[h] = r < 32 ? __funnelshift_r(ag[h], agn[h], r) : agn[h];
                } else {
                    b[h] = Sn[u + h + r][lane];
                    if (MODEL == 1) bg[h] = Sg[u + h + r][lane];
                }
            }
            if constexpr (MODEL == 0) {
                const uint32_t x1 = (a[0] ^ b[0]) & m, x2 = (a[1] ^ b[1]) & m;
                acc[d] = mad_acc(acc[d], __popc(csa_carry(ones[d], x1, x2)), one);
                ones[d] = csa_sum(ones[d], x1, x2);
            } else {
                // pairs of non-zero sites, and those of opposite sign
                const uint32_t b1 = a[0] & b[0] & m, b2 = a[1] & b[1] & m;
                const uint32_t n1 = b1 & (ag[0] ^ bg[0]), n2 = b2 & (ag[1] ^ bg[1]);
                acc[d] = mad_acc(acc[d], __popc(csa_carry(ones[d], b1, b2)), one);
                ones[d] = csa_sum(ones[d], b1, b2);
                acc2[d] = mad_acc(acc2[d], __popc(csa_carry(ones2[d], n1, n2)), one);
                ones2[d] = csa_sum(ones2[d], n1, n2);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d)
        v[d] = MODEL == 0 ? 2ll * acc[d] + __popc(ones[d])  // unequal pairs
                          : (2ll * acc[d] + __popc(ones[d])) - 2 * (2ll * acc2[d] + __popc(ones2[d]));
}

template <int MODEL>
__global__ void __launch_bounds__(256, MODEL == 0 ? 6 : 4) k_corr_near(const void* spins, uint32_t L, uint32_t rmax, long long* cx,
                                                   long long* cy, uint32_t one)
{
    constexpr int P = Planes<MODEL>::n;
    constexpr uint32_t NR = kNearRows + kNear;  // staged rows
    __shared__ uint32_t S[P][NR][kNearStride];
    const uint32_t W32 = L / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t j0 = blockIdx.x * 32;
    const uint32_t tw = min(32u, W32 - j0);
    const uint32_t y0 = blockIdx.y * kNearRows;
    // column words j0 .. j0+tw of rows y0 .. y0+NR-1 (word j0+tw is the one
    // right of the strip, periodic); zero beyond
    for (uint32_t t = threadIdx.x; t < NR * kNearStride; t += blockDim.x) {
        const uint32_t rr = t / kNearStride, c = t % kNearStride;
        const uint64_t y = ((uint64_t)y0 + rr) % L;
        uint32_t vn, vg;
        load_strip_word<MODEL>(spins, W32, y, (j0 + c) % W32, c <= tw, vn, vg);
        S[0][rr][c] = vn;
        if constexpr (P == 2) S[P - 1][rr][c] = vg;
    }
    __syncthreads();
    const uint32_t m = (uint32_t)lane < tw ? ~0u : 0u;
    const uint32_t (*Sn)[kNearStride] = S[0];
    const uint32_t (*Sg)[kNearStride] = S[P - 1];
    long long v[8];
    switch (warp) {
        case 0: near_rows<MODEL, true, 1>(Sn, Sg, lane, m, one, v); break;
        case 1: near_rows<MODEL, true, 9>(Sn, Sg, lane, m, one, v); break;
        case 2: near_rows<MODEL, true, 17>(Sn, Sg, lane, m, one, v); break;
        case 3: near_rows<MODEL, true, 25>(Sn, Sg, lane, m, one, v); break;
        case 4: near_rows<MODEL, false, 1>(Sn, Sg, lane, m, one, v); break;
        case 5: near_rows<MODEL, false, 9>(Sn, Sg, lane, m, one, v); break;
        case 6: near_rows<MODEL, false, 17>(Sn, Sg, lane, m, one, v); break;
        default: near_rows<MODEL, false, 25>(Sn, Sg, lane, m, one, v); break;
    }
    const bool xw = warp < 4;
    const uint32_t rbase = 8u * (uint32_t)(warp & 3) + 1;
    long long* out = xw ? cx : cy;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        long long t = v[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        if (lane == 0 && rbase + d <= rmax) {
            const long long pairs = (long long)kNearRows * 32 * tw;
            const long long c = MODEL == 0 ? pairs - 2 * t : t;
            atomicAdd(reinterpret_cast<unsigned long long*>(out + rbase + d), (unsigned long long)c);
        }
    }
    // distance 0: every site (Ising) or every non-zero site (Blume-Capel)
    if (warp == 0) {
        long long z = 0;
        if (MODEL == 1)
            for (uint32_t u = 0; u < kNearRows; ++u) z += __popc(Sn[u][lane] & m);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(kFull, z, o);
        if (lane == 0) {
            const long long c0 = MODEL == 0 ? (long long)kNearRows * 32 * tw : z;
            atomicAdd(reinterpret_cast<unsigned long long*>(cx), (unsigned long long)c0);
            atomicAdd(reinterpret_cast<unsigned long long*>(cy), (unsigned long long)c0);
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
cudaError_t launch_x(const void* spins, uint32_t L, uint32_t rmax, long long* cx, int sms, cudaStream_t st)
{
    const uint32_t W32 = L / 32;
    const uint32_t groups = (rmax / 32 + 1 + NQ - 1) / NQ;   // word-offset groups of NQ
    const uint32_t gpb = groups < (uint32_t)kXGroupsMax ? groups : (uint32_t)kXGroupsMax;  // groups per block
    const uint32_t gy = (groups + gpb - 1) / gpb;
    // row parts: as many warps as fit kXWarpsMax, each part at least 8 groups of 2 NQ words
    uint32_t parts = kXWarpsMax / gpb;
    const uint32_t most = W32 / (16 * NQ);
    parts = parts < most ? parts : (most < 1 ? 1 : most);
    const uint32_t span = ((W32 + parts - 1) / parts + 2 * NQ - 1) / (2 * NQ) * (2 * NQ);
    const uint32_t nwarps = gpb * parts;
    // the largest word a warp reads is q0 + NQ + W32 (entering words run
    // from q0 + NQ + i0 up to word i1 - 1 <= W32 - 1, plus the next word of
    // each funnel shift), with q0 < gy * gpb * NQ
    const uint32_t ext = gy * gpb * NQ + NQ + W32 + 1;
    const size_t one_buf = (size_t)ext * Planes<MODEL>::n * sizeof(uint32_t);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const uint32_t nbuf = 2 * one_buf <= (size_t)optin ? 2u : 1u;  // two row buffers when they fit
    const size_t smem = nbuf * one_buf;
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(k_corr_x<MODEL, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // rows per block: enough blocks for about eight full waves, so the last
    // partial wave costs little; at least 8 rows per block
    int resident = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_corr_x<MODEL, NQ>, nwarps * 32, smem);
    if (e != cudaSuccess) return e;
    const uint64_t want_blocks = (uint64_t)sms * (resident < 1 ? 1 : resident) * 8 / gy + 1;
    uint32_t rpb = (uint32_t)((L + want_blocks - 1) / want_blocks);
    rpb = rpb < 8 ? 8 : rpb;
    // per-lane popcount sums stay below 2^31: at most L per row
    const uint32_t rmax_rows = (1u << 30) / L;
    rpb = rpb > rmax_rows ? rmax_rows : rpb;
    const dim3 grid((L + rpb - 1) / rpb, gy);
    k_corr_x<MODEL, NQ><<<grid, nwarps * 32, smem, st>>>(spins, L, rmax, rpb, cx, ext, nbuf, gpb, span, 1u);
    return cudaGetLastError();
}

template <int MODEL, int NQ>
cudaError_t launch_y(const void* spins, uint32_t L, uint32_t rmax, long long* cy, int sms, cudaStream_t st)
{
    const uint32_t W32 = L / 32;
    const size_t smem = (size_t)(YRing<NQ>::rows + 2 * YRing<NQ>::step) * 32 * Planes<MODEL>::n * sizeof(uint32_t);  // ring + two A buffers
    cudaError_t e = cudaFuncSetAttribute(k_corr_y<MODEL, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const uint32_t per_block = kYWarps * NQ;
    const uint32_t strips = (W32 + 31) / 32, chunks = (rmax + per_block) / per_block;
    // row segments: enough blocks for about eight full waves, segments of at least two steps
    int resident = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_corr_y<MODEL, NQ>, kYWarps * 32, smem);
    if (e != cudaSuccess) return e;
    const uint64_t want = (uint64_t)sms * (resident < 1 ? 1 : resident) * 8 / ((uint64_t)strips * chunks) + 1;
    uint32_t rpb = (uint32_t)((L + want - 1) / want);
    const uint32_t step = YRing<NQ>::step;
    const uint32_t minrows = 2 * step;
    rpb = rpb < minrows ? minrows : rpb;
    rpb = (rpb + step - 1) / step * step;  // a multiple of the (even) step, so every segment has an even row count
    const uint64_t nblocks = (uint64_t)strips * chunks * ((L + rpb - 1) / rpb);
    if (nblocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
    k_corr_y<MODEL, NQ><<<(unsigned)nblocks, kYWarps * 32, smem, st>>>(spins, L, rmax, rpb, cy, chunks, strips, 1u);
    return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch_xy(const void* spins, uint32_t L, uint32_t rmax, long long* cx, long long* cy, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    switch (pick_nq(rmax / 32 + 1, 1)) {
        case 4: e = launch_x<MODEL, 4>(spins, L, rmax, cx, sms, st); break;
        case 8: e = launch_x<MODEL, 8>(spins, L, rmax, cx, sms, st); break;
        case 11: e = launch_x<MODEL, 11>(spins, L, rmax, cx, sms, st); break;
        case 13: e = launch_x<MODEL, 13>(spins, L, rmax, cx, sms, st); break;
        default: e = launch_x<MODEL, 16>(spins, L, rmax, cx, sms, st); break;
    }
    if (e != cudaSuccess) return e;
    switch (pick_nq(rmax + 1, kYWarps)) {
        case 4: return launch_y<MODEL, 4>(spins, L, rmax, cy, sms, st);
        case 8: return launch_y<MODEL, 8>(spins, L, rmax, cy, sms, st);
        case 11: return launch_y<MODEL, 11>(spins, L, rmax, cy, sms, st);
        case 13: return launch_y<MODEL, 13>(spins, L, rmax, cy, sms, st);
        default: return launch_y<MODEL, 16>(spins, L, rmax, cy, sms, st);
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
    if (rmax <= kNear) {
        const dim3 grid((L / 32 + 31) / 32, L / kNearRows);
        if (model == 0) k_corr_near<0><<<grid, 256, 0, st>>>(spins, L, rmax, cx, cy, 1u);
        else k_corr_near<1><<<grid, 256, 0, st>>>(spins, L, rmax, cx, cy, 1u);
        return cudaGetLastError();
    }
    return model == 0 ? launch_xy<0>(spins, L, rmax, cx, cy, st) : launch_xy<1>(spins, L, rmax, cx, cy, st);
}

}  // namespace latk
