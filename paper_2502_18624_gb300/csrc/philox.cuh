// philox.cuh -- Philox4x32-10 for the sweep kernels (sm_103a).
//
// Generator of section 3.2 (the paper draws it through cuRAND's device API);
// written here from Salmon et al., SC'11.  State (c0,c1,c2,c3), key (k0,k1);
// one round maps it to
//     (hi(B*c2) ^ c1 ^ k0,  lo(B*c2),  hi(A*c0) ^ c3 ^ k1,  lo(A*c0))
// with A = 0xD2511F53, B = 0xCD9E8D57, and the key advances by
// (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.
//
// The ten round keys are computed once on the host and passed as kernel
// parameters, so every XOR with a key reads the constant bank.  The counter
// of a lattice decision is (site_lo, site_hi, sweep, colour): within one
// 128-site chunk of one phase only site_lo varies, so the first round's B*c2
// product and the second round's A*c0 product are the same for every site of
// the chunk.  PhiloxChunk holds those shared parts; philox_site_w0/w01 finish
// the remaining per-site work (17 multiplies instead of 20).
#pragma once
#include <cstdint>

namespace latk {

constexpr uint32_t kPhiloxA = 0xD2511F53u;
constexpr uint32_t kPhiloxB = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;
constexpr uint32_t kQuenchSweep = 0xFFFFFFFFu;

struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += kWeyl0;
        b += kWeyl1;
    }
    return rk;
}

__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t m, uint32_t& hi, uint32_t& lo)
{
    const uint64_t p = (uint64_t)a * (uint64_t)m;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Full generator, all four output words.
__device__ __forceinline__ uint4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         const RoundKeys& rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t h0, l0, h1, l1;
        mul_wide(c0, kPhiloxA, h0, l0);
        mul_wide(c2, kPhiloxB, h1, l1);
        c0 = h1 ^ c1 ^ rk.k0[r];
        c1 = l1;
        c2 = h0 ^ c3 ^ rk.k1[r];
        c3 = l0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Parts of rounds 1 and 2 shared by every site of a chunk with fixed
// (site_hi, sweep, colour).
struct PhiloxChunk {
    uint32_t r1_c1;   // state word 1 after round 1 (lo(B*sweep))
    uint32_t r2_h;    // hi(A * state word 0 after round 1) ^ k1[1]
    uint32_t r2_l;    // lo(A * state word 0 after round 1)
    uint32_t c3k;     // colour ^ k1[0]
};

__device__ __forceinline__ PhiloxChunk philox_chunk(uint32_t site_hi, uint32_t sweep, uint32_t colour,
                                                    const RoundKeys& rk)
{
    PhiloxChunk pc;
    uint32_t h1, l1;
    mul_wide(sweep, kPhiloxB, h1, l1);
    const uint32_t s0 = h1 ^ site_hi ^ rk.k0[0];  // round-1 state word 0
    pc.r1_c1 = l1;
    uint32_t h0, l0;
    mul_wide(s0, kPhiloxA, h0, l0);
    pc.r2_h = h0 ^ rk.k1[1];
    pc.r2_l = l0;
    pc.c3k = colour ^ rk.k1[0];
    return pc;
}

// Rounds 1..9 for one site; returns the state before round 10.
__device__ __forceinline__ void philox_site_r9(uint32_t site_lo, const PhiloxChunk& pc, const RoundKeys& rk,
                                               uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3)
{
    // Round 1: word 0 and 1 are chunk-wide; A*site_lo is per site.
    uint32_t h, l;
    mul_wide(site_lo, kPhiloxA, h, l);
    const uint32_t s2 = h ^ pc.c3k;
    const uint32_t s3 = l;
    // Round 2: A*s0 is chunk-wide.
    mul_wide(s2, kPhiloxB, h, l);
    c0 = h ^ pc.r1_c1 ^ rk.k0[1];
    c1 = l;
    c2 = pc.r2_h ^ s3;
    c3 = pc.r2_l;
#pragma unroll
    for (int r = 2; r < 9; ++r) {
        uint32_t h0, l0, h1, l1;
        mul_wide(c0, kPhiloxA, h0, l0);
        mul_wide(c2, kPhiloxB, h1, l1);
        c0 = h1 ^ c1 ^ rk.k0[r];
        c1 = l1;
        c2 = h0 ^ c3 ^ rk.k1[r];
        c3 = l0;
    }
}

// Output word 0 only (Ising decision).
__device__ __forceinline__ uint32_t philox_site_w0(uint32_t site_lo, const PhiloxChunk& pc, const RoundKeys& rk)
{
    uint32_t c0, c1, c2, c3;
    philox_site_r9(site_lo, pc, rk, c0, c1, c2, c3);
    return __umulhi(c2, kPhiloxB) ^ c1 ^ rk.k0[9];
}

// All four output words (lookup-table random bits).
__device__ __forceinline__ uint4 philox_site_w4(uint32_t site_lo, const PhiloxChunk& pc, const RoundKeys& rk)
{
    uint32_t c0, c1, c2, c3;
    philox_site_r9(site_lo, pc, rk, c0, c1, c2, c3);
    uint32_t h0, l0, h1, l1;
    mul_wide(c0, kPhiloxA, h0, l0);
    mul_wide(c2, kPhiloxB, h1, l1);
    return make_uint4(h1 ^ c1 ^ rk.k0[9], l1, h0 ^ c3 ^ rk.k1[9], l0);
}

// Output words 0 and 1 (Blume-Capel decision and proposal).
__device__ __forceinline__ uint2 philox_site_w01(uint32_t site_lo, const PhiloxChunk& pc, const RoundKeys& rk)
{
    uint32_t c0, c1, c2, c3;
    philox_site_r9(site_lo, pc, rk, c0, c1, c2, c3);
    uint32_t h, l;
    mul_wide(c2, kPhiloxB, h, l);
    return make_uint2(h ^ c1 ^ rk.k0[9], l);
}

}  // namespace latk
