/*
 * oracle.c -- plain, slow, obviously correct CPU restatement of the
 * checkerboard Metropolis method of Bisson et al., "Massive-Scale Simulations
 * of 2D Ising and Blume-Capel Models on Rack-Scale Multi-GPU Systems"
 * (arXiv 2502.18624).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may load this
 * code.  It shares no source with the CUDA library (its Philox, threshold
 * tables, packing and hash are written here independently), and the CUDA
 * library never calls it.
 *
 * Representation: one int8 per spin, s[y*L + x], x the column (fastest),
 * values -1/+1 (Ising) or -1/0/+1 (Blume-Capel).  All sums are exact int64.
 * The only floating point is the FP64 threshold table and the
 * Schwinger-Dyson combination done by callers.
 *
 * Parity pins (what fixes each function independently of this file):
 *   or_philox4x32_10   cuRAND's host-side Philox4_32_10 generator
 *                      (tests/test_oracle_philox.py) and, on a GPU, the
 *                      cuRAND device API.
 *   or_thresholds_*    closed form in 80-digit arithmetic and detailed
 *                      balance (tests/test_oracle_thresholds.py).
 *   or_init/or_sweep   exact enumeration of 4x4 Ising and 3x3 Blume-Capel,
 *                      Onsager's u(T), +-flip symmetry, T->0 monotonicity
 *                      (tests/test_oracle_physics.py).
 *   or_measure         brute-force energy of each enumerated state.
 *   or_correlation     numpy FFT autocorrelation; C(0), reflection and the
 *                      bond identity B = Cx(1) + Cy(1).
 *   or_sd_hist         Eq. (3) equals 1 exactly under the enumerated
 *                      Boltzmann weights.
 *   or_protocol_*      the integers the section 3.3 formulas give when
 *                      evaluated in 60-digit decimal arithmetic, and the
 *                      structure of the distance and time sets
 *                      (tests/test_oracle_protocol.py).
 *   or_correlation_sampled  equals or_correlation at R = 1; numpy array
 *                      form (strided sources, rolled targets).
 *   or_lut_table       80-digit closed form of the cumulative pattern
 *                      probabilities (tests/test_oracle_lut.py).
 *   or_sweep_lut       Kaufman's exact finite-torus energy and Onsager's
 *                      energy reproduced by long runs; frequencies of the
 *                      generated bits; +-flip symmetry.
 *   or_init_window, or_sweep_window, or_sweep_window_lut  the interior
 *                      after t calls equals the periodic lattice's after t
 *                      sweeps (or_run / or_run_lut), windows across the seams
 *                      (tests/test_oracle_window.py).
 *   or_sweep_par, or_sweep_strip_par  equal to or_sweep / or_sweep_strip for
 *                      every thread count tried (tests/test_oracle_threads.py).
 *   or_pack            numpy.packbits (tests/test_oracle_measure.py).
 *   or_hash_words/or_hash  every one-bit change of every canonical word and
 *                      every exchange of two unequal words changes the hash;
 *                      the Blume-Capel planes are not interchangeable; the
 *                      mixer's avalanche (each input bit flips each output bit
 *                      with frequency near 1/2) (tests/test_oracle_hash.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror and Shaw, "Parallel      */
/* random numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter, a 2-word    */
/* key, ten rounds; each round multiplies words 0 and 2 by the two round      */
/* multipliers (32x32->64), and the new state is                              */
/*   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0));        */
/* the key is bumped by the two Weyl constants between rounds.  The paper     */
/* uses this generator through cuRAND's device API (section 3.2).             */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += OR_PHILOX_W0;
        k1 += OR_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Vectorised form for tests: n counters (4 words each) under one key. */
void or_philox_many(const uint32_t* ctrs, size_t n, const uint32_t key[2], uint32_t* outs)
{
    for (size_t i = 0; i < n; ++i) or_philox4x32_10(ctrs + 4 * i, key, outs + 4 * i);
}

/* The random stream of a lattice: key = (seed low word, seed high word);    */
/* counter = (site low word, site high word, sweep, colour), site = y*L + x. */
/* Sweep index 0xFFFFFFFF with colour 0 is the initial quench.               */
static void or_draw(uint64_t seed, uint64_t site, uint32_t sweep, uint32_t colour, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)site, (uint32_t)(site >> 32), sweep, colour};
    or_philox4x32_10(ctr, key, w);
}

#define OR_INIT_SWEEP 0xFFFFFFFFu
#define OR_ALWAYS (((uint64_t)1) << 32)

/* ------------------------------------------------------------------------ */
/* Acceptance thresholds.  Metropolis accepts a move of energy change dE      */
/* with probability min(1, exp(-dE/T)) (section 3.2 states the Ising case:    */
/* e^{-4 beta}, e^{-8 beta}, else 1).  Integer form: thr = 2^32 (ALWAYS) when */
/* dE <= 0, else floor(2^32 exp(-dE/T)) clamped to 2^32; a move is accepted   */
/* iff thr == ALWAYS or u < thr for a uniform 32-bit u.                       */
/* ------------------------------------------------------------------------ */
static uint64_t or_thr(double dE, double T)
{
    if (dE <= 0.0) return OR_ALWAYS;
    double v = floor(ldexp(exp(-dE / T), 32));
    if (v >= 4294967296.0) return OR_ALWAYS;
    if (v <= 0.0) return 0;
    return (uint64_t)v;
}

/* Ising, Eq. (1): flipping s with neighbour sum h costs dE = 2 J s h.       */
/* Entry i (0..4) is for the product k = s*h = 2*i - 4.                       */
void or_thresholds_ising(double J, double T, uint64_t thr[5])
{
    for (int i = 0; i < 5; ++i) {
        int k = 2 * i - 4;
        thr[i] = or_thr(2.0 * J * (double)k, T);
    }
}

/* The two values a Blume-Capel spin s may move to, in ascending order.     */
static int or_bc_other(int s, int b)
{
    static const int others[3][2] = {{0, 1}, {-1, 1}, {-1, 0}};
    return others[s + 1][b];
}

/* Blume-Capel, Eq. (2): moving s -> s' with neighbour sum h costs           */
/* dE = -J (s' - s) h + Delta (s'^2 - s^2).  Entry ((s+1)*2 + b)*9 + (h+4),  */
/* s' the b-th other value of s in ascending order.                          */
void or_thresholds_bc(double J, double Delta, double T, uint64_t thr[54])
{
    for (int s = -1; s <= 1; ++s)
        for (int b = 0; b < 2; ++b)
            for (int h = -4; h <= 4; ++h) {
                int sp = or_bc_other(s, b);
                double dE = -J * (double)(sp - s) * (double)h + Delta * (double)(sp * sp - s * s);
                thr[((s + 1) * 2 + b) * 9 + (h + 4)] = or_thr(dE, T);
            }
}

/* ------------------------------------------------------------------------ */
/* Initial quench from infinite temperature (section 1: the system starts    */
/* at high temperature).  Ising: s = +1 iff bit 31 of word 0 is set.          */
/* Blume-Capel: s = floor(3 * w0 / 2^32) - 1, uniform over {-1,0,+1}.         */
/* ------------------------------------------------------------------------ */
void or_init(int model, uint32_t L, uint64_t seed, int8_t* s)
{
    for (uint64_t y = 0; y < L; ++y)
        for (uint64_t x = 0; x < L; ++x) {
            uint64_t site = y * L + x;
            uint32_t w[4];
            or_draw(seed, site, OR_INIT_SWEEP, 0, w);
            if (model == 0)
                s[site] = (w[0] >> 31) ? 1 : -1;
            else
                s[site] = (int8_t)((int)(((uint64_t)w[0] * 3u) >> 32) - 1);
        }
}

/* The same quench for rows y0 .. y0+nrows-1 (mod L) only, into an          */
/* nrows x L array: used to check lattices too large to hold as int8.       */
void or_init_rows(int model, uint32_t L, uint64_t seed, uint64_t y0, uint32_t nrows, int8_t* s)
{
    for (uint64_t r = 0; r < nrows; ++r) {
        uint64_t y = (y0 + r) % L;
        for (uint64_t x = 0; x < L; ++x) {
            uint32_t w[4];
            or_draw(seed, y * L + x, OR_INIT_SWEEP, 0, w);
            int8_t v;
            if (model == 0)
                v = (w[0] >> 31) ? 1 : -1;
            else
                v = (int8_t)((int)(((uint64_t)w[0] * 3u) >> 32) - 1);
            s[r * L + x] = v;
        }
    }
}

/* One Metropolis decision for the spin value sv with neighbour sum h at the  */
/* given site, during sweep `sweep` and colour phase `colour`.                */
static int8_t or_update_site(int model, int sv, int h, uint64_t site, uint32_t sweep, uint32_t colour,
                             uint64_t seed, const uint64_t* thr)
{
    if (model == 0) {
        /* Ising: the proposal is -sv; word 0 decides. */
        uint64_t t = thr[(sv * h + 4) / 2];
        if (t == OR_ALWAYS) return (int8_t)(-sv);
        uint32_t w[4];
        or_draw(seed, site, sweep, colour, w);
        return (uint64_t)w[0] < t ? (int8_t)(-sv) : (int8_t)sv;
    } else {
        /* Blume-Capel: word 1's low bit picks the proposal, word 0 decides. */
        uint32_t w[4];
        or_draw(seed, site, sweep, colour, w);
        int b = (int)(w[1] & 1u);
        int sp = or_bc_other(sv, b);
        uint64_t t = thr[((sv + 1) * 2 + b) * 9 + (h + 4)];
        if (t == OR_ALWAYS || (uint64_t)w[0] < t) return (int8_t)sp;
        return (int8_t)sv;
    }
}

/* ------------------------------------------------------------------------ */
/* One sweep (section 3.1): colour 0 (x+y even) then colour 1 (x+y odd).     */
/* Same-colour sites have no common bond when L is even, so the in-colour    */
/* order is irrelevant; the loop below is plainly sequential and in place.   */
/* Periodic boundaries (Eq. (1)).                                            */
/* ------------------------------------------------------------------------ */
void or_sweep(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep, int8_t* s)
{
    for (uint32_t colour = 0; colour < 2; ++colour)
        for (uint64_t y = 0; y < L; ++y)
            for (uint64_t x = 0; x < L; ++x) {
                if (((x + y) & 1u) != colour) continue;
                uint64_t site = y * L + x;
                int h = s[((y + L - 1) % L) * L + x] + s[((y + 1) % L) * L + x] +
                        s[y * L + (x + L - 1) % L] + s[y * L + (x + 1) % L];
                s[site] = or_update_site(model, s[site], h, site, sweep, colour, seed, thr);
            }
}

/* Several sweeps, recording (M, B, Q) after each one when obs != NULL.      */
void or_measure(int model, uint32_t L, const int8_t* s, int64_t out[3]);
void or_run(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t first_sweep,
            uint32_t nsweeps, int8_t* s, int64_t* obs)
{
    for (uint32_t i = 0; i < nsweeps; ++i) {
        or_sweep(model, L, seed, thr, first_sweep + i, s);
        if (obs) or_measure(model, L, s, obs + 3 * (size_t)i);
    }
}

/* The same sweep restricted to a horizontal strip, for lattices too large   */
/* to hold as int8.  `strip` holds the H+4 full rows y0-2 .. y0+H+1 (mod L). */
/* Colour 0 is updated on strip rows 1..H+2 and colour 1 on rows 2..H+1;     */
/* afterwards rows 2..H+1 equal global rows y0..y0+H-1 after the sweep,      */
/* because each phase reads only nearest neighbours.  Sites keep their       */
/* global index y*L + x for the random stream.                               */
void or_sweep_strip(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep,
                    uint64_t y0, uint32_t H, int8_t* strip)
{
    for (uint32_t colour = 0; colour < 2; ++colour) {
        uint32_t r_lo = colour == 0 ? 1 : 2;
        uint32_t r_hi = colour == 0 ? H + 3 : H + 2;
        for (uint32_t r = r_lo; r < r_hi; ++r) {
            uint64_t y = (y0 + (uint64_t)L * 4 + r - 2) % L;
            for (uint64_t x = 0; x < L; ++x) {
                if (((x + y) & 1u) != colour) continue;
                int8_t* row = strip + (size_t)r * L;
                int h = strip[(size_t)(r - 1) * L + x] + strip[(size_t)(r + 1) * L + x] +
                        row[(x + L - 1) % L] + row[(x + 1) % L];
                row[x] = or_update_site(model, row[x], h, y * L + x, sweep, colour, seed, thr);
            }
        }
    }
}

/* The quench of a window: win[i*Wd + j] = the initial spin of the global    */
/* site ((y0 + i) mod L, (x0 + j) mod L), i < H, j < Wd.                     */
void or_init_window(int model, uint32_t L, uint64_t seed, uint64_t y0, uint64_t x0, uint32_t H, uint32_t Wd,
                    int8_t* win)
{
    for (uint64_t i = 0; i < H; ++i)
        for (uint64_t j = 0; j < Wd; ++j) {
            uint64_t y = (y0 + i) % L, x = (x0 + j) % L;
            uint32_t w[4];
            or_draw(seed, y * L + x, OR_INIT_SWEEP, 0, w);
            if (model == 0)
                win[i * Wd + j] = (w[0] >> 31) ? 1 : -1;
            else
                win[i * Wd + j] = (int8_t)((int)(((uint64_t)w[0] * 3u) >> 32) - 1);
        }
}

/* One sweep of a window that is not periodic (a light-cone check for       */
/* lattices too large to hold as int8).  win holds H x Wd spins, element    */
/* (i, j) being the global site ((y0 + i) mod L, (x0 + j) mod L); H, Wd <= L. */
/* Colour 0 is updated where 1 <= i < H-1 and 1 <= j < Wd-1 (every such site */
/* has its four neighbours in the window), then colour 1 where 2 <= i < H-2  */
/* and 2 <= j < Wd-2, each site with its global index for the random stream. */
/* A phase reads only nearest neighbours, so after t calls the block         */
/* 2t <= i < H-2t, 2t <= j < Wd-2t equals the periodic lattice after the     */
/* same t sweeps; the band outside it holds values of no meaning.            */
void or_sweep_window(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep, uint64_t y0,
                     uint64_t x0, uint32_t H, uint32_t Wd, int8_t* win)
{
    for (uint32_t colour = 0; colour < 2; ++colour) {
        uint32_t m = colour == 0 ? 1 : 2;
        for (uint64_t i = m; i + m < H; ++i)
            for (uint64_t j = m; j + m < Wd; ++j) {
                uint64_t y = (y0 + i) % L, x = (x0 + j) % L;
                if (((x + y) & 1u) != colour) continue;
                int8_t* c = win + i * Wd + j;
                int h = c[-(int64_t)Wd] + c[Wd] + c[-1] + c[1];
                *c = or_update_site(model, *c, h, y * L + x, sweep, colour, seed, thr);
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Multi-threaded forms, for timing the oracle on every host core.  A colour  */
/* phase updates sites that share no bond (section 3.1), so its rows can be   */
/* shared out among threads in any way: each site is updated by the same      */
/* or_update_site as in the sequential loops, from the same neighbours, and   */
/* the result equals or_sweep / or_sweep_strip exactly.  Built with OpenMP    */
/* when the host compiler has it; otherwise these run on one thread.          */
/* ------------------------------------------------------------------------ */
int or_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void or_phase_rows(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep,
                          uint32_t colour, uint64_t y, int8_t* row, const int8_t* up, const int8_t* down)
{
    for (uint64_t x = (colour + y) & 1u; x < L; x += 2) {
        int h = up[x] + down[x] + row[(x + L - 1) % L] + row[(x + 1) % L];
        row[x] = or_update_site(model, row[x], h, y * L + x, sweep, colour, seed, thr);
    }
}

void or_sweep_par(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep, int8_t* s,
                  int nthreads)
{
    (void)nthreads;
    for (uint32_t colour = 0; colour < 2; ++colour) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int64_t y = 0; y < (int64_t)L; ++y)
            or_phase_rows(model, L, seed, thr, sweep, colour, (uint64_t)y, s + (size_t)y * L,
                          s + (size_t)((y + L - 1) % L) * L, s + (size_t)((y + 1) % L) * L);
    }
}

/* Strip form (as or_sweep_strip: strip rows 2..H+1 become exact). */
void or_sweep_strip_par(int model, uint32_t L, uint64_t seed, const uint64_t* thr, uint32_t sweep, uint64_t y0,
                        uint32_t H, int8_t* strip, int nthreads)
{
    (void)nthreads;
    for (uint32_t colour = 0; colour < 2; ++colour) {
        int64_t r_lo = colour == 0 ? 1 : 2;
        int64_t r_hi = colour == 0 ? (int64_t)H + 3 : (int64_t)H + 2;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int64_t r = r_lo; r < r_hi; ++r) {
            uint64_t y = (y0 + (uint64_t)L * 4 + (uint64_t)r - 2) % L;
            or_phase_rows(model, L, seed, thr, sweep, colour, y, strip + (size_t)r * L, strip + (size_t)(r - 1) * L,
                          strip + (size_t)(r + 1) * L);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* The paper's lookup-table random bits for the Ising model (section 3.2).   */
/* A word of random bits, each set independently with probability           */
/* p = exp(-4 J / T), is produced four bits at a time: a uniform 32-bit u    */
/* is located in a sorted table of 16 entries, and the index of the largest  */
/* entry not above u is itself the four bits.  Table: tbl[j] = floor(2^32 *  */
/* sum over patterns m < j of p^popcount(m) (1-p)^(4-popcount(m))), so index */
/* j comes out with probability of pattern j (to within 2^-32).  A site with */
/* all four neighbours equal to it flips iff its bit in one such word AND    */
/* its bit in a second, independent word are set (probability p^2 =          */
/* exp(-8J/T)); with exactly three iff its bit in the first word is set;     */
/* every other site flips.  (The paper defers the table construction to a    */
/* companion reference; the construction above is this library's reading.)  */
/*                                                                           */
/* Stream: the 64-bit word w = y*(L/64) + x/64 draws, in sweep t and colour  */
/* phase c, the Philox blocks at counters (4w+q low, 4w+q high, t, c+2),     */
/* q = 0..3; uniform i = 4q + k is word k of block q.  Uniforms 0..7 give    */
/* the first word of bits, uniforms 8..15 the second, lookup l giving bits   */
/* 4l .. 4l+3.  The word's active sites (those of colour c, in increasing x) */
/* take bits 0..31 in order.                                                 */
/* ------------------------------------------------------------------------ */
void or_lut_table(double J, double T, uint32_t tbl[16])
{
    double p = exp(-4.0 * J / T);
    double cum = 0.0;
    for (int j = 0; j < 16; ++j) {
        double v = floor(ldexp(cum, 32));
        tbl[j] = v >= 4294967295.0 ? 4294967295u : (uint32_t)v;
        int k = __builtin_popcount((unsigned)j);
        cum += pow(p, k) * pow(1.0 - p, 4 - k);
    }
}

static int or_lut_index(const uint32_t tbl[16], uint32_t u)
{
    int best = 0;
    for (int j = 0; j < 16; ++j)
        if (tbl[j] <= u) best = j;
    return best;
}

/* Bit `bit` (0..31) of random word `which` (0 or 1) of the word w. */
static int or_lut_bit(uint64_t seed, const uint32_t tbl[16], uint64_t w, uint32_t sweep, uint32_t colour,
                      int which, int bit)
{
    int i = 8 * which + bit / 4;              /* uniform index 0..15 */
    uint64_t ctr = 4 * w + (uint64_t)(i / 4);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c[4] = {(uint32_t)ctr, (uint32_t)(ctr >> 32), sweep, colour + 2u};
    uint32_t out[4];
    or_philox4x32_10(c, key, out);
    int j = or_lut_index(tbl, out[i % 4]);
    return (j >> (bit % 4)) & 1;
}

void or_sweep_lut(uint32_t L, uint64_t seed, const uint32_t tbl[16], uint32_t sweep, int8_t* s)
{
    for (uint32_t colour = 0; colour < 2; ++colour)
        for (uint64_t y = 0; y < L; ++y)
            for (uint64_t x = 0; x < L; ++x) {
                if (((x + y) & 1u) != colour) continue;
                uint64_t site = y * L + x;
                int sv = s[site];
                int agree = (s[((y + L - 1) % L) * L + x] == sv) + (s[((y + 1) % L) * L + x] == sv) +
                            (s[y * L + (x + L - 1) % L] == sv) + (s[y * L + (x + 1) % L] == sv);
                uint64_t w = y * (L / 64) + x / 64;
                int k = (int)((x % 64) / 2); /* rank of x among the word's colour-c sites */
                int flip;
                if (agree == 4)
                    flip = or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 0, k) &
                           or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 1, k);
                else if (agree == 3)
                    flip = or_lut_bit(seed, tbl, w, (uint32_t)sweep, colour, 0, k);
                else
                    flip = 1;
                if (flip) s[site] = (int8_t)(-sv);
            }
}

/* The lookup-table sweep restricted to a strip (as or_sweep_strip): strip  */
/* holds the H+4 full rows y0-2 .. y0+H+1 (mod L); rows 2..H+1 become the    */
/* global rows y0..y0+H-1 after the sweep.                                   */
void or_sweep_strip_lut(uint32_t L, uint64_t seed, const uint32_t tbl[16], uint32_t sweep, uint64_t y0,
                        uint32_t H, int8_t* strip)
{
    for (uint32_t colour = 0; colour < 2; ++colour) {
        uint32_t r_lo = colour == 0 ? 1 : 2;
        uint32_t r_hi = colour == 0 ? H + 3 : H + 2;
        for (uint32_t r = r_lo; r < r_hi; ++r) {
            uint64_t y = (y0 + (uint64_t)L * 4 + r - 2) % L;
            int8_t* row = strip + (size_t)r * L;
            for (uint64_t x = 0; x < L; ++x) {
                if (((x + y) & 1u) != colour) continue;
                int sv = row[x];
                int agree = (strip[(size_t)(r - 1) * L + x] == sv) + (strip[(size_t)(r + 1) * L + x] == sv) +
                            (row[(x + L - 1) % L] == sv) + (row[(x + 1) % L] == sv);
                uint64_t w = y * (L / 64) + x / 64;
                int k = (int)((x % 64) / 2);
                int flip;
                if (agree == 4)
                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k) & or_lut_bit(seed, tbl, w, sweep, colour, 1, k);
                else if (agree == 3)
                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k);
                else
                    flip = 1;
                if (flip) row[x] = (int8_t)(-sv);
            }
        }
    }
}

/* The lookup-table sweep of a window that is not periodic (as             */
/* or_sweep_window, with the flip rule and stream of or_sweep_lut).         */
void or_sweep_window_lut(uint32_t L, uint64_t seed, const uint32_t tbl[16], uint32_t sweep, uint64_t y0,
                         uint64_t x0, uint32_t H, uint32_t Wd, int8_t* win)
{
    for (uint32_t colour = 0; colour < 2; ++colour) {
        uint32_t m = colour == 0 ? 1 : 2;
        for (uint64_t i = m; i + m < H; ++i)
            for (uint64_t j = m; j + m < Wd; ++j) {
                uint64_t y = (y0 + i) % L, x = (x0 + j) % L;
                if (((x + y) & 1u) != colour) continue;
                int8_t* c = win + i * Wd + j;
                int sv = *c;
                int agree = (c[-(int64_t)Wd] == sv) + (c[Wd] == sv) + (c[-1] == sv) + (c[1] == sv);
                uint64_t w = y * (L / 64) + x / 64;
                int k = (int)((x % 64) / 2);
                int flip;
                if (agree == 4)
                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k) & or_lut_bit(seed, tbl, w, sweep, colour, 1, k);
                else if (agree == 3)
                    flip = or_lut_bit(seed, tbl, w, sweep, colour, 0, k);
                else
                    flip = 1;
                if (flip) *c = (int8_t)(-sv);
            }
    }
}

/* Several lookup-table sweeps, recording (M, B, Q) after each when obs != NULL. */
void or_run_lut(uint32_t L, uint64_t seed, const uint32_t tbl[16], uint32_t first_sweep, uint32_t nsweeps,
                int8_t* s, int64_t* obs)
{
    for (uint32_t i = 0; i < nsweeps; ++i) {
        or_sweep_lut(L, seed, tbl, first_sweep + i, s);
        if (obs) or_measure(0, L, s, obs + 3 * (size_t)i);
    }
}

/* Random bit words for tests: bits of word `which` for the word w. */
uint32_t or_lut_word(uint64_t seed, const uint32_t tbl[16], uint64_t w, uint32_t sweep, uint32_t colour, int which)
{
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) v |= (uint32_t)or_lut_bit(seed, tbl, w, sweep, colour, which, b) << b;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Observables of Eqs. (1)-(2): M = sum s, Q = sum s^2 and the bond sum      */
/* B = sum over nearest-neighbour pairs s_x s_y, each bond counted once      */
/* (right and down neighbours, periodic).  E = -J B + Delta Q.               */
/* ------------------------------------------------------------------------ */
void or_measure(int model, uint32_t L, const int8_t* s, int64_t out[3])
{
    (void)model;
    int64_t M = 0, B = 0, Q = 0;
    for (uint64_t y = 0; y < L; ++y)
        for (uint64_t x = 0; x < L; ++x) {
            int v = s[y * L + x];
            M += v;
            Q += v * v;
            B += v * s[y * L + (x + 1) % L];
            B += v * s[((y + 1) % L) * L + x];
        }
    out[0] = M; out[1] = B; out[2] = Q;
}

/* Spin-spin correlation from every site along both lattice axes (section    */
/* 3.3, first item of the protocol, applied to every distance asked for):    */
/* cx[r] = sum_{x,y} s(x,y) s(x+r,y), cy[r] = sum_{x,y} s(x,y) s(x,y+r),     */
/* periodic, r = 0..rmax, raw int64 sums.                                    */
void or_correlation(uint32_t L, const int8_t* s, uint32_t rmax, int64_t* cx, int64_t* cy)
{
    for (uint32_t r = 0; r <= rmax; ++r) {
        int64_t ax = 0, ay = 0;
        for (uint64_t y = 0; y < L; ++y)
            for (uint64_t x = 0; x < L; ++x) {
                int v = s[y * L + x];
                ax += v * s[y * L + (x + r) % L];
                ay += v * s[((y + r) % L) * L + x];
            }
        cx[r] = ax;
        cy[r] = ay;
    }
}

/* ------------------------------------------------------------------------ */
/* The correlation protocol of section 3.3.                                   */
/*   R = 16; every site is a source for r <= 2R; beyond that the sources are  */
/*   one site per R x R square (its top-left corner, x % R == 0 and           */
/*   y % R == 0), for every r up to r_c(t) and then for the log-spaced        */
/*   distances floor(2^(x/32)) up to L/2.                                     */
/*   r_c(t) = max{256, floor(g(L) sqrt(t) + 0.5)},                            */
/*   g(L)   = 6 sqrt(ln(L / 2^16) / 3.3^2 + 1)   (natural logarithm).         */
/*   Measurement times: t = floor(2^(x/8) + 0.5), x = 1, 2, ...               */
/* All of it is computed in FP64, in the order the formulas are written.      */
/* ------------------------------------------------------------------------ */
uint64_t or_protocol_rc(uint32_t L, uint64_t t)
{
    const double g = 6.0 * sqrt(log((double)L / 65536.0) / (3.3 * 3.3) + 1.0);
    const double v = floor(g * sqrt((double)t) + 0.5);
    return v > 256.0 ? (uint64_t)v : 256u;
}

/* The distances measured from the downsampled sources at time t, ascending: */
/* every r with 2R < r <= min(r_c, L/2), then every distinct floor(2^(x/32)) */
/* with r_c < floor(2^(x/32)), for x up to 32 (log2(L) - 1) (i.e. r <= L/2). */
/* Returns the count; writes at most cap values.                             */
uint32_t or_protocol_distances(uint32_t L, uint64_t t, uint32_t R, uint32_t* out, uint32_t cap)
{
    const uint64_t rc = or_protocol_rc(L, t);
    const uint64_t half = L / 2;
    const uint64_t dense_end = rc < half ? rc : half;
    uint32_t n = 0;
    for (uint64_t r = 2 * (uint64_t)R + 1; r <= dense_end; ++r) {
        if (n < cap) out[n] = (uint32_t)r;
        ++n;
    }
    uint64_t last = dense_end;
    for (uint32_t x = 1;; ++x) {
        const double v = floor(exp2((double)x / 32.0));
        if (v > (double)half) break;
        const uint64_t r = (uint64_t)v;
        if (r <= rc || r <= last) continue;
        if (n < cap) out[n] = (uint32_t)r;
        ++n;
        last = r;
    }
    return n;
}

/* Distinct measurement times floor(2^(x/8) + 0.5) <= tmax, x = 1, 2, ...,   */
/* ascending.  Returns the count; writes at most cap values.                 */
uint32_t or_protocol_times(uint64_t tmax, uint64_t* out, uint32_t cap)
{
    uint32_t n = 0;
    uint64_t last = 0;
    for (uint32_t x = 1;; ++x) {
        const double v = floor(exp2((double)x / 8.0) + 0.5);
        if (v > (double)tmax) break;
        const uint64_t t = (uint64_t)v;
        if (t == last) continue;
        if (n < cap) out[n] = t;
        ++n;
        last = t;
    }
    return n;
}

/* Correlation from the downsampled sources (one per R x R square, the       */
/* top-left corner): for each listed r,                                      */
/* cx = sum over x % R == 0, y % R == 0 of s(x,y) s(x+r,y), cy likewise with */
/* s(x,y+r); periodic, raw int64 sums over (L/R)^2 sources.                  */
void or_correlation_sampled(uint32_t L, const int8_t* s, uint32_t R, const uint32_t* r, uint32_t nr,
                            int64_t* cx, int64_t* cy)
{
    for (uint32_t i = 0; i < nr; ++i) {
        int64_t ax = 0, ay = 0;
        for (uint64_t y = 0; y < L; y += R)
            for (uint64_t x = 0; x < L; x += R) {
                int v = s[y * L + x];
                ax += v * s[y * L + (x + r[i]) % L];
                ay += v * s[((y + r[i]) % L) * L + x];
            }
        cx[i] = ax;
        cy[i] = ay;
    }
}

/* Schwinger-Dyson check of Eq. (3): histogram of sigma_x * h_x over all     */
/* sites, bins v = -4..4 at index v+4.  Eq. (3)'s right-hand side is then    */
/* L^-2 sum_v hist[v] exp(-2 J beta v).                                      */
void or_sd_hist(uint32_t L, const int8_t* s, int64_t hist[9])
{
    for (int i = 0; i < 9; ++i) hist[i] = 0;
    for (uint64_t y = 0; y < L; ++y)
        for (uint64_t x = 0; x < L; ++x) {
            int h = s[((y + L - 1) % L) * L + x] + s[((y + 1) % L) * L + x] +
                    s[y * L + (x + L - 1) % L] + s[y * L + (x + 1) % L];
            hist[s[y * L + x] * h + 4] += 1;
        }
}

/* ------------------------------------------------------------------------ */
/* Canonical packing and lattice hash, used to compare a lattice with one    */
/* kept elsewhere without moving it.  Words per row W = L/64; bit b of word  */
/* (y, j) is the site x = 64 j + b.  Ising: one plane, bit set iff s = +1.   */
/* Blume-Capel: plane 0 (words 0 .. L*W-1) bit set iff s != 0, plane 1      */
/* (words L*W .. 2*L*W-1) bit set iff s = -1.                                 */
/* hash = sum over canonical words i of mix(i ^ word_i) mod 2^64, mix the    */
/* SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014).                */
/* ------------------------------------------------------------------------ */
void or_pack(int model, uint32_t L, const int8_t* s, uint64_t* words)
{
    uint64_t W = L / 64, n = (uint64_t)L * W;
    memset(words, 0, (model == 0 ? n : 2 * n) * sizeof(uint64_t));
    for (uint64_t y = 0; y < L; ++y)
        for (uint64_t x = 0; x < L; ++x) {
            int v = s[y * L + x];
            uint64_t i = y * W + x / 64, bit = ((uint64_t)1) << (x % 64);
            if (model == 0) {
                if (v == 1) words[i] |= bit;
            } else {
                if (v != 0) words[i] |= bit;
                if (v == -1) words[n + i] |= bit;
            }
        }
}

static uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t or_hash_words(const uint64_t* words, uint64_t nwords)
{
    uint64_t h = 0;
    for (uint64_t i = 0; i < nwords; ++i) h += or_mix64(i ^ words[i]);
    return h;
}

uint64_t or_hash(int model, uint32_t L, const int8_t* s)
{
    uint64_t W = L / 64, n = (uint64_t)L * W * (model == 0 ? 1 : 2);
    uint64_t* words = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!words) return 0;
    or_pack(model, L, s, words);
    uint64_t h = or_hash_words(words, n);
    free(words);
    return h;
}
