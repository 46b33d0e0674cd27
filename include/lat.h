/*
 * lat.h -- C ABI of the GB300 (sm_103a) checkerboard Metropolis library for
 * the 2D Ising and Blume-Capel models (Bisson et al., arXiv 2502.18624).
 *
 * The problem (section "Nature of problem", section 2): an L x L square
 * lattice with periodic boundaries, Hamiltonian Eq. (1) (Ising, s = +-1) or
 * Eq. (2) (Blume-Capel, s in {-1, 0, +1}), evolved by single-spin-flip
 * Metropolis dynamics (section 1) in checkerboard order: every sweep updates
 * the sites with x+y even (colour 0), then those with x+y odd (colour 1)
 * (section 3.1).  Measurements are the exact integer sums behind the energy
 * and magnetisation, and the spin-spin correlation from every site along
 * both axes (section 3.3).
 *
 * Random stream.  Every decision draws Philox4x32-10 (section 3.2) with
 * key = (seed low 32 bits, seed high 32 bits) and counter
 * (site low 32 bits, site high 32 bits, sweep index, colour), site = y*L + x.
 * The initial quench uses sweep index 0xFFFFFFFF and colour 0.  Ising: a
 * site with dE = 2 J s h <= 0 flips; otherwise it flips iff word 0 < thr[dE].
 * Blume-Capel: every site draws; the low bit of word 1 picks the proposal
 * among the two other values in ascending order, and the move is accepted
 * iff dE <= 0 or word 0 < thr.  thr = floor(2^32 exp(-dE/T)), built once in
 * FP64 on the host.  Because the stream is counter-based and same-colour
 * sites share no bond, every result is independent of launch shape, tiling
 * and batching.
 *
 * Conventions for every call:
 *   - return 0 (LAT_OK) on success or a negative LAT_E* code; no call throws.
 *   - handles are not thread-safe; one handle is used by one host thread.
 *   - device work is ordered on the handle's CUDA stream; calls that return
 *     host data synchronise that stream before returning.
 *   - there is no CPU fallback: without a usable CUDA device the calls that
 *     need one return LAT_ECUDA.
 */
#ifndef LAT_H
#define LAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define LAT_OK 0
#define LAT_EINVAL (-1)    /* bad argument (see each call) */
#define LAT_ENOMEM (-2)    /* device buffer too small, or allocation failed */
#define LAT_ECUDA (-3)     /* a CUDA call failed (no device, launch error, ...) */
#define LAT_ETIMEDOUT (-4) /* a bounded device-side wait gave up */
#define LAT_ESTATE (-5)    /* handle in the wrong state for this call */

/* Models. */
#define LAT_ISING 0
#define LAT_BLUME_CAPEL 1

/* Random-number modes (lat_params.rng). */
#define LAT_RNG_SITE 0  /* one Philox4x32-10 block per decision, counter (site, sweep, colour) */
#define LAT_RNG_TABLE 1 /* Ising only: the paper's lookup-table random bits (section 3.2) */

/* Largest accepted linear size: 2^20 (2^40 spins, 128 GiB as Ising). */
#define LAT_MAX_L (1u << 20)

typedef struct lat lat_t; /* opaque; owned by the library */

/* Simulation parameters (Eqs. (1)-(2); section 2).
 *   model  LAT_ISING or LAT_BLUME_CAPEL.
 *   L      linear size, a multiple of 64, 64 <= L <= LAT_MAX_L.
 *   J      ferromagnetic coupling, J > 0 (section 2 takes J > 0).
 *   Delta  crystal-field coupling of Eq. (2); ignored for Ising.
 *   T      temperature, T > 0 (k_B = 1).
 *   seed   64-bit key of the random stream.
 *   rng    LAT_RNG_SITE (default) or LAT_RNG_TABLE.  LAT_RNG_TABLE (Ising
 *          only) draws the flips of section 3.2: per 64-bit word and phase,
 *          two words of independent random bits with P(1) = p = exp(-4J/T),
 *          each made four bits at a time by locating a 32-bit uniform in a
 *          sorted 16-entry table (lat_lut_table); a site with four equal
 *          neighbours flips iff both words' bits are set (probability p^2),
 *          with three iff the first word's bit is set, otherwise always.
 *          Uniforms: word w = y*(L/64) + x/64 uses Philox blocks at counters
 *          (4w+q low, 4w+q high, sweep, colour+2), q = 0..3; uniform 4q+k is
 *          word k of block q; uniforms 0..7 make the first bit word and 8..15
 *          the second, four bits per uniform; the word's active sites take
 *          bits 0..31 in increasing x. */
typedef struct {
    int32_t model;
    uint32_t L;
    double J;
    double Delta;
    double T;
    uint64_t seed;
    int32_t rng;
} lat_params;

/* Exact observables after a sweep (Eqs. (1)-(2)):
 *   M = sum of s, B = sum over nearest-neighbour bonds (each once) of s s',
 *   Q = sum of s^2, so that E = -J B + Delta Q (Delta term for BC only).
 *   sweep = number of sweeps completed on the lattice when measured.
 *   draws = Philox blocks drawn during that sweep (both colours): the
 *   uphill Ising sites whose threshold is neither 0 nor 2^32, or every
 *   Blume-Capel site (L^2).  A work count, not an observable; 0 from
 *   lat_measure. */
typedef struct {
    int64_t M;
    int64_t B;
    int64_t Q;
    uint64_t sweep;
    uint64_t draws;
} lat_obs;

/* Device bytes lat_create needs for these parameters: the packed lattice
 * (L*L/8 bytes Ising, L*L/4 bytes Blume-Capel) plus a workspace for
 * per-sweep observables, correlation sums, a transfer stage and the compact
 * copy of the source columns used by lat_correlation_sampled (1/16 of the
 * lattice).
 * Returns 0 if the parameters are invalid.  Host only; needs no GPU. */
size_t lat_footprint(const lat_params* p);

/* The acceptance table the library builds for p (section 3.2: flip
 * probabilities e^{-4 beta}, e^{-8 beta} or 1 for Ising; Eq. (2) for BC),
 * written to out[0..n).  Entries are 2^32 for "always accept" (dE <= 0),
 * else floor(2^32 exp(-dE/T)).  Ising: 5 entries, entry i for the product
 * s*h = 2i - 4.  Blume-Capel: 54 entries, entry ((s+1)*2 + b)*9 + (h+4)
 * for the move from s to the b-th other value (ascending) with neighbour
 * sum h.  n must be >= 5 (Ising) or >= 54 (BC), else LAT_EINVAL.  Host only. */
int lat_thresholds(const lat_params* p, uint64_t* out, size_t n);

/* The 16-entry table of LAT_RNG_TABLE for p: entry j = floor(2^32 * sum
 * over 4-bit patterns m < j of p^popcount(m) (1-p)^(4-popcount(m))),
 * p = exp(-4J/T), clamped to 2^32-1; a uniform u selects the largest j with
 * entry j <= u, and j is the four random bits.  (The paper leaves the
 * construction to a companion reference; this is the library's reading.)
 * Host only; LAT_EINVAL unless p describes an Ising lattice. */
int lat_lut_table(const lat_params* p, uint32_t out[16]);

/* Create a lattice and draw its initial quench (infinite-temperature start,
 * section 1) on the device.
 *   dev_buf  caller-owned device memory of at least lat_footprint(p) bytes,
 *            256-byte aligned, that outlives the handle; or NULL to let the
 *            library cudaMalloc (and later free) its own buffer.
 *   bytes    size of dev_buf (ignored when dev_buf is NULL).
 *   stream   cudaStream_t to order all of this handle's work on (NULL = the
 *            legacy default stream).
 *   out      receives the handle.
 * Errors: LAT_EINVAL (bad params: L not a multiple of 64, L < 64 or
 * L > LAT_MAX_L, J <= 0, T <= 0, model unknown, NULL out, misaligned
 * dev_buf), LAT_ENOMEM (bytes < lat_footprint or allocation failure),
 * LAT_ECUDA.  The quench is enqueued, not synchronised. */
int lat_create(const lat_params* p, void* dev_buf, size_t bytes, void* stream, lat_t** out);

/* Run nsweeps checkerboard sweeps (section 3.1), with sweep indices
 * next .. next+nsweeps-1 where next = lat_sweep_index().  When per_sweep is
 * not NULL it receives nsweeps host records: the exact (M, B, Q) after each
 * sweep, computed on the device inside the colour-1 phase.  Sweep indices
 * must stay below 0xFFFFFFFF (reserved for the quench): LAT_EINVAL otherwise.
 * Synchronises the stream only when per_sweep is not NULL. */
int lat_sweep(lat_t* h, uint32_t nsweeps, lat_obs* per_sweep);

/* lat_sweep with the Schwinger-Dyson histogram of Eq. (3) after every sweep,
 * fused into the sweep kernels (section 4: the identity
 * <exp(-2 beta s_x h_x)> = 1 is the paper's check of equilibrium).
 * sd_hist is a host array of 9 * nsweeps int64: entry [i*9 + v+4] = number
 * of sites with s_x * h_x = v, v = -4..4, h_x the sum of the four
 * neighbours, in the lattice after sweep i of the call (the same values as
 * lat_sd_hist after that sweep).  Each colour phase counts its own sites:
 * the colour-1 sites after their update, the colour-0 sites before their
 * update in the next sweep; one separate pass over the lattice per call
 * (per 1024 sweeps) counts the colour-0 sites after the last sweep.
 * per_sweep as in lat_sweep (may be NULL).  LAT_EINVAL if sd_hist is NULL
 * and nsweeps > 0, and as lat_sweep otherwise.  Synchronises. */
int lat_sweep_sd(lat_t* h, uint32_t nsweeps, lat_obs* per_sweep, int64_t* sd_hist);

/* Exact (M, B, Q) of the current lattice by a separate reduction kernel
 * (an independent check of the fused per-sweep values).  Synchronises. */
int lat_measure(lat_t* h, lat_obs* out);

/* Spin-spin correlation from every site along both axes (section 3.3,
 * all sources, every distance): cx[r] = sum_{x,y} s(x,y) s(x+r,y) and
 * cy[r] = sum_{x,y} s(x,y) s(x,y+r), periodic, r = 0..rmax, exact int64
 * raw sums (no mean subtracted, no normalisation).  cx and cy are host
 * arrays of rmax+1 entries.  rmax must be <= L/2 (LAT_EINVAL).  Synchronises. */
int lat_correlation(lat_t* h, uint32_t rmax, int64_t* cx, int64_t* cy);

/* lat_correlation without waiting: the correlation kernels and the copies
 * of the sums into cx and cy are enqueued on the handle's stream and the
 * call returns.  cx and cy (rmax+1 entries each) hold the sums once the
 * stream has passed this point (cudaStreamSynchronize, or any later call on
 * the same stream that synchronises it); they should be page-locked host
 * memory, without which the copies wait for the stream.  A later
 * correlation call on the same handle reuses its device accumulators after
 * this one, in stream order.  Errors as lat_correlation. */
int lat_correlation_async(lat_t* h, uint32_t rmax, int64_t* cx, int64_t* cy);

/* The correlation protocol of section 3.3.  Every site is a source for
 * r <= 2R.  Beyond that, only one site per R x R square is a source (its
 * top-left corner, x % R == 0 and y % R == 0), and the distances are:
 *   - every r in (2R, r_c(t)];
 *   - the log-spaced floor(2^(x/32)) > r_c(t), 32 per octave, up to L/2;
 * with r_c(t) = max{256, floor(g(L) sqrt(t) + 1/2)} and
 * g(L) = 6 sqrt(ln(L / 2^16) / 3.3^2 + 1), natural logarithm.
 * Measurements are taken at the times t = floor(2^(x/8) + 1/2), x = 1, 2, ...
 * The formulas are evaluated on the host in FP64, in the order written and
 * without floating-point contraction.  The functions below need no device. */

/* r_c(t) for a lattice of side L. */
uint64_t lat_protocol_rc(uint32_t L, uint64_t t);

/* The downsampled distances at time t, ascending and distinct: every r in
 * (2R, min(r_c, L/2)], then every floor(2^(x/32)) in (r_c, L/2].  Returns
 * their number and writes the first min(number, cap) to out (which may be
 * NULL when cap is 0). */
uint32_t lat_protocol_distances(uint32_t L, uint64_t t, uint32_t R, uint32_t* out, uint32_t cap);

/* The distinct measurement times floor(2^(x/8) + 1/2) <= tmax, ascending.
 * Returns their number and writes the first min(number, cap) to out. */
uint32_t lat_protocol_times(uint64_t tmax, uint64_t* out, uint32_t cap);

/* Correlation from downsampled sources, for an arbitrary list of distances:
 *   cx[i] = sum over x % R == 0, y % R == 0 of s(x,y) s(x + r[i], y),
 *   cy[i] = the same with s(x, y + r[i]);
 * periodic, exact int64 raw sums over (L/R)^2 sources.
 *   R          a power of two, 1..64 (the paper uses 16).
 *   r, nr      host array of nr distances, each <= L/2.  Repeats and any
 *              order are allowed; lists longer than L/2 + 1 are processed
 *              in pieces of that size.
 *   cx, cy     host arrays of nr entries.
 * With R >= 16, the y sums read a compact copy of the source columns that
 * the handle's buffer holds: L/16 bits per row and plane, counted in
 * lat_footprint.  With R < 16 they read the lattice directly.
 * Errors: LAT_EINVAL (R not a power of two in 1..64, a distance > L/2,
 * a NULL array with nr > 0), LAT_ECUDA.  Synchronises. */
int lat_correlation_sampled(lat_t* h, uint32_t R, const uint32_t* r, uint32_t nr, int64_t* cx, int64_t* cy);

/* One protocol measurement at time t.  Output rows are in ascending r:
 *   - rows 0..min(2R, L/2) hold every distance from every site
 *     (nsrc = L^2, as lat_correlation);
 *   - the remaining rows hold lat_protocol_distances(L, t, R) from the
 *     downsampled sources (nsrc = (L/R)^2, as lat_correlation_sampled).
 * *n_out always receives the row count.  A call with cap == 0 and every
 * array NULL only queries that count and returns LAT_OK.  Otherwise all
 * four arrays are needed, each of cap >= *n_out entries (LAT_EINVAL if
 * fewer).  The host divides cx and cy by nsrc to normalise.  Synchronises. */
int lat_correlation_protocol(lat_t* h, uint64_t t, uint32_t R, uint32_t cap, uint32_t* n_out, uint32_t* r_out,
                             int64_t* cx, int64_t* cy, uint64_t* nsrc);

/* Spin counts, the consistency check the paper's runs perform (Table 3
 * caption: the total number of spins stays unchanged): counts[0], [1], [2]
 * = number of sites holding -1, 0, +1, and counts[3] = number of
 * Blume-Capel 2-bit codes that are not a spin (g set without n; always 0 for
 * Ising).  On a sound lattice counts[0] + counts[1] + counts[2] = L^2,
 * counts[3] = 0, M = counts[2] - counts[0] and Q = counts[0] + counts[2].
 * Synchronises. */
int lat_spin_counts(lat_t* h, int64_t counts[4]);

/* Schwinger-Dyson histogram of Eq. (3): hist[v+4] = number of sites with
 * s_x * h_x = v, v = -4..4, h_x the sum of the four neighbours.  Eq. (3)'s
 * right-hand side is L^-2 sum_v hist[v+4] exp(-2 J v / T).  hist is a host
 * array of 9 entries.  Synchronises. */
int lat_sd_hist(lat_t* h, int64_t* hist);

/* Canonical lattice hash: sum over canonical words i of
 * mix(i XOR word_i) mod 2^64, mix the SplitMix64 finaliser.  Canonical
 * words: W = L/64 per row, bit b of word (y, j) is site x = 64j + b; Ising
 * one plane (bit set iff s = +1); Blume-Capel plane 0 (bit set iff s != 0)
 * at words 0..L*W-1 then plane 1 (bit set iff s = -1).  Synchronises. */
int lat_hash(lat_t* h, uint64_t* out);

/* lat_hash without waiting: the hash is written to *out (page-locked host
 * memory) once the handle's stream has passed this point. */
int lat_hash_async(lat_t* h, uint64_t* out);

/* Copy the whole lattice to host int8 values (L*L bytes, row-major,
 * s[y*L + x]).  Synchronises. */
int lat_get_spins(lat_t* h, int8_t* host_out);

/* Copy nrows rows starting at row y0 (wrapping modulo L) to host int8
 * (nrows*L bytes).  y0 < L and nrows <= L, else LAT_EINVAL.  Synchronises. */
int lat_get_rows(lat_t* h, uint32_t y0, uint32_t nrows, int8_t* host_out);

/* Replace the lattice with host int8 values (L*L bytes, -1/+1 for Ising,
 * -1/0/+1 for Blume-Capel; any other value gives LAT_EINVAL and leaves the
 * lattice unspecified).  Does not change the sweep index.  Synchronises. */
int lat_set_spins(lat_t* h, const int8_t* host_in);

/* Bytes of the packed device state (the lattice alone). */
size_t lat_state_bytes(const lat_params* p);

/* Raw packed state to/from host memory (checkpointing).  Layout: Ising,
 * L rows of L/64 little-endian uint64 words, bit b of word j = site 64j+b,
 * set iff s = +1; Blume-Capel, L rows of L/64 word pairs (plane n: s != 0,
 * plane g: s = -1), pair j covering sites 64j..64j+63.  bytes must equal
 * lat_state_bytes.  Host memory may be pinned or pageable.  lat_set_state
 * copies the words as they are (a Blume-Capel pair with g set and n clear
 * is not a spin; lat_spin_counts reports how many there are).
 * Synchronises. */
int lat_get_state(lat_t* h, void* host, size_t bytes);
int lat_set_state(lat_t* h, const void* host, size_t bytes);

/* Number of sweeps completed (the index of the next sweep), and its setter
 * for resuming from a checkpoint (must be < 0xFFFFFFFF). */
int lat_get_sweep_index(lat_t* h, uint64_t* next);
int lat_set_sweep_index(lat_t* h, uint64_t next);

/* The acceptance table in use by this handle (see lat_thresholds). */
int lat_get_thresholds(lat_t* h, uint64_t* out, size_t n);

/* Release the handle (and the buffer, if the library allocated it).
 * Synchronises the stream first.  NULL is accepted. */
int lat_destroy(lat_t* h);

/* ---- Many lattices in one persistent launch ------------------------------
 *
 * A runner advances a set of lattices (handles from lat_create, of any mix
 * of models, sizes and temperatures) by per-lattice sweep counts in one
 * persistent kernel launch, replayed from a CUDA graph captured when the
 * runner is created.  Every lattice ends bit-identical to the same sweeps
 * run on it alone with lat_sweep (same counters, same per-site update), and
 * its sweep index advances the same way.  The paper runs one lattice at a
 * time (section 4); batching independent lattices is this library's own
 * addition for many small systems.
 *
 * Inside the launch, phase k of a lattice waits for every tile of its phase
 * k-1; each such wait is bounded (lat_runner_set_timeout), and a wait that
 * gives up makes the run return LAT_ETIMEDOUT with the lattices in an
 * unspecified state. */
typedef struct lat_runner lat_runner_t;

/* Device bytes a runner needs for up to max_lattices lattices and
 * max_sweeps sweeps per lattice per run (0 if either is 0 or > 2^20). */
size_t lat_runner_footprint(uint32_t max_lattices, uint32_t max_sweeps);

/* Create a runner.  dev_buf/bytes/stream as in lat_create (NULL dev_buf
 * lets the library allocate).  The runner also allocates a small pinned
 * host staging area.  Errors: LAT_EINVAL, LAT_ENOMEM, LAT_ECUDA. */
int lat_runner_create(uint32_t max_lattices, uint32_t max_sweeps, void* dev_buf, size_t bytes, void* stream,
                      lat_runner_t** out);

/* Schedule: items per tile for lattices of this model and L (a multiple of
 * 256; 0 restores the default of 4096).  Results do not depend on it. */
int lat_runner_set_tile(lat_runner_t* r, int32_t model, uint32_t L, uint32_t tile_items);

/* Limit of one device-side wait, in nanoseconds (default 10 s). */
int lat_runner_set_timeout(lat_runner_t* r, uint64_t ns);

/* Failure-path testing: in later runs, every wait of lattices[index] (as
 * passed to lat_runner_run) waits for a count that is never reached, so the
 * run ends with LAT_ETIMEDOUT after the wait limit instead of hanging.
 * index = 0xFFFFFFFF switches this off (the default). */
int lat_runner_inject_stall(lat_runner_t* r, uint32_t index);

/* Boundary testing: the per-lattice tile counters of later runs start at
 * base instead of 0.  Inside a run the counter of a lattice with ntiles tiles
 * per phase counts up to base + 2 * nsweeps * ntiles; a run in which that
 * would reach 2^64 - 1 is rejected with LAT_EINVAL before anything is
 * launched.  With base just below 2^32 a test crosses the 32-bit boundary in
 * a few phases.  Results do not depend on base.  LAT_EINVAL for
 * base = 2^64 - 1. */
int lat_runner_set_counter_base(lat_runner_t* r, uint64_t base);

/* Advance lattices[i] by nsweeps[i] sweeps (0 allowed), all in one launch
 * on the runner's stream.  1 <= n <= max_lattices, nsweeps[i] <=
 * max_sweeps, each handle at most once, Ising and Blume-Capel L <= 2^19.
 * per_sweep may be NULL, or an array of n host pointers (each NULL or of
 * nsweeps[i] records) that receive the exact (M, B, Q) and draw count after
 * every sweep, as lat_sweep would.  The run is ordered after all earlier
 * work of every handle (by stream order when a handle uses the runner's
 * stream, else by a device-side wait on the handle's stream), and the call
 * synchronises the runner's stream before it returns.  Errors: LAT_EINVAL (including a run whose tile counters would
 * not fit, see lat_runner_set_counter_base), LAT_ECUDA, LAT_ETIMEDOUT, and LAT_ESTATE if
 * the tile maps built on the host fail their consistency check (an internal
 * error; nothing is launched). */
int lat_runner_run(lat_runner_t* r, lat_t* const* lattices, uint32_t n, const uint32_t* nsweeps,
                   lat_obs* const* per_sweep);

/* lat_runner_run in two halves, so that the host can prepare other work
 * while the run is on the device.  lat_runner_submit checks the arguments
 * (as lat_runner_run), orders the run after the lattices' earlier work as
 * lat_runner_run does, enqueues it on the runner's stream and returns
 * without waiting.
 * lat_runner_collect waits for it, then writes the per-sweep records
 * (per_sweep as in lat_runner_run; may be NULL) and advances the lattices'
 * sweep indices.  Between the two, a lattice of the run may only be given
 * work that is ordered after the run on the runner's stream (for example
 * lat_correlation_async on a handle created on that stream); no second run
 * may be submitted (LAT_ESTATE); the runner's other settings may be changed
 * and apply to later runs.  lat_runner_collect without a pending run is
 * LAT_ESTATE; a run whose device waits timed out is collected as
 * LAT_ETIMEDOUT, with its lattices in an unspecified state and their sweep
 * indices unchanged. */
int lat_runner_submit(lat_runner_t* r, lat_t* const* lattices, uint32_t n, const uint32_t* nsweeps);
int lat_runner_collect(lat_runner_t* r, lat_obs* const* per_sweep);

/* Release the runner (and its buffer, if the library allocated it). */
int lat_runner_destroy(lat_runner_t* r);

/* Largest rmax accepted by lat_correlation_static. */
#define LAT_STATIC_RMAX 4096u

/* lat_correlation without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they measure, such as a library running inside another
 * framework whose caching allocator owns the GPU's memory, or a serving loop
 * in which cudaMalloc/cudaFree would synchronise the device.
 *   model, L   as in lat_params (L a multiple of 64 within the same limits).
 *   dev_spins  device pointer to a packed lattice in the layout of
 *              lat_get_state (lat_create places it at the start of the
 *              caller's dev_buf); read only; 16-byte aligned (LAT_EINVAL
 *              otherwise, checked before anything is launched).
 *   rmax       0 <= rmax <= min(L/2, LAT_STATIC_RMAX); larger values give
 *              LAT_EINVAL.
 *   cx, cy     host arrays of rmax+1 entries, filled exactly as by
 *              lat_correlation.
 *   stream     cudaStream_t to run on (NULL = legacy default stream); the
 *              call synchronises it before returning.
 * Scratch: a fixed file-scope device array of 2*(LAT_STATIC_RMAX+1) int64
 * (64 KiB) that every GPU loading the library keeps until the process
 * exits.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current and keeps it for the rest of
 * the process; make that first call before any stream capture, and make no
 * call after a cudaDeviceReset (the kept address belonged to the context
 * that the reset ended).  All calls share the array (it is cleared on
 * the stream before each use), so calls whose work overlaps on the GPU race.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: LAT_EINVAL (bad arguments), LAT_ECUDA. */
int lat_correlation_static(int32_t model, uint32_t L, const void* dev_spins, uint32_t rmax, int64_t* cx,
                           int64_t* cy, void* stream);

/* ---- Diagnostics ----------------------------------------------------------
 *
 * Measured issue rates of the integer pipes the hot path is bound by, the
 * denominators of its roofline fractions (the paper has no counterpart).
 * Runs register-only microkernels on the current device, each for a few tens
 * of milliseconds at full occupancy, and writes to rates[0..LAT_PROBE_RATES):
 *   rates[0]  IMAD-ops/s: 32x32->64 multiply-adds (mad.wide.u32, the
 *             Philox4x32-10 round multiply), each counted as two IMAD-ops
 *             (the faster of two chain layouts);
 *   rates[1]  LOP3/s: 3-input logic operations (lop3.b32);
 *   rates[2]  POPC/s: population counts (popc.b32);
 *   rates[3]  Philox4x32-10 blocks/s: full ten-round blocks, all four words;
 *   rates[4]  32-bit multiply-adds (mad.lo.u32) per second.
 * seconds (may be NULL) receives each rate's CUDA-event time.  The rates
 * hold at the SM clock during the call, which the caller should record.
 * Uses a private stream and synchronises it; allocates nothing.
 * Errors: LAT_EINVAL (NULL rates), LAT_ECUDA. */
#define LAT_PROBE_RATES 5
int lat_probe_rates(double rates[LAT_PROBE_RATES], double seconds[LAT_PROBE_RATES]);

/* Static description of an error code. */
const char* lat_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LAT_H */
