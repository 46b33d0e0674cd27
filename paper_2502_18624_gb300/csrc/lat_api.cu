// lat_api.cu -- the extern "C" entry points declared in include/lat.h.
//
// Host responsibilities only: argument checks, the FP64 acceptance table
// (built once per lattice and passed to the kernels as data), carving the
// device buffer, and ordering launches and copies on the handle's stream.
// Every step of the simulation and every measurement runs in the kernels of
// k_sweep.cu, k_lattice.cu and k_corr.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lat.h"
#include "lat_handle.h"
#include "lat_internal.cuh"

using namespace latk;

namespace {

constexpr uint32_t kObsCap = 1024;  // per-sweep records buffered on the device per batch
constexpr size_t kStageCap = 4u << 20;
constexpr size_t kAlign = 256;
constexpr uint64_t kLastSweep = 0xFFFFFFFFull;  // index reserved for the quench

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool params_ok(const lat_params* p)
{
    if (!p) return false;
    if (p->model != LAT_ISING && p->model != LAT_BLUME_CAPEL) return false;
    if (p->L < 64 || p->L % 64 != 0 || p->L > LAT_MAX_L) return false;
    if (p->model == LAT_BLUME_CAPEL && p->L > LAT_MAX_L / 2) return false;
    if (!(p->J > 0.0) || !std::isfinite(p->J)) return false;
    if (!(p->T > 0.0) || !std::isfinite(p->T)) return false;
    if (p->model == LAT_BLUME_CAPEL && !std::isfinite(p->Delta)) return false;
    if (p->rng != LAT_RNG_SITE && p->rng != LAT_RNG_TABLE) return false;
    if (p->rng == LAT_RNG_TABLE && p->model != LAT_ISING) return false;
    return true;
}

size_t spins_bytes(const lat_params* p)
{
    return (size_t)p->L * (p->L / 64) * sizeof(uint64_t) * (p->model == LAT_ISING ? 1 : 2);
}

Layout layout_of(const lat_params* p)
{
    Layout l;
    size_t off = 0;
    l.spins = off;
    off = align_up(off + spins_bytes(p));
    l.obs = off;
    off = align_up(off + (size_t)kObsCap * kObsWords * sizeof(long long));
    l.sd = off;
    off = align_up(off + (size_t)kObsCap * 9 * sizeof(long long));
    l.corr = off;
    off = align_up(off + 2 * ((size_t)p->L / 2 + 1) * sizeof(long long));
    l.misc = off;
    off = align_up(off + 32 * sizeof(long long));
    const size_t lsq = (size_t)p->L * p->L;
    l.stage_bytes = lsq < kStageCap ? lsq : (kStageCap / p->L) * p->L;
    l.stage = off;
    off = align_up(off + l.stage_bytes);
    l.ds = off;
    off = align_up(off + ds_scratch_words(p->model, p->L) * sizeof(uint64_t));
    l.rlist = off;
    off = align_up(off + ((size_t)p->L / 2 + 1) * sizeof(uint32_t));
    l.total = off;
    return l;
}

// Integer Metropolis bound for an energy change dE at temperature T:
// 2^32 (accept without drawing) when dE <= 0, else floor(2^32 e^{-dE/T}).
uint64_t acceptance_bound(double dE, double T)
{
    if (!(dE > 0.0)) return kAlways;
    const double x = std::exp(-dE / T) * 4294967296.0;
    if (x >= 4294967296.0) return kAlways;
    return (uint64_t)std::floor(x);
}

size_t build_table(const lat_params* p, uint64_t* t)
{
    if (p->model == LAT_ISING) {
        // Eq. (1): flipping s with neighbour sum h costs 2 J s h; index i <-> s*h = 2i - 4.
        for (int i = 0; i < 5; ++i) t[i] = acceptance_bound(p->J * (double)(2 * (2 * i - 4)), p->T);
        return 5;
    }
    // Eq. (2): s -> s' costs -J (s'-s) h + Delta (s'^2 - s^2); s' is the b-th
    // of the two other values in ascending order.
    static const int kOther[3][2] = {{0, 1}, {-1, 1}, {-1, 0}};
    for (int si = 0; si < 3; ++si)
        for (int b = 0; b < 2; ++b)
            for (int h = -4; h <= 4; ++h) {
                const int s = si - 1, sp = kOther[si][b];
                const double dE = p->J * (double)(-(sp - s) * h) + p->Delta * (double)(sp * sp - s * s);
                t[(si * 2 + b) * 9 + (h + 4)] = acceptance_bound(dE, p->T);
            }
    return 54;
}

// LAT_RNG_TABLE: cumulative probabilities of the 16 four-bit patterns in
// index order, each bit independently 1 with p = exp(-4J/T).
void build_lut(const lat_params* p, uint32_t* out)
{
    const double q = std::exp(-4.0 * p->J / p->T);
    double cum = 0.0;
    for (int j = 0; j < 16; ++j) {
        const double scaled = std::floor(cum * 4294967296.0);
        out[j] = scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
        const int ones = __builtin_popcount((unsigned)j);
        cum += std::pow(q, (double)ones) * std::pow(1.0 - q, (double)(4 - ones));
    }
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LAT_OK : LAT_ECUDA; }

// Section 3.3: r_c(t) = max{256, floor(g(L) sqrt(t) + 1/2)} with
// g(L) = 6 sqrt(ln(L / 2^16) / 3.3^2 + 1), evaluated in FP64 in that order
// (the library is compiled without floating-point contraction).
uint64_t protocol_rc(uint32_t L, uint64_t t)
{
    const double g = 6.0 * std::sqrt(std::log((double)L / 65536.0) / (3.3 * 3.3) + 1.0);
    const double v = std::floor(g * std::sqrt((double)t) + 0.5);
    return v > 256.0 ? (uint64_t)v : 256u;
}

bool valid_R(uint32_t R) { return R >= 1 && R <= 64 && (R & (R - 1)) == 0; }

}  // namespace

extern "C" {

uint64_t lat_protocol_rc(uint32_t L, uint64_t t) { return protocol_rc(L, t); }

uint32_t lat_protocol_distances(uint32_t L, uint64_t t, uint32_t R, uint32_t* out, uint32_t cap)
{
    const uint64_t rc = protocol_rc(L, t), half = L / 2;
    std::vector<uint32_t> d;
    // every distance in (2R, min(r_c, L/2)]
    for (uint64_t r = 2 * (uint64_t)R + 1; r <= std::min(rc, half); ++r) d.push_back((uint32_t)r);
    // floor(2^(x/32)) beyond r_c, 32 per octave, up to 2^(log2(L) - 1) = L/2
    for (uint32_t x = 1; std::floor(std::exp2(x / 32.0)) <= (double)half; ++x) {
        const uint64_t r = (uint64_t)std::floor(std::exp2(x / 32.0));
        if (r > rc && (d.empty() || r > d.back())) d.push_back((uint32_t)r);
    }
    if (out)
        for (size_t i = 0; i < d.size() && i < cap; ++i) out[i] = d[i];
    return (uint32_t)d.size();
}

uint32_t lat_protocol_times(uint64_t tmax, uint64_t* out, uint32_t cap)
{
    uint32_t n = 0;
    uint64_t prev = 0;
    for (uint32_t x = 1;; ++x) {
        const double v = std::floor(std::exp2(x / 8.0) + 0.5);
        if (v > (double)tmax) break;
        if ((uint64_t)v == prev) continue;
        prev = (uint64_t)v;
        if (out && n < cap) out[n] = prev;
        ++n;
    }
    return n;
}

size_t lat_footprint(const lat_params* p) { return params_ok(p) ? layout_of(p).total : 0; }

size_t lat_state_bytes(const lat_params* p) { return params_ok(p) ? spins_bytes(p) : 0; }

int lat_thresholds(const lat_params* p, uint64_t* out, size_t n)
{
    if (!params_ok(p) || !out) return LAT_EINVAL;
    uint64_t t[54];
    const size_t k = build_table(p, t);
    if (n < k) return LAT_EINVAL;
    std::memcpy(out, t, k * sizeof(uint64_t));
    return LAT_OK;
}

int lat_lut_table(const lat_params* p, uint32_t out[16])
{
    if (!params_ok(p) || !out || p->model != LAT_ISING) return LAT_EINVAL;
    build_lut(p, out);
    return LAT_OK;
}

int lat_create(const lat_params* p, void* dev_buf, size_t bytes, void* stream, lat_t** out)
{
    const NvtxRange range("lat_create");
    if (!out || !params_ok(p)) return LAT_EINVAL;
    *out = nullptr;
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) % kAlign) != 0) return LAT_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LAT_ECUDA;
    lat* h = new (std::nothrow) lat();
    if (!h) return LAT_ENOMEM;
    h->p = *p;
    h->W = p->L / 64;
    h->nthr = build_table(p, h->thr);
    build_lut(p, h->lut);
    h->lay = layout_of(p);
    h->stream = static_cast<cudaStream_t>(stream);
    h->next_sweep = 0;
    h->rk = make_round_keys(p->seed);
    if (query_sweep_occupancy(h->ls) != cudaSuccess) {
        delete h;
        return LAT_ECUDA;
    }
    if (dev_buf) {
        if (bytes < h->lay.total) {
            delete h;
            return LAT_ENOMEM;
        }
        h->buf = static_cast<char*>(dev_buf);
        h->owns = false;
    } else {
        if (cudaMalloc(&h->buf, h->lay.total) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return LAT_ENOMEM;
        }
        h->owns = true;
    }
    const cudaError_t e = launch_init(p->model, h->spins(), p->L, h->W, h->rk, h->ls.sms, h->stream);
    if (e != cudaSuccess) {
        if (h->owns) cudaFree(h->buf);
        delete h;
        return LAT_ECUDA;
    }
    *out = h;
    return LAT_OK;
}

// nsweeps sweeps; per_sweep (or NULL) receives the fused (M, B, Q) records and
// sd (or NULL) the fused Schwinger-Dyson histogram after every sweep (9 per
// sweep).  The histogram of the state after sweep t is taken in two parts:
// its colour-1 sites after their update in the colour-1 phase of sweep t,
// its colour-0 sites before their update in the colour-0 phase of sweep
// t+1; after the last sweep of each batch of records a separate pass counts
// the colour-0 sites.
static int sweep_impl(lat_t* h, uint32_t nsweeps, lat_obs* per_sweep, int64_t* sd)
{
    if (!h) return LAT_EINVAL;
    if (h->next_sweep + nsweeps > kLastSweep) return LAT_EINVAL;
    const uint32_t L = h->p.L, W = h->W;
    IsingPhaseArgs ia;
    BcPhaseArgs ba;
    if (h->p.model == LAT_ISING) {
        ia.spins = static_cast<uint64_t*>(h->spins());
        ia.L = L;
        ia.W = W;
        ia.thr4 = (uint32_t)(h->thr[3] >= kAlways ? 0 : h->thr[3]);
        ia.thr8 = (uint32_t)(h->thr[4] >= kAlways ? 0 : h->thr[4]);
        ia.mode4 = class_mode(h->thr[3]);
        ia.mode8 = class_mode(h->thr[4]);
        ia.rng = (uint32_t)h->p.rng;
        std::memcpy(ia.lut, h->lut, sizeof(ia.lut));
        ia.rk = h->rk;
    } else {
        ba.spins = static_cast<ulonglong2*>(h->spins());
        ba.L = L;
        ba.W = W;
        ba.rk = h->rk;
        for (int i = 0; i < 54; ++i) ba.thr[i] = h->thr[i];
    }
    uint32_t done = 0;
    while (done < nsweeps) {
        const uint32_t batch = nsweeps - done < kObsCap ? nsweeps - done : kObsCap;
        if (per_sweep) {
            const cudaError_t e = cudaMemsetAsync(h->obs(), 0, (size_t)batch * kObsWords * sizeof(long long), h->stream);
            if (e != cudaSuccess) return LAT_ECUDA;
        }
        if (sd) {
            const cudaError_t e = cudaMemsetAsync(h->sd(), 0, (size_t)batch * 9 * sizeof(long long), h->stream);
            if (e != cudaSuccess) return LAT_ECUDA;
        }
        for (uint32_t i = 0; i < batch; ++i) {
            const uint32_t t = (uint32_t)(h->next_sweep + done + i);
            long long* rec = per_sweep ? h->obs() + (size_t)i * kObsWords : nullptr;
            for (uint32_t colour = 0; colour < 2; ++colour) {
                cudaError_t e;
                // colour 0 counts the previous record's colour-0 sites, colour 1 this one's colour-1 sites
                long long* sdrec = !sd ? nullptr : colour == 1 ? h->sd() + (size_t)i * 9
                                                 : (i > 0 ? h->sd() + (size_t)(i - 1) * 9 : nullptr);
                if (h->p.model == LAT_ISING) {
                    ia.sweep = t;
                    ia.colour = colour;
                    ia.obs = colour == 1 ? rec : nullptr;
                    ia.draws = rec ? rec + kObsDraws : nullptr;
                    ia.sd = sdrec;
                    e = launch_ising_phase(ia, h->ls, h->stream);
                } else {
                    ba.sweep = t;
                    ba.colour = colour;
                    ba.obs = colour == 1 ? rec : nullptr;
                    ba.draws = rec ? rec + kObsDraws : nullptr;
                    ba.sd = sdrec;
                    e = launch_bc_phase(ba, h->ls, h->stream);
                }
                if (e != cudaSuccess) return LAT_ECUDA;
            }
        }
        if (per_sweep) {
            h->host_obs.resize((size_t)batch * kObsWords);
            cudaError_t e = cudaMemcpyAsync(h->host_obs.data(), h->obs(), h->host_obs.size() * sizeof(long long),
                                            cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return LAT_ECUDA;
            for (uint32_t i = 0; i < batch; ++i) {
                lat_obs& o = per_sweep[done + i];
                o.M = h->host_obs[(size_t)i * kObsWords + kObsM];
                o.B = h->host_obs[(size_t)i * kObsWords + kObsB];
                o.Q = h->host_obs[(size_t)i * kObsWords + kObsQ];
                o.sweep = h->next_sweep + done + i + 1;
                o.draws = (uint64_t)h->host_obs[(size_t)i * kObsWords + kObsDraws];
            }
        }
        if (sd) {
            // the last record's colour-0 sites (no later colour-0 phase in this batch)
            cudaError_t e = launch_sd_hist_add(h->p.model, h->spins(), L, W, h->sd() + (size_t)(batch - 1) * 9, 1u,
                                               h->ls.sms, h->stream);
            h->host_sd.resize((size_t)batch * 9);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->host_sd.data(), h->sd(), h->host_sd.size() * sizeof(long long),
                                    cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) return LAT_ECUDA;
            for (size_t k = 0; k < h->host_sd.size(); ++k) sd[(size_t)done * 9 + k] = h->host_sd[k];
        }
        done += batch;
    }
    h->next_sweep += nsweeps;
    return LAT_OK;
}

int lat_sweep(lat_t* h, uint32_t nsweeps, lat_obs* per_sweep)
{
    const NvtxRange range("lat_sweep");
    return sweep_impl(h, nsweeps, per_sweep, nullptr);
}

int lat_sweep_sd(lat_t* h, uint32_t nsweeps, lat_obs* per_sweep, int64_t* sd_hist)
{
    const NvtxRange range("lat_sweep_sd");
    if (!sd_hist && nsweeps > 0) return LAT_EINVAL;
    return sweep_impl(h, nsweeps, per_sweep, sd_hist);
}

int lat_measure(lat_t* h, lat_obs* out)
{
    const NvtxRange range("lat_measure");
    if (!h || !out) return LAT_EINVAL;
    long long v[3];
    cudaError_t e = launch_measure(h->p.model, h->spins(), h->p.L, h->W, h->misc(), h->ls.sms, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v, h->misc(), sizeof(v), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LAT_ECUDA;
    out->M = v[0];
    out->B = v[1];
    out->Q = v[2];
    out->sweep = h->next_sweep;
    out->draws = 0;
    return LAT_OK;
}

int lat_correlation(lat_t* h, uint32_t rmax, int64_t* cx, int64_t* cy)
{
    const NvtxRange range("lat_correlation");
    if (!h || !cx || !cy || rmax > h->p.L / 2) return LAT_EINVAL;
    long long* dcx = h->corr();
    long long* dcy = dcx + (rmax + 1);
    cudaError_t e = launch_correlation(h->p.model, h->spins(), h->p.L, h->W, rmax, dcx, dcy, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cx, dcx, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cy, dcy, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_correlation_async(lat_t* h, uint32_t rmax, int64_t* cx, int64_t* cy)
{
    const NvtxRange range("lat_correlation_async");
    if (!h || !cx || !cy || rmax > h->p.L / 2) return LAT_EINVAL;
    long long* dcx = h->corr();
    long long* dcy = dcx + (rmax + 1);
    cudaError_t e = launch_correlation(h->p.model, h->spins(), h->p.L, h->W, rmax, dcx, dcy, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cx, dcx, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cy, dcy, (rmax + 1) * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    return cuda_err(e);
}

int lat_correlation_sampled(lat_t* h, uint32_t R, const uint32_t* r, uint32_t nr, int64_t* cx, int64_t* cy)
{
    const NvtxRange range("lat_correlation_sampled");
    if (!h || !valid_R(R) || (nr && (!r || !cx || !cy))) return LAT_EINVAL;
    for (uint32_t i = 0; i < nr; ++i)
        if (r[i] > h->p.L / 2) return LAT_EINVAL;
    // the device list and accumulators hold L/2 + 1 distances: longer lists go in pieces
    const uint32_t piece = h->p.L / 2 + 1;
    long long* dcx = h->corr();
    long long* dcy = dcx + piece;
    cudaError_t e = cudaSuccess;
    for (uint32_t i0 = 0; i0 < nr && e == cudaSuccess; i0 += piece) {
        const uint32_t n = std::min(piece, nr - i0);
        e = cudaMemcpyAsync(h->rlist(), r + i0, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = launch_correlation_sampled(h->p.model, h->spins(), h->p.L, h->W, R, h->rlist(), n, dcx, dcy,
                                           h->ds_scratch(), h->ls.sms, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cx + i0, dcx, (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cy + i0, dcy, (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
        // the list and accumulators are reused by the next piece; r is read before return
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    return cuda_err(e);
}

int lat_correlation_protocol(lat_t* h, uint64_t t, uint32_t R, uint32_t cap, uint32_t* n_out, uint32_t* r_out,
                             int64_t* cx, int64_t* cy, uint64_t* nsrc)
{
    const NvtxRange range("lat_correlation_protocol");
    if (!h || !n_out || !valid_R(R)) return LAT_EINVAL;
    const uint32_t L = h->p.L;
    const uint32_t rfull = std::min<uint32_t>(2 * R, L / 2);
    const uint32_t nds = lat_protocol_distances(L, t, R, nullptr, 0);
    const uint32_t n = rfull + 1 + nds;
    *n_out = n;
    if (cap < n) return cap == 0 && !r_out && !cx && !cy && !nsrc ? LAT_OK : LAT_EINVAL;
    if (!r_out || !cx || !cy || !nsrc) return LAT_EINVAL;
    int rc = lat_correlation(h, rfull, cx, cy);
    if (rc != LAT_OK) return rc;
    const uint64_t all = (uint64_t)L * L, sampled = (uint64_t)(L / R) * (L / R);
    for (uint32_t r = 0; r <= rfull; ++r) {
        r_out[r] = r;
        nsrc[r] = all;
    }
    lat_protocol_distances(L, t, R, r_out + rfull + 1, nds);
    for (uint32_t i = rfull + 1; i < n; ++i) nsrc[i] = sampled;
    return lat_correlation_sampled(h, R, r_out + rfull + 1, nds, cx + rfull + 1, cy + rfull + 1);
}

int lat_spin_counts(lat_t* h, int64_t counts[4])
{
    const NvtxRange range("lat_spin_counts");
    if (!h || !counts) return LAT_EINVAL;
    cudaError_t e = launch_spin_counts(h->p.model, h->spins(), h->p.L, h->W, h->misc() + 24, h->ls.sms, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, h->misc() + 24, 4 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_sd_hist(lat_t* h, int64_t* hist)
{
    const NvtxRange range("lat_sd_hist");
    if (!h || !hist) return LAT_EINVAL;
    cudaError_t e = launch_sd_hist(h->p.model, h->spins(), h->p.L, h->W, h->misc() + 4, h->ls.sms, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist, h->misc() + 4, 9 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_hash(lat_t* h, uint64_t* out)
{
    if (!h || !out) return LAT_EINVAL;
    unsigned long long* d = reinterpret_cast<unsigned long long*>(h->misc() + 16);
    cudaError_t e = launch_hash(h->p.model, h->spins(), h->p.L, h->W, d, h->ls.sms, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_hash_async(lat_t* h, uint64_t* out)
{
    if (!h || !out) return LAT_EINVAL;
    unsigned long long* d = reinterpret_cast<unsigned long long*>(h->misc() + 16);
    cudaError_t e = launch_hash(h->p.model, h->spins(), h->p.L, h->W, d, h->ls.sms, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream);
    return cuda_err(e);
}

int lat_get_rows(lat_t* h, uint32_t y0, uint32_t nrows, int8_t* host_out)
{
    if (!h || !host_out || y0 >= h->p.L || nrows > h->p.L) return LAT_EINVAL;
    const uint32_t L = h->p.L;
    const uint32_t per = (uint32_t)(h->lay.stage_bytes / L);
    for (uint32_t r = 0; r < nrows; r += per) {
        const uint32_t n = nrows - r < per ? nrows - r : per;
        const uint32_t y = (uint32_t)(((uint64_t)y0 + r) % L);
        cudaError_t e = launch_unpack_rows(h->p.model, h->spins(), L, h->W, y, n, h->stage(), h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_out + (size_t)r * L, h->stage(), (size_t)n * L, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return LAT_ECUDA;
    }
    return LAT_OK;
}

int lat_get_spins(lat_t* h, int8_t* host_out)
{
    if (!h) return LAT_EINVAL;
    return lat_get_rows(h, 0, h->p.L, host_out);
}

int lat_set_spins(lat_t* h, const int8_t* host_in)
{
    if (!h || !host_in) return LAT_EINVAL;
    const uint32_t L = h->p.L;
    const uint32_t per = (uint32_t)(h->lay.stage_bytes / L);
    unsigned int* bad = reinterpret_cast<unsigned int*>(h->misc() + 20);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), h->stream);
    for (uint32_t r = 0; r < L && e == cudaSuccess; r += per) {
        const uint32_t n = L - r < per ? L - r : per;
        e = cudaMemcpyAsync(h->stage(), host_in + (size_t)r * L, (size_t)n * L, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_pack_rows(h->p.model, h->spins(), L, h->W, r, n, h->stage(), bad, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the stage is reused
    }
    unsigned int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, bad, sizeof(flag), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return LAT_ECUDA;
    return flag ? LAT_EINVAL : LAT_OK;
}

int lat_get_state(lat_t* h, void* host, size_t bytes)
{
    if (!h || !host || bytes != spins_bytes(&h->p)) return LAT_EINVAL;
    cudaError_t e = cudaMemcpyAsync(host, h->spins(), bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_set_state(lat_t* h, const void* host, size_t bytes)
{
    if (!h || !host || bytes != spins_bytes(&h->p)) return LAT_EINVAL;
    cudaError_t e = cudaMemcpyAsync(h->spins(), host, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_err(e);
}

int lat_get_sweep_index(lat_t* h, uint64_t* next)
{
    if (!h || !next) return LAT_EINVAL;
    *next = h->next_sweep;
    return LAT_OK;
}

int lat_set_sweep_index(lat_t* h, uint64_t next)
{
    if (!h || next >= kLastSweep) return LAT_EINVAL;
    h->next_sweep = next;
    return LAT_OK;
}

int lat_get_thresholds(lat_t* h, uint64_t* out, size_t n)
{
    if (!h || !out || n < h->nthr) return LAT_EINVAL;
    std::memcpy(out, h->thr, h->nthr * sizeof(uint64_t));
    return LAT_OK;
}

int lat_destroy(lat_t* h)
{
    if (!h) return LAT_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (h->owns) {
        const cudaError_t f = cudaFree(h->buf);
        if (e == cudaSuccess) e = f;
    }
    delete h;
    return cuda_err(e);
}

const char* lat_strerror(int code)
{
    switch (code) {
        case LAT_OK: return "success";
        case LAT_EINVAL: return "invalid argument";
        case LAT_ENOMEM: return "device buffer too small or allocation failed";
        case LAT_ECUDA: return "CUDA error";
        case LAT_ETIMEDOUT: return "a bounded device wait timed out";
        case LAT_ESTATE: return "handle in the wrong state for this call";
        default: return "unknown error";
    }
}

}  // extern "C"
