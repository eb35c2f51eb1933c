// C ABI of the simulator (declared in include/ea.h): argument validation,
// device state, the FP64 threshold tables, and the host-side schedule that
// splits a sweep range into kernel launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <new>
#include <vector>

#include "../../include/ea.h"
#include "ea_internal.h"


namespace {

int cuda_fail(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return EA_ENOMEM;
    return EA_ECUDA;
}

#define EA_TRY(expr)                                      \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_);      \
    } while (0)

uint32_t prob_to_u32(double p)
{
    const double v = std::floor(std::ldexp(p, 32));
    if (v >= 4294967295.0) return 4294967295u;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

bool swap_after(uint64_t s, uint32_t every) { return every != 0 && (s + 1) % every == 0; }
bool measured(uint64_t s, uint64_t from, uint32_t every)
{
    return every != 0 && s >= from && (s - from) % every == 0;
}

int validate_tables(const uint32_t *metro, const uint32_t *swapt, uint32_t NT, uint32_t len)
{
    for (uint32_t t = 0; metro && t < NT; ++t)
        if (metro[t * 3] > metro[t * 3 + 1] || metro[t * 3 + 1] > metro[t * 3 + 2]) return EA_EINVAL;
    if (NT > 1 && len > 0) {
        if (!swapt) return EA_EINVAL;
        for (uint32_t p = 0; p + 1 < NT; ++p)
            for (uint32_t k = 1; k < len; ++k)
                if (swapt[(size_t)p * len + k] > swapt[(size_t)p * len + k - 1]) return EA_EINVAL;
    }
    return EA_OK;
}

ea::SweepLaunch base_launch(ea_ctx *c)
{
    ea::SweepLaunch a;
    std::memset(&a, 0, sizeof(a));
    a.spins = c->d_spins;
    a.bonds = c->d_bonds;
    a.metro = c->d_metro;
    a.swapt = c->d_swapt;
    a.swap_len = c->swap_len;
    a.energy = c->d_energy;
    a.G = c->G;
    a.NT = c->NT;
    a.C = c->C;
    a.rk = c->rk;
    a.err = c->d_err;
    a.metro_f = c->d_metro_f;
    a.mag = c->d_mag;
    a.h_num = c->h_num;
    a.h_den = c->h_den;
    a.step = c->step;
    a.g_base = c->g_base;
    return a;
}

// Device memory of a context: plain allocations, or stream-ordered ones from
// a memory pool (no implicit device synchronisation on either side).
cudaError_t ctx_alloc(ea_ctx *c, void **p, size_t bytes, cudaStream_t st)
{
    if (c->pool) return cudaMallocFromPoolAsync(p, bytes, c->pool, st);
    return cudaMalloc(p, bytes);
}

void ctx_free(ea_ctx *c, void *p, cudaStream_t st)
{
    if (!p) return;
    if (c->pool) cudaFreeAsync(p, st);
    else cudaFree(p);
}

void free_ctx(ea_ctx *c, cudaStream_t st)
{
    if (!c) return;
    ctx_free(c, c->d_spins, st);
    ctx_free(c, c->d_bonds, st);
    ctx_free(c, c->d_metro, st);
    ctx_free(c, c->d_swapt, st);
    ctx_free(c, c->d_masks, st);
    ctx_free(c, c->d_energy, st);
    ctx_free(c, c->d_err, st);
    ctx_free(c, c->d_metro_f, st);
    ctx_free(c, c->d_mag, st);
    delete c;
}

}  // namespace

namespace ea {

size_t ctx_device_bytes(const ea_config *cfg)
{
    const size_t N = (size_t)cfg->L * cfg->L * cfg->L;
    const size_t n_spin = (size_t)cfg->n_groups * cfg->n_temps * cfg->n_copies * N;
    const size_t n_bond = (size_t)cfg->n_groups * 3 * N;
    const size_t n_swap = (size_t)(cfg->n_temps > 1 ? cfg->n_temps - 1 : 0) * cfg->swap_len;
    // resident arrays plus the import staging (spins and bonds once more)
    return 2 * (n_spin + n_bond) * 4 + (size_t)cfg->n_temps * 12 + (n_swap ? n_swap : 1) * 4 +
           (size_t)cfg->n_groups * cfg->n_copies * (kMaxTemps + cfg->n_temps * kLanes) * 4 + 4;
}

}  // namespace ea

extern "C" {

const char *ea_strerror(int code)
{
    switch (code) {
    case EA_OK: return "ok";
    case EA_PENDING: return "pending";
    case EA_EINVAL: return "invalid argument";
    case EA_ENOMEM: return "out of memory";
    case EA_ECUDA: return "CUDA error";
    case EA_ETIMEOUT: return "timed out";
    case EA_EUNSUPPORTED: return "unsupported lattice size";
    case EA_ESTATE: return "invalid state";
    default: return "unknown error";
    }
}

int ea_supported_L(uint32_t L) { return ea::supported_L((int)L) ? 1 : 0; }

int ea_build_tables(const double *beta, uint32_t n_temps, uint32_t n_sites, uint32_t *metro_out,
                    uint32_t *swap_out, uint32_t swap_cap, uint32_t *swap_len_out)
{
    if (!beta || n_temps == 0 || n_sites == 0 || !swap_len_out) return EA_EINVAL;
    for (uint32_t t = 0; t < n_temps; ++t) {
        if (!(beta[t] >= 0.0) || !std::isfinite(beta[t])) return EA_EINVAL;
        if (t > 0 && !(beta[t] <= beta[t - 1])) return EA_EINVAL;
    }
    if (metro_out)
        for (uint32_t t = 0; t < n_temps; ++t)
            for (int u = 0; u < 3; ++u)
                metro_out[t * 3 + u] = prob_to_u32(std::exp(-beta[t] * (12.0 - 4.0 * u)));
    // largest k with a non-zero threshold in any row, k <= 3N/2
    const uint32_t kmax = 3u * n_sites / 2u;
    uint32_t len = 0;
    for (uint32_t p = 0; p + 1 < n_temps; ++p) {
        const double db = beta[p] - beta[p + 1];
        // thresholds decrease in k: find the last non-zero one by bisection
        uint32_t lo = 0, hi = kmax;   // invariant: entry lo is non-zero (lo = 0: none known)
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (prob_to_u32(std::exp(-db * 4.0 * (double)mid)) != 0) lo = mid; else hi = mid - 1;
        }
        if (lo > len) len = lo;
    }
    *swap_len_out = len;
    if (swap_out && swap_cap >= len && len > 0)
        for (uint32_t p = 0; p + 1 < n_temps; ++p) {
            const double db = beta[p] - beta[p + 1];
            for (uint32_t k = 1; k <= len; ++k)
                swap_out[(size_t)p * swap_cap + (k - 1)] = prob_to_u32(std::exp(-db * 4.0 * (double)k));
        }
    return EA_OK;
}

int ea_build_tables_field(const double *beta, uint32_t n_temps, uint32_t n_sites, int32_t h_num,
                          int32_t h_den, uint64_t *metro_out, uint32_t *swap_out, uint32_t swap_cap,
                          uint32_t *swap_len_out)
{
    if (!beta || n_temps == 0 || n_sites == 0 || !swap_len_out || h_den < 1) return EA_EINVAL;
    if (3LL * h_den + std::llabs((long long)h_num) >= (1LL << 15)) return EA_EINVAL;
    for (uint32_t t = 0; t < n_temps; ++t) {
        if (!(beta[t] >= 0.0) || !std::isfinite(beta[t])) return EA_EINVAL;
        if (t > 0 && !(beta[t] <= beta[t - 1])) return EA_EINVAL;
    }
    const double h = (double)h_num / (double)h_den;
    if (metro_out)
        for (uint32_t t = 0; t < n_temps; ++t)
            for (int sp = 0; sp < 2; ++sp) {
                const int S = sp ? 1 : -1;
                for (int u = 0; u < 7; ++u) {
                    // the change of Et = h_den E - h_num M; accepted always where <= 0
                    const long long d = (long long)h_den * (12 - 4 * u) + 2LL * h_num * S;
                    metro_out[((size_t)t * 2 + sp) * 7 + u] =
                        d <= 0 ? (1ull << 32)
                               : prob_to_u32(std::exp(-beta[t] * (12.0 - 4.0 * u + 2.0 * h * S)));
                }
            }
    const long long step = std::gcd(4LL * h_den, 2LL * std::llabs((long long)h_num));
    const uint64_t kmax = (uint64_t)((6LL * n_sites * h_den + 2LL * n_sites * std::llabs((long long)h_num)) / step);
    const double stepd = (double)step;
    uint64_t len = 0;
    for (uint32_t p = 0; p + 1 < n_temps; ++p) {
        const double db = beta[p] - beta[p + 1];
        uint64_t lo = 0, hi = kmax;   // entry lo non-zero (lo = 0: none known); entries decrease in k
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo + 1) / 2;
            if (prob_to_u32(std::exp(-db * stepd * (double)mid / h_den)) != 0) lo = mid; else hi = mid - 1;
        }
        if (lo > len) len = lo;
    }
    if (len > 0xFFFFFFFFull) return EA_EINVAL;
    *swap_len_out = (uint32_t)len;
    if (swap_out && swap_cap >= len && len > 0)
        for (uint32_t p = 0; p + 1 < n_temps; ++p) {
            const double db = beta[p] - beta[p + 1];
            for (uint64_t k = 1; k <= len; ++k)
                swap_out[(size_t)p * swap_cap + (k - 1)] = prob_to_u32(std::exp(-db * stepd * (double)k / h_den));
        }
    return EA_OK;
}

int ea_create(const ea_config *cfg, void *stream, ea_ctx **out)
{
    return ea::create_ctx(cfg, (cudaStream_t)stream, nullptr, out);
}

int ea_create_field(const ea_config *cfg, const ea_field *field, void *stream, ea_ctx **out)
{
    return ea::create_ctx(cfg, (cudaStream_t)stream, nullptr, out, field);
}

void ea_destroy(ea_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx, ctx->stream);
}

}  // extern "C"

namespace ea {

// Checks a field's tables.  h_num == 0: the field-free method; its
// thresholds are written to metro0 [NT][3].
int validate_field(const ea_field *f, uint32_t NT, uint32_t *metro0)
{
    if (!f->metro || f->h_den < 1) return EA_EINVAL;
    if (3LL * f->h_den + std::llabs((long long)f->h_num) >= (1LL << 15)) return EA_EINVAL;
    for (uint32_t t = 0; t < NT; ++t)
        for (int sp = 0; sp < 2; ++sp) {
            const uint64_t *row = f->metro + ((size_t)t * 2 + sp) * 7;
            for (int u = 0; u < 7; ++u) {
                if (row[u] > (1ull << 32)) return EA_EINVAL;
                if (u > 0 && row[u] < row[u - 1]) return EA_EINVAL;
            }
            if (f->h_num == 0)
                for (int u = 0; u < 7; ++u) {
                    const uint64_t other = f->metro[((size_t)t * 2 + (1 - sp)) * 7 + u];
                    if (row[u] != other || (u < 3 && row[u] >= (1ull << 32)) ||
                        (u >= 3 && row[u] != (1ull << 32)))
                        return EA_EINVAL;
                    if (u < 3) metro0[t * 3 + u] = (uint32_t)row[u];
                }
        }
    return EA_OK;
}

// The wavefront kernel's kind for a field table (ea_field::metro, validated):
// the first u at which every slot's thresholds reach 2^32 ("always"), per spin
// value, must be 3 for one value and 4 for the other; 0 otherwise.
int field_wave_kind(const ea_field *f, uint32_t NT)
{
    int ua[2] = {-1, -1};
    for (uint32_t t = 0; t < NT; ++t)
        for (int sp = 0; sp < 2; ++sp) {
            const uint64_t *row = f->metro + ((size_t)t * 2 + sp) * 7;
            int first = 7;
            for (int u = 6; u >= 0 && row[u] == (1ull << 32); --u) first = u;
            if (ua[sp] >= 0 && ua[sp] != first) return 0;
            ua[sp] = first;
        }
    return wave_field_kind(ua[0], ua[1]);
}

int create_ctx(const ea_config *cfg_in, cudaStream_t stream, cudaMemPool_t pool, ea_ctx **out,
               const ea_field *field)
{
    if (!cfg_in || !out) return EA_EINVAL;
    *out = nullptr;
    ea_config cfg_copy = *cfg_in;
    const ea_config *cfg = &cfg_copy;
    uint32_t metro0[kMaxTemps * 3];
    if (field) {
        if (cfg->n_temps == 0 || cfg->n_temps > (uint32_t)kMaxTemps) return EA_EINVAL;
        const int rc = validate_field(field, cfg->n_temps, metro0);
        if (rc != EA_OK) return rc;
        if (field->h_num == 0) {   // exactly the field-free method
            cfg_copy.metro = metro0;
            field = nullptr;
        } else {
            cfg_copy.metro = nullptr;
        }
    }
    const uint32_t L = cfg->L;
    if (L < 4 || (L & 1u)) return EA_EINVAL;
    if (!ea::supported_L((int)L)) return EA_EUNSUPPORTED;
    if (cfg->n_groups == 0 || cfg->n_temps == 0 || cfg->n_temps > (uint32_t)ea::kMaxTemps)
        return EA_EINVAL;
    if (cfg->n_copies < 1 || cfg->n_copies > 2) return EA_EINVAL;
    if ((uint64_t)cfg->group_base + cfg->n_groups > (1ull << 32)) return EA_EINVAL;
    if (!cfg->bonds || !cfg->spins0 || (!cfg->metro && !field)) return EA_EINVAL;
    if (cfg->n_temps > 1 && cfg->swap_len > 0 && !cfg->swapt) return EA_EINVAL;
    int rc = validate_tables(cfg->metro, cfg->swapt, cfg->n_temps, cfg->swap_len);
    if (rc != EA_OK) return rc;

    ea_ctx *c = new (std::nothrow) ea_ctx();
    if (!c) return EA_ENOMEM;
    c->L = L;
    c->G = cfg->n_groups;
    c->NT = cfg->n_temps;
    c->C = cfg->n_copies;
    c->N = L * L * L;
    c->swap_len = cfg->swap_len;
    c->seed = cfg->seed;
    c->g_base = cfg->group_base;
    c->stream = stream;
    c->pool = pool;
    c->rk = ea::make_round_keys(cfg->seed);
    c->h_num = field ? field->h_num : 0;
    c->h_den = field ? field->h_den : 1;
    c->step = field ? std::gcd(4 * field->h_den, 2 * std::abs(field->h_num)) : 4;

    cudaError_t e = cudaGetDevice(&c->device);
    int optin = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e); }
    c->smem_optin = (size_t)optin;
    c->plans = ea::make_plans((int)L, (int)c->NT, (int)c->C, c->swap_len, c->smem_optin, field != nullptr,
                              field ? field_wave_kind(field, c->NT) : 0);
    if (c->plans.empty()) {
        delete c;
        return EA_EUNSUPPORTED;
    }
    c->plan_idx = 0;
    c->plan = c->plans[0];

    const size_t n_spin = (size_t)c->G * c->NT * c->C * c->N;
    const size_t n_bond = (size_t)c->G * 3 * c->N;
    const size_t n_swap = (size_t)(c->NT > 1 ? c->NT - 1 : 0) * c->swap_len;
    uint32_t *stage_s = nullptr, *stage_b = nullptr;
    cudaStream_t st = c->stream;
    auto fail = [&](cudaError_t err) {
        if (pool) cudaStreamSynchronize(st);
        ctx_free(c, stage_s, st);
        ctx_free(c, stage_b, st);
        free_ctx(c, st);
        return cuda_fail(err);
    };
    auto alloc = [&](auto **p, size_t bytes) { return ctx_alloc(c, reinterpret_cast<void **>(p), bytes, st); };
    if ((e = alloc(&c->d_spins, n_spin * 4)) != cudaSuccess) return fail(e);
    if ((e = alloc(&c->d_bonds, n_bond * 4)) != cudaSuccess) return fail(e);
    if (!field && (e = alloc(&c->d_metro, (size_t)c->NT * 3 * 4)) != cudaSuccess) return fail(e);
    if (field && (e = alloc(&c->d_metro_f, (size_t)c->NT * 14 * 8)) != cudaSuccess) return fail(e);
    if (field && (e = alloc(&c->d_mag, (size_t)c->G * c->C * c->NT * ea::kLanes * 4)) != cudaSuccess)
        return fail(e);
    if ((e = alloc(&c->d_swapt, (n_swap ? n_swap : 1) * 4)) != cudaSuccess) return fail(e);
    if ((e = alloc(&c->d_masks, (size_t)c->G * c->C * ea::kMaxTemps * 4)) != cudaSuccess)
        return fail(e);
    if ((e = alloc(&c->d_energy, (size_t)c->G * c->C * c->NT * ea::kLanes * 4)) != cudaSuccess)
        return fail(e);
    if ((e = alloc(&c->d_err, sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = alloc(&stage_s, n_spin * 4)) != cudaSuccess) return fail(e);
    if ((e = alloc(&stage_b, n_bond * 4)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(c->d_err, 0, sizeof(int), st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(stage_s, cfg->spins0, n_spin * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpyAsync(stage_b, cfg->bonds, n_bond * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if (!field &&
        (e = cudaMemcpyAsync(c->d_metro, cfg->metro, (size_t)c->NT * 3 * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if (field && (e = cudaMemcpyAsync(c->d_metro_f, field->metro, (size_t)c->NT * 14 * 8,
                                      cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if (n_swap &&
        (e = cudaMemcpyAsync(c->d_swapt, cfg->swapt, n_swap * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if ((e = ea::launch_import(stage_s, stage_b, c->d_spins, c->d_bonds, (int)L, c->G, c->NT, c->C, st,
                               &c->launches)) != cudaSuccess)
        return fail(e);
    if ((e = ea::launch_energy(c->d_spins, c->d_bonds, c->d_energy, (int)L, c->G, c->NT, c->C, st,
                               &c->launches, c->d_mag)) != cudaSuccess)
        return fail(e);
    if (pool) {
        // stream-ordered: the staging buffers are released after the import
        // kernels; the host waits for nothing (pageable sources are staged
        // by the copy calls themselves)
        ctx_free(c, stage_s, st);
        ctx_free(c, stage_b, st);
    } else {
        // the staging buffers are freed once the copies above have run
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
        cudaFree(stage_s);
        cudaFree(stage_b);
    }
    *out = c;
    return EA_OK;
}

void destroy_ctx(ea_ctx *c, cudaStream_t st)
{
    free_ctx(c, st);
}

}  // namespace ea

namespace {

// Enqueues the kernels of n sweeps starting at the context's counters with
// the given plan; does not advance the counters.
int run_sweeps(ea_ctx *c, const ea_sweep_args *args, const ea::Plan &plan)
{
    const uint32_t n = args->n_sweeps;
    cudaStream_t st = c->stream;
    ea::SweepLaunch a = base_launch(c);
    a.swap_every = args->swap_every;
    a.energy_log = args->energy_log;
    a.log_s0 = c->sweep;
    a.swap_log = args->swap_log;
    a.qhist = args->qhist;
    a.esum = args->esum;
    a.measure_from = args->measure_from;
    a.measure_every = args->measure_every;
    const uint64_t s_begin = c->sweep;
    if (plan.unit) {
        a.s0 = s_begin;
        a.n_sweeps = n;
        a.P0 = c->pass;
        a.pass_local0 = 0;
        const bool overlaps = c->C == 2 && args->qhist != nullptr && args->measure_every != 0;
        if (plan.form == ea::kFormUnitWave) {
            const bool meas = args->measure_every != 0 && (args->qhist != nullptr || args->esum != nullptr);
            const bool log = args->energy_log != nullptr || args->swap_log != nullptr;
            if (!meas) {
                EA_TRY(ea::launch_sweep_unit_wave(a, plan.swap_in_smem, plan.field_kind, 0, st, &c->launches));
                return EA_OK;
            }
            if (plan.field_kind == 0 && !log) {
                // field-free measured calls: energy sums, and with two copies the q histogram
                EA_TRY(ea::launch_sweep_unit_wave(a, plan.swap_in_smem, 0, overlaps ? 2 : 1, st, &c->launches));
                return EA_OK;
            }
            // measured calls with logs or in a field run under the first other unit plan (same results)
            for (const ea::Plan &q : c->plans)
                if (q.unit && q.form != ea::kFormUnitWave) return run_sweeps(c, args, q);
            return EA_EUNSUPPORTED;
        }
        if (plan.form == ea::kFormUnitFast)
            EA_TRY(ea::launch_sweep_unit_fast(a, (int)c->L, plan.threads_per_lattice,
                                              plan.swap_in_smem, overlaps, c->smem_optin, st,
                                              &c->launches));
        else
            EA_TRY(ea::launch_sweep_unit(a, (int)c->L, plan, overlaps, st, &c->launches));
        return EA_OK;
    }
    // Chunked form: sweep kernels run up to each swap or measured sweep;
    // swap passes and measurements run as their own kernels in between.
    uint64_t s = s_begin;
    uint32_t pass_local = 0;
    const uint64_t s_end = s_begin + n;
    while (s < s_end) {
        uint64_t e = s;
        while (e + 1 < s_end && !swap_after(e, args->swap_every) &&
               !measured(e, args->measure_from, args->measure_every))
            ++e;
        // sweeps [s, e]
        ea::SweepLaunch b = a;
        b.s0 = s;
        b.n_sweeps = (uint32_t)(e - s + 1);
        b.qhist = nullptr;
        b.esum = nullptr;
        b.measure_every = 0;
        const bool sw = swap_after(e, args->swap_every);
        const bool me = measured(e, args->measure_from, args->measure_every);
        b.compute_energy_last = 1;
        EA_TRY(ea::launch_sweep_chunk(b, (int)c->L, plan, st, &c->launches));
        if (sw) {
            b.P0 = c->pass + pass_local;
            b.pass_local0 = pass_local;
            int32_t *elog_row = args->energy_log
                ? args->energy_log + (size_t)(e - s_begin) * c->G * c->NT * c->C * ea::kLanes
                : nullptr;
            EA_TRY(ea::launch_swap_global(b, (int)c->L, c->pass + pass_local, c->d_masks, elog_row,
                                          st, &c->launches));
            ++pass_local;
        }
        if (me)
            EA_TRY(ea::launch_measure(c->d_spins, c->d_energy, (int)c->L, c->G, c->NT, c->C,
                                      nullptr, nullptr, args->qhist, args->esum, st, &c->launches));
        s = e + 1;
    }
    return EA_OK;
}

}  // namespace

extern "C" {

int ea_sweep(ea_ctx *c, const ea_sweep_args *args)
{
    if (!c || !args) return EA_EINVAL;
    if ((args->qhist) && c->C != 2) return EA_EINVAL;
    const uint32_t n = args->n_sweeps;
    if (n == 0) return EA_OK;
    uint64_t passes = 0;
    for (uint64_t s = c->sweep; s < c->sweep + n; ++s) passes += swap_after(s, args->swap_every);
    const int rc = run_sweeps(c, args, c->plan);
    if (rc != EA_OK) return rc;
    c->sweep += n;
    c->pass += passes;
    return EA_OK;
}

int ea_plan_count(const ea_ctx *c) { return c ? (int)c->plans.size() : EA_EINVAL; }

int ea_plan_current(const ea_ctx *c) { return c ? c->plan_idx : EA_EINVAL; }

int ea_plan_info(const ea_ctx *c, int index, ea_plan_desc *out)
{
    if (!c || !out || index < 0 || index >= (int)c->plans.size()) return EA_EINVAL;
    const ea::Plan &p = c->plans[(size_t)index];
    out->form = p.form;
    out->threads = p.threads;
    out->group_threads = p.threads_per_lattice;
    out->lattices_per_cta = p.lattices_per_cta;
    out->smem_bytes = p.smem;
    out->units_per_cta = p.unit ? 1 : 0;
    return EA_OK;
}

int ea_plan_select(ea_ctx *c, int index)
{
    if (!c || index < 0 || index >= (int)c->plans.size()) return EA_EINVAL;
    c->plan_idx = index;
    c->plan = c->plans[(size_t)index];
    return EA_OK;
}

int ea_autotune(ea_ctx *c, uint32_t probe_sweeps, uint32_t swap_every, float *ms_out)
{
    if (!c || probe_sweeps == 0) return EA_EINVAL;
    const size_t n_spin = (size_t)c->G * c->NT * c->C * c->N;
    const size_t n_e = (size_t)c->G * c->C * c->NT * ea::kLanes;
    uint32_t *save_s = nullptr;
    int32_t *save_e = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaError_t e = cudaMalloc(&save_s, n_spin * 4);
    if (e == cudaSuccess) e = cudaMalloc(&save_e, n_e * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save_s, c->d_spins, n_spin * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save_e, c->d_energy, n_e * 4, cudaMemcpyDeviceToDevice, c->stream);
    int32_t *save_m = nullptr;
    if (e == cudaSuccess && c->d_mag) e = cudaMalloc(&save_m, n_e * 4);
    if (e == cudaSuccess && c->d_mag)
        e = cudaMemcpyAsync(save_m, c->d_mag, n_e * 4, cudaMemcpyDeviceToDevice, c->stream);
    int best = c->plan_idx, rc = EA_OK;
    float best_ms = 0.f;
    ea_sweep_args args;
    std::memset(&args, 0, sizeof(args));
    args.n_sweeps = probe_sweeps;
    args.swap_every = swap_every;
    for (size_t i = 0; e == cudaSuccess && rc == EA_OK && i < c->plans.size(); ++i) {
        float ms = 0.f;
        for (int rep = 0; rep < 2 && rc == EA_OK && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(ev0, c->stream);
            if (e == cudaSuccess) rc = run_sweeps(c, &args, c->plans[i]);
            if (e == cudaSuccess && rc == EA_OK) e = cudaEventRecord(ev1, c->stream);
            if (e == cudaSuccess && rc == EA_OK) e = cudaEventSynchronize(ev1);
            if (e == cudaSuccess && rc == EA_OK) e = cudaEventElapsedTime(&ms, ev0, ev1);
            // every plan starts from the same state
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->d_spins, save_s, n_spin * 4, cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->d_energy, save_e, n_e * 4, cudaMemcpyDeviceToDevice, c->stream);
            if (e == cudaSuccess && save_m)
                e = cudaMemcpyAsync(c->d_mag, save_m, n_e * 4, cudaMemcpyDeviceToDevice, c->stream);
        }
        if (ms_out) ms_out[i] = ms;
        if (e == cudaSuccess && rc == EA_OK && (i == 0 || ms < best_ms)) {
            best_ms = ms;
            best = (int)i;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(save_s);
    cudaFree(save_e);
    cudaFree(save_m);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (rc != EA_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e);
    return ea_plan_select(c, best);
}

int ea_pt_swap(ea_ctx *c, uint32_t *masks)
{
    if (!c) return EA_EINVAL;
    cudaStream_t st = c->stream;
    EA_TRY(ea::launch_energy(c->d_spins, c->d_bonds, c->d_energy, (int)c->L, c->G, c->NT, c->C, st,
                             &c->launches, c->d_mag));
    ea::SweepLaunch a = base_launch(c);
    a.swap_log = masks;   // row 0 of a one-pass log
    a.pass_local0 = 0;
    EA_TRY(ea::launch_swap_global(a, (int)c->L, c->pass, c->d_masks, nullptr, st, &c->launches));
    c->pass += 1;
    return EA_OK;
}

int ea_measure(ea_ctx *c, int32_t *energies, uint32_t *ndiff, uint64_t *qhist)
{
    if (!c) return EA_EINVAL;
    if ((ndiff || qhist) && c->C != 2) return EA_EINVAL;
    cudaStream_t st = c->stream;
    EA_TRY(ea::launch_energy(c->d_spins, c->d_bonds, c->d_energy, (int)c->L, c->G, c->NT, c->C, st,
                             &c->launches, c->d_mag));
    EA_TRY(ea::launch_measure(c->d_spins, c->d_energy, (int)c->L, c->G, c->NT, c->C, energies, ndiff,
                              qhist, nullptr, st, &c->launches));
    return EA_OK;
}

int ea_measure_planes(ea_ctx *c, int mode, int32_t *out)
{
    if (!c || !out || (mode != 0 && mode != 1)) return EA_EINVAL;
    if (mode == 0 && c->C != 2) return EA_EINVAL;
    EA_TRY(ea::launch_measure_planes(c->d_spins, (int)c->L, c->G, c->NT, c->C, mode, out, c->stream,
                                     &c->launches));
    return EA_OK;
}

int ea_magnetisations(ea_ctx *c, int32_t *out)
{
    if (!c || !out) return EA_EINVAL;
    EA_TRY(ea::launch_magnetisation(c->d_spins, (int)c->L, c->G, c->NT, c->C, out, c->stream,
                                    &c->launches));
    return EA_OK;
}

int ea_read_spins(ea_ctx *c, uint32_t *dst)
{
    if (!c || !dst) return EA_EINVAL;
    EA_TRY(ea::launch_export(c->d_spins, dst, (int)c->L, c->G, c->NT, c->C, c->stream, &c->launches));
    return EA_OK;
}

int ea_read_spins_host(ea_ctx *c, uint32_t *dst)
{
    if (!c || !dst) return EA_EINVAL;
    const size_t bytes = (size_t)c->G * c->NT * c->C * c->N * 4;
    uint32_t *tmp = nullptr;
    EA_TRY(cudaMalloc(&tmp, bytes));
    cudaError_t e = ea::launch_export(c->d_spins, tmp, (int)c->L, c->G, c->NT, c->C, c->stream,
                                      &c->launches);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    return e == cudaSuccess ? EA_OK : cuda_fail(e);
}

int ea_write_spins(ea_ctx *c, const uint32_t *src, uint64_t sweep_index, uint64_t pass_index)
{
    if (!c || !src) return EA_EINVAL;
    EA_TRY(ea::launch_import_spins(src, c->d_spins, (int)c->L, c->G, c->NT, c->C, c->stream,
                                   &c->launches));
    EA_TRY(ea::launch_energy(c->d_spins, c->d_bonds, c->d_energy, (int)c->L, c->G, c->NT, c->C,
                             c->stream, &c->launches, c->d_mag));
    c->sweep = sweep_index;
    c->pass = pass_index;
    return EA_OK;
}

int ea_get_counters(const ea_ctx *c, uint64_t *sweep_index, uint64_t *pass_index)
{
    if (!c) return EA_EINVAL;
    if (sweep_index) *sweep_index = c->sweep;
    if (pass_index) *pass_index = c->pass;
    return EA_OK;
}

int ea_sync(ea_ctx *c)
{
    if (!c) return EA_EINVAL;
    EA_TRY(cudaStreamSynchronize(c->stream));
    EA_TRY(cudaGetLastError());
    // a bounded device-side wait that ran out raises the context's error flag
    int err = 0;
    EA_TRY(cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) {
        EA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
        return EA_ETIMEOUT;
    }
    return EA_OK;
}

uint64_t ea_launch_count(const ea_ctx *c) { return c ? c->launches : 0; }

int ea_run(const ea_config *cfg, const ea_sweep_args *args, void *stream, int32_t *energies_host,
           uint32_t *spins_host, uint64_t *qhist_host, int64_t *esum_host)
{
    if (!cfg || !args) return EA_EINVAL;
    if (args->energy_log || args->swap_log || args->qhist || args->esum) return EA_EINVAL;
    ea_ctx *c = nullptr;
    int rc = ea_create(cfg, stream, &c);
    if (rc != EA_OK) return rc;
    const size_t nq = (size_t)c->NT * (c->N + 1);
    const size_t ne = (size_t)c->G * c->NT * c->C * ea::kLanes;
    uint64_t *d_q = nullptr;
    int64_t *d_es = nullptr;
    int32_t *d_e = nullptr;
    cudaError_t e = cudaSuccess;
    ea_sweep_args a2 = *args;
    if (qhist_host) {
        if (c->C != 2) { ea_destroy(c); return EA_EINVAL; }
        e = cudaMalloc(&d_q, nq * 8);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_q, 0, nq * 8, c->stream);
        a2.qhist = d_q;
    }
    if (e == cudaSuccess && esum_host) {
        e = cudaMalloc(&d_es, (size_t)c->NT * 8);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_es, 0, (size_t)c->NT * 8, c->stream);
        a2.esum = d_es;
    }
    if (e == cudaSuccess) {
        rc = ea_sweep(c, &a2);
        if (rc == EA_OK && energies_host) {
            e = cudaMalloc(&d_e, ne * 4);
            if (e == cudaSuccess)
                e = ea::launch_measure(c->d_spins, c->d_energy, (int)c->L, c->G, c->NT, c->C, d_e,
                                       nullptr, nullptr, nullptr, c->stream, &c->launches);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(energies_host, d_e, ne * 4, cudaMemcpyDeviceToHost, c->stream);
        }
        if (rc == EA_OK && e == cudaSuccess && qhist_host)
            e = cudaMemcpyAsync(qhist_host, d_q, nq * 8, cudaMemcpyDeviceToHost, c->stream);
        if (rc == EA_OK && e == cudaSuccess && esum_host)
            e = cudaMemcpyAsync(esum_host, d_es, (size_t)c->NT * 8, cudaMemcpyDeviceToHost, c->stream);
        if (rc == EA_OK && e == cudaSuccess) rc = ea_sync(c);
        if (rc == EA_OK && e == cudaSuccess && spins_host) rc = ea_read_spins_host(c, spins_host);
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(d_q);
    cudaFree(d_es);
    cudaFree(d_e);
    ea_destroy(c);
    if (rc != EA_OK) return rc;
    return e == cudaSuccess ? EA_OK : cuda_fail(e);
}

}  // extern "C"
