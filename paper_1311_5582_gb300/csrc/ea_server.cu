// Serving loop: admits simulation requests by device memory, keeps their
// state resident on the device, and advances every resident request together
// in rounds of one persistent batched launch (continuous batching).
//
// One worker thread owns the GPU work.  Rounds run back to back on one
// compute stream: while round k runs, the worker
//   1. decides and launches round k+1 (ea_batch_sweep_each on the other of two
//      batch objects, so neither overwrites the tables of a call in flight):
//      the resident requests with the least work left -- as many as give
//      about two (group, copy) units per SM -- advance by min(q, sweeps left)
//      sweeps, q sized so that a round lasts about round_ms at the measured
//      rate (shortest remaining work first, which minimises mean latency when
//      requests queue, while keeping the GPU full);
//   2. right behind each round, enqueues the export of the requests that the
//      round finishes (their sweep counts are known when it is launched), and
//      an event;
//   3. admits queued requests in arrival order as long as their device bytes
//      fit the budget (contexts are created on a second stream from a
//      stream-ordered memory pool); they join the next round;
//   4. waits for the previous round's event only, then copies the finished
//      requests' outputs to their host buffers on a third stream and releases
//      their memory -- the GPU meanwhile runs the round already queued.
// Every request's trajectory is the one ea_sweep would give it alone: the
// batch keeps each member's own counters, tables and swap schedule.
// Temperature-packed requests (ea_submit_tp) take part in the same rounds
// with their own launches (ea_tp_sweep) behind the batched ones; their
// contexts use cudaMalloc / cudaFree, so admitting or finishing one
// synchronises the device once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/ea.h"
#include "ea_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    uint64_t ticket = 0;
    ea_config cfg{};                              // points into the copies below
    std::vector<uint32_t> bonds, spins0, metro, swapt;
    uint32_t n_sweeps = 0, swap_every = 0;
    uint32_t *spins_out = nullptr;
    int32_t *energies_out = nullptr;
    int32_t *mags_out = nullptr;
    bool field = false;                           // in an external field (runs in the field batches)
    bool has_fld = false;                         // submitted with ea_submit_field (h_num may be 0)
    ea_field fld{};                               // points into metro_f
    std::vector<uint64_t> metro_f;
    size_t bytes = 0;                             // device bytes while resident
    Clock::time_point t_submit;
    ea_ctx *ctx = nullptr;
    bool tp = false;                              // temperature-packed (ea_submit_tp): tcfg, tctx
    ea_tp_config tcfg{};                          // points into the copies (bonds in tbonds)
    std::vector<uint8_t> tbonds;
    ea_tp *tctx = nullptr;
    double flips_per_sweep = 0.0;                 // flip attempts of one sweep
    uint64_t units = 0;                           // CTAs of one launch ((group or realization) x copy)
    uint32_t left = 0;                            // sweeps not yet launched
    uint64_t words = 0;                           // site-words of one sweep (N * NT * C * G)
    uint32_t waited = 0;                          // consecutive rounds left out
    uint32_t *d_spins = nullptr;                  // export scratch (pool) of a finishing request
    int32_t *d_energies = nullptr, *d_mags = nullptr;
    int status = EA_OK;                           // of the export
};

// A launched round: its completion event and the requests it finishes.
struct Round {
    cudaEvent_t start = nullptr, done = nullptr;
    std::vector<std::unique_ptr<Request>> finishing;
    double work = 0.0;                            // site-word updates of the round
    bool active = false;
};

// A request left out of this many consecutive rounds goes first in the next.
constexpr uint32_t kAgeRounds = 64;

}  // namespace

struct ea_server {
    int device = 0, sms = 1;
    size_t budget = 0, used = 0, peak = 0;
    uint32_t max_live = 256;
    double round_ms = 20.0;
    cudaStream_t compute = nullptr, admit = nullptr, copy = nullptr;
    cudaEvent_t admitted = nullptr;
    cudaMemPool_t pool = nullptr;
    ea_batch *batch[2] = {nullptr, nullptr};      // rounds alternate between the two
    ea_batch *batch_f[2] = {nullptr, nullptr};    // the same for requests in a field (own kernel)
    Round rounds_ring[2];
    uint64_t round_index = 0;
    std::thread worker;
    Clock::time_point t0;

    std::mutex mu;                                // guards everything below up to `live`
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<std::unique_ptr<Request>> queue;   // submitted, not yet admitted
    std::unordered_set<uint64_t> open;            // submitted, not yet finished
    std::unordered_map<uint64_t, int> finished;   // finished, not yet polled: status
    uint64_t next_ticket = 1;
    std::vector<double> lat_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, rounds = 0;
    double flips = 0.0, busy_s = 0.0;
    double first_submit_s = -1.0, last_done_s = 0.0;
    size_t n_live = 0;

    std::vector<std::unique_ptr<Request>> live;   // worker thread only
    double rate = 2.0e8;                          // site-words per ms (updated each round)
};

namespace {

// Records the end of a request (status EA_OK or an error); takes the lock.
void finish(ea_server *s, Request &r, int status)
{
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->open.erase(r.ticket);
    s->finished[r.ticket] = status;
    if (status == EA_OK) {
        s->completed += 1;
        s->lat_ms.push_back(ms_between(r.t_submit, now));
        s->flips += r.flips_per_sweep * r.n_sweeps;
        s->last_done_s = ms_between(s->t0, now) * 1e-3;
    } else {
        s->failed += 1;
    }
    s->cv_done.notify_all();
}

// Admits queued requests, in arrival order, while they fit the memory budget
// and the resident-request limit.  Contexts are created on the admission
// stream; the compute stream waits for them before its next launch.
void admit(ea_server *s)
{
    bool any = false;
    for (;;) {
        std::unique_ptr<Request> r;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty() || s->live.size() >= s->max_live) break;
            Request &h = *s->queue.front();
            if (s->used + h.bytes > s->budget) {
                if (!s->live.empty() || h.bytes <= s->budget) break;   // waits for memory
            }
            r = std::move(s->queue.front());
            s->queue.pop_front();
        }
        if (r->bytes > s->budget) {            // can never fit
            finish(s, *r, EA_ENOMEM);
            continue;
        }
        ea_ctx *ctx = nullptr;
        ea_tp *tctx = nullptr;
        // a temperature-packed context is created (cudaMalloc) and filled on the
        // admission stream, which ea_tp_create synchronises before it returns
        const int rc = r->tp ? ea_tp_create(&r->tcfg, s->admit, &tctx)
                             : ea::create_ctx(&r->cfg, s->admit, s->pool, &ctx, r->has_fld ? &r->fld : nullptr);
        if (rc == EA_ENOMEM && !s->live.empty()) {
            // the budget was optimistic: retry once resident requests finish
            std::lock_guard<std::mutex> lk(s->mu);
            s->queue.push_front(std::move(r));
            break;
        }
        if (rc != EA_OK) {
            finish(s, *r, rc);
            continue;
        }
        if (r->tp) {
            ea::tp_set_stream(tctx, s->compute);  // all later work of this context
            r->tctx = tctx;
        } else {
            ctx->stream = s->compute;
            r->ctx = ctx;
        }
        r->left = r->n_sweeps;
        // the host copies of the inputs are no longer needed
        std::vector<uint32_t>().swap(r->bonds);
        std::vector<uint32_t>().swap(r->spins0);
        std::vector<uint8_t>().swap(r->tbonds);
        s->used += r->bytes;
        s->peak = std::max(s->peak, s->used);
        s->live.push_back(std::move(r));
        any = true;
    }
    if (any) {
        cudaEventRecord(s->admitted, s->admit);
        cudaStreamWaitEvent(s->compute, s->admitted, 0);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->n_live = s->live.size();
}

// Frees a request's context (stream-ordered on the compute stream for pooled
// contexts; a temperature-packed one synchronises it and frees with cudaFree).
void release_request(ea_server *s, Request &r)
{
    if (r.ctx) ea::destroy_ctx(r.ctx, s->compute);
    if (r.tctx) ea_tp_destroy(r.tctx);
    r.ctx = nullptr;
    r.tctx = nullptr;
}

// Enqueues on the compute stream, behind the round that finishes request r,
// the export of its final energies and spins into pool scratch.
void enqueue_export(ea_server *s, Request &r)
{
    if (r.tp) {
        const ea_tp_config &t = r.tcfg;
        const size_t W = (t.n_temps + 31) / 32, N = (size_t)t.L * t.L * t.L;
        const size_t nsp = (size_t)t.n_real * t.n_copies * W * N, nen = (size_t)t.n_real * t.n_temps * t.n_copies;
        cudaError_t e = cudaSuccess;
        if (r.spins_out)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.d_spins), nsp * 4, s->pool, s->compute);
        if (e == cudaSuccess && r.energies_out)
            e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.d_energies), nen * 4, s->pool, s->compute);
        int rc = EA_OK;
        if (e == cudaSuccess) rc = ea_tp_read(r.tctx, r.d_spins, r.d_energies);
        r.status = e != cudaSuccess ? (e == cudaErrorMemoryAllocation ? EA_ENOMEM : EA_ECUDA) : rc;
        return;
    }
    ea_ctx *c = r.ctx;
    const size_t nsp = (size_t)c->G * c->NT * c->C * c->N, nen = (size_t)c->G * c->NT * c->C * ea::kLanes;
    cudaError_t e = cudaSuccess;
    int rc = EA_OK;
    if (r.energies_out) {
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.d_energies), nen * 4, s->pool, s->compute);
        if (e == cudaSuccess) rc = ea_measure(c, r.d_energies, nullptr, nullptr);
    }
    if (e == cudaSuccess && rc == EA_OK && r.spins_out) {
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.d_spins), nsp * 4, s->pool, s->compute);
        if (e == cudaSuccess) rc = ea_read_spins(c, r.d_spins);
    }
    if (e == cudaSuccess && rc == EA_OK && r.mags_out) {
        e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.d_mags), nen * 4, s->pool, s->compute);
        if (e == cudaSuccess) rc = ea_magnetisations(c, r.d_mags);
    }
    r.status = e != cudaSuccess ? (e == cudaErrorMemoryAllocation ? EA_ENOMEM : EA_ECUDA) : rc;
}

// Waits for a launched round (and the exports behind it), copies the outputs
// of the requests it finished to their host buffers on the copy stream, and
// releases their scratch and device state.
void deliver(ea_server *s, Round &rd)
{
    const cudaError_t es = cudaEventSynchronize(rd.done);
    float ms = 0.0f;
    if (es == cudaSuccess && cudaEventElapsedTime(&ms, rd.start, rd.done) == cudaSuccess && ms > 0.5f)
        s->rate = 0.5 * s->rate + 0.5 * (rd.work / (double)ms);
    std::vector<int> status(rd.finishing.size(), EA_OK);
    for (size_t j = 0; j < rd.finishing.size(); ++j) {
        Request &r = *rd.finishing[j];
        int st = es != cudaSuccess ? EA_ECUDA : r.status;
        cudaError_t e = cudaSuccess;
        if (r.tp) {
            const ea_tp_config &t = r.tcfg;
            const size_t W = (t.n_temps + 31) / 32, N = (size_t)t.L * t.L * t.L;
            if (st == EA_OK && r.spins_out)
                e = cudaMemcpyAsync(r.spins_out, r.d_spins, (size_t)t.n_real * t.n_copies * W * N * 4,
                                    cudaMemcpyDeviceToHost, s->copy);
            if (st == EA_OK && e == cudaSuccess && r.energies_out)
                e = cudaMemcpyAsync(r.energies_out, r.d_energies, (size_t)t.n_real * t.n_temps * t.n_copies * 4,
                                    cudaMemcpyDeviceToHost, s->copy);
            if (e != cudaSuccess) st = EA_ECUDA;
            status[j] = st;
            continue;
        }
        ea_ctx *c = r.ctx;
        if (st == EA_OK && r.energies_out)
            e = cudaMemcpyAsync(r.energies_out, r.d_energies, (size_t)c->G * c->NT * c->C * ea::kLanes * 4,
                                cudaMemcpyDeviceToHost, s->copy);
        if (st == EA_OK && e == cudaSuccess && r.spins_out)
            e = cudaMemcpyAsync(r.spins_out, r.d_spins, (size_t)c->G * c->NT * c->C * c->N * 4,
                                cudaMemcpyDeviceToHost, s->copy);
        if (st == EA_OK && e == cudaSuccess && r.mags_out)
            e = cudaMemcpyAsync(r.mags_out, r.d_mags, (size_t)c->G * c->NT * c->C * ea::kLanes * 4,
                                cudaMemcpyDeviceToHost, s->copy);
        if (e != cudaSuccess) st = EA_ECUDA;
        status[j] = st;
    }
    const cudaError_t ec = cudaStreamSynchronize(s->copy);
    for (size_t j = 0; j < rd.finishing.size(); ++j) {
        Request &r = *rd.finishing[j];
        if (r.d_spins) cudaFreeAsync(r.d_spins, s->copy);
        if (r.d_energies) cudaFreeAsync(r.d_energies, s->copy);
        if (r.d_mags) cudaFreeAsync(r.d_mags, s->copy);
        r.d_spins = nullptr;
        r.d_energies = nullptr;
        r.d_mags = nullptr;
        release_request(s, r);                    // after every round already queued
        s->used -= r.bytes;
        finish(s, r, ec != cudaSuccess ? EA_ECUDA : status[j]);
    }
    rd.finishing.clear();
    rd.active = false;
}

// Launches round k on batch object k % 2 (whose previous call, round k - 2,
// has been delivered): the resident requests in order of least work left
// until their (group, copy) units give about two tasks per SM; then the
// exports of the requests this round finishes and the round's event.
void run_round(ea_server *s, uint64_t k)
{
    Round &rd = s->rounds_ring[k & 1];
    ea_batch *b = s->batch[k & 1];
    const size_t n = s->live.size();
    // requests with nothing to run (zero sweeps) finish with this round
    std::vector<char> in_round(n, 0);
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const Request &a = *s->live[x], &bq = *s->live[y];
        const bool aged_a = a.waited >= kAgeRounds, aged_b = bq.waited >= kAgeRounds;
        if (aged_a != aged_b) return aged_a;      // starved requests first
        return (double)a.left * (double)a.words < (double)bq.left * (double)bq.words;
    });
    double words = 0.0;
    uint64_t units = 0;
    for (size_t j = 0; j < n; ++j) {
        const Request &r = *s->live[order[j]];
        if (r.left == 0) continue;
        if (units >= 2ull * (uint64_t)s->sms && words > 0.0) break;
        in_round[order[j]] = 1;
        words += (double)r.words;
        units += r.units;
    }
    const double qd = s->round_ms * s->rate / (words > 0 ? words : 1.0);
    const uint32_t q = (uint32_t)std::max(1.0, std::min(qd, 1048576.0));
    // requests in a field run in the field batch kernel: one call per kind
    ea_batch *bf = s->batch_f[k & 1];
    ea_batch_clear(b);
    ea_batch_clear(bf);
    std::vector<uint32_t> nsw[2], kev[2];
    int rc = EA_OK;
    double work = 0.0, kind_work[2] = {0.0, 0.0};
    std::vector<uint32_t> nsw_all(n);
    for (size_t i = 0; i < n && rc == EA_OK; ++i) {
        Request &r = *s->live[i];
        nsw_all[i] = in_round[i] ? std::min(q, r.left) : 0u;
        r.waited = in_round[i] ? 0u : r.waited + 1u;
        const double w = (double)nsw_all[i] * (double)r.words;
        work += w;
        if (r.tp) continue;                       // launched on its own below
        const int kd = r.field ? 1 : 0;
        rc = ea_batch_add(kd ? bf : b, r.ctx);
        nsw[kd].push_back(nsw_all[i]);
        kev[kd].push_back(r.swap_every);
        kind_work[kd] += w;
    }
    cudaEventRecord(rd.start, s->compute);
    if (rc == EA_OK && kind_work[0] > 0.0) rc = ea_batch_sweep_each(b, nsw[0].data(), kev[0].data());
    if (rc == EA_OK && kind_work[1] > 0.0) rc = ea_batch_sweep_each(bf, nsw[1].data(), kev[1].data());
    // temperature-packed requests: their own launches, behind the batches
    for (size_t i = 0; i < n && rc == EA_OK; ++i) {
        Request &r = *s->live[i];
        if (r.tp && nsw_all[i] > 0) rc = ea_tp_sweep(r.tctx, nsw_all[i], r.swap_every, nullptr, nullptr);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->rounds += 1;
    }
    if (rc != EA_OK) {
        // the round failed: every resident request fails with its status
        cudaStreamSynchronize(s->compute);
        for (size_t i = 0; i < n; ++i) {
            Request &r = *s->live[i];
            release_request(s, r);
            s->used -= r.bytes;
            finish(s, r, rc);
        }
        s->live.clear();
        cudaStreamSynchronize(s->compute);
        std::lock_guard<std::mutex> lk(s->mu);
        s->n_live = 0;
        return;
    }
    // requests whose sweeps are now all launched finish with this round
    std::vector<std::unique_ptr<Request>> keep;
    for (size_t i = 0; i < n; ++i) {
        std::unique_ptr<Request> &r = s->live[i];
        r->left -= nsw_all[i];
        if (r->left == 0) {
            enqueue_export(s, *r);
            rd.finishing.push_back(std::move(r));
        } else {
            keep.push_back(std::move(r));
        }
    }
    s->live.swap(keep);
    cudaEventRecord(rd.done, s->compute);
    rd.work = work;
    rd.active = true;
    std::lock_guard<std::mutex> lk(s->mu);
    s->n_live = s->live.size();
}

void worker_main(ea_server *s)
{
    cudaSetDevice(s->device);
    Clock::time_point busy_from;
    bool busy = false;
    for (;;) {
        const bool in_flight = s->rounds_ring[0].active || s->rounds_ring[1].active;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->live.empty() && !in_flight)
                s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->stop) break;
        }
        admit(s);
        if (!busy && (!s->live.empty() || in_flight)) {
            busy = true;
            busy_from = Clock::now();
        }
        const uint64_t k = s->round_index;
        Round &prev = s->rounds_ring[(k + 1) & 1];       // round k - 1, if any
        if (!s->live.empty()) {
            run_round(s, k);                              // queued behind round k - 1
            s->round_index = k + 1;
        }
        if (prev.active) deliver(s, prev);
        const bool idle = s->live.empty() && !s->rounds_ring[0].active && !s->rounds_ring[1].active;
        if (idle && busy) {
            busy = false;
            std::lock_guard<std::mutex> lk(s->mu);
            s->busy_s += ms_between(busy_from, Clock::now()) * 1e-3;
        }
    }
    // shutting down: drop what is left
    cudaStreamSynchronize(s->compute);
    cudaStreamSynchronize(s->admit);
    cudaStreamSynchronize(s->copy);
    for (Round &rd : s->rounds_ring) {
        for (auto &r : rd.finishing) {
            if (r->d_spins) cudaFreeAsync(r->d_spins, s->compute);
            if (r->d_energies) cudaFreeAsync(r->d_energies, s->compute);
            if (r->d_mags) cudaFreeAsync(r->d_mags, s->compute);
            release_request(s, *r);
        }
        rd.finishing.clear();
        rd.active = false;
    }
    for (auto &r : s->live) release_request(s, *r);
    s->live.clear();
    cudaStreamSynchronize(s->compute);
}

// Frees a server's streams, events, pool and batch objects (worker stopped).
void release_server(ea_server *s)
{
    for (ea_batch *b : s->batch)
        if (b) ea_batch_destroy(b);
    for (ea_batch *b : s->batch_f)
        if (b) ea_batch_destroy(b);
    for (Round &rd : s->rounds_ring) {
        if (rd.start) cudaEventDestroy(rd.start);
        if (rd.done) cudaEventDestroy(rd.done);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->admitted) cudaEventDestroy(s->admitted);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->admit) cudaStreamDestroy(s->admit);
    if (s->compute) cudaStreamDestroy(s->compute);
    delete s;
}

// Up-front checks of a request (the tables are validated at admission).
int check_request(const ea_config *cfg, bool need_metro)
{
    if (cfg->L < 4 || (cfg->L & 1u)) return EA_EINVAL;
    if (!ea::supported_L((int)cfg->L)) return EA_EUNSUPPORTED;
    if (cfg->n_groups == 0 || cfg->n_temps == 0 || cfg->n_temps > (uint32_t)ea::kMaxTemps) return EA_EINVAL;
    if (cfg->n_copies < 1 || cfg->n_copies > 2) return EA_EINVAL;
    if ((uint64_t)cfg->group_base + cfg->n_groups > (1ull << 32)) return EA_EINVAL;
    if (!cfg->bonds || !cfg->spins0 || (need_metro && !cfg->metro)) return EA_EINVAL;
    if (cfg->n_temps > 1 && cfg->swap_len > 0 && !cfg->swapt) return EA_EINVAL;
    return EA_OK;
}

}  // namespace

extern "C" {

int ea_server_create(const ea_server_opts *opts, ea_server **out)
{
    if (!out) return EA_EINVAL;
    *out = nullptr;
    ea_server *s = new (std::nothrow) ea_server();
    if (!s) return EA_ENOMEM;
    s->t0 = Clock::now();
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    const size_t cap = free_b / 10 * 9;
    s->budget = (opts && opts->mem_budget) ? std::min((size_t)opts->mem_budget, cap) : cap / 10 * 9;
    if (opts && opts->max_live) s->max_live = opts->max_live;
    if (opts && opts->round_ms) s->round_ms = opts->round_ms;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->admitted, cudaEventDisableTiming);
    for (Round &rd : s->rounds_ring) {
        if (e == cudaSuccess) e = cudaEventCreate(&rd.start);
        if (e == cudaSuccess) e = cudaEventCreate(&rd.done);
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        e = cudaMemPoolCreate(&s->pool, &props);
    }
    if (e == cudaSuccess) {
        // keep freed blocks for reuse up to the budget instead of returning them
        uint64_t thr = s->budget;
        e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    int rc = e == cudaSuccess ? EA_OK : EA_ECUDA;
    if (rc == EA_OK) rc = ea_batch_create(s->compute, &s->batch[0]);
    if (rc == EA_OK) rc = ea_batch_create(s->compute, &s->batch[1]);
    if (rc == EA_OK) rc = ea_batch_create(s->compute, &s->batch_f[0]);
    if (rc == EA_OK) rc = ea_batch_create(s->compute, &s->batch_f[1]);
    if (rc == EA_OK) {
        try {
            s->worker = std::thread(worker_main, s);
        } catch (...) {
            rc = EA_ENOMEM;
        }
    }
    if (rc != EA_OK) {
        release_server(s);
        return rc;
    }
    *out = s;
    return EA_OK;
}

int ea_submit(ea_server *s, const ea_config *cfg, const ea_request *req, uint64_t *ticket)
{
    return ea_submit_field(s, cfg, nullptr, req, ticket);
}

int ea_submit_field(ea_server *s, const ea_config *cfg, const ea_field *field, const ea_request *req,
                    uint64_t *ticket)
{
    if (!s || !cfg || !req || !ticket) return EA_EINVAL;
    const bool in_field = field != nullptr && field->h_num != 0;
    if (field && (!field->metro || field->h_den < 1)) return EA_EINVAL;
    const int chk = check_request(cfg, field == nullptr);
    if (chk != EA_OK) return chk;
    auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
    if (!r) return EA_ENOMEM;
    const size_t N = (size_t)cfg->L * cfg->L * cfg->L;
    const size_t nsp = (size_t)cfg->n_groups * cfg->n_temps * cfg->n_copies * N;
    const size_t nbo = (size_t)cfg->n_groups * 3 * N;
    const size_t nsw = (size_t)(cfg->n_temps > 1 ? cfg->n_temps - 1 : 0) * cfg->swap_len;
    try {
        r->bonds.assign(cfg->bonds, cfg->bonds + nbo);
        r->spins0.assign(cfg->spins0, cfg->spins0 + nsp);
        if (cfg->metro) r->metro.assign(cfg->metro, cfg->metro + (size_t)cfg->n_temps * 3);
        if (nsw) r->swapt.assign(cfg->swapt, cfg->swapt + nsw);
        if (field) r->metro_f.assign(field->metro, field->metro + (size_t)cfg->n_temps * 14);
    } catch (...) {
        return EA_ENOMEM;
    }
    r->cfg = *cfg;
    r->cfg.bonds = r->bonds.data();
    r->cfg.spins0 = r->spins0.data();
    r->cfg.metro = cfg->metro ? r->metro.data() : nullptr;
    r->cfg.swapt = nsw ? r->swapt.data() : nullptr;
    if (field) {
        // the field's tables (h_num == 0 gives the field-free method, as ea_create_field)
        r->has_fld = true;
        r->field = in_field;
        r->fld = *field;
        r->fld.metro = r->metro_f.data();
    }
    r->mags_out = in_field ? req->magnetisations_out : nullptr;
    r->n_sweeps = req->n_sweeps;
    r->swap_every = req->swap_every;
    r->spins_out = req->spins_out;
    r->energies_out = req->energies_out;
    r->words = (uint64_t)nsp;
    r->flips_per_sweep = (double)nsp * 32.0;
    r->units = (uint64_t)cfg->n_groups * cfg->n_copies;
    // resident state plus the output scratch taken at completion
    const size_t nen = (size_t)cfg->n_groups * cfg->n_temps * cfg->n_copies * ea::kLanes;
    r->bytes = ea::ctx_device_bytes(cfg) + (r->spins_out ? nsp * 4 : 0) + (r->energies_out ? nen * 4 : 0) +
               (r->field ? nen * 4 * (r->mags_out ? 2 : 1) + (size_t)cfg->n_temps * 14 * 8 : 0);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return EA_ESTATE;
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->open.insert(r->ticket);
        s->submitted += 1;
        if (s->first_submit_s < 0) s->first_submit_s = ms_between(s->t0, r->t_submit) * 1e-3;
        s->queue.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return EA_OK;
}

int ea_submit_tp(ea_server *s, const ea_tp_config *cfg, const ea_tp_request *req, uint64_t *ticket)
{
    if (!s || !cfg || !req || !ticket) return EA_EINVAL;
    if (cfg->L < 4 || (cfg->L & 1u)) return EA_EINVAL;
    if (!ea::supported_L((int)cfg->L)) return EA_EUNSUPPORTED;
    if (cfg->n_real == 0 || cfg->n_temps == 0 || cfg->n_temps > 64 || cfg->n_copies < 1 || cfg->n_copies > 2)
        return EA_EINVAL;
    if ((uint64_t)cfg->real_base + cfg->n_real > (1ull << 32)) return EA_EINVAL;
    if (!cfg->bonds || !cfg->spins0 || !cfg->metro) return EA_EINVAL;
    if (cfg->n_temps > 1 && cfg->swap_len > 0 && !cfg->swapt) return EA_EINVAL;
    auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
    if (!r) return EA_ENOMEM;
    const size_t N = (size_t)cfg->L * cfg->L * cfg->L, W = (cfg->n_temps + 31) / 32;
    const size_t nsp = (size_t)cfg->n_real * cfg->n_copies * W * N, nbo = (size_t)cfg->n_real * 3 * N;
    const size_t nen = (size_t)cfg->n_real * cfg->n_temps * cfg->n_copies;
    const size_t nsw = (size_t)(cfg->n_temps > 1 ? cfg->n_temps - 1 : 0) * cfg->swap_len;
    try {
        r->tbonds.assign(cfg->bonds, cfg->bonds + nbo);
        r->spins0.assign(cfg->spins0, cfg->spins0 + nsp);
        r->metro.assign(cfg->metro, cfg->metro + (size_t)cfg->n_temps * 3);
        if (nsw) r->swapt.assign(cfg->swapt, cfg->swapt + nsw);
    } catch (...) {
        return EA_ENOMEM;
    }
    r->tp = true;
    r->tcfg = *cfg;
    r->tcfg.bonds = r->tbonds.data();
    r->tcfg.spins0 = r->spins0.data();
    r->tcfg.metro = r->metro.data();
    r->tcfg.swapt = nsw ? r->swapt.data() : nullptr;
    r->n_sweeps = req->n_sweeps;
    r->swap_every = req->swap_every;
    r->spins_out = req->spins_out;
    r->energies_out = req->energies_out;
    // work in units of a realization-packed site-word update (32 flip attempts):
    // one flip attempt of this form costs about a third of one (one uniform per
    // attempt instead of one per 32)
    r->flips_per_sweep = (double)cfg->n_real * cfg->n_copies * N * cfg->n_temps;
    r->words = (uint64_t)std::ceil(r->flips_per_sweep / 3.0);
    r->units = (uint64_t)cfg->n_real * cfg->n_copies * W;
    r->bytes = ea::tp_device_bytes(cfg) + (r->spins_out ? nsp * 4 : 0) + (r->energies_out ? nen * 4 : 0);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return EA_ESTATE;
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->open.insert(r->ticket);
        s->submitted += 1;
        if (s->first_submit_s < 0) s->first_submit_s = ms_between(s->t0, r->t_submit) * 1e-3;
        s->queue.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return EA_OK;
}

int ea_poll(ea_server *s, uint64_t ticket, uint32_t timeout_us)
{
    if (!s) return EA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->finished.count(ticket) != 0; };
    if (!ready()) {
        if (!s->open.count(ticket)) return EA_EINVAL;     // unknown or already collected
        if (timeout_us) s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
        if (!ready()) return EA_PENDING;
    }
    const int st = s->finished[ticket];
    s->finished.erase(ticket);
    return st;
}

int ea_server_stats_get(ea_server *s, ea_server_stats *out)
{
    if (!s || !out) return EA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = s->queue.size();
    out->live = s->n_live;
    out->rounds = s->rounds;
    out->flip_attempts = s->flips;
    out->busy_s = s->busy_s;
    out->span_s = s->first_submit_s >= 0 ? s->last_done_s - s->first_submit_s : 0.0;
    out->mem_budget = s->budget;
    out->peak_bytes = s->peak;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto rank = [&](double q) {
            size_t k = (size_t)std::ceil(q * (double)v.size());
            return v[k > 0 ? k - 1 : 0];
        };
        double sum = 0.0;
        for (double x : v) sum += x;
        out->p50_ms = rank(0.50);
        out->p99_ms = rank(0.99);
        out->mean_ms = sum / (double)v.size();
        out->max_ms = v.back();
    }
    return EA_OK;
}

void ea_server_destroy(ea_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    release_server(s);
}

}  // extern "C"
