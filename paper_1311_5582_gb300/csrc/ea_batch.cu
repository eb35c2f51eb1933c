// Persistent batch executor: one launch advances several ensembles (contexts
// of any supported L, temperature ladder and size) by the same number of
// sweeps, each exactly as if it ran alone.
//
// Work is cut into tasks:
//  * unit piece: a whole (group, copy) unit resident in one CTA for a segment
//    of sweeps, swap passes in-kernel; its successor is the next segment;
//  * chunk piece: the slots [j*nlat, (j+1)*nlat) of a unit that does not fit
//    one CTA, for one swap interval; the last chunk of an interval to finish
//    runs the unit's swap pass (in global memory) and publishes the chunks of
//    the next interval.
// A device-side FIFO holds the tasks; each CTA takes the next index, waits
// until that task is published, runs it, and publishes its successors.  A
// task is published only by a task that was taken before it and that runs to
// completion without waiting, so the queue always progresses, whatever
// number of CTAs is resident; waits are bounded all the same and raise an
// error flag instead of hanging.  Initial tasks are ordered by the work left
// in their unit (longest first).  The upload, the queue reset and the launch
// are captured in a CUDA graph, replayed while the batch's shape is unchanged.

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ea.h"
#include "ea_batch_kernel.cuh"

namespace ea {
namespace {

// Publishes the initial tasks and resets the queue (one CTA).
__global__ void k_batch_init(const BatchHdr *hdr, uint32_t *ready, BatchCtl *ctl)
{
    const uint32_t epoch = hdr->epoch, ninit = hdr->ninit;
    for (uint32_t i = threadIdx.x; i < ninit; i += blockDim.x) ready[i] = epoch;
    if (threadIdx.x == 0) {
        ctl->head = 0;
        ctl->tail = ninit;
        ctl->err = 0;
    }
}

size_t plan_task_smem(const ea_ctx *c, const Plan &p)
{
    const int N = (int)c->N, NT = (int)c->NT;
    size_t b = 0;
    if (p.form == kFormUnitFast)
        b = fast_unit_smem((int)c->L, NT, c->swap_len, p.swap_in_smem, false, false);
    else if (p.form == kFormUnit)
        b = UnitSmem::base_bytes(N, NT) + (p.swap_in_smem ? UnitSmem::swap_bytes(NT, c->swap_len) : 0);
    else
        b = p.smem;
    const size_t swap_need = (size_t)(kMaxTemps * kLanes + kMaxTemps) * 4;
    return b > swap_need ? b : swap_need;
}

}  // namespace
}  // namespace ea

struct ea_batch {
    cudaStream_t stream;
    int device;
    std::vector<ea_ctx *> ctxs;
    std::vector<int> plan_override;        // per context: plan index or -1 (automatic)
    uint32_t seg_target;                   // site-words per unit piece (0: default)
    // device buffers: upload area (header + instance table), task queue, flags, joins
    unsigned char *d_up;
    ea::BatchTask *d_tasks;
    uint32_t *d_ready, *d_join;
    ea::BatchCtl *d_ctl;
    size_t cap_up, cap_tasks, cap_join;
    // pinned copies of the upload area and of the initial tasks
    unsigned char *h_up;
    ea::BatchTask *h_init;
    size_t cap_h_up, cap_h_init;
    uint32_t epoch;
    // captured graph of the last shape
    cudaGraphExec_t gexec;
    bool have_graph;
    size_t g_ninst, g_ninit, g_total;
    int g_grid, g_threads;
    size_t g_smem;
    cudaEvent_t done;
    bool pending;
    uint64_t launches;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaErrorMemoryAllocation ? EA_ENOMEM : EA_ECUDA; }

template <typename T>
cudaError_t grow_dev(T **p, size_t *cap, size_t need)
{
    if (*cap >= need) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = need < 64 ? 64 : need;
    n += n / 2;
    const cudaError_t e = cudaMalloc(p, n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

template <typename T>
cudaError_t grow_host(T **p, size_t *cap, size_t need)
{
    if (*cap >= need) return cudaSuccess;
    cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = need < 64 ? 64 : need;
    n += n / 2;
    const cudaError_t e = cudaMallocHost(p, n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

// Thread counts of the two batch kernels: 384 (up to 168 registers a
// thread, which the L % 8 == 0 unit kernel needs to run without spills) and 512.
constexpr int kBatchSmallThreads = 384;

// The plan a context runs under in a batch: an explicit choice if the batch
// kernel can host it (<= 512 threads); else its selected plan, or the first
// in its list, that fits 384 threads; else the first that fits 512.
const ea::Plan *batch_plan(const ea_ctx *c, int override_idx)
{
    if (override_idx >= 0 && override_idx < (int)c->plans.size() &&
        c->plans[(size_t)override_idx].threads <= ea::kBatchMaxThreads)
        return &c->plans[(size_t)override_idx];
    if (c->plan.threads <= kBatchSmallThreads) return &c->plan;
    for (const ea::Plan &p : c->plans)
        if (p.threads <= kBatchSmallThreads) return &p;
    if (c->plan.threads <= ea::kBatchMaxThreads) return &c->plan;
    for (const ea::Plan &p : c->plans)
        if (p.threads <= ea::kBatchMaxThreads) return &p;
    return nullptr;
}

}  // namespace

extern "C" {

int ea_batch_create(void *stream, ea_batch **out)
{
    if (!out) return EA_EINVAL;
    *out = nullptr;
    ea_batch *b = new (std::nothrow) ea_batch();
    if (!b) return EA_ENOMEM;
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(ea::BatchCtl));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaFree(b->d_ctl);
        delete b;
        return cuda_err(e);
    }
    *out = b;
    return EA_OK;
}

int ea_batch_add(ea_batch *b, ea_ctx *ctx)
{
    if (!b || !ctx) return EA_EINVAL;
    if (ctx->device != b->device) return EA_EINVAL;
    if (!batch_plan(ctx, -1)) return EA_EUNSUPPORTED;
    for (const ea_ctx *m : b->ctxs)
        if (m == ctx) return EA_EINVAL;      // a member runs once per call
    b->ctxs.push_back(ctx);
    b->plan_override.push_back(-1);
    b->have_graph = false;
    return EA_OK;
}

int ea_batch_clear(ea_batch *b)
{
    if (!b) return EA_EINVAL;
    b->ctxs.clear();
    b->plan_override.clear();
    b->have_graph = false;
    return EA_OK;
}

int ea_batch_set_plan(ea_batch *b, uint32_t member, int plan_index)
{
    if (!b || member >= b->ctxs.size()) return EA_EINVAL;
    const ea_ctx *c = b->ctxs[member];
    if (plan_index >= (int)c->plans.size()) return EA_EINVAL;
    if (plan_index >= 0 && c->plans[(size_t)plan_index].threads > ea::kBatchMaxThreads)
        return EA_EUNSUPPORTED;
    b->plan_override[member] = plan_index;
    b->have_graph = false;
    return EA_OK;
}

int ea_batch_set_segment(ea_batch *b, uint32_t site_words)
{
    if (!b) return EA_EINVAL;
    b->seg_target = site_words;
    b->have_graph = false;
    return EA_OK;
}

int ea_batch_sweep(ea_batch *b, uint32_t n_sweeps, uint32_t swap_every)
{
    using namespace ea;
    if (!b) return EA_EINVAL;
    if (n_sweeps == 0 || b->ctxs.empty()) return EA_OK;
    cudaError_t e = cudaSuccess;
    // the pinned upload buffers are rewritten below: the previous call must be done
    if (b->pending) {
        e = cudaEventSynchronize(b->done);
        if (e != cudaSuccess) return cuda_err(e);
        b->pending = false;
        BatchCtl ctl;
        e = cudaMemcpy(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(e);
        if (ctl.err) {
            b->have_graph = false;           // re-capture: join counters are zeroed again
            return EA_ETIMEOUT;
        }
    }
    const size_t ninst = b->ctxs.size();
    const size_t up_bytes = sizeof(BatchHdr) + ninst * sizeof(BatchInst);
    if ((e = grow_host(&b->h_up, &b->cap_h_up, up_bytes)) != cudaSuccess) return cuda_err(e);
    BatchHdr *hdr = reinterpret_cast<BatchHdr *>(b->h_up);
    BatchInst *insts = reinterpret_cast<BatchInst *>(b->h_up + sizeof(BatchHdr));
    std::vector<BatchTask> init;
    std::vector<uint64_t> work;      // work left in the task's unit (ordering key)
    uint64_t total = 0;
    uint32_t njoin = 0;
    size_t smem = 0;
    int maxt = 0;
    const uint32_t seg_target = b->seg_target ? b->seg_target : (1u << 21);
    std::vector<uint64_t> passes(ninst);
    for (size_t i = 0; i < ninst; ++i) {
        ea_ctx *c = b->ctxs[i];
        const Plan *p = batch_plan(c, b->plan_override[i]);
        if (!p) return EA_EUNSUPPORTED;
        BatchInst &I = insts[i];
        std::memset(&I, 0, sizeof(I));
        I.a.spins = c->d_spins;
        I.a.bonds = c->d_bonds;
        I.a.metro = c->d_metro;
        I.a.swapt = c->d_swapt;
        I.a.swap_len = c->swap_len;
        I.a.energy = c->d_energy;
        I.a.G = c->G;
        I.a.NT = c->NT;
        I.a.C = c->C;
        I.a.rk = c->rk;
        I.a.err = c->d_err;
        I.a.s0 = c->sweep;
        I.a.n_sweeps = n_sweeps;
        I.a.swap_every = swap_every;
        I.a.P0 = c->pass;
        I.L = (int32_t)c->L;
        I.units = c->G * c->C;
        I.swap_smem = p->swap_in_smem ? 1 : 0;
        I.j_smem = p->j_in_smem ? 1 : 0;
        passes[i] = swaps_between(c->sweep, c->sweep + n_sweeps, swap_every);
        const uint64_t unit_work = (uint64_t)n_sweeps * c->N * c->NT;
        if (p->form == kFormChunked) {
            I.form = kBChunk;
            I.p1 = p->threads_per_lattice;
            I.p2 = p->lattices_per_cta;
            I.nchunks = (c->NT + (uint32_t)p->lattices_per_cta - 1) / (uint32_t)p->lattices_per_cta;
            I.pieces = intervals_of(c->sweep, n_sweeps, swap_every);
            I.join_base = njoin;
            njoin += I.units;
            total += (uint64_t)I.units * I.pieces * I.nchunks;
            for (uint32_t u = 0; u < I.units; ++u)
                for (uint32_t j = 0; j < I.nchunks; ++j) {
                    init.push_back({(uint32_t)i, u, 0u, j});
                    work.push_back(unit_work);
                }
        } else {
            I.form = p->form == kFormUnitFast ? kBFast : kBUnit;
            I.p1 = p->threads_per_lattice;
            const uint64_t per_sweep = (uint64_t)c->N * c->NT;
            uint64_t seg = seg_target / (per_sweep ? per_sweep : 1);
            if (seg < 8) seg = 8;
            if (seg > n_sweeps) seg = n_sweeps;
            I.seg = (uint32_t)seg;
            I.pieces = (uint32_t)((n_sweeps + seg - 1) / seg);
            total += (uint64_t)I.units * I.pieces;
            for (uint32_t u = 0; u < I.units; ++u) {
                init.push_back({(uint32_t)i, u, 0u, 0u});
                work.push_back(unit_work);
            }
        }
        const size_t need = plan_task_smem(c, *p);
        if (need > smem) smem = need;
        if (p->threads > maxt) maxt = p->threads;
    }
    if (total > 0xFFFFFFF0ull) return EA_EINVAL;
    // longest unit first
    std::vector<size_t> order(init.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return work[x] > work[y]; });
    if ((e = grow_host(&b->h_init, &b->cap_h_init, init.size())) != cudaSuccess) return cuda_err(e);
    for (size_t i = 0; i < order.size(); ++i) b->h_init[i] = init[order[i]];
    b->epoch += 1;
    hdr->total = (uint32_t)total;
    hdr->epoch = b->epoch;
    hdr->ninit = (uint32_t)init.size();
    hdr->ninst = (uint32_t)ninst;

    const int threads = maxt <= kBatchSmallThreads ? kBatchSmallThreads : kBatchMaxThreads;
    const void *kern = threads == kBatchSmallThreads ? batch_kernel_384() : batch_kernel_512();
    const bool same_shape = b->have_graph && b->g_ninst == ninst && b->g_ninit == init.size() &&
                            b->g_total == total && b->g_smem == smem && b->g_threads == threads;
    if (!same_shape) {
        if (b->have_graph) {
            cudaGraphExecDestroy(b->gexec);
            b->have_graph = false;
        }
        if ((e = grow_dev(&b->d_up, &b->cap_up, up_bytes)) != cudaSuccess) return cuda_err(e);
        if (b->cap_tasks < (size_t)total) {
            if ((e = grow_dev(&b->d_tasks, &b->cap_tasks, (size_t)total)) != cudaSuccess) return cuda_err(e);
            // ready flags never equal a future epoch: zero them when (re)allocated
            cudaFree(b->d_ready);
            b->d_ready = nullptr;
            if ((e = cudaMalloc(&b->d_ready, b->cap_tasks * sizeof(uint32_t))) != cudaSuccess) return cuda_err(e);
            if ((e = cudaMemset(b->d_ready, 0, b->cap_tasks * sizeof(uint32_t))) != cudaSuccess) return cuda_err(e);
        }
        if (b->cap_join < (size_t)njoin || !b->d_join) {
            cudaFree(b->d_join);
            b->d_join = nullptr;
            b->cap_join = njoin ? njoin : 1;
            if ((e = cudaMalloc(&b->d_join, b->cap_join * sizeof(uint32_t))) != cudaSuccess) return cuda_err(e);
        }
        // joins are reset by the closing chunk of each interval; zero them once here
        if ((e = cudaMemset(b->d_join, 0, b->cap_join * sizeof(uint32_t))) != cudaSuccess) return cuda_err(e);
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_err(e);
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        if (e != cudaSuccess) return cuda_err(e);
        if (per_sm < 1) return EA_EUNSUPPORTED;
        b->g_grid = per_sm * sms;
        b->g_ninst = ninst;
        b->g_ninit = init.size();
        b->g_total = total;
        b->g_smem = smem;
        b->g_threads = threads;
        // capture: upload, publish the initial tasks, the persistent launch
        cudaStream_t cap = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_up, b->h_up, up_bytes, cudaMemcpyHostToDevice, cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_tasks, b->h_init, init.size() * sizeof(BatchTask),
                                cudaMemcpyHostToDevice, cap);
        const BatchHdr *d_hdr = reinterpret_cast<const BatchHdr *>(b->d_up);
        const BatchInst *d_insts = reinterpret_cast<const BatchInst *>(b->d_up + sizeof(BatchHdr));
        if (e == cudaSuccess) {
            k_batch_init<<<1, 1024, 0, cap>>>(d_hdr, b->d_ready, b->d_ctl);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(b->g_grid);
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = cap;
            void *args[] = {(void *)&d_hdr, (void *)&d_insts, (void *)&b->d_tasks, (void *)&b->d_ready,
                            (void *)&b->d_join, (void *)&b->d_ctl};
            e = cudaLaunchKernelExC(&cfg, kern, args);
        }
        const cudaError_t e2 = cap ? cudaStreamEndCapture(cap, &graph) : cudaSuccess;
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_err(e);
        b->have_graph = true;
    }
    e = cudaGraphLaunch(b->gexec, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
    if (e != cudaSuccess) return cuda_err(e);
    b->pending = true;
    b->launches += 2;
    for (size_t i = 0; i < ninst; ++i) {
        b->ctxs[i]->sweep += n_sweeps;
        b->ctxs[i]->pass += passes[i];
        b->ctxs[i]->launches += 1;
    }
    return EA_OK;
}

int ea_batch_sync(ea_batch *b)
{
    if (!b) return EA_EINVAL;
    if (!b->pending) return EA_OK;
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return cuda_err(e);
    b->pending = false;
    ea::BatchCtl ctl;
    e = cudaMemcpy(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    if (ctl.err) {
        b->have_graph = false;
        return EA_ETIMEOUT;
    }
    return EA_OK;
}

uint64_t ea_batch_launch_count(const ea_batch *b) { return b ? b->launches : 0; }

void ea_batch_destroy(ea_batch *b)
{
    if (!b) return;
    if (b->pending) cudaEventSynchronize(b->done);
    if (b->have_graph) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->d_up);
    cudaFree(b->d_tasks);
    cudaFree(b->d_ready);
    cudaFree(b->d_join);
    cudaFree(b->d_ctl);
    cudaFreeHost(b->h_up);
    cudaFreeHost(b->h_init);
    cudaEventDestroy(b->done);
    delete b;
}

}  // extern "C"
