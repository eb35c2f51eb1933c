// Device side of the persistent batch executor (the host side is in
// ea_batch.cu): task records, the interval arithmetic shared with the host,
// and the kernel template k_batch<MAXT>, instantiated for 384 and 512
// threads in ea_batch_k384.cu and ea_batch_k512.cu.
#pragma once
#include <cuda/atomic>

#include "ea_bodies.cuh"
#include "ea_fast.cuh"
#include "ea_wave.cuh"

namespace ea {

constexpr int kBatchMaxThreads = 512;
constexpr uint32_t kSpinLimit = 1u << 26;   // default wait: ~ tens of seconds of 256 ns naps

enum BatchForm { kBUnit = 0, kBFast = 1, kBChunk = 2, kBWave = 3 };

struct BatchInst {
    SweepLaunch a;          // s0, n_sweeps, P0, swap_every of this call
    int32_t L, form, p1, p2;    // p1: threads per lattice (unit, chunk), HP (fast), 16 (wave);
                                // p2: units per task (unit) or lattices per chunk (chunked)
    int32_t swap_smem, j_smem;
    int32_t field_kind;     // field members of the field kernel, wave form: 34 or 43 (else 0)
    uint32_t units;         // G * C; a unit task starts at unit `task.unit`
    uint32_t pieces;        // unit forms: sweep segments; chunked: swap intervals
    uint32_t seg;           // unit forms: sweeps per segment
    uint32_t nchunks;       // chunked: CTAs per unit and interval
    uint32_t join_base;     // chunked: join counter of unit 0
};

struct __align__(16) BatchTask {
    uint32_t inst, unit, piece, chunk;
};

struct BatchCtl {
    uint32_t head;          // next task index to take
    uint32_t tail;          // next free task index
    int32_t err;            // a wait ran out
    uint32_t pad;
};

// Per-call header, uploaded with the instance table (a captured graph replays
// the upload, so these change from call to call without re-capture).
struct BatchHdr {
    uint32_t total;         // tasks of the whole call
    uint32_t epoch;         // ready[i] == epoch: task i is published
    uint32_t ninit;         // initial tasks, already in tasks[0 .. ninit)
    uint32_t ninst;
    uint32_t spin_limit;    // naps a CTA waits for a task before raising the error flag
    uint32_t pad[3];
};

__host__ __device__ inline uint64_t swaps_between(uint64_t a, uint64_t b, uint32_t k)
{
    return k ? (b / k - a / k) : 0;    // sweeps s in [a, b) with (s + 1) % k == 0
}

// Sweep range [*s, *s + *len) of swap interval i of a call starting at sweep
// s_begin with n sweeps: intervals end right after each swap sweep.
__host__ __device__ inline void interval_of(uint64_t s_begin, uint32_t n, uint32_t k, uint32_t i,
                                            uint64_t *s, uint32_t *len)
{
    const uint64_t end = s_begin + n;
    if (k == 0) {
        *s = s_begin;
        *len = n;
        return;
    }
    const uint64_t e0 = (s_begin / k + 1) * k;          // exclusive end of interval 0
    uint64_t st = i == 0 ? s_begin : e0 + (uint64_t)(i - 1) * k;
    uint64_t en = i == 0 ? e0 : st + k;
    if (en > end) en = end;
    *s = st;
    *len = (uint32_t)(en - st);
}

__host__ __device__ inline uint32_t intervals_of(uint64_t s_begin, uint32_t n, uint32_t k)
{
    if (k == 0) return 1;
    const uint64_t end = s_begin + n;
    const uint64_t sw = swaps_between(s_begin, end, k);
    return (uint32_t)(sw + ((end % k) != 0 ? 1 : 0));
}

namespace {

template <bool FIELD>
__device__ __forceinline__ void run_unit(int L, uint32_t *base, const SweepLaunch &a, uint32_t unit,
                                         int tpl, int swap_smem, int m)
{
    switch (L) {
#define EA_U(X) case X: unit_body<X, false, FIELD>(base, a, unit, tpl, 0, swap_smem, m); break;
        EA_U(4) EA_U(6) EA_U(8) EA_U(10) EA_U(12) EA_U(14) EA_U(16) EA_U(20) EA_U(24) EA_U(32)
#undef EA_U
    default: break;
    }
}

__device__ __forceinline__ void run_fast(int L, int HP, uint32_t *base, const SweepLaunch &a,
                                         uint32_t unit, int swap_smem)
{
    if (L == 8 && HP == 4) unit_fast_body<8, 4, false>(base, a, unit, 0, swap_smem, 0, 0);
    else if (L == 8 && HP == 8) unit_fast_body<8, 8, false>(base, a, unit, 0, swap_smem, 0, 0);
    else if (L == 16 && HP == 32) unit_fast_body<16, 32, false>(base, a, unit, 0, swap_smem, 0, 0);
    else if (L == 16 && HP == 64) unit_fast_body<16, 64, false>(base, a, unit, 0, swap_smem, 0, 0);
}

template <bool FIELD>
__device__ __forceinline__ void run_chunk(int L, int j_smem, uint32_t *base, const SweepLaunch &a,
                                          uint32_t unit, int chunk, int tpl, int nlat)
{
    switch (L) {
#define EA_C(X)                                                                          \
    case X:                                                                              \
        if (j_smem) chunk_body<X, true, false, FIELD>(base, a, unit, chunk, tpl, nlat);  \
        else chunk_body<X, false, false, FIELD>(base, a, unit, chunk, tpl, nlat);        \
        break;
        EA_C(4) EA_C(6) EA_C(8) EA_C(10) EA_C(12) EA_C(14) EA_C(16) EA_C(20) EA_C(24) EA_C(32)
#undef EA_C
    default: break;
    }
}

__device__ __forceinline__ void publish(BatchTask *tasks, uint32_t *ready, BatchCtl *ctl,
                                        uint32_t epoch, const BatchTask &t0, uint32_t count)
{
    // thread 0 only: reserve `count` slots, write the tasks, then release their flags
    const uint32_t idx = atomicAdd(&ctl->tail, count);
    for (uint32_t j = 0; j < count; ++j) {
        BatchTask t = t0;
        t.chunk = j;
        tasks[idx + j] = t;
    }
    __threadfence();
    for (uint32_t j = 0; j < count; ++j) {
        cuda::atomic_ref<uint32_t, cuda::thread_scope_device> r(ready[idx + j]);
        r.store(epoch, cuda::memory_order_release);
    }
}

// FIELD = true: the kernel for batches of ensembles in an external field (its
// members run the field bodies: the generic unit and chunk forms, the
// wavefront form for the fields it takes).
template <int MAXT, bool FIELD = false>
__global__ void __launch_bounds__(MAXT, 1)
k_batch(const BatchHdr *hdr, const BatchInst *__restrict__ insts, BatchTask *tasks, uint32_t *ready,
        uint32_t *join, BatchCtl *ctl)
{
    extern __shared__ uint4 smem_u4[];
    const uint32_t total = hdr->total, epoch = hdr->epoch, spin_limit = hdr->spin_limit;
    uint32_t *base = reinterpret_cast<uint32_t *>(smem_u4);
    __shared__ SweepLaunch s_a;
    __shared__ BatchTask s_t;
    __shared__ int s_state;      // 0 run, 1 stop
    __shared__ int s_last;       // chunk piece: this CTA closes the interval
    for (;;) {
        if (threadIdx.x == 0) {
            int state = 0;
            const uint32_t idx = atomicAdd(&ctl->head, 1u);
            if (idx >= total) {
                state = 1;
            } else {
                cuda::atomic_ref<uint32_t, cuda::thread_scope_device> r(ready[idx]);
                cuda::atomic_ref<int32_t, cuda::thread_scope_device> er(ctl->err);
                uint32_t n = 0;
                while (r.load(cuda::memory_order_acquire) != epoch) {
                    if (++n > spin_limit || er.load(cuda::memory_order_relaxed) != 0) {
                        er.store(1, cuda::memory_order_relaxed);
                        state = 1;
                        break;
                    }
                    __nanosleep(256);
                }
                if (state == 0) {
                    const uint4 tv = __ldcg(reinterpret_cast<const uint4 *>(tasks + idx));
                    s_t.inst = tv.x;
                    s_t.unit = tv.y;
                    s_t.piece = tv.z;
                    s_t.chunk = tv.w;
                    const BatchInst &I = insts[s_t.inst];
                    s_a = I.a;
                    const uint32_t k = I.a.swap_every;
                    if (I.form == kBChunk) {
                        uint64_t s;
                        uint32_t len;
                        interval_of(I.a.s0, I.a.n_sweeps, k, s_t.piece, &s, &len);
                        s_a.s0 = s;
                        s_a.n_sweeps = len;
                        s_a.compute_energy_last = 1;
                    } else {
                        const uint64_t s = I.a.s0 + (uint64_t)s_t.piece * I.seg;
                        const uint64_t end = I.a.s0 + I.a.n_sweeps;
                        s_a.s0 = s;
                        s_a.n_sweeps = (uint32_t)((end - s) < I.seg ? (end - s) : I.seg);
                        s_a.P0 = I.a.P0 + swaps_between(I.a.s0, s, k);
                    }
                    s_a.energy_log = nullptr;
                    s_a.swap_log = nullptr;
                    s_a.qhist = nullptr;
                    s_a.esum = nullptr;
                    s_a.measure_every = 0;
                }
            }
            s_state = state;
            s_last = 0;
        }
        __syncthreads();
        if (s_state) break;
        const BatchTask t = s_t;
        const BatchInst &I = insts[t.inst];
        if (I.form == kBUnit)
            run_unit<FIELD>(I.L, base, s_a, t.unit, I.p1, I.swap_smem,
                            (int)min((uint32_t)I.p2, I.units - t.unit));
        else if (I.form == kBChunk) run_chunk<FIELD>(I.L, I.j_smem, base, s_a, t.unit, (int)t.chunk, I.p1, I.p2);
        else if constexpr (FIELD) {
            if (I.form == kBWave && I.field_kind == 34) unit_wave_body<false, 34>(base, s_a, t.unit, I.swap_smem);
            else if (I.form == kBWave && I.field_kind == 43) unit_wave_body<false, 43>(base, s_a, t.unit, I.swap_smem);
        } else {
            if (I.form == kBFast) run_fast(I.L, I.p1, base, s_a, t.unit, I.swap_smem);
            else if (I.form == kBWave) unit_wave_body<false>(base, s_a, t.unit, I.swap_smem);
        }
        __syncthreads();
        if (I.form == kBWave) {
            wave_release(base, (int)I.a.NT, FIELD);
            __syncthreads();
        }
        if (I.form != kBChunk) {
            if (threadIdx.x == 0 && t.piece + 1 < I.pieces) {
                __threadfence();
                BatchTask nt = t;
                nt.piece = t.piece + 1;
                publish(tasks, ready, ctl, epoch, nt, 1);
            }
        } else {
            if (threadIdx.x == 0) {
                __threadfence();   // this chunk's spins and energies before the count
                cuda::atomic_ref<uint32_t, cuda::thread_scope_device> j(join[I.join_base + t.unit]);
                const uint32_t done = j.fetch_add(1u, cuda::memory_order_acq_rel) + 1u;
                if (done == I.nchunks) {
                    j.store(0u, cuda::memory_order_relaxed);
                    s_last = 1;
                }
            }
            __syncthreads();
            if (s_last) {
                const uint32_t k = I.a.swap_every;
                const uint64_t e = s_a.s0 + s_a.n_sweeps;      // exclusive end of the interval
                if (k != 0 && e % k == 0)
                    swap_unit_body(base, s_a, t.unit, I.a.P0 + t.piece, I.L * I.L * I.L);
                if (threadIdx.x == 0 && t.piece + 1 < I.pieces) {
                    __threadfence();
                    BatchTask nt = t;
                    nt.piece = t.piece + 1;
                    publish(tasks, ready, ctl, epoch, nt, I.nchunks);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

// Kernel entry points of one instantiation (defined in ea_batch_k*.cu).
const void *batch_kernel_384();
const void *batch_kernel_512();
const void *batch_kernel_field_384();

}  // namespace ea
