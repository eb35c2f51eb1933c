// Sweep bodies shared by the standalone kernels and the persistent batch
// kernel: each runs one task on the calling CTA, given the CTA's shared
// memory.  Loads of mutable state (spins, energies) bypass L1 (ld.global.cg):
// in the persistent kernel another SM may have written them since this SM
// last read them.
#pragma once

#include "ea_device.cuh"

namespace ea {
namespace {

// ------------------------------------------------------------------ unit kernel
// One CTA owns all NT lattices of one (group, copy) unit in shared memory and
// runs the whole sweep range: Metropolis half-sweeps, per-lane energies,
// replica-exchange passes and measurements.  With C = 2 and overlap
// measurement the two copies of a group form a 2-CTA cluster and read each
// other's lattices through distributed shared memory.
//
// The persistent batch kernel may give one CTA m > 1 consecutive units of an
// ensemble (m * NT <= 64), run in lockstep: slot l of the CTA is slot l % NT
// of unit unit0 + l / NT.  Measurements and the cluster form need m = 1.

// MEAS = false compiles the body without the measurement, cluster and log
// paths (launches that use none of them; cluster_measure must then be 0).
// FIELD = true runs the method in an external field (ea_device.cuh): field
// flips, magnetisations counted with the energies, decisions on Et; it needs
// kMaxTemps x 32 more words of shared memory (after the masks).
template <int L, bool MEAS = true, bool FIELD = false>
__device__ __forceinline__ void unit_body(uint32_t *base, const SweepLaunch &a, uint32_t unit0, int tpl,
                                          int cluster_measure_arg, int swap_in_smem, int m = 1)
{
    const int cluster_measure = MEAS ? cluster_measure_arg : 0;
    int32_t *const energy_log = MEAS ? a.energy_log : nullptr;
    uint32_t *const swap_log = MEAS ? a.swap_log : nullptr;
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    const int NT = (int)a.NT;
    const int MT = m * NT;                                    // slots of the CTA
    uint32_t *S = base;                                       // [m][NT][2][H]
    uint32_t *Js = S + (size_t)MT * N;                        // [m][3][2][H]
    int *E = reinterpret_cast<int *>(Js + (size_t)m * 3 * N); // [64][32] energies by slot
    int *bnd = E + kMaxTemps * kLanes;                        // [64][32] swap accept bounds
    int *nd = bnd + kMaxTemps * kLanes;                       // [64][32] overlap counts
    uint32_t *msk = reinterpret_cast<uint32_t *>(nd + kMaxTemps * kLanes);  // [64]
    int *Mv = reinterpret_cast<int *>(msk + kMaxTemps);       // [64][32] magnetisations (FIELD)
    uint32_t *Tsw = msk + kMaxTemps + (FIELD ? kMaxTemps * kLanes : 0);  // [NT-1][swap_len]

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const bool act = tid < tpl * MT;                    // threads beyond the units' groups idle
    const int lf = act ? tid / tpl : 0, tl = tid - (tid / tpl) * tpl;   // my CTA slot and rank
    const int ui = lf / NT, l = lf - ui * NT;            // my unit (within the CTA) and slot
    const uint32_t unit = unit0 + (uint32_t)ui;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const uint32_t gr = g + a.g_base;                   // group index of the random numbers
    const int qper = (Gm::Q + tpl - 1) / tpl;

    uint32_t *gS = a.spins + (size_t)unit0 * NT * N;
    for (int w = tid; w < MT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
    for (int w = tid; w < m * 3 * N / 4; w += nthr) {
        const int i = w / (3 * N / 4), r = w - i * (3 * N / 4);
        const uint32_t gi = (unit0 + (uint32_t)i) / a.C;
        reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(a.bonds + (size_t)gi * 3 * N)[r];
    }
    const uint32_t *swt = a.swapt;
    if (swap_in_smem) {
        const int nsw = (NT - 1) * (int)a.swap_len;
        for (int w = tid; w < nsw; w += nthr) Tsw[w] = a.swapt[w];
        swt = Tsw;
    }
    uint32_t t0 = 0, t1 = 0, t2 = 0;
    uint64_t T[14];
    if constexpr (FIELD) {
#pragma unroll
        for (int k = 0; k < 14; ++k) T[k] = 0ull - a.metro_f[(size_t)l * 14 + k];   // 2^64 - T
    } else {
        t0 = a.metro[l * 3 + 0];
        t1 = a.metro[l * 3 + 1];
        t2 = a.metro[l * 3 + 2];
    }
    uint32_t *mine = S + (size_t)lf * N;
    const uint32_t *myJ = Js + (size_t)ui * 3 * N;
    __syncthreads();

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    SwapCountdown swap_cd(a.s0, a.swap_every);
    MeasureCountdown meas_cd(a.s0, a.measure_from, MEAS ? a.measure_every : 0u);
    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_s = swap_cd.step();             // a pass follows sweep s
        const bool swap_now = swap_s && NT > 1;
        const bool meas = MEAS && meas_cd.step();
        const bool needE = swap_now || energy_log != nullptr || meas || (n + 1 == a.n_sweeps);
        uint32_t acc[kPlanes], accM[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = accM[p] = 0;
        if (needE)   // counters add 2 per unsatisfied bond: E = 2U - 3N
            for (int i = tid; i < MT * kLanes; i += nthr) E[i] = -3 * N;
        if (FIELD && needE)   // and 2 per up spin: M = 2 up - N
            for (int i = tid; i < MT * kLanes; i += nthr) Mv[i] = -N;
        if (swap_now) {
            // Swap acceptance bounds depend only on the pass index: compute them
            // now; they are read after the half-sweeps' barriers.  Row
            // i * (NT - 1) + p: pair p of unit i.
            for (int i = tid; i < m * (NT - 1) * kLanes; i += nthr) {
                const int row = i >> 5, b = i & 31;
                const int ub = row / (NT - 1), p = row - ub * (NT - 1);
                const uint32_t un = unit0 + (uint32_t)ub;
                const uint32_t r = swap_uniform(a.rk, p, b, P, un / a.C + a.g_base, (int)(un % a.C));
                const int b4 = accept_bound(swt + (size_t)p * a.swap_len, a.swap_len, r);
                bnd[i] = FIELD ? (b4 / 4) * a.step : b4;      // -K x the step of Et
            }
        }
        const uint32_t tag0 = (0u << 16) | ((uint32_t)c << 8) | (uint32_t)l;
        const uint32_t tag1 = (1u << 16) | ((uint32_t)c << 8) | (uint32_t)l;
        if constexpr (FIELD) {
            if (act) {
                if (needE)
                    half_sweep_field<L, false, true>(mine, myJ, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk, T,
                                                     acc, accM);
                else
                    half_sweep_field<L, false, false>(mine, myJ, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk,
                                                      T, acc, accM);
            }
            __syncthreads();
            if (needE) {
                if (act)
                    half_sweep_field<L, true, true>(mine, myJ, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, T,
                                                    acc, accM);
                reduce_counters(acc, tpl, E, lane, warp, 2, MT);
                reduce_counters(accM, tpl, Mv, lane, warp, 2, MT);
            } else if (act) {
                half_sweep_field<L, false, false>(mine, myJ, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, T,
                                                  acc, accM);
            }
        } else {
            if (act)
                half_sweep<L, false>(mine, myJ, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk, t0, t1, t2, acc);
            __syncthreads();
            if (needE) {
                if (act)
                    half_sweep<L, true>(mine, myJ, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
                reduce_counters(acc, tpl, E, lane, warp, 2, MT);
            } else if (act) {
                half_sweep<L, false>(mine, myJ, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
            }
        }
        __syncthreads();
        if (swap_now) {
            for (int uw = warp; uw < m; uw += nthr / 32) {
                // Sequential pairs (0,1), (1,2), ... of unit `uw` per realization
                // lane; the configuration carried upward is `cur`.  Loads run one
                // pair ahead.
                int *Eu = E + uw * NT * kLanes;
                const int *bu = bnd + uw * (NT - 1) * kLanes;
                uint32_t *mu = msk + uw * (NT - 1);
                if constexpr (FIELD) {
                    // decisions on Et = h_den E - h_num M; E and M travel together
                    int *Mu = Mv + uw * NT * kLanes;
                    int ce = Eu[lane], cm = Mu[lane];
                    for (int p = 0; p + 1 < NT; ++p) {
                        const int ne = Eu[(p + 1) * kLanes + lane], nm = Mu[(p + 1) * kLanes + lane];
                        const int xc = a.h_den * ce - a.h_num * cm, xn = a.h_den * ne - a.h_num * nm;
                        const bool ok = (xc - xn) >= bu[p * kLanes + lane];
                        const uint32_t msk_p = __ballot_sync(kFull, ok);
                        Eu[p * kLanes + lane] = ok ? ne : ce;
                        Mu[p * kLanes + lane] = ok ? nm : cm;
                        ce = ok ? ce : ne;
                        cm = ok ? cm : nm;
                        if (lane == 0) mu[p] = msk_p;
                    }
                    Eu[(NT - 1) * kLanes + lane] = ce;
                    Mu[(NT - 1) * kLanes + lane] = cm;
                    continue;
                }
                int cur = Eu[lane];
                int nxt = Eu[kLanes + lane];
                int bb = bu[lane];
                for (int p = 0; p + 1 < NT; ++p) {
                    const int nxt2 = (p + 2 < NT) ? Eu[(p + 2) * kLanes + lane] : 0;
                    const int bb2 = (p + 2 < NT) ? bu[(p + 1) * kLanes + lane] : 0;
                    const bool ok = (cur - nxt) >= bb;
                    const uint32_t msk_p = __ballot_sync(kFull, ok);
                    Eu[p * kLanes + lane] = ok ? nxt : cur;
                    cur = ok ? cur : nxt;
                    if (lane == 0) mu[p] = msk_p;
                    nxt = nxt2;
                    bb = bb2;
                }
                Eu[(NT - 1) * kLanes + lane] = cur;
            }
            __syncthreads();
            // Masked exchange chain, pairs in order (0,1), (1,2), ..., two words a thread
            for (int wf = tid; wf < m * (N / 2); wf += nthr) {
                const int ub = wf / (N / 2), w = wf - ub * (N / 2);
                uint32_t *Su = S + (size_t)ub * NT * N;
                const uint32_t *mu = msk + ub * (NT - 1);
                uint2 x = reinterpret_cast<const uint2 *>(Su)[w];
                for (int p = 0; p + 1 < NT; ++p) {
                    const uint2 y = reinterpret_cast<const uint2 *>(Su + (size_t)(p + 1) * N)[w];
                    const uint32_t mp = mu[p];
                    const uint32_t dx = (x.x ^ y.x) & mp, dy = (x.y ^ y.y) & mp;
                    reinterpret_cast<uint2 *>(Su + (size_t)p * N)[w] = make_uint2(x.x ^ dx, x.y ^ dy);
                    x = make_uint2(y.x ^ dx, y.y ^ dy);
                }
                reinterpret_cast<uint2 *>(Su + (size_t)(NT - 1) * N)[w] = x;
            }
            if (swap_log != nullptr)
                for (int i = tid; i < m * (NT - 1); i += nthr) {
                    const int ub = i / (NT - 1), p = i - ub * (NT - 1);
                    const uint32_t un = unit0 + (uint32_t)ub;
                    swap_log[(((size_t)pass_local * a.G + un / a.C) * a.C + un % a.C) * (NT - 1) + p] =
                        msk[i];
                }
            __syncthreads();
        }
        if (swap_s) {
            ++P;
            ++pass_local;
        }
        if (energy_log != nullptr) {
            const size_t row = (size_t)(s - a.log_s0);
            for (int i = tid; i < MT * kLanes; i += nthr) {
                const int lf2 = i >> 5, b = i & 31;
                const int ub = lf2 / NT, t = lf2 - ub * NT;
                const uint32_t un = unit0 + (uint32_t)ub;
                energy_log[(((row * a.G + un / a.C) * NT + t) * a.C + un % a.C) * kLanes + b] = E[i];
            }
        }
        if (meas) {
            if (a.esum != nullptr) {
                // one warp per slot
                for (int t = warp; t < NT; t += nthr / 32) {
                    long long v = E[t * kLanes + lane];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0)
                        atomicAdd(reinterpret_cast<unsigned long long *>(a.esum + t),
                                  (unsigned long long)v);
                }
            }
            if (cluster_measure) {
                cg::cluster_group cl = cg::this_cluster();
                for (int i = tid; i < NT * kLanes; i += nthr) nd[i] = 0;
                cl.sync();   // both copies have finished sweep s and its swap pass
                const uint32_t *other = cl.map_shared_rank(S, c ^ 1);
                uint32_t oacc[kPlanes];
#pragma unroll
                for (int p = 0; p < kPlanes; ++p) oacc[p] = 0;
                if (act && (l & 1) == c) {
                    const uint4 *A4 = reinterpret_cast<const uint4 *>(S + (size_t)l * N);
                    const uint4 *B4 = reinterpret_cast<const uint4 *>(other + (size_t)l * N);
                    for (int w = tl; w < N / 4; w += tpl) {
                        const uint4 x = A4[w], y = B4[w];
                        acc_add_words4(oacc, x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w);
                    }
                }
                reduce_counters(oacc, tpl, nd, lane, warp, 1, NT);
                cl.sync();   // the other copy may now modify its lattices again
                if (a.qhist != nullptr)
                    for (int i = tid; i < NT * kLanes; i += nthr) {
                        const int t = i >> 5;
                        if ((t & 1) == c)
                            atomicAdd(reinterpret_cast<unsigned long long *>(
                                          a.qhist + (size_t)t * (N + 1) + nd[i]), 1ull);
                    }
            }
            __syncthreads();   // E and nd are rewritten by the next sweep
        }
    }
    // energies of the final state, spins back to global memory
    for (int i = tid; i < MT * kLanes; i += nthr) a.energy[(size_t)unit0 * NT * kLanes + i] = E[i];
    if constexpr (FIELD)
        for (int i = tid; i < MT * kLanes; i += nthr) a.mag[(size_t)unit0 * NT * kLanes + i] = Mv[i];
    for (int w = tid; w < MT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

// ------------------------------------------------------------------ chunked kernel
// For ensembles whose NT lattices do not fit one CTA: each CTA stages
// lattices [t0, t0 + nlat) of one unit, runs the sweeps up to the next swap
// point, and writes them back; the swap pass runs as its own kernels.

// LOG = false compiles the body without the energy-log path (energy_log must
// then be null).  FIELD = true: field flips (ea_device.cuh), and the
// magnetisations after the last sweep go to a.mag with the energies; needs
// kMaxTemps x 32 more words of shared memory after the energies.
template <int L, bool J_SMEM, bool LOG = true, bool FIELD = false>
__device__ __forceinline__ void chunk_body(uint32_t *base, const SweepLaunch &a, uint32_t unit,
                                           int chunk, int tpl, int nlat)
{
    int32_t *const energy_log = LOG ? a.energy_log : nullptr;
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    uint32_t *S = base;                                                   // [nlat][2][H]
    uint32_t *Js = S + (size_t)nlat * N;                                 // [3][2][H] if J_SMEM
    int *E = reinterpret_cast<int *>(Js + (J_SMEM ? 3 * N : 0));         // [64][32]
    int *Mv = E + kMaxTemps * kLanes;                                    // [64][32] if FIELD

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const uint32_t gr = g + a.g_base;                   // group index of the random numbers
    const int tbase = chunk * nlat;
    const int NT = (int)a.NT;
    const int l = tid / tpl, tl = tid - l * tpl;
    const int slot = tbase + l;
    const int nl_here = min(nlat, NT - tbase);
    const bool active = l < nl_here;
    const int qper = (Gm::Q + tpl - 1) / tpl;

    uint32_t *gS = a.spins + ((size_t)unit * NT + tbase) * N;
    const uint32_t *gJ = a.bonds + (size_t)g * 3 * N;
    for (int w = tid; w < nl_here * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
    const uint32_t *J = gJ;
    if constexpr (J_SMEM) {
        for (int w = tid; w < 3 * N / 4; w += nthr)
            reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
        J = Js;
    }
    uint32_t t0 = 0, t1 = 0, t2 = 0;
    uint64_t T[14];
    if constexpr (FIELD) {
#pragma unroll
        for (int k = 0; k < 14; ++k) T[k] = active ? 0ull - a.metro_f[(size_t)slot * 14 + k] : 0;   // 2^64 - T
    } else if (active) {
        t0 = a.metro[slot * 3]; t1 = a.metro[slot * 3 + 1]; t2 = a.metro[slot * 3 + 2];
    }
    uint32_t *mine = S + (size_t)l * N;
    __syncthreads();

    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool last = n + 1 == a.n_sweeps;
        const bool needE = energy_log != nullptr || (last && a.compute_energy_last);
        uint32_t acc[kPlanes], accM[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = accM[p] = 0;
        if (needE)
            for (int i = tid; i < kMaxTemps * kLanes; i += nthr) E[i] = -3 * N;
        const bool needM = FIELD && last && a.compute_energy_last;
        if (needM)
            for (int i = tid; i < kMaxTemps * kLanes; i += nthr) Mv[i] = -N;
        const uint32_t tag0 = (0u << 16) | ((uint32_t)c << 8) | (uint32_t)slot;
        const uint32_t tag1 = (1u << 16) | ((uint32_t)c << 8) | (uint32_t)slot;
        if (active) {
            if constexpr (FIELD) {
                if (needM)
                    half_sweep_field<L, false, true>(mine, J, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk, T,
                                                     acc, accM);
                else
                    half_sweep_field<L, false, false>(mine, J, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk, T,
                                                      acc, accM);
            } else {
                half_sweep<L, false>(mine, J, 0, tl, tpl, qper, (uint32_t)s, gr, tag0, a.rk, t0, t1, t2, acc);
            }
        }
        __syncthreads();
        if (needE) {
            if (active) {
                if constexpr (FIELD) {
                    if (needM)
                        half_sweep_field<L, true, true>(mine, J, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk,
                                                        T, acc, accM);
                    else
                        half_sweep_field<L, true, false>(mine, J, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk,
                                                         T, acc, accM);
                } else {
                    half_sweep<L, true>(mine, J, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
                }
            }
            reduce_counters(acc, tpl, E, lane, warp, 2, nlat);
            if (needM) reduce_counters(accM, tpl, Mv, lane, warp, 2, nlat);
            __syncthreads();
            for (int i = tid; i < nl_here * kLanes; i += nthr) {
                const int e = E[i];
                const int t = tbase + (i >> 5), b = i & 31;
                if (energy_log != nullptr) {
                    const size_t row = (size_t)(s - a.log_s0);
                    energy_log[(((row * a.G + g) * NT + t) * a.C + c) * kLanes + b] = e;
                }
                if (last) a.energy[((size_t)unit * NT + t) * kLanes + b] = e;
                if (needM) a.mag[((size_t)unit * NT + t) * kLanes + b] = Mv[i];
            }
        } else if (active) {
            if constexpr (FIELD)
                half_sweep_field<L, false, false>(mine, J, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, T, acc,
                                                  accM);
            else
                half_sweep<L, false>(mine, J, 1, tl, tpl, qper, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
        }
        __syncthreads();
    }
    for (int w = tid; w < nl_here * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

// One replica-exchange pass of one unit whose spins and energies are in
// global memory, run by one CTA (the persistent batch kernel's inline pass):
// acceptance bounds of every (pair, realization) by all threads, the decision
// chain by warp 0 on the unit's energies (permuted in place), then the masked
// exchange of all slots by all threads.  `base` needs 64 x 32 + 64 words.
__device__ __forceinline__ void swap_unit_body(uint32_t *base, const SweepLaunch &a, uint32_t unit,
                                               uint64_t P, int N)
{
    int *bnd = reinterpret_cast<int *>(base);                       // [64][32]
    uint32_t *msk = reinterpret_cast<uint32_t *>(bnd + kMaxTemps * kLanes);  // [64]
    const int NT = (int)a.NT;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (NT < 2) return;
    for (int i = tid; i < (NT - 1) * kLanes; i += nthr) {
        const int p = i >> 5, b = i & 31;
        bnd[i] = accept_bound(a.swapt + (size_t)p * a.swap_len, a.swap_len,
                              swap_uniform(a.rk, p, b, P, g + a.g_base, c));
    }
    __syncthreads();
    if (warp == 0 && a.h_num != 0) {
        // field: decisions on Et = h_den E - h_num M in steps of a.step; E and M travel together
        int32_t *E = a.energy + (size_t)unit * NT * kLanes;
        int32_t *M = a.mag + (size_t)unit * NT * kLanes;
        int ce = __ldcg(E + lane), cm = __ldcg(M + lane);
        for (int p = 0; p + 1 < NT; ++p) {
            const int ne = __ldcg(E + (p + 1) * kLanes + lane), nm = __ldcg(M + (p + 1) * kLanes + lane);
            const int xc = a.h_den * ce - a.h_num * cm, xn = a.h_den * ne - a.h_num * nm;
            const bool ok = (xc - xn) >= (bnd[p * kLanes + lane] / 4) * a.step;
            const uint32_t m = __ballot_sync(kFull, ok);
            E[p * kLanes + lane] = ok ? ne : ce;
            M[p * kLanes + lane] = ok ? nm : cm;
            ce = ok ? ce : ne;
            cm = ok ? cm : nm;
            if (lane == 0) msk[p] = m;
        }
        E[(NT - 1) * kLanes + lane] = ce;
        M[(NT - 1) * kLanes + lane] = cm;
    } else if (warp == 0) {
        int32_t *E = a.energy + (size_t)unit * NT * kLanes;
        int cur = __ldcg(E + lane);
        for (int p = 0; p + 1 < NT; ++p) {
            const int nxt = __ldcg(E + (p + 1) * kLanes + lane);
            const bool ok = (cur - nxt) >= bnd[p * kLanes + lane];
            const uint32_t m = __ballot_sync(kFull, ok);
            E[p * kLanes + lane] = ok ? nxt : cur;
            cur = ok ? cur : nxt;
            if (lane == 0) msk[p] = m;
        }
        E[(NT - 1) * kLanes + lane] = cur;
    }
    __syncthreads();
    uint4 *S = reinterpret_cast<uint4 *>(a.spins + (size_t)unit * NT * N);
    const int W = N / 4;
    for (int w = tid; w < W; w += nthr) {
        uint4 x = __ldcg(S + w);
        for (int p = 0; p + 1 < NT; ++p) {
            const uint4 y = __ldcg(S + (size_t)(p + 1) * W + w);
            const uint32_t m = msk[p];
            const uint4 d = make_uint4((x.x ^ y.x) & m, (x.y ^ y.y) & m, (x.z ^ y.z) & m, (x.w ^ y.w) & m);
            S[(size_t)p * W + w] = make_uint4(x.x ^ d.x, x.y ^ d.y, x.z ^ d.z, x.w ^ d.w);
            x = make_uint4(y.x ^ d.x, y.y ^ d.y, y.z ^ d.z, y.w ^ d.w);
        }
        S[(size_t)(NT - 1) * W + w] = x;
    }
    __syncthreads();
}

}  // namespace
}  // namespace ea
