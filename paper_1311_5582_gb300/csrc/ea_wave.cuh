// Unit sweep body for L = 8 with the replica exchange run as a wavefront.
//
// Same method and results as the other unit kernels (one CTA per (group,
// copy) unit, all slots in shared memory for the whole call); what differs is
// how the exchange pass of Sec. 2.4 is scheduled.  The pass after sweep s is
// sequential in the pair index: pair p compares the energy `cur` of the
// configuration carried up from slot p (the product of pairs 0..p-1) with
// E_{p+1}, and an accepted pair moves the carried configuration on (the
// masked exchange chain of the swap pass).  Slot p's configuration for sweep
// s+1 is final as soon as pair p is decided and applied, and slots never
// interact during a sweep, so nothing needs the whole CTA to wait:
//  * warp k owns slots 2k (lanes 0-15) and 2k+1 (lanes 16-31) and sweeps them
//    on its own;
//  * after sweep s it reduces its two slots' energies (lane b = realization
//    b), publishes E_{2k} for warp k-1, takes the carried energy of pair 2k-1
//    from warp k-1, decides pair 2k and applies it to its own two slots,
//    then waits for E_{2k+2} of warp k+1, decides pair 2k+1 and applies it to
//    slots 2k+1 and 2k+2 (the latter then holds the carried configuration),
//    hands the carried energy to warp k+1 and starts sweep s+1 at once.
// The warps run staggered by about two pair steps each; the exchange, the
// decisions and the bound search of the next pass overlap the sweeps of the
// other warps instead of stopping the CTA.  Hand-offs are shared-memory
// mbarriers (the waiting warp is suspended, not spinning); every wait is
// bounded (on expiry the unit raises the context's error flag and stops).
// Each decision uses exactly the energies, bounds and order of the
// sequential pass, so the trajectory is that of every other kernel.
#pragma once

#include "ea_fast.cuh"

namespace ea {
namespace {

constexpr int kWaveWaitLimit = 1 << 22;    // suspending polls of one wait (seconds) before giving up

// Shared-memory layout of the wavefront kernel, in 32-bit words.
struct WaveLayout {
    size_t s, js, eo, cur, bar_e, bar_h, abort, tsw, words;
    __host__ __device__ WaveLayout(int N, int NT, uint32_t swap_len, bool swap_smem)
    {
        const int nw = (NT + 1) / 2;
        size_t o = 0;
        s = o; o += (size_t)NT * N;               // [NT][2][H] spins by slot
        js = o; o += (size_t)3 * N;               // [3][2][H] bonds
        eo = o; o += (size_t)NT * kLanes;         // energy of slot 2k after the sweep, for warp k-1
        cur = o; o += (size_t)nw * kLanes;        // carried energy from warp k to warp k+1
        o = (o + 1) & ~(size_t)1;                 // 8-byte alignment of the barriers
        bar_e = o; o += 2 * (size_t)nw;           // mbarrier k: E_{2k+2} of warp k+1 is published
        bar_h = o; o += 2 * (size_t)nw;           // mbarrier k: warp k applied its pass steps
        abort = o; o += 1;
        tsw = o; o += swap_smem && NT > 1 ? (size_t)(NT - 1) * swap_len : 0;
        words = o;
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Hand-offs between warps: a shared-memory mbarrier that completes one phase
// when the 32 lanes of the producer warp have arrived (arrive has release
// semantics for each lane's earlier writes, the consumer's wait acquire).
// A waiting warp is suspended by the hardware instead of spinning, so it
// takes no issue slots from the warps that are sweeping.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Invalidates the hand-off barriers of a finished unit (after a CTA barrier)
// before the shared memory is used for anything else.
__device__ __forceinline__ void wave_release(uint32_t *base, int NT)
{
    const WaveLayout lay(8 * 8 * 8, NT, 0, false);
    uint64_t *bar_e = reinterpret_cast<uint64_t *>(base + lay.bar_e);
    uint64_t *bar_h = reinterpret_cast<uint64_t *>(base + lay.bar_h);
    for (int i = threadIdx.x; i < (NT + 1) / 2; i += blockDim.x) {
        mbar_inval(&bar_e[i]);
        mbar_inval(&bar_h[i]);
    }
}

// Waits (whole warp) for the phase of `bar` with the given parity.  Returns
// false if the unit was aborted or the wait ran out; the latter raises the
// abort flag and the context's error flag.
__device__ __forceinline__ bool wave_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort, int *err)
{
    for (int it = 0; it < kWaveWaitLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort != 0u) return false;
    }
    *abort = 1u;
    atomicExch(err, 1);
    return false;
}

// (a & ~m) | (b & m): one LOP3.
__device__ __forceinline__ uint32_t mux(uint32_t a, uint32_t b, uint32_t m) { return (a & ~m) | (b & m); }

// One quad of the lane: quad J of (row parity J >> 1, row index base + 16 (J & 1)).
template <int COL, int J, bool WITH_E, int PL>
__device__ __forceinline__ void wave_quad(uint32_t *mine, const uint32_t *Js, const QuadRow &d, uint4 r,
                                          uint64_t t0, uint64_t t1, uint64_t t2, uint32_t (&acc)[PL])
{
    constexpr int PX = ((J >> 1) + COL) & 1;
    quad_fast<8, COL, PX, WITH_E, PL>(mine, Js, d, r, t0, t1, t2, acc);
}

// Half-sweep of colour COL over the lane's four quads; the uniforms of the
// next quad are drawn while the current one is updated.
template <int COL, bool WITH_E, int PL>
__device__ __forceinline__ void wave_half(uint32_t *mine, const uint32_t *Js, const QuadRow (&qd)[4],
                                          uint32_t s, uint32_t gr, uint32_t ctag, const RoundKeys &rk,
                                          uint64_t t0, uint64_t t1, uint64_t t2, uint32_t (&acc)[PL])
{
    uint4 r0 = philox((uint32_t)(qd[0].k0 >> 2), ctag, s, gr, rk);
    uint4 r1 = philox((uint32_t)(qd[1].k0 >> 2), ctag, s, gr, rk);
    wave_quad<COL, 0, WITH_E, PL>(mine, Js, qd[0], r0, t0, t1, t2, acc);
    r0 = philox((uint32_t)(qd[2].k0 >> 2), ctag, s, gr, rk);
    wave_quad<COL, 1, WITH_E, PL>(mine, Js, qd[1], r1, t0, t1, t2, acc);
    r1 = philox((uint32_t)(qd[3].k0 >> 2), ctag, s, gr, rk);
    wave_quad<COL, 2, WITH_E, PL>(mine, Js, qd[2], r0, t0, t1, t2, acc);
    wave_quad<COL, 3, WITH_E, PL>(mine, Js, qd[3], r1, t0, t1, t2, acc);
}

// Unsatisfied-bond totals of the warp's two slots: each half-warp sums its
// lanes' bit-sliced counters with a butterfly of shuffles and bit-sliced
// adders, lane t of each half then holds plane t, and one 32x32 bit transpose
// leaves in lane b the total of realization b of slot A (bits 0..15) and of
// slot B (bits 16..31).
template <int PL>
__device__ __forceinline__ void wave_reduce(const uint32_t (&acc)[PL], int lane, int &UA, int &UB)
{
    constexpr int PT = PL + 4;
    static_assert(PT <= 16, "counter too wide for a half-warp transpose");
    uint32_t v[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) v[p] = p < PL ? acc[p] : 0u;
#pragma unroll
    for (int lv = 0; lv < 4; ++lv) {
        uint32_t cy = 0;
#pragma unroll
        for (int p = 0; p < PL + lv + 1; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, v[p], 1 << lv);
            uint32_t s2, c2;
            full_add(v[p], o, cy, s2, c2);
            v[p] = s2;
            cy = c2;
        }
    }
    const int t = lane & 15;
    uint32_t x = 0;
#pragma unroll
    for (int p = 0; p < PT; ++p) x = (t == p) ? v[p] : x;
    const uint32_t y = warp_transpose(x, lane);
    UA = (int)(y & 0xFFFFu);
    UB = (int)(y >> 16);
}

// Acceptance bounds of the warp's pairs 2k and 2k+1 in pass P for the
// realization of this lane (Sec. 2.4 with the integer table of Sec. 4.3.2):
// pair p is accepted iff E_p - E_{p+1} >= bound.  Lanes 0-7 draw the Philox
// blocks of pair 2k (realizations 4q..4q+3 from lane q), lanes 8-15 those of
// pair 2k+1; each lane then searches both rows for its own uniforms.
__device__ __forceinline__ void wave_bounds(const uint32_t *swt, uint32_t len, uint32_t top, int k, int NT,
                                            int c, uint64_t P, uint32_t gr, const RoundKeys &rk,
                                            int lane, int &bA, int &bB)
{
    const int pq = (lane >> 3) & 1, bq = lane & 7;
    const int p = 2 * k + pq;
    const uint4 v = philox(((uint32_t)p << 3) | (uint32_t)bq, (1u << 24) | ((uint32_t)c << 8), (uint32_t)P,
                           gr, rk);
    const int src = lane >> 2, w = lane & 3;
    uint32_t ra, rb;
    {
        const uint32_t x = __shfl_sync(kFull, v.x, src), y = __shfl_sync(kFull, v.y, src);
        const uint32_t z = __shfl_sync(kFull, v.z, src), q = __shfl_sync(kFull, v.w, src);
        ra = w == 0 ? x : w == 1 ? y : w == 2 ? z : q;
    }
    {
        const uint32_t x = __shfl_sync(kFull, v.x, src + 8), y = __shfl_sync(kFull, v.y, src + 8);
        const uint32_t z = __shfl_sync(kFull, v.z, src + 8), q = __shfl_sync(kFull, v.w, src + 8);
        rb = w == 0 ? x : w == 1 ? y : w == 2 ? z : q;
    }
    const int pa = min(2 * k, NT - 2), pb = min(2 * k + 1, NT - 2);   // rows in range; unused otherwise
    const uint32_t *rowa = swt + (size_t)max(pa, 0) * len, *rowb = swt + (size_t)max(pb, 0) * len;
    uint32_t ka = 0, kb = 0;                  // invariant: row[0..k) > r
    for (uint32_t st = top; st != 0; st >>= 1) {
        const uint32_t na = ka + st, nb = kb + st;
        const uint32_t ea = na <= len ? rowa[na - 1] : 0u;
        const uint32_t eb = nb <= len ? rowb[nb - 1] : 0u;
        ka = ea > ra ? na : ka;
        kb = eb > rb ? nb : kb;
    }
    bA = -4 * (int)ka;
    bB = -4 * (int)kb;
}

// LOG = false compiles the body without the energy and swap logs (their
// pointers must then be null).  Launches that measure (qhist / esum) use
// another kernel.
template <bool LOG>
__device__ __forceinline__ void unit_wave_body(uint32_t *const base, const SweepLaunch &a, uint32_t unit,
                                               int swap_in_smem)
{
    constexpr int L = 8;
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    constexpr int PL = planes_for(24 * 4);          // counter planes of four quads (<= 96)
    int32_t *const energy_log = LOG ? a.energy_log : nullptr;
    uint32_t *const swap_log = LOG ? a.swap_log : nullptr;
    const int NT = (int)a.NT;
    const WaveLayout lay(N, NT, a.swap_len, swap_in_smem != 0);
    uint32_t *S = base + lay.s;
    uint32_t *Js = base + lay.js;
    int *Eo = reinterpret_cast<int *>(base + lay.eo);
    int *Cur = reinterpret_cast<int *>(base + lay.cur);
    uint64_t *bar_e = reinterpret_cast<uint64_t *>(base + lay.bar_e);
    uint64_t *bar_h = reinterpret_cast<uint64_t *>(base + lay.bar_h);
    volatile uint32_t *abort = base + lay.abort;

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, k = tid >> 5;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const uint32_t gr = g + a.g_base;                   // group index of the random numbers
    const int half = lane >> 4, li = lane & 15;
    const int slot = 2 * k + half;
    const bool act = slot < NT;                         // idle half of the last warp (odd NT)
    const int ls = act ? slot : 0;
    const bool hasB = 2 * k + 1 < NT, hasC = 2 * k + 2 < NT;   // pairs 2k and 2k+1 exist

    uint32_t *gS = a.spins + (size_t)unit * NT * N;
    const uint32_t *gJ = a.bonds + (size_t)g * 3 * N;
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
    for (int w = tid; w < 3 * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
    const uint32_t *swt = a.swapt;
    if (swap_in_smem) {
        uint32_t *Tsw = base + lay.tsw;
        for (int w = tid; w < (NT - 1) * (int)a.swap_len; w += nthr) Tsw[w] = a.swapt[w];
        swt = Tsw;
    }
    for (int i = tid; i < (NT + 1) / 2; i += nthr) {
        mbar_init(&bar_e[i], kLanes);
        mbar_init(&bar_h[i], kLanes);
    }
    if (tid == 0) *abort = 0u;
    const uint64_t t0 = 0ull - (uint64_t)a.metro[ls * 3 + 0];
    const uint64_t t1 = 0ull - (uint64_t)a.metro[ls * 3 + 1];
    const uint64_t t2 = 0ull - (uint64_t)a.metro[ls * 3 + 2];
    QuadRow qd[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) qd[j] = quad_row<L>(j >> 1, li + 16 * (j & 1));
    uint32_t *mine = S + (size_t)ls * N;
    const uint32_t tag0 = ((uint32_t)c << 8) | (uint32_t)ls;
    const uint32_t tag1 = (1u << 16) | tag0;
    const uint32_t len = a.swap_len;
    uint32_t top = 0;                                   // largest power of two <= len
    if (len != 0) {
        top = 1;
        while (top <= (len >> 1)) top <<= 1;
    }
    __syncthreads();   // staged lattices, bonds, table and flags are complete; no CTA barrier after this
    if (2 * k >= NT) return;                            // warps beyond the slots (wider CTAs of a batch)

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    int bA = 0, bB = 0;
    if (NT > 1 && a.swap_every != 0 && hasB) wave_bounds(swt, len, top, k, NT, c, P, gr, a.rk, lane, bA, bB);
    int EA = 0, EB = 0;                                 // energies of slots 2k, 2k+1 (lane = realization)
    bool ok_run = true;
    uint32_t ph_e = 0, ph_h = 0;                        // parity of the next phase this warp waits for

    for (uint32_t n = 0; n < a.n_sweeps && ok_run; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_now = swap_after(s, a.swap_every) && NT > 1;
        const bool needE = swap_now || energy_log != nullptr || (n + 1 == a.n_sweeps);
        uint32_t acc[PL];
#pragma unroll
        for (int p = 0; p < PL; ++p) acc[p] = 0;
        if (act) wave_half<0, false, PL>(mine, Js, qd, (uint32_t)s, gr, tag0, a.rk, t0, t1, t2, acc);
        __syncwarp();
        if (needE) {
            if (act) wave_half<1, true, PL>(mine, Js, qd, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
            int UA, UB;
            wave_reduce<PL>(acc, lane, UA, UB);          // also orders the colour-1 stores (shuffles)
            EA = 2 * UA - 3 * N;
            EB = 2 * UB - 3 * N;
        } else if (act) {
            wave_half<1, false, PL>(mine, Js, qd, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
        }
        __syncwarp();
        if (swap_now) {
            // publish E_{2k} (pre-exchange) for pair 2k-1 of warp k-1
            Eo[2 * k * kLanes + lane] = EA;
            if (k > 0) mbar_arrive(&bar_e[k - 1]);
            int cur = EA;
            if (k > 0) {
                if (!wave_wait(&bar_h[k - 1], ph_h, abort, a.err)) { ok_run = false; break; }
                ph_h ^= 1u;
                cur = Cur[(k - 1) * kLanes + lane];
            }
            uint32_t mA = 0, mB = 0;
            if (hasB) {
                // pair 2k: slot 2k holds the carried configuration (energy cur)
                const bool okA = cur - EB >= bA;
                mA = __ballot_sync(kFull, okA);
                const int nEA = okA ? EB : cur;
                cur = okA ? cur : EB;
                uint4 *pa = reinterpret_cast<uint4 *>(S + (size_t)(2 * k) * N);
                uint4 *pb = reinterpret_cast<uint4 *>(S + (size_t)(2 * k + 1) * N);
                uint4 xb[N / 128];                      // slot 2k+1 after pair 2k (the carry)
#pragma unroll
                for (int j = 0; j < N / 128; ++j) {
                    const uint4 x = pa[lane + 32 * j], y = pb[lane + 32 * j];
                    pa[lane + 32 * j] = make_uint4(mux(x.x, y.x, mA), mux(x.y, y.y, mA), mux(x.z, y.z, mA),
                                                   mux(x.w, y.w, mA));
                    xb[j] = make_uint4(mux(y.x, x.x, mA), mux(y.y, x.y, mA), mux(y.z, x.z, mA), mux(y.w, x.w, mA));
                }
                int nEB;
                if (hasC) {
                    if (!wave_wait(&bar_e[k], ph_e, abort, a.err)) { ok_run = false; break; }
                    ph_e ^= 1u;
                    const int e2 = Eo[(2 * k + 2) * kLanes + lane];
                    const bool okB = cur - e2 >= bB;
                    mB = __ballot_sync(kFull, okB);
                    nEB = okB ? e2 : cur;
                    cur = okB ? cur : e2;
                    uint4 *pc = reinterpret_cast<uint4 *>(S + (size_t)(2 * k + 2) * N);
#pragma unroll
                    for (int j = 0; j < N / 128; ++j) {
                        const uint4 x = xb[j], y = pc[lane + 32 * j];
                        pb[lane + 32 * j] = make_uint4(mux(x.x, y.x, mB), mux(x.y, y.y, mB), mux(x.z, y.z, mB),
                                                       mux(x.w, y.w, mB));
                        pc[lane + 32 * j] = make_uint4(mux(y.x, x.x, mB), mux(y.y, x.y, mB), mux(y.z, x.z, mB),
                                                       mux(y.w, x.w, mB));
                    }
                    Cur[k * kLanes + lane] = cur;
                    mbar_arrive(&bar_h[k]);
                } else {
#pragma unroll
                    for (int j = 0; j < N / 128; ++j) pb[lane + 32 * j] = xb[j];
                    nEB = cur;                          // slot 2k+1 is the last
                }
                EA = nEA;
                EB = nEB;
            } else {
                EA = cur;                               // slot 2k is the last (odd NT)
            }
            __syncwarp();
            if (swap_log != nullptr && lane == 0) {
                uint32_t *row = swap_log + ((size_t)pass_local * a.G + g) * a.C * (NT - 1) + (size_t)c * (NT - 1);
                if (hasB) row[2 * k] = mA;
                if (hasC) row[2 * k + 1] = mB;
            }
            ++P;
            ++pass_local;
            if (hasB) wave_bounds(swt, len, top, k, NT, c, P, gr, a.rk, lane, bA, bB);
        } else if (swap_after(s, a.swap_every)) {
            ++P;                                        // NT == 1: passes count, nothing to exchange
            ++pass_local;
        }
        if (energy_log != nullptr) {
            const size_t row = (size_t)(s - a.log_s0);
            int32_t *el = energy_log + ((row * a.G + g) * NT) * a.C * kLanes + (size_t)c * kLanes;
            el[(size_t)(2 * k) * a.C * kLanes + lane] = EA;
            if (hasB) el[(size_t)(2 * k + 1) * a.C * kLanes + lane] = EB;
        }
    }
    if (!ok_run) return;                                // the error flag is raised; state is not written
    int32_t *gE = a.energy + (size_t)unit * NT * kLanes;
    gE[(2 * k) * kLanes + lane] = EA;
    if (hasB) gE[(2 * k + 1) * kLanes + lane] = EB;
    // this warp's slots are final (no later pass step touches them)
    const int nslot = hasB ? 2 : 1;
    for (int w = lane; w < nslot * N / 4; w += 32)
        reinterpret_cast<uint4 *>(gS + (size_t)(2 * k) * N)[w] =
            reinterpret_cast<const uint4 *>(S + (size_t)(2 * k) * N)[w];
}

}  // namespace
}  // namespace ea
