// Temperature-packed form: one word per (realization, copy, site) whose bit t
// holds the spin of temperature slot t.  This is the word layout of the
// paper's compact asynchronous multispin coding (Sec. 3.2, Sec. 4.3.3): the
// temperature replicas of one realization share a word, the six bond XORs of
// Eq. e act on all of them at once, and a replica exchange (Sec. 2.4) moves
// bits inside the word instead of moving words.
//
// Random numbers are the realization's own: realization r draws the stream of
// word-group r of the realization-packed form (of which it is realization 32r,
// i.e. bit 0), so no two realizations share a uniform.  Each flip attempt gets
// its own uniform (the paper's per-replica random numbers, Sec. 4.3.2), which
// makes this form suited to ensembles with few realizations and many
// temperatures; the realization-packed form shares one uniform among 32
// realizations and is the faster form when realizations are plentiful.
//
// Kernel shape (one CTA per (realization, copy) unit, the whole call in one
// launch, state in shared memory): four threads per quad of four sites.  For
// each slot t it owns (t = i, i + 4, ...), thread i draws the quad's four
// uniforms with one Philox4x32-10 call and tests them against the slot's three
// thresholds on the FMA pipe (r < T as the high word of r + 2^64 - T), setting
// bit t of twelve partial masks; two OR-shuffles complete the masks and thread
// i updates site i of the quad with the bit-sliced adder of the other forms.
// Energies per slot come from a bit-sliced counter over the colour-1 sites
// (E = 2U - 3N), reduced by a shuffle butterfly; the swap pass runs its chain
// on one warp and applies the accepted pairs to every word as a bit
// permutation: new bit t = old bit t + 1 where pair t was accepted, else the
// bit at the start of the run of accepted pairs that ends at t (an integer
// addition carries each run's start bit to its end).
//
// Few realizations leave most SMs idle with one CTA per unit, so a unit can be
// split into slot groups (slots do not interact between swap passes): one CTA
// per group sweeps only its slots' bits up to the next pass and stores them in
// its slice, and k_tp_merge ORs the slices and runs the pass.
//
// More than 32 temperatures take several words per site (the paper's several
// integer cubes, Sec. 3.2): word w holds slots 32w .. 32w + 31.  Slot groups
// then never straddle a word, every group sweeps its word as above, and the
// merge runs the pass over all words: the bit permutation above is a shift and
// an addition of 32W-bit integers, whose carries cross the words.
#include <new>

#include "../../include/ea.h"
#include "ea_device.cuh"

namespace ea {
namespace {

constexpr int kTpMaxTemps = 64;      // two words per site
constexpr int kTpMaxWords = kTpMaxTemps / 32;
constexpr int kTpThreads = 1024;   // at most 64 registers a thread

struct TpLaunch {
    uint32_t *spins;            // [R][C][W][2][H]: word w, bit b = slot 32 w + b
    const uint32_t *bonds;      // [R][3][2][H], words 0 (J = +1) or ~0 (J = -1)
    const uint64_t *nthr;       // [NT][3]: 2^64 - metro threshold
    const uint32_t *swapt;      // [NT-1][swap_len]
    uint32_t swap_len;
    int32_t *energy;            // [R][C][32 W] by slot
    uint32_t R, NT, C;
    RoundKeys rk;
    uint64_t s0;                // global index of the first sweep
    uint32_t n_sweeps, swap_every;
    uint64_t P0;                // global index of the first swap pass of this call
    uint32_t pass_local0;       // row of swap_log for that pass
    int32_t *energy_log;        // [n_sweeps][R][NT][C] or null
    uint32_t *swap_log;         // [passes][R][C][W] (bit b of word w = pair 32 w + b) or null
    // slot split: CTA (unit, y) owns slots [32 w + j spg, 32 w + (j + 1) spg) of
    // word w = y / gpw (j = y % gpw, clipped to the word's slots) and writes them
    // to slices[y]; null = one CTA per unit owning every slot (W = 1)
    uint32_t *slices;           // [nsplit][R][C][2][H]
    uint32_t spg;               // slots per group
    uint32_t gpw;               // groups per word
    uint32_t nsplit;            // groups (gridDim.y) = W gpw
    uint32_t W;                 // words per site = ceil(NT / 32)
    uint32_t r_base;            // global index of realization 0 in the random-number counters
};

// The words a site update reads: own spin word, its six neighbours and the six
// bond words (+x, -x, +y, -y, +z, -z; the -d bond's J is stored at the
// neighbour).  k is the site's class index in colour col.
template <int L>
__device__ __forceinline__ void tp_load_site(const uint32_t *S, const uint32_t *J, int col, int k,
                                             uint32_t &own, uint32_t (&nb)[6], uint32_t (&jb)[6])
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N, H = Gm::H, R = Gm::R;
    const uint32_t *Sc = S + col * H;
    const uint32_t *So = S + (col ^ 1) * H;
    const int row = k / R, m = k - row * R;
    const int y = row % L, z = row / L;
    const int px = (y + z + col) & 1;           // x parity of the site
    const int rowb = row * R;
    const int kxp = rowb + (px ? (m + 1 == R ? 0 : m + 1) : m);
    const int kxm = rowb + (px ? m : (m == 0 ? R - 1 : m - 1));
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
    const int kyp = m + R * (yp + L * z), kym = m + R * (ym + L * z);
    const int kzp = m + R * (y + L * zp), kzm = m + R * (y + L * zm);
    own = Sc[k];
    nb[0] = So[kxp];
    nb[1] = So[kxm];
    nb[2] = So[kyp];
    nb[3] = So[kym];
    nb[4] = So[kzp];
    nb[5] = So[kzm];
    jb[0] = J[0 * N + col * H + k];
    jb[1] = J[0 * N + (col ^ 1) * H + kxm];
    jb[2] = J[1 * N + col * H + k];
    jb[3] = J[1 * N + (col ^ 1) * H + kym];
    jb[4] = J[2 * N + col * H + k];
    jb[5] = J[2 * N + (col ^ 1) * H + kzm];
}

__device__ __forceinline__ uint32_t pick4(const uint32_t (&v)[4], int i)
{
    return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : v[3];
}

// acc += (x2 x1 x0), bit-sliced per slot bit.
__device__ __forceinline__ void tp_acc_add3(uint32_t (&acc)[kPlanes], uint32_t x0, uint32_t x1,
                                            uint32_t x2)
{
    uint32_t cy = acc[0] & x0;
    acc[0] ^= x0;
    uint32_t s, c;
    full_add(acc[1], x1, cy, s, c);
    acc[1] = s;
    cy = c;
    full_add(acc[2], x2, cy, s, c);
    acc[2] = s;
    cy = c;
#pragma unroll
    for (int p = 3; p < kPlanes; ++p) {
        c = acc[p] & cy;
        acc[p] ^= cy;
        cy = c;
    }
}

// Sets bit t of m_k[x] iff uniform x of v is below threshold k of slot t.  The
// tests are wide multiply-adds on the FMA pipe (below_wide).  Bit t of m_0 is
// ORed in on the integer ALU pipe; those of m_1 and m_2 are added on the FMA
// pipe as m += below * (-2^t) (below is 0 or all ones and bit t is still
// clear), which balances the two pipes (the Philox rounds load both).
__device__ __forceinline__ void tp_mask_bits(uint32_t (&m0)[4], uint32_t (&m1)[4], uint32_t (&m2)[4],
                                             const uint4 v, const uint64_t *th, int t)
{
    const uint64_t n0 = th[0], n1 = th[1], n2 = th[2];
    const uint32_t negbit = 0u - (1u << t);
    const uint32_t rr[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        m0[x] |= below_wide(rr[x], n0) & (0u - negbit);
        m1[x] = below_wide(rr[x], n1) * negbit + m1[x];
        m2[x] = below_wide(rr[x], n2) * negbit + m2[x];
    }
}

// One half-sweep (colour col) of one word of a unit, slots [t_lo, t_hi) of the
// word whose bit 0 is slot wb (omask = their bits; the other bits of the words
// are left as they are).  Thread (quad group
// qg, site i) takes quads qg, qg + nqg, ...; the trip count qper is the same
// for every thread so that the whole warp takes part in each shuffle.  MODE 0: update
// without counting; 1: update and count the post-update unsatisfied bonds of
// the (colour-1) sites; 2: count the current unsatisfied bonds, no update.
template <int L, int MODE>
__device__ __forceinline__ void tp_half(uint32_t *S, const uint32_t *J, const uint64_t *nthr, int col,
                                        int qg, int nqg, int qper, int i, int t_lo, int t_hi, int wb,
                                        uint32_t omask, uint32_t s, uint32_t r, uint32_t ctag,
                                        const RoundKeys &rk, uint32_t (&acc)[kPlanes])
{
    constexpr int Q = Geo<L>::Q, H = Geo<L>::H;
    for (int j = 0; j < qper; ++j) {
        const int q0 = qg + j * nqg;
        const bool inq = q0 < Q;
        const int q = inq ? q0 : 0;
        uint32_t f = 0;
        if constexpr (MODE != 2) {
            uint32_t m0[4] = {0u, 0u, 0u, 0u}, m1[4] = {0u, 0u, 0u, 0u}, m2[4] = {0u, 0u, 0u, 0u};
            if (inq) {
                for (int t = t_lo + i; t < t_hi; t += 4) {
                    const uint4 v = philox((uint32_t)q, ctag | (uint32_t)t, s, r, rk);
                    tp_mask_bits(m0, m1, m2, v, nthr + 3 * t, t - wb);
                }
            }
#pragma unroll
            for (int d = 1; d <= 2; d <<= 1) {
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    m0[x] |= __shfl_xor_sync(kFull, m0[x], d);
                    m1[x] |= __shfl_xor_sync(kFull, m1[x], d);
                    m2[x] |= __shfl_xor_sync(kFull, m2[x], d);
                }
            }
            if (!inq) continue;
            const uint32_t M0 = pick4(m0, i), M1 = pick4(m1, i), M2 = pick4(m2, i);
            uint32_t own, nb[6], jb[6];
            tp_load_site<L>(S, J, col, 4 * q + i, own, nb, jb);
            uint32_t e[6];
#pragma unroll
            for (int d = 0; d < 6; ++d) e[d] = own ^ nb[d] ^ jb[d];
            uint32_t a0, a1, b0, b1, u0, u1, u2;
            full_add(e[0], e[1], e[2], a0, a1);
            full_add(e[3], e[4], e[5], b0, b1);
            u0 = a0 ^ b0;
            full_add(a1, b1, a0 & b0, u1, u2);
            const uint32_t ge3 = u2 | (u1 & u0), ge2 = u2 | u1, ge1 = ge2 | u0;
            f = (ge3 | (ge2 & M2) | (ge1 & M1) | M0) & omask;
            S[col * H + 4 * q + i] = own ^ f;
            if constexpr (MODE == 1) {
                // flipped sites hold 6 - u unsatisfied bonds
                tp_acc_add3(acc, u0, u1 ^ (f & ~u0), u2 ^ (f & ~(u0 & u1)));
            }
        } else {
            if (!inq) continue;
            uint32_t own, nb[6], jb[6];
            tp_load_site<L>(S, J, col, 4 * q + i, own, nb, jb);
            uint32_t e[6];
#pragma unroll
            for (int d = 0; d < 6; ++d) e[d] = own ^ nb[d] ^ jb[d];
            uint32_t a0, a1, b0, b1, u0, u1, u2;
            full_add(e[0], e[1], e[2], a0, a1);
            full_add(e[3], e[4], e[5], b0, b1);
            u0 = a0 ^ b0;
            full_add(a1, b1, a0 & b0, u1, u2);
            tp_acc_add3(acc, u0, u1, u2);
        }
    }
}

// Adds 2 x (the warp's per-slot counts) into E[t], t in [t_lo, t_hi): a
// shuffle butterfly of bit-sliced adders leaves the warp total (kPlanes + 5
// planes) in every lane, then lane t reads bit t of each plane.
__device__ __forceinline__ void tp_reduce_energy(const uint32_t (&acc)[kPlanes], int *E, int lane, int t_lo,
                                                 int t_hi)
{
    constexpr int PT = kPlanes + 5;
    uint32_t v[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) v[p] = p < kPlanes ? acc[p] : 0u;
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        uint32_t cy = 0;
#pragma unroll
        for (int p = 0; p < kPlanes + lv + 1; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, v[p], 1 << lv);
            uint32_t s2, c2;
            full_add(v[p], o, cy, s2, c2);
            v[p] = s2;
            cy = c2;
        }
    }
    int cnt = 0;
#pragma unroll
    for (int p = 0; p < PT; ++p) cnt += (int)((v[p] >> lane) & 1u) << p;
    if (lane >= t_lo && lane < t_hi && cnt != 0) atomicAdd(&E[lane], 2 * cnt);
}

// Layout of the dynamic shared memory: spins [2][H], then (J_SMEM) bonds [3][2][H].
template <int L, bool J_SMEM>
__global__ void __launch_bounds__(kTpThreads)
k_tp_sweep(TpLaunch a, int recompute_only)
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N, Q = Gm::Q;
    extern __shared__ __align__(16) uint32_t tp_smem[];
    __shared__ uint64_t nthr[kTpMaxTemps * 3];
    __shared__ int E[32];                               // by bit of the word this CTA updates
    __shared__ uint32_t smask;
    uint32_t *S = tp_smem;
    const uint32_t unit = blockIdx.x;
    const uint32_t c = unit % a.C, r = unit / a.C;
    const uint32_t rr = r + a.r_base;                   // realization index of the random numbers
    const int NT = (int)a.NT;
    const int tid = threadIdx.x, nthr_cta = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int i = tid & 3, qg = tid >> 2, nqg = nthr_cta >> 2;
    const int qper = (Q + nqg - 1) / nqg;
    // the word of the unit this CTA updates (bit 0 = slot wb) and its slots [t_lo, t_hi)
    int w = 0, t_lo = 0, t_hi = NT;
    if (a.slices) {
        w = (int)(blockIdx.y / a.gpw);
        t_lo = 32 * w + (int)((blockIdx.y % a.gpw) * a.spg);
        t_hi = max(t_lo, min(min(NT, 32 * w + 32), t_lo + (int)a.spg));
    } else if (recompute_only) {
        w = (int)blockIdx.y;
        t_lo = 32 * w;
        t_hi = min(NT, t_lo + 32);
    }
    const int wb = 32 * w, nw = min(32, NT - wb);
    const uint32_t valid = nw >= 32 ? kFull : ((1u << nw) - 1u);
    const int b_lo = t_lo - wb, b_hi = t_hi - wb;       // bits of the word, 0 <= b_lo <= b_hi <= 32
    const uint32_t own = (b_hi >= 32 ? kFull : ((1u << b_hi) - 1u)) & ~((1u << b_lo) - 1u);
    int32_t *const gE = a.energy + (size_t)unit * kLanes * a.W + wb;

    uint32_t *gS = a.spins + ((size_t)unit * a.W + w) * N;
    const uint32_t *gJ = a.bonds + (size_t)r * 3 * N;
    for (int w = tid; w < N / 4; w += nthr_cta)
        reinterpret_cast<uint4 *>(S)[w] = __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
    const uint32_t *J = gJ;
    if constexpr (J_SMEM) {
        uint32_t *Js = tp_smem + N;
        for (int w = tid; w < 3 * N / 4; w += nthr_cta)
            reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
        J = Js;
    }
    for (int x = tid; x < NT * 3; x += nthr_cta) nthr[x] = a.nthr[x];
    if (tid < 32) E[tid] = -3 * N;
    __syncthreads();

    uint32_t acc[kPlanes];
    if (recompute_only) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
        tp_half<L, 2>(S, J, nthr, 1, qg, nqg, qper, i, 0, 0, wb, valid, 0u, rr, 0u, a.rk, acc);
        tp_reduce_energy(acc, E, lane, 0, nw);
        __syncthreads();
        if (tid < 32) gE[tid] = tid < nw ? E[tid] : 0;
        return;
    }

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    const uint32_t tag0 = (c << 8), tag1 = (1u << 16) | (c << 8);
    SwapCountdown swap_cd(a.s0, a.swap_every);
    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_s = swap_cd.step();             // a pass follows sweep s
        const bool swap_now = swap_s && NT > 1;
        const bool needE = swap_now || a.energy_log != nullptr || (n + 1 == a.n_sweeps);
        if (needE && tid < 32) E[tid] = -3 * N;
        tp_half<L, 0>(S, J, nthr, 0, qg, nqg, qper, i, t_lo, t_hi, wb, own, (uint32_t)s, rr, tag0, a.rk, acc);
        __syncthreads();
        if (needE) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
            tp_half<L, 1>(S, J, nthr, 1, qg, nqg, qper, i, t_lo, t_hi, wb, own, (uint32_t)s, rr, tag1, a.rk, acc);
            tp_reduce_energy(acc, E, lane, b_lo, b_hi);
        } else {
            tp_half<L, 0>(S, J, nthr, 1, qg, nqg, qper, i, t_lo, t_hi, wb, own, (uint32_t)s, rr, tag1, a.rk, acc);
        }
        __syncthreads();
        if (swap_now) {                                 // one word (W = 1): the pass in this kernel
            if (warp == 0) {
                // lane t: energy of slot t and the acceptance bound of pair t
                const int e = lane < NT ? E[lane] : 0;
                int bnd = 0;
                if (lane + 1 < NT) {
                    const uint4 v = philox((uint32_t)lane << 3, (1u << 24) | (c << 8), (uint32_t)P, rr, a.rk);
                    bnd = accept_bound(a.swapt + (size_t)lane * a.swap_len, a.swap_len, v.x);
                }
                // sequential pairs 0..NT-2 on the energies carried upward
                int cur = __shfl_sync(kFull, e, 0), mine = e;
                uint32_t m = 0;
                for (int p = 0; p + 1 < NT; ++p) {
                    const int nx = __shfl_sync(kFull, e, p + 1);
                    const int bp = __shfl_sync(kFull, bnd, p);
                    const bool ok = cur - nx >= bp;
                    if (lane == p) mine = ok ? nx : cur;
                    cur = ok ? cur : nx;
                    m |= (uint32_t)ok << p;
                }
                if (lane == NT - 1) mine = cur;
                if (lane < NT) E[lane] = mine;
                if (lane == 0) {
                    smask = m;
                    if (a.swap_log) a.swap_log[((size_t)pass_local * a.R + r) * a.C + c] = m;
                }
            }
            __syncthreads();
            // the pass as a bit permutation of every word of the unit
            const uint32_t M = smask;
            const uint32_t ends = ~M & valid;
            const uint32_t starts = ((~M << 1) | 1u) & valid;
            for (int w = tid; w < N; w += nthr_cta) {
                const uint32_t x = S[w];
                S[w] = ((x >> 1) & M) | ((M + (starts & x)) & ends);
            }
            __syncthreads();
        }
        if (swap_s) {
            ++P;
            ++pass_local;
        }
        if (a.energy_log != nullptr && tid >= b_lo && tid < b_hi)
            a.energy_log[(((size_t)n * a.R + r) * NT + wb + tid) * a.C + c] = E[tid];
        // E is rewritten at the top of the next sweep only by the thread that logged it
    }
    __syncthreads();
    if (a.slices) {
        // this group's bits go to its slice; the merge kernel ORs the slices
        uint32_t *sl = a.slices + ((size_t)blockIdx.y * gridDim.x + unit) * N;
        for (int w = tid; w < N / 4; w += nthr_cta) {
            const uint4 x = reinterpret_cast<const uint4 *>(S)[w];
            __stcg(reinterpret_cast<uint4 *>(sl) + w, make_uint4(x.x & own, x.y & own, x.z & own, x.w & own));
        }
    } else {
        for (int w = tid; w < N / 4; w += nthr_cta)
            __stcg(reinterpret_cast<uint4 *>(gS) + w, reinterpret_cast<const uint4 *>(S)[w]);
    }
    if (tid >= b_lo && tid < b_hi) gE[tid] = E[tid];
    else if (!a.slices && tid < 32) gE[tid] = 0;
}

// Slot-split form: merges the groups' slices into the unit's words and, with
// do_swap, runs the swap pass on them (one CTA per unit): warp 0 takes the
// decision chain as in k_tp_sweep (lane t holds slots t and t + 32), then
// every site gets the pass's bit permutation over its W words.  elog_row (or
// null): the energy-log row of the interval's last sweep, rewritten with the
// energies after the pass.
__global__ void __launch_bounds__(256)
k_tp_merge(TpLaunch a, int N, int do_swap, uint64_t P, uint32_t pass_local, int32_t *elog_row)
{
    static_assert(kTpMaxWords == 2, "the chain holds two slots a lane");
    __shared__ uint32_t smask[kTpMaxWords];
    const uint32_t unit = blockIdx.x;
    const uint32_t c = unit % a.C, r = unit / a.C;
    const uint32_t rr = r + a.r_base;                   // realization index of the random numbers
    const int NT = (int)a.NT, W = (int)a.W, tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        int32_t *Eg = a.energy + (size_t)unit * kLanes * W;
        const int e0 = lane < NT ? Eg[lane] : 0;
        const int e1 = lane + 32 < NT ? Eg[lane + 32] : 0;
        uint32_t m0 = 0, m1 = 0;
        int mine0 = e0, mine1 = e1;
        if (do_swap) {
            int bnd0 = 0, bnd1 = 0;
            if (lane + 1 < NT) {
                const uint4 v = philox((uint32_t)lane << 3, (1u << 24) | (c << 8), (uint32_t)P, rr, a.rk);
                bnd0 = accept_bound(a.swapt + (size_t)lane * a.swap_len, a.swap_len, v.x);
            }
            if (lane + 33 < NT) {
                const uint4 v = philox((uint32_t)(lane + 32) << 3, (1u << 24) | (c << 8), (uint32_t)P, rr, a.rk);
                bnd1 = accept_bound(a.swapt + (size_t)(lane + 32) * a.swap_len, a.swap_len, v.x);
            }
            // sequential pairs 0..NT-2 on the energies carried upward (the word of
            // a slot is the same for every lane, so each shuffle is warp-wide)
            int cur = __shfl_sync(kFull, e0, 0);
            for (int p = 0; p + 1 < NT; ++p) {
                const int q = p + 1;
                const int nx = q < 32 ? __shfl_sync(kFull, e0, q) : __shfl_sync(kFull, e1, q - 32);
                const int bp = p < 32 ? __shfl_sync(kFull, bnd0, p) : __shfl_sync(kFull, bnd1, p - 32);
                const bool ok = cur - nx >= bp;
                if (p < 32) {
                    if (lane == p) mine0 = ok ? nx : cur;
                    m0 |= (uint32_t)ok << p;
                } else {
                    if (lane == p - 32) mine1 = ok ? nx : cur;
                    m1 |= (uint32_t)ok << (p - 32);
                }
                cur = ok ? cur : nx;
            }
            if (NT - 1 < 32) {
                if (lane == NT - 1) mine0 = cur;
            } else if (lane == NT - 33) {
                mine1 = cur;
            }
            if (lane < NT) Eg[lane] = mine0;
            if (lane + 32 < NT) Eg[lane + 32] = mine1;
            if (lane == 0 && a.swap_log) {
                uint32_t *sl = a.swap_log + (((size_t)pass_local * a.R + r) * a.C + c) * W;
                sl[0] = m0;
                if (W > 1) sl[1] = m1;
            }
            if (elog_row) {
                if (lane < NT) elog_row[((size_t)r * NT + lane) * a.C + c] = mine0;
                if (lane + 32 < NT) elog_row[((size_t)r * NT + lane + 32) * a.C + c] = mine1;
            }
        }
        if (lane == 0) {
            smask[0] = m0;
            smask[1] = m1;
        }
    }
    __syncthreads();
    // the pass on the 32W-bit integer of a site's words: bit t <- bit t + 1 where
    // pair t was accepted, else the bit at the start of the run of accepted pairs
    // ending at t (M + (starts & x) carries each run's start bit to its end)
    const uint32_t M0 = smask[0], M1 = W > 1 ? smask[1] : 0u;
    const uint32_t valid0 = NT >= 32 ? kFull : ((1u << NT) - 1u);
    const uint32_t valid1 = W < 2 ? 0u : (NT >= 64 ? kFull : ((1u << (NT - 32)) - 1u));
    const uint32_t ends0 = ~M0 & valid0, ends1 = ~M1 & valid1;
    const uint32_t starts0 = ((~M0 << 1) | 1u) & valid0;
    const uint32_t starts1 = ((~M1 << 1) | (~M0 >> 31)) & valid1;
    const size_t stride = (size_t)gridDim.x * N;
    const uint32_t gpw = a.gpw;
    const uint32_t *src = a.slices + (size_t)unit * N;
    uint32_t *dst = a.spins + (size_t)unit * W * N;
    for (int w = tid; w < N; w += blockDim.x) {
        uint32_t x0 = 0, x1 = 0;
        for (uint32_t g = 0; g < gpw; ++g) x0 |= __ldcg(src + g * stride + w);
        if (W > 1)
            for (uint32_t g = gpw; g < 2 * gpw; ++g) x1 |= __ldcg(src + g * stride + w);
        if (do_swap) {
            const uint32_t sh0 = (x0 >> 1) | (x1 << 31), sh1 = x1 >> 1;
            const uint32_t s0 = M0 + (starts0 & x0);
            const uint32_t cy = s0 < M0 ? 1u : 0u;      // carry into slot 32
            const uint32_t s1 = M1 + (starts1 & x1) + cy;
            x0 = (sh0 & M0) | (s0 & ends0);
            x1 = (sh1 & M1) | (s1 & ends1);
        }
        dst[w] = x0;
        if (W > 1) dst[N + w] = x1;
    }
}

// spins: API [R][C][W][N] (site order) <-> device [R][C][W][2][H] (colour-split),
// bits of slots >= NT cleared on import.
__global__ void k_tp_import_spins(const uint32_t *api, uint32_t *dev, int L, size_t total, int NT, int W)
{
    const int N = L * L * L, H = N / 2, R = L / 2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t unit = idx / N;                    // (realization, copy, word)
        const int nw = NT - 32 * (int)(unit % W);       // slots in this word (>= 1)
        const uint32_t valid = nw >= 32 ? kFull : ((1u << nw) - 1u);
        const int col = w / H, k = w - col * H;
        const int row = k / R, y = row % L, z = row / L;
        const int site = 2 * k + ((col + y + z) & 1);
        dev[idx] = api[unit * N + site] & valid;
    }
}

__global__ void k_tp_export_spins(const uint32_t *dev, uint32_t *api, int L, size_t total)
{
    const int N = L * L * L, H = N / 2, R = L / 2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t unit = idx / N;
        const int col = w / H, k = w - col * H;
        const int row = k / R, y = row % L, z = row / L;
        api[unit * N + 2 * k + ((col + y + z) & 1)] = dev[idx];
    }
}

// bonds: API [R][3][N] bytes (1 <=> J = -1) -> device [R][3][2][H] words 0 / ~0.
__global__ void k_tp_import_bonds(const uint8_t *api, uint32_t *dev, int L, size_t total)
{
    const int N = L * L * L, H = N / 2, R = L / 2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t rd = idx / N;
        const int col = w / H, k = w - col * H;
        const int row = k / R, y = row % L, z = row / L;
        dev[idx] = api[rd * N + 2 * k + ((col + y + z) & 1)] ? kFull : 0u;
    }
}

// energies: device [R][C][32 W] -> API [R][NT][C]
__global__ void k_tp_export_energy(const int32_t *dev, int32_t *api, uint32_t R, uint32_t NT, uint32_t C,
                                   uint32_t W)
{
    const size_t total = (size_t)R * NT * C;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(idx % C), t = (uint32_t)((idx / C) % NT);
        const size_t r = idx / ((size_t)C * NT);
        api[idx] = dev[(r * C + c) * kLanes * W + t];
    }
}

int tp_grid(size_t total)
{
    size_t b = (total + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

bool tp_j_smem(int L) { return L <= 24; }

size_t tp_smem_bytes(int L)
{
    const size_t N = (size_t)L * L * L;
    return N * 4 * (tp_j_smem(L) ? 4 : 1);
}

int tp_threads(int L)
{
    const int Q = L * L * L / 8;
    int t = 4 * Q;
    t = (t + 31) / 32 * 32;
    return t > kTpThreads ? kTpThreads : t;
}

template <int L>
cudaError_t tp_launch_L(const TpLaunch &a, int recompute_only, cudaStream_t st)
{
    constexpr bool JS = L <= 24;
    const size_t smem = tp_smem_bytes(L);
    const cudaError_t e = cudaFuncSetAttribute(k_tp_sweep<L, JS>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid(a.R * a.C, a.slices ? a.nsplit : (recompute_only ? a.W : 1));
    k_tp_sweep<L, JS><<<grid, tp_threads(L), smem, st>>>(a, recompute_only);
    return cudaGetLastError();
}

cudaError_t tp_launch(int L, const TpLaunch &a, int recompute_only, cudaStream_t st)
{
    switch (L) {
#define EA_TP_CASE(X) case X: return tp_launch_L<X>(a, recompute_only, st);
        EA_TP_CASE(4) EA_TP_CASE(6) EA_TP_CASE(8) EA_TP_CASE(10) EA_TP_CASE(12)
        EA_TP_CASE(14) EA_TP_CASE(16) EA_TP_CASE(20) EA_TP_CASE(24) EA_TP_CASE(32)
#undef EA_TP_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace ea

struct ea_tp {
    uint32_t L, R, NT, C, N, swap_len;
    uint32_t W;                    // words per site, ceil(NT / 32)
    cudaStream_t stream;
    uint32_t *d_spins, *d_bonds, *d_swapt;
    uint64_t *d_nthr;
    int32_t *d_energy;
    uint64_t sweep, pass, launches;
    ea::RoundKeys rk;
    uint32_t r_base;               // ea_tp_config::real_base
    uint32_t split, spg, gpw, nsplit;   // requested groups per word, slots per group,
                                        // groups per word in use, groups in use (W gpw)
    uint32_t *d_slices;            // [nsplit][R][C][N] when nsplit > 1
};

namespace {

int tp_cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? EA_ENOMEM : EA_ECUDA; }

void tp_free(ea_tp *t)
{
    if (!t) return;
    cudaFree(t->d_spins);
    cudaFree(t->d_bonds);
    cudaFree(t->d_swapt);
    cudaFree(t->d_nthr);
    cudaFree(t->d_energy);
    cudaFree(t->d_slices);
    delete t;
}

// Slot groups per word: k groups of ceil(n0 / k) slots, n0 = min(NT, 32) the
// slots of the first word (the groups in use are the ones non-empty there; a
// shorter last word may leave some empty); slices for them are (re)allocated
// here.  More than one word always takes the slot-group path.
int tp_apply_split(ea_tp *t, uint32_t k)
{
    const uint32_t n0 = t->NT < 32 ? t->NT : 32;
    const uint32_t spg = (n0 + k - 1) / k;
    const uint32_t gpw = (n0 + spg - 1) / spg;
    const uint32_t nsplit = t->W * gpw;
    if (t->d_slices && nsplit != t->nsplit) {
        const cudaError_t e = cudaStreamSynchronize(t->stream);
        if (e != cudaSuccess) return tp_cuda_fail(e);
        cudaFree(t->d_slices);
        t->d_slices = nullptr;
    }
    if (nsplit > 1 && !t->d_slices) {
        const cudaError_t e = cudaMalloc(&t->d_slices, (size_t)nsplit * t->R * t->C * t->N * 4);
        if (e != cudaSuccess) return tp_cuda_fail(e);
    }
    t->split = k;
    t->spg = spg;
    t->gpw = gpw;
    t->nsplit = nsplit;
    return EA_OK;
}

bool tp_supported_L(uint32_t L)
{
    switch (L) {
    case 4: case 6: case 8: case 10: case 12: case 14: case 16: case 20: case 24: case 32: return true;
    default: return false;
    }
}

}  // namespace

#define EA_TP_TRY(expr)                                   \
    do {                                                  \
        const cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) {                          \
            tp_free(t);                                   \
            cudaFree(staging);                            \
            return tp_cuda_fail(e_);                      \
        }                                                 \
    } while (0)

extern "C" int ea_tp_create(const ea_tp_config *cfg, void *stream, ea_tp **out)
{
    if (!cfg || !out || !cfg->bonds || !cfg->spins0 || !cfg->metro) return EA_EINVAL;
    *out = nullptr;
    const uint32_t L = cfg->L, R = cfg->n_real, NT = cfg->n_temps, C = cfg->n_copies;
    if (L < 4 || (L & 1u) || R == 0 || NT == 0 || NT > (uint32_t)ea::kTpMaxTemps || C < 1 || C > 2)
        return EA_EINVAL;
    if (!tp_supported_L(L)) return EA_EUNSUPPORTED;
    if ((uint64_t)cfg->real_base + R > (1ull << 32)) return EA_EINVAL;
    for (uint32_t t = 0; t < NT; ++t)
        if (cfg->metro[t * 3] > cfg->metro[t * 3 + 1] || cfg->metro[t * 3 + 1] > cfg->metro[t * 3 + 2])
            return EA_EINVAL;
    const uint32_t len = NT > 1 ? cfg->swap_len : 0;
    if (len > 0) {
        if (!cfg->swapt) return EA_EINVAL;
        for (uint32_t p = 0; p + 1 < NT; ++p)
            for (uint32_t k = 1; k < len; ++k)
                if (cfg->swapt[(size_t)p * len + k] > cfg->swapt[(size_t)p * len + k - 1]) return EA_EINVAL;
    }
    const size_t N = (size_t)L * L * L;
    ea_tp *t = new (std::nothrow) ea_tp();
    if (!t) return EA_ENOMEM;
    void *staging = nullptr;
    t->L = L;
    t->R = R;
    t->NT = NT;
    t->C = C;
    t->N = (uint32_t)N;
    t->W = (NT + 31) / 32;
    t->swap_len = len;
    t->stream = (cudaStream_t)stream;
    t->rk = ea::make_round_keys(cfg->seed);
    t->r_base = cfg->real_base;
    const size_t n_spin = (size_t)R * C * t->W * N, n_bond = (size_t)R * 3 * N;
    EA_TP_TRY(cudaMalloc(&t->d_spins, n_spin * 4));
    EA_TP_TRY(cudaMalloc(&t->d_bonds, n_bond * 4));
    EA_TP_TRY(cudaMalloc(&t->d_swapt, (len ? (size_t)(NT - 1) * len : 1) * 4));
    EA_TP_TRY(cudaMalloc(&t->d_nthr, (size_t)NT * 3 * 8));
    EA_TP_TRY(cudaMalloc(&t->d_energy, (size_t)R * C * ea::kLanes * t->W * 4));
    std::vector<uint64_t> nthr((size_t)NT * 3);
    for (size_t x = 0; x < nthr.size(); ++x) nthr[x] = 0ull - (uint64_t)cfg->metro[x];
    cudaStream_t st = t->stream;
    EA_TP_TRY(cudaMemcpyAsync(t->d_nthr, nthr.data(), nthr.size() * 8, cudaMemcpyHostToDevice, st));
    if (len)
        EA_TP_TRY(cudaMemcpyAsync(t->d_swapt, cfg->swapt, (size_t)(NT - 1) * len * 4,
                                  cudaMemcpyHostToDevice, st));
    EA_TP_TRY(cudaMalloc(&staging, (n_spin > n_bond ? n_spin : n_bond) * 4));
    EA_TP_TRY(cudaMemcpyAsync(staging, cfg->spins0, n_spin * 4, cudaMemcpyHostToDevice, st));
    ea::k_tp_import_spins<<<ea::tp_grid(n_spin), 256, 0, st>>>((const uint32_t *)staging, t->d_spins,
                                                                (int)L, n_spin, (int)NT, (int)t->W);
    EA_TP_TRY(cudaGetLastError());
    EA_TP_TRY(cudaMemcpyAsync(staging, cfg->bonds, n_bond, cudaMemcpyHostToDevice, st));
    ea::k_tp_import_bonds<<<ea::tp_grid(n_bond), 256, 0, st>>>((const uint8_t *)staging, t->d_bonds,
                                                                (int)L, n_bond);
    EA_TP_TRY(cudaGetLastError());
    // initial energies
    ea::TpLaunch a{};
    a.spins = t->d_spins;
    a.bonds = t->d_bonds;
    a.nthr = t->d_nthr;
    a.swapt = t->d_swapt;
    a.swap_len = len;
    a.energy = t->d_energy;
    a.R = R;
    a.NT = NT;
    a.C = C;
    a.rk = t->rk;
    a.r_base = t->r_base;
    a.W = t->W;
    EA_TP_TRY(ea::tp_launch((int)L, a, 1, st));
    t->launches = 3;
    // the staging buffer is read by the import kernels: wait before freeing it
    EA_TP_TRY(cudaStreamSynchronize(st));
    cudaFree(staging);
    staging = nullptr;
    // slot groups while R * C is small: the most groups (at most eight) that keep
    // the CTAs within one wave, at most one CTA per SM (a second wave costs more
    // than the extra groups gain: 2.40 against 1.74 ps per flip at L = 16 with
    // 32 realizations)
    int dev = 0, sms = 0;
    EA_TP_TRY(cudaGetDevice(&dev));
    EA_TP_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t k = 1;
    while (k * 2 <= 8 && k * 2 <= NT && (uint64_t)R * C * t->W * (k * 2) <= (uint64_t)sms) k *= 2;
    const int rc = tp_apply_split(t, k);
    if (rc != EA_OK) {
        tp_free(t);
        return rc;
    }
    *out = t;
    return EA_OK;
}
#undef EA_TP_TRY

extern "C" int ea_tp_sweep(ea_tp *t, uint32_t n_sweeps, uint32_t swap_every, int32_t *energy_log,
                           uint32_t *swap_log)
{
    if (!t) return EA_EINVAL;
    if (n_sweeps == 0) return EA_OK;
    ea::TpLaunch a{};
    a.spins = t->d_spins;
    a.bonds = t->d_bonds;
    a.nthr = t->d_nthr;
    a.swapt = t->d_swapt;
    a.swap_len = t->swap_len;
    a.energy = t->d_energy;
    a.R = t->R;
    a.NT = t->NT;
    a.C = t->C;
    a.rk = t->rk;
    a.r_base = t->r_base;
    a.W = t->W;
    if (t->nsplit <= 1) {
        // one CTA per unit: sweeps and swap passes of the whole call in one launch
        a.s0 = t->sweep;
        a.n_sweeps = n_sweeps;
        a.swap_every = swap_every;
        a.P0 = t->pass;
        a.pass_local0 = 0;
        a.energy_log = energy_log;
        a.swap_log = swap_log;
        const cudaError_t e = ea::tp_launch((int)t->L, a, 0, t->stream);
        if (e != cudaSuccess) return tp_cuda_fail(e);
        ++t->launches;
        uint64_t passes = 0;
        if (swap_every != 0)
            passes = (t->sweep + n_sweeps) / swap_every - t->sweep / swap_every;
        t->sweep += n_sweeps;
        t->pass += passes;
        return EA_OK;
    }
    // slot groups: each interval (sweeps up to the next swap pass) is one launch
    // of nsplit CTAs per unit, then one merge launch that runs the pass
    a.slices = t->d_slices;
    a.spg = t->spg;
    a.gpw = t->gpw;
    a.nsplit = t->nsplit;
    a.swap_every = 0;
    a.swap_log = swap_log;
    const size_t row_words = (size_t)t->R * t->NT * t->C;
    const uint64_t end = t->sweep + n_sweeps;
    uint64_t s = t->sweep;
    uint32_t row = 0, pass_local = 0;
    while (s < end) {
        uint64_t last = end - 1;
        bool sw = false;
        if (swap_every != 0) {
            const uint64_t nxt = (s / swap_every + 1) * swap_every - 1;
            if (nxt < end) {
                last = nxt;
                sw = true;
            }
        }
        const uint32_t n_int = (uint32_t)(last - s + 1);
        a.s0 = s;
        a.n_sweeps = n_int;
        a.energy_log = energy_log ? energy_log + (size_t)row * row_words : nullptr;
        cudaError_t e = ea::tp_launch((int)t->L, a, 0, t->stream);
        if (e != cudaSuccess) return tp_cuda_fail(e);
        const int do_swap = sw && t->NT > 1;
        int32_t *elog_row = (energy_log && do_swap) ? energy_log + (size_t)(row + n_int - 1) * row_words : nullptr;
        ea::k_tp_merge<<<t->R * t->C, 256, 0, t->stream>>>(a, (int)t->N, do_swap, t->pass, pass_local, elog_row);
        e = cudaGetLastError();
        if (e != cudaSuccess) return tp_cuda_fail(e);
        t->launches += 2;
        if (sw) {
            ++t->pass;
            ++pass_local;
        }
        s += n_int;
        row += n_int;
    }
    t->sweep = end;
    return EA_OK;
}

extern "C" int ea_tp_set_split(ea_tp *t, uint32_t k)
{
    if (!t || k == 0 || k > 32 || (k & (k - 1)) != 0 || k > t->NT) return EA_EINVAL;   // k <= min(NT, 32)
    return tp_apply_split(t, k);
}

extern "C" int ea_tp_read(ea_tp *t, uint32_t *spins, int32_t *energies)
{
    if (!t) return EA_EINVAL;
    if (spins) {
        const size_t total = (size_t)t->R * t->C * t->W * t->N;
        ea::k_tp_export_spins<<<ea::tp_grid(total), 256, 0, t->stream>>>(t->d_spins, spins, (int)t->L, total);
        ++t->launches;
    }
    if (energies) {
        const size_t total = (size_t)t->R * t->NT * t->C;
        ea::k_tp_export_energy<<<ea::tp_grid(total), 256, 0, t->stream>>>(t->d_energy, energies, t->R,
                                                                           t->NT, t->C, t->W);
        ++t->launches;
    }
    return cudaGetLastError() == cudaSuccess ? EA_OK : EA_ECUDA;
}

extern "C" int ea_tp_info(const ea_tp *t, uint64_t *sweep_index, uint64_t *pass_index, uint64_t *launches,
                          uint32_t *split)
{
    if (!t) return EA_EINVAL;
    if (split) *split = t->nsplit;
    if (sweep_index) *sweep_index = t->sweep;
    if (pass_index) *pass_index = t->pass;
    if (launches) *launches = t->launches;
    return EA_OK;
}

namespace ea {

void tp_set_stream(ea_tp *t, cudaStream_t st) { t->stream = st; }

size_t tp_device_bytes(const ea_tp_config *cfg)
{
    const size_t N = (size_t)cfg->L * cfg->L * cfg->L, R = cfg->n_real, C = cfg->n_copies;
    const size_t W = (cfg->n_temps + 31) / 32, NT = cfg->n_temps;
    const size_t n_spin = R * C * W * N, n_bond = R * 3 * N;
    const size_t len = NT > 1 ? cfg->swap_len : 0;
    return n_spin * 4 + n_bond * 4 + (len ? (NT - 1) * len : 1) * 4 + NT * 3 * 8 + R * C * kLanes * W * 4 +
           (n_spin > n_bond ? n_spin : n_bond) * 4 +       // import staging
           W * 8 * R * C * N * 4;                           // slot-group slices
}

}  // namespace ea

extern "C" void ea_tp_destroy(ea_tp *t)
{
    if (!t) return;
    cudaStreamSynchronize(t->stream);
    tp_free(t);
}
