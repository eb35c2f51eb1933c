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
constexpr uint32_t kWaveSuspendNs = 2000;  // suspend-time hint of the field kernel's polls
constexpr int kWaveWaitLimitHint = 1 << 22;   // its polls before giving up (<= 8.4 s)

// Shared-memory layout of the wavefront kernel, in 32-bit words.
struct WaveLayout {
    size_t s, js, eo, cur, bar_e, bar_h, bar_r, bar_d, abort, tsw, hist, words;
    // overlaps: the copy-pair rendezvous barriers and the q histogram of the
    // slots this CTA measures (t = c mod 2)
    __host__ __device__ WaveLayout(int N, int NT, uint32_t swap_len, bool swap_smem, bool field = false,
                                   bool overlaps = false)
    {
        const int nw = (NT + 1) / 2, rec = field ? 3 : 1;   // Et (and E, M in a field)
        const int sn = field ? 3 * N / 2 : N;     // words of a lattice: [c0][c1] ([c0][c1][c0'] in a field)
        size_t o = 0;
        s = o; o += (size_t)NT * sn;              // [NT][sn] spins by slot
        js = o; o += (size_t)3 * sn;              // [3][sn] bonds
        eo = o; o += (size_t)rec * NT * kLanes;   // slot 2k after the sweep, for warp k-1
        cur = o; o += (size_t)rec * nw * kLanes;  // the carried configuration, warp k to warp k+1
        o = (o + 1) & ~(size_t)1;                 // 8-byte alignment of the barriers
        bar_e = o; o += 2 * (size_t)nw;           // mbarrier k: E_{2k+2} of warp k+1 is published
        bar_h = o; o += 2 * (size_t)nw;           // mbarrier k: warp k applied its pass steps
        bar_r = o; o += overlaps ? 2 * (size_t)nw : 0;   // mbarrier k: the partner's warp k slots are final
        bar_d = o; o += overlaps ? 2 * (size_t)nw : 0;   // mbarrier k: the partner read my warp k slot
        abort = o; o += 1;
        tsw = o; o += swap_smem && NT > 1 ? (size_t)(NT - 1) * swap_len : 0;
        hist = o; o += overlaps ? (size_t)nw * (N + 1) : 0;
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
// The same with a suspend-time hint: the waiting warp sleeps until the phase
// completes or hint_ns pass, instead of polling at the hardware's default
// interval.  The field kernel gains from it (~2 %); the field-free one, whose
// waits are shorter, measured ~2 % slower with it and polls without.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
                 : "memory");
    return ok != 0;
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

// Arrive (release at cluster scope) on the barrier at the same offset in the
// shared memory of CTA `rank` of the cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint64_t *bar, uint32_t rank)
{
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(smem_addr(bar)), "r"(rank));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(ra) : "memory");
}
// try_wait that also acquires the partner CTA's writes made before its arrive.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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
__device__ __forceinline__ void wave_release(uint32_t *base, int NT, bool field)
{
    const WaveLayout lay(8 * 8 * 8, NT, 0, false, field);
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
// HINT: sleep up to kWaveSuspendNs per poll (at most kWaveWaitLimitHint polls).
// Without the hint the abort flag is read every 32nd poll: the polls of the
// field-free kernel's short waits then cost fewer issue slots (0.0937 ->
// 0.0912 ps/flip on the bench ensemble); with it, every poll (the field kernel
// measured slower with the sparse check).
template <bool HINT = false>
__device__ __forceinline__ bool wave_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort, int *err)
{
    for (int it = 0; it < (HINT ? kWaveWaitLimitHint : kWaveWaitLimit); ++it) {
        if (HINT ? mbar_try_wait_hint(bar, parity, kWaveSuspendNs) : mbar_try_wait(bar, parity)) return true;
        if ((HINT || (it & 31) == 31) && *abort != 0u) return false;
    }
    *abort = 1u;
    atomicExch(err, 1);
    return false;
}
// The same for a barrier the partner CTA of the cluster arrives on (the abort
// flag read every 32nd poll, as for the field-free waits above).
__device__ __forceinline__ bool wave_wait_cluster(uint64_t *bar, uint32_t parity, volatile uint32_t *abort,
                                                  int *err)
{
    for (int it = 0; it < kWaveWaitLimit; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 31) == 31 && *abort != 0u) return false;
    }
    *abort = 1u;
    atomicExch(err, 1);
    return false;
}

// (a & ~m) | (b & m): one LOP3.
__device__ __forceinline__ uint32_t mux(uint32_t a, uint32_t b, uint32_t m) { return lop3<0xD8u>(a, b, m); }
static_assert((((0xF0u & ~0xAAu) | (0xCCu & 0xAAu)) & 0xFFu) == 0xD8u, "mux truth table");

// Per-quad constants of the lane: shared-window byte addresses of the words
// the quad reads (the colour and direction of each word are immediate offsets
// from these), and the parts of the first two Philox rounds that depend on
// the quad's counter word q = k0 / 4 and the group only.
struct WaveQuad {
    uint32_t s, yp, ym, zp, zm;     // lattice + k0, + yp, + ym, + zp, + zm
    uint32_t j, jym, jzm;           // bonds + k0, + ym, + zm
    uint32_t plo0, plo1, phi1;      // M0 q, M1 n, umulhi(M1, n) with n = umulhi(M0, q) ^ g ^ key1
};

__device__ __forceinline__ WaveQuad wave_quad_setup(const uint32_t *mine, const uint32_t *Js, const QuadRow &d,
                                                    uint32_t gr, const RoundKeys &rk)
{
    WaveQuad w;
    const uint32_t sb = smem_addr(mine), jb = smem_addr(Js);
    w.s = sb + 4u * (uint32_t)d.k0;
    w.yp = sb + 4u * (uint32_t)d.yp;
    w.ym = sb + 4u * (uint32_t)d.ym;
    w.zp = sb + 4u * (uint32_t)d.zp;
    w.zm = sb + 4u * (uint32_t)d.zm;
    w.j = jb + 4u * (uint32_t)d.k0;
    w.jym = jb + 4u * (uint32_t)d.ym;
    w.jzm = jb + 4u * (uint32_t)d.zm;
    const uint32_t q = (uint32_t)d.k0 >> 2;
    w.plo0 = kM0 * q;
    const uint32_t n = __umulhi(kM0, q) ^ gr ^ rk.k[1];
    w.plo1 = kM1 * n;
    w.phi1 = __umulhi(kM1, n);
    return w;
}

// Rounds 2..9 of Philox4x32-10 from the state after round 1.
__device__ __forceinline__ uint4 philox_from2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const RoundKeys &rk)
{
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint32_t lo0 = kM0 * c0, hi0 = __umulhi(kM0, c0);
        const uint32_t lo1 = kM1 * c2, hi1 = __umulhi(kM1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ rk.k[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk.k[2 * r + 1];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Shared-memory vector load and store at a byte address plus an immediate.
// The loads are not volatile (the scheduler may move them); `dep`, an opaque
// zero made after the last barrier, keeps them from being moved above it.
template <int OFF>
__device__ __forceinline__ uint4 lds4(uint32_t addr, uint32_t dep)
{
    uint4 v;
    asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4+%5];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "r"(addr), "n"(OFF), "r"(dep));
    return v;
}
template <int OFF>
__device__ __forceinline__ void sts4(uint32_t addr, uint4 v)
{
    asm volatile("st.shared.v4.u32 [%0+%1], {%2, %3, %4, %5};" ::"r"(addr), "n"(OFF), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w));
}
__device__ __forceinline__ uint32_t opaque_zero()
{
    uint32_t z;
    asm volatile("mov.u32 %0, 0;" : "=r"(z));
    return z;
}

// Metropolis update of one quad of colour COL with x parity PX (L = 8).
template <int COL, int PX, bool WITH_E, int Q, typename Acc>
__device__ __forceinline__ void wave_quad(const WaveQuad &q, uint4 r, uint64_t t0, uint64_t t1, uint64_t t2,
                                          Acc &acc, uint32_t dep)
{
    constexpr int H4 = 256 * 4, N4 = 512 * 4;           // bytes of a colour half and of a bond direction
    constexpr int C4 = COL * H4, O4 = (1 - COL) * H4;
    const uint4 own = lds4<C4>(q.s, dep), xo = lds4<O4>(q.s, dep);
    const uint4 vyp = lds4<O4>(q.yp, dep), vym = lds4<O4>(q.ym, dep);
    const uint4 vzp = lds4<O4>(q.zp, dep), vzm = lds4<O4>(q.zm, dep);
    const uint4 jcx = lds4<C4>(q.j, dep), jcy = lds4<N4 + C4>(q.j, dep), jcz = lds4<2 * N4 + C4>(q.j, dep);
    const uint4 jox = lds4<O4>(q.j, dep), joy = lds4<N4 + O4>(q.jym, dep), joz = lds4<2 * N4 + O4>(q.jzm, dep);
    const uint32_t xe_s = PX ? xo.x : xo.w;             // x neighbour across the row's edge (R = 4)
    sts4<C4>(q.s, quad_core<PX, WITH_E, Q>(own, xo, vyp, vym, vzp, vzm, jcx, jcy, jcz, jox, joy, joz, xe_s,
                                            jox.w, r, t0, t1, t2, acc));
}

// Half-sweep of colour COL over the lane's four quads (quad j: row parity
// j >> 1, x parity ((j >> 1) + COL) & 1).  The sweep- and colour-only parts
// of the first two Philox rounds are formed once; the uniforms of the next
// quad are drawn while the current one is updated.  With WITH_E, acc
// receives the lane's sum of the post-update counts u' of its 16 sites (a
// carry-save counter over the four quads, resolved at the end).
template <int COL, bool WITH_E, int PL>
__device__ __forceinline__ void wave_half(const WaveQuad (&wq)[4], uint32_t s, uint32_t ctag,
                                          const RoundKeys &rk, uint64_t t0, uint64_t t1, uint64_t t2,
                                          uint32_t (&acc)[PL])
{
    const uint32_t dep = opaque_zero();
    const uint32_t lo1 = kM1 * s, n0 = __umulhi(kM1, s) ^ ctag ^ rk.k[0];
    const uint32_t lo0b = kM0 * n0, hi0b = __umulhi(kM0, n0);
    auto draw = [&](const WaveQuad &q) {
        return philox_from2(q.phi1 ^ lo1 ^ rk.k[2], q.plo1, hi0b ^ q.plo0 ^ rk.k[3], lo0b, rk);
    };
    CountAcc cs;
    cs.clear();
    uint4 r0 = draw(wq[0]);
    uint4 r1 = draw(wq[1]);
    wave_quad<COL, COL, WITH_E, 0>(wq[0], r0, t0, t1, t2, cs, dep);
    r0 = draw(wq[2]);
    wave_quad<COL, COL, WITH_E, 1>(wq[1], r1, t0, t1, t2, cs, dep);
    r1 = draw(wq[3]);
    wave_quad<COL, 1 - COL, WITH_E, 2>(wq[2], r0, t0, t1, t2, cs, dep);
    wave_quad<COL, 1 - COL, WITH_E, 3>(wq[3], r1, t0, t1, t2, cs, dep);
    if constexpr (WITH_E) cs.resolve<4>(acc);
}

// External field h = h_num / h_den (Eq. 1 with the field term; the field runs
// of Sec. 5), for fields whose always-accept boundary is u >= UA0 for spin
// value S = -1 and u >= UA1 for S = +1 with {UA0, UA1} = {3, 4} (0 < |h| < 2).
// A spin flips iff r < T[S][u]; below the boundary the thresholds are
// non-decreasing in u, so the masks m[k] = [r < T[k]] are nested and the
// flip mask of one spin value follows from the partial sums (a, b) of the
// six unsatisfied-bond bits in a few LOP3s:
//   UA = 3: [u>=3] | m2 [u>=2] | m1 [u>=1] | m0
//         = maj(a1, b1, a0 | b0 | m2) | (m2 & maj(a0, b0, m1)) | m0
//   UA = 4: [u>=4] | m3 [u>=3] | m2 [u>=2] | m1 [u>=1] | m0
//         = maj(a1, b1, maj(a0, b0, m3)) | (m2 & (a1 | b1 | maj(a0, b0, m1))) | m0
template <int UA>
__device__ __forceinline__ uint32_t field_mask(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1,
                                               const uint32_t (&m)[UA])
{
    if constexpr (UA == 3) {
        const uint32_t v = lop3<kOr3>(a0, b0, m[2]);
        return lop3<kOr3>(lop3<kMaj3>(a1, b1, v), m[2] & lop3<kMaj3>(a0, b0, m[1]), m[0]);
    } else {
        static_assert(UA == 4, "always-accept boundary 3 or 4");
        const uint32_t z = lop3<kMaj3>(a0, b0, m[3]);
        const uint32_t w = lop3<kOr3>(a1, b1, lop3<kMaj3>(a0, b0, m[1]));
        return lop3<kOr3>(lop3<kMaj3>(a1, b1, z), m[2] & w, m[0]);
    }
}

// Up-spin counts: the four quads of one half-sweep (<= 16) and their sum over
// the sweep's two halves (<= 32).
constexpr int kPlanesM = 6;
constexpr int kPlanesHalfM = 5;
using HalfUpAcc = CsaAcc<1, kPlanesHalfM>;

// In a field one body serves both colours, so that the code of a sweep fits
// the instruction cache (two colour-specialised copies of the field update
// did not: their fetch stalls cost about a fifth of the kernel's time).  A
// slot's lattice is held as [c0][c1][c0'] and each bond direction as
// [c0][c1][c0'] (H words each), c0' a copy of colour 0 that the colour-0
// half-sweep writes beside c0.  For colour col the quad's own words lie
// col * H words beyond its colour-0 addresses and the other colour's words H
// words beyond its own, so both colours load with the same immediate
// offsets.  The x parity of the quad's sites is chosen at run time: with v the
// other colour's row words rotated left by px, the +x neighbours are v and
// the -x neighbours v rotated right (likewise the -x bonds).
constexpr uint32_t kWaveH4 = 256u * 4u;        // bytes of a colour half (L = 8)
constexpr int kWaveFieldD4 = 3 * 256 * 4;      // bytes of a bond direction in the field layout

// v rotated left by one word where pm is all ones (one LOP3 a word).
__device__ __forceinline__ uint4 rot_left_if(uint32_t pm, uint4 v)
{
    return make_uint4(mux(v.x, v.y, pm), mux(v.y, v.z, pm), mux(v.z, v.w, pm), mux(v.w, v.x, pm));
}

// Metropolis update of one quad in the field (L = 8), colour `col` (d =
// col * H bytes): the flip mask per spin value from field_mask, selected per
// lane by the spin bit; WITH_E adds the post-update unsatisfied-bond counts to
// ce in colour 1 (as quad Q of the half), WITH_M the new spins to cm.
template <bool WITH_E, bool WITH_M, int UA0, int UA1, int Q>
__device__ __forceinline__ void wave_quad_field(const WaveQuad &q, uint32_t d, uint32_t px, bool col0, uint4 r,
                                                const uint64_t (&n0)[UA0], const uint64_t (&n1)[UA1],
                                                CountAcc &ce, HalfUpAcc &cm, uint32_t dep)
{
    constexpr int H4 = (int)kWaveH4, D4 = kWaveFieldD4;
    const uint32_t sa = q.s + d, ja = q.j + d;
    const uint4 own = lds4<0>(sa, dep), xo = lds4<H4>(sa, dep);
    const uint4 vyp = lds4<H4>(q.yp + d, dep), vym = lds4<H4>(q.ym + d, dep);
    const uint4 vzp = lds4<H4>(q.zp + d, dep), vzm = lds4<H4>(q.zm + d, dep);
    const uint4 jcx = lds4<0>(ja, dep), jcy = lds4<D4>(ja, dep), jcz = lds4<2 * D4>(ja, dep);
    const uint4 jox = lds4<H4>(ja, dep), joy = lds4<D4 + H4>(q.jym + d, dep);
    const uint4 joz = lds4<2 * D4 + H4>(q.jzm + d, dep);
    const uint4 v = rot_left_if(px, xo), w = rot_left_if(px, jox);
    const uint32_t nxp[4] = {v.x, v.y, v.z, v.w}, nxm[4] = {v.w, v.x, v.y, v.z};
    const uint32_t jxm[4] = {w.w, w.x, w.y, w.z};
    const uint32_t sv[4] = {own.x, own.y, own.z, own.w};
    const uint32_t jx[4] = {jcx.x, jcx.y, jcx.z, jcx.w};
    const uint32_t ny[4] = {vyp.x, vyp.y, vyp.z, vyp.w}, my[4] = {vym.x, vym.y, vym.z, vym.w};
    const uint32_t nz[4] = {vzp.x, vzp.y, vzp.z, vzp.w}, mz[4] = {vzm.x, vzm.y, vzm.z, vzm.w};
    const uint32_t jy[4] = {jcy.x, jcy.y, jcy.z, jcy.w}, jym[4] = {joy.x, joy.y, joy.z, joy.w};
    const uint32_t jz[4] = {jcz.x, jcz.y, jcz.z, jcz.w}, jzm[4] = {joz.x, joz.y, joz.z, joz.w};
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    uint32_t ns[4], A0[4], A1[4], B0[4], B1[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t sj = sv[j];
        const uint32_t e0 = lop3<kXor3>(sj, nxp[j], jx[j]);
        const uint32_t e1 = lop3<kXor3>(sj, nxm[j], jxm[j]);
        const uint32_t e2 = lop3<kXor3>(sj, ny[j], jy[j]);
        const uint32_t e3 = lop3<kXor3>(sj, my[j], jym[j]);
        const uint32_t e4 = lop3<kXor3>(sj, nz[j], jz[j]);
        const uint32_t e5 = lop3<kXor3>(sj, mz[j], jzm[j]);
        const uint32_t a0 = lop3<kXor3>(e0, e1, e2), a1 = lop3<kMaj3>(e0, e1, e2);
        const uint32_t b0 = lop3<kXor3>(e3, e4, e5), b1 = lop3<kMaj3>(e3, e4, e5);
        uint32_t m0[UA0], m1[UA1];
#pragma unroll
        for (int u = 0; u < UA0; ++u) m0[u] = below_mask(rr[j], n0[u]);
#pragma unroll
        for (int u = 0; u < UA1; ++u) m1[u] = below_mask(rr[j], n1[u]);
        const uint32_t F0 = field_mask<UA0>(a0, a1, b0, b1, m0), F1 = field_mask<UA1>(a0, a1, b0, b1, m1);
        ns[j] = lop3<kSelNot>(sj, F1, F0);              // s ^ f with f = S > 0 ? F1 : F0
        A0[j] = a0;
        A1[j] = a1;
        B0[j] = b0;
        B1[j] = b1;
    }
    const uint4 nsv = make_uint4(ns[0], ns[1], ns[2], ns[3]);
    sts4<0>(sa, nsv);
    if (col0) sts4<2 * H4>(sa, nsv);                   // colour 0 also refreshes its copy c0'
    if constexpr (WITH_E) {
        if (!col0) {
            uint32_t x[3][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t f = sv[j] ^ ns[j];
                const uint32_t u0 = A0[j] ^ B0[j], c0 = A0[j] & B0[j];
                const uint32_t u1 = lop3<kXor3>(A1[j], B1[j], c0), u2 = lop3<kMaj3>(A1[j], B1[j], c0);
                x[0][j] = u0;
                x[1][j] = lop3<kXorAndN>(u1, f, u0);
                x[2][j] = lop3<kXorAndN>(u2, f, u0 & u1);
            }
            ce.template add<Q>(x);
        }
    }
    if constexpr (WITH_M) {
        const uint32_t up[1][4] = {{ns[0], ns[1], ns[2], ns[3]}};
        cm.template add<Q>(up);
    }
}

// Half-sweep of colour col in the field.  With WITH_E, colour 1 writes the
// lane's post-update counts of its 16 sites to acc (colour 0 leaves acc as it
// is); with WITH_M, up receives the up-spin count of its 16 new spins.
template <bool WITH_E, bool WITH_M, int UA0, int UA1>
__device__ __forceinline__ void wave_half_field(const WaveQuad (&wq)[4], int col, uint32_t s, uint32_t ctag,
                                                const RoundKeys &rk, const uint64_t (&n0)[UA0],
                                                const uint64_t (&n1)[UA1], uint32_t (&acc)[7],
                                                uint32_t (&up)[kPlanesHalfM])
{
    const uint32_t dep = opaque_zero();
    const uint32_t lo1 = kM1 * s, n0r = __umulhi(kM1, s) ^ ctag ^ rk.k[0];
    const uint32_t lo0b = kM0 * n0r, hi0b = __umulhi(kM0, n0r);
    auto draw = [&](const WaveQuad &q) {
        return philox_from2(q.phi1 ^ lo1 ^ rk.k[2], q.plo1, hi0b ^ q.plo0 ^ rk.k[3], lo0b, rk);
    };
    const bool col0 = col == 0;
    const uint32_t d = col0 ? 0u : kWaveH4;
    const uint32_t pxa = col0 ? 0u : ~0u;              // x parity of quads 0, 1 (row parity 0); 2, 3 the other
    CountAcc ce;
    ce.clear();
    HalfUpAcc cm;
    cm.clear();
    uint4 r0 = draw(wq[0]);
    uint4 r1 = draw(wq[1]);
    wave_quad_field<WITH_E, WITH_M, UA0, UA1, 0>(wq[0], d, pxa, col0, r0, n0, n1, ce, cm, dep);
    r0 = draw(wq[2]);
    wave_quad_field<WITH_E, WITH_M, UA0, UA1, 1>(wq[1], d, pxa, col0, r1, n0, n1, ce, cm, dep);
    r1 = draw(wq[3]);
    wave_quad_field<WITH_E, WITH_M, UA0, UA1, 2>(wq[2], d, ~pxa, col0, r0, n0, n1, ce, cm, dep);
    wave_quad_field<WITH_E, WITH_M, UA0, UA1, 3>(wq[3], d, ~pxa, col0, r1, n0, n1, ce, cm, dep);
    if constexpr (WITH_E) {
        if (!col0) ce.resolve<4>(acc);
    }
    if constexpr (WITH_M) cm.resolve<4>(up);
}

// Adds a half-sweep's up-spin count (5 planes) to the sweep's (6 planes).
__device__ __forceinline__ void add_up_planes(uint32_t (&acc)[kPlanesM], const uint32_t (&up)[kPlanesHalfM])
{
    uint32_t cy = 0u;
#pragma unroll
    for (int p = 0; p < kPlanesHalfM; ++p) {
        const uint32_t x = acc[p];
        acc[p] = lop3<kXor3>(x, up[p], cy);
        cy = lop3<kMaj3>(x, up[p], cy);
    }
    acc[kPlanesHalfM] ^= cy;
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
        // planes 0 .. PL + lv - 1 hold the partial sums; the next one is zero
        // in both lanes and receives only the carry
        uint32_t cy = 0;
#pragma unroll
        for (int p = 0; p < PL + lv; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, v[p], 1 << lv);
            uint32_t s2, c2;
            full_add(v[p], o, cy, s2, c2);
            v[p] = s2;
            cy = c2;
        }
        v[PL + lv] = cy;
    }
    const int t = lane & 15;
    uint32_t x = 0;
#pragma unroll
    for (int p = 0; p < PT; ++p) x = (t == p) ? v[p] : x;
    const uint32_t y = warp_transpose(x, lane);
    UA = (int)(y & 0xFFFFu);
    UB = (int)(y >> 16);
}

// Number of leading entries of a non-increasing threshold row above r (the
// acceptance bound of Sec. 2.4 with the table of Sec. 4.3.2 is -4 times it).
// Entry k-1 is floor(exp(-4k dbeta) 2^32), so the count is close to
// log2(2^32 / (r + 1)) / (32 - log2 row[0]); `slope` holds the reciprocal of
// that denominator.  The estimate is then corrected by stepping along the row
// until the defining inequalities hold, so the result is exact whatever the
// rounding of the estimate (usually no step or one).
__device__ __forceinline__ uint32_t count_above(const uint32_t *row, uint32_t len, uint32_t r, float slope)
{
    const float g = (32.0f - __log2f((float)r + 1.0f)) * slope;
    uint32_t k = g < (float)len ? (uint32_t)g : len;    // also catches an infinite slope
    while (k < len && row[k] > r) ++k;
    while (k > 0 && row[k - 1] <= r) --k;
    return k;
}

__device__ __forceinline__ float count_slope(const uint32_t *row, uint32_t len)
{
    if (len == 0 || row[0] == 0u) return 0.0f;
    return 1.0f / (32.0f - __log2f((float)row[0]));    // +inf when row[0] rounds to 2^32
}

// Acceptance bounds of the warp's pairs 2k and 2k+1 in pass P for the
// realization of this lane (Sec. 2.4 with the integer table of Sec. 4.3.2):
// pair p is accepted iff E_p - E_{p+1} >= bound (in a field: Et_p - Et_{p+1},
// the table in units of `step`; without one step = 4).  Lanes 0-7 draw the Philox
// blocks of pair 2k (realizations 4q..4q+3 from lane q), lanes 8-15 those of
// pair 2k+1; each lane then counts both rows for its own uniforms.
__device__ __forceinline__ void wave_bounds(const uint32_t *rowa, const uint32_t *rowb, uint32_t len, float sa,
                                            float sb, int k, int c, uint64_t P, uint32_t gr,
                                            const RoundKeys &rk, int lane, int step, int &bA, int &bB)
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
    bA = -step * (int)count_above(rowa, len, ra, sa);
    bB = -step * (int)count_above(rowb, len, rb, sb);
}

// Number of sites where the two copies of one slot differ (the overlap of
// Sec. 5: q = 1 - 2 n / N), per realization: lane b receives the count of
// realization b.  A4 is the slot in this CTA, B4 the same slot of the other
// copy (distributed shared memory).  Each lane XORs four 16-byte words of both
// copies, counts its 16 difference words in a carry-save counter, and the warp
// sums the counters with a butterfly of bit-sliced adders.
__device__ __forceinline__ int wave_overlap(const uint4 *A4, const uint4 *B4, int lane)
{
    CsaAcc<1, 5> cd;
    cd.clear();
#define EA_OVQ(Q)                                                                                  \
    {                                                                                              \
        const uint4 x = A4[lane + 32 * (Q)], y = B4[lane + 32 * (Q)];                              \
        const uint32_t d[1][4] = {{x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w}};                   \
        cd.add<Q>(d);                                                                              \
    }
    EA_OVQ(0) EA_OVQ(1) EA_OVQ(2) EA_OVQ(3)
#undef EA_OVQ
    uint32_t pl[5], v[10];
    cd.resolve<4>(pl);
#pragma unroll
    for (int p = 0; p < 10; ++p) v[p] = p < 5 ? pl[p] : 0u;
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
        uint32_t cy = 0;
#pragma unroll
        for (int p = 0; p < 5 + lv; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, v[p], 1 << lv);
            uint32_t s2, c2;
            full_add(v[p], o, cy, s2, c2);
            v[p] = s2;
            cy = c2;
        }
        v[5 + lv] = cy;
    }
    int nd = 0;
#pragma unroll
    for (int p = 0; p < 10; ++p) nd |= (int)((v[p] >> lane) & 1u) << p;
    return nd;
}

// LOG = false compiles the body without the energy and swap logs (their
// pointers must then be null).  FLD = 0 runs the field-free method; FLD = 34
// (43) the external field with always-accept boundaries u >= 3 (4) for S = -1
// and u >= 4 (3) for S = +1: decisions of the pass on Et = h_den E - h_num M,
// magnetisations M counted beside the energies.  MEAS (field-free only): 0 no
// measurement; 1 energy sums of the measured sweeps (esum); 2 also the q
// histogram (C = 2, the two copies of a group in one 2-CTA cluster): after its
// pass of a measured sweep, warp k of each copy meets warp k of the other copy
// (cluster-scope mbarriers: "my slots are final"), counts the overlap of slot
// 2k + c from its own words and the other copy's (distributed shared memory),
// signals that it has read them, and waits for the same signal before it
// next writes its own slots.
template <bool LOG, int FLD = 0, int MEAS = 0>
__device__ __forceinline__ void unit_wave_body(uint32_t *const base, const SweepLaunch &a, uint32_t unit,
                                               int swap_in_smem)
{
    constexpr int L = 8;
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    constexpr bool F = FLD != 0;
    constexpr int UA0 = FLD == 43 ? 4 : 3, UA1 = FLD == 34 ? 4 : 3;
    constexpr int PL = planes_for(24 * 4);          // counter planes of four quads (<= 96)
    constexpr int PLM = planes_for(32);             // up spins of eight quads (<= 32)
    static_assert(PL == 7 && PLM == kPlanesM, "counter planes of the carry-save counters");
    int32_t *const energy_log = LOG ? a.energy_log : nullptr;
    uint32_t *const swap_log = LOG ? a.swap_log : nullptr;
    const int NT = (int)a.NT;
    static_assert(MEAS == 0 || FLD == 0, "measurement in the field-free form only");
    const WaveLayout lay(N, NT, a.swap_len, swap_in_smem != 0, F, MEAS == 2);
    uint32_t *S = base + lay.s;
    uint32_t *Js = base + lay.js;
    int *Eo = reinterpret_cast<int *>(base + lay.eo);          // [3][NT][32]: Et, E, M of slot 2k
    int *Cur = reinterpret_cast<int *>(base + lay.cur);        // [3][nw][32]: the carry's Et, E, M
    uint64_t *bar_e = reinterpret_cast<uint64_t *>(base + lay.bar_e);
    uint64_t *bar_h = reinterpret_cast<uint64_t *>(base + lay.bar_h);
    volatile uint32_t *abort = base + lay.abort;
    const int nw = (NT + 1) / 2;

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
    constexpr int SN = F ? 3 * N / 2 : N;               // words of a slot's lattice in shared memory
    if constexpr (F) {
        // [c0][c1] of each slot; c0' is written by the first colour-0 half-sweep
        for (int w = tid; w < NT * N / 4; w += nthr)
            reinterpret_cast<uint4 *>(S)[(w / (N / 4)) * (SN / 4) + w % (N / 4)] =
                __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
        // [c0][c1][c0'] of each bond direction
        for (int w = tid; w < 3 * N / 4; w += nthr) {
            const uint4 v = reinterpret_cast<const uint4 *>(gJ)[w];
            const int dir = w / (N / 4), o = w % (N / 4);
            reinterpret_cast<uint4 *>(Js)[dir * (SN / 4) + o] = v;
            if (o < N / 8) reinterpret_cast<uint4 *>(Js)[dir * (SN / 4) + N / 4 + o] = v;
        }
    } else {
        for (int w = tid; w < NT * N / 4; w += nthr)
            reinterpret_cast<uint4 *>(S)[w] = __ldcg(reinterpret_cast<const uint4 *>(gS) + w);
        for (int w = tid; w < 3 * N / 4; w += nthr)
            reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
    }
    const uint32_t *swt = a.swapt;
    if (swap_in_smem) {
        uint32_t *Tsw = base + lay.tsw;
        for (int w = tid; w < (NT - 1) * (int)a.swap_len; w += nthr) Tsw[w] = a.swapt[w];
        swt = Tsw;
    }
    for (int i = tid; i < nw; i += nthr) {
        mbar_init(&bar_e[i], kLanes);
        mbar_init(&bar_h[i], kLanes);
    }
    uint64_t *bar_r = reinterpret_cast<uint64_t *>(base + lay.bar_r);
    uint64_t *bar_d = reinterpret_cast<uint64_t *>(base + lay.bar_d);
    uint32_t *hist = base + lay.hist;                   // [nw][N + 1]: slot 2k + c
    const uint32_t *S_other = nullptr;                  // the other copy's lattices (MEAS == 2)
    if constexpr (MEAS == 2) {
        for (int i = tid; i < nw; i += nthr) {
            mbar_init(&bar_r[i], kLanes);
            mbar_init(&bar_d[i], kLanes);
        }
        for (int i = tid; i < nw * (N + 1); i += nthr) hist[i] = 0u;
        S_other = cg::this_cluster().map_shared_rank(S, (unsigned int)(c ^ 1));
    }
    if (tid == 0) *abort = 0u;
    // Metropolis thresholds of my slot as 2^64 - T (see below_mask)
    uint64_t t0 = 0, t1 = 0, t2 = 0;
    uint64_t n0[UA0], n1[UA1];
    if constexpr (F) {
#pragma unroll
        for (int u = 0; u < UA0; ++u) n0[u] = 0ull - a.metro_f[((size_t)ls * 2 + 0) * 7 + u];
#pragma unroll
        for (int u = 0; u < UA1; ++u) n1[u] = 0ull - a.metro_f[((size_t)ls * 2 + 1) * 7 + u];
    } else {
        t0 = 0ull - (uint64_t)a.metro[ls * 3 + 0];
        t1 = 0ull - (uint64_t)a.metro[ls * 3 + 1];
        t2 = 0ull - (uint64_t)a.metro[ls * 3 + 2];
    }
    uint32_t *mine = S + (size_t)ls * SN;
    WaveQuad wq[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wq[j] = wave_quad_setup(mine, Js, quad_row<L>(j >> 1, li + 16 * (j & 1)), gr, a.rk);
    const uint32_t tag0 = ((uint32_t)c << 8) | (uint32_t)ls;
    const uint32_t tag1 = (1u << 16) | tag0;
    const uint32_t len = a.swap_len;
    const int step = F ? a.step : 4;
    const int hn = a.h_num, hd = a.h_den;
    if constexpr (MEAS == 2)
        cg::this_cluster().sync();   // both copies staged, their barriers initialised
    else
        __syncthreads();   // staged lattices, bonds, table and flags are complete; no CTA barrier after this
    if (2 * k >= NT) {                                  // warps beyond the slots (wider CTAs of a batch)
        if constexpr (MEAS == 2) cg::this_cluster().sync();
        return;
    }
    // rows of the warp's pairs 2k and 2k+1 (clamped into range; unused when the pair does not exist)
    const uint32_t *rowa = swt + (size_t)max(min(2 * k, NT - 2), 0) * len;
    const uint32_t *rowb = swt + (size_t)max(min(2 * k + 1, NT - 2), 0) * len;
    const float sa = count_slope(rowa, len), sb = count_slope(rowb, len);

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    int bA = 0, bB = 0;
    if (NT > 1 && a.swap_every != 0 && hasB)
        wave_bounds(rowa, rowb, len, sa, sb, k, c, P, gr, a.rk, lane, step, bA, bB);
    // energies (and in a field magnetisations) of slots 2k, 2k+1; lane = realization
    int EA = 0, EB = 0, MA = 0, MB = 0;
    bool ok_run = true;
    uint32_t ph_e = 0, ph_h = 0;                        // parity of the next phase this warp waits for
    uint32_t ph_r = 0, ph_d = 0;                        // (MEAS == 2) the copy-pair rendezvous
    bool pend_d = false;                                // the other copy may still read my slots
    long long esA = 0, esB = 0;                         // energy sums of the measured sweeps (MEAS)

    SwapCountdown swap_cd(a.s0, a.swap_every);
    MeasureCountdown meas_cd(a.s0, a.measure_from, MEAS != 0 ? a.measure_every : 0u);
    for (uint32_t n = 0; n < a.n_sweeps && ok_run; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_s = swap_cd.step();             // a pass follows sweep s
        const bool swap_now = swap_s && NT > 1;
        const bool meas = MEAS != 0 && meas_cd.step();
        const bool needE = swap_now || energy_log != nullptr || meas || (n + 1 == a.n_sweeps);
        if constexpr (MEAS == 2) {
            if (pend_d) {                               // before this sweep writes my slots
                if (!wave_wait_cluster(&bar_d[k], ph_d, abort, a.err)) { ok_run = false; break; }
                ph_d ^= 1u;
                pend_d = false;
            }
        }
        uint32_t acc[PL], accM[PLM];
#pragma unroll
        for (int p = 0; p < PL; ++p) acc[p] = 0;
#pragma unroll
        for (int p = 0; p < PLM; ++p) accM[p] = 0;
        if constexpr (F) {
            // one body for both colours (kept a loop: two copies overflow the instruction cache)
            if (needE) {
#pragma unroll 1
                for (int col = 0; col < 2; ++col) {
                    uint32_t up[kPlanesHalfM] = {};
                    if (act)
                        wave_half_field<true, true, UA0, UA1>(wq, col, (uint32_t)s, col ? tag1 : tag0, a.rk, n0, n1,
                                                              acc, up);
                    add_up_planes(accM, up);
                    __syncwarp();
                }
            } else {
#pragma unroll 1
                for (int col = 0; col < 2; ++col) {
                    uint32_t up[kPlanesHalfM] = {};
                    if (act)
                        wave_half_field<false, false, UA0, UA1>(wq, col, (uint32_t)s, col ? tag1 : tag0, a.rk, n0,
                                                                n1, acc, up);
                    __syncwarp();
                }
            }
        } else {
            if (act) wave_half<0, false, PL>(wq, (uint32_t)s, tag0, a.rk, t0, t1, t2, acc);
            __syncwarp();
            if (needE) {
                if (act) wave_half<1, true, PL>(wq, (uint32_t)s, tag1, a.rk, t0, t1, t2, acc);
            } else if (act) {
                wave_half<1, false, PL>(wq, (uint32_t)s, tag1, a.rk, t0, t1, t2, acc);
            }
        }
        if (needE) {
            int UA, UB;
            wave_reduce<PL>(acc, lane, UA, UB);          // also orders the colour-1 stores (shuffles)
            EA = 2 * UA - 3 * N;
            EB = 2 * UB - 3 * N;
            if constexpr (F) {
                int upA, upB;
                wave_reduce<PLM>(accM, lane, upA, upB);
                MA = 2 * upA - N;
                MB = 2 * upB - N;
            }
        }
        __syncwarp();
        if (swap_now) {
            // decisions on Et = h_den E - h_num M (E itself without a field)
            const int etA = F ? hd * EA - hn * MA : EA, etB = F ? hd * EB - hn * MB : EB;
            // publish slot 2k (pre-exchange) for pair 2k-1 of warp k-1
            Eo[2 * k * kLanes + lane] = etA;
            if constexpr (F) {
                Eo[(NT + 2 * k) * kLanes + lane] = EA;
                Eo[(2 * NT + 2 * k) * kLanes + lane] = MA;
            }
            if (k > 0) mbar_arrive(&bar_e[k - 1]);
            int cur = etA, curE = EA, curM = MA;        // the carried configuration
            // Field-free: warps after the first form the next pass's bounds (they
            // depend on its index only) while warp k - 1 decides and applies its
            // pairs (0.0913 -> 0.0902 ps/flip); the field kernel measured slower so.
            constexpr bool kEarlyBounds = !F;
            int nbA = 0, nbB = 0;
            if (k > 0) {
                if (kEarlyBounds && hasB)
                    wave_bounds(rowa, rowb, len, sa, sb, k, c, P + 1, gr, a.rk, lane, step, nbA, nbB);
                if (!wave_wait<F>(&bar_h[k - 1], ph_h, abort, a.err)) { ok_run = false; break; }
                ph_h ^= 1u;
                cur = Cur[(k - 1) * kLanes + lane];
                if constexpr (F) {
                    curE = Cur[(nw + k - 1) * kLanes + lane];
                    curM = Cur[(2 * nw + k - 1) * kLanes + lane];
                }
            }
            uint32_t mA = 0, mB = 0;
            if (hasB) {
                // pair 2k: slot 2k holds the carried configuration (energy cur)
                const bool okA = cur - etB >= bA;
                mA = __ballot_sync(kFull, okA);
                const int nEA = okA ? EB : (F ? curE : cur), nMA = okA ? MB : curM;
                if (!okA) {
                    cur = etB;
                    if constexpr (F) {
                        curE = EB;
                        curM = MB;
                    }
                }
                uint4 *pa = reinterpret_cast<uint4 *>(S + (size_t)(2 * k) * SN);
                uint4 *pb = reinterpret_cast<uint4 *>(S + (size_t)(2 * k + 1) * SN);
                uint4 xb[N / 128];                      // slot 2k+1 after pair 2k (the carry)
#pragma unroll
                for (int j = 0; j < N / 128; ++j) {
                    const uint4 x = pa[lane + 32 * j], y = pb[lane + 32 * j];
                    pa[lane + 32 * j] = make_uint4(mux(x.x, y.x, mA), mux(x.y, y.y, mA), mux(x.z, y.z, mA),
                                                   mux(x.w, y.w, mA));
                    xb[j] = make_uint4(mux(y.x, x.x, mA), mux(y.y, x.y, mA), mux(y.z, x.z, mA), mux(y.w, x.w, mA));
                }
                int nEB, nMB;
                if (hasC) {
                    if (!wave_wait<F>(&bar_e[k], ph_e, abort, a.err)) { ok_run = false; break; }
                    ph_e ^= 1u;
                    const int e2 = Eo[(2 * k + 2) * kLanes + lane];
                    int e2E = e2, e2M = 0;
                    if constexpr (F) {
                        e2E = Eo[(NT + 2 * k + 2) * kLanes + lane];
                        e2M = Eo[(2 * NT + 2 * k + 2) * kLanes + lane];
                    }
                    const bool okB = cur - e2 >= bB;
                    mB = __ballot_sync(kFull, okB);
                    nEB = okB ? e2E : (F ? curE : cur);
                    nMB = okB ? e2M : curM;
                    if (!okB) {
                        cur = e2;
                        if constexpr (F) {
                            curE = e2E;
                            curM = e2M;
                        }
                    }
                    uint4 *pc = reinterpret_cast<uint4 *>(S + (size_t)(2 * k + 2) * SN);
#pragma unroll
                    for (int j = 0; j < N / 128; ++j) {
                        const uint4 x = xb[j], y = pc[lane + 32 * j];
                        pb[lane + 32 * j] = make_uint4(mux(x.x, y.x, mB), mux(x.y, y.y, mB), mux(x.z, y.z, mB),
                                                       mux(x.w, y.w, mB));
                        pc[lane + 32 * j] = make_uint4(mux(y.x, x.x, mB), mux(y.y, x.y, mB), mux(y.z, x.z, mB),
                                                       mux(y.w, x.w, mB));
                    }
                    Cur[k * kLanes + lane] = cur;
                    if constexpr (F) {
                        Cur[(nw + k) * kLanes + lane] = curE;
                        Cur[(2 * nw + k) * kLanes + lane] = curM;
                    }
                    mbar_arrive(&bar_h[k]);
                } else {
#pragma unroll
                    for (int j = 0; j < N / 128; ++j) pb[lane + 32 * j] = xb[j];
                    nEB = F ? curE : cur;               // slot 2k+1 is the last
                    nMB = curM;
                }
                EA = nEA;
                EB = nEB;
                MA = nMA;
                MB = nMB;
            } else {
                EA = F ? curE : cur;                    // slot 2k is the last (odd NT)
                MA = curM;
            }
            __syncwarp();
            if (swap_log != nullptr && lane == 0) {
                uint32_t *row = swap_log + ((size_t)pass_local * a.G + g) * a.C * (NT - 1) + (size_t)c * (NT - 1);
                if (hasB) row[2 * k] = mA;
                if (hasC) row[2 * k + 1] = mB;
            }
            ++P;
            ++pass_local;
            if (kEarlyBounds && k > 0) {
                bA = nbA;
                bB = nbB;
            } else if (hasB) {
                wave_bounds(rowa, rowb, len, sa, sb, k, c, P, gr, a.rk, lane, step, bA, bB);
            }
        } else if (swap_s) {
            ++P;                                        // NT == 1: passes count, nothing to exchange
            ++pass_local;
        }
        if (energy_log != nullptr) {
            const size_t row = (size_t)(s - a.log_s0);
            int32_t *el = energy_log + ((row * a.G + g) * NT) * a.C * kLanes + (size_t)c * kLanes;
            el[(size_t)(2 * k) * a.C * kLanes + lane] = EA;
            if (hasB) el[(size_t)(2 * k + 1) * a.C * kLanes + lane] = EB;
        }
        if constexpr (MEAS != 0) {
            if (meas) {
                esA += EA;                              // slots 2k, 2k+1 after the sweep and its pass
                esB += hasB ? EB : 0;
                if constexpr (MEAS == 2) {
                    mbar_arrive_remote(&bar_r[k], (uint32_t)(c ^ 1));   // my slots are final
                    if (!wave_wait_cluster(&bar_r[k], ph_r, abort, a.err)) { ok_run = false; break; }
                    ph_r ^= 1u;
                    const int t = 2 * k + c;
                    if (t < NT) {
                        const int nd = wave_overlap(reinterpret_cast<const uint4 *>(S + (size_t)t * N),
                                                    reinterpret_cast<const uint4 *>(S_other + (size_t)t * N),
                                                    lane);
                        atomicAdd(&hist[(size_t)k * (N + 1) + nd], 1u);
                    }
                    __syncwarp();
                    mbar_arrive_remote(&bar_d[k], (uint32_t)(c ^ 1));   // done reading the other copy
                    pend_d = true;
                }
            }
        }
    }
    if constexpr (MEAS != 0) {
        if (ok_run && a.esum != nullptr) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                esA += __shfl_xor_sync(kFull, esA, o);
                esB += __shfl_xor_sync(kFull, esB, o);
            }
            if (lane == 0) {
                atomicAdd(reinterpret_cast<unsigned long long *>(a.esum + 2 * k), (unsigned long long)esA);
                if (hasB)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.esum + 2 * k + 1), (unsigned long long)esB);
            }
        }
    }
    if (!ok_run) {                                      // the error flag is raised; state is not written
        if constexpr (MEAS == 2) cg::this_cluster().sync();
        return;
    }
    int32_t *gE = a.energy + (size_t)unit * NT * kLanes;
    gE[(2 * k) * kLanes + lane] = EA;
    if (hasB) gE[(2 * k + 1) * kLanes + lane] = EB;
    if constexpr (F) {
        int32_t *gM = a.mag + (size_t)unit * NT * kLanes;
        gM[(2 * k) * kLanes + lane] = MA;
        if (hasB) gM[(2 * k + 1) * kLanes + lane] = MB;
    }
    // this warp's slots are final (no later pass step touches them)
    const int nslot = hasB ? 2 : 1;
    if constexpr (F) {
        for (int i = 0; i < nslot; ++i)
            for (int w = lane; w < N / 4; w += 32)
                reinterpret_cast<uint4 *>(gS + (size_t)(2 * k + i) * N)[w] =
                    reinterpret_cast<const uint4 *>(S + (size_t)(2 * k + i) * SN)[w];
    } else {
        for (int w = lane; w < nslot * N / 4; w += 32)
            reinterpret_cast<uint4 *>(gS + (size_t)(2 * k) * N)[w] =
                reinterpret_cast<const uint4 *>(S + (size_t)(2 * k) * N)[w];
    }
    if constexpr (MEAS == 2) {
        // every warp of both copies is done: the histogram is complete and no
        // read of this CTA's shared memory is pending
        cg::this_cluster().sync();
        if (a.qhist != nullptr)
            for (int i = tid; i < nw * (N + 1); i += nthr) {
                const int j = i / (N + 1), bin = i - j * (N + 1);
                const int t = 2 * j + c;
                if (t < NT && hist[i] != 0u)
                    atomicAdd(reinterpret_cast<unsigned long long *>(a.qhist + (size_t)t * (N + 1) + bin),
                              (unsigned long long)hist[i]);
            }
    }
}

}  // namespace
}  // namespace ea
