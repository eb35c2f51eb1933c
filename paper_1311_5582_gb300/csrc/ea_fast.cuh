// Unit sweep body specialised for lattices with L % 8 == 0 (L = 8, 16).
//
// Same method and results as the generic unit kernel; the thread mapping is
// chosen for the hardware:
//  * Rows (y, z) are split by the parity of y + z.  In a row of parity pi the
//    sites of colour c sit at x parity (pi + c) & 1, which fixes which way the
//    x neighbours are shifted.  Every warp holds rows of one parity only, so
//    that choice is a warp-uniform branch instead of per-lane selects.
//  * HP threads work on one (lattice, parity) class and the number of quads
//    each one updates is a compile-time constant: addresses are computed once
//    per thread, outside the sweep loop.
//  * The replica-exchange bounds draw each Philox output block once (four
//    realizations per call) and search a shared-memory copy of the table.
#pragma once

#include "ea_device.cuh"

namespace ea {
namespace {


__host__ __device__ constexpr int planes_for(int maxval)
{
    int p = 0;
    while ((1 << p) <= maxval) ++p;
    return p;
}

template <int HP>
struct FastMap {
    // lattices per warp (HP < 32): a block of 64 threads covers M lattices,
    // its first warp their parity-0 rows, its second warp their parity-1 rows
    static constexpr int M = HP >= 32 ? 1 : 32 / HP;
    __device__ static void map(int tid, int &l, int &par, int &tl)
    {
        if constexpr (HP >= 32) {
            l = tid / (2 * HP);
            const int r = tid - l * 2 * HP;
            par = r / HP;
            tl = r - par * HP;
        } else {
            const int blk = tid >> 6, within = tid & 63;
            par = within >> 5;
            const int idx = within & 31;
            l = blk * M + idx / HP;
            tl = idx % HP;
        }
    }
    __device__ static int group_lattice(int warp, int gi)
    {
        if constexpr (HP >= 32) return (warp * 32) / (2 * HP);
        else return (warp >> 1) * M + gi;
    }
    static int threads(int NT) { return HP >= 32 ? NT * 2 * HP : ((NT + M - 1) / M) * 64; }
};

// Class indices of one quad and of the quads it reads (valid in either colour array).
struct QuadRow {
    int k0;                 // own quad
    int yp, ym, zp, zm;     // matching quads in the rows y +- 1, z +- 1
    int xe0, xe1;           // the x neighbour across the quad edge: x - 1 of the first
                            // site (x parity 0) or x + 1 of the last site (x parity 1)
};

template <int L>
__device__ __forceinline__ QuadRow quad_row(int par, int i)
{
    constexpr int R = L / 2, QR = L / 8;
    const int irow = i / QR, sub = i - irow * QR;
    const int z = irow / (L / 2), yh = irow - z * (L / 2);
    const int y = 2 * yh + ((z + par) & 1);
    const int m0 = 4 * sub;
    const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
    const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
    QuadRow d;
    const int rowb = R * (y + L * z);
    d.k0 = rowb + m0;
    d.yp = m0 + R * (yp + L * z);
    d.ym = m0 + R * (ym + L * z);
    d.zp = m0 + R * (y + L * zp);
    d.zm = m0 + R * (y + L * zm);
    d.xe0 = rowb + (m0 == 0 ? R - 1 : m0 - 1);
    d.xe1 = rowb + (m0 + 4 == R ? 0 : m0 + 4);
    return d;
}

__device__ __forceinline__ uint4 ld4(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }

// All-ones iff r < t: the high word of r - t in 64-bit arithmetic, formed as
// r * 1 + (2^64 - t) by one wide multiply-add (the assembler makes it an add
// with carry: one ALU and one FMA-pipe instruction).
__device__ __forceinline__ uint32_t below_mask(uint32_t r, uint64_t neg_t)
{
    uint64_t d;
    asm("mad.wide.u32 %0, %1, 1, %2;" : "=l"(d) : "r"(r), "l"(neg_t));
    return (uint32_t)(d >> 32);
}

// Flip mask (same decision as flip_mask): lanes with u >= 3, or u >= 2 and
// r < t2, or u >= 1 and r < t1, or r < t0.  The masks m_i = [r < t_i] are
// all-ones or all-zeros words and, the thresholds being monotone, m0 implies
// m1 implies m2, so
//   [u>=3] | [u>=2] m2 | [u>=1] m1 | m0 = u2 | u1 (u0 | m2) | u0 m1 | m0,
// three LOP3s before the last OR (which the caller may fold into its XOR).
__device__ __forceinline__ uint32_t flip_mask_part(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t m1,
                                                   uint32_t m2)
{
    const uint32_t a = u0 | m2;
    const uint32_t t = u2 | (u1 & a);
    return t | (u0 & m1);
}
__device__ __forceinline__ uint32_t flip_mask_fma(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t r,
                                                  uint64_t n0, uint64_t n1, uint64_t n2)
{
    const uint32_t m0 = below_mask(r, n0), m1 = below_mask(r, n1), m2 = below_mask(r, n2);
    return flip_mask_part(u0, u1, u2, m1, m2) | m0;
}

template <int PL>
__device__ __forceinline__ void acc_add_sum5(uint32_t (&acc)[PL], const uint32_t (&A)[5])
{
    uint32_t cy = acc[0] & A[0];
    acc[0] ^= A[0];
#pragma unroll
    for (int i = 1; i < PL; ++i) {
        if (i < 5) {
            uint32_t s2, c2;
            full_add(acc[i], A[i], cy, s2, c2);
            acc[i] = s2;
            cy = c2;
        } else {
            const uint32_t c2 = acc[i] & cy;
            acc[i] ^= cy;
            cy = c2;
        }
    }
}

// Adds the post-update counts (x2 x1 x0)[j] of one quad to a ripple counter
// of PL planes: the quad's 5-bit sum, then a ripple add.
template <int PL>
struct RippleAcc {
    uint32_t (&acc)[PL];
    template <int Q>
    __device__ __forceinline__ void add(const uint32_t (&x)[3][4])
    {
        uint32_t A[5];
        quad_sum(x[0], x[1], x[2], A);
        acc_add_sum5<PL>(acc, A);
    }
};

// Carry-save counter of per-lane sums over the quads a lane updates: each quad
// brings four bits at each of the weights 2^0 .. 2^(NIN-1) (NIN = 3 for the
// post-update counts u' of four sites, NIN = 1 for four spin bits), and NP
// planes hold the largest total.  Plane S[w] holds one bit of weight 2^w per
// lane; each full adder S[w] + b + b' -> S[w] + 2 c moves one carry up, and a
// bit left over at a weight waits in P[w] for the next quad.  Which weights
// hold a waiting bit before quad Q follows from the bit counts alone, so the
// whole schedule is resolved at compile time (for four quads of u': ~45 full
// adders, against 128 LOP3s for four 5-bit quad sums rippled into a counter).
__host__ __device__ constexpr uint32_t csa_pending(int Q, int NIN, int NP)
{
    uint32_t pend = 0;
    for (int q = 0; q < Q; ++q) {
        int carry = 0;
        for (int w = 0; w < NP; ++w) {
            const int n = (w < NIN ? 4 : 0) + carry + (int)((pend >> w) & 1u);
            carry = n / 2;
            pend = (pend & ~(1u << w)) | ((uint32_t)(n & 1) << w);
        }
    }
    return pend;
}

template <int NIN, int NP>
struct CsaAcc {
    uint32_t S[NP], P[NP];

    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int w = 0; w < NP; ++w) S[w] = P[w] = 0u;
    }

    template <int Q, int W, int NC>
    __device__ __forceinline__ void weight(const uint32_t (&x)[NIN][4], const uint32_t (&cin)[NC > 0 ? NC : 1])
    {
        constexpr bool pend = ((csa_pending(Q, NIN, NP) >> W) & 1u) != 0;
        constexpr int NI = W < NIN ? 4 : 0;
        constexpr int N = NI + NC + (pend ? 1 : 0);
        constexpr int NF = N / 2;
        uint32_t bag[N > 0 ? N : 1];
#pragma unroll
        for (int i = 0; i < NI; ++i) bag[i] = x[W < NIN ? W : 0][i];
#pragma unroll
        for (int i = 0; i < NC; ++i) bag[NI + i] = cin[i];
        if constexpr (pend) bag[N - 1] = P[W];
        uint32_t cout[NF > 0 ? NF : 1];
#pragma unroll
        for (int i = 0; i < NF; ++i) {
            const uint32_t sw = S[W];
            S[W] = lop3<kXor3>(sw, bag[2 * i], bag[2 * i + 1]);
            cout[i] = lop3<kMaj3>(sw, bag[2 * i], bag[2 * i + 1]);
        }
        if constexpr ((N & 1) != 0) P[W] = bag[N - 1];
        if constexpr (W + 1 < NP) weight<Q, W + 1, NF>(x, cout);    // a carry out of the top plane is 0
    }

    // Adds quad Q of the sequence (Q counts from 0 after clear()).
    template <int Q>
    __device__ __forceinline__ void add(const uint32_t (&x)[NIN][4])
    {
        const uint32_t none[1] = {0u};
        weight<Q, 0, 0>(x, none);
    }

    // The binary counter after NQ quads: the waiting bits rippled into S.
    template <int NQ>
    __device__ __forceinline__ void resolve(uint32_t (&acc)[NP])
    {
        constexpr uint32_t pend = csa_pending(NQ, NIN, NP);
        uint32_t cy = 0u;
        bool has_cy = false;
#pragma unroll
        for (int w = 0; w < NP; ++w) {
            const bool p = ((pend >> w) & 1u) != 0;
            if (p && has_cy) {
                const uint32_t sw = S[w];
                S[w] = lop3<kXor3>(sw, P[w], cy);
                cy = lop3<kMaj3>(sw, P[w], cy);
            } else if (p || has_cy) {
                const uint32_t b = p ? P[w] : cy;
                cy = S[w] & b;
                S[w] ^= b;
                has_cy = true;
            }
            acc[w] = S[w];
        }
    }
};

// Post-update counts of four quads per lane (<= 96): seven planes.
using CountAcc = CsaAcc<3, 7>;

// Metropolis update of the four sites of one quad whose rows have x parity
// PX, from its loaded words: own spins, the other colour's words at the same
// class index (xo) and in the rows y +- 1, z +- 1, the bonds of the own colour
// (+x, +y, +z at the site) and of the other colour (-x at xo, -y at the y - 1
// row, -z at the z - 1 row).  Valid for rows of four class indices (L = 8),
// where the x neighbour across the quad edge is in xo itself, and through
// xe_s / xe_j otherwise.  Returns the new own spins; with WITH_E adds the
// post-update unsatisfied-bond counts to acc (as quad Q of its half-sweep).
template <int PX, bool WITH_E, int Q, typename Acc>
__device__ __forceinline__ uint4 quad_core(uint4 own, uint4 xo, uint4 vyp, uint4 vym, uint4 vzp, uint4 vzm,
                                           uint4 jcx, uint4 jcy, uint4 jcz, uint4 jox, uint4 joy, uint4 joz,
                                           uint32_t xe_s, uint32_t xe_j, const uint4 r, uint64_t t0,
                                           uint64_t t1, uint64_t t2, Acc &acc)
{
    uint32_t nxp[4], nxm[4], jxm[4];
    if constexpr (PX == 0) {
        nxp[0] = xo.x; nxp[1] = xo.y; nxp[2] = xo.z; nxp[3] = xo.w;
        nxm[0] = xe_s; nxm[1] = xo.x; nxm[2] = xo.y; nxm[3] = xo.z;
        jxm[0] = xe_j; jxm[1] = jox.x; jxm[2] = jox.y; jxm[3] = jox.z;
    } else {
        nxp[0] = xo.y; nxp[1] = xo.z; nxp[2] = xo.w; nxp[3] = xe_s;
        nxm[0] = xo.x; nxm[1] = xo.y; nxm[2] = xo.z; nxm[3] = xo.w;
        jxm[0] = jox.x; jxm[1] = jox.y; jxm[2] = jox.z; jxm[3] = jox.w;
        (void)xe_j;
    }
    const uint32_t sv[4] = {own.x, own.y, own.z, own.w};
    const uint32_t jx[4] = {jcx.x, jcx.y, jcx.z, jcx.w};
    const uint32_t ny[4] = {vyp.x, vyp.y, vyp.z, vyp.w}, my[4] = {vym.x, vym.y, vym.z, vym.w};
    const uint32_t nz[4] = {vzp.x, vzp.y, vzp.z, vzp.w}, mz[4] = {vzm.x, vzm.y, vzm.z, vzm.w};
    const uint32_t jy[4] = {jcy.x, jcy.y, jcy.z, jcy.w}, jym[4] = {joy.x, joy.y, joy.z, joy.w};
    const uint32_t jz[4] = {jcz.x, jcz.y, jcz.z, jcz.w}, jzm[4] = {joz.x, joz.y, joz.z, joz.w};
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    uint32_t ns[4], x0[4], x1[4], x2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t sj = sv[j];
        const uint32_t e0 = lop3<kXor3>(sj, nxp[j], jx[j]);
        const uint32_t e1 = lop3<kXor3>(sj, nxm[j], jxm[j]);
        const uint32_t e2 = lop3<kXor3>(sj, ny[j], jy[j]);
        const uint32_t e3 = lop3<kXor3>(sj, my[j], jym[j]);
        const uint32_t e4 = lop3<kXor3>(sj, nz[j], jz[j]);
        const uint32_t e5 = lop3<kXor3>(sj, mz[j], jzm[j]);
        // u = (a0 + 2 a1) + (b0 + 2 b1)
        const uint32_t a0 = lop3<kXor3>(e0, e1, e2), a1 = lop3<kMaj3>(e0, e1, e2);
        const uint32_t b0 = lop3<kXor3>(e3, e4, e5), b1 = lop3<kMaj3>(e3, e4, e5);
        const uint32_t m0 = below_mask(rr[j], t0), m1 = below_mask(rr[j], t1), m2 = below_mask(rr[j], t2);
        if constexpr (WITH_E) {
            // the energy counters need u itself: u0, u1, u2, then the mask
            //   f = u2 | u1 (u0 | m2) | u0 m1 | m0
            const uint32_t u0 = a0 ^ b0, c0 = a0 & b0;
            const uint32_t u1 = lop3<kXor3>(a1, b1, c0), u2 = lop3<kMaj3>(a1, b1, c0);
            const uint32_t f = lop3<kOrAnd>(lop3<kOr3>(lop3<kAndOr2>(u1, u0, m2), u2, m0), u0, m1);
            ns[j] = sj ^ f;
            // post-flip counts: u -> 6 - u where f (u0 unchanged)
            x0[j] = u0;
            x1[j] = lop3<kXorAndN>(u1, f, u0);
            x2[j] = lop3<kXorAndN>(u2, f, u0 & u1);
        } else {
            // the mask straight from the two partial sums (m0 => m1 => m2):
            //   [u>=3] | m2 [u>=2] | m1 [u>=1] | m0
            //     = maj(a1, b1, a0 | b0 | m2) | (m2 & maj(a0, b0, m1)) | m0,
            // four LOP3s and the flip folded into the last
            const uint32_t v = lop3<kOr3>(a0, b0, m2);
            const uint32_t t = lop3<kAndOr>(m2, lop3<kMaj3>(a0, b0, m1), lop3<kMaj3>(a1, b1, v));
            ns[j] = lop3<kXorOr>(sj, t, m0);
        }
    }
    if constexpr (WITH_E) {
        const uint32_t x[3][4] = {{x0[0], x0[1], x0[2], x0[3]}, {x1[0], x1[1], x1[2], x1[3]},
                                  {x2[0], x2[1], x2[2], x2[3]}};
        acc.template add<Q>(x);
    }
    return make_uint4(ns[0], ns[1], ns[2], ns[3]);
}

// Metropolis update of one quad of colour COL whose rows have x parity PX.
template <int L, int COL, int PX, bool WITH_E, int PL>
__device__ __forceinline__ void quad_fast(uint32_t *S, const uint32_t *J, const QuadRow &d,
                                          const uint4 r, uint64_t t0, uint64_t t1, uint64_t t2,
                                          uint32_t (&acc)[PL])
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N, H = Gm::H, R = Gm::R;
    uint32_t *Sc = S + COL * H;
    const uint32_t *So = S + (1 - COL) * H;
    const uint32_t *Jc = J + COL * H;
    const uint32_t *Jo = J + (1 - COL) * H;
    const uint4 own = ld4(Sc + d.k0), xo = ld4(So + d.k0);
    const uint4 vyp = ld4(So + d.yp), vym = ld4(So + d.ym);
    const uint4 vzp = ld4(So + d.zp), vzm = ld4(So + d.zm);
    const uint4 jcx = ld4(Jc + d.k0), jcy = ld4(Jc + N + d.k0), jcz = ld4(Jc + 2 * N + d.k0);
    const uint4 jox = ld4(Jo + d.k0), joy = ld4(Jo + N + d.ym), joz = ld4(Jo + 2 * N + d.zm);
    uint32_t xe_s, xe_j;
    if constexpr (R == 4) {
        xe_s = PX ? xo.x : xo.w;
        xe_j = jox.w;
    } else {
        const int ie = PX ? d.xe1 : d.xe0;
        xe_s = So[ie];
        xe_j = Jo[ie];
    }
    RippleAcc<PL> ra{acc};
    *reinterpret_cast<uint4 *>(Sc + d.k0) = quad_core<PX, WITH_E, 0>(
        own, xo, vyp, vym, vzp, vzm, jcx, jcy, jcz, jox, joy, joz, xe_s, xe_j, r, t0, t1, t2, ra);
}

template <int L, int HP, int QPER, int COL, int PX, bool WITH_E, int PL>
__device__ __forceinline__ void half_fast(uint32_t *S, const uint32_t *J, const QuadRow (&qd)[QPER],
                                          const bool (&qv)[QPER], uint32_t s, uint32_t g,
                                          uint32_t ctag, const RoundKeys &rk, uint64_t t0,
                                          uint64_t t1, uint64_t t2, uint32_t (&acc)[PL])
{
    // The uniforms of quad j + 1 are drawn while quad j is updated (they are
    // independent), which gives the scheduler two dependency chains to interleave.
    constexpr bool ALL = (Geo<L>::Q / 2) % HP == 0;   // every active thread has QPER valid quads
    uint4 rn = philox((uint32_t)(qd[0].k0 >> 2), ctag, s, g, rk);
#pragma unroll
    for (int j = 0; j < QPER; ++j) {
        const uint4 rj = rn;
        if (j + 1 < QPER) rn = philox((uint32_t)(qd[j + 1 < QPER ? j + 1 : j].k0 >> 2), ctag, s, g, rk);
        if (ALL || qv[j]) quad_fast<L, COL, PX, WITH_E, PL>(S, J, qd[j], rj, t0, t1, t2, acc);
    }
}

// Adds scale x (per-lane value of each thread group's bit-sliced counter)
// into out[lattice][lane].  A group is the HP threads of one (lattice, row
// parity) class.  The group's counters are first summed with a butterfly of
// shuffles and bit-sliced adders (every member ends with the total, PL +
// log2(HP) planes); then member t holds plane t, and a 32x32 bit transpose
// leaves in lane b a word whose bits [gi*G, gi*G + G) are, in order, the
// planes of group gi at lane b -- i.e. the group's value for realization b.
template <int PL, int HP>
__device__ __forceinline__ void reduce_groups(const uint32_t (&acc)[PL], int *out, int lane,
                                              int warp, int scale, int NT)
{
    constexpr int GW = HP < 32 ? HP : 32;           // group width inside a warp
    constexpr int LV = GW == 1 ? 0 : GW == 2 ? 1 : GW == 4 ? 2 : GW == 8 ? 3 : GW == 16 ? 4 : 5;
    constexpr int PT = PL + LV;                      // planes of the group total
    constexpr int NR = (PT + GW - 1) / GW;           // transposes needed
    uint32_t v[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) v[p] = p < PL ? acc[p] : 0u;
#pragma unroll
    for (int lv = 0; lv < LV; ++lv) {
        const int m = 1 << lv;
        uint32_t cy = 0;
#pragma unroll
        for (int p = 0; p < PL + lv + 1; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, v[p], m);
            uint32_t s2, c2;
            full_add(v[p], o, cy, s2, c2);
            v[p] = s2;
            cy = c2;
        }
    }
    const int t = lane % GW;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        // member t contributes plane r*GW + t
        uint32_t x = 0;
#pragma unroll
        for (int p = 0; p < PT; ++p)
            if (p / GW == r) x = (t == p % GW) ? v[p] : x;
        const uint32_t y = warp_transpose(x, lane);
#pragma unroll
        for (int gi = 0; gi < 32 / GW; ++gi) {
            constexpr uint32_t gmask = (uint32_t)((1ull << GW) - 1ull);
            const int val = (int)((y >> (gi * GW)) & gmask) << (r * GW);
            const int l = FastMap<HP>::group_lattice(warp, gi);
            if (l < NT && val != 0) atomicAdd(&out[l * kLanes + lane], scale * val);
        }
    }
}

// Shared-memory layout of the specialised unit kernel, in 32-bit words.
struct FastLayout {
    size_t s, js, e, bnd0, bnd1, nd, msk, esum, tsw, snap0, snap1, hist, words;
    __host__ __device__ FastLayout(int N, int NT, uint32_t swap_len, bool swap_smem, bool snap,
                                   bool hist_smem)
    {
        const int half = (NT + 1) / 2;
        size_t o = 0;
        s = o; o += (size_t)NT * N;
        js = o; o += (size_t)3 * N;
        e = o; o += (size_t)kMaxTemps * kLanes;
        bnd0 = o; o += (size_t)kMaxTemps * kLanes;
        bnd1 = o; o += (size_t)kMaxTemps * kLanes;
        nd = o; o += (size_t)kMaxTemps * kLanes;
        msk = o; o += kMaxTemps;
        esum = o; o += 2 * kMaxTemps;            // int64 per slot (offset even: 8-byte aligned)
        tsw = o; o += swap_smem && NT > 1 ? (size_t)(NT - 1) * swap_len : 0;
        o = (o + 3) & ~(size_t)3;                // 16-byte alignment for the snapshots
        snap0 = o; o += snap ? (size_t)half * N : 0;
        snap1 = o; o += snap ? (size_t)half * N : 0;
        hist = o; o += hist_smem ? (size_t)half * (N + 1) : 0;
        words = o;
    }
};

// Sum over the 32 lanes of a warp of each lane's bit-sliced per-realization
// counter; out[b] receives the total of realization b.  Butterfly of shuffles
// and bit-sliced adders (every lane ends with the total, PL + 5 planes), then
// lane t holds plane t and a 32x32 transpose leaves the binary value of
// realization b in lane b.
template <int PL>
__device__ __forceinline__ void warp_sum_to_lanes(const uint32_t (&acc)[PL], int lane, int *out)
{
    constexpr int PT = PL + 5;
    static_assert(PT <= 32, "counter too wide");
    uint32_t v[PT];
#pragma unroll
    for (int p = 0; p < PT; ++p) v[p] = p < PL ? acc[p] : 0u;
#pragma unroll
    for (int lv = 0; lv < 5; ++lv) {
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
    uint32_t x = 0;
#pragma unroll
    for (int p = 0; p < PT; ++p) x = (lane == p) ? v[p] : x;
    out[lane] = (int)warp_transpose(x, lane);
}

// Named CTA barriers (ids 1..15; 0 is __syncthreads): the producer warp
// arrives without waiting, the consumer warps wait until `count` threads have
// arrived.  Both order the shared-memory accesses made before them.
__device__ __forceinline__ void named_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// MEAS = false compiles the body without the measurement and log paths
// (launches that measure and log nothing); the flags then must be 0 and the
// log pointers null.
template <int L, int HP, bool MEAS = true>
__device__ __forceinline__ void unit_fast_body(uint32_t *const base, const SweepLaunch &a, uint32_t unit,
                                               int cluster_measure_arg, int swap_in_smem, int snap_mode_arg,
                                               int hist_smem_arg)
{
    const int cluster_measure = MEAS ? cluster_measure_arg : 0;
    const int snap_mode = MEAS ? snap_mode_arg : 0;
    const int hist_smem = MEAS ? hist_smem_arg : 0;
    int32_t *const energy_log = MEAS ? a.energy_log : nullptr;
    uint32_t *const swap_log = MEAS ? a.swap_log : nullptr;
    using Gm = Geo<L>;
    using Mp = FastMap<HP>;
    constexpr int N = Gm::N;
    constexpr int QP = Gm::Q / 2;                       // quads per (colour, row parity)
    constexpr int QPER = (QP + HP - 1) / HP;            // quads per thread per half-sweep
    constexpr int PL = planes_for(24 * QPER);           // energy counter planes
    const int NT = (int)a.NT;
    const FastLayout lay(N, NT, a.swap_len, swap_in_smem != 0, snap_mode != 0, hist_smem != 0);
    uint32_t *S = base + lay.s;                                // [NT][2][H]
    uint32_t *Js = base + lay.js;                              // [3][2][H]
    int *E = reinterpret_cast<int *>(base + lay.e);            // [64][32] energies by slot
    // acceptance bounds of the swap pass, for even and odd pass indices
    int *const bnd0 = reinterpret_cast<int *>(base + lay.bnd0);
    int *const bnd1 = reinterpret_cast<int *>(base + lay.bnd1);
    int *nd = reinterpret_cast<int *>(base + lay.nd);          // [64][32] overlap counts
    uint32_t *msk = base + lay.msk;                            // [64]
    unsigned long long *esum_s = reinterpret_cast<unsigned long long *>(base + lay.esum);
    uint32_t *const snap0 = base + lay.snap0;                  // partner's slots, ping-pong
    uint32_t *const snap1 = base + lay.snap1;
    uint32_t *hist = base + lay.hist;                          // [ceil(NT/2)][N+1]

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const uint32_t gr = g + a.g_base;                   // group index of the random numbers
    const int half = (NT + 1) / 2;
    int l, par, tl;
    Mp::map(tid, l, par, tl);
    const bool active = l < NT;
    const int ls = active ? l : 0;

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
    for (int i = tid; i < kMaxTemps; i += nthr) esum_s[i] = 0ull;
    if (hist_smem)
        for (int i = tid; i < half * (N + 1); i += nthr) hist[i] = 0u;
    // thresholds of my slot as 2^64 - t (see below_mask)
    const uint64_t t0 = 0ull - (uint64_t)a.metro[ls * 3 + 0];
    const uint64_t t1 = 0ull - (uint64_t)a.metro[ls * 3 + 1];
    const uint64_t t2 = 0ull - (uint64_t)a.metro[ls * 3 + 2];
    QuadRow qd[QPER];
    bool qv[QPER];
#pragma unroll
    for (int j = 0; j < QPER; ++j) {
        const int i = tl + HP * j;
        qv[j] = active && i < QP;
        qd[j] = quad_row<L>(par, qv[j] ? i : 0);
    }
    uint32_t *mine = S + (size_t)ls * N;
    const uint32_t tag0 = ((uint32_t)c << 8) | (uint32_t)ls;
    const uint32_t tag1 = (1u << 16) | tag0;

    // Acceptance bounds of swap pass Q (depend on the pass index only): one
    // Philox call gives the uniforms of four realizations of a pair.
    // Acceptance bounds of swap pass Q (they depend on the pass index only).
    // One Philox call gives the uniforms of four realizations of a pair; their
    // four bounds come from one branchless binary search run in lockstep: the
    // number of leading entries of the non-increasing row above r is found by
    // binary lifting with a trip count fixed by the row length.
    auto bounds = [&](uint64_t Q, int *out, int first, int step) {
        const uint32_t len = a.swap_len;
        uint32_t top = 0;                    // largest power of two <= len
        if (len != 0) {
            top = 1;
            while (top <= (len >> 1)) top <<= 1;
        }
        for (int i = first; i < (NT - 1) * 8; i += step) {
            const int p = i >> 3, bq = i & 7;
            const uint4 v = philox(((uint32_t)p << 3) | (uint32_t)bq,
                                   (1u << 24) | ((uint32_t)c << 8), (uint32_t)Q, gr, a.rk);
            const uint32_t *row = swt + (size_t)p * len;
            uint32_t k0 = 0, k1 = 0, k2 = 0, k3 = 0;      // invariant: row[0..k) > r
            for (uint32_t st = top; st != 0; st >>= 1) {
                const uint32_t n0 = k0 + st, n1 = k1 + st, n2 = k2 + st, n3 = k3 + st;
                const uint32_t e0 = n0 <= len ? row[n0 - 1] : 0u;
                const uint32_t e1 = n1 <= len ? row[n1 - 1] : 0u;
                const uint32_t e2 = n2 <= len ? row[n2 - 1] : 0u;
                const uint32_t e3 = n3 <= len ? row[n3 - 1] : 0u;
                k0 = e0 > v.x ? n0 : k0;
                k1 = e1 > v.y ? n1 : k1;
                k2 = e2 > v.z ? n2 : k2;
                k3 = e3 > v.w ? n3 : k3;
            }
            int *o = out + p * kLanes + 4 * bq;
            o[0] = -4 * (int)k0;
            o[1] = -4 * (int)k1;
            o[2] = -4 * (int)k2;
            o[3] = -4 * (int)k3;
        }
    };
    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    uint32_t n_meas = 0;
    __syncthreads();   // staged lattices, bonds and swap table are complete
    if (NT > 1 && a.swap_every != 0) bounds(P, (P & 1) ? bnd1 : bnd0, tid, nthr);
    __syncthreads();

    SwapCountdown swap_cd(a.s0, a.swap_every);
    MeasureCountdown meas_cd(a.s0, a.measure_from, MEAS ? a.measure_every : 0u);
    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_s = swap_cd.step();             // a pass follows sweep s
        const bool swap_now = swap_s && NT > 1;
        const bool meas = MEAS && meas_cd.step();
        const bool needE = swap_now || energy_log != nullptr || meas || (n + 1 == a.n_sweeps);
        uint32_t acc[PL];
#pragma unroll
        for (int p = 0; p < PL; ++p) acc[p] = 0;
        if (needE)   // groups add 2 per unsatisfied bond: E = 2U - 3N
            for (int i = tid; i < NT * kLanes; i += nthr) E[i] = -3 * N;
        // colour 0: x parity = par; colour 1: x parity = par ^ 1 (warp-uniform)
        if (!active) {
        } else if (par == 0)
            half_fast<L, HP, QPER, 0, 0, false, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag0, a.rk, t0, t1, t2, acc);
        else
            half_fast<L, HP, QPER, 0, 1, false, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag0, a.rk, t0, t1, t2, acc);
        __syncthreads();
        if (needE) {
            if (!active) {
            } else if (par == 0)
                half_fast<L, HP, QPER, 1, 1, true, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
            else
                half_fast<L, HP, QPER, 1, 0, true, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
            reduce_groups<PL, HP>(acc, E, lane, warp, 2, NT);
        } else {
            if (!active) {
            } else if (par == 0)
                half_fast<L, HP, QPER, 1, 1, false, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
            else
                half_fast<L, HP, QPER, 1, 0, false, PL>(mine, Js, qd, qv, (uint32_t)s, gr, tag1, a.rk, t0, t1, t2, acc);
        }
        __syncthreads();
        if (swap_now) {
            const int *bnd = (P & 1) ? bnd1 : bnd0;
            // Pipelined exchange (L = 8, 16 threads per lattice, at least 12 warps):
            // warp 0 releases each batch of eight decided pairs through named
            // barrier 1 + batch; warps 1..4 (two 8-byte columns of the lattices
            // each) exchange that batch meanwhile; the remaining warps (at least
            // seven: one item each) compute the next pass's bounds.  Every thread
            // of warps 0..4 passes each of the batch barriers exactly once (160
            // threads).
            constexpr int kXW = 4;                     // exchange warps
            bool pipe = false;
            if constexpr (L == 8 && HP == 8) pipe = nthr >= 32 * (kXW + 8);
            const int kPipeThreads = 32 * (kXW + 1);
            if (warp == 0) {
                // Sequential pairs (0,1), (1,2), ... per realization lane.  The
                // configuration carried upward has energy `cur`; pair p accepts iff
                // cur - E[p+1] >= bound, i.e. cur >= E[p+1] + bound.  The right
                // sides of eight pairs are loaded before their eight decisions.
                int cur = E[lane];
                for (int p0 = 0; p0 + 1 < NT; p0 += 8) {
                    int nx[8], th[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int p = p0 + q;
                        nx[q] = 0;
                        th[q] = 0;
                        if (p + 1 < NT) {
                            nx[q] = E[(p + 1) * kLanes + lane];
                            th[q] = nx[q] + bnd[p * kLanes + lane];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int p = p0 + q;
                        if (p + 1 < NT) {
                            const bool ok = cur >= th[q];
                            const uint32_t m = __ballot_sync(kFull, ok);
                            E[p * kLanes + lane] = ok ? nx[q] : cur;
                            cur = ok ? cur : nx[q];
                            if (lane == 0) msk[p] = m;
                        }
                    }
                    if (pipe) {
                        __syncwarp();
                        named_arrive(1 + p0 / 8, kPipeThreads);   // masks of this batch are final
                    }
                }
                E[(NT - 1) * kLanes + lane] = cur;
            } else if (pipe && warp <= kXW) {
                if constexpr (L == 8 && HP == 8) {
                    constexpr int RW = N / 2;                     // 256 columns, two a thread
                    constexpr int CW = 32 * kXW;                  // column stride between them
                    const int w = tid - 32;
                    const uint2 *src = reinterpret_cast<const uint2 *>(S) + w;
                    uint2 *dst = reinterpret_cast<uint2 *>(S) + w;
                    uint2 x0 = src[0], x1 = src[CW];
                    for (int p0 = 0; p0 + 1 < NT; p0 += 8) {
                        uint2 y0[8], y1[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const bool in = p0 + q + 1 < NT;
                            y0[q] = in ? src[(size_t)(p0 + 1 + q) * RW] : make_uint2(0u, 0u);
                            y1[q] = in ? src[(size_t)(p0 + 1 + q) * RW + CW] : make_uint2(0u, 0u);
                        }
                        named_sync(1 + p0 / 8, kPipeThreads);     // wait for this batch's masks
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (p0 + q + 1 < NT) {
                                const uint32_t m = msk[p0 + q];
                                const uint32_t a0 = (x0.x ^ y0[q].x) & m, b0 = (x0.y ^ y0[q].y) & m;
                                const uint32_t a1 = (x1.x ^ y1[q].x) & m, b1 = (x1.y ^ y1[q].y) & m;
                                dst[(size_t)(p0 + q) * RW] = make_uint2(x0.x ^ a0, x0.y ^ b0);
                                dst[(size_t)(p0 + q) * RW + CW] = make_uint2(x1.x ^ a1, x1.y ^ b1);
                                x0 = make_uint2(y0[q].x ^ a0, y0[q].y ^ b0);
                                x1 = make_uint2(y1[q].x ^ a1, y1[q].y ^ b1);
                            }
                        }
                    }
                    dst[(size_t)(NT - 1) * RW] = x0;
                    dst[(size_t)(NT - 1) * RW + CW] = x1;
                }
            } else if (pipe) {
                if constexpr (L == 8 && HP == 8)
                    bounds(P + 1, (P & 1) ? bnd0 : bnd1, tid - kPipeThreads, nthr - kPipeThreads);
            } else {
                // meanwhile: bounds of the next pass (other buffer)
                bounds(P + 1, (P & 1) ? bnd0 : bnd1, tid - 32, nthr - 32);
            }
            __syncthreads();
            for (int w = tid; !pipe && w < N / 2; w += nthr) {
                // masked exchange chain; the words of eight slots are loaded before
                // any of them is stored (slot rows never alias)
                const uint2 *src = reinterpret_cast<const uint2 *>(S) + w;
                uint2 *dst = reinterpret_cast<uint2 *>(S) + w;
                constexpr int RW = N / 2;                 // uint2 words per lattice
                uint2 x = src[0];
                int p = 0;
                for (; p + 8 < NT; p += 8) {
                    uint2 ys[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) ys[q] = src[(size_t)(p + 1 + q) * RW];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t m = msk[p + q];
                        const uint32_t dx = (x.x ^ ys[q].x) & m, dy = (x.y ^ ys[q].y) & m;
                        dst[(size_t)(p + q) * RW] = make_uint2(x.x ^ dx, x.y ^ dy);
                        x = make_uint2(ys[q].x ^ dx, ys[q].y ^ dy);
                    }
                }
                for (; p + 1 < NT; ++p) {
                    const uint2 y = src[(size_t)(p + 1) * RW];
                    const uint32_t m = msk[p];
                    const uint32_t dx = (x.x ^ y.x) & m, dy = (x.y ^ y.y) & m;
                    dst[(size_t)p * RW] = make_uint2(x.x ^ dx, x.y ^ dy);
                    x = make_uint2(y.x ^ dx, y.y ^ dy);
                }
                dst[(size_t)(NT - 1) * RW] = x;
            }
            if (swap_log != nullptr)
                for (int p = tid; p + 1 < NT; p += nthr)
                    swap_log[(((size_t)pass_local * a.G + g) * a.C + c) * (NT - 1) + p] = msk[p];
            __syncthreads();
        }
        if (swap_s) {
            ++P;
            ++pass_local;
        }
        if (energy_log != nullptr) {
            const size_t row = (size_t)(s - a.log_s0);
            for (int i = tid; i < NT * kLanes; i += nthr) {
                const int t = i >> 5, b = i & 31;
                energy_log[(((row * a.G + g) * NT + t) * a.C + c) * kLanes + b] = E[i];
            }
        }
        if (meas) {
            if (a.esum != nullptr)
                for (int t = warp; t < NT; t += nthr / 32) {
                    long long v = E[t * kLanes + lane];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                    if (lane == 0) esum_s[t] += (unsigned long long)v;   // one warp per slot
                }
            if (cluster_measure) {
                cg::cluster_group cl = cg::this_cluster();
                for (int i = tid; i < NT * kLanes; i += nthr) nd[i] = 0;
                const uint32_t *other;
                if (snap_mode) {
                    // snapshot of my slots the partner measures (parity 1 - c)
                    uint32_t *sn = (n_meas & 1) ? snap1 : snap0;
                    for (int i = tid; i < half * N / 4; i += nthr) {
                        const int j = i / (N / 4), w = i - j * (N / 4);
                        const int t = 2 * j + (1 - c);
                        if (t < NT)
                            reinterpret_cast<uint4 *>(sn + (size_t)j * N)[w] =
                                reinterpret_cast<const uint4 *>(S + (size_t)t * N)[w];
                    }
                    cl.sync();   // both snapshots of sweep s are complete
                    other = cl.map_shared_rank(sn, c ^ 1);
                } else {
                    cl.sync();   // both copies have finished sweep s and its swap pass
                    other = cl.map_shared_rank(S, c ^ 1);
                }
                // one warp per measured slot t (parity c): lane-wise popcount of
                // copy0 ^ copy1 over the slot's words, summed over the warp
                constexpr int WPL = (N / 4 + 31) / 32;     // 16-byte words per lane
                constexpr int PLW = planes_for(4 * WPL);
                for (int t = 2 * warp + c; t < NT; t += 2 * (nthr / 32)) {
                    const uint4 *A4 = reinterpret_cast<const uint4 *>(S + (size_t)t * N);
                    const uint4 *B4 = reinterpret_cast<const uint4 *>(
                        other + (size_t)(snap_mode ? (t - c) / 2 : t) * N);
                    uint32_t oacc[PLW];
#pragma unroll
                    for (int q = 0; q < PLW; ++q) oacc[q] = 0;
#pragma unroll
                    for (int j = 0; j < WPL; ++j) {
                        const int w = lane + 32 * j;
                        if (w < N / 4) {
                            const uint4 x = A4[w], y = B4[w];
                            uint32_t s3, c1;
                            const uint32_t d0 = x.x ^ y.x, d1 = x.y ^ y.y, d2 = x.z ^ y.z, d3 = x.w ^ y.w;
                            full_add(d0, d1, d2, s3, c1);
                            uint32_t A[5] = {s3 ^ d3, c1 ^ (s3 & d3), c1 & (s3 & d3), 0u, 0u};
                            acc_add_sum5<PLW>(oacc, A);
                        }
                    }
                    warp_sum_to_lanes<PLW>(oacc, lane, &nd[t * kLanes]);
                }
                // live mode: the partner may modify its lattices only after this
                if (!snap_mode) cl.sync();
                else __syncthreads();
                if (a.qhist != nullptr)
                    for (int i = tid; i < NT * kLanes; i += nthr) {
                        const int t = i >> 5;
                        if ((t & 1) != c) continue;
                        if (hist_smem) atomicAdd(&hist[(size_t)(t >> 1) * (N + 1) + nd[i]], 1u);
                        else atomicAdd(reinterpret_cast<unsigned long long *>(
                                           a.qhist + (size_t)t * (N + 1) + nd[i]), 1ull);
                    }
                ++n_meas;
            }
            __syncthreads();   // E and nd are rewritten by the next sweep
        }
    }
    if (cluster_measure && snap_mode) cg::this_cluster().sync();   // partner done reading my snapshot
    for (int i = tid; i < NT * kLanes; i += nthr) a.energy[(size_t)unit * NT * kLanes + i] = E[i];
    if (a.esum != nullptr)
        for (int t = tid; t < NT; t += nthr)
            if (esum_s[t] != 0ull) atomicAdd(reinterpret_cast<unsigned long long *>(a.esum + t), esum_s[t]);
    if (hist_smem && a.qhist != nullptr)
        for (int i = tid; i < half * (N + 1); i += nthr) {
            const int j = i / (N + 1), k = i - j * (N + 1);
            const int t = 2 * j + c;
            if (t < NT && hist[i] != 0u)
                atomicAdd(reinterpret_cast<unsigned long long *>(a.qhist + (size_t)t * (N + 1) + k),
                          (unsigned long long)hist[i]);
        }
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

}  // namespace
}  // namespace ea
