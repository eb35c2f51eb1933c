// Device building blocks shared by the sweep kernels (included by each
// kernel translation unit; everything here is internal linkage).
//
// Sec. 4.3 of the paper turns the Metropolis step into bit operations on
// multispin-coded words (XOR bond energies, a local energy E in 0..6, a table
// compare).  Here 32 disorder realizations share a word (one bit each), so one
// 32-bit operation advances 32 realizations:
//   e_d = s ^ s_nb ^ J_d                      (Eq. e: 1 = unsatisfied bond)
//   (u2 u1 u0) = e_0 + ... + e_5              (bit-sliced full-adder tree)
//   flip lanes with u >= m, m = #thresholds r has passed (Eq. r, Sec. 4.3.2)
// which is exact because the three thresholds of a slot are monotone.
// Random numbers come from Philox4x32-10 (Sec. 4.3.2 evaluates this generator
// family), one 32-bit output per (group, slot, copy, sweep, site) shared by
// the 32 lanes; one call serves the four sites of a quad.
#pragma once

#include <cooperative_groups.h>

#include "ea_internal.h"

namespace ea {
namespace {

namespace cg = cooperative_groups;


constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;   // Philox4x32 multipliers
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;   // Philox Weyl key increments
constexpr uint32_t kFull = 0xFFFFFFFFu;

template <int L>
struct Geo {
    static constexpr int N = L * L * L;
    static constexpr int H = N / 2;   // sites per colour
    static constexpr int R = L / 2;   // sites per row per colour
    static constexpr int Q = N / 8;   // quads (four consecutive class indices) per colour
};

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const RoundKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kM0 * c0, hi0 = __umulhi(kM0, c0);
        const uint32_t lo1 = kM1 * c2, hi1 = __umulhi(kM1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ rk.k[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk.k[2 * r + 1];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// One three-input logic operation with the truth table LUT over the operand
// patterns a = 0xF0, b = 0xCC, c = 0xAA, written out so that the compiler
// keeps the bit-sliced expressions in the form given here.
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}
constexpr uint32_t kXor3 = 0x96u;                   // a ^ b ^ c
constexpr uint32_t kMaj3 = 0xE8u;                   // majority
constexpr uint32_t kOr3 = 0xFEu;                    // a | b | c
constexpr uint32_t kAndOr = 0xEAu;                  // (a & b) | c
constexpr uint32_t kXorOr = 0x1Eu;                  // a ^ (b | c)
constexpr uint32_t kAndOr2 = 0xE0u;                 // a & (b | c)
constexpr uint32_t kOrAnd = 0xF8u;                  // a | (b & c)
constexpr uint32_t kXorAndN = 0xB4u;                // a ^ (b & ~c)
constexpr uint32_t kSelNot = 0x3Au;                 // a ? ~b : c
static_assert(((0xF0u ^ 0xCCu ^ 0xAAu) & 0xFFu) == kXor3 && (((0xF0u & 0xCCu) | (0xAAu & (0xF0u | 0xCCu))) & 0xFFu) == kMaj3 &&
              ((0xF0u | 0xCCu | 0xAAu) & 0xFFu) == kOr3 && (((0xF0u & 0xCCu) | 0xAAu) & 0xFFu) == kAndOr &&
              ((0xF0u ^ (0xCCu | 0xAAu)) & 0xFFu) == kXorOr && ((0xF0u & (0xCCu | 0xAAu)) & 0xFFu) == kAndOr2 &&
              ((0xF0u | (0xCCu & 0xAAu)) & 0xFFu) == kOrAnd && ((0xF0u ^ (0xCCu & ~0xAAu)) & 0xFFu) == kXorAndN &&
              (((0xF0u & ~0xCCu) | (~0xF0u & 0xAAu)) & 0xFFu) == kSelNot,
              "truth tables");

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return lop3<kMaj3>(a, b, c); }
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy)
{
    s = lop3<kXor3>(a, b, c);
    cy = lop3<kMaj3>(a, b, c);
}

// The words one quad update reads: own spins, the six neighbour spins and the
// six bond words of each of its four sites.  Index order of the six:
// +x, -x, +y, -y, +z, -z; the -d bond's J is stored at the neighbour.
struct Quad {
    uint32_t s[4];
    uint32_t nb[6][4];
    uint32_t jb[6][4];
};

// Loads quad q of colour col.  S: lattice base [2][H]; J: bond base [3][2][H].
// Works on shared or global pointers.
template <int L>
__device__ __forceinline__ void load_quad(const uint32_t *__restrict__ S,
                                          const uint32_t *__restrict__ J, int col, int q, Quad &o)
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N, H = Gm::H, R = Gm::R;
    const uint32_t *Sc = S + col * H;
    const uint32_t *So = S + (col ^ 1) * H;
    const int k0 = 4 * q;
    if constexpr (L % 8 == 0) {
        // The quad's four sites sit in one x-row: vector loads.
        const int row = k0 / R, m0 = k0 - row * R;
        const int y = row % L, z = row / L;
        const int px = (y + z + col) & 1;      // x parity of this colour in this row
        const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
        const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
        const int rowb = row * R;
        const uint4 own = *reinterpret_cast<const uint4 *>(Sc + k0);
        const uint4 xo = *reinterpret_cast<const uint4 *>(So + k0);
        const uint4 vyp = *reinterpret_cast<const uint4 *>(So + m0 + R * (yp + L * z));
        const uint4 vym = *reinterpret_cast<const uint4 *>(So + m0 + R * (ym + L * z));
        const uint4 vzp = *reinterpret_cast<const uint4 *>(So + m0 + R * (y + L * zp));
        const uint4 vzm = *reinterpret_cast<const uint4 *>(So + m0 + R * (y + L * zm));
        const uint4 jcx = *reinterpret_cast<const uint4 *>(J + 0 * N + col * H + k0);
        const uint4 jcy = *reinterpret_cast<const uint4 *>(J + 1 * N + col * H + k0);
        const uint4 jcz = *reinterpret_cast<const uint4 *>(J + 2 * N + col * H + k0);
        const uint4 jox = *reinterpret_cast<const uint4 *>(J + 0 * N + (col ^ 1) * H + k0);
        const uint4 joy = *reinterpret_cast<const uint4 *>(J + 1 * N + (col ^ 1) * H + m0 + R * (ym + L * z));
        const uint4 joz = *reinterpret_cast<const uint4 *>(J + 2 * N + (col ^ 1) * H + m0 + R * (y + L * zm));
        // x neighbours: same class index in the other colour, plus one word
        // across the quad edge (x-1 of the first site when px = 0, x+1 of the
        // last site when px = 1), wrapping inside the row.
        uint32_t xs_extra, xj_extra;
        if constexpr (R == 4) {
            xs_extra = px ? xo.x : xo.w;
            xj_extra = jox.w;   // only used when px = 0
        } else {
            const int ie = px ? (m0 + 4 == R ? 0 : m0 + 4) : (m0 == 0 ? R - 1 : m0 - 1);
            xs_extra = So[rowb + ie];
            xj_extra = J[0 * N + (col ^ 1) * H + rowb + ie];
        }
        o.s[0] = own.x; o.s[1] = own.y; o.s[2] = own.z; o.s[3] = own.w;
        // +x
        o.nb[0][0] = px ? xo.y : xo.x;
        o.nb[0][1] = px ? xo.z : xo.y;
        o.nb[0][2] = px ? xo.w : xo.z;
        o.nb[0][3] = px ? xs_extra : xo.w;
        // -x
        o.nb[1][0] = px ? xo.x : xs_extra;
        o.nb[1][1] = px ? xo.y : xo.x;
        o.nb[1][2] = px ? xo.z : xo.y;
        o.nb[1][3] = px ? xo.w : xo.z;
        o.nb[2][0] = vyp.x; o.nb[2][1] = vyp.y; o.nb[2][2] = vyp.z; o.nb[2][3] = vyp.w;
        o.nb[3][0] = vym.x; o.nb[3][1] = vym.y; o.nb[3][2] = vym.z; o.nb[3][3] = vym.w;
        o.nb[4][0] = vzp.x; o.nb[4][1] = vzp.y; o.nb[4][2] = vzp.z; o.nb[4][3] = vzp.w;
        o.nb[5][0] = vzm.x; o.nb[5][1] = vzm.y; o.nb[5][2] = vzm.z; o.nb[5][3] = vzm.w;
        o.jb[0][0] = jcx.x; o.jb[0][1] = jcx.y; o.jb[0][2] = jcx.z; o.jb[0][3] = jcx.w;
        // -x bond: J of the -x neighbour
        o.jb[1][0] = px ? jox.x : xj_extra;
        o.jb[1][1] = px ? jox.y : jox.x;
        o.jb[1][2] = px ? jox.z : jox.y;
        o.jb[1][3] = px ? jox.w : jox.z;
        o.jb[2][0] = jcy.x; o.jb[2][1] = jcy.y; o.jb[2][2] = jcy.z; o.jb[2][3] = jcy.w;
        o.jb[3][0] = joy.x; o.jb[3][1] = joy.y; o.jb[3][2] = joy.z; o.jb[3][3] = joy.w;
        o.jb[4][0] = jcz.x; o.jb[4][1] = jcz.y; o.jb[4][2] = jcz.z; o.jb[4][3] = jcz.w;
        o.jb[5][0] = joz.x; o.jb[5][1] = joz.y; o.jb[5][2] = joz.z; o.jb[5][3] = joz.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = k0 + j;
            const int row = k / R, m = k - row * R;
            const int y = row % L, z = row / L;
            const int px = (y + z + col) & 1;
            const int rowb = row * R;
            const int kxp = rowb + (px ? (m + 1 == R ? 0 : m + 1) : m);
            const int kxm = rowb + (px ? m : (m == 0 ? R - 1 : m - 1));
            const int yp = (y + 1 == L) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
            const int zp = (z + 1 == L) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
            const int kyp = m + R * (yp + L * z), kym = m + R * (ym + L * z);
            const int kzp = m + R * (y + L * zp), kzm = m + R * (y + L * zm);
            o.s[j] = Sc[k];
            o.nb[0][j] = So[kxp];
            o.nb[1][j] = So[kxm];
            o.nb[2][j] = So[kyp];
            o.nb[3][j] = So[kym];
            o.nb[4][j] = So[kzp];
            o.nb[5][j] = So[kzm];
            o.jb[0][j] = J[0 * N + col * H + k];
            o.jb[1][j] = J[0 * N + (col ^ 1) * H + kxm];
            o.jb[2][j] = J[1 * N + col * H + k];
            o.jb[3][j] = J[1 * N + (col ^ 1) * H + kym];
            o.jb[4][j] = J[2 * N + col * H + k];
            o.jb[5][j] = J[2 * N + (col ^ 1) * H + kzm];
        }
    }
}

// Number of unsatisfied bonds u = (u2 u1 u0) of the 32 lanes of one site.
__device__ __forceinline__ void unsat_count(uint32_t s, const uint32_t (&nb)[6][4],
                                            const uint32_t (&jb)[6][4], int j, uint32_t &u0,
                                            uint32_t &u1, uint32_t &u2)
{
    const uint32_t e0 = lop3<kXor3>(s, nb[0][j], jb[0][j]);
    const uint32_t e1 = lop3<kXor3>(s, nb[1][j], jb[1][j]);
    const uint32_t e2 = lop3<kXor3>(s, nb[2][j], jb[2][j]);
    const uint32_t e3 = lop3<kXor3>(s, nb[3][j], jb[3][j]);
    const uint32_t e4 = lop3<kXor3>(s, nb[4][j], jb[4][j]);
    const uint32_t e5 = lop3<kXor3>(s, nb[5][j], jb[5][j]);
    uint32_t a0, a1, b0, b1;
    full_add(e0, e1, e2, a0, a1);
    full_add(e3, e4, e5, b0, b1);
    u0 = a0 ^ b0;
    const uint32_t c = a0 & b0;
    full_add(a1, b1, c, u1, u2);
}

// All-ones iff r < T, for a threshold T <= 2^32 held as 2^64 - T: the high
// word of r + 2^64 - T, formed by one wide multiply-add (an add with carry
// after assembly: one ALU and one FMA-pipe instruction).
__device__ __forceinline__ uint32_t below_wide(uint32_t r, uint64_t neg_t)
{
    uint64_t d;
    asm("mad.wide.u32 %0, %1, 1, %2;" : "=l"(d) : "r"(r), "l"(neg_t));
    return (uint32_t)(d >> 32);
}

// Flip mask of a site: all lanes with dE <= 0 (u >= 3), and lanes with
// u >= m where m counts the thresholds r is not below (t0 <= t1 <= t2, given
// as 2^64 - t).
__device__ __forceinline__ uint32_t flip_mask(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t r,
                                              uint64_t n0, uint64_t n1, uint64_t n2)
{
    // the masks are nested (m0 => m1 => m2), so
    //   [u>=3] | m2 [u>=2] | m1 [u>=1] | m0 = u2 | u1 (u0 | m2) | u0 m1 | m0
    const uint32_t m0 = below_wide(r, n0), m1 = below_wide(r, n1), m2 = below_wide(r, n2);
    return lop3<kOrAnd>(lop3<kOr3>(lop3<kAndOr2>(u1, u0, m2), u2, m0), u0, m1);
}

// Sum of four 3-bit lane values (x2 x1 x0)[j] into a 5-bit value A.
__device__ __forceinline__ void quad_sum(const uint32_t (&x0)[4], const uint32_t (&x1)[4],
                                         const uint32_t (&x2)[4], uint32_t (&A)[5])
{
    uint32_t s, ca, cb, c1, c2, c3, s2, k1, k2, k3;
    full_add(x0[0], x0[1], x0[2], s, ca);
    A[0] = s ^ x0[3]; cb = s & x0[3];
    full_add(ca, cb, x1[0], s, c1);
    full_add(s, x1[1], x1[2], s2, c2);
    A[1] = s2 ^ x1[3]; c3 = s2 & x1[3];
    full_add(c1, c2, c3, s, k1);
    full_add(x2[0], x2[1], x2[2], s2, k2);
    full_add(s, s2, x2[3], A[2], k3);
    full_add(k1, k2, k3, A[3], A[4]);
}

// acc += A (bit-sliced ripple add of a 5-bit value into kPlanes planes).
__device__ __forceinline__ void acc_add5(uint32_t (&acc)[kPlanes], const uint32_t (&A)[5])
{
    uint32_t cy = acc[0] & A[0];
    acc[0] ^= A[0];
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        uint32_t s, c;
        full_add(acc[i], A[i], cy, s, c);
        acc[i] = s;
        cy = c;
    }
#pragma unroll
    for (int i = 5; i < kPlanes; ++i) {
        const uint32_t c = acc[i] & cy;
        acc[i] ^= cy;
        cy = c;
    }
}

// acc += popcount-per-lane of four words (3-bit partial sum, then ripple).
__device__ __forceinline__ void acc_add_words4(uint32_t (&acc)[kPlanes], uint32_t w0, uint32_t w1,
                                               uint32_t w2, uint32_t w3)
{
    uint32_t s, c1;
    full_add(w0, w1, w2, s, c1);
    const uint32_t b0 = s ^ w3, c2 = s & w3;
    const uint32_t b1 = c1 ^ c2, b2 = c1 & c2;
    uint32_t A[5] = {b0, b1, b2, 0u, 0u};
    acc_add5(acc, A);
}

// 32x32 bit transpose across a warp: afterwards bit j of lane b's word is
// bit b of lane j's word before.
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane)
{
#define EA_TSTEP(S, M)                                                              \
    {                                                                               \
        const uint32_t y = __shfl_xor_sync(kFull, x, S);                            \
        x = (lane & S) ? ((x & ~(M)) | ((y >> S) & (M))) : ((x & (M)) | ((y << S) & ~(M))); \
    }
    EA_TSTEP(16, 0x0000FFFFu)
    EA_TSTEP(8, 0x00FF00FFu)
    EA_TSTEP(4, 0x0F0F0F0Fu)
    EA_TSTEP(2, 0x33333333u)
    EA_TSTEP(1, 0x55555555u)
#undef EA_TSTEP
    return x;
}

// Adds scale x each thread's bit-sliced per-lane counter into out[group][lane],
// where a group is tpl consecutive threads (tpl a power of two dividing 32,
// or a multiple of 32); groups at or beyond ngroups are idle threads and add
// nothing.  The whole warp must call this.
__device__ __forceinline__ void reduce_counters(const uint32_t (&acc)[kPlanes], int tpl,
                                                int *out, int lane, int warp, int scale, int ngroups)
{
    uint32_t y[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) y[p] = warp_transpose(acc[p], lane);
    if (tpl >= 32) {
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p]) << p;
        const int grp = (warp * 32) / tpl;
        if (grp < ngroups) atomicAdd(&out[grp * kLanes + lane], scale * cnt);
    } else {
        const int ng = 32 / tpl;
        const uint32_t base = (tpl == 32) ? kFull : ((1u << tpl) - 1u);
        for (int gi = 0; gi < ng; ++gi) {
            const uint32_t gm = base << (gi * tpl);
            int cnt = 0;
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p] & gm) << p;
            const int grp = (warp * 32 + gi * tpl) / tpl;
            if (grp < ngroups) atomicAdd(&out[grp * kLanes + lane], scale * cnt);
        }
    }
}

// One half-sweep (colour col) of one lattice by the tpl threads of its group;
// thread tl takes quads tl, tl + tpl, ...  With WITH_E, acc receives the
// post-update unsatisfied-bond counts of the colour-1 sites (every bond has
// exactly one colour-1 end, so they sum to U, E = 2U - 3N).
template <int L, bool WITH_E>
__device__ __forceinline__ void half_sweep(uint32_t *S, const uint32_t *J, int col, int tl, int tpl,
                                           int qper, uint32_t s, uint32_t g, uint32_t ctag,
                                           const RoundKeys &rk, uint32_t t0, uint32_t t1,
                                           uint32_t t2, uint32_t (&acc)[kPlanes])
{
    using Gm = Geo<L>;
    uint32_t *Sc = S + col * Gm::H;
    const uint64_t n0 = 0ull - (uint64_t)t0, n1 = 0ull - (uint64_t)t1, n2 = 0ull - (uint64_t)t2;
    for (int j = 0; j < qper; ++j) {
        const int q = tl + j * tpl;
        if (q >= Gm::Q) break;
        Quad o;
        load_quad<L>(S, J, col, q, o);
        const uint4 r = philox((uint32_t)q, ctag, s, g, rk);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        uint32_t x0[4], x1[4], x2[4], ns[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t u0, u1, u2;
            unsat_count(o.s[i], o.nb, o.jb, i, u0, u1, u2);
            const uint32_t f = flip_mask(u0, u1, u2, rr[i], n0, n1, n2);
            ns[i] = o.s[i] ^ f;
            if constexpr (WITH_E) {
                // after a flip the six bonds change state: u' = 6 - u
                x0[i] = u0;
                x1[i] = u1 ^ (f & ~u0);
                x2[i] = u2 ^ (f & ~(u0 & u1));
            }
        }
        *reinterpret_cast<uint4 *>(Sc + 4 * q) = make_uint4(ns[0], ns[1], ns[2], ns[3]);
        if constexpr (WITH_E) {
            uint32_t A[5];
            quad_sum(x0, x1, x2, A);
            acc_add5(acc, A);
        }
    }
}

// ------------------------------------------------------------ external field
// With h = h_num / h_den != 0 (Eq. 1) a flip of spin S with u unsatisfied
// bonds changes Et = h_den E - h_num M by h_den (12 - 4u) + 2 h_num S; it is
// accepted iff r < T[S > 0][u], with T[sp][u] = 2^32 (always) where that change
// is <= 0.  The kernels hold each threshold as 2^64 - T (below_wide), which
// also gives "always" for T = 2^32 and "never" for T = 0.

// Flip mask in a field: s the spin word, NTh the slot's 14 thresholds [sp][u]
// as 2^64 - T.  For each spin value the table is non-decreasing in u, so the
// accepted u form a suffix and the mask is the OR over u of [u_lane >= u] and
// "r < T[u]".
__device__ __forceinline__ uint32_t flip_mask_field(uint32_t s, uint32_t u0, uint32_t u1, uint32_t u2,
                                                    uint32_t r, const uint64_t (&NTh)[14])
{
    const uint32_t ge2 = u1 | u2, ge1 = ge2 | u0, ge3 = u2 | (u1 & u0);
    const uint32_t ge4 = u2, ge5 = u2 & (u1 | u0), ge6 = u2 & u1;
    uint32_t f[2];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        const int o = 7 * sp;
        f[sp] = below_wide(r, NTh[o]) | (ge1 & below_wide(r, NTh[o + 1])) |
                (ge2 & below_wide(r, NTh[o + 2])) | (ge3 & below_wide(r, NTh[o + 3])) |
                (ge4 & below_wide(r, NTh[o + 4])) | (ge5 & below_wide(r, NTh[o + 5])) |
                (ge6 & below_wide(r, NTh[o + 6]));
    }
    return (s & f[1]) | (~s & f[0]);
}

// Adds one word to a bit-sliced per-lane counter.
__device__ __forceinline__ void acc_add_word(uint32_t (&acc)[kPlanes], uint32_t w)
{
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const uint32_t c = acc[p] & w;
        acc[p] ^= w;
        w = c;
    }
}

// half_sweep in a field (thresholds as 2^64 - T): WITH_E as there; WITH_M
// counts the up spins of the updated sites into accM.
template <int L, bool WITH_E, bool WITH_M>
__device__ __forceinline__ void half_sweep_field(uint32_t *S, const uint32_t *J, int col, int tl, int tpl,
                                                 int qper, uint32_t s, uint32_t g, uint32_t ctag,
                                                 const RoundKeys &rk, const uint64_t (&NTh)[14],
                                                 uint32_t (&acc)[kPlanes], uint32_t (&accM)[kPlanes])
{
    using Gm = Geo<L>;
    uint32_t *Sc = S + col * Gm::H;
    for (int j = 0; j < qper; ++j) {
        const int q = tl + j * tpl;
        if (q >= Gm::Q) break;
        Quad o;
        load_quad<L>(S, J, col, q, o);
        const uint4 r = philox((uint32_t)q, ctag, s, g, rk);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        uint32_t x0[4], x1[4], x2[4], ns[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t u0, u1, u2;
            unsat_count(o.s[i], o.nb, o.jb, i, u0, u1, u2);
            const uint32_t f = flip_mask_field(o.s[i], u0, u1, u2, rr[i], NTh);
            ns[i] = o.s[i] ^ f;
            if constexpr (WITH_E) {
                x0[i] = u0;
                x1[i] = u1 ^ (f & ~u0);
                x2[i] = u2 ^ (f & ~(u0 & u1));
            }
        }
        *reinterpret_cast<uint4 *>(Sc + 4 * q) = make_uint4(ns[0], ns[1], ns[2], ns[3]);
        if constexpr (WITH_E) {
            uint32_t A[5];
            quad_sum(x0, x1, x2, A);
            acc_add5(acc, A);
        }
        if constexpr (WITH_M) {
#pragma unroll
            for (int i = 0; i < 4; ++i) acc_add_word(accM, ns[i]);
        }
    }
}

__device__ __forceinline__ bool swap_after(uint64_t s, uint32_t swap_every)
{
    return swap_every != 0 && ((s + 1) % swap_every) == 0;
}
__device__ __forceinline__ bool measured(uint64_t s, uint64_t from, uint32_t every)
{
    return every != 0 && s >= from && ((s - from) % every) == 0;
}

// The same schedules without a 64-bit division per sweep: the number of
// sweeps until the next selected one is formed once (one division) and
// counted down.  step() tells whether the current sweep is selected and
// moves on to the next.
struct SwapCountdown {          // sweeps s with (s + 1) % every == 0
    uint32_t every, left;
    __device__ SwapCountdown(uint64_t s0, uint32_t every_) : every(every_), left(0)
    {
        if (every) left = every - 1u - (uint32_t)(s0 % every);
    }
    __device__ __forceinline__ bool step()
    {
        if (every == 0) return false;
        const bool now = left == 0;
        left = now ? every - 1u : left - 1u;
        return now;
    }
};
struct MeasureCountdown {       // sweeps s >= from with (s - from) % every == 0
    uint32_t every;
    uint64_t left;
    __device__ MeasureCountdown(uint64_t s0, uint64_t from, uint32_t every_) : every(every_), left(0)
    {
        if (every) left = s0 >= from ? (uint64_t)((every - (uint32_t)((s0 - from) % every)) % every) : from - s0;
    }
    __device__ __forceinline__ bool step()
    {
        if (every == 0) return false;
        const bool now = left == 0;
        left = now ? (uint64_t)(every - 1u) : left - 1u;
        return now;
    }
};

// Number of leading entries of a non-increasing threshold row above r: the
// swap of pair p is accepted iff E_p - E_{p+1} >= -4 * K (Sec. 2.4 with the
// integer table of Sec. 4.3.2).
__device__ __forceinline__ int accept_bound(const uint32_t *row, uint32_t len, uint32_t r)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (row[mid] > r) lo = mid + 1; else hi = mid;   // row: shared or global
    }
    return -4 * (int)lo;
}

__device__ __forceinline__ uint32_t swap_uniform(const RoundKeys &rk, int p, int b, uint64_t P,
                                                 uint32_t g, int c)
{
    const uint4 v = philox(((uint32_t)p << 3) | ((uint32_t)b >> 2), (1u << 24) | ((uint32_t)c << 8),
                           (uint32_t)P, g, rk);
    const int w = b & 3;
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}


struct UnitSmem {
    // m units of NT lattices and their bonds, energies, bounds, overlap counts, masks
    static size_t base_bytes(int N, int NT, int m = 1)
    {
        return (size_t)m * NT * N * 4 + (size_t)m * 3 * N * 4 + (size_t)kMaxTemps * kLanes * 4 * 3 +
               (size_t)kMaxTemps * 4;
    }
    static size_t swap_bytes(int NT, uint32_t swap_len)
    {
        return NT > 1 ? (size_t)(NT - 1) * swap_len * 4 : 0;
    }
};

}  // namespace
}  // namespace ea
