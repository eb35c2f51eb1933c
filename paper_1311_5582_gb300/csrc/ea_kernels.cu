// Kernels of the parallel-tempering Metropolis simulation of the 3D +-J
// Edwards-Anderson model, written for sm_103a.
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
#include <cooperative_groups.h>

#include "ea_internal.h"

namespace cg = cooperative_groups;

namespace ea {

namespace {

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

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c)
{
    return (a & b) | (c & (a | b));
}
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy)
{
    s = a ^ b ^ c;
    cy = maj3(a, b, c);
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
    const uint32_t e0 = s ^ nb[0][j] ^ jb[0][j];
    const uint32_t e1 = s ^ nb[1][j] ^ jb[1][j];
    const uint32_t e2 = s ^ nb[2][j] ^ jb[2][j];
    const uint32_t e3 = s ^ nb[3][j] ^ jb[3][j];
    const uint32_t e4 = s ^ nb[4][j] ^ jb[4][j];
    const uint32_t e5 = s ^ nb[5][j] ^ jb[5][j];
    uint32_t a0, a1, b0, b1;
    full_add(e0, e1, e2, a0, a1);
    full_add(e3, e4, e5, b0, b1);
    u0 = a0 ^ b0;
    const uint32_t c = a0 & b0;
    full_add(a1, b1, c, u1, u2);
}

// Flip mask of a site: all lanes with dE <= 0 (u >= 3), and lanes with
// u >= m where m counts the thresholds r is not below (t0 <= t1 <= t2).
__device__ __forceinline__ uint32_t flip_mask(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t r,
                                              uint32_t t0, uint32_t t1, uint32_t t2)
{
    const uint32_t ge2 = u2 | u1;
    const uint32_t ge1 = ge2 | u0;
    const uint32_t ge3 = u2 | (u1 & u0);
    return (r < t0) ? kFull : (r < t1) ? ge1 : (r < t2) ? ge2 : ge3;
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

// Adds each thread's bit-sliced per-lane counter into out[group][lane],
// where a group is tpl consecutive threads (tpl a power of two dividing 32,
// or a multiple of 32).  The whole warp must call this.
__device__ __forceinline__ void reduce_counters(const uint32_t (&acc)[kPlanes], int tpl,
                                                int *out, int lane, int warp)
{
    uint32_t y[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) y[p] = warp_transpose(acc[p], lane);
    if (tpl >= 32) {
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p]) << p;
        const int grp = (warp * 32) / tpl;
        atomicAdd(&out[grp * kLanes + lane], cnt);
    } else {
        const int ng = 32 / tpl;
        const uint32_t base = (tpl == 32) ? kFull : ((1u << tpl) - 1u);
        for (int gi = 0; gi < ng; ++gi) {
            const uint32_t gm = base << (gi * tpl);
            int cnt = 0;
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p] & gm) << p;
            const int grp = (warp * 32 + gi * tpl) / tpl;
            atomicAdd(&out[grp * kLanes + lane], cnt);
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
    for (int j = 0; j < qper; ++j) {
        const int q = tl + j * tpl;
        if (q >= Gm::Q) break;
        Quad o;
        load_quad<L>(S, J, col, q, o);
        const uint4 r = philox((uint32_t)q, s, g, ctag, rk);
        const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
        uint32_t x0[4], x1[4], x2[4], ns[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t u0, u1, u2;
            unsat_count(o.s[i], o.nb, o.jb, i, u0, u1, u2);
            const uint32_t f = flip_mask(u0, u1, u2, rr[i], t0, t1, t2);
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

__device__ __forceinline__ bool swap_after(uint64_t s, uint32_t swap_every)
{
    return swap_every != 0 && ((s + 1) % swap_every) == 0;
}
__device__ __forceinline__ bool measured(uint64_t s, uint64_t from, uint32_t every)
{
    return every != 0 && s >= from && ((s - from) % every) == 0;
}

// Number of leading entries of a non-increasing threshold row above r: the
// swap of pair p is accepted iff E_p - E_{p+1} >= -4 * K (Sec. 2.4 with the
// integer table of Sec. 4.3.2).
__device__ __forceinline__ int accept_bound(const uint32_t *row, uint32_t len, uint32_t r)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(row + mid) > r) lo = mid + 1; else hi = mid;
    }
    return -4 * (int)lo;
}

__device__ __forceinline__ uint32_t swap_uniform(const RoundKeys &rk, int p, int b, uint64_t P,
                                                 uint32_t g, int c)
{
    const uint4 v = philox(((uint32_t)p << 3) | ((uint32_t)b >> 2), (uint32_t)P, g,
                           (1u << 24) | ((uint32_t)c << 8), rk);
    const int w = b & 3;
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

// ------------------------------------------------------------------ unit kernel
// One CTA owns all NT lattices of one (group, copy) unit in shared memory and
// runs the whole sweep range: Metropolis half-sweeps, per-lane energies,
// replica-exchange passes and measurements.  With C = 2 and overlap
// measurement the two copies of a group form a 2-CTA cluster and read each
// other's lattices through distributed shared memory.

struct UnitSmem {
    static size_t bytes(int N, int NT)
    {
        return (size_t)NT * N * 4 + (size_t)3 * N * 4 + (size_t)kMaxTemps * kLanes * 4 * 3 +
               (size_t)kMaxTemps * 4;
    }
};

template <int L>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sweep_unit(const __grid_constant__ SweepLaunch a, int tpl, int cluster_measure)
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    extern __shared__ uint4 smem_u4[];
    const int NT = (int)a.NT;
    uint32_t *S = reinterpret_cast<uint32_t *>(smem_u4);     // [NT][2][H]
    uint32_t *Js = S + (size_t)NT * N;                        // [3][2][H]
    int *E = reinterpret_cast<int *>(Js + 3 * N);             // [64][32] U, then E, by slot
    int *bnd = E + kMaxTemps * kLanes;                        // [64][32] swap accept bounds
    int *nd = bnd + kMaxTemps * kLanes;                       // [64][32] overlap counts
    uint32_t *msk = reinterpret_cast<uint32_t *>(nd + kMaxTemps * kLanes);  // [64]

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const int l = tid / tpl, tl = tid - l * tpl;   // my slot and rank in its group
    const int qper = (Gm::Q + tpl - 1) / tpl;

    uint32_t *gS = a.spins + (size_t)unit * NT * N;
    const uint32_t *gJ = a.bonds + (size_t)g * 3 * N;
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = reinterpret_cast<const uint4 *>(gS)[w];
    for (int w = tid; w < 3 * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
    const uint32_t t0 = a.metro[l * 3 + 0], t1 = a.metro[l * 3 + 1], t2 = a.metro[l * 3 + 2];
    uint32_t *mine = S + (size_t)l * N;
    __syncthreads();

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_now = swap_after(s, a.swap_every);
        const bool meas = measured(s, a.measure_from, a.measure_every);
        const bool needE = swap_now || a.energy_log != nullptr || meas || (n + 1 == a.n_sweeps);
        uint32_t acc[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
        if (needE)
            for (int i = tid; i < NT * kLanes; i += nthr) E[i] = 0;
        half_sweep<L, false>(mine, Js, 0, tl, tpl, qper, (uint32_t)s, g,
                             (0u << 16) | ((uint32_t)c << 8) | (uint32_t)l, a.rk, t0, t1, t2, acc);
        __syncthreads();
        if (needE) {
            half_sweep<L, true>(mine, Js, 1, tl, tpl, qper, (uint32_t)s, g,
                                (1u << 16) | ((uint32_t)c << 8) | (uint32_t)l, a.rk, t0, t1, t2, acc);
            reduce_counters(acc, tpl, E, lane, warp);
            __syncthreads();
            for (int i = tid; i < NT * kLanes; i += nthr) E[i] = 2 * E[i] - 3 * N;
            __syncthreads();
        } else {
            half_sweep<L, false>(mine, Js, 1, tl, tpl, qper, (uint32_t)s, g,
                                 (1u << 16) | ((uint32_t)c << 8) | (uint32_t)l, a.rk, t0, t1, t2, acc);
            __syncthreads();
        }
        if (swap_now) {
            if (NT > 1) {
                for (int i = tid; i < (NT - 1) * kLanes; i += nthr) {
                    const int p = i >> 5, b = i & 31;
                    const uint32_t r = swap_uniform(a.rk, p, b, P, g, c);
                    bnd[i] = accept_bound(a.swapt + (size_t)p * a.swap_len, a.swap_len, r);
                }
                __syncthreads();
                if (warp == 0) {
                    int cur = E[lane];
                    for (int p = 0; p + 1 < NT; ++p) {
                        const int nxt = E[(p + 1) * kLanes + lane];
                        const bool ok = (cur - nxt) >= bnd[p * kLanes + lane];
                        const uint32_t m = __ballot_sync(kFull, ok);
                        E[p * kLanes + lane] = ok ? nxt : cur;
                        cur = ok ? cur : nxt;
                        if (lane == 0) msk[p] = m;
                    }
                    E[(NT - 1) * kLanes + lane] = cur;
                }
                __syncthreads();
                // Masked exchange chain, pairs in order (0,1), (1,2), ...
                for (int w = tid; w < N; w += nthr) {
                    uint32_t x = S[w];
                    for (int p = 0; p + 1 < NT; ++p) {
                        const uint32_t y = S[(size_t)(p + 1) * N + w];
                        const uint32_t d = (x ^ y) & msk[p];
                        S[(size_t)p * N + w] = x ^ d;
                        x = y ^ d;
                    }
                    S[(size_t)(NT - 1) * N + w] = x;
                }
                if (a.swap_log != nullptr)
                    for (int p = tid; p + 1 < NT; p += nthr)
                        a.swap_log[(((size_t)pass_local * a.G + g) * a.C + c) * (NT - 1) + p] = msk[p];
                __syncthreads();
            }
            ++P;
            ++pass_local;
        }
        if (a.energy_log != nullptr) {
            const size_t row = (size_t)(s - a.log_s0);
            for (int i = tid; i < NT * kLanes; i += nthr) {
                const int t = i >> 5, b = i & 31;
                a.energy_log[(((row * a.G + g) * NT + t) * a.C + c) * kLanes + b] = E[i];
            }
        }
        if (meas) {
            if (a.esum != nullptr && warp < NT) {
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
                if ((l & 1) == c) {
                    const uint4 *A4 = reinterpret_cast<const uint4 *>(S + (size_t)l * N);
                    const uint4 *B4 = reinterpret_cast<const uint4 *>(other + (size_t)l * N);
                    for (int w = tl; w < N / 4; w += tpl) {
                        const uint4 x = A4[w], y = B4[w];
                        acc_add_words4(oacc, x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w);
                    }
                }
                reduce_counters(oacc, tpl, nd, lane, warp);
                cl.sync();   // the other copy may now modify its lattices again
                if (a.qhist != nullptr)
                    for (int i = tid; i < NT * kLanes; i += nthr) {
                        const int t = i >> 5;
                        if ((t & 1) == c)
                            atomicAdd(reinterpret_cast<unsigned long long *>(
                                          a.qhist + (size_t)t * (N + 1) + nd[i]), 1ull);
                    }
                __syncthreads();
            }
        }
    }
    // energies of the final state, spins back to global memory
    for (int i = tid; i < NT * kLanes; i += nthr) a.energy[(size_t)unit * NT * kLanes + i] = E[i];
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

// ------------------------------------------------------------------ chunked kernel
// For ensembles whose NT lattices do not fit one CTA: each CTA stages
// lattices [t0, t0 + nlat) of one unit, runs the sweeps up to the next swap
// point, and writes them back; the swap pass runs as its own kernels.

template <int L, bool J_SMEM>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sweep_chunk(const __grid_constant__ SweepLaunch a, int tpl, int nlat)
{
    using Gm = Geo<L>;
    constexpr int N = Gm::N;
    extern __shared__ uint4 smem_u4[];
    uint32_t *S = reinterpret_cast<uint32_t *>(smem_u4);                // [nlat][2][H]
    uint32_t *Js = S + (size_t)nlat * N;                                 // [3][2][H] if J_SMEM
    int *E = reinterpret_cast<int *>(Js + (J_SMEM ? 3 * N : 0));         // [64][32]

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const int tbase = (int)blockIdx.y * nlat;
    const int NT = (int)a.NT;
    const int l = tid / tpl, tl = tid - l * tpl;
    const int slot = tbase + l;
    const int nl_here = min(nlat, NT - tbase);
    const bool active = l < nl_here;
    const int qper = (Gm::Q + tpl - 1) / tpl;

    uint32_t *gS = a.spins + ((size_t)unit * NT + tbase) * N;
    const uint32_t *gJ = a.bonds + (size_t)g * 3 * N;
    for (int w = tid; w < nl_here * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = reinterpret_cast<const uint4 *>(gS)[w];
    const uint32_t *J = gJ;
    if constexpr (J_SMEM) {
        for (int w = tid; w < 3 * N / 4; w += nthr)
            reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
        J = Js;
    }
    uint32_t t0 = 0, t1 = 0, t2 = 0;
    if (active) { t0 = a.metro[slot * 3]; t1 = a.metro[slot * 3 + 1]; t2 = a.metro[slot * 3 + 2]; }
    uint32_t *mine = S + (size_t)l * N;
    __syncthreads();

    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool last = n + 1 == a.n_sweeps;
        const bool needE = a.energy_log != nullptr || (last && a.compute_energy_last);
        uint32_t acc[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
        if (needE)
            for (int i = tid; i < kMaxTemps * kLanes; i += nthr) E[i] = 0;
        if (active)
            half_sweep<L, false>(mine, J, 0, tl, tpl, qper, (uint32_t)s, g,
                                 (0u << 16) | ((uint32_t)c << 8) | (uint32_t)slot, a.rk, t0, t1, t2, acc);
        __syncthreads();
        if (needE) {
            if (active)
                half_sweep<L, true>(mine, J, 1, tl, tpl, qper, (uint32_t)s, g,
                                    (1u << 16) | ((uint32_t)c << 8) | (uint32_t)slot, a.rk, t0, t1, t2, acc);
            reduce_counters(acc, tpl, E, lane, warp);
            __syncthreads();
            for (int i = tid; i < nl_here * kLanes; i += nthr) {
                const int e = 2 * E[i] - 3 * N;
                const int t = tbase + (i >> 5), b = i & 31;
                if (a.energy_log != nullptr) {
                    const size_t row = (size_t)(s - a.log_s0);
                    a.energy_log[(((row * a.G + g) * NT + t) * a.C + c) * kLanes + b] = e;
                }
                if (last) a.energy[((size_t)unit * NT + t) * kLanes + b] = e;
            }
        } else if (active) {
            half_sweep<L, false>(mine, J, 1, tl, tpl, qper, (uint32_t)s, g,
                                 (1u << 16) | ((uint32_t)c << 8) | (uint32_t)slot, a.rk, t0, t1, t2, acc);
        }
        __syncthreads();
    }
    for (int w = tid; w < nl_here * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

// Swap decision of one pass for every unit: one CTA per unit.  Reads the
// energies by slot, writes the accepted-pair masks, permutes the energies.
__global__ void __launch_bounds__(256)
k_swap_decide(const __grid_constant__ SweepLaunch a, uint64_t P, uint32_t *masks_out,
              uint32_t *swap_log_row, int32_t *energy_log_row)
{
    __shared__ int bnd[kMaxTemps * kLanes];
    const int NT = (int)a.NT;
    const uint32_t unit = blockIdx.x;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < (NT - 1) * kLanes; i += blockDim.x) {
        const int p = i >> 5, b = i & 31;
        bnd[i] = accept_bound(a.swapt + (size_t)p * a.swap_len, a.swap_len,
                              swap_uniform(a.rk, p, b, P, g, c));
    }
    __syncthreads();
    if (warp == 0) {
        int32_t *E = a.energy + (size_t)unit * NT * kLanes;
        int cur = E[lane];
        for (int p = 0; p + 1 < NT; ++p) {
            const int nxt = E[(p + 1) * kLanes + lane];
            const bool ok = (cur - nxt) >= bnd[p * kLanes + lane];
            const uint32_t m = __ballot_sync(kFull, ok);
            E[p * kLanes + lane] = ok ? nxt : cur;
            cur = ok ? cur : nxt;
            if (lane == 0) {
                masks_out[(size_t)unit * (NT - 1) + p] = m;
                if (swap_log_row) swap_log_row[(size_t)unit * (NT - 1) + p] = m;
            }
        }
        E[(NT - 1) * kLanes + lane] = cur;
        if (energy_log_row)
            for (int t = 0; t < NT; ++t)
                energy_log_row[(((size_t)g * NT + t) * a.C + c) * kLanes + lane] = E[t * kLanes + lane];
    }
}

// Applies the masked exchange chain of one pass to spins in global memory.
__global__ void __launch_bounds__(256)
k_swap_apply(uint32_t *spins, const uint32_t *masks, int N, int NT)
{
    const uint32_t unit = blockIdx.y;
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= N) return;
    uint32_t *S = spins + (size_t)unit * NT * N;
    const uint32_t *m = masks + (size_t)unit * (NT - 1);
    uint32_t x = S[w];
    for (int p = 0; p + 1 < NT; ++p) {
        const uint32_t y = S[(size_t)(p + 1) * N + w];
        const uint32_t d = (x ^ y) & __ldg(m + p);
        S[(size_t)p * N + w] = x ^ d;
        x = y ^ d;
    }
    S[(size_t)(NT - 1) * N + w] = x;
}

// Energies recomputed from the spins: one CTA per lattice.
template <int L>
__global__ void __launch_bounds__(kMaxThreads)
k_energy(const uint32_t *spins, const uint32_t *bonds, int32_t *energy, uint32_t NT, uint32_t C)
{
    using Gm = Geo<L>;
    __shared__ int U[kLanes];
    const size_t lat = blockIdx.x;              // (unit, t)
    const uint32_t unit = (uint32_t)(lat / NT);
    const uint32_t g = unit / C;
    const uint32_t *S = spins + lat * Gm::N;
    const uint32_t *J = bonds + (size_t)g * 3 * Gm::N;
    const int tid = threadIdx.x, tpl = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kLanes) U[tid] = 0;
    __syncthreads();
    uint32_t acc[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
    for (int q = tid; q < Gm::Q; q += tpl) {
        Quad o;
        load_quad<L>(S, J, 1, q, o);
        uint32_t x0[4], x1[4], x2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) unsat_count(o.s[i], o.nb, o.jb, i, x0[i], x1[i], x2[i]);
        uint32_t A[5];
        quad_sum(x0, x1, x2, A);
        acc_add5(acc, A);
    }
    // all threads of the block form one group
    uint32_t y[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) y[p] = warp_transpose(acc[p], lane);
    int cnt = 0;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p]) << p;
    (void)warp;
    atomicAdd(&U[lane], cnt);
    __syncthreads();
    if (tid < kLanes) energy[lat * kLanes + tid] = 2 * U[tid] - 3 * Gm::N;
}

// Measurement pass: per (group, slot) overlap counts between the two copies,
// q histogram, energy sums and per-lane outputs by slot.
__global__ void __launch_bounds__(256)
k_measure(const uint32_t *spins, const int32_t *energy, int N, uint32_t NT, uint32_t C,
          int32_t *energies_out, uint32_t *ndiff_out, uint64_t *qhist, int64_t *esum)
{
    __shared__ int nd[kLanes];
    const uint32_t g = blockIdx.x / NT, t = blockIdx.x % NT;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < kLanes) nd[tid] = 0;
    __syncthreads();
    if (energies_out != nullptr && tid < (int)(C * kLanes)) {
        const int c = tid >> 5;
        energies_out[(((size_t)g * NT + t) * C + c) * kLanes + lane] =
            energy[(((size_t)g * C + c) * NT + t) * kLanes + lane];
    }
    if (esum != nullptr && tid < 32) {
        long long v = 0;
        for (uint32_t c = 0; c < C; ++c) v += energy[(((size_t)g * C + c) * NT + t) * kLanes + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(esum + t), (unsigned long long)v);
    }
    if (C == 2 && (ndiff_out != nullptr || qhist != nullptr)) {
        const uint4 *A4 = reinterpret_cast<const uint4 *>(spins + (((size_t)g * C + 0) * NT + t) * N);
        const uint4 *B4 = reinterpret_cast<const uint4 *>(spins + (((size_t)g * C + 1) * NT + t) * N);
        uint32_t acc[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
        // per-thread count <= 4 * ceil(N / 1024) <= 128 for L <= 32 (N <= 32768)
        for (int w = tid; w < N / 4; w += blockDim.x) {
            const uint4 x = A4[w], y = B4[w];
            acc_add_words4(acc, x.x ^ y.x, x.y ^ y.y, x.z ^ y.z, x.w ^ y.w);
        }
        uint32_t y[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) y[p] = warp_transpose(acc[p], lane);
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) cnt += __popc(y[p]) << p;
        atomicAdd(&nd[lane], cnt);
        __syncthreads();
        if (tid < kLanes) {
            if (ndiff_out != nullptr) ndiff_out[((size_t)g * NT + t) * kLanes + tid] = (uint32_t)nd[tid];
            if (qhist != nullptr)
                atomicAdd(reinterpret_cast<unsigned long long *>(qhist + (size_t)t * (N + 1) + nd[tid]), 1ull);
        }
    }
}

// API order [G][NT][C][N] (site order) <-> device [G][C][NT][2][H] (colour-split).
__device__ __forceinline__ int site_of(int L, int col, int k)
{
    const int R = L / 2;
    const int row = k / R;
    const int y = row % L, z = row / L;
    return 2 * k + ((col + y + z) & 1);
}

__global__ void k_import_spins(const uint32_t *api, uint32_t *dev, int L, uint32_t G, uint32_t NT,
                               uint32_t C)
{
    const int N = L * L * L, H = N / 2;
    const size_t total = (size_t)G * C * NT * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t lat = idx / N;              // (g, c, t)
        const uint32_t t = (uint32_t)(lat % NT);
        const uint32_t c = (uint32_t)((lat / NT) % C);
        const uint32_t g = (uint32_t)(lat / ((size_t)NT * C));
        const int col = w / H, k = w - col * H;
        dev[idx] = api[(((size_t)g * NT + t) * C + c) * N + site_of(L, col, k)];
    }
}

__global__ void k_export_spins(const uint32_t *dev, uint32_t *api, int L, uint32_t G, uint32_t NT,
                               uint32_t C)
{
    const int N = L * L * L, H = N / 2;
    const size_t total = (size_t)G * C * NT * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t lat = idx / N;
        const uint32_t t = (uint32_t)(lat % NT);
        const uint32_t c = (uint32_t)((lat / NT) % C);
        const uint32_t g = (uint32_t)(lat / ((size_t)NT * C));
        const int col = w / H, k = w - col * H;
        api[(((size_t)g * NT + t) * C + c) * N + site_of(L, col, k)] = dev[idx];
    }
}

__global__ void k_import_bonds(const uint32_t *api, uint32_t *dev, int L, uint32_t G)
{
    const int N = L * L * L, H = N / 2;
    const size_t total = (size_t)G * 3 * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(idx % N);
        const size_t gd = idx / N;               // (g, d)
        const int col = w / H, k = w - col * H;
        dev[idx] = api[gd * N + site_of(L, col, k)];
    }
}

int grid_for(size_t total, int threads)
{
    size_t b = (total + threads - 1) / threads;
    if (b > 65535 * 8) b = 65535 * 8;
    return (int)(b < 1 ? 1 : b);
}

template <int L>
cudaError_t launch_unit_L(const SweepLaunch &a, const Plan &plan, bool cluster_measure,
                          cudaStream_t st)
{
    auto kern = k_sweep_unit<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.G * a.C);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int nattr = 0;
    if (cluster_measure) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        nattr = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    return cudaLaunchKernelEx(&cfg, kern, a, plan.threads_per_lattice, cluster_measure ? 1 : 0);
}

template <int L>
cudaError_t launch_chunk_L(const SweepLaunch &a, const Plan &plan, cudaStream_t st)
{
    const int nchunks = ((int)a.NT + plan.lattices_per_cta - 1) / plan.lattices_per_cta;
    dim3 grid(a.G * a.C, nchunks);
    if (plan.j_in_smem) {
        auto kern = k_sweep_chunk<L, true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, plan.threads, plan.smem, st>>>(a, plan.threads_per_lattice, plan.lattices_per_cta);
    } else {
        auto kern = k_sweep_chunk<L, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, plan.threads, plan.smem, st>>>(a, plan.threads_per_lattice, plan.lattices_per_cta);
    }
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_energy_L(const uint32_t *spins, const uint32_t *bonds, int32_t *energy,
                            uint32_t G, uint32_t NT, uint32_t C, cudaStream_t st)
{
    constexpr int Q = Geo<L>::Q;
    int threads = 32;
    while (threads < kMaxThreads && (Q + threads - 1) / threads > kMaxQuadsPerThread) threads *= 2;
    k_energy<L><<<(unsigned)((size_t)G * C * NT), threads, 0, st>>>(spins, bonds, energy, NT, C);
    return cudaGetLastError();
}

#define EA_FOR_EACH_L(X) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(32)

}  // namespace

RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += kW0;
        k1 += kW1;
    }
    return rk;
}

bool supported_L(int L)
{
    switch (L) {
#define EA_CASE(X) case X: return true;
        EA_FOR_EACH_L(EA_CASE)
#undef EA_CASE
    default: return false;
    }
}

static int pow2_at_least(int x)
{
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

bool make_plan(int L, int NT, int C, size_t smem_optin, int tpl_override, Plan *plan)
{
    (void)C;
    if (NT < 1 || NT > kMaxTemps) return false;
    const int N = L * L * L, Q = N / 8;
    const int tpl_min = pow2_at_least((Q + kMaxQuadsPerThread - 1) / kMaxQuadsPerThread);
    auto fix_tpl = [&](int tpl, int nlat) {
        if (tpl < tpl_min) tpl = tpl_min;
        // whole warps only: shuffles in the energy reduction use full masks
        while ((tpl * nlat) % 32 != 0) tpl *= 2;
        return tpl;
    };
    // unit form: all NT lattices of a (group, copy) in one CTA
    {
        int tpl = tpl_override > 0 ? tpl_override : pow2_at_least((Q + 3) / 4);
        tpl = fix_tpl(tpl, NT);
        while (tpl * NT > kMaxThreads && tpl / 2 >= tpl_min && ((tpl / 2) * NT) % 32 == 0) tpl /= 2;
        const size_t smem = UnitSmem::bytes(N, NT);
        // overlap counting: per-thread words N / tpl must fit the 8-plane counter
        if (tpl * NT <= kMaxThreads && smem <= smem_optin && (N + tpl - 1) / tpl <= 255) {
            plan->unit = true;
            plan->threads_per_lattice = tpl;
            plan->lattices_per_cta = NT;
            plan->threads = tpl * NT;
            plan->smem = smem;
            plan->j_in_smem = true;
            return true;
        }
    }
    // chunked form: nlat lattices per CTA, swaps in their own kernels
    const size_t lat_bytes = (size_t)N * 4, j_bytes = (size_t)3 * N * 4;
    const size_t e_bytes = (size_t)kMaxTemps * kLanes * 4;
    const bool j_smem = j_bytes + lat_bytes + e_bytes <= smem_optin;
    const size_t budget = smem_optin - (j_smem ? j_bytes : 0) - e_bytes;
    int nlat = (int)(budget / lat_bytes);
    if (nlat < 1) return false;
    if (nlat > NT) nlat = NT;
    int tpl = tpl_override > 0 ? tpl_override : pow2_at_least((Q + 3) / 4);
    if (tpl < tpl_min) tpl = tpl_min;
    if (tpl > kMaxThreads) tpl = kMaxThreads;
    if (tpl < tpl_min) return false;
    while (nlat * tpl > kMaxThreads && nlat > 1) --nlat;
    while (nlat * tpl > kMaxThreads && tpl / 2 >= tpl_min) tpl /= 2;
    // prefer a divisor of NT so every CTA is full
    for (int d = nlat; d >= 1; --d)
        if (NT % d == 0) { nlat = d; break; }
    tpl = fix_tpl(tpl, nlat);
    if (nlat * tpl > kMaxThreads) return false;
    plan->unit = false;
    plan->threads_per_lattice = tpl;
    plan->lattices_per_cta = nlat;
    plan->threads = tpl * nlat;
    plan->smem = (size_t)nlat * lat_bytes + (j_smem ? j_bytes : 0) + e_bytes;
    plan->j_in_smem = j_smem;
    return true;
}

cudaError_t launch_import(const uint32_t *api_spins, const uint32_t *api_bonds, uint32_t *spins,
                          uint32_t *bonds, int L, uint32_t G, uint32_t NT, uint32_t C,
                          cudaStream_t st, uint64_t *launches)
{
    const size_t N = (size_t)L * L * L;
    k_import_spins<<<grid_for(G * C * NT * N, 256), 256, 0, st>>>(api_spins, spins, L, G, NT, C);
    k_import_bonds<<<grid_for(G * 3 * N, 256), 256, 0, st>>>(api_bonds, bonds, L, G);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_import_spins(const uint32_t *api_spins, uint32_t *spins, int L, uint32_t G,
                                uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches)
{
    const size_t N = (size_t)L * L * L;
    k_import_spins<<<grid_for(G * C * NT * N, 256), 256, 0, st>>>(api_spins, spins, L, G, NT, C);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_export(const uint32_t *spins, uint32_t *api_spins, int L, uint32_t G,
                          uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches)
{
    const size_t N = (size_t)L * L * L;
    k_export_spins<<<grid_for(G * C * NT * N, 256), 256, 0, st>>>(spins, api_spins, L, G, NT, C);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_sweep_unit(const SweepLaunch &a, int L, const Plan &plan, bool cluster_measure,
                              cudaStream_t st, uint64_t *launches)
{
    *launches += 1;
    switch (L) {
#define EA_CASE(X) case X: return launch_unit_L<X>(a, plan, cluster_measure, st);
        EA_FOR_EACH_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_chunk(const SweepLaunch &a, int L, const Plan &plan, cudaStream_t st,
                               uint64_t *launches)
{
    *launches += 1;
    switch (L) {
#define EA_CASE(X) case X: return launch_chunk_L<X>(a, plan, st);
        EA_FOR_EACH_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_swap_global(const SweepLaunch &a, int L, uint64_t P, uint32_t *masks,
                               int32_t *energy_log_row, cudaStream_t st, uint64_t *launches)
{
    if (a.NT < 2) return cudaSuccess;
    const int N = L * L * L;
    uint32_t *swap_log_row =
        a.swap_log ? a.swap_log + (size_t)a.pass_local0 * a.G * a.C * (a.NT - 1) : nullptr;
    k_swap_decide<<<a.G * a.C, 256, 0, st>>>(a, P, masks, swap_log_row, energy_log_row);
    dim3 grid((N + 255) / 256, a.G * a.C);
    k_swap_apply<<<grid, 256, 0, st>>>(a.spins, masks, N, (int)a.NT);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_energy(const uint32_t *spins, const uint32_t *bonds, int32_t *energy, int L,
                          uint32_t G, uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches)
{
    *launches += 1;
    switch (L) {
#define EA_CASE(X) case X: return launch_energy_L<X>(spins, bonds, energy, G, NT, C, st);
        EA_FOR_EACH_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_measure(const uint32_t *spins, const int32_t *energy, int L, uint32_t G,
                           uint32_t NT, uint32_t C, int32_t *energies_out, uint32_t *ndiff_out,
                           uint64_t *qhist, int64_t *esum, cudaStream_t st, uint64_t *launches)
{
    const int N = L * L * L;
    k_measure<<<G * NT, 256, 0, st>>>(spins, energy, N, NT, C, energies_out, ndiff_out, qhist, esum);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace ea
