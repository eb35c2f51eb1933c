// Unit sweep kernel specialised for lattices with L % 8 == 0 (L = 8, 16).
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

// Metropolis update of one quad of colour COL whose rows have x parity PX.
template <int L, int COL, int PX, bool WITH_E, int PL>
__device__ __forceinline__ void quad_fast(uint32_t *S, const uint32_t *J, const QuadRow &d,
                                          uint32_t s, uint32_t g, uint32_t ctag, const RoundKeys &rk,
                                          uint32_t t0, uint32_t t1, uint32_t t2, uint32_t (&acc)[PL])
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
    const uint4 r = philox((uint32_t)(d.k0 >> 2), ctag, s, g, rk);
    const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
    uint32_t ns[4], x0[4], x1[4], x2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t sj = sv[j];
        const uint32_t e0 = sj ^ nxp[j] ^ jx[j];
        const uint32_t e1 = sj ^ nxm[j] ^ jxm[j];
        const uint32_t e2 = sj ^ ny[j] ^ jy[j];
        const uint32_t e3 = sj ^ my[j] ^ jym[j];
        const uint32_t e4 = sj ^ nz[j] ^ jz[j];
        const uint32_t e5 = sj ^ mz[j] ^ jzm[j];
        uint32_t a0, a1, b0, b1, u0, u1, u2;
        full_add(e0, e1, e2, a0, a1);
        full_add(e3, e4, e5, b0, b1);
        u0 = a0 ^ b0;
        full_add(a1, b1, a0 & b0, u1, u2);
        const uint32_t f = flip_mask(u0, u1, u2, rr[j], t0, t1, t2);
        ns[j] = sj ^ f;
        if constexpr (WITH_E) {
            x0[j] = u0;
            x1[j] = u1 ^ (f & ~u0);
            x2[j] = u2 ^ (f & ~(u0 & u1));
        }
    }
    *reinterpret_cast<uint4 *>(Sc + d.k0) = make_uint4(ns[0], ns[1], ns[2], ns[3]);
    if constexpr (WITH_E) {
        uint32_t A[5];
        quad_sum(x0, x1, x2, A);
        acc_add_sum5<PL>(acc, A);
    }
}

template <int L, int QPER, int COL, int PX, bool WITH_E, int PL>
__device__ __forceinline__ void half_fast(uint32_t *S, const uint32_t *J, const QuadRow (&qd)[QPER],
                                          const bool (&qv)[QPER], uint32_t s, uint32_t g,
                                          uint32_t ctag, const RoundKeys &rk, uint32_t t0,
                                          uint32_t t1, uint32_t t2, uint32_t (&acc)[PL])
{
#pragma unroll
    for (int j = 0; j < QPER; ++j)
        if (qv[j]) quad_fast<L, COL, PX, WITH_E, PL>(S, J, qd[j], s, g, ctag, rk, t0, t1, t2, acc);
}

template <int PL, int HP>
__device__ __forceinline__ void reduce_fast(const uint32_t (&acc)[PL], int *out, int lane, int warp,
                                            int scale, int NT)
{
    uint32_t y[PL];
#pragma unroll
    for (int p = 0; p < PL; ++p) y[p] = warp_transpose(acc[p], lane);
    if constexpr (HP >= 32) {
        int cnt = 0;
#pragma unroll
        for (int p = 0; p < PL; ++p) cnt += __popc(y[p]) << p;
        const int l = FastMap<HP>::group_lattice(warp, 0);
        if (l < NT) atomicAdd(&out[l * kLanes + lane], scale * cnt);
    } else {
#pragma unroll
        for (int gi = 0; gi < 32 / HP; ++gi) {
            const uint32_t gm = ((1u << HP) - 1u) << (gi * HP);
            int cnt = 0;
#pragma unroll
            for (int p = 0; p < PL; ++p) cnt += __popc(y[p] & gm) << p;
            const int l = FastMap<HP>::group_lattice(warp, gi);
            if (l < NT) atomicAdd(&out[l * kLanes + lane], scale * cnt);
        }
    }
}

template <int L, int HP>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sweep_unit_fast(const __grid_constant__ SweepLaunch a, int cluster_measure, int swap_in_smem)
{
    using Gm = Geo<L>;
    using Mp = FastMap<HP>;
    constexpr int N = Gm::N;
    constexpr int QP = Gm::Q / 2;                       // quads per (colour, row parity)
    constexpr int QPER = (QP + HP - 1) / HP;            // quads per thread per half-sweep
    constexpr int PL = planes_for(24 * QPER);           // energy counter planes
    constexpr int W4 = (N / 4 + 2 * HP - 1) / (2 * HP); // overlap: 16-byte words per thread
    constexpr int PLO = planes_for(4 * W4);
    extern __shared__ uint4 smem_u4[];
    const int NT = (int)a.NT;
    uint32_t *S = reinterpret_cast<uint32_t *>(smem_u4);     // [NT][2][H]
    uint32_t *Js = S + (size_t)NT * N;                        // [3][2][H]
    int *E = reinterpret_cast<int *>(Js + 3 * N);             // [64][32] energies by slot
    int *bnd = E + kMaxTemps * kLanes;                        // [64][32] swap accept bounds
    int *nd = bnd + kMaxTemps * kLanes;                       // [64][32] overlap counts
    uint32_t *msk = reinterpret_cast<uint32_t *>(nd + kMaxTemps * kLanes);  // [64]
    uint32_t *Tsw = msk + kMaxTemps;                          // [NT-1][swap_len] if swap_in_smem

    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t unit = blockIdx.x;
    const int c = (int)(unit % a.C);
    const uint32_t g = unit / a.C;
    int l, par, tl;
    Mp::map(tid, l, par, tl);
    const bool active = l < NT;
    const int ls = active ? l : 0;

    uint32_t *gS = a.spins + (size_t)unit * NT * N;
    const uint32_t *gJ = a.bonds + (size_t)g * 3 * N;
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(S)[w] = reinterpret_cast<const uint4 *>(gS)[w];
    for (int w = tid; w < 3 * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(Js)[w] = reinterpret_cast<const uint4 *>(gJ)[w];
    const uint32_t *swt = a.swapt;
    if (swap_in_smem) {
        const int nsw = (NT - 1) * (int)a.swap_len;
        for (int w = tid; w < nsw; w += nthr) Tsw[w] = a.swapt[w];
        swt = Tsw;
    }
    const uint32_t t0 = a.metro[ls * 3 + 0], t1 = a.metro[ls * 3 + 1], t2 = a.metro[ls * 3 + 2];
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
    __syncthreads();

    uint64_t P = a.P0;
    uint32_t pass_local = a.pass_local0;
    for (uint32_t n = 0; n < a.n_sweeps; ++n) {
        const uint64_t s = a.s0 + n;
        const bool swap_now = swap_after(s, a.swap_every) && NT > 1;
        const bool meas = measured(s, a.measure_from, a.measure_every);
        const bool needE = swap_now || a.energy_log != nullptr || meas || (n + 1 == a.n_sweeps);
        uint32_t acc[PL];
#pragma unroll
        for (int p = 0; p < PL; ++p) acc[p] = 0;
        if (needE)   // counters add 2 per unsatisfied bond: E = 2U - 3N
            for (int i = tid; i < NT * kLanes; i += nthr) E[i] = -3 * N;
        if (swap_now) {
            // one Philox call gives the uniforms of four realizations of a pair
            for (int i = tid; i < (NT - 1) * 8; i += nthr) {
                const int p = i >> 3, bq = i & 7;
                const uint4 v = philox(((uint32_t)p << 3) | (uint32_t)bq,
                                       (1u << 24) | ((uint32_t)c << 8), (uint32_t)P, g, a.rk);
                const uint32_t *row = swt + (size_t)p * a.swap_len;
                int *o = bnd + p * kLanes + 4 * bq;
                o[0] = accept_bound(row, a.swap_len, v.x);
                o[1] = accept_bound(row, a.swap_len, v.y);
                o[2] = accept_bound(row, a.swap_len, v.z);
                o[3] = accept_bound(row, a.swap_len, v.w);
            }
        }
        // colour 0: x parity = par; colour 1: x parity = par ^ 1 (warp-uniform)
        if (par == 0)
            half_fast<L, QPER, 0, 0, false, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag0, a.rk, t0, t1, t2, acc);
        else
            half_fast<L, QPER, 0, 1, false, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag0, a.rk, t0, t1, t2, acc);
        __syncthreads();
        if (needE) {
            if (par == 0)
                half_fast<L, QPER, 1, 1, true, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag1, a.rk, t0, t1, t2, acc);
            else
                half_fast<L, QPER, 1, 0, true, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag1, a.rk, t0, t1, t2, acc);
            reduce_fast<PL, HP>(acc, E, lane, warp, 2, NT);
        } else {
            if (par == 0)
                half_fast<L, QPER, 1, 1, false, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag1, a.rk, t0, t1, t2, acc);
            else
                half_fast<L, QPER, 1, 0, false, PL>(mine, Js, qd, qv, (uint32_t)s, g, tag1, a.rk, t0, t1, t2, acc);
        }
        __syncthreads();
        if (swap_now) {
            if (warp == 0) {
                // Sequential pairs (0,1), (1,2), ... per realization lane; the
                // configuration carried upward is `cur`.  Loads run one pair ahead.
                int cur = E[lane];
                int nxt = E[kLanes + lane];
                int bb = bnd[lane];
                for (int p = 0; p + 1 < NT; ++p) {
                    const int nxt2 = (p + 2 < NT) ? E[(p + 2) * kLanes + lane] : 0;
                    const int bb2 = (p + 2 < NT) ? bnd[(p + 1) * kLanes + lane] : 0;
                    const bool ok = (cur - nxt) >= bb;
                    const uint32_t m = __ballot_sync(kFull, ok);
                    E[p * kLanes + lane] = ok ? nxt : cur;
                    cur = ok ? cur : nxt;
                    if (lane == 0) msk[p] = m;
                    nxt = nxt2;
                    bb = bb2;
                }
                E[(NT - 1) * kLanes + lane] = cur;
            }
            __syncthreads();
            for (int w = tid; w < N / 2; w += nthr) {
                uint2 x = reinterpret_cast<const uint2 *>(S)[w];
                for (int p = 0; p + 1 < NT; ++p) {
                    const uint2 y = reinterpret_cast<const uint2 *>(S + (size_t)(p + 1) * N)[w];
                    const uint32_t m = msk[p];
                    const uint32_t dx = (x.x ^ y.x) & m, dy = (x.y ^ y.y) & m;
                    reinterpret_cast<uint2 *>(S + (size_t)p * N)[w] = make_uint2(x.x ^ dx, x.y ^ dy);
                    x = make_uint2(y.x ^ dx, y.y ^ dy);
                }
                reinterpret_cast<uint2 *>(S + (size_t)(NT - 1) * N)[w] = x;
            }
            if (a.swap_log != nullptr)
                for (int p = tid; p + 1 < NT; p += nthr)
                    a.swap_log[(((size_t)pass_local * a.G + g) * a.C + c) * (NT - 1) + p] = msk[p];
            __syncthreads();
        }
        if (swap_after(s, a.swap_every)) {
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
            if (a.esum != nullptr) {
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
                uint32_t oacc[PLO];
#pragma unroll
                for (int p = 0; p < PLO; ++p) oacc[p] = 0;
                if (active && (l & 1) == c) {
                    const uint4 *A4 = reinterpret_cast<const uint4 *>(S + (size_t)l * N);
                    const uint4 *B4 = reinterpret_cast<const uint4 *>(other + (size_t)l * N);
#pragma unroll 4
                    for (int j = 0; j < W4; ++j) {
                        const int w = par * HP + tl + j * 2 * HP;
                        if (w < N / 4) {
                            const uint4 x = A4[w], y = B4[w];
                            uint32_t s3, c1;
                            const uint32_t d0 = x.x ^ y.x, d1 = x.y ^ y.y, d2 = x.z ^ y.z, d3 = x.w ^ y.w;
                            full_add(d0, d1, d2, s3, c1);
                            uint32_t A[5] = {s3 ^ d3, c1 ^ (s3 & d3), c1 & (s3 & d3), 0u, 0u};
                            acc_add_sum5<PLO>(oacc, A);
                        }
                    }
                }
                reduce_fast<PLO, HP>(oacc, nd, lane, warp, 1, NT);
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
    for (int i = tid; i < NT * kLanes; i += nthr) a.energy[(size_t)unit * NT * kLanes + i] = E[i];
    for (int w = tid; w < NT * N / 4; w += nthr)
        reinterpret_cast<uint4 *>(gS)[w] = reinterpret_cast<const uint4 *>(S)[w];
}

template <int L, int HP>
cudaError_t launch_fast(const SweepLaunch &a, size_t smem, bool swap_in_smem, bool cluster_measure,
                        cudaStream_t st)
{
    auto kern = k_sweep_unit_fast<L, HP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.G * a.C);
    cfg.blockDim = dim3(FastMap<HP>::threads((int)a.NT));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    cfg.numAttrs = 0;
    if (cluster_measure) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, a, cluster_measure ? 1 : 0, swap_in_smem ? 1 : 0);
}

}  // namespace

// Variants compiled here: (L, HP).  Returns the thread count for a variant,
// or 0 if it does not exist / does not fit.
int fast_unit_threads(int L, int HP, int NT)
{
    if (!((L == 8 && (HP == 4 || HP == 8)) || (L == 16 && (HP == 32 || HP == 64)))) return 0;
    const int t = HP >= 32 ? NT * 2 * HP : ((NT + 32 / HP - 1) / (32 / HP)) * 64;
    return t <= kMaxThreads ? t : 0;
}

cudaError_t launch_sweep_unit_fast(const SweepLaunch &a, int L, int HP, size_t smem,
                                   bool swap_in_smem, bool cluster_measure, cudaStream_t st,
                                   uint64_t *launches)
{
    *launches += 1;
    if (L == 8 && HP == 4) return launch_fast<8, 4>(a, smem, swap_in_smem, cluster_measure, st);
    if (L == 8 && HP == 8) return launch_fast<8, 8>(a, smem, swap_in_smem, cluster_measure, st);
    if (L == 16 && HP == 32) return launch_fast<16, 32>(a, smem, swap_in_smem, cluster_measure, st);
    if (L == 16 && HP == 64) return launch_fast<16, 64>(a, smem, swap_in_smem, cluster_measure, st);
    return cudaErrorInvalidValue;
}

}  // namespace ea
