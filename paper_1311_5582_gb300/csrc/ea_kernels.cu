// Generic kernels of the parallel-tempering Metropolis simulation of the 3D
// +-J Edwards-Anderson model for sm_103a (any supported even L): the unit and
// chunked sweep kernels, the global swap pass, energy recomputation,
// measurement and layout conversion, plus the launch plan.
#include "ea_bodies.cuh"

namespace ea {

namespace {
template <int L, bool MEAS>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sweep_unit(const __grid_constant__ SweepLaunch a, int tpl, int cluster_measure, int swap_in_smem)
{
    extern __shared__ uint4 smem_u4[];
    unit_body<L, MEAS>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x, tpl, cluster_measure,
                       swap_in_smem);
}

template <int L, bool J_SMEM, bool LOG>
__global__ void __launch_bounds__(kMaxThreads, 1)
k_sweep_chunk(const __grid_constant__ SweepLaunch a, int tpl, int nlat)
{
    extern __shared__ uint4 smem_u4[];
    chunk_body<L, J_SMEM, LOG>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x, (int)blockIdx.y,
                               tpl, nlat);
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
                              swap_uniform(a.rk, p, b, P, g + a.g_base, c));
    }
    __syncthreads();
    if (warp == 0 && a.h_num != 0) {
        // field: bounds in steps of Et = h_den E - h_num M; E and M travel together
        int32_t *E = a.energy + (size_t)unit * NT * kLanes;
        int32_t *M = a.mag + (size_t)unit * NT * kLanes;
        int ce = E[lane], cm = M[lane];
        for (int p = 0; p + 1 < NT; ++p) {
            const int ne = E[(p + 1) * kLanes + lane], nm = M[(p + 1) * kLanes + lane];
            const int xc = a.h_den * ce - a.h_num * cm, xn = a.h_den * ne - a.h_num * nm;
            const bool ok = (xc - xn) >= (bnd[p * kLanes + lane] / 4) * a.step;
            const uint32_t m = __ballot_sync(kFull, ok);
            E[p * kLanes + lane] = ok ? ne : ce;
            M[p * kLanes + lane] = ok ? nm : cm;
            ce = ok ? ce : ne;
            cm = ok ? cm : nm;
            if (lane == 0) {
                masks_out[(size_t)unit * (NT - 1) + p] = m;
                if (swap_log_row) swap_log_row[(size_t)unit * (NT - 1) + p] = m;
            }
        }
        E[(NT - 1) * kLanes + lane] = ce;
        M[(NT - 1) * kLanes + lane] = cm;
        if (energy_log_row)
            for (int t = 0; t < NT; ++t)
                energy_log_row[(((size_t)g * NT + t) * a.C + c) * kLanes + lane] = E[t * kLanes + lane];
    } else if (warp == 0) {
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

// Energies (and, with mag != null, magnetisations M = 2 up - N) recomputed
// from the spins: one CTA per lattice.
template <int L>
__global__ void __launch_bounds__(kMaxThreads)
k_energy(const uint32_t *spins, const uint32_t *bonds, int32_t *energy, int32_t *mag, uint32_t NT,
         uint32_t C)
{
    using Gm = Geo<L>;
    __shared__ int U[kLanes], Up[kLanes];
    const size_t lat = blockIdx.x;              // (unit, t)
    const uint32_t unit = (uint32_t)(lat / NT);
    const uint32_t g = unit / C;
    const uint32_t *S = spins + lat * Gm::N;
    const uint32_t *J = bonds + (size_t)g * 3 * Gm::N;
    const int tid = threadIdx.x, tpl = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kLanes) U[tid] = Up[tid] = 0;
    __syncthreads();
    if (mag != nullptr) {
        // per-thread count <= 4 x 2 x kMaxQuadsPerThread = 80 (N / 4 vectors, 2Q)
        uint32_t accM[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) accM[p] = 0;
        const uint4 *S4 = reinterpret_cast<const uint4 *>(S);
        for (int w = tid; w < Gm::N / 4; w += tpl) {
            const uint4 x = S4[w];
            acc_add_words4(accM, x.x, x.y, x.z, x.w);
        }
        int cm = 0;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) cm += __popc(warp_transpose(accM[p], lane)) << p;
        atomicAdd(&Up[lane], cm);
    }
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
    if (mag != nullptr && tid < kLanes) mag[lat * kLanes + tid] = 2 * Up[tid] - Gm::N;
}

// Magnetisations M = 2 up - N of every lattice in API order [G][NT][C][32]:
// one CTA per lattice (g, c, t).
__global__ void __launch_bounds__(256)
k_magnetisation(const uint32_t *spins, int N, uint32_t NT, uint32_t C, int32_t *out)
{
    __shared__ int up[kLanes];
    const size_t lat = blockIdx.x;              // device order (g, c, t)
    const uint32_t t = (uint32_t)(lat % NT), gc = (uint32_t)(lat / NT);
    const uint32_t c = gc % C, g = gc / C;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < kLanes) up[tid] = 0;
    __syncthreads();
    // per-thread count <= 4 x ceil(N / 1024) <= 128 for N <= 32768
    uint32_t acc[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) acc[p] = 0;
    const uint4 *S4 = reinterpret_cast<const uint4 *>(spins + lat * N);
    for (int w = tid; w < N / 4; w += blockDim.x) {
        const uint4 x = S4[w];
        acc_add_words4(acc, x.x, x.y, x.z, x.w);
    }
    int cnt = 0;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) cnt += __popc(warp_transpose(acc[p], lane)) << p;
    atomicAdd(&up[lane], cnt);
    __syncthreads();
    if (tid < kLanes) out[(((size_t)g * NT + t) * C + c) * kLanes + tid] = 2 * up[tid] - N;
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

// Per-plane counts for Fourier-mode observables (Sec. 5): one warp per plane
// (axis blockIdx.y, index = warp), one block per unit.  mode 0: unit (g, t),
// sites of the plane where the two copies differ; mode 1: unit (g, t, c), up
// spins of the plane.  out [unit][3][L][32] in API order.  Each lane adds its
// words into a bit-sliced counter; a 32 x 32 transpose gives each lane its
// realization's count.
__global__ void k_measure_planes(const uint32_t *spins, int L, uint32_t NT, uint32_t C, int mode,
                                 int32_t *out)
{
    const int N = L * L * L, H = N / 2;
    const uint32_t unit = blockIdx.x;
    const int a = (int)blockIdx.y, plane = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    uint32_t g, t, c;
    if (mode == 0) {
        g = unit / NT;
        t = unit % NT;
        c = 0;
    } else {
        g = unit / (NT * C);
        t = (unit / C) % NT;
        c = unit % C;
    }
    const uint32_t *A = spins + (((size_t)g * C + c) * NT + t) * N;
    const uint32_t *B = spins + (((size_t)g * C + (C - 1)) * NT + t) * N;
    uint32_t acc[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) acc[q] = 0;
    // per lane at most ceil(L^2 / 32) <= 32 words: the 8-plane counter cannot overflow
    for (int j = lane; j < L * L; j += 32) {
        const int u = j % L, v = j / L;
        const int x = a == 0 ? plane : u;
        const int y = a == 1 ? plane : (a == 0 ? u : v);
        const int z = a == 2 ? plane : v;
        const int i = x + L * (y + L * z);
        const int w = ((x + y + z) & 1) * H + (i >> 1);
        uint32_t cy = mode == 0 ? (A[w] ^ B[w]) : A[w];
#pragma unroll
        for (int q = 0; q < kPlanes; ++q) {
            const uint32_t t2 = acc[q] & cy;
            acc[q] ^= cy;
            cy = t2;
        }
    }
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) cnt += __popc(warp_transpose(acc[q], lane)) << q;
    out[(((size_t)unit * 3 + a) * L + plane) * kLanes + lane] = cnt;
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
    // launches that measure and log nothing run the body compiled without those paths
    const bool full = a.measure_every != 0 || a.energy_log != nullptr || a.swap_log != nullptr;
    auto kern = full ? k_sweep_unit<L, true> : k_sweep_unit<L, false>;
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
    return cudaLaunchKernelEx(&cfg, kern, a, plan.threads_per_lattice, cluster_measure ? 1 : 0,
                              plan.swap_in_smem ? 1 : 0);
}

template <int L>
cudaError_t launch_chunk_L(const SweepLaunch &a, const Plan &plan, cudaStream_t st)
{
    const int nchunks = ((int)a.NT + plan.lattices_per_cta - 1) / plan.lattices_per_cta;
    dim3 grid(a.G * a.C, nchunks);
    const bool log = a.energy_log != nullptr;
    if (plan.j_in_smem) {
        auto kern = log ? k_sweep_chunk<L, true, true> : k_sweep_chunk<L, true, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, plan.threads, plan.smem, st>>>(a, plan.threads_per_lattice, plan.lattices_per_cta);
    } else {
        auto kern = log ? k_sweep_chunk<L, false, true> : k_sweep_chunk<L, false, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)plan.smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, plan.threads, plan.smem, st>>>(a, plan.threads_per_lattice, plan.lattices_per_cta);
    }
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_energy_L(const uint32_t *spins, const uint32_t *bonds, int32_t *energy, int32_t *mag,
                            uint32_t G, uint32_t NT, uint32_t C, cudaStream_t st)
{
    constexpr int Q = Geo<L>::Q;
    int threads = 32;
    while (threads < kMaxThreads && (Q + threads - 1) / threads > kMaxQuadsPerThread) threads *= 2;
    k_energy<L><<<(unsigned)((size_t)G * C * NT), threads, 0, st>>>(spins, bonds, energy, mag, NT, C);
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

// Threads a CTA of the sweep kernels may have: the field kernels are
// compiled for at most field_max_threads(L) (more registers a thread).
static int max_threads(int L, bool field) { return field ? field_max_threads(L) : kMaxThreads; }

static int pow2_at_least(int x)
{
    int p = 1;
    while (p < x) p *= 2;
    return p;
}

static bool unit_generic_plan(int L, int NT, uint32_t swap_len, size_t smem_optin, int tpl_pref,
                              bool field, Plan *plan)
{
    const int kMaxThreads = max_threads(L, field);
    const int N = L * L * L, Q = N / 8;
    const int tpl_min = pow2_at_least((Q + kMaxQuadsPerThread - 1) / kMaxQuadsPerThread);
    int tpl = tpl_pref > 0 ? tpl_pref : pow2_at_least((Q + 3) / 4);
    if (tpl < tpl_min) tpl = tpl_min;
    // whole warps only: shuffles in the energy reduction use full masks
    while ((tpl * NT) % 32 != 0) tpl *= 2;
    while (tpl * NT > kMaxThreads && tpl / 2 >= tpl_min && ((tpl / 2) * NT) % 32 == 0) tpl /= 2;
    size_t smem = UnitSmem::base_bytes(N, NT) + (field ? (size_t)kMaxTemps * kLanes * 4 : 0);
    const size_t sw = UnitSmem::swap_bytes(NT, swap_len);
    const bool sw_smem = smem + sw <= smem_optin;
    if (sw_smem) smem += sw;
    // overlap counting: per-thread words N / tpl must fit the 8-plane counter
    if (tpl * NT > kMaxThreads || smem > smem_optin || (N + tpl - 1) / tpl > 255) return false;
    plan->form = kFormUnit;
    plan->unit = true;
    plan->threads_per_lattice = tpl;
    plan->lattices_per_cta = NT;
    plan->threads = tpl * NT;
    plan->smem = smem;
    plan->j_in_smem = true;
    plan->swap_in_smem = sw_smem;
    return true;
}

static bool chunk_plan(int L, int NT, size_t smem_optin, int tpl_pref, int nlat_cap, bool field,
                       Plan *plan)
{
    const int kMaxThreads = max_threads(L, field);
    const int N = L * L * L, Q = N / 8;
    const int tpl_min = pow2_at_least((Q + kMaxQuadsPerThread - 1) / kMaxQuadsPerThread);
    const size_t lat_bytes = (size_t)N * 4, j_bytes = (size_t)3 * N * 4;
    const size_t e_bytes = (size_t)kMaxTemps * kLanes * 4 * (field ? 2 : 1);
    const bool j_smem = j_bytes + lat_bytes + e_bytes <= smem_optin;
    const size_t budget = smem_optin - (j_smem ? j_bytes : 0) - e_bytes;
    int nlat = (int)(budget / lat_bytes);
    if (nlat < 1) return false;
    if (nlat > NT) nlat = NT;
    if (nlat_cap > 0 && nlat > nlat_cap) nlat = nlat_cap;
    int tpl = tpl_pref > 0 ? tpl_pref : pow2_at_least((Q + 3) / 4);
    if (tpl < tpl_min) tpl = tpl_min;
    if (tpl > kMaxThreads) tpl = kMaxThreads;
    if (tpl < tpl_min) return false;
    while (nlat * tpl > kMaxThreads && nlat > 1) --nlat;
    while (nlat * tpl > kMaxThreads && tpl / 2 >= tpl_min) tpl /= 2;
    // prefer a divisor of NT so every CTA is full
    for (int d = nlat; d >= 1; --d)
        if (NT % d == 0) { nlat = d; break; }
    while ((tpl * nlat) % 32 != 0) tpl *= 2;
    if (nlat * tpl > kMaxThreads) return false;
    plan->form = kFormChunked;
    plan->unit = false;
    plan->threads_per_lattice = tpl;
    plan->lattices_per_cta = nlat;
    plan->threads = tpl * nlat;
    plan->smem = (size_t)nlat * lat_bytes + (j_smem ? j_bytes : 0) + e_bytes;
    plan->j_in_smem = j_smem;
    plan->swap_in_smem = false;
    return true;
}

std::vector<Plan> make_plans(int L, int NT, int C, uint32_t swap_len, size_t smem_optin, bool field,
                             int field_kind)
{
    (void)C;
    std::vector<Plan> out;
    if (NT < 1 || NT > kMaxTemps || !supported_L(L)) return out;
    // wavefront unit form (L = 8): best first; field-free, or the fields it takes
    if ((!field || field_kind != 0) && wave_unit_threads(L, NT) != 0) {
        const bool sw_smem = wave_unit_smem(L, NT, swap_len, true, field) <= smem_optin;
        const size_t smem = wave_unit_smem(L, NT, swap_len, sw_smem, field);
        if (smem <= smem_optin) {
            Plan p;
            p.form = kFormUnitWave;
            p.unit = true;
            p.threads_per_lattice = 16;
            p.lattices_per_cta = NT;
            p.threads = wave_unit_threads(L, NT);
            p.smem = smem;
            p.j_in_smem = true;
            p.swap_in_smem = sw_smem;
            p.field_kind = field ? field_kind : 0;
            out.push_back(p);
        }
    }
    // fast unit form (L % 8 == 0); field-free only
    if (!field) {
        const bool sw_smem = fast_unit_smem(L, NT, swap_len, true, false, false) <= smem_optin;
        const size_t smem = fast_unit_smem(L, NT, swap_len, sw_smem, false, false);
        const int hps[] = {8, 16, 4, 64, 32};
        if (smem <= smem_optin)
            for (int hp : hps) {
                const int t = fast_unit_threads(L, hp, NT);
                if (t == 0) continue;
                Plan p;
                p.form = kFormUnitFast;
                p.unit = true;
                p.threads_per_lattice = hp;
                p.lattices_per_cta = NT;
                p.threads = t;
                p.smem = smem;
                p.j_in_smem = true;
                p.swap_in_smem = sw_smem;
                out.push_back(p);
            }
    }
    // generic unit form with a few group sizes
    {
        const int prefs[] = {0, 8, 16, 32, 64, 128};
        for (int tp : prefs) {
            Plan p;
            if (!unit_generic_plan(L, NT, swap_len, smem_optin, tp, field, &p)) continue;
            bool dup = false;
            for (const Plan &q : out)
                if (q.form == p.form && q.threads_per_lattice == p.threads_per_lattice) dup = true;
            if (!dup) out.push_back(p);
        }
    }
    // chunked form: always possible when one lattice fits
    {
        const int caps[] = {0, 1, 2, 4};
        const int prefs[] = {0, 64, 128, 256};
        for (int cap : caps)
            for (int tp : prefs) {
                Plan p;
                if (!chunk_plan(L, NT, smem_optin, tp, cap, field, &p)) continue;
                bool dup = false;
                for (const Plan &q : out)
                    if (q.form == p.form && q.threads_per_lattice == p.threads_per_lattice &&
                        q.lattices_per_cta == p.lattices_per_cta)
                        dup = true;
                if (!dup) out.push_back(p);
            }
    }
    return out;
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

cudaError_t launch_measure_planes(const uint32_t *spins, int L, uint32_t G, uint32_t NT, uint32_t C,
                                  int mode, int32_t *out, cudaStream_t st, uint64_t *launches)
{
    const uint32_t units = mode == 0 ? G * NT : G * NT * C;
    k_measure_planes<<<dim3(units, 3), 32 * L, 0, st>>>(spins, L, NT, C, mode, out);
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
    if (a.h_num != 0) return launch_sweep_unit_field(a, L, plan, cluster_measure, st);
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
    if (a.h_num != 0) return launch_sweep_chunk_field(a, L, plan, st);
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
                          uint32_t G, uint32_t NT, uint32_t C, cudaStream_t st, uint64_t *launches,
                          int32_t *mag)
{
    *launches += 1;
    switch (L) {
#define EA_CASE(X) case X: return launch_energy_L<X>(spins, bonds, energy, mag, G, NT, C, st);
        EA_FOR_EACH_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_magnetisation(const uint32_t *spins, int L, uint32_t G, uint32_t NT, uint32_t C,
                                 int32_t *out, cudaStream_t st, uint64_t *launches)
{
    const int N = L * L * L;
    k_magnetisation<<<G * C * NT, 256, 0, st>>>(spins, N, NT, C, out);
    *launches += 1;
    return cudaGetLastError();
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
