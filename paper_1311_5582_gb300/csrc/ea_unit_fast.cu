// Launchers of the unit kernel specialised for L % 8 == 0 (the body is in
// ea_fast.cuh): one CTA per (group, copy), variants (L, HP, max threads).
#include "ea_fast.cuh"

namespace ea {
namespace {
template <int L, int HP, int MAXT, bool MEAS>
__global__ void __launch_bounds__(MAXT, 1)
k_sweep_unit_fast(const __grid_constant__ SweepLaunch a, int cluster_measure, int swap_in_smem,
                  int snap_mode, int hist_smem)
{
    extern __shared__ uint4 smem_u4[];
    unit_fast_body<L, HP, MEAS>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x, cluster_measure,
                                swap_in_smem, snap_mode, hist_smem);
}

template <int L, int HP, int MAXT>
cudaError_t launch_fast(const SweepLaunch &a, size_t smem, bool swap_in_smem, bool cluster_measure,
                        bool snap_mode, bool hist_smem, cudaStream_t st)
{
    // launches that measure and log nothing run the body compiled without those paths
    const bool meas = a.measure_every != 0 || a.energy_log != nullptr || a.swap_log != nullptr;
    auto kern = meas ? k_sweep_unit_fast<L, HP, MAXT, true> : k_sweep_unit_fast<L, HP, MAXT, false>;
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
    return cudaLaunchKernelEx(&cfg, kern, a, cluster_measure ? 1 : 0, swap_in_smem ? 1 : 0,
                              snap_mode ? 1 : 0, hist_smem ? 1 : 0);
}

}  // namespace

// Variants compiled here: (L, HP).  Returns the thread count for a variant,
// or 0 if it does not exist / does not fit.
int fast_unit_threads(int L, int HP, int NT)
{
    if (!((L == 8 && (HP == 4 || HP == 8 || HP == 16)) || (L == 16 && (HP == 32 || HP == 64))))
        return 0;
    const int t = HP >= 32 ? NT * 2 * HP : ((NT + 32 / HP - 1) / (32 / HP)) * 64;
    const int cap = (L == 8 && HP == 16) ? 768 : kMaxThreads;
    return t <= cap ? t : 0;
}

size_t fast_unit_smem(int L, int NT, uint32_t swap_len, bool swap_smem, bool snap, bool hist_smem)
{
    const int N = L * L * L;
    return FastLayout(N, NT, swap_len, swap_smem, snap, hist_smem).words * 4;
}

cudaError_t launch_sweep_unit_fast(const SweepLaunch &a, int L, int HP, bool swap_in_smem,
                                   bool cluster_measure, size_t smem_optin, cudaStream_t st,
                                   uint64_t *launches)
{
    *launches += 1;
    // measurement extras (partner snapshots, shared-memory histogram) when they fit
    const int NT = (int)a.NT;
    bool snap = false, hist = false;
    if (cluster_measure) {
        snap = fast_unit_smem(L, NT, a.swap_len, swap_in_smem, true, false) <= smem_optin;
        hist = a.qhist != nullptr &&
               fast_unit_smem(L, NT, a.swap_len, swap_in_smem, snap, true) <= smem_optin;
    }
    const size_t smem = fast_unit_smem(L, NT, a.swap_len, swap_in_smem, snap, hist);
    // up to 384 threads a CTA the kernel may use 170 registers a thread
    const int threads = fast_unit_threads(L, HP, NT);
    if (L == 8 && HP == 4) return launch_fast<8, 4, 512>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    if (L == 8 && HP == 8 && threads <= 384)
        return launch_fast<8, 8, 384>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    if (L == 8 && HP == 8) return launch_fast<8, 8, 512>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    if (L == 8 && HP == 16) return launch_fast<8, 16, 768>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    if (L == 16 && HP == 32) return launch_fast<16, 32, 512>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    if (L == 16 && HP == 64) return launch_fast<16, 64, 512>(a, smem, swap_in_smem, cluster_measure, snap, hist, st);
    return cudaErrorInvalidValue;
}

}  // namespace ea
