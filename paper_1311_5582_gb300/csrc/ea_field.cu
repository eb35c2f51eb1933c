// Sweep kernels of the simulation in an external field h = h_num / h_den
// (Eq. 1 with h != 0; the field runs of Sec. 5): the generic unit and chunked
// bodies instantiated with field flips, magnetisation counters and swap
// decisions on Et = h_den E - h_num M.  Kept in their own translation unit so
// that they compile in parallel with the field-free kernels.
#include "ea_bodies.cuh"

namespace ea {
namespace {

template <int L>
__global__ void __launch_bounds__(field_max_threads(L), 1)
k_sweep_unit_field(const __grid_constant__ SweepLaunch a, int tpl, int cluster_measure, int swap_in_smem)
{
    extern __shared__ uint4 smem_u4[];
    unit_body<L, true, true>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x, tpl, cluster_measure,
                             swap_in_smem);
}

template <int L, bool J_SMEM>
__global__ void __launch_bounds__(field_max_threads(L), 1)
k_sweep_chunk_field(const __grid_constant__ SweepLaunch a, int tpl, int nlat)
{
    extern __shared__ uint4 smem_u4[];
    chunk_body<L, J_SMEM, true, true>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x,
                                      (int)blockIdx.y, tpl, nlat);
}

template <int L>
cudaError_t launch_unit_field_L(const SweepLaunch &a, const Plan &plan, bool cluster_measure,
                                cudaStream_t st)
{
    auto kern = k_sweep_unit_field<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.G * a.C);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
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
    return cudaLaunchKernelEx(&cfg, kern, a, plan.threads_per_lattice, cluster_measure ? 1 : 0,
                              plan.swap_in_smem ? 1 : 0);
}

template <int L>
cudaError_t launch_chunk_field_L(const SweepLaunch &a, const Plan &plan, cudaStream_t st)
{
    const int nchunks = ((int)a.NT + plan.lattices_per_cta - 1) / plan.lattices_per_cta;
    dim3 grid(a.G * a.C, nchunks);
    auto kern = plan.j_in_smem ? k_sweep_chunk_field<L, true> : k_sweep_chunk_field<L, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plan.smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, plan.threads, plan.smem, st>>>(a, plan.threads_per_lattice, plan.lattices_per_cta);
    return cudaGetLastError();
}

#define EA_FIELD_L(X) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(32)

}  // namespace

cudaError_t launch_sweep_unit_field(const SweepLaunch &a, int L, const Plan &plan, bool cluster_measure,
                                    cudaStream_t st)
{
    switch (L) {
#define EA_CASE(X) case X: return launch_unit_field_L<X>(a, plan, cluster_measure, st);
        EA_FIELD_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_chunk_field(const SweepLaunch &a, int L, const Plan &plan, cudaStream_t st)
{
    switch (L) {
#define EA_CASE(X) case X: return launch_chunk_field_L<X>(a, plan, st);
        EA_FIELD_L(EA_CASE)
#undef EA_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ea
