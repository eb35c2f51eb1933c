// Launcher of the L = 8 unit kernel with the wavefront replica exchange (the
// body is in ea_wave.cuh): one CTA per (group, copy), one warp per two slots;
// field-free, or in an external field whose always-accept boundaries are
// u >= 3 and u >= 4 for the two spin values.  Field-free calls that measure
// run the MEAS instantiations (energy sums; with the q histogram the two
// copies of a group form a 2-CTA cluster).
#include "ea_wave.cuh"

namespace ea {
namespace {
template <int MAXT, bool LOG, int FLD, int MEAS>
__global__ void __launch_bounds__(MAXT, 1)
k_sweep_unit_wave(const __grid_constant__ SweepLaunch a, int swap_in_smem)
{
    extern __shared__ uint4 smem_u4[];
    unit_wave_body<LOG, FLD, MEAS>(reinterpret_cast<uint32_t *>(smem_u4), a, blockIdx.x, swap_in_smem);
}

template <int MAXT, bool LOG, int FLD, int MEAS = 0>
cudaError_t launch_wave(const SweepLaunch &a, int threads, size_t smem, bool swap_in_smem, cudaStream_t st)
{
    auto kern = k_sweep_unit_wave<MAXT, LOG, FLD, MEAS>;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (MEAS == 2) {
        // the two copies of a group (units 2g, 2g + 1) form one cluster
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.G * a.C);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, a, swap_in_smem ? 1 : 0);
    } else {
        kern<<<a.G * a.C, threads, smem, st>>>(a, swap_in_smem ? 1 : 0);
        return cudaGetLastError();
    }
}

template <int FLD>
cudaError_t launch_wave_fld(const SweepLaunch &a, int threads, size_t smem, bool swap_in_smem, bool log,
                            cudaStream_t st)
{
    if (threads <= 384)
        return log ? launch_wave<384, true, FLD>(a, threads, smem, swap_in_smem, st)
                   : launch_wave<384, false, FLD>(a, threads, smem, swap_in_smem, st);
    return log ? launch_wave<512, true, FLD>(a, threads, smem, swap_in_smem, st)
               : launch_wave<512, false, FLD>(a, threads, smem, swap_in_smem, st);
}

template <int MEAS>
cudaError_t launch_wave_meas(const SweepLaunch &a, int threads, size_t smem, bool swap_in_smem, cudaStream_t st)
{
    if (threads <= 384) return launch_wave<384, false, 0, MEAS>(a, threads, smem, swap_in_smem, st);
    return launch_wave<512, false, 0, MEAS>(a, threads, smem, swap_in_smem, st);
}
}  // namespace

int wave_unit_threads(int L, int NT)
{
    return (L == 8 && NT >= 1 && NT <= kWaveMaxTemps) ? 32 * ((NT + 1) / 2) : 0;
}

size_t wave_unit_smem(int L, int NT, uint32_t swap_len, bool swap_smem, bool field, bool overlaps)
{
    return WaveLayout(L * L * L, NT, swap_len, swap_smem, field, overlaps).words * 4;
}

int wave_field_kind(int ua0, int ua1)
{
    if (ua0 == 3 && ua1 == 4) return 34;
    if (ua0 == 4 && ua1 == 3) return 43;
    return 0;
}

cudaError_t launch_sweep_unit_wave(const SweepLaunch &a, bool swap_in_smem, int field_kind, int meas,
                                   cudaStream_t st, uint64_t *launches)
{
    const int threads = wave_unit_threads(8, (int)a.NT);
    if (threads == 0) return cudaErrorInvalidValue;
    const bool field = field_kind != 0;
    if (field != (a.h_num != 0)) return cudaErrorInvalidValue;
    const bool log = a.energy_log != nullptr || a.swap_log != nullptr;
    if (meas != 0) {
        // field-free, without logs; the q histogram needs the copy pair
        if (field || log || meas > 2 || (meas == 2 && a.C != 2)) return cudaErrorInvalidValue;
        const size_t smem = wave_unit_smem(8, (int)a.NT, a.swap_len, swap_in_smem, false, meas == 2);
        *launches += 1;
        return meas == 2 ? launch_wave_meas<2>(a, threads, smem, swap_in_smem, st)
                         : launch_wave_meas<1>(a, threads, smem, swap_in_smem, st);
    }
    const size_t smem = wave_unit_smem(8, (int)a.NT, a.swap_len, swap_in_smem, field, false);
    *launches += 1;
    if (field_kind == 34) return launch_wave_fld<34>(a, threads, smem, swap_in_smem, log, st);
    if (field_kind == 43) return launch_wave_fld<43>(a, threads, smem, swap_in_smem, log, st);
    if (field_kind != 0) return cudaErrorInvalidValue;
    return launch_wave_fld<0>(a, threads, smem, swap_in_smem, log, st);
}

}  // namespace ea
