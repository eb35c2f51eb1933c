// One replica-exchange pass that allocates nothing.
//
// Some callers cannot allocate device memory while they run: an application
// that reserves all device memory for its own pool up front, a host thread
// that must not call cudaMalloc (which can synchronise the device and stall
// other streams), or code that has handed its allocator to another runtime.
// ea_pt_swap_static gives them the replica-exchange pass on buffers they
// already own.  Its only scratch -- the accepted-pair masks passed from the
// decision kernel to the exchange kernel -- lives in the file-scope device
// array below, which every GPU that loads this library keeps until the
// process exits.
#include <mutex>

#include "../../include/ea.h"
#include "ea_device.cuh"

namespace ea {
namespace {

// Largest G * C one call may handle; masks take kMaxTemps words per unit (1 MiB).
constexpr uint32_t kStaticMaxUnits = 4096;
static __device__ __align__(256) uint32_t g_static_masks[kStaticMaxUnits * kMaxTemps];

// Device address of g_static_masks per device, looked up once with that
// device current (the host-side name is only a stand-in for the symbol).  The
// cache assumes the device's primary context lives as long as the process: a
// cudaDeviceReset unloads the module, and this call must not be used after one.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint32_t *g_static_ptr[kMaxDevices] = {};

cudaError_t static_masks_ptr(int dev, uint32_t **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_masks);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// Decision for one (group, copy) unit per CTA on energies in API order
// [G][NT][C][32]; permutes them in place and writes the masks to scratch.
__global__ void __launch_bounds__(256)
k_static_decide(int32_t *energies, const uint32_t *swapt, uint32_t swap_len, uint32_t NT,
                uint32_t C, RoundKeys rk, uint64_t P, uint32_t *scratch, uint32_t *masks_out)
{
    __shared__ int bnd[kMaxTemps * kLanes];
    const uint32_t unit = blockIdx.x;
    const int c = (int)(unit % C);
    const uint32_t g = unit / C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < ((int)NT - 1) * kLanes; i += blockDim.x) {
        const int p = i >> 5, b = i & 31;
        bnd[i] = accept_bound(swapt + (size_t)p * swap_len, swap_len, swap_uniform(rk, p, b, P, g, c));
    }
    __syncthreads();
    if (warp != 0) return;
    auto E = [&](int t) -> int32_t & {
        return energies[(((size_t)g * NT + t) * C + c) * kLanes + lane];
    };
    int cur = E(0);
    for (int p = 0; p + 1 < (int)NT; ++p) {
        const int nxt = E(p + 1);
        const bool ok = (cur - nxt) >= bnd[p * kLanes + lane];
        const uint32_t m = __ballot_sync(kFull, ok);
        E(p) = ok ? nxt : cur;
        cur = ok ? cur : nxt;
        if (lane == 0) {
            scratch[(size_t)unit * kMaxTemps + p] = m;
            if (masks_out) masks_out[(size_t)unit * (NT - 1) + p] = m;
        }
    }
    E((int)NT - 1) = cur;
}

// Masked exchange chain over the slots of each unit, spins in API order
// [G][NT][C][N]; masks from scratch.
__global__ void __launch_bounds__(256)
k_static_apply(uint32_t *spins, const uint32_t *scratch, uint32_t N, uint32_t NT, uint32_t C)
{
    const uint32_t unit = blockIdx.y;
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= N) return;
    const uint32_t c = unit % C, g = unit / C;
    const size_t stride = (size_t)C * N;                 // next slot, same copy
    uint32_t *S = spins + ((size_t)g * NT * C + c) * N + w;
    const uint32_t *m = scratch + (size_t)unit * kMaxTemps;
    uint32_t x = S[0];
    for (uint32_t p = 0; p + 1 < NT; ++p) {
        const uint32_t y = S[(p + 1) * stride];
        const uint32_t d = (x ^ y) & m[p];
        S[p * stride] = x ^ d;
        x = y ^ d;
    }
    S[(NT - 1) * stride] = x;
}

}  // namespace
}  // namespace ea

extern "C" int ea_pt_swap_static(uint32_t *spins, int32_t *energies, const uint32_t *swapt,
                                 uint32_t swap_len, uint32_t L, uint32_t n_groups, uint32_t n_temps,
                                 uint32_t n_copies, uint64_t seed, uint64_t pass_index,
                                 uint32_t *masks, void *stream)
{
    using namespace ea;
    if (!spins || !energies) return EA_EINVAL;
    if (L < 2 || (L & 1u) || n_groups == 0 || n_temps == 0 || n_temps > (uint32_t)kMaxTemps ||
        n_copies < 1 || n_copies > 2)
        return EA_EINVAL;
    if ((uint64_t)L * L * L > 0xFFFFFFFFull) return EA_EINVAL;              // N in 32 bits
    if ((uint64_t)n_groups * n_copies > kStaticMaxUnits) return EA_EINVAL;   // scratch limit
    if (n_temps > 1 && swap_len > 0 && !swapt) return EA_EINVAL;
    if (n_temps < 2) return EA_OK;    // no pairs: nothing to exchange
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    uint32_t *scratch = nullptr;
    if (e == cudaSuccess) e = static_masks_ptr(dev, &scratch);
    if (e != cudaSuccess) return EA_ECUDA;
    const uint32_t units = n_groups * n_copies;
    const uint32_t N = L * L * L;
    cudaStream_t st = (cudaStream_t)stream;
    k_static_decide<<<units, 256, 0, st>>>(energies, swapt, swap_len, n_temps, n_copies,
                                           make_round_keys(seed), pass_index, scratch, masks);
    dim3 grid((N + 255) / 256, units);
    k_static_apply<<<grid, 256, 0, st>>>(spins, scratch, N, n_temps, n_copies);
    return cudaGetLastError() == cudaSuccess ? EA_OK : EA_ECUDA;
}
