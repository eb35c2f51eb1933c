// Instantiation of the persistent batch kernel for CTAs of up to 512 threads
// (own translation unit so that the variants compile in parallel).
#include "ea_batch_kernel.cuh"

namespace ea {
const void *batch_kernel_512() { return reinterpret_cast<const void *>(&k_batch<512>); }
}  // namespace ea
