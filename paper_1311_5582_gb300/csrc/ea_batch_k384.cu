// Instantiation of the persistent batch kernel for CTAs of up to 384 threads
// (own translation unit so that the variants compile in parallel).
#include "ea_batch_kernel.cuh"

namespace ea {
const void *batch_kernel_384() { return reinterpret_cast<const void *>(&k_batch<384>); }
}  // namespace ea
