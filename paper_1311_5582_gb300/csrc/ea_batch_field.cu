// Instantiation of the persistent batch kernel for ensembles in an external
// field, CTAs of up to 384 threads (own translation unit: it compiles in
// parallel with the field-free variants).
#include "ea_batch_kernel.cuh"

namespace ea {
const void *batch_kernel_field_384() { return reinterpret_cast<const void *>(&k_batch<384, true>); }
}  // namespace ea
