// Instantiations of the fused eigensolver kernel for matrices of up to 32 rows.
#include "bed_kernel.cuh"

namespace bed {
template cudaError_t launch_eigh_t<32, 2>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<32, 4>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<32, 4, true>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                                  const KParams&, bed_counters*, bool, cudaStream_t);
}  // namespace bed
