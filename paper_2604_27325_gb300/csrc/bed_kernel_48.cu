// Instantiations of the fused eigensolver kernel for matrices of 33 to 48 rows.
#include "bed_kernel.cuh"

namespace bed {
template cudaError_t launch_eigh_t<48, 2>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<48, 4>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<48, 4, true>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                                  const KParams&, bed_counters*, bool, cudaStream_t);
}  // namespace bed
