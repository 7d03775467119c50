// Instantiations of the fused eigensolver kernel for matrices of up to 64 rows.
#include "bed_kernel.cuh"

namespace bed {
template cudaError_t launch_eigh_t<64, 2>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<64, 4>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                            const KParams&, bed_counters*, bool, cudaStream_t);
template cudaError_t launch_eigh_t<64, 4, true>(const float*, float*, float*, int32_t*, int64_t, int64_t, const Plan&,
                                                  const KParams&, bed_counters*, bool, cudaStream_t);
}  // namespace bed
