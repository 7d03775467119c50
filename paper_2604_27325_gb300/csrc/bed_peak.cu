// FP32 FMA throughput probe: the measured denominator of the eigensolver's FP32 ALU roofline.
//
// Every thread runs kChains independent FMA chains for `iters` rounds, so that each warp scheduler
// always has a ready FMA to issue; the result is stored so the work cannot be removed. The host times
// the launch with CUDA events and divides 2 * kChains * iters * threads FLOPs by it. Nothing here is
// part of the eigensolver; it only measures what the SMs deliver at the clocks they run at.
#include <cuda_runtime.h>

#include "bed_internal.h"

namespace bed {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) fma_peak_kernel(float* __restrict__ out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = static_cast<float>(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace bed

extern "C" {

int bed_fma_peak_chains(void) { return bed::kChains; }

bed_status bed_fma_peak_launch(float* out, int blocks, int threads, int iters, cudaStream_t stream)
{
    if (!out || blocks < 1 || threads < 32 || threads > 256 || threads % 32 != 0 || iters < 1)
        return BED_ERR_INVALID_ARG;
    // a, b keep x bounded (|x| -> b / (1 - a)) without letting the compiler fold the chain
    bed::fma_peak_kernel<<<blocks, threads, 0, stream>>>(out, iters, 0.999999f, 1e-6f);
    return cudaGetLastError() == cudaSuccess ? BED_OK : BED_ERR_CUDA;
}

}  // extern "C"
