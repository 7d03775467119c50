// Backward of the batched eigendecomposition: dL/dA from (W, V) and the loss gradients (gW, gV).
//
//   K  = diag(gW) + F o (V^T gV),  F_ij = 1/(W_j - W_i) for |W_j - W_i| > gap_eps (i != j), else 0
//   G  = V K V^T,                  gA = (G + G^T) / 2
//
// First-order perturbation theory of the symmetric eigenproblem (dW_i = v_i^T dA v_i,
// dv_i = sum_{j != i} v_j v_j^T dA v_i / (W_i - W_j)); gA is the gradient over symmetric
// perturbations of A. One thread block per matrix, the three products in shared memory with FP32
// FMA: thread (column j, row group g) owns rows g, g + G, ... of column j of each product.
#include <atomic>
#include <cfloat>

#include <cuda_runtime.h>

#include "bed_internal.h"

namespace bed {

template <int NMAX>
struct BwdSmem {
    static constexpr int LD = NMAX + 1;  // odd stride: the column walk of the last product is conflict-free
    float V[NMAX * LD];
    float X[NMAX * LD];  // gV, then V K
    float K[NMAX * LD];  // diag(gW) + F o (V^T gV), then G = V K V^T
    float lam[NMAX], gl[NMAX];
};

template <int NMAX, int G>
__global__ void __launch_bounds__(NMAX * G)
    eigh_backward_kernel(const float* __restrict__ W, const float* __restrict__ V, const float* __restrict__ gW,
                         const float* __restrict__ gV, float* __restrict__ gA, int64_t batch, int n, float gap_eps)
{
    constexpr int NT = NMAX * G;
    constexpr int LD = BwdSmem<NMAX>::LD;
    constexpr int RPT = NMAX / G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem<NMAX>& S = *reinterpret_cast<BwdSmem<NMAX>*>(smem_raw);
    const int tid = threadIdx.x;
    const int col = tid % NMAX;
    const int grp = tid / NMAX;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NW = NT / 32;

    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        const float* Vb = V + b * (int64_t)n * n;
        const float* gVb = gV ? gV + b * (int64_t)n * n : nullptr;
        for (int i = warp; i < n; i += NW)
            for (int j = lane; j < n; j += 32) {
                S.V[i * LD + j] = __ldg(Vb + i * n + j);
                S.X[i * LD + j] = gVb ? __ldg(gVb + i * n + j) : 0.f;
            }
        if (tid < n) {
            S.lam[tid] = __ldg(W + b * n + tid);
            S.gl[tid] = gW ? __ldg(gW + b * n + tid) : 0.f;
        }
        __syncthreads();
        float acc[RPT];
        // K = diag(gW) + F o (V^T gV)
        if (col < n) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) acc[t] = 0.f;
            for (int k = 0; k < n; ++k) {
                const float x = S.X[k * LD + col];
#pragma unroll
                for (int t = 0; t < RPT; ++t) acc[t] = fmaf(S.V[k * LD + grp + G * t], x, acc[t]);
            }
            const float lj = S.lam[col];
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int i = grp + G * t;
                if (i < n) {
                    const float gap = lj - S.lam[i];
                    float kv;
                    if (i == col) kv = S.gl[i];
                    else kv = (fabsf(gap) > gap_eps) ? acc[t] / gap : 0.f;
                    S.K[i * LD + col] = kv;
                }
            }
        }
        __syncthreads();
        // X = V K
        if (col < n) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) acc[t] = 0.f;
            for (int k = 0; k < n; ++k) {
                const float kv = S.K[k * LD + col];
#pragma unroll
                for (int t = 0; t < RPT; ++t) {
                    const int i = grp + G * t;
                    if (i < n) acc[t] = fmaf(S.V[i * LD + k], kv, acc[t]);
                }
            }
        }
        __syncthreads();
        if (col < n) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int i = grp + G * t;
                if (i < n) S.X[i * LD + col] = acc[t];
            }
        }
        __syncthreads();
        // K = X V^T
        if (col < n) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) acc[t] = 0.f;
            for (int k = 0; k < n; ++k) {
                const float v = S.V[col * LD + k];
#pragma unroll
                for (int t = 0; t < RPT; ++t) {
                    const int i = grp + G * t;
                    if (i < n) acc[t] = fmaf(S.X[i * LD + k], v, acc[t]);
                }
            }
        }
        __syncthreads();
        if (col < n) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int i = grp + G * t;
                if (i < n) S.K[i * LD + col] = acc[t];
            }
        }
        __syncthreads();
        float* gAb = gA + b * (int64_t)n * n;
        for (int i = warp; i < n; i += NW)
            for (int j = lane; j < n; j += 32) gAb[i * n + j] = 0.5f * (S.K[i * LD + j] + S.K[j * LD + i]);
        __syncthreads();
    }
}

template <int NMAX>
static cudaError_t launch_bwd(const float* W, const float* V, const float* gW, const float* gV, float* gA,
                              int64_t batch, int n, float gap_eps, cudaStream_t stream)
{
    constexpr int G = 4;
    const size_t smem = sizeof(BwdSmem<NMAX>);
    auto kern = eigh_backward_kernel<NMAX, G>;
    static std::atomic<unsigned long long> configured{0};  // per device, set on its first launch
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(configured.load(std::memory_order_acquire) & (1ull << (dev & 63)))) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        configured.fetch_or(1ull << (dev & 63), std::memory_order_release);
    }
    const unsigned grid = static_cast<unsigned>(batch < 2147483647LL ? batch : 2147483647LL);
    kern<<<grid, NMAX * G, smem, stream>>>(W, V, gW, gV, gA, batch, n, gap_eps);
    return cudaGetLastError();
}

cudaError_t launch_backward(const float* W, const float* V, const float* gW, const float* gV, float* gA,
                            int64_t batch, int n, float gap_eps, cudaStream_t stream)
{
    if (n <= 16) return launch_bwd<16>(W, V, gW, gV, gA, batch, n, gap_eps, stream);
    if (n <= 32) return launch_bwd<32>(W, V, gW, gV, gA, batch, n, gap_eps, stream);
    return launch_bwd<64>(W, V, gW, gV, gA, batch, n, gap_eps, stream);
}

}  // namespace bed
