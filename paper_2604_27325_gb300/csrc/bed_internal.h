// Internal declarations shared by the C-ABI layer and the kernel translation units.
#pragma once

#include <cstdint>

#include <cuda_runtime_api.h>

#include "../../include/bed.h"

namespace bed {

constexpr int kMaxN = 64;
constexpr int kMaxLeaf = 8;  // largest leaf of the divide tree (3..8 rows: implicit QL leaf solver)
constexpr int kMaxLevels = 8;  // merge levels of a tree over n <= 64 rows (6 with 1x1 leaves)

// The divide tree of Sec. 2.1 for one n: blocks are split at floor(s/2) until they have at most
// leaf_size rows. Passed by value to the kernel (a __grid_constant__ parameter), so every thread
// reads it from the constant bank.
struct Plan {
    int n;
    int nleaves;
    int nmerge;
    int nlevels;                            // merge levels; level 0 is the deepest
    int max_leaf;                           // rows of the largest leaf
    unsigned long long cut_mask;            // bit t: the tridiagonal is torn between rows t and t+1
    uint8_t leaf_lo[kMaxN], leaf_hi[kMaxN]; // leaves [lo, hi), 1 to kMaxLeaf rows
    uint8_t m_lo[kMaxN], m_mid[kMaxN], m_hi[kMaxN];  // merges, grouped by level (deepest first)
    uint8_t level_start[kMaxLevels + 1];    // merges of level L: [level_start[L], level_start[L+1])
    uint8_t blk[kMaxLevels][kMaxN];         // merge that owns row/column t at level L, 0xFF if none
};

// Constants of the secular solver and deflation (bed_params minus the launch shape).
struct KParams {
    int k_ms;         // k of Eq. (16)
    int max_sec;      // multi-section cap
    int max_halley;   // Halley cap
    float sec_eps;    // Eq. (17), relative to the initial bracket
    float stop_c;     // Halley stop: |f| <= stop_c * u * err
    float defl_c;     // deflation tolerance scale
    int retire;       // warp-vote retirement of converged roots
    int merge_tc;     // merge products on the tensor cores (split-3xTF32)
    int n_bisect;     // bisection steps before the multi-section of Eq. (16), >= 1
    unsigned long long stage_wait_ns;  // limit of the wait for a matrix's staging copy
};

bool build_plan(int n, int leaf_size, Plan* P);

// Leaf size used for n when bed_params.leaf_size is 0 (automatic).
int auto_leaf(int n);

// One kernel launch over the whole batch. nmax in {16, 32, 64}, g in {2, 4} (threads = nmax * g);
// `blocks` thread blocks (>= 1), block i solving matrices i, i + blocks, ...
// bulk: stage each matrix with a TMA bulk copy (requires 16-byte aligned A and even n).
cudaError_t launch_eigh(int nmax, int g, const float* A, float* W, float* V, int32_t* info,
                        int64_t batch, int64_t blocks, const Plan& P, const KParams& kp,
                        bed_counters* counters, bool bulk, cudaStream_t stream);

cudaError_t launch_ragged(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count, float* W,
                          const int64_t* w_offsets, float* V, int32_t* info, const bed_ragged_tuning& tuning,
                          const KParams& kp, void* workspace, bed_counters* counters, cudaStream_t stream);
size_t ragged_workspace_bytes(int64_t count);
cudaError_t launch_backward(const float* W, const float* V, const float* gW, const float* gV, float* gA,
                            int64_t batch, int n, float gap_eps, cudaStream_t stream);
// Device address of the allocation-free entry point's scratch on the current device (looked up once).
cudaError_t noalloc_scratch(void** ptr);

// One uniform-size launch after full argument validation (the body of bed_eigh_f32); host_mapped: A, W,
// V, info may be device-visible addresses of page-locked host memory, read and written with plain
// loads and stores (no bulk-copy staging).
bed_status eigh_common(const float* A, float* W, float* V, int32_t* info, int64_t batch, int n,
                       const bed_params* p, bed_counters* counters, cudaStream_t stream, bool host_mapped);

// Device address of the page-locked host range [p, p + bytes) in the current context, or nullptr.
const void* mapped_range(const void* p, size_t bytes);

// Records a CUDA error for bed_last_cuda_error() and returns BED_ERR_CUDA.
bed_status cuda_fail(cudaError_t e);

// Addresses of one matrix of a ragged launch in descriptor form (any mix of device memory and
// device-visible page-locked host memory).
struct MatDesc {
    const float* A;  // n x n input, row-major, lower triangle read
    float* W;        // n eigenvalues
    float* V;        // n x n eigenvectors (columns)
    int32_t* info;   // one flag word (may be null)
};

// Ragged launch over descriptors: matrix b has size ns[b] and the addresses desc[b]; desc and ns may
// themselves be device-visible page-locked host memory. Inputs are read with plain loads.
cudaError_t launch_ragged_desc(const MatDesc* desc, const int32_t* ns, int64_t count,
                               const bed_ragged_tuning& tuning, const KParams& kp, void* workspace,
                               cudaStream_t stream);

// Validates bed_params and derives the kernel constants (false: out of range).
bool make_kparams(const bed_params* p, bed_params* prm, KParams* kp);

// TC: the merge products on the tensor cores (split-3xTF32), instantiated for G = 4 teams only.
template <int NMAX, int G, bool TC = false>
cudaError_t launch_eigh_t(const float* A, float* W, float* V, int32_t* info, int64_t batch, int64_t blocks,
                          const Plan& P, const KParams& kp, bed_counters* counters, bool bulk,
                          cudaStream_t stream);

}  // namespace bed
