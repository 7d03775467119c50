// C ABI of the batched eigensolver: argument validation, the divide-tree plan, launch selection.
#include <algorithm>
#include <cfloat>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "bed_internal.h"

namespace bed {

namespace {

struct MergeRec {
    int lo, mid, hi, depth;
};

// Sec. 2.1: blocks are torn at floor(s/2) until they have at most leaf_size rows.
void split(int lo, int hi, int depth, int leaf, std::vector<MergeRec>& merges, std::vector<int>& leaves)
{
    const int s = hi - lo;
    if (s <= leaf) {
        leaves.push_back(lo);
        leaves.push_back(hi);
        return;
    }
    const int mid = lo + s / 2;
    split(lo, mid, depth + 1, leaf, merges, leaves);
    split(mid, hi, depth + 1, leaf, merges, leaves);
    merges.push_back({lo, mid, hi, depth});
}

thread_local char g_last_cuda_error[256] = "";

}  // namespace

bed_status cuda_fail(cudaError_t e)
{
    std::snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
    return BED_ERR_CUDA;
}

bool build_plan(int n, int leaf_size, Plan* P)
{
    if (n < 1 || n > kMaxN || leaf_size < 1 || leaf_size > kMaxLeaf) return false;
    std::vector<MergeRec> merges;
    std::vector<int> leaves;
    split(0, n, 0, leaf_size, merges, leaves);
    std::memset(P, 0, sizeof *P);
    P->n = n;
    P->nleaves = static_cast<int>(leaves.size() / 2);
    P->nmerge = static_cast<int>(merges.size());
    for (int i = 0; i < P->nleaves; ++i) {
        P->leaf_lo[i] = static_cast<uint8_t>(leaves[2 * i]);
        P->leaf_hi[i] = static_cast<uint8_t>(leaves[2 * i + 1]);
        P->max_leaf = std::max(P->max_leaf, leaves[2 * i + 1] - leaves[2 * i]);
    }
    int maxd = -1;
    for (const auto& m : merges) maxd = m.depth > maxd ? m.depth : maxd;
    P->nlevels = maxd + 1;
    if (P->nlevels > kMaxLevels) return false;
    std::memset(P->blk, 0xFF, sizeof P->blk);
    int idx = 0;
    for (int L = 0; L < P->nlevels; ++L) {  // level 0 = deepest merges
        const int depth = maxd - L;
        P->level_start[L] = static_cast<uint8_t>(idx);
        for (const auto& m : merges) {
            if (m.depth != depth) continue;
            P->m_lo[idx] = static_cast<uint8_t>(m.lo);
            P->m_mid[idx] = static_cast<uint8_t>(m.mid);
            P->m_hi[idx] = static_cast<uint8_t>(m.hi);
            for (int t = m.lo; t < m.hi; ++t) P->blk[L][t] = static_cast<uint8_t>(idx);
            P->cut_mask |= 1ull << (m.mid - 1);
            ++idx;
        }
    }
    P->level_start[P->nlevels] = static_cast<uint8_t>(idx);
    return true;
}

// Leaf size of the divide tree for leaf_size = 0 (automatic), by n: the autotuner's choice on a GB300
// (per-n timing of every team shape and leaf size of 2, 4 and 8 rows, batch 2048; the team shapes it
// chose are the built-in ones of bed_ragged_default_tuning). Leaves of up to 4 rows pay for 4 register
// slots of the QL leaf solver, of 5-6 rows for 6 and of 7-8 for 8, so whether a deeper tree pays
// depends on n.
constexpr unsigned char kAutoLeaf[kMaxN + 1] = {
    0, 4, 2, 8, 8, 8, 8, 4, 4, 8, 8, 8, 8, 4, 4, 4,
    4, 4, 8, 8, 8, 8, 8, 8, 8, 4, 4, 4, 4, 4, 4, 4,
    4, 4, 4, 4, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8,
    8, 8, 8, 8, 8, 8, 8, 8, 8, 4, 4, 4, 4, 4, 4, 4,
    4,
};

int auto_leaf(int n) { return (n >= 1 && n <= kMaxN) ? kAutoLeaf[n] : 8; }

// Divide trees of every n and leaf size, built once on first use (host memory, read-only afterwards).
const Plan* cached_plan(int n, int leaf_size)
{
    if (leaf_size == 0) leaf_size = auto_leaf(n);
    static Plan plans[kMaxLeaf][kMaxN + 1];
    static bool ok[kMaxLeaf][kMaxN + 1];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int leaf = 1; leaf <= kMaxLeaf; ++leaf)
            for (int m = 1; m <= kMaxN; ++m) ok[leaf - 1][m] = build_plan(m, leaf, &plans[leaf - 1][m]);
    });
    if (n < 1 || n > kMaxN || leaf_size < 1 || leaf_size > kMaxLeaf || !ok[leaf_size - 1][n]) return nullptr;
    return &plans[leaf_size - 1][n];
}

cudaError_t launch_eigh(int nmax, int g, const float* A, float* W, float* V, int32_t* info,
                        int64_t batch, int64_t blocks, const Plan& P, const KParams& kp,
                        bed_counters* counters, bool bulk, cudaStream_t stream)
{
#define BED_CASE(NM, GG)                                                                                   \
    if (nmax == NM && g == GG) {                                                                           \
        if (GG == 4 && kp.merge_tc)                                                                        \
            return launch_eigh_t<NM, 4, true>(A, W, V, info, batch, blocks, P, kp, counters, bulk, stream); \
        return launch_eigh_t<NM, GG>(A, W, V, info, batch, blocks, P, kp, counters, bulk, stream);         \
    }
    BED_CASE(16, 2)
    BED_CASE(16, 4)
    BED_CASE(32, 2)
    BED_CASE(32, 4)
    BED_CASE(48, 2)
    BED_CASE(48, 4)
    BED_CASE(64, 2)
    BED_CASE(64, 4)
#undef BED_CASE
    return cudaErrorInvalidValue;
}

// Validates the parameters shared by every entry point and derives the kernel constants.
bool make_kparams(const bed_params* p, bed_params* prm, KParams* kp)
{
    bed_default_params(prm);
    if (p) *prm = *p;
    if (prm->leaf_size < 0 || prm->leaf_size > kMaxLeaf) return false;
    if (prm->k_multisection < 2 || prm->k_multisection > 64) return false;
    if (prm->max_section_iters < 0 || prm->max_section_iters > 256) return false;
    if (prm->max_halley_iters < 1 || prm->max_halley_iters > 256) return false;
    if (!(prm->section_rel_eps > 0.f && prm->section_rel_eps < 1.f)) return false;
    if (!(prm->stop_c >= 1.f && prm->stop_c <= 1e6f)) return false;
    if (!(prm->deflation_tol_scale >= 1.f && prm->deflation_tol_scale <= 1e6f)) return false;
    if (prm->retire_by_vote != 0 && prm->retire_by_vote != 1) return false;
    if (prm->merge_tensor_cores != 0 && prm->merge_tensor_cores != 1) return false;
    if (prm->stage_wait_us < 0 || prm->stage_wait_us > 60000000) return false;
    if (prm->matrices_per_cta < 0 || prm->matrices_per_cta > (1 << 20)) return false;
    if (prm->n_bisect_first < 1 || prm->n_bisect_first > 64) return false;
    kp->k_ms = prm->k_multisection;
    kp->max_sec = prm->max_section_iters;
    kp->max_halley = prm->max_halley_iters;
    kp->sec_eps = prm->section_rel_eps;
    kp->stop_c = prm->stop_c;
    kp->defl_c = prm->deflation_tol_scale;
    kp->retire = prm->retire_by_vote;
    kp->merge_tc = prm->merge_tensor_cores;
    kp->n_bisect = prm->n_bisect_first;
    kp->stage_wait_ns = 1000ull * static_cast<unsigned long long>(prm->stage_wait_us);
    return true;
}

namespace {

// Team shape: nmax rows of tiles, G lanes per row; the smallest nmax that holds n unless the caller
// asks for a thread count, which then selects the smallest (nmax >= n, G) with G * nmax equal to it.
// Automatic: G = 4, except G = 2 for the 64-row team (128 threads with up to 128 registers each: half
// the warps repeat the tridiagonalization's per-step vector work, and a warp's 16-column tile still
// fits in registers; measured faster alone and beside the other sizes). The tensor-core merge variant
// is instantiated for G = 4 only, so it keeps G = 4.
bool team_shape(int n, const bed_params& prm, int* nmax_out, int* g_out)
{
    int nmax = n <= 16 ? 16 : (n <= 32 ? 32 : (n <= 48 ? 48 : 64));
    int g = (nmax == 64 && !prm.merge_tensor_cores) ? 2 : 4;
    if (prm.threads_per_matrix != 0) {
        bool found = false;
        for (const int nm : {16, 32, 48, 64}) {
            if (nm < n || found) continue;
            for (const int gg : {4, 2})
                if (!found && prm.threads_per_matrix == gg * nm) {
                    nmax = nm;
                    g = gg;
                    found = true;
                }
        }
        if (!found) return false;
    }
    *nmax_out = nmax;
    *g_out = g;
    return true;
}

}  // namespace

bed_status eigh_common(const float* A, float* W, float* V, int32_t* info, int64_t batch, int n,
                       const bed_params* p, bed_counters* counters, cudaStream_t stream, bool host_mapped)
{
    if (n < 1 || n > kMaxN) return BED_ERR_UNSUPPORTED_N;
    if (batch < 0) return BED_ERR_INVALID_ARG;
    bed_params prm;
    KParams kp;
    if (!make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    int nmax = 0, g = 0;
    if (!team_shape(n, prm, &nmax, &g)) return BED_ERR_INVALID_ARG;
    if (batch == 0) return BED_OK;
    if (!A || !W || !V) return BED_ERR_INVALID_ARG;
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(W) |
                           reinterpret_cast<uintptr_t>(V)) & 3u;
    if (mis || (reinterpret_cast<uintptr_t>(info) & 3u) || (reinterpret_cast<uintptr_t>(counters) & 7u))
        return BED_ERR_INVALID_ARG;
    if (A == V) return BED_ERR_INVALID_ARG;
    const Plan* P = cached_plan(n, prm.leaf_size);
    if (!P) return BED_ERR_INVALID_ARG;
    // TMA bulk staging needs a 16-byte aligned source and a size that is a multiple of 16 bytes for
    // every matrix: A 16-byte aligned and n even.
    // Matrices in mapped host memory are read with plain loads.
    const bool bulk = !host_mapped && ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) && (n % 2 == 0);
    const int64_t mpc = prm.matrices_per_cta;
    const int64_t blocks = mpc > 0 ? (batch + mpc - 1) / mpc : batch;
    const cudaError_t e = launch_eigh(nmax, g, A, W, V, info, batch, blocks, *P, kp, counters, bulk, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return BED_OK;
}

namespace {

bool tuning_valid(const bed_ragged_tuning& t)
{
    for (int n = 1; n <= kMaxN; ++n) {
        if (t.leaf[n] < 1 || t.leaf[n] > kMaxLeaf) return false;
        const int tt = t.team[n];
        if (tt > 4) return false;
        const int cap = tt == 0 ? 64 : (tt == 4 ? 48 : (tt == 1 ? 32 : 16));
        if (n > cap) return false;
    }
    return true;
}

}  // namespace

}  // namespace bed

extern "C" {

void bed_ragged_default_tuning(bed_ragged_tuning* t)
{
    if (!t) return;
    std::memset(t, 0, sizeof *t);
    for (int n = 0; n <= bed::kMaxN; ++n) {
        t->team[n] = static_cast<unsigned char>(n <= 16 ? 2 : (n <= 32 ? 1 : (n <= 48 ? 4 : 0)));
        t->leaf[n] = static_cast<unsigned char>(n >= 1 ? bed::auto_leaf(n) : 8);
    }
}

size_t bed_eigh_ragged_workspace_size(int64_t count) { return bed::ragged_workspace_bytes(count < 0 ? 0 : count); }

bed_status bed_eigh_ragged_f32(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count,
                               float* W, const int64_t* w_offsets, float* V, int32_t* info,
                               const bed_params* p, const bed_ragged_tuning* tuning, void* workspace,
                               size_t workspace_bytes, bed_counters* counters, cudaStream_t stream)
{
    if (count < 0) return BED_ERR_INVALID_ARG;
    bed_params prm;
    bed::KParams kp;
    if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    bed_ragged_tuning tune;
    bed_ragged_default_tuning(&tune);
    if (tuning) tune = *tuning;
    if (!bed::tuning_valid(tune)) return BED_ERR_INVALID_ARG;
    if (count == 0) return BED_OK;
    if (!A || !offsets || !ns || !W || !w_offsets || !V || !workspace) return BED_ERR_INVALID_ARG;
    const uintptr_t mis4 = (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(W) |
                            reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(ns) |
                            reinterpret_cast<uintptr_t>(info)) & 3u;
    const uintptr_t mis8 = (reinterpret_cast<uintptr_t>(offsets) | reinterpret_cast<uintptr_t>(w_offsets) |
                            reinterpret_cast<uintptr_t>(counters)) & 7u;
    if (mis4 || mis8 || (reinterpret_cast<uintptr_t>(workspace) & 15u)) return BED_ERR_INVALID_ARG;
    if (A == V) return BED_ERR_INVALID_ARG;
    if (workspace_bytes < bed::ragged_workspace_bytes(count)) return BED_ERR_INVALID_ARG;
    if (count > 2147483647LL) return BED_ERR_INVALID_ARG;
    const cudaError_t e = bed::launch_ragged(A, offsets, ns, count, W, w_offsets, V, info, tune, kp, workspace,
                                             counters, stream);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    return BED_OK;
}

void bed_default_params(bed_params* p)
{
    if (!p) return;
    p->leaf_size = 0;
    p->k_multisection = 4;
    p->max_section_iters = 24;
    p->max_halley_iters = 32;
    p->section_rel_eps = 0x1p-1f;
    p->stop_c = 8.f;
    p->deflation_tol_scale = 8.f;
    p->threads_per_matrix = 0;
    p->retire_by_vote = 1;
    p->merge_tensor_cores = 0;
    p->stage_wait_us = 2000000;
    p->matrices_per_cta = 0;
    p->n_bisect_first = 1;
}

bed_status bed_eigh_f32(const float* A, float* W, float* V, int32_t* info, int64_t batch, int n,
                        const bed_params* p, cudaStream_t stream)
{
    return bed::eigh_common(A, W, V, info, batch, n, p, nullptr, stream, false);
}

bed_status bed_eigh_f32_counted(const float* A, float* W, float* V, int32_t* info, int64_t batch,
                                int n, const bed_params* p, bed_counters* counters,
                                cudaStream_t stream)
{
    if (!counters) return BED_ERR_INVALID_ARG;
    return bed::eigh_common(A, W, V, info, batch, n, p, counters, stream, false);
}

bed_status bed_eigh_f32_host(const float* A_host, float* W_host, float* V_host, int32_t* info_host,
                             int64_t batch, int n, const bed_params* p, float* A_dev, float* W_dev,
                             float* V_dev, int32_t* info_dev, int chunks, cudaStream_t s0,
                             cudaStream_t s1)
{
    if (n < 1 || n > bed::kMaxN) return BED_ERR_UNSUPPORTED_N;
    if (batch < 0 || chunks < 0) return BED_ERR_INVALID_ARG;
    if (batch == 0) return BED_OK;
    if (!A_host || !W_host || !V_host || !A_dev || !W_dev || !V_dev) return BED_ERR_INVALID_ARG;
    if ((info_host == nullptr) != (info_dev == nullptr)) return BED_ERR_INVALID_ARG;
    {
        // validate the parameters and the device buffers once, before anything is enqueued
        bed_params prm;
        bed::KParams kp;
        if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
        const uintptr_t mis = (reinterpret_cast<uintptr_t>(A_dev) | reinterpret_cast<uintptr_t>(W_dev) |
                               reinterpret_cast<uintptr_t>(V_dev) | reinterpret_cast<uintptr_t>(info_dev)) & 3u;
        if (mis || A_dev == V_dev) return BED_ERR_INVALID_ARG;
    }
    // automatic: two pieces (one per stream) from 256 matrices on; more pieces measured slower (each
    // piece is a smaller launch and four more copies)
    int64_t nc = chunks ? chunks : (batch >= 256 ? 2 : 1);
    if (nc > batch) nc = batch;
    const size_t nn = static_cast<size_t>(n) * n;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t b0 = batch * c / nc, b1 = batch * (c + 1) / nc, nb = b1 - b0;
        if (nb == 0) continue;
        cudaStream_t s = (c & 1) ? s1 : s0;
        cudaError_t e = cudaMemcpyAsync(A_dev + b0 * nn, A_host + b0 * nn, nb * nn * sizeof(float),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return bed::cuda_fail(e);
        const bed_status st = bed::eigh_common(A_dev + b0 * nn, W_dev + b0 * n, V_dev + b0 * nn,
                                               info_dev ? info_dev + b0 : nullptr, nb, n, p, nullptr, s, false);
        if (st != BED_OK) return st;
        e = cudaMemcpyAsync(W_host + b0 * n, W_dev + b0 * n, nb * n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(V_host + b0 * nn, V_dev + b0 * nn, nb * nn * sizeof(float),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && info_host)
            e = cudaMemcpyAsync(info_host + b0, info_dev + b0, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return bed::cuda_fail(e);
    }
    return BED_OK;
}

}  // extern "C"

namespace bed {

// Device address of the page-locked host range [p, p + bytes) in the current context, or nullptr when
// any part of it is not page-locked memory mapped into the device's address space. Both ends must lie
// in the same mapping (their device addresses differ by bytes - 1).
const void* mapped_range(const void* p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    const void* last = static_cast<const char*>(p) + (bytes - 1);
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();  // clear the error of an unregistered pointer
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<const char*>(b.devicePointer) - static_cast<const char*>(a.devicePointer) !=
        static_cast<ptrdiff_t>(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

}  // namespace bed

extern "C" {

bed_status bed_eigh_f32_pinned(const float* A_host, float* W_host, float* V_host, int32_t* info_host,
                               int64_t batch, int n, const bed_params* p, cudaStream_t stream)
{
    if (n < 1 || n > bed::kMaxN) return BED_ERR_UNSUPPORTED_N;
    if (batch < 0) return BED_ERR_INVALID_ARG;
    {
        bed_params prm;
        bed::KParams kp;
        if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    }
    if (batch == 0) return BED_OK;
    const size_t nn = static_cast<size_t>(n) * n, b = static_cast<size_t>(batch);
    const float* A = static_cast<const float*>(bed::mapped_range(A_host, b * nn * sizeof(float)));
    float* W = static_cast<float*>(const_cast<void*>(bed::mapped_range(W_host, b * n * sizeof(float))));
    float* V = static_cast<float*>(const_cast<void*>(bed::mapped_range(V_host, b * nn * sizeof(float))));
    int32_t* info = nullptr;
    if (info_host) {
        info = static_cast<int32_t*>(const_cast<void*>(bed::mapped_range(info_host, b * sizeof(int32_t))));
        if (!info) return BED_ERR_INVALID_ARG;
    }
    if (!A || !W || !V) return BED_ERR_INVALID_ARG;
    return bed::eigh_common(A, W, V, info, batch, n, p, nullptr, stream, true);
}

bed_status bed_eigh_many_f32_pinned(int count, const int* ns, const int64_t* batches, const float* const* A_host,
                                    float* const* W_host, float* const* V_host, int32_t* const* info_host,
                                    const bed_params* p, cudaStream_t origin, const cudaStream_t* side, int nside)
{
    if (count < 0 || (count > 0 && (!ns || !batches || !A_host || !W_host || !V_host || !side || nside < 1)))
        return BED_ERR_INVALID_ARG;
    bed_params prm;
    {
        bed::KParams kp;
        if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    }
    // validate every batch (and translate its buffers to device addresses) before anything is enqueued
    struct Dev {
        const float* A;
        float *W, *V;
        int32_t* info;
    };
    std::vector<Dev> dp(count);
    std::vector<int> order;
    for (int k = 0; k < count; ++k) {
        const int n = ns[k];
        if (n < 1 || n > bed::kMaxN) return BED_ERR_UNSUPPORTED_N;
        int nmax = 0, g = 0;
        if (batches[k] < 0 || !bed::team_shape(n, prm, &nmax, &g)) return BED_ERR_INVALID_ARG;
        if (batches[k] == 0) continue;
        const size_t nn = static_cast<size_t>(n) * n, b = static_cast<size_t>(batches[k]);
        Dev& d = dp[k];
        d.A = static_cast<const float*>(bed::mapped_range(A_host[k], b * nn * sizeof(float)));
        d.W = static_cast<float*>(const_cast<void*>(bed::mapped_range(W_host[k], b * n * sizeof(float))));
        d.V = static_cast<float*>(const_cast<void*>(bed::mapped_range(V_host[k], b * nn * sizeof(float))));
        d.info = nullptr;
        if (info_host && info_host[k]) {
            d.info = static_cast<int32_t*>(const_cast<void*>(bed::mapped_range(info_host[k], b * sizeof(int32_t))));
            if (!d.info) return BED_ERR_INVALID_ARG;
        }
        if (!d.A || !d.W || !d.V || d.A == d.V) return BED_ERR_INVALID_ARG;
        order.push_back(k);
    }
    if (order.empty()) return BED_OK;
    // largest n first: its launch is the longest
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
    // fork from and join back to `origin` through two events of this thread (one record / wait pair at a
    // time, so that reusing them is safe)
    struct Events {
        int dev = -1;
        cudaEvent_t fork = nullptr, join = nullptr;
    };
    thread_local std::vector<Events> evs;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    Events* ev = nullptr;
    for (auto& x : evs)
        if (x.dev == dev) ev = &x;
    if (!ev) {
        Events x;
        x.dev = dev;
        e = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return bed::cuda_fail(e);
        evs.push_back(x);
        ev = &evs.back();
    }
    e = cudaEventRecord(ev->fork, origin);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    const int used = nside < static_cast<int>(order.size()) ? nside : static_cast<int>(order.size());
    for (int s = 0; s < used; ++s) {
        e = cudaStreamWaitEvent(side[s], ev->fork, 0);
        if (e != cudaSuccess) return bed::cuda_fail(e);
    }
    // With the team shape left automatic and several batches side by side, sizes 17..32 run 64-thread
    // teams (two lanes per row): half the registers of the 128-thread team, so that more of them share
    // the SMs with the larger sizes' blocks (a lone launch of such a batch is faster with 128 threads)
    const bool concurrent = used > 1 && prm.threads_per_matrix == 0;
    bed_status st = BED_OK;
    for (size_t j = 0; j < order.size() && st == BED_OK; ++j) {
        const int k = order[j];
        bed_params pk = prm;
        if (concurrent && ns[k] > 16 && ns[k] <= 32) pk.threads_per_matrix = 64;
        st = bed::eigh_common(dp[k].A, dp[k].W, dp[k].V, dp[k].info, batches[k], ns[k], &pk, nullptr,
                              side[j % used], true);
    }
    // join even after a failed launch, so that `origin` still orders after whatever was enqueued
    for (int s = 0; s < used; ++s) {
        e = cudaEventRecord(ev->join, side[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev->join, 0);
        if (e != cudaSuccess && st == BED_OK) st = bed::cuda_fail(e);
    }
    return st;
}

bed_status bed_eigh_ragged_f32_noalloc(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count,
                                       float* W, const int64_t* w_offsets, float* V, int32_t* info,
                                       const bed_params* p, const bed_ragged_tuning* tuning,
                                       bed_counters* counters, cudaStream_t stream)
{
    if (count < 0) return BED_ERR_INVALID_ARG;
    if (count > BED_NOALLOC_MAX_COUNT) return BED_ERR_TOO_LARGE;
    bed_params prm;
    bed::KParams kp;
    if (!bed::make_kparams(p, &prm, &kp)) return BED_ERR_INVALID_ARG;
    bed_ragged_tuning tune;
    bed_ragged_default_tuning(&tune);
    if (tuning) tune = *tuning;
    if (!bed::tuning_valid(tune)) return BED_ERR_INVALID_ARG;
    if (count == 0) return BED_OK;
    if (!A || !offsets || !ns || !W || !w_offsets || !V) return BED_ERR_INVALID_ARG;
    const uintptr_t mis4 = (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(W) |
                            reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(ns) |
                            reinterpret_cast<uintptr_t>(info)) & 3u;
    const uintptr_t mis8 = (reinterpret_cast<uintptr_t>(offsets) | reinterpret_cast<uintptr_t>(w_offsets) |
                            reinterpret_cast<uintptr_t>(counters)) & 7u;
    if (mis4 || mis8 || A == V) return BED_ERR_INVALID_ARG;
    void* scratch = nullptr;
    cudaError_t e = bed::noalloc_scratch(&scratch);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    e = bed::launch_ragged(A, offsets, ns, count, W, w_offsets, V, info, tune, kp, scratch, counters, stream);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    return BED_OK;
}

bed_status bed_eigh_backward_f32(const float* W, const float* V, const float* gW, const float* gV, float* gA,
                                 int64_t batch, int n, float gap_eps, cudaStream_t stream)
{
    if (n < 1 || n > bed::kMaxN) return BED_ERR_UNSUPPORTED_N;
    if (batch < 0 || !(gap_eps >= 0.f && gap_eps <= FLT_MAX)) return BED_ERR_INVALID_ARG;
    if (batch == 0) return BED_OK;
    if (!W || !V || !gA || gA == V) return BED_ERR_INVALID_ARG;
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(W) | reinterpret_cast<uintptr_t>(V) |
                           reinterpret_cast<uintptr_t>(gW) | reinterpret_cast<uintptr_t>(gV) |
                           reinterpret_cast<uintptr_t>(gA)) & 3u;
    if (mis) return BED_ERR_INVALID_ARG;
    const cudaError_t e = bed::launch_backward(W, V, gW, gV, gA, batch, n, gap_eps, stream);
    if (e != cudaSuccess) return bed::cuda_fail(e);
    return BED_OK;
}

int bed_max_n(void) { return bed::kMaxN; }

const char* bed_status_string(bed_status s)
{
    switch (s) {
    case BED_OK: return "BED_OK";
    case BED_ERR_INVALID_ARG: return "BED_ERR_INVALID_ARG";
    case BED_ERR_UNSUPPORTED_N: return "BED_ERR_UNSUPPORTED_N";
    case BED_ERR_CUDA: return "BED_ERR_CUDA";
    case BED_ERR_TOO_LARGE: return "BED_ERR_TOO_LARGE";
    case BED_ERR_TIMEOUT: return "BED_ERR_TIMEOUT";
    }
    return "BED_UNKNOWN_STATUS";
}

const char* bed_last_cuda_error(void) { return bed::g_last_cuda_error; }

int bed_plan_describe(int n, int leaf_size, int* merges, int* level_of)
{
    if (leaf_size == 0) leaf_size = bed::auto_leaf(n);
    bed::Plan P;
    if (!bed::build_plan(n, leaf_size, &P)) return -1;
    for (int L = 0; L < P.nlevels; ++L)
        for (int i = P.level_start[L]; i < P.level_start[L + 1]; ++i) {
            if (merges) {
                merges[3 * i] = P.m_lo[i];
                merges[3 * i + 1] = P.m_mid[i];
                merges[3 * i + 2] = P.m_hi[i];
            }
            if (level_of) level_of[i] = L;
        }
    return P.nmerge;
}

}  // extern "C"
