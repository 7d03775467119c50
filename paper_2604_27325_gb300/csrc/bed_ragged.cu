// Ragged batches: one persistent launch over matrices of mixed n (1 <= n <= 64).
//
// Every thread block has 256 threads and works through "units" taken from an atomic counter in the
// caller's workspace. A unit is one team configuration and up to as many matrices as it has teams:
//   team type 0: one team of 256 threads (the n <= 64 code path: NMAX 64, 4 lanes per row)
//   team type 1: two teams of 128 threads (NMAX 32, 4 lanes per row)
//   team type 2: four teams of 64 threads (NMAX 16, 4 lanes per row)
//   team type 3: eight teams of 32 threads (NMAX 16, 2 lanes per row)
//   team type 4: one team of 192 threads (NMAX 48, 4 lanes per row; the block's last 64 threads idle)
// Each team runs the same per-matrix code as the uniform launch (solve_matrix) on its own slice of
// shared memory, with its own named barrier and mbarrier. A one-block pre-kernel sorts the matrices by
// (rank of their team type, n descending) into the workspace and resets the counter; both launches are
// stream-ordered and can be captured into a CUDA graph.
#include <cstring>
#include <mutex>

#include "bed_kernel.cuh"

namespace bed {

constexpr int kRaggedThreads = 256;
constexpr int kTeamTypes = 5;
constexpr int kMaxTeams = 8;

__host__ __device__ constexpr int team_count(int t) { return (t == 0 || t == 4) ? 1 : (t == 1 ? 2 : (t == 2 ? 4 : 8)); }

// Units are handed out by rank: rank r holds the units of the team type in hex digit r of kRankTypes,
// read from the left. The order is measured, not largest first: the 32-row pairs, then the 64-row teams,
// the 16-row teams, and the 48-row teams last. Against plain type order (64, 32, 16, 16, 48 rows) it
// runs the 8192-matrix ragged workload 1.8 % faster (8.47 -> 8.62 M matrices/s) and 4 x 512 uniform
// sizes 1 % faster; largest first (64, 48, 32, 16) is slower on both (8.38 M/s, 297 us against 281 us),
// as are the 48-row teams first (283-308 us): a 48-row team pairs badly with the 64-row teams on an SM.
constexpr unsigned kRankTypes = 0x10234u;
__host__ __device__ constexpr int type_of_rank(int r) { return static_cast<int>((kRankTypes >> (4 * (4 - r))) & 0xFu); }
__host__ __device__ constexpr int rank_of_type(int t)
{
    return type_of_rank(0) == t ? 0 : (type_of_rank(1) == t ? 1 : (type_of_rank(2) == t ? 2 : (type_of_rank(3) == t ? 3 : 4)));
}
static_assert(type_of_rank(0) < kTeamTypes && type_of_rank(1) < kTeamTypes && type_of_rank(2) < kTeamTypes &&
                  type_of_rank(3) < kTeamTypes && type_of_rank(4) < kTeamTypes &&
                  rank_of_type(type_of_rank(0)) == 0 && rank_of_type(type_of_rank(1)) == 1 &&
                  rank_of_type(type_of_rank(2)) == 2 && rank_of_type(type_of_rank(3)) == 3 &&
                  rank_of_type(type_of_rank(4)) == 4,
              "the ranks are a permutation of the team types");

template <int NMAX, int G>
__host__ __device__ constexpr size_t slice_bytes()
{
    return (sizeof(Smem<NMAX, G>) + 15) / 16 * 16;
}

__host__ __device__ constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kRaggedSmem = cmax(cmax(cmax(slice_bytes<64, 4>(), 2 * slice_bytes<32, 4>()),
                                         cmax(4 * slice_bytes<16, 4>(), 8 * slice_bytes<16, 2>())),
                                    slice_bytes<48, 4>());

// Divide trees for every n and every leaf size, written once per device (setup before first use).
__device__ Plan g_plans[kMaxLeaf][kMaxN + 1];

struct RaggedHeader {
    unsigned int next_unit;                   // work counter (reset by the pre-kernel)
    unsigned int total_units;
    unsigned int unit_start[kTeamTypes + 1];  // first unit of each rank (rank_of_type)
    unsigned int mat_start[kTeamTypes + 1];   // first position in `order` of each rank
    unsigned int pad[2];
};
static_assert(sizeof(RaggedHeader) == 64, "workspace header is 64 bytes");

struct RaggedTune {
    uint8_t team[kMaxN + 1];
    uint8_t leaf[kMaxN + 1];
};

// Orders the matrices by (rank of their team type, n descending) with a counting sort; invalid sizes are
// flagged. Each thread loads PER sizes at a time so that their global loads are in flight together; the
// bins of each rank are scanned by one warp (two bins per lane).
__global__ void __launch_bounds__(1024) ragged_order_kernel(const int32_t* __restrict__ ns, int64_t count,
                                                            const RaggedTune tune, RaggedHeader* __restrict__ hdr,
                                                            int32_t* __restrict__ order, int32_t* __restrict__ info)
{
    constexpr int NK = kTeamTypes * kMaxN;  // key = rank * 64 + (64 - n)
    constexpr int PER = 8;
    __shared__ unsigned int hist[NK];
    __shared__ unsigned int offs[NK];
    __shared__ unsigned int tsum[kTeamTypes], tbase[kTeamTypes];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < NK; i += nt) hist[i] = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += static_cast<int64_t>(nt) * PER) {
        int v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int64_t i = base + static_cast<int64_t>(k) * nt + tid;
            v[k] = (i < count) ? ns[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int64_t i = base + static_cast<int64_t>(k) * nt + tid;
            if (i >= count) continue;
            const int n = v[k];
            if (n < 1 || n > kMaxN) {
                if (info) info[i] = BED_INFO_BAD_N;
                continue;
            }
            atomicAdd(&hist[rank_of_type(tune.team[n]) * kMaxN + (kMaxN - n)], 1u);
        }
    }
    __syncthreads();
    static_assert(kMaxN == 64, "two bins per lane");
    if (warp < kTeamTypes) {
        const int b0 = warp * kMaxN + 2 * lane;
        const unsigned int h0 = hist[b0], h1 = hist[b0 + 1];
        unsigned int x = h0 + h1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        offs[b0] = x - h0 - h1;  // relative to the start of the rank
        offs[b0 + 1] = x - h1;
        if (lane == 31) tsum[warp] = x;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned int acc = 0, units = 0;
        for (int r = 0; r < kTeamTypes; ++r) {
            hdr->mat_start[r] = acc;
            hdr->unit_start[r] = units;
            tbase[r] = acc;
            acc += tsum[r];
            const int per = team_count(type_of_rank(r));
            units += (tsum[r] + per - 1) / per;
        }
        hdr->mat_start[kTeamTypes] = acc;
        hdr->unit_start[kTeamTypes] = units;
        hdr->total_units = units;
        hdr->next_unit = 0;
    }
    __syncthreads();
    for (int i = tid; i < NK; i += nt) offs[i] += tbase[i / kMaxN];
    __syncthreads();
    for (int64_t base = 0; base < count; base += static_cast<int64_t>(nt) * PER) {
        int v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int64_t i = base + static_cast<int64_t>(k) * nt + tid;
            v[k] = (i < count) ? ns[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int64_t i = base + static_cast<int64_t>(k) * nt + tid;
            const int n = v[k];
            if (i >= count || n < 1 || n > kMaxN) continue;
            const unsigned int p = atomicAdd(&offs[rank_of_type(tune.team[n]) * kMaxN + (kMaxN - n)], 1u);
            order[p] = static_cast<int32_t>(i);
        }
    }
}

struct RaggedArgs {
    const MatDesc* desc;  // descriptor form (the request loop): per-matrix addresses, plain loads
    const float* A;
    const int64_t* offsets;
    const int32_t* ns;
    float* W;
    const int64_t* w_offsets;
    float* V;
    int32_t* info;
    RaggedHeader* hdr;
    const int32_t* order;
    bed_counters* counters;
};

template <int NMAX, int G>
__device__ __forceinline__ bool run_team(unsigned char* smem, const RaggedArgs& a, const RaggedTune& tune,
                                         const KParams& kp, int team, int ttid, unsigned first, unsigned last,
                                         unsigned long long* mbars, uint32_t* phases)
{
    const unsigned slot = first + team;
    if (slot >= last) return true;  // the whole team is idle in a partial unit
    const int i = a.order[slot];
    const int n = a.ns[i];
    const Plan& plan = g_plans[tune.leaf[n] - 1][n];
    Smem<NMAX, G>& S = *reinterpret_cast<Smem<NMAX, G>*>(smem + team * slice_bytes<NMAX, G>());
    const float* Ab;
    float *Wb, *Vb;
    int32_t* Ib;
    bool bulk;
    if (a.desc) {
        const MatDesc d = a.desc[i];
        Ab = d.A;
        Wb = d.W;
        Vb = d.V;
        Ib = d.info;
        bulk = false;  // the input may be page-locked host memory
    } else {
        Ab = a.A + a.offsets[i];
        Wb = a.W + a.w_offsets[i];
        Vb = a.V + a.offsets[i];
        Ib = a.info ? a.info + i : nullptr;
        bulk = (n % 2 == 0) && ((reinterpret_cast<uintptr_t>(Ab) & 15u) == 0);
    }
    uint32_t phase = phases[team];
    const bool ok = solve_matrix<NMAX, G>(S, plan, kp, ttid, 1 + team, smem_u32(&mbars[team]), phase, Ab, Wb, Vb,
                                          Ib, a.counters, bulk);
    if (ttid == 0) phases[team] = phase;
    return ok;
}

__global__ void __launch_bounds__(kRaggedThreads, 4)
    ragged_kernel(const RaggedArgs a, const RaggedTune tune, const KParams kp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long mbars[kMaxTeams];
    __shared__ uint32_t phases[kMaxTeams];
    __shared__ unsigned int s_unit;
    __shared__ int s_stop;
    const int tid = threadIdx.x;
    if (tid < kMaxTeams) {
        mbar_init(smem_u32(&mbars[tid]));
        phases[tid] = 0;
    }
    if (tid == 0) s_stop = 0;
    __syncthreads();
    const unsigned total = a.hdr->total_units;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(&a.hdr->next_unit, 1u);
        __syncthreads();
        const unsigned u = s_unit;
        if (u >= total || s_stop) break;
        int rk = 0;
        while (rk + 1 < kTeamTypes && u >= a.hdr->unit_start[rk + 1]) ++rk;
        const int t = type_of_rank(rk);
        const unsigned first = a.hdr->mat_start[rk] + (u - a.hdr->unit_start[rk]) * team_count(t);
        const unsigned last = a.hdr->mat_start[rk + 1];
        bool ok = true;
        switch (t) {
        case 0: ok = run_team<64, 4>(smem_raw, a, tune, kp, 0, tid, first, last, mbars, phases); break;
        case 1: ok = run_team<32, 4>(smem_raw, a, tune, kp, tid / 128, tid % 128, first, last, mbars, phases); break;
        case 2: ok = run_team<16, 4>(smem_raw, a, tune, kp, tid / 64, tid % 64, first, last, mbars, phases); break;
        case 3: ok = run_team<16, 2>(smem_raw, a, tune, kp, tid / 32, tid % 32, first, last, mbars, phases); break;
        default:  // one 192-thread team; the last 64 threads wait at the block barrier below
            if (tid < 192) ok = run_team<48, 4>(smem_raw, a, tune, kp, 0, tid, first, last, mbars, phases);
            break;
        }
        if (!ok) s_stop = 1;  // a timed-out staging copy never landed: this block stops taking work
        // the next unit may stage a matrix by bulk copy into memory any thread wrote in this one
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
}

namespace {

std::mutex g_setup_mutex;
bool g_setup_done[64] = {};
int g_ragged_grid[64] = {};

// Per-device setup: divide trees for every n into g_plans, shared-memory attribute, grid size.
cudaError_t ragged_setup(int* grid)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_setup_done[dev]) {
        static Plan host_plans[kMaxLeaf][kMaxN + 1];
        std::memset(host_plans, 0, sizeof host_plans);
        for (int leaf = 1; leaf <= kMaxLeaf; ++leaf)
            for (int n = 1; n <= kMaxN; ++n) build_plan(n, leaf, &host_plans[leaf - 1][n]);
        e = cudaMemcpyToSymbol(g_plans, host_plans, sizeof host_plans);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(kRaggedSmem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(ragged_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_kernel, kRaggedThreads, kRaggedSmem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_ragged_grid[dev] = (per_sm > 0 ? per_sm : 1) * sms;
        g_setup_done[dev] = true;
    }
    *grid = g_ragged_grid[dev];
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_ragged(const float* A, const int64_t* offsets, const int32_t* ns, int64_t count, float* W,
                          const int64_t* w_offsets, float* V, int32_t* info, const bed_ragged_tuning& tuning,
                          const KParams& kp, void* workspace, bed_counters* counters, cudaStream_t stream)
{
    int grid = 0;
    cudaError_t e = ragged_setup(&grid);
    if (e != cudaSuccess) return e;
    RaggedTune tune;
    std::memcpy(tune.team, tuning.team, sizeof tune.team);
    std::memcpy(tune.leaf, tuning.leaf, sizeof tune.leaf);
    RaggedHeader* hdr = static_cast<RaggedHeader*>(workspace);
    int32_t* order = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + sizeof(RaggedHeader));
    ragged_order_kernel<<<1, 1024, 0, stream>>>(ns, count, tune, hdr, order, info);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RaggedArgs a{nullptr, A, offsets, ns, W, w_offsets, V, info, hdr, order, counters};
    ragged_kernel<<<grid, kRaggedThreads, kRaggedSmem, stream>>>(a, tune, kp);
    return cudaGetLastError();
}

cudaError_t launch_ragged_desc(const MatDesc* desc, const int32_t* ns, int64_t count,
                               const bed_ragged_tuning& tuning, const KParams& kp, void* workspace,
                               cudaStream_t stream)
{
    int grid = 0;
    cudaError_t e = ragged_setup(&grid);
    if (e != cudaSuccess) return e;
    RaggedTune tune;
    std::memcpy(tune.team, tuning.team, sizeof tune.team);
    std::memcpy(tune.leaf, tuning.leaf, sizeof tune.leaf);
    RaggedHeader* hdr = static_cast<RaggedHeader*>(workspace);
    int32_t* order = reinterpret_cast<int32_t*>(static_cast<char*>(workspace) + sizeof(RaggedHeader));
    // sizes outside [1, 64] are flagged through the descriptors' info words by the persistent kernel's
    // callers (the request loop admits only valid sizes), so the ordering pass gets no info array
    ragged_order_kernel<<<1, 1024, 0, stream>>>(ns, count, tune, hdr, order, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RaggedArgs a{desc, nullptr, nullptr, ns, nullptr, nullptr, nullptr, nullptr, hdr, order, nullptr};
    ragged_kernel<<<grid, kRaggedThreads, kRaggedSmem, stream>>>(a, tune, kp);
    return cudaGetLastError();
}

size_t ragged_workspace_bytes(int64_t count)
{
    return (sizeof(RaggedHeader) + static_cast<size_t>(count) * sizeof(int32_t) + 255) / 256 * 256;
}

// Scratch of the allocation-free ragged entry point: the workspace of a batch of at most
// BED_NOALLOC_MAX_COUNT matrices, as a file-scope device array that every GPU loading the library
// holds until the process exits. In host code `g_noalloc_scratch` only names the symbol; its device
// address is looked up once per device below and is what the kernels receive.
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[(sizeof(RaggedHeader) + BED_NOALLOC_MAX_COUNT * sizeof(int32_t) + 255) / 256 * 256];

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {};
}  // namespace

cudaError_t noalloc_scratch(void** ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // with device `dev` current
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace bed
