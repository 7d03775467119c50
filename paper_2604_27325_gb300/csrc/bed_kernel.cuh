// Fused per-matrix kernel of the batched divide-and-conquer symmetric eigensolver (sm_103a).
//
// One thread block solves one matrix at a time, entirely in shared memory:
//   a0  stage A[b] into shared memory (TMA bulk copy + mbarrier, or coalesced loads), read the lower
//       triangle, check finiteness, scale by a power of two
//   a1  Householder tridiagonalization; the reflector dot products are warp-shuffle reductions
//   a2  tear the tridiagonal along the static divide tree (Sec. 2.1, Eq. (2)-(3))
//   a3  2x2 leaves by one Jacobi rotation (Sec. 2.2)
//   a4  per merge (Eq. (4)-(5)): coupling vector z, pole ordering, deflation
//   a5  secular roots (Eq. (8)-(21)): one thread per root, hybrid-section then Halley in coordinates
//       relative to the nearer pole; a warp stops iterating when all of its lanes have converged
//       (the GPU form of the progressive batch shrinkage, Eq. (22))
//   a6  Gu-Eisenstat z-hat (Eq. (25)) and normalized eigenvectors (Eq. (24))
//   a7  merge GEMM Q <- blkdiag(Q1, Q2) Q^ (Eq. (4))
//   a8  back-transform through the Householder reflectors
//   a9  ascending order, sign convention, store
// Thread layout: NT = NMAX * G threads; "column" col = tid % NMAX, "group" grp = tid / NMAX. Phases
// indexed by a row/column/root use threads tid < n.
#pragma once

#include <cfloat>
#include <cstdint>

#include <cuda_runtime.h>

#include "bed_internal.h"

namespace bed {

constexpr float kU = 0x1p-24f;  // unit roundoff of binary32

template <int NMAX, int G>
struct Smem {
    static constexpr int LD = NMAX + 1;  // odd stride: column walks hit distinct banks
    float A[NMAX * LD];  // matrix; after a1 row k holds reflector k in columns k+2..n-1
    float Q[NMAX * LD];  // eigenvectors of the current blocks (block diagonal)
    float M[NMAX * LD];  // staging of A[b] (dense n x n); merge workspace (rows = sorted poles)
    float P[G * NMAX];   // per-group partial sums
    float vv[NMAX], ww[NMAX];              // reflector v and w of the current step
    float d[NMAX], e[NMAX], tau[NMAX];     // tridiagonal and reflector scalars
    float lam[NMAX];                       // eigenvalue of each column of Q
    float ds[NMAX], zs[NMAX];              // merge: poles and z in ascending pole order
    float cd[NMAX], cz[NMAX];              // merge: compacted (non-deflated first) poles and z
    float tq[NMAX], zh[NMAX];              // merge: root offsets from their poles, z-hat
    float rc[NMAX], rs[NMAX];              // merge: Givens deflation rotations (by sorted position)
    float sgn[NMAX];
    float brho[NMAX], bnz[NMAX], btol[NMAX];  // per merge block: rho = |beta|, |z|, tolerance
    float bsc[NMAX];  // per merge block: power of two that brings max(max|d|, rho|z|^2) into [0.5, 1)
    int rank[NMAX];   // column c of the children -> its sorted position
    int inv[NMAX];    // compacted index -> sorted position
    int org[NMAX];    // root -> compacted index of the pole it is measured from
    int rotj[NMAX];   // sorted position -> rotation partner (-1: none)
    int defl[NMAX];
    int bK[NMAX];     // per merge block: number of secular roots
    int brot[NMAX];   // per merge block: close-pole rotations present
    int outc[NMAX];   // output column j <- column outc[j] of Q
    float red[32];
    int flag_rot;
    int info;
    unsigned int evals, roots, deflated;
    alignas(8) unsigned long long mbar;
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sort key with a total order: NaN sorts last, ties broken by index by the callers.
__device__ __forceinline__ float sort_key(float x) { return isnan(x) ? INFINITY : x; }

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the mbarrier; gives up after `limit_ns` and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------------------------------------------
// a5: one secular root (Eq. (8)) of the compacted, ascending poles d[0] < ... < d[K-1].
// Root q lies in (d_q, d_{q+1}) for q < K-1 (Eq. (9)) and in (d_{K-1}, upper] for q = K-1
// (Eq. (10)-(11)). Every participating lane of the warp (mask) runs the same number of loop trips,
// so that the vote that retires the warp is taken convergently.
// ---------------------------------------------------------------------------------------------
struct RootOut {
    int org;      // pole index the offset is measured from (0..K-1)
    float tau;    // lambda - d[org]
    int evals;    // f evaluations
    bool conv;
};

__device__ __forceinline__ RootOut secular_root(const float* __restrict__ d, const float* __restrict__ z,
                                                int K, int q, float rho, const KParams& kp,
                                                unsigned mask)
{
    RootOut r{q, 0.f, 0, false};
    bool done = false;
    const bool top = (q == K - 1);
    float L = 0.f, U;
    if (!top) {
        U = d[q + 1] - d[q];
    } else {
        // Eq. (10)-(11): lambda_top <= d_top + rho |z|^2 and lambda_top <= |D + rho z z^T|_F.
        // Both bounds are raised by their FP32 rounding error so the bracket keeps the root.
        float zn2 = 0.f, sd2 = 0.f, sdz = 0.f, sdza = 0.f;
        for (int j = 0; j < K; ++j) {
            const float z2 = z[j] * z[j];
            zn2 += z2;
            sd2 = fmaf(d[j], d[j], sd2);
            sdz = fmaf(d[j], z2, sdz);
            sdza = fmaf(fabsf(d[j]), z2, sdza);
        }
        U = rho * zn2 * (1.f + 2.f * (K + 2) * kU);
        const float rz = rho * zn2;
        const float fro2 = fmaf(rz, rz, fmaf(2.f * rho, sdz, sd2));
        const float err2 = 4.f * (K + 4) * kU * fmaf(rz, rz, fmaf(2.f * rho, sdza, sd2));
        const float fro = sqrtf(fmaxf(fro2 + err2, 0.f));
        const float uf = (fro - d[K - 1]) + 4.f * kU * (fro + fabsf(d[K - 1]));
        if (uf > 0.f && uf < U) U = uf;
        if (K == 1) {  // one pole: 1 + rho z^2/(d - lambda) = 0 has lambda = d + rho z^2
            r.tau = rho * z[0] * z[0];
            r.conv = true;
            done = true;
        }
    }
    const float width0 = U;
    int o = q;
    int state = 0;  // 0: first bisection (Eq. (13)-(15)); 1: multi-section (Eq. (16)); 2: Halley (Eq. (20))
    int nsec = 0, nh = 0;
    float h = 0.5f * U;
    const float kinv = 1.f / static_cast<float>(kp.k_ms);
    const int cap = 2 + kp.max_sec + kp.max_halley;
    for (int it = 0; it < cap; ++it) {
        if (kp.retire && !__any_sync(mask, !done)) break;  // progressive shrinkage (Eq. (22))
        if (done) continue;
        // Eq. (8), (18), (21) at lambda = d[o] + h, with d_j - lambda = (d_j - d_o) - h
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, sa = 0.f;
        const float dorg = d[o];
        for (int j = 0; j < K; ++j) {
            const float del = (d[j] - dorg) - h;
            const float inv = __frcp_rn(del);
            const float zj = z[j];
            const float t = zj * zj * inv;
            const float ti = t * inv;
            s0 += t;
            s1 += ti;
            s2 = fmaf(ti, inv, s2);
            sa += fabsf(t);
        }
        const float f = fmaf(rho, s0, 1.f);
        const float f1 = rho * s1;
        const float f2 = 2.f * rho * s2;
        const float err = fmaf(rho, sa, 1.f);
        ++r.evals;
        if (state < 2) {
            // Eq. (14): keep the root bracketed
            if (f > 0.f) U = h;
            else if (f < 0.f) L = h;
            else { done = true; r.conv = true; }
            if (state == 0) {
                if (!done && !top && f < 0.f) {
                    // root in the upper half of (d_q, d_{q+1}): measure it from d_{q+1}
                    const float sh = d[q + 1] - d[q];
                    o = q + 1;
                    L -= sh;
                    U = 0.f;
                }
                state = 1;
            } else {
                ++nsec;
            }
            if (!done) {
                if ((U - L) < kp.sec_eps * width0 || nsec >= kp.max_sec) {
                    state = 2;
                    h = 0.5f * (L + U);
                } else {
                    h = fmaf(U - L, kinv, L);  // Eq. (16)
                }
            }
        } else {
            if (f == 0.f || fabsf(f) <= kp.stop_c * kU * err) {
                done = true;
                r.conv = true;
            } else {
                if (f > 0.f) U = h;
                else L = h;
                if ((U - L) <= 2.f * kU * fmaxf(fabsf(L), fabsf(U))) {
                    // the bracket has shrunk to rounding level: the sign of f no longer says more
                    done = true;
                    r.conv = true;
                } else if (++nh > kp.max_halley) {
                    done = true;  // not converged: keep the last iterate
                } else {
                    const float den = 2.f * f1 * f1 - f * f2;
                    float hn = h - 2.f * f * f1 / den;  // Eq. (20)
                    const bool inside = (hn > L) && (top ? hn <= U : hn < U);
                    if (!(den > 0.f) || !inside) hn = 0.5f * (L + U);
                    if (fabsf(hn - h) <= 4.f * kU * fabsf(hn)) {
                        done = true;
                        r.conv = true;
                    }
                    h = hn;
                }
            }
        }
    }
    r.org = o;
    if (!(top && K == 1)) r.tau = h;
    return r;
}

// ---------------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------------
template <int NMAX, int G>
__global__ void __launch_bounds__(NMAX * G)
    eigh_kernel(const float* __restrict__ A, float* __restrict__ W, float* __restrict__ V,
                int32_t* __restrict__ info, int64_t batch, const __grid_constant__ Plan plan,
                const KParams kp, bed_counters* __restrict__ counters, int bulk)
{
    constexpr int NT = NMAX * G;
    constexpr int NW = NT / 32;
    constexpr int LD = Smem<NMAX, G>::LD;
    constexpr int RPT = NMAX / G;  // merge-GEMM rows per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<NMAX, G>& S = *reinterpret_cast<Smem<NMAX, G>*>(smem_raw);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int col = tid % NMAX;
    const int grp = tid / NMAX;
    const int n = plan.n;
    const uint32_t bar = smem_u32(&S.mbar);
    uint32_t phase = 0;

    if (bulk) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }

    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        const float* Ab = A + b * (int64_t)n * n;
        float* Wb = W + b * (int64_t)n;
        float* Vb = V + b * (int64_t)n * n;

        // ---------------- a0: stage the matrix -------------------------------------------------
        if (bulk) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (tid == 0) {
            S.info = 0;
            S.evals = 0;
            S.roots = 0;
            S.deflated = 0;
        }
        __syncthreads();
        bool timed_out = false;
        if (bulk) {
            const uint32_t bytes = static_cast<uint32_t>(n * n * sizeof(float));
            if (tid == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(S.M)),
                    "l"(Ab), "r"(bytes), "r"(bar)
                    : "memory");
            }
            if (!mbar_wait_bounded(bar, phase, 2000000000ull)) {
                timed_out = true;
                // wait once more, again bounded, for the copy still in flight
                mbar_wait_bounded(bar, phase, 2000000000ull);
            }
            phase ^= 1u;
        } else {
            for (int i = tid; i < n * n; i += NT) S.M[i] = __ldg(Ab + i);
        }
        if (timed_out) atomicOr(&S.info, BED_INFO_TIMEOUT);
        __syncthreads();

        // lower triangle -> max |a|, finiteness
        float amax = 0.f;
        bool bad = false;
        for (int i = warp; i < n; i += NW)
            for (int j = lane; j <= i; j += 32) {
                const float x = S.M[i * n + j];
                if (!(fabsf(x) <= FLT_MAX)) bad = true;
                else amax = fmaxf(amax, fabsf(x));
            }
        amax = warp_max(amax);
        if (lane == 0) S.red[warp] = amax;
        if (bad) atomicOr(&S.info, BED_INFO_NONFINITE);
        __syncthreads();
        if (S.info & (BED_INFO_NONFINITE | BED_INFO_TIMEOUT)) {
            const float qnan = __int_as_float(0x7fc00000);
            for (int i = tid; i < n; i += NT) Wb[i] = qnan;
            for (int i = tid; i < n * n; i += NT) Vb[i] = qnan;
            if (info && tid == 0) info[b] = S.info;
            const bool stop = (S.info & BED_INFO_TIMEOUT) != 0;
            __syncthreads();
            if (stop) return;  // the barrier phase is no longer known: leave the remaining matrices
            continue;
        }
        amax = S.red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) amax = fmaxf(amax, S.red[w]);
        // exact power-of-two scaling to max|a| in [0.5, 1): norms below cannot overflow or underflow
        int ex = 0;
        if (amax > 0.f) frexpf(amax, &ex);
        const float scale = ldexpf(1.f, -ex);
        const float unscale = ldexpf(1.f, ex);
        for (int i = warp; i < n; i += NW)
            for (int j = lane; j <= i; j += 32) {
                const float x = S.M[i * n + j] * scale;
                S.A[i * LD + j] = x;
                S.A[j * LD + i] = x;
            }
        __syncthreads();

        // ---------------- a1: Householder tridiagonalization ------------------------------------
        for (int k = 0; k + 2 < n; ++k) {
            const int r0 = k + 1;
            const int m = n - r0;
            // every warp forms reflector k from row k (= column k; the matrix is kept symmetric)
            const float alpha = S.A[k * LD + r0];
            float part = 0.f;
            for (int j = r0 + 1 + lane; j < n; j += 32) {
                const float x = S.A[k * LD + j];
                part = fmaf(x, x, part);
            }
            const float xn2 = warp_sum(part);
            float tau = 0.f, beta = alpha, scal = 0.f;
            if (xn2 > 0.f) {
                const float nrm = sqrtf(fmaf(alpha, alpha, xn2));
                beta = (alpha >= 0.f) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = 1.f / (alpha - beta);
            }
            // partial products p = A22 v over row groups
            if (col < m) {
                const int i = r0 + col;
                float acc = 0.f;
                for (int j = r0 + grp; j < n; j += G) {
                    const float vj = (j == r0) ? 1.f : S.A[k * LD + j] * scal;
                    acc = fmaf(S.A[j * LD + i], vj, acc);
                }
                S.P[grp * NMAX + i] = acc;
                if (grp == 0) S.vv[i] = (i == r0) ? 1.f : S.A[k * LD + i] * scal;
            }
            __syncthreads();
            // w = p - (tau/2)(p.v) v with p = tau A22 v
            if (warp == 0) {
                float pl[2] = {0.f, 0.f};
                float pvp = 0.f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = r0 + lane + 32 * h;
                    if (i < n) {
                        float p = 0.f;
#pragma unroll
                        for (int g = 0; g < G; ++g) p += S.P[g * NMAX + i];
                        p *= tau;
                        pl[h] = p;
                        pvp = fmaf(p, S.vv[i], pvp);
                    }
                }
                const float c = 0.5f * tau * warp_sum(pvp);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = r0 + lane + 32 * h;
                    if (i < n) S.ww[i] = fmaf(-c, S.vv[i], pl[h]);
                }
            }
            if (tid == 0) {
                S.d[k] = S.A[k * LD + k];
                S.e[k] = beta;
                S.tau[k] = tau;
            }
            __syncthreads();
            // A22 -= v w^T + w v^T; row k keeps v (columns r0+1..n-1)
            if (col < m) {
                const int j = r0 + col;
                const float vj = S.vv[j], wj = S.ww[j];
                for (int i = r0 + grp; i < n; i += G)
                    S.A[i * LD + j] -= fmaf(S.vv[i], wj, S.ww[i] * vj);
                if (grp == 0 && j > r0) S.A[k * LD + j] = vj;
            }
            __syncthreads();
        }
        if (tid == 0) {
            if (n >= 2) {
                S.d[n - 2] = S.A[(n - 2) * LD + n - 2];
                S.d[n - 1] = S.A[(n - 1) * LD + n - 1];
                S.e[n - 2] = S.A[(n - 1) * LD + n - 2];
            } else {
                S.d[0] = S.A[0];
            }
        }
        __syncthreads();

        // ---------------- a2: tear (Eq. (3)) ----------------------------------------------------
        if (tid < n) {
            float dt = S.d[tid];
            if ((plan.cut_mask >> tid) & 1ull) dt -= fabsf(S.e[tid]);
            if (tid > 0 && ((plan.cut_mask >> (tid - 1)) & 1ull)) dt -= fabsf(S.e[tid - 1]);
            S.d[tid] = dt;
        }
        __syncthreads();

        // ---------------- a3: leaves ------------------------------------------------------------
        if (tid < plan.nleaves) {
            const int lo = plan.leaf_lo[tid];
            if (plan.leaf_hi[tid] - lo == 1) {
                S.lam[lo] = S.d[lo];
                S.Q[lo * LD + lo] = 1.f;
            } else {
                const float a = S.d[lo], bb = S.e[lo], c = S.d[lo + 1];
                float t = 0.f;
                if (bb != 0.f) {
                    const float th = (c - a) / (2.f * bb);
                    t = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                }
                const float cs = rsqrtf(fmaf(t, t, 1.f));
                const float sn = t * cs;
                S.lam[lo] = fmaf(-t, bb, a);
                S.lam[lo + 1] = fmaf(t, bb, c);
                S.Q[lo * LD + lo] = cs;
                S.Q[lo * LD + lo + 1] = sn;
                S.Q[(lo + 1) * LD + lo] = -sn;
                S.Q[(lo + 1) * LD + lo + 1] = cs;
            }
        }
        __syncthreads();

        // ---------------- a4-a7: merges, deepest level first -----------------------------------
        for (int L = 0; L < plan.nlevels; ++L) {
            const int bi = (tid < n) ? plan.blk[L][tid] : 0xFF;
            const bool act = (bi != 0xFF);
            int lo = 0, mid = 0, hi = 0;
            if (act) {
                lo = plan.m_lo[bi];
                mid = plan.m_mid[bi];
                hi = plan.m_hi[bi];
            }
            // P1: z (Eq. (5)), pole order, block scalars
            if (act) {
                const int c = tid;
                const float beta = S.e[mid - 1];
                const float rho = fabsf(beta);
                const float sig = (beta >= 0.f) ? 1.f : -1.f;
                const float* z1 = &S.Q[(mid - 1) * LD];  // last row of Q1
                const float* z2 = &S.Q[mid * LD];        // first row of Q2
                const float zc = (c < mid) ? sig * z1[c] : z2[c];
                const float kc = sort_key(S.lam[c]);
                int p = 0;
                float nz2 = 0.f, dmax = 0.f;
                for (int c2 = lo; c2 < hi; ++c2) {
                    const float l2 = S.lam[c2];
                    const float k2 = sort_key(l2);
                    p += (k2 < kc) || (k2 == kc && c2 < c);
                    const float zz = (c2 < mid) ? z1[c2] : z2[c2];
                    nz2 = fmaf(zz, zz, nz2);
                    dmax = fmaxf(dmax, fabsf(l2));
                }
                S.rank[c] = lo + p;
                S.ds[lo + p] = S.lam[c];
                S.zs[lo + p] = zc;
                if (c == lo) {
                    const float bscale = fmaxf(dmax, rho * nz2);
                    int ex = 0;
                    if (bscale > 0.f) frexpf(bscale, &ex);
                    S.brho[bi] = rho;
                    S.bnz[bi] = sqrtf(nz2);
                    S.btol[bi] = kp.defl_c * kU * bscale;
                    S.bsc[bi] = ldexpf(1.f, -ex);
                    S.brot[bi] = 0;
                }
            }
            if (tid == 0) S.flag_rot = 0;
            __syncthreads();
            // P2: deflation of negligible couplings; detect close-pole pairs
            if (act) {
                const int t = tid;
                const float rho = S.brho[bi], nz = S.bnz[bi], tol = S.btol[bi];
                const float zp = S.zs[t];
                const int dfl = (rho * fabsf(zp) * nz <= tol);
                S.defl[t] = dfl;
                S.rotj[t] = -1;
                if (!dfl) {
                    int j = t + 1;
                    while (j < hi && rho * fabsf(S.zs[j]) * nz <= tol) ++j;
                    if (j < hi) {
                        const float zj = S.zs[j];
                        const float r = hypotf(zp, zj);
                        const float cc = zj / r, ss = zp / r;
                        if (fabsf((S.ds[j] - S.ds[t]) * cc * ss) <= tol) {
                            S.brot[bi] = 1;
                            S.flag_rot = 1;
                        }
                    }
                }
            }
            __syncthreads();
            // P3: close-pole Givens deflation, one pass in pole order (rare)
            if (S.flag_rot) {
                if (act && tid == lo && S.brot[bi]) {
                    const float tol = S.btol[bi];
                    int pj = -1;
                    for (int p = lo; p < hi; ++p) {
                        if (S.defl[p]) continue;
                        if (pj < 0) {
                            pj = p;
                            continue;
                        }
                        const float r = hypotf(S.zs[pj], S.zs[p]);
                        const float cc = S.zs[p] / r, ss = S.zs[pj] / r;
                        if (fabsf((S.ds[p] - S.ds[pj]) * cc * ss) <= tol) {
                            const float a = S.ds[pj], bb = S.ds[p];
                            S.ds[pj] = fmaf(cc * cc, a, ss * ss * bb);
                            S.ds[p] = fmaf(ss * ss, a, cc * cc * bb);
                            S.zs[p] = r;
                            S.zs[pj] = 0.f;
                            S.defl[pj] = 1;
                            S.rotj[pj] = p;
                            S.rc[pj] = cc;
                            S.rs[pj] = ss;
                        }
                        pj = p;
                    }
                }
                __syncthreads();
            }
            // P4: compaction, non-deflated poles first (ascending). The secular problem of the block is
            // scaled exactly by a power of two to unit size: the derivatives of f grow like
            // 1/(d - lambda)^3 and would overflow FP32 for blocks whose spectrum is far below 1
            if (act) {
                const int t = tid;
                const float sc = S.bsc[bi];
                int nb = 0, K = 0;
                for (int p = lo; p < hi; ++p) {
                    const int nd = !S.defl[p];
                    K += nd;
                    nb += (p < t) & nd;
                }
                const int q = S.defl[t] ? (K + (t - lo - nb)) : nb;
                S.inv[lo + q] = t;
                S.cd[lo + q] = S.ds[t] * sc;
                S.cz[lo + q] = S.zs[t];
                if (t == lo) {
                    S.bK[bi] = K;
                    atomicAdd(&S.deflated, static_cast<unsigned>(hi - lo - K));
                }
            }
            __syncthreads();
            // P5: secular roots, one thread per root
            {
                int K = 0, q = 0;
                if (act) {
                    K = S.bK[bi];
                    q = tid - lo;
                }
                const bool part = act && (q < K);
                const unsigned mask = __ballot_sync(0xffffffffu, part);
                if (part) {
                    const float sc = S.bsc[bi];
                    const RootOut r = secular_root(S.cd + lo, S.cz + lo, K, q, S.brho[bi] * sc, kp, mask);
                    S.org[lo + q] = lo + r.org;
                    S.tq[lo + q] = r.tau;
                    S.lam[lo + q] = (S.cd[lo + r.org] + r.tau) * (1.f / sc);
                    atomicAdd(&S.evals, static_cast<unsigned>(r.evals));
                    atomicAdd(&S.roots, 1u);
                    if (!r.conv) atomicOr(&S.info, BED_INFO_NOT_CONVERGED);
                } else if (act) {
                    S.org[lo + q] = lo + q;
                    S.tq[lo + q] = 0.f;
                    S.lam[lo + q] = S.cd[lo + q] * (1.f / S.bsc[bi]);
                }
            }
            __syncthreads();
            // P6: Gu-Eisenstat z-hat, Eq. (25), as a product of interlaced ratios
            if (act) {
                const int K = S.bK[bi];
                const int i = tid - lo;
                if (i < K) {
                    const float di = S.cd[lo + i];
                    const float rho = S.brho[bi] * S.bsc[bi];
                    // (lambda_{K-1} - d_i)/rho first: it is the only factor that may exceed 1, so the
                    // running product falls monotonically to its result and cannot underflow early
                    float prod = ((S.cd[S.org[lo + K - 1]] - di) + S.tq[lo + K - 1]) / rho;
                    for (int j = 0; j < K - 1; ++j) {
                        const float num = (S.cd[S.org[lo + j]] - di) + S.tq[lo + j];  // lambda_j - d_i
                        const float den = (j < i) ? (S.cd[lo + j] - di) : (S.cd[lo + j + 1] - di);
                        prod *= num / den;
                    }
                    S.zh[lo + i] = copysignf(sqrtf(fmaxf(prod, 0.f)), S.cz[lo + i]);
                }
            }
            __syncthreads();
            // P7: eigenvectors of the merge (Eq. (24)) in sorted-pole rows, rotations undone
            if (act) {
                const int K = S.bK[bi];
                const int q = tid - lo;
                const int cq = tid;
                for (int p = lo; p < hi; ++p) S.M[p * LD + cq] = 0.f;
                if (q < K) {
                    const float dorg = S.cd[S.org[lo + q]];
                    const float tq = S.tq[lo + q];
                    float nrm2 = 0.f;
                    for (int i = 0; i < K; ++i) {
                        const float v = S.zh[lo + i] / ((S.cd[lo + i] - dorg) - tq);
                        S.M[S.inv[lo + i] * LD + cq] = v;
                        nrm2 = fmaf(v, v, nrm2);
                    }
                    const float inv = 1.f / sqrtf(nrm2);
                    for (int i = 0; i < K; ++i) S.M[S.inv[lo + i] * LD + cq] *= inv;
                } else {
                    S.M[S.inv[lo + q] * LD + cq] = 1.f;
                }
                if (S.brot[bi]) {
                    for (int p = hi - 1; p >= lo; --p) {
                        const int j = S.rotj[p];
                        if (j >= 0) {
                            const float cc = S.rc[p], ss = S.rs[p];
                            const float yp = S.M[p * LD + cq], yj = S.M[j * LD + cq];
                            S.M[p * LD + cq] = fmaf(cc, yp, ss * yj);
                            S.M[j * LD + cq] = fmaf(-ss, yp, cc * yj);
                        }
                    }
                }
            }
            __syncthreads();
            // P8: Q <- blkdiag(Q1, Q2) Q^ (Eq. (4)); rows of Q^ are gathered through the pole order
            {
                const int bc = (col < n) ? plan.blk[L][col] : 0xFF;
                float acc[RPT];
                int clo = 0, cmid = 0, chi = 0;
                if (bc != 0xFF) {
                    clo = plan.m_lo[bc];
                    cmid = plan.m_mid[bc];
                    chi = plan.m_hi[bc];
#pragma unroll
                    for (int k = 0; k < RPT; ++k) acc[k] = 0.f;
                    for (int c = clo; c < chi; ++c) {
                        const float mv = S.M[S.rank[c] * LD + col];
                        const bool left = c < cmid;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            const int r = clo + grp + G * k;
                            if (r < chi && ((r < cmid) == left)) acc[k] = fmaf(S.Q[r * LD + c], mv, acc[k]);
                        }
                    }
                }
                __syncthreads();
                if (bc != 0xFF) {
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        const int r = clo + grp + G * k;
                        if (r < chi) S.Q[r * LD + col] = acc[k];
                    }
                }
            }
            __syncthreads();
        }

        // ---------------- a8: back-transform V = H_0 ... H_{n-3} Q_T --------------------------
        for (int k = n - 3; k >= 0; --k) {
            const float tk = S.tau[k];
            if (tk == 0.f) continue;
            const int r0 = k + 1;
            if (col < n) {
                float acc = 0.f;
                for (int i = r0 + grp; i < n; i += G) {
                    const float vi = (i == r0) ? 1.f : S.A[k * LD + i];
                    acc = fmaf(vi, S.Q[i * LD + col], acc);
                }
                S.P[grp * NMAX + col] = acc;
            }
            __syncthreads();
            if (col < n) {
                float w = 0.f;
#pragma unroll
                for (int g = 0; g < G; ++g) w += S.P[g * NMAX + col];
                w *= tk;
                for (int i = r0 + grp; i < n; i += G) {
                    const float vi = (i == r0) ? 1.f : S.A[k * LD + i];
                    S.Q[i * LD + col] = fmaf(-vi, w, S.Q[i * LD + col]);
                }
            }
            __syncthreads();
        }

        // ---------------- a9: ascending order, signs, store ------------------------------------
        if (tid < n) {
            const float kc = sort_key(S.lam[tid]);
            int r = 0;
            for (int t2 = 0; t2 < n; ++t2) {
                const float k2 = sort_key(S.lam[t2]);
                r += (k2 < kc) || (k2 == kc && t2 < tid);
            }
            S.outc[r] = tid;
        }
        __syncthreads();
        if (tid < n) {
            const int src = S.outc[tid];
            int im = 0;
            float vm = fabsf(S.Q[src]);
            for (int i = 1; i < n; ++i) {
                const float v = fabsf(S.Q[i * LD + src]);
                if (v > vm) {
                    vm = v;
                    im = i;
                }
            }
            S.sgn[tid] = (S.Q[im * LD + src] < 0.f) ? -1.f : 1.f;
            Wb[tid] = S.lam[src] * unscale;
        }
        __syncthreads();
        for (int i = warp; i < n; i += NW)
            for (int j = lane; j < n; j += 32) Vb[i * n + j] = S.sgn[j] * S.Q[i * LD + S.outc[j]];
        if (tid == 0) {
            if (info) info[b] = S.info;
            if (counters) {
                atomicAdd(&counters->matrices, 1ull);
                atomicAdd(&counters->roots, static_cast<unsigned long long>(S.roots));
                atomicAdd(&counters->evals, static_cast<unsigned long long>(S.evals));
                atomicAdd(&counters->deflated, static_cast<unsigned long long>(S.deflated));
            }
        }
        __syncthreads();
    }
}

template <int NMAX, int G>
cudaError_t launch_eigh_t(const float* A, float* W, float* V, int32_t* info, int64_t batch,
                          const Plan& P, const KParams& kp, bed_counters* counters, bool bulk,
                          cudaStream_t stream)
{
    const size_t smem = sizeof(Smem<NMAX, G>);
    auto kern = eigh_kernel<NMAX, G>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    const int64_t max_grid = 2147483647LL;
    const unsigned grid = static_cast<unsigned>(batch < max_grid ? batch : max_grid);
    kern<<<grid, NMAX * G, smem, stream>>>(A, W, V, info, batch, P, kp, counters, bulk ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace bed
