// Fused per-matrix kernel of the batched divide-and-conquer symmetric eigensolver (sm_103a).
//
// One thread block solves one matrix at a time, entirely in shared memory:
//   a0  stage A[b] into shared memory (TMA bulk copy + mbarrier, or coalesced loads), read the lower
//       triangle, check finiteness, scale by a power of two
//   a1  Householder tridiagonalization: A in column-owned register tiles, p = tau A v from the
//       column sums of each warp's block (A is symmetric), one block barrier per reflector; the
//       steps run in phases of 16 that drop the rows below the phase's first step
//   a2  tear the tridiagonal along the static divide tree (Sec. 2.1, Eq. (2)-(3))
//   a3  leaves (Sec. 2.2): 1x1; 2x2 by one Jacobi rotation; 3 to 8 rows by implicit QL with
//       Wilkinson shifts
//   a4  per merge (Eq. (4)-(5)): coupling vector z, pole ordering, deflation
//   a5  secular roots (Eq. (8)-(21)): 1 or 2 lanes per root (G for 16- and 32-row teams), hybrid-section
//       then Halley in coordinates relative to the nearer pole; a warp stops iterating when all of
//       its lanes have converged (the GPU form of the progressive batch shrinkage, Eq. (22))
//   a6  Gu-Eisenstat z-hat (Eq. (25)) and eigenvectors (Eq. (24)), normalized by a7
//   a7  merge GEMM Q <- blkdiag(Q1, Q2) Q^ (Eq. (4)) in register tiles of 4 rows x 16/G columns
//   a8  back-transform through the Householder reflectors, 8 at a time as I - Y T Y^T, with each
//       column of Q held in the registers of its G lanes and the rows above each block skipped
//   a9  ascending order, sign convention, store
// Thread layouts (NT = NMAX * G threads): "position" pos = tid / G, sub = tid % G: G consecutive
// lanes share one row / column and combine their partial results with shuffles inside the group;
// a1 and a7 use their own register tilings and a5 its own lanes per root, described where they run.
#pragma once

#include <atomic>
#include <cfloat>
#include <cstdint>

#include <cuda_runtime.h>

#include "bed_internal.h"

namespace bed {

constexpr float kU = 0x1p-24f;  // unit roundoff of binary32
constexpr unsigned kFull = 0xffffffffu;
constexpr int kBT = 8;          // reflectors per back-transform block

template <int NMAX, int G>
struct Smem {
    static constexpr int LD = NMAX + 1;  // odd stride: column walks hit distinct banks
    static constexpr int NB = NMAX / 2;  // merges per level, at most
    alignas(16) float A[NMAX * LD];  // the reflectors of a1, transposed (yt_index)
    float Q[NMAX * LD + 3 * LD];      // eigenvectors of the current blocks (block diagonal); P8 tiles read
                                      // up to 3 rows past the last one
    alignas(16) float M[NMAX * LD + 8];  // staging of A[b]; merge workspace (rows = sorted poles); a8
                                         // workspace; P8 tiles read up to 7 columns past the last one
    float d[NMAX], e[NMAX], tau[NMAX];     // tridiagonal and reflector scalars
    float lam[NMAX];                       // eigenvalue of each column of Q
    float ds[NMAX], zs[NMAX];              // merge: poles and z in ascending pole order
    union alignas(16) {  // a1 and the merges never run at the same time
        struct {
            float2 cdz[NMAX];  // merge: compacted (non-deflated first) scaled poles (x) and z^2 (y)
            float cz[NMAX];    // merge: z in the compacted order
            float tq[NMAX], zh[NMAX];             // merge: root offsets from their poles, z-hat
            float rc[NMAX], rs[NMAX];             // merge: Givens deflation rotations (by sorted position)
        };
        struct {
            float hp[2][NMAX];  // a1: p = tau A22 v of the last reflector (by step parity)
            float hu[2][NMAX];  // a1: the last reflector v, 0 before its leading 1
            float hy[2][NMAX];  // a1: the next column, before the last update
        };
    };
    float sgn[NMAX];
    float cinv[NMAX];  // merge: 1 / norm of each column of Q^ (P7), applied by P8
    float brho[NB], btol[NB], bsc[NB];  // per merge of a level: |beta|, tolerance, scale
    int colof[NMAX];  // sorted position -> the column of the children it came from
    int inv[NMAX];    // compacted index -> column of the children (the row of Q^ in M)
    float dorg[NMAX];  // root -> the (scaled) pole it is measured from, d_o
    int rotj[NMAX];   // sorted position -> rotation partner (-1: none)
    int defl[NMAX];
    int outc[NMAX];   // output column j <- column outc[j] of Q
    int bK[NB];       // per merge of a level: number of secular roots
    int brot[NB];     // per merge of a level: close-pole rotations present
    float red[32];
    int flag_rot;
    float unscale;      // 2^e of the input scaling (a0), for the eigenvalues stored in a9
    float* out_w;       // this matrix's outputs, kept here rather than in registers through a1-a8
    float* out_v;
    int32_t* out_info;
    int info;
    unsigned int evals, roots, deflated;
    alignas(8) unsigned long long mbar;
};

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Reductions over the G lanes of a position group; every lane of the warp must call them. xor
// partners combine the same two values in both lanes, so all G lanes obtain bitwise identical results.
template <int G>
__device__ __forceinline__ float gsum(float v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ int gsumi(int v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ float gmax(float v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
template <int G>
__device__ __forceinline__ float gprod(float v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v *= __shfl_xor_sync(kFull, v, o);
    return v;
}

// One-instruction reciprocal (relative error below 1 ulp); its argument here is a distance to a pole of
// a secular problem scaled to unit size, far from the subnormal range.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Vector shared-memory access of N consecutive floats (16- or 8-byte aligned when N is 4, 8 or 2).
template <int N>
__device__ __forceinline__ void load_vec(const float* p, float (&v)[N])
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 t = reinterpret_cast<const float4*>(p)[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else if constexpr (N == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x;
        v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] = p[q];
    }
}
template <int N>
__device__ __forceinline__ void store_vec(float* p, const float (&v)[N])
{
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if constexpr (N == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) p[q] = v[q];
    }
}

// Sum over the 32 / NTC lanes that share lane % NTC (the row lanes of the a1 tile layout); all of
// them get the same value.
template <int NTC>
__device__ __forceinline__ float row_lane_sum(float v)
{
#pragma unroll
    for (int o = NTC; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Lanes along the columns of a warp's block in the a1 tile layout (the rest run along the rows).
template <int NMAX, int G>
__host__ __device__ constexpr int a1_col_lanes()
{
    return 2;
}

// One-instruction square root (relative error about 2^-23) of a non-negative argument, subnormals
// flushed to zero; used for the Householder norms and the Gu-Eisenstat z-hat.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Sort key with a total order: NaN sorts last, ties broken by index by the callers.
__device__ __forceinline__ float sort_key(float x) { return isnan(x) ? INFINITY : x; }

// Reflectors of a1, stored transposed over the storage of S.A once a1 has read the matrix: entry i of
// v_k at Yt[i * NMAX + k], with the 4-float chunks of each row permuted by an XOR of the row index so
// that 16-byte reads of rows i, i + 1, i + 2, i + 3 at the same column fall in distinct banks.
template <int NMAX>
__device__ __forceinline__ int yt_index(int i, int k)
{
    // XOR by at most 8 chunks, and by a divisor of the row's chunk count so that it stays in the row
    constexpr int CH = NMAX / 4;
    constexpr int SW = ((CH % 8 == 0) ? 8 : ((CH % 4 == 0) ? 4 : ((CH % 2 == 0) ? 2 : 1))) - 1;
    return i * NMAX + ((((k >> 2) ^ (i & SW)) << 2) | (k & 3));
}

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

// Waits for phase `parity` of the mbarrier; gives up once `limit_ns` have passed (checked before every
// poll, so a limit of 0 gives up without polling) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (global_timer_ns() - t0 >= limit_ns) return false;
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
}

// Internal flag of S.info (never stored): a staging copy that timed out was still in flight after the
// second, draining wait, so the mbarrier phase is unknown and the team must stop.
constexpr int kInfoUndrained = 1 << 16;
constexpr uint64_t kDrainWaitNs = 2000000000ull;

// ---------------------------------------------------------------------------------------------
// a3 for leaves of 3..8 rows: implicit QL iteration with Wilkinson shifts (the small-block solver the
// paper offers in place of dividing down to 2x2 blocks, Sec. 2.2; the step recurrence is the published
// one of the EISPACK routine tql2). Every lane of a group of LM (4 or 8) runs the same scalar recurrence
// on its own register copy of (d, e) -- no communication -- and applies each plane rotation to its own
// row r of the leaf's eigenvector block. The loops are unrolled over the LM possible positions and
// predicated on the runtime bounds, so d, e and z stay in registers.
// Writes the eigenvalues (lane 0) and row r of the eigenvectors; returns false if an eigenvalue hit
// the iteration cap.
// ---------------------------------------------------------------------------------------------
// c ? a : b through an explicit predicate select: written this way so that a chain of them over an
// unrolled register array is not turned back into an indexed (local-memory) load
__device__ __forceinline__ float selp(bool c, float a, float b)
{
    float r;
    asm("{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %3, 0;\n\tselp.f32 %0, %1, %2, p;\n\t}"
        : "=f"(r)
        : "f"(a), "f"(b), "r"(static_cast<int>(c)));
    return r;
}

constexpr int kLeafMax = 8;

// LM: the register arrays' length, at least the leaf's row count m. The unrolled steps cost LM positions
// whatever m is, so leaves of up to 4 rows run the LM = 4 instance.
template <int LM>
__device__ __forceinline__ bool ql_leaf(const float* __restrict__ dg, const float* __restrict__ eg, int m,
                                        int r, float* __restrict__ lam_out, float* __restrict__ q_row)
{
    float d[LM], e[LM], z[LM];
#pragma unroll
    for (int j = 0; j < LM; ++j) {
        d[j] = (j < m) ? dg[j] : 0.f;
        e[j] = (j < m - 1) ? eg[j] : 0.f;
        z[j] = (j == r) ? 1.f : 0.f;
    }
    bool ok = true;
    // One QL step per pass. Eigenvalue l is final once coupling e[l] is negligible; each pass first moves l
    // past every such coupling, so that the lanes of a warp (up to four leaves) advance together, one
    // step per pass, rather than waiting for each other at every eigenvalue.
    int l = 0, iter = 0;
    for (int pass = 0; pass < 31 * LM; ++pass) {
        int mm = m - 1;
        {
            bool negl[LM - 1];
#pragma unroll
            for (int j = 0; j < LM - 1; ++j)
                negl[j] = (j >= m - 1) || fabsf(e[j]) <= 0x1p-23f * (fabsf(d[j]) + fabsf(d[j + 1]));
            int ln = m - 1;
#pragma unroll
            for (int j = LM - 2; j >= 0; --j)
                if (j >= l && !negl[j]) ln = j;
            if (ln != l) iter = 0;
            l = ln;
            if (l >= m - 1) break;
            if (iter >= 30) {  // not converged: leave eigenvalue l as it is and go on with the next
                ok = false;
                ++l;
                iter = 0;
                continue;
            }
            ++iter;
            // the first negligible coupling after l bounds the unreduced block [l, mm]
#pragma unroll
            for (int j = LM - 2; j >= 0; --j)
                if (j > l && j < m - 1 && negl[j]) mm = j;
        }
        {
            float dl = 0.f, dl1 = 0.f, el = 0.f, dmm = 0.f;
#pragma unroll
            for (int j = 0; j < LM; ++j) {
                dl = selp(j == l, d[j], dl);
                el = selp(j == l, e[j], el);
                dl1 = selp(j == l + 1, d[j], dl1);
                dmm = selp(j == mm, d[j], dmm);
            }
            // Wilkinson shift: the eigenvalue of the top 2x2 block nearer to d_l; the chase starts from
            // d_mm minus it
            float g = (dl1 - dl) * rcp_approx(2.f * el);
            const float rr = sqrt_approx(fmaf(g, g, 1.f));
            g = dmm - dl + el * rcp_approx(g + copysignf(rr, g));
            float sn = 1.f, cs = 1.f, p = 0.f;
            bool split = false;  // the bulge vanished: the block splits, the step ends early
#pragma unroll
            for (int i = LM - 2; i >= 0; --i) {
                if (i < mm && i >= l && !split) {
                    const float f = sn * e[i], b = cs * e[i];
                    const float h2 = fmaf(f, f, g * g);
                    const float ih = rsqrtf(h2);  // one reciprocal square root gives h and 1/h
                    const float h = h2 * ih;
                    e[i + 1] = h;
                    if (h2 < FLT_MIN) {  // (a subnormal square flushes too: the bulge has vanished)
                        e[i + 1] = 0.f;
                        d[i + 1] -= p;
                        split = true;
                    } else {
                        sn = f * ih;
                        cs = g * ih;
                        g = d[i + 1] - p;
                        const float t = fmaf(d[i] - g, sn, 2.f * cs * b);
                        p = sn * t;
                        d[i + 1] = g + p;
                        g = fmaf(cs, t, -b);
                        const float za = z[i], zb = z[i + 1];
                        z[i + 1] = fmaf(sn, za, cs * zb);
                        z[i] = fmaf(cs, za, -sn * zb);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < LM; ++j) {
                if (j == l && !split) {
                    d[j] -= p;
                    e[j] = g;
                }
                if (j == mm) e[j] = 0.f;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < LM; ++j)
        if (j < m) {
            if (r == 0) lam_out[j] = d[j];
            if (r < m) q_row[j] = z[j];
        }
    return ok;
}

// ---------------------------------------------------------------------------------------------
// a5: one secular root (Eq. (8)) of the compacted, ascending, unit-scaled poles
// d[0] < ... < d[K-1] with couplings z_j^2, stored as pairs dz[j] = (d[j], z_j^2). Root q lies in (d_q, d_{q+1}) for q < K-1
// (Eq. (9)) and in (d_{K-1}, upper] for q = K-1 (Eq. (10)-(11)). Called by EVERY lane of the warp (non-participating lanes pass
// part = false): the G lanes of a root split the pole sums and combine them with shuffles, and the
// vote that retires the warp is taken by all 32 lanes.
// ---------------------------------------------------------------------------------------------
struct RootOut {
    int org;      // pole index the offset is measured from (0..K-1)
    float tau;    // lambda - d[org]
    int evals;    // f evaluations
    bool conv;
};

template <int G>
__device__ __forceinline__ RootOut secular_root(const float2* __restrict__ dz, int K, int q, float rho,
                                                const KParams& kp, bool part, int sub)
{
    RootOut r{q, 0.f, 0, false};
    bool done = !part;
    const bool top = part && (q == K - 1);
    float L = 0.f, U = 1.f;
    {
        // Eq. (10)-(11): lambda_top <= d_top + rho |z|^2 and lambda_top <= |D + rho z z^T|_F.
        // Both bounds are raised by their FP32 rounding error so that the bracket keeps the root.
        float zn2 = 0.f, sd2 = 0.f, sdz = 0.f, sdza = 0.f;
        if (top)
            for (int j = sub; j < K; j += G) {
                const float2 p = dz[j];
                zn2 += p.y;
                sd2 = fmaf(p.x, p.x, sd2);
                sdz = fmaf(p.x, p.y, sdz);
                sdza = fmaf(fabsf(p.x), p.y, sdza);
            }
        zn2 = gsum<G>(zn2);
        sd2 = gsum<G>(sd2);
        sdz = gsum<G>(sdz);
        sdza = gsum<G>(sdza);
        if (top) {
            U = rho * zn2 * (1.f + 2.f * (K + 2) * kU);
            const float rz = rho * zn2;
            const float fro2 = fmaf(rz, rz, fmaf(2.f * rho, sdz, sd2));
            const float err2 = 4.f * (K + 4) * kU * fmaf(rz, rz, fmaf(2.f * rho, sdza, sd2));
            const float fro = sqrt_approx(fmaxf(fro2 + err2, 0.f));  // 2^-23: inside the 4u margin below
            const float dtop = dz[K - 1].x;
            const float uf = (fro - dtop) + 4.f * kU * (fro + fabsf(dtop));
            if (uf > 0.f && uf < U) U = uf;
            if (K == 1) {  // one pole: 1 + rho z^2/(d - lambda) = 0 has lambda = d + rho z^2
                r.tau = rho * dz[0].y;
                r.conv = true;
                done = true;
            }
        } else if (part) {
            U = dz[q + 1].x - dz[q].x;
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
        if (kp.retire && !__any_sync(kFull, !done)) break;  // progressive shrinkage (Eq. (22))
        // Eq. (8) at lambda = d[o] + h, with d_j - lambda = (d_j - d_o) - h; the sectioning steps need
        // only the sign of f, Halley's steps also f' (Eq. (18)), f'' (Eq. (21)) and the error scale
        const bool deriv = __any_sync(kFull, !done && state == 2);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, sa = 0.f;
        if (!done) {
            const float dorg = dz[o].x;
            // four poles per pass (their loads and reciprocals in flight together), accumulated in two
            // independent partial sums, two passes unrolled so that the next pass's loads and
            // reciprocals overlap this one's sums; then one pole at a time for the remainder
            if (deriv) {
                float s0b = 0.f, s1b = 0.f, s2b = 0.f, sab = 0.f;
                int j = sub;
#pragma unroll 2
                for (; j + 3 * G < K; j += 4 * G) {
                    const float2 pa = dz[j], pb = dz[j + G], pc = dz[j + 2 * G], pd = dz[j + 3 * G];
                    const float ia = rcp_approx((pa.x - dorg) - h), ib = rcp_approx((pb.x - dorg) - h);
                    const float ic = rcp_approx((pc.x - dorg) - h), id = rcp_approx((pd.x - dorg) - h);
                    const float ta = pa.y * ia, tb = pb.y * ib, tc = pc.y * ic, td = pd.y * id;
                    const float tia = ta * ia, tib = tb * ib, tic = tc * ic, tid = td * id;
                    s0 += ta + tc;
                    s0b += tb + td;
                    s1 += tia + tic;
                    s1b += tib + tid;
                    s2 = fmaf(tia, ia, fmaf(tic, ic, s2));
                    s2b = fmaf(tib, ib, fmaf(tid, id, s2b));
                    sa += fabsf(ta) + fabsf(tc);
                    sab += fabsf(tb) + fabsf(td);
                }
                for (; j < K; j += G) {
                    const float2 pa = dz[j];
                    const float ia = rcp_approx((pa.x - dorg) - h);
                    const float ta = pa.y * ia;
                    const float tia = ta * ia;
                    s0 += ta;
                    s1 += tia;
                    s2 = fmaf(tia, ia, s2);
                    sa += fabsf(ta);
                }
                s0 += s0b;
                s1 += s1b;
                s2 += s2b;
                sa += sab;
            } else {
                float s0b = 0.f, s0c = 0.f, s0d = 0.f;
                int j = sub;
#pragma unroll 2
                for (; j + 3 * G < K; j += 4 * G) {
                    const float2 pa = dz[j], pb = dz[j + G], pc = dz[j + 2 * G], pd = dz[j + 3 * G];
                    s0 = fmaf(pa.y, rcp_approx((pa.x - dorg) - h), s0);
                    s0b = fmaf(pb.y, rcp_approx((pb.x - dorg) - h), s0b);
                    s0c = fmaf(pc.y, rcp_approx((pc.x - dorg) - h), s0c);
                    s0d = fmaf(pd.y, rcp_approx((pd.x - dorg) - h), s0d);
                }
                for (; j < K; j += G) {
                    const float2 pa = dz[j];
                    s0 = fmaf(pa.y, rcp_approx((pa.x - dorg) - h), s0);
                }
                s0 = (s0 + s0b) + (s0c + s0d);
            }
        }
        s0 = gsum<G>(s0);
        if (deriv) {
            s1 = gsum<G>(s1);
            s2 = gsum<G>(s2);
            sa = gsum<G>(sa);
        }
        if (done) continue;
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
            float hev = h;  // the point just evaluated, relative to the current origin
            if (state == 0) {
                if (!done && !top && f < 0.f) {
                    // root in the upper half of (d_q, d_{q+1}): measure it from d_{q+1}
                    const float sh = dz[q + 1].x - dz[q].x;
                    o = q + 1;
                    L -= sh;
                    U = 0.f;
                    hev = h - sh;
                }
                state = 1;
            } else {
                ++nsec;
            }
            if (!done) {
                if ((U - L) < kp.sec_eps * width0 || nsec >= kp.max_sec) {
                    // Halley starts from the root of the one-pole model of f at the last point (the
                    // same model as its fallback below) when that lies in the bracket, else the midpoint
                    state = 2;
                    float hn = 0.5f * (L + U);
                    if (hev != 0.f) {
                        const float rz = rho * dz[o].y;
                        const float g = f + rz / hev;
                        if (g != 0.f) {
                            const float he = rz / g;
                            if ((he > L) && (top ? he <= U : he < U)) hn = he;
                        }
                    }
                    h = hn;
                } else {
                    // Eq. (16); the first n_bisect - 1 of these steps bisect (Eq. (13)-(15))
                    h = fmaf(U - L, (nsec + 1 < kp.n_bisect) ? 0.5f : kinv, L);
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
                    float hn = h - (2.f * f * f1) * rcp_approx(den);  // Eq. (20)
                    const bool inside = (hn > L) && (top ? hn <= U : hn < U);
                    if (!(den > 0.f) || !inside) {
                        // Halley's step left the bracket: far from a root that hugs its pole d_o, f is
                        // nearly flat. Write f = rho z_o^2 / (d_o - lambda) + g with the rest g taken
                        // constant at its value here; the root of that model, h = rho z_o^2 / g, is the
                        // next iterate when it lies inside the bracket, else the midpoint.
                        hn = 0.5f * (L + U);
                        if (h != 0.f) {
                            const float rz = rho * dz[o].y;
                            const float g = f + rz / h;
                            if (g != 0.f) {
                                const float he = rz / g;
                                if ((he > L) && (top ? he <= U : he < U)) hn = he;
                            }
                        }
                    }
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
// Tensor-core variant of the merge product (a7): split-3xTF32 on mma.sync m16n8k8. Each FP32 operand
// x is split as x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact), and a product
// is accumulated in FP32 as hi*hi + hi*lo + lo*hi, which keeps about 21 bits of each operand.
// Fragment layout (PTX ISA, mma.m16n8k8 with .tf32; gid = lane / 4, tig = lane % 4):
//   A (16 x 8, row):  a0 (gid, tig), a1 (gid + 8, tig), a2 (gid, tig + 4), a3 (gid + 8, tig + 4)
//   B (8 x 8, col):   b0 (k = tig, n = gid), b1 (k = tig + 4, n = gid)
//   C (16 x 8, f32):  c0 (gid, 2 tig), c1 (gid, 2 tig + 1), c2 (gid + 8, 2 tig), c3 (gid + 8, 2 tig + 1)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_16x8x8(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Tiles of 16 rows x 8 columns of one merge level's products: per merge, the row tiles of the left
// half, then of the right half, each with all column tiles of the merge.
__device__ __forceinline__ int tc_level_tiles(const Plan& plan, int L)
{
    int t = 0;
    for (int m = plan.level_start[L]; m < plan.level_start[L + 1]; ++m) {
        const int lo = plan.m_lo[m], md = plan.m_mid[m], hi = plan.m_hi[m];
        t += ((md - lo + 15) / 16 + (hi - md + 15) / 16) * ((hi - lo + 7) / 8);
    }
    return t;
}

// ---------------------------------------------------------------------------------------------
// One matrix, solved by a team of NMAX * G threads (tid = index within the team) that synchronizes
// on named barrier bar_id. `bar` is the team's mbarrier (initialized by the caller) and `phase` its
// current phase bit. Returns false only when the staging copy timed out (the caller then stops).
// ---------------------------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void team_sync(int bar_id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "n"(NT) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// a7 on the FP32 FMA pipes. Register tiles: the rows of one half of a merge times its columns form a
// small product over the half's columns c. The level's tiles (PR rows x PC columns, merges in order, the
// left half's tiles, then the right half's, each half column tile by column tile) are dealt one per thread;
// per c a thread reads PR entries of Q, one row of Q^ (PC entries) and does PR x PC FMAs. The products
// are scaled by the reciprocal column norms of Q^ when stored (after the team barrier: Q is read by all).
template <int NMAX, int G>
__device__ __forceinline__ void merge_product_fma(Smem<NMAX, G>& S, const Plan& plan, int L, int tid, int bar_id)
{
    constexpr int NT = NMAX * G;
    constexpr int LD = Smem<NMAX, G>::LD;
    constexpr int PR = 4;
    constexpr int PC = 16 / G;
    int r0 = 0, rend = 0, c0 = 0, c1 = 0, q0 = 0, qend = 0;
    bool have = false;
    {
        int tbase = 0;
        for (int m = plan.level_start[L]; m < plan.level_start[L + 1]; ++m) {
            const int lo = plan.m_lo[m], md = plan.m_mid[m], hi = plan.m_hi[m];
            const int rtl = (md - lo + PR - 1) / PR, rtr = (hi - md + PR - 1) / PR;
            const int ctn = (hi - lo + PC - 1) / PC;
            const int cnt = (rtl + rtr) * ctn;
            if (tid >= tbase && tid < tbase + cnt) {
                // a half's tiles are dealt down its row tiles first: the lanes of a warp then span
                // more row tiles and fewer column tiles, so that a warp's reads of one row of Q^ fall in
                // distinct banks
                const int u = tid - tbase;
                const bool left = u < rtl * ctn;
                const int uh = left ? u : u - rtl * ctn;
                const int rth = left ? rtl : rtr;
                const int ct = uh / rth, rr = uh - ct * rth;
                r0 = left ? lo + PR * rr : md + PR * rr;
                rend = left ? md : hi;
                c0 = left ? lo : md;
                c1 = left ? md : hi;
                q0 = lo + PC * ct;
                qend = hi;
                have = true;
            }
            tbase += cnt;
        }
    }
    float acc[PR][PC];
#pragma unroll
    for (int i = 0; i < PR; ++i)
#pragma unroll
        for (int j = 0; j < PC; ++j) acc[i][j] = 0.f;
    if (have) {
        // rows past rend and columns past qend read padding or neighbouring entries; their
        // sums are never stored
        const float* qrow = S.Q + r0 * LD;
#pragma unroll 2
        for (int c = c0; c < c1; ++c) {
            const float* mrow = S.M + c * LD + q0;
            float mv[PC];
#pragma unroll
            for (int j = 0; j < PC; ++j) mv[j] = mrow[j];
#pragma unroll
            for (int i = 0; i < PR; ++i) {
                const float qv = qrow[i * LD + c];
#pragma unroll
                for (int j = 0; j < PC; ++j) acc[i][j] = fmaf(qv, mv[j], acc[i][j]);
            }
        }
    }
    team_sync<NT>(bar_id);
    if (have) {
#pragma unroll
        for (int i = 0; i < PR; ++i)
#pragma unroll
            for (int j = 0; j < PC; ++j)
                if (r0 + i < rend && q0 + j < qend) S.Q[(r0 + i) * LD + q0 + j] = acc[i][j] * S.cinv[q0 + j];
    }
}

// a7 on the tensor cores (split-3xTF32, see above): tiles of 16 rows x 8 columns in the order of
// tc_level_tiles; warp w computes tiles w, w + NW, ... (at most TPW) in registers, then, after the team
// barrier, stores them scaled by the reciprocal column norms of Q^.
template <int NMAX, int G, int TPW>
__device__ __forceinline__ void merge_product_tc(Smem<NMAX, G>& S, const Plan& plan, int L, int tid, int bar_id)
{
    constexpr int NT = NMAX * G;
    constexpr int NW = NT / 32;
    constexpr int LD = Smem<NMAX, G>::LD;
    const int lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    // tile t of this level: rows [r0, rend), columns from q0 (below qend), inner index over [c0, c1)
    auto tile = [&](int t, int& r0, int& rend, int& c0, int& c1, int& q0, int& qend) {
        r0 = rend = c0 = c1 = q0 = qend = 0;
        int tbase = 0;
        for (int m = plan.level_start[L]; m < plan.level_start[L + 1]; ++m) {
            const int lo = plan.m_lo[m], md = plan.m_mid[m], hi = plan.m_hi[m];
            const int rtl = (md - lo + 15) / 16, rtr = (hi - md + 15) / 16, ctn = (hi - lo + 7) / 8;
            const int cnt = (rtl + rtr) * ctn;
            if (t >= tbase && t < tbase + cnt) {
                const int u = t - tbase;
                const int rr = u / ctn, ct = u - rr * ctn;
                const bool left = rr < rtl;
                r0 = left ? lo + 16 * rr : md + 16 * (rr - rtl);
                rend = left ? md : hi;
                c0 = left ? lo : md;
                c1 = left ? md : hi;
                q0 = lo + 8 * ct;
                qend = hi;
            }
            tbase += cnt;
        }
    };
    float acc[TPW][4];
#pragma unroll
    for (int j = 0; j < TPW; ++j) {
        acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
        int r0, rend, c0, c1, q0, qend;
        tile(warp + j * NW, r0, rend, c0, c1, q0, qend);  // past the last tile: c0 == c1, nothing to do
        const int ra = r0 + gid, rb = ra + 8, nq = q0 + gid;
        for (int kc = c0; kc < c1; kc += 8) {
            const int ka = kc + tig, kb = ka + 4;
            const float x0 = (ra < rend && ka < c1) ? S.Q[ra * LD + ka] : 0.f;
            const float x1 = (rb < rend && ka < c1) ? S.Q[rb * LD + ka] : 0.f;
            const float x2 = (ra < rend && kb < c1) ? S.Q[ra * LD + kb] : 0.f;
            const float x3 = (rb < rend && kb < c1) ? S.Q[rb * LD + kb] : 0.f;
            const float y0 = (ka < c1 && nq < qend) ? S.M[ka * LD + nq] : 0.f;
            const float y1 = (kb < c1 && nq < qend) ? S.M[kb * LD + nq] : 0.f;
            uint32_t ah[4], al[4], bh[2], bl[2];
            split_tf32(x0, ah[0], al[0]);
            split_tf32(x1, ah[1], al[1]);
            split_tf32(x2, ah[2], al[2]);
            split_tf32(x3, ah[3], al[3]);
            split_tf32(y0, bh[0], bl[0]);
            split_tf32(y1, bh[1], bl[1]);
            mma_tf32_16x8x8(acc[j], al, bh);
            mma_tf32_16x8x8(acc[j], ah, bl);
            mma_tf32_16x8x8(acc[j], ah, bh);
        }
    }
    team_sync<NT>(bar_id);
#pragma unroll
    for (int j = 0; j < TPW; ++j) {
        int r0, rend, c0, c1, q0, qend;
        tile(warp + j * NW, r0, rend, c0, c1, q0, qend);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = r0 + gid + ((e & 2) ? 8 : 0), q = q0 + 2 * tig + (e & 1);
            if (r < rend && q < qend) S.Q[r * LD + q] = acc[j][e] * S.cinv[q];
        }
    }
}

// ---------------------------------------------------------------------------------------------
// a1 in phases of 16 steps. Rows below step k are finished, so phase p (steps 16 p .. 16 p + 15) keeps
// only rows 16 p .. NMAX - 1 of its warp's columns in registers: TRP = (NMAX - 16 p) / 16 rows per lane,
// rows r0 + TRP tr + [0, TRP) with r0 = 16 p. Between phases a warp moves its tile to the smaller shape
// through the staging area (free during a1), so every later step updates and sums fewer rows.
// ---------------------------------------------------------------------------------------------
template <int NMAX, int G>
__host__ __device__ constexpr int a1_tile_cols()
{
    return (NMAX / (NMAX * G / 32)) / a1_col_lanes<NMAX, G>();
}

// steps k0 .. k1 - 1 with the rows r0 .. NMAX - 1 in registers
template <int NMAX, int G, int TRP>
__device__ __forceinline__ void a1_steps(Smem<NMAX, G>& S, float (&a)[TRP][a1_tile_cols<NMAX, G>()], int r0,
                                         int k0, int k1, int n, float& tau_prev, int tid, int bar_id)
{
    constexpr int NT = NMAX * G;
    constexpr int NW = NT / 32;
    constexpr int WC = NMAX / NW;
    constexpr int NTC = a1_col_lanes<NMAX, G>();
    constexpr int TC = a1_tile_cols<NMAX, G>();
    constexpr int LOG_TC = ilog2(TC);
    constexpr int LOG_NTC = ilog2(NTC);
    const int lane = tid & 31, warp = tid >> 5;
    const int tr = lane / NTC, tc = lane % NTC;
    const int i0 = r0 + tr * TRP, j0 = warp * WC + tc * TC;
    const int wlast = (n - 1) / WC;  // owns column n - 1: active in every step; stores reflectors
    for (int k = k0; k < k1; ++k) {
        const float* Pr = S.hp[(k + 1) & 1];
        const float* Ur = S.hu[(k + 1) & 1];
        const float* Yr = S.hy[(k + 1) & 1];
        float tau = 0.f;
        if (warp * WC + WC > k + 1 && warp <= wlast) {
            // the three vectors on this lane's rows; every warp holds all rows from r0, so sums over
            // rows are sums over the 16 row lanes (the two column lanes of a row agree). v_{k-1} is
            // zero on the rows below r0 <= k, which therefore add nothing to p.v
            float pr[TRP], ur[TRP], yr[TRP];
            load_vec<TRP>(Pr + i0, pr);
            load_vec<TRP>(Ur + i0, ur);
            load_vec<TRP>(Yr + i0, yr);
            float dot = 0.f;
#pragma unroll
            for (int ii = 0; ii < TRP; ++ii) dot = fmaf(pr[ii], ur[ii], dot);
            const float c = 0.5f * tau_prev * row_lane_sum<NTC>(dot);  // (tau/2) p.v of step k - 1
            const float uk = Ur[k];
            const float wk = fmaf(-c, uk, Pr[k]);
            if (warp == wlast && lane == 0) S.d[k] = fmaf(-2.f * uk, wk, Yr[k]);
            // w of step k - 1 and x = column k of the updated matrix. v_{k-1} is zero on the
            // finished rows i < k, so the update below leaves the active block exact without
            // masking; the finished rows and columns pick up bounded values that no later step
            // reads (the column sums and x are taken against v_k, zero there). Rows >= n stay zero.
            float wr[TRP], xr[TRP];
            float part = 0.f;
#pragma unroll
            for (int ii = 0; ii < TRP; ++ii) {
                const int i = i0 + ii;
                wr[ii] = fmaf(-c, ur[ii], pr[ii]);
                xr[ii] = fmaf(-wr[ii], uk, fmaf(-ur[ii], wk, yr[ii]));
                if (i > k + 1) part = fmaf(xr[ii], xr[ii], part);
            }
            // the update of step k - 1 needs only c: apply it to the tile (rows and columns >= k)
            // while the reduction for reflector k is in flight
            float pc[TC], uc[TC];
            load_vec<TC>(Pr + j0, pc);
            load_vec<TC>(Ur + j0, uc);
#pragma unroll
            for (int jj = 0; jj < TC; ++jj) {
                const float u = uc[jj];
                const float w = fmaf(-c, u, pc[jj]);
#pragma unroll
                for (int ii = 0; ii < TRP; ++ii) a[ii][jj] = fmaf(-ur[ii], w, fmaf(-wr[ii], u, a[ii][jj]));
            }
            // column k + 1 of the updated matrix, for step k + 1
            if (warp == (k + 1) / WC && tc == ((k + 1) % WC) / TC) {
                const int kj = (k + 1) % TC;
                float yk[TRP];
#pragma unroll
                for (int ii = 0; ii < TRP; ++ii) {
                    float x = 0.f;
#pragma unroll
                    for (int jj = 0; jj < TC; ++jj) x = (jj == kj) ? a[ii][jj] : x;
                    yk[ii] = x;
                }
                store_vec<TRP>(S.hy[k & 1] + i0, yk);
            }
            const float xn2 = row_lane_sum<NTC>(part);
            const float u1 = Ur[k + 1];
            const float alpha = fmaf(-fmaf(-c, u1, Pr[k + 1]), uk, fmaf(-u1, wk, Yr[k + 1]));
            // reflector k; when x is already zero below its first entry, tau = 0 and beta = alpha.
            // |beta| = nrm and |alpha - beta| >= nrm: both normal, far from overflow
            const float nrm = sqrt_approx(fmaf(alpha, alpha, xn2));
            const bool refl = xn2 > 0.f;
            const float beta = refl ? ((alpha >= 0.f) ? -nrm : nrm) : alpha;
            tau = refl ? (beta - alpha) * rcp_approx(beta) : 0.f;
            const float scal = refl ? rcp_approx(alpha - beta) : 0.f;
            float vr[TRP];
#pragma unroll
            for (int ii = 0; ii < TRP; ++ii) {
                const int i = i0 + ii;
                vr[ii] = (i > k + 1) ? xr[ii] * scal : ((i == k + 1) ? 1.f : 0.f);
            }
            // reflector k: for the next step and, transposed, for the back-transform (its rows
            // below r0 are zero and stay as a1 cleared them)
            if (warp == wlast && tc == 0) {
                store_vec<TRP>(S.hu[k & 1] + i0, vr);
#pragma unroll
                for (int ii = 0; ii < TRP; ++ii) S.A[yt_index<NMAX>(i0 + ii, k)] = vr[ii];
                if (lane == 0) {
                    S.e[k] = beta;
                    S.tau[k] = tau;
                }
            }
            // column sums of the updated tile with v_k
            float s[TC];
#pragma unroll
            for (int jj = 0; jj < TC; ++jj) {
                float acc = 0.f;
#pragma unroll
                for (int ii = 0; ii < TRP; ++ii) acc = fmaf(a[ii][jj], vr[ii], acc);
                s[jj] = acc;
            }
            // sum over the row lanes: halving exchanges leave the lowest LOG_TC row-lane bits
            // holding one column each, plain butterflies finish the sum
            int cb = 0;
#pragma unroll
            for (int l = 0; l < LOG_TC; ++l) {
                const int h = TC >> (l + 1);
                const int o = NTC << l;
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int t = 0; t < h; ++t) {
                    const float send = up ? s[t] : s[t + h];
                    const float keep = up ? s[t + h] : s[t];
                    s[t] = keep + __shfl_xor_sync(kFull, send, o);
                }
                if (up) cb += h;
            }
#pragma unroll
            for (int o = NTC << LOG_TC; o < 32; o <<= 1) s[0] += __shfl_xor_sync(kFull, s[0], o);
            float* Pw = S.hp[k & 1];
            if ((lane >> (LOG_NTC + LOG_TC)) == 0) Pw[j0 + cb] = tau * s[0];
        }
        tau_prev = tau;
        team_sync<NT>(bar_id);
    }
}

// the trailing 2 x 2 block after the last update (the whole matrix when n <= 2), from the tile of the
// last phase (rows r0 .. NMAX - 1, r0 <= n - 2)
template <int NMAX, int G, int TRP>
__device__ __forceinline__ void a1_last(Smem<NMAX, G>& S, const float (&a)[TRP][a1_tile_cols<NMAX, G>()],
                                        int r0, int n, float tau_prev, int tid)
{
    constexpr int NW = NMAX * G / 32;
    constexpr int WC = NMAX / NW;
    constexpr int NTC = a1_col_lanes<NMAX, G>();
    constexpr int TC = a1_tile_cols<NMAX, G>();
    const int lane = tid & 31, warp = tid >> 5;
    const int tr = lane / NTC, tc = lane % NTC;
    const int i0 = r0 + tr * TRP, j0 = warp * WC + tc * TC;
    const int wlast = (n - 1) / WC;
    const int kf = n - 2;
    if (n >= 2 && warp * WC + WC > kf && warp <= wlast) {
        const float* Pr = S.hp[(kf + 1) & 1];
        const float* Ur = S.hu[(kf + 1) & 1];
        float dot = 0.f;
#pragma unroll
        for (int ii = 0; ii < TRP; ++ii) dot = fmaf(Pr[i0 + ii], Ur[i0 + ii], dot);
        const float c = 0.5f * tau_prev * row_lane_sum<NTC>(dot);
#pragma unroll
        for (int ii = 0; ii < TRP; ++ii)
#pragma unroll
            for (int jj = 0; jj < TC; ++jj) {
                const int i = i0 + ii, j = j0 + jj;
                if (i >= kf && j >= kf && i < n && j < n && j <= i) {
                    const float ui = Ur[i], uj = Ur[j];
                    const float wi = fmaf(-c, ui, Pr[i]), wj = fmaf(-c, uj, Pr[j]);
                    const float x = fmaf(-ui, wj, fmaf(-wi, uj, a[ii][jj]));
                    if (i == j) S.d[i] = x;
                    else S.e[kf] = x;
                }
            }
    } else if (n == 1 && tid == 0) {
        S.d[0] = a[0][0];
    }
}

// phase r0 / 16 and the ones after it
template <int NMAX, int G, int TRP>
__device__ __forceinline__ void a1_run(Smem<NMAX, G>& S, float (&a)[TRP][a1_tile_cols<NMAX, G>()], int r0, int n,
                                       float& tau_prev, int tid, int bar_id)
{
    constexpr int NW = NMAX * G / 32;
    constexpr int WC = NMAX / NW;
    constexpr int NTC = a1_col_lanes<NMAX, G>();
    constexpr int TC = a1_tile_cols<NMAX, G>();
    constexpr int LD = Smem<NMAX, G>::LD;
    const int ks = n - 2;  // steps k = 0 .. n - 3
    if constexpr (TRP > 1) {
        if (ks > r0 + 16) {
            a1_steps<NMAX, G, TRP>(S, a, r0, r0, r0 + 16, n, tau_prev, tid, bar_id);
            // rows r0 + 16 .. of this warp's columns to the next phase's layout, through the staging
            // area (each warp moves only its own columns)
            const int lane = tid & 31, warp = tid >> 5;
            const int tr = lane / NTC, tc = lane % NTC;
            const int j0 = warp * WC + tc * TC;
#pragma unroll
            for (int ii = 0; ii < TRP; ++ii) {
                const int i = r0 + tr * TRP + ii;
                if (i >= r0 + 16)
#pragma unroll
                    for (int jj = 0; jj < TC; ++jj) S.M[i * LD + j0 + jj] = a[ii][jj];
            }
            __syncwarp();
            float b[TRP - 1][TC];
#pragma unroll
            for (int ii = 0; ii < TRP - 1; ++ii) {
                const int i = r0 + 16 + tr * (TRP - 1) + ii;
#pragma unroll
                for (int jj = 0; jj < TC; ++jj) b[ii][jj] = S.M[i * LD + j0 + jj];
            }
            a1_run<NMAX, G, TRP - 1>(S, b, r0 + 16, n, tau_prev, tid, bar_id);
            return;
        }
    }
    a1_steps<NMAX, G, TRP>(S, a, r0, r0, ks, n, tau_prev, tid, bar_id);
    a1_last<NMAX, G, TRP>(S, a, r0, n, tau_prev, tid);
}

template <int NMAX, int G, bool TC = false>
__device__ __forceinline__ bool solve_matrix(Smem<NMAX, G>& S, const Plan& plan, const KParams& kp, const int tid,
                                             const int bar_id, const uint32_t bar, uint32_t& phase,
                                             const float* __restrict__ Ab, float* __restrict__ Wb,
                                             float* __restrict__ Vb, int32_t* __restrict__ info_b,
                                             bed_counters* __restrict__ counters, const bool bulk)
{
    constexpr int NT = NMAX * G;
    constexpr int NW = NT / 32;
    constexpr int LD = Smem<NMAX, G>::LD;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int pos = tid / G;
    const int sub = tid % G;
    const int n = plan.n;

    // ---------------- a0: stage the matrix -------------------------------------------------
    if (bulk) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        S.info = 0;
        S.evals = 0;
        S.roots = 0;
        S.deflated = 0;
    }
    team_sync<NT>(bar_id);
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
        if (!mbar_wait_bounded(bar, phase, kp.stage_wait_ns)) {
            timed_out = true;
            // wait once more, again bounded, for the copy still in flight: once it has landed the
            // mbarrier phase is known again and the team can go on with its next matrix
            if (!mbar_wait_bounded(bar, phase, kDrainWaitNs)) atomicOr(&S.info, kInfoUndrained);
        }
        phase ^= 1u;
    } else {
        // all loads of a thread in flight at once: the source may be host memory across the link
        constexpr int PER = NMAX / G;  // NMAX^2 / NT
        float r[PER];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int i = tid + t * NT;
            r[t] = (i < n * n) ? Ab[i] : 0.f;
        }
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int i = tid + t * NT;
            if (i < n * n) S.M[i] = r[t];
        }
    }
    if (timed_out) atomicOr(&S.info, BED_INFO_TIMEOUT);
    team_sync<NT>(bar_id);

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
    team_sync<NT>(bar_id);
    if (S.info & (BED_INFO_NONFINITE | BED_INFO_TIMEOUT)) {
        const float qnan = __int_as_float(0x7fc00000);
        for (int i = tid; i < n; i += NT) Wb[i] = qnan;
        for (int i = tid; i < n * n; i += NT) Vb[i] = qnan;
        if (info_b && tid == 0) *info_b = S.info & ~kInfoUndrained;
        const bool stop = (S.info & kInfoUndrained) != 0;
        team_sync<NT>(bar_id);
        return !stop;  // a copy still in flight: the mbarrier phase is no longer known, the caller stops
    }
    amax = S.red[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) amax = fmaxf(amax, S.red[w]);
    // exact power-of-two scaling to max|a| in [0.5, 1): norms below cannot overflow or underflow
    int ex = 0;
    if (amax > 0.f) frexpf(amax, &ex);
    const float scale = ldexpf(1.f, -ex);
    if (tid == 0) {
        S.unscale = ldexpf(1.f, ex);
        S.out_w = Wb;
        S.out_v = Vb;
        S.out_info = info_b;
    }

    // ---------------- a1: Householder tridiagonalization ------------------------------------
    // Column-owned register tiles, one barrier per reflector. Warp w keeps columns
    // [w WC, (w + 1) WC) of A in registers: lane (tr, tc) = (lane / NTC, lane % NTC) holds rows
    // [TR tr, TR tr + TR) of columns w WC + TC tc + [0, TC). A is symmetric, so the column sums of a
    // warp's block are the entries of A v at its columns: p = tau A22 v needs shuffles inside the warp
    // only. Step k reads three vectors that step k-1 left in shared memory (double-buffered by step
    // parity): p_{k-1}, v_{k-1} and column k of A before the update of step k-1. From them every warp
    // forms, redundantly and identically, w_{k-1} = p - (tau/2)(p.v) v, column k of the updated matrix
    // and reflector k (each warp holds every row, so the sums over rows are shuffle sums over its row
    // lanes); it applies A22 -= v w^T + w v^T of step k-1 to its tile and forms the column sums with
    // v_k. A warp whose columns are all finished skips the step. The steps run in phases of 16 (a1_run):
    // rows below the phase's first step are finished, so each phase keeps 16 rows fewer per column
    // (the tile starts with all NMAX rows, TR per lane).
    {
        constexpr int WC = NMAX / NW;             // columns per warp
        constexpr int NTC = a1_col_lanes<NMAX, G>();  // lanes along the columns
        constexpr int NTR = 32 / NTC;             // lanes along the rows
        constexpr int TCOL = WC / NTC;            // tile columns per lane
        constexpr int TR = NMAX / NTR;            // tile rows per lane
        constexpr int LOG_TCOL = ilog2(TCOL);
        constexpr int LOG_NTC = ilog2(NTC);
        static_assert(WC * NW == NMAX && TR * NTR == NMAX && TCOL * NTC == WC && (1 << LOG_TCOL) == TCOL &&
                          (1 << LOG_NTC) == NTC && NTR == 16 && TCOL == a1_tile_cols<NMAX, G>(),
                      "tile shape");
        const int tr = lane / NTC, tc = lane % NTC;
        const int i0 = tr * TR, j0 = warp * WC + tc * TCOL;
        float a[TR][TCOL];
        // the tile comes straight from the staged input (row-major n x n, lower triangle read), scaled
#pragma unroll
        for (int ii = 0; ii < TR; ++ii)
#pragma unroll
            for (int jj = 0; jj < TCOL; ++jj) {
                const int i = i0 + ii, j = j0 + jj;
                a[ii][jj] = (i < n && j < n) ? S.M[(j <= i) ? (i * n + j) : (j * n + i)] * scale : 0.f;
            }
        // step 0 reads buffer 1: p = v = 0 and column 0 of A
        for (int i = tid; i < NMAX; i += NT) {
            S.hp[0][i] = 0.f;
            S.hu[0][i] = 0.f;
            S.hy[0][i] = 0.f;
            S.hp[1][i] = 0.f;
            S.hu[1][i] = 0.f;
            S.hy[1][i] = (i < n) ? S.M[i * n] * scale : 0.f;
        }
        // the reflectors' rows above each phase are not stored by the steps: they start out zero
        for (int i = tid; i < NMAX * NMAX / 4; i += NT)
            reinterpret_cast<float4*>(S.A)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        team_sync<NT>(bar_id);  // every tile is loaded before the merge phases reuse the staging area
        float tau_prev = 0.f;
        a1_run<NMAX, G, TR>(S, a, 0, n, tau_prev, tid, bar_id);
        // reflector columns n - 2 .. of the last back-transform block are zero
        for (int idx = tid; idx < NMAX * kBT; idx += NT) {
            const int i = idx / kBT, kk = n - 2 + idx % kBT;
            if (n >= 3 && kk < NMAX) S.A[yt_index<NMAX>(i, kk)] = 0.f;
        }
        team_sync<NT>(bar_id);
    }

    // ---------------- a2: tear (Eq. (3)) ----------------------------------------------------
    if (tid < n) {
        float dt = S.d[tid];
        if ((plan.cut_mask >> tid) & 1ull) dt -= fabsf(S.e[tid]);
        if (tid > 0 && ((plan.cut_mask >> (tid - 1)) & 1ull)) dt -= fabsf(S.e[tid - 1]);
        S.d[tid] = dt;
    }
    team_sync<NT>(bar_id);

    // ---------------- a3: leaves ------------------------------------------------------------
    // a leaf of m >= 3 rows is solved by a group of lanes (one per row of its eigenvector block) with
    // LM register slots: LM = 4 when every leaf of the tree has at most 4 rows, 6 for at most 6, else 8
    if (plan.max_leaf <= 4) {
        for (int lf = tid >> 2; lf < plan.nleaves; lf += NT >> 2) {
            const int lo = plan.leaf_lo[lf], m = plan.leaf_hi[lf] - lo;
            if (m >= 3) {
                const int r = tid & 3;
                const bool ok =
                    ql_leaf<4>(&S.d[lo], &S.e[lo], m, r, &S.lam[lo], &S.Q[(lo + min(r, m - 1)) * LD + lo]);
                if (!ok && r == 0) atomicOr(&S.info, BED_INFO_NOT_CONVERGED);
            }
        }
    } else if (plan.max_leaf <= 6) {
        for (int lf = tid >> 3; lf < plan.nleaves; lf += NT >> 3) {
            const int lo = plan.leaf_lo[lf], m = plan.leaf_hi[lf] - lo;
            if (m >= 3) {
                const int r = tid & 7;
                const bool ok =
                    ql_leaf<6>(&S.d[lo], &S.e[lo], m, r, &S.lam[lo], &S.Q[(lo + min(r, m - 1)) * LD + lo]);
                if (!ok && r == 0) atomicOr(&S.info, BED_INFO_NOT_CONVERGED);
            }
        }
    } else {
        for (int lf = tid >> 3; lf < plan.nleaves; lf += NT >> 3) {
            const int lo = plan.leaf_lo[lf], m = plan.leaf_hi[lf] - lo;
            if (m >= 3) {
                const int r = tid & 7;
                const bool ok =
                    ql_leaf<8>(&S.d[lo], &S.e[lo], m, r, &S.lam[lo], &S.Q[(lo + min(r, m - 1)) * LD + lo]);
                if (!ok && r == 0) atomicOr(&S.info, BED_INFO_NOT_CONVERGED);
            }
        }
    }
    if (tid < plan.nleaves && plan.leaf_hi[tid] - plan.leaf_lo[tid] <= 2) {
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
    team_sync<NT>(bar_id);

    // ---------------- a4-a7: merges, deepest level first -----------------------------------
    for (int L = 0; L < plan.nlevels; ++L) {
        const int l0 = plan.level_start[L];
        // position layout: this group's row/column/root t = pos belongs to merge bi
        const int bi = (pos < n) ? plan.blk[L][pos] : 0xFF;
        const bool act = (bi != 0xFF);
        const int lb = bi - l0;  // merge index within the level
        int lo = 0, mid = 0, hi = 0;
        if (act) {
            lo = plan.m_lo[bi];
            mid = plan.m_mid[bi];
            hi = plan.m_hi[bi];
        }
        // P1: z (Eq. (5)), pole order, block scalars, negligible couplings. Every group of the merge
        // forms the block scalars from the same sums in the same order, so all agree exactly
        {
            const int c = pos;
            float zc = 0.f, kc = 0.f;
            int p = 0;
            float nz2 = 0.f, dmax = 0.f;
            if (act) {
                const float sig = (S.e[mid - 1] >= 0.f) ? 1.f : -1.f;
                const float* z1 = &S.Q[(mid - 1) * LD];  // last row of Q1
                const float* z2 = &S.Q[mid * LD];        // first row of Q2
                zc = (c < mid) ? sig * z1[c] : z2[c];
                kc = sort_key(S.lam[c]);
#pragma unroll 4
                for (int c2 = lo + sub; c2 < hi; c2 += G) {
                    const float l2 = S.lam[c2];
                    const float k2 = sort_key(l2);
                    p += (k2 < kc) || (k2 == kc && c2 < c);
                    const float zz = (c2 < mid) ? z1[c2] : z2[c2];
                    nz2 = fmaf(zz, zz, nz2);
                    dmax = fmaxf(dmax, fabsf(l2));
                }
            }
            p = gsumi<G>(p);
            nz2 = gsum<G>(nz2);
            dmax = gmax<G>(dmax);
            if (act && sub == 0) {
                const float rho = fabsf(S.e[mid - 1]);
                const float bscale = fmaxf(dmax, rho * nz2);
                const float nz = sqrt_approx(nz2);
                const float tol = kp.defl_c * kU * bscale;
                S.colof[lo + p] = c;
                S.ds[lo + p] = S.lam[c];
                S.zs[lo + p] = zc;
                S.defl[lo + p] = (rho * fabsf(zc) * nz <= tol);  // deflation of a negligible coupling
                S.rotj[lo + p] = -1;
                if (c == lo) {
                    int bex = 0;
                    if (bscale > 0.f) frexpf(bscale, &bex);
                    S.brho[lb] = rho;
                    S.btol[lb] = tol;
                    S.bsc[lb] = ldexpf(1.f, -bex);
                    S.brot[lb] = 0;
                }
            }
        }
        if (tid == 0) S.flag_rot = 0;
        team_sync<NT>(bar_id);
        // P4: compaction, non-deflated poles first (ascending). The secular problem of the block is
        // scaled exactly by a power of two to unit size: the derivatives of f grow like
        // 1/(d - lambda)^3 and would overflow FP32 for blocks whose spectrum is far below 1
        auto compact = [&]() {
            const int t = pos;
            int nb = 0, K = 0;
            if (act)
#pragma unroll 4
                for (int p2 = lo + sub; p2 < hi; p2 += G) {
                    const int nd = !S.defl[p2];
                    K += nd;
                    nb += (p2 < t) & nd;
                }
            nb = gsumi<G>(nb);
            K = gsumi<G>(K);
            if (act && sub == 0) {
                const int q = S.defl[t] ? (K + (t - lo - nb)) : nb;
                S.inv[lo + q] = S.colof[t];
                S.cdz[lo + q] = make_float2(S.ds[t] * S.bsc[lb], S.zs[t] * S.zs[t]);
                S.cz[lo + q] = S.zs[t];
                if (t == lo) S.bK[lb] = K;
            }
        };
        // P2 (detect close-pole pairs) with the compaction in the same phase; in the rare case that a
        // pair is found, P3 rotates and the compaction is redone
        if (act && sub == 0 && !S.defl[pos]) {
            const int t = pos;
            const float tol = S.btol[lb];
            const float zp = S.zs[t];
            int j = t + 1;
            while (j < hi && S.defl[j]) ++j;
            if (j < hi) {
                // c s = zp zj / (zp^2 + zj^2); the test is loosened by 2 so that no pair the exact
                // test of P3 (with hypot) would rotate is missed
                const float zj = S.zs[j];
                const float cs = zp * zj * rcp_approx(fmaf(zp, zp, zj * zj));
                if (fabsf((S.ds[j] - S.ds[t]) * cs) <= 2.f * tol) {
                    S.brot[lb] = 1;
                    S.flag_rot = 1;
                }
            }
        }
        compact();
        team_sync<NT>(bar_id);
        // P3: close-pole Givens deflation, one pass in pole order (rare)
        if (S.flag_rot) {
            if (act && sub == 0 && pos == lo && S.brot[lb]) {
                const float tol = S.btol[lb];
                int pj = -1;
                for (int p2 = lo; p2 < hi; ++p2) {
                    if (S.defl[p2]) continue;
                    if (pj < 0) {
                        pj = p2;
                        continue;
                    }
                    const float r = hypotf(S.zs[pj], S.zs[p2]);
                    const float cc = S.zs[p2] / r, ss = S.zs[pj] / r;
                    if (fabsf((S.ds[p2] - S.ds[pj]) * cc * ss) <= tol) {
                        const float a2 = S.ds[pj], bb = S.ds[p2];
                        S.ds[pj] = fmaf(cc * cc, a2, ss * ss * bb);
                        S.ds[p2] = fmaf(ss * ss, a2, cc * cc * bb);
                        S.zs[p2] = r;
                        S.zs[pj] = 0.f;
                        S.defl[pj] = 1;
                        S.rotj[pj] = p2;
                        S.rc[pj] = cc;
                        S.rs[pj] = ss;
                    }
                    pj = p2;
                }
            }
            team_sync<NT>(bar_id);
            compact();
            team_sync<NT>(bar_id);
        }
        // P5: secular roots, GS lanes per root (root t on threads GS t ..). Every root repeats the same
        // scalar step logic around its pole sums, so splitting a root's sums over several lanes repeats
        // that logic on each of them: fewer lanes per root issue fewer instructions. Measured best:
        // two lanes per root for 64-row teams (the roots then fill four warps, one per scheduler of
        // the SM), one for 48 rows; 16- and 32-row teams have too few warps and keep G lanes per root.
        constexpr int GS = (NMAX == 64) ? 2 : ((NMAX == 48) ? 1 : G);  // lanes per root
        if (warp * (32 / GS) < n) {  // warps holding no root skip the phase (the vote inside is per warp)
            const int t = tid / GS;
            const int bt = (t < n) ? plan.blk[L][t] : 0xFF;
            int K = 0, q = 0, lot = 0, hit = 0;
            float sc = 1.f, rho = 0.f;
            if (bt != 0xFF) {
                const int lbt = bt - l0;
                lot = plan.m_lo[bt];
                hit = plan.m_hi[bt];
                K = S.bK[lbt];
                q = t - lot;
                sc = S.bsc[lbt];
                rho = S.brho[lbt] * sc;
            }
            const bool part = (bt != 0xFF) && (q < K);
            if (bt != 0xFF && q == 0 && tid % GS == 0) atomicAdd(&S.deflated, static_cast<unsigned>(hit - lot - K));
            const RootOut r = secular_root<GS>(S.cdz + lot, K, q, rho, kp, part, tid % GS);
            if (part && tid % GS == 0) {
                S.dorg[t] = S.cdz[lot + r.org].x;
                S.tq[t] = r.tau;
                S.lam[t] = (S.cdz[lot + r.org].x + r.tau) * (1.f / sc);
                atomicAdd(&S.evals, static_cast<unsigned>(r.evals));
                atomicAdd(&S.roots, 1u);
                if (!r.conv) atomicOr(&S.info, BED_INFO_NOT_CONVERGED);
            } else if (bt != 0xFF && tid % GS == 0) {
                S.dorg[t] = S.cdz[t].x;
                S.tq[t] = 0.f;
                S.lam[t] = S.cdz[t].x * (1.f / sc);
            }
        }
        team_sync<NT>(bar_id);
        // P6: Gu-Eisenstat z-hat, Eq. (25), as a product of interlaced ratios, each in (0, 1):
        //   (lambda_{K-1} - d_i)/rho * prod_{j<i} (lambda_j - d_i)/(d_j - d_i)
        //                            * prod_{i<=j<K-1} (lambda_j - d_i)/(d_{j+1} - d_i)
        {
            int K = 0;
            if (act) K = S.bK[lb];
            const int i = pos - lo;
            const bool own = act && (i < K);
            float prod = 1.f;
            if (own) {
                const float di = S.cdz[lo + i].x;
                if (sub == 0)
                    prod = ((S.dorg[lo + K - 1] - di) + S.tq[lo + K - 1]) / (S.brho[lb] * S.bsc[lb]);
                // two ratios per division: their indices differ by G >= 2, so at most one of the two
                // numerators is a root hugging d_i, and both products stay far inside the FP32 range
                int j = sub;
#pragma unroll 2
                for (; j + G < K - 1; j += 2 * G) {
                    const int jb = j + G;
                    const float na = (S.dorg[lo + j] - di) + S.tq[lo + j];  // lambda_j - d_i
                    const float nb = (S.dorg[lo + jb] - di) + S.tq[lo + jb];
                    const float da = (j < i) ? (S.cdz[lo + j].x - di) : (S.cdz[lo + j + 1].x - di);
                    const float db = (jb < i) ? (S.cdz[lo + jb].x - di) : (S.cdz[lo + jb + 1].x - di);
                    prod *= (na * nb) * rcp_approx(da * db);
                }
                if (j < K - 1) {
                    const float num = (S.dorg[lo + j] - di) + S.tq[lo + j];
                    const float den = (j < i) ? (S.cdz[lo + j].x - di) : (S.cdz[lo + j + 1].x - di);
                    prod *= num / den;
                }
            }
            prod = gprod<G>(prod);
            // (a product below the normal range flushes to zero: |z-hat| < 1e-19 is a negligible coupling)
            if (own && sub == 0) S.zh[lo + i] = copysignf(sqrt_approx(fmaxf(prod, 0.f)), S.cz[lo + i]);
        }
        team_sync<NT>(bar_id);
        // P7: eigenvectors of the merge (Eq. (24)), row of sorted pole p at row colof[p] of M, rotations undone
        {
            int K = 0;
            if (act) K = S.bK[lb];
            const int q = pos - lo;
            const int cq = pos;
            float nrm2 = 0.f;
            if (act) {
                if (q < K) {
                    const float dorg = S.dorg[lo + q];
                    const float tq = S.tq[lo + q];
#pragma unroll 4
                    for (int i = sub; i < K; i += G) {
                        const float v = __fdividef(S.zh[lo + i], (S.cdz[lo + i].x - dorg) - tq);
                        S.M[S.inv[lo + i] * LD + cq] = v;
                        nrm2 = fmaf(v, v, nrm2);
                    }
                    // rows of the deflated poles (compacted indices K ..) are zero
                    for (int i = K + sub; i < hi - lo; i += G) S.M[S.inv[lo + i] * LD + cq] = 0.f;
                } else {
                    const int tgt = S.inv[lo + q];
                    for (int p = lo + sub; p < hi; p += G) S.M[p * LD + cq] = (p == tgt) ? 1.f : 0.f;
                }
            }
            // the columns are normalized by P8, which scales its products by 1 / |column|
            nrm2 = gsum<G>(nrm2);
            if (act && sub == 0) S.cinv[cq] = (q < K) ? rsqrtf(nrm2) : 1.f;
            __syncwarp();
            if (act && sub == 0 && S.brot[lb]) {
                for (int p = hi - 1; p >= lo; --p) {
                    const int j = S.rotj[p];
                    if (j >= 0) {
                        const float cc = S.rc[p], ss = S.rs[p];
                        const int rp = S.colof[p] * LD + cq, rj = S.colof[j] * LD + cq;
                        const float yp = S.M[rp], yj = S.M[rj];
                        S.M[rp] = fmaf(cc, yp, ss * yj);
                        S.M[rj] = fmaf(-ss, yp, cc * yj);
                    }
                }
            }
        }
        team_sync<NT>(bar_id);
        // P8: Q <- blkdiag(Q1, Q2) Q^ (Eq. (4)); P7 stored row c of Q^ (the sorted pole that column c of
        // the children became) at row c of M, so that the product reads M in the children's column order
        if constexpr (TC) {
            constexpr int TPW = (32 / NW < 2) ? 2 : ((32 / NW > 8) ? 8 : 32 / NW);  // tiles per warp
            if (tc_level_tiles(plan, L) <= TPW * NW)
                merge_product_tc<NMAX, G, TPW>(S, plan, L, tid, bar_id);
            else
                merge_product_fma<NMAX, G>(S, plan, L, tid, bar_id);
        } else {
            merge_product_fma<NMAX, G>(S, plan, L, tid, bar_id);
        }
        team_sync<NT>(bar_id);
    }

    // ---------------- a8: back-transform V = H_0 ... H_{n-3} Q_T ----------------------------
    // Blocks of kBT reflectors: H_{k0} ... H_{k0+b-1} = I - Y T Y^T with T upper triangular
    // (forward accumulation); column r of Y is v_{k0+r}, zero above its unit entry. Each block is
    // stored once more as W = Y T, so that applying it is two passes over the rows,
    // Q <- Q - W (Y^T Q). Blocks are applied last to first, with column pos of Q held in registers by
    // its G lanes (rows sub + G t): Y^T Q is a sum over those lanes, so no barrier separates the blocks.
    if (n >= 3) {
        const int nr = n - 2;
        const int ngr = (nr + kBT - 1) / kBT;
        const float* Yt = S.A;
        float* Wt = S.M;  // W, in the layout of Yt (the merges are done with M)
        static_assert(kBT == 8, "two 16-byte reads per row of a block");
        for (int g = warp; g < ngr; g += NW) {
            const int k0 = g * kBT;
            const int bsz = min(kBT, nr - k0);
            // Gram entries Y[:, r]^T Y[:, j], r < j (28 pairs, r-major): every lane forms the products
            // of its rows (two 16-byte reads per row), then a halving exchange over the 32 lanes
            // leaves pair `lane` summed on lane `lane`
            float gram;
            {
                float v[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) v[t] = 0.f;
#pragma unroll
                for (int m = 0; m < (NMAX + 31) / 32; ++m) {
                    const int i = lane + 32 * m;
                    if (32 * m + 31 <= k0) continue;  // rows up to k0 are zero in Y
                    if (i < NMAX) {
                        const float4 ya = *reinterpret_cast<const float4*>(Yt + yt_index<NMAX>(i, k0));
                        const float4 yb = *reinterpret_cast<const float4*>(Yt + yt_index<NMAX>(i, k0 + 4));
                        const float y[kBT] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
                        int pp = 0;
#pragma unroll
                        for (int r = 0; r < kBT - 1; ++r)
#pragma unroll
                            for (int j = r + 1; j < kBT; ++j) {
                                v[pp] = fmaf(y[r], y[j], v[pp]);
                                ++pp;
                            }
                    }
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int t = 0; t < o; ++t) {
                        const float send = up ? v[t] : v[t + o];
                        const float keep = up ? v[t + o] : v[t];
                        v[t] = keep + __shfl_xor_sync(kFull, send, o);
                    }
                }
                gram = v[0];
            }
            // T[jj][jj] = tau_jj; T[0:jj, jj] = -tau_jj T[0:jj, 0:jj] Gram[0:jj, jj]: lane r keeps row r
            // of T in registers; Gram(s, jj) is pair s (15 - s) / 2 + jj - s - 1, read from its lane
            float trow[kBT];
#pragma unroll
            for (int t = 0; t < kBT; ++t) trow[t] = 0.f;
#pragma unroll
            for (int jj = 0; jj < kBT; ++jj) {
                float acc = 0.f;
#pragma unroll
                for (int s2 = 0; s2 < jj; ++s2)
                    acc = fmaf(trow[s2], __shfl_sync(kFull, gram, s2 * (15 - s2) / 2 + jj - s2 - 1), acc);
                const float tj = (jj < bsz) ? S.tau[k0 + jj] : 0.f;
                trow[jj] = (lane < jj) ? -tj * acc : ((lane == jj) ? tj : 0.f);
            }
            // W = Y T for this lane's rows; T[r][c] (r <= c) comes from lane r
#pragma unroll
            for (int m = 0; m < (NMAX + 31) / 32; ++m) {
                const int i = lane + 32 * m;
                if (32 * m + 31 < k0) continue;  // rows below k0 of W are never read
                float y[kBT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (i < NMAX) {
                    const float4 ya = *reinterpret_cast<const float4*>(Yt + yt_index<NMAX>(i, k0));
                    const float4 yb = *reinterpret_cast<const float4*>(Yt + yt_index<NMAX>(i, k0 + 4));
                    y[0] = ya.x, y[1] = ya.y, y[2] = ya.z, y[3] = ya.w;
                    y[4] = yb.x, y[5] = yb.y, y[6] = yb.z, y[7] = yb.w;
                }
                float w[kBT];
#pragma unroll
                for (int c = 0; c < kBT; ++c) {
                    float acc = 0.f;
#pragma unroll
                    for (int r = 0; r <= c; ++r) acc = fmaf(y[r], __shfl_sync(kFull, trow[c], r), acc);
                    w[c] = acc;
                }
                if (i < NMAX) {
                    *reinterpret_cast<float4*>(Wt + yt_index<NMAX>(i, k0)) = make_float4(w[0], w[1], w[2], w[3]);
                    *reinterpret_cast<float4*>(Wt + yt_index<NMAX>(i, k0 + 4)) = make_float4(w[4], w[5], w[6], w[7]);
                }
            }
        }
        team_sync<NT>(bar_id);
        constexpr int RPT = NMAX / G;
        float q[RPT];
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
            const int i = sub + G * t;
            q[t] = (pos < n && i < n) ? S.Q[i * LD + pos] : 0.f;
        }
        // Rows i = sub + G t of this lane fall into PER classes of i & SW (the XOR swizzle of yt_index), so a
        // block's two 16-byte chunks of row t sit at a class offset plus a compile-time row offset: the
        // addresses cost a few instructions per block instead of per row
        constexpr int CH = NMAX / 4;
        constexpr int SWP = (CH % 8 == 0) ? 8 : ((CH % 4 == 0) ? 4 : ((CH % 2 == 0) ? 2 : 1));
        constexpr int PER = SWP > G ? SWP / G : 1;
        const float* Yrow = Yt + sub * NMAX;
        const float* Wrow = Wt + sub * NMAX;
        for (int g = ngr - 1; g >= 0; --g) {
            const int k0 = g * kBT;
            int offa[PER], offb[PER];  // yt_index(i, k0) - i NMAX and yt_index(i, k0 + 4) - i NMAX per class
#pragma unroll
            for (int c = 0; c < PER; ++c) {
                const int sw = (sub + G * c) & (SWP - 1);
                offa[c] = ((2 * g) ^ sw) << 2;
                offb[c] = ((2 * g + 1) ^ sw) << 2;
            }
            // W1 = Y^T q over this lane's rows; rows up to k0 are zero in every column of Y and W. The
            // rows go in chunks of 8 (TPC values of t): a chunk wholly above row k0 is skipped by a test
            // that is the same on every lane, so its loads and FMAs are not issued at all (a test per
            // row would only predicate them off)
            constexpr int TPC = 8 / G;
            float w1[kBT];
#pragma unroll
            for (int r = 0; r < kBT; ++r) w1[r] = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < RPT / TPC; ++c8) {
                if (8 * c8 + 7 <= k0) continue;
#pragma unroll
                for (int t = c8 * TPC; t < c8 * TPC + TPC; ++t) {
                    const float4 ya = *reinterpret_cast<const float4*>(Yrow + G * t * NMAX + offa[t % PER]);
                    const float4 yb = *reinterpret_cast<const float4*>(Yrow + G * t * NMAX + offb[t % PER]);
                    w1[0] = fmaf(ya.x, q[t], w1[0]);
                    w1[1] = fmaf(ya.y, q[t], w1[1]);
                    w1[2] = fmaf(ya.z, q[t], w1[2]);
                    w1[3] = fmaf(ya.w, q[t], w1[3]);
                    w1[4] = fmaf(yb.x, q[t], w1[4]);
                    w1[5] = fmaf(yb.y, q[t], w1[5]);
                    w1[6] = fmaf(yb.z, q[t], w1[6]);
                    w1[7] = fmaf(yb.w, q[t], w1[7]);
                }
            }
#pragma unroll
            for (int r = 0; r < kBT; ++r) w1[r] = gsum<G>(w1[r]);
            // q -= W W1, over the same chunks
#pragma unroll
            for (int c8 = 0; c8 < RPT / TPC; ++c8) {
                if (8 * c8 + 7 <= k0) continue;
#pragma unroll
                for (int t = c8 * TPC; t < c8 * TPC + TPC; ++t) {
                    const float4 wa = *reinterpret_cast<const float4*>(Wrow + G * t * NMAX + offa[t % PER]);
                    const float4 wb = *reinterpret_cast<const float4*>(Wrow + G * t * NMAX + offb[t % PER]);
                    float v = q[t];
                    v = fmaf(-wa.x, w1[0], v);
                    v = fmaf(-wa.y, w1[1], v);
                    v = fmaf(-wa.z, w1[2], v);
                    v = fmaf(-wa.w, w1[3], v);
                    v = fmaf(-wb.x, w1[4], v);
                    v = fmaf(-wb.y, w1[5], v);
                    v = fmaf(-wb.z, w1[6], v);
                    q[t] = fmaf(-wb.w, w1[7], v);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
            const int i = sub + G * t;
            if (pos < n && i < n) S.Q[i * LD + pos] = q[t];
        }
        team_sync<NT>(bar_id);
    }

    // ---------------- a9: ascending order, signs, store ------------------------------------
    {
        int r = 0;
        if (pos < n) {
            const float kc = sort_key(S.lam[pos]);
#pragma unroll 4
            for (int t2 = sub; t2 < n; t2 += G) {
                const float k2 = sort_key(S.lam[t2]);
                r += (k2 < kc) || (k2 == kc && t2 < pos);
            }
        }
        r = gsumi<G>(r);
        if (pos < n && sub == 0) S.outc[r] = pos;
    }
    team_sync<NT>(bar_id);
    {
        int src = 0;
        float vm = -1.f;
        int im = 0;
        if (pos < n) {
            src = S.outc[pos];
#pragma unroll 4
            for (int i = sub; i < n; i += G) {
                const float v = fabsf(S.Q[i * LD + src]);
                if (v > vm) {
                    vm = v;
                    im = i;
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) {
            const float v2 = __shfl_xor_sync(kFull, vm, o);
            const int i2 = __shfl_xor_sync(kFull, im, o);
            if (v2 > vm || (v2 == vm && i2 < im)) {
                vm = v2;
                im = i2;
            }
        }
        if (pos < n && sub == 0) {
            S.sgn[pos] = (S.Q[im * LD + src] < 0.f) ? -1.f : 1.f;
            S.out_w[pos] = S.lam[src] * S.unscale;
        }
    }
    team_sync<NT>(bar_id);
    {
        // each lane stores the same output columns j = lane + 32 t of every row: their signs and source
        // columns are read once
        constexpr int JPL = (NMAX + 31) / 32;
        float sj[JPL];
        int cj[JPL];
#pragma unroll
        for (int t = 0; t < JPL; ++t) {
            const int j = lane + 32 * t;
            sj[t] = (j < n) ? S.sgn[j] : 0.f;
            cj[t] = (j < n) ? S.outc[j] : 0;
        }
        float* ov = S.out_v;
        for (int i = warp; i < n; i += NW) {
            const float* qi = S.Q + i * LD;
#pragma unroll
            for (int t = 0; t < JPL; ++t) {
                const int j = lane + 32 * t;
                if (j < n) ov[i * n + j] = sj[t] * qi[cj[t]];
            }
        }
    }
    if (tid == 0) {
        if (S.out_info) *S.out_info = S.info;
        if (counters) {
            atomicAdd(&counters->matrices, 1ull);
            atomicAdd(&counters->roots, static_cast<unsigned long long>(S.roots));
            atomicAdd(&counters->evals, static_cast<unsigned long long>(S.evals));
            atomicAdd(&counters->deflated, static_cast<unsigned long long>(S.deflated));
        }
    }
    team_sync<NT>(bar_id);
    return true;
}

// ---------------------------------------------------------------------------------------------
// Uniform-size kernel: one team = one thread block, matrices b = blockIdx.x, blockIdx.x + gridDim.x, ...
// ---------------------------------------------------------------------------------------------
// Blocks per SM the launch bounds promise: as many as 64 registers a thread allows, but no more than
// the shared memory lets reside (228 KB per SM, 1 KB of it reserved per block), so that a block whose
// residency is set by shared memory gets the registers that it can use (the 64 x 64 team of 128
// threads: 4 blocks, 128 registers).
template <int NMAX, int G>
constexpr int eigh_min_blocks()
{
    constexpr int by_regs = 65536 / (NMAX * G * 64);
    constexpr int by_smem = static_cast<int>((228 * 1024) / (sizeof(Smem<NMAX, G>) + 1024));
    constexpr int m = by_regs < by_smem ? by_regs : by_smem;
    return m < 1 ? 1 : m;
}

template <int NMAX, int G, bool TC>
__global__ void __launch_bounds__(NMAX * G, eigh_min_blocks<NMAX, G>())
    eigh_kernel(const float* __restrict__ A, float* __restrict__ W, float* __restrict__ V,
                int32_t* __restrict__ info, int64_t batch, const __grid_constant__ Plan plan,
                const KParams kp, bed_counters* __restrict__ counters, int bulk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<NMAX, G>& S = *reinterpret_cast<Smem<NMAX, G>*>(smem_raw);
    const int n = plan.n;
    const uint32_t bar = smem_u32(&S.mbar);
    uint32_t phase = 0;
    if (bulk) {
        if (threadIdx.x == 0) mbar_init(bar);
        __syncthreads();
    }
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        if (!solve_matrix<NMAX, G, TC>(S, plan, kp, threadIdx.x, 0, bar, phase, A + b * (int64_t)n * n,
                                   W + b * (int64_t)n, V + b * (int64_t)n * n, info ? info + b : nullptr,
                                   counters, bulk != 0))
            return;
    }
}

template <int NMAX, int G, bool TC>
cudaError_t launch_eigh_t(const float* A, float* W, float* V, int32_t* info, int64_t batch, int64_t blocks,
                          const Plan& P, const KParams& kp, bed_counters* counters, bool bulk,
                          cudaStream_t stream)
{
    const size_t smem = sizeof(Smem<NMAX, G>);
    auto kern = eigh_kernel<NMAX, G, TC>;
    // the function attributes are per device: set them on the first launch there (setting them again
    // from a racing thread is harmless), keeping later launches to the launch itself
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load(std::memory_order_acquire) & bit)) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (err != cudaSuccess) return err;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared);
        if (err != cudaSuccess) return err;
        configured.fetch_or(bit, std::memory_order_release);
    }
    const int64_t max_grid = 2147483647LL;
    const unsigned grid = static_cast<unsigned>(blocks < max_grid ? blocks : max_grid);
    kern<<<grid, NMAX * G, smem, stream>>>(A, W, V, info, batch, P, kp, counters, bulk ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace bed
