// Mixed-precision Sylvester / Lyapunov solvers with FP64-accurate iterative
// refinement.
//
// Per instance (one CTA):
//   1. r_ij = 1 / (l_ii + u_jj) in FP64 (the divisions stay FP64), stored as
//      FP32 in scratch; tiny or NaN divisors set info = 1.
//   2. Low-precision solve of L D + D U = C: the lazy blocked recurrence of the
//      FP64 kernels with FP32 tiles.  Off-diagonal block updates run in FP32
//      FMA (CUDA cores) or on the tensor cores in TF32 / BF16 with FP32
//      accumulation (mma.sync); the diagonal-block wavefront runs in FP32 and
//      multiplies by the FP64-computed reciprocals.
//   3. X = D in FP64.  Then repeat: R = C - L X - X U with FP64-class accuracy
//      (double-float arithmetic on the FP32 pipe, or FP64 FMA), solve
//      L D + D U = R in low precision, X += D, until the predicted error
//      |D|^2 / |D_prev| (or |D| itself) is below SS_REFINE_TOL * |X|.
// The Lyapunov form is the Sylvester one with U = L^T over the lower blocks.
// Every instance is rescaled by powers of two (DfScale: L and U by 2^op, C by
// 2^rhs, so X carries 2^x) before anything enters FP32: each FP64 value is
// shifted as it is converted (the `sh` arguments below), X in global memory
// stays in the caller's units.  Without it data outside FP32's exponent
// range (or residuals that shrink below it) would be lost in conversion.
//
// Double-float arithmetic (split, TwoProduct / TwoSum updates) is in df.cuh.
#pragma once

#include <cuda_bf16.h>

#include "df.cuh"
#include "ss_device.cuh"
#include "ss_internal.h"

namespace ss {
namespace mx {

enum Prec { P_FP32 = 0, P_TF32 = 1, P_BF16 = 2 };
enum Res { R_DF = 0, R_FP64 = 1 };

constexpr int MAXIT = SS_REFINE_MAXIT;

// FP64 -> FP32 by truncating the significand, integer operations only (the
// low-precision solve does not need round-to-nearest; values outside the FP32
// normal range take the hardware conversion).
__device__ __forceinline__ float d2f_trunc(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
    const int ef = (int)((u >> 52) & 0x7FF) - 896;
    if (ef >= 1 && ef <= 254)
        return __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
    if ((u << 1) == 0ull) return __uint_as_float(sgn);
    return __double2float_rz(x);
}


// x * 2^sh -> FP32 by truncation (the high part of split_df_s, with its
// flush below 2^-126 and +-Inf above the range).
__device__ __forceinline__ float d2f_trunc_s(double x, int sh)
{
    float hi, lo;
    split_df_s(x, sh, hi, lo);
    return hi;
}

// Staging conversions of one element: FP64 sources are scaled by 2^sh and
// truncated to FP32 (float) or split (float2); FP32 sources (scratch that is
// already in scaled units) are copied.
__device__ __forceinline__ float to_f(float v, int) { return v; }
__device__ __forceinline__ float to_f(double v, int sh) { return d2f_trunc_s(v, sh); }

template <typename Elem, typename Src>
__device__ __forceinline__ Elem cvt_elem(Src v, int sh);
template <>
__device__ __forceinline__ float cvt_elem<float, float>(float v, int) { return v; }
template <>
__device__ __forceinline__ float cvt_elem<float, double>(double v, int sh) { return d2f_trunc_s(v, sh); }
template <>
__device__ __forceinline__ float2 cvt_elem<float2, double>(double v, int sh)
{
    float2 r;
    split_df_s(v, sh, r.x, r.y);
    return r;
}


// ------------------------------------------------------------------ tiles

// Shared tiles: natural layout uses LD = B + 1; every tile slot holds
// B * (B + 4) elements so the k-major micro-tile layouts fit as well.
template <int B>
struct FTile {
    static constexpr int LD = B + 1;
    static constexpr int SZ = B * (B + 4);
};

// Modes of staging a B x B tile from a column-major global matrix.
enum Fill { F_FULL, F_LOWER, F_UPPER, F_SYM_LOWER };

template <Fill F>
__device__ __forceinline__ bool fill_keep(int r, int c) {
    return F == F_FULL || F == F_SYM_LOWER || (F == F_LOWER ? r >= c : r <= c);
}

// Float tile from a double (scaled by 2^sh) or float source (rows x cols
// valid, zero elsewhere).
template <int B, int T, Fill F, typename Src>
__device__ __forceinline__ void stage_f(float *S, const Src *G, long ldg, int rows, int cols, int sh)
{
    constexpr int LD = FTile<B>::LD;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        float v = 0.0f;
        if (r < rows && c < cols && fill_keep<F>(r, c)) {
            const long idx = (F == F_SYM_LOWER && r < c) ? (c + (long)r * ldg) : (r + (long)c * ldg);
            v = to_f(G[idx], sh);
        }
        S[r + c * LD] = v;
    }
}

// Double-float tile (float2 hi/lo) of a double source scaled by 2^sh.
template <int B, int T, Fill F>
__device__ __forceinline__ void stage_df(float2 *S, const double *G, long ldg, int rows, int cols, int sh)
{
    constexpr int LD = FTile<B>::LD;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows && c < cols && fill_keep<F>(r, c)) {
            const long idx = (F == F_SYM_LOWER && r < c) ? (c + (long)r * ldg) : (r + (long)c * ldg);
            split_df_s(G[idx], sh, v.x, v.y);
        }
        S[r + c * LD] = v;
    }
}

// Double tile (for the FP64-FMA residual) of a double source scaled by 2^sh
// (exact products by powers of two).
template <int B, int T, Fill F>
__device__ __forceinline__ void stage_d(double *S, const double *G, long ldg, int rows, int cols, int sh)
{
    constexpr int LD = Tile<B>::LD;
    const Pow2 f(sh);
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        double v = 0.0;
        if (r < rows && c < cols && fill_keep<F>(r, c)) {
            const long idx = (F == F_SYM_LOWER && r < c) ? (c + (long)r * ldg) : (r + (long)c * ldg);
            v = f(G[idx]);
        }
        S[r + c * LD] = v;
    }
}

// ------------------------------------------------------- block updates (FP32)

template <int B, int T, bool TA, bool TB>
__device__ __forceinline__ void slot_update_f(float (&acc)[B * B / T], const Slots<B, T> &s,
                                              const float *A, const float *Bm, int kk)
{
    constexpr int LD = FTile<B>::LD;
    constexpr int E = B * B / T;
#pragma unroll 2
    for (int k = 0; k < kk; ++k) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (s.ok(r)) {
                const float a = TA ? A[k + s.row[r] * LD] : A[s.row[r] + k * LD];
                const float b = TB ? Bm[s.col[r] + k * LD] : Bm[k + s.col[r] * LD];
                acc[r] = fmaf(-a, b, acc[r]);
            }
        }
    }
}

template <int B, int T, bool TA, bool TB>
__device__ __forceinline__ void slot_update_df(float (&ah)[B * B / T], float (&al)[B * B / T],
                                               const Slots<B, T> &s, const float2 *A,
                                               const float2 *Bm, int kk)
{
    constexpr int LD = FTile<B>::LD;
    constexpr int E = B * B / T;
#pragma unroll 1
    for (int k = 0; k < kk; ++k) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (s.ok(r)) {
                const float2 a = TA ? A[k + s.row[r] * LD] : A[s.row[r] + k * LD];
                const float2 b = TB ? Bm[s.col[r] + k * LD] : Bm[k + s.col[r] * LD];
                df_msub(ah[r], al[r], a.x, a.y, b.x, b.y);
            }
        }
    }
}

// ---------------------------------------- register micro-tiles (full blocks)
//
// For a full B x B output block each thread owns an MR x MC micro-tile at rows
// r0 = (tid % TX) * MR and columns c0 = (tid / TX) * MC.  Operands are staged
// "k-major": sOA[r + k*LDA] = op(A)(r, k) (LDA = B + 4, so a column of MR = 4
// rows is one aligned 16-byte load) and sOB[c + k*LDB] = op(B)(k, c)
// (LDB = B + 1), transposing at staging time when the operand is read
// transposed.  One k step is MR/4 + MC loads for MR * MC FMAs.
template <int B, int T>
struct Micro {
    static constexpr int P = (B * B) / T >= 1 ? (B * B) / T : 1;   // outputs per thread
    static constexpr int MR = P >= 4 ? 4 : P;
    static constexpr int MC = P / MR;
    static constexpr int TX = B / MR;
    static constexpr int TY = B / MC;
    static constexpr int LDA = B + 4;
    static constexpr int LDB = B + 1;
    static constexpr bool OK = B * B >= T && TX * TY == T && TX * MR == B && TY * MC == B;
    __device__ __forceinline__ static int r0() { return (threadIdx.x % TX) * MR; }
    __device__ __forceinline__ static int c0() { return (threadIdx.x / TX) * MC; }
};

// Stage op(A) (rows x kk valid, zero elsewhere) k-major: sOA[r + k*LDA].
// TRANS: op(A)(r, k) = G(k, r).
template <int B, int T, bool TRANS, typename Src, typename Elem>
__device__ __forceinline__ void stage_opA(Elem *S, const Src *G, long ldg, int rows, int kk, int sh)
{
    constexpr int LDA = Micro<B, T>::LDA;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int x = e % B, y = e / B;      // fast index x walks memory
        const int r = TRANS ? y : x, k = TRANS ? x : y;
        Elem v{};
        if (r < rows && k < kk) v = cvt_elem<Elem>(G[x + (long)y * ldg], sh);
        S[r + k * LDA] = v;
    }
}

// Stage op(B) (kk x cols valid) k-major: sOB[c + k*LDB].  TRANS: op(B)(k, c) = G(c, k).
template <int B, int T, bool TRANS, typename Src, typename Elem>
__device__ __forceinline__ void stage_opB(Elem *S, const Src *G, long ldg, int kk, int cols, int sh)
{
    constexpr int LDB = Micro<B, T>::LDB;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int x = e % B, y = e / B;
        const int k = TRANS ? y : x, c = TRANS ? x : y;
        Elem v{};
        if (k < kk && c < cols) v = cvt_elem<Elem>(G[x + (long)y * ldg], sh);
        S[c + k * LDB] = v;
    }
}

template <int B, int T>
__device__ __forceinline__ void micro_update_f(float (&acc)[Micro<B, T>::MR][Micro<B, T>::MC],
                                               const float *sOA, const float *sOB, int kk)
{
    using M = Micro<B, T>;
    const int r0 = M::r0(), c0 = M::c0();
#pragma unroll 4
    for (int k = 0; k < kk; ++k) {
        float a[M::MR], b[M::MC];
        if constexpr (M::MR == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(sOA + r0 + k * M::LDA);
            a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
        } else {
#pragma unroll
            for (int i = 0; i < M::MR; ++i) a[i] = sOA[r0 + i + k * M::LDA];
        }
#pragma unroll
        for (int j = 0; j < M::MC; ++j) b[j] = sOB[c0 + j + k * M::LDB];
#pragma unroll
        for (int i = 0; i < M::MR; ++i)
#pragma unroll
            for (int j = 0; j < M::MC; ++j) acc[i][j] = fmaf(-a[i], b[j], acc[i][j]);
    }
}

template <int B, int T>
__device__ __forceinline__ void micro_update_df(float (&ah)[Micro<B, T>::MR][Micro<B, T>::MC],
                                                float (&al)[Micro<B, T>::MR][Micro<B, T>::MC],
                                                const float2 *sOA, const float2 *sOB, int kk)
{
    using M = Micro<B, T>;
    const int r0 = M::r0(), c0 = M::c0();
#pragma unroll 1
    for (int k = 0; k < kk; ++k) {
        float2 a[M::MR], b[M::MC];
#pragma unroll
        for (int i = 0; i < M::MR; ++i) a[i] = sOA[r0 + i + k * M::LDA];
#pragma unroll
        for (int j = 0; j < M::MC; ++j) b[j] = sOB[c0 + j + k * M::LDB];
#pragma unroll
        for (int i = 0; i < M::MR; ++i)
#pragma unroll
            for (int j = 0; j < M::MC; ++j) df_msub(ah[i][j], al[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
    }
}

// ----------------------------------------- block updates (tensor cores, mma.sync)
//
// The B x B output is cut into 16 x 8 tiles; warp w owns tiles w*TPW .. w*TPW+TPW-1
// (tile t covers rows 16*(t / (B/8)) and columns 8*(t % (B/8))).  Fragment
// layouts are those of mma.m16n8k8 (TF32) and mma.m16n8k16 (BF16).

template <int B, int T>
struct MmaShape {
    static constexpr int TILES = (B / 16) * (B / 8);
    static constexpr int NW = T / 32;
    static constexpr int TPW = TILES / NW;
    static_assert(TILES % NW == 0 && TPW >= 1, "mma tiling needs whole tiles per warp");
};

// Tensor-core fragments per warp (1 for the FP32 path, which uses none).
template <int B, int T, int P>
struct FragN { static constexpr int value = MmaShape<B, T>::TPW; };
template <int B, int T>
struct FragN<B, T, P_FP32> { static constexpr int value = 1; };

__device__ __forceinline__ unsigned to_tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&v);
}

template <int B, int T>
__device__ __forceinline__ void frag_load(float (&c)[MmaShape<B, T>::TPW][4], const float *S)
{
    constexpr int LD = FTile<B>::LD;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < MmaShape<B, T>::TPW; ++q) {
        const int t = w * MmaShape<B, T>::TPW + q;
        const int r = 16 * (t / (B / 8)) + (lane >> 2), cc = 8 * (t % (B / 8)) + 2 * (lane & 3);
        c[q][0] = S[r + cc * LD];
        c[q][1] = S[r + (cc + 1) * LD];
        c[q][2] = S[r + 8 + cc * LD];
        c[q][3] = S[r + 8 + (cc + 1) * LD];
    }
}

template <int B, int T>
__device__ __forceinline__ void frag_store(const float (&c)[MmaShape<B, T>::TPW][4], float *S)
{
    constexpr int LD = FTile<B>::LD;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < MmaShape<B, T>::TPW; ++q) {
        const int t = w * MmaShape<B, T>::TPW + q;
        const int r = 16 * (t / (B / 8)) + (lane >> 2), cc = 8 * (t % (B / 8)) + 2 * (lane & 3);
        S[r + cc * LD] = c[q][0];
        S[r + (cc + 1) * LD] = c[q][1];
        S[r + 8 + cc * LD] = c[q][2];
        S[r + 8 + (cc + 1) * LD] = c[q][3];
    }
}

// c -= op(A) op(Bm) over kk (a multiple of 8 for TF32, 16 for BF16) terms.
template <int B, int T, int P, bool TA, bool TB>
__device__ __forceinline__ void mma_update(float (&c)[MmaShape<B, T>::TPW][4], const float *A,
                                           const float *Bm, int kk)
{
    constexpr int LD = FTile<B>::LD;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int g = lane >> 2, h = lane & 3;
    auto Aat = [&](int i, int k) { return TA ? A[k + i * LD] : A[i + k * LD]; };
    auto Bat = [&](int k, int j) { return TB ? Bm[j + k * LD] : Bm[k + j * LD]; };
#pragma unroll
    for (int q = 0; q < MmaShape<B, T>::TPW; ++q) {
        const int t = w * MmaShape<B, T>::TPW + q;
        const int r0 = 16 * (t / (B / 8)), c0 = 8 * (t % (B / 8));
        if (P == P_TF32) {
            for (int k0 = 0; k0 < kk; k0 += 8) {
                const unsigned a0 = to_tf32(-Aat(r0 + g, k0 + h));
                const unsigned a1 = to_tf32(-Aat(r0 + g + 8, k0 + h));
                const unsigned a2 = to_tf32(-Aat(r0 + g, k0 + h + 4));
                const unsigned a3 = to_tf32(-Aat(r0 + g + 8, k0 + h + 4));
                const unsigned b0 = to_tf32(Bat(k0 + h, c0 + g));
                const unsigned b1 = to_tf32(Bat(k0 + h + 4, c0 + g));
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                    "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        } else {
            for (int k0 = 0; k0 < kk; k0 += 16) {
                const unsigned a0 = pack_bf16(-Aat(r0 + g, k0 + 2 * h), -Aat(r0 + g, k0 + 2 * h + 1));
                const unsigned a1 = pack_bf16(-Aat(r0 + g + 8, k0 + 2 * h), -Aat(r0 + g + 8, k0 + 2 * h + 1));
                const unsigned a2 = pack_bf16(-Aat(r0 + g, k0 + 2 * h + 8), -Aat(r0 + g, k0 + 2 * h + 9));
                const unsigned a3 = pack_bf16(-Aat(r0 + g + 8, k0 + 2 * h + 8), -Aat(r0 + g + 8, k0 + 2 * h + 9));
                const unsigned b0 = pack_bf16(Bat(k0 + 2 * h, c0 + g), Bat(k0 + 2 * h + 1, c0 + g));
                const unsigned b1 = pack_bf16(Bat(k0 + 2 * h + 8, c0 + g), Bat(k0 + 2 * h + 9, c0 + g));
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                    "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                    : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
    }
}

// ------------------------------------------------------ diagonal block (FP32)

__device__ __forceinline__ float group_sum_f(float v, int split)
{
    for (int o = split >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Solve Lt Y + Y Ut = T in place (m x nn block in sT), multiplying by the
// FP64-computed reciprocals Rg[i + j*ldr] (global, float), which are first
// staged into the shared tile sR so no step of the wavefront waits on a
// global load.  UT: Ut is the transpose of the lower-triangular sU.
template <int B, int T, bool UT>
__device__ void syl_diag_f(const float *sL, const float *sU, float *sT, int m, int nn,
                           const float *Rg, long ldr, float *sR)
{
    constexpr int LD = FTile<B>::LD;
    for (int e = threadIdx.x; e < m * nn; e += T) {
        const int i = e % m, j = e / m;
        sR[i + j * LD] = Rg[i + (long)j * ldr];
    }
    __syncthreads();
    for (int d = 0; d <= m + nn - 2; ++d) {
        const int ilo = max(0, d - nn + 1), ihi = min(d, m - 1);
        const int cnt = ihi - ilo + 1;
        const int split = pick_split<T>(cnt, d);
        if (warp_has_work(cnt, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < cnt;
            const int i = ilo + (act ? idx : 0), j = d - i;
            float s = 0.0f;
            if (act) {
                for (int t = part; t < d; t += split) {
                    const bool lt = t < i;
                    const int k = t - i;
                    const float a = lt ? sL[i + t * LD] : sT[i + k * LD];
                    const float b = lt ? sT[t + j * LD] : (UT ? sU[j + k * LD] : sU[k + j * LD]);
                    s = fmaf(a, b, s);
                }
            }
            s = group_sum_f(s, split);
            if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * sR[i + j * LD];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float block_sum_f(float v, float *s_red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += s_red[w];
    __syncthreads();
    return r;
}

}  // namespace mx
}  // namespace ss
