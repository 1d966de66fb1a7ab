// Warp-block wavefront variant of the mixed-precision Sylvester / Lyapunov
// solver (FP32 low-precision solves, double-float residual).
//
// The latency of one instance, not arithmetic, bounds the FP32 solves, so this
// variant shortens the dependency chain:
//   * the 32 x 32 blocks of X are solved by block anti-diagonals D = I + J;
//     the blocks of one anti-diagonal are independent and each is solved by
//     one warp on its own (staging its tiles in its private shared memory,
//     register micro-tiles of 4 x 8 per lane for the updates
//       T_IJ = R_IJ - sum_{K<I} L_IK D_KJ - sum_{K<J} D_IK U_KJ,
//     then the diagonal-block recurrence as an anti-diagonal wavefront with
//     warp-level synchronisation only); one CTA barrier per block
//     anti-diagonal (2 * ceil(n/32) - 1 per solve);
//   * the residual blocks R_IJ = C_IJ - (L X)_IJ - (X U)_IJ are independent, so
//     warps compute them with no CTA barrier at all (double-float micro-tiles,
//     operands split on staging with integer operations).
// L and U are converted to FP32 once per instance into scratch (for the
// Lyapunov form U = L^T is stored explicitly), as are the FP64 reciprocals
// 1/(l_ii + u_jj).  Scratch per instance: 4 n^2 floats (D, reciprocals, L, U).
//
// Tensor-memory configurations (TF32 / BF16, n <= 128) replace the
// low-precision solve by a right-looking one whose right-hand side stays in
// TMEM as the tensor cores' FP32 accumulator (tsolve below); the residual and
// the correction steps are the same.
#pragma once

#include "mixed_solver.cuh"
#include "umma.cuh"

namespace ss {
namespace mx {
namespace wb {

constexpr int BW = 32;           // block size (one lane per block column)
constexpr int LDK = BW + 4;      // k-major operand tiles (16-byte aligned rows of 4)
constexpr int LDN = BW + 1;      // natural tiles
constexpr int TILE = BW * LDK;   // floats per tile slot (>= BW * LDN)
constexpr int SLOTS = 4;         // per warp: A, B, T, R

__host__ __device__ constexpr size_t smem_bytes(int wpc) { return (size_t)wpc * SLOTS * TILE * sizeof(float) + 256; }

// Lane (tx, ty) owns rows 4tx..4tx+3 and columns 8ty..8ty+7 of a block.
__device__ __forceinline__ int lane_r0() { return ((threadIdx.x & 31) & 7) * 4; }
__device__ __forceinline__ int lane_c0() { return ((threadIdx.x & 31) >> 3) * 8; }

// Warp-staging of a BW x BW float source block into k-major op(A):
// S[r + k*LDK] = op(A)(r, k).  TRANS: op(A)(r, k) = G(k, r).
template <bool TRANS>
__device__ __forceinline__ void wstage_A(float *S, const float *G, long ld, int rows, int kk)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 16
    for (int y = 0; y < BW; ++y) {
        const int x = lane;
        const int r = TRANS ? y : x, k = TRANS ? x : y;
        float v = 0.0f;
        if (r < rows && k < kk) v = G[x + (long)y * ld];
        S[r + k * LDK] = v;
    }
}

// S[c + k*LDK] = op(B)(k, c); TRANS: op(B)(k, c) = G(c, k).
template <bool TRANS>
__device__ __forceinline__ void wstage_B(float *S, const float *G, long ld, int kk, int cols)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 16
    for (int y = 0; y < BW; ++y) {
        const int x = lane;
        const int k = TRANS ? y : x, c = TRANS ? x : y;
        float v = 0.0f;
        if (k < kk && c < cols) v = G[x + (long)y * ld];
        S[c + k * LDK] = v;
    }
}

// acc -= op(A) op(B) over kk terms (k-major tiles).
__device__ __forceinline__ void wmicro_f(float (&acc)[4][8], const float *A, const float *B, int kk)
{
    const int r0 = lane_r0(), c0 = lane_c0();
#pragma unroll 4
    for (int k = 0; k < kk; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(A + r0 + k * LDK);
        const float4 b0 = *reinterpret_cast<const float4 *>(B + c0 + k * LDK);
        const float4 b1 = *reinterpret_cast<const float4 *>(B + c0 + 4 + k * LDK);
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(-av[i], bv[j], acc[i][j]);
    }
}

// One warp solves block (I, J) of L D + D U = RHS in place on W (ld n):
// Lf, Uf are FP32 copies (Uf = L^T for the Lyapunov form), R the reciprocals.
template <bool LYAP>
__device__ void warp_block(int n, int I, int J, const float *Lf, const float *Uf, const float *R, float *W,
                           float *sm)
{
    float *sA = sm, *sB = sm + TILE, *sT = sm + 2 * TILE, *sR = sm + 3 * TILE;
    const int lane = threadIdx.x & 31;
    const long ldn = n;
    const int i0 = I * BW, j0 = J * BW;
    const int mI = min(BW, n - i0), nJ = min(BW, n - j0);
    const int r0 = lane_r0(), c0 = lane_c0();
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = r0 + i, c = c0 + j;
            acc[i][j] = (r < mI && c < nJ) ? W[(i0 + r) + (long)(j0 + c) * ldn] : 0.0f;
        }
    // sum_{K<I} L_IK D_KJ   (Lyapunov: D_KJ = D_JK^T for K < J)
    for (int K = 0; K < I; ++K) {
        const int k0 = K * BW;
        __syncwarp();
        wstage_A<false>(sA, Lf + i0 + (long)k0 * ldn, ldn, mI, BW);
        if (LYAP && K < J) wstage_B<true>(sB, W + j0 + (long)k0 * ldn, ldn, BW, nJ);
        else wstage_B<false>(sB, W + k0 + (long)j0 * ldn, ldn, BW, nJ);
        __syncwarp();
        wmicro_f(acc, sA, sB, BW);
    }
    // sum_{K<J} D_IK U_KJ
    for (int K = 0; K < J; ++K) {
        const int k0 = K * BW;
        __syncwarp();
        wstage_A<false>(sA, W + i0 + (long)k0 * ldn, ldn, mI, BW);
        wstage_B<false>(sB, Uf + k0 + (long)j0 * ldn, ldn, BW, nJ);
        __syncwarp();
        wmicro_f(acc, sA, sB, BW);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sT[(r0 + i) + (c0 + j) * LDN] = acc[i][j];
    // Diagonal blocks of L and U, and the reciprocals, in natural layout.
#pragma unroll 8
    for (int y = 0; y < BW; ++y) {
        const int x = lane;
        sA[x + y * LDN] = (x < mI && y < mI && x > y) ? Lf[(i0 + x) + (long)(i0 + y) * ldn] : 0.0f;
        sB[x + y * LDN] = (x < nJ && y < nJ && x < y) ? Uf[(j0 + x) + (long)(j0 + y) * ldn] : 0.0f;
        sR[x + y * LDN] = (x < mI && y < nJ) ? R[(i0 + x) + (long)(j0 + y) * ldn] : 0.0f;
    }
    __syncwarp();
    // Wavefront: lane j finishes entry (d - j, j) at step d (d - j terms from
    // the strict lower row of L_II, j from the strict upper column of U_JJ).
    for (int d = 0; d <= mI + nJ - 2; ++d) {
        const int j = lane, i = d - j;
        if (j < nJ && i >= 0 && i < mI) {
            // d terms in one uniform loop: t < i from the L row, then the U column.
            float s0 = 0.0f, s1 = 0.0f;
            int t = 0;
            for (; t + 1 < d; t += 2) {
                const bool l0 = t < i, l1 = t + 1 < i;
                const float a0 = l0 ? sA[i + t * LDN] : sT[i + (t - i) * LDN];
                const float b0 = l0 ? sT[t + j * LDN] : sB[(t - i) + j * LDN];
                const float a1 = l1 ? sA[i + (t + 1) * LDN] : sT[i + (t + 1 - i) * LDN];
                const float b1 = l1 ? sT[t + 1 + j * LDN] : sB[(t + 1 - i) + j * LDN];
                s0 = fmaf(a0, b0, s0);
                s1 = fmaf(a1, b1, s1);
            }
            if (t < d) {
                const bool l0 = t < i;
                const float a0 = l0 ? sA[i + t * LDN] : sT[i + (t - i) * LDN];
                const float b0 = l0 ? sT[t + j * LDN] : sB[(t - i) + j * LDN];
                s0 = fmaf(a0, b0, s0);
            }
            sT[i + j * LDN] = (sT[i + j * LDN] - (s0 + s1)) * sR[i + j * LDN];
        }
        __syncwarp();
    }
#pragma unroll 8
    for (int y = 0; y < nJ; ++y) {
        const int x = lane;
        if (x < mI) W[(i0 + x) + (long)(j0 + y) * ldn] = sT[x + y * LDN];
    }
    __syncwarp();
}

// Low-precision solve of L D + D U = W (in place), block anti-diagonals in
// order, their blocks spread over the CTA's warps.
template <int WPC, bool LYAP>
__device__ void wsolve(int n, const float *Lf, const float *Uf, const float *R, float *W, float *smem)
{
    const int warp = threadIdx.x >> 5;
    float *sm = smem + warp * SLOTS * TILE;
    const int nb = (n + BW - 1) / BW;
    for (int D = 0; D <= 2 * nb - 2; ++D) {
        const int ilo = max(LYAP ? (D + 1) / 2 : 0, D - nb + 1), ihi = min(D, nb - 1);
        for (int I = ilo + warp; I <= ihi; I += WPC) warp_block<LYAP>(n, I, D - I, Lf, Uf, R, W, sm);
        __syncthreads();
    }
}

// Double-float operand tile staged k-major by one warp from an FP64 block
// scaled by 2^sh (rows x cols valid; triangle / symmetric-mirror fills as in
// the blocked path).
__device__ __forceinline__ void wstage_df(float2 *S, const double *G, long ld, int rows, int cols, Fill f,
                                          bool asA, bool trans, int sh)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 8
    for (int y = 0; y < BW; ++y) {
        const int x = lane;
        float2 v = make_float2(0.f, 0.f);
        bool keep = x < rows && y < cols;
        if (keep && f == F_LOWER) keep = x >= y;
        if (keep && f == F_UPPER) keep = x <= y;
        if (keep) {
            const long idx = (f == F_SYM_LOWER && x < y) ? (y + (long)x * ld) : (x + (long)y * ld);
            split_df_s(G[idx], sh, v.x, v.y);
        }
        // source element (x, y): as op(A)(r = x, k = y); as op(B)(k = x, c = y),
        // or transposed op(B)(k = y, c = x).
        if (asA) S[x + y * LDK] = v;
        else if (!trans) S[y + x * LDK] = v;
        else S[x + y * LDK] = v;
    }
}

__device__ __forceinline__ void wmicro_df(float (&h)[4][8], float (&l)[4][8], const float2 *A, const float2 *B,
                                          int kk)
{
    const int r0 = lane_r0(), c0 = lane_c0();
#pragma unroll 1
    for (int k = 0; k < kk; ++k) {
        float2 a[4], b[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[r0 + i + k * LDK];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = B[c0 + j + k * LDK];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) df_msub(h[i][j], l[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
    }
}

// Residual block (I, J) by one warp into W (ld n), in the scaled units of sc.
template <bool LYAP>
__device__ void warp_residual_block(int n, int I, int J, const double *L, long ldl, const double *U, long ldu,
                                    const double *C, long ldc, const double *X, long ldx, float *W, float *sm,
                                    const DfScale &sc)
{
    float2 *sA = reinterpret_cast<float2 *>(sm), *sB = sA + TILE;
    const int i0 = I * BW, j0 = J * BW;
    const int mI = min(BW, n - i0), nJ = min(BW, n - j0);
    const int r0 = lane_r0(), c0 = lane_c0();
    float h[4][8], l[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int r = r0 + i, c = c0 + j;
            h[i][j] = 0.f;
            l[i][j] = 0.f;
            if (r < mI && c < nJ) {
                if (LYAP && I == J && r < c) { const int t = r; r = c; c = t; }
                split_df_s(C[(i0 + r) + (long)(j0 + c) * ldc], sc.rhs, h[i][j], l[i][j]);
            }
        }
    for (int K = 0; K <= I; ++K) {                          // L_IK X_KJ
        const int k0 = K * BW, kw = min(BW, n - k0);
        __syncwarp();
        wstage_df(sA, L + i0 + (long)k0 * ldl, ldl, mI, kw, K == I ? F_LOWER : F_FULL, true, false, sc.op);
        if (!LYAP || K > J) wstage_df(sB, X + k0 + (long)j0 * ldx, ldx, kw, nJ, F_FULL, false, false, sc.x);
        else if (K == J) wstage_df(sB, X + j0 + (long)j0 * ldx, ldx, kw, nJ, F_SYM_LOWER, false, false, sc.x);
        else wstage_df(sB, X + j0 + (long)k0 * ldx, ldx, nJ, kw, F_FULL, false, true, sc.x);
        __syncwarp();
        wmicro_df(h, l, sA, sB, kw);
    }
    for (int K = 0; K <= J; ++K) {                          // X_IK U_KJ
        const int k0 = K * BW, kw = min(BW, n - k0);
        __syncwarp();
        if (LYAP && K == I) wstage_df(sA, X + i0 + (long)i0 * ldx, ldx, mI, kw, F_SYM_LOWER, true, false, sc.x);
        else wstage_df(sA, X + i0 + (long)k0 * ldx, ldx, mI, kw, F_FULL, true, false, sc.x);
        if (!LYAP) wstage_df(sB, U + k0 + (long)j0 * ldu, ldu, kw, nJ, K == J ? F_UPPER : F_FULL, false, false, sc.op);
        else wstage_df(sB, L + j0 + (long)k0 * ldl, ldl, nJ, kw, K == J ? F_LOWER : F_FULL, false, true, sc.op);
        __syncwarp();
        wmicro_df(h, l, sA, sB, kw);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = r0 + i, c = c0 + j;
            if (r < mI && c < nJ) W[(i0 + r) + (long)(j0 + c) * n] = __fadd_rn(h[i][j], l[i][j]);
        }
    __syncwarp();
}

// All residual blocks (Lyapunov: the lower ones), largest first, over the
// warps; one barrier at the end.
template <int WPC, bool LYAP>
__device__ void wresidual(int n, const double *L, long ldl, const double *U, long ldu, const double *C,
                          long ldc, const double *X, long ldx, float *W, float *smem, const DfScale &sc)
{
    const int warp = threadIdx.x >> 5;
    float *sm = smem + warp * SLOTS * TILE;
    const int nb = (n + BW - 1) / BW;
    // Enumerate blocks by decreasing I + J (the K extent), round-robin to warps.
    int q = 0;
    for (int D = 2 * nb - 2; D >= 0; --D) {
        const int ilo = max(LYAP ? (D + 1) / 2 : 0, D - nb + 1), ihi = min(D, nb - 1);
        for (int I = ilo; I <= ihi; ++I, ++q)
            if (q % WPC == warp) warp_residual_block<LYAP>(n, I, D - I, L, ldl, U, ldu, C, ldc, X, ldx, W, sm, sc);
    }
    __syncthreads();
}

// ---- Tensor-memory low-precision solve (n <= 128) -------------------------
//
// TMEM holds -R' (rows = lanes, 128 columns), R' the right-hand side less
// every trailing update applied so far.  Block column K (k0 = 32 K):
//   * the diagonal block D_KK, then the column chain D_IK (I > K; warp I,
//     the owner of those lanes): T = R'_IK - sum_{K <= K' < I} L_IK' D_K'K,
//     solved as L_II D + D U_KK = T by the block wavefront; for Sylvester
//     also the row chain D_KJ (J > K; warp K): T = R'_KJ - sum D_KK' U_K'J;
//   * the trailing update of every block (I, J), I, J > K, by the tensor
//     cores: R' -= L_p D_r + D_c U_r  (Sylvester) or L_p D_c^T + D_c L_p^T
//     (Lyapunov), with L_p / D_c the block column K of L / D below the
//     block and D_r / U_r the block row K right of it, as one MMA sequence
//     [L_p | D_c] [D_r^T | U_r^T]^T of K = 64 into the TMEM columns right of
//     the block (Lyapunov: one operand buffer, read with its two K halves
//     swapped for B).
// The operand buffers overlay the warps' tiles (idle while the MMAs run).
// The kernel runs one CTA per SM (TMEM); it has TC_WARPS warps so that the
// double-float residual and the other CTA-wide phases fill the SM, while the
// TMEM traffic and the block chains stay on warps 0..3 (warp w reaches lane
// quarter w % 4 only).
constexpr int TC_MAXN = 128, TC_WARPS = 12, TC_THREADS = 32 * TC_WARPS;

// The block (I, J) of the chain of block column K, by the warp owning lanes
// 32 I .. 32 I + 31.
template <bool LYAP>
__device__ void tblock(int n, int I, int J, int K, const float *Lf, const float *Uf, const float *R, float *W,
                       float *sm, uint32_t tbase)
{
    float *sA = sm, *sB = sm + TILE, *sT = sm + 2 * TILE, *sR = sm + 3 * TILE;
    const int lane = threadIdx.x & 31;
    const long ldn = n;
    const int i0 = I * BW, j0 = J * BW;
    const int mI = min(BW, n - i0), nJ = min(BW, n - j0);
    const int r0 = lane_r0(), c0 = lane_c0();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float v[16];
        tc::ld16(tc::taddr(tbase, I, j0 + 16 * h), v);
#pragma unroll
        for (int q = 0; q < 16; ++q) sT[lane + (16 * h + q) * LDN] = -v[q];
    }
    __syncwarp();
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = sT[(r0 + i) + (c0 + j) * LDN];
    if (I > J) {
        for (int Kp = K; Kp < I; ++Kp) {          // L_IK' D_K'K
            const int k0 = Kp * BW;
            __syncwarp();
            wstage_A<false>(sA, Lf + i0 + (long)k0 * ldn, ldn, mI, BW);
            wstage_B<false>(sB, W + k0 + (long)j0 * ldn, ldn, BW, nJ);
            __syncwarp();
            wmicro_f(acc, sA, sB, BW);
        }
    } else if (J > I) {
        for (int Kp = K; Kp < J; ++Kp) {          // D_KK' U_K'J
            const int k0 = Kp * BW;
            __syncwarp();
            wstage_A<false>(sA, W + i0 + (long)k0 * ldn, ldn, mI, BW);
            wstage_B<false>(sB, Uf + k0 + (long)j0 * ldn, ldn, BW, nJ);
            __syncwarp();
            wmicro_f(acc, sA, sB, BW);
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sT[(r0 + i) + (c0 + j) * LDN] = acc[i][j];
#pragma unroll 8
    for (int y = 0; y < BW; ++y) {
        const int x = lane;
        sA[x + y * LDN] = (x < mI && y < mI && x > y) ? Lf[(i0 + x) + (long)(i0 + y) * ldn] : 0.0f;
        sB[x + y * LDN] = (x < nJ && y < nJ && x < y) ? Uf[(j0 + x) + (long)(j0 + y) * ldn] : 0.0f;
        sR[x + y * LDN] = (x < mI && y < nJ) ? R[(i0 + x) + (long)(j0 + y) * ldn] : 0.0f;
    }
    __syncwarp();
    for (int d = 0; d <= mI + nJ - 2; ++d) {
        const int j = lane, i = d - j;
        if (j < nJ && i >= 0 && i < mI) {
            float s0 = 0.0f, s1 = 0.0f;
            int t = 0;
            for (; t + 1 < d; t += 2) {
                const bool l0 = t < i, l1 = t + 1 < i;
                const float a0 = l0 ? sA[i + t * LDN] : sT[i + (t - i) * LDN];
                const float b0 = l0 ? sT[t + j * LDN] : sB[(t - i) + j * LDN];
                const float a1 = l1 ? sA[i + (t + 1) * LDN] : sT[i + (t + 1 - i) * LDN];
                const float b1 = l1 ? sT[t + 1 + j * LDN] : sB[(t + 1 - i) + j * LDN];
                s0 = fmaf(a0, b0, s0);
                s1 = fmaf(a1, b1, s1);
            }
            if (t < d) {
                const bool l0 = t < i;
                const float a0 = l0 ? sA[i + t * LDN] : sT[i + (t - i) * LDN];
                const float b0 = l0 ? sT[t + j * LDN] : sB[(t - i) + j * LDN];
                s0 = fmaf(a0, b0, s0);
            }
            sT[i + j * LDN] = (sT[i + j * LDN] - (s0 + s1)) * sR[i + j * LDN];
        }
        __syncwarp();
    }
#pragma unroll 8
    for (int y = 0; y < nJ; ++y) {
        const int x = lane;
        if (x < mI) W[(i0 + x) + (long)(j0 + y) * ldn] = sT[x + y * LDN];
    }
    __syncwarp();
}

struct TcSolve {
    uint32_t base;       // TMEM columns (128)
    uint64_t *mbar;
    uint32_t phase;
};

// Low-precision solve of L D + D U = W in place (n <= 128) with the
// right-hand side in TMEM.  `smem` is 1024-byte aligned, the warps' tiles.
// Returns false if a bounded wait for the tensor cores ran out.
template <bool LYAP, int KIND>
__device__ bool tsolve(int n, const float *Lf, const float *Uf, const float *R, float *W, float *smem, TcSolve &t)
{
    constexpr int KT = 2 * BW, S = KT / tc::KindTraits<KIND>::KSTEP;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *sm = smem + warp * SLOTS * TILE;
    unsigned char *za = reinterpret_cast<unsigned char *>(smem);
    unsigned char *zb = za + (size_t)TC_MAXN * KT * tc::KindTraits<KIND>::ES;
    const int nb = (n + BW - 1) / BW, nr = (n + 15) & ~15;
    if (warp < 4) {
        const int i = 32 * warp + lane;
        for (int cc = 0; cc < nr; cc += 16) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = cc + q;
                v[q] = (i < n && j < n) ? -W[i + (long)j * n] : 0.0f;
            }
            tc::st16(tc::taddr(t.base, warp, cc), v);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    for (int K = 0; K < nb; ++K) {
        const int k0 = K * BW, c0 = k0 + BW;
        if (warp == K) tblock<LYAP>(n, K, K, K, Lf, Uf, R, W, sm, t.base);
        __syncthreads();
        for (int s = 1; K + s < nb; ++s) {
            if (warp == K + s) tblock<LYAP>(n, K + s, K, K, Lf, Uf, R, W, sm, t.base);
            if (!LYAP && warp == K) tblock<LYAP>(n, K, K + s, K, Lf, Uf, R, W, sm, t.base);
            __syncthreads();
        }
        if (c0 >= n) break;
        // Operands: A row r = [L(r, k0..) | D(r, k0..)] for c0 <= r < n;
        // Sylvester B row r = [D(k0.., r) | U(k0.., r)], Lyapunov B = A with
        // its K halves swapped.
        for (int e = tid; e < TC_MAXN * KT; e += TC_THREADS) {
            const int r = e % TC_MAXN, k = e / TC_MAXN;
            float v = 0.0f;
            if (r >= c0 && r < n) v = k < BW ? Lf[r + (long)(k0 + k) * n] : W[r + (long)(k0 + k - BW) * n];
            tc::op_store<KIND>(za, r, k, KT, v);
        }
        if (!LYAP) {
            for (int e = tid; e < TC_MAXN * KT; e += TC_THREADS) {
                const int k = e % KT, r = e / KT;
                float v = 0.0f;
                if (r >= c0 && r < n) v = k < BW ? W[(k0 + k) + (long)r * n] : Uf[(k0 + k - BW) + (long)r * n];
                tc::op_store<KIND>(zb, r, k, KT, v);
            }
        }
        tc::fence_smem_to_async();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const uint32_t id = tc::idesc<KIND>(128, nr - c0, false);
#pragma unroll
            for (int sk = 0; sk < S; ++sk) {
                const uint64_t a = tc::op_desc<KIND>(za, 0, sk, KT);
                const uint64_t b = LYAP ? tc::op_desc<KIND>(za, c0, (sk + S / 2) % S, KT)
                                        : tc::op_desc<KIND>(zb, c0, sk, KT);
                tc::mma<KIND>(t.base + c0, a, b, id, true);
            }
            tc::commit(t.mbar);
        }
        const bool ok = tc::mbar_wait(t.mbar, t.phase);
        if (__syncthreads_or(!ok)) {
            tc::mbar_wait(t.mbar, t.phase, 1u << 26);
            return false;
        }
        t.phase ^= 1u;
        tc::fence_after();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return true;
}

template <int WPC, bool LYAP, int TCK = -1>
__device__ bool warp_instance(int n, const double *L, long ldl, const double *U, long ldu, const double *C,
                              long ldc, double *X, long ldx, int *info, float *W, bool raw, float *smem,
                              TcSolve *ts = nullptr)
{
    constexpr int T = 32 * WPC;
    const long nn = (long)n * n;
    float *R = W + nn, *Lf = W + 2 * nn, *Uf = W + 3 * nn;
    float *s_red = smem + WPC * SLOTS * TILE;
    const DfScale sc = instance_scale<T, LYAP>(n, L, ldl, U, ldu, C, ldc, s_red);
    const int bad = reciprocal_divisors<T, LYAP>(n, L, ldl, U, ldu, R, s_red, sc.op);
#pragma unroll 4
    for (long e = threadIdx.x; e < nn; e += T) {
        const int a = (int)(e % n), b = (int)(e / n);
        Lf[e] = a > b ? d2f_trunc_s(L[a + (long)b * ldl], sc.op) : 0.0f;
        const double u = LYAP ? L[b + (long)a * ldl] : U[a + (long)b * ldu];
        Uf[e] = a < b ? d2f_trunc_s(u, sc.op) : 0.0f;
        const double c = (LYAP && a < b) ? C[b + (long)a * ldc] : C[a + (long)b * ldc];
        W[e] = d2f_trunc_s(c, sc.rhs);
    }
    __syncthreads();
    auto solve = [&]() -> bool {
        if constexpr (TCK >= 0) {
            if (n <= TC_MAXN) return tsolve<LYAP, TCK>(n, Lf, Uf, R, W, smem, *ts);
        }
        wsolve<WPC, LYAP>(n, Lf, Uf, R, W, smem);
        return true;
    };
    if (!solve()) {
        if (threadIdx.x == 0) *info = SS_INFO_TIMEOUT;
        return false;
    }
    const float nx = sqrtf(update_x<T, LYAP>(n, X, ldx, W, n, true, s_red, sc.x));
    int conv = nx == 0.0f || raw;
    float prev = nx;
    for (int it = 0; it < MAXIT && !conv; ++it) {
        wresidual<WPC, LYAP>(n, L, ldl, U, ldu, C, ldc, X, ldx, W, smem, sc);
        if (LYAP) {
            for (long e = threadIdx.x; e < nn; e += T) {
                const int a = (int)(e % n), b = (int)(e / n);
                if (a < b) W[e] = W[b + (long)a * n];
            }
            __syncthreads();
        }
        if (!solve()) {
            if (threadIdx.x == 0) *info = SS_INFO_TIMEOUT;
            return false;
        }
        const float nd = sqrtf(update_x<T, LYAP>(n, X, ldx, W, n, false, s_red, sc.x));
        const float pred = prev > 0.0f ? nd * (nd / prev) : nd;
        conv = (nd <= (float)SS_REFINE_TOL * nx) || (pred <= (float)SS_REFINE_TOL * nx);
        prev = nd;
    }
    if (threadIdx.x == 0) *info = bad ? 1 : (conv ? 0 : n + 1);
    return true;
}

template <int WPC, bool LYAP>
__global__ void __launch_bounds__(32 * WPC) warp_syl_kernel(Operands o, Sched s, int group, int raw)
{
    extern __shared__ __align__(16) float smf[];
    __shared__ int s_slot;
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    claim_init(&s_slot);
    for (;;) {
        const int w = lo + claim_slot(s.meta + META_HEAD + group, &s_slot);
        if (w >= hi) break;
        const int b = s.perm[w];
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        // The refinement reads the original right-hand side at every step,
        // so it cannot run in place: an aliased X is left untouched.
        if (!raw && o.X[b] == o.C[b]) { if (threadIdx.x == 0) o.info[b] = SS_INFO_ALIASED; continue; }
        const long long off = s.scr[w];
        if (off + 4ll * n * n > s.scratch_elems) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
            continue;
        }
        float *W = static_cast<float *>(s.scratch) + off;
        warp_instance<WPC, LYAP>(n, o.A[b], o.lda[b], LYAP ? nullptr : o.U[b], LYAP ? 0 : o.ldu[b], o.C[b],
                                 o.ldc[b], o.X[b], o.ldx[b], o.info + b, W, raw != 0, smf);
    }
}

// Tensor-memory configurations: four warps, TMEM (128 columns) held for the
// whole launch; instances with n > 128 take the warp-block wavefront.
template <bool LYAP, int P>
__global__ void __launch_bounds__(TC_THREADS) warp_tc_kernel(Operands o, Sched s, int group, int raw)
{
    constexpr int KIND = P == P_TF32 ? tc::K_TF32 : tc::K_BF16;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_slot;
    __shared__ uint64_t s_mbar;
    __shared__ uint32_t s_tmem;
    float *smf = reinterpret_cast<float *>(smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u));
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    claim_init(&s_slot);
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&s_tmem, 128);
    if (threadIdx.x == 0) tc::mbar_init(&s_mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    TcSolve ts{s_tmem, &s_mbar, 0u};
    for (;;) {
        const int w = lo + claim_slot(s.meta + META_HEAD + group, &s_slot);
        if (w >= hi) break;
        const int b = s.perm[w];
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        if (!raw && o.X[b] == o.C[b]) { if (threadIdx.x == 0) o.info[b] = SS_INFO_ALIASED; continue; }
        const long long off = s.scr[w];
        if (off + 4ll * n * n > s.scratch_elems) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
            continue;
        }
        float *W = static_cast<float *>(s.scratch) + off;
        if (!warp_instance<TC_WARPS, LYAP, KIND>(n, o.A[b], o.lda[b], LYAP ? nullptr : o.U[b], LYAP ? 0 : o.ldu[b],
                                          o.C[b], o.ldc[b], o.X[b], o.ldx[b], o.info + b, W, raw != 0, smf, &ts))
            break;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(s_tmem, 128);
}

template <bool LYAP, int P>
cudaError_t launch_warp_tc(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, int raw)
{
    auto kern = warp_tc_kernel<LYAP, P>;
    const size_t smem = smem_bytes(TC_WARPS) + 1024;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TC_THREADS, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm > 4 ? 4 : (per_sm < 1 ? 1 : per_sm);   // 4 x 128 TMEM columns per SM
    long grid = (long)per_sm * sm_count();
    if (grid > l.batch) grid = l.batch;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, TC_THREADS, smem, st>>>(o, s, l.group, raw);
    return cudaGetLastError();
}

template <int WPC, bool LYAP>
cudaError_t launch_warp_syl(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, int raw)
{
    auto kern = warp_syl_kernel<WPC, LYAP>;
    const size_t smem = smem_bytes(WPC);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WPC, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long grid = (long)per_sm * sm_count();
    if (grid > l.batch) grid = l.batch;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, 32 * WPC, smem, st>>>(o, s, l.group, raw);
    return cudaGetLastError();
}

}  // namespace wb
}  // namespace mx
}  // namespace ss
