// Triangular Sylvester (L X + X U = C), Lyapunov (L X + X L^T = S) and
// Cholesky with warp-specialised CTAs, in FP64 or double-float arithmetic.
//
// The blocked lazy algorithm (the Bartels-Stewart back substitution of the
// paper's triangular Sylvester and Lyapunov solves, done block by block)
// alternates two kinds of work per B x B block (I, J):
//
//   T_IJ = C_IJ - sum_{K<I} L_IK X_KJ - sum_{K<J} X_IK U_KJ   (block updates)
//   L_II X_IJ + X_IJ U_JJ = T_IJ                             (diagonal block)
//
// The updates are plain FMA streams; the diagonal-block solve is a wavefront
// whose dependent chain of FP64 operations, queued behind other warps' FMAs in
// the SM's narrow FP64 pipe, makes it latency-bound.  Done one after the other
// under CTA-wide barriers (solve_fp64.cu), the update warps sit idle during
// every wavefront.  Here warp 0 (the diagonal warp) only solves diagonal
// blocks and warps 1..NU (the update warps) only form right-hand sides, in the
// same row-by-row block order.  While the diagonal warp solves block t, the
// update warps already form T for block t+1 except the one term that needs
// X of block t (K = J-1 of the second sum), which they add as soon as block t
// is done.  The two roles meet at two named barriers per block:
//
//   barrier 2 "T ready": update warps arrive, the diagonal warp waits;
//   barrier 3 "X ready": the diagonal warp arrives, the update warps wait.
//
// Each role makes exactly one arrival at each of them per block (the update
// warps wait once more after their last block), so the phases of a barrier
// never overlap.  Barrier 1 synchronises the update warps' tile staging.
// T and X of consecutive blocks alternate between two shared tiles.
//
// The same pipelines with double-float arithmetic (SS_MODE_DF, template flag
// DF): the block updates run as TwoProduct / TwoSum updates on the FP32 pipe,
// which on this GPU is 58 times wider than the FP64 pipe; for Sylvester /
// Lyapunov the diagonal-block wavefront does too, on operands the update
// warps prepare; divisions, square roots and pivots stay FP64.  The warp
// roles, barriers and block order are the FP64 ones.  The warp-specialised
// Cholesky (X^T X = A) follows the Sylvester kernel.
#include <type_traits>

#include "df.cuh"
#include "ss_internal.h"
#include "ss_device.cuh"

namespace ss {
namespace {

constexpr int kBarUpd = 1, kBarT = 2, kBarX = 3;

__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int count)
{
    __threadfence_block();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A double tile's memory as double-float pairs (same size per element).
__device__ __forceinline__ float2 *df2(double *p) { return reinterpret_cast<float2 *>(p); }
__device__ __forceinline__ const float2 *df2(const double *p) { return reinterpret_cast<const float2 *>(p); }

// Largest |p_ii| over i < n (all threads of the CTA take part).
__device__ __forceinline__ double max_abs_diag(const double *P, long ld, int n, double *s_red)
{
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(P[i + (long)i * ld]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, s_red[w]);
    __syncthreads();
    return r;
}

// ------------------------------------------------------------ diagonal warp

// Stage the lower (lower = true) or upper triangle of the m x m block at G
// into tile S with the 32 lanes of one warp; zero elsewhere.
template <int B>
__device__ __forceinline__ void warp_stage_tri(double *S, const double *G, long ldg, int m, bool lower, int lane)
{
    constexpr int LD = Tile<B>::LD;
    for (int e = lane; e < B * B; e += 32) {
        const int r = e % B, c = e / B;
        const bool keep = lower ? (r >= c) : (r <= c);
        S[r + c * LD] = (r < m && c < m && keep) ? G[r + (long)c * ldg] : 0.0;
    }
}

// In place: Lt Y + Y Ut = T for the m x nn block in sT, Lt = sL lower, Ut =
// sU upper or (UT) the transpose of the lower sU, reciprocal divisors in sR.
// Anti-diagonal d = i + j at a time; each entry is a dot product of d terms,
// split over `split` lanes (power of two, at most 32 / entries and at most
// d) with two partial sums per lane to halve the dependent chain.  SYM (a
// Lyapunov diagonal block, Ut = Lt^T, Y symmetric): only the entries i >= j
// are solved and read; y_tj with t < j is read as y_jt.
template <int B, bool UT, bool SYM>
__device__ void warp_diag_solve(const double *sL, const double *sU, double *sT, const double *sR, int m,
                                int nn, int lane)
{
    constexpr int LD = Tile<B>::LD;
    for (int d = 0; d <= m + nn - 2; ++d) {
        const int ilo = SYM ? max((d + 1) / 2, d - nn + 1) : max(0, d - nn + 1), ihi = min(d, m - 1);
        const int cnt = ihi - ilo + 1;
        // split = min(pow2_floor(32 / cnt), pow2_floor(d)), a power of two:
        // shifts and masks instead of divisions on the dependent chain.
        int split = cnt >= 32 ? 1 : (32 >> ceil_log2(cnt));
        const int byLen = pow2_floor(d > 1 ? d : 1);
        split = split < byLen ? split : byLen;
        const int lg = 31 - __clz(split);
        const int idx = lane >> lg, part = lane & (split - 1);
        const bool act = idx < cnt;
        const int i = ilo + (act ? idx : 0), j = d - i;
        double s0 = 0.0, s1 = 0.0;
        if (act) {
            int t = part;
            for (; t + split < d; t += 2 * split) {
                const int t1 = t + split;
                const double a0 = t < i ? sL[i + t * LD] : sT[i + (t - i) * LD];
                const double b0 = t < i ? (SYM && t < j ? sT[j + t * LD] : sT[t + j * LD])
                                        : (UT ? sU[j + (t - i) * LD] : sU[(t - i) + j * LD]);
                const double a1 = t1 < i ? sL[i + t1 * LD] : sT[i + (t1 - i) * LD];
                const double b1 = t1 < i ? (SYM && t1 < j ? sT[j + t1 * LD] : sT[t1 + j * LD])
                                         : (UT ? sU[j + (t1 - i) * LD] : sU[(t1 - i) + j * LD]);
                s0 = fma(a0, b0, s0);
                s1 = fma(a1, b1, s1);
            }
            if (t < d) {
                const double a0 = t < i ? sL[i + t * LD] : sT[i + (t - i) * LD];
                const double b0 = t < i ? (SYM && t < j ? sT[j + t * LD] : sT[t + j * LD])
                                        : (UT ? sU[j + (t - i) * LD] : sU[(t - i) + j * LD]);
                s0 = fma(a0, b0, s0);
            }
        }
        const double s = group_sum(s0 + s1, split);
        if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * sR[i + j * LD];
        __syncwarp();
    }
}

// Double-float form of warp_diag_solve for the DF pipeline: T and X in sT,
// the strict lower triangle of Lt and the strict upper triangle of Ut in one
// tile sLU, reciprocal divisors in sR, all as (hi, lo) float pairs with
// leading dimension LDT.  The lane that finishes entry (i, j) starts its sum at
// t_ij; x_ij = (t_ij - sum) * r_ij is a normalised double-float product.  One
// accumulator per lane: the loop-carried chain of a double-float term is one
// addition on each half, so a second one would only add the merge.  Only the
// FP32 pipe is used.
template <int B, int LDT, bool SYM>
__device__ void warp_diag_solve_df(const float2 *sLU, float2 *sT, const float2 *sR, int m, int nn, int lane)
{
    for (int d = 0; d <= m + nn - 2; ++d) {
        const int ilo = SYM ? max((d + 1) / 2, d - nn + 1) : max(0, d - nn + 1), ihi = min(d, m - 1);
        const int cnt = ihi - ilo + 1;
        // split = min(pow2_floor(32 / cnt), pow2_floor(d)), a power of two:
        // shifts and masks instead of divisions on the dependent chain.
        int split = cnt >= 32 ? 1 : (32 >> ceil_log2(cnt));
        const int byLen = pow2_floor(d > 1 ? d : 1);
        split = split < byLen ? split : byLen;
        const int lg = 31 - __clz(split);
        const int idx = lane >> lg, part = lane & (split - 1);
        const bool act = idx < cnt;
        const int i = ilo + (act ? idx : 0), j = d - i;
        float h0 = 0.f, l0 = 0.f;
        if (act) {
            if (part == 0) {
                const float2 tv = sT[i + j * LDT];
                h0 = tv.x;
                l0 = tv.y;
            }
            int t = part;
            if constexpr (!SYM) {
                // Offsets from sT: term t reads L_it (sLU) and Y_tj (sT) for
                // t < i, Y_i,t-i (sT) and U_t-i,j (sLU) from t = i on, that
                // is base + t * LDT and base + t with the bases of its part.
                const int dlu = (int)(sLU - sT);
                const int aL = dlu + i, aU = i - i * LDT, bL = j * LDT, bU = dlu - i + j * LDT;
                for (; t + split < d; t += 2 * split) {
                    const int t1 = t + split;
                    const float2 a0 = sT[(t < i ? aL : aU) + t * LDT], b0 = sT[(t < i ? bL : bU) + t];
                    const float2 a1 = sT[(t1 < i ? aL : aU) + t1 * LDT], b1 = sT[(t1 < i ? bL : bU) + t1];
                    df_msub(h0, l0, a0.x, a0.y, b0.x, b0.y);
                    df_msub(h0, l0, a1.x, a1.y, b1.x, b1.y);
                }
                if (t < d) {
                    const float2 a0 = sT[(t < i ? aL : aU) + t * LDT], b0 = sT[(t < i ? bL : bU) + t];
                    df_msub(h0, l0, a0.x, a0.y, b0.x, b0.y);
                }
            } else {
                for (; t + split < d; t += 2 * split) {
                    const int t1 = t + split;
                    const float2 a0 = t < i ? sLU[i + t * LDT] : sT[i + (t - i) * LDT];
                    const float2 b0 = t < i ? (t < j ? sT[j + t * LDT] : sT[t + j * LDT]) : sLU[(t - i) + j * LDT];
                    const float2 a1 = t1 < i ? sLU[i + t1 * LDT] : sT[i + (t1 - i) * LDT];
                    const float2 b1 = t1 < i ? (t1 < j ? sT[j + t1 * LDT] : sT[t1 + j * LDT]) : sLU[(t1 - i) + j * LDT];
                    df_msub(h0, l0, a0.x, a0.y, b0.x, b0.y);
                    df_msub(h0, l0, a1.x, a1.y, b1.x, b1.y);
                }
                if (t < d) {
                    const float2 a0 = t < i ? sLU[i + t * LDT] : sT[i + (t - i) * LDT];
                    const float2 b0 = t < i ? (t < j ? sT[j + t * LDT] : sT[t + j * LDT]) : sLU[(t - i) + j * LDT];
                    df_msub(h0, l0, a0.x, a0.y, b0.x, b0.y);
                }
            }
        }
        df_group_sum(h0, l0, split);
        if (act && part == 0) {
            df_norm(h0, l0);
            const float2 r = sR[i + j * LDT];
            float2 x;
            df_mul(h0, l0, r.x, r.y, x.x, x.y);
            sT[i + j * LDT] = x;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------- update warps

// Outputs of one update thread: flat index e = ut + TU*r over the m x nn
// valid entries of the block (column-major), as in Slots.
template <int B, int TU>
struct OutMap {
    static constexpr int E = B * B / TU;
    int row[E], col[E];
    unsigned valid;
    bool same_row;    // every output in row row[0] (full blocks)
    __device__ __forceinline__ void set(int m, int nn, int ut)
    {
        same_row = m == B && TU % B == 0;
        valid = 0u;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = ut + TU * r;
            row[r] = 0;
            col[r] = 0;
            if (e < m * nn) {
                row[r] = e % m;
                col[r] = e / m;
                valid |= 1u << r;
            }
        }
    }
    // The m(m+1)/2 entries with row <= col of an m x m block (a Cholesky
    // diagonal block).
    __device__ __forceinline__ void set_upper(int m, int ut)
    {
        set_lower(m, ut);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int x = row[r];
            row[r] = col[r];
            col[r] = x;
        }
    }
    // The m(m+1)/2 entries with row >= col of an m x m block (a Lyapunov
    // diagonal block, whose upper part is the transpose).
    __device__ __forceinline__ void set_lower(int m, int ut)
    {
        same_row = false;
        valid = 0u;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = ut + TU * r;
            row[r] = 0;
            col[r] = 0;
            if (e < m * (m + 1) / 2) {
                int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
                while (c * (c + 1) / 2 > e) --c;
                while ((c + 1) * (c + 2) / 2 <= e) ++c;
                row[r] = c;
                col[r] = e - c * (c + 1) / 2;
                valid |= 1u << r;
            }
        }
    }
    __device__ __forceinline__ bool ok(int r) const { return (valid >> r) & 1u; }
};

// Where one operand tile of a block-update step comes from: rows x cols at
// P (leading dimension ld); sym: the symmetric diagonal block whose lower
// triangle is stored (rows = cols = m); sh: the operand's power-of-two shift
// in the double-float pipelines (DfScale; 0 and unused in FP64).
struct Src {
    const double *P;
    long ld;
    int rows, cols;
    bool sym;
    int sh;
};

// The tile elements one update thread loads: e = ut + TU*q, (r, c) = (e % B, e / B).
template <int B, int TU>
struct Prefetch {
    static constexpr int PE = B * B / TU;
    double a[PE], b[PE];

    __device__ __forceinline__ static double get(const Src &s, int r, int c)
    {
        if (r >= s.rows || c >= s.cols) return 0.0;
        if (s.sym && r < c) return s.P[c + (long)r * s.ld];
        return s.P[r + (long)c * s.ld];
    }
    __device__ __forceinline__ void load(const Src &sa, const Src &sb, bool has_a, int ut)
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            a[q] = has_a ? get(sa, r, c) : 0.0;
            b[q] = get(sb, r, c);
        }
    }
    __device__ __forceinline__ void store(double *tA, double *tB, bool has_a, int ut) const
    {
        constexpr int LD = Tile<B>::LD;
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            if (has_a) tA[r + c * LD] = a[q];
            tB[r + c * LD] = b[q];
        }
    }
    // The same tiles as double-float pairs (DF update warps), leading
    // dimension LDT, each operand scaled by 2^sha / 2^shb.
    template <int LDT>
    __device__ __forceinline__ void store_df(float2 *tA, float2 *tB, bool has_a, int ut, int sha, int shb) const
    {
        constexpr int LD = LDT;
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            float2 v;
            if (has_a) {
                split_df_s(a[q], sha, v.x, v.y);
                tA[r + c * LD] = v;
            }
            split_df_s(b[q], shb, v.x, v.y);
            tB[r + c * LD] = v;
        }
    }
    // Bulk-step tiles K-contiguous, for upd_dfk: op(A)(row, k) at
    // tA[k + row * LDT], op(B)(k, col) at tB[k + col * LDT] (tb: op(B) is the
    // staged tile transposed).
    template <int LDT>
    __device__ __forceinline__ void store_dfk(float2 *tA, float2 *tB, bool has_a, bool tb, int ut, int sha,
                                              int shb) const
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            float2 v;
            if (has_a) {
                split_df_s(a[q], sha, v.x, v.y);
                tA[c + r * LDT] = v;
            }
            split_df_s(b[q], shb, v.x, v.y);
            if (tb) tB[c + r * LDT] = v;
            else    tB[r + c * LDT] = v;
        }
    }
};

// Double-float Sylvester / Lyapunov pipeline: the operand tiles come from
// per-instance copies already split into double-float pairs (L and U when
// the instance starts, X as the diagonal warp finishes each block; see
// syl_ws_instance), so staging only copies.  Layout of the copies in the
// instance's scratch, leading dimensions m, n, m: L (m x m), U (n x n),
// X (m x n).
struct SrcF {
    const float2 *F;
    long ld;
    int rows, cols;
    bool sym;   // the symmetric diagonal block, its lower triangle stored
};

template <int B, int TU>
struct PrefetchF {
    static constexpr int PE = B * B / TU;
    float2 a[PE], b[PE];

    __device__ __forceinline__ static float2 get(const SrcF &s, int r, int c)
    {
        if (r >= s.rows || c >= s.cols) return make_float2(0.f, 0.f);
        if (s.sym && r < c) return s.F[c + (long)r * s.ld];
        return s.F[r + (long)c * s.ld];
    }
    __device__ __forceinline__ void load(const SrcF &sa, const SrcF &sb, bool has_a, int ut)
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            a[q] = has_a ? get(sa, r, c) : make_float2(0.f, 0.f);
            b[q] = get(sb, r, c);
        }
    }
    // Bulk-step tiles, K-contiguous (see upd_dfk).
    template <int LDT>
    __device__ __forceinline__ void store_k(float2 *tA, float2 *tB, bool tb, int ut) const
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            tA[c + r * LDT] = a[q];
            if (tb) tB[c + r * LDT] = b[q];
            else    tB[r + c * LDT] = b[q];
        }
    }
    // Both tiles in natural layout (the Cholesky pipeline's X_KI^T X_KJ).
    template <int LDT>
    __device__ __forceinline__ void store_nat(float2 *tA, float2 *tB, bool has_a, int ut) const
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            if (has_a) tA[r + c * LDT] = a[q];
            tB[r + c * LDT] = b[q];
        }
    }
    // The last phase's tile, natural layout.
    template <int LDT>
    __device__ __forceinline__ void store_b(float2 *tB, int ut) const
    {
#pragma unroll
        for (int q = 0; q < PE; ++q) {
            const int e = ut + TU * q, r = e % B, c = e / B;
            tB[r + c * LDT] = b[q];
        }
    }
};

// acc -= A * op(Bm) over B terms, A(row, k) = A[row + k*LD],
// op(Bm)(k, col) = TB ? Bm[col + k*LD] : Bm[k + col*LD]; even and odd k go to
// separate accumulators (two independent FMA chains per output).
template <int B, int TU, bool TB>
__device__ __forceinline__ void upd_fma(double (&ae)[B * B / TU], double (&ao)[B * B / TU],
                                        const OutMap<B, TU> &om, const double *A, const double *Bm)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int E = B * B / TU;
#pragma unroll 2
    for (int k = 0; k < B; k += 2) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (om.ok(r)) {
                const double a0 = A[om.row[r] + k * LD], a1 = A[om.row[r] + (k + 1) * LD];
                const double b0 = TB ? Bm[om.col[r] + k * LD] : Bm[k + om.col[r] * LD];
                const double b1 = TB ? Bm[om.col[r] + (k + 1) * LD] : Bm[k + 1 + om.col[r] * LD];
                ae[r] = fma(-a0, b0, ae[r]);
                ao[r] = fma(-a1, b1, ao[r]);
            }
        }
    }
}

// acc -= A^T * Bm over B terms: A(row, k) read as A[k + row*LD] (the tile
// holds X_KI, used as X_KI^T), Bm(k, col) = Bm[k + col*LD].
template <int B, int TU>
__device__ __forceinline__ void upd_fma_ta(double (&ae)[B * B / TU], double (&ao)[B * B / TU],
                                           const OutMap<B, TU> &om, const double *A, const double *Bm)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int E = B * B / TU;
#pragma unroll 2
    for (int k = 0; k < B; k += 2) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (om.ok(r)) {
                ae[r] = fma(-A[k + om.row[r] * LD], Bm[k + om.col[r] * LD], ae[r]);
                ao[r] = fma(-A[k + 1 + om.row[r] * LD], Bm[k + 1 + om.col[r] * LD], ao[r]);
            }
        }
    }
}

template <int B, int TU>
__device__ __forceinline__ void upd_fma_rt(bool tb, double (&ae)[B * B / TU], double (&ao)[B * B / TU],
                                           const OutMap<B, TU> &om, const double *A, const double *Bm)
{
    if (tb) upd_fma<B, TU, true>(ae, ao, om, A, Bm);
    else    upd_fma<B, TU, false>(ae, ao, om, A, Bm);
}

// Double-float forms of the three products above: (ah, al) -= A op(Bm) with
// A and Bm tiles of double-float pairs (leading dimension LDT); one
// TwoProduct / TwoSum update per term on the FP32 pipe.
template <int B, int TU, int LDT, bool TB>
__device__ __forceinline__ void upd_df(float (&ah)[B * B / TU], float (&al)[B * B / TU], const OutMap<B, TU> &om,
                                       const float2 *A, const float2 *Bm)
{
    constexpr int E = B * B / TU;
#pragma unroll 2
    for (int k = 0; k < B; ++k) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (om.ok(r)) {
                const float2 a = A[om.row[r] + k * LDT];
                const float2 b = TB ? Bm[om.col[r] + k * LDT] : Bm[k + om.col[r] * LDT];
                df_msub(ah[r], al[r], a.x, a.y, b.x, b.y);
            }
        }
    }
}

// (ah, al) -= op(A) op(B) over B terms from K-contiguous tiles (store_dfk):
// each 16-byte load brings two terms, and with om.same_row the A pair is
// loaded once for all of the thread's outputs.
template <int B, int TU, int LDT>
__device__ __forceinline__ void upd_dfk(float (&ah)[B * B / TU], float (&al)[B * B / TU], const OutMap<B, TU> &om,
                                        const float2 *A, const float2 *Bm)
{
    constexpr int E = B * B / TU;
    static_assert(B % 2 == 0 && LDT % 2 == 0, "16-byte pairs of terms");
#pragma unroll 1
    for (int k = 0; k < B; k += 2) {
        const float4 a0 = *reinterpret_cast<const float4 *>(A + k + om.row[0] * LDT);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (om.ok(r)) {
                const float4 a = (r == 0 || om.same_row) ? a0
                                                         : *reinterpret_cast<const float4 *>(A + k + om.row[r] * LDT);
                const float4 b = *reinterpret_cast<const float4 *>(Bm + k + om.col[r] * LDT);
                df_msub(ah[r], al[r], a.x, a.y, b.x, b.y);
                df_msub(ah[r], al[r], a.z, a.w, b.z, b.w);
            }
        }
    }
}

template <int B, int TU, int LDT>
__device__ __forceinline__ void upd_df_ta(float (&ah)[B * B / TU], float (&al)[B * B / TU], const OutMap<B, TU> &om,
                                          const float2 *A, const float2 *Bm)
{
    constexpr int E = B * B / TU;
#pragma unroll 2
    for (int k = 0; k < B; ++k) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (om.ok(r)) {
                const float2 a = A[k + om.row[r] * LDT];
                const float2 b = Bm[k + om.col[r] * LDT];
                df_msub(ah[r], al[r], a.x, a.y, b.x, b.y);
            }
        }
    }
}

// All update threads: the B x B double tile S as double-float pairs into D
// (both leading dimension LDT).
template <int B, int TU, int LDT>
__device__ __forceinline__ void tile_to_df(float2 *D, const double *S, int ut)
{
#pragma unroll
    for (int e = ut; e < B * B; e += TU) {
        const int r = e % B, c = e / B;
        float2 v;
        split_df_s(S[r + c * LDT], 0, v.x, v.y);
        D[r + c * LDT] = v;
    }
}

template <int B, int TU, int LDT>
__device__ __forceinline__ void upd_df_rt(bool tb, float (&ah)[B * B / TU], float (&al)[B * B / TU],
                                          const OutMap<B, TU> &om, const float2 *A, const float2 *Bm)
{
    if (tb) upd_df<B, TU, LDT, true>(ah, al, om, A, Bm);
    else    upd_df<B, TU, LDT, false>(ah, al, om, A, Bm);
}

// Operands of bulk step s of block (I, J): s < P1 is K = s of the first sum,
// then K = s - P1 (< J - 1) of the second.  P1 = I, except for a Lyapunov
// diagonal block, whose first-sum term K = I-1 reads X_{I-1,I} = X_{I,I-1}^T,
// the block solved just before it: that term joins the last phase.  *tb: use
// op(Bm) transposed.
template <int B, bool LYAP>
__device__ __forceinline__ void step_src(int s, int P1, int I, int J, int mI, int nJ, const double *L, long ldl,
                                         const double *U, long ldu, const double *X, long ldx, Src &a, Src &b,
                                         bool &tb, const DfScale &sc)
{
    const int i0 = I * B, j0 = J * B;
    if (s < P1) {
        const int k0 = s * B;
        a = Src{L + i0 + (long)k0 * ldl, ldl, mI, B, false, sc.op};         // L_IK
        if (!LYAP || s > J) {
            b = Src{X + k0 + (long)j0 * ldx, ldx, B, nJ, false, sc.x};       // X_KJ
            tb = false;
        } else if (s == J) {
            b = Src{X + j0 + (long)j0 * ldx, ldx, nJ, nJ, true, sc.x};       // X_JJ (symmetric)
            tb = false;
        } else {
            b = Src{X + j0 + (long)k0 * ldx, ldx, nJ, B, false, sc.x};       // X_JK, used transposed
            tb = true;
        }
    } else {
        const int k0 = (s - P1) * B;
        a = Src{X + i0 + (long)k0 * ldx, ldx, mI, B, false, sc.x};           // X_IK
        if (!LYAP) {
            b = Src{U + k0 + (long)j0 * ldu, ldu, B, nJ, false, sc.op};      // U_KJ
            tb = false;
        } else {
            b = Src{L + j0 + (long)k0 * ldl, ldl, nJ, B, false, sc.op};      // L_JK, used transposed
            tb = true;
        }
    }
}

// The staged tile of the last phase: U_{J-1,J} (Lyapunov: L_{J,J-1}, used
// transposed) for J > 0; for J = 0 (a first-sum term, see has_first_last):
// L_{I,I-1} (not transposed).
template <int B, bool LYAP>
__device__ __forceinline__ void last_src_t(int I, int J, int mI, int nJ, const double *L, long ldl,
                                           const double *U, long ldu, Src &b, bool &tb, const DfScale &sc)
{
    const int j0 = J * B;
    if (J == 0) {
        b = Src{L + I * B + (long)(I - 1) * B * ldl, ldl, mI, B, false, sc.op};
        tb = false;
        return;
    }
    const int k0 = (J - 1) * B;
    b = LYAP ? Src{L + j0 + (long)k0 * ldl, ldl, nJ, B, false, sc.op}
             : Src{U + k0 + (long)j0 * ldu, ldu, B, nJ, false, sc.op};
    tb = LYAP;
}

// step_src / last_src_t on the pre-split copies (dfw: L, then U, then X).
template <int B, bool LYAP>
__device__ __forceinline__ void step_src_f(int s, int P1, int I, int J, int mI, int nJ, int m, int n,
                                           const float2 *dfw, SrcF &a, SrcF &b, bool &tb)
{
    const int i0 = I * B, j0 = J * B;
    const float2 *Lf = dfw, *Uf = dfw + (long)m * m, *Xf = Uf + (long)n * n;
    if (s < P1) {
        const int k0 = s * B;
        a = SrcF{Lf + i0 + (long)k0 * m, m, mI, B, false};                 // L_IK
        if (!LYAP || s > J) {
            b = SrcF{Xf + k0 + (long)j0 * m, m, B, nJ, false};             // X_KJ
            tb = false;
        } else if (s == J) {
            b = SrcF{Xf + j0 + (long)j0 * m, m, nJ, nJ, true};             // X_JJ (symmetric)
            tb = false;
        } else {
            b = SrcF{Xf + j0 + (long)k0 * m, m, nJ, B, false};             // X_JK, used transposed
            tb = true;
        }
    } else {
        const int k0 = (s - P1) * B;
        a = SrcF{Xf + i0 + (long)k0 * m, m, mI, B, false};                 // X_IK
        if (!LYAP) {
            b = SrcF{Uf + k0 + (long)j0 * n, n, B, nJ, false};             // U_KJ
            tb = false;
        } else {
            b = SrcF{Lf + j0 + (long)k0 * m, m, nJ, B, false};             // L_JK, used transposed
            tb = true;
        }
    }
}

template <int B, bool LYAP>
__device__ __forceinline__ void last_src_f(int I, int J, int mI, int nJ, int m, int n, const float2 *dfw, SrcF &b,
                                           bool &tb)
{
    const int j0 = J * B;
    const float2 *Lf = dfw, *Uf = dfw + (long)m * m;
    if (J == 0) {
        b = SrcF{Lf + I * B + (long)(I - 1) * B * m, m, mI, B, false};
        tb = false;
        return;
    }
    const int k0 = (J - 1) * B;
    b = LYAP ? SrcF{Lf + j0 + (long)k0 * m, m, nJ, B, false} : SrcF{Uf + k0 + (long)j0 * n, n, B, nJ, false};
    tb = LYAP;
}

// Shared tiles of the warp-specialised kernels: FP64 uses nine tiles of
// Tile<B>; DF uses ten tiles of B x (B + 2) double-float pairs (an even
// leading dimension of 8-byte elements puts the entries of an anti-diagonal,
// which the wavefront reads together, in distinct banks).
template <int B, bool DF>
struct WsTile {
    static constexpr int LD = DF ? B + 2 : Tile<B>::LD;
    static constexpr int SZ = B * LD;
    static constexpr int N = DF ? 10 : 9;
};
template <int B, bool DF = false>
constexpr size_t ws_smem_bytes() { return (size_t)WsTile<B, DF>::N * WsTile<B, DF>::SZ * sizeof(double) + 32 * sizeof(double); }

// One instance.  X is m x n (L m x m, U n x n); Lyapunov has m = n.
// FP64 shared tiles: sT[2] (T / X of consecutive blocks), sL, sU, sR
// (diagonal warp), sA[2], sB[2] (update warps' staging).
// DF: the update warps form T in double-float arithmetic on the FP32 pipe
// (operands split on staging) and, for each block, also prepare the diagonal
// warp's operands in double-buffered tiles: sLU[t & 1] (strict lower L_II,
// strict upper U_JJ or L_JJ^T) and sR[t & 1] (1 / (l_ii + u_jj), divided in
// FP64, then split).  The diagonal warp then solves on the FP32 pipe only
// (warp_diag_solve_df) and writes X rounded to FP64.  sT holds T and X as
// double-float pairs, so the update warps' last phase reads X of block t-1
// without conversion.  Buffer t & 1 is free when block t starts: the diagonal
// warp last read it for block t-2, before the "X ready" arrival the update
// warps waited for in block t-1.
//
// DF status (the return value, valid on thread 0 only): 1 if some
// double-float intermediate left its range (df_out_of_range: a reciprocal
// divisor or an entry of X more than 2^60 times the rescaled data, or Inf /
// NaN), in which case X is not reliable and the caller solves the instance
// again in FP64; else 0.  The FP64 form always returns 0.
//
// DF without SC finds, in its first pass over the instance (the one that
// splits L and U), the largest exponents and diagonal magnitudes: data in
// DfScale's band is solved with the constant zero shifts, which keeps the
// pipeline's registers as without rescaling; other data returns 4 after
// writing its record (di) for the SC pass, which reads the shifts and the
// divisor threshold from there.
//
// PD = 2 (configurations for one or two CTAs per SM, where no other CTA
// hides a global load): the update warps load the operands of step s + 2
// while computing step s, through two register sets used alternately.
//
// DF: dfw, the instance's scratch for the pre-split copies (SrcF), holds
// m*m + n*n + m*n double-float pairs.
template <int B, int NU, bool LYAP, bool DF, bool SC = false, int PD = 1>
__device__ int syl_ws_instance(int m, int n, const double *L, long ldl, const double *U, long ldu,
                               const double *C, long ldc, double *X, long ldx, int *info, double *sm,
                               DfInst *di, float2 *dfw = nullptr)
{
    constexpr int LD = WsTile<B, DF>::LD, SZ = WsTile<B, DF>::SZ;
    constexpr int TU = 32 * NU, TALL = TU + 32;
    static_assert((B * B) % TU == 0, "update threads must divide the block");
    double *sT0 = sm, *sL = sm + 2 * SZ, *sU = sm + 3 * SZ, *sR = sm + 4 * SZ;
    double *sA0 = sm + 5 * SZ, *sB0 = sm + 7 * SZ;
    if constexpr (DF) {
        sA0 = sm + 6 * SZ;
        sB0 = sm + 8 * SZ;
    }
    double *s_red = sm + WsTile<B, DF>::N * SZ;
    int *s_bad = reinterpret_cast<int *>(s_red + 24);     // DF: a divisor check failed
    int *s_rng = reinterpret_cast<int *>(s_red + 25);     // DF: range left (see above)
    const int mb = (m + B - 1) / B, nb = (n + B - 1) / B;

    double delta;
    DfScale sc{0, 0, 0};
    if constexpr (DF) {
        if (threadIdx.x == 0) {
            *s_bad = 0;
            *s_rng = 0;
        }
        if constexpr (SC) {
            const DfInst d = *di;
            sc = DfScale::sylvester(d.eo, d.ec);
            delta = divisor_delta(max(m, n), __longlong_as_double((long long)d.maxdiag));
        }
        // One pass over L and U: split the strict triangles once (scaled;
        // the diagonal blocks' operands are prepared per block as before)
        // and, in the zero-shift pass, the largest exponents and diagonal
        // magnitudes that decide whether the instance needs rescaling
        // (Inf / NaN exponents are left to the range check, as in DfScale).
        int eo = 0, ec = 0;
        double md = 0.0;                                 // fmax drops NaN, as the FP64 solves' maximum does
        for (long e = threadIdx.x; e < (long)m * m; e += blockDim.x) {
            const int r = (int)(e % m), c = (int)(e / m);
            if (r >= c) {
                const double x = L[r + (long)c * ldl];
                if constexpr (!SC) {
                    const int ex = exp_bits(x);
                    eo = max(eo, ex == 0x7FF ? 0 : ex);
                    if (r == c) md = fmax(md, fabs(x));
                }
                if (r > c) {
                    float2 v;
                    split_df_s(x, sc.op, v.x, v.y);
                    dfw[e] = v;
                }
            }
        }
        if (!LYAP) {
            float2 *Uf = dfw + (long)m * m;
            for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
                const int r = (int)(e % n), c = (int)(e / n);
                if (r <= c) {
                    const double x = U[r + (long)c * ldu];
                    if constexpr (!SC) {
                        const int ex = exp_bits(x);
                        eo = max(eo, ex == 0x7FF ? 0 : ex);
                        if (r == c) md = fmax(md, fabs(x));
                    }
                    if (r < c) {
                        float2 v;
                        split_df_s(x, sc.op, v.x, v.y);
                        Uf[e] = v;
                    }
                }
            }
        }
        if constexpr (!SC) {
            const unsigned *hC = reinterpret_cast<const unsigned *>(C) + 1;   // high words
            for (long e = threadIdx.x; e < (long)m * n; e += blockDim.x) {
                const int r = (int)(e % m), c = (int)(e / m);
                if (LYAP && r < c) continue;                 // S: lower triangle
                const int ex = (int)((hC[2 * (r + (long)c * ldc)] >> 20) & 0x7FFu);
                ec = max(ec, ex == 0x7FF ? 0 : ex);
            }
            // CTA maxima: the exponents through s_red[0 .. 2 * warps) as ints,
            // the warps' md at s_red + 12; cta_max2's barriers also order the
            // split copies before the update warps read them.
            for (int k = 16; k > 0; k >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, k));
            if ((threadIdx.x & 31) == 0) s_red[12 + (threadIdx.x >> 5)] = md;
            cta_max2(eo, ec, reinterpret_cast<int *>(s_red));
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) md = fmax(md, s_red[12 + k]);
            if (!DfScale::sylvester(eo, ec).zero()) {
                if (threadIdx.x == 0) *di = DfInst{eo, ec, 1, 0, (unsigned long long)__double_as_longlong(md)};
                return 4;                                // to the rescaled pass (the same on every thread)
            }
            delta = divisor_delta(max(m, n), md);
        }
        __syncthreads();
    } else {
        double md = max_abs_diag(L, ldl, m, s_red);
        if (!LYAP) md = fmax(md, max_abs_diag(U, ldu, n, s_red));
        delta = divisor_delta(max(m, n), md);
    }

    if (threadIdx.x < 32) {
        // ------------------------------------------------ diagonal warp
        const int lane = threadIdx.x;
        int bad = 0, t = 0, rng = 0;
        for (int I = 0; I < mb; ++I) {
            const int mI = min(B, m - I * B), i0 = I * B;
            if constexpr (!DF) warp_stage_tri<B>(sL, L + i0 + (long)i0 * ldl, ldl, mI, true, lane);
            const int jend = LYAP ? I + 1 : nb;
            for (int J = 0; J < jend; ++J, ++t) {
                const int nJ = min(B, n - J * B), j0 = J * B;
                const bool sym = LYAP && I == J;
                double *sT = sT0 + (t & 1) * SZ;
                if constexpr (DF) {
                    named_sync(kBarT, TALL);               // T and the diagonal operands of block t
                    float2 *dT = df2(sT);
                    const float2 *dLU = df2(sL + (t & 1) * SZ), *dR = df2(sR + (t & 1) * SZ);
                    if (sym) {
                        warp_diag_solve_df<B, LD, true>(dLU, dT, dR, mI, nJ, lane);
                        for (int e = lane; e < mI * mI; e += 32) {
                            const int i = e % mI, j = e / mI;
                            if (i < j) dT[i + j * LD] = dT[j + i * LD];
                        }
                        __syncwarp();
                    } else {
                        warp_diag_solve_df<B, LD, false>(dLU, dT, dR, mI, nJ, lane);
                    }
                    // The pairs in scaled units first, for the update warps'
                    // staging of later blocks; then "X final" (the update
                    // warps read this block from shared memory); then X
                    // rounded to FP64 and its range check, while the update
                    // warps finish the next block's T.
                    float2 *dX = dfw + (long)m * m + (long)n * n + i0 + (long)j0 * m;
                    for (int e = lane; e < mI * nJ; e += 32) {
                        const int r = e % mI, c = e / mI;
                        if (!LYAP || I != J || r >= c) dX[r + (long)c * m] = dT[r + c * LD];
                    }
                    named_arrive(kBarX, TALL);             // X of block t is final
                    for (int e = lane; e < mI * nJ; e += 32) {
                        const int r = e % mI, c = e / mI;
                        if (!LYAP || I != J || r >= c) {
                            const float2 v = dT[r + c * LD];
                            rng |= df_out_of_range(v.x);          // every entry of X passes here once
                            X[(i0 + r) + (long)(j0 + c) * ldx] = df_to_double_s(v.x, v.y, -sc.x);
                        }
                    }
                } else {
                    if (!LYAP) warp_stage_tri<B>(sU, U + j0 + (long)j0 * ldu, ldu, nJ, false, lane);
                    else       warp_stage_tri<B>(sU, L + j0 + (long)j0 * ldl, ldl, nJ, true, lane);
                    __syncwarp();
                    for (int e = lane; e < mI * nJ; e += 32) {
                        const int i = e % mI, j = e / mI;
                        if (sym && i < j) continue;
                        const double dd = sL[i + i * LD] + sU[j + j * LD];
                        if (!(fabs(dd) > delta)) bad = 1;
                        sR[i + j * LD] = 1.0 / dd;
                    }
                    __syncwarp();
                    named_sync(kBarT, TALL);               // T of block t is in sT
                    if (sym) {
                        warp_diag_solve<B, LYAP, true>(sL, sU, sT, sR, mI, nJ, lane);
                        // Mirror: the block after X_00 reads it whole from here.
                        for (int e = lane; e < mI * mI; e += 32) {
                            const int i = e % mI, j = e / mI;
                            if (i < j) sT[i + j * LD] = sT[j + i * LD];
                        }
                        __syncwarp();
                    } else {
                        warp_diag_solve<B, LYAP, false>(sL, sU, sT, sR, mI, nJ, lane);
                    }
                    for (int e = lane; e < mI * nJ; e += 32) {
                        const int r = e % mI, c = e / mI;
                        if (!LYAP || I != J || r >= c) X[(i0 + r) + (long)(j0 + c) * ldx] = sT[r + c * LD];
                    }
                    named_arrive(kBarX, TALL);             // X of block t is final
                }
            }
        }
        // DF: the update warps set s_bad and s_rng before their last "T ready"
        // arrival, which this warp waited for.
        if (DF) bad = *s_bad;
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) *info = bad ? 1 : 0;
        if constexpr (DF) return (__any_sync(0xffffffffu, rng) || *s_rng) ? 1 : 0;
        return 0;
    } else {
        // ------------------------------------------------- update warps
        constexpr int E = B * B / TU;
        const int ut = threadIdx.x - 32;
        OutMap<B, TU> om;
        using Acc = typename std::conditional<DF, float, double>::type;
        int t = 0;
        for (int I = 0; I < mb; ++I) {
            const int mI = min(B, m - I * B), i0 = I * B;
            const int jend = LYAP ? I + 1 : nb;
            for (int J = 0; J < jend; ++J, ++t) {
                const int nJ = min(B, n - J * B), j0 = J * B;
                if (LYAP && I == J) om.set_lower(mI, ut);   // symmetric diagonal block: i >= j only
                else                om.set(mI, nJ, ut);
                if constexpr (DF) {
                    // The diagonal warp's operands of block t (see above).
                    float2 *pLU = df2(sL + (t & 1) * SZ), *pR = df2(sR + (t & 1) * SZ);
                    const bool sym = LYAP && I == J;
                    int bad = 0;
                    for (int e = ut; e < B * B; e += TU) {
                        const int r = e % B, c = e / B;
                        float2 v = make_float2(0.f, 0.f), w = make_float2(0.f, 0.f);
                        if (r > c && r < mI) {
                            split_df_s(L[(i0 + r) + (long)(i0 + c) * ldl], sc.op, v.x, v.y);
                        } else if (r < c && c < nJ) {
                            const double u = LYAP ? L[(j0 + c) + (long)(j0 + r) * ldl] : U[(j0 + r) + (long)(j0 + c) * ldu];
                            split_df_s(u, sc.op, v.x, v.y);
                        }
                        if (r < mI && c < nJ && !(sym && r < c)) {
                            const double dd = L[(i0 + r) + (long)(i0 + r) * ldl] +
                                              (LYAP ? L[(j0 + c) + (long)(j0 + c) * ldl] : U[(j0 + c) + (long)(j0 + c) * ldu]);
                            if (!(fabs(dd) > delta)) bad = 1;
                            split_df_s(1.0 / dd, -sc.op, w.x, w.y);   // 1 / (2^op dd)
                            if (df_out_of_range(w.x)) bad |= 2;
                        }
                        pLU[r + c * LD] = v;
                        pR[r + c * LD] = w;
                    }
                    if (bad & 1) *s_bad = 1;
                    if (bad & 2) *s_rng = 1;
                }
                // FP64: even / odd terms; DF: hi / lo of one double-float sum.
                Acc ae[E], ao[E];
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    ao[r] = 0;
                    ae[r] = 0;
                    if (om.ok(r)) {
                        int rr = om.row[r], cc = om.col[r];
                        if (LYAP && I == J && rr < cc) { const int x = rr; rr = cc; cc = x; }
                        const double c = C[(i0 + rr) + (long)(j0 + cc) * ldc];
                        if constexpr (DF) split_df_s(c, sc.rhs, ae[r], ao[r]);
                        else ae[r] = c;
                    }
                }
                // Bulk steps, then (J > 0) the staged operand of the last phase.
                // Blocks right after the block whose X they need in the first
                // sum (term K = I-1): the Lyapunov diagonal block (I, I), and
                // block (I, 0) when block (I-1, 0) is solved just before it
                // (Lyapunov I = 1; Sylvester with a single block column).
                const bool ldiag = LYAP && I == J && I > 0;
                const bool lfirst = J == 0 && I > 0 && (LYAP ? I == 1 : nb == 1);
                const int P1 = (ldiag || lfirst) ? I - 1 : I;
                const bool has_last = J > 0 || lfirst;
                const int nsteps = P1 + (J > 0 ? J - 1 : 0);
                const int nload = nsteps + (has_last ? 1 : 0);
                using SrcT = typename std::conditional<DF, SrcF, Src>::type;
                using PfT = typename std::conditional<DF, PrefetchF<B, TU>, Prefetch<B, TU>>::type;
                // Operands of step q (q == nsteps: the last phase's tile).
                auto src = [&](int q, SrcT &a, SrcT &b, bool &tq) {
                    if constexpr (DF) {
                        if (q < nsteps) step_src_f<B, LYAP>(q, P1, I, J, mI, nJ, m, n, dfw, a, b, tq);
                        else last_src_f<B, LYAP>(I, J, mI, nJ, m, n, dfw, b, tq);
                    } else {
                        if (q < nsteps) step_src<B, LYAP>(q, P1, I, J, mI, nJ, L, ldl, U, ldu, X, ldx, a, b, tq, sc);
                        else last_src_t<B, LYAP>(I, J, mI, nJ, L, ldl, U, ldu, b, tq, sc);
                    }
                };
                // The tiles of step q into buffer q & 1.
                auto stage = [&](const PfT &p, bool tq, int q) {
                    const int bf = q & 1;
                    if constexpr (DF) {
                        if (q < nsteps) p.template store_k<LD>(df2(sA0 + bf * SZ), df2(sB0 + bf * SZ), tq, ut);
                        else p.template store_b<LD>(df2(sB0 + bf * SZ), ut);
                    } else {
                        p.store(sA0 + bf * SZ, sB0 + bf * SZ, q < nsteps, ut);
                    }
                };
                auto compute = [&](bool tq, int bf) {
                    if constexpr (DF) upd_dfk<B, TU, LD>(ae, ao, om, df2(sA0 + bf * SZ), df2(sB0 + bf * SZ));
                    else upd_fma_rt<B, TU>(tq, ae, ao, om, sA0 + bf * SZ, sB0 + bf * SZ);
                };
                bool tb_next = false;
                if constexpr (PD == 2) {
                    // Step q's operands live in register set q & 1: loaded at
                    // step q - 2, stored to tile buffer q & 1 after step q - 1.
                    PfT pf0, pf1;
                    SrcT sa0{}, sb0{}, sa1{}, sb1{};
                    bool tb0 = false, tb1 = false;
                    auto iter = [&](int q, PfT &pc, SrcT &ac, SrcT &bc, bool &tc, const PfT &pn, const bool &tn) {
                        const bool tq = tc;
                        if (q + 2 < nload) {
                            src(q + 2, ac, bc, tc);
                            pc.load(ac, bc, q + 2 < nsteps, ut);
                        }
                        compute(tq, q & 1);
                        if (q + 1 < nload) stage(pn, tn, q + 1);
                        named_sync(kBarUpd, TU);
                    };
                    if (nload > 0) {
                        src(0, sa0, sb0, tb0);
                        pf0.load(sa0, sb0, nsteps > 0, ut);
                        stage(pf0, tb0, 0);
                    }
                    if (nload > 1) {
                        src(1, sa1, sb1, tb1);
                        pf1.load(sa1, sb1, nsteps > 1, ut);
                    }
                    if (nload > 0) named_sync(kBarUpd, TU);
                    for (int q = 0; q < nsteps; q += 2) {
                        iter(q, pf0, sa0, sb0, tb0, pf1, tb1);
                        if (q + 1 < nsteps) iter(q + 1, pf1, sa1, sb1, tb1, pf0, tb0);
                    }
                    tb_next = (nsteps & 1) ? tb1 : tb0;
                } else {
                    PfT pf;
                    SrcT sa{}, sb{};
                    if (nload > 0) {
                        src(0, sa, sb, tb_next);
                        pf.load(sa, sb, nsteps > 0, ut);
                        stage(pf, tb_next, 0);
                        named_sync(kBarUpd, TU);
                    }
                    for (int q = 0; q < nsteps; ++q) {
                        const bool tq = tb_next;
                        const bool more = q + 1 < nload;
                        if (more) {
                            src(q + 1, sa, sb, tb_next);
                            pf.load(sa, sb, q + 1 < nsteps, ut);
                        }
                        compute(tq, q & 1);
                        if (more) stage(pf, tb_next, q + 1);
                        named_sync(kBarUpd, TU);
                    }
                }
                if (t > 0) named_sync(kBarX, TALL);        // X of block t-1 is final
                if (has_last) {
                    // Last phase: the X block of block t-1 is still in shared
                    // memory (for a Lyapunov diagonal block: all of it).
                    const double *sXp = sT0 + ((t - 1) & 1) * SZ;
                    const double *sV = sB0 + (nsteps & 1) * SZ;
                    if constexpr (DF) {
                        const float2 *dX = df2(sXp), *dV = df2(sV);
                        if (J > 0) {
                            upd_df_rt<B, TU, LD>(tb_next, ae, ao, om, dX, dV);
                            if (ldiag) upd_df<B, TU, LD, true>(ae, ao, om, dV, dX);
                        } else {
                            upd_df<B, TU, LD, false>(ae, ao, om, dV, dX);
                        }
                    } else if (J > 0) {
                        upd_fma_rt<B, TU>(tb_next, ae, ao, om, sXp, sV);      // X_{I,J-1} U_{J-1,J}
                        if (ldiag) upd_fma<B, TU, true>(ae, ao, om, sV, sXp); // L_{I,I-1} X_{I,I-1}^T
                    } else {
                        upd_fma<B, TU, false>(ae, ao, om, sV, sXp);           // L_{I,I-1} X_{I-1,0}
                    }
                }
                double *sT = sT0 + (t & 1) * SZ;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (om.ok(r)) {
                        if constexpr (DF) df2(sT)[om.row[r] + om.col[r] * LD] = make_float2(ae[r], ao[r]);
                        else sT[om.row[r] + om.col[r] * LD] = ae[r] + ao[r];
                    }
                }
                named_sync(kBarUpd, TU);                   // staging tiles free again
                named_arrive(kBarT, TALL);                 // T of block t is in sT
            }
        }
        named_sync(kBarX, TALL);                           // X of the last block is final
    }
    return 0;
}

// ------------------------------------------------ Cholesky, warp-specialised
//
// The lazy blocked Cholesky (X^T X = A, X upper), blocks (I, J) by columns,
// I = 0..J: T_IJ = A_IJ - sum_{K<I} X_KI^T X_KJ, then X_JJ = chol(T_JJ) or
// X_IJ = X_II^{-T} T_IJ.  Warp 0 factors diagonal blocks and runs the panel
// solves (latency-bound); the update warps form T.  The term K = I-1 needs
// X_{I-1,J}, the block solved just before, so it is added from shared memory
// once that block is final (its other operand X_{I-1,I} is in an earlier
// column, or for I = J the same tile); the other terms overlap the diagonal
// warp's previous block.  Same two named barriers per block as the Sylvester
// pipeline.  After a failing pivot both roles finish the schedule (columns
// from the failing one on are undefined) so that every barrier phase
// completes; info is the first failure.

// Factor the m x m upper block in sT in place (rows in order, 32/B lanes per
// column, one FP64 rsqrt per row).  Returns 0 or the failing pivot + 1.
template <int B>
__device__ int warp_chol_diag(double *sT, int m, int lane)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int S = 32 / B;
    const int idx = lane / S, part = lane % S;
    for (int i = 0; i < m; ++i) {
        const int j = i + idx;
        const bool act = j < m;
        double s = 0.0;
        if (act)
            for (int k = part; k < i; k += S) s = fma(sT[k + i * LD], sT[k + j * LD], s);
        for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double t = act ? sT[i + j * LD] - s : 0.0;
        const double d = __shfl_sync(0xffffffffu, t, 0);
        if (!(d > 0.0)) return i + 1;
        const double r = rsqrt(d);
        if (act && part == 0) sT[i + j * LD] = (j == i) ? d * r : t * r;
        __syncwarp();
    }
    return 0;
}

// X_II^T Y = T in place for the B x nn block in sT (X_II upper in sD,
// reciprocal diagonal in sR): rows in order, 32/B lanes per column.
template <int B>
__device__ void warp_trsm_ut(const double *sD, const double *sR, double *sT, int nn, int lane)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int S = 32 / B;
    const int idx = lane / S, part = lane % S;
    const bool act = idx < nn;
    for (int i = 0; i < B; ++i) {
        double s = 0.0;
        if (act)
            for (int k = part; k < i; k += S) s = fma(sD[k + i * LD], sT[k + idx * LD], s);
        for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (act && part == 0) sT[i + idx * LD] = (sT[i + idx * LD] - s) * sR[i];
        __syncwarp();
    }
}

// DF: the update warps form T in double-float arithmetic (operands split on
// staging, X_{I-1,J} split into the staging tile the last step leaves free)
// and round it to FP64; the diagonal warp is the FP64 one.  The instance is
// rescaled by powers of two (DfScale::cholesky: A by 4^s, X by 2^s): shared
// tiles hold scaled values, global X the caller's; the diagonal warp scales
// the X blocks it stages and unscales what it writes (exact FP64 products).
//
// SC, the band check without SC and the status (valid on thread 0): as for
// syl_ws_instance (the check covers every entry of A, each staged once).
//
// DF: dfx, the instance's scratch, receives X (scaled) as double-float pairs
// (ld n) as the diagonal warp finishes each block; the update warps stage
// X_KI and X_KJ from there without splitting.
template <int B, int NU, bool DF, bool SC = false>
__device__ int chol_ws_instance(int n, const double *A, long lda, double *X, long ldx, int *info, double *sm,
                                const DfScale &scin, float2 *dfx = nullptr)
{
    constexpr bool VAL = DF && !SC;
    constexpr int W = DfScale::BAND_CHOL;
    constexpr int LD = Tile<B>::LD, SZ = Tile<B>::SZ;
    constexpr int TU = 32 * NU, TALL = TU + 32;
    static_assert((B * B) % TU == 0, "update threads must divide the block");
    double *sT0 = sm, *sD = sm + 2 * SZ, *sR = sm + 3 * SZ;
    double *sA0 = sm + 5 * SZ, *sB0 = sm + 7 * SZ;
    const int nb = (n + B - 1) / B;
    DfScale sc{0, 0, 0};
    if constexpr (SC) sc = scin;
    int *s_chk = reinterpret_cast<int *>(sm + 9 * SZ + 26);    // band bits of A (VAL)
    if constexpr (VAL) {
        if (threadIdx.x == 0) *s_chk = 0;
        __syncthreads();                       // before any update warp can set a bit
    }

    if (threadIdx.x < 32) {
        // ------------------------------------------------ diagonal warp
        const int lane = threadIdx.x;
        int fail = 0, t = 0;
        for (int J = 0; J < nb; ++J) {
            const int nJ = min(B, n - J * B), j0 = J * B;
            for (int I = 0; I <= J; ++I, ++t) {
                const int i0 = I * B;
                if (I < J) {
                    warp_stage_tri<B>(sD, X + i0 + (long)i0 * ldx, ldx, B, false, lane);
                    if constexpr (DF) {
                        const double f = pow2d(sc.x);            // each lane scales the entries it staged
                        for (int e = lane; e < B * B; e += 32) sD[e % B + (e / B) * LD] *= f;
                    }
                    __syncwarp();
                    if (lane < B) sR[lane] = 1.0 / sD[lane * (LD + 1)];
                    __syncwarp();
                }
                double *sT = sT0 + (t & 1) * SZ;
                named_sync(kBarT, TALL);                   // T of block t is in sT
                int f = 0;
                if (I < J) warp_trsm_ut<B>(sD, sR, sT, nJ, lane);
                else       f = warp_chol_diag<B>(sT, nJ, lane);
                if (f && !fail) fail = j0 + f;
                const int mI = I < J ? B : nJ;
                for (int e = lane; e < mI * nJ; e += 32) {
                    const int r = e % mI, c = e / mI;
                    // diagonal block: upper part; after a failing pivot only
                    // the rows above it are final.
                    if (I < J || (r <= c && (!f || r < f - 1))) {
                        if constexpr (DF) {
                            const double v = sT[r + c * LD];
                            X[(i0 + r) + (long)(j0 + c) * ldx] = v * pow2d(-sc.x);
                            // Pairs (scaled) for the update warps: only block rows
                            // that later blocks stage (K <= I - 2 in the bulk steps,
                            // I - 1 <= J - 2 in the last phase), i.e. I <= nb - 3.
                            if (I + 3 <= nb) {
                                float2 p;
                                split_df_s(v, 0, p.x, p.y);
                                dfx[(i0 + r) + (long)(j0 + c) * n] = p;
                            }
                        } else {
                            X[(i0 + r) + (long)(j0 + c) * ldx] = sT[r + c * LD];
                        }
                    }
                }
                named_arrive(kBarX, TALL);                 // X of block t is final
            }
        }
        if (lane == 0) *info = fail;
        if constexpr (VAL) {
            // The update warps set s_chk before their last "T ready" arrival.
            const unsigned k = (unsigned)*s_chk;
            return ((k & BAND_BIG) || !(k & BAND_OP)) ? 2 : 0;
        }
        return 0;
    } else {
        // ------------------------------------------------- update warps
        constexpr int E = B * B / TU;
        const int ut = threadIdx.x - 32;
        OutMap<B, TU> om;
        using Acc = typename std::conditional<DF, float, double>::type;
        unsigned chk = 0;                                  // band bits (VAL)
        int t = 0;
        for (int J = 0; J < nb; ++J) {
            const int nJ = min(B, n - J * B), j0 = J * B;
            for (int I = 0; I <= J; ++I, ++t) {
                const int i0 = I * B;
                const bool diag = I == J;
                const int mI = diag ? nJ : B;
                if (diag) om.set_upper(nJ, ut);
                else      om.set(mI, nJ, ut);
                // Bulk K = 0..I-2; then, for I < J, the staged X_{I-1,I} of the last term.
                const int nsteps = I > 1 ? I - 1 : 0;
                const bool has_last = I >= 1;
                const int nload = nsteps + (has_last && !diag ? 1 : 0);
                using SrcT = typename std::conditional<DF, SrcF, Src>::type;
                using PfT = typename std::conditional<DF, PrefetchF<B, TU>, Prefetch<B, TU>>::type;
                // Operands of step q: X_KI (used transposed) and X_KJ for K = q;
                // q == nsteps: the last phase's X_{I-1,I}.
                auto src = [&](int q, SrcT &sa, SrcT &sb) {
                    if constexpr (DF) {
                        if (q < nsteps) {
                            sa = SrcF{dfx + q * B + (long)i0 * n, n, B, mI, false};
                            sb = SrcF{dfx + q * B + (long)j0 * n, n, B, nJ, false};
                        } else {
                            sb = SrcF{dfx + (long)(I - 1) * B + (long)i0 * n, n, B, mI, false};
                        }
                    } else {
                        if (q < nsteps) {
                            const int k0 = q * B;
                            sa = Src{X + k0 + (long)i0 * ldx, ldx, B, mI, false, sc.x};
                            sb = Src{X + k0 + (long)j0 * ldx, ldx, B, nJ, false, sc.x};
                        } else {
                            sb = Src{X + (long)(I - 1) * B + (long)i0 * ldx, ldx, B, mI, false, sc.x};
                        }
                    }
                };
                auto stage = [&](const PfT &p, int q) {           // step q's tiles into buffer q & 1
                    const int bf = q & 1;
                    if constexpr (DF) p.template store_nat<LD>(df2(sA0 + bf * SZ), df2(sB0 + bf * SZ), q < nsteps, ut);
                    else p.store(sA0 + bf * SZ, sB0 + bf * SZ, q < nsteps, ut);
                };
                PfT pf;
                SrcT sa{}, sb{};
                if (nload > 0) {
                    src(0, sa, sb);
                    pf.load(sa, sb, nsteps > 0, ut);
                    stage(pf, 0);
                    named_sync(kBarUpd, TU);
                }
                // FP64: even / odd terms; DF: hi / lo of one double-float sum.
                Acc ae[E], ao[E];
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    ao[r] = 0;
                    ae[r] = 0;
                    if (om.ok(r)) {
                        const double a = A[(i0 + om.row[r]) + (long)(j0 + om.col[r]) * lda];
                        if constexpr (DF) split_df_s(a, sc.op, ae[r], ao[r]);
                        else ae[r] = a;
                        if constexpr (VAL) chk |= band_bits<W>(a, BAND_OP);
                    }
                }
                for (int q = 0; q < nsteps; ++q) {
                    const int buf = q & 1;
                    const bool more = q + 1 < nload;
                    if (more) {
                        src(q + 1, sa, sb);
                        pf.load(sa, sb, q + 1 < nsteps, ut);
                    }
                    if constexpr (DF) upd_df_ta<B, TU, LD>(ae, ao, om, df2(sA0 + buf * SZ), df2(sB0 + buf * SZ));
                    else upd_fma_ta<B, TU>(ae, ao, om, sA0 + buf * SZ, sB0 + buf * SZ);
                    if (more) stage(pf, q + 1);
                    named_sync(kBarUpd, TU);
                }
                if (t > 0) named_sync(kBarX, TALL);        // X of block t-1 is final
                if (has_last) {
                    // K = I-1: X_{I-1,J} is block t-1, in shared memory; X_{I-1,I}
                    // is the staged tile, or for I = J that same block.
                    const double *sXp = sT0 + ((t - 1) & 1) * SZ;
                    const double *sV = diag ? sXp : sB0 + (nsteps & 1) * SZ;
                    if constexpr (DF) {
                        // X_{I-1,J} split into the free staging tile sA[nsteps & 1]
                        // (the last step stages no A operand).
                        float2 *dX = df2(sA0 + (nsteps & 1) * SZ);
                        tile_to_df<B, TU, LD>(dX, sXp, ut);
                        named_sync(kBarUpd, TU);
                        upd_df_ta<B, TU, LD>(ae, ao, om, diag ? dX : df2(sV), dX);
                    } else {
                        upd_fma_ta<B, TU>(ae, ao, om, sV, sXp);
                    }
                }
                double *sT = sT0 + (t & 1) * SZ;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (om.ok(r)) {
                        if constexpr (DF) sT[om.row[r] + om.col[r] * LD] = df_to_double(ae[r], ao[r]);
                        else sT[om.row[r] + om.col[r] * LD] = ae[r] + ao[r];
                    }
                }
                named_sync(kBarUpd, TU);                   // staging tiles free again
                if (VAL && J == nb - 1 && I == J) {
                    // Before the last arrival: the band bits of the whole instance.
                    chk = __reduce_or_sync(0xffffffffu, chk);
                    if ((threadIdx.x & 31) == 0) atomicOr(s_chk, (int)chk);
                }
                named_arrive(kBarT, TALL);                 // T of block t is in sT
            }
        }
        named_sync(kBarX, TALL);                           // X of the last block is final
    }
    return 0;
}

__device__ __forceinline__ bool next_instance(const Sched &s, int group, int *s_slot, int &b,
                                              int head = META_HEAD, int *wpos = nullptr)
{
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    const int w = lo + claim_slot(s.meta + head + group, s_slot);
    if (w >= hi) return false;
    b = s.perm[w];
    if (wpos) *wpos = w;
    return true;
}

// MINB: CTAs per SM the register allocation must allow (the two roles share
// one register budget, set by the larger of them).
// DF without SC: the persistent queue over the group, solving with zero
// shifts the instances whose data lies in DfScale's band (found by the
// solve's first pass); the others are left to the SC pass (DfInst::pend and
// the group's META_SCL flag).  DF with SC: only those instances, solved with their
// shifts, from a second queue over the group's positions (longest first, as
// the first); it returns at once when the group's flag is clear.
template <int B, int NU, bool LYAP, int MINB, bool DF, bool SC>
__global__ void __launch_bounds__(32 * NU + 32, MINB) syl_ws_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    __shared__ int s_slot;
    auto one = [&](int b, int w) {
        const int n = o.n[b], m = o.m != nullptr ? o.m[b] : n;
        if (n == 0 || m == 0) { if (threadIdx.x == 0) o.info[b] = 0; return; }
        // DF: the instance's share of the workspace scratch (pre-split copies).
        float2 *dfw = nullptr;
        if constexpr (DF) {
            const long long need = 2ll * ((long long)m * m + (long long)n * n + (long long)m * n);
            if (s.scr == nullptr || s.scratch == nullptr || s.scr[w] + need > s.scratch_elems) {
                if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
                return;
            }
            dfw = reinterpret_cast<float2 *>(static_cast<float *>(s.scratch) + s.scr[w]);
        }
        const double *U = LYAP ? nullptr : o.U[b];
        const int ldu = LYAP ? 0 : o.ldu[b];
        const int st = syl_ws_instance<B, NU, LYAP, DF, SC, MINB <= 2 ? 2 : 1>(m, n, o.A[b], o.lda[b], U, ldu, o.C[b],
                                                                              o.ldc[b], o.X[b], o.ldx[b], o.info + b,
                                                                              sm, DF ? const_cast<DfInst *>(s.dfs) + b : nullptr,
                                                                              dfw);
        // Zero-shift pass: the instance's data is outside DfScale's band; its
        // record (written by the instance) hands it to the rescaled pass.
        if (DF && !SC && st == 4) {
            if (threadIdx.x == 0) s.meta[META_SCL + group] = 1;
            return;
        }
        // Out of the double-float range: syl_ws_fixup_kernel, launched last,
        // solves the instance again in FP64 (unless X overwrote C).
        if (DF && st != 0 && threadIdx.x == 0) {
            o.info[b] = SS_INFO_RANGE;
            s.meta[META_RNG + group] = 1;
        }
    };
    int b, w = 0;
    claim_init(&s_slot);
    if constexpr (SC) {
        if (s.meta[META_SCL + group] == 0) return;            // the same on every thread
        while (next_instance(s, group, &s_slot, b, META_SCL_HEAD, &w))
            if (s.dfs[b].pend != 0) one(b, w);                // the same on every thread
    } else {
        while (next_instance(s, group, &s_slot, b, META_HEAD, &w)) one(b, w);
    }
}

// After a double-float launch group: every instance of the group whose info
// is SS_INFO_RANGE is solved again in FP64 from its right-hand side, unless X
// overwrote it (X == C), where the code stays.  Usually the group's range
// flag is clear and every CTA returns after one load; otherwise one CTA per
// SM strides over the group's positions.  (A separate launch keeps the FP64
// code out of the double-float kernel's register allocation.)
template <int B, int NU, bool LYAP, int MINB>
__global__ void __launch_bounds__(32 * NU + 32, MINB) syl_ws_fixup_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    if (s.meta[META_RNG + group] == 0) return;            // the same on every thread
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    for (int w = lo + (int)blockIdx.x; w < hi; w += (int)gridDim.x) {
        const int b = s.perm[w];
        if (o.info[b] != SS_INFO_RANGE || o.X[b] == o.C[b]) continue;   // the same on every thread
        const int n = o.n[b], m = o.m != nullptr ? o.m[b] : n;
        __syncthreads();                                      // the previous instance's shared data is dead
        syl_ws_instance<B, NU, LYAP, false>(m, n, o.A[b], o.lda[b], LYAP ? nullptr : o.U[b], LYAP ? 0 : o.ldu[b],
                                           o.C[b], o.ldc[b], o.X[b], o.ldx[b], o.info + b, sm, nullptr);
    }
}

template <typename K>
cudaError_t launch_ws(K kernel, int threads, size_t smem, int batch, cudaStream_t st, const Operands &o,
                      const Sched &s, int group)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long grid = (long)per_sm * sm_count();
    if (grid > batch) grid = batch;
    if (grid < 1) grid = 1;
    kernel<<<(int)grid, threads, smem, st>>>(o, s, group);
    return cudaGetLastError();
}

// The range fix-up pass after a double-float group: one CTA per SM (or per
// instance, if fewer).
template <typename K>
cudaError_t launch_fixup(K kernel, int threads, size_t smem, int batch, cudaStream_t st, const Operands &o,
                         const Sched &s, int group)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = sm_count();
    if (grid > batch) grid = batch;
    if (grid < 1) grid = 1;
    kernel<<<grid, threads, smem, st>>>(o, s, group);
    return cudaGetLastError();
}

}  // namespace

// DF without SC / with SC: as for syl_ws_kernel (an instance out of the band,
// or solved in place, X == A, is left to the rescaled pass).
template <int B, int NU, int MINB, bool DF, bool SC>
__global__ void __launch_bounds__(32 * NU + 32, MINB) chol_ws_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    __shared__ int s_slot;
    int *s_scan = reinterpret_cast<int *>(sm + 9 * Tile<B>::SZ);
    auto pend = [&](int b) {
        if (threadIdx.x == 0) {
            const_cast<DfInst *>(s.dfs)[b].pend = 1;
            s.meta[META_SCL + group] = 1;
        }
    };
    auto one = [&](int b, int w) {
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; return; }
        // DF: the instance's share of the workspace scratch (X as pairs).
        float2 *dfx = nullptr;
        if constexpr (DF) {
            if (s.scr == nullptr || s.scratch == nullptr || s.scr[w] + 2ll * n * n > s.scratch_elems) {
                if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
                return;
            }
            dfx = reinterpret_cast<float2 *>(static_cast<float *>(s.scratch) + s.scr[w]);
        }
        DfScale sc{0, 0, 0};
        if constexpr (DF && !SC) {
            if (o.X[b] == o.A[b]) { pend(b); return; }           // in place: scanned first by the SC pass
        }
        if constexpr (SC) {
            int ea, unused;
            scan_exp3(ScanOp{o.A[b], o.lda[b], n, n, 2}, ScanOp{nullptr, 0, 0, 0, 0}, ScanOp{nullptr, 0, 0, 0, 0},
                      threadIdx.x >> 5, (int)(blockDim.x >> 5), threadIdx.x & 31, ea, unused);
            cta_max2(ea, unused, s_scan);
            sc = DfScale::cholesky(ea);
        }
        const int st = chol_ws_instance<B, NU, DF, SC>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], o.info + b, sm, sc, dfx);
        if (DF && (st & 2)) pend(b);                            // out of the band: solve again rescaled
    };
    int b, w = 0;
    claim_init(&s_slot);
    if constexpr (SC) {
        if (s.meta[META_SCL + group] == 0) return;              // the same on every thread
        while (next_instance(s, group, &s_slot, b, META_SCL_HEAD, &w))
            if (s.dfs[b].pend != 0) one(b, w);                  // the same on every thread
    } else {
        while (next_instance(s, group, &s_slot, b, META_HEAD, &w)) one(b, w);
    }
}

// Warp-specialised Cholesky configurations: block B, NU update warps; df:
// double-float update warps (the diagonal warp stays FP64), then the scaled
// pass.
template <int BB, int NN, int MB>
cudaError_t launch_chol_df(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st)
{
    cudaError_t e = launch_ws(chol_ws_kernel<BB, NN, MB, true, false>, 32 * NN + 32, ws_smem_bytes<BB>(), l.batch, st,
                              o, s, l.group);
    if (e != cudaSuccess) return e;
    return launch_ws(chol_ws_kernel<BB, NN, MB, true, true>, 32 * NN + 32, ws_smem_bytes<BB>(), l.batch, st, o, s,
                     l.group);
}

cudaError_t launch_potrf_ws(int block, int nu, bool df, const Operands &o, const Sched &s, const Launch &l,
                            cudaStream_t st, bool few)
{
#define CWS_CASE(BB, NN, MB, FEW)                                                                         \
    if (block == BB && nu == NN && few == FEW)                                                            \
        return df ? launch_chol_df<BB, NN, MB>(o, s, l, st)                                               \
                  : launch_ws(chol_ws_kernel<BB, NN, MB, false, false>, 32 * NN + 32, ws_smem_bytes<BB>(), l.batch, \
                              st, o, s, l.group);
    CWS_CASE(16, 2, 8, false)
    CWS_CASE(16, 4, 7, false)
    CWS_CASE(16, 4, 2, true)     // few instances per SM: all of the registers
#undef CWS_CASE
    return cudaErrorInvalidValue;
}

// A double-float Sylvester / Lyapunov group (three launches): the unscaled
// pipeline over the queue, the scaled pipeline for the instances it left,
// then the range fix-up pass.
template <int BB, int NN, int MB, bool LY>
cudaError_t launch_syl_df(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st)
{
    cudaError_t e = launch_ws(syl_ws_kernel<BB, NN, LY, MB, true, false>, 32 * NN + 32, ws_smem_bytes<BB, true>(),
                              l.batch, st, o, s, l.group);
    if (e != cudaSuccess) return e;
    e = launch_ws(syl_ws_kernel<BB, NN, LY, MB, true, true>, 32 * NN + 32, ws_smem_bytes<BB, true>(), l.batch, st, o,
                  s, l.group);
    if (e != cudaSuccess) return e;
    return launch_fixup(syl_ws_fixup_kernel<BB, NN, LY, MB>, 32 * NN + 32, ws_smem_bytes<BB, false>(), l.batch, st, o,
                        s, l.group);
}

// Warp-specialised configurations: block B, NU update warps (+1 diagonal warp);
// df: double-float update warps (plus the scaled pass and the range fix-up pass);
// few: at most two CTAs per SM and the two-step operand prefetch.
cudaError_t launch_syl_ws(int block, int nu, bool lyap, bool df, const Operands &o, const Sched &s, const Launch &l,
                          cudaStream_t st, bool few)
{
#define WS_ONE(BB, NN, MB, LY, D)                                                                          \
    launch_ws(syl_ws_kernel<BB, NN, LY, MB, D, false>, 32 * NN + 32, ws_smem_bytes<BB, D>(), l.batch, st, o, s, l.group)
#define WS_CASE(BB, NN, MB, FEW)                                                                           \
    if (block == BB && nu == NN && few == FEW)                                                             \
        return df ? (lyap ? launch_syl_df<BB, NN, MB, true>(o, s, l, st) : launch_syl_df<BB, NN, MB, false>(o, s, l, st)) \
                  : (lyap ? WS_ONE(BB, NN, MB, true, false) : WS_ONE(BB, NN, MB, false, false));
    WS_CASE(16, 4, 6, false)
    WS_CASE(16, 2, 8, false)
    WS_CASE(16, 1, 8, false)
    WS_CASE(16, 4, 2, true)    // few instances per SM: two-step operand prefetch
    WS_CASE(16, 8, 1, true)
    WS_CASE(32, 8, 1, true)
#undef WS_CASE
#undef WS_ONE
    return cudaErrorInvalidValue;
}

}  // namespace ss
