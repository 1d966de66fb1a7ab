// Plain FP64 batched solvers: upper Cholesky (Fig. 2a), triangular Lyapunov
// (Fig. 2b) and triangular Sylvester (Fig. 2c) of the paper.
//
// One CTA solves one instance at a time and pulls instances from a persistent
// queue ordered by size, largest first.  Each instance is processed in B x B
// blocks with the "lazy" (left-looking) loop order: a block of the result is
// finished in one visit, after accumulating every update it needs from
// already finished blocks, and is then written once.  The updates are the
// GEMM/SYRK part (register-tiled, FP64 FMA); the diagonal work (square roots,
// the divisions by x_ii and by l_ii + u_jj) is a wavefront of split dot
// products over the block in shared memory.
//
// Blocked recurrences (2 x 2 partitioning of the defining equations):
//   Cholesky   X_IJ = X_II^{-T} (A_IJ - sum_{K<I} X_KI^T X_KJ),  I < J,
//              X_JJ = chol(A_JJ - sum_{K<J} X_KJ^T X_KJ);
//   Sylvester  L_II X_IJ + X_IJ U_JJ = C_IJ - sum_{K<I} L_IK X_KJ - sum_{K<J} X_IK U_KJ;
//   Lyapunov   the Sylvester recurrence with U = L^T over the blocks I >= J,
//              reading X_KJ (K < J) as X_JK^T.
#include "ss_device.cuh"
#include "ss_internal.h"

namespace ss {
namespace {

// Shared memory of one CTA: five tiles plus a few scalars.
template <int B>
constexpr size_t smem_bytes() { return (size_t)5 * Tile<B>::SZ * sizeof(double) + 2 * B * sizeof(double); }

__device__ __forceinline__ double block_max_abs_diag(const double *P, long ld, int n, double *s_red)
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

// ---------------------------------------------------------------- Sylvester
//
// Solve Lt Y + Y Ut = T in place for an m x nn block in sT, Lt = sL (lower
// triangular m x m), Ut = sU (upper, nn x nn) or, with UT, the transpose of
// the lower triangular sU.  First the block's reciprocal divisors
// 1 / (l_ii + u_jj) go to sR with every lane busy; then a wavefront over the
// anti-diagonals d = i + j: the entries of one anti-diagonal are independent,
// and each is one dot product of exactly d terms (i from the L row, j from the
// U column), split over `split` lanes so that one anti-diagonal fills one
// warp.  FP64 lanes are the scarce resource on this GPU, so idle warps are
// preferred to partially filled ones.  Returns 1 if a divisor was tiny.
template <int B, int T, bool UT>
__device__ int syl_diag(const double *sL, const double *sU, double *sT, double *sR, int m, int nn,
                        double delta)
{
    constexpr int LD = Tile<B>::LD;
    int bad = 0;
    for (int e = threadIdx.x; e < m * nn; e += T) {
        const int i = e % m, j = e / m;
        const double dd = sL[i + i * LD] + sU[j + j * LD];
        if (!(fabs(dd) > delta)) bad = 1;
        sR[i + j * LD] = 1.0 / dd;
    }
    __syncthreads();
    for (int d = 0; d <= m + nn - 2; ++d) {
        const int ilo = max(0, d - nn + 1), ihi = min(d, m - 1);
        const int cnt = ihi - ilo + 1;
        int split = cnt >= 32 ? 1 : pow2_floor(32 / cnt);
        const int byLen = pow2_floor(d > 1 ? d : 1);
        split = split < byLen ? split : byLen;
        if (warp_has_work(cnt, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < cnt;
            const int i = ilo + (act ? idx : 0), j = d - i;
            double s = 0.0;
            if (act) {
                for (int t = part; t < d; t += split) {
                    const bool lt = t < i;
                    const int k = t - i;
                    const double a = lt ? sL[i + t * LD] : sT[i + k * LD];
                    const double b = lt ? sT[t + j * LD] : (UT ? sU[j + k * LD] : sU[k + j * LD]);
                    s = fma(a, b, s);
                }
            }
            s = group_sum(s, split);
            if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * sR[i + j * LD];
        }
        __syncthreads();
    }
    return bad;
}

// Warp-level version of syl_diag (B <= 32): warp 0 alone runs the
// reciprocals and the wavefront, synchronising with __syncwarp only; each
// entry of an anti-diagonal gets 32/B lanes.  The other warps wait at the
// closing barrier.  Shortens the per-instance critical path when latency,
// not the FP64 pipe, bounds the call.
template <int B, int T, bool UT>
__device__ int syl_diag_warp(const double *sL, const double *sU, double *sT, double *sR, int m, int nn,
                             double delta)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int S = 32 / B;          // lanes per entry
    int bad = 0;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int e = lane; e < m * nn; e += 32) {
            const int i = e % m, j = e / m;
            const double dd = sL[i + i * LD] + sU[j + j * LD];
            if (!(fabs(dd) > delta)) bad = 1;
            sR[i + j * LD] = 1.0 / dd;
        }
        __syncwarp();
        const int idx = lane / S, part = lane % S;
        for (int d = 0; d <= m + nn - 2; ++d) {
            const int ilo = max(0, d - nn + 1), ihi = min(d, m - 1);
            const int cnt = ihi - ilo + 1;
            const bool act = idx < cnt;
            const int i = ilo + (act ? idx : 0), j = d - i;
            double s = 0.0;
            if (act) {
                for (int t = part; t < d; t += S) {
                    const bool lt = t < i;
                    const int k = t - i;
                    const double a = lt ? sL[i + t * LD] : sT[i + k * LD];
                    const double b = lt ? sT[t + j * LD] : (UT ? sU[j + k * LD] : sU[k + j * LD]);
                    s = fma(a, b, s);
                }
            }
            for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * sR[i + j * LD];
            __syncwarp();
        }
    }
    return __syncthreads_or(bad);
}

// One Sylvester (LYAP = false) or Lyapunov (LYAP = true, U unused) instance.
// X is m x n (L m x m, U n x n); Lyapunov has m = n.
template <int B, int T, bool LYAP, int VAR>
__device__ void syl_instance(int m, int n, const double *L, long ldl, const double *U, long ldu,
                             const double *C, long ldc, double *X, long ldx, int *info,
                             double *sm)
{
    constexpr int LD = Tile<B>::LD, SZ = Tile<B>::SZ, E = B * B / T;
    double *sA = sm, *sB = sm + SZ, *sT = sm + 2 * SZ, *sL = sm + 3 * SZ, *sU = sm + 4 * SZ;
    double *s_red = sm + 5 * SZ;
    const int mb = (m + B - 1) / B, nb = (n + B - 1) / B;

    double md = block_max_abs_diag(L, ldl, m, s_red);
    if (!LYAP) md = fmax(md, block_max_abs_diag(U, ldu, n, s_red));
    const double delta = divisor_delta(max(m, n), md);

    int bad = 0;
    Slots<B, T> sl;
    for (int I = 0; I < mb; ++I) {
        const int mI = min(B, m - I * B);
        const int i0 = I * B;
        __syncthreads();
        stage_tri<B, T>(sL, L + i0 + (long)i0 * ldl, ldl, mI, true);
        const int jend = LYAP ? I + 1 : nb;
        for (int J = 0; J < jend; ++J) {
            const int nJ = min(B, n - J * B);
            const int j0 = J * B;
            sl.set(Shape::Full, mI, nJ);
            double acc[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                acc[r] = 0.0;
                if (sl.ok(r)) {
                    int rr = sl.row[r], cc = sl.col[r];
                    // Lyapunov diagonal block: read S through its lower triangle.
                    if (LYAP && I == J && rr < cc) { int t = rr; rr = cc; cc = t; }
                    acc[r] = C[(i0 + rr) + (long)(j0 + cc) * ldc];
                }
            }
            // sum_{K<I} L_IK X_KJ
            for (int K = 0; K < I; ++K) {
                const int k0 = K * B;
                __syncthreads();
                stage_tile<B, T>(sA, L + i0 + (long)k0 * ldl, ldl, mI, B);
                const bool tr = LYAP && K < J;
                if (LYAP && K == J) stage_sym_lower<B, T>(sB, X + j0 + (long)j0 * ldx, ldx, nJ);
                else if (!tr) stage_tile<B, T>(sB, X + k0 + (long)j0 * ldx, ldx, B, nJ);
                else          stage_tile<B, T>(sB, X + j0 + (long)k0 * ldx, ldx, nJ, B);   // X_JK
                __syncthreads();
                if (!tr) slot_update<B, T, false, false>(acc, sl, sA, sB, B);
                else     slot_update<B, T, false, true>(acc, sl, sA, sB, B);
            }
            // sum_{K<J} X_IK U_KJ  (Lyapunov: U_KJ = L_JK^T)
            for (int K = 0; K < J; ++K) {
                const int k0 = K * B;
                __syncthreads();
                stage_tile<B, T>(sA, X + i0 + (long)k0 * ldx, ldx, mI, B);
                if (!LYAP) stage_tile<B, T>(sB, U + k0 + (long)j0 * ldu, ldu, B, nJ);
                else       stage_tile<B, T>(sB, L + j0 + (long)k0 * ldl, ldl, nJ, B);
                __syncthreads();
                if (!LYAP) slot_update<B, T, false, false>(acc, sl, sA, sB, B);
                else       slot_update<B, T, false, true>(acc, sl, sA, sB, B);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < E; ++r)
                if (sl.ok(r)) sT[sl.row[r] + sl.col[r] * LD] = acc[r];
            if (!LYAP) stage_tri<B, T>(sU, U + j0 + (long)j0 * ldu, ldu, nJ, false);
            else       stage_tri<B, T>(sU, L + j0 + (long)j0 * ldl, ldl, nJ, true);
            __syncthreads();
            if (VAR == 0) bad |= syl_diag<B, T, LYAP>(sL, sU, sT, sA, mI, nJ, delta);
            else bad |= syl_diag_warp<B, T, LYAP>(sL, sU, sT, sA, mI, nJ, delta);
            // syl_diag ends with a barrier.
#pragma unroll
            for (int r = 0; r < E; ++r) {
                if (sl.ok(r)) {
                    const int rr = sl.row[r], cc = sl.col[r];
                    if (!LYAP || I != J || rr >= cc)
                        X[(i0 + rr) + (long)(j0 + cc) * ldx] = sT[rr + cc * LD];
                }
            }
        }
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) *info = bad ? 1 : 0;
}

// ----------------------------------------------------------------- Cholesky
//
// Factor the m x m block in sT (upper triangle) in place: X^T X = T.  Row i
// of X needs only rows < i, so rows go one at a time and the entries of a row
// are independent split dot products.  Returns 0 or the failing pivot + 1.
template <int B, int T>
__device__ int chol_diag(double *sT, int m, double *s_scal)
{
    constexpr int LD = Tile<B>::LD;
    for (int i = 0; i < m; ++i) {
        const int cnt = m - i;
        const int split = pick_split<T>(cnt, i);
        if (warp_has_work(cnt, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < cnt;
            const int j = i + (act ? idx : 0);
            double s = 0.0;
            if (act)
                for (int k = part; k < i; k += split) s = fma(sT[k + i * LD], sT[k + j * LD], s);
            s = group_sum(s, split);
            if (act && part == 0) sT[i + j * LD] -= s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double d = sT[i + i * LD];
            if (d > 0.0) {
                const double p = sqrt(d);
                sT[i + i * LD] = p;
                s_scal[0] = 1.0 / p;
                s_scal[1] = 0.0;
            } else {
                s_scal[1] = 1.0;
            }
        }
        __syncthreads();
        if (s_scal[1] != 0.0) return i + 1;
        const double rinv = s_scal[0];
        for (int j = i + 1 + threadIdx.x; j < m; j += T) sT[i + j * LD] *= rinv;
        __syncthreads();
    }
    return 0;
}

// Solve X_II^T Y = T in place for the B x nn block in sT, X_II the upper
// triangular factor in sD with reciprocal diagonal s_rinv.  Row i of Y needs
// rows < i only.
template <int B, int T>
__device__ void chol_trsm(const double *sD, const double *s_rinv, double *sT, int m, int nn)
{
    constexpr int LD = Tile<B>::LD;
    for (int i = 0; i < m; ++i) {
        const int split = pick_split<T>(nn, i);
        if (warp_has_work(nn, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < nn;
            const int j = act ? idx : 0;
            double s = 0.0;
            if (act)
                for (int k = part; k < i; k += split) s = fma(sD[k + i * LD], sT[k + j * LD], s);
            s = group_sum(s, split);
            if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * s_rinv[i];
        }
        __syncthreads();
    }
}

// Warp-level Cholesky of the m x m upper block in sT (B <= 32): warp 0 alone,
// rows in order, 32/B lanes per column; every lane takes the pivot from the
// row's first entry and forms 1/sqrt once (FP64 rsqrt), so a row costs one
// __syncwarp.  Returns 0 or the failing pivot + 1 (uniform over the CTA).
template <int B, int T>
__device__ int chol_diag_warp(double *sT, int m, double *s_scal)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int S = 32 / B;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, idx = lane / S, part = lane % S;
        int fail = 0;
        for (int i = 0; i < m; ++i) {
            const int j = i + idx;
            const bool act = j < m;
            double s = 0.0;
            if (act)
                for (int k = part; k < i; k += S) s = fma(sT[k + i * LD], sT[k + j * LD], s);
            for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const double t = act ? sT[i + j * LD] - s : 0.0;
            const double d = __shfl_sync(0xffffffffu, t, 0);    // pivot argument of row i
            if (!(d > 0.0)) { fail = i + 1; break; }
            const double r = rsqrt(d);
            if (act && part == 0) sT[i + j * LD] = (j == i) ? d * r : t * r;
            __syncwarp();
        }
        if (lane == 0) s_scal[1] = (double)fail;
    }
    __syncthreads();
    return (int)s_scal[1];
}

// Warp-level solve of X_II^T Y = T for the B x nn block in sT (B <= 32):
// warp 0, rows in order, 32/B lanes per column.
template <int B, int T>
__device__ void chol_trsm_warp(const double *sD, const double *s_rinv, double *sT, int m, int nn)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int S = 32 / B;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, idx = lane / S, part = lane % S;
        const bool act = idx < nn;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            if (act)
                for (int k = part; k < i; k += S) s = fma(sD[k + i * LD], sT[k + idx * LD], s);
            for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (act && part == 0) sT[i + idx * LD] = (sT[i + idx * LD] - s) * s_rinv[i];
            __syncwarp();
        }
    }
    __syncthreads();
}

template <int B, int T, int VAR>
__device__ void potrf_instance(int n, const double *A, long lda, double *X, long ldx, int *info,
                               double *sm)
{
    constexpr int LD = Tile<B>::LD, SZ = Tile<B>::SZ, E = B * B / T;
    double *sA = sm, *sB = sm + SZ, *sT = sm + 2 * SZ, *sD = sm + 3 * SZ;
    double *s_rinv = sm + 5 * SZ, *s_scal = s_rinv + B;
    const int nb = (n + B - 1) / B;
    Slots<B, T> sl;
    for (int J = 0; J < nb; ++J) {
        const int nJ = min(B, n - J * B);
        const int j0 = J * B;
        for (int I = 0; I <= J; ++I) {
            const int i0 = I * B;
            const bool diag = I == J;
            const int mI = diag ? nJ : B;
            if (diag) sl.set(Shape::Upper, nJ, nJ);
            else      sl.set(Shape::Full, mI, nJ);
            double acc[E];
#pragma unroll
            for (int r = 0; r < E; ++r)
                acc[r] = sl.ok(r) ? A[(i0 + sl.row[r]) + (long)(j0 + sl.col[r]) * lda] : 0.0;
            // sum_{K<I} X_KI^T X_KJ
            for (int K = 0; K < I; ++K) {
                const int k0 = K * B;
                __syncthreads();
                stage_tile<B, T>(sA, X + k0 + (long)i0 * ldx, ldx, B, mI);   // X_KI
                stage_tile<B, T>(sB, X + k0 + (long)j0 * ldx, ldx, B, nJ);   // X_KJ
                __syncthreads();
                slot_update<B, T, true, false>(acc, sl, sA, sB, B);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < E; ++r)
                if (sl.ok(r)) sT[sl.row[r] + sl.col[r] * LD] = acc[r];
            if (!diag) {
                stage_tri<B, T>(sD, X + i0 + (long)i0 * ldx, ldx, B, false);
                __syncthreads();
                for (int i = threadIdx.x; i < B; i += T) s_rinv[i] = 1.0 / sD[i + i * LD];
                __syncthreads();
                if (VAR == 0) chol_trsm<B, T>(sD, s_rinv, sT, B, nJ);
                else chol_trsm_warp<B, T>(sD, s_rinv, sT, B, nJ);
            } else {
                __syncthreads();
                const int f = VAR == 0 ? chol_diag<B, T>(sT, nJ, s_scal) : chol_diag_warp<B, T>(sT, nJ, s_scal);
                if (f) {
                    // Rows above the failing pivot are final (both diagonal
                    // solvers go row by row): write them, i.e. every column
                    // of the block before the pivot.
#pragma unroll
                    for (int r = 0; r < E; ++r)
                        if (sl.ok(r) && sl.row[r] < f - 1)
                            X[(i0 + sl.row[r]) + (long)(j0 + sl.col[r]) * ldx] = sT[sl.row[r] + sl.col[r] * LD];
                    if (threadIdx.x == 0) *info = j0 + f;
                    return;     // uniform: every thread saw the same pivot
                }
            }
#pragma unroll
            for (int r = 0; r < E; ++r)
                if (sl.ok(r)) X[(i0 + sl.row[r]) + (long)(j0 + sl.col[r]) * ldx] = sT[sl.row[r] + sl.col[r] * LD];
        }
    }
    if (threadIdx.x == 0) *info = 0;
}

// ------------------------------------- Cholesky, right-looking in shared memory
//
// For n <= NMAX the upper triangle of A sits in shared memory and is factored
// in place column by column (right-looking): pivot k, row k scaled by
// 1/sqrt(pivot), then the rank-1 update of the trailing upper triangle.  No
// global traffic inside the factorisation, two CTA barriers per column, and
// the update's FP64 instructions all carry useful FMAs (a flat map over the
// trailing triangle).  Returns 0 or the failing pivot + 1; on failure at
// pivot k the final rows 0..k-1 of X (so every column < k) are written.

// Column c of the flat upper-triangle index e: c(c+1)/2 <= e < (c+1)(c+2)/2.
__device__ __forceinline__ int tri_col(int e)
{
    int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (c * (c + 1) / 2 > e) --c;
    while ((c + 1) * (c + 2) / 2 <= e) ++c;
    return c;
}

template <int NMAX, int T>
__device__ int chol_rl_smem(int n, const double *A, long lda, double *X, long ldx, double *S)
{
    constexpr int LD = NMAX + 1;
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int i = e % n, j = e / n;
        if (i <= j) S[i + j * LD] = A[i + (long)j * lda];
    }
    __syncthreads();
    int done = n, fail = 0;
    for (int k = 0; k < n; ++k) {
        const double d = S[k + k * LD];
        if (!(d > 0.0)) { done = k; fail = k + 1; break; }   // every thread read the same pivot
        const double r = rsqrt(d);
        for (int j = k + 1 + threadIdx.x; j < n; j += T) S[k + j * LD] *= r;
        __syncthreads();
        // The pivot is read by all threads above; it is overwritten only now.
        if (threadIdx.x == 0) S[k + k * LD] = d * r;
        const int m = n - k - 1;
        const int cnt = m * (m + 1) / 2;
        for (int e = threadIdx.x; e < cnt; e += T) {
            const int c = tri_col(e);
            const int i = k + 1 + (e - c * (c + 1) / 2), j = k + 1 + c;
            S[i + j * LD] = fma(-S[k + i * LD], S[k + j * LD], S[i + j * LD]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int i = e % n, j = e / n;
        if (i <= j && i < done) X[i + (long)j * ldx] = S[i + j * LD];
    }
    return fail;
}

// --------------------------------------------------------------- kernels

__device__ __forceinline__ bool next_instance(const Sched &s, int group, int *s_slot, int &b)
{
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    const int w = lo + claim_slot(s.meta + META_HEAD + group, s_slot);
    if (w >= hi) return false;
    b = s.perm[w];
    return true;
}

template <int B, int T, int VAR>
__global__ void __launch_bounds__(T) potrf_fp64_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    __shared__ int s_slot;
    int b;
    claim_init(&s_slot);
    while (next_instance(s, group, &s_slot, b)) {
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        potrf_instance<B, T, VAR>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], o.info + b, sm);
    }
}

// Right-looking shared-memory Cholesky for n <= NMAX; larger n in the same
// call take the blocked lazy path (B = 16, one-warp diagonal blocks).
template <int NMAX, int T>
__global__ void __launch_bounds__(T) potrf_rl_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    __shared__ int s_slot;
    int b;
    claim_init(&s_slot);
    while (next_instance(s, group, &s_slot, b)) {
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        if (n <= NMAX) {
            const int f = chol_rl_smem<NMAX, T>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], sm);
            if (threadIdx.x == 0) o.info[b] = f;
            __syncthreads();
        } else {
            potrf_instance<16, T, 1>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], o.info + b, sm);
        }
    }
}

template <int B, int T, bool LYAP, int VAR>
__global__ void __launch_bounds__(T) syl_fp64_kernel(Operands o, Sched s, int group)
{
    extern __shared__ double sm[];
    __shared__ int s_slot;
    int b;
    claim_init(&s_slot);
    while (next_instance(s, group, &s_slot, b)) {
        const int n = o.n[b], m = o.m != nullptr ? o.m[b] : n;
        if (n == 0 || m == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        syl_instance<B, T, LYAP, VAR>(m, n, o.A[b], o.lda[b], LYAP ? nullptr : o.U[b], LYAP ? 0 : o.ldu[b],
                                 o.C[b], o.ldc[b], o.X[b], o.ldx[b], o.info + b, sm);
    }
}

template <typename K>
cudaError_t launch_persistent(K kernel, int threads, size_t smem, int batch, cudaStream_t st,
                              const Operands &o, const Sched &s, int group)
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

}  // namespace

// The (B, T, diagonal variant: 0 CTA-wide, 1 one warp) instantiations the
// FP64 configuration tables (api.cu) draw from, per operation.
#define SS_POTRF_CONFIGS(X) X(16, 64, 0) X(32, 128, 0) X(32, 256, 0) X(16, 64, 1) X(16, 128, 1)
#define SS_SYL_CONFIGS(X) X(8, 64, 0) X(16, 64, 0) X(16, 128, 0) X(32, 128, 0) X(16, 128, 1)

cudaError_t launch_potrf_fp64(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st)
{
    const Config *c = config_get(SS_OP_POTRF, SS_MODE_FP64, l.cfg);
    if (c == nullptr) return cudaErrorInvalidValue;
    if (c->variant == 2) return launch_potrf_ws(c->block, (c->threads - 32) / 32, false, o, s, l, st, false);
    if (c->variant == 3 && c->block == 64 && c->threads == 128) {
        constexpr size_t rl = (size_t)64 * 65 * sizeof(double);
        const size_t smem = rl > smem_bytes<16>() ? rl : smem_bytes<16>();
        return launch_persistent(potrf_rl_kernel<64, 128>, 128, smem, l.batch, st, o, s, l.group);
    }
#define CASE(B, T, V) \
    if (c->block == B && c->threads == T && c->variant == V) \
        return launch_persistent(potrf_fp64_kernel<B, T, V>, T, smem_bytes<B>(), l.batch, st, o, s, l.group);
    SS_POTRF_CONFIGS(CASE)
#undef CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_syl_fp64(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, bool lyap)
{
    const Config *c = config_get(lyap ? SS_OP_TRLYAP : SS_OP_TRSYL, SS_MODE_FP64, l.cfg);
    if (c == nullptr) return cudaErrorInvalidValue;
    if (c->variant == 2) return launch_syl_ws(c->block, (c->threads - 32) / 32, lyap, false, o, s, l, st, false);
#define CASE(B, T, V)                                                                                    \
    if (c->block == B && c->threads == T && c->variant == V)                                             \
        return lyap ? launch_persistent(syl_fp64_kernel<B, T, true, V>, T, smem_bytes<B>(), l.batch, st, o, s, l.group) \
                    : launch_persistent(syl_fp64_kernel<B, T, false, V>, T, smem_bytes<B>(), l.batch, st, o, s, l.group);
    SS_SYL_CONFIGS(CASE)
#undef CASE
    return cudaErrorInvalidValue;
}

}  // namespace ss
