// Mixed-precision upper Cholesky X^T X = A (Fig. 2a) with FP64-accurate
// refinement of the factor.
//
// Per instance (one CTA, lazy blocked order as the FP64 kernel):
//   1. X0 = low-precision factor of A: block updates A_IJ - sum X_KI^T X_KJ in
//      FP32 FMA (CUDA cores) or TF32 / BF16 on the tensor cores (mma.sync,
//      FP32 accumulation); in the diagonal blocks the pivots' square roots and
//      reciprocals are computed in FP64.
//   2. Refinement of the factor (a Newton step on X^T X = A): with
//        E = A - X^T X                    (FP64-class accuracy: double-float on
//                                          the FP32 pipe, or FP64 FMA),
//        F = X^{-T} E X^{-1}              (two FP32 triangular solves),
//        M = Phi(F)  (strict upper triangle of F plus half its diagonal),
//      X <- X + M X.  Since X^T (M X) + (M X)^T X = F' with F' = X^T F X = E,
//      the step removes E to first order; the remaining error is the square of
//      the previous one plus the FP32 rounding of the correction.  Stop as the
//      Sylvester driver does (|D| or |D|^2/|D_prev| below SS_REFINE_TOL |X|).
// The instance is rescaled by powers of two first (DfScale::cholesky: A by
// 4^s, X by 2^s; F is unchanged), each FP64 value shifted as it is converted;
// X in global memory stays in the caller's units.
// Scratch: two n x n float buffers (W1, W2, ld n).
//
// The tensor-memory variant (TF32 / BF16, n <= 256) replaces step 1 by a
// right-looking factorization whose whole trailing matrix stays on chip as
// the FP32 accumulator of the fifth-generation tensor cores: per block row
// of 32, the warp that owns those TMEM lanes reads the panel out, the CTA
// factors its diagonal block and solves the panel (FP32, FP64 pivots), and
// one thread issues the SYRK update A' -= P^T P of the trailing matrix as
// 128-row MMA tiles (umma.cuh).  Refinement is the same.
#include "mixed.cuh"
#include "umma.cuh"

namespace ss {
namespace mx {
namespace {

template <int B>
constexpr size_t chol_smem_bytes() { return (size_t)5 * FTile<B>::SZ * sizeof(float) + 64 * sizeof(float) + 2 * B * sizeof(float); }

// Factor the m x m upper block in sT in place (FP32 dots; square root and
// reciprocal of each pivot in FP64).  Returns 0 or the failing pivot + 1.
template <int B, int T>
__device__ int chol_diag_f(float *sT, int m, float *s_scal)
{
    constexpr int LD = FTile<B>::LD;
    for (int i = 0; i < m; ++i) {
        const int cnt = m - i;
        const int split = pick_split<T>(cnt, i);
        if (warp_has_work(cnt, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < cnt;
            const int j = i + (act ? idx : 0);
            float s = 0.0f;
            if (act)
                for (int k = part; k < i; k += split) s = fmaf(sT[k + i * LD], sT[k + j * LD], s);
            s = group_sum_f(s, split);
            if (act && part == 0) sT[i + j * LD] -= s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double d = f2d_exact(sT[i + i * LD]);
            if (d > 0.0) {
                const double p = sqrt(d);
                sT[i + i * LD] = d2f_trunc(p);
                s_scal[0] = d2f_trunc(1.0 / p);
                s_scal[1] = 0.0f;
            } else {
                s_scal[1] = 1.0f;
            }
        }
        __syncthreads();
        if (s_scal[1] != 0.0f) return i + 1;
        const float rinv = s_scal[0];
        for (int j = i + 1 + threadIdx.x; j < m; j += T) sT[i + j * LD] *= rinv;
        __syncthreads();
    }
    return 0;
}

// Solve D^T Y = T in place for the m x nn block in sT, D upper triangular in
// sD with reciprocal diagonal s_rinv (row i of Y needs rows < i only).
template <int B, int T>
__device__ void trsm_ut_f(const float *sD, const float *s_rinv, float *sT, int m, int nn)
{
    constexpr int LD = FTile<B>::LD;
    for (int i = 0; i < m; ++i) {
        const int split = pick_split<T>(nn, i);
        if (warp_has_work(nn, split)) {
            const int idx = threadIdx.x / split, part = threadIdx.x % split;
            const bool act = idx < nn;
            const int j = act ? idx : 0;
            float s = 0.0f;
            if (act)
                for (int k = part; k < i; k += split) s = fmaf(sD[k + i * LD], sT[k + j * LD], s);
            s = group_sum_f(s, split);
            if (act && part == 0) sT[i + j * LD] = (sT[i + j * LD] - s) * s_rinv[i];
        }
        __syncthreads();
    }
}

// Stage the upper-triangular diagonal block X_II (FP64 source, scaled by
// 2^shx) as floats and its reciprocal diagonal computed in FP64.
template <int B, int T>
__device__ void stage_pivots(float *sD, float *s_rinv, const double *X, long ldx, int i0, int m, int shx)
{
    stage_f<B, T, F_UPPER>(sD, X + i0 + (long)i0 * ldx, ldx, m, m, shx);
    for (int i = threadIdx.x; i < m; i += T) s_rinv[i] = d2f_trunc_s(1.0 / X[(i0 + i) + (long)(i0 + i) * ldx], -shx);
    __syncthreads();
}

// Low-precision factor of A into W (upper triangle, ld n).  Returns 0 or the
// failing leading minor.
template <int B, int T, int P>
__device__ int chol_low(int n, const double *A, long lda, float *W, float *sm, int sha)
{
    constexpr int LD = FTile<B>::LD, SZ = FTile<B>::SZ, E = B * B / T;
    float *sA = sm, *sB = sm + SZ, *sT = sm + 2 * SZ, *sD = sm + 3 * SZ;
    float *s_rinv = sm + 5 * SZ + 64, *s_scal = sm + 5 * SZ;
    const int nb = (n + B - 1) / B;
    const long ldw = n;
    Slots<B, T> sl;
    for (int J = 0; J < nb; ++J) {
        const int nJ = min(B, n - J * B), j0 = J * B;
        for (int I = 0; I <= J; ++I) {
            const int i0 = I * B;
            const bool diag = I == J;
            const int mI = diag ? nJ : B;
            __syncthreads();
            if (diag) stage_f<B, T, F_UPPER>(sT, A + i0 + (long)j0 * lda, lda, mI, nJ, sha);
            else stage_f<B, T, F_FULL>(sT, A + i0 + (long)j0 * lda, lda, mI, nJ, sha);
            __syncthreads();
            float acc[E];
            float frag[FragN<B, T, P>::value][4];
            if constexpr (P == P_FP32) {
                sl.set(Shape::Full, mI, nJ);
#pragma unroll
                for (int r = 0; r < E; ++r) acc[r] = sl.ok(r) ? sT[sl.row[r] + sl.col[r] * LD] : 0.0f;
            } else {
                frag_load<B, T>(frag, sT);
            }
            for (int K = 0; K < I; ++K) {
                const int k0 = K * B;
                __syncthreads();
                stage_f<B, T, F_FULL>(sA, W + k0 + (long)i0 * ldw, ldw, B, mI, 0);   // X_KI
                stage_f<B, T, F_FULL>(sB, W + k0 + (long)j0 * ldw, ldw, B, nJ, 0);   // X_KJ
                __syncthreads();
                if constexpr (P == P_FP32) slot_update_f<B, T, true, false>(acc, sl, sA, sB, B);
                else mma_update<B, T, P, true, false>(frag, sA, sB, B);
            }
            __syncthreads();
            if constexpr (P == P_FP32) {
#pragma unroll
                for (int r = 0; r < E; ++r)
                    if (sl.ok(r)) sT[sl.row[r] + sl.col[r] * LD] = acc[r];
            } else {
                frag_store<B, T>(frag, sT);
            }
            __syncthreads();
            if (!diag) {
                stage_f<B, T, F_UPPER>(sD, W + i0 + (long)i0 * ldw, ldw, B, B, 0);
                // Pivot reciprocals in FP64 from the stored FP32 diagonal.
                for (int i = threadIdx.x; i < B; i += T) s_rinv[i] = d2f_trunc(1.0 / f2d_exact(W[(i0 + i) + (long)(i0 + i) * ldw]));
                __syncthreads();
                trsm_ut_f<B, T>(sD, s_rinv, sT, B, nJ);
            } else {
                const int f = chol_diag_f<B, T>(sT, nJ, s_scal);
                if (f) return j0 + f;
            }
            for (int e = threadIdx.x; e < mI * nJ; e += T) {
                const int r = e % mI, c = e / mI;
                if (!diag || r <= c) W[(i0 + r) + (long)(j0 + c) * ldw] = sT[r + c * LD];
            }
        }
    }
    __syncthreads();
    return 0;
}

// ---- Tensor-memory (tcgen05) variant of step 1 ----------------------------
constexpr int TCB = 32, TCT = 128, TCLD = TCB + 1, TCMAXN = 256;

template <int KIND>
constexpr size_t tc_q_bytes() { return (size_t)TCMAXN * TCB * tc::KindTraits<KIND>::ES; }
// Float region: the panel (TCLD x TCMAXN; the refinement's tiles reuse it),
// 64 pivot scalars, 32 pivot reciprocals.
constexpr int TC_FLOATS = TCLD * TCMAXN + 64 + TCB;
static_assert(chol_smem_bytes<32>() <= (size_t)TCLD * TCMAXN * sizeof(float), "refinement tiles fit the panel");
template <int KIND>
constexpr size_t tc_chol_smem_bytes() { return 1024 + tc_q_bytes<KIND>() + (size_t)TC_FLOATS * sizeof(float) + 16; }

struct TcChol {
    unsigned char *q;    // SYRK operand, K-major, TCMAXN rows x 32
    float *sm;           // panel P (column-major, ld TCLD) / refinement tiles
    float *s_scal, *s_rinv;
    uint64_t *mbar;      // MMA completion
    uint32_t *slot;      // TMEM base address
};

template <int KIND>
__device__ TcChol tc_chol_carve(unsigned char *raw)
{
    TcChol c;
    const uint32_t mis = tc::smem_u32(raw) & 1023u;
    c.q = raw + ((1024u - mis) & 1023u);
    c.sm = reinterpret_cast<float *>(c.q + tc_q_bytes<KIND>());
    c.s_scal = c.sm + TCLD * TCMAXN;
    c.s_rinv = c.s_scal + 64;
    c.mbar = reinterpret_cast<uint64_t *>(c.sm + TC_FLOATS);
    c.slot = reinterpret_cast<uint32_t *>(c.mbar + 1);
    return c;
}

// Low-precision factor of A (n <= TCMAXN) into W (upper, ld n) with the
// trailing matrix in TMEM as -A' (tile 0: rows 0..127 x columns 0..255;
// tile 1: rows 128..255 x columns 128..255 at TMEM columns 256..383).
// Returns 0, the failing leading minor, or -1 if a bounded wait for the
// tensor cores ran out (the CTA must then stop).  `phase` is the mbarrier
// parity, carried across calls.
template <int KIND>
__device__ int chol_low_tc(int n, const double *A, long lda, float *W, const TcChol &c, uint32_t &phase, int sha)
{
    constexpr int KS = TCB / tc::KindTraits<KIND>::KSTEP;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nr = (n + 15) & ~15;
    const bool two = n > 128;
    const uint32_t ncols = two ? 512u : 128u;
    float *P = c.sm;
    if (warp == 0) tc::tmem_alloc(c.slot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t base = *c.slot;
    {
        const int i = 32 * warp + lane;
        for (int cc = 0; cc < nr; cc += 16) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = cc + q;
                v[q] = (i <= j && j < n) ? -d2f_trunc_s(A[i + (long)j * lda], sha) : 0.0f;
            }
            tc::st16(tc::taddr(base, warp, cc), v);
        }
        if (two) {
            const int i1 = 128 + i;
            for (int cc = 128; cc < nr; cc += 16) {
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = cc + q;
                    v[q] = (i1 <= j && j < n) ? -d2f_trunc_s(A[i1 + (long)j * lda], sha) : 0.0f;
                }
                tc::st16(tc::taddr(base, warp, 256 + cc - 128), v);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int nb = (n + TCB - 1) / TCB;
    const int rq = two ? 256 : 128;
    int fail = 0;
    for (int K = 0; K < nb; ++K) {
        const int k0 = K * TCB, kb = min(TCB, n - k0), w = n - k0;
        // Panel rows k0 .. k0 + 31 (columns k0 .. n-1) out of TMEM.
        if (warp == ((k0 & 127) >> 5)) {
            for (int cc = k0; cc < nr; cc += 16) {
                float v[16];
                tc::ld16(tc::taddr(base, warp, k0 >= 128 ? 256 + cc - 128 : cc), v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = cc + q - k0;
                    if (j < w) P[lane + j * TCLD] = -v[q];
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        const int f = chol_diag_f<TCB, TCT>(P, kb, c.s_scal);
        if (f) { fail = k0 + f; break; }
        for (int i = tid; i < kb; i += TCT) c.s_rinv[i] = d2f_trunc(1.0 / f2d_exact(P[i + i * TCLD]));
        __syncthreads();
        // Panel solve X_KK^T Y = P[:, kb:], one column per thread (kb = 32 here).
        for (int j = kb + tid; j < w; j += TCT) {
            float y[TCB];
#pragma unroll
            for (int i = 0; i < TCB; ++i) y[i] = P[i + j * TCLD];
#pragma unroll
            for (int i = 0; i < TCB; ++i) {
                float sacc = y[i];
#pragma unroll
                for (int k = 0; k < i; ++k) sacc = fmaf(-P[k + i * TCLD], y[k], sacc);
                y[i] = sacc * c.s_rinv[i];
            }
#pragma unroll
            for (int i = 0; i < TCB; ++i) P[i + j * TCLD] = y[i];
        }
        __syncthreads();
        for (int e = tid; e < kb * w; e += TCT) {
            const int r = e % kb, j = e / kb;
            if (j >= r) W[(k0 + r) + (long)(k0 + j) * n] = P[r + j * TCLD];
        }
        const int c0 = k0 + kb;
        if (c0 >= n) break;
        // Operand rows r = trailing-matrix indices, K = the panel's 32 rows;
        // rows outside [c0, n) are zero (rows below k0 already are).
        const int r0 = K == 0 ? 0 : k0;
        for (int e = tid; e < (rq - r0) * TCB; e += TCT) {
            const int r = r0 + e / TCB, k = e % TCB;
            tc::op_store<KIND>(c.q, r, k, TCB, (r >= c0 && r < n) ? P[k + (r - k0) * TCLD] : 0.0f);
        }
        tc::fence_smem_to_async();
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            if (c0 < 128) {
                const uint32_t id = tc::idesc<KIND>(128, nr - c0, false);
#pragma unroll
                for (int sk = 0; sk < KS; ++sk)
                    tc::mma<KIND>(base + c0, tc::op_desc<KIND>(c.q, 0, sk, TCB), tc::op_desc<KIND>(c.q, c0, sk, TCB),
                                  id, true);
            }
            if (two) {
                const int c1 = max(c0, 128);
                const uint32_t id = tc::idesc<KIND>(128, nr - c1, false);
#pragma unroll
                for (int sk = 0; sk < KS; ++sk)
                    tc::mma<KIND>(base + 256 + (c1 - 128), tc::op_desc<KIND>(c.q, 128, sk, TCB),
                                  tc::op_desc<KIND>(c.q, c1, sk, TCB), id, true);
            }
            tc::commit(c.mbar);
        }
        const bool ok = tc::mbar_wait(c.mbar, phase);
        if (__syncthreads_or(!ok)) {
            tc::mbar_wait(c.mbar, phase, 1u << 26);
            fail = -1;
            break;
        }
        phase ^= 1u;
        tc::fence_after();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(base, ncols);
    return fail;
}

// E = A - X^T X (X: FP64 upper factor), all blocks I <= J, written to W in
// full (both triangles, E is symmetric).
template <int B, int T, int RS>
__device__ void chol_residual(int n, const double *A, long lda, const double *X, long ldx, float *W,
                              float *sm, const DfScale &sc)
{
    constexpr int E = B * B / T;
    using Elem = typename std::conditional<RS == R_DF, float2, double>::type;
    Elem *sA = reinterpret_cast<Elem *>(sm);
    Elem *sB = sA + FTile<B>::SZ;
    const int nb = (n + B - 1) / B;
    const long ldw = n;
    Slots<B, T> sl;
    for (int J = 0; J < nb; ++J) {
        const int nJ = min(B, n - J * B), j0 = J * B;
        for (int I = 0; I <= J; ++I) {
            const int i0 = I * B, mI = min(B, n - i0);
            sl.set(Shape::Full, mI, nJ);
            float ah[E], al[E];
            double ad[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                ah[r] = 0.f; al[r] = 0.f; ad[r] = 0.0;
                if (sl.ok(r)) {
                    int rr = i0 + sl.row[r], cc = j0 + sl.col[r];
                    if (rr > cc) { const int t = rr; rr = cc; cc = t; }   // upper triangle of A
                    const double a = A[rr + (long)cc * lda];
                    if constexpr (RS == R_DF) split_df_s(a, sc.op, ah[r], al[r]);
                    else ad[r] = Pow2(sc.op)(a);
                }
            }
            for (int K = 0; K <= I; ++K) {
                const int k0 = K * B, kw = min(B, n - k0);
                __syncthreads();
                // X_KI (upper when K == I) and X_KJ (upper when K == J).
                if constexpr (RS == R_DF) {
                    float2 *a2 = reinterpret_cast<float2 *>(sA), *b2 = reinterpret_cast<float2 *>(sB);
                    if (K == I) stage_df<B, T, F_UPPER>(a2, X + k0 + (long)i0 * ldx, ldx, kw, mI, sc.x);
                    else stage_df<B, T, F_FULL>(a2, X + k0 + (long)i0 * ldx, ldx, kw, mI, sc.x);
                    if (K == J) stage_df<B, T, F_UPPER>(b2, X + k0 + (long)j0 * ldx, ldx, kw, nJ, sc.x);
                    else stage_df<B, T, F_FULL>(b2, X + k0 + (long)j0 * ldx, ldx, kw, nJ, sc.x);
                    __syncthreads();
                    slot_update_df<B, T, true, false>(ah, al, sl, a2, b2, kw);
                } else {
                    double *a = reinterpret_cast<double *>(sA), *b = reinterpret_cast<double *>(sB);
                    if (K == I) stage_d<B, T, F_UPPER>(a, X + k0 + (long)i0 * ldx, ldx, kw, mI, sc.x);
                    else stage_d<B, T, F_FULL>(a, X + k0 + (long)i0 * ldx, ldx, kw, mI, sc.x);
                    if (K == J) stage_d<B, T, F_UPPER>(b, X + k0 + (long)j0 * ldx, ldx, kw, nJ, sc.x);
                    else stage_d<B, T, F_FULL>(b, X + k0 + (long)j0 * ldx, ldx, kw, nJ, sc.x);
                    __syncthreads();
                    slot_update<B, T, true, false>(ad, sl, a, b, kw);
                }
            }
#pragma unroll
            for (int r = 0; r < E; ++r) {
                if (sl.ok(r)) {
                    const float v = RS == R_DF ? __fadd_rn(ah[r], al[r]) : (float)ad[r];
                    const int rr = i0 + sl.row[r], cc = j0 + sl.col[r];
                    W[rr + (long)cc * ldw] = v;
                    W[cc + (long)rr * ldw] = v;
                }
            }
        }
    }
    __syncthreads();
}

// Z = X^{-T} R in place on W (n x n, ld n) with X the FP64 upper factor
// (staged as FP32; pivot reciprocals in FP64).  With TRANS the right-hand
// side is read from Wsrc transposed (R = Wsrc^T) and the result goes to W.
template <int B, int T, bool TRANS>
__device__ void trsm_ut_blocked(int n, const double *X, long ldx, const float *Wsrc, float *W, float *sm, int shx)
{
    constexpr int LD = FTile<B>::LD, SZ = FTile<B>::SZ, E = B * B / T;
    float *sA = sm, *sB = sm + SZ, *sT = sm + 2 * SZ, *sD = sm + 3 * SZ;
    float *s_rinv = sm + 5 * SZ + 64;
    const int nb = (n + B - 1) / B;
    const long ldw = n;
    Slots<B, T> sl;
    for (int I = 0; I < nb; ++I) {
        const int i0 = I * B, mI = min(B, n - i0);
        __syncthreads();
        stage_pivots<B, T>(sD, s_rinv, X, ldx, i0, mI, shx);
        for (int J = 0; J < nb; ++J) {
            const int j0 = J * B, nJ = min(B, n - j0);
            sl.set(Shape::Full, mI, nJ);
            float acc[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                acc[r] = 0.0f;
                if (sl.ok(r)) {
                    const int rr = i0 + sl.row[r], cc = j0 + sl.col[r];
                    acc[r] = TRANS ? Wsrc[cc + (long)rr * ldw] : W[rr + (long)cc * ldw];
                }
            }
            for (int K = 0; K < I; ++K) {
                const int k0 = K * B;
                __syncthreads();
                stage_f<B, T, F_FULL>(sA, X + k0 + (long)i0 * ldx, ldx, B, mI, shx);   // X_KI
                stage_f<B, T, F_FULL>(sB, W + k0 + (long)j0 * ldw, ldw, B, nJ, 0);     // Z_KJ
                __syncthreads();
                slot_update_f<B, T, true, false>(acc, sl, sA, sB, B);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < E; ++r)
                if (sl.ok(r)) sT[sl.row[r] + sl.col[r] * LD] = acc[r];
            __syncthreads();
            trsm_ut_f<B, T>(sD, s_rinv, sT, mI, nJ);
            for (int e = threadIdx.x; e < mI * nJ; e += T) {
                const int r = e % mI, c = e / mI;
                W[(i0 + r) + (long)(j0 + c) * ldw] = sT[r + c * LD];
            }
        }
    }
    __syncthreads();
}

// D = Phi(F) X (upper, F in Wf) into Wd (upper blocks), then X += D in FP64.
// Returns |D|_F^2.
template <int B, int T>
__device__ float chol_correct(int n, double *X, long ldx, const float *Wf, float *Wd, float *sm,
                              float *s_red, int shx)
{
    constexpr int LD = FTile<B>::LD, SZ = FTile<B>::SZ, E = B * B / T;
    float *sA = sm, *sB = sm + SZ;
    const int nb = (n + B - 1) / B;
    const long ldw = n;
    Slots<B, T> sl;
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * B, nJ = min(B, n - j0);
        for (int I = 0; I <= J; ++I) {
            const int i0 = I * B, mI = min(B, n - i0);
            sl.set(Shape::Full, mI, nJ);
            float acc[E];
#pragma unroll
            for (int r = 0; r < E; ++r) acc[r] = 0.0f;
            // D_IJ = sum_{I <= K <= J} M_IK X_KJ with M = Phi(F).
            for (int K = I; K <= J; ++K) {
                const int k0 = K * B, kw = min(B, n - k0);
                __syncthreads();
                for (int e = threadIdx.x; e < B * B; e += T) {
                    const int r = e % B, c = e / B;
                    float v = 0.0f;
                    const int gr = i0 + r, gc = k0 + c;
                    if (r < mI && c < kw && gr <= gc) {
                        v = Wf[gr + (long)gc * ldw];
                        if (gr == gc) v *= 0.5f;
                    }
                    sA[r + c * LD] = v;
                }
                if (K == J) stage_f<B, T, F_UPPER>(sB, X + k0 + (long)j0 * ldx, ldx, kw, nJ, shx);
                else stage_f<B, T, F_FULL>(sB, X + k0 + (long)j0 * ldx, ldx, kw, nJ, shx);
                __syncthreads();
                // acc += M X : slot_update_f subtracts, so negate via the sign of M.
                slot_update_f<B, T, false, false>(acc, sl, sA, sB, kw);
            }
#pragma unroll
            for (int r = 0; r < E; ++r)
                if (sl.ok(r)) Wd[(i0 + sl.row[r]) + (long)(j0 + sl.col[r]) * ldw] = -acc[r];
        }
    }
    __syncthreads();
    float ss = 0.0f;
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int r = e % n, c = e / n;
        if (r > c) continue;
        const float d = Wd[e];
        ss = fmaf(d, d, ss);
        X[r + (long)c * ldx] += f2d_exact_s(d, -shx);
    }
    return block_sum_f(ss, s_red);
}

template <int T>
__device__ DfScale chol_scale(int n, const double *A, long lda, float *s_red)
{
    int ea, dummy;
    scan_exp3(ScanOp{A, lda, n, n, 2}, ScanOp{nullptr, 0, 0, 0, 0}, ScanOp{nullptr, 0, 0, 0, 0}, threadIdx.x >> 5, T / 32,
              threadIdx.x & 31, ea, dummy);
    cta_max2(ea, dummy, reinterpret_cast<int *>(s_red));
    return DfScale::cholesky(ea);
}

// X = the low-precision factor in W1, then (unless raw) the refinement.
template <int B, int T, int RS>
__device__ void chol_refine(int n, const double *A, long lda, double *X, long ldx, int *info, float *W1, float *W2,
                            bool raw, float *sm, const DfScale &sc)
{
    float *s_red = sm + 5 * FTile<B>::SZ;
    float ss = 0.0f;
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int r = e % n, c = e / n;
        if (r > c) continue;
        const float v = W1[e];
        ss = fmaf(v, v, ss);
        X[r + (long)c * ldx] = f2d_exact_s(v, -sc.x);
    }
    const float nx = sqrtf(block_sum_f(ss, s_red));
    int conv = raw || nx == 0.0f;
    float prev = nx;
    for (int it = 0; it < MAXIT && !conv; ++it) {
        chol_residual<B, T, RS>(n, A, lda, X, ldx, W1, sm, sc);        // E -> W1
        trsm_ut_blocked<B, T, false>(n, X, ldx, W1, W1, sm, sc.x);     // Y = X^-T E in W1
        trsm_ut_blocked<B, T, true>(n, X, ldx, W1, W2, sm, sc.x);      // F = X^-T Y^T in W2
        const float nd = sqrtf(chol_correct<B, T>(n, X, ldx, W2, W1, sm, s_red, sc.x));
        const float pred = prev > 0.0f ? nd * (nd / prev) : nd;
        conv = (nd <= (float)SS_REFINE_TOL * nx) || (pred <= (float)SS_REFINE_TOL * nx);
        prev = nd;
    }
    if (threadIdx.x == 0) *info = conv ? 0 : n + 1;
}

template <int B, int T, int P, int RS>
__device__ void chol_mixed_instance(int n, const double *A, long lda, double *X, long ldx, int *info,
                                    float *W1, float *W2, bool raw, float *sm)
{
    const DfScale sc = chol_scale<T>(n, A, lda, sm + 5 * FTile<B>::SZ);
    const int f = chol_low<B, T, P>(n, A, lda, W1, sm, sc.op);
    if (f) {
        if (threadIdx.x == 0) *info = f;
        return;
    }
    chol_refine<B, T, RS>(n, A, lda, X, ldx, info, W1, W2, raw, sm, sc);
}

template <int B, int T, int P, int RS>
__global__ void __launch_bounds__(T, 1024 / T) chol_mixed_kernel(Operands o, Sched s, int group, int raw)
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
        if (!raw && o.X[b] == o.A[b]) { if (threadIdx.x == 0) o.info[b] = SS_INFO_ALIASED; continue; }
        const long long off = s.scr[w];
        if (off + 2ll * n * n > s.scratch_elems) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
            continue;
        }
        float *W1 = static_cast<float *>(s.scratch) + off;
        chol_mixed_instance<B, T, P, RS>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], o.info + b, W1,
                                         W1 + (long)n * n, raw != 0, smf);
    }
}

// Tensor-memory variant, pass 1: the low-precision factor of every instance
// into W1 (TF32 or BF16 SYRK updates on the tensor cores for n <= 256, the
// blocked path above), info = 0 or the failing minor.  Few CTAs per SM fit
// (TMEM, shared memory), so the refinement runs as pass 2.
template <int P>
__global__ void __launch_bounds__(TCT) chol_tc_factor_kernel(Operands o, Sched s, int group, int raw)
{
    constexpr int KIND = P == P_TF32 ? tc::K_TF32 : tc::K_BF16;
    extern __shared__ unsigned char smraw[];
    __shared__ int s_slot;
    const TcChol c = tc_chol_carve<KIND>(smraw);
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    claim_init(&s_slot);
    if (threadIdx.x == 0) tc::mbar_init(c.mbar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        const int w = lo + claim_slot(s.meta + META_HEAD + group, &s_slot);
        if (w >= hi) break;
        const int b = s.perm[w];
        const int n = o.n[b];
        if (n == 0) { if (threadIdx.x == 0) o.info[b] = 0; continue; }
        if (!raw && o.X[b] == o.A[b]) { if (threadIdx.x == 0) o.info[b] = SS_INFO_ALIASED; continue; }
        const long long off = s.scr[w];
        if (off + 2ll * n * n > s.scratch_elems) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
            continue;
        }
        float *W1 = static_cast<float *>(s.scratch) + off;
        const DfScale sc = chol_scale<TCT>(n, o.A[b], o.lda[b], c.sm);
        const int f = n <= TCMAXN ? chol_low_tc<KIND>(n, o.A[b], o.lda[b], W1, c, phase, sc.op)
                                  : chol_low<TCB, TCT, P>(n, o.A[b], o.lda[b], W1, c.sm, sc.op);
        if (threadIdx.x == 0) o.info[b] = f < 0 ? SS_INFO_TIMEOUT : f;
        if (f < 0) break;
    }
}

// Pass 2: X from W1 and the refinement, for every instance pass 1 left at
// info = 0 (its own queue: the group's second-pass head).
template <int P, int RS>
__global__ void __launch_bounds__(TCT, 1024 / TCT) chol_tc_refine_kernel(Operands o, Sched s, int group, int raw)
{
    extern __shared__ __align__(16) float smf[];
    __shared__ int s_slot;
    const int lo = s.meta[META_RANGE + 2 * group], hi = s.meta[META_RANGE + 2 * group + 1];
    claim_init(&s_slot);
    for (;;) {
        const int w = lo + claim_slot(s.meta + META_SCL_HEAD + group, &s_slot);
        if (w >= hi) break;
        const int b = s.perm[w];
        const int n = o.n[b];
        if (n == 0 || o.info[b] != 0) continue;
        float *W1 = static_cast<float *>(s.scratch) + s.scr[w];
        const DfScale sc = chol_scale<TCT>(n, o.A[b], o.lda[b], smf + 5 * FTile<TCB>::SZ);
        chol_refine<TCB, TCT, RS>(n, o.A[b], o.lda[b], o.X[b], o.ldx[b], o.info + b, W1, W1 + (long)n * n,
                                  raw != 0, smf, sc);
    }
}

template <int P, int RS>
cudaError_t launch_chol_tc(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, int raw)
{
    constexpr int KIND = P == P_TF32 ? tc::K_TF32 : tc::K_BF16;
    auto k1 = chol_tc_factor_kernel<P>;
    auto k2 = chol_tc_refine_kernel<P, RS>;
    const size_t smem1 = tc_chol_smem_bytes<KIND>(), smem2 = chol_smem_bytes<TCB>();
    cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    int per1 = 0, per2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k1, TCT, smem1);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, TCT, smem2);
    if (e != cudaSuccess) return e;
    // TMEM: 128 columns per CTA for n <= 128 (512 per SM).
    per1 = per1 > 4 ? 4 : (per1 < 1 ? 1 : per1);
    per2 = per2 < 1 ? 1 : per2;
    long g1 = (long)per1 * sm_count(), g2 = (long)per2 * sm_count();
    if (g1 > l.batch) g1 = l.batch;
    if (g2 > l.batch) g2 = l.batch;
    k1<<<(int)(g1 < 1 ? 1 : g1), TCT, smem1, st>>>(o, s, l.group, raw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k2<<<(int)(g2 < 1 ? 1 : g2), TCT, smem2, st>>>(o, s, l.group, raw);
    return cudaGetLastError();
}

template <int B, int T, int P, int RS>
cudaError_t launch_chol(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, int raw)
{
    auto kern = chol_mixed_kernel<B, T, P, RS>;
    const size_t smem = chol_smem_bytes<B>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long grid = (long)per_sm * sm_count();
    if (grid > l.batch) grid = l.batch;
    if (grid < 1) grid = 1;
    kern<<<(int)grid, T, smem, st>>>(o, s, l.group, raw);
    return cudaGetLastError();
}

}  // namespace
}  // namespace mx

// cfg -> (B, T, residual) per precision; mirrored by the potrf table in mixed_api.cu.
cudaError_t launch_mixed_potrf(int prec, int cfg, const Operands &o, const Sched &s, const Launch &l,
                               cudaStream_t st, int raw)
{
    using namespace mx;
    if (prec == P_FP32) {
        switch (cfg) {
        case 0: return launch_chol<16, 64, P_FP32, R_DF>(o, s, l, st, raw);
        case 1: return launch_chol<16, 128, P_FP32, R_DF>(o, s, l, st, raw);
        case 2: return launch_chol<32, 128, P_FP32, R_DF>(o, s, l, st, raw);
        case 3: return launch_chol<32, 128, P_FP32, R_FP64>(o, s, l, st, raw);
        }
    } else if (prec == P_TF32) {
        switch (cfg) {
        case 0: return launch_chol<16, 64, P_TF32, R_DF>(o, s, l, st, raw);
        case 1: return launch_chol<32, 128, P_TF32, R_DF>(o, s, l, st, raw);
        case 2: return launch_chol<32, 128, P_TF32, R_FP64>(o, s, l, st, raw);
        case 3: return launch_chol_tc<P_TF32, R_DF>(o, s, l, st, raw);
        }
    } else if (prec == P_BF16) {
        switch (cfg) {
        case 0: return launch_chol<16, 64, P_BF16, R_DF>(o, s, l, st, raw);
        case 1: return launch_chol<32, 128, P_BF16, R_DF>(o, s, l, st, raw);
        case 2: return launch_chol<32, 128, P_BF16, R_FP64>(o, s, l, st, raw);
        case 3: return launch_chol_tc<P_BF16, R_DF>(o, s, l, st, raw);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace ss
