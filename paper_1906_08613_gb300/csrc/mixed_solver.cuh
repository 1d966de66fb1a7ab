// Mixed-precision Sylvester / Lyapunov instance driver and persistent kernel
// (see mixed.cuh for the method).  Included by mixed_syl.cu (Sylvester) and
// mixed_lyap.cu (Lyapunov), one translation unit each.
#pragma once

#include "mixed.cuh"

namespace ss {
namespace mx {

template <int B>
constexpr size_t mixed_smem_bytes()
{
    // Five float tiles for the solve; the residual reuses the same memory as
    // two 8-byte tiles (float2 or double); plus a reduction buffer.
    return (size_t)5 * FTile<B>::SZ * sizeof(float) + 64 * sizeof(float);
}

// Low-precision solve of L D + D U = RHS into W (FP32, ld n), in place when
// the right-hand side is W itself (SRC_D = false) or from the FP64 C.  All in
// the instance's scaled units (sc): W and Rinv already are, L, U and C are
// shifted as they are staged.
template <int B, int T, bool LYAP, int P, bool SRC_D>
__device__ void low_solve(int n, const double *L, long ldl, const double *U, long ldu,
                          const double *Cd, long ldc, float *W, const float *Rinv, float *sm, const DfScale &sc)
{
    constexpr int LD = FTile<B>::LD, SZ = FTile<B>::SZ, E = B * B / T;
    float *sA = sm, *sB = sm + SZ, *sT = sm + 2 * SZ, *sL = sm + 3 * SZ, *sU = sm + 4 * SZ;
    const int nb = (n + B - 1) / B;
    const long ldw = n;
    Slots<B, T> sl;
    for (int I = 0; I < nb; ++I) {
        const int mI = min(B, n - I * B), i0 = I * B;
        __syncthreads();
        stage_f<B, T, F_LOWER>(sL, L + i0 + (long)i0 * ldl, ldl, mI, mI, sc.op);
        const int jend = LYAP ? I + 1 : nb;
        for (int J = 0; J < jend; ++J) {
            const int nJ = min(B, n - J * B), j0 = J * B;
            __syncthreads();
            if (SRC_D) {
                if (LYAP && I == J) stage_f<B, T, F_SYM_LOWER>(sT, Cd + i0 + (long)j0 * ldc, ldc, mI, nJ, sc.rhs);
                else stage_f<B, T, F_FULL>(sT, Cd + i0 + (long)j0 * ldc, ldc, mI, nJ, sc.rhs);
            } else {
                stage_f<B, T, F_FULL>(sT, W + i0 + (long)j0 * ldw, ldw, mI, nJ, 0);
            }
            __syncthreads();
            using MT = Micro<B, T>;
            const bool micro = MT::OK && (P == P_FP32) && mI == B && nJ == B;
            float acc[E];
            float macc[MT::MR][MT::MC];
            float frag[FragN<B, T, P>::value][4];
            if constexpr (P == P_FP32) {
                if (micro) {
#pragma unroll
                    for (int i = 0; i < MT::MR; ++i)
#pragma unroll
                        for (int j = 0; j < MT::MC; ++j) macc[i][j] = sT[(MT::r0() + i) + (MT::c0() + j) * LD];
                } else {
                    sl.set(Shape::Full, mI, nJ);
#pragma unroll
                    for (int r = 0; r < E; ++r) acc[r] = sl.ok(r) ? sT[sl.row[r] + sl.col[r] * LD] : 0.0f;
                }
            } else {
                frag_load<B, T>(frag, sT);
            }
            auto update = [&](bool tb) {
                if constexpr (P == P_FP32) {
                    if (micro) micro_update_f<B, T>(macc, sA, sB, B);
                    else if (tb) slot_update_f<B, T, false, true>(acc, sl, sA, sB, B);
                    else slot_update_f<B, T, false, false>(acc, sl, sA, sB, B);
                } else {
                    if (tb) mma_update<B, T, P, false, true>(frag, sA, sB, B);
                    else mma_update<B, T, P, false, false>(frag, sA, sB, B);
                }
            };
            // Stage A (not transposed) and B (transposed when tb) for either
            // layout, FP64 sources shifted by sha / shb.
            auto stageAB = [&](const auto *GA, long lda_, int ra, int sha, const auto *GB, long ldb_, int rb, int cb,
                               int shb, bool tb) {
                if (micro) {
                    stage_opA<B, T, false>(sA, GA, lda_, ra, B, sha);
                    if (tb) stage_opB<B, T, true>(sB, GB, ldb_, B, rb, shb);
                    else stage_opB<B, T, false>(sB, GB, ldb_, B, cb, shb);
                } else {
                    stage_f<B, T, F_FULL>(sA, GA, lda_, ra, B, sha);
                    stage_f<B, T, F_FULL>(sB, GB, ldb_, rb, cb, shb);
                }
            };
            // sum_{K<I} L_IK D_KJ
            for (int K = 0; K < I; ++K) {
                const int k0 = K * B;
                __syncthreads();
                const bool tr = LYAP && K < J;
                if (!tr) stageAB(L + i0 + (long)k0 * ldl, ldl, mI, sc.op, W + k0 + (long)j0 * ldw, ldw, B, nJ, 0, false);
                else stageAB(L + i0 + (long)k0 * ldl, ldl, mI, sc.op, W + j0 + (long)k0 * ldw, ldw, nJ, B, 0, true);
                __syncthreads();
                update(tr);
            }
            // sum_{K<J} D_IK U_KJ   (Lyapunov: U_KJ = L_JK^T)
            for (int K = 0; K < J; ++K) {
                const int k0 = K * B;
                __syncthreads();
                if (!LYAP) stageAB(W + i0 + (long)k0 * ldw, ldw, mI, 0, U + k0 + (long)j0 * ldu, ldu, B, nJ, sc.op, false);
                else stageAB(W + i0 + (long)k0 * ldw, ldw, mI, 0, L + j0 + (long)k0 * ldl, ldl, nJ, B, sc.op, true);
                __syncthreads();
                update(LYAP);
            }
            __syncthreads();
            if constexpr (P == P_FP32) {
                if (micro) {
#pragma unroll
                    for (int i = 0; i < MT::MR; ++i)
#pragma unroll
                        for (int j = 0; j < MT::MC; ++j) sT[(MT::r0() + i) + (MT::c0() + j) * LD] = macc[i][j];
                } else {
#pragma unroll
                    for (int r = 0; r < E; ++r)
                        if (sl.ok(r)) sT[sl.row[r] + sl.col[r] * LD] = acc[r];
                }
            } else {
                frag_store<B, T>(frag, sT);
            }
            if (!LYAP) stage_f<B, T, F_UPPER>(sU, U + j0 + (long)j0 * ldu, ldu, nJ, nJ, sc.op);
            else stage_f<B, T, F_LOWER>(sU, L + j0 + (long)j0 * ldl, ldl, nJ, nJ, sc.op);
            __syncthreads();
            syl_diag_f<B, T, LYAP>(sL, sU, sT, mI, nJ, Rinv + i0 + (long)j0 * ldw, ldw, sA);
            for (int e = threadIdx.x; e < mI * nJ; e += T) {
                const int r = e % mI, c = e / mI;
                W[(i0 + r) + (long)(j0 + c) * ldw] = sT[r + c * LD];
            }
        }
    }
    __syncthreads();
}

// R = C - L X - X U (Lyapunov: U = L^T, lower blocks, X read through its
// lower triangle) into W with FP64-class accuracy: double-float on the FP32
// pipe (RS = R_DF) or FP64 FMA (RS = R_FP64); in the scaled units of sc.
template <int B, int T, bool LYAP, int RS>
__device__ void residual(int n, const double *L, long ldl, const double *U, long ldu,
                         const double *C, long ldc, const double *X, long ldx, float *W, long ldw,
                         float *sm, const DfScale &sc)
{
    constexpr int E = B * B / T;
    using Elem = typename std::conditional<RS == R_DF, float2, double>::type;
    Elem *sA = reinterpret_cast<Elem *>(sm);
    Elem *sB = sA + FTile<B>::SZ;
    const int nb = (n + B - 1) / B;
    Slots<B, T> sl;

    auto stage = [&](Elem *S, const double *G, long ld, int rows, int cols, Fill f, int sh) {
        if constexpr (RS == R_DF) {
            float2 *S2 = reinterpret_cast<float2 *>(S);
            switch (f) {
            case F_FULL: stage_df<B, T, F_FULL>(S2, G, ld, rows, cols, sh); break;
            case F_LOWER: stage_df<B, T, F_LOWER>(S2, G, ld, rows, cols, sh); break;
            case F_UPPER: stage_df<B, T, F_UPPER>(S2, G, ld, rows, cols, sh); break;
            default: stage_df<B, T, F_SYM_LOWER>(S2, G, ld, rows, cols, sh); break;
            }
        } else {
            double *Sd = reinterpret_cast<double *>(S);
            switch (f) {
            case F_FULL: stage_d<B, T, F_FULL>(Sd, G, ld, rows, cols, sh); break;
            case F_LOWER: stage_d<B, T, F_LOWER>(Sd, G, ld, rows, cols, sh); break;
            case F_UPPER: stage_d<B, T, F_UPPER>(Sd, G, ld, rows, cols, sh); break;
            default: stage_d<B, T, F_SYM_LOWER>(Sd, G, ld, rows, cols, sh); break;
            }
        }
    };

    for (int I = 0; I < nb; ++I) {
        const int mI = min(B, n - I * B), i0 = I * B;
        const int jend = LYAP ? I + 1 : nb;
        for (int J = 0; J < jend; ++J) {
            const int nJ = min(B, n - J * B), j0 = J * B;
            using MT = Micro<B, T>;
            const bool micro = MT::OK && RS == R_DF && mI == B && nJ == B;
            float mh[MT::MR][MT::MC], ml[MT::MR][MT::MC];
            float ah[E], al[E];
            double ad[E];
            if (micro) {
#pragma unroll
                for (int i = 0; i < MT::MR; ++i)
#pragma unroll
                    for (int j = 0; j < MT::MC; ++j) {
                        int rr = MT::r0() + i, cc = MT::c0() + j;
                        if (LYAP && I == J && rr < cc) { const int t = rr; rr = cc; cc = t; }
                        split_df_s(C[(i0 + rr) + (long)(j0 + cc) * ldc], sc.rhs, mh[i][j], ml[i][j]);
                    }
            } else {
                sl.set(Shape::Full, mI, nJ);
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    ah[r] = 0.f; al[r] = 0.f; ad[r] = 0.0;
                    if (sl.ok(r)) {
                        int rr = sl.row[r], cc = sl.col[r];
                        if (LYAP && I == J && rr < cc) { const int t = rr; rr = cc; cc = t; }
                        const double c = C[(i0 + rr) + (long)(j0 + cc) * ldc];
                        if (RS == R_DF) split_df_s(c, sc.rhs, ah[r], al[r]);
                        else ad[r] = Pow2(sc.rhs)(c);
                    }
                }
            }
            auto upd = [&](bool tb, int kw) {
                if constexpr (RS == R_DF) {
                    const float2 *a = reinterpret_cast<const float2 *>(sA);
                    const float2 *b = reinterpret_cast<const float2 *>(sB);
                    if (micro) micro_update_df<B, T>(mh, ml, a, b, kw);
                    else if (tb) slot_update_df<B, T, false, true>(ah, al, sl, a, b, kw);
                    else slot_update_df<B, T, false, false>(ah, al, sl, a, b, kw);
                } else {
                    const double *a = reinterpret_cast<const double *>(sA);
                    const double *b = reinterpret_cast<const double *>(sB);
                    if (tb) slot_update<B, T, false, true>(ad, sl, a, b, kw);
                    else slot_update<B, T, false, false>(ad, sl, a, b, kw);
                }
            };
            // Micro-tile staging (double-float, k-major) of one A / B operand;
            // triangles (F_LOWER/F_UPPER) and the symmetric mirror are applied
            // by staging through the natural layout first when needed.
            auto stageM = [&](bool isA, const double *G, long ld, int rows, int cols, Fill f, bool tb, int sh) {
                float2 *S = reinterpret_cast<float2 *>(isA ? sA : sB);
                constexpr int LDA = MT::LDA, LDB = MT::LDB;
                for (int e = threadIdx.x; e < B * B; e += T) {
                    const int x = e % B, y = e / B;            // (x, y) of the source block
                    float2 v = make_float2(0.f, 0.f);
                    bool keep = x < rows && y < cols;
                    if (keep) {
                        if (f == F_LOWER) keep = x >= y;
                        else if (f == F_UPPER) keep = x <= y;
                    }
                    if (keep) {
                        const long idx = (f == F_SYM_LOWER && x < y) ? (y + (long)x * ld) : (x + (long)y * ld);
                        split_df_s(G[idx], sh, v.x, v.y);
                    }
                    if (isA) S[x + y * LDA] = v;                 // op(A)(r=x, k=y)
                    else if (!tb) S[y + x * LDB] = v;            // op(B)(k=x, c=y)
                    else S[x + y * LDB] = v;                     // op(B)(k=y, c=x) = G(x, y)
                }
            };
            auto stage2 = [&](const double *GA, long lda_, int ra, int ca, Fill fa, int sha,
                              const double *GB, long ldb_, int rb, int cb, Fill fb, int shb, bool tb) {
                if (micro) {
                    stageM(true, GA, lda_, ra, ca, fa, false, sha);
                    stageM(false, GB, ldb_, rb, cb, fb, tb, shb);
                } else {
                    stage(sA, GA, lda_, ra, ca, fa, sha);
                    stage(sB, GB, ldb_, rb, cb, fb, shb);
                }
            };
            // sum_{K<=I} L_IK X_KJ
            for (int K = 0; K <= I; ++K) {
                const int k0 = K * B, kw = min(B, n - k0);
                __syncthreads();
                const Fill fa = K == I ? F_LOWER : F_FULL;
                bool tb = false;
                if (!LYAP || K > J)
                    stage2(L + i0 + (long)k0 * ldl, ldl, mI, kw, fa, sc.op, X + k0 + (long)j0 * ldx, ldx, kw, nJ, F_FULL, sc.x,
                           false);
                else if (K == J)
                    stage2(L + i0 + (long)k0 * ldl, ldl, mI, kw, fa, sc.op, X + j0 + (long)j0 * ldx, ldx, kw, nJ,
                           F_SYM_LOWER, sc.x, false);
                else {
                    stage2(L + i0 + (long)k0 * ldl, ldl, mI, kw, fa, sc.op, X + j0 + (long)k0 * ldx, ldx, nJ, kw, F_FULL, sc.x,
                           true);
                    tb = true;
                }
                __syncthreads();
                upd(tb, kw);
            }
            // sum_{K<=J} X_IK U_KJ   (Lyapunov: L_JK^T)
            for (int K = 0; K <= J; ++K) {
                const int k0 = K * B, kw = min(B, n - k0);
                __syncthreads();
                const Fill fa = (LYAP && K == I) ? F_SYM_LOWER : F_FULL;
                const long aoff = (LYAP && K == I) ? (i0 + (long)i0 * ldx) : (i0 + (long)k0 * ldx);
                if (!LYAP)
                    stage2(X + aoff, ldx, mI, kw, fa, sc.x, U + k0 + (long)j0 * ldu, ldu, kw, nJ, K == J ? F_UPPER : F_FULL,
                           sc.op, false);
                else
                    stage2(X + aoff, ldx, mI, kw, fa, sc.x, L + j0 + (long)k0 * ldl, ldl, nJ, kw, K == J ? F_LOWER : F_FULL,
                           sc.op, true);
                __syncthreads();
                upd(LYAP, kw);
            }
            if (micro) {
#pragma unroll
                for (int i = 0; i < MT::MR; ++i)
#pragma unroll
                    for (int j = 0; j < MT::MC; ++j)
                        W[(i0 + MT::r0() + i) + (long)(j0 + MT::c0() + j) * ldw] = __fadd_rn(mh[i][j], ml[i][j]);
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (sl.ok(r)) {
                        const float v = RS == R_DF ? __fadd_rn(ah[r], al[r]) : (float)ad[r];
                        W[(i0 + sl.row[r]) + (long)(j0 + sl.col[r]) * ldw] = v;
                    }
                }
            }
        }
    }
    __syncthreads();
}

// X (FP64, the meaningful triangle, caller's units) = X + D * 2^-shx (first:
// X = D * 2^-shx), D in scaled units; returns |D|_F^2.
template <int T, bool LYAP>
__device__ float update_x(int n, double *X, long ldx, const float *W, long ldw, bool first,
                          float *s_red, int shx)
{
    float ss = 0.0f;
#pragma unroll 4
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int r = e % n, c = e / n;
        if (LYAP && r < c) continue;
        const float d = W[r + (long)c * ldw];
        ss = fmaf(d, d, ss);
        double *p = X + r + (long)c * ldx;
        *p = first ? f2d_exact_s(d, -shx) : *p + f2d_exact_s(d, -shx);
    }
    return block_sum_f(ss, s_red);
}

// r_ij = 1 / (l_ii + u_jj) computed in FP64, stored (rounded) as FP32 into
// Rinv (ld n) in the units of L and U scaled by 2^sho; returns 1 if a divisor
// is tiny or NaN.
template <int T, bool LYAP>
__device__ int reciprocal_divisors(int n, const double *L, long ldl, const double *U, long ldu,
                                   float *Rinv, float *s_red, int sho)
{
    double md = 0.0;
    for (int i = threadIdx.x; i < n; i += T) {
        md = fmax(md, fabs(L[i + (long)i * ldl]));
        if (!LYAP) md = fmax(md, fabs(U[i + (long)i * ldu]));
    }
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
    double *s_md = reinterpret_cast<double *>(s_red);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_md[threadIdx.x >> 5] = md;
    __syncthreads();
    md = 0.0;
    for (int w = 0; w < T / 32; ++w) md = fmax(md, s_md[w]);
    const double delta = divisor_delta(n, md);
    int bad = 0;
#pragma unroll 4
    for (int e = threadIdx.x; e < n * n; e += T) {
        const int i = e % n, j = e / n;
        const double d = L[i + (long)i * ldl] + (LYAP ? L[j + (long)j * ldl] : U[j + (long)j * ldu]);
        if (!(fabs(d) > delta)) bad = 1;
        Rinv[e] = d2f_trunc_s(1.0 / d, -sho);
    }
    return __syncthreads_or(bad);
}

// The instance's power-of-two scaling (DfScale) from the largest entries of
// L, U and C (Lyapunov: the lower triangles of L and S); s_buf: 2 ints per
// warp.
template <int T, bool LYAP>
__device__ DfScale instance_scale(int n, const double *L, long ldl, const double *U, long ldu, const double *C,
                                  long ldc, float *s_buf)
{
    int eo, ec;
    scan_exp3(ScanOp{L, ldl, n, n, 1}, ScanOp{LYAP ? nullptr : U, ldu, n, n, 2}, ScanOp{C, ldc, n, n, LYAP ? 1 : 0},
              threadIdx.x >> 5, T / 32, threadIdx.x & 31, eo, ec);
    cta_max2(eo, ec, reinterpret_cast<int *>(s_buf));
    return DfScale::sylvester(eo, ec);
}

template <int B, int T, bool LYAP, int P, int RS>
__device__ void mixed_instance(int n, const double *L, long ldl, const double *U, long ldu,
                               const double *C, long ldc, double *X, long ldx, int *info,
                               float *W, float *Rinv, bool raw, float *sm)
{
    float *s_red = sm + 5 * FTile<B>::SZ;
    const DfScale sc = instance_scale<T, LYAP>(n, L, ldl, U, ldu, C, ldc, s_red);
    const int bad = reciprocal_divisors<T, LYAP>(n, L, ldl, U, ldu, Rinv, s_red, sc.op);
    low_solve<B, T, LYAP, P, true>(n, L, ldl, U, ldu, C, ldc, W, Rinv, sm, sc);
    const float nx2 = update_x<T, LYAP>(n, X, ldx, W, n, true, s_red, sc.x);
    int conv = nx2 == 0.0f;
    if (!raw) {
        const float tol = (float)SS_REFINE_TOL;
        const float nx = sqrtf(nx2);
        float prev = nx;
        for (int it = 0; it < MAXIT && !conv; ++it) {
            residual<B, T, LYAP, RS>(n, L, ldl, U, ldu, C, ldc, X, ldx, W, n, sm, sc);
            low_solve<B, T, LYAP, P, false>(n, L, ldl, U, ldu, C, ldc, W, Rinv, sm, sc);
            const float nd = sqrtf(update_x<T, LYAP>(n, X, ldx, W, n, false, s_red, sc.x));
            const float pred = prev > 0.0f ? nd * (nd / prev) : nd;
            conv = (nd <= tol * nx) || (pred <= tol * nx);
            prev = nd;
        }
    } else {
        conv = 1;
    }
    if (threadIdx.x == 0) *info = bad ? 1 : (conv ? 0 : n + 1);
}

template <int B, int T, bool LYAP, int P, int RS>
__global__ void __launch_bounds__(T, 1024 / T) mixed_syl_kernel(Operands o, Sched s, int group, int raw)
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
        if (off + 2ll * n * n > s.scratch_elems) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_NO_WORK;
            continue;
        }
        float *W = static_cast<float *>(s.scratch) + off;
        mixed_instance<B, T, LYAP, P, RS>(n, o.A[b], o.lda[b], LYAP ? nullptr : o.U[b],
                                          LYAP ? 0 : o.ldu[b], o.C[b], o.ldc[b], o.X[b], o.ldx[b],
                                          o.info + b, W, W + (long)n * n, raw != 0, smf);
    }
}

template <int B, int T, bool LYAP, int P, int RS>
cudaError_t launch_mixed_syl(const Operands &o, const Sched &s, const Launch &l, cudaStream_t st, int raw)
{
    auto kern = mixed_syl_kernel<B, T, LYAP, P, RS>;
    const size_t smem = mixed_smem_bytes<B>();
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

}  // namespace mx
}  // namespace ss
