// Second stage of the SPD solve A X = B: with the upper Cholesky factor R
// (R^T R = A, computed by the Cholesky kernels into R) solve
//   R^T Y = B   (forward, row blocks I ascending),
//   R X = Y     (backward, row blocks I descending),
// for the k right-hand sides, Y held in X.  The paper names the Cholesky
// factorisation as a building block of linear-system solves; this is that use.
//
// One CTA per instance (persistent queue over the same size-sorted order as
// the factor launch, on a queue head of its own).  Right-hand sides go in
// chunks of 32 columns (16 when every instance has k <= 16).  Per row block I
// the lazy update
//   T = B_I - sum_{K<I} R_KI^T Y_K      (forward)
//   T = Y_I - sum_{K>I} R_IK X_K        (backward)
// is a B x (chunk) block product by all threads from shared tiles; the diagonal
// block solve R_II^T Y_I = T (R_II X_I = T) is done by one warp, one lane per
// column, the column's B entries in registers: x_i = t_i / r_ii, then every
// later entry of the column subtracts its r * x_i at once, so the dependent
// chain is one multiply and one FMA per row.  In SS_MODE_DF the block
// products are double-float on the FP32 pipe; the diagonal solves stay FP64.
#include "df.cuh"
#include "ss_internal.h"
#include "ss_device.cuh"

namespace ss {
namespace {

constexpr int KC = 32;   // right-hand-side columns per chunk (one per lane)

struct PosvOps {
    const int *n, *k;
    const double *const *R;
    const int *ldr;
    const double *const *B;
    const int *ldb;
    double *const *X;
    const int *ldx;
    int *info;
    int max_k;
};

template <int BS>
struct PTile {
    static constexpr int LD = BS + 1;
};

// Stage rows x cols of the column-major G (ld) into S (ld LDS), zero elsewhere
// of the R x C tile.
template <int R, int C, int LDS, int T>
__device__ __forceinline__ void stage(double *S, const double *G, long ld, int rows, int cols)
{
#pragma unroll 4
    for (int e = threadIdx.x; e < R * C; e += T) {
        const int r = e % R, c = e / R;
        S[r + c * LDS] = (r < rows && c < cols) ? G[r + (long)c * ld] : 0.0;
    }
}

// The same staging as double-float pairs of G * 2^sh (a float2 slot has the
// size of a double, so the tile layout is unchanged).
template <int R, int C, int LDS, int T>
__device__ __forceinline__ void stage_df(float2 *S, const double *G, long ld, int rows, int cols, int sh)
{
#pragma unroll 4
    for (int e = threadIdx.x; e < R * C; e += T) {
        const int r = e % R, c = e / R;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows && c < cols) split_df_s(G[r + (long)c * ld], sh, v.x, v.y);
        S[r + c * LDS] = v;
    }
}

// CW: right-hand-side columns per chunk (16 or 32; the kernel picks 16 when
// k <= 16 so that no update multiplies padding columns).  DF (SS_MODE_DF):
// the block updates in double-float arithmetic on the FP32 pipe, T rounded
// to FP64 for the FP64 diagonal solve.  DF rescales the system by powers of
// two so that the largest entries of R and of B lie in [1, 2): R by 2^r and B
// by 2^q make Y = R^-T B carry 2^(q-r) and X = R^-1 Y carry 2^(q-2r), exactly.
// The double-float operands take their shift in the split, the FP64 diagonal
// solves work on the scaled values, and X (holding Y between the passes) is
// stored in the caller's units.
template <int BS, int T, int CW, bool DF>
__device__ void posv_instance(int n, int k, const double *R, long ldr, const double *Bm, long ldb, double *X,
                              long ldx, double *sm)
{
    constexpr int LDR = PTile<BS>::LD, LDK = BS + 1;
    constexpr int E = BS * CW / T;          // outputs per thread of a BS x CW block
    static_assert((BS * CW) % T == 0 && CW <= KC, "threads must divide the block");
    double *sR = sm;                          // BS x BS (ld LDR): R_KI or R_IK of a step
    double *sY = sR + BS * LDR;               // BS x KC (ld LDK): Y_K or X_K of a step
    double *sD = sY + KC * LDK;               // BS x BS: R_II
    double *sT = sD + BS * LDR;               // BS x KC: T handed to the diagonal warp
    double *sInv = sT + KC * LDK;             // BS reciprocals 1 / r_ii
    const int nb = (n + BS - 1) / BS;
    int shR = 0, shY = 0, shX = 0;            // DF: shifts of R, Y and X
    if constexpr (DF) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int er, eb;
        scan_exp3(ScanOp{R, ldr, n, n, 2}, ScanOp{nullptr, 0, 0, 0, 0}, ScanOp{Bm, ldb, n, k, 0}, w, T / 32, lane, er, eb);
        cta_max2(er, eb, reinterpret_cast<int *>(sInv + BS));
        shR = er ? 1023 - er : 0;
        const int shB = eb ? 1023 - eb : shR;
        shY = shB - shR;
        shX = shB - 2 * shR;
    }
    for (int c0 = 0; c0 < k; c0 += CW) {
        const int kc = min(CW, k - c0);
        for (int pass = 0; pass < 2; ++pass) {
            const bool fwd = pass == 0;
            for (int q = 0; q < nb; ++q) {
                const int I = fwd ? q : nb - 1 - q;
                const int i0 = I * BS, mI = min(BS, n - i0);
                double acc[E];
                float ah[E], al[E];
                const double *src = fwd ? Bm : X;
                const long lds = fwd ? ldb : ldx;
                const int shs = fwd ? shY + shR : shY;            // B: 2^q, Y: 2^(q-r)
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int e = threadIdx.x + T * r, row = e % BS, col = e / BS;
                    acc[r] = (row < mI && col < kc) ? src[(i0 + row) + (long)(c0 + col) * lds] : 0.0;
                    if constexpr (DF) split_df_s(acc[r], shs, ah[r], al[r]);
                }
                const int K0 = fwd ? 0 : I + 1, K1 = fwd ? I : nb;
                for (int K = K0; K < K1; ++K) {
                    const int k0 = K * BS, mK = min(BS, n - k0);
                    __syncthreads();
                    if constexpr (DF) {
                        float2 *dR = reinterpret_cast<float2 *>(sR), *dY = reinterpret_cast<float2 *>(sY);
                        if (fwd) stage_df<BS, BS, LDR, T>(dR, R + k0 + (long)i0 * ldr, ldr, mK, mI, shR);
                        else     stage_df<BS, BS, LDR, T>(dR, R + i0 + (long)k0 * ldr, ldr, mI, mK, shR);
                        stage_df<BS, CW, LDK, T>(dY, X + k0 + (long)c0 * ldx, ldx, mK, kc, fwd ? shY : shX);
                    } else {
                        if (fwd) stage<BS, BS, LDR, T>(sR, R + k0 + (long)i0 * ldr, ldr, mK, mI);   // R_KI
                        else     stage<BS, BS, LDR, T>(sR, R + i0 + (long)k0 * ldr, ldr, mI, mK);   // R_IK
                        stage<BS, CW, LDK, T>(sY, X + k0 + (long)c0 * ldx, ldx, mK, kc);           // Y_K / X_K
                    }
                    __syncthreads();
#pragma unroll
                    for (int r = 0; r < E; ++r) {
                        const int e = threadIdx.x + T * r, row = e % BS, col = e / BS;
                        if (col >= kc) continue;    // whole half-warps of padding columns skip
                        if constexpr (DF) {
                            const float2 *dR = reinterpret_cast<const float2 *>(sR);
                            const float2 *dY = reinterpret_cast<const float2 *>(sY);
                            float h = ah[r], l = al[r];
#pragma unroll 4
                            for (int t = 0; t < mK; ++t) {
                                const float2 a = fwd ? dR[t + row * LDR] : dR[row + t * LDR];
                                const float2 y = dY[t + col * LDK];
                                df_msub(h, l, a.x, a.y, y.x, y.y);
                            }
                            ah[r] = h;
                            al[r] = l;
                        } else {
                            double s = acc[r];
#pragma unroll 4
                            for (int t = 0; t < mK; ++t) {
                                // forward: (R_KI^T)(row, t) = R_KI(t, row); backward: R_IK(row, t)
                                const double a = fwd ? sR[t + row * LDR] : sR[row + t * LDR];
                                s = fma(-a, sY[t + col * LDK], s);
                            }
                            acc[r] = s;
                        }
                    }
                }
                if constexpr (DF) {
#pragma unroll
                    for (int r = 0; r < E; ++r) acc[r] = df_to_double(ah[r], al[r]);
                }
                __syncthreads();
                stage<BS, BS, LDR, T>(sD, R + i0 + (long)i0 * ldr, ldr, mI, mI);
                if constexpr (DF) {
                    // Same thread-to-element map as stage(): each thread scales its own entries.
                    const Pow2 fr(shR);
                    for (int e = threadIdx.x; e < BS * BS; e += T) sD[e % BS + (e / BS) * LDR] = fr(sD[e % BS + (e / BS) * LDR]);
                }
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int e = threadIdx.x + T * r, row = e % BS, col = e / BS;
                    sT[row + col * LDK] = acc[r];
                }
                __syncthreads();
                if (threadIdx.x < BS) sInv[threadIdx.x] = threadIdx.x < mI ? 1.0 / sD[threadIdx.x * (LDR + 1)] : 0.0;
                __syncthreads();
                if (threadIdx.x < 32) {
                    const int j = threadIdx.x;          // column of the chunk
                    const Pow2 fo(DF ? (fwd ? -shY : -shX) : 0);   // back to the caller's units
                    double t[BS];
#pragma unroll
                    for (int i = 0; i < BS; ++i) t[i] = sT[i + j * LDK];
                    if (fwd) {
                        // R_II^T lower: row i of Y needs rows < i.
#pragma unroll
                        for (int i = 0; i < BS; ++i) {
                            if (i < mI) {
                                t[i] *= sInv[i];
#pragma unroll
                                for (int l = i + 1; l < BS; ++l) t[l] = fma(-sD[i + l * LDR], t[i], t[l]);
                            }
                        }
                    } else {
                        // R_II upper: row i of X needs rows > i.
#pragma unroll
                        for (int i = BS - 1; i >= 0; --i) {
                            if (i < mI) {
                                t[i] *= sInv[i];
#pragma unroll
                                for (int l = 0; l < i; ++l) t[l] = fma(-sD[l + i * LDR], t[i], t[l]);
                            }
                        }
                    }
                    if (j < kc)
#pragma unroll
                        for (int i = 0; i < BS; ++i)
                            if (i < mI) {
                                if constexpr (DF) X[(i0 + i) + (long)(c0 + j) * ldx] = fo(t[i]);
                                else X[(i0 + i) + (long)(c0 + j) * ldx] = t[i];
                            }
                }
                __syncthreads();
            }
        }
    }
}

// One persistent CTA per system, over the same size-sorted order as the
// factor launch.
template <int CW, bool DF>
__device__ __forceinline__ void posv_loop(const PosvOps &o, const Sched &s, int group)
{
    constexpr int BS = 16, T = 128;
    extern __shared__ double sm[];
    __shared__ int s_slot;
    claim_init(&s_slot);
    const int hi = s.meta[META_COUNT];
    for (;;) {
        const int w = claim_slot(s.meta + META_HEAD + group, &s_slot);
        if (w >= hi) break;
        const int b = s.perm[w];
        if (o.info[b] != 0) continue;           // factor failed or bad size: X untouched
        const int n = o.n[b], k = o.k[b];
        if (k < 0 || k > o.max_k) {
            if (threadIdx.x == 0) o.info[b] = SS_INFO_BAD_SIZE;
            continue;
        }
        if (n == 0 || k == 0) continue;
        posv_instance<BS, T, CW, DF>(n, k, o.R[b], o.ldr[b], o.B[b], o.ldb[b], o.X[b], o.ldx[b], sm);
    }
}

// FP64 and double-float forms; the double-float one is held to five CTAs per
// SM (seven for 16-column chunks), as without its scaling shifts.
template <int CW>
__global__ void __launch_bounds__(128) posv_kernel(PosvOps o, Sched s, int group)
{
    posv_loop<CW, false>(o, s, group);
}

template <int CW>
__global__ void __launch_bounds__(128, CW == 16 ? 7 : 5) posv_df_kernel(PosvOps o, Sched s, int group)
{
    posv_loop<CW, true>(o, s, group);
}

}  // namespace

// The solve stage on the queue head `group` over all valid instances.
cudaError_t launch_posv_solve(const int *d_n, const int *d_k, int max_k, const double *const *d_R, const int *d_ldr,
                              const double *const *d_B, const int *d_ldb, double *const *d_X, const int *d_ldx,
                              int *d_info, const Sched &s, int group, int batch, cudaStream_t st, bool df)
{
    constexpr int BS = 16, T = 128;
    const size_t smem = (size_t)(2 * BS * (BS + 1) + 2 * KC * (BS + 1) + BS + 4) * sizeof(double);
    auto kernel = max_k <= 16 ? (df ? posv_df_kernel<16> : posv_kernel<16>)
                              : (df ? posv_df_kernel<KC> : posv_kernel<KC>);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long grid = (long)per_sm * sm_count();
    if (grid > batch) grid = batch;
    if (grid < 1) grid = 1;
    PosvOps o{d_n, d_k, d_R, d_ldr, d_B, d_ldb, d_X, d_ldx, d_info, max_k};
    kernel<<<(int)grid, T, smem, st>>>(o, s, group);
    return cudaGetLastError();
}

}  // namespace ss
