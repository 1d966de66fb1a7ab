// Device building blocks shared by the solve kernels: the persistent work
// queue, shared-memory tile staging, the register-tiled block update, and
// split dot products.
//
// Tiles are B x B blocks of one instance, staged column-major in shared
// memory with leading dimension B + 1 (odd, so a transposed read walks the
// banks).  A CTA of T threads owns the B*B outputs of a block update with
// element e = tid + T * r  ->  (row, col) = (e % B, e / B): each thread keeps
// E = B*B/T accumulators for one row and E columns spaced T/B apart.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ss {

template <int B>
struct Tile {
    static constexpr int LD = B + 1;
    static constexpr int SZ = B * (B + 1);
};

// Claim the next slot of the persistent queue; every thread gets the value.
// A CTA's first slot is its block index; later slots come from the atomic
// counter, offset by the grid size, so every slot is handed out exactly once
// whether or not all CTAs are resident.  Why the first claim is static: the
// queue is in longest-first order, so the first gridDim.x slots hold the
// largest instances, and consecutive block indices are dispatched to
// different SMs, so each SM receives one instance from every stretch of
// (number of SMs) consecutive slots.  Claimed in arrival order at the atomic
// instead, some SMs reach it first repeatedly and start with several of the
// largest instances, and the FP64 pipes of the others idle at the end.
// *s_slot holds the previous slot, negative before the first claim
// (claim_init); the choice is made by thread 0 on that shared value, which
// keeps it out of the solver's registers.
__device__ __forceinline__ void claim_init(int *s_slot)
{
    if (threadIdx.x == 0) *s_slot = -1;
}

__device__ __forceinline__ int claim_slot(int *head, int *s_slot)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_slot = *s_slot < 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(head, 1);
    __syncthreads();
    return *s_slot;
}

// Stage a rows x cols sub-block of a column-major global matrix (leading
// dimension ldg) into tile S, zero-filling the rest of the B x B tile.
template <int B, int T, typename Src>
__device__ __forceinline__ void stage_tile(double *S, const Src *G, long ldg, int rows, int cols)
{
    constexpr int LD = Tile<B>::LD;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        double v = 0.0;
        if (r < rows && c < cols) v = (double)G[r + (long)c * ldg];
        S[r + c * LD] = v;
    }
}

// Same, but keep only the lower (lower=true) or upper triangle of the
// sub-block (diagonal included); the other strict triangle becomes zero.
template <int B, int T>
__device__ __forceinline__ void stage_tri(double *S, const double *G, long ldg, int m, bool lower)
{
    constexpr int LD = Tile<B>::LD;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        double v = 0.0;
        const bool keep = lower ? (r >= c) : (r <= c);
        if (r < m && c < m && keep) v = G[r + (long)c * ldg];
        S[r + c * LD] = v;
    }
}

// Stage the symmetric m x m diagonal block whose lower triangle is stored in
// G, mirroring it into the upper triangle of S; zero elsewhere.
template <int B, int T>
__device__ __forceinline__ void stage_sym_lower(double *S, const double *G, long ldg, int m)
{
    constexpr int LD = Tile<B>::LD;
#pragma unroll 4
    for (int e = threadIdx.x; e < B * B; e += T) {
        const int r = e % B, c = e / B;
        double v = 0.0;
        if (r < m && c < m) v = r >= c ? G[r + (long)c * ldg] : G[c + (long)r * ldg];
        S[r + c * LD] = v;
    }
}

// Register-tiled block update  acc -= op(A) * op(Bm)  over kk terms, with
// op(A)(row, k) = TA ? A[k + row*LD] : A[row + k*LD] and
// op(Bm)(k, col) = TB ? Bm[col + k*LD] : Bm[k + col*LD].
template <int B, int T, bool TA, bool TB>
__device__ __forceinline__ void block_update(double (&acc)[B * B / T], const double *A,
                                             const double *Bm, int kk)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int E = B * B / T;
    constexpr int CS = T / B;
    const int row = threadIdx.x % B;
    const int col0 = threadIdx.x / B;
#pragma unroll 2
    for (int k = 0; k < kk; ++k) {
        const double a = TA ? A[k + row * LD] : A[row + k * LD];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int col = col0 + CS * r;
            const double b = TB ? Bm[col + k * LD] : Bm[k + col * LD];
            acc[r] = fma(-a, b, acc[r]);
        }
    }
}

// Sum over aligned groups of `split` lanes (a power of two <= 32).  Every lane
// of the warp must call it.
__device__ __forceinline__ double group_sum(double v, int split)
{
    for (int o = split >> 1; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int pow2_floor(int x)
{
    return x <= 1 ? 1 : (1 << (31 - __clz(x)));
}

// Smallest k with 2^k >= x (x >= 1).
__device__ __forceinline__ int ceil_log2(int x)
{
    return x <= 1 ? 0 : 32 - __clz(x - 1);
}

// Lanes per dot product when `cnt` dot products of length about `len` share T
// threads: a power of two, at most 32, at most T/cnt, and small enough that
// each lane still does about four terms.
template <int T>
__device__ __forceinline__ int pick_split(int cnt, int len)
{
    int s = pow2_floor(T / (cnt > 0 ? cnt : 1));
    int byLen = pow2_floor(len / 4 > 0 ? len / 4 : 1);
    s = s < byLen ? s : byLen;
    return s > 32 ? 32 : s;
}

// One operand of an exponent scan: the entries (i, j), 0 <= i < rows,
// 0 <= j < cols, of the column-major p that `tri` keeps (0: all, 1: i >= j,
// 2: i <= j); p == nullptr: none.
struct ScanOp {
    const double *p;
    long ld;
    int rows, cols, tri;
};

__device__ __forceinline__ int scan_e(double v)
{
    const int e = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
    return e == 0x7FF ? 0 : e;
}

// Largest biased FP64 exponents over the operands a and b (-> e0) and c
// (-> e1); Inf and NaN are left out, zero counts as exponent 0.  This
// thread's part only (reduce with cta_max2): warp w of nw takes columns
// w, w + nw, ..., two at a time, its lanes four rows each of all three
// operands, so that one round trip to memory brings up to 24 loads per lane
// (a scan is latency-bound: one instance's data, once).
__device__ __forceinline__ void scan_exp3(const ScanOp &a, const ScanOp &b, const ScanOp &c, int w, int nw,
                                          int lane, int &e0, int &e1)
{
    const int cols = max(max(a.p ? a.cols : 0, b.p ? b.cols : 0), c.p ? c.cols : 0);
    const int rows = max(max(a.p ? a.rows : 0, b.p ? b.rows : 0), c.p ? c.rows : 0);
    auto keep = [](const ScanOp &o, int i, int j) {
        return o.p != nullptr && i < o.rows && j < o.cols && (o.tri == 0 || (o.tri == 1 ? i >= j : i <= j));
    };
    int m0 = 0, m1 = 0;
#pragma unroll 2
    for (int j = w; j < cols; j += nw) {
        for (int r0 = 0; r0 < rows; r0 += 128) {
            double va[4], vb[4], vc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = r0 + lane + 32 * q;
                va[q] = keep(a, i, j) ? __ldg(a.p + i + (long)j * a.ld) : 0.0;
                vb[q] = keep(b, i, j) ? __ldg(b.p + i + (long)j * b.ld) : 0.0;
                vc[q] = keep(c, i, j) ? __ldg(c.p + i + (long)j * c.ld) : 0.0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                m0 = max(m0, max(scan_e(va[q]), scan_e(vb[q])));
                m1 = max(m1, scan_e(vc[q]));
            }
        }
    }
    e0 = m0;
    e1 = m1;
}

// CTA-wide maxima of two ints (every thread of the CTA calls it and gets
// both); s_buf holds 2 ints per warp.
__device__ __forceinline__ void cta_max2(int &x, int &y, int *s_buf)
{
    const unsigned ux = __reduce_max_sync(0xffffffffu, (unsigned)x);
    const unsigned uy = __reduce_max_sync(0xffffffffu, (unsigned)y);
    const int w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        s_buf[2 * w] = (int)ux;
        s_buf[2 * w + 1] = (int)uy;
    }
    __syncthreads();
    x = 0;
    y = 0;
    for (int k = 0; k < nw; ++k) {
        x = max(x, s_buf[2 * k]);
        y = max(y, s_buf[2 * k + 1]);
    }
    __syncthreads();
}

// Power-of-two rescaling of one instance for the double-float pipelines.
// The equations are homogeneous: for Sylvester / Lyapunov, L X + X U = C
// holds with (2^a L, 2^a U, 2^(a+b) C, 2^b X), and for Cholesky X^T X = A
// with (2^(2s) A, 2^s X), all exactly in binary floating point.  An operand
// whose largest entry lies in the deadband [2^-W, 2^(W+1)) keeps shift 0 (so
// that typical data needs no rescaling at all); one outside it is moved to
// [1, 2).  Built from the largest biased FP64 exponents eo (operator: L and
// U, or A) and ec (right-hand side); an all-zero operand gets shift 0.
//
// Why the bands keep FP64 accuracy: a double-float value loses at most 2^-126
// absolutely (a hi or lo part below FP32's normal range is flushed), so one
// product term errs by at most 2^-126 times its other factor.  Sylvester /
// Lyapunov, W = 12: L, U and C stay below 2^13 and X below 2^60 (checked by
// the solve), so products stay below 2^73 and a dot product of up to 4096
// terms errs by at most 2^-54 absolutely, 2^-42 relative to a right-hand side
// whose largest entry is at least 2^-12.  Cholesky, W = 40: the largest entry
// of an SPD matrix is on its diagonal and |x_ij| <= sqrt(a_jj) < 2^21, so a
// dot product of up to 4096 terms errs by at most 2^-93 absolutely, 2^-53
// relative to a matrix whose largest entry is at least 2^-40.
struct DfScale {
    int op;    // shift of L and U (Cholesky: of A)
    int rhs;   // shift of C
    int x;     // shift of X: rhs - op (Cholesky: op / 2)
    static constexpr int BAND_SYL = 12, BAND_CHOL = 40;
    __device__ __forceinline__ static int to_one(int e, int band)
    {
        const int d = e ? 1023 - e : 0;
        return (d >= -band && d <= band) ? 0 : d;
    }
    __device__ __forceinline__ static DfScale sylvester(int eo, int ec)
    {
        DfScale s;
        s.op = to_one(eo, BAND_SYL);
        s.rhs = ec ? to_one(ec, BAND_SYL) : s.op;
        s.x = s.rhs - s.op;
        return s;
    }
    __device__ __forceinline__ static DfScale cholesky(int ea)
    {
        DfScale s;
        const int d = to_one(ea, BAND_CHOL);
        s.x = d >= 0 ? d / 2 : -((1 - d) / 2);   // floor(d / 2)
        s.op = 2 * s.x;
        s.rhs = s.op;
        return s;
    }
    __device__ __forceinline__ bool zero() const { return (op | rhs | x) == 0; }
};

// Band check of one input value for the unscaled double-float pipelines:
// bit 0 if |v| >= 2^(W+1) (or v is Inf / NaN), bit `cls` if |v| >= 2^-W.  An
// instance whose operator and right-hand side each have their largest entry
// in [2^-W, 2^(W+1)) has all DfScale shifts zero: OR-ing these bits over every
// input value decides that exactly.
template <int W>
__device__ __forceinline__ unsigned band_bits(double v, unsigned cls)
{
    const int e = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
    return (e > 1023 + W ? 1u : 0u) | (e >= 1023 - W ? cls : 0u);
}
constexpr unsigned BAND_BIG = 1u, BAND_OP = 2u, BAND_RHS = 4u;

// 2^k as a double, -1022 <= k <= 1023.
__device__ __forceinline__ double pow2d(int k)
{
    return __longlong_as_double((long long)((unsigned long long)(1023 + k) << 52));
}

// Multiplication by 2^k, |k| <= 2044, as two exact factors 2^(k/2) and
// 2^(k - k/2) (each within FP64's normal range): v * 2^k exactly unless the
// result itself leaves FP64's normal range.
struct Pow2 {
    double f1, f2;
    __device__ __forceinline__ explicit Pow2(int k) : f1(pow2d(k / 2)), f2(pow2d(k - k / 2)) {}
    __device__ __forceinline__ double operator()(double v) const { return v * f1 * f2; }
};

// Threshold below which a Sylvester/Lyapunov divisor counts as singular:
// n * DBL_EPSILON * (largest diagonal magnitude).
__device__ __forceinline__ double divisor_delta(int n, double maxdiag)
{
    return (double)n * 2.220446049250313e-16 * maxdiag;
}

}  // namespace ss

namespace ss {

// Which outputs of a block a thread owns.  Slot r of thread tid is flat index
// e = tid + T*r over the block's valid elements, so lanes only ever hold real
// outputs and padded rows or columns cost no arithmetic.
enum class Shape { Full, Upper, Lower };

template <int B, int T>
struct Slots {
    static constexpr int E = B * B / T;
    int row[E];
    int col[E];
    unsigned valid;

    // Column index c with c(c+1)/2 <= e < (c+1)(c+2)/2.
    __device__ __forceinline__ static int tri_decode(int e)
    {
        int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (c * (c + 1) / 2 > e) --c;
        while ((c + 1) * (c + 2) / 2 <= e) ++c;
        return c;
    }

    __device__ __forceinline__ void set(Shape s, int m, int nn)
    {
        valid = 0u;
        const int cnt = s == Shape::Full ? m * nn : nn * (nn + 1) / 2;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = threadIdx.x + T * r;
            int rr = 0, cc = 0;
            if (e < cnt) {
                if (s == Shape::Full) {
                    rr = e % m;
                    cc = e / m;
                } else {
                    const int t = tri_decode(e);
                    const int u = e - t * (t + 1) / 2;   // 0 <= u <= t
                    if (s == Shape::Upper) { rr = u; cc = t; }
                    else                   { rr = t; cc = u; }
                }
                valid |= 1u << r;
            }
            row[r] = rr;
            col[r] = cc;
        }
    }
    __device__ __forceinline__ bool ok(int r) const { return (valid >> r) & 1u; }
};

// acc[r] -= sum_k op(A)(row[r], k) * op(Bm)(k, col[r]) over kk terms, with
// op(A)(i, k) = TA ? A[k + i*LD] : A[i + k*LD] and
// op(Bm)(k, j) = TB ? Bm[j + k*LD] : Bm[k + j*LD].
template <int B, int T, bool TA, bool TB>
__device__ __forceinline__ void slot_update(double (&acc)[B * B / T], const Slots<B, T> &s,
                                            const double *A, const double *Bm, int kk)
{
    constexpr int LD = Tile<B>::LD;
    constexpr int E = B * B / T;
#pragma unroll 2
    for (int k = 0; k < kk; ++k) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if (s.ok(r)) {
                const double a = TA ? A[k + s.row[r] * LD] : A[s.row[r] + k * LD];
                const double b = TB ? Bm[s.col[r] + k * LD] : Bm[k + s.col[r] * LD];
                acc[r] = fma(-a, b, acc[r]);
            }
        }
    }
}

// True if any lane of this warp handles one of the first `cnt` work items
// when items are spread `split` lanes apiece (warp-uniform).
__device__ __forceinline__ bool warp_has_work(int cnt, int split)
{
    const int first = (threadIdx.x & ~31) / split;
    return first < cnt;
}

}  // namespace ss
