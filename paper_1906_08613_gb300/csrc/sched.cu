// Binning pre-pass of the persistent batched scheduler.
//
// One CTA of 1024 threads sorts the instance indices by order n, largest
// first (a counting sort over n = 0..max_n), so that the persistent solve
// kernels start the longest instances first and finish with the short ones
// (longest-processing-time-first list scheduling).  It also records where
// each size bin bin(n) = ceil(log2 n) starts in the sorted order, the range
// of every launch group, and the offset of each instance's scratch area, and
// resets the work-queue heads.  Instances whose device-side order is negative
// or above max_n get info = SS_INFO_BAD_SIZE and are left out.  For the
// rectangular Sylvester solve the order used is max(m, n).
#include "ss_device.cuh"
#include "ss_internal.h"

namespace ss {
namespace {

constexpr int BIN_THREADS = 1024;

struct GroupMap {
    int group_of_bin[NUM_BINS];
    int ngroups;
};


// Sort key of instance b: its order n; with d_m, max(m, n), or -1 when m or
// n is out of range.
__device__ __forceinline__ int size_key(const int *d_n, const int *d_m, int max_n, int max_m, int b)
{
    const int n = d_n[b];
    if (d_m == nullptr) return n;
    const int m = d_m[b];
    if (m < 0 || m > max_m || n < 0 || n > max_n) return -1;
    return m > n ? m : n;
}

__global__ void __launch_bounds__(BIN_THREADS)
bin_kernel(int batch, int max_key, const int *d_n, const int *d_m, int max_n_in, int max_m, int *d_info,
           int *meta, int *perm, long long *scr, long long scr_per_n2, GroupMap gm, DfInst *dfs)
{
    const int max_n = max_key;
    extern __shared__ unsigned char raw[];
    const int M = max_n + 1;
    long long *sq = reinterpret_cast<long long *>(raw);          // [M]
    int *hist = reinterpret_cast<int *>(sq + M);                  // [M]
    int *pos = hist + M;                                          // [M]
    __shared__ int s_part[BIN_THREADS];
    __shared__ long long s_psq[BIN_THREADS];
    __shared__ int s_total;
    const int tid = threadIdx.x;

    for (int i = tid; i < M; i += BIN_THREADS) hist[i] = 0;
    __syncthreads();
    for (int b = tid; b < batch; b += BIN_THREADS) {
        const int n = size_key(d_n, d_m, max_n_in, max_m, b);
        if (n < 0 || n > max_n) d_info[b] = SS_INFO_BAD_SIZE;
        else atomicAdd(&hist[n], 1);
        if (dfs) dfs[b] = DfInst{0, 0, 0, 0, 0ull};
    }
    __syncthreads();

    // Exclusive scan in descending n: pos[n] = #instances of order > n,
    // sq[n] = sum of m^2 over those instances.  Thread t owns the chunk of
    // q = max_n - n in [t*chunk, (t+1)*chunk).
    const int chunk = (M + BIN_THREADS - 1) / BIN_THREADS;
    int c_sum = 0;
    long long s_sum = 0;
    for (int q = tid * chunk; q < min(M, (tid + 1) * chunk); ++q) {
        const int n = max_n - q;
        c_sum += hist[n];
        s_sum += (long long)hist[n] * n * n;
    }
    s_part[tid] = c_sum;
    s_psq[tid] = s_sum;
    __syncthreads();
    if (tid < 32) {
        // Warp 0 scans the 1024 partial sums: 32 per lane, then across lanes.
        int c = 0;
        long long v = 0;
        for (int t = tid * 32; t < tid * 32 + 32; ++t) { c += s_part[t]; v += s_psq[t]; }
        int ci = c;
        long long vi = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ci, o);
            const long long z = __shfl_up_sync(0xffffffffu, vi, o);
            if (tid >= o) { ci += y; vi += z; }
        }
        int run = ci - c;
        long long rsq = vi - v;
        for (int t = tid * 32; t < tid * 32 + 32; ++t) {
            const int cc = s_part[t];
            const long long vv = s_psq[t];
            s_part[t] = run;
            s_psq[t] = rsq;
            run += cc;
            rsq += vv;
        }
        if (tid == 31) s_total = ci;
    }
    __syncthreads();
    {
        int run = s_part[tid];
        long long rsq = s_psq[tid];
        for (int q = tid * chunk; q < min(M, (tid + 1) * chunk); ++q) {
            const int n = max_n - q;
            pos[n] = run;
            sq[n] = rsq;
            run += hist[n];
            rsq += (long long)hist[n] * n * n;
        }
    }
    __syncthreads();
    for (int i = tid; i < M; i += BIN_THREADS) hist[i] = pos[i];   // cursors
    __syncthreads();
    for (int b = tid; b < batch; b += BIN_THREADS) {
        const int n = size_key(d_n, d_m, max_n_in, max_m, b);
        if (n < 0 || n > max_n) continue;
        const int w = atomicAdd(&hist[n], 1);
        perm[w] = b;
        if (scr) scr[w] = (sq[n] + (long long)(w - pos[n]) * n * n) * scr_per_n2;
    }
    if (tid == 0) {
        const int count = s_total;
        meta[META_COUNT] = count;
        // pos of "order > x": x >= max_n -> 0; x < 0 -> count.
        auto posf = [&](int x) { return x >= max_n ? 0 : (x < 0 ? count : pos[x]); };
        int glo[MAX_GROUPS], ghi[MAX_GROUPS];
        for (int g = 0; g < MAX_GROUPS; ++g) { glo[g] = 0x7fffffff; ghi[g] = 0; }
        for (int k = 0; k < NUM_BINS; ++k) {
            const int a = k == 0 ? -1 : (1 << (k - 1));
            const int bmax = k == 0 ? 1 : (1 << k);
            int lo = 0, hi = 0;
            if (a < max_n) {
                lo = posf(bmax < max_n ? bmax : max_n);
                hi = posf(a);
            }
            meta[META_BIN_LO + k] = lo;
            meta[META_BIN_HI + k] = hi;
            const int g = gm.group_of_bin[k];
            if (g >= 0 && g < MAX_GROUPS && hi > lo) {
                glo[g] = min(glo[g], lo);
                ghi[g] = max(ghi[g], hi);
            }
        }
        for (int g = 0; g < MAX_GROUPS; ++g) {
            const bool used = ghi[g] > 0 && glo[g] < ghi[g];
            meta[META_RANGE + 2 * g] = used ? glo[g] : 0;
            meta[META_RANGE + 2 * g + 1] = used ? ghi[g] : 0;
            meta[META_HEAD + g] = 0;
            meta[META_RNG + g] = 0;
            meta[META_SCL + g] = 0;
            meta[META_SCL_HEAD + g] = 0;
        }
    }
}

}  // namespace

cudaError_t launch_binning(int batch, int max_n, const int *d_n, int *d_info, const Sched &s,
                           const int *group_of_bin, int ngroups, long long scratch_per_n2,
                           cudaStream_t st, const int *d_m, int max_m)
{
    const int max_key = d_m != nullptr && max_m > max_n ? max_m : max_n;
    GroupMap gm;
    for (int k = 0; k < NUM_BINS; ++k) gm.group_of_bin[k] = group_of_bin[k];
    gm.ngroups = ngroups;
    const size_t smem = (size_t)(max_key + 1) * (sizeof(long long) + 2 * sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    bin_kernel<<<1, BIN_THREADS, smem, st>>>(batch, max_key, d_n, d_m, max_n, max_m, d_info, s.meta,
                                             const_cast<int *>(s.perm),
                                             const_cast<long long *>(s.scr), scratch_per_n2, gm,
                                             const_cast<DfInst *>(s.dfs));
    return cudaGetLastError();
}

}  // namespace ss
