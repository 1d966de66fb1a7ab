// Tensor-core self-test: one 128 x N tile D (+)= op(A) B^T through the same
// operand layout, descriptors, TMEM accumulator and completion path as the
// refined modes' trailing updates (umma.cuh), so that a test can pin each
// encoding against a host product.
#include "ss_internal.h"
#include "umma.cuh"

namespace ss {
namespace {

constexpr int kSelfTestThreads = 128;

__host__ __device__ constexpr size_t selftest_smem(int n, int k, int es)
{
    return 1024 + (size_t)128 * k * es + (size_t)n * k * es + 64;
}

template <int KIND>
__global__ void __launch_bounds__(kSelfTestThreads) umma_selftest_kernel(int n, int k, const float *A, const float *B,
                                                                       const float *C, float *D, int flags,
                                                                       int *status)
{
    using KT = tc::KindTraits<KIND>;
    extern __shared__ unsigned char smraw[];
    const uint32_t mis = tc::smem_u32(smraw) & 1023u;
    unsigned char *sA = smraw + ((1024u - mis) & 1023u);
    unsigned char *sB = sA + (size_t)128 * k * KT::ES;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + (size_t)n * k * KT::ES);
    uint32_t *slot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < 128 * k; e += kSelfTestThreads) tc::op_store<KIND>(sA, e / k, e % k, k, A[e]);
    for (int e = tid; e < n * k; e += kSelfTestThreads) tc::op_store<KIND>(sB, e / k, e % k, k, B[e]);
    tc::fence_smem_to_async();
    const uint32_t ncols = tc::tmem_cols(n);
    if (warp == 0) tc::tmem_alloc(slot, ncols);
    if (tid == 0) tc::mbar_init(mbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t base = *slot;
    const bool acc = (flags & 1) != 0;
    if (acc) {
        for (int c = 0; c < n; c += 16) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = C[(long)(32 * warp + lane) * n + c + i];
            tc::st16(tc::taddr(base, warp, c), v);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
        const uint32_t id = tc::idesc<KIND>(128, n, (flags & 2) != 0);
        for (int s = 0; s < k / KT::KSTEP; ++s)
            tc::mma<KIND>(base, tc::op_desc<KIND>(sA, 0, s, k), tc::op_desc<KIND>(sB, 0, s, k), id, acc || s > 0);
        tc::commit(mbar);
    }
    bool ok = tc::mbar_wait(mbar, 0);
    if (!ok) ok = tc::mbar_wait(mbar, 0);   // let an MMA still in flight finish before TMEM is freed
    tc::fence_after();
    if (ok) {
        for (int c = 0; c < n; c += 16) {
            float v[16];
            tc::ld16(tc::taddr(base, warp, c), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(long)(32 * warp + lane) * n + c + i] = v[i];
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(base, ncols);
    if (tid == 0) *status = ok ? 0 : 1;
}

}  // namespace
}  // namespace ss

extern "C" int ss_umma_selftest(int kind, int n, int k, const float *d_a, const float *d_b, const float *d_c,
                                float *d_d, int flags, int *d_status, void *stream)
{
    using namespace ss;
    if (kind != tc::K_TF32 && kind != tc::K_BF16) return -1;
    if (n < 16 || n > 256 || n % 16) return -2;
    const int kstep = kind == tc::K_TF32 ? tc::KindTraits<tc::K_TF32>::KSTEP : tc::KindTraits<tc::K_BF16>::KSTEP;
    if (k < kstep || k > 64 || k % kstep) return -3;
    if (!d_a) return -4;
    if (!d_b) return -5;
    if ((flags & 1) && !d_c) return -6;
    if (!d_d) return -7;
    if (flags & ~3) return -8;
    if (!d_status) return -9;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int es = kind == tc::K_TF32 ? 4 : 2;
    const size_t smem = selftest_smem(n, k, es);
    cudaError_t e;
    if (kind == tc::K_TF32) {
        e = cudaFuncSetAttribute(umma_selftest_kernel<tc::K_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            umma_selftest_kernel<tc::K_TF32><<<1, kSelfTestThreads, smem, st>>>(n, k, d_a, d_b, d_c, d_d, flags,
                                                                                d_status);
    } else {
        e = cudaFuncSetAttribute(umma_selftest_kernel<tc::K_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            umma_selftest_kernel<tc::K_BF16><<<1, kSelfTestThreads, smem, st>>>(n, k, d_a, d_b, d_c, d_d, flags,
                                                                                d_status);
    }
    if (e != cudaSuccess) return SS_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : SS_ERR_CUDA;
}
