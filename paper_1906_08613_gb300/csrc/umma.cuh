// Fifth-generation tensor cores (tcgen05) for the refined modes' trailing
// updates: tensor memory (TMEM) accumulators, shared-memory operand
// descriptors, single-thread MMA issue, completion through an mbarrier.
//
// Operand layout (K-major, no swizzle).  An operand with R rows and KT
// elements of K per row is stored as 8-row x 16-byte core matrices:
//   byte(r, k) = (r / 8) * SBO + (k / EPC) * 128 + (r % 8) * 16 + (k % EPC) * ES
// with ES the element size, EPC = 16 / ES elements per 16 bytes, the K-adjacent
// core matrices 128 bytes apart (the descriptor's leading-dimension offset)
// and row groups SBO = (KT / EPC) * 128 bytes apart (its stride-dimension
// offset).  One MMA consumes 32 bytes of K per row (8 TF32 or 16 BF16
// elements), so step s of a K loop starts s * 256 bytes further.
//
// Accumulator layout (M = 128, one CTA): row i of D is TMEM lane i, column j
// is TMEM column c0 + j, FP32.  Warp w of the CTA reads and writes lanes
// 32 (w % 4) .. 32 (w % 4) + 31 only.
//
// Every wait on an mbarrier is bounded; a wait that runs out sets the
// caller's error flag instead of hanging.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace ss {
namespace tc {

enum Kind { K_TF32 = 0, K_BF16 = 1 };

template <int KIND> struct KindTraits;
template <> struct KindTraits<K_TF32> {
    static constexpr int ES = 4, EPC = 4, KSTEP = 8;   // element bytes, elements per 16 B, K per MMA
    static constexpr uint32_t FMT = 2;
};
template <> struct KindTraits<K_BF16> {
    static constexpr int ES = 2, EPC = 8, KSTEP = 16;
    static constexpr uint32_t FMT = 1;
};

// Byte offset of element (r, k) in a K-major operand whose rows hold kt
// elements of K.
template <int KIND>
__host__ __device__ __forceinline__ uint32_t op_offset(int r, int k, int kt)
{
    using KT = KindTraits<KIND>;
    const uint32_t sbo = (uint32_t)(kt / KT::EPC) * 128u;
    return (uint32_t)(r >> 3) * sbo + (uint32_t)(k / KT::EPC) * 128u + (uint32_t)(r & 7) * 16u +
           (uint32_t)(k % KT::EPC) * KT::ES;
}

// Store one FP32 value as an operand element (TF32 rounded to nearest, or
// BF16 rounded to nearest even).
template <int KIND>
__device__ __forceinline__ void op_store(unsigned char *base, int r, int k, int kt, float v)
{
    if constexpr (KIND == K_TF32) {
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
        *reinterpret_cast<uint32_t *>(base + op_offset<KIND>(r, k, kt)) = t;
    } else {
        *reinterpret_cast<__nv_bfloat16 *>(base + op_offset<KIND>(r, k, kt)) = __float2bfloat16_rn(v);
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K-adjacent core matrices), stride-dimension byte offset (8-row
// groups), the fixed version bits 0b001 at 46..48, base offset 0, relative
// leading-dimension mode, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Descriptor of K step s of an operand (rows from r0, a multiple of 8) laid
// out as op_offset<KIND> with kt elements of K per row.
template <int KIND>
__device__ __forceinline__ uint64_t op_desc(const unsigned char *base, int r0, int s, int kt)
{
    using KT = KindTraits<KIND>;
    const uint32_t sbo = (uint32_t)(kt / KT::EPC) * 128u;
    const uint32_t a = smem_u32(base) + (uint32_t)(r0 >> 3) * sbo + (uint32_t)s * 256u;
    return sdesc(a, 128u, sbo);
}

// Instruction descriptor of kind::tf32 / kind::f16 with FP32 accumulation,
// both operands K-major: D format at bits 4..5, A / B formats at 7..9 and
// 10..12, negate A at 13, N / 8 at 17..22, M / 16 at 24..28.
template <int KIND>
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool neg_a)
{
    return (1u << 4) | (KindTraits<KIND>::FMT << 7) | (KindTraits<KIND>::FMT << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One MMA, issued by a single thread: D[tmem] (+)= A * B^T.
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, bool accumulate)
{
    const uint32_t acc = accumulate ? 1u : 0u;
    if constexpr (KIND == K_TF32) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
    } else {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                     :: "r"(d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
    }
}

// Arrive once on the mbarrier when every MMA this thread issued so far has
// completed.
__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make this thread's generic-proxy shared-memory writes visible to the
// tensor cores (async proxy).
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the mbarrier completes the phase with the given parity, at most
// `limit` polls.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, uint32_t limit = 1u << 22)
{
    const uint32_t a = smem_u32(mbar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// TMEM allocation by one whole warp: ncols (a power of two, 32..512)
// columns, the base address written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(slot)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}

// TMEM address of lane quarter q (lanes 32 q ..), column c.
__device__ __forceinline__ uint32_t taddr(uint32_t base, int q, int c)
{
    return base + ((uint32_t)(32 * q) << 16) + (uint32_t)c;
}

// Warp-wide load of 16 consecutive columns of this warp's 32 lanes: thread t
// gets lane 32 q + t, columns c .. c + 15.
__device__ __forceinline__ void ld16(uint32_t ta, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Warp-wide store of 16 consecutive columns of this warp's 32 lanes.
__device__ __forceinline__ void st16(uint32_t ta, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
                 :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                    "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                    "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                    "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                    "r"(__float_as_uint(v[15]))
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Smallest legal TMEM allocation holding `cols` columns.
__host__ __device__ constexpr uint32_t tmem_cols(int cols)
{
    return cols <= 32 ? 32u : cols <= 64 ? 64u : cols <= 128 ? 128u : cols <= 256 ? 256u : 512u;
}

}  // namespace tc
}  // namespace ss
