// tc_ptx.cuh -- inline-PTX helpers for the tcgen05 kernels (sm_103a): shared-memory addresses,
// bounded mbarrier waits, UMMA shared-memory descriptors (K-major, no swizzle), the BF16 MMA
// with FP32 accumulation in tensor memory, and tensor-memory loads and stores.
#pragma once

#include <cstdint>

namespace mcmcdet {

constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Per-thread tensor-memory row segments (shape 32x32b: thread i of the warp owns lane
// quadrant-base + i): NS consecutive 32-bit columns at address a and 8 at address b, moved in one
// statement together with the completion wait, so that no use of the loaded registers (or reuse
// of the stored ones) can be scheduled before the transfer has completed.
template <int NS>
__device__ __forceinline__ void tmem_ld_pair(uint32_t a, uint32_t b, uint32_t (&s)[NS], uint32_t (&e)[8]);
template <int NS>
__device__ __forceinline__ void tmem_st_pair(uint32_t a, uint32_t b, const uint32_t (&s)[NS],
                                             const uint32_t (&e)[8]);

template <>
__device__ __forceinline__ void tmem_ld_pair<4>(uint32_t a, uint32_t b, uint32_t (&s)[4], uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%4,%5,%6,%7,%8,%9,%10,%11}, [%13];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(e[0]), "=r"(e[1]), "=r"(e[2]), "=r"(e[3]), "=r"(e[4]), "=r"(e[5]), "=r"(e[6]), "=r"(e[7])
        : "r"(a), "r"(b)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_st_pair<4>(uint32_t a, uint32_t b, const uint32_t (&s)[4],
                                                const uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%2,%3,%4,%5};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%6,%7,%8,%9,%10,%11,%12,%13};\n"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(a), "r"(b), "r"(s[0]), "r"(s[1]), "r"(s[2]), "r"(s[3]), "r"(e[0]), "r"(e[1]), "r"(e[2]), "r"(e[3]), "r"(e[4]), "r"(e[5]), "r"(e[6]), "r"(e[7])
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_ld_pair<8>(uint32_t a, uint32_t b, uint32_t (&s)[8], uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(e[0]), "=r"(e[1]), "=r"(e[2]), "=r"(e[3]), "=r"(e[4]), "=r"(e[5]), "=r"(e[6]), "=r"(e[7])
        : "r"(a), "r"(b)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_st_pair<8>(uint32_t a, uint32_t b, const uint32_t (&s)[8],
                                                const uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2,%3,%4,%5,%6,%7,%8,%9};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%10,%11,%12,%13,%14,%15,%16,%17};\n"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(a), "r"(b), "r"(s[0]), "r"(s[1]), "r"(s[2]), "r"(s[3]), "r"(s[4]), "r"(s[5]), "r"(s[6]), "r"(s[7]), "r"(e[0]), "r"(e[1]), "r"(e[2]), "r"(e[3]), "r"(e[4]), "r"(e[5]), "r"(e[6]), "r"(e[7])
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_ld_pair<16>(uint32_t a, uint32_t b, uint32_t (&s)[16], uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%25];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]), "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15]), "=r"(e[0]), "=r"(e[1]), "=r"(e[2]), "=r"(e[3]), "=r"(e[4]), "=r"(e[5]), "=r"(e[6]), "=r"(e[7])
        : "r"(a), "r"(b)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_st_pair<16>(uint32_t a, uint32_t b, const uint32_t (&s)[16],
                                                const uint32_t (&e)[8])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17};\n"
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%1], {%18,%19,%20,%21,%22,%23,%24,%25};\n"
        "tcgen05.wait::st.sync.aligned;"
        :
        : "r"(a), "r"(b), "r"(s[0]), "r"(s[1]), "r"(s[2]), "r"(s[3]), "r"(s[4]), "r"(s[5]), "r"(s[6]), "r"(s[7]), "r"(s[8]), "r"(s[9]), "r"(s[10]), "r"(s[11]), "r"(s[12]), "r"(s[13]), "r"(s[14]), "r"(s[15]), "r"(e[0]), "r"(e[1]), "r"(e[2]), "r"(e[3]), "r"(e[4]), "r"(e[5]), "r"(e[6]), "r"(e[7])
        : "memory");
}

}  // namespace mcmcdet
