// Helpers shared by the tcgen05 (5th-generation tensor core) kernels: shared-memory and
// instruction descriptors, and a bounded mbarrier wait.
#pragma once
#include <stdint.h>

namespace qm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; lbo = byte stride between core
// matrices (8 rows x 16 bytes) adjacent along K, sbo = byte stride between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version (fixed 0b001)
    return d;                // base offset 0, relative LBO, swizzle none
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// wait for the phase `phase` of the mbarrier to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long limit) {
    for (long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace tc
}  // namespace qm
