// Helpers for the 5th-generation tensor-core kernels (tcgen05 MMA with
// operands in shared memory and the accumulator in tensor memory).
#pragma once

#include <stdint.h>

namespace nfl {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N)
// byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Byte offset of element (row, k) in a K-major, no-swizzle operand holding
// K values per row: core matrices of 8 rows x 16 bytes, the K/4 core
// matrices of an 8-row group 128 B apart (leading offset), 8-row groups
// K * 32 B apart (stride offset).
template <int K>
__device__ __forceinline__ uint32_t kmajor_off_k(int row, int k) {
    return (uint32_t)((((row >> 3) * (K / 4) + (k >> 2)) * 128) + ((row & 7) * 16) + ((k & 3) * 4));
}
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) { return kmajor_off_k<16>(row, k); }

// One D (+)= A B step of kind::tf32 with operands described in shared memory.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate));
}

// Device clock in nanoseconds.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, at most `limit` polls and `limit_ns`
// nanoseconds; true if it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar_addr, uint32_t parity, uint32_t limit,
                                                  uint64_t limit_ns = 2000000000ull) {
    const uint64_t t0 = global_ns();
    uint32_t done = 0, spins = 0;
    while (!done) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar_addr), "r"(parity));
        if (done) break;
        if (++spins > limit) break;
        if ((spins & 31u) == 0u && global_ns() - t0 > limit_ns) break;
    }
    return done != 0;
}

// Limits of the bounded waits on an MMA-completion mbarrier (polls, and 2 s of
// device time unless a fault test shortens it): a wait that runs out sets the
// plan's error flag and the kernel skips its remaining work.
constexpr uint32_t kSpinLimit = 1u << 26;

}  // namespace nfl
