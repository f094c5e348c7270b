// akra_tc.cuh -- the tcgen05 (5th-generation tensor core) primitives the FP32 Legendre
// contraction uses: TMEM allocation, shared-memory matrix descriptors, the TF32 MMA with an FP32
// accumulator in tensor memory, its completion barrier and the TMEM -> register loads.
//
// Operand layout: no-swizzle, K-major, "canonical" core matrices of 8 rows x 16 bytes
// (8 rows x 4 TF32 elements, 128 contiguous bytes); the core matrix holding (row, k) starts at
// (row / 8) * SBO + (k / 4) * LBO.  Every operand here is a tile of 8 K-elements per row, with
// LBO = 128 B (the two core matrices along K adjacent) and SBO = 256 B (8-row groups).
#pragma once
#include <cstdint>

#include "akra_internal.cuh"

namespace akra {
namespace tc {

constexpr uint32_t kLBO = 128, kSBO = 256;   // bytes, see above

// byte offset of element (row, k), 0 <= k < 8, in a K = 8 operand tile
__device__ __forceinline__ uint32_t tile_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1
// (bits 46-48 = 0b001), base offset 0, relative LBO, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::tf32: D = F32, A = B = TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// arrive on the mbarrier once every MMA this thread issued so far has completed
__device__ __forceinline__ void commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(count));
}

// an mbarrier with no pending arrivals goes back to plain shared memory (before a re-init)
__device__ __forceinline__ void mbar_inval(uint64_t *mbar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(mbar)) : "memory");
}

// wait for the completion of the mbarrier phase with the given parity, at most `limit` polls,
// and not at all once the launch's error flag is set; returns false on timeout (the caller
// records an error instead of waiting forever)
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int limit, const int *err)
{
    uint32_t done = 0;
    for (int it = 0; it < limit; it++) {
        if (err && (it & 1023) == 1023 && *(volatile const int *)err) return false;
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// TMEM allocation (one warp), address written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(dst)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory writes of this thread become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 4 consecutive TMEM columns of this warp's 32 lanes (lane = row); taddr holds the warp's lane
// base in bits 31..16 and the column in bits 15..0
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r0, r1, r2, r3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
}

// 16-byte asynchronous copy global -> shared (cp.async, L2 only); src_bytes = 0 zero-fills the
// destination without reading the source
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_u32(smem_dst)), "l"(__cvta_generic_to_global(gsrc)), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed copy groups are still pending
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// split x into a TF32 head (the top 11 significant bits, exactly representable) and the FP32
// remainder x - head (exact); the tensor core reads the remainder's top 11 bits, so
// head*b_head + head*b_rest + rest*b_head carries ~21 bits of each product
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

}  // namespace tc
}  // namespace akra
