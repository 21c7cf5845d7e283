// tma_util.cuh -- tensor-memory-accelerator (TMA) tile loads and mbarrier
// waits for the TMA-staged stage kernels (sm_90+ PTX, used on sm_103a).
//
// A 4-D tensor map (x, y, z, field) describes one state's fields in HBM; a
// tile load copies a box of (width, height, 1 plane, fields) doubles into
// shared memory, x fastest, and signals completion of its bytes on an
// mbarrier.  Loads only: this GPU's own memory, no multicast, no stores.
// Every wait is bounded: after kWaitCycles SM clocks without completion the
// caller is told, records an error status and stops waiting.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hydro {

// tensor maps of one stage input: conserved fields (5) and primitives
// (p, v_x, v_y, v_z); the box covers the fields a stage kernel stages
struct TmaMaps {
    CUtensorMap u;
    CUtensorMap w;
};

// about one second at the GB300's SM clock
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// the calling thread arrives and announces `bytes` of transactions
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// wait for the phase with parity `parity` to complete; false after the cycle budget
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// order this thread's earlier shared-memory accesses (generic proxy) before
// later TMA writes to the same memory (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// box load at element coordinates (x, y, z, f) of map `m` into `dst`
// (16-byte aligned; x * 8 bytes must be a multiple of 16)
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* m, int x, int y, int z, int f, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace hydro
