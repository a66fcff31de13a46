// pw_common.cuh -- device helpers shared by the PW advection kernels:
// mbarrier and TMA (cp.async.bulk.tensor) wrappers in inline PTX for sm_103a,
// bounded waits, and the library's device status word.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pw {

// Longest a kernel waits on one mbarrier phase before giving up (ns). A
// tile load completes in microseconds; this bound only matters if a copy
// never lands, in which case the kernel records PW status and returns.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

// Bits of the device status word: a bounded wait expired; a batched kernel
// was given a plan built for another dtype or variant.
constexpr unsigned int kStatusTimeout = 1u;
constexpr unsigned int kStatusBadPlan = 2u;

namespace {
// Device status word of this translation unit (each kernel .cu file has its
// own copy; the library ORs them when the host asks).
__device__ unsigned int tu_status;

// Copy this unit's status word to the host and clear it (ordered on st).
__host__ inline cudaError_t read_and_clear_tu_status(unsigned int* out, cudaStream_t st) {
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(out, tu_status, sizeof(unsigned int), 0, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(tu_status, &zero, sizeof(unsigned int), 0, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}
}  // namespace

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Second bound on a wait, independent of the timer: try_wait polls.
constexpr unsigned int kWaitMaxPolls = 1u << 28;

// Wait for the phase with the given parity to complete, for at most limit_ns
// (and at most kWaitMaxPolls polls). Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned int n = 0; n < kWaitMaxPolls; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

// 3D tiled TMA load of one box into shared memory, completing on `bar`.
// x must be a multiple of 16 bytes / element size (checked by the host).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory
// before later async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace pw
