// pw_noalloc.cu -- batched evaluation without any caller-provided or
// library-allocated device buffer.
//
// pw_advect_batched needs the batch plan in device memory: it holds the TMA
// descriptors the persistent kernel reads and the atomic counter it takes
// work from. Some callers cannot obtain that memory: real-time loops that
// must not call cudaMalloc (it can synchronise the device, and its latency
// is unbounded), plug-ins inside a host program that owns every device
// allocation, and programs whose device memory another allocator has wholly
// reserved. For them this entry point keeps the plan in a fixed file-scope
// device array that every GPU loading the library holds until the process
// exits, and copies the caller's host plan into it per call.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "pw.h"
#include "pw_internal.h"

namespace {

// Room for the largest plan this entry point accepts (PW_NOALLOC_MAX_DOMAINS).
constexpr size_t kScratchBytes =
    offsetof(pw::BatchPlan, dom) + (size_t)PW_NOALLOC_MAX_DOMAINS * sizeof(pw::BatchDomain);

// The plan scratch: one per device, shared by every call on that device.
static __device__ __align__(256) unsigned char g_plan_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_plan_scratch, per device

thread_local std::string t_err;

int fail(int code, const char* fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    t_err = buf;
    return code;
}

}  // namespace

// Error text of this entry point's last failure in this thread (pw_last_error
// reports the failures of every other entry point).
extern "C" const char* pw_noalloc_last_error(void) { return t_err.c_str(); }

extern "C" int pw_advect_batched_noalloc(pw_dtype dtype, int variant, const void* plan_host, size_t plan_bytes,
                                         long long n_items, void* stream) {
    if (!plan_host) return fail(PW_ENULL, "pw_advect_batched_noalloc: plan_host is NULL");
    if (dtype != PW_F64_PAIRED && dtype != PW_F32 && dtype != PW_F32_SPLIT)
        return fail(PW_EUNSUPPORTED, "pw_advect_batched_noalloc: no batched kernel for dtype %lld", (long long)dtype);
    if (variant < 0 || variant >= pw_variant_count(dtype))
        return fail(PW_EINVAL, "pw_advect_batched_noalloc: variant %lld out of range", variant);
    if (plan_bytes < offsetof(pw::BatchPlan, dom))
        return fail(PW_EINVAL, "pw_advect_batched_noalloc: plan_bytes %lld too small", (long long)plan_bytes);
    const pw::BatchPlan* hp = static_cast<const pw::BatchPlan*>(plan_host);
    if (hp->n_domains < 1 || hp->n_domains > PW_NOALLOC_MAX_DOMAINS)
        return fail(PW_EINVAL, "pw_advect_batched_noalloc: %lld domains, at most %lld are supported",
                    hp->n_domains, PW_NOALLOC_MAX_DOMAINS);
    const size_t need = pw::batch_plan_bytes(hp->n_domains);
    if (plan_bytes < need || need > kScratchBytes)
        return fail(PW_EINVAL, "pw_advect_batched_noalloc: plan_bytes %lld < %lld", (long long)plan_bytes,
                    (long long)need);
    if (hp->dtype != (int)dtype || hp->variant != variant || hp->n_items != n_items || n_items < 1)
        return fail(PW_EINVAL, "pw_advect_batched_noalloc: plan was built for another dtype, variant or size");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PW_ECUDA, "pw_advect_batched_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return fail(PW_EINVAL, "pw_advect_batched_noalloc: device %lld", dev);
    void* scratch = nullptr;
    {
        // first call on this device (with it current): look up the array's address
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_plan_scratch);
            if (e != cudaSuccess || !p)
                return fail(PW_ECUDA, "pw_advect_batched_noalloc: cudaGetSymbolAddress failed");
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    pw::BatchPlan* plan = static_cast<pw::BatchPlan*>(scratch);
    // the array keeps the previous call's plan: overwrite it, then zero the
    // work counter the kernel takes items from
    e = cudaMemcpyAsync(scratch, plan_host, need, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&plan->counter, 0, sizeof(plan->counter), st);
    if (e != cudaSuccess) return fail(PW_ECUDA, "pw_advect_batched_noalloc: copying the plan failed");
    e = dtype == PW_F64_PAIRED ? pw::launch_paired_batched(variant, plan, n_items, st)
                               : pw::launch_split_batched(variant, plan, n_items, st);
    if (e != cudaSuccess) return fail(PW_ECUDA, "pw_advect_batched_noalloc: launch failed");
    return PW_OK;
}
