// diag.cu -- latency of dependent device-memory loads (pointer chasing).
//
// No counterpart in the paper.  The insertion loop of Algorithms 1 and 2 is a
// chain of dependent round trips (a probe of a sorted row, then the gathers
// of S, then the index update), so its bound is memory latency, not
// bandwidth; this measures the two latencies that bound it on the device it
// runs on: an L2 hit and a DRAM miss (with the address-translation misses of
// a multi-gigabyte working set, as the loop sees them).
//
// The buffer is `bytes` rounded down to a power of two of 128-byte lines;
// line i holds the index of the next line, (a*i + c) mod L with a = 1 mod 4
// and c odd -- a full-period linear congruential step, so the chain visits
// every line once per period in a scattered order.  One thread follows it
// with L1-bypassing loads; the device clock times `hops` of them.
#include "ctx.cuh"

namespace tmfg {
namespace {

constexpr uint32_t kLcgA = 1664525u, kLcgC = 1013904223u;

__global__ void chase_init_kernel(uint32_t *buf, uint32_t mask)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i <= mask;
         i += (size_t)gridDim.x * blockDim.x)
        buf[i * 32] = (kLcgA * (uint32_t)i + kLcgC) & mask;
}

__global__ void chase_kernel(const uint32_t *buf, uint32_t warm, uint32_t hops, double *ns_out)
{
    uint32_t p = 0;
    for (uint32_t i = 0; i < warm; ++i) p = __ldcg(buf + (size_t)p * 32);
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0; i < hops; ++i) p = __ldcg(buf + (size_t)p * 32);
    const uint64_t t1 = globaltimer_ns();
    // p keeps the chain live; it is always a line index, never ~0
    ns_out[0] = p == 0xFFFFFFFFu ? -1.0 : (double)(t1 - t0) / (double)hops;
}

}  // namespace
}  // namespace tmfg

extern "C" int tmfg_memory_latency(tmfg_ctx *ctx, int64_t bytes, int32_t hops, int32_t warm,
                                   double *ns_per_hop)
{
    using namespace tmfg;
    if (!ctx || !ns_per_hop || bytes < 4096 || hops < 1 || warm < 0) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    uint64_t lines = 1;
    while (lines * 2 * 128 <= (uint64_t)bytes && lines * 2 <= (1ull << 31)) lines *= 2;
    uint32_t *buf = nullptr;
    double *dns = nullptr;
    if (cudaMalloc(&buf, lines * 128) != cudaSuccess) {
        cudaGetLastError();
        return TMFG_ENOMEM;
    }
    if (cudaMalloc(&dns, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return TMFG_ENOMEM;
    }
    const uint32_t mask = (uint32_t)(lines - 1);
    chase_init_kernel<<<4 * ctx->num_sms, 256>>>(buf, mask);
    chase_kernel<<<1, 1>>>(buf, (uint32_t)warm, (uint32_t)hops, dns);
    double ns = -1.0;
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpy(&ns, dns, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(dns);
    cudaFree(buf);
    if (!ok || ns < 0.0) return TMFG_ECUDA;
    *ns_per_hop = ns;
    return TMFG_OK;
}
