// diag.cu -- latency of dependent device-memory loads (pointer chasing).
//
// No counterpart in the paper.  The insertion loop of Algorithms 1 and 2 is a
// chain of dependent round trips (a probe of a sorted row, then the gathers
// of S, then the index update), so its bound is memory latency, not
// bandwidth; this measures the two latencies that bound it on the device it
// runs on: an L2 hit and a DRAM miss (with the address-translation misses of
// a multi-gigabyte working set, as the loop sees them).
//
// A second diagnostic times the step that the cluster loop kernel takes once
// per insertion: every CTA of a thread-block cluster stores a 16-byte record
// into a slot of every CTA's shared memory, then the cluster passes a
// barrier (release / acquire).
//
// The buffer is `bytes` rounded down to a power of two of 128-byte lines;
// line i holds the index of the next line, (a*i + c) mod L with a = 1 mod 4
// and c odd -- a full-period linear congruential step, so the chain visits
// every line once per period in a scattered order.  One thread follows it
// with L1-bypassing loads; the device clock times `hops` of them.
#include <cooperative_groups.h>

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

// One cluster of C CTAs of 64 threads: `iters` exchanges of a 16-byte record
// (lane j of warp 0 stores into CTA j) each followed by a cluster barrier.
template <int C>
__global__ void __launch_bounds__(64, 1) exchange_kernel(int iters, double *ns_out)
{
    __shared__ uint4 slot[2][C];
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    const unsigned r = cl.block_rank();
    if (threadIdx.x < 2 * C) (&slot[0][0])[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
    cl.sync();
    uint32_t acc = 0;
    const uint64_t t0 = globaltimer_ns();
    for (int k = 0; k < iters; ++k) {
        const int par = k & 1;
        if (threadIdx.x < C) {
            uint4 *dst = cl.map_shared_rank(&slot[par][r], threadIdx.x);
            *dst = make_uint4((uint32_t)k, r, acc, 0u);
        }
        asm volatile("barrier.cluster.arrive.release;\n\t"
                     "barrier.cluster.wait.acquire;" ::: "memory");
        acc += slot[par][(k + r) % C].x;
    }
    const uint64_t t1 = globaltimer_ns();
    cl.sync();
    // acc keeps the reads live; it is a sum of loop counters, never ~0
    if (r == 0 && threadIdx.x == 0)
        ns_out[0] = acc == 0xFFFFFFFFu ? -1.0 : (double)(t1 - t0) / (double)iters;
}

template <int C>
cudaError_t launch_exchange(int iters, double *dns)
{
    if (C > 8) {
        const cudaError_t e = cudaFuncSetAttribute(
            exchange_kernel<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1, 1);
    cfg.blockDim = dim3(64, 1, 1);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, exchange_kernel<C>, iters, dns);
}

}  // namespace
}  // namespace tmfg

extern "C" int tmfg_cluster_exchange_latency(tmfg_ctx *ctx, int32_t cluster, int32_t iters,
                                             double *ns_per_exchange)
{
    using namespace tmfg;
    if (!ctx || !ns_per_exchange || iters < 1 || (cluster != 8 && cluster != 16))
        return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    double *dns = nullptr;
    if (cudaMalloc(&dns, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return TMFG_ENOMEM;
    }
    const cudaError_t e = cluster == 16 ? launch_exchange<16>(iters, dns)
                                        : launch_exchange<8>(iters, dns);
    double ns = -1.0;
    const bool ok = e == cudaSuccess && cudaGetLastError() == cudaSuccess &&
                    cudaMemcpy(&ns, dns, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(dns);
    if (!ok || ns < 0.0) {
        cudaGetLastError();
        return TMFG_ECUDA;
    }
    *ns_per_exchange = ns;
    return TMFG_OK;
}

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
