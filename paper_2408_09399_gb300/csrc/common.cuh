// common.cuh -- device helpers shared by the libtmfg kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tmfg.h"

namespace tmfg {

constexpr int kWarp = 32;
constexpr uint16_t kNone16 = 0xFFFFu;  // "no vertex" in 16-bit vertex arrays

// Record the first error of a run in the device status word.
__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// -0.0 and +0.0 are the same similarity.
template <typename T>
__device__ __forceinline__ T canon(T x)
{
    return x == T(0) ? T(0) : x;
}

// Order-preserving unsigned image of a (canonical, non-NaN) float/double.
__device__ __forceinline__ uint32_t ord_key(float x)
{
    uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ uint64_t ord_key(double x)
{
    uint64_t u = (uint64_t)__double_as_longlong(x);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// Exact-rounding adds (no FMA contraction can touch these).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// x * 2^40 rounded to the nearest integer (ties to even), as int64.
template <typename T>
__device__ __forceinline__ long long quantize40(T x)
{
    return __double2ll_rn((double)x * 1099511627776.0);
}

// Valid off-diagonal entry: finite and |x| <= 64.  Returns 0 or a code.
template <typename T>
__device__ __forceinline__ int check_entry(T x)
{
    if (!(x == x) || x - x != T(0)) return TMFG_ENONFINITE;  // NaN or +-inf
    if (x > T(64) || x < T(-64)) return TMFG_ERANGE;
    return 0;
}

template <typename T>
__device__ __forceinline__ T shfl(T v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

}  // namespace tmfg
