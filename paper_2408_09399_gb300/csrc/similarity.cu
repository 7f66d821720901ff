// similarity.cu -- the Pearson similarity matrix of n series (the input the
// paper's TMFG is built from: Section 5, "Datasets", Pearson correlation of
// every pair of series), on the device.
//
// rho_ij = <x_i - mean_i, x_j - mean_j> / (|x_i - mean_i| |x_j - mean_j|).
// Centring and norms are computed in double, one CTA per series; each
// normalised series y_i (unit norm, in double) is then stored for the
// product in the requested precision:
//   F64     y in double, SIMT double dot products;
//   F32     y rounded to float, SIMT float dot products (FMA);
//   BF16X3  y = hi + lo with hi = bf16(y), lo = bf16(y - hi); rho = hi.hi' +
//           hi.lo' + lo.hi' on the tensor cores (tcgen05.mma kind::f16, FP32
//           accumulation in tensor memory); the lo.lo' term (< 2^-16
//           relative) is dropped;
//   TF32X3  the same split with TF32 halves (tcgen05.mma kind::tf32).
// Only the tiles on or above the diagonal are computed; each value is written
// to (i,j) and (j,i), so S is exactly symmetric, and the diagonal is 1.
//
// Tensor-core kernel: persistent, one CTA per SM, walking 128 x 128 output
// tiles on or above the diagonal.  Warp 0 lane 0 streams 128-byte-wide K
// slices of the four operand tiles (A hi/lo, B hi/lo) into shared memory
// with TMA (128-byte swizzle), three stages deep, across tile boundaries,
// each stage guarded by a "full" and an "empty" mbarrier.  Warp 1 owns the
// tensor memory (512 columns: two tiles' accumulators, two accumulators of
// 128 columns each per tile) and lane 0 issues the MMAs (4 K steps x 3
// products per slice, slice k into accumulator k mod 2) and commits each
// slice's completion to its "empty" barrier and each tile's to its buffer's
// "full" barrier.  Warps 2..5 drain a finished buffer while the next tile
// accumulates into the other: tcgen05.ld 32x32b of their 32 rows, the two
// accumulators added in FP32, rows stored as 16-byte vectors and the
// transpose with consecutive lanes on consecutive addresses; then the
// buffer's "drained" barrier.  The tensor core's FP32 accumulation
// truncates, so its error grows with the number of accumulation steps and
// the size of the partial sums; two accumulators halve both.  Every
// mbarrier wait is bounded by the device clock; a wait that runs out
// records TMFG_ETIMEOUT, and the CTA still frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace tmfg {

namespace {

constexpr int kTile = 128;        // output tile (M = N = 128)
constexpr int kStages = 3;
constexpr int kRowBytes = 128;    // bytes of one K slice of one row
constexpr int kOpBytes = kTile * kRowBytes;  // one operand tile slice: 16 KB
constexpr int kStageBytes = 4 * kOpBytes;    // A hi, A lo, B hi, B lo
constexpr int kTcThreads = 192;   // warp 0: TMA, warp 1: MMA, warps 2..5: epilogue
constexpr int kAcc = 2;           // accumulators per tile (128 TMEM columns each)
constexpr int kBufCols = kAcc * kTile;  // one tile's accumulators; two tiles in flight
constexpr size_t kTcSmem = kStages * kStageBytes + 1024 + 256;

// --------------------------------------------------------------- prep
// One CTA per series: mean and sum of squares in double (block reduction in
// a fixed order), then the normalised values in the product's format.
template <int Prec>
__global__ void __launch_bounds__(256) sim_prep_kernel(const float *X, int n, int T, long long ldx,
                                                       void *hi, void *lo, long long ldy,
                                                       int *status)
{
    __shared__ double red[256];
    const int i = blockIdx.x, t0 = threadIdx.x;
    if (i >= n) return;
    const float *x = X + (long long)i * ldx;
    double s = 0.0;
    bool bad = false;
    for (int t = t0; t < T; t += 256) {
        const float v = x[t];
        bad |= !(v - v == 0.0f);
        s += (double)v;
    }
    const int any_bad = __syncthreads_or(bad);
    red[t0] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t0 < o) red[t0] += red[t0 + o];
        __syncthreads();
    }
    const double mean = red[0] / (double)T;
    __syncthreads();
    double q = 0.0;
    for (int t = t0; t < T; t += 256) {
        const double d = (double)x[t] - mean;
        q += d * d;
    }
    red[t0] = q;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t0 < o) red[t0] += red[t0 + o];
        __syncthreads();
    }
    const double ss = red[0];
    if (any_bad || !(ss > 0.0)) {  // non-finite values, or a constant series
        if (t0 == 0) set_status(status, TMFG_ENONFINITE);
        return;
    }
    const double inv = 1.0 / sqrt(ss);
    for (int t = t0; t < (int)ldy; t += 256) {
        const double y = t < T ? ((double)x[t] - mean) * inv : 0.0;
        const long long o = (long long)i * ldy + t;
        if (Prec == TMFG_SIM_F64) {
            static_cast<double *>(hi)[o] = y;
        } else if (Prec == TMFG_SIM_F32) {
            static_cast<float *>(hi)[o] = (float)y;
        } else if (Prec == TMFG_SIM_BF16X3) {
            const __nv_bfloat16 h = __double2bfloat16(y);
            static_cast<__nv_bfloat16 *>(hi)[o] = h;
            static_cast<__nv_bfloat16 *>(lo)[o] = __double2bfloat16(y - (double)__bfloat162float(h));
        } else {  // TF32X3: round to 10 explicit mantissa bits (nearest, ties away)
            uint32_t h, l;
            const float yf = (float)y;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(yf));
            const float r = (float)(y - (double)__uint_as_float(h));
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
            static_cast<uint32_t *>(hi)[o] = h;
            static_cast<uint32_t *>(lo)[o] = l;
        }
    }
}

// Tile pair (I <= J) of linear index b over the upper triangle of nt x nt,
// in groups of G tile rows: within a group, column J is visited by the
// group's rows one after the other, so the CTAs that run at the same time
// share their B tiles and the group's A tiles stay in L2 for the sweep.
template <int G>
__device__ __forceinline__ void tri_tile_grouped(int b, int nt, int &I, int &J)
{
    int I0 = 0;
    for (;;) {
        const int I1 = min(I0 + G, nt) - 1;
        const int g = I1 - I0 + 1;
        const int total = g * (g + 1) / 2 + (nt - 1 - I1) * g;
        if (b < total) {
            const int tri = g * (g + 1) / 2;
            if (b < tri) {
                int j = 0;
                while ((j + 1) * (j + 2) / 2 <= b) ++j;
                J = I0 + j;
                I = I0 + (b - j * (j + 1) / 2);
            } else {
                b -= tri;
                J = I1 + 1 + b / g;
                I = I0 + b % g;
            }
            return;
        }
        b -= total;
        I0 += G;
    }
}

// tile pair (I <= J) of linear index b over the upper triangle of nt x nt
__device__ __forceinline__ void tri_tile(int b, int nt, int &I, int &J)
{
    int i = 0, off = 0;
    while (b >= off + (nt - i)) {
        off += nt - i;
        ++i;
    }
    I = i;
    J = i + (b - off);
}

// --------------------------------------------------------------- SIMT paths
// 64 x 64 output tile per CTA (256 threads, 4 x 4 each), K staged through
// shared memory 16 at a time; upper-triangle tiles only.
template <typename T>
__global__ void __launch_bounds__(256) sim_simt_kernel(const T *Y, int n, int K, long long ldy,
                                                       float *S, long long ld, const int *status)
{
    if (*status) return;
    __shared__ T As[16][64 + 1];
    __shared__ T Bs[16][64 + 1];
    const int nt = (n + 63) / 64;
    int I, J;
    tri_tile(blockIdx.x, nt, I, J);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int r = e >> 4, k = e & 15;
            const int gi = I * 64 + r, gj = J * 64 + r;
            As[k][r] = (gi < n && k0 + k < K) ? Y[(long long)gi * ldy + k0 + k] : T(0);
            Bs[k][r] = (gj < n && k0 + k < K) ? Y[(long long)gj * ldy + k0 + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ty * 4 + u];
                b[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = I * 64 + ty * 4 + u, gj = J * 64 + tx * 4 + v;
            if (gi >= n || gj >= n || gi > gj) continue;
            const float r = gi == gj ? 1.0f : (float)acc[u][v];
            S[(long long)gi * ld + gj] = r;
            S[(long long)gj * ld + gi] = r;
        }
}

// --------------------------------------------------------------- tcgen05 path
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Wait for the phase of the given parity to complete; false once the device
// clock passes `deadline`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline)
{
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && globaltimer_ns() > deadline) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand tile, rows of 128 bytes,
// 128-byte swizzle, 8-row groups 1024 bytes apart (tile base 1024-aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of the given format
// (1 = BF16 for kind::f16, 2 = TF32 for kind::tf32), both K-major, M = N = 128.
__host__ __device__ constexpr uint32_t idesc_128x128(uint32_t fmt)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) |
           ((uint32_t)(kTile >> 4) << 24);
}

template <bool kTf32>
__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    if (kTf32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
            : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

template <bool kTf32>
__global__ void __launch_bounds__(kTcThreads, 1)
    sim_tc_kernel(const __grid_constant__ CUtensorMap map_hi,
                  const __grid_constant__ CUtensorMap map_lo, int n, int kblocks, int tiles,
                  float *S, long long ld, bool vec, int *status, unsigned long long timeout_ns)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    // bars[0..S): stage full, [S..2S): stage empty, [2S..2S+2): accumulator
    // buffer full, [2S+2..2S+4): accumulator buffer drained
    uint64_t *full = bars, *empty = bars + kStages, *tfull = bars + 2 * kStages,
             *tempty = bars + 2 * kStages + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = (n + kTile - 1) / kTile;
    constexpr int kElems = kTf32 ? 32 : 64;  // elements per 128-byte K slice
    constexpr uint32_t kIdesc = idesc_128x128(kTf32 ? 2u : 1u);
    const uint64_t deadline = globaltimer_ns() + timeout_ns;
    auto give_up = [&]() {
        set_status(status, TMFG_ETIMEOUT);
        s_abort = 1;
    };

    if (threadIdx.x == 0) {
        s_abort = *status != 0;
        for (int s = 0; s < 2 * kStages + 2; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int b = 0; b < 2; ++b) mbar_init(smem_u32(&tempty[b]), 4);  // 4 epilogue warps
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tmem_slot)),
            "r"(2 * kBufCols)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const bool skip = s_abort != 0;

    if (!skip && warp == 0) {
        if (lane == 0) {  // producer: the K slices of this CTA's tiles, back to back
            int it = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
                int I, J;
                tri_tile_grouped<16>(t, nt, I, J);
                bool ok = true;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % kStages;
                    if (it >= kStages &&
                        !mbar_wait(smem_u32(&empty[s]), ((it / kStages) & 1) ^ 1, deadline)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full[s]);
                    uint8_t *st = smem + s * kStageBytes;
                    mbar_expect_tx(fb, kStageBytes);
                    tma_load_2d(smem_u32(st), &map_hi, kb * kElems, I * kTile, fb);
                    tma_load_2d(smem_u32(st + kOpBytes), &map_lo, kb * kElems, I * kTile, fb);
                    tma_load_2d(smem_u32(st + 2 * kOpBytes), &map_hi, kb * kElems, J * kTile, fb);
                    tma_load_2d(smem_u32(st + 3 * kOpBytes), &map_lo, kb * kElems, J * kTile, fb);
                }
                if (!ok || *(volatile int *)&s_abort) break;
            }
        }
    } else if (!skip && warp == 1) {
        if (lane == 0) {  // MMA issuer: tile lt into accumulator buffer lt & 1
            int it = 0, lt = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
                const int buf = lt & 1;
                if (lt >= 2 &&
                    !mbar_wait(smem_u32(&tempty[buf]), ((lt >> 1) & 1) ^ 1, deadline)) {
                    give_up();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t accb = tmem + (uint32_t)(buf * kBufCols);
                bool ok = true;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % kStages;
                    if (!mbar_wait(smem_u32(&full[s]), (it / kStages) & 1, deadline)) {
                        give_up();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = smem_u32(smem + s * kStageBytes);
                    const uint32_t acc = accb + (uint32_t)((kb % kAcc) * kTile);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ah = sw128_desc(st + kk * 32);
                        const uint64_t al = sw128_desc(st + kOpBytes + kk * 32);
                        const uint64_t bh = sw128_desc(st + 2 * kOpBytes + kk * 32);
                        const uint64_t bl = sw128_desc(st + 3 * kOpBytes + kk * 32);
                        mma_issue<kTf32>(acc, ah, bh, kIdesc, (kb >= kAcc || kk != 0) ? 1u : 0u);
                        mma_issue<kTf32>(acc, ah, bl, kIdesc, 1u);
                        mma_issue<kTf32>(acc, al, bh, kIdesc, 1u);
                    }
                    mma_commit(smem_u32(&empty[s]));
                }
                if (!ok || *(volatile int *)&s_abort) break;
                mma_commit(smem_u32(&tfull[buf]));  // completes once the tile's MMAs have
            }
        }
    } else if (!skip) {
        // epilogue warps 2..5: warp w reads TMEM lanes 32*(w % 4) .. +31 (its
        // rows of the tile); row stores as 16-byte vectors where aligned, the
        // transpose with consecutive lanes on consecutive addresses
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const int nacc = kblocks < kAcc ? kblocks : kAcc;
        int lt = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++lt) {
            const int buf = lt & 1;
            bool ok = mbar_wait(smem_u32(&tfull[buf]), (lt >> 1) & 1, deadline);
            ok = __all_sync(0xffffffffu, ok && !*(volatile int *)&s_abort);
            if (!ok) {
                if (lane == 0 && !*(volatile int *)&s_abort) give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int I, J;
            tri_tile_grouped<16>(t, nt, I, J);
            const int gi = I * kTile + r;
            const uint32_t accb =
                tmem + (uint32_t)(buf * kBufCols) + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
            for (int c0 = 0; c0 < kTile; c0 += 16) {
                float sum[16];
#pragma unroll 1
                for (int a = 0; a < nacc; ++a) {
                    uint32_t v[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
                        "%8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
                          "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
                          "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                          "=r"(v[15])
                        : "r"(accb + (uint32_t)(a * kTile + c0)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        sum[u] = a ? __fadd_rn(sum[u], __uint_as_float(v[u]))
                                   : __uint_as_float(v[u]);
                }
                const int gj0 = J * kTile + c0;
                if (gi < n) {
                    if (I != J && vec && gj0 + 16 <= n) {
                        float4 *dst = reinterpret_cast<float4 *>(S + (long long)gi * ld + gj0);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            dst[u] = make_float4(sum[4 * u], sum[4 * u + 1], sum[4 * u + 2],
                                                 sum[4 * u + 3]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int gj = gj0 + u;
                            if (gj < n && gj >= gi)
                                S[(long long)gi * ld + gj] = gi == gj ? 1.0f : sum[u];
                        }
                    }
                    // the transpose: S[gj, gi] for gj > gi (lanes write neighbours)
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int gj = gj0 + u;
                        if (gj < n && gj > gi) S[(long long)gj * ld + gi] = sum[u];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * kBufCols)
                     : "memory");
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// 2-D map over rows of `ldy` elements (n rows), box = one 128-byte K slice
// of 128 rows, 128-byte swizzle; rows past n read as zero.
int make_map(CUtensorMap *m, void *base, int n, long long ldy, bool tf32)
{
    EncodeTiled enc = encoder();
    if (!enc) return TMFG_ECUDA;
    const int esz = tf32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)ldy, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(ldy * esz)};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)kTile};
    cuuint32_t estr[2] = {1, 1};
    // TF32 operands are stored already rounded (low 13 bits zero): plain
    // 32-bit copies
    const CUresult r = enc(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace

// Columns of the normalised series (a multiple of one 128-byte K slice).
long long sim_ldy(int T, int prec)
{
    const int per = prec == TMFG_SIM_F64 ? 16 : (prec == TMFG_SIM_BF16X3 ? 64 : 32);
    return ((long long)T + per - 1) / per * per;
}

size_t sim_work_bytes(int n, int T, int prec)
{
    const long long ldy = sim_ldy(T, prec);
    const size_t esz = prec == TMFG_SIM_F64 ? 8 : (prec == TMFG_SIM_BF16X3 ? 2 : 4);
    const size_t one = (((size_t)n * ldy * esz) + 1023) & ~size_t(1023);
    return (prec == TMFG_SIM_BF16X3 || prec == TMFG_SIM_TF32X3) ? 2 * one : one;
}

int launch_similarity(const float *X, int n, int T, long long ldx, int prec, float *S, long long ld,
                      void *work, int *status, unsigned long long timeout_ns, cudaStream_t stream)
{
    const long long ldy = sim_ldy(T, prec);
    const size_t esz = prec == TMFG_SIM_F64 ? 8 : (prec == TMFG_SIM_BF16X3 ? 2 : 4);
    const size_t one = (((size_t)n * ldy * esz) + 1023) & ~size_t(1023);
    void *hi = work;
    void *lo = static_cast<char *>(work) + one;
    switch (prec) {
        case TMFG_SIM_F64:
            sim_prep_kernel<TMFG_SIM_F64><<<n, 256, 0, stream>>>(X, n, T, ldx, hi, nullptr, ldy, status);
            break;
        case TMFG_SIM_F32:
            sim_prep_kernel<TMFG_SIM_F32><<<n, 256, 0, stream>>>(X, n, T, ldx, hi, nullptr, ldy, status);
            break;
        case TMFG_SIM_BF16X3:
            sim_prep_kernel<TMFG_SIM_BF16X3><<<n, 256, 0, stream>>>(X, n, T, ldx, hi, lo, ldy, status);
            break;
        default:
            sim_prep_kernel<TMFG_SIM_TF32X3><<<n, 256, 0, stream>>>(X, n, T, ldx, hi, lo, ldy, status);
            break;
    }
    if (prec == TMFG_SIM_F64 || prec == TMFG_SIM_F32) {
        const int nt = (n + 63) / 64;
        const int tiles = nt * (nt + 1) / 2;
        if (prec == TMFG_SIM_F64)
            sim_simt_kernel<double><<<tiles, 256, 0, stream>>>(static_cast<const double *>(hi), n,
                                                               T, ldy, S, ld, status);
        else
            sim_simt_kernel<float><<<tiles, 256, 0, stream>>>(static_cast<const float *>(hi), n, T,
                                                              ldy, S, ld, status);
        return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
    }
    const bool tf32 = prec == TMFG_SIM_TF32X3;
    CUtensorMap mh, ml;
    int rc = make_map(&mh, hi, n, ldy, tf32);
    if (!rc) rc = make_map(&ml, lo, n, ldy, tf32);
    if (rc) return rc;
    const int nt = (n + kTile - 1) / kTile;
    const int tiles = nt * (nt + 1) / 2;
    const int kblocks = (int)(ldy / (tf32 ? 32 : 64));
    auto k = tf32 ? sim_tc_kernel<true> : sim_tc_kernel<false>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) !=
        cudaSuccess)
        return TMFG_ECUDA;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent: one CTA per SM (the pipeline's shared memory allows no
    // second one, so the whole tensor memory is this CTA's)
    const int grid = tiles < sms ? tiles : sms;
    const bool vec = (ld % 4 == 0) && (reinterpret_cast<uintptr_t>(S) % 16 == 0);
    k<<<grid, kTcThreads, kTcSmem, stream>>>(mh, ml, n, kblocks, tiles, S, ld, vec, status,
                                             timeout_ns);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace tmfg
