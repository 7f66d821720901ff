// rowsort.cu -- per-row key/index sort of S and exact row sums
// (Algorithm 1, sort loop and initial 4-clique row sums).
//
// One CTA sorts one row at a time (persistent grid, one CTA per SM):
//   * the row is read once from HBM with 16-byte loads, each entry mapped
//     to a 32-bit (float) or 64-bit (double) unsigned key whose ascending
//     order is descending similarity (-0.0 folded into +0.0);
//   * the same pass accumulates the exact row sum sum_u q(S[v,u]) in int64
//     (q = x*2^40 rounded to nearest-even, order independent) and checks that
//     every off-diagonal entry is finite with |x| <= 64;
//   * a stable LSD radix sort on 8-bit digits runs in shared memory; ranks
//     inside a warp come from eight ballots (one per digit bit: the lanes
//     holding the same digit), ranks across warps from a
//     block-wide scan of per-warp digit counts (digit-major), which keeps
//     equal keys in ascending column order: (S desc, u asc);
//   * for float rows the key shrinks by 8 bits per pass (32 -> 24 -> 16 -> 8
//     -> 0) and is packed with the 16-bit position, so the whole row needs
//     10 bytes of shared memory per entry (n up to 21581);
//   * the sorted positions are converted to vertex ids (skipping the
//     diagonal) and written with 16-byte stores, rows padded to ldi with
//     0xFFFF.
#include <type_traits>

#include "internal.cuh"

namespace tmfg {

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kHistBytes = kSortWarps * 256 * 4;
constexpr int kSortSmemMax = 232448;  // 227 KB opt-in shared memory per CTA

__host__ __device__ constexpr int sort_smem_f32(int m) { return kHistBytes + 256 + 10 * m + 64; }
__host__ __device__ constexpr int sort_smem_f64(int m) { return kHistBytes + 256 + 20 * m + 64; }

// Block-wide exclusive scan of the per-warp digit counts, digit-major
// (digit d of warp w gets sum of all counts with smaller digit, plus the
// counts of digit d in warps before w).  hist[w*256 + d] is replaced by
// that offset.
__device__ __forceinline__ void scan_hist(uint32_t *hist, uint32_t *wsum)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // thread t owns digit d = t>>1 and warps [8*(t&1), 8*(t&1)+8)
    const int d = t >> 1, w0 = (t & 1) * (kSortWarps / 2);
    uint32_t v[kSortWarps / 2];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kSortWarps / 2; ++i) {
        v[i] = hist[(w0 + i) * 256 + d];
        s += v[i];
    }
    // inclusive warp scan of s
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t ws = lane < kSortWarps ? wsum[lane] : 0;
        uint32_t z = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < kSortWarps) wsum[lane] = z - ws;  // exclusive
    }
    __syncthreads();
    uint32_t run = wsum[warp] + x - s;
#pragma unroll
    for (int i = 0; i < kSortWarps / 2; ++i) {
        hist[(w0 + i) * 256 + d] = run;
        run += v[i];
    }
    __syncthreads();
}

// One stable counting pass over m entries held warp-striped: warp w owns
// positions [w*32*I, (w+1)*32*I), lane l position base + j*32 + l.
// digit_of(p) gives the 8-bit digit of the entry at position p; emit(p, q)
// moves it to position q of the destination buffer.
template <int I, class DigitOf, class Emit>
__device__ __forceinline__ void radix_pass(int m, uint32_t *hist, uint32_t *wsum,
                                           DigitOf digit_of, Emit emit)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *h = hist + warp * 256;
#pragma unroll
    for (int i = 0; i < 8; ++i) h[lane + 32 * i] = 0;
    __syncwarp();
    const int base = warp * 32 * I;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t rank[I];
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int p = base + j * 32 + lane;
        const bool valid = p < m;
        const uint32_t d = valid ? digit_of(p) : 0u;
        // lanes with the same digit: one ballot per digit bit
        unsigned peers = __ballot_sync(0xffffffffu, valid);
        peers = valid ? peers : (1u << lane);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned mb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? mb : ~mb;
        }
        uint32_t before = valid ? h[d] : 0u;
        rank[j] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) h[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    scan_hist(hist, wsum);
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const int p = base + j * 32 + lane;
        if (p < m) emit(p, h[digit_of(p)] + rank[j]);
    }
    __syncthreads();
}

// Sum an int64 over the block; result valid in thread 0.
__device__ __forceinline__ long long block_sum_ll(long long x, long long *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp] = x;
    __syncthreads();
    long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kSortWarps; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Write the sorted row: positions -> vertex ids (skip the diagonal), pad
// to ldi with 0xFFFF.
__device__ __forceinline__ void store_row(const uint16_t *pos, int m, int v, uint16_t *out,
                                          long long ldi, bool vec)
{
    if (vec) {
        const int chunks = (int)(ldi / 8);
        for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
            uint16_t e[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = c * 8 + k;
                if (j < m) {
                    const int p = pos[j];
                    e[k] = (uint16_t)(p + (p >= v));
                } else {
                    e[k] = kNone16;
                }
            }
            uint4 q;
            q.x = e[0] | ((uint32_t)e[1] << 16);
            q.y = e[2] | ((uint32_t)e[3] << 16);
            q.z = e[4] | ((uint32_t)e[5] << 16);
            q.w = e[6] | ((uint32_t)e[7] << 16);
            reinterpret_cast<uint4 *>(out)[c] = q;
        }
    } else {
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const int p = pos[j];
            out[j] = (uint16_t)(p + (p >= v));
        }
    }
}

// ------------------------------------------------------- 32-bit key radix
// Stable sort of m 32-bit keys (key0, at smem + kHistBytes + 256) in four
// 8-bit passes; the key shrinks by a byte per pass and is packed with the
// 16-bit position, so the buffers take 10 bytes per entry.  Leaves the sorted
// positions in out16 (the start of the same region).
template <int I>
__device__ __forceinline__ void radix_key32(int m, unsigned char *smem)
{
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    uint32_t *wsum = reinterpret_cast<uint32_t *>(smem + kHistBytes);
    unsigned char *r1 = smem + kHistBytes + 256;  // 4m bytes: KEY0, then P2, then OUT16
    const int r1_bytes = ((4 * m + 15) / 16) * 16;
    unsigned char *r2 = r1 + r1_bytes;            // 6m bytes: P1 (key24 + pos), then P3
    uint32_t *key0 = reinterpret_cast<uint32_t *>(r1);
    uint32_t *p2 = reinterpret_cast<uint32_t *>(r1);
    uint16_t *out16 = reinterpret_cast<uint16_t *>(r1);
    uint32_t *p1k = reinterpret_cast<uint32_t *>(r2);
    uint16_t *p1v = reinterpret_cast<uint16_t *>(r2 + 4 * (size_t)m);
    uint32_t *p3 = reinterpret_cast<uint32_t *>(r2);
    radix_pass<I>(m, hist, wsum,
        [&](int p) { return key0[p] & 0xFFu; },
        [&](int p, uint32_t q) { p1k[q] = key0[p] >> 8; p1v[q] = (uint16_t)p; });
    radix_pass<I>(m, hist, wsum,
        [&](int p) { return p1k[p] & 0xFFu; },
        [&](int p, uint32_t q) { p2[q] = ((p1k[p] >> 8) << 16) | p1v[p]; });
    radix_pass<I>(m, hist, wsum,
        [&](int p) { return (p2[p] >> 16) & 0xFFu; },
        [&](int p, uint32_t q) { p3[q] = ((p2[p] >> 24) << 16) | (p2[p] & 0xFFFFu); });
    radix_pass<I>(m, hist, wsum,
        [&](int p) { return p3[p] >> 16; },
        [&](int p, uint32_t q) { out16[q] = (uint16_t)(p3[p] & 0xFFFFu); });
}

// ------------------------------------------------------- 64-bit key radix
// Stable sort of m 64-bit keys (k0 at smem + kHistBytes + 256, then k1, v0,
// v1: 20 bytes per entry) in eight 8-bit passes; leaves the sorted positions
// in v0 (returned).
template <int I>
__device__ __forceinline__ uint16_t *radix_key64(int m, unsigned char *smem)
{
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    uint32_t *wsum = reinterpret_cast<uint32_t *>(smem + kHistBytes);
    unsigned char *base = smem + kHistBytes + 256;
    uint64_t *k0 = reinterpret_cast<uint64_t *>(base);
    uint64_t *k1 = k0 + m;
    uint16_t *v0 = reinterpret_cast<uint16_t *>(k1 + m);
    uint16_t *v1 = v0 + m;
    // pass 0: positions are implicit
    radix_pass<I>(m, hist, wsum,
        [&](int p) { return (uint32_t)(k0[p] & 0xFFu); },
        [&](int p, uint32_t q) { k1[q] = k0[p]; v1[q] = (uint16_t)p; });
#pragma unroll 1
    for (int pass = 1; pass < 8; ++pass) {
        const int sh = 8 * pass;
        uint64_t *ks = (pass & 1) ? k1 : k0;
        uint64_t *kd = (pass & 1) ? k0 : k1;
        uint16_t *vs = (pass & 1) ? v1 : v0;
        uint16_t *vd = (pass & 1) ? v0 : v1;
        radix_pass<I>(m, hist, wsum,
            [&](int p) { return (uint32_t)((ks[p] >> sh) & 0xFFu); },
            [&](int p, uint32_t q) { kd[q] = ks[p]; vd[q] = vs[p]; });
    }
    return v0;  // after 8 passes the result is in (k0, v0)
}

// ---------------------------------------------------------------- float rows
// Sort row v of an n x n float matrix (row = S + v*ld) into out (ldi ids).
template <int I>
__device__ __forceinline__ void sort_row_f32(const float *__restrict__ row, int n, int v,
                                             bool vec_in, uint16_t *__restrict__ out,
                                             long long ldi, bool vec_out, long long *rowsum_v,
                                             int *status, unsigned char *smem)
{
    const int m = n - 1;
    long long *red = reinterpret_cast<long long *>(smem + kHistBytes + 64);
    uint32_t *key0 = reinterpret_cast<uint32_t *>(smem + kHistBytes + 256);
    const uint16_t *out16 = reinterpret_cast<const uint16_t *>(smem + kHistBytes + 256);

    long long acc = 0;
    int bad = 0;
    auto take = [&](int u, float x) {
        if (u == v) return;
        x = canon(x);
        int c = check_entry(x);
        if (c) bad = c;
        acc += quantize40(x);
        key0[u - (u > v)] = ~ord_key(x);  // ascending key = descending S
    };
    if (vec_in) {
        const int n4 = n >> 2;
        const float4 *row4 = reinterpret_cast<const float4 *>(row);
        for (int q = threadIdx.x; q < n4; q += blockDim.x) {
            float4 x = __ldcs(row4 + q);
            take(4 * q, x.x);
            take(4 * q + 1, x.y);
            take(4 * q + 2, x.z);
            take(4 * q + 3, x.w);
        }
        for (int u = 4 * n4 + threadIdx.x; u < n; u += blockDim.x) take(u, row[u]);
    } else {
        for (int u = threadIdx.x; u < n; u += blockDim.x) take(u, row[u]);
    }
    if (bad) set_status(status, bad);
    __syncthreads();
    const long long rs = block_sum_ll(acc, red);
    if (threadIdx.x == 0 && rowsum_v) *rowsum_v = rs;

    radix_key32<I>(m, smem);
    store_row(out16, m, v, out, ldi, vec_out);
    __syncthreads();
}

// --------------------------------------------------------------- double rows
template <int I>
__device__ __forceinline__ void sort_row_f64(const double *__restrict__ row, int n, int v,
                                             bool vec_in, uint16_t *__restrict__ out,
                                             long long ldi, bool vec_out, long long *rowsum_v,
                                             int *status, unsigned char *smem)
{
    const int m = n - 1;
    long long *red = reinterpret_cast<long long *>(smem + kHistBytes + 64);
    uint64_t *k0 = reinterpret_cast<uint64_t *>(smem + kHistBytes + 256);

    long long acc = 0;
    int bad = 0;
    auto take = [&](int u, double x) {
        if (u == v) return;
        x = canon(x);
        int c = check_entry(x);
        if (c) bad = c;
        acc += quantize40(x);
        k0[u - (u > v)] = ~ord_key(x);
    };
    if (vec_in) {
        const int n2 = n >> 1;
        const double2 *row2 = reinterpret_cast<const double2 *>(row);
        for (int q = threadIdx.x; q < n2; q += blockDim.x) {
            double2 x = __ldcs(row2 + q);
            take(2 * q, x.x);
            take(2 * q + 1, x.y);
        }
        for (int u = 2 * n2 + threadIdx.x; u < n; u += blockDim.x) take(u, row[u]);
    } else {
        for (int u = threadIdx.x; u < n; u += blockDim.x) take(u, row[u]);
    }
    if (bad) set_status(status, bad);
    __syncthreads();
    const long long rs = block_sum_ll(acc, red);
    if (threadIdx.x == 0 && rowsum_v) *rowsum_v = rs;

    const uint16_t *sorted = radix_key64<I>(m, smem);
    store_row(sorted, m, v, out, ldi, vec_out && ((uintptr_t)sorted % 16 == 0));
    __syncthreads();
}

template <int I, typename T>
__device__ __forceinline__ void sort_row(const T *row, int n, int v, bool vec_in, uint16_t *out,
                                         long long ldi, bool vec_out, long long *rowsum_v,
                                         int *status, unsigned char *smem)
{
    if constexpr (sizeof(T) == 4)
        sort_row_f32<I>(row, n, v, vec_in, out, ldi, vec_out, rowsum_v, status, smem);
    else
        sort_row_f64<I>(row, n, v, vec_in, out, ldi, vec_out, rowsum_v, status, smem);
}

// ------------------------------------------------------------ long rows
// A row longer than one CTA's shared memory sorts in three steps: the
// positions [0, h) and [h, m) (h = ceil(m / 2)) are each sorted as above
// and their ids written to the output row; then the whole row is read again
// (with the exact sum and the entry checks), its keys kept in shared memory
// by position, and the two sorted halves are merged by merge path.  Every
// id of the first half is smaller than every id of the second, so taking
// the first half's entry on equal keys keeps the (S desc, u asc) order.

template <typename T>
using key_of_t = std::conditional_t<sizeof(T) == 4, uint32_t, uint64_t>;

// Sort positions [p0, p0 + cnt) of row v by key (ties in position order);
// ids to out[p0 + j].
template <int I, typename T>
__device__ __forceinline__ void sort_part(const T *__restrict__ row, int v, int p0, int cnt,
                                          uint16_t *__restrict__ out, unsigned char *smem)
{
    using K = key_of_t<T>;
    K *key0 = reinterpret_cast<K *>(smem + kHistBytes + 256);
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int p = p0 + j;
        const int u = p + (p >= v);
        key0[j] = ~ord_key(canon(row[u]));
    }
    __syncthreads();
    const uint16_t *sorted;
    if constexpr (sizeof(T) == 4) {
        radix_key32<I>(cnt, smem);
        sorted = reinterpret_cast<const uint16_t *>(smem + kHistBytes + 256);
    } else {
        sorted = radix_key64<I>(cnt, smem);
    }
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
        const int p = p0 + sorted[j];
        out[p0 + j] = (uint16_t)(p + (p >= v));
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void merge_halves(const T *__restrict__ row, int n, int v,
                                             uint16_t *__restrict__ out, long long ldi,
                                             long long *rowsum_v, int *status,
                                             unsigned char *smem)
{
    using K = key_of_t<T>;
    const int m = n - 1, na = (m + 1) / 2, nb = m - na;
    long long *red = reinterpret_cast<long long *>(smem + kHistBytes + 64);
    K *key = reinterpret_cast<K *>(smem + kHistBytes + 256);
    uint16_t *ids = reinterpret_cast<uint16_t *>(key + m);
    long long acc = 0;
    int bad = 0;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        if (u == v) continue;
        const T x = canon(row[u]);
        const int c = check_entry(x);
        if (c) bad = c;
        acc += quantize40(x);
        key[u - (u > v)] = ~ord_key(x);
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) ids[j] = out[j];
    if (bad) set_status(status, bad);
    __syncthreads();
    const long long rs = block_sum_ll(acc, red);
    if (threadIdx.x == 0 && rowsum_v) *rowsum_v = rs;
    const uint16_t *A = ids, *B = ids + na;
    auto kof = [&](int id) { return key[id - (id > v)]; };
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int d0 = threadIdx.x * per;
    if (d0 < m) {
        const int d1 = d0 + per < m ? d0 + per : m;
        // merge path: i = the number of first-half entries among the first d0
        int lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (kof(A[mid]) <= kof(B[d0 - mid - 1])) lo = mid + 1;
            else hi = mid;
        }
        int i = lo, j = d0 - lo;
        for (int d = d0; d < d1; ++d) {
            const bool takeA = j >= nb || (i < na && kof(A[i]) <= kof(B[j]));
            out[d] = takeA ? A[i++] : B[j++];
        }
    }
    for (int j = m + threadIdx.x; j < ldi; j += blockDim.x) out[j] = kNone16;
    __syncthreads();
}

template <int I, typename T>
__global__ void __launch_bounds__(kSortThreads, 1)
rowsort_long_kernel(const T *__restrict__ S, int n, long long ld, uint16_t *__restrict__ idx,
                    long long ldi, long long *__restrict__ rowsum, int *status, int row0,
                    int row1)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int m = n - 1, na = (m + 1) / 2;
    for (int v = row0 + blockIdx.x; v < row1; v += gridDim.x) {
        const T *row = S + (long long)v * ld;
        uint16_t *out = idx + (long long)v * ldi;
        sort_part<I, T>(row, v, 0, na, out, smem);
        sort_part<I, T>(row, v, na, m - na, out, smem);
        merge_halves<T>(row, n, v, out, ldi, rowsum ? rowsum + v : nullptr, status, smem);
    }
}

// One matrix: a persistent grid walks its rows.
template <int I, typename T>
__global__ void __launch_bounds__(kSortThreads, 1)
rowsort_kernel(const T *__restrict__ S, int n, long long ld, bool vec_in, uint16_t *__restrict__ idx,
               long long ldi, bool vec_out, long long *__restrict__ rowsum, int *status, int row0,
               int row1)
{
    extern __shared__ __align__(16) unsigned char smem[];
    for (int v = row0 + blockIdx.x; v < row1; v += gridDim.x)
        sort_row<I, T>(S + (long long)v * ld, n, v, vec_in, idx + (long long)v * ldi, ldi, vec_out,
                       rowsum ? rowsum + v : nullptr, status, smem);
}

// Many matrices: a persistent grid walks the rows of all jobs (row r of the
// launch is row r - row_begin[j] of job j).
template <int I, typename T>
__global__ void __launch_bounds__(kSortThreads, 1)
rowsort_batch_kernel(const SortJob *__restrict__ jobs, const int *__restrict__ row_begin, int njobs,
                     int *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int total = row_begin[njobs];
    for (int r = blockIdx.x; r < total; r += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_begin[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const SortJob &J = jobs[lo];
        const int v = r - row_begin[lo];
        const T *S = static_cast<const T *>(J.S);
        sort_row<I, T>(S + (long long)v * J.ld, J.n, v, J.vec_in, J.idx + (long long)v * J.ldi,
                       J.ldi, J.vec_out, J.rowsum ? J.rowsum + v : nullptr, status, smem);
    }
}

// ------------------------------------------------------------------- launch
static const int kItemsF32[] = {1, 2, 4, 8, 16, 24, 32, 43};
static const int kItemsF64[] = {1, 2, 4, 8, 16, 22};

static int pick_items(int m, int dtype)
{
    const int *c = dtype == TMFG_F32 ? kItemsF32 : kItemsF64;
    const int nc = dtype == TMFG_F32 ? 8 : 6;
    for (int i = 0; i < nc; ++i)
        if ((long long)c[i] * kSortThreads >= m) return c[i];
    return -1;
}

// Shared memory of the one-pass sort of a row of n, and of the long-row
// sort (two halves, then the merge).
size_t rowsort_smem(int n, int dtype)
{
    return dtype == TMFG_F32 ? (size_t)sort_smem_f32(n - 1) : (size_t)sort_smem_f64(n - 1);
}

static size_t rowsort_long_smem(int n, int dtype)
{
    const size_t m = (size_t)n - 1, na = (m + 1) / 2;
    const size_t part = dtype == TMFG_F32 ? ((4 * na + 15) / 16) * 16 + 6 * na : 20 * na;
    const size_t merge = dtype == TMFG_F32 ? 6 * m : 10 * m;
    return kHistBytes + 256 + (part > merge ? part : merge) + 64;
}

static bool rowsort_fits(int n, int dtype)
{
    return pick_items(n - 1, dtype) > 0 && rowsort_smem(n, dtype) <= (size_t)kSortSmemMax;
}

static bool rowsort_long_fits(int n, int dtype)
{
    return pick_items(n / 2, dtype) > 0 && rowsort_long_smem(n, dtype) <= (size_t)kSortSmemMax;
}

int64_t rowsort_max_n(int dtype)
{
    // the largest n that one of the two paths sorts (ids are 16 bits)
    int n = 65535;
    while (n > 2 && !rowsort_fits(n, dtype) && !rowsort_long_fits(n, dtype)) --n;
    return n;
}

// Launch one kernel instance K<I, T> for the items count I (a switch over
// the instantiated values).
template <typename T, class F>
static int dispatch_items(int I, F &&f)
{
    switch (I) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        case 16: return f(std::integral_constant<int, 16>{});
        case 22:
            if constexpr (sizeof(T) == 8) return f(std::integral_constant<int, 22>{});
            return TMFG_EINTERNAL;
        case 24:
            if constexpr (sizeof(T) == 4) return f(std::integral_constant<int, 24>{});
            return TMFG_EINTERNAL;
        case 32:
            if constexpr (sizeof(T) == 4) return f(std::integral_constant<int, 32>{});
            return TMFG_EINTERNAL;
        case 43:
            if constexpr (sizeof(T) == 4) return f(std::integral_constant<int, 43>{});
            return TMFG_EINTERNAL;
        default: return TMFG_EINTERNAL;
    }
}

template <typename T>
static int launch_rowsort_t(const void *S, int n, long long ld, uint16_t *idx, long long ldi,
                            long long *rowsum, int *status, int num_sms, int row0, int row1,
                            cudaStream_t stream)
{
    const int dtype = sizeof(T) == 4 ? TMFG_F32 : TMFG_F64;
    const int rows = row1 - row0;
    if (rows <= 0) return TMFG_OK;
    const int grid = rows < num_sms ? rows : num_sms;
    if (!rowsort_fits(n, dtype)) {
        if (!rowsort_long_fits(n, dtype)) return TMFG_ETOOBIG;
        const size_t smem = rowsort_long_smem(n, dtype);
        return dispatch_items<T>(pick_items((n - 1 + 1) / 2, dtype), [&](auto ic) {
            constexpr int II = decltype(ic)::value;
            auto k = rowsort_long_kernel<II, T>;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return (int)TMFG_ECUDA;
            k<<<grid, kSortThreads, smem, stream>>>(static_cast<const T *>(S), n, ld, idx, ldi,
                                                     rowsum, status, row0, row1);
            return cudaGetLastError() == cudaSuccess ? (int)TMFG_OK : (int)TMFG_ECUDA;
        });
    }
    const int I = pick_items(n - 1, dtype);
    const size_t smem = rowsort_smem(n, dtype);
    const bool vec_out = (ldi % 8 == 0) && ((uintptr_t)idx % 16 == 0);
    const bool vec_in = (ld % (16 / sizeof(T)) == 0) && ((uintptr_t)S % 16 == 0);
    return dispatch_items<T>(I, [&](auto ic) {
        constexpr int II = decltype(ic)::value;
        auto k = rowsort_kernel<II, T>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return (int)TMFG_ECUDA;
        k<<<grid, kSortThreads, smem, stream>>>(static_cast<const T *>(S), n, ld, vec_in, idx, ldi,
                                                 vec_out, rowsum, status, row0, row1);
        return cudaGetLastError() == cudaSuccess ? (int)TMFG_OK : (int)TMFG_ECUDA;
    });
}

int launch_rowsort(const void *S, int n, long long ld, int dtype, uint16_t *idx, long long ldi,
                   long long *rowsum, int *status, int num_sms, cudaStream_t stream, int row0,
                   int row1)
{
    if (row1 < 0) row1 = n;
    if (dtype == TMFG_F32)
        return launch_rowsort_t<float>(S, n, ld, idx, ldi, rowsum, status, num_sms, row0, row1,
                                       stream);
    return launch_rowsort_t<double>(S, n, ld, idx, ldi, rowsum, status, num_sms, row0, row1,
                                    stream);
}

int launch_rowsort_batch(const SortJob *d_jobs, const int *d_row_begin, int njobs, int max_n,
                         int dtype, int *status, int grid, cudaStream_t stream)
{
    // the batched sort keeps every row in one pass (the serving sizes)
    if (!rowsort_fits(max_n, dtype)) return TMFG_ETOOBIG;
    const int I = pick_items(max_n - 1, dtype);
    const size_t smem = rowsort_smem(max_n, dtype);
    auto go = [&](auto tag) {
        using T = decltype(tag);
        return dispatch_items<T>(I, [&](auto ic) {
            constexpr int II = decltype(ic)::value;
            auto k = rowsort_batch_kernel<II, T>;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return (int)TMFG_ECUDA;
            k<<<grid, kSortThreads, smem, stream>>>(d_jobs, d_row_begin, njobs, status);
            return cudaGetLastError() == cudaSuccess ? (int)TMFG_OK : (int)TMFG_ECUDA;
        });
    };
    return dtype == TMFG_F32 ? go(float{}) : go(double{});
}

}  // namespace tmfg
