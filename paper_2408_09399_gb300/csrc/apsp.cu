// apsp.cu -- all-pairs shortest paths over the TMFG (Section 2: APSP by one
// single-source search per vertex; Section 4.3: hub-based approximation).
//
// Distances are float: the length of edge (a,b) is
// sqrt(max(0, 2(1 - S[a,b]))) rounded to float, and the distance from s to t
// is the least left-to-right float sum of the lengths along a path.  Both the
// exact and the approximate forms compute that quantity exactly for the
// pairs they search, so they agree bit for bit with a float Dijkstra.
//
// Kernels:
//   csr_*           degree count, exclusive scan, arc fill (col, len) packed
//                   into 8 bytes; 6n-12 arcs, L2-resident;
//   sssp_kernel     one CTA per source (persistent grid, one CTA per SM):
//                   dist[] in shared memory, frontier bitmaps, Bellman-Ford
//                   rounds where 8-lane groups relax the arcs of one frontier
//                   vertex with shared-memory atomicMin on the float bits;
//                   writes the finished row with 16-byte stores.  A bounded
//                   variant does not expand vertices beyond the radius r_s
//                   and writes the approximate row instead;
//   hub_select      top-h degrees (ties to the smaller id) by a degree
//                   histogram in one CTA;
//   nearest_hub     per vertex, the closest hub (ties to the lower rank);
//   sym_min         D = min(R, R^T) tile by tile (32x32), in place.
#include <cfloat>
#include <mutex>

#include "internal.cuh"

namespace tmfg {

constexpr int kSsspThreads = 512;  // default CTA size of the SSSP kernels

// ------------------------------------------------------------------ CSR
__global__ void csr_degree_kernel(const int *__restrict__ edges, int ne, int n, int *deg,
                                  int *status)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) {
            set_status(status, TMFG_EINVAL);
            continue;
        }
        atomicAdd(&deg[a], 1);
        atomicAdd(&deg[b], 1);
    }
}

// rowptr[0] = 0, rowptr[v+1] = sum of deg[0..v]; one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) csr_scan_kernel(const int *__restrict__ deg, int n,
                                                        int *rowptr, int *cursor)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n + 1023) / 1024;
    const int lo = t * per, hi = min(n, lo + per);
    int s = 0;
    for (int v = lo; v < hi; ++v) s += deg[v];
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z - w;
    }
    __syncthreads();
    int run = wsum[warp] + x - s;
    if (t == 0) rowptr[0] = 0;
    for (int v = lo; v < hi; ++v) {
        cursor[v] = run;
        run += deg[v];
        rowptr[v + 1] = run;
    }
}

template <typename T>
__device__ __forceinline__ float edge_length(T s);

template <>
__device__ __forceinline__ float edge_length<float>(float s)
{
    const float t = __fmul_rn(2.0f, __fsub_rn(1.0f, s));
    return __fsqrt_rn(fmaxf(t, 0.0f));
}

template <>
__device__ __forceinline__ float edge_length<double>(double s)
{
    const double t = __dmul_rn(2.0, __dsub_rn(1.0, s));
    return __double2float_rn(__dsqrt_rn(fmax(t, 0.0)));
}

template <typename T>
__global__ void csr_fill_kernel(const int *__restrict__ edges, int ne, int n,
                                const T *__restrict__ S, long long ld, int *cursor,
                                uint2 *__restrict__ arcs)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) continue;
        const float l = edge_length<T>(canon(S[(long long)a * ld + b]));
        const int pa = atomicAdd(&cursor[a], 1);
        const int pb = atomicAdd(&cursor[b], 1);
        arcs[pa] = make_uint2((unsigned)b, __float_as_uint(l));
        arcs[pb] = make_uint2((unsigned)a, __float_as_uint(l));
    }
}

// ----------------------------------------------------------------- SSSP

// Shared memory: dist[n] floats, two frontier bitmaps, a frontier list of at
// most list_cap ids, and a list of high-degree frontier vertices with their
// arc ranges.  The list holds at least 32 entries, so that any one bitmap
// word fits an empty window, and at most 8192.
__host__ __device__ inline int sssp_list_cap(int n)
{
    const int c = (((n / 2) > 32 ? (n / 2) : 32) + 15) & ~15;
    return c < 8192 ? c : 8192;
}
constexpr int kHeavyCap = 512;
constexpr int kHeavyDeg = 16;

// Single-source search for source index i of a (row i of a.out).  Returns
// false when the run must stop (an earlier error or the time limit).
template <bool kBounded, int NT>
__device__ __forceinline__ bool sssp_source(const SsspArgs &a, int i, uint64_t t0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cnt, s_listed, s_hcnt, s_abort, s_wnext;
    const int n = a.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = (n + 31) / 32;
    const int cap = sssp_list_cap(n);
    float *dist = reinterpret_cast<float *>(smem);
    uint32_t *bm0 = reinterpret_cast<uint32_t *>(smem + ((4 * (size_t)n + 15) & ~size_t(15)));
    uint32_t *bm1 = bm0 + W;
    int2 *hrange = reinterpret_cast<int2 *>(bm0 + 2 * W);  // 8-byte aligned
    uint16_t *list = reinterpret_cast<uint16_t *>(hrange + kHeavyCap);
    uint16_t *heavy = list + cap;
    {
        if (tid == 0) s_abort = (*(volatile int *)a.status != 0) ||
                                (globaltimer_ns() - t0 > a.timeout_ns);
        const int s = a.src ? a.src[i] : a.src0 + i;
        for (int v = tid; v < n; v += NT) dist[v] = __int_as_float(0x7f800000);
        for (int w = tid; w < W; w += NT) { bm0[w] = 0; bm1[w] = 0; }
        __syncthreads();
        if (s_abort) {
            if (tid == 0 && *(volatile int *)a.status == 0) set_status(a.status, TMFG_ETIMEOUT);
            return false;
        }
        const float r = kBounded ? __fmul_rn(a.rf, a.dnear[s]) : __int_as_float(0x7f800000);
        if (tid == 0) {
            dist[s] = 0.0f;
            bm0[s >> 5] = 1u << (s & 31);
        }
        uint32_t *cur = bm0, *nxt = bm1;
        __syncthreads();
        int rounds = 0;
        for (;;) {
            // one Bellman-Ford round over the frontier in cur, in windows of
            // at most cap frontier vertices
            int wstart = 0;
            bool any = false;
            while (wstart < W) {
                if (tid == 0) { s_cnt = 0; s_listed = 0; s_hcnt = 0; s_wnext = W; }
                __syncthreads();
                for (int w = wstart + tid; w < W; w += NT) {
                    uint32_t b = cur[w];
                    if (!b) continue;
                    const int c = __popc(b);
                    const int pos = atomicAdd(&s_cnt, c);
                    if (pos + c > cap) {  // the window is full: resume from this word
                        atomicMin(&s_wnext, w);
                        continue;
                    }
                    cur[w] = 0;
                    atomicAdd(&s_listed, c);
                    int q = pos;
                    while (b) {
                        const int bit = __ffs(b) - 1;
                        b &= b - 1;
                        list[q++] = (uint16_t)(w * 32 + bit);
                    }
                }
                __syncthreads();
                // successful reservations form the prefix [0, s_listed); a
                // word that did not fit stays set and starts the next window
                const int cnt = s_listed;
                const int wn = s_wnext;
                any |= cnt > 0;
                if (cnt == 0 && wn < W) {  // no progress is impossible; stop rather than spin
                    if (tid == 0) set_status(a.status, TMFG_EINTERNAL);
                    return false;
                }
                // relax: light vertices one per thread (two per pass, their
                // loads issued together), heavy ones a warp each
                auto relax = [&](float du, const uint2 &arc) {
                    const int w = (int)arc.x;
                    if (w < 0 || w >= n) return;
                    const float nd = __fadd_rn(du, __uint_as_float(arc.y));
                    if (nd < dist[w]) {
                        const int old = atomicMin(reinterpret_cast<int *>(&dist[w]),
                                                  __float_as_int(nd));
                        if (__float_as_int(nd) < old) atomicOr(&nxt[w >> 5], 1u << (w & 31));
                    }
                };
                for (int j = tid; j < cnt; j += 2 * NT) {
                    int us[2], q0[2], q1[2];
                    float du[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int jj = j + h * NT;
                        us[h] = jj < cnt ? list[jj] : n;
                        q0[h] = 0;
                        q1[h] = 0;
                        du[h] = 0.0f;
                        if (us[h] < n) {
                            du[h] = dist[us[h]];
                            if (!(kBounded && du[h] > r)) {
                                q0[h] = a.rowptr[us[h]];
                                q1[h] = a.rowptr[us[h] + 1];
                            }
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int p0 = q0[h], p1 = q1[h];
                        if (p1 - p0 > kHeavyDeg) {
                            const int hh = atomicAdd(&s_hcnt, 1);
                            if (hh < kHeavyCap) {
                                heavy[hh] = (uint16_t)us[h];
                                hrange[hh] = make_int2(p0, p1);
                                continue;
                            }
                        }
                        for (int p = p0; p < p1; p += 8) {
                            uint2 arc[8];
#pragma unroll
                            for (int t = 0; t < 8; ++t)
                                arc[t] = p + t < p1 ? a.arcs[p + t] : make_uint2(0xFFFFFFFFu, 0u);
#pragma unroll
                            for (int t = 0; t < 8; ++t) relax(du[h], arc[t]);
                        }
                    }
                }
                __syncthreads();
                const int hc = s_hcnt < kHeavyCap ? s_hcnt : kHeavyCap;
                for (int j = warp; j < hc; j += NT / 32) {
                    const int u = heavy[j];
                    const float du = dist[u];
                    const int2 pr = hrange[j];
                    for (int p = pr.x + lane; p < pr.y; p += 4 * 32) {
                        uint2 arc[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t)
                            arc[t] = p + 32 * t < pr.y ? a.arcs[p + 32 * t]
                                                      : make_uint2(0xFFFFFFFFu, 0u);
#pragma unroll
                        for (int t = 0; t < 4; ++t) relax(du, arc[t]);
                    }
                }
                __syncthreads();
                wstart = wn;
            }
            if (!any) break;
            uint32_t *t = cur; cur = nxt; nxt = t;
            if (++rounds > n + 1) {  // cannot happen for a finite graph
                if (tid == 0) set_status(a.status, TMFG_EINTERNAL);
                break;
            }
        }
        // write the row
        float *orow = a.out + (long long)i * a.ldo;
        const bool vec = ((a.ldo & 3) == 0) && (((uintptr_t)a.out & 15) == 0);
        if (!kBounded) {
            if (vec) {
                const int n4 = n >> 2;
                for (int q = tid; q < n4; q += NT)
                    __stcs(reinterpret_cast<float4 *>(orow) + q,
                           make_float4(dist[4 * q], dist[4 * q + 1], dist[4 * q + 2], dist[4 * q + 3]));
                for (int t = 4 * n4 + tid; t < n; t += NT) orow[t] = dist[t];
            } else {
                for (int t = tid; t < n; t += NT) orow[t] = dist[t];
            }
        } else {
            const float ds = a.dnear[s];
            const float *hrow = a.DH + (long long)a.near[s] * n;
            for (int t = tid; t < n; t += NT) {
                const float es = __fadd_rn(ds, hrow[t]);
                const float et = __fadd_rn(a.dnear[t], a.DH[(long long)a.near[t] * n + s]);
                float v = fminf(es, et);
                const float dt = dist[t];
                if (dt <= r) v = fminf(v, dt);
                orow[t] = v;
            }
        }
        __syncthreads();
    }
    return true;
}

template <bool kBounded, int NT>
__global__ void __launch_bounds__(NT, 2) sssp_kernel(SsspArgs a)
{
    const uint64_t t0 = globaltimer_ns();
    for (int i = blockIdx.x; i < a.nsrc; i += gridDim.x)
        if (!sssp_source<kBounded, NT>(a, i, t0)) return;
}

// Many graphs: source g of the launch is source g - src_begin[j] of job j.
template <int NT>
__global__ void __launch_bounds__(NT, 2) sssp_batch_kernel(const SsspArgs *__restrict__ args,
                                                           const int *__restrict__ src_begin,
                                                           int njobs)
{
    __shared__ SsspArgs s_a;
    const uint64_t t0 = globaltimer_ns();
    const int total = src_begin[njobs];
    for (int g = blockIdx.x; g < total; g += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (src_begin[mid] <= g) lo = mid; else hi = mid - 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_a = args[lo];
        __syncthreads();
        if (!sssp_source<false, NT>(s_a, g - src_begin[lo], t0)) return;
    }
}

size_t sssp_smem_bytes(int n)
{
    const size_t W = (n + 31) / 32;
    return ((4 * (size_t)n + 15) & ~size_t(15)) + 8 * W + 8 * (size_t)kHeavyCap +
           2 * (size_t)sssp_list_cap(n) + 2 * (size_t)kHeavyCap + 16;
}

// ------------------------------------------------------------- hubs
// Top-h vertices by (degree desc, id asc), in that rank order; one CTA.
// Dynamic shared memory: hist[n] (counts per degree) then sel[h].
__global__ void __launch_bounds__(1024) hub_select_kernel(const int *__restrict__ rowptr, int n,
                                                          int h, int *hubs, int *status)
{
    extern __shared__ int hist[];
    int *sel = hist + n;
    __shared__ int s_thr, s_above, s_cnt, s_cnt_eq;
    __shared__ int wc[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int d = t; d < n; d += 1024) hist[d] = 0;
    __syncthreads();
    for (int v = t; v < n; v += 1024) {
        const int d = rowptr[v + 1] - rowptr[v];
        atomicAdd(&hist[d < n ? (d >= 0 ? d : 0) : n - 1], 1);
    }
    __syncthreads();
    if (t == 0) {
        // threshold degree T: count(deg > T) < h <= count(deg >= T)
        int above = 0, T = 0;
        for (int d = n - 1; d >= 0; --d) {
            if (above + hist[d] >= h) { T = d; break; }
            above += hist[d];
        }
        s_thr = T;
        s_above = above;
        s_cnt = 0;
        s_cnt_eq = 0;
    }
    __syncthreads();
    const int T = s_thr, above = s_above, need_eq = h - above;
    // every vertex above the threshold
    for (int v = t; v < n; v += 1024) {
        const int d = rowptr[v + 1] - rowptr[v];
        if (d > T) {
            const int pos = atomicAdd(&s_cnt, 1);
            if (pos < above) sel[pos] = v;
        }
    }
    // then the smallest ids at the threshold, in id order (1024 ids a pass)
    for (int base = 0; base < n; base += 1024) {
        __syncthreads();
        if (s_cnt_eq >= need_eq) break;
        const int v = base + t;
        const int flag = (v < n) && (rowptr[v + 1] - rowptr[v] == T);
        const unsigned bal = __ballot_sync(0xffffffffu, flag);
        if (lane == 0) wc[warp] = __popc(bal);
        __syncthreads();
        int pre = 0, blk_total = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) pre += wc[w];
            blk_total += wc[w];
        }
        pre += __popc(bal & ((1u << lane) - 1u));
        const int rank = s_cnt_eq + pre;
        if (flag && rank < need_eq) sel[above + rank] = v;
        __syncthreads();
        if (t == 0) s_cnt_eq += blk_total;
    }
    __syncthreads();
    // rank sort of the h selected by (deg desc, id asc)
    for (int i = t; i < h; i += 1024) {
        const int v = sel[i];
        const int dv = rowptr[v + 1] - rowptr[v];
        int rank = 0;
        for (int j = 0; j < h; ++j) {
            const int u = sel[j];
            const int du = rowptr[u + 1] - rowptr[u];
            rank += (du > dv) || (du == dv && u < v);
        }
        hubs[rank] = v;
    }
    if (t == 0 && (s_cnt != above || s_cnt_eq < need_eq)) set_status(status, TMFG_EINTERNAL);
}

// d_s = min over hub ranks of DH[rank][s] (ties to the lower rank).
__global__ void nearest_hub_kernel(const float *__restrict__ DH, int h, int n, int *near,
                                   float *dnear)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        int bi = 0;
        float bd = DH[s];
        for (int i = 1; i < h; ++i) {
            const float d = DH[(long long)i * n + s];
            if (d < bd) { bd = d; bi = i; }
        }
        near[s] = bi;
        dnear[s] = bd;
    }
}

// ------------------------------------------------------------ sym min
// D = min(D, D^T) in place; block (32, 8) per pair of 32x32 tiles (I <= J).
__global__ void sym_min_kernel(float *D, long long ldd, int n)
{
    __shared__ float ta[32][33];
    __shared__ float tb[32][33];
    const int I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int i = I * 32 + r, j = J * 32 + tx;
        ta[r][tx] = (i < n && j < n) ? D[(long long)i * ldd + j] : 0.0f;
        const int i2 = J * 32 + r, j2 = I * 32 + tx;
        tb[r][tx] = (i2 < n && j2 < n) ? D[(long long)i2 * ldd + j2] : 0.0f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = I * 32 + r, j = J * 32 + tx;
        const float m = fminf(ta[r][tx], tb[tx][r]);  // D[i][j] vs D[j][i]
        if (i < n && j < n) D[(long long)i * ldd + j] = m;
        const int i2 = J * 32 + r, j2 = I * 32 + tx;
        const float m2 = fminf(tb[r][tx], ta[tx][r]);
        if (i2 < n && j2 < n) D[(long long)i2 * ldd + j2] = m2;
    }
}

// --------------------------------------------------------------- launch
struct ApspWork {
    int *deg, *rowptr, *cursor;
    uint2 *arcs;
    int *hubs, *near;
    float *dnear, *DH;
};

size_t apsp_work_bytes(int n, int approx, int h)
{
    const size_t ne = 3 * (size_t)n - 6;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
    add(4 * (size_t)n);          // deg
    add(4 * ((size_t)n + 1));    // rowptr
    add(4 * (size_t)n);          // cursor
    add(8 * 2 * ne);             // arcs
    if (approx) {
        add(4 * (size_t)h);
        add(4 * (size_t)n);
        add(4 * (size_t)n);
        add(4 * (size_t)h * n);
    }
    return b;
}

ApspWork apsp_carve(void *base, int n, int approx, int h)
{
    const size_t ne = 3 * (size_t)n - 6;
    ApspWork w{};
    char *p = static_cast<char *>(base);
    auto take = [&](size_t x) { void *r = p; p += (x + 255) & ~size_t(255); return r; };
    w.deg = static_cast<int *>(take(4 * (size_t)n));
    w.rowptr = static_cast<int *>(take(4 * ((size_t)n + 1)));
    w.cursor = static_cast<int *>(take(4 * (size_t)n));
    w.arcs = static_cast<uint2 *>(take(8 * 2 * ne));
    if (approx) {
        w.hubs = static_cast<int *>(take(4 * (size_t)h));
        w.near = static_cast<int *>(take(4 * (size_t)n));
        w.dnear = static_cast<float *>(take(4 * (size_t)n));
        w.DH = static_cast<float *>(take(4 * (size_t)h * n));
    }
    return w;
}

int launch_apsp_csr(const void *S, int n, long long ld, int dtype, const int *edges, void *work,
                    int *status, cudaStream_t stream)
{
    const int ne = 3 * n - 6;
    ApspWork w = apsp_carve(work, n, 0, 1);
    if (cudaMemsetAsync(w.deg, 0, 4 * (size_t)n, stream) != cudaSuccess) return TMFG_ECUDA;
    const int eb = (ne + 255) / 256;
    csr_degree_kernel<<<eb, 256, 0, stream>>>(edges, ne, n, w.deg, status);
    csr_scan_kernel<<<1, 1024, 0, stream>>>(w.deg, n, w.rowptr, w.cursor);
    if (dtype == TMFG_F32)
        csr_fill_kernel<float><<<eb, 256, 0, stream>>>(edges, ne, n, static_cast<const float *>(S),
                                                       ld, w.cursor, w.arcs);
    else
        csr_fill_kernel<double><<<eb, 256, 0, stream>>>(edges, ne, n,
                                                        static_cast<const double *>(S), ld,
                                                        w.cursor, w.arcs);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

int launch_apsp_exact_rows(int n, void *work, float *D, long long ldd, int s0, int s1, int *status,
                           int num_sms, unsigned long long timeout_ns, cudaStream_t stream)
{
    ApspWork w = apsp_carve(work, n, 0, 1);
    const size_t smem = sssp_smem_bytes(n);
    if (smem > 232448) return TMFG_ETOOBIG;
    if (cudaFuncSetAttribute(sssp_kernel<false, kSsspThreads>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return TMFG_ECUDA;
    SsspArgs a{};
    a.n = n;
    a.rowptr = w.rowptr;
    a.arcs = w.arcs;
    a.status = status;
    a.timeout_ns = timeout_ns;
    a.src = nullptr;
    a.src0 = s0;
    a.nsrc = s1 - s0;
    a.out = D + (long long)s0 * ldd;
    a.ldo = ldd;
    const int rows = s1 - s0;
    if (rows <= 0) return TMFG_OK;
    const int grid = rows < 2 * num_sms ? rows : 2 * num_sms;
    sssp_kernel<false, kSsspThreads><<<grid, kSsspThreads, smem, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

int launch_apsp(const void *S, int n, long long ld, int dtype, const int *edges, int approx,
                int h, float rf, float *D, long long ldd, void *work, int *status, int num_sms,
                unsigned long long timeout_ns, cudaStream_t stream)
{
    const int ne = 3 * n - 6;
    ApspWork w = apsp_carve(work, n, approx, h);
    if (cudaMemsetAsync(w.deg, 0, 4 * (size_t)n, stream) != cudaSuccess) return TMFG_ECUDA;
    const int eb = (ne + 255) / 256;
    csr_degree_kernel<<<eb, 256, 0, stream>>>(edges, ne, n, w.deg, status);
    csr_scan_kernel<<<1, 1024, 0, stream>>>(w.deg, n, w.rowptr, w.cursor);
    if (dtype == TMFG_F32)
        csr_fill_kernel<float><<<eb, 256, 0, stream>>>(edges, ne, n, static_cast<const float *>(S),
                                                       ld, w.cursor, w.arcs);
    else
        csr_fill_kernel<double><<<eb, 256, 0, stream>>>(edges, ne, n,
                                                        static_cast<const double *>(S), ld,
                                                        w.cursor, w.arcs);
    const size_t smem = sssp_smem_bytes(n);
    if (smem > 232448) return TMFG_ETOOBIG;
    if (cudaFuncSetAttribute(sssp_kernel<false, kSsspThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(sssp_kernel<true, kSsspThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return TMFG_ECUDA;
    SsspArgs a{};
    a.n = n;
    a.rowptr = w.rowptr;
    a.arcs = w.arcs;
    a.status = status;
    a.timeout_ns = timeout_ns;
    if (!approx) {
        a.src = nullptr;
        a.nsrc = n;
        a.out = D;
        a.ldo = ldd;
        const int grid = n < 2 * num_sms ? n : 2 * num_sms;
        sssp_kernel<false, kSsspThreads><<<grid, kSsspThreads, smem, stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
    }
    // hubs and their exact rows
    const size_t hsm = 4 * (size_t)n + 4 * (size_t)h;
    if (hsm > kSmemLimit - 1024) return TMFG_ETOOBIG;
    if (cudaFuncSetAttribute(hub_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hsm) != cudaSuccess)
        return TMFG_ECUDA;
    hub_select_kernel<<<1, 1024, hsm, stream>>>(w.rowptr, n, h, w.hubs, status);
    a.src = w.hubs;
    a.nsrc = h;
    a.out = w.DH;
    a.ldo = n;
    sssp_kernel<false, kSsspThreads><<<h < 2 * num_sms ? h : 2 * num_sms, kSsspThreads, smem, stream>>>(a);
    nearest_hub_kernel<<<(n + 255) / 256, 256, 0, stream>>>(w.DH, h, n, w.near, w.dnear);
    // bounded search from every vertex, approximate rows, then min with the transpose
    a.src = nullptr;
    a.nsrc = n;
    a.out = D;
    a.ldo = ldd;
    a.dnear = w.dnear;
    a.near = w.near;
    a.DH = w.DH;
    a.rf = rf;
    sssp_kernel<true, kSsspThreads><<<n < 2 * num_sms ? n : 2 * num_sms, kSsspThreads, smem, stream>>>(a);
    const int T = (n + 31) / 32;
    sym_min_kernel<<<dim3(T, T), dim3(32, 8), 0, stream>>>(D, ldd, n);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace tmfg

// ------------------------------------------------------------ batched
namespace tmfg {

// Exact APSP of many graphs at once: the CSR of every job is built by
// kernels over the concatenated edge lists, then one persistent grid runs a
// search per (job, source) pair.

__device__ __forceinline__ int find_job(const int *__restrict__ begin, int njobs, int x)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void csr_degree_batch_kernel(const ApspJob *__restrict__ jobs,
                                        const int *__restrict__ edge_begin, int njobs, int *status)
{
    const int total = edge_begin[njobs];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int j = find_job(edge_begin, njobs, e);
        const ApspJob &J = jobs[j];
        const int le = e - edge_begin[j];
        const int a = J.edges[2 * le], b = J.edges[2 * le + 1];
        if (a < 0 || b < 0 || a >= J.n || b >= J.n || a == b) {
            set_status(status, TMFG_EINVAL);
            continue;
        }
        atomicAdd(&J.deg[a], 1);
        atomicAdd(&J.deg[b], 1);
    }
}

// one CTA per job: row pointers and fill cursors from the degrees
__global__ void __launch_bounds__(1024) csr_scan_batch_kernel(const ApspJob *__restrict__ jobs)
{
    const ApspJob &J = jobs[blockIdx.x];
    __shared__ int wsum[32];
    const int n = J.n;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n + 1023) / 1024;
    const int lo = t * per, hi = min(n, lo + per);
    int sum = 0;
    for (int v = lo; v < hi; ++v) sum += J.deg[v];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z - w;
    }
    __syncthreads();
    int run = wsum[warp] + x - sum;
    if (t == 0) J.rowptr[0] = 0;
    for (int v = lo; v < hi; ++v) {
        J.cursor[v] = run;
        run += J.deg[v];
        J.rowptr[v + 1] = run;
    }
}

template <typename T>
__global__ void csr_fill_batch_kernel(const ApspJob *__restrict__ jobs,
                                      const int *__restrict__ edge_begin, int njobs)
{
    const int total = edge_begin[njobs];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int j = find_job(edge_begin, njobs, e);
        const ApspJob &J = jobs[j];
        const int le = e - edge_begin[j];
        const int a = J.edges[2 * le], b = J.edges[2 * le + 1];
        if (a < 0 || b < 0 || a >= J.n || b >= J.n || a == b) continue;
        const T *S = static_cast<const T *>(J.S);
        const float l = edge_length<T>(canon(S[(long long)a * J.ld + b]));
        const int pa = atomicAdd(&J.cursor[a], 1);
        const int pb = atomicAdd(&J.cursor[b], 1);
        J.arcs[pa] = make_uint2((unsigned)b, __float_as_uint(l));
        J.arcs[pb] = make_uint2((unsigned)a, __float_as_uint(l));
    }
}

// d_jobs / d_sargs: device copies of the job and SSSP tables; edge_begin and
// src_begin: device prefix sums (njobs + 1).  The degree arrays of every job
// must be zero on entry.
int launch_apsp_batch(const ApspJob *d_jobs, const SsspArgs *d_sargs, const int *d_edge_begin,
                      const int *d_src_begin, int njobs, int total_edges, int max_n, int dtype,
                      int sssp_threads, int *status, int num_sms, cudaStream_t stream)
{
    const int eb = (total_edges + 255) / 256;
    const int egrid = eb < 8 * num_sms ? (eb > 0 ? eb : 1) : 8 * num_sms;
    csr_degree_batch_kernel<<<egrid, 256, 0, stream>>>(d_jobs, d_edge_begin, njobs, status);
    csr_scan_batch_kernel<<<njobs, 1024, 0, stream>>>(d_jobs);
    if (dtype == TMFG_F32)
        csr_fill_batch_kernel<float><<<egrid, 256, 0, stream>>>(d_jobs, d_edge_begin, njobs);
    else
        csr_fill_batch_kernel<double><<<egrid, 256, 0, stream>>>(d_jobs, d_edge_begin, njobs);
    const size_t smem = sssp_smem_bytes(max_n);
    if (smem > kSmemLimit) return TMFG_ETOOBIG;
    auto go = [&](auto k, int nt) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return (int)TMFG_ECUDA;
        k<<<2 * num_sms, nt, smem, stream>>>(d_sargs, d_src_begin, njobs);
        return cudaGetLastError() == cudaSuccess ? (int)TMFG_OK : (int)TMFG_ECUDA;
    };
    if (sssp_threads == 256) return go(sssp_batch_kernel<256>, 256);
    return go(sssp_batch_kernel<512>, 512);
}

}  // namespace tmfg

// ------------------------------------------------- allocation-free variant
// Exact APSP whose scratch (the CSR: degrees, row pointers, cursors, arcs)
// lives in one file-scope device array instead of a context workspace, for
// callers that cannot allocate device memory.  Every GPU that loads this
// library holds the array (about 1.3 MB) until the process exits.
namespace tmfg {

constexpr size_t noalloc_round(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNoAllocBytes =
    noalloc_round(4 * (size_t)TMFG_NOALLOC_MAX_N) +          // deg
    noalloc_round(4 * ((size_t)TMFG_NOALLOC_MAX_N + 1)) +    // rowptr
    noalloc_round(4 * (size_t)TMFG_NOALLOC_MAX_N) +          // cursor
    noalloc_round(8 * 2 * (3 * (size_t)TMFG_NOALLOC_MAX_N - 6));  // arcs

static __device__ __align__(256) unsigned char g_apsp_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int g_noalloc_sms[kNoAllocMaxDevices];

// Device address of the scratch array in the context current on the calling
// thread, and the SM count of the current device.  The address is looked up
// on every call (a host-side table lookup once the module is loaded), so it
// stays right after a device reset or with a different context current; only
// the SM count, a property of the device, is kept between calls.
int noalloc_setup(void **ptr, int *sms)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return TMFG_ECUDA;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_apsp_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return TMFG_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_sms[dev]) {
        int s = 0;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            s <= 0) {
            cudaGetLastError();
            return TMFG_ECUDA;
        }
        g_noalloc_sms[dev] = s;
    }
    *ptr = p;
    *sms = g_noalloc_sms[dev];
    return TMFG_OK;
}
}  // namespace

}  // namespace tmfg

extern "C" int tmfg_apsp_exact_noalloc(const void *S, int64_t n, int64_t ld, int32_t dtype,
                                       const int32_t *edges, float *D, int64_t ldd,
                                       int32_t *status, void *stream)
{
    using namespace tmfg;
    if (!S || !edges || !D || !status || n < 4 || ld < n || ldd < n) return TMFG_EINVAL;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (n > TMFG_NOALLOC_MAX_N || sssp_smem_bytes((int)n) > kSmemLimit) return TMFG_ETOOBIG;
    // the exact path's carve of the workspace must fit the static array
    if (apsp_work_bytes((int)n, 0, 1) > kNoAllocBytes) return TMFG_EINTERNAL;
    void *work = nullptr;
    int sms = 0;
    int rc = noalloc_setup(&work, &sms);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the status output starts at zero; the degree counts are cleared by
    // launch_apsp itself before they are accumulated
    if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return TMFG_ECUDA;
    return launch_apsp(S, (int)n, ld, dtype, edges, 0, 0, 0.0f, D, ldd, work, status, sms,
                       device_timeout_ns(), st);
}
