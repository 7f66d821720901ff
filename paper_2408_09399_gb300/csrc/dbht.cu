// dbht.cu -- the DBHT dendrogram on the device (Section 2, "PMFG, TMFG, and
// DBHT": bubble tree, edge directions, converging bubbles, vertex -> group
// and vertex -> bubble assignment, three-level complete linkage).
//
// The paper sketches DBHT without fixing its rules; this file implements the
// reading documented in include/tmfg.h for dbht_cluster, so the linkage
// matrix equals the CPU oracle's exactly:
//   * bubble 0 = the initial clique, bubble k = {v_k} + t_k.  The inside of
//     the separating triangle t_k is the set of vertices introduced by the
//     bubbles of k's subtree, tested with an Euler-tour numbering;
//   * edge k points inside iff sum q(S[a,b]) over TMFG edges from t_k to the
//     inside exceeds that to the outside (q = S*2^40 rounded, int64 sums);
//   * converging bubbles have no outgoing edge; a vertex joins the converging
//     bubble of least mean D to its 4 vertices, every other bubble the
//     converging bubble of least mean inter-bubble D, and a vertex then the
//     bubble of least mean D among its group's (means in double, summed in
//     a fixed order; ties to the smaller bubble id);
//   * complete linkage inside each (group, bubble) cell, then among the cells
//     of each group, then among the groups; ties to the pair with the
//     smallest (min leaf id, max leaf id); rows in the scipy layout, written
//     at offsets fixed by prefix sums so that the row order is independent
//     of scheduling.
#include "internal.cuh"

namespace tmfg {

namespace {

constexpr int kDbThreads = 256;   // linkage CTAs
constexpr int kResCap = 1024;     // rows re-scanned cooperatively per merge
constexpr int kCapG = 2048;       // groups whose maxima fit shared memory
constexpr int kCapC = 4096;       // cells of one group whose maxima fit shared memory

struct DbWork {
    int n, nb;
    int *status;
    int *bv;              // [4 nb] bubble vertices
    int *intro;           // [n] bubble that introduced each vertex
    int *tin, *tsz;       // [nb] Euler-tour entry, subtree size
    int *rowptr;          // [n+1] TMFG adjacency
    int *cursor;          // [n]
    int2 *adj;            // [2 ne] {neighbour, edge id}
    int *dir;             // [nb] edge k points inside (k >= 1)
    int *outdeg;          // [nb]
    int *conv;            // [nb] converging bubbles, ascending
    int *gidx;            // [nb] group index of a converging bubble, -1 otherwise
    int *group;           // [n] converging bubble of each vertex
    int *hidx;            // [nb] group index of each bubble's home
    int *glist, *gbeg;    // bubbles of each group (ascending) + offsets [nb+1]
    int *bub;             // [n] bubble of each vertex
    int *cell_list, *cell_beg;  // vertices of each bubble (ascending) + offsets [nb+1]
    int *bcnt, *bcur, *btmp;    // bucket scratch [nb], [nb], [n]
    int *pos;             // [nb+1] scan scratch
    int *scal;            // [0] nc, [1] rows of level 1, [2] rows of level 2, [3] ngroups
    long long *lscal;     // [0] level-2 matrices, [1] level-3 matrix, [2] end (floats)
    int *l1_off;          // [nb+1] first linkage row of each cell
    long long *dm_off1;   // [nb+1] offsets of the cell distance matrices
    int *cid, *crep, *csz;        // [nb] final id / rep / size of each cell
    int *gcells_beg;      // [nb+1] nonempty cells of each group
    int *gcells;          // [nb]
    int *bslot;           // [nb] slot of a nonempty cell within its group
    int *l2_off;          // [nb+1]
    long long *dm_off2;   // [nb+1]
    int *gid, *grep, *gsz, *gslot;  // [nb] per group
    int2 *vinfo;          // [n] {group index, cell slot} of each vertex
    int *items_id, *items_rep, *items_sz;  // [n] linkage scratch (disjoint slices)
    unsigned long long *rowkey;            // [n]
    int *rowbest, *alive;                  // [n]
    float *dm;            // distance matrices of the three levels
    long long dm_cap;     // floats
};

__device__ __forceinline__ float dsym(const float *D, long long ldd, int i, int j)
{
    return i <= j ? D[(long long)i * ldd + j] : D[(long long)j * ldd + i];
}

// Exclusive scan over one CTA: out[i] = sum_{j<i} val(j), out[m] = total.
// Every thread calls it; returns the total.
template <typename T, typename F>
__device__ T cta_scan(int m, F val, T *out)
{
    __shared__ T ws[32];
    __shared__ T s_tot;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const int per = (m + (int)blockDim.x - 1) / (int)blockDim.x;
    const int lo = min(m, t * per), hi = min(m, lo + per);
    T s = 0;
    for (int i = lo; i < hi; ++i) s += val(i);
    T x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const T orig = lane < nwarp ? ws[lane] : T(0);
        T z = orig;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nwarp) ws[lane] = z - orig;
        if (lane == 31) s_tot = z;
    }
    __syncthreads();
    T run = ws[warp] + x - s;
    for (int i = lo; i < hi; ++i) {
        out[i] = run;
        run += val(i);
    }
    if (t == 0) out[m] = s_tot;
    const T total = s_tot;
    __syncthreads();
    return total;
}

// ------------------------------------------------------------ input checks
// order a permutation of 0..n-1, parent[0] = -1 and 0 <= parent[k] < k,
// every ins_face and edge endpoint in [0, n).  `seen` starts at zero.
__global__ void dbht_check_kernel(int n, const int *order, const int *edges, const int *ins_face,
                                  const int *parent, int *seen, int *status)
{
    const int nb = n - 3, ne = 3 * n - 6;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ne; i += stride) {
        const int x = edges[i];
        if (x < 0 || x >= n) set_status(status, TMFG_EINVAL);
        if (i < n) {
            const int v = order[i];
            if (v < 0 || v >= n || atomicAdd(&seen[v], 1) != 0) set_status(status, TMFG_EINVAL);
        }
        if (i < 3 * (nb - 1)) {
            const int f = ins_face[i];
            if (f < 0 || f >= n) set_status(status, TMFG_EINVAL);
        }
        if (i < nb) {
            const int p = parent[i];
            if (i == 0 ? p != -1 : (p < 0 || p >= i)) set_status(status, TMFG_EINVAL);
        }
    }
}

// ------------------------------------------------------------ bubble tree
// Bubble vertex sets and the introducing bubble of each vertex (parallel);
// subtree sizes and the Euler-tour numbering (one thread, on shared memory;
// parents always have smaller ids than their children).
__global__ void __launch_bounds__(1024) dbht_tree_kernel(DbWork w, const int *order,
                                                         const int *ins_face, const int *parent)
{
    if (*w.status) return;
    extern __shared__ int sm[];
    const int nb = w.nb, n = w.n, t = threadIdx.x;
    int *sz = sm;                                               // [nb]
    int *nxt = sm + nb;                                         // [nb]
    uint16_t *par = reinterpret_cast<uint16_t *>(sm + 2 * nb);  // [nb]
    for (int b = t; b < nb; b += blockDim.x) {
        sz[b] = 1;
        par[b] = b ? (uint16_t)parent[b] : (uint16_t)0;
        if (b == 0) {
            for (int i = 0; i < 4; ++i) w.bv[i] = order[i];
        } else {
            w.bv[4 * b] = order[b + 3];
            for (int i = 0; i < 3; ++i) w.bv[4 * b + 1 + i] = ins_face[3 * (b - 1) + i];
        }
    }
    for (int i = t; i < n; i += blockDim.x) w.intro[order[i]] = i < 4 ? 0 : i - 3;
    __syncthreads();
    if (t == 0) {
        for (int k = nb - 1; k >= 1; --k) sz[par[k]] += sz[k];
        nxt[0] = 1;
        w.tin[0] = 0;
        for (int k = 1; k < nb; ++k) {
            const int p = par[k];
            const int tk = nxt[p];
            w.tin[k] = tk;
            nxt[p] = tk + sz[k];
            nxt[k] = tk + 1;
        }
    }
    __syncthreads();
    for (int b = t; b < nb; b += blockDim.x) w.tsz[b] = sz[b];
}

__global__ void dbht_deg_kernel(const int *edges, int ne, int *deg, const int *status)
{
    if (*status) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        atomicAdd(&deg[edges[2 * e]], 1);
        atomicAdd(&deg[edges[2 * e + 1]], 1);
    }
}

// out[0..m] = exclusive scan of cnt[0..m); copy[0..m) = out[0..m) if given.
__global__ void __launch_bounds__(1024) scan_kernel(const int *cnt, int m, int *out, int *copy,
                                                    const int *status)
{
    if (*status) return;
    cta_scan<int>(m, [&](int i) { return cnt[i]; }, out);
    if (copy)
        for (int i = threadIdx.x; i < m; i += blockDim.x) copy[i] = out[i];
}

__global__ void dbht_fill_kernel(const int *edges, int ne, int *cursor, int2 *adj,
                                 const int *status)
{
    if (*status) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int a = edges[2 * e], b = edges[2 * e + 1];
        adj[atomicAdd(&cursor[a], 1)] = make_int2(b, e);
        adj[atomicAdd(&cursor[b], 1)] = make_int2(a, e);
    }
}

// ------------------------------------------------------------ directions
// One warp per bubble-tree edge k >= 1: exact int64 sums of q(S) over the
// TMFG edges from t_k to the inside and to the outside.
template <typename T>
__global__ void dbht_dir_kernel(DbWork w, const T *S, long long ld, const int *edges,
                                const int *ins_face, const int *parent)
{
    if (*w.status) return;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = 1 + wid; k < w.nb; k += nw) {
        const int t0 = ins_face[3 * (k - 1)], t1 = ins_face[3 * (k - 1) + 1],
                  t2 = ins_face[3 * (k - 1) + 2];
        const int lo = w.tin[k], hi = w.tin[k] + w.tsz[k];
        long long win = 0, wout = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int a = i == 0 ? t0 : (i == 1 ? t1 : t2);
            for (int p = w.rowptr[a] + lane; p < w.rowptr[a + 1]; p += 32) {
                const int2 x = w.adj[p];
                const int j = x.x;
                if (j == t0 || j == t1 || j == t2) continue;
                const int ea = edges[2 * x.y], eb = edges[2 * x.y + 1];
                const long long q = quantize40(canon(S[(long long)ea * ld + eb]));
                const int ti = w.tin[w.intro[j]];
                if (ti >= lo && ti < hi) win += q; else wout += q;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            win += __shfl_xor_sync(0xffffffffu, win, o);
            wout += __shfl_xor_sync(0xffffffffu, wout, o);
        }
        if (lane == 0) {
            const int d = win > wout ? 1 : 0;
            w.dir[k] = d;
            atomicAdd(&w.outdeg[d ? parent[k] : k], 1);
        }
    }
}

// The converging bubbles (no outgoing edge) in ascending order; one CTA.
__global__ void __launch_bounds__(1024) dbht_conv_kernel(DbWork w)
{
    if (*w.status) return;
    __shared__ int wsum[32];
    __shared__ int s_base;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_base = 0;
    __syncthreads();
    for (int b0 = 0; b0 < w.nb; b0 += 1024) {
        const int b = b0 + t;
        const int f = (b < w.nb && w.outdeg[b] == 0) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int i = 0; i < 32; ++i) {
            pre += i < warp ? wsum[i] : 0;
            tot += wsum[i];
        }
        pre += __popc(bal & ((1u << lane) - 1u));
        if (b < w.nb) w.gidx[b] = f ? s_base + pre : -1;
        if (f) w.conv[s_base + pre] = b;
        __syncthreads();
        if (t == 0) s_base += tot;
        __syncthreads();
    }
    if (t == 0) w.scal[0] = s_base;
}

// ------------------------------------------------------------ assignments
// Group of each vertex: the converging bubble of least mean D to its four
// vertices (double, summed in vertex order; ties to the smaller id).
__global__ void dbht_group_kernel(DbWork w, const float *D, long long ldd)
{
    if (*w.status) return;
    const int nc = w.scal[0];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < w.n; v += gridDim.x * blockDim.x) {
        int bc = -1;
        double bm = 0.0;
        for (int c = 0; c < nc; ++c) {
            const int cb = w.conv[c];
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) s = __dadd_rn(s, (double)dsym(D, ldd, v, w.bv[4 * cb + i]));
            s = __ddiv_rn(s, 4.0);
            if (bc < 0 || s < bm) { bc = cb; bm = s; }
        }
        w.group[v] = bc;
    }
}

// Home of each bubble: itself if converging, else the converging bubble of
// least mean D over the 16 vertex pairs; stored as a group index.
__global__ void dbht_home_kernel(DbWork w, const float *D, long long ldd)
{
    if (*w.status) return;
    const int nc = w.scal[0];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < w.nb; b += gridDim.x * blockDim.x) {
        if (w.outdeg[b] == 0) { w.hidx[b] = w.gidx[b]; continue; }
        int bc = -1;
        double bm = 0.0;
        for (int c = 0; c < nc; ++c) {
            const int cb = w.conv[c];
            double s = 0.0;
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    s = __dadd_rn(s, (double)dsym(D, ldd, w.bv[4 * b + i], w.bv[4 * cb + j]));
            s = __ddiv_rn(s, 16.0);
            if (bc < 0 || s < bm) { bc = c; bm = s; }
        }
        w.hidx[b] = bc;
    }
}

// Bubble of each vertex: least mean D among the bubbles of its group.
__global__ void dbht_bubble_kernel(DbWork w, const float *D, long long ldd)
{
    if (*w.status) return;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < w.n; v += gridDim.x * blockDim.x) {
        const int g = w.gidx[w.group[v]];
        int bb = -1;
        double bm = 0.0;
        for (int p = w.gbeg[g]; p < w.gbeg[g + 1]; ++p) {
            const int b = w.glist[p];
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) s = __dadd_rn(s, (double)dsym(D, ldd, v, w.bv[4 * b + i]));
            s = __ddiv_rn(s, 4.0);
            if (bb < 0 || s < bm) { bb = b; bm = s; }
        }
        w.bub[v] = bb;
    }
}

// ------------------------------------------------------------ stable buckets
// Lists the items 0..count-1 of each key in ascending item order: counts by
// atomics, scan, unordered scatter, then each item finds its rank among the
// smaller items of its bucket.
__global__ void bucket_count_kernel(const int *key, int count, int *cnt, const int *status)
{
    if (*status) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        atomicAdd(&cnt[key[i]], 1);
}

__global__ void bucket_scatter_kernel(const int *key, int count, int *cur, int *tmp,
                                      const int *status)
{
    if (*status) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        tmp[atomicAdd(&cur[key[i]], 1)] = i;
}

__global__ void bucket_order_kernel(const int *key, int count, const int *beg, const int *tmp,
                                    int *out, const int *status)
{
    if (*status) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
        const int item = tmp[q];
        const int k = key[item];
        const int lo = beg[k], hi = beg[k + 1];
        int rank = 0;
        for (int r = lo; r < hi; ++r) rank += tmp[r] < item;
        out[lo + rank] = item;
    }
}

// ------------------------------------------------------------ plan
// One CTA: linkage row offsets and distance-matrix offsets of the three
// levels, the nonempty cells of each group, the group slots of level 3 and
// {group, cell slot} of every vertex.
__global__ void __launch_bounds__(1024) dbht_plan_kernel(DbWork w)
{
    if (*w.status) return;
    const int nb = w.nb, n = w.n, nc = w.scal[0], t = threadIdx.x;
    auto csize = [&](int b) { return w.cell_beg[b + 1] - w.cell_beg[b]; };
    const int rows1 = cta_scan<int>(nb, [&](int b) { return max(csize(b) - 1, 0); }, w.l1_off);
    const long long dm1 = cta_scan<long long>(
        nb, [&](int b) { const long long m = csize(b); return m >= 2 ? m * m : 0ll; }, w.dm_off1);
    // nonempty cells of each group, ascending bubble id within a group
    cta_scan<int>(nb, [&](int p) { return csize(w.glist[p]) > 0 ? 1 : 0; }, w.pos);
    for (int c = t; c <= nc; c += blockDim.x) w.gcells_beg[c] = w.pos[w.gbeg[c]];
    __syncthreads();
    for (int p = t; p < nb; p += blockDim.x) {
        const int b = w.glist[p];
        if (csize(b) > 0) {
            w.gcells[w.pos[p]] = b;
            w.bslot[b] = w.pos[p] - w.gcells_beg[w.hidx[b]];
        }
    }
    __syncthreads();
    auto gsize = [&](int c) { return w.gcells_beg[c + 1] - w.gcells_beg[c]; };
    const int rows2 = cta_scan<int>(nc, [&](int c) { return max(gsize(c) - 1, 0); }, w.l2_off);
    const long long dm2 = cta_scan<long long>(
        nc, [&](int c) { const long long m = gsize(c); return m >= 2 ? m * m : 0ll; }, w.dm_off2);
    const int ng = cta_scan<int>(nc, [&](int c) { return gsize(c) > 0 ? 1 : 0; }, w.pos);
    for (int c = t; c < nc; c += blockDim.x) {
        w.l2_off[c] += rows1;
        w.dm_off2[c] += dm1;
        w.gslot[c] = gsize(c) > 0 ? w.pos[c] : -1;
    }
    for (int v = t; v < n; v += blockDim.x)
        w.vinfo[v] = make_int2(w.gidx[w.group[v]], w.bslot[w.bub[v]]);
    if (t == 0) {
        w.scal[1] = rows1;
        w.scal[2] = rows2;
        w.scal[3] = ng;
        w.lscal[0] = dm1;
        w.lscal[1] = dm1 + dm2;
        w.lscal[2] = dm1 + dm2 + (long long)ng * ng;
        if (w.lscal[2] > w.dm_cap || rows1 + rows2 + ng != n) set_status(w.status, TMFG_EINTERNAL);
    }
}

// level-2 and level-3 matrices start at zero (maxima of non-negative floats)
__global__ void dbht_zero_kernel(DbWork w)
{
    if (*w.status) return;
    const long long lo = w.lscal[0], hi = w.lscal[2];
    for (long long i = lo + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < hi;
         i += (long long)gridDim.x * blockDim.x)
        w.dm[i] = 0.0f;
}

// ------------------------------------------------------------ complete linkage
// Key of a candidate merge: distance bits (non-negative floats order as
// their bits), then the smaller and the larger representative leaf id.
__device__ __forceinline__ unsigned long long lk_key(float d, int ra, int rb)
{
    const int r0 = ra < rb ? ra : rb, r1 = ra < rb ? rb : ra;
    return ((unsigned long long)__float_as_uint(d) << 30) | ((unsigned long long)r0 << 15) |
           (unsigned long long)r1;
}

// Best merge partner of row i (one warp, four columns per lane in flight).
__device__ __forceinline__ void lk_row_scan(int i, int m, const float *dm, const int *rep,
                                            const int *alive, unsigned long long *rowkey,
                                            int *rowbest, int lane)
{
    unsigned long long bk = ~0ull;
    int bj = -1;
    const int ri = rep[i];
    const float *row = dm + (long long)i * m;
    for (int j0 = lane; j0 < m; j0 += 4 * 32) {
        float dv[4];
        int rj[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + 32 * u;
            ok[u] = j < m && j != i && alive[j];
            dv[u] = ok[u] ? row[j] : 0.0f;
            rj[u] = ok[u] ? rep[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (ok[u]) {
                const unsigned long long k = lk_key(dv[u], ri, rj[u]);
                if (k < bk) { bk = k; bj = j0 + 32 * u; }
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
        if (k2 < bk) { bk = k2; bj = j2; }
    }
    if (lane == 0) {
        rowkey[i] = bk;
        rowbest[i] = bj;
    }
}

// Items whose per-item state (row key, best partner, alive flag,
// representative, id, size: 28 bytes) the linkage keeps in shared memory.
constexpr int kLkCap = 3072;
constexpr size_t kLkSmem = 28 * (size_t)kLkCap;
constexpr int kRB = 4;         // rows re-scanned together by the whole CTA
constexpr int kLkUnroll = 4;   // columns per thread in flight during a re-scan
constexpr int kLkUpd = 4;      // rows per thread in flight during a merge update
constexpr int kLkMaxWarps = kDbThreads / 32;

// Complete linkage of m >= 2 items by one CTA.  dm: m x m distances in
// global memory (destroyed); id/rep/sz per item.  Each merge takes the
// smallest key over all pairs (keys are unique per pair: they carry both
// representatives).  The row minima stay current: after a merge (a, b), one
// pass over the other rows writes row and column a as the maxima of rows a
// and b and updates each row's minimum with its new distance to a; rows
// whose partner was a or b, and row a, are re-scanned by the whole CTA.
// Merge `step` writes linkage row row0 + step and leaves the merged cluster
// in the lower slot; the final cluster goes to out_*.  With m <= cap the
// per-item state lives in `sm` (cap * 28 bytes of shared memory).
__device__ void linkage_cta(int m, float *dm, int *id_g, int *rep_g, int *sz_g,
                            unsigned long long *rowkey_g, int *rowbest_g, int *alive_g, int n,
                            int row0, double *Z, int *status, int *out_id, int *out_rep,
                            int *out_sz, unsigned char *sm, int cap)
{
    __shared__ unsigned long long s_k[32];
    __shared__ int s_i[32];
    __shared__ int s_a, s_b, s_nres, s_fail;
    __shared__ int s_res[kResCap];
    __shared__ unsigned long long s_pk[kRB * kLkMaxWarps];
    __shared__ int s_pj[kRB * kLkMaxWarps];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    const bool fits = m <= cap;
    unsigned long long *rowkey =
        fits ? reinterpret_cast<unsigned long long *>(sm) : rowkey_g;
    int *rowbest = fits ? reinterpret_cast<int *>(sm + 8 * (size_t)cap) : rowbest_g;
    int *alive = fits ? reinterpret_cast<int *>(sm + 12 * (size_t)cap) : alive_g;
    int *rep = fits ? reinterpret_cast<int *>(sm + 16 * (size_t)cap) : rep_g;
    int *id = fits ? reinterpret_cast<int *>(sm + 20 * (size_t)cap) : id_g;
    int *sz = fits ? reinterpret_cast<int *>(sm + 24 * (size_t)cap) : sz_g;
    for (int i = t; i < m; i += blockDim.x) {
        alive[i] = 1;
        if (fits) {
            rep[i] = rep_g[i];
            id[i] = id_g[i];
            sz[i] = sz_g[i];
        }
    }
    if (t == 0) s_fail = 0;
    __syncthreads();
    for (int i = warp; i < m; i += nw) lk_row_scan(i, m, dm, rep, alive, rowkey, rowbest, lane);
    __syncthreads();
    for (int step = 0; step + 1 < m; ++step) {
        unsigned long long bk = ~0ull;
        int bi = -1;
        for (int i = t; i < m; i += blockDim.x)
            if (alive[i] && rowkey[i] < bk) { bk = rowkey[i]; bi = i; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (k2 < bk || (k2 == bk && i2 >= 0 && (bi < 0 || i2 < bi))) { bk = k2; bi = i2; }
        }
        if (lane == 0) { s_k[warp] = bk; s_i[warp] = bi; }
        __syncthreads();
        if (t == 0) {
            unsigned long long k = s_k[0];
            int i = s_i[0];
            for (int q = 1; q < nw; ++q)
                if (s_k[q] < k || (s_k[q] == k && s_i[q] >= 0 && (i < 0 || s_i[q] < i))) {
                    k = s_k[q];
                    i = s_i[q];
                }
            const int j = i >= 0 ? rowbest[i] : -1;
            if (i < 0 || j < 0 || j == i || !alive[j]) {
                s_fail = 1;
                set_status(status, TMFG_EINTERNAL);
            } else {
                const int a = i < j ? i : j, b = i < j ? j : i;
                s_a = a;
                s_b = b;
                const int row = row0 + step;
                const int ia = id[a], ib = id[b];
                Z[4 * row + 0] = (double)(ia < ib ? ia : ib);
                Z[4 * row + 1] = (double)(ia < ib ? ib : ia);
                // the key carries the pair's distance bits (dm[a][b])
                Z[4 * row + 2] = (double)__uint_as_float((unsigned)(k >> 30));
                Z[4 * row + 3] = (double)(sz[a] + sz[b]);
                id[a] = n + row;
                rep[a] = rep[a] < rep[b] ? rep[a] : rep[b];
                sz[a] += sz[b];
                alive[b] = 0;
            }
            s_nres = 0;
        }
        __syncthreads();
        if (s_fail) break;
        const int a = s_a, b = s_b, repa = rep[a];
        // row and column a = max of rows a and b; minima of the other rows
        // (kLkUpd rows per thread with their loads in flight)
        for (int k0 = t; k0 < m; k0 += kLkUpd * blockDim.x) {
            float d1[kLkUpd], d2[kLkUpd];
            bool live[kLkUpd];
#pragma unroll
            for (int u = 0; u < kLkUpd; ++u) {
                const int k = k0 + u * blockDim.x;
                live[u] = k < m && alive[k];
                const bool ld = live[u] && k != a;
                d1[u] = ld ? dm[(long long)a * m + k] : 0.0f;
                d2[u] = ld ? dm[(long long)b * m + k] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < kLkUpd; ++u) {
                const int k = k0 + u * blockDim.x;
                if (!live[u]) continue;
                bool again = k == a;
                if (!again) {
                    const float d = d1[u] > d2[u] ? d1[u] : d2[u];
                    dm[(long long)a * m + k] = d;
                    dm[(long long)k * m + a] = d;
                    const int pb = rowbest[k];
                    again = pb == a || pb == b;
                    if (!again) {
                        const unsigned long long kk = lk_key(d, rep[k], repa);
                        if (kk < rowkey[k]) { rowkey[k] = kk; rowbest[k] = a; }
                    }
                }
                if (again) {
                    const int slot = atomicAdd(&s_nres, 1);
                    if (slot < kResCap) s_res[slot] = k;
                    else rowbest[k] = -2;  // re-scanned by this thread below
                }
            }
        }
        __syncthreads();
        // rows beyond the list (more than kResCap re-scans in one merge)
        if (s_nres > kResCap)
            for (int k = t; k < m; k += blockDim.x) {
                if (!alive[k] || rowbest[k] != -2) continue;
                unsigned long long bk2 = ~0ull;
                int bj2 = -1;
                for (int j = 0; j < m; ++j) {
                    if (j == k || !alive[j]) continue;
                    const unsigned long long kk = lk_key(dm[(long long)k * m + j], rep[k], rep[j]);
                    if (kk < bk2) { bk2 = kk; bj2 = j; }
                }
                rowkey[k] = bk2;
                rowbest[k] = bj2;
            }
        // the listed rows, kRB at a time, by the whole CTA
        const int nres = min(s_nres, kResCap);
        for (int r0 = 0; r0 < nres; r0 += kRB) {
            int ri[kRB], rr[kRB];
            unsigned long long bq[kRB];
            int bjq[kRB];
#pragma unroll
            for (int q = 0; q < kRB; ++q) {
                ri[q] = r0 + q < nres ? s_res[r0 + q] : -1;
                rr[q] = ri[q] >= 0 ? rep[ri[q]] : 0;
                bq[q] = ~0ull;
                bjq[q] = -1;
            }
            for (int j0 = t; j0 < m; j0 += kLkUnroll * blockDim.x) {
                float dv[kLkUnroll][kRB];
                int rj[kLkUnroll];
                bool ok[kLkUnroll];
#pragma unroll
                for (int u = 0; u < kLkUnroll; ++u) {
                    const int j = j0 + u * blockDim.x;
                    ok[u] = j < m && alive[j];
                    rj[u] = ok[u] ? rep[j] : 0;
#pragma unroll
                    for (int q = 0; q < kRB; ++q)
                        dv[u][q] = (ok[u] && ri[q] >= 0 && ri[q] != j) ? dm[(long long)ri[q] * m + j]
                                                                       : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < kLkUnroll; ++u) {
                    const int j = j0 + u * blockDim.x;
#pragma unroll
                    for (int q = 0; q < kRB; ++q)
                        if (ok[u] && ri[q] >= 0 && ri[q] != j) {
                            const unsigned long long kk = lk_key(dv[u][q], rr[q], rj[u]);
                            if (kk < bq[q]) { bq[q] = kk; bjq[q] = j; }
                        }
                }
            }
#pragma unroll
            for (int q = 0; q < kRB; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bq[q], o);
                    const int j2 = __shfl_xor_sync(0xffffffffu, bjq[q], o);
                    if (k2 < bq[q]) { bq[q] = k2; bjq[q] = j2; }
                }
                if (lane == 0) {
                    s_pk[q * kLkMaxWarps + warp] = bq[q];
                    s_pj[q * kLkMaxWarps + warp] = bjq[q];
                }
            }
            __syncthreads();
            if (t < kRB && r0 + t < nres) {
                unsigned long long k = s_pk[t * kLkMaxWarps];
                int j = s_pj[t * kLkMaxWarps];
                for (int q = 1; q < nw; ++q)
                    if (s_pk[t * kLkMaxWarps + q] < k) {
                        k = s_pk[t * kLkMaxWarps + q];
                        j = s_pj[t * kLkMaxWarps + q];
                    }
                rowkey[s_res[r0 + t]] = k;
                rowbest[s_res[r0 + t]] = j;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        for (int i = 0; i < m; ++i)
            if (alive[i]) { *out_id = id[i]; *out_rep = rep[i]; *out_sz = sz[i]; break; }
    }
    __syncthreads();
}

// Complete linkage by the nearest-neighbour chain (one CTA, 2 <= m <=
// kChainMax items, state in `sm`).  Complete linkage is reducible --
// d(i+j, k) = max(d(i,k), d(j,k)) >= min(d(i,k), d(j,k)) -- and the keys
// order all pairs strictly (with equal distances the merged cluster's key to
// k equals one of its parts' keys, since its representative is the smaller
// of the two), so merging reciprocal nearest neighbours as the chain finds
// them builds the same hierarchy as always merging the globally smallest
// key, and the merge keys of that sequential order increase strictly.  The
// merges are therefore recorded with their keys, sorted, and replayed in
// key order to write the linkage rows and cluster ids exactly as the
// sequential order does.  Each chain step is one row scan by the whole CTA
// (no row minima to keep current), a merge one more pass over rows a and b.
constexpr int kChainMax = 2048;
// keys (8 B) and six int arrays per item, inside the linkage kernels' shared memory
static_assert(32 * (size_t)kChainMax <= kLkSmem, "chain state exceeds the linkage shared memory");
constexpr int kChainUnroll = 8;   // row entries per thread in flight (m <= 2048)
__device__ void linkage_chain_cta(int m, float *dm, const int *id_g, const int *rep_g,
                                  const int *sz_g, int n, int row0, double *Z, int *status,
                                  int *out_id, int *out_rep, int *out_sz, unsigned char *sm)
{
    __shared__ unsigned long long s_pk[kLkMaxWarps];
    __shared__ int s_pj[kLkMaxWarps];
    __shared__ int s_x, s_len, s_merges, s_start, s_act, s_a, s_b, s_fail;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    unsigned long long *mkey = reinterpret_cast<unsigned long long *>(sm);
    int *mab = reinterpret_cast<int *>(sm + 8 * (size_t)kChainMax);
    int *chain = mab + kChainMax;
    int *alive = chain + kChainMax;
    int *rep = alive + kChainMax;
    int *id = rep + kChainMax;
    int *sz = id + kChainMax;
    for (int i = t; i < m; i += blockDim.x) {
        alive[i] = 1;
        rep[i] = rep_g[i];
        id[i] = id_g[i];
        sz[i] = sz_g[i];
    }
    if (t == 0) {
        s_len = 1;
        chain[0] = 0;
        s_x = 0;
        s_merges = 0;
        s_start = 0;
        s_fail = 0;
    }
    __syncthreads();
    const int nmerge = m - 1;
    // at most 2m - 1 pushes and m - 1 merges
    for (int iter = 0; s_merges < nmerge; ++iter) {
        if (iter > 3 * m) {
            if (t == 0) set_status(status, TMFG_EINTERNAL);
            return;
        }
        // nearest neighbour of the chain's top x
        const int x = s_x, rx = rep[x];
        const float *row = dm + (long long)x * m;
        unsigned long long bk = ~0ull;
        int bj = -1;
        for (int j0 = t; j0 < m; j0 += kChainUnroll * blockDim.x) {
            float dv[kChainUnroll];
            int rj[kChainUnroll];
            bool ok[kChainUnroll];
#pragma unroll
            for (int u = 0; u < kChainUnroll; ++u) {
                const int j = j0 + u * blockDim.x;
                ok[u] = j < m && j != x && alive[j];
                dv[u] = ok[u] ? row[j] : 0.0f;
                rj[u] = ok[u] ? rep[j] : 0;
            }
#pragma unroll
            for (int u = 0; u < kChainUnroll; ++u)
                if (ok[u]) {
                    const unsigned long long k = lk_key(dv[u], rx, rj[u]);
                    if (k < bk) { bk = k; bj = j0 + u * blockDim.x; }
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
            const int j2 = __shfl_xor_sync(0xffffffffu, bj, o);
            if (k2 < bk) { bk = k2; bj = j2; }
        }
        if (lane == 0) { s_pk[warp] = bk; s_pj[warp] = bj; }
        __syncthreads();
        if (t == 0) {
            unsigned long long k = s_pk[0];
            int y = s_pj[0];
            for (int q = 1; q < nw; ++q)
                if (s_pk[q] < k) { k = s_pk[q]; y = s_pj[q]; }
            s_act = 0;
            if (y < 0) {
                s_fail = 1;
                set_status(status, TMFG_EINTERNAL);
            } else if (s_len >= 2 && chain[s_len - 2] == y) {
                // reciprocal nearest neighbours: merge into the lower slot
                const int a = x < y ? x : y, b = x < y ? y : x;
                mkey[s_merges] = k;
                mab[s_merges] = a | (b << 16);
                ++s_merges;
                rep[a] = rep[a] < rep[b] ? rep[a] : rep[b];
                alive[b] = 0;
                s_len -= 2;
                s_a = a;
                s_b = b;
                s_act = 1;
                if (s_len == 0) {  // restart the chain at the smallest live item
                    while (s_start < m && !alive[s_start]) ++s_start;
                    chain[s_len++] = s_start < m ? s_start : a;
                }
                s_x = chain[s_len - 1];
            } else if (s_len >= m) {  // a chain longer than the items: cannot happen
                s_fail = 1;
                set_status(status, TMFG_EINTERNAL);
            } else {
                chain[s_len++] = y;
                s_x = y;
            }
        }
        __syncthreads();
        if (s_fail) return;
        if (s_act) {
            // row and column a = max of rows a and b
            const int a = s_a, b = s_b;
            for (int k0 = t; k0 < m; k0 += kChainUnroll * blockDim.x) {
                float d1[kChainUnroll], d2[kChainUnroll];
                bool ok[kChainUnroll];
#pragma unroll
                for (int u = 0; u < kChainUnroll; ++u) {
                    const int k = k0 + u * blockDim.x;
                    ok[u] = k < m && k != a && alive[k];
                    d1[u] = ok[u] ? dm[(long long)a * m + k] : 0.0f;
                    d2[u] = ok[u] ? dm[(long long)b * m + k] : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < kChainUnroll; ++u)
                    if (ok[u]) {
                        const int k = k0 + u * blockDim.x;
                        const float d = d1[u] > d2[u] ? d1[u] : d2[u];
                        dm[(long long)a * m + k] = d;
                        dm[(long long)k * m + a] = d;
                    }
            }
            __syncthreads();
        }
    }
    // the merges in key order (bitonic sort of the key / pair records)
    int P = 1;
    while (P < nmerge) P <<= 1;
    for (int i = nmerge + t; i < P; i += blockDim.x) {
        mkey[i] = ~0ull;
        mab[i] = 0;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = t; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long ki = mkey[i], kj = mkey[j];
                    if ((ki > kj) == up) {
                        mkey[i] = kj;
                        mkey[j] = ki;
                        const int tmp = mab[i];
                        mab[i] = mab[j];
                        mab[j] = tmp;
                    }
                }
            }
            __syncthreads();
        }
    // replay: linkage rows and cluster ids in the sequential order
    if (t == 0) {
        int last = 0;
        for (int r = 0; r < nmerge; ++r) {
            const int a = mab[r] & 0xFFFF, b = (mab[r] >> 16) & 0xFFFF;
            const int row = row0 + r;
            const int ia = id[a], ib = id[b];
            Z[4 * row + 0] = (double)(ia < ib ? ia : ib);
            Z[4 * row + 1] = (double)(ia < ib ? ib : ia);
            Z[4 * row + 2] = (double)__uint_as_float((unsigned)(mkey[r] >> 30));
            Z[4 * row + 3] = (double)(sz[a] + sz[b]);
            id[a] = n + row;
            sz[a] += sz[b];
            last = a;
        }
        *out_id = id[last];
        *out_rep = rep[last];
        *out_sz = sz[last];
    }
    __syncthreads();
}

// level 1: complete linkage inside each cell (one CTA per cell)
__global__ void __launch_bounds__(kDbThreads) dbht_l1_kernel(DbWork w, const float *D,
                                                             long long ldd, double *Z)
{
    if (*w.status) return;
    for (int b = blockIdx.x; b < w.nb; b += gridDim.x) {
        const int beg = w.cell_beg[b], m = w.cell_beg[b + 1] - beg;
        if (m == 0) continue;
        if (m == 1) {
            if (threadIdx.x == 0) {
                const int v = w.cell_list[beg];
                w.cid[b] = v;
                w.crep[b] = v;
                w.csz[b] = 1;
            }
            continue;
        }
        float *dm = w.dm + w.dm_off1[b];
        int *id = w.items_id + beg, *rep = w.items_rep + beg, *sz = w.items_sz + beg;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const int v = w.cell_list[beg + i];
            id[i] = v;
            rep[i] = v;
            sz[i] = 1;
            for (int j = 0; j < m; ++j)
                dm[(long long)i * m + j] = i == j ? 0.0f : dsym(D, ldd, v, w.cell_list[beg + j]);
        }
        __syncthreads();
        linkage_cta(m, dm, id, rep, sz, w.rowkey + beg, w.rowbest + beg, w.alive + beg, w.n,
                    w.l1_off[b], Z, w.status, &w.cid[b], &w.crep[b], &w.csz[b], nullptr, 0);
    }
}

// Level-2 and level-3 cluster distances in one pass over the upper triangle
// of D (row u, columns v > u, coalesced): a pair in one group but different
// cells raises that group's cell matrix, a pair in different groups the
// group matrix.  Maxima of non-negative floats as int bits; each row's
// maxima gather in shared memory first (global atomics when a group has too
// many cells or there are too many groups).  Only the (su, sv) entry is
// raised; the linkage kernels take max(M, M^T).
__global__ void __launch_bounds__(256) dbht_dist_kernel(DbWork w, const float *D, long long ldd)
{
    if (*w.status) return;
    __shared__ int gmax[kCapG];
    __shared__ int cmax[kCapC];
    const int n = w.n, nc = w.scal[0], ng = w.scal[3], t = threadIdx.x;
    int *dm3 = reinterpret_cast<int *>(w.dm + w.lscal[1]);
    const bool g_sm = nc <= kCapG;
    for (int u = blockIdx.x; u < n - 1; u += gridDim.x) {
        const int2 iu = w.vinfo[u];
        const int gu = iu.x, su = iu.y;
        const int mc = w.gcells_beg[gu + 1] - w.gcells_beg[gu];
        const bool c_sm = mc <= kCapC;
        int *row2 = reinterpret_cast<int *>(w.dm + w.dm_off2[gu]) + (long long)su * mc;
        int *row3 = dm3 + (long long)w.gslot[gu] * ng;
        if (g_sm)
            for (int c = t; c < nc; c += blockDim.x) gmax[c] = 0;
        if (c_sm)
            for (int i = t; i < mc; i += blockDim.x) cmax[i] = 0;
        __syncthreads();
        const float *Drow = D + (long long)u * ldd;
        for (int v = u + 1 + t; v < n; v += blockDim.x) {
            const int d = __float_as_int(Drow[v]);
            const int2 iv = w.vinfo[v];
            if (iv.x == gu) {
                if (iv.y != su) {
                    if (c_sm) {
                        if (d > cmax[iv.y]) atomicMax(&cmax[iv.y], d);
                    } else {
                        atomicMax(&row2[iv.y], d);
                    }
                }
            } else if (g_sm) {
                if (d > gmax[iv.x]) atomicMax(&gmax[iv.x], d);
            } else {
                atomicMax(&row3[w.gslot[iv.x]], d);
            }
        }
        __syncthreads();
        if (g_sm)
            for (int c = t; c < nc; c += blockDim.x)
                if (gmax[c] > 0) atomicMax(&row3[w.gslot[c]], gmax[c]);
        if (c_sm)
            for (int i = t; i < mc; i += blockDim.x)
                if (cmax[i] > 0) atomicMax(&row2[i], cmax[i]);
        __syncthreads();
    }
}

__device__ void symmetrize_max(float *dm, int m)
{
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        dm[(long long)i * m + i] = 0.0f;
        for (int j = i + 1; j < m; ++j) {
            const float x = fmaxf(dm[(long long)i * m + j], dm[(long long)j * m + i]);
            dm[(long long)i * m + j] = x;
            dm[(long long)j * m + i] = x;
        }
    }
    __syncthreads();
}

// level 2: complete linkage of the cells of each group (one CTA per group)
__global__ void __launch_bounds__(kDbThreads) dbht_l2_kernel(DbWork w, double *Z)
{
    extern __shared__ __align__(16) unsigned char lk_smem[];
    if (*w.status) return;
    const int nc = w.scal[0];
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        const int beg = w.gcells_beg[c], m = w.gcells_beg[c + 1] - beg;
        if (m == 0) continue;
        if (m == 1) {
            if (threadIdx.x == 0) {
                const int b = w.gcells[beg];
                w.gid[c] = w.cid[b];
                w.grep[c] = w.crep[b];
                w.gsz[c] = w.csz[b];
            }
            continue;
        }
        float *dm = w.dm + w.dm_off2[c];
        int *id = w.items_id + beg, *rep = w.items_rep + beg, *sz = w.items_sz + beg;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const int b = w.gcells[beg + i];
            id[i] = w.cid[b];
            rep[i] = w.crep[b];
            sz[i] = w.csz[b];
        }
        symmetrize_max(dm, m);
        if (m <= kChainMax)
            linkage_chain_cta(m, dm, id, rep, sz, w.n, w.l2_off[c], Z, w.status, &w.gid[c],
                              &w.grep[c], &w.gsz[c], lk_smem);
        else
            linkage_cta(m, dm, id, rep, sz, w.rowkey + beg, w.rowbest + beg, w.alive + beg, w.n,
                        w.l2_off[c], Z, w.status, &w.gid[c], &w.grep[c], &w.gsz[c], lk_smem,
                        kLkCap);
    }
}

// level 3: complete linkage of the groups (one CTA)
__global__ void __launch_bounds__(kDbThreads) dbht_l3_kernel(DbWork w, double *Z)
{
    extern __shared__ __align__(16) unsigned char lk_smem[];
    if (*w.status) return;
    __shared__ int s_id, s_rep, s_sz;
    const int nc = w.scal[0], ng = w.scal[3];
    float *dm = w.dm + w.lscal[1];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int s = w.gslot[c];
        if (s >= 0) {
            w.items_id[s] = w.gid[c];
            w.items_rep[s] = w.grep[c];
            w.items_sz[s] = w.gsz[c];
        }
    }
    symmetrize_max(dm, ng);
    if (ng >= 2 && ng <= kChainMax)
        linkage_chain_cta(ng, dm, w.items_id, w.items_rep, w.items_sz, w.n,
                          w.scal[1] + w.scal[2], Z, w.status, &s_id, &s_rep, &s_sz, lk_smem);
    else if (ng >= 2)
        linkage_cta(ng, dm, w.items_id, w.items_rep, w.items_sz, w.rowkey, w.rowbest, w.alive,
                    w.n, w.scal[1] + w.scal[2], Z, w.status, &s_id, &s_rep, &s_sz, lk_smem,
                    kLkCap);
}

// optional per-vertex / per-bubble outputs
__global__ void dbht_extra_kernel(DbWork w, int *direction, int *converging, int *group,
                                  int *bubble)
{
    if (*w.status) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) {
        if (direction && i >= 1 && i < w.nb) direction[i - 1] = w.dir[i];
        if (converging && i < w.nb) converging[i] = w.outdeg[i] == 0;
        if (group) group[i] = w.group[i];
        if (bubble) bubble[i] = w.bub[i];
    }
}

// Workspace carving; with base 0 it only measures.
struct Carver {
    uintptr_t base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        T *r = reinterpret_cast<T *>(base + off);
        off += (count * sizeof(T) + 255) & ~size_t(255);
        return r;
    }
};

long long dm_floats(int n) { return (long long)n * n + 4ll * n + 1024; }

DbWork carve(Carver &c, int n, int *status)
{
    const size_t nb = (size_t)n - 3, ne = 3 * (size_t)n - 6, nn = (size_t)n;
    DbWork w{};
    w.n = n;
    w.nb = (int)nb;
    w.status = status;
    w.bv = c.take<int>(4 * nb);
    w.intro = c.take<int>(nn);
    w.tin = c.take<int>(nb);
    w.tsz = c.take<int>(nb);
    w.rowptr = c.take<int>(nn + 1);
    w.cursor = c.take<int>(nn);
    w.adj = c.take<int2>(2 * ne);
    w.dir = c.take<int>(nb);
    w.outdeg = c.take<int>(nb);
    w.conv = c.take<int>(nb);
    w.gidx = c.take<int>(nb);
    w.group = c.take<int>(nn);
    w.hidx = c.take<int>(nb);
    w.glist = c.take<int>(nb);
    w.gbeg = c.take<int>(nb + 1);
    w.bub = c.take<int>(nn);
    w.cell_list = c.take<int>(nn);
    w.cell_beg = c.take<int>(nb + 1);
    w.bcnt = c.take<int>(nb);
    w.bcur = c.take<int>(nb);
    w.btmp = c.take<int>(nn);
    w.pos = c.take<int>(nb + 1);
    w.scal = c.take<int>(16);
    w.lscal = c.take<long long>(4);
    w.l1_off = c.take<int>(nb + 1);
    w.dm_off1 = c.take<long long>(nb + 1);
    w.cid = c.take<int>(nb);
    w.crep = c.take<int>(nb);
    w.csz = c.take<int>(nb);
    w.gcells_beg = c.take<int>(nb + 1);
    w.gcells = c.take<int>(nb);
    w.bslot = c.take<int>(nb);
    w.l2_off = c.take<int>(nb + 1);
    w.dm_off2 = c.take<long long>(nb + 1);
    w.gid = c.take<int>(nb);
    w.grep = c.take<int>(nb);
    w.gsz = c.take<int>(nb);
    w.gslot = c.take<int>(nb);
    w.vinfo = c.take<int2>(nn);
    w.items_id = c.take<int>(nn);
    w.items_rep = c.take<int>(nn);
    w.items_sz = c.take<int>(nn);
    w.rowkey = c.take<unsigned long long>(nn);
    w.rowbest = c.take<int>(nn);
    w.alive = c.take<int>(nn);
    w.dm_cap = dm_floats(n);
    w.dm = c.take<float>((size_t)w.dm_cap);
    return w;
}

}  // namespace

size_t dbht_smem_bytes(int n) { return 10 * (size_t)(n - 3); }

size_t dbht_work_bytes(int n)
{
    Carver c{0};
    carve(c, n, nullptr);
    return c.off;
}

int launch_dbht(const void *S, int n, long long ld, int dtype, const int *order, const int *edges,
                const int *ins_face, const int *parent, const float *D, long long ldd, double *Z,
                int *direction, int *converging, int *group, int *bubble, void *work, int *status,
                int num_sms, cudaStream_t stream)
{
    const int nb = n - 3, ne = 3 * n - 6;
    Carver c{reinterpret_cast<uintptr_t>(work)};
    DbWork w = carve(c, n, status);
    const int g = 4 * num_sms;
    const size_t tsm = dbht_smem_bytes(n);
    if (tsm > kSmemLimit) return TMFG_ETOOBIG;
    if (cudaFuncSetAttribute(dbht_tree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tsm) != cudaSuccess)
        return TMFG_ECUDA;
    // input checks (the permutation test counts in the cursor scratch)
    cudaMemsetAsync(w.cursor, 0, 4 * (size_t)n, stream);
    dbht_check_kernel<<<g, 256, 0, stream>>>(n, order, edges, ins_face, parent, w.cursor, status);
    // bubble tree and TMFG adjacency
    dbht_tree_kernel<<<1, 1024, tsm, stream>>>(w, order, ins_face, parent);
    int *deg = w.btmp;  // [n]
    cudaMemsetAsync(deg, 0, 4 * (size_t)n, stream);
    dbht_deg_kernel<<<g, 256, 0, stream>>>(edges, ne, deg, status);
    scan_kernel<<<1, 1024, 0, stream>>>(deg, n, w.rowptr, w.cursor, status);
    dbht_fill_kernel<<<g, 256, 0, stream>>>(edges, ne, w.cursor, w.adj, status);
    // directions and converging bubbles
    cudaMemsetAsync(w.outdeg, 0, 4 * (size_t)nb, stream);
    if (dtype == TMFG_F32)
        dbht_dir_kernel<float><<<g, 256, 0, stream>>>(w, static_cast<const float *>(S), ld, edges,
                                                      ins_face, parent);
    else
        dbht_dir_kernel<double><<<g, 256, 0, stream>>>(w, static_cast<const double *>(S), ld,
                                                       edges, ins_face, parent);
    dbht_conv_kernel<<<1, 1024, 0, stream>>>(w);
    // assignments
    dbht_group_kernel<<<g, 256, 0, stream>>>(w, D, ldd);
    dbht_home_kernel<<<g, 256, 0, stream>>>(w, D, ldd);
    // bubbles of each group
    cudaMemsetAsync(w.bcnt, 0, 4 * (size_t)nb, stream);
    bucket_count_kernel<<<g, 256, 0, stream>>>(w.hidx, nb, w.bcnt, status);
    scan_kernel<<<1, 1024, 0, stream>>>(w.bcnt, nb, w.gbeg, w.bcur, status);
    bucket_scatter_kernel<<<g, 256, 0, stream>>>(w.hidx, nb, w.bcur, w.btmp, status);
    bucket_order_kernel<<<g, 256, 0, stream>>>(w.hidx, nb, w.gbeg, w.btmp, w.glist, status);
    dbht_bubble_kernel<<<g, 256, 0, stream>>>(w, D, ldd);
    // vertices of each bubble
    cudaMemsetAsync(w.bcnt, 0, 4 * (size_t)nb, stream);
    bucket_count_kernel<<<g, 256, 0, stream>>>(w.bub, n, w.bcnt, status);
    scan_kernel<<<1, 1024, 0, stream>>>(w.bcnt, nb, w.cell_beg, w.bcur, status);
    bucket_scatter_kernel<<<g, 256, 0, stream>>>(w.bub, n, w.bcur, w.btmp, status);
    bucket_order_kernel<<<g, 256, 0, stream>>>(w.bub, n, w.cell_beg, w.btmp, w.cell_list, status);
    // the three linkage levels
    dbht_plan_kernel<<<1, 1024, 0, stream>>>(w);
    dbht_zero_kernel<<<g, 256, 0, stream>>>(w);
    dbht_l1_kernel<<<g, kDbThreads, 0, stream>>>(w, D, ldd, Z);
    dbht_dist_kernel<<<8 * num_sms, 256, 0, stream>>>(w, D, ldd);
    if (cudaFuncSetAttribute(dbht_l2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLkSmem) != cudaSuccess ||
        cudaFuncSetAttribute(dbht_l3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kLkSmem) != cudaSuccess)
        return TMFG_ECUDA;
    dbht_l2_kernel<<<g, kDbThreads, kLkSmem, stream>>>(w, Z);
    dbht_l3_kernel<<<1, kDbThreads, kLkSmem, stream>>>(w, Z);
    if (direction || converging || group || bubble)
        dbht_extra_kernel<<<g, 256, 0, stream>>>(w, direction, converging, group, bubble);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace tmfg
