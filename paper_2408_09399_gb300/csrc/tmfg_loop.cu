// tmfg_loop.cu -- the greedy TMFG insertion loop (Algorithm 1 corr-tmfg with
// prefix P, Algorithm 2 heap-tmfg), entirely on the device.
//
// One CTA runs the whole sequence of n-4 insertions with no host round trip.
// State:
//   shared  inserted bitmap, per-vertex lazy pointer ptr[w] into its sorted
//           row and the cached MaxCorrs Mc[w] = row[w][ptr[w]] (16-bit ids),
//           the stored best vertex fv[f] of each face, and a two-level max
//           index over the face keys: level 1 = max of each group of 32
//           faces, level 2 = max of each group of 32 level-1 nodes, then a
//           root; dirty groups are recomputed after each batch of updates;
//   global  the face triples and owners (int4), the per-face keys (leaves,
//           L2-resident), the sorted rows (from the row sort) and S.
// A face key is (gain desc, vertex asc, face id asc); with one entry per
// face, popping the max of Algorithm 2's heap is the argmax over the faces'
// stored keys, which is what the index returns.
//
// MaxCorrs[w] is read fresh (Algorithm 1 recomputes it for every vertex of
// an updated face before reading it; Algorithm 2 likewise for the vertices
// of the face it just popped or created): the cached Mc[w] is valid while it
// is uninserted, else one warp scans row w from ptr[w]+1 with 16-byte loads
// (256 entries per step) and a ballot over the inserted bitmap (the pointer
// of Section 4.3, vectorised across a warp instead of AVX lanes).
//
// A face's best vertex is computed by one warp: 9 lanes gather S[x,u] for
// the 3 candidates u x 3 face vertices x; gain = (S[a,u] + S[b,u]) + S[c,u]
// with round-to-nearest adds in the dtype of S; ties go to the smaller u.
//
// The loop checks the device clock every iteration and stops with
// TMFG_ETIMEOUT past its limit, so it always terminates.
#include <climits>

#include "internal.cuh"

namespace tmfg {

constexpr int kLoopThreads = 256;
constexpr int kLoopWarps = kLoopThreads / kWarp;
constexpr int kChunk = 256;    // faces per recompute batch
constexpr int kMaxPrefix = 256;

struct Node {
    unsigned long long gk;  // order-preserving image of the gain (0 = empty)
    int v;
    int f;
};

__device__ __forceinline__ bool above(const Node &a, const Node &b)
{
    if (a.gk != b.gk) return a.gk > b.gk;
    if (a.v != b.v) return a.v < b.v;
    return a.f < b.f;
}

__device__ __forceinline__ Node node_empty() { return Node{0ull, INT_MAX, INT_MAX}; }

__device__ __forceinline__ Node warp_max(Node x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Node y;
        y.gk = __shfl_xor_sync(0xffffffffu, x.gk, o);
        y.v = __shfl_xor_sync(0xffffffffu, x.v, o);
        y.f = __shfl_xor_sync(0xffffffffu, x.f, o);
        if (above(y, x)) x = y;
    }
    return x;
}

// Shared-memory layout (dynamic part), computed identically on the host.
struct LoopLayout {
    int W;      // words of an n-bit bitmap
    int nfmax;  // 2n-4
    int G1, G2; // level-1 / level-2 node counts
    size_t off_ins, off_vmark, off_round, off_mc, off_ptr, off_fv, off_l1, off_l2, off_d1bits,
        off_d2bits, off_d1list, off_d2list, off_vlist, off_flist, off_sel, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline LoopLayout loop_layout(int n)
{
    LoopLayout L;
    L.W = (n + 31) / 32;
    L.nfmax = 2 * n - 4;
    L.G1 = (L.nfmax + 31) / 32;
    L.G2 = (L.G1 + 31) / 32;
    size_t o = 0;
    L.off_ins = o;    o = align16(o + 4 * (size_t)L.W);
    L.off_vmark = o;  o = align16(o + 4 * (size_t)L.W);
    L.off_round = o;  o = align16(o + 4 * (size_t)L.W);
    L.off_mc = o;     o = align16(o + 2 * (size_t)n);
    L.off_ptr = o;    o = align16(o + 2 * (size_t)n);
    L.off_fv = o;     o = align16(o + 2 * (size_t)L.nfmax);
    L.off_l1 = o;     o = align16(o + sizeof(Node) * (size_t)L.G1);
    L.off_l2 = o;     o = align16(o + sizeof(Node) * (size_t)L.G2);
    L.off_d1bits = o; o = align16(o + 4 * (size_t)((L.G1 + 31) / 32));
    L.off_d2bits = o; o = align16(o + 4 * (size_t)((L.G2 + 31) / 32));
    L.off_d1list = o; o = align16(o + 2 * (size_t)L.G1);
    L.off_d2list = o; o = align16(o + 2 * (size_t)L.G2);
    L.off_vlist = o;  o = align16(o + 4 * (size_t)(3 * kChunk));
    L.off_flist = o;  o = align16(o + 4 * (size_t)4);
    L.off_sel = o;    o = align16(o + sizeof(Node) * (size_t)kMaxPrefix);
    L.total = o;
    return L;
}

template <typename T>
struct Loop {
    const LoopArgs &a;
    const T *S;
    int n;
    uint32_t *ins, *vmark, *rnd, *d1bits, *d2bits;
    uint16_t *mc, *ptr, *fv, *d1list, *d2list;
    Node *l1, *l2, *sel;
    int *vlist, *flist;
    int G1, G2;
    // scalars (static shared)
    Node *root;
    int *nf, *k, *vcount, *nd1, *nd2, *scan_chunks, *face_evals;

    __device__ bool is_ins(int v) const { return (ins[v >> 5] >> (v & 31)) & 1u; }

    __device__ void mark_d1(int g)
    {
        const uint32_t bit = 1u << (g & 31);
        if (!(atomicOr(&d1bits[g >> 5], bit) & bit)) d1list[atomicAdd(nd1, 1)] = (uint16_t)g;
    }
    __device__ void mark_d2(int g)
    {
        const uint32_t bit = 1u << (g & 31);
        if (!(atomicOr(&d2bits[g >> 5], bit) & bit)) d2list[atomicAdd(nd2, 1)] = (uint16_t)g;
    }

    // Fresh MaxCorrs of vertex w (one warp): keep Mc[w] while uninserted,
    // else advance ptr[w] to the first uninserted entry of row w.
    __device__ void refresh(int w)
    {
        const int lane = threadIdx.x & 31;
        const uint16_t m = mc[w];
        if (m == kNone16 || !is_ins(m)) return;
        const int mlen = n - 1;
        const uint16_t *row = a.idx + (long long)w * a.ldi;
        int p = ptr[w] + 1;
        while (p < mlen) {
            const int base = p & ~7;
            const int q0 = base + lane * 8;
            int first = 8;
            uint16_t e[8] = {kNone16, kNone16, kNone16, kNone16, kNone16, kNone16, kNone16, kNone16};
            if (q0 < a.ldi) {
                const uint4 c = *reinterpret_cast<const uint4 *>(row + q0);
                e[0] = c.x & 0xFFFF; e[1] = c.x >> 16; e[2] = c.y & 0xFFFF; e[3] = c.y >> 16;
                e[4] = c.z & 0xFFFF; e[5] = c.z >> 16; e[6] = c.w & 0xFFFF; e[7] = c.w >> 16;
#pragma unroll
                for (int t = 7; t >= 0; --t) {
                    const int q = q0 + t;
                    if (q >= p && q < mlen && e[t] < n && !is_ins(e[t])) first = t;
                }
            }
            if (lane == 0) atomicAdd(scan_chunks, 1);
            const unsigned bal = __ballot_sync(0xffffffffu, first < 8);
            if (bal) {
                const int src = __ffs(bal) - 1;
                const int t = __shfl_sync(0xffffffffu, first, src);
                uint16_t hit = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (u == t) hit = e[u];
                hit = (uint16_t)__shfl_sync(0xffffffffu, (int)hit, src);
                if (lane == 0) {
                    ptr[w] = (uint16_t)(base + src * 8 + t);
                    mc[w] = hit;
                }
                __syncwarp();
                return;
            }
            p = base + 256;
        }
        if (lane == 0) {
            ptr[w] = (uint16_t)mlen;
            mc[w] = kNone16;
        }
        __syncwarp();
    }

    // Best vertex of face f from the fresh MaxCorrs of its vertices (one warp).
    __device__ void face_best(int f)
    {
        const int lane = threadIdx.x & 31;
        const int4 fc = a.face[f];
        const int m0 = mc[fc.x], m1 = mc[fc.y], m2 = mc[fc.z];
        const int ci = lane / 3, cj = lane - 3 * (lane / 3);
        T val = T(0);
        if (lane < 9) {
            const int cand = ci == 0 ? m0 : (ci == 1 ? m1 : m2);
            const int fx = cj == 0 ? fc.x : (cj == 1 ? fc.y : fc.z);
            if (cand != kNone16 && cand < n) val = canon(S[(long long)fx * a.ld + cand]);
        }
        const int l3 = (3 * lane) & 31;
        const T x0 = shfl(val, l3), x1 = shfl(val, (l3 + 1) & 31), x2 = shfl(val, (l3 + 2) & 31);
        const T g = canon(add_rn(add_rn(x0, x1), x2));
        const T g1 = shfl(g, 1), g2 = shfl(g, 2);
        if (lane == 0) {
            int bv = -1;
            T bg = T(0);
            const int cs[3] = {m0, m1, m2};
            const T gs[3] = {g, g1, g2};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const int c = cs[i];
                if (c == kNone16 || c >= n) continue;
                if (bv < 0 || gs[i] > bg || (gs[i] == bg && c < bv)) { bv = c; bg = gs[i]; }
            }
            if (bv < 0) {
                a.leaf_gk[f] = 0ull;
                a.leaf_v[f] = INT_MAX;
                fv[f] = kNone16;
            } else {
                a.leaf_gk[f] = (unsigned long long)ord_key(bg);
                a.leaf_v[f] = bv;
                fv[f] = (uint16_t)bv;
            }
            atomicAdd(face_evals, 1);
            mark_d1(f >> 5);
        }
        __syncwarp();
    }

    // Recompute the faces of list[0..cnt) (list in shared or global memory).
    __device__ void recompute(const int *list, int cnt)
    {
        const int tid = threadIdx.x, warp = tid >> 5;
        for (int c0 = 0; c0 < cnt; c0 += kChunk) {
            const int m = cnt - c0 < kChunk ? cnt - c0 : kChunk;
            if (tid == 0) *vcount = 0;
            __syncthreads();
            for (int i = tid; i < m; i += kLoopThreads) {
                const int4 fc = a.face[list[c0 + i]];
                const int vs[3] = {fc.x, fc.y, fc.z};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int w = vs[j];
                    const uint32_t bit = 1u << (w & 31);
                    if (!(atomicOr(&vmark[w >> 5], bit) & bit)) vlist[atomicAdd(vcount, 1)] = w;
                }
            }
            __syncthreads();
            const int nv = *vcount;
            for (int i = warp; i < nv; i += kLoopWarps) refresh(vlist[i]);
            __syncthreads();
            for (int i = tid; i < nv; i += kLoopThreads) {
                const int w = vlist[i];
                atomicAnd(&vmark[w >> 5], ~(1u << (w & 31)));
            }
            for (int i = warp; i < m; i += kLoopWarps) face_best(list[c0 + i]);
            __syncthreads();
        }
    }

    // Bring the max index up to date after leaf writes (ends synchronised).
    __device__ void tree_update()
    {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int nfc = *nf;
        const int c1 = *nd1;
        for (int i = warp; i < c1; i += kLoopWarps) {
            const int g = d1list[i];
            const int f = g * 32 + lane;
            Node x = node_empty();
            if (f < nfc) {
                x.gk = a.leaf_gk[f];
                x.v = a.leaf_v[f];
                x.f = f;
                if (x.gk == 0ull) x = node_empty();
            }
            x = warp_max(x);
            if (lane == 0) {
                l1[g] = x;
                atomicAnd(&d1bits[g >> 5], ~(1u << (g & 31)));
                mark_d2(g >> 5);
            }
        }
        __syncthreads();
        const int c2 = *nd2;
        for (int i = warp; i < c2; i += kLoopWarps) {
            const int g = d2list[i];
            const int j = g * 32 + lane;
            Node x = j < G1 ? l1[j] : node_empty();
            x = warp_max(x);
            if (lane == 0) {
                l2[g] = x;
                atomicAnd(&d2bits[g >> 5], ~(1u << (g & 31)));
            }
        }
        __syncthreads();
        if (warp == 0) {
            Node x = lane < G2 ? l2[lane] : node_empty();
            Node y = lane + 32 < G2 ? l2[lane + 32] : node_empty();
            if (above(y, x)) x = y;
            x = warp_max(x);
            if (lane == 0) {
                *root = x;
                *nd1 = 0;
                *nd2 = 0;
            }
        }
        __syncthreads();
    }

    // Thread 0 only: insert v into face f (Algorithm 1/2 insertion step);
    // writes the outputs and the 3 new faces; returns their ids in out3.
    __device__ void insert_pair(int v, int f, int *out3)
    {
        const int4 fc = a.face[f];
        const int x = fc.x, y = fc.y, z = fc.z;
        const int kk = *k;
        const int nfc = *nf;
        a.order[4 + kk] = v;
        int *e = a.edges + 2 * (6 + 3 * kk);
        e[0] = v; e[1] = x; e[2] = v; e[3] = y; e[4] = v; e[5] = z;
        a.ins_face[3 * kk + 0] = x;
        a.ins_face[3 * kk + 1] = y;
        a.ins_face[3 * kk + 2] = z;
        a.parent[kk + 1] = fc.w;
        ins[v >> 5] |= 1u << (v & 31);
        const int bub = kk + 1;
        auto sorted = [&](int p, int q, int r) {
            int t;
            if (p > q) { t = p; p = q; q = t; }
            if (q > r) { t = q; q = r; r = t; }
            if (p > q) { t = p; p = q; q = t; }
            return make_int4(p, q, r, bub);
        };
        a.face[f] = sorted(v, x, y);
        a.face[nfc] = sorted(v, y, z);
        a.face[nfc + 1] = sorted(v, x, z);
        fv[nfc] = kNone16;
        fv[nfc + 1] = kNone16;
        out3[0] = f;
        out3[1] = nfc;
        out3[2] = nfc + 1;
        *nf = nfc + 2;
        *k = kk + 1;
    }
};

template <typename T>
__global__ void __launch_bounds__(kLoopThreads, 1) tmfg_loop_kernel(LoopArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Node s_root;
    __shared__ int s_nf, s_k, s_vcount, s_nd1, s_nd2, s_scan, s_evals, s_stop, s_nsel, s_fcount;
    __shared__ int s_clique[4];
    __shared__ unsigned long long s_red_r[kLoopWarps];
    __shared__ int s_red_i[kLoopWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.n;
    if (*(volatile int *)a.status != 0) return;  // an earlier step failed
    const uint64_t t0 = globaltimer_ns();
    const LoopLayout L = loop_layout(n);

    Loop<T> st{a};
    st.S = reinterpret_cast<const T *>(a.S);
    st.n = n;
    st.ins = reinterpret_cast<uint32_t *>(smem + L.off_ins);
    st.vmark = reinterpret_cast<uint32_t *>(smem + L.off_vmark);
    st.rnd = reinterpret_cast<uint32_t *>(smem + L.off_round);
    st.mc = reinterpret_cast<uint16_t *>(smem + L.off_mc);
    st.ptr = reinterpret_cast<uint16_t *>(smem + L.off_ptr);
    st.fv = reinterpret_cast<uint16_t *>(smem + L.off_fv);
    st.l1 = reinterpret_cast<Node *>(smem + L.off_l1);
    st.l2 = reinterpret_cast<Node *>(smem + L.off_l2);
    st.d1bits = reinterpret_cast<uint32_t *>(smem + L.off_d1bits);
    st.d2bits = reinterpret_cast<uint32_t *>(smem + L.off_d2bits);
    st.d1list = reinterpret_cast<uint16_t *>(smem + L.off_d1list);
    st.d2list = reinterpret_cast<uint16_t *>(smem + L.off_d2list);
    st.vlist = reinterpret_cast<int *>(smem + L.off_vlist);
    st.flist = reinterpret_cast<int *>(smem + L.off_flist);
    st.sel = reinterpret_cast<Node *>(smem + L.off_sel);
    st.G1 = L.G1;
    st.G2 = L.G2;
    st.root = &s_root;
    st.nf = &s_nf;
    st.k = &s_k;
    st.vcount = &s_vcount;
    st.nd1 = &s_nd1;
    st.nd2 = &s_nd2;
    st.scan_chunks = &s_scan;
    st.face_evals = &s_evals;

    // ---- initial state
    for (int i = tid; i < L.W; i += kLoopThreads) { st.ins[i] = 0; st.vmark[i] = 0; st.rnd[i] = 0; }
    for (int w = tid; w < n; w += kLoopThreads) {
        st.ptr[w] = 0;
        const uint16_t m0 = a.idx[(long long)w * a.ldi];
        st.mc[w] = m0 < n ? m0 : kNone16;
    }
    for (int f = tid; f < L.nfmax; f += kLoopThreads) st.fv[f] = kNone16;
    for (int g = tid; g < L.G1; g += kLoopThreads) st.l1[g] = node_empty();
    for (int g = tid; g < L.G2; g += kLoopThreads) st.l2[g] = node_empty();
    for (int i = tid; i < (L.G1 + 31) / 32; i += kLoopThreads) st.d1bits[i] = 0;
    for (int i = tid; i < (L.G2 + 31) / 32; i += kLoopThreads) st.d2bits[i] = 0;
    if (tid == 0) {
        s_nf = 4; s_k = 0; s_vcount = 0; s_nd1 = 0; s_nd2 = 0; s_scan = 0; s_evals = 0;
        s_stop = 0; s_nsel = 0; s_fcount = 0;
    }
    __syncthreads();

    // ---- initial 4-clique: top four row sums (r desc, id asc)
    for (int c = 0; c < 4; ++c) {
        long long br = LLONG_MIN;
        int bi = INT_MAX;
        for (int v = tid; v < n; v += kLoopThreads) {
            bool taken = false;
            for (int j = 0; j < c; ++j) taken |= (s_clique[j] == v);
            if (taken) continue;
            const long long r = a.rowsum[v];
            if (r > br || (r == br && v < bi)) { br = r; bi = v; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long r2 = __shfl_xor_sync(0xffffffffu, br, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (r2 > br || (r2 == br && i2 < bi)) { br = r2; bi = i2; }
        }
        if (lane == 0) { s_red_r[warp] = (unsigned long long)br; s_red_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            long long r = (long long)s_red_r[0];
            int i = s_red_i[0];
            for (int w = 1; w < kLoopWarps; ++w) {
                const long long r2 = (long long)s_red_r[w];
                const int i2 = s_red_i[w];
                if (r2 > r || (r2 == r && i2 < i)) { r = r2; i = i2; }
            }
            s_clique[c] = i;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int *c = s_clique;
        for (int i = 0; i < 4; ++i) {
            a.order[i] = c[i];
            st.ins[c[i] >> 5] |= 1u << (c[i] & 31);
        }
        const int pr[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        for (int i = 0; i < 6; ++i) {
            a.edges[2 * i] = c[pr[i][0]];
            a.edges[2 * i + 1] = c[pr[i][1]];
        }
        a.parent[0] = -1;
        const int tri[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
        for (int f = 0; f < 4; ++f) {
            int p = c[tri[f][0]], q = c[tri[f][1]], r = c[tri[f][2]], t;
            if (p > q) { t = p; p = q; q = t; }
            if (q > r) { t = q; q = r; r = t; }
            if (p > q) { t = p; p = q; q = t; }
            a.face[f] = make_int4(p, q, r, 0);
            st.flist[f] = f;
        }
    }
    __syncthreads();
    st.recompute(st.flist, 4);
    st.tree_update();

    // ---- main loop
    const int total = n - 4;
    long long stale = 0, rounds = 0;
    while (s_k < total) {
        if (tid == 0 && globaltimer_ns() - t0 > a.timeout_ns) s_stop = TMFG_ETIMEOUT;
        __syncthreads();
        if (s_stop) break;
        if (a.mode == TMFG_HEAP) {
            const Node r = s_root;
            if (r.gk == 0ull || r.v >= n || r.f >= s_nf) {
                if (tid == 0) s_stop = TMFG_EINTERNAL;
                __syncthreads();
                break;
            }
            if (st.is_ins(r.v)) {
                // stale pair: recompute this face alone and re-push it
                ++stale;
                if (tid == 0) st.flist[0] = r.f;
                __syncthreads();
                st.recompute(st.flist, 1);
                st.tree_update();
                continue;
            }
            if (tid == 0) st.insert_pair(r.v, r.f, st.flist);
            __syncthreads();
            ++rounds;
            st.recompute(st.flist, 3);
            st.tree_update();
        } else {
            // L = the P best pairs (repeated extraction from the max index)
            if (tid == 0) s_nsel = 0;
            __syncthreads();
            for (int i = 0; i < a.P; ++i) {
                const Node r = s_root;
                if (r.gk == 0ull) break;
                if (tid == 0) {
                    st.sel[s_nsel++] = r;
                    if (a.P > 1) {
                        a.leaf_gk[r.f] = 0ull;
                        a.leaf_v[r.f] = INT_MAX;
                        st.mark_d1(r.f >> 5);
                    }
                }
                __syncthreads();
                if (a.P == 1) break;
                st.tree_update();
            }
            const int nsel = s_nsel;
            if (nsel == 0) {
                if (tid == 0) s_stop = TMFG_EINTERNAL;
                __syncthreads();
                break;
            }
            const int nf_old = s_nf;
            if (tid == 0) {
                // keep the first (best) pair of each vertex, insert in rank order
                int out3[3];
                for (int i = 0; i < nsel; ++i) {
                    const int v = st.sel[i].v;
                    if (v >= n) {
                        s_stop = TMFG_EINTERNAL;
                        continue;
                    }
                    if (st.is_ins(v)) {
                        // a later pair of a vertex kept this round; any other
                        // inserted vertex breaks the corr-tmfg invariant
                        if (!((st.rnd[v >> 5] >> (v & 31)) & 1u)) s_stop = TMFG_EINTERNAL;
                        continue;
                    }
                    st.rnd[v >> 5] |= 1u << (v & 31);
                    st.insert_pair(v, st.sel[i].f, out3);
                }
                s_fcount = 0;
            }
            __syncthreads();
            if (s_stop) break;
            ++rounds;
            // F_update: faces whose stored vertex was inserted this round,
            // and the appended faces
            const int nf_new = s_nf;
            for (int f = tid; f < nf_old; f += kLoopThreads) {
                const int v = st.fv[f];
                if (v != kNone16 && ((st.rnd[v >> 5] >> (v & 31)) & 1u))
                    a.fu_buf[atomicAdd(&s_fcount, 1)] = f;
            }
            for (int f = nf_old + tid; f < nf_new; f += kLoopThreads)
                a.fu_buf[atomicAdd(&s_fcount, 1)] = f;
            __syncthreads();
            st.recompute(a.fu_buf, s_fcount);
            if (tid == 0)
                for (int i = 0; i < nsel; ++i) {
                    const int v = st.sel[i].v;
                    if (v < n) st.rnd[v >> 5] &= ~(1u << (v & 31));
                }
            st.tree_update();
        }
    }
    if (tid == 0) {
        if (s_stop) set_status(a.status, s_stop);
        a.stats[0] = s_evals;
        a.stats[1] = stale;
        a.stats[2] = s_scan;
        a.stats[3] = rounds;
        a.stats[4] = (long long)(globaltimer_ns() - t0);
    }
}

size_t loop_smem_bytes(int n) { return loop_layout(n).total; }

int launch_loop(const LoopArgs &args, int dtype, cudaStream_t stream)
{
    const size_t smem = loop_smem_bytes(args.n);
    if (smem > 232448) return TMFG_ETOOBIG;
    if (dtype == TMFG_F32) {
        auto k = tmfg_loop_kernel<float>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return TMFG_ECUDA;
        k<<<1, kLoopThreads, smem, stream>>>(args);
    } else {
        auto k = tmfg_loop_kernel<double>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return TMFG_ECUDA;
        k<<<1, kLoopThreads, smem, stream>>>(args);
    }
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace tmfg
