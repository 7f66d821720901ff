// loop_cluster.cu -- the insertion loop of corr-tmfg with prefix 1 (Algorithm
// 1 with P = 1: every round inserts the single best face-vertex pair) on a
// thread-block cluster of C CTAs, one per SM, that share one insertion at a
// time through distributed shared memory.
//
// Why a cluster.  One insertion is a short chain of dependent steps (find the
// faces whose stored vertex is the inserted v, refresh the sorted-row
// pointers that v made stale, gather S for the faces' candidates, update a
// max index).  On one SM every step also pays for work proportional to the
// whole face set (scans of the stored vertices) and for hundreds of scattered
// loads issued by one SM.  Split over C SMs, each step does 1/C of that work,
// and the C partial maxima meet once per insertion.
//
// Ownership.  Face f belongs to CTA f mod C (local index f / C): its record
// {x, y, z, creating bubble}, its stored best vertex and its key live in that
// CTA's shared memory, with a one-level max index (groups of 32 keys) over
// them.  Row w belongs to CTA w mod C.  Every CTA holds a replica of the
// inserted-vertex bitmap and of every row's pointer word (ptr << 16 | Mc).
//
// Pointers (Section 4.3, MaxCorrs read fresh).  The owner keeps the word of
// every inserted row fresh: inserting v makes stale exactly the inserted rows
// whose Mc is v (and v's own row if its Mc was inserted earlier), so at each
// insertion every CTA scans the Mc of its own rows for v, refreshes the ones
// it finds and stores each new word into every CTA's replica.  A CTA that
// evaluates a face whose vertex's word is still stale in its replica waits
// for the owner's store (a bounded poll of its own shared memory) and
// refreshes its replica itself if the bound runs out.  Every word is valid at
// all times (Mc is the id at position ptr, every id before ptr is inserted),
// so neither path can give a wrong Mc.
//
// One insertion (all 256 threads of every CTA):
//  A. read the C slots that the last cluster barrier published (each CTA's
//     best pair and its face's record); the best of them is (v, t).
//  B. the owner of t rewrites it as {v,x,y}; the owners of faces nf, nf+1
//     write {v,y,z} and {v,x,z}; every CTA scans the Mc of its rows for v
//     (the rows to refresh).                                       -- barrier
//  C. groups of PL lanes refresh the listed rows (steps of PL x 8 sorted
//     ids) and store the new words into every CTA; meanwhile the warps with
//     no row scan the stored vertices of the CTA's faces for v (the faces
//     to recompute).                                               -- barrier
//  D. one thread per listed face: the fresh Mc of its three vertices, 9
//     gathers of S, gain (S[a,u] + S[b,u]) + S[c,u] in the dtype of S, ties
//     to the smaller u, the best pair's key into its leaf.         -- barrier
//  E. a warp per touched group: the group's maximum.               -- barrier
//  F. warp 0: the CTA's best pair and its face record into slot k+1 of every
//     CTA of the cluster; then a cluster barrier (release / acquire).
// Within an insertion v counts as inserted in every check; its bit is set
// after E, so no thread sees the bitmap change before the cluster barrier.
// Every CTA reads the same slots, so every CTA takes the same decisions,
// including leaving the loop (time limit, bad pair); the barriers therefore
// always match.  The only poll (D) is bounded and has a fallback.
//
// Segments.  Like the other loop kernels the build runs in segments with the
// sorted rows compacted in between; the state format in global memory is the
// one of loop_common.cuh (inserted bitmap, ptr, Mc, stored vertices) plus the
// face records and keys in the build's face and leaf arrays.
#include <cooperative_groups.h>

#include "loop_common.cuh"

namespace cg = cooperative_groups;

namespace tmfg {

constexpr int kClThreads = 256;
constexpr int kClWaitPolls = 1 << 16;  // polls of a stale word before refreshing it locally

// One CTA's best pair and its face record, stored into every CTA with one
// 16-byte store (float keys; two for double keys).  The bubble takes 15 bits
// (n <= 32770).
template <class Key>
struct alignas(16) ClSlot {
    Key key;      // the CTA's best pair (empty: none)
    uint32_t xy;  // its face's vertices x | y << 16 (x < y < z)
    uint32_t zb;  // z | creating bubble << 16 | time limit passed (CTA 0) << 31
};

struct ClLayout {
    int C, NL, NL8, G1L, W, n8, NR, NR8;
    size_t off_ins, off_mco, off_pm, off_frec, off_fv, off_leaf, off_l1, off_b1, off_q1,
        off_flist, off_rows, off_slot, total;
};

// Shared-memory layout of one CTA (dynamic part), computed identically on the
// host.  ks = key bytes; a slot is 16 bytes (float keys) or 32 (double).
__host__ __device__ inline ClLayout cl_layout(int n, int C, size_t ks)
{
    ClLayout L;
    L.C = C;
    const int nfmax = 2 * n - 4;
    L.NL = (nfmax + C - 1) / C;
    L.NL8 = (L.NL + 7) & ~7;
    L.G1L = (L.NL + 31) / 32;
    L.W = (n + 31) / 32;
    L.n8 = (n + 7) & ~7;
    L.NR = (n + C - 1) / C;
    L.NR8 = (L.NR + 7) & ~7;
    size_t o = 0;
    L.off_ins = o;   o = align16(o + 4 * (size_t)L.W);
    L.off_mco = o;   o = align16(o + 2 * (size_t)L.NR8);
    L.off_pm = o;    o = align16(o + 4 * (size_t)L.n8);
    L.off_frec = o;  o = align16(o + 8 * (size_t)L.NL);
    L.off_fv = o;    o = align16(o + 2 * (size_t)L.NL8);
    L.off_leaf = o;  o = align16(o + ks * (size_t)L.NL);
    L.off_l1 = o;    o = align16(o + ks * (size_t)L.G1L);
    L.off_b1 = o;    o = align16(o + 4 * (size_t)((L.G1L + 31) / 32));
    L.off_q1 = o;    o = align16(o + 2 * (size_t)L.G1L);
    L.off_flist = o; o = align16(o + 2 * (size_t)L.NL8);
    L.off_rows = o;  o = align16(o + 2 * (size_t)L.NR8);  // each own row at most once
    L.off_slot = o;  o = align16(o + 2 * (size_t)C * (ks == 8 ? 16 : 32));
    L.total = o;
    return L;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\t"
                 "barrier.cluster.wait.acquire;" ::: "memory");
}

// x | y << 16, z | bub << 16 of the face {p, q, s} (any order) made by bubble bub
__device__ __forceinline__ uint2 face_record(int p, int q, int s, int bub)
{
    int t;
    if (p > q) { t = p; p = q; q = t; }
    if (q > s) { t = q; q = s; s = t; }
    if (p > q) { t = p; p = q; q = t; }
    return make_uint2((uint32_t)p | ((uint32_t)q << 16), (uint32_t)s | ((uint32_t)bub << 16));
}

// One thread's refresh of a CTA's replica `word` of a sorted row, when the
// owner's word did not arrive within the poll bound (out of line: the path is
// rare and its loop would otherwise be copied into every face evaluation).
// The word is read again first: the owner's store may have landed meanwhile.
__device__ __noinline__ uint32_t cl_refresh_thread(const uint16_t *row, const uint32_t *ins,
                                                   uint32_t *word, int n, int cur_v)
{
    auto inserted = [&](int u) { return u == cur_v || ((ins[u >> 5] >> (u & 31)) & 1u); };
    const int mlen = n - 1;
    const uint32_t w0 = *(volatile const uint32_t *)word;
    const int m0 = (int)(w0 & 0xFFFFu);
    if (m0 == kNone16 || !inserted(m0)) return w0;
    int p = (int)(w0 >> 16) + 1;
    int fq = mlen, fe = kNone16;
    while (p < mlen) {
        const int base = p & ~7;  // base + 8 <= ldi: both multiples of 8, base < n - 1
        const uint4 c = *reinterpret_cast<const uint4 *>(row + base);
        const uint32_t wd[4] = {c.x, c.y, c.z, c.w};
        bool done = false;
        for (int t = 0; t < 8 && !done; ++t) {
            const int q = base + t;
            if (q < p) continue;
            const int e = (wd[t >> 1] >> (16 * (t & 1))) & 0xFFFF;
            if (q >= mlen || e >= n) {
                fq = q < mlen ? q : mlen;
                done = true;
            } else if (!inserted(e)) {
                fq = q;
                fe = e;
                done = true;
            }
        }
        if (done) break;
        p = base + 8;
    }
    const uint32_t nw = ((uint32_t)fq << 16) | (uint32_t)fe;
    atomicMax(word, nw);
    return nw;
}

template <typename T, int C, int PL>
struct ClLoop {
    using KO = KeyOps<T>;
    using Key = typename KO::Key;
    static constexpr int NT = kClThreads, NW = NT / kWarp, NG = NT / PL;
    static_assert(PL >= 1 && PL <= 32 && (PL & (PL - 1)) == 0, "PL: a power of two <= 32");
    static_assert(sizeof(ClSlot<Key>) % 16 == 0, "a slot is whole 16-byte words");

    const LoopArgs &a;
    const T *S;
    int n, r, NL, NR, G1L;
    uint32_t *ins, *pm, *b1;
    uint2 *frec;
    uint16_t *mco, *fv, *flist, *rows, *q1;
    Key *leaf, *l1;
    ClSlot<Key> *slot;  // [2][C]
    int *fcount, *rcount, *n1;
    // the vertex being inserted: inserted for every check of this insertion,
    // although its bit is set only at its end
    int cur_v = -1;
    // this thread's counters
    long long c_rows = 0, c_cont = 0, c_steps = 0, c_evals = 0, c_wait = 0, c_slow = 0;

    __device__ bool is_ins(int u) const { return (ins[u >> 5] >> (u & 31)) & 1u; }
    __device__ static int mc_of(uint32_t w) { return (int)(w & 0xFFFFu); }
    __device__ static int ptr_of(uint32_t w) { return (int)(w >> 16); }
    __device__ static bool same(const Key &x, const Key &y) { return !KO::gt(x, y) && !KO::gt(y, x); }
    __device__ bool inserted(int u) const { return u == cur_v || is_ins(u); }
    // a word is stale when its Mc was inserted (the row's end is never stale)
    __device__ bool stale(uint32_t w) const { return mc_of(w) != kNone16 && inserted(mc_of(w)); }
    __device__ uint32_t word_at(int w) const { return *(volatile const uint32_t *)(pm + w); }

    // The entries of one 16-byte load (8 ids) equal to v, as bits 0..7.
    __device__ static uint32_t match8(const uint4 &q, uint32_t vv)
    {
        const uint32_t m0 = __vcmpeq2(q.x, vv), m1 = __vcmpeq2(q.y, vv);
        const uint32_t m2 = __vcmpeq2(q.z, vv), m3 = __vcmpeq2(q.w, vv);
        return (m0 & 1u) | ((m0 >> 15) & 2u) | ((m1 & 1u) << 2) | ((m1 >> 13) & 8u) |
               ((m2 & 1u) << 4) | ((m2 >> 11) & 32u) | ((m3 & 1u) << 6) | ((m3 >> 9) & 128u);
    }

    // Every index i < count of a 16-bit array (16-byte aligned, padded to a
    // multiple of 8 entries) whose entry is v: on_hit(i), by `stride` threads
    // (g = this thread's index among them).  Two 16-byte loads (16 entries)
    // in flight per thread; the matches become one bit mask, handled by a
    // single copy of on_hit (the loop runs once per insertion, so its code
    // size is what it costs).
    template <class F>
    __device__ __forceinline__ void scan_eq(const uint16_t *arr, int count, int v, int g,
                                            int stride, F on_hit)
    {
        const uint32_t vv = (uint32_t)v | ((uint32_t)v << 16);
        const uint4 *a8 = reinterpret_cast<const uint4 *>(arr);
        const int nq = (count + 7) >> 3;
        for (int i0 = g; i0 < nq; i0 += 2 * stride) {
            const uint4 q0 = a8[i0];
            const uint4 q1 = i0 + stride < nq ? a8[i0 + stride] : make_uint4(~vv, ~vv, ~vv, ~vv);
            uint32_t hits = match8(q0, vv) | (match8(q1, vv) << 8);
            while (hits) {
                const int j = __ffs(hits) - 1;
                hits &= hits - 1;
                const int e = 8 * (j < 8 ? i0 : i0 + stride) + (j & 7);
                if (e < count) on_hit(e);
            }
        }
    }

    // Row w of this CTA to refresh in this insertion (a row is
    // listed at most once, so the list holds NR entries).
    __device__ void list_row(int w)
    {
        const int i = atomicAdd(rcount, 1);
        if (i < NR) rows[i] = (uint16_t)w;
    }

    // The owner's refresh of row w by the PL lanes of this lane's
    // group: from ptr + 1, steps of one 16-byte load (8 sorted ids) per lane,
    // until the first uninserted id or the end of the row (an id >= n or
    // position n - 1); the new word goes to this CTA's Mc list and to every
    // CTA's replica (lane sl stores into CTAs sl, sl + PL, ...).
    __device__ void refresh_row(int w)
    {
        const int lane = threadIdx.x & 31, sl = lane & (PL - 1), g0 = lane - sl;
        const unsigned gmask = PL == 32 ? 0xffffffffu : (((1u << PL) - 1u) << g0);
        const int mlen = n - 1;
        const uint16_t *row = a.idx + (long long)w * a.ldi;
        int p = ptr_of(pm[w]) + 1;
        int fq = mlen, fe = kNone16;
        int steps = 0;
        while (p < mlen) {
            const int base = p & ~7;
            const int q0 = base + sl * 8;
            const uint4 c = q0 < a.ldi ? *reinterpret_cast<const uint4 *>(row + q0)
                                       : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu,
                                                    0xFFFFFFFFu);
            ++steps;
            const uint32_t wd[4] = {c.x, c.y, c.z, c.w};
            // bit t: position q0 + t ends the scan (at or after p; the row's
            // end or an uninserted id)
            uint32_t um = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int q = q0 + t;
                const int e = (wd[t >> 1] >> (16 * (t & 1))) & 0xFFFF;
                const bool stop = q >= mlen || e >= n;
                const int ec = stop ? 0 : e;
                const bool ins_e = ec == cur_v || ((ins[ec >> 5] >> (ec & 31)) & 1u);
                um |= (uint32_t)(q >= p && (stop || !ins_e)) << t;
            }
            // lanes hold consecutive runs of 8: the lowest lane with a bit
            // holds the first such position
            const unsigned hit = __ballot_sync(gmask, um != 0u) & gmask;
            if (hit) {
                const int t = um ? __ffs(um) - 1 : 0;
                const uint32_t sel = t < 2 ? c.x : t < 4 ? c.y : t < 6 ? c.z : c.w;
                const int e = (int)((sel >> (16 * (t & 1))) & 0xFFFFu);
                const int q = q0 + t;
                const bool stop = q >= mlen || e >= n;
                const uint32_t pk = ((uint32_t)q << 16) | (uint32_t)(stop ? kNone16 : e);
                const uint32_t got = __shfl_sync(gmask, pk, __ffs(hit) - 1);
                fq = (int)(got >> 16);
                fe = (int)(got & 0xFFFFu);
                break;
            }
            p = base + PL * 8;
        }
        const uint32_t word = (fe != kNone16 && fq < mlen)
                                  ? ((uint32_t)fq << 16) | (uint32_t)fe
                                  : ((uint32_t)(fq < mlen ? fq : mlen) << 16) | kNone16;
        for (int j = sl; j < C; j += PL) {
            if (j == r) {
                mco[w / C] = (uint16_t)(word & 0xFFFFu);
                *(volatile uint32_t *)(pm + w) = word;
            } else {
                *(volatile uint32_t *)cg::this_cluster().map_shared_rank(pm + w, j) = word;
            }
        }
        if (sl == 0) {
            ++c_rows;
            c_steps += steps;
            if (steps > 1) ++c_cont;
        }
    }

    // The fresh word of vertex w of a face: at once if this CTA's
    // replica is fresh, else after the owner's store arrives (bounded poll),
    // else by a local refresh.
    __device__ uint32_t fresh_word(int w)
    {
        uint32_t x = word_at(w);
        if (!stale(x)) return x;
        ++c_wait;
        for (int i = 0; i < kClWaitPolls; ++i) {
            x = word_at(w);
            if (!stale(x)) return x;
        }
        ++c_slow;
        return cl_refresh_thread(a.idx + (long long)w * a.ldi, ins, pm + w, n, cur_v);
    }

    __device__ void mark_group(int g)
    {
        const uint32_t bit = 1u << (g & 31);
        if (!(atomicOr(&b1[g >> 5], bit) & bit)) q1[atomicAdd(n1, 1)] = (uint16_t)g;
    }

    // Best pair of local face lf from the fresh Mc of its
    // vertices: 9 independent gathers; gain (S[a,u] + S[b,u]) + S[c,u]
    // round-to-nearest in the dtype of S; ties to the smaller u.  The key
    // (with the global face id) goes to the face's leaf.  The gathers of the
    // vertices whose replica word is already fresh are issued before the
    // wait for the others.
    __device__ void eval_face(int lf)
    {
        const uint2 fr = frec[lf];
        const int xs[3] = {(int)(fr.x & 0xFFFFu), (int)(fr.x >> 16), (int)(fr.y & 0xFFFFu)};
        int cs[3];
        bool st[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const uint32_t w = word_at(xs[i]);
            st[i] = stale(w);
            cs[i] = mc_of(w);
        }
        T v[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (st[i]) continue;
            const int col = cs[i] < n ? cs[i] : 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) v[i][j] = S[(long long)xs[j] * a.ld + col];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (!st[i]) continue;
            cs[i] = mc_of(fresh_word(xs[i]));
            const int col = cs[i] < n ? cs[i] : 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) v[i][j] = S[(long long)xs[j] * a.ld + col];
        }
        int bv = -1;
        T bg = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int c = cs[i];
            if (c >= n) continue;
            const T g = canon(add_rn(add_rn(canon(v[i][0]), canon(v[i][1])), canon(v[i][2])));
            if (bv < 0 || g > bg || (g == bg && c < bv)) { bv = c; bg = g; }
        }
        leaf[lf] = bv < 0 ? KO::empty() : KO::make(bg, bv, lf * C + r);
        fv[lf] = bv < 0 ? kNone16 : (uint16_t)bv;
        mark_group(lf >> 5);
        ++c_evals;
    }

    __device__ void list_face(int lf) { flist[atomicAdd(fcount, 1)] = (uint16_t)lf; }

    // C, D, E of an insertion over the listed rows and faces (the caller has
    // just passed the barrier after the row scan).  The warps that no row
    // refresh needs run face_scan(g, stride) meanwhile (all warps after
    // their refreshes when every warp has one).  Ends with a barrier.
    template <class FS>
    __device__ void round(long long &cyc_ref, long long &cyc_eval, long long &cyc_l1,
                          FS face_scan)
    {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        long long c0 = clock64();
        const int rc = *rcount < NR ? *rcount : NR;
        const int groups = rc < NG ? rc : NG;         // row groups with a row
        const int rw = (groups * PL + kWarp - 1) / kWarp;  // the warps they occupy
        if (warp < rw)
            for (int i = tid / PL; i < rc; i += NG) refresh_row(rows[i]);
        if (rw < NW) {
            if (warp >= rw) face_scan(tid - kWarp * rw, NT - kWarp * rw);
        } else {
            face_scan(tid, NT);
        }
        __syncthreads();
        long long c1 = clock64();
        cyc_ref += c1 - c0;
        // faces spread over all warps: face i to lane i / NW of warp i % NW
        const int m = *fcount;
        for (int i = lane * NW + warp; i < m; i += NT) eval_face(flist[i]);
        __syncthreads();
        long long c2 = clock64();
        cyc_eval += c2 - c1;
        const int c1n = *n1;
        for (int j = warp; j < c1n; j += NW) {
            const int g = q1[j];
            const int lf = g * 32 + lane;
            const Key mx = warp_max<KO>(lf < NL ? leaf[lf] : KO::empty());
            if (lane == 0) {
                l1[g] = mx;
                atomicAnd(&b1[g >> 5], ~(1u << (g & 31)));
            }
        }
        __syncthreads();
        cyc_l1 += clock64() - c2;
    }

    // Warp 0: this CTA's best pair and its face record into slot `par` of
    // every CTA of the cluster (the caller then passes a cluster barrier).
    __device__ void push_root(int par, uint32_t flag)
    {
        const int lane = threadIdx.x & 31;
        Key x = KO::empty();
        for (int g = lane; g < G1L; g += 32) {
            const Key y = l1[g];
            if (KO::gt(y, x)) x = y;
        }
        x = warp_max<KO>(x);
        uint2 fr = make_uint2(0u, 0u);
        if (!KO::is_empty(x)) fr = frec[KO::face(x) / C];
        if (lane < C) {
            ClSlot<Key> val;
            val.key = x;
            val.xy = fr.x;
            val.zb = fr.y | (flag << 31);
            const uint4 *src = reinterpret_cast<const uint4 *>(&val);
            uint4 *dst = reinterpret_cast<uint4 *>(
                cg::this_cluster().map_shared_rank(slot + par * C + r, lane));
#pragma unroll
            for (int i = 0; i < (int)(sizeof(val) / 16); ++i) dst[i] = src[i];
        }
    }
};

template <typename T, int C, int PL>
__device__ __forceinline__ void cluster_body(const LoopArgs &a)
{
    using L_ = ClLoop<T, C, PL>;
    using KO = typename L_::KO;
    using Key = typename L_::Key;
    constexpr int NT = kClThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_fcount, s_rcount, s_n1, s_status;
    __shared__ int s_clique[4];
    __shared__ long long s_red_r[NT / kWarp];
    __shared__ int s_red_i[NT / kWarp];
    __shared__ unsigned long long s_cnt[8];  // CTA 0: the cluster's counters

    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = (int)cl.block_rank();
    const int n = a.n;

    // one decision for the whole cluster: CTA 0's reading of the status word
    if (tid == 0) s_status = *(volatile int *)a.status;
    if (tid < 8) s_cnt[tid] = 0;
    if (tid == 0) { s_fcount = 0; s_rcount = 0; s_n1 = 0; }
    cluster_barrier();
    const int st0 = *cl.map_shared_rank(&s_status, 0);
    cluster_barrier();
    if (st0 != 0) return;  // an earlier step failed (every CTA leaves)

    const uint64_t t0 = globaltimer_ns();
    const ClLayout L = cl_layout(n, C, sizeof(Key));
    L_ st{a};
    st.S = reinterpret_cast<const T *>(a.S);
    st.n = n;
    st.r = r;
    st.NL = L.NL;
    st.NR = L.NR;
    st.G1L = L.G1L;
    st.ins = reinterpret_cast<uint32_t *>(smem + L.off_ins);
    st.mco = reinterpret_cast<uint16_t *>(smem + L.off_mco);
    st.pm = reinterpret_cast<uint32_t *>(smem + L.off_pm);
    st.frec = reinterpret_cast<uint2 *>(smem + L.off_frec);
    st.fv = reinterpret_cast<uint16_t *>(smem + L.off_fv);
    st.leaf = reinterpret_cast<Key *>(smem + L.off_leaf);
    st.l1 = reinterpret_cast<Key *>(smem + L.off_l1);
    st.b1 = reinterpret_cast<uint32_t *>(smem + L.off_b1);
    st.q1 = reinterpret_cast<uint16_t *>(smem + L.off_q1);
    st.flist = reinterpret_cast<uint16_t *>(smem + L.off_flist);
    st.rows = reinterpret_cast<uint16_t *>(smem + L.off_rows);
    st.slot = reinterpret_cast<ClSlot<Key> *>(smem + L.off_slot);
    st.fcount = &s_fcount;
    st.rcount = &s_rcount;
    st.n1 = &s_n1;

    const StateLayout SL = state_layout(n, sizeof(Key128));
    unsigned char *gs = reinterpret_cast<unsigned char *>(a.state);
    long long *gscal = reinterpret_cast<long long *>(gs + SL.off_scal);
    uint32_t *gins = reinterpret_cast<uint32_t *>(gs + SL.off_ins);
    uint16_t *gmc = reinterpret_cast<uint16_t *>(gs + SL.off_mc);
    uint16_t *gptr = reinterpret_cast<uint16_t *>(gs + SL.off_ptr);
    uint16_t *gfv = reinterpret_cast<uint16_t *>(gs + SL.off_fv);
    Key *gleaf = reinterpret_cast<Key *>(a.leaf_fresh);
    const int mlen = n - 1;

    long long cyc_sel = 0, cyc_scan = 0, cyc_ref = 0, cyc_eval = 0, cyc_l1 = 0, cyc_root = 0;
    int k;
    // common to both starts
    for (int i = tid; i < (L.G1L + 31) / 32; i += NT) st.b1[i] = 0;
    for (int lf = tid; lf < L.NL8; lf += NT) st.fv[lf] = kNone16;
    if (a.resume) {
        k = (int)gscal[17];
        const int nf = 4 + 2 * k;
        for (int i = tid; i < L.W; i += NT) st.ins[i] = gins[i];
        for (int w = tid; w < L.n8; w += NT)
            st.pm[w] = w < n ? ((uint32_t)gptr[w] << 16) | (uint32_t)gmc[w]
                             : ((uint32_t)mlen << 16) | kNone16;
        for (int i = tid; i < L.NR8; i += NT) {
            const int w = r + C * i;
            st.mco[i] = (i < L.NR && w < n) ? gmc[w] : kNone16;
        }
        for (int lf = tid; lf < L.NL; lf += NT) {
            const int f = lf * C + r;
            if (f < nf) {
                const int4 fc = a.face[f];
                st.frec[lf] = make_uint2((uint32_t)fc.x | ((uint32_t)fc.y << 16),
                                         (uint32_t)fc.z | ((uint32_t)fc.w << 16));
                st.fv[lf] = gfv[f];
                st.leaf[lf] = gleaf[f];
            } else {
                st.frec[lf] = make_uint2(0u, 0u);
                st.leaf[lf] = KO::empty();
            }
        }
        __syncthreads();
        for (int gr = warp; gr < L.G1L; gr += NT / kWarp) {
            const int lf = gr * 32 + lane;
            const Key mx = warp_max<KO>(lf < L.NL ? st.leaf[lf] : KO::empty());
            if (lane == 0) st.l1[gr] = mx;
        }
        __syncthreads();
    } else {
        k = 0;
        for (int i = tid; i < L.W; i += NT) st.ins[i] = 0;
        for (int w = tid; w < L.n8; w += NT) {
            uint32_t word = ((uint32_t)mlen << 16) | kNone16;
            if (w < n) {
                const uint16_t e = a.idx[(long long)w * a.ldi];
                word = e < n ? (uint32_t)e : ((uint32_t)mlen << 16) | kNone16;
            }
            st.pm[w] = word;
        }
        __syncthreads();
        for (int i = tid; i < L.NR8; i += NT) {
            const int w = r + C * i;
            st.mco[i] = (i < L.NR && w < n) ? (uint16_t)(st.pm[w] & 0xFFFFu) : kNone16;
        }
        for (int lf = tid; lf < L.NL; lf += NT) {
            st.frec[lf] = make_uint2(0u, 0u);
            st.leaf[lf] = KO::empty();
        }
        for (int gr = tid; gr < L.G1L; gr += NT) st.l1[gr] = KO::empty();
        __syncthreads();
        // every replica is initialised before any owner stores a word into it
        cluster_barrier();
        // the initial 4-clique (Algorithm 1): top four row sums, found by
        // every CTA alike
        pick_clique<NT>(a.rowsum, n, s_clique, s_red_r, s_red_i);
        const int *c = s_clique;
        if (tid == 0) {
            for (int i = 0; i < 4; ++i) st.ins[c[i] >> 5] |= 1u << (c[i] & 31);
            if (r == 0) {
                for (int i = 0; i < 4; ++i) a.order[i] = c[i];
                const int pr[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
                for (int i = 0; i < 6; ++i) {
                    a.edges[2 * i] = c[pr[i][0]];
                    a.edges[2 * i + 1] = c[pr[i][1]];
                }
                a.parent[0] = -1;
            }
        }
        if (tid == 0) {
            // this CTA's clique rows whose first id is another clique vertex,
            // and its clique faces
            for (int i = 0; i < 4; ++i)
                if (c[i] % C == r && st.stale(st.pm[c[i]])) st.list_row(c[i]);
            const int tri[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
            for (int f = 0; f < 4; ++f) {
                if (f % C != r) continue;
                st.frec[f / C] = face_record(c[tri[f][0]], c[tri[f][1]], c[tri[f][2]], 0);
                st.list_face(f / C);
            }
        }
        __syncthreads();
        st.round(cyc_ref, cyc_eval, cyc_l1, [](int, int) {});
    }
    // the first slot exchange
    if (warp == 0) st.push_root(0, 0u);
    if (tid == 0) { s_fcount = 0; s_rcount = 0; s_n1 = 0; }
    cluster_barrier();

    // ---- main loop: one insertion per round
    const int total = n - 4;
    const int k_stop = a.k_stop < total ? a.k_stop : total;
    long long rounds = 0;
    int par = 0, stop = 0;
    while (k < k_stop) {
        long long c0 = clock64();
        // the best of the C slots (every warp alike)
        const ClSlot<Key> *sl = st.slot + par * C;
        const Key x = lane < C ? sl[lane].key : KO::empty();
        const uint32_t fl = lane < C ? sl[lane].zb >> 31 : 0u;
        const Key best = warp_max<KO>(x);
        const uint32_t flags = __reduce_or_sync(0xffffffffu, fl);
        const unsigned who = __ballot_sync(0xffffffffu, lane < C && L_::same(x, best));
        const int wr = who ? __ffs(who) - 1 : 0;
        const uint32_t xy = sl[wr].xy, zb = sl[wr].zb & 0x7FFFFFFFu;
        const int nf_old = 4 + 2 * k;
        const int v = KO::is_empty(best) ? -1 : KO::vert(best);
        const int t = KO::is_empty(best) ? -1 : KO::face(best);
        if (flags & 1u) { stop = TMFG_ETIMEOUT; break; }
        if (v < 0 || v >= n || t < 0 || t >= nf_old || st.is_ins(v)) {
            stop = TMFG_EINTERNAL;
            break;
        }
        const int fx = (int)(xy & 0xFFFFu), fy = (int)(xy >> 16), fz = (int)(zb & 0xFFFFu);
        const int tb = (int)(zb >> 16);
        st.cur_v = v;
        long long c1 = clock64();
        cyc_sel += c1 - c0;
        // B. the three faces made by inserting v into t = {x < y < z} that
        // belong to this CTA (threads 0, 1, 2), v's own row if its Mc was
        // inserted before v, this CTA's inserted rows whose Mc is v, and this
        // CTA's faces whose stored vertex is v
        const int tl = t / C, tr = t % C;
        if (tid < 3) {
            const int fid = tid == 0 ? t : nf_old + tid - 1;
            if (fid % C == r) {
                st.frec[fid / C] = tid == 0 ? face_record(v, fx, fy, k + 1)
                                 : tid == 1 ? face_record(v, fy, fz, k + 1)
                                            : face_record(v, fx, fz, k + 1);
                st.list_face(fid / C);
            }
        }
        if (tid == 32 && v % C == r && st.stale(st.pm[v])) st.list_row(v);
        if (r == 0 && tid == 64) {
            a.order[4 + k] = v;
            int *e = a.edges + 2 * (6 + 3 * k);
            e[0] = v; e[1] = fx; e[2] = v; e[3] = fy; e[4] = v; e[5] = fz;
            a.ins_face[3 * k + 0] = fx;
            a.ins_face[3 * k + 1] = fy;
            a.ins_face[3 * k + 2] = fz;
            a.parent[k + 1] = tb;
        }
        st.scan_eq(st.mco, L.NR, v, tid, NT, [&](int i) {
            const int w = r + C * i;
            if (w < n && st.is_ins(w)) st.list_row(w);
        });
        __syncthreads();
        long long c2 = clock64();
        cyc_scan += c2 - c1;
        // C (with the face scan on the warps that refresh no row), D, E
        const int nlcur = r < nf_old ? (nf_old - 1 - r) / C + 1 : 0;
        st.round(cyc_ref, cyc_eval, cyc_l1, [&](int g, int stride) {
            st.scan_eq(st.fv, nlcur, v, g, stride, [&](int lf) {
                if (!(tr == r && lf == tl)) st.list_face(lf);
            });
        });
        long long c3 = clock64();
        ++k;
        ++rounds;
        par ^= 1;
        // F. this CTA's best pair to every CTA; v's bit; then the cluster barrier
        uint32_t flag = 0u;
        if (warp == 0) {
            if (r == 0 && lane == 0 && globaltimer_ns() - t0 > a.timeout_ns) flag = 1u;
            flag = __shfl_sync(0xffffffffu, flag, 0);
            st.push_root(par, flag);
        }
        if (tid == 0) {
            st.ins[v >> 5] |= 1u << (v & 31);
            s_fcount = 0;
            s_rcount = 0;
            s_n1 = 0;
        }
        cluster_barrier();
        cyc_root += clock64() - c3;
    }

    // ---- statistics (summed over the cluster and over segments) and the
    // state for the next segment
    {
        unsigned long long *c0p = cl.map_shared_rank(s_cnt, 0);
        unsigned long long v6[6] = {(unsigned long long)st.c_evals, (unsigned long long)st.c_rows,
                                    (unsigned long long)st.c_cont, (unsigned long long)st.c_steps,
                                    (unsigned long long)st.c_slow, (unsigned long long)st.c_wait};
        for (int i = 0; i < 6; ++i)
            if (v6[i]) atomicAdd(c0p + i, v6[i]);
    }
    const bool save = gs && k < total && !stop;
    if (save) {
        const int nf = 4 + 2 * k;
        if (r == 0)
            for (int i = tid; i < L.W; i += NT) gins[i] = st.ins[i];
        for (int lf = tid; lf < L.NL; lf += NT) {
            const int f = lf * C + r;
            if (f >= nf) continue;
            const uint2 fr = st.frec[lf];
            a.face[f] = make_int4((int)(fr.x & 0xFFFFu), (int)(fr.x >> 16), (int)(fr.y & 0xFFFFu),
                                  (int)(fr.y >> 16));
            gfv[f] = st.fv[lf];
            gleaf[f] = st.leaf[lf];
        }
        // this CTA's rows (their owner's words are the fresh ones)
        for (int i = tid; i < L.NR; i += NT) {
            const int w = r + C * i;
            if (w >= n) continue;
            gptr[w] = (uint16_t)(st.pm[w] >> 16);
            gmc[w] = (uint16_t)(st.pm[w] & 0xFFFFu);
        }
    }
    cluster_barrier();  // no CTA leaves while another reads its shared memory
    if (r == 0 && tid == 0) {
        if (stop) set_status(a.status, stop);
        long long acc[16];
        for (int i = 0; i < 16; ++i) acc[i] = a.resume ? gscal[i] : 0;
        // slots: 0 face evaluations, 1 cycles of A, 2 pointer steps, 3
        // rounds, 4 ns; cycles of CTA 0's thread 0: 5 B (with its barrier),
        // 8 C, 10 D, 6 E, 7 F (push and cluster barrier); 9 one-thread
        // refreshes after a poll ran out, 11 rows refreshed, 12 rows that
        // took more than one step, 13 the steps beyond the first; 14 cluster
        // size; 15 reads of a stale word that waited for its owner
        const long long seg[16] = {(long long)s_cnt[0], cyc_sel, (long long)s_cnt[3], rounds,
                                   (long long)(globaltimer_ns() - t0), cyc_scan, cyc_l1, cyc_root,
                                   cyc_ref, (long long)s_cnt[4], cyc_eval, (long long)s_cnt[1],
                                   (long long)s_cnt[2], (long long)(s_cnt[3] - s_cnt[1]), 0,
                                   (long long)s_cnt[5]};
        for (int i = 0; i < 16; ++i) acc[i] += seg[i];
        acc[14] = C;
        for (int i = 0; i < 16; ++i) {
            a.stats[i] = acc[i];
            if (gs) gscal[i] = acc[i];
        }
        if (gs) {
            gscal[16] = 4 + 2 * k;
            gscal[17] = k;
        }
    }
}

template <typename T, int C, int PL>
__global__ void __launch_bounds__(kClThreads, 1) tmfg_cluster_kernel(LoopArgs a)
{
    cluster_body<T, C, PL>(a);
}

// ------------------------------------------------------------------- host

size_t cluster_smem_bytes(int n, int dtype, int C)
{
    // a slot keeps the bubble in 15 bits: n - 3 bubbles must fit
    if (n > 32770) return ~(size_t)0;
    const size_t ks = dtype == TMFG_F32 ? sizeof(unsigned long long) : sizeof(Key128);
    return cl_layout(n, C, ks).total;
}

bool cluster_shape_ok(int C, int lanes)
{
    return (C == 8 || C == 16) && (lanes == 8 || lanes == 16 || lanes == 32);
}

namespace {
// The launch configuration of one cluster of C CTAs; false if the kernel's
// attributes cannot be set or the device cannot place such a cluster.
template <typename T, int C, int PL>
bool cluster_config(size_t smem, cudaStream_t stream, cudaLaunchConfig_t *cfg,
                    cudaLaunchAttribute *at)
{
    auto kern = tmfg_cluster_kernel<T, C, PL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(C, 1, 1);
    cfg->blockDim = dim3(kClThreads, 1, 1);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T, int C, int PL>
int go_cluster(const LoopArgs &a, size_t smem, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    if (!cluster_config<T, C, PL>(smem, stream, &cfg, at)) return TMFG_ETOOBIG;
    if (cudaLaunchKernelEx(&cfg, tmfg_cluster_kernel<T, C, PL>, a) != cudaSuccess)
        return TMFG_ECUDA;
    return TMFG_OK;
}
}  // namespace

bool cluster_placeable(int n, int dtype, int C, int lanes)
{
    if (!cluster_shape_ok(C, lanes)) return false;
    const size_t smem = cluster_smem_bytes(n, dtype, C);
    if (smem > kSmemLimit) return false;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    // the placement does not depend on the lanes (same threads and memory)
    if (dtype == TMFG_F32)
        return C == 16 ? cluster_config<float, 16, 32>(smem, 0, &cfg, at)
                       : cluster_config<float, 8, 32>(smem, 0, &cfg, at);
    return C == 16 ? cluster_config<double, 16, 32>(smem, 0, &cfg, at)
                   : cluster_config<double, 8, 32>(smem, 0, &cfg, at);
}

namespace {
template <typename T, int C>
int go_cluster_lanes(const LoopArgs &a, int lanes, size_t smem, cudaStream_t stream)
{
    if (lanes == 32) return go_cluster<T, C, 32>(a, smem, stream);
    if (lanes == 16) return go_cluster<T, C, 16>(a, smem, stream);
    return go_cluster<T, C, 8>(a, smem, stream);
}
}  // namespace

int launch_cluster_loop(const LoopArgs &a, int dtype, int C, int lanes, cudaStream_t stream)
{
    if (!cluster_shape_ok(C, lanes)) return TMFG_EINVAL;
    const size_t smem = cluster_smem_bytes(a.n, dtype, C);
    if (smem > kSmemLimit) return TMFG_ETOOBIG;
    if (dtype == TMFG_F32)
        return C == 16 ? go_cluster_lanes<float, 16>(a, lanes, smem, stream)
                       : go_cluster_lanes<float, 8>(a, lanes, smem, stream);
    return C == 16 ? go_cluster_lanes<double, 16>(a, lanes, smem, stream)
                   : go_cluster_lanes<double, 8>(a, lanes, smem, stream);
}

}  // namespace tmfg
