// loop_corr1.cu -- the insertion loop of corr-tmfg with prefix 1 (Algorithm 1
// with P = 1: every round inserts the single best face-vertex pair), in a
// kernel of its own whose chain of dependent steps per insertion is shorter
// than the general loop kernel's.
//
// Invariant: every inserted vertex's cached MaxCorrs Mc is fresh (the first
// uninserted id of its sorted row).  Inserting v makes stale exactly the
// inserted rows whose Mc is v, plus v's own row if its Mc was inserted
// earlier; all of them are refreshed in the round that inserts v.  The
// paper's pointer (Section 4.3) is read fresh at every use; refreshing a row
// at the insertion of its Mc gives the same value at its next use, since
// the first uninserted id of a sorted row only moves forward and nothing
// else changes it.  The rows to refresh are found by a scan of Mc, not by
// gathering the vertices of the faces to recompute, so their probes start
// at once.
//
// One insertion, all NT threads of the CTA:
//  1. thread 0 inserts the root pair (v, t) (three edges, face t becomes
//     {v,x,y}, {v,y,z} and {v,x,z} are appended); every thread scans the
//     stored vertices of the faces for v (F_update: the faces to
//     recompute) and the Mc of the inserted vertices for v (the rows to
//     refresh), and marks the index groups of the faces to recompute.
//                                                               -- barrier
//  2. groups of PL lanes refresh the listed rows, each from its pointer in
//     steps of PL x 8, 2 PL x 8, 4 PL x 8 ids until an uninserted id or the
//     row's end; meanwhile each thread loads the record of its face and the
//     warps copy the current keys of the marked groups to shared memory.
//                                                               -- barrier
//  3. one thread per face: 9 independent gathers of S, gains summed in the
//     fixed order, the best pair's key into its leaf and its group's copy.
//                                                               -- barrier
//  4. a warp per marked group: the group's maximum (level 1).   -- barrier
//  5. a warp per marked level-2 group: its maximum.             -- barrier
// Every warp then reads the root, the next pair, from level 2.
//
// The keys, the two-level index and the state kept between the segments of
// a build are those of the general loop kernel (loop_common.cuh), so the row
// compaction between segments serves both.
#include "loop_common.cuh"

namespace tmfg {

constexpr int kC1RowCap = 1024;   // rows to refresh listed in shared memory (the rest in global)
constexpr int kC1FuCap = 1024;    // faces to recompute listed in shared memory (the rest in global)
constexpr int kC1StageMax = 256;  // index groups whose keys are copied to shared memory

// Shared-memory layout (dynamic part), computed identically on the host; the
// copies of the marked groups' keys come last, `cap` groups of 32 keys.
struct Corr1Layout {
    int W, nfmax, G1, G2, n8, nf8;
    size_t off_ins, off_mc, off_ptr, off_fv, off_tree, off_gslot, off_rows, off_fus, off_stage;
    size_t total;
};

// gp: the pointers live in global memory (the loop state's array) instead of
// shared memory, which leaves room for n up to 32768.
__host__ __device__ inline Corr1Layout corr1_layout(int n, size_t ks, int cap, bool gp)
{
    Corr1Layout L;
    L.W = (n + 31) / 32;
    L.nfmax = 2 * n - 4;
    L.G1 = (L.nfmax + 31) / 32;
    L.G2 = (L.G1 + 31) / 32;
    L.n8 = (n + 7) & ~7;
    L.nf8 = (L.nfmax + 7) & ~7;
    size_t o = 0;
    L.off_ins = o;   o = align16(o + 4 * (size_t)L.W);
    L.off_mc = o;    o = align16(o + 2 * (size_t)L.n8);
    L.off_ptr = o;   o = align16(o + (gp ? 0 : 2 * (size_t)n));
    L.off_fv = o;    o = align16(o + 2 * (size_t)L.nf8);
    L.off_tree = o;  o += tree_layout_bytes(L.G1, L.G2, ks);
    L.off_gslot = o; o = align16(o + 2 * (size_t)L.G1);
    L.off_rows = o;  o = align16(o + 2 * (size_t)kC1RowCap);
    L.off_fus = o;   o = align16(o + 4 * (size_t)kC1FuCap);
    L.off_stage = o;
    L.total = o + ks * 32 * (size_t)cap;
    return L;
}

__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

template <typename T, int NT, int PL>
struct Corr1 {
    using KO = KeyOps<T>;
    using Key = typename KO::Key;
    static constexpr int NW = NT / kWarp;  // warps
    static constexpr int NG = NT / PL;     // row-refresh groups
    static_assert(PL >= 1 && PL <= 32 && (PL & (PL - 1)) == 0, "PL: a power of two <= 32");

    const LoopArgs &a;
    const T *S;
    int n, nfmax, G1, G2, n8, cap;
    uint32_t *ins;
    uint16_t *mc, *ptr, *fv, *gslot, *rows;
    int *fus, *rows_over;
    Key *leaf, *stage;
    Key *l1, *l2;
    uint32_t *b1, *b2;
    uint16_t *q1, *q2;
    int *n1, *n2, *fcount, *rcount;
    // this thread's counters, added to the shared ones once per segment
    long long c_rows = 0, c_cont = 0, c_steps = 0, c_evals = 0;
    long long cyc_own = 0;  // thread 0: its own share of the gathers

    __device__ bool is_ins(int v) const { return (ins[v >> 5] >> (v & 31)) & 1u; }

    __device__ void fu_put(int i, int f)
    {
        if (i < kC1FuCap) fus[i] = f;
        else a.fu_buf[i] = f;
    }
    __device__ int fu_get(int i) const { return i < kC1FuCap ? fus[i] : a.fu_buf[i]; }
    __device__ void row_put(int i, int w)
    {
        if (i < kC1RowCap) rows[i] = (uint16_t)w;
        else rows_over[i] = w;
    }
    __device__ int row_get(int i) const { return i < kC1RowCap ? (int)rows[i] : rows_over[i]; }

    // Mark the level-1 group of face f for the index update; its position in
    // the list of marked groups is its slot for the copy of its keys.
    __device__ void mark(int f)
    {
        const int g = f >> 5;
        const uint32_t bit = 1u << (g & 31);
        if (!(atomicOr(&b1[g >> 5], bit) & bit)) {
            const int j = atomicAdd(n1, 1);
            q1[j] = (uint16_t)g;
            gslot[g] = (uint16_t)j;
        }
    }

    // Every index i < count of a 16-bit array (16-byte aligned, padded to a
    // multiple of 8 entries) whose entry is v: on_hit(i).  Four 16-byte
    // loads per thread are in flight at a time; a word holds a match when
    // one of its halves of word ^ vv is zero.
    template <class F>
    __device__ __forceinline__ void scan_eq(const uint16_t *arr, int count, int v, F on_hit)
    {
        const uint32_t vv = (uint32_t)v | ((uint32_t)v << 16);
        const uint4 *a8 = reinterpret_cast<const uint4 *>(arr);
        const int nq = (count + 7) >> 3;
        for (int i0 = threadIdx.x; i0 < nq; i0 += 4 * NT) {
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * NT;
                q[u] = i < nq ? a8[i] : make_uint4(~vv, ~vv, ~vv, ~vv);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t wd[4] = {q[u].x ^ vv, q[u].y ^ vv, q[u].z ^ vv, q[u].w ^ vv};
                uint32_t any = 0;
#pragma unroll
                for (int h = 0; h < 4; ++h) any |= (wd[h] - 0x00010001u) & ~wd[h] & 0x80008000u;
                if (!any) continue;  // no half is zero: no match in these 8
#pragma unroll
                for (int h = 0; h < 4; ++h)
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int e = 8 * (i0 + u * NT) + 2 * h + b;
                        if (e < count && ((wd[h] >> (16 * b)) & 0xFFFFu) == 0) on_hit(e);
                    }
            }
        }
    }

    // Faces f < nf whose stored vertex is v go to the face-update list and
    // have their groups marked.
    __device__ void scan_faces(int v, int nf)
    {
        scan_eq(fv, nf, v, [&](int f) {
            fu_put(atomicAdd(fcount, 1), f);
            mark(f);
        });
    }

    // Inserted rows w whose Mc is v go to the list of rows to refresh.
    __device__ void scan_rows(int v)
    {
        scan_eq(mc, n, v, [&](int w) {
            if (is_ins(w)) row_put(atomicAdd(rcount, 1), w);
        });
    }

    // Refresh row w (its Mc is inserted) by the PL lanes of this thread's
    // group: from ptr[w] + 1, steps of 1, 2, then 4 16-byte loads per lane,
    // until the first uninserted id or the end of the row (an id >= n or
    // position n - 1).  Lane 0 of the group writes ptr[w] and Mc[w].
    __device__ void refresh_row(int w)
    {
        const int lane = threadIdx.x & 31, sl = lane & (PL - 1), g0 = lane - sl;
        const unsigned gmask = PL == 32 ? 0xffffffffu : (((1u << PL) - 1u) << g0);
        const int mlen = n - 1;
        const uint16_t *row = a.idx + (long long)w * a.ldi;
        int p = ptr[w] + 1;
        int fq = mlen, fe = kNone16;
        int span = 1, steps = 0;
        while (p < mlen) {
            const int base = p & ~7;
            uint4 c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q0 = base + (u * PL + sl) * 8;
                c[u] = (u < span && q0 < a.ldi)
                           ? *reinterpret_cast<const uint4 *>(row + q0)
                           : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
            }
            ++steps;
            // bit t of um[u]: position base + (u * PL + sl) * 8 + t ends the
            // scan (at or after p; the row's end or an uninserted id)
            uint32_t um[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u >= span) continue;
                const uint32_t wd[4] = {c[u].x, c[u].y, c[u].z, c[u].w};
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int q = base + (u * PL + sl) * 8 + t;
                    const int e = (wd[t >> 1] >> (16 * (t & 1))) & 0xFFFF;
                    const bool stop = q >= mlen || e >= n;
                    um[u] |= (uint32_t)(q >= p && (stop || !is_ins(stop ? 0 : e))) << t;
                }
            }
            // positions run chunk by chunk (chunk u of every lane before
            // chunk u + 1), lane by lane within a chunk: the first chunk with
            // a bit, its lowest lane with one, that lane's lowest bit
            int hu = -1;
            unsigned hit = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned h = __ballot_sync(gmask, um[u] != 0u) & gmask;
                if (hu < 0 && h) {
                    hu = u;
                    hit = h;
                }
            }
            if (hu >= 0) {
                const uint32_t mk = hu == 0 ? um[0] : hu == 1 ? um[1] : hu == 2 ? um[2] : um[3];
                const uint4 ch = hu == 0 ? c[0] : hu == 1 ? c[1] : hu == 2 ? c[2] : c[3];
                const int t = mk ? __ffs(mk) - 1 : 0;
                const uint32_t sel = t < 2 ? ch.x : t < 4 ? ch.y : t < 6 ? ch.z : ch.w;
                const int e = (int)((sel >> (16 * (t & 1))) & 0xFFFFu);
                const int q = base + (hu * PL + sl) * 8 + t;
                const bool stop = q >= mlen || e >= n;
                const uint32_t pk = ((uint32_t)q << 16) | (uint32_t)(stop ? kNone16 : e);
                const uint32_t got = __shfl_sync(gmask, pk, __ffs(hit) - 1);
                fq = (int)(got >> 16);
                fe = (int)(got & 0xFFFFu);
                break;
            }
            p = base + span * PL * 8;
            if (span < 4) span <<= 1;
        }
        if (sl == 0) {
            if (fe != kNone16 && fq < mlen) {
                ptr[w] = (uint16_t)fq;
                mc[w] = (uint16_t)fe;
            } else {
                ptr[w] = (uint16_t)(fq < mlen ? fq : mlen);
                mc[w] = kNone16;
            }
            ++c_rows;
            c_steps += steps;
            if (steps > 1) ++c_cont;
        }
    }

    // Best pair of face f = {fc.x < fc.y < fc.z} from the fresh Mc of its
    // vertices (9 independent gathers; gain (S[a,u] + S[b,u]) + S[c,u],
    // round-to-nearest in the dtype of S; ties to the smaller u).  The key
    // goes to the face's leaf and, when its group has a slot, to the copy.
    __device__ void eval_face(int f, int4 fc)
    {
        const int cs[3] = {mc[fc.x], mc[fc.y], mc[fc.z]};
        const int xs[3] = {fc.x, fc.y, fc.z};
        // all nine loads unconditional (a missing candidate reads column 0
        // and is ignored), so they are all in flight together
        T v[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
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
        const Key key = bv < 0 ? KO::empty() : KO::make(bg, bv, f);
        leaf[f] = key;
        fv[f] = bv < 0 ? kNone16 : (uint16_t)bv;
        const int slot = gslot[f >> 5];
        if (slot < cap) stage[slot * 32 + (f & 31)] = key;
        ++c_evals;
    }

    // Phases 2-5 of a round over the listed faces and rows (the lists and
    // marks are complete: the caller has just passed a barrier).  Ends with
    // a barrier after which level 2 holds the new maxima.
    __device__ void round(long long &cyc_load, long long &cyc_gain, long long &cyc_index)
    {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        const int m = *fcount, r = *rcount, c1 = *n1;
        if (tid == 0) *n2 = 0;  // read after the level-1 phase of the previous round
        long long c0 = clock64();
        // 2. face records, copies of the marked groups' keys, row refreshes
        int4 fc0 = make_int4(0, 0, 0, 0);
        int f0 = -1;
        // face i goes to lane i / NW of warp i % NW: the faces (and their
        // gathers) are spread over all warps, not packed into the first ones
        const int fi = lane * NW + warp;
        if (fi < m) {
            f0 = fu_get(fi);
            fc0 = a.face[f0];
        }
        // the keys of this warp's first four copy slots are loaded before
        // the row refreshes and stored after them, so the loads overlap
        const int cs = c1 < cap ? c1 : cap;
        Key kr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = warp + u * NW;
            const int f = j < cs ? (int)q1[j] * 32 + lane : nfmax;
            kr[u] = f < nfmax ? leaf[f] : KO::empty();
        }
        for (int i = tid / PL; i < r; i += NG) refresh_row(row_get(i));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = warp + u * NW;
            if (j < cs) stage[j * 32 + lane] = kr[u];
        }
        for (int j = warp + 4 * NW; j < cs; j += NW) {
            const int f = (int)q1[j] * 32 + lane;
            stage[j * 32 + lane] = f < nfmax ? leaf[f] : KO::empty();
        }
        __syncthreads();
        long long c1t = clock64();
        cyc_load += c1t - c0;
        // 3. the faces' best pairs
        if (f0 >= 0) eval_face(f0, fc0);
        for (int i = fi + NT; i < m; i += NT) {
            const int f = fu_get(i);
            eval_face(f, a.face[f]);
        }
        cyc_own += clock64() - c1t;
        __syncthreads();
        long long c2t = clock64();
        cyc_gain += c2t - c1t;
        // 4. level 1: the maxima of the marked groups
        for (int j = warp; j < c1; j += NW) {
            const int g = q1[j];
            const int f = g * 32 + lane;
            const Key x = j < cap ? stage[j * 32 + lane] : (f < nfmax ? leaf[f] : KO::empty());
            const Key mx = warp_max<KO>(x);
            if (lane == 0) {
                l1[g] = mx;
                atomicAnd(&b1[g >> 5], ~(1u << (g & 31)));
                const int g2 = g >> 5;
                const uint32_t bit = 1u << (g2 & 31);
                if (!(atomicOr(&b2[g2 >> 5], bit) & bit)) q2[atomicAdd(n2, 1)] = (uint16_t)g2;
            }
        }
        if (tid == 0) *n1 = 0;
        __syncthreads();
        // 5. level 2
        const int c2 = *n2;
        for (int j = warp; j < c2; j += NW) {
            const int g2 = q2[j];
            const int g = g2 * 32 + lane;
            const Key mx = warp_max<KO>(g < G1 ? l1[g] : KO::empty());
            if (lane == 0) {
                l2[g2] = mx;
                atomicAnd(&b2[g2 >> 5], ~(1u << (g2 & 31)));
            }
        }
        if (tid == 0) {
            *fcount = 2;  // the next insertion lists its two appended faces first
            *rcount = 0;
        }
        __syncthreads();
        cyc_index += clock64() - c2t;
    }

    // The root (the best pair over all faces), read by every warp from level 2.
    __device__ Key root() const
    {
        const int lane = threadIdx.x & 31;
        Key x = lane < G2 ? l2[lane] : KO::empty();
        const Key y = lane + 32 < G2 ? l2[lane + 32] : KO::empty();
        if (KO::gt(y, x)) x = y;
        return warp_max<KO>(x);
    }
};

template <typename T, int NT, int PL, bool GP>
__device__ __forceinline__ void corr1_body(const LoopArgs &a)
{
    using C = Corr1<T, NT, PL>;
    using KO = typename C::KO;
    using Key = typename C::Key;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_n1, s_n2, s_fcount, s_rcount, s_stop;
    __shared__ int s_clique[4];
    __shared__ long long s_red_r[NT / kWarp];
    __shared__ int s_red_i[NT / kWarp];
    __shared__ unsigned long long s_cnt[4];

    const int tid = threadIdx.x;
    const int n = a.n;
    if (*(volatile int *)a.status != 0) return;  // an earlier step failed
    const uint64_t t0 = globaltimer_ns();
    const Corr1Layout L = corr1_layout(n, sizeof(Key), 0, GP);
    const uint32_t dyn = dynamic_smem_bytes();
    int cap = dyn > L.total ? (int)((dyn - L.total) / (32 * sizeof(Key))) : 0;
    if (cap > kC1StageMax) cap = kC1StageMax;

    C st{a};
    st.S = reinterpret_cast<const T *>(a.S);
    st.n = n;
    st.nfmax = L.nfmax;
    st.G1 = L.G1;
    st.G2 = L.G2;
    st.n8 = L.n8;
    st.cap = cap;
    st.ins = reinterpret_cast<uint32_t *>(smem + L.off_ins);
    st.mc = reinterpret_cast<uint16_t *>(smem + L.off_mc);
    const StateLayout SL = state_layout(n, sizeof(Key128));
    unsigned char *gs = reinterpret_cast<unsigned char *>(a.state);
    st.ptr = GP ? reinterpret_cast<uint16_t *>(gs + SL.off_ptr)
                : reinterpret_cast<uint16_t *>(smem + L.off_ptr);
    st.fv = reinterpret_cast<uint16_t *>(smem + L.off_fv);
    {
        unsigned char *b = smem + L.off_tree;
        size_t o = 0;
        st.l1 = reinterpret_cast<Key *>(b + o);      o = align16(o + sizeof(Key) * (size_t)L.G1);
        st.l2 = reinterpret_cast<Key *>(b + o);      o = align16(o + sizeof(Key) * (size_t)L.G2);
        st.b1 = reinterpret_cast<uint32_t *>(b + o); o = align16(o + 4 * (size_t)((L.G1 + 31) / 32));
        st.b2 = reinterpret_cast<uint32_t *>(b + o); o = align16(o + 4 * (size_t)((L.G2 + 31) / 32));
        st.q1 = reinterpret_cast<uint16_t *>(b + o); o = align16(o + 2 * (size_t)L.G1);
        st.q2 = reinterpret_cast<uint16_t *>(b + o);
    }
    st.gslot = reinterpret_cast<uint16_t *>(smem + L.off_gslot);
    st.rows = reinterpret_cast<uint16_t *>(smem + L.off_rows);
    st.fus = reinterpret_cast<int *>(smem + L.off_fus);
    st.stage = reinterpret_cast<Key *>(smem + L.off_stage);
    st.leaf = reinterpret_cast<Key *>(a.leaf_fresh);
    // prefix 1 has no pending keys: their candidate buffer (8 bytes per face
    // slot, more than 4 bytes per vertex) holds the overflow of the row list
    st.rows_over = reinterpret_cast<int *>(a.pend_cand);
    st.n1 = &s_n1;
    st.n2 = &s_n2;
    st.fcount = &s_fcount;
    st.rcount = &s_rcount;

    long long *gscal = reinterpret_cast<long long *>(gs + SL.off_scal);
    long long acc[16];
    for (int i = 0; i < 16; ++i) acc[i] = 0;
    long long cyc_load = 0, cyc_gain = 0, cyc_index = 0, cyc_scan = 0, cyc_root = 0;
    long long cyc_sf = 0, cyc_sr = 0, cyc_ins = 0;  // parts of the scan phase
    if (tid < 4) s_cnt[tid] = 0;
    int k;  // insertions done
    if (a.resume) {
        for (int i = 0; i < 16; ++i) acc[i] = gscal[i];
        const uint32_t *gins = reinterpret_cast<const uint32_t *>(gs + SL.off_ins);
        const uint16_t *gmc = reinterpret_cast<const uint16_t *>(gs + SL.off_mc);
        const uint16_t *gptr = reinterpret_cast<const uint16_t *>(gs + SL.off_ptr);
        const uint16_t *gfv = reinterpret_cast<const uint16_t *>(gs + SL.off_fv);
        const Key *gt = reinterpret_cast<const Key *>(gs + SL.off_tree[0]);
        for (int i = tid; i < L.W; i += NT) st.ins[i] = gins[i];
        for (int w = tid; w < L.n8; w += NT) st.mc[w] = w < n ? gmc[w] : kNone16;
        if (!GP)
            for (int w = tid; w < n; w += NT) st.ptr[w] = gptr[w];
        for (int f = tid; f < L.nf8; f += NT) st.fv[f] = f < L.nfmax ? gfv[f] : kNone16;
        for (int i = tid; i < L.G1; i += NT) st.l1[i] = gt[i];
        for (int i = tid; i < L.G2; i += NT) st.l2[i] = gt[L.G1 + i];
        for (int i = tid; i < (L.G1 + 31) / 32; i += NT) st.b1[i] = 0;
        for (int i = tid; i < (L.G2 + 31) / 32; i += NT) st.b2[i] = 0;
        k = (int)gscal[17];
        if (tid == 0) { s_n1 = 0; s_n2 = 0; s_fcount = 2; s_rcount = 0; s_stop = 0; }
        __syncthreads();
    } else {
        // ---- initial state: nothing inserted, every Mc the row's first id
        for (int i = tid; i < L.W; i += NT) st.ins[i] = 0;
        for (int w = tid; w < L.n8; w += NT) {
            uint16_t m0 = kNone16;
            if (w < n) {
                st.ptr[w] = 0;
                const uint16_t e = a.idx[(long long)w * a.ldi];
                m0 = e < n ? e : kNone16;
            }
            st.mc[w] = m0;
        }
        for (int f = tid; f < L.nf8; f += NT) {
            st.fv[f] = kNone16;
            if (f < L.nfmax) st.leaf[f] = KO::empty();
        }
        for (int g = tid; g < L.G1; g += NT) st.l1[g] = KO::empty();
        for (int g = tid; g < L.G2; g += NT) st.l2[g] = KO::empty();
        for (int i = tid; i < (L.G1 + 31) / 32; i += NT) st.b1[i] = 0;
        for (int i = tid; i < (L.G2 + 31) / 32; i += NT) st.b2[i] = 0;
        if (tid == 0) { s_n1 = 0; s_n2 = 0; s_fcount = 0; s_rcount = 0; s_stop = 0; }
        __syncthreads();
        // ---- initial 4-clique (Algorithm 1): top four row sums
        pick_clique<NT>(a.rowsum, n, s_clique, s_red_r, s_red_i);
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
                st.fu_put(f, f);
                st.mark(f);
            }
            s_fcount = 4;
            // the clique's rows whose first id is another clique vertex
            for (int i = 0; i < 4; ++i) {
                const int m0 = st.mc[c[i]];
                if (m0 != kNone16 && st.is_ins(m0)) st.row_put(s_rcount++, c[i]);
            }
        }
        __syncthreads();
        st.round(cyc_load, cyc_gain, cyc_index);
        k = 0;
    }

    // ---- main loop: one insertion per round
    const int total = n - 4;
    const int k_stop = a.k_stop < total ? a.k_stop : total;
    long long rounds = 0;
    while (k < k_stop) {
        long long c0 = clock64();
        const Key r = st.root();
        const int v = KO::is_empty(r) ? -1 : KO::vert(r);
        const int fsel = KO::is_empty(r) ? -1 : KO::face(r);
        const int nf_old = 4 + 2 * k;
        if (v < 0 || v >= n || fsel < 0 || fsel >= nf_old || st.is_ins(v)) {
            // every thread read the same root: all leave together
            if (tid == 0) s_stop = TMFG_EINTERNAL;
            break;
        }
        int4 fc = make_int4(0, 0, 0, 0);
        if (tid == 0) {
            if (globaltimer_ns() - t0 > a.timeout_ns) s_stop = TMFG_ETIMEOUT;
            fc = a.face[fsel];  // its load overlaps thread 0's share of the scans
        }
        long long c1 = clock64();
        cyc_root += c1 - c0;
        st.scan_faces(v, nf_old);
        long long c2 = clock64();
        cyc_sf += c2 - c1;
        st.scan_rows(v);
        long long c3 = clock64();
        cyc_sr += c3 - c2;
        if (tid == 0 && !s_stop) {
            // insert v into face fsel = {x < y < z}: outputs, then the faces
            // {v,x,y} (slot fsel), {v,y,z} and {v,x,z} (appended)
            const int x = fc.x, y = fc.y, z = fc.z;
            a.order[4 + k] = v;
            int *e = a.edges + 2 * (6 + 3 * k);
            e[0] = v; e[1] = x; e[2] = v; e[3] = y; e[4] = v; e[5] = z;
            a.ins_face[3 * k + 0] = x;
            a.ins_face[3 * k + 1] = y;
            a.ins_face[3 * k + 2] = z;
            a.parent[k + 1] = fc.w;
            st.ins[v >> 5] |= 1u << (v & 31);
            const int bub = k + 1;
            auto sorted = [&](int p, int q, int s) {
                int t;
                if (p > q) { t = p; p = q; q = t; }
                if (q > s) { t = q; q = s; s = t; }
                if (p > q) { t = p; p = q; q = t; }
                return make_int4(p, q, s, bub);
            };
            a.face[fsel] = sorted(v, x, y);
            a.face[nf_old] = sorted(v, y, z);
            a.face[nf_old + 1] = sorted(v, x, z);
            st.fv[nf_old] = kNone16;
            st.fv[nf_old + 1] = kNone16;
            st.fu_put(0, nf_old);
            st.fu_put(1, nf_old + 1);
            st.mark(nf_old);
            st.mark(nf_old + 1);
            // v's own row, if its Mc was inserted before v
            const int mv = st.mc[v];
            if (mv != kNone16 && st.is_ins(mv)) st.row_put(atomicAdd(&s_rcount, 1), v);
        }
        long long c4 = clock64();
        cyc_ins += c4 - c3;
        __syncthreads();
        cyc_scan += clock64() - c1;
        if (s_stop) break;
        st.round(cyc_load, cyc_gain, cyc_index);
        ++k;
        ++rounds;
    }

    // ---- statistics (summed over segments) and the state for the next segment
    if (st.c_rows) atomicAdd(&s_cnt[0], (unsigned long long)st.c_rows);
    if (st.c_cont) atomicAdd(&s_cnt[1], (unsigned long long)st.c_cont);
    if (st.c_steps) atomicAdd(&s_cnt[2], (unsigned long long)st.c_steps);
    if (st.c_evals) atomicAdd(&s_cnt[3], (unsigned long long)st.c_evals);
    __syncthreads();
    const Key rfin = st.root();  // a warp-wide reduction: every warp computes it
    if (tid == 0) {
        if (s_stop) set_status(a.status, s_stop);
        // slots: 0 face evaluations, 2 pointer steps, 3 rounds, 4 ns; cycles
        // (thread 0): 5 scans + insertion + barrier, 6 index, 7 root, 8 loads
        // and row refreshes, 10 gathers; 11 rows refreshed, 12 rows that took
        // more than one step, 13 the steps beyond the first; the scan phase
        // in parts: 1 face scan, 9 row scan, 14 insertion (the rest of 5 is
        // the barrier wait); 15 thread 0's own share of the gathers
        const long long seg[16] = {(long long)s_cnt[3], cyc_sf, (long long)s_cnt[2], rounds,
                                   (long long)(globaltimer_ns() - t0), cyc_scan, cyc_index, cyc_root,
                                   cyc_load, cyc_sr, cyc_gain, (long long)s_cnt[0],
                                   (long long)s_cnt[1], (long long)(s_cnt[2] - s_cnt[0]), cyc_ins,
                                   st.cyc_own};
        for (int i = 0; i < 16; ++i) {
            acc[i] += seg[i];
            a.stats[i] = acc[i];
            if (gs) gscal[i] = acc[i];
        }
        if (gs) {
            gscal[16] = 4 + 2 * k;
            gscal[17] = k;
            Key *gr = reinterpret_cast<Key *>(gs + SL.off_roots);
            gr[0] = rfin;
            gr[1] = KO::empty();
        }
    }
    if (gs && k < total && !s_stop) {
        uint32_t *gins = reinterpret_cast<uint32_t *>(gs + SL.off_ins);
        uint16_t *gmc = reinterpret_cast<uint16_t *>(gs + SL.off_mc);
        uint16_t *gptr = reinterpret_cast<uint16_t *>(gs + SL.off_ptr);
        uint16_t *gfv = reinterpret_cast<uint16_t *>(gs + SL.off_fv);
        Key *gt = reinterpret_cast<Key *>(gs + SL.off_tree[0]);
        for (int i = tid; i < L.W; i += NT) gins[i] = st.ins[i];
        for (int w = tid; w < n; w += NT) {
            gmc[w] = st.mc[w];
            if (!GP) gptr[w] = st.ptr[w];
        }
        for (int f = tid; f < L.nfmax; f += NT) gfv[f] = st.fv[f];
        for (int i = tid; i < L.G1; i += NT) gt[i] = st.l1[i];
        for (int i = tid; i < L.G2; i += NT) gt[L.G1 + i] = st.l2[i];
    }
}

// One instance per launch (the arguments by value).
template <typename T, int NT, int PL, bool GP>
__global__ void __launch_bounds__(NT, 1) tmfg_corr1_kernel(LoopArgs a)
{
    corr1_body<T, NT, PL, GP>(a);
}

// Many instances per launch: CTA b runs instance b.
template <typename T, int NT, int PL>
__global__ void __launch_bounds__(NT, NT > 256 ? 1 : 2) tmfg_corr1_batch_kernel(const LoopArgs *args)
{
    __shared__ LoopArgs s_args;
    if (threadIdx.x == 0) s_args = args[blockIdx.x];
    __syncthreads();
    corr1_body<T, NT, PL, false>(s_args);
}

// ------------------------------------------------------------------- host

size_t corr1_smem_bytes(int n, int dtype, int groups, bool gp)
{
    const size_t ks = dtype == TMFG_F32 ? sizeof(unsigned long long) : sizeof(Key128);
    return corr1_layout(n, ks, groups, gp).total;
}

int corr1_fit_groups(int n, int dtype, int want, size_t limit, bool gp)
{
    const size_t ks = dtype == TMFG_F32 ? sizeof(unsigned long long) : sizeof(Key128);
    const size_t base = corr1_layout(n, ks, 0, gp).total;
    if (base > limit) return -1;
    size_t g = (limit - base) / (32 * ks);
    if (g > (size_t)kC1StageMax) g = kC1StageMax;
    return want < (int)g ? want : (int)g;
}

bool corr1_shape_ok(int threads, int lanes)
{
    return (threads == 256 && (lanes == 4 || lanes == 8 || lanes == 16)) ||
           (threads == 512 && (lanes == 8 || lanes == 16));
}

namespace {
template <typename T, int NT, int PL, bool GP>
int go_corr1(const LoopArgs *a, const LoopArgs *d_args, int count, size_t smem, int ctas,
             cudaStream_t stream)
{
    const void *kp = a ? (const void *)tmfg_corr1_kernel<T, NT, PL, GP>
                       : (const void *)tmfg_corr1_batch_kernel<T, NT, PL>;
    if (cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kp, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carveout_percent(smem, ctas)) != cudaSuccess)
        return TMFG_ECUDA;
    if (a)
        tmfg_corr1_kernel<T, NT, PL, GP><<<1, NT, smem, stream>>>(*a);
    else
        tmfg_corr1_batch_kernel<T, NT, PL><<<count, NT, smem, stream>>>(d_args);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

template <typename T>
int go_corr1_shape(int threads, int lanes, const LoopArgs *a, const LoopArgs *d_args, int count,
                   size_t smem, int ctas, cudaStream_t stream)
{
    if (threads == 512)
        return lanes == 16 ? go_corr1<T, 512, 16, false>(a, d_args, count, smem, ctas, stream)
                           : go_corr1<T, 512, 8, false>(a, d_args, count, smem, ctas, stream);
    if (lanes == 4) return go_corr1<T, 256, 4, false>(a, d_args, count, smem, ctas, stream);
    if (lanes == 16) return go_corr1<T, 256, 16, false>(a, d_args, count, smem, ctas, stream);
    return go_corr1<T, 256, 8, false>(a, d_args, count, smem, ctas, stream);
}
}  // namespace

int launch_corr1(const LoopArgs &a, const LoopShape &shape, int dtype, size_t smem, bool gp,
                 cudaStream_t stream)
{
    if (gp) {  // large n: the one shape with pointers in global memory
        if (!a.state) return TMFG_EINVAL;
        return dtype == TMFG_F32 ? go_corr1<float, 256, 8, true>(&a, nullptr, 1, smem, 1, stream)
                                 : go_corr1<double, 256, 8, true>(&a, nullptr, 1, smem, 1, stream);
    }
    if (dtype == TMFG_F32)
        return go_corr1_shape<float>(shape.threads, shape.lanes, &a, nullptr, 1, smem, 1, stream);
    return go_corr1_shape<double>(shape.threads, shape.lanes, &a, nullptr, 1, smem, 1, stream);
}

int launch_corr1_batch(const LoopArgs *d_args, int count, const LoopShape &shape, int dtype,
                       size_t smem, cudaStream_t stream)
{
    if (dtype == TMFG_F32)
        return go_corr1_shape<float>(shape.threads, shape.lanes, nullptr, d_args, count, smem, 2,
                                     stream);
    return go_corr1_shape<double>(shape.threads, shape.lanes, nullptr, d_args, count, smem, 2,
                                  stream);
}

}  // namespace tmfg
