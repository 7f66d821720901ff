// tmfg_loop.cu -- the greedy TMFG insertion loop (Algorithm 1 corr-tmfg with
// prefix P, Algorithm 2 heap-tmfg), entirely on the device.
//
// One CTA runs the whole sequence of n-4 insertions with no host round trip.
//
// Keys.  A face-vertex pair ranks by (gain desc, vertex asc, face id asc).
// For float input the whole rank is one 64-bit word: the order-preserving
// image of the gain in the high 32 bits, then 0xFFFF-vertex and 0xFFFF-face
// (n <= 32770 keeps both in 16 bits), so a pair comparison is one unsigned
// compare; for double input the gain image takes 64 bits and a second word
// holds the rest.  Key 0 means "no pair".
//
// Max index.  For a set of faces, a two-level index: level 1 = max of each
// group of 32 face keys (the keys themselves, the leaves, live in global
// memory and stay in L2), level 2 = max of each group of 32 level-1 nodes,
// then a root.  Writers mark the groups they touch; one batched update
// recomputes the marked groups (a warp per group) and the root.
//
// MaxCorrs[w] is read fresh: the cached Mc[w] is kept while uninserted, else
// the lazily advanced pointer of Section 4.3 moves on -- first the next 64
// sorted ids are probed (corr-tmfg: by a group of 8 lanes, one 16-byte load
// and 8 inserted-bitmap checks each, the rows to probe listed while the
// update's vertices are gathered; heap-tmfg: by one thread, eight 16-byte
// loads), and only rows whose probe finds nothing go to a warp that scans
// 256 sorted ids per step with 16-byte loads and a ballot.  A face's best
// vertex is computed by one thread: 9 independent gathers S[x,u] (3
// candidates u x 3 face vertices x), gain = (S[a,u] + S[b,u]) + S[c,u] with
// round-to-nearest adds in the dtype of S, ties to the smaller u.
//
// Segments.  The loop runs as a few launches (ending after 1/2, 3/4, ...,
// 31/32 of the insertions); between them every sorted row is compacted to
// its uninserted ids, so the pointers of late insertions do not wade through
// long runs of inserted ids.  The loop state is saved to global memory at
// the end of a segment and restored at the start of the next.
//
// corr-tmfg: one index over all faces.  A round takes the P best pairs
// (repeated extraction), keeps the first pair of each vertex, inserts in
// rank order, and recomputes F_update = {faces whose stored vertex was
// inserted} + {new faces}.
//
// heap-tmfg: each face has exactly one heap entry, so Algorithm 2's pop is
// the argmax over the faces' stored keys.  The faces are split between two
// indexes: FRESH (stored vertex uninserted) and STALE (stored vertex
// inserted).  After inserting v, the faces whose stored vertex is v move to
// STALE keeping their (stale) keys, and their recomputation with the current
// MaxCorrs is done at once, in parallel with the three new faces, and kept
// as a pending result with the three candidates it used.  Algorithm 2 pops
// stale faces in key order until the top of the heap is fresh; that epoch
// is resolved in one batch: the stale faces ranking above the best fresh
// key are extracted, sorted, and scanned in order -- a stale face is popped
// while its stale key ranks above the running best, and its pending key
// joins the running best.  A pending result is what a recompute at pop time
// gives as long as its three candidates are still uninserted (the first
// uninserted entry of a sorted row cannot change otherwise); if one was
// inserted meanwhile, the face is recomputed before the scan.
//
// Every loop checks the device clock and stops with TMFG_ETIMEOUT past its
// limit, so the kernel always terminates.
#include <climits>

#include "loop_common.cuh"

namespace tmfg {

size_t loop_state_bytes(int n) { return state_layout(n, sizeof(Key128)).total; }

template <typename T>
struct Loop {
    using KO = KeyOps<T>;
    using Key = typename KO::Key;
    const LoopArgs &a;
    const T *S;
    int n, nfmax, G1, G2;
    uint32_t *ins, *vmark, *rnd;
    uint16_t *mc, *ptr, *fv;
    Tree<KO> tf, ts;  // FRESH (all faces in corr mode), STALE (heap mode)
    int *vlist, *vslowlist, *plist;
    int *pcount;
    Key *sel, *xkey, *xpend;
    int *xf;
    uint16_t *xs, *q1x, *q2x;
    Key *pend_key;
    unsigned long long *pend_cand;
    // shared scalars
    int *nf, *k, *vcount, *vslow, *scan_chunks, *face_evals;
    int *probes, *warp_refreshes, *warp_steps;
    // this thread's share of the counters, added to them once per segment
    int n_scan = 0, n_probes = 0, n_wsteps = 0, n_evals = 0;
    __device__ void flush_counters()
    {
        if (n_scan) atomicAdd(scan_chunks, n_scan);
        if (n_probes) atomicAdd(probes, n_probes);
        if (n_wsteps) atomicAdd(warp_steps, n_wsteps);
        if (n_evals) atomicAdd(face_evals, n_evals);
    }
    long long cyc_push = 0, cyc_refresh = 0, cyc_gain = 0;  // thread 0's view

    __device__ bool is_ins(int v) const { return (ins[v >> 5] >> (v & 31)) & 1u; }

    // Append to the face-update list every face f < nf whose stored vertex
    // is v.  Eight stored vertices per 16-byte load; a branch-free test
    // (some 16-bit lane of x ^ vv is zero) filters the loads, the exact
    // per-lane comparison runs only on a hit.
    __device__ void scan_faces_of(int v, int nf, int *count)
    {
        const uint32_t vv = (uint32_t)v | ((uint32_t)v << 16);
        const uint4 *fv8 = reinterpret_cast<const uint4 *>(fv);
        const int nq = (nf + 7) >> 3;
        for (int i = threadIdx.x; i < nq; i += kLoopThreads) {
            const uint4 q = fv8[i];
            const uint32_t x0 = q.x ^ vv, x1 = q.y ^ vv, x2 = q.z ^ vv, x3 = q.w ^ vv;
            auto z = [](uint32_t y) { return (y - 0x00010001u) & ~y & 0x80008000u; };
            if (!(z(x0) | z(x1) | z(x2) | z(x3))) continue;  // no lane equals v
            const uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
            for (int h = 0; h < 4; ++h)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int f = 8 * i + 2 * h + b;
                    if (f < nf && ((xs[h] >> (16 * b)) & 0xFFFFu) == 0)
                        fu_put(atomicAdd(count, 1), f | (kToFresh << 28));
                }
        }
    }
    int *fus;  // the face-update list's first kFuCap entries (the rest in a.fu_buf)
    __device__ int fu_get(int i) const { return i < kFuCap ? fus[i] : a.fu_buf[i]; }
    __device__ void fu_put(int i, int e)
    {
        if (i < kFuCap) fus[i] = e;
        else a.fu_buf[i] = e;
    }

    // Fresh MaxCorrs of vertex w (one warp): keep Mc[w] while uninserted,
    // else advance ptr[w] to the first uninserted entry of row w.  An id
    // >= n (0xFFFF) ends the row.
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
            }
#pragma unroll
            for (int t = 7; t >= 0; --t) {
                const int q = q0 + t;
                if (q >= p && (q >= mlen || e[t] >= n || !is_ins(e[t]))) first = t;
            }
            if (lane == 0) {
                ++n_scan;
                ++n_wsteps;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, first < 8);
            if (bal) {
                const int src = __ffs(bal) - 1;
                const int t = __shfl_sync(0xffffffffu, first, src);
                int hit = kNone16;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (u == t) hit = e[u];
                hit = __shfl_sync(0xffffffffu, hit, src);
                const int q = base + src * 8 + t;
                if (lane == 0) {
                    if (q < mlen && hit < n) {
                        ptr[w] = (uint16_t)q;
                        mc[w] = (uint16_t)hit;
                    } else {
                        ptr[w] = (uint16_t)(q < mlen ? q : mlen);
                        mc[w] = kNone16;
                    }
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

    // One thread's first look for the fresh MaxCorrs of w: the 64 sorted ids
    // from ptr[w] + 1 rounded down to 8 (eight 16-byte loads).  Returns false
    // if w still needs the warp-wide scan.
    __device__ bool refresh_probe(int w)
    {
        const uint16_t m = mc[w];
        if (m == kNone16 || !is_ins(m)) return true;
        const int mlen = n - 1;
        const int p = ptr[w] + 1;
        if (p >= mlen) {
            ptr[w] = (uint16_t)mlen;
            mc[w] = kNone16;
            return true;
        }
        const uint16_t *row = a.idx + (long long)w * a.ldi;
        const int base = p & ~7;
        uint4 c[8];
#pragma unroll
        for (int h = 0; h < 8; ++h)
            c[h] = base + 8 * h < a.ldi ? *reinterpret_cast<const uint4 *>(row + base + 8 * h)
                                        : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        ++n_scan;
        ++n_probes;
        // all 64 checks independent (their shared-memory reads overlap); the
        // first candidate wins
        int first = 64, hit = kNone16;
#pragma unroll
        for (int j = 63; j >= 0; --j) {
            const uint4 &cc = c[j >> 3];
            const uint32_t wd = ((j >> 1) & 3) == 0 ? cc.x : ((j >> 1) & 3) == 1 ? cc.y
                              : ((j >> 1) & 3) == 2 ? cc.z : cc.w;
            const int e = (wd >> (16 * (j & 1))) & 0xFFFF;
            const int q = base + j;
            const bool stop = q >= mlen || e >= n;
            const bool cand = q >= p && (stop || !is_ins(e));
            if (cand) { first = j; hit = stop ? kNone16 : e; }
        }
        if (first < 64) {
            const int q = base + first;
            if (hit != kNone16) {
                ptr[w] = (uint16_t)q;
                mc[w] = (uint16_t)hit;
            } else {
                ptr[w] = (uint16_t)(q < mlen ? q : mlen);
                mc[w] = kNone16;
            }
            return true;
        }
        ptr[w] = (uint16_t)(base + 63);  // all 64 inserted (so base + 63 < mlen)
        return false;
    }

    // The first look for row w by an 8-lane group (lanes 8g..8g+7 of a warp,
    // sl = lane & 7): each lane loads 8 sorted ids (16 bytes), the group's
    // first candidate wins.  Same outcome as refresh_probe.  Returns false
    // (to every lane of the group) if w still needs the warp-wide scan.
    __device__ bool refresh_probe8(int w)
    {
        const int lane = threadIdx.x & 31, sl = lane & 7, g0 = lane & ~7;
        const unsigned gmask = 0xFFu << g0;
        const int mlen = n - 1;
        const int p = ptr[w] + 1;
        if (p >= mlen) {
            __syncwarp(gmask);
            if (sl == 0) { ptr[w] = (uint16_t)mlen; mc[w] = kNone16; }
            return true;
        }
        const uint16_t *row = a.idx + (long long)w * a.ldi;
        const int base = p & ~7;
        const int q0 = base + 8 * sl;
        uint16_t e[8] = {kNone16, kNone16, kNone16, kNone16, kNone16, kNone16, kNone16, kNone16};
        if (q0 < a.ldi) {
            const uint4 c = *reinterpret_cast<const uint4 *>(row + q0);
            e[0] = c.x & 0xFFFF; e[1] = c.x >> 16; e[2] = c.y & 0xFFFF; e[3] = c.y >> 16;
            e[4] = c.z & 0xFFFF; e[5] = c.z >> 16; e[6] = c.w & 0xFFFF; e[7] = c.w >> 16;
        }
        int first = 8;
#pragma unroll
        for (int t = 7; t >= 0; --t) {
            const int q = q0 + t;
            if (q >= p && (q >= mlen || e[t] >= n || !is_ins(e[t]))) first = t;
        }
        int hit = kNone16;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u == first) hit = e[u];
        const unsigned bal = (__ballot_sync(gmask, first < 8) >> g0) & 0xFFu;
        if (bal) {
            const int src = g0 + __ffs(bal) - 1;
            const int t = __shfl_sync(gmask, first, src);
            const int h = __shfl_sync(gmask, hit, src);
            if (sl == 0) {
                const int q = base + (src - g0) * 8 + t;
                ++n_scan;
                ++n_probes;
                if (q < mlen && h < n) {
                    ptr[w] = (uint16_t)q;
                    mc[w] = (uint16_t)h;
                } else {
                    ptr[w] = (uint16_t)(q < mlen ? q : mlen);
                    mc[w] = kNone16;
                }
            }
            return true;
        }
        if (sl == 0) {
            ++n_scan;
            ++n_probes;
            ptr[w] = (uint16_t)(base + 63);  // all 64 inserted (so base + 63 < mlen)
        }
        return false;
    }

    // Best vertex of face f = {fc.x < fc.y < fc.z} from the fresh MaxCorrs of
    // its vertices (one thread: 9 independent gathers), stored per dest.
    __device__ void face_best_thread(int f, int4 fc, int dest)
    {
        const int cs[3] = {mc[fc.x], mc[fc.y], mc[fc.z]};
        const int xs[3] = {fc.x, fc.y, fc.z};
        Key old = KO::empty();
        if (dest == kToPendMove) old = tf.leaf[f];
        T v[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                v[i][j] = (cs[i] != kNone16 && cs[i] < n) ? S[(long long)xs[j] * a.ld + cs[i]] : T(0);
        int bv = -1;
        T bg = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int c = cs[i];
            if (c == kNone16 || c >= n) continue;
            const T g = canon(add_rn(add_rn(canon(v[i][0]), canon(v[i][1])), canon(v[i][2])));
            if (bv < 0 || g > bg || (g == bg && c < bv)) { bv = c; bg = g; }
        }
        const Key key = bv < 0 ? KO::empty() : KO::make(bg, bv, f);
        if (dest == kToFresh) {
            tf.set(f, key);
            fv[f] = bv < 0 ? kNone16 : (uint16_t)bv;
        } else {
            pend_key[f] = key;
            pend_cand[f] = (unsigned long long)(unsigned)cs[0] |
                           ((unsigned long long)(unsigned)cs[1] << 16) |
                           ((unsigned long long)(unsigned)cs[2] << 32);
            if (dest == kToPendMove) {
                ts.set(f, old);
                tf.set(f, KO::empty());
            }
        }
        ++n_evals;
    }

    // Recompute the faces of the face-update list [0..cnt): entry = face |
    // dest << 28.  One thread per face, one thread per vertex to refresh (a
    // warp per vertex when the first 64 sorted ids are all inserted).  Ends
    // synchronised.
    __device__ void recompute(int cnt)
    {
        const int tid = threadIdx.x, warp = tid >> 5;
        for (int c0 = 0; c0 < cnt; c0 += kChunk) {
            const int m = cnt - c0 < kChunk ? cnt - c0 : kChunk;
            long long c0t = clock64();
            if (tid == 0) { *vcount = 0; *vslow = 0; *pcount = 0; }
            __syncthreads();
            int4 fc = make_int4(0, 0, 0, 0);
            int fe = 0;
            // thread t keeps face t for its evaluation; the marks of the
            // 3m (face, vertex) pairs are spread over all threads, one
            // dependent chain of shared-memory atomics each
            const int np3 = 3 * m;
            int pf[2], pj[2];
            int4 pc[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int q = tid + r * kLoopThreads;
                pf[r] = q < np3 ? fu_get(c0 + q / 3) & 0x0FFFFFFF : -1;
                pj[r] = q % 3;
            }
            if (tid < m) {
                fe = fu_get(c0 + tid);
                fc = a.face[fe & 0x0FFFFFFF];
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) pc[r] = pf[r] >= 0 ? a.face[pf[r]] : make_int4(0, 0, 0, 0);
            for (int q = tid + 2 * kLoopThreads; q < np3; q += kLoopThreads) {
                // more than 2 pairs per thread: only for chunks of over 170 faces
                const int4 c = a.face[fu_get(c0 + q / 3) & 0x0FFFFFFF];
                const int w = q % 3 == 0 ? c.x : q % 3 == 1 ? c.y : c.z;
                const uint32_t bit = 1u << (w & 31);
                if (!(atomicOr(&vmark[w >> 5], bit) & bit)) {
                    vlist[atomicAdd(vcount, 1)] = w;
                    const uint16_t mw = mc[w];
                    if (plist && mw != kNone16 && is_ins(mw)) plist[atomicAdd(pcount, 1)] = w;
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (pf[r] < 0) continue;
                const int w = pj[r] == 0 ? pc[r].x : pj[r] == 1 ? pc[r].y : pc[r].z;
                const uint32_t bit = 1u << (w & 31);
                if (!(atomicOr(&vmark[w >> 5], bit) & bit)) {
                    vlist[atomicAdd(vcount, 1)] = w;
                    const uint16_t mw = mc[w];
                    if (plist && mw != kNone16 && is_ins(mw)) plist[atomicAdd(pcount, 1)] = w;
                }
            }
            __syncthreads();
            long long c1t = clock64();
            cyc_push += c1t - c0t;
            const int nv = *vcount;
            if (plist) {
                // rows whose MaxCorrs was inserted: an 8-lane group each
                const int np = *pcount;
                for (int i = tid >> 3; i < np; i += kLoopThreads / 8) {
                    const int w = plist[i];
                    if (!refresh_probe8(w) && (tid & 7) == 0) vslowlist[atomicAdd(vslow, 1)] = w;
                }
            } else {
                for (int i = tid; i < nv; i += kLoopThreads) {
                    const int w = vlist[i];
                    if (!refresh_probe(w)) vslowlist[atomicAdd(vslow, 1)] = w;
                }
            }
            __syncthreads();
            const int ns = *vslow;
            if (tid == 0) *warp_refreshes += ns;
            for (int i = warp; i < ns; i += kLoopWarps) refresh(vslowlist[i]);
            __syncthreads();
            long long c2t = clock64();
            cyc_refresh += c2t - c1t;
            // the gathers first, then the marks' clearing (needed by the next
            // chunk or insertion only, after the barrier)
            if (tid < m) face_best_thread(fe & 0x0FFFFFFF, fc, (fe >> 28) & 3);
            for (int i = tid; i < nv; i += kLoopThreads) {
                const int w = vlist[i];
                atomicAnd(&vmark[w >> 5], ~(1u << (w & 31)));
            }
            __syncthreads();
            cyc_gain += clock64() - c2t;
        }
    }

    // Level-1 recompute of the marked groups of index x: a warp takes up to 4
    // groups at once, with all their leaf loads in flight together.
    __device__ void update_l1(Tree<KO> &x)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int c1 = *x.n1;
        for (int i0 = 4 * warp; i0 < c1; i0 += 4 * kLoopWarps) {
            Key v[4];
            int g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                g[u] = i0 + u < c1 ? x.q1[i0 + u] : -1;
                const int f = g[u] * 32 + lane;
                v[u] = (g[u] >= 0 && f < nfmax) ? x.leaf[f] : KO::empty();
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (g[u] < 0) break;
                const Key m = warp_max<KO>(v[u]);
                if (lane == 0) {
                    x.l1[g[u]] = m;
                    atomicAnd(&x.b1[g[u] >> 5], ~(1u << (g[u] & 31)));
                    const int g2 = g[u] >> 5;
                    const uint32_t bit = 1u << (g2 & 31);
                    if (!(atomicOr(&x.b2[g2 >> 5], bit) & bit)) x.q2[atomicAdd(x.n2, 1)] = (uint16_t)g2;
                }
            }
        }
    }
    __device__ void update_l2(Tree<KO> &x)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int c2 = *x.n2;
        for (int i = warp; i < c2; i += kLoopWarps) {
            const int g = x.q2[i];
            const int j = g * 32 + lane;
            Key v = j < G1 ? x.l1[j] : KO::empty();
            v = warp_max<KO>(v);
            if (lane == 0) {
                x.l2[g] = v;
                atomicAnd(&x.b2[g >> 5], ~(1u << (g & 31)));
            }
        }
    }
    __device__ void update_root(Tree<KO> &x)
    {
        const int lane = threadIdx.x & 31;
        Key v = lane < G2 ? x.l2[lane] : KO::empty();
        const Key y = lane + 32 < G2 ? x.l2[lane + 32] : KO::empty();
        if (KO::gt(y, v)) v = y;
        v = warp_max<KO>(v);
        if (lane == 0) {
            *x.root = v;
            *x.n1 = 0;
            *x.n2 = 0;
        }
    }

    // Batched update of the marked groups of the FRESH index (and of the
    // STALE index when both is set).  Starts and ends synchronised.
    __device__ void update(int both)
    {
        const int warp = threadIdx.x >> 5;
        __syncthreads();
        update_l1(tf);
        if (both) update_l1(ts);
        __syncthreads();
        update_l2(tf);
        if (both) update_l2(ts);
        __syncthreads();
        if (warp == 0) update_root(tf);
        if (both && warp == 1) update_root(ts);
        __syncthreads();
    }

    // Thread 0 only: insert v into face f; writes the outputs and the 3 new
    // faces (slot f, then nf, nf+1).
    __device__ void insert_pair(int v, int f, bool have_face = false,
                                int4 known = make_int4(0, 0, 0, 0))
    {
        const int4 fc = have_face ? known : a.face[f];
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
        *nf = nfc + 2;
        *k = kk + 1;
    }

    __device__ bool pend_valid(int f) const
    {
        const unsigned long long c = pend_cand[f];
        if (KO::is_empty(pend_key[f])) return false;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int u = (int)((c >> (16 * i)) & 0xFFFFu);
            if (u != kNone16 && (u >= n || is_ins(u))) return false;
        }
        return true;
    }
};

// kHeap selects Algorithm 2 (heap-tmfg) or Algorithm 1 (corr-tmfg) at
// compile time: each kernel holds only its own path, which keeps the code
// that one SM runs for every insertion compact.
template <typename T, bool kHeap>
__device__ __forceinline__ void loop_body(const LoopArgs &a)
{
    using KO = KeyOps<T>;
    using Key = typename KO::Key;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Key s_root[2], s_win;
    __shared__ int s_n1[2], s_n2[2];
    __shared__ int s_vslow, s_pcount;
    __shared__ int s_nf, s_k, s_vcount, s_scan, s_evals, s_stop, s_nsel, s_fcount;
    __shared__ int s_nx, s_ninv, s_nq1, s_np, s_more;
    __shared__ int s_probes, s_wref, s_wsteps;
    __shared__ Key s_tau;
    __shared__ int s_clique[4];
    __shared__ long long s_red_r[kLoopWarps];
    __shared__ int s_red_i[kLoopWarps];

    const int tid = threadIdx.x;
    const int n = a.n;
    if (*(volatile int *)a.status != 0) return;  // an earlier step failed
    const uint64_t t0 = globaltimer_ns();
    constexpr bool heap = kHeap;
    const LoopLayout L = loop_layout(n, sizeof(Key), heap ? 2 : 1);

    Loop<T> st{a};
    st.S = reinterpret_cast<const T *>(a.S);
    st.n = n;
    st.nfmax = L.nfmax;
    st.G1 = L.G1;
    st.G2 = L.G2;
    st.ins = reinterpret_cast<uint32_t *>(smem + L.off_ins);
    st.vmark = reinterpret_cast<uint32_t *>(smem + L.off_vmark);
    st.rnd = reinterpret_cast<uint32_t *>(smem + L.off_rnd);
    st.mc = reinterpret_cast<uint16_t *>(smem + L.off_mc);
    st.ptr = reinterpret_cast<uint16_t *>(smem + L.off_ptr);
    st.fv = reinterpret_cast<uint16_t *>(smem + L.off_fv);
    auto bind = [&](Tree<KO> &x, int t, void *leaf) {
        unsigned char *b = smem + L.off_tree[t];
        size_t o = 0;
        x.leaf = reinterpret_cast<Key *>(leaf);
        x.l1 = reinterpret_cast<Key *>(b + o);      o = align16(o + sizeof(Key) * (size_t)L.G1);
        x.l2 = reinterpret_cast<Key *>(b + o);      o = align16(o + sizeof(Key) * (size_t)L.G2);
        x.b1 = reinterpret_cast<uint32_t *>(b + o); o = align16(o + 4 * (size_t)((L.G1 + 31) / 32));
        x.b2 = reinterpret_cast<uint32_t *>(b + o); o = align16(o + 4 * (size_t)((L.G2 + 31) / 32));
        x.q1 = reinterpret_cast<uint16_t *>(b + o); o = align16(o + 2 * (size_t)L.G1);
        x.q2 = reinterpret_cast<uint16_t *>(b + o);
        x.n1 = &s_n1[t];
        x.n2 = &s_n2[t];
        x.root = &s_root[t];
    };
    bind(st.tf, 0, a.leaf_fresh);
    bind(st.ts, 1, a.leaf_stale);
    st.vlist = reinterpret_cast<int *>(smem + L.off_vlist);
    st.vslowlist = reinterpret_cast<int *>(smem + L.off_vslow);
    st.plist = heap ? nullptr : reinterpret_cast<int *>(smem + L.off_plist);
    st.pcount = &s_pcount;
    st.fus = reinterpret_cast<int *>(smem + L.off_fus);
    st.sel = reinterpret_cast<Key *>(smem + L.off_sel);
    st.xf = reinterpret_cast<int *>(smem + L.off_x);
    st.xkey = reinterpret_cast<Key *>(smem + L.off_xkey);
    st.xpend = reinterpret_cast<Key *>(smem + L.off_xpend);
    st.xs = reinterpret_cast<uint16_t *>(smem + L.off_xs);
    st.q1x = reinterpret_cast<uint16_t *>(smem + L.off_q1x);
    st.q2x = reinterpret_cast<uint16_t *>(smem + L.off_q2x);
    st.pend_key = reinterpret_cast<Key *>(a.pend_key);
    st.pend_cand = a.pend_cand;
    st.nf = &s_nf;
    st.k = &s_k;
    st.vcount = &s_vcount;
    st.vslow = &s_vslow;
    st.scan_chunks = &s_scan;
    st.face_evals = &s_evals;
    st.probes = &s_probes;
    st.warp_refreshes = &s_wref;
    st.warp_steps = &s_wsteps;

    const StateLayout SL = state_layout(n, sizeof(Key128));
    unsigned char *gs = reinterpret_cast<unsigned char *>(a.state);
    long long *gscal = reinterpret_cast<long long *>(gs + SL.off_scal);
    // stats carried across segments: 0 evals, 1 stale, 2 scan, 3 rounds, 4 ns,
    // 5..14 cycle counters, 15 epoch iterations; 16 nf, 17 k
    long long acc[16];
    for (int i = 0; i < 16; ++i) acc[i] = 0;
    if (a.resume) {
        for (int i = 0; i < 16; ++i) acc[i] = gscal[i];
        const uint32_t *gins = reinterpret_cast<const uint32_t *>(gs + SL.off_ins);
        const uint16_t *gmc = reinterpret_cast<const uint16_t *>(gs + SL.off_mc);
        const uint16_t *gptr = reinterpret_cast<const uint16_t *>(gs + SL.off_ptr);
        const uint16_t *gfv = reinterpret_cast<const uint16_t *>(gs + SL.off_fv);
        for (int i = tid; i < L.W; i += kLoopThreads) { st.ins[i] = gins[i]; st.vmark[i] = 0; st.rnd[i] = 0; }
        for (int w = tid; w < n; w += kLoopThreads) { st.mc[w] = gmc[w]; st.ptr[w] = gptr[w]; }
        for (int f = tid; f < L.nfmax; f += kLoopThreads) st.fv[f] = gfv[f];
        auto load_tree = [&](Tree<KO> &x, int t) {
            const Key *g = reinterpret_cast<const Key *>(gs + SL.off_tree[t]);
            for (int i = tid; i < L.G1; i += kLoopThreads) x.l1[i] = g[i];
            for (int i = tid; i < L.G2; i += kLoopThreads) x.l2[i] = g[L.G1 + i];
            for (int i = tid; i < (L.G1 + 31) / 32; i += kLoopThreads) x.b1[i] = 0;
            for (int i = tid; i < (L.G2 + 31) / 32; i += kLoopThreads) x.b2[i] = 0;
        };
        load_tree(st.tf, 0);
        if (heap) load_tree(st.ts, 1);
        if (tid == 0) {
            const Key *gr = reinterpret_cast<const Key *>(gs + SL.off_roots);
            s_nf = (int)gscal[16]; s_k = (int)gscal[17];
            s_vcount = 0; s_scan = 0; s_evals = 0; s_stop = 0; s_nsel = 0; s_fcount = 0;
            s_probes = 0; s_wref = 0; s_wsteps = 0;
            s_n1[0] = s_n1[1] = s_n2[0] = s_n2[1] = 0;
            s_root[0] = gr[0];
            s_root[1] = heap ? gr[1] : KO::empty();
        }
        __syncthreads();
    } else {
    // ---- initial state
        for (int i = tid; i < L.W; i += kLoopThreads) { st.ins[i] = 0; st.vmark[i] = 0; st.rnd[i] = 0; }
        for (int w = tid; w < n; w += kLoopThreads) {
            st.ptr[w] = 0;
            const uint16_t m0 = a.idx[(long long)w * a.ldi];
            st.mc[w] = m0 < n ? m0 : kNone16;
        }
        for (int f = tid; f < L.nfmax; f += kLoopThreads) {
            st.fv[f] = kNone16;
            st.tf.leaf[f] = KO::empty();
            if (heap) {
                st.ts.leaf[f] = KO::empty();
                st.pend_key[f] = KO::empty();
            }
        }
        auto clear_tree = [&](Tree<KO> &x) {
            for (int g = tid; g < L.G1; g += kLoopThreads) x.l1[g] = KO::empty();
            for (int g = tid; g < L.G2; g += kLoopThreads) x.l2[g] = KO::empty();
            for (int i = tid; i < (L.G1 + 31) / 32; i += kLoopThreads) x.b1[i] = 0;
            for (int i = tid; i < (L.G2 + 31) / 32; i += kLoopThreads) x.b2[i] = 0;
        };
        clear_tree(st.tf);
        if (heap) clear_tree(st.ts);
        if (tid == 0) {
            s_nf = 4; s_k = 0; s_vcount = 0; s_scan = 0; s_evals = 0; s_stop = 0; s_nsel = 0;
            s_probes = 0; s_wref = 0; s_wsteps = 0;
            s_fcount = 0;
            s_n1[0] = s_n1[1] = s_n2[0] = s_n2[1] = 0;
            s_root[0] = s_root[1] = KO::empty();
        }
        __syncthreads();

        // ---- initial 4-clique: top four row sums (r desc, id asc)
        pick_clique<kLoopThreads>(a.rowsum, n, s_clique, s_red_r, s_red_i);
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
                st.fu_put(f, f | (kToFresh << 28));
            }
        }
        __syncthreads();
        st.recompute(4);
        st.update(heap);
    }

    // thread 0 reads the face of the next root ahead of time (corr mode):
    // the read overlaps the barriers before the insertion that uses it
    int pf_f = -1;
    int4 pf_fc = make_int4(0, 0, 0, 0);
    auto prefetch_face = [&]() {
        if (tid == 0 && !heap) {
            const Key r = s_root[0];
            pf_f = KO::is_empty(r) ? -1 : KO::face(r);
            if (pf_f >= 0 && pf_f < L.nfmax) pf_fc = a.face[pf_f];
            else pf_f = -1;
        }
    };
    prefetch_face();

    // ---- main loop
    const int total = n - 4;
    const int k_stop = a.k_stop < total ? a.k_stop : total;
    long long stale = 0, rounds = 0;
    long long cyc_rec = 0, cyc_tree = 0, cyc_sel = 0;
    long long cyc_x = 0, cyc_v = 0, cyc_sim = 0, cyc_scan = 0, n_epoch_iters = 0, n_x = 0;
    long long c_mark = clock64();
    auto lap = [&](long long &acc) {
        const long long c = clock64();
        acc += c - c_mark;
        c_mark = c;
    };
    while (s_k < k_stop) {
        const int nf_top = s_nf;  // every thread reads it before thread 0 may change it
        if (tid == 0 && globaltimer_ns() - t0 > a.timeout_ns) s_stop = TMFG_ETIMEOUT;
        if (tid == 0) s_fcount = 2;  // prefix 1: the two appended faces come first
        __syncthreads();
        if (s_stop) break;
        if (heap) {
            // ---- resolve the epoch: which pair does Algorithm 2 insert next?
            // Stale faces are taken in key order, at most 8 level-1 groups
            // (256 faces) at a time: the stale keys >= tau, tau = the 8th
            // largest group maximum (or the best fresh key if fewer than 8
            // groups rank above it).  Every stale key above tau is in the
            // batch, so the batch is a prefix of the key order.
            for (;;) {
                const Key kf = s_root[0], ks = s_root[1];
                if (!KO::gt(ks, kf)) {
                    if (tid == 0) s_win = kf;
                    __syncthreads();
                    break;
                }
                long long e0 = clock64();
                ++n_epoch_iters;
                if (tid == 0) { s_nx = 0; s_ninv = 0; s_tau = kf; s_nq1 = 0; }
                // (a) the top 8 level-2 groups above kf
                if (tid < 64) {
                    const Key x = tid < L.G2 ? st.ts.l2[tid] : KO::empty();
                    st.xkey[tid] = x;
                }
                __syncthreads();
                if (tid < 64) {
                    const Key x = st.xkey[tid];
                    if (KO::gt(x, kf)) {
                        int r = 0;
                        for (int j = 0; j < 64; ++j) r += KO::gt(st.xkey[j], x);
                        if (r < 8) st.q2x[r] = (uint16_t)tid;
                    }
                }
                __syncthreads();
                int nq2 = 0;
                for (int j = 0; j < 64 && j < L.G2; ++j) nq2 += KO::gt(st.xkey[j], kf);
                nq2 = nq2 < 8 ? nq2 : 8;
                __syncthreads();
                // (b) their level-1 nodes; the top 8 above kf give tau
                {
                    const int gi = tid >> 5, j = gi < nq2 ? st.q2x[gi] * 32 + (tid & 31) : -1;
                    const Key x = (j >= 0 && j < L.G1) ? st.ts.l1[j] : KO::empty();
                    st.xpend[tid] = KO::gt(x, kf) ? x : KO::empty();
                    __syncthreads();
                    const Key y = st.xpend[tid];
                    if (!KO::is_empty(y)) {
                        int r = 0;
                        for (int q = 0; q < kLoopThreads; ++q) r += KO::gt(st.xpend[q], y);
                        if (r < 8) st.q1x[r] = (uint16_t)j;
                        if (r == 7) s_tau = y;
                        atomicAdd(&s_nq1, 1);
                    }
                }
                __syncthreads();
                const int nq1 = s_nq1 < 8 ? s_nq1 : 8;
                const Key tau = s_tau;  // kf when fewer than 8 groups qualify
                // (c) the leaves >= tau (and > kf) of those groups
                {
                    const int gi = tid >> 5;
                    if (gi < nq1) {
                        const int f = st.q1x[gi] * 32 + (tid & 31);
                        if (f < L.nfmax) {
                            const Key kk = st.ts.leaf[f];
                            if (KO::gt(kk, kf) && !KO::gt(tau, kk)) {
                                const int pos = atomicAdd(&s_nx, 1);
                                st.xf[pos] = f;
                                st.xkey[pos] = kk;
                            }
                        }
                    }
                }
                __syncthreads();
                long long e1 = clock64();
                cyc_x += e1 - e0;
                const int nx = s_nx;
                n_x += nx;
                // pending results still valid? (recompute the others)
                for (int i = tid; i < nx; i += kLoopThreads) {
                    const int f = st.xf[i];
                    if (!st.pend_valid(f)) st.fu_put(atomicAdd(&s_ninv, 1), f | (kToPend << 28));
                }
                __syncthreads();
                if (s_ninv) st.recompute(s_ninv);
                long long e2 = clock64();
                cyc_v += e2 - e1;
                for (int i = tid; i < nx; i += kLoopThreads) {
                    st.xpend[i] = st.pend_key[st.xf[i]];
                    int r = 0;
                    const Key ki = st.xkey[i];
                    for (int j = 0; j < nx; ++j) r += KO::gt(st.xkey[j], ki);
                    st.xs[r] = (uint16_t)i;
                }
                __syncthreads();
                // the pops of Algorithm 2, in key order
                if (tid == 0) {
                    Key run = kf;
                    int np = 0;
                    for (int r = 0; r < nx; ++r) {
                        const int i = st.xs[r];
                        if (!KO::gt(st.xkey[i], run)) break;
                        ++np;
                        if (KO::gt(st.xpend[i], run)) run = st.xpend[i];
                    }
                    s_np = np;
                    s_win = run;
                    // the whole batch was popped and more stale keys may rank
                    // above the running best: resolve the next batch
                    s_more = (np == nx && KO::gt(tau, kf)) ? 1 : 0;
                }
                __syncthreads();
                const int np = s_np;
                for (int r = tid; r < np; r += kLoopThreads) {
                    const int i = st.xs[r];
                    const int f = st.xf[i];
                    const Key p = st.xpend[i];
                    st.tf.set(f, p);
                    st.fv[f] = KO::is_empty(p) ? kNone16 : (uint16_t)KO::vert(p);
                    st.ts.set(f, KO::empty());
                }
                stale += np;
                cyc_sim += clock64() - e2;
                st.update(1);
                if (!s_more) break;
                if (tid == 0 && globaltimer_ns() - t0 > a.timeout_ns) s_stop = TMFG_ETIMEOUT;
                __syncthreads();
                if (s_stop) break;
            }
            if (s_stop) break;
            lap(cyc_sel);
            const Key w = s_win;
            const int v = KO::vert(w), fs = KO::face(w);
            if (KO::is_empty(w) || v >= n || fs >= s_nf || st.is_ins(v)) {
                if (tid == 0) s_stop = TMFG_EINTERNAL;
                __syncthreads();
                break;
            }
            // ---- insert, then recompute the new faces and the faces it made stale
            const int nf_old = s_nf;
            if (tid == 0) {
                st.insert_pair(v, fs);
                st.fu_put(0, fs | (kToFresh << 28));
                st.fu_put(1, nf_old | (kToFresh << 28));
                st.fu_put(2, (nf_old + 1) | (kToFresh << 28));
                s_fcount = 3;
            }
            __syncthreads();
            {
                const uint32_t vv = (uint32_t)v | ((uint32_t)v << 16);
                const uint4 *fv8 = reinterpret_cast<const uint4 *>(st.fv);
                for (int i = tid; 8 * i < nf_old; i += kLoopThreads) {
                    const uint4 q = fv8[i];
                    const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const uint32_t m = __vcmpeq2(wd[h], vv);
                        if (m) {
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                const int f = 8 * i + 2 * h + b;
                                if (f < nf_old && f != fs && ((m >> (16 * b)) & 0xFFFFu))
                                    st.fu_put(atomicAdd(&s_fcount, 1), f | (kToPendMove << 28));
                            }
                        }
                    }
                }
            }
            __syncthreads();
            {
                long long c = clock64();
                cyc_scan += c - c_mark;
            }
            ++rounds;
            st.recompute(s_fcount);
            lap(cyc_rec);
            st.update(1);
            lap(cyc_tree);
        } else {
            if (a.P == 1) {
                // prefix 1: the pair is the root, known to every thread since
                // the last index update.  Thread 0 inserts it while all
                // threads list the faces whose stored vertex it is.
                const Key r = s_root[0];
                const int v = KO::is_empty(r) ? -1 : KO::vert(r);
                const int fsel = KO::is_empty(r) ? -1 : KO::face(r);
                if (v < 0 || v >= n || fsel >= nf_top || st.is_ins(v)) {
                    if (tid == 0) s_stop = TMFG_EINTERNAL;
                    __syncthreads();
                    break;
                }
                lap(cyc_sel);
                const int nf_old = nf_top;
                if (tid == 0) {
                    // the scan below reads stored vertices of faces < nf_old
                    // only; the insertion writes the two new faces' entries
                    st.insert_pair(v, fsel, fsel == pf_f, pf_fc);
                    st.fu_put(0, nf_old | (kToFresh << 28));
                    st.fu_put(1, (nf_old + 1) | (kToFresh << 28));
                }
                st.scan_faces_of(v, nf_old, &s_fcount);
                __syncthreads();
                ++rounds;
                st.recompute(s_fcount);
                lap(cyc_rec);
                st.update(0);
                prefetch_face();
                lap(cyc_tree);
                continue;
            }
            // L = the P best pairs (repeated extraction from the index)
            if (tid == 0) s_nsel = 0;
            __syncthreads();
            for (int i = 0; i < a.P; ++i) {
                const Key r = s_root[0];
                if (KO::is_empty(r)) break;
                if (tid == 0) {
                    st.sel[s_nsel++] = r;
                    if (a.P > 1) st.tf.set(KO::face(r), KO::empty());
                }
                __syncthreads();
                if (a.P == 1) break;
                st.update(0);
            }
            const int nsel = s_nsel;
            if (nsel == 0) {
                if (tid == 0) s_stop = TMFG_EINTERNAL;
                __syncthreads();
                break;
            }
            lap(cyc_sel);
            const int nf_old = s_nf;
            if (tid == 0) {
                // keep the first (best) pair of each vertex, insert in rank order
                for (int i = 0; i < nsel; ++i) {
                    const int v = KO::vert(st.sel[i]);
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
                    const int fsel = KO::face(st.sel[i]);
                    st.insert_pair(v, fsel, i == 0 && fsel == pf_f, pf_fc);
                }
                s_fcount = 0;
            }
            __syncthreads();
            if (s_stop) break;
            ++rounds;
            // F_update: faces whose stored vertex was inserted this round,
            // and the appended faces
            const int nf_new = s_nf;
            if (nsel == 1) {
                // one inserted vertex: compare 8 stored vertices per 16-byte load
                const int v = KO::vert(st.sel[0]);
                const uint32_t vv = (uint32_t)v | ((uint32_t)v << 16);
                const uint4 *fv8 = reinterpret_cast<const uint4 *>(st.fv);
                for (int i = tid; 8 * i < nf_old; i += kLoopThreads) {
                    const uint4 q = fv8[i];
                    const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const uint32_t m = __vcmpeq2(wd[h], vv);
                        if (m) {
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                const int f = 8 * i + 2 * h + b;
                                if (f < nf_old && ((m >> (16 * b)) & 0xFFFFu))
                                    st.fu_put(atomicAdd(&s_fcount, 1), f | (kToFresh << 28));
                            }
                        }
                    }
                }
            } else {
                for (int f = tid; f < nf_old; f += kLoopThreads) {
                    const int v = st.fv[f];
                    if (v != kNone16 && ((st.rnd[v >> 5] >> (v & 31)) & 1u))
                        st.fu_put(atomicAdd(&s_fcount, 1), f | (kToFresh << 28));
                }
            }
            for (int f = nf_old + tid; f < nf_new; f += kLoopThreads)
                st.fu_put(atomicAdd(&s_fcount, 1), f | (kToFresh << 28));
            __syncthreads();
            st.recompute(s_fcount);
            lap(cyc_rec);
            if (tid == 0)
                for (int i = 0; i < nsel; ++i) {
                    const int v = KO::vert(st.sel[i]);
                    if (v < n) st.rnd[v >> 5] &= ~(1u << (v & 31));
                }
            st.update(0);
            prefetch_face();
            lap(cyc_tree);
        }
    }
    // ---- statistics (summed over segments) and the state for the next segment
    st.flush_counters();
    __syncthreads();
    if (tid == 0) {
        if (s_stop) set_status(a.status, s_stop);
        // slots 11..13: heap: cycles of extraction / validation / resolution;
        // corr: pointer probes, warp refreshes after a probe found nothing,
        // and the warp refreshes' 256-id steps
        const long long seg[16] = {s_evals, stale, s_scan, rounds,
                                   (long long)(globaltimer_ns() - t0), cyc_rec, cyc_tree, cyc_sel,
                                   st.cyc_push, st.cyc_refresh, st.cyc_gain,
                                   heap ? cyc_x : (long long)s_probes,
                                   heap ? cyc_v : (long long)s_wref,
                                   heap ? cyc_sim : (long long)s_wsteps, cyc_scan, n_epoch_iters};
        for (int i = 0; i < 16; ++i) {
            acc[i] += seg[i];
            a.stats[i] = acc[i];
            if (gs) gscal[i] = acc[i];
        }
        if (gs) {
            gscal[16] = s_nf;
            gscal[17] = s_k;
            Key *gr = reinterpret_cast<Key *>(gs + SL.off_roots);
            gr[0] = s_root[0];
            gr[1] = s_root[1];
        }
    }
    if (gs && s_k < total && !s_stop) {
        uint32_t *gins = reinterpret_cast<uint32_t *>(gs + SL.off_ins);
        uint16_t *gmc = reinterpret_cast<uint16_t *>(gs + SL.off_mc);
        uint16_t *gptr = reinterpret_cast<uint16_t *>(gs + SL.off_ptr);
        uint16_t *gfv = reinterpret_cast<uint16_t *>(gs + SL.off_fv);
        for (int i = tid; i < L.W; i += kLoopThreads) gins[i] = st.ins[i];
        for (int w = tid; w < n; w += kLoopThreads) { gmc[w] = st.mc[w]; gptr[w] = st.ptr[w]; }
        for (int f = tid; f < L.nfmax; f += kLoopThreads) gfv[f] = st.fv[f];
        auto save_tree = [&](Tree<KO> &x, int t) {
            Key *g = reinterpret_cast<Key *>(gs + SL.off_tree[t]);
            for (int i = tid; i < L.G1; i += kLoopThreads) g[i] = x.l1[i];
            for (int i = tid; i < L.G2; i += kLoopThreads) g[L.G1 + i] = x.l2[i];
        };
        save_tree(st.tf, 0);
        if (heap) save_tree(st.ts, 1);
    }
}

// One instance per launch (the arguments by value).
template <typename T, bool kHeap>
__global__ void __launch_bounds__(kLoopThreads, 1) tmfg_loop_kernel(LoopArgs a)
{
    loop_body<T, kHeap>(a);
}

// Many instances per launch: CTA b runs instance b (arguments in global memory).
template <typename T, bool kHeap>
__global__ void __launch_bounds__(kLoopThreads, 2) tmfg_loop_batch_kernel(const LoopArgs *args)
{
    __shared__ LoopArgs s_args;
    if (threadIdx.x == 0) s_args = args[blockIdx.x];
    __syncthreads();
    loop_body<T, kHeap>(s_args);
}

// Between loop segments: drop the inserted ids from every sorted row.  Row
// w keeps, in order, the ids after ptr[w] that are still uninserted, moved to
// the front of the row and ended by 0xFFFF; ptr[w] = 0 and Mc[w] = the new
// first id.  MaxCorrs (the first uninserted id of the sorted row) is
// unchanged by construction.  One CTA per row (grid-stride); each thread
// reads 8 ids with one 16-byte load, so a round covers 2048 ids; a round's
// reads all happen before its writes, and writes land at or before the read
// positions, so the compaction is in place.
__global__ void __launch_bounds__(256) compact_rows_kernel(uint16_t *idx, long long ldi, int n,
                                                           void *state, const int *status)
{
    __shared__ int s_cnt[8], s_end;
    if (*(volatile const int *)status != 0) return;
    const StateLayout SL = state_layout(n, sizeof(Key128));
    unsigned char *gs = reinterpret_cast<unsigned char *>(state);
    const uint32_t *ins = reinterpret_cast<const uint32_t *>(gs + SL.off_ins);
    uint16_t *gmc = reinterpret_cast<uint16_t *>(gs + SL.off_mc);
    uint16_t *gptr = reinterpret_cast<uint16_t *>(gs + SL.off_ptr);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mlen = n - 1;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        uint16_t *row = idx + (long long)w * ldi;
        const int p0 = gptr[w];
        int out = 0;
        bool done = false;
        for (int base = p0 & ~7; base < mlen && !done; base += 2048) {
            const int q0 = base + 8 * tid;
            uint16_t e[8];
            if (q0 < ldi) {
                const uint4 c = *reinterpret_cast<const uint4 *>(row + q0);
                e[0] = c.x & 0xFFFF; e[1] = c.x >> 16; e[2] = c.y & 0xFFFF; e[3] = c.y >> 16;
                e[4] = c.z & 0xFFFF; e[5] = c.z >> 16; e[6] = c.w & 0xFFFF; e[7] = c.w >> 16;
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) e[t] = kNone16;
            }
            // phase 1: the first end marker of the round (an id >= n or the
            // row end), block-wide
            int first_end = 8;
#pragma unroll
            for (int t = 7; t >= 0; --t) {
                const int q = q0 + t;
                if (q >= mlen || e[t] >= n) first_end = t;
            }
            int m = first_end < 8 ? q0 + first_end : 0x7FFFFFFF;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (tid == 0) s_end = 0x7FFFFFFF;
            __syncthreads();
            if (lane == 0) atomicMin(&s_end, m);
            __syncthreads();
            const int gend = s_end;
            // phase 2: keep the uninserted ids in [p0, gend), compact in order
            uint32_t keepm = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int q = q0 + t;
                if (q >= p0 && q < gend && !((ins[e[t] >> 5] >> (e[t] & 31)) & 1u))
                    keepm |= 1u << t;
            }
            const int c = __popc(keepm);
            int x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_cnt[warp] = x;
            __syncthreads();
            int before = 0, tot = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                before += i < warp ? s_cnt[i] : 0;
                tot += s_cnt[i];
            }
            int pos = out + before + x - c;
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if ((keepm >> t) & 1u) row[pos++] = e[t];
            out += tot;
            done = gend != 0x7FFFFFFF;
            __syncthreads();
        }
        if (tid == 0) {
            if (out < ldi) row[out] = kNone16;
            gptr[w] = 0;
            gmc[w] = out > 0 ? row[0] : kNone16;
        }
        __syncthreads();
    }
}

size_t loop_smem_bytes(int n, int dtype, int mode)
{
    const size_t ks = dtype == TMFG_F32 ? sizeof(unsigned long long) : sizeof(Key128);
    return loop_layout(n, ks, mode == TMFG_HEAP ? 2 : 1).total;
}

// The smallest shared-memory carve-out (percent of the SM's maximum) that
// holds `ctas` CTAs of `smem` dynamic bytes (plus static and reserved
// space): the rest of the unified L1/shared memory stays L1 cache, which
// keeps recently probed sorted-row lines and faces close to the loop.
int carveout_percent(size_t smem, int ctas)
{
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        per_sm <= 0)
        return 100;
    const size_t need = (size_t)ctas * (smem + 2048);
    const size_t pct = (need * 100 + (size_t)per_sm - 1) / (size_t)per_sm;
    return pct > 100 ? 100 : (int)pct;
}

bool loop_shape_from(const tmfg_loop_shape *in, LoopShape *out)
{
    LoopShape s;
    if (in) {
        if (in->threads) s.threads = in->threads;
        if (in->probe_lanes) s.lanes = in->probe_lanes;
        if (in->stage_groups > 0) s.groups = in->stage_groups;
        if (in->stage_groups < 0) s.groups = 0;
        if (in->kernel < 0 || in->kernel > 3) return false;
        s.general = in->kernel - 1;
        if (in->cluster) s.cluster = in->cluster;
        if (s.general == 2) {
            // the cluster kernel's lanes per row refresh (default 32)
            s.cluster_lanes = in->probe_lanes ? in->probe_lanes : 32;
            s.lanes = 8;
        }
    }
    if (!corr1_shape_ok(s.threads, s.lanes) || !cluster_shape_ok(s.cluster, s.cluster_lanes))
        return false;
    *out = s;
    return true;
}

// The insertion loop runs in segments; between them every sorted row is
// compacted to its uninserted ids, so the lazy pointers keep finding an
// uninserted id in their first probe.  Segments end after 1/2, 3/4, 7/8,
// 15/16, 31/32 of the insertions (for n >= 1024).  corr-tmfg with prefix 1
// runs on its own kernel (loop_corr1.cu), every other mode on this file's.
int64_t loop_max_n(int dtype, int mode, int prefix)
{
    int64_t m = 32769;  // 2n - 4 face ids in 16 bits
    if (mode == TMFG_CORR && prefix == 1) {
        while (m > 4 && corr1_fit_groups((int)m, dtype, 0, kSmemLimit, true) < 0) --m;
        return m;
    }
    while (m > 4 && loop_smem_bytes((int)m, dtype, mode) > kSmemLimit) --m;
    return m;
}

int launch_loop(const LoopArgs &args, int dtype, cudaStream_t stream, const LoopShape &shape_in)
{
    if (2 * (size_t)args.n - 4 > 65535) return TMFG_ETOOBIG;
    const bool p1 = args.mode == TMFG_CORR && args.P == 1;
    LoopShape shape = shape_in;
    if (p1 && shape.general < 0 && args.state && args.n >= kClusterAutoMinN &&
        cluster_placeable(args.n, dtype, 16, 32)) {
        shape.general = 2;
        shape.cluster = 16;
        shape.cluster_lanes = 32;
    }
    const size_t gen_smem = loop_smem_bytes(args.n, dtype, args.mode);
    const bool clus = p1 && shape.general == 2;
    if (clus && (!args.state || cluster_smem_bytes(args.n, dtype, shape.cluster) > kSmemLimit))
        return TMFG_ETOOBIG;
    // corr-tmfg with prefix 1 off the cluster kernel: the prefix-1 kernel
    // unless the general one is asked for
    const bool corr1 = p1 && !clus && shape.general <= 0;
    const bool heap = args.mode == TMFG_HEAP;
    auto kf = heap ? tmfg_loop_kernel<float, true> : tmfg_loop_kernel<float, false>;
    auto kd = heap ? tmfg_loop_kernel<double, true> : tmfg_loop_kernel<double, false>;
    size_t smem;
    bool gp = false;
    if (corr1) {
        if (!corr1_shape_ok(shape.threads, shape.lanes)) return TMFG_EINVAL;
        int g = corr1_fit_groups(args.n, dtype, shape.groups, kSmemLimit, false);
        if (g < 0) {
            gp = true;
            g = corr1_fit_groups(args.n, dtype, shape.groups, kSmemLimit, true);
            if (g < 0) return TMFG_ETOOBIG;
        }
        smem = corr1_smem_bytes(args.n, dtype, g, gp);
    } else if (clus) {
        smem = 0;
    } else {
        smem = gen_smem;
        if (smem > kSmemLimit) return TMFG_ETOOBIG;
        const void *kp = dtype == TMFG_F32 ? (const void *)kf : (const void *)kd;
        if (cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(kp, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 carveout_percent(smem, 1)) != cudaSuccess)
            return TMFG_ECUDA;
    }
    const int total = args.n - 4;
    int stops[8];
    int ns = 0;
    if (args.n >= 1024)
        for (int j = 1; j <= 5; ++j) {
            const int s = total - (total >> j);
            if (s > 0 && (ns == 0 || s > stops[ns - 1])) stops[ns++] = s;
        }
    stops[ns++] = total;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < ns; ++i) {
        LoopArgs a = args;
        a.k_stop = stops[i];
        a.resume = i > 0;
        if (clus) {
            const int rc = launch_cluster_loop(a, dtype, shape.cluster, shape.cluster_lanes, stream);
            if (rc) return rc;
        } else if (corr1) {
            const int rc = launch_corr1(a, shape, dtype, smem, gp, stream);
            if (rc) return rc;
        } else if (dtype == TMFG_F32) {
            kf<<<1, kLoopThreads, smem, stream>>>(a);
        } else {
            kd<<<1, kLoopThreads, smem, stream>>>(a);
        }
        if (i + 1 < ns)
            compact_rows_kernel<<<2 * sms, 256, 0, stream>>>(const_cast<uint16_t *>(args.idx),
                                                             args.ldi, args.n, args.state,
                                                             args.status);
    }
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

int launch_loop_batch(const LoopArgs *d_args, int count, int max_n, int dtype, int mode, int P,
                      cudaStream_t stream, const LoopShape &shape)
{
    if (2 * (size_t)max_n - 4 > 65535) return TMFG_ETOOBIG;
    if (shape.general == 2) return TMFG_EINVAL;  // the cluster kernel runs single builds only
    const size_t smem = loop_smem_bytes(max_n, dtype, mode);
    // corr-tmfg with prefix 1 runs on the prefix-1 kernel unless the general
    // one is asked for
    if (mode == TMFG_CORR && P == 1 && shape.general <= 0) {
        if (!corr1_shape_ok(shape.threads, shape.lanes)) return TMFG_EINVAL;
        // two CTAs per SM when they fit, else one
        int g = corr1_fit_groups(max_n, dtype, shape.groups, kSmemLimit / 2 - 4096, false);
        if (g < 0) g = corr1_fit_groups(max_n, dtype, shape.groups, kSmemLimit, false);
        if (g < 0) return TMFG_ETOOBIG;
        return launch_corr1_batch(d_args, count, shape, dtype,
                                  corr1_smem_bytes(max_n, dtype, g, false), stream);
    }
    if (smem > kSmemLimit) return TMFG_ETOOBIG;
    const bool heap = mode == TMFG_HEAP;
    auto kf = heap ? tmfg_loop_batch_kernel<float, true> : tmfg_loop_batch_kernel<float, false>;
    auto kd = heap ? tmfg_loop_batch_kernel<double, true> : tmfg_loop_batch_kernel<double, false>;
    const void *kp = dtype == TMFG_F32 ? (const void *)kf : (const void *)kd;
    if (cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kp, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carveout_percent(smem, 2)) != cudaSuccess)
        return TMFG_ECUDA;
    if (dtype == TMFG_F32)
        kf<<<count, kLoopThreads, smem, stream>>>(d_args);
    else
        kd<<<count, kLoopThreads, smem, stream>>>(d_args);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace tmfg
