// loop_common.cuh -- what the insertion-loop kernels share: the pair keys,
// the two-level max index over face keys, the shared-memory layout of the
// general loop kernel and the loop state kept in global memory between the
// segments of a build (its format is the same for every loop kernel, so the
// row compaction between segments serves them all).
#pragma once

#include <climits>

#include "internal.cuh"

namespace tmfg {

constexpr int kLoopThreads = 256;
constexpr int kLoopWarps = kLoopThreads / kWarp;
constexpr int kChunk = kLoopThreads;  // faces per recompute batch (one per thread)
constexpr int kMaxPrefix = 256;  // largest corr-tmfg prefix
constexpr int kXCap = 256;       // stale faces resolved in one batch
constexpr int kFuCap = 512;      // face-update list entries kept in shared memory

// recompute destinations (encoded in bits 28..29 of a list entry)
constexpr int kToFresh = 0;      // store as the face's key in the FRESH index
constexpr int kToPendMove = 1;   // store as pending; move the face FRESH -> STALE
constexpr int kToPend = 2;       // store as pending only

// ------------------------------------------------------------------- keys
template <typename T>
struct KeyOps;

template <>
struct KeyOps<float> {
    using Key = unsigned long long;
    __device__ static Key empty() { return 0ull; }
    __device__ static Key make(float g, int v, int f)
    {
        return ((Key)ord_key(g) << 32) | ((Key)(0xFFFFu - (unsigned)v) << 16) |
               (Key)(0xFFFFu - (unsigned)f);
    }
    __device__ static bool gt(const Key &a, const Key &b) { return a > b; }
    __device__ static bool is_empty(const Key &k) { return k == 0ull; }
    __device__ static int vert(const Key &k) { return 0xFFFF - (int)((k >> 16) & 0xFFFFu); }
    __device__ static int face(const Key &k) { return 0xFFFF - (int)(k & 0xFFFFu); }
    __device__ static Key shfl_xor(const Key &k, int o) { return __shfl_xor_sync(0xffffffffu, k, o); }
};

struct Key128 {
    unsigned long long hi;  // order-preserving image of the double gain
    unsigned long long lo;  // (0xFFFF - vertex) << 16 | (0xFFFF - face)
};

template <>
struct KeyOps<double> {
    using Key = Key128;
    __device__ static Key empty() { return Key128{0ull, 0ull}; }
    __device__ static Key make(double g, int v, int f)
    {
        return Key128{ord_key(g), ((unsigned long long)(0xFFFFu - (unsigned)v) << 16) |
                                      (unsigned long long)(0xFFFFu - (unsigned)f)};
    }
    __device__ static bool gt(const Key &a, const Key &b)
    {
        return a.hi != b.hi ? a.hi > b.hi : a.lo > b.lo;
    }
    __device__ static bool is_empty(const Key &k) { return k.hi == 0ull; }
    __device__ static int vert(const Key &k) { return 0xFFFF - (int)((k.lo >> 16) & 0xFFFFu); }
    __device__ static int face(const Key &k) { return 0xFFFF - (int)(k.lo & 0xFFFFu); }
    __device__ static Key shfl_xor(const Key &k, int o)
    {
        return Key128{__shfl_xor_sync(0xffffffffu, k.hi, o), __shfl_xor_sync(0xffffffffu, k.lo, o)};
    }
};

template <class KO>
__device__ __forceinline__ typename KO::Key warp_max(typename KO::Key x)
{
    if constexpr (sizeof(typename KO::Key) == 8) {
        // 64-bit key: the largest high word, then the largest low word among
        // the lanes holding it (two warp reductions instead of five
        // shuffle-and-compare steps)
        const unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
        const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
        const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
        return ((typename KO::Key)mh << 32) | ml;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const typename KO::Key y = KO::shfl_xor(x, o);
            if (KO::gt(y, x)) x = y;
        }
        return x;
    }
}

// ------------------------------------------------------------- max index
template <class KO>
struct Tree {
    using Key = typename KO::Key;
    Key *leaf;         // global [nfmax]
    Key *l1, *l2;      // shared [G1], [G2]
    uint32_t *b1, *b2; // dirty bits
    uint16_t *q1, *q2; // dirty lists
    int *n1, *n2;      // dirty counts (shared scalars)
    Key *root;         // shared scalar

    __device__ void mark(int f)
    {
        const int g = f >> 5;
        const uint32_t bit = 1u << (g & 31);
        if (!(atomicOr(&b1[g >> 5], bit) & bit)) q1[atomicAdd(n1, 1)] = (uint16_t)g;
    }
    __device__ void set(int f, const Key &k)
    {
        leaf[f] = k;
        mark(f);
    }
};

// Shared-memory layout (dynamic part), computed identically on the host.
struct LoopLayout {
    int W, nfmax, G1, G2;
    size_t off_ins, off_vmark, off_rnd, off_mc, off_ptr, off_fv, off_tree[2], off_vlist, off_vslow, off_plist,
        off_sel, off_x, off_xkey, off_xpend, off_xs, off_q1x, off_q2x, off_fus, total;
    size_t tree_bytes;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Per index: l1 [G1] keys, l2 [G2] keys, b1, b2 bits, q1 [G1], q2 [G2].
__host__ __device__ inline size_t tree_layout_bytes(int G1, int G2, size_t ks)
{
    size_t o = 0;
    o = align16(o + ks * (size_t)G1);
    o = align16(o + ks * (size_t)G2);
    o = align16(o + 4 * (size_t)((G1 + 31) / 32));
    o = align16(o + 4 * (size_t)((G2 + 31) / 32));
    o = align16(o + 2 * (size_t)G1);
    o = align16(o + 2 * (size_t)G2);
    return o;
}

__host__ __device__ inline LoopLayout loop_layout(int n, size_t ks, int ntrees)
{
    LoopLayout L;
    L.W = (n + 31) / 32;
    L.nfmax = 2 * n - 4;
    L.G1 = (L.nfmax + 31) / 32;
    L.G2 = (L.G1 + 31) / 32;
    L.tree_bytes = tree_layout_bytes(L.G1, L.G2, ks);
    size_t o = 0;
    L.off_ins = o;   o = align16(o + 4 * (size_t)L.W);
    L.off_vmark = o; o = align16(o + 4 * (size_t)L.W);
    L.off_rnd = o;   o = align16(o + 4 * (size_t)L.W);
    L.off_mc = o;    o = align16(o + 2 * (size_t)n);
    L.off_ptr = o;   o = align16(o + 2 * (size_t)n);
    L.off_fv = o;    o = align16(o + 2 * (size_t)L.nfmax);
    L.off_tree[0] = o; o += L.tree_bytes;
    L.off_tree[1] = o; o += ntrees > 1 ? L.tree_bytes : 0;
    L.off_vlist = o; o = align16(o + 4 * (size_t)(3 * kChunk));
    L.off_vslow = o; o = align16(o + 4 * (size_t)(3 * kChunk));
    // the list of rows to probe by 8-lane groups: corr-tmfg only (heap mode
    // probes one row per thread and keeps its shared memory for two indexes)
    L.off_plist = o; o = align16(o + (ntrees > 1 ? 0 : 4 * (size_t)(3 * kChunk)));
    L.off_sel = o;   o = align16(o + ks * (size_t)kMaxPrefix);
    // the stale-pop resolution arrays exist in heap mode (two indexes) only
    const size_t hx = ntrees > 1 ? 1 : 0;
    L.off_x = o;     o = align16(o + hx * 4 * (size_t)kXCap);
    L.off_xkey = o;  o = align16(o + hx * ks * (size_t)kXCap);
    L.off_xpend = o; o = align16(o + hx * ks * (size_t)kXCap);
    L.off_xs = o;    o = align16(o + hx * 2 * (size_t)kXCap);
    L.off_q1x = o;   o = align16(o + hx * 2 * (size_t)L.G1);
    L.off_q2x = o;   o = align16(o + hx * 2 * (size_t)64);
    L.off_fus = o;   o = align16(o + 4 * (size_t)kFuCap);
    L.total = o;
    return L;
}

// Loop state kept in global memory between segments of the loop (the rows
// are compacted between segments): scalars, then the shared arrays.
struct StateLayout {
    size_t off_scal, off_roots, off_ins, off_mc, off_ptr, off_fv, off_tree[2], total;
};

__host__ __device__ inline StateLayout state_layout(int n, size_t ks)
{
    const LoopLayout L = loop_layout(n, ks, 2);
    StateLayout S;
    size_t o = 0;
    S.off_scal = o;  o = align16(o + 8 * 32);
    S.off_roots = o; o = align16(o + 2 * ks);
    S.off_ins = o;   o = align16(o + 4 * (size_t)L.W);
    S.off_mc = o;    o = align16(o + 2 * (size_t)n);
    S.off_ptr = o;   o = align16(o + 2 * (size_t)n);
    S.off_fv = o;    o = align16(o + 2 * (size_t)L.nfmax);
    for (int t = 0; t < 2; ++t) {
        S.off_tree[t] = o;
        o = align16(o + ks * (size_t)(L.G1 + L.G2));
    }
    S.total = o;
    return S;
}

// The initial 4-clique (Algorithm 1; reading R2): the four largest row sums
// by (r desc, id asc), written to s_clique in rank order.  All NT threads of
// the CTA call it; s_red_r / s_red_i hold one entry per warp.
template <int NT>
__device__ void pick_clique(const long long *rowsum, int n, int *s_clique, long long *s_red_r,
                            int *s_red_i)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < 4; ++c) {
        long long br = LLONG_MIN;
        int bi = INT_MAX;
        for (int v = tid; v < n; v += NT) {
            bool taken = false;
            for (int j = 0; j < c; ++j) taken |= (s_clique[j] == v);
            if (taken) continue;
            const long long r = rowsum[v];
            if (r > br || (r == br && v < bi)) { br = r; bi = v; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long r2 = __shfl_xor_sync(0xffffffffu, br, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            if (r2 > br || (r2 == br && i2 < bi)) { br = r2; bi = i2; }
        }
        if (lane == 0) { s_red_r[warp] = br; s_red_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            long long r = s_red_r[0];
            int i = s_red_i[0];
            for (int w = 1; w < NT / 32; ++w)
                if (s_red_r[w] > r || (s_red_r[w] == r && s_red_i[w] < i)) { r = s_red_r[w]; i = s_red_i[w]; }
            s_clique[c] = i;
        }
        __syncthreads();
    }
}

}  // namespace tmfg
