// pipeline.cu -- the whole clustering of many raw-series instances in one
// call (no counterpart in the paper: the request shape of a clustering
// service): Pearson similarity of each instance's series (Section 5, the
// input the method takes), then the batched TMFG and exact APSP of every
// instance (tmfg_batch_run: one launch per stage for all of them), then each
// instance's DBHT dendrogram (Section 2) and its cut at k clusters
// (Section 5, the labels the evaluation scores).  The stages are launched in
// stream order on the context's workspace, sized once for the largest stage.
#include <climits>
#include <vector>

#include "ctx.cuh"

namespace tmfg {

// Labels after the first n - k merges of a linkage (scipy layout): the
// clusters are numbered 0..k-1 in the order of their smallest member.  One
// CTA, every step parallel over the nodes:
//  1. parent[a] = parent[b] = n + r for each kept merge r < n - k (a node
//     has at most one parent, and it has a larger id);
//  2. roots by pointer jumping (each node's pointer to its parent replaced
//     by its parent's until nothing changes: O(log depth) rounds);
//  3. each root's smallest leaf (atomic minimum);
//  4. a leaf that is its cluster's smallest marks the cluster; an exclusive
//     scan of the marks over the leaves numbers the clusters in that order.
// buf holds 3 (2n - 1) ints: in shared memory when they fit, else in the
// caller's global scratch.
constexpr int kCutThreads = 512;

__host__ __device__ inline size_t cut_buf_bytes(int64_t n) { return 12 * (2 * (size_t)n - 1); }

__global__ void __launch_bounds__(kCutThreads) cut_labels_kernel(
    const double *__restrict__ Z, int n, int k, int *__restrict__ labels,
    int *__restrict__ gbuf, int use_smem, int *status)
{
    extern __shared__ int sm[];
    __shared__ int s_flag, s_warp[kCutThreads / 32], s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_flag = *(volatile int *)status;
    __syncthreads();
    if (s_flag) return;  // an earlier step failed (every thread leaves)
    const int m = 2 * n - 1;
    int *par = use_smem ? sm : gbuf;  // parent, then root
    int *minv = par + m;              // smallest leaf of each root
    int *rank = minv + m;             // clusters before the leaf (leaves only)
    for (int i = tid; i < m; i += kCutThreads) {
        par[i] = i;
        minv[i] = INT_MAX;
    }
    __syncthreads();
    // 1. the kept merges
    for (int r = tid; r < n - k; r += kCutThreads) {
        const int a = (int)Z[4 * (size_t)r], b = (int)Z[4 * (size_t)r + 1];
        if (a < 0 || b < 0 || a >= n + r || b >= n + r || a == b) {
            atomicExch(&s_flag, 1);
            continue;
        }
        par[a] = n + r;
        par[b] = n + r;
    }
    __syncthreads();
    if (s_flag) {
        if (tid == 0) set_status(status, TMFG_EINVAL);
        return;
    }
    // 2. pointer jumping; parents have larger ids, so there is no cycle and
    // a round that changes nothing ends it (at most ~log2 m + 1 rounds)
    // (the decision to go on is the barrier's own reduction, the same value
    // in every thread)
    for (int it = 0; it < 64; ++it) {
        int changed = 0;
        for (int i = tid; i < m; i += kCutThreads) {
            const int p = par[i], pp = par[p];
            if (pp != p) {
                par[i] = pp;
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    // 3. each root's smallest leaf
    for (int v = tid; v < n; v += kCutThreads) atomicMin(&minv[par[v]], v);
    __syncthreads();
    // 4. exclusive scan over the leaves of "v is its cluster's smallest"
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int v0 = 0; v0 < n; v0 += kCutThreads) {
        const int v = v0 + tid;
        const int f = (v < n && minv[par[v]] == v) ? 1 : 0;
        int x = f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int ws = lane < kCutThreads / 32 ? s_warp[lane] : 0;
            int z = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            if (lane < kCutThreads / 32) s_warp[lane] = z - ws;  // exclusive over warps
        }
        __syncthreads();
        if (v < n) rank[v] = s_carry + s_warp[warp] + x - f;
        __syncthreads();
        if (tid == kCutThreads - 1) s_carry += s_warp[warp] + x;
        __syncthreads();
    }
    for (int v = tid; v < n; v += kCutThreads) labels[v] = rank[minv[par[v]]];
}

// Launch the cut on one CTA; gbuf: cut_buf_bytes(n) of global scratch (used
// when the buffers do not fit shared memory).
int launch_cut_labels(const double *Z, int n, int k, int *labels, void *gbuf, int *status,
                      cudaStream_t st)
{
    const size_t bytes = cut_buf_bytes(n);
    const bool use_smem = bytes + 1024 <= (size_t)kSmemLimit;
    const int smem = use_smem ? (int)bytes : 0;
    if (use_smem && smem > 48 * 1024 &&
        cudaFuncSetAttribute(cut_labels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
        return TMFG_ECUDA;
    cut_labels_kernel<<<1, kCutThreads, smem, st>>>(Z, n, k, labels, static_cast<int *>(gbuf),
                                                   use_smem ? 1 : 0, status);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

// requests whose per-request stages (similarity, DBHT, cut) run side by side:
// each request's stages are a chain of small launches, mostly one or a few
// CTAs each, so many streams are needed to fill the GPU (measured on the
// 4096-request serving workload: 8 streams 1557 solves/s, 16 1686, 32 1811,
// 64 1850)
constexpr int kPipeStreams = 32;

int ensure_aux_streams(tmfg_ctx *c)
{
    if (c->aux_ready) return TMFG_OK;
    for (cudaStream_t &a : c->aux)
        if (cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) != cudaSuccess) return TMFG_ECUDA;
    for (cudaEvent_t &e : c->aux_ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return TMFG_ECUDA;
    c->aux_ready = true;
    return TMFG_OK;
}

// The first `k` side streams wait for `st`'s work so far.
bool fork_aux(tmfg_ctx *c, cudaStream_t st, int k)
{
    if (cudaEventRecord(c->aux_ev[kPipeStreams], st) != cudaSuccess) return false;
    for (int i = 0; i < k; ++i)
        if (cudaStreamWaitEvent(c->aux[i], c->aux_ev[kPipeStreams], 0) != cudaSuccess) return false;
    return true;
}

// `st` waits for the first `k` side streams' work so far.
bool join_aux(tmfg_ctx *c, cudaStream_t st, int k)
{
    for (int i = 0; i < k; ++i)
        if (cudaEventRecord(c->aux_ev[i], c->aux[i]) != cudaSuccess ||
            cudaStreamWaitEvent(st, c->aux_ev[i], 0) != cudaSuccess)
            return false;
    return true;
}

size_t pipeline_scratch_bytes(int64_t n, int64_t T, int precision)
{
    size_t b = sim_work_bytes((int)n, (int)T, precision);
    const size_t d = dbht_work_bytes((int)n);
    if (d > b) b = d;
    const size_t c = cut_buf_bytes(n);
    return c > b ? c : b;
}

}  // namespace tmfg

using namespace tmfg;

extern "C" {

size_t tmfg_pipeline_request_bytes(int64_t n, int64_t T, int32_t precision)
{
    if (n < 4 || T < 2) return 0;
    return batch_request_bytes(n, true) + round256(pipeline_scratch_bytes(n, T, precision));
}

int tmfg_cut_labels(tmfg_ctx *ctx, const double *Z, int64_t n, int32_t k, int32_t *labels,
                    void *stream)
{
    if (!ctx || !Z || !labels || n < 2 || k < 1 || k > n) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(ctx, cut_buf_bytes(n), st);
    if (rc) return rc;
    return launch_cut_labels(Z, (int)n, k, labels, ctx->work, ctx->status, st);
}

int tmfg_pipeline_run(tmfg_ctx *ctx, const tmfg_pipeline_job *jobs, int32_t count,
                      const tmfg_pipeline_params *pp, const tmfg_batch_config *cfg, void *stream)
{
    if (!ctx || !jobs || count < 1 || !pp) return TMFG_EINVAL;
    const int prec = pp->precision;
    if (prec < TMFG_SIM_F64 || prec > TMFG_SIM_TF32X3) return TMFG_EINVAL;
    if (pp->tmfg.dtype != TMFG_F32) return TMFG_EINVAL;  // the similarity is float
    size_t scratch = 0;
    for (int i = 0; i < count; ++i) {
        const tmfg_pipeline_job &J = jobs[i];
        if (!J.X || !J.S || !J.order || !J.edges || !J.bubble_parent || !J.D || !J.Z ||
            J.n < 4 || J.T < 2 || J.ldx < J.T || (J.n > 4 && !J.ins_face) || J.k < 0 ||
            J.k > J.n || (J.k > 0 && !J.labels))
            return TMFG_EINVAL;
        if (J.n > DBHT_MAX_N) return TMFG_ETOOBIG;
        const size_t b = pipeline_scratch_bytes(J.n, J.T, prec);
        if (b > scratch) scratch = b;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return TMFG_ECUDA;
    // the per-request stages of request i run on side stream i mod k, each
    // stream on its own slice of the workspace
    int k = count < kPipeStreams ? count : kPipeStreams;
    scratch = round256(scratch);
    if (cs != cudaStreamCaptureStatusNone) {
        // under capture nothing is allocated: as many streams as the
        // workspace already holds slices for
        while (k > 1 && (size_t)k * scratch > ctx->work_bytes) k >>= 1;
        if (!ctx->aux_ready || (size_t)k * scratch > ctx->work_bytes) return TMFG_ENOMEM;
    } else {
        int rc = ensure_aux_streams(ctx);
        if (rc) return rc;
        // fewer streams when the context's budget does not hold k slices
        while (k > 1 && ctx->budget && (size_t)k * scratch > ctx->budget) k >>= 1;
        rc = ensure_work(ctx, (size_t)k * scratch, st);
        if (rc) return rc;
    }
    auto slice = [&](int i) { return static_cast<char *>(ctx->work) + (size_t)(i % k) * scratch; };
    // 1. the similarity of each instance's series
    if (!fork_aux(ctx, st, k)) return TMFG_ECUDA;
    for (int i = 0; i < count; ++i) {
        const tmfg_pipeline_job &J = jobs[i];
        const int rc = launch_similarity(J.X, (int)J.n, (int)J.T, J.ldx, prec, J.S, J.n,
                                         slice(i), ctx->status, ctx->timeout_ns,
                                         ctx->aux[i % k]);
        if (rc) return rc;
    }
    if (!join_aux(ctx, st, k)) return TMFG_ECUDA;
    // 2. the batched TMFG and exact APSP
    std::vector<tmfg_job> bj(count);
    for (int i = 0; i < count; ++i) {
        const tmfg_pipeline_job &J = jobs[i];
        tmfg_job &b = bj[i];
        b = tmfg_job{};
        b.S = J.S;
        b.n = J.n;
        b.ld = J.n;
        b.order = J.order;
        b.edges = J.edges;
        b.ins_face = J.ins_face;
        b.bubble_parent = J.bubble_parent;
        b.D = J.D;
        b.ldd = J.n;
    }
    int rc = tmfg_batch_run(ctx, bj.data(), count, &pp->tmfg, cfg, stream);
    if (rc) return rc;
    // 3. each dendrogram, then its cut (the batch's tables in the workspace
    // are done with once the batched stages have run: the side streams wait)
    if (!fork_aux(ctx, st, k)) return TMFG_ECUDA;
    for (int i = 0; i < count; ++i) {
        const tmfg_pipeline_job &J = jobs[i];
        cudaStream_t as = ctx->aux[i % k];
        rc = launch_dbht(J.S, (int)J.n, J.n, TMFG_F32, J.order, J.edges, J.ins_face,
                         J.bubble_parent, J.D, J.n, J.Z, nullptr, nullptr, nullptr, nullptr,
                         slice(i), ctx->status, ctx->num_sms, as);
        if (rc) return rc;
        if (J.k > 0) {
            rc = launch_cut_labels(J.Z, (int)J.n, J.k, J.labels, slice(i), ctx->status, as);
            if (rc) return rc;
        }
    }
    return join_aux(ctx, st, k) ? TMFG_OK : TMFG_ECUDA;
}

}  // extern "C"
