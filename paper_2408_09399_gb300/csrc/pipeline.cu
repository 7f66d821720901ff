// pipeline.cu -- the whole clustering of many raw-series instances in one
// call (no counterpart in the paper: the request shape of a clustering
// service): Pearson similarity of each instance's series (Section 5, the
// input the method takes), then the batched TMFG and exact APSP of every
// instance (tmfg_batch_run: one launch per stage for all of them), then each
// instance's DBHT dendrogram (Section 2) and its cut at k clusters
// (Section 5, the labels the evaluation scores).  The stages are launched in
// stream order on the context's workspace, sized once for the largest stage.
#include <vector>

#include "ctx.cuh"

namespace tmfg {

// Labels after the first n - k merges of a linkage (scipy layout): the
// clusters are numbered 0..k-1 in the order of their smallest member.  One
// thread (n is a request's size); scratch holds 2 (2n - 1) ints.
__global__ void cut_labels_kernel(const double *__restrict__ Z, int n, int k,
                                  int *__restrict__ labels, int *__restrict__ scratch, int *status)
{
    if (threadIdx.x != 0 || *(volatile int *)status != 0) return;
    const int m = 2 * n - 1;
    int *uf = scratch, *lab = scratch + m;
    for (int i = 0; i < m; ++i) { uf[i] = i; lab[i] = -1; }
    for (int r = 0; r < n - k; ++r) {
        const int a = (int)Z[4 * r], b = (int)Z[4 * r + 1];
        if (a < 0 || b < 0 || a >= n + r || b >= n + r) { set_status(status, TMFG_EINVAL); return; }
        uf[a] = n + r;
        uf[b] = n + r;
    }
    int next = 0;
    for (int v = 0; v < n; ++v) {
        int r = v;
        while (uf[r] != r) r = uf[r];
        // path compression: later leaves of the cluster stop at the root
        for (int x = v; uf[x] != r && x != r;) { const int y = uf[x]; uf[x] = r; x = y; }
        if (lab[r] < 0) lab[r] = next++;
        labels[v] = lab[r];
    }
}

constexpr int kPipeStreams = 8;  // requests whose per-request stages run side by side

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
    const size_t c = 8 * (2 * (size_t)n - 1);
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
    int rc = ensure_work(ctx, 8 * (2 * (size_t)n - 1), st);
    if (rc) return rc;
    cut_labels_kernel<<<1, 32, 0, st>>>(Z, (int)n, k, labels, static_cast<int *>(ctx->work),
                                        ctx->status);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
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
    const int k = count < kPipeStreams ? count : kPipeStreams;
    scratch = round256(scratch);
    if (cs != cudaStreamCaptureStatusNone) {
        if (!ctx->aux_ready || (size_t)k * scratch > ctx->work_bytes) return TMFG_ENOMEM;
    } else {
        int rc = ensure_aux_streams(ctx);
        if (!rc) rc = ensure_work(ctx, (size_t)k * scratch, st);
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
            cut_labels_kernel<<<1, 32, 0, as>>>(J.Z, (int)J.n, J.k, J.labels,
                                                reinterpret_cast<int *>(slice(i)), ctx->status);
            if (cudaGetLastError() != cudaSuccess) return TMFG_ECUDA;
        }
    }
    return join_aux(ctx, st, k) ? TMFG_OK : TMFG_ECUDA;
}

}  // extern "C"
