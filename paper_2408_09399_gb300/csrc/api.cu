// api.cu -- the C ABI of libtmfg.so (declared in include/tmfg.h): context
// and workspace management, argument checks, kernel launches.
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ctx.cuh"

namespace tmfg {

constexpr int kMaxPrefixApi = 256;

// Bitwise symmetry of S (with -0 == +0), 32x32 tiles above the diagonal.
template <typename T>
__global__ void symmetry_kernel(const T *__restrict__ S, long long ld, int n, int *status)
{
    __shared__ T tile[32][33];
    const int I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int i = J * 32 + r, j = I * 32 + tx;
        tile[r][tx] = (i < n && j < n) ? canon(S[(long long)i * ld + j]) : T(0);
    }
    __syncthreads();
    bool bad = false;
    for (int r = ty; r < 32; r += 8) {
        const int i = I * 32 + r, j = J * 32 + tx;
        if (i < n && j < n && i != j) {
            const T x = canon(S[(long long)i * ld + j]);
            const T y = tile[tx][r];  // S[j][i]
            bad |= !(x == y) && !(x != x && y != y);
        }
    }
    if (bad) set_status(status, TMFG_EASYMMETRIC);
}

}  // namespace tmfg

using namespace tmfg;


namespace tmfg {

unsigned long long device_timeout_ns()
{
    unsigned long long ns = 60ull * 1000000000ull;
    if (const char *e = std::getenv("TMFG_TIMEOUT_MS")) {
        const long long ms = std::atoll(e);
        if (ms > 0) ns = (unsigned long long)ms * 1000000ull;
    }
    return ns;
}

int ensure_work(tmfg_ctx *c, size_t bytes, cudaStream_t stream)
{
    if (bytes <= c->work_bytes) return TMFG_OK;
    if (c->budget && bytes > c->budget) return TMFG_ENOMEM;
    if (c->work) {
        if (cudaStreamSynchronize(stream) != cudaSuccess) return TMFG_ECUDA;
        cudaFree(c->work);
        c->work = nullptr;
        c->work_bytes = 0;
    }
    if (cudaMalloc(&c->work, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->work = nullptr;
        return TMFG_ENOMEM;
    }
    c->work_bytes = bytes;
    return TMFG_OK;
}

int ensure_stage(tmfg_ctx *c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return TMFG_OK;
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    if (cudaHostAlloc(&c->stage, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return TMFG_ENOMEM;
    }
    c->stage_bytes = bytes;
    return TMFG_OK;
}

size_t batch_table_bytes(int count, int napsp)
{
    return round256(sizeof(SortJob) * count) + round256(sizeof(int) * (count + 1)) +
           round256(sizeof(LoopArgs) * count) + round256(sizeof(ApspJob) * (napsp + 1)) +
           round256(sizeof(SsspArgs) * (napsp + 1)) + 2 * round256(sizeof(int) * (napsp + 1));
}

size_t batch_request_bytes(int64_t n, bool apsp)
{
    const size_t nf = 2 * (size_t)n - 4;
    size_t b = round256(2 * (size_t)n * (size_t)ldi_for(n)) + round256(8 * (size_t)n) +
               round256(16 * nf) * 4 + round256(8 * nf) + round256(4 * nf) + 256;
    if (apsp)
        b += round256(4 * (size_t)n) + round256(4 * ((size_t)n + 1)) + round256(4 * (size_t)n) +
             round256(8 * 2 * (3 * (size_t)n - 6));
    return b;
}

}  // namespace tmfg

namespace {


struct BuildWork {
    uint16_t *idx;
    long long *rowsum;
    int4 *face;
    void *leaf_fresh, *leaf_stale, *pend_key;
    unsigned long long *pend_cand;
    int *fu_buf;
    void *state;
};

size_t build_work_bytes(int64_t n)
{
    const size_t nf = 2 * (size_t)n - 4;
    return round256(2 * (size_t)n * (size_t)ldi_for(n)) + round256(8 * (size_t)n) +
           round256(16 * nf) + 3 * round256(16 * nf) + round256(8 * nf) + round256(4 * nf) +
           round256(loop_state_bytes((int)n));
}

BuildWork build_carve(void *base, int64_t n)
{
    const size_t nf = 2 * (size_t)n - 4;
    char *p = static_cast<char *>(base);
    auto take = [&](size_t x) { void *r = p; p += round256(x); return r; };
    BuildWork w;
    w.idx = static_cast<uint16_t *>(take(2 * (size_t)n * (size_t)ldi_for(n)));
    w.rowsum = static_cast<long long *>(take(8 * (size_t)n));
    w.face = static_cast<int4 *>(take(16 * nf));
    w.leaf_fresh = take(16 * nf);
    w.leaf_stale = take(16 * nf);
    w.pend_key = take(16 * nf);
    w.pend_cand = static_cast<unsigned long long *>(take(8 * nf));
    w.fu_buf = static_cast<int *>(take(4 * nf));
    w.state = take(loop_state_bytes((int)n));
    return w;
}

int hubs_for(int64_t n, int n_hubs)
{
    int64_t h = n_hubs > 0 ? n_hubs : (int64_t)std::ceil(std::sqrt((double)n));
    if (h > n) h = n;
    return (int)h;
}

int check_symmetry(tmfg_ctx *c, const void *S, int64_t n, int64_t ld, int dtype,
                   cudaStream_t stream)
{
    const int T = (int)((n + 31) / 32);
    if (dtype == TMFG_F32)
        symmetry_kernel<float><<<dim3(T, T), dim3(32, 8), 0, stream>>>(
            static_cast<const float *>(S), ld, (int)n, c->status);
    else
        symmetry_kernel<double><<<dim3(T, T), dim3(32, 8), 0, stream>>>(
            static_cast<const double *>(S), ld, (int)n, c->status);
    return cudaGetLastError() == cudaSuccess ? TMFG_OK : TMFG_ECUDA;
}

}  // namespace

namespace {
// The insertion loop of tmfg_build over rows already sorted into w.
int launch_build_loop(tmfg_ctx *ctx, const BuildWork &w, const void *S, int64_t n, int64_t ld,
                      const tmfg_params *params, int32_t *order, int32_t *edges,
                      int32_t *ins_face, int32_t *bubble_parent, cudaStream_t st)
{
    const int dtype = params->dtype;
    LoopArgs a{};
    a.S = S;
    a.ld = ld;
    a.n = (int)n;
    a.mode = params->mode;
    a.P = params->prefix;
    a.idx = w.idx;
    a.ldi = ldi_for(n);
    a.rowsum = w.rowsum;
    a.order = order;
    a.edges = edges;
    a.ins_face = ins_face;
    a.parent = bubble_parent;
    a.face = w.face;
    a.leaf_fresh = w.leaf_fresh;
    a.leaf_stale = w.leaf_stale;
    a.pend_key = w.pend_key;
    a.pend_cand = w.pend_cand;
    a.fu_buf = w.fu_buf;
    a.state = w.state;
    a.status = ctx->status;
    a.stats = ctx->stats;
    a.timeout_ns = ctx->timeout_ns;
    return launch_loop(a, dtype, st, ctx->loop_shape);
}

// The device block of tmfg_solve_host (grown like the workspace).
int ensure_io(tmfg_ctx *c, size_t bytes, cudaStream_t stream)
{
    if (bytes <= c->io_bytes) return TMFG_OK;
    if (c->budget && c->work_bytes + bytes > c->budget) return TMFG_ENOMEM;
    if (c->io) {
        if (cudaStreamSynchronize(stream) != cudaSuccess) return TMFG_ECUDA;
        cudaFree(c->io);
        c->io = nullptr;
        c->io_bytes = 0;
    }
    if (cudaMalloc(&c->io, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->io = nullptr;
        return TMFG_ENOMEM;
    }
    c->io_bytes = bytes;
    return TMFG_OK;
}

int ensure_stage_events(tmfg_ctx *c)
{
    if (!c->tev_ready) {
        for (cudaEvent_t &e : c->tev)
            if (cudaEventCreate(&e) != cudaSuccess) return TMFG_ECUDA;
        c->tev_ready = true;
    }
    for (bool &u : c->tev_used) u = false;
    return TMFG_OK;
}

int ensure_copy_stream(tmfg_ctx *c)
{
    if (!c->cstream &&
        cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking) != cudaSuccess)
        return TMFG_ECUDA;
    if (!c->ev_ready) {
        for (cudaEvent_t &e : c->ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return TMFG_ECUDA;
        c->ev_ready = true;
    }
    return TMFG_OK;
}

}  // namespace

extern "C" {

int tmfg_create(tmfg_ctx **out, int device, size_t workspace_budget_bytes)
{
    if (!out) return TMFG_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return TMFG_ECUDA;
    }
    DeviceGuard g(device);
    if (!g.ok) return TMFG_ECUDA;
    tmfg_ctx *c = new (std::nothrow) tmfg_ctx();
    if (!c) return TMFG_ENOMEM;
    c->device = device;
    c->budget = workspace_budget_bytes;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&c->status, 256) != cudaSuccess) {
        delete c;
        return TMFG_ECUDA;
    }
    c->stats = reinterpret_cast<long long *>(reinterpret_cast<char *>(c->status) + 64);
    if (cudaMemset(c->status, 0, 256) != cudaSuccess) {
        cudaFree(c->status);
        delete c;
        return TMFG_ECUDA;
    }
    if (cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(c->status);
        delete c;
        return TMFG_ECUDA;
    }
    c->timeout_ns = device_timeout_ns();
    *out = c;
    return TMFG_OK;
}

void tmfg_destroy(tmfg_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->work) cudaFree(ctx->work);
    if (ctx->status) cudaFree(ctx->status);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    cudaEventDestroy(ctx->stage_ev);
    if (ctx->io) cudaFree(ctx->io);
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    if (ctx->ev_ready)
        for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->tev_ready)
        for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
    if (ctx->aux_ready) {
        for (cudaStream_t a : ctx->aux) cudaStreamDestroy(a);
        for (cudaEvent_t e : ctx->aux_ev) cudaEventDestroy(e);
    }
    delete ctx;
}

int64_t tmfg_max_n_mode(int dtype, int mode, int prefix)
{
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return 0;
    if (mode != TMFG_CORR && mode != TMFG_HEAP) return 0;
    int64_t m = rowsort_max_n(dtype);
    const int64_t lm = loop_max_n(dtype, mode, prefix > 1 ? 2 : 1);
    if (lm < m) m = lm;
    while (m > 4 && (sssp_smem_bytes((int)m) > kSmemLimit || 2 * m - 4 > 65535)) --m;
    return m;
}

int64_t tmfg_max_n(int dtype) { return tmfg_max_n_mode(dtype, TMFG_CORR, 1); }

size_t tmfg_workspace_bytes(int64_t n, int dtype, int what, int n_hubs)
{
    (void)dtype;
    if (n < 4) return 0;
    if (what == 0) return build_work_bytes(n);
    if (what == 3) return dbht_work_bytes((int)n);
    return apsp_work_bytes((int)n, what == 2, hubs_for(n, n_hubs));
}

int tmfg_row_sort(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                  uint16_t *idx, int64_t ldi, int64_t *rowsum, void *stream)
{
    if (!ctx || !S || !idx || n < 2 || ld < n || ldi < n - 1) return TMFG_EINVAL;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (n > rowsort_max_n(dtype)) return TMFG_ETOOBIG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    return launch_rowsort(S, (int)n, ld, dtype, idx, ldi, reinterpret_cast<long long *>(rowsum),
                          ctx->status, ctx->num_sms, static_cast<cudaStream_t>(stream));
}

int tmfg_build(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, const tmfg_params *params,
               int32_t *order, int32_t *edges, int32_t *ins_face, int32_t *bubble_parent,
               void *stream)
{
    if (!ctx || !S || !params || !order || !edges || !bubble_parent || n < 4 || ld < n)
        return TMFG_EINVAL;
    if (n > 4 && !ins_face) return TMFG_EINVAL;
    const int dtype = params->dtype;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (params->mode != TMFG_CORR && params->mode != TMFG_HEAP) return TMFG_EINVAL;
    if (params->prefix < 1 || params->prefix > kMaxPrefixApi) return TMFG_EINVAL;
    if (params->mode == TMFG_HEAP && params->prefix != 1) return TMFG_EINVAL;
    if (n > tmfg_max_n_mode(dtype, params->mode, params->prefix)) return TMFG_ETOOBIG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(ctx, build_work_bytes(n), st);
    if (rc) return rc;
    BuildWork w = build_carve(ctx->work, n);
    if (params->flags & TMFG_CHECK_SYMMETRY) {
        rc = check_symmetry(ctx, S, n, ld, dtype, st);
        if (rc) return rc;
    }
    rc = launch_rowsort(S, (int)n, ld, dtype, w.idx, ldi_for(n), w.rowsum, ctx->status,
                        ctx->num_sms, st);
    if (rc) return rc;
    return launch_build_loop(ctx, w, S, n, ld, params, order, edges, ins_face, bubble_parent, st);
}



int tmfg_batch_run(tmfg_ctx *ctx, const tmfg_job *jobs, int32_t count, const tmfg_params *params,
                   const tmfg_batch_config *cfg, void *stream)
{
    if (!ctx || !jobs || count < 1 || !params) return TMFG_EINVAL;
    const int dtype = params->dtype;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (params->mode != TMFG_CORR && params->mode != TMFG_HEAP) return TMFG_EINVAL;
    if (params->prefix < 1 || params->prefix > kMaxPrefixApi) return TMFG_EINVAL;
    if (params->mode == TMFG_HEAP && params->prefix != 1) return TMFG_EINVAL;
    const int sssp_threads = (cfg && cfg->sssp_threads) ? cfg->sssp_threads : 512;
    if (sssp_threads != 256 && sssp_threads != 512) return TMFG_EINVAL;
    LoopShape shape;
    if (!loop_shape_from(cfg ? &cfg->loop : nullptr, &shape)) return TMFG_EINVAL;
    if (shape.general == 2) return TMFG_EINVAL;  // the cluster kernel runs single builds only
    const int64_t maxn_lib = tmfg_max_n_mode(dtype, params->mode, params->prefix);
    int max_n = 0, napsp = 0;
    for (int i = 0; i < count; ++i) {
        const tmfg_job &J = jobs[i];
        if (!J.S || J.n < 4 || J.ld < J.n || !J.order || !J.edges || !J.bubble_parent ||
            (J.n > 4 && !J.ins_face) || (J.D && J.ldd < J.n))
            return TMFG_EINVAL;
        if (J.n > maxn_lib) return TMFG_ETOOBIG;
        if (J.n > max_n) max_n = (int)J.n;
        napsp += J.D != nullptr;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- sizes: descriptor tables, then per-instance blocks
    const size_t t_sort = round256(sizeof(SortJob) * count);
    const size_t t_rows = round256(sizeof(int) * (count + 1));
    const size_t t_loop = round256(sizeof(LoopArgs) * count);
    const size_t t_ajob = round256(sizeof(ApspJob) * (napsp + 1));
    const size_t t_sarg = round256(sizeof(SsspArgs) * (napsp + 1));
    const size_t t_ebeg = round256(sizeof(int) * (napsp + 1));
    const size_t t_sbeg = round256(sizeof(int) * (napsp + 1));
    const size_t tables = t_sort + t_rows + t_loop + t_ajob + t_sarg + t_ebeg + t_sbeg;
    if (tables != batch_table_bytes(count, napsp)) return TMFG_EINTERNAL;
    size_t build_bytes = 0, apsp_bytes = 0, deg_bytes = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t n = jobs[i].n;
        const size_t nf = 2 * (size_t)n - 4;
        build_bytes += round256(2 * (size_t)n * (size_t)ldi_for(n)) + round256(8 * (size_t)n) +
                       round256(16 * nf) * 4 + round256(8 * nf) + round256(4 * nf) + 256;
        if (jobs[i].D) {
            deg_bytes += 4 * (size_t)n;
            apsp_bytes += round256(4 * ((size_t)n + 1)) + round256(4 * (size_t)n) +
                          round256(8 * 2 * (3 * (size_t)n - 6));
        }
    }
    deg_bytes = round256(deg_bytes);
    const size_t total = tables + build_bytes + deg_bytes + apsp_bytes;
    // Under stream capture nothing may allocate or wait: the workspace and
    // the staging buffer must already be large enough (run the same batch
    // once uncaptured first), and the captured descriptor copy reads the
    // staging buffer when the graph is replayed.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return TMFG_ECUDA;
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    if (capturing && (total > ctx->work_bytes || tables > ctx->stage_bytes)) return TMFG_ENOMEM;
    int rc = ensure_work(ctx, total, st);
    if (rc) return rc;

    // ---- host staging buffer (reused once its last copy has completed)
    if (!capturing && ctx->stage_used && cudaEventSynchronize(ctx->stage_ev) != cudaSuccess)
        return TMFG_ECUDA;
    rc = ensure_stage(ctx, tables);
    if (rc) return rc;
    char *hb = static_cast<char *>(ctx->stage);
    char *db = static_cast<char *>(ctx->work);
    SortJob *h_sort = reinterpret_cast<SortJob *>(hb);
    int *h_rows = reinterpret_cast<int *>(hb + t_sort);
    LoopArgs *h_loop = reinterpret_cast<LoopArgs *>(hb + t_sort + t_rows);
    ApspJob *h_ajob = reinterpret_cast<ApspJob *>(hb + t_sort + t_rows + t_loop);
    SsspArgs *h_sarg = reinterpret_cast<SsspArgs *>(hb + t_sort + t_rows + t_loop + t_ajob);
    int *h_ebeg = reinterpret_cast<int *>(hb + t_sort + t_rows + t_loop + t_ajob + t_sarg);
    int *h_sbeg = reinterpret_cast<int *>(hb + t_sort + t_rows + t_loop + t_ajob + t_sarg + t_ebeg);
    const SortJob *d_sort = reinterpret_cast<const SortJob *>(db);
    const int *d_rows = reinterpret_cast<const int *>(db + t_sort);
    const LoopArgs *d_loop = reinterpret_cast<const LoopArgs *>(db + t_sort + t_rows);
    const ApspJob *d_ajob = reinterpret_cast<const ApspJob *>(db + t_sort + t_rows + t_loop);
    const SsspArgs *d_sarg = reinterpret_cast<const SsspArgs *>(db + t_sort + t_rows + t_loop + t_ajob);
    const int *d_ebeg = reinterpret_cast<const int *>(db + t_sort + t_rows + t_loop + t_ajob + t_sarg);
    const int *d_sbeg = reinterpret_cast<const int *>(db + t_sort + t_rows + t_loop + t_ajob + t_sarg + t_ebeg);

    char *p = db + tables;
    char *deg = p + build_bytes;
    char *ap = deg + deg_bytes;
    auto take = [&](char *&q, size_t x) { void *r = q; q += round256(x); return r; };
    int row_acc = 0, edge_acc = 0, src_acc = 0, a = 0;
    size_t deg_off = 0;
    for (int i = 0; i < count; ++i) {
        const tmfg_job &J = jobs[i];
        const int n = (int)J.n;
        const size_t nf = 2 * (size_t)n - 4;
        const long long ldi = ldi_for(n);
        uint16_t *idx = static_cast<uint16_t *>(take(p, 2 * (size_t)n * (size_t)ldi));
        long long *rowsum = static_cast<long long *>(take(p, 8 * (size_t)n));
        int4 *face = static_cast<int4 *>(take(p, 16 * nf));
        void *lf = take(p, 16 * nf);
        void *ls = take(p, 16 * nf);
        void *pk = take(p, 16 * nf);
        unsigned long long *pc = static_cast<unsigned long long *>(take(p, 8 * nf));
        int *fu = static_cast<int *>(take(p, 4 * nf));
        long long *stats = static_cast<long long *>(take(p, 128));
        SortJob &sj = h_sort[i];
        sj.S = J.S;
        sj.ld = J.ld;
        sj.n = n;
        sj.vec_in = (J.ld % (dtype == TMFG_F32 ? 4 : 2) == 0) && ((uintptr_t)J.S % 16 == 0);
        sj.vec_out = true;
        sj.idx = idx;
        sj.ldi = ldi;
        sj.rowsum = rowsum;
        h_rows[i] = row_acc;
        row_acc += n;
        LoopArgs &la = h_loop[i];
        la = LoopArgs{};
        la.S = J.S;
        la.ld = J.ld;
        la.n = n;
        la.mode = params->mode;
        la.P = params->prefix;
        la.idx = idx;
        la.ldi = ldi;
        la.rowsum = rowsum;
        la.order = J.order;
        la.edges = J.edges;
        la.ins_face = J.ins_face;
        la.parent = J.bubble_parent;
        la.face = face;
        la.leaf_fresh = lf;
        la.leaf_stale = ls;
        la.pend_key = pk;
        la.pend_cand = pc;
        la.fu_buf = fu;
        la.status = ctx->status;
        la.stats = stats;
        la.timeout_ns = ctx->timeout_ns;
        la.state = nullptr;
        la.k_stop = n - 4;
        la.resume = 0;
        if (J.D) {
            ApspJob &aj = h_ajob[a];
            aj.S = J.S;
            aj.ld = J.ld;
            aj.n = n;
            aj.edges = J.edges;
            aj.deg = reinterpret_cast<int *>(deg + deg_off);
            deg_off += 4 * (size_t)n;
            aj.rowptr = static_cast<int *>(take(ap, 4 * ((size_t)n + 1)));
            aj.cursor = static_cast<int *>(take(ap, 4 * (size_t)n));
            aj.arcs = static_cast<uint2 *>(take(ap, 8 * 2 * (3 * (size_t)n - 6)));
            SsspArgs &sa = h_sarg[a];
            sa = SsspArgs{};
            sa.n = n;
            sa.rowptr = aj.rowptr;
            sa.arcs = aj.arcs;
            sa.src = nullptr;
            sa.nsrc = n;
            sa.out = J.D;
            sa.ldo = J.ldd;
            sa.status = ctx->status;
            sa.timeout_ns = ctx->timeout_ns;
            h_ebeg[a] = edge_acc;
            h_sbeg[a] = src_acc;
            edge_acc += 3 * n - 6;
            src_acc += n;
            ++a;
        }
    }
    h_rows[count] = row_acc;
    h_ebeg[napsp] = edge_acc;
    h_sbeg[napsp] = src_acc;
    if (cudaMemcpyAsync(db, hb, tables, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return TMFG_ECUDA;
    if (!capturing) {
        if (cudaEventRecord(ctx->stage_ev, st) != cudaSuccess) return TMFG_ECUDA;
        ctx->stage_used = true;
    }
    if (napsp && cudaMemsetAsync(deg, 0, deg_bytes, st) != cudaSuccess) return TMFG_ECUDA;

    rc = launch_rowsort_batch(d_sort, d_rows, count, max_n, dtype, ctx->status,
                              ctx->num_sms * 2, st);
    if (rc) return rc;
    rc = launch_loop_batch(d_loop, count, max_n, dtype, params->mode, params->prefix, st, shape);
    if (rc) return rc;
    if (napsp)
        rc = launch_apsp_batch(d_ajob, d_sarg, d_ebeg, d_sbeg, napsp, edge_acc, max_n, dtype,
                               sssp_threads, ctx->status, ctx->num_sms, st);
    return rc;
}

int tmfg_apsp(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
              const int32_t *edges, const tmfg_apsp_params *params, float *D, int64_t ldd,
              void *stream)
{
    if (!ctx || !S || !edges || !D || n < 4 || ld < n || ldd < n) return TMFG_EINVAL;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (n > 65535 || sssp_smem_bytes((int)n) > kSmemLimit) return TMFG_ETOOBIG;
    const int approx = params ? params->approx : 0;
    const int h = hubs_for(n, params ? params->n_hubs : 0);
    const float rf = (params && params->radius_factor > 0.0f) ? params->radius_factor : 2.0f;
    if (approx && (h < 1 || 4 * (n + h) > (int64_t)kSmemLimit - 1024)) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(ctx, apsp_work_bytes((int)n, approx, h), st);
    if (rc) return rc;
    return launch_apsp(S, (int)n, ld, dtype, edges, approx, h, rf, D, ldd, ctx->work, ctx->status,
                       ctx->num_sms, ctx->timeout_ns, st);
}

int tmfg_similarity(tmfg_ctx *ctx, const float *X, int64_t n, int64_t T, int32_t precision,
                    float *S, int64_t ld, void *stream)
{
    if (!ctx || !X || !S || n < 2 || T < 2 || ld < n || n > INT32_MAX / 2 || T > INT32_MAX / 2)
        return TMFG_EINVAL;
    if (precision < TMFG_SIM_F64 || precision > TMFG_SIM_TF32X3) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(ctx, sim_work_bytes((int)n, (int)T, precision), st);
    if (rc) return rc;
    return launch_similarity(X, (int)n, (int)T, T, precision, S, ld, ctx->work, ctx->status,
                             ctx->timeout_ns, st);
}

int dbht_cluster_detail(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                        const int32_t *order, const int32_t *edges, const int32_t *ins_face,
                        const int32_t *bubble_parent, const float *D, int64_t ldd,
                        double *linkage, const dbht_outputs *out, void *stream)
{
    if (!ctx || !S || !order || !edges || !bubble_parent || !D || !linkage || n < 4 || ld < n ||
        ldd < n)
        return TMFG_EINVAL;
    if (n > 4 && !ins_face) return TMFG_EINVAL;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (n > DBHT_MAX_N || dbht_smem_bytes((int)n) > kSmemLimit) return TMFG_ETOOBIG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_work(ctx, dbht_work_bytes((int)n), st);
    if (rc) return rc;
    return launch_dbht(S, (int)n, ld, dtype, order, edges, ins_face, bubble_parent, D, ldd,
                       linkage, out ? out->direction : nullptr, out ? out->converging : nullptr,
                       out ? out->group : nullptr, out ? out->bubble : nullptr, ctx->work,
                       ctx->status, ctx->num_sms, st);
}

int dbht_cluster(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                 const int32_t *order, const int32_t *edges, const int32_t *ins_face,
                 const int32_t *bubble_parent, const float *D, int64_t ldd, double *linkage,
                 void *stream)
{
    return dbht_cluster_detail(ctx, S, n, ld, dtype, order, edges, ins_face, bubble_parent, D, ldd,
                               linkage, nullptr, stream);
}

int tmfg_solve_host(tmfg_ctx *ctx, const void *S_host, int64_t n, int64_t ld,
                    const tmfg_params *params, const tmfg_solve_params *sp, int32_t *order,
                    int32_t *edges, int32_t *ins_face, int32_t *bubble_parent, float *D_exact,
                    float *D_approx, int64_t ldd, void *stream)
{
    if (!ctx || !S_host || !params || !order || !edges || !bubble_parent || n < 4 || ld < n)
        return TMFG_EINVAL;
    if (n > 4 && !ins_face) return TMFG_EINVAL;
    if ((D_exact || D_approx) && ldd < n) return TMFG_EINVAL;
    const int dtype = params->dtype;
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return TMFG_EINVAL;
    if (params->mode != TMFG_CORR && params->mode != TMFG_HEAP) return TMFG_EINVAL;
    if (params->prefix < 1 || params->prefix > kMaxPrefixApi) return TMFG_EINVAL;
    if (params->mode == TMFG_HEAP && params->prefix != 1) return TMFG_EINVAL;
    if (n > tmfg_max_n_mode(dtype, params->mode, params->prefix)) return TMFG_ETOOBIG;
    const int h = hubs_for(n, sp ? sp->n_hubs : 0);
    const float rf = (sp && sp->radius_factor > 0.0f) ? sp->radius_factor : 2.0f;
    if (D_approx && (h < 1 || 4 * (n + h) > (int64_t)kSmemLimit - 1024)) return TMFG_EINVAL;
    int blocks = sp && sp->row_blocks > 0 ? sp->row_blocks : 8;
    if (blocks > 32) blocks = 32;
    if (blocks > n) blocks = (int)n;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = ensure_copy_stream(ctx);
    if (rc) return rc;
    rc = ensure_stage_events(ctx);
    if (rc) return rc;
    cudaStream_t cs = ctx->cstream;
    auto mark = [&](int i, cudaStream_t on) {
        ctx->tev_used[i] = true;
        return cudaEventRecord(ctx->tev[i], on) != cudaSuccess;
    };
    // one workspace for every stage (no reallocation between them)
    size_t wb = build_work_bytes(n);
    if (D_exact) wb = wb > apsp_work_bytes((int)n, 0, h) ? wb : apsp_work_bytes((int)n, 0, h);
    if (D_approx) wb = wb > apsp_work_bytes((int)n, 1, h) ? wb : apsp_work_bytes((int)n, 1, h);
    rc = ensure_work(ctx, wb, st);
    if (rc) return rc;
    // device block: S, D, D approx, then the TMFG outputs
    const size_t esz = dtype == TMFG_F32 ? 4 : 8;
    const size_t bS = round256((size_t)n * (size_t)ld * esz);
    const size_t bD = round256((size_t)n * (size_t)n * 4);
    const size_t bo = round256(4 * (size_t)n) + round256(8 * (3 * (size_t)n - 6)) +
                      round256(12 * (size_t)(n > 4 ? n - 4 : 1)) + round256(4 * (size_t)n);
    rc = ensure_io(ctx, bS + (D_exact ? bD : 0) + (D_approx ? bD : 0) + bo, st);
    if (rc) return rc;
    char *p = static_cast<char *>(ctx->io);
    void *dS = p;
    p += bS;
    float *dD = D_exact ? reinterpret_cast<float *>(p) : nullptr;
    p += D_exact ? bD : 0;
    float *dDa = D_approx ? reinterpret_cast<float *>(p) : nullptr;
    p += D_approx ? bD : 0;
    int32_t *d_order = reinterpret_cast<int32_t *>(p);
    p += round256(4 * (size_t)n);
    int32_t *d_edges = reinterpret_cast<int32_t *>(p);
    p += round256(8 * (3 * (size_t)n - 6));
    int32_t *d_face = reinterpret_cast<int32_t *>(p);
    p += round256(12 * (size_t)(n > 4 ? n - 4 : 1));
    int32_t *d_parent = reinterpret_cast<int32_t *>(p);

    cudaEvent_t *ev = ctx->ev;
    auto fail = [](cudaError_t e) { return e != cudaSuccess; };
    // copies wait for the compute stream's earlier work on these buffers
    if (fail(cudaEventRecord(ev[0], st)) || fail(cudaStreamWaitEvent(cs, ev[0], 0)) ||
        mark(0, cs))
        return TMFG_ECUDA;
    BuildWork w = build_carve(ctx->work, n);
    // S in row blocks: each block is sorted as soon as it has arrived
    for (int b = 0; b < blocks; ++b) {
        const int64_t r0 = n * b / blocks, r1 = n * (b + 1) / blocks;
        const size_t off = (size_t)r0 * (size_t)ld * esz;
        // rows r0..r1-1, reading no further than the last row's n elements
        const size_t bytes = ((size_t)(r1 - r0 - 1) * (size_t)ld + (size_t)n) * esz;
        if (fail(cudaMemcpyAsync(static_cast<char *>(dS) + off,
                                 static_cast<const char *>(S_host) + off, bytes,
                                 cudaMemcpyHostToDevice, cs)) ||
            fail(cudaEventRecord(ev[1 + b], cs)) || fail(cudaStreamWaitEvent(st, ev[1 + b], 0)))
            return TMFG_ECUDA;
        rc = launch_rowsort(dS, (int)n, ld, dtype, w.idx, ldi_for(n), w.rowsum, ctx->status,
                            ctx->num_sms, st, (int)r0, (int)r1);
        if (rc) return rc;
    }
    if (mark(1, cs)) return TMFG_ECUDA;
    if (params->flags & TMFG_CHECK_SYMMETRY) {
        rc = check_symmetry(ctx, dS, n, ld, dtype, st);
        if (rc) return rc;
    }
    rc = launch_build_loop(ctx, w, dS, n, ld, params, d_order, d_edges, d_face, d_parent, st);
    if (rc) return rc;
    if (mark(2, st)) return TMFG_ECUDA;
    // the TMFG goes back while the distances are computed
    auto out_copy = [&](int e, void *dst, const void *src, size_t bytes) {
        return fail(cudaEventRecord(ev[e], st)) || fail(cudaStreamWaitEvent(cs, ev[e], 0)) ||
               fail(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cs));
    };
    if (out_copy(33, order, d_order, 4 * (size_t)n) ||
        fail(cudaMemcpyAsync(edges, d_edges, 8 * (3 * (size_t)n - 6), cudaMemcpyDeviceToHost, cs)) ||
        (n > 4 && fail(cudaMemcpyAsync(ins_face, d_face, 12 * (size_t)(n - 4),
                                       cudaMemcpyDeviceToHost, cs))) ||
        fail(cudaMemcpyAsync(bubble_parent, d_parent, 4 * (size_t)(n - 3), cudaMemcpyDeviceToHost,
                             cs)))
        return TMFG_ECUDA;
    // rows [r0, r1) of a distance matrix to the host, after the work on st so far
    auto d_copy = [&](int e, float *dst, const float *src, int64_t r0, int64_t r1) {
        if (fail(cudaEventRecord(ev[e], st)) || fail(cudaStreamWaitEvent(cs, ev[e], 0)))
            return true;
        if (ldd == n)  // one contiguous block: the plain copy runs at full link speed
            return fail(cudaMemcpyAsync(dst + r0 * n, src + r0 * n, 4 * (size_t)n * (r1 - r0),
                                        cudaMemcpyDeviceToHost, cs));
        return fail(cudaMemcpy2DAsync(dst + r0 * ldd, 4 * (size_t)ldd, src + r0 * n, 4 * (size_t)n,
                                      4 * (size_t)n, (size_t)(r1 - r0), cudaMemcpyDeviceToHost,
                                      cs));
    };
    // the approximate matrix first: its download (one block, after its
    // symmetric pass) overlaps the exact searches
    if (D_approx) {
        rc = launch_apsp(dS, (int)n, ld, dtype, d_edges, 1, h, rf, dDa, n, ctx->work,
                         ctx->status, ctx->num_sms, ctx->timeout_ns, st);
        if (rc) return rc;
        if (d_copy(38, D_approx, dDa, 0, n) || mark(7, cs)) return TMFG_ECUDA;
    }
    if (D_exact) {
        // four pieces of sources: each piece's rows go back while the next computes
        rc = launch_apsp_csr(dS, (int)n, ld, dtype, d_edges, ctx->work, ctx->status, st);
        if (rc) return rc;
        constexpr int kPieces = 4;
        for (int b = 0; b < kPieces; ++b) {
            const int64_t s0 = n * b / kPieces, s1 = n * (b + 1) / kPieces;
            rc = launch_apsp_exact_rows((int)n, ctx->work, dD, n, (int)s0, (int)s1, ctx->status,
                                        ctx->num_sms, ctx->timeout_ns, st);
            if (rc) return rc;
            if (d_copy(34 + b, D_exact, dD, s0, s1) || mark(3 + b, cs)) return TMFG_ECUDA;
        }
    }
    // the call completes on `stream` once every copy has
    if (fail(cudaEventRecord(ev[39], cs)) || fail(cudaStreamWaitEvent(st, ev[39], 0)))
        return TMFG_ECUDA;
    return TMFG_OK;
}

int tmfg_sync_status(tmfg_ctx *ctx, void *stream)
{
    if (!ctx) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return TMFG_ECUDA;
    }
    int code = 0;
    if (cudaMemcpy(&code, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ctx->host_stats, ctx->stats, sizeof(ctx->host_stats), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return TMFG_ECUDA;
    if (code && cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess) return TMFG_ECUDA;
    return code;
}

int tmfg_solve_host_stages(tmfg_ctx *ctx, float *ms, int32_t count)
{
    if (!ctx || !ms || count < 0) return TMFG_EINVAL;
    if (!ctx->tev_ready || !ctx->tev_used[0]) return TMFG_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return TMFG_ECUDA;
    for (int i = 0; i < count && i < 8; ++i) {
        ms[i] = -1.0f;
        if (!ctx->tev_used[i]) continue;
        if (cudaEventSynchronize(ctx->tev[i]) != cudaSuccess ||
            cudaEventElapsedTime(&ms[i], ctx->tev[0], ctx->tev[i]) != cudaSuccess)
            return TMFG_ECUDA;
    }
    return TMFG_OK;
}

int tmfg_set_loop_shape(tmfg_ctx *ctx, const tmfg_loop_shape *shape)
{
    if (!ctx) return TMFG_EINVAL;
    LoopShape s;
    if (!loop_shape_from(shape, &s)) return TMFG_EINVAL;
    ctx->loop_shape = s;
    return TMFG_OK;
}

int tmfg_last_stats(tmfg_ctx *ctx, int64_t *out, int count)
{
    if (!ctx || !out || count < 0) return TMFG_EINVAL;
    for (int i = 0; i < count && i < 16; ++i) out[i] = ctx->host_stats[i];
    return TMFG_OK;
}

const char *tmfg_strerror(int code)
{
    switch (code) {
        case TMFG_OK: return "ok";
        case TMFG_EINVAL: return "invalid argument";
        case TMFG_ENOMEM: return "out of memory (workspace budget or device)";
        case TMFG_ENONFINITE: return "S has a NaN or infinite off-diagonal entry";
        case TMFG_EASYMMETRIC: return "S is not symmetric";
        case TMFG_ETIMEOUT: return "a device loop reached its time limit";
        case TMFG_ECUDA: return "CUDA runtime error";
        case TMFG_ERANGE: return "an off-diagonal |S| exceeds 64";
        case TMFG_ETOOBIG: return "n exceeds the supported size for this dtype";
        case TMFG_EINTERNAL: return "internal consistency check failed";
        default: return "unknown error";
    }
}

}  // extern "C"
