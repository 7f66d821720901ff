// api.cu -- the C ABI of libtmfg.so (declared in include/tmfg.h): context
// and workspace management, argument checks, kernel launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

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

struct tmfg_ctx {
    int device;
    int num_sms;
    size_t budget;
    void *work;
    size_t work_bytes;
    int *status;        // device word
    long long *stats;   // device [8]
    long long host_stats[16];
    unsigned long long timeout_ns;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

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

long long ldi_for(int64_t n) { return ((n - 1) + 7) / 8 * 8; }

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
    c->timeout_ns = 60ull * 1000000000ull;
    if (const char *e = std::getenv("TMFG_TIMEOUT_MS")) {
        const long long ms = std::atoll(e);
        if (ms > 0) c->timeout_ns = (unsigned long long)ms * 1000000ull;
    }
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
    delete ctx;
}

int64_t tmfg_max_n(int dtype)
{
    if (dtype != TMFG_F32 && dtype != TMFG_F64) return 0;
    int64_t m = rowsort_max_n(dtype);
    while (m > 4 && (loop_smem_bytes((int)m, dtype, TMFG_HEAP) > kSmemLimit ||
                      loop_smem_bytes((int)m, dtype, TMFG_CORR) > kSmemLimit ||
                      sssp_smem_bytes((int)m) > kSmemLimit || 2 * m - 4 > 65535))
        --m;
    return m;
}

size_t tmfg_workspace_bytes(int64_t n, int dtype, int what, int n_hubs)
{
    (void)dtype;
    if (n < 4) return 0;
    if (what == 0) return build_work_bytes(n);
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
    if (n > tmfg_max_n(dtype)) return TMFG_ETOOBIG;
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
    return launch_loop(a, dtype, st);
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
