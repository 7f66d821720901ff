// ctx.cuh -- the context object behind tmfg_ctx and the host helpers that
// the entry points (api.cu) and the request server (serve.cu) share.
#pragma once

#include "internal.cuh"

struct tmfg_ctx {
    int device;
    int num_sms;
    size_t budget;
    void *work;
    size_t work_bytes;
    int *status;        // device word
    long long *stats;   // device [8]
    long long host_stats[16];
    tmfg::LoopShape loop_shape;  // shape of the corr-tmfg prefix-1 loop (tmfg_set_loop_shape)
    unsigned long long timeout_ns;
    void *stage;          // pinned host staging buffer for batch descriptor tables
    size_t stage_bytes;
    cudaEvent_t stage_ev; // recorded after the last copy out of the staging buffer
    bool stage_used;
    // tmfg_solve_host: device copies of its inputs and outputs, a copy stream
    // and the events that order the two streams
    void *io;
    size_t io_bytes;
    cudaStream_t cstream;
    cudaEvent_t ev[40];
    bool ev_ready;
    // timing events of the last tmfg_solve_host: start, uploads done, TMFG
    // done, the four exact-distance pieces downloaded, approximate downloaded
    cudaEvent_t tev[8];
    bool tev_ready;
    bool tev_used[8];
    // tmfg_pipeline_run: streams that run the per-request stages side by
    // side, and the events that fork them from and join them to the caller's
    cudaStream_t aux[32];
    cudaEvent_t aux_ev[33];
    bool aux_ready;
};

namespace tmfg {

// Makes `dev` current for the lifetime of the guard.
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

inline size_t round256(size_t x) { return (x + 255) & ~size_t(255); }
inline long long ldi_for(int64_t n) { return ((n - 1) + 7) / 8 * 8; }

// Grow the context workspace to `bytes` (synchronises `stream` and frees the
// old block first when it must grow).
int ensure_work(tmfg_ctx *c, size_t bytes, cudaStream_t stream);
// Grow the pinned staging buffer to `bytes` (only between batches).
int ensure_stage(tmfg_ctx *c, size_t bytes);

// Workspace of a batched run: the descriptor tables of `count` instances
// (`napsp` of them with APSP), and an upper bound of one instance's own
// blocks (sorted rows, loop buffers, and with APSP its CSR).
size_t batch_table_bytes(int count, int napsp);
size_t batch_request_bytes(int64_t n, bool apsp);

}  // namespace tmfg
