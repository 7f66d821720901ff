// serve.cu -- a request server with continuous batching over tmfg_batch_run.
//
// No counterpart in the paper: it turns the batched construction into a
// service.  Callers submit TMFG (+ exact APSP) jobs whose buffers are already
// resident in device memory; one host worker thread groups waiting jobs into
// batches and runs each batch on one of several lanes.  A lane is a context
// (its workspace sized once, at start, to the lane's memory budget) plus a
// non-blocking stream, so batches on different lanes overlap on the GPU, and
// jobs that arrive while other batches run are admitted as soon as a lane
// frees up -- FIFO, as many as fit the lane's memory and the batch cap.
// Completion reaches the worker through a host function enqueued after each
// batch (no polling of the device); the batch's status word is copied to
// pinned memory and cleared on the lane's stream before that.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "ctx.cuh"

using namespace tmfg;

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int64_t id;
    tmfg_job job;
    tmfg_pipeline_job pjob;  // pipeline servers
    size_t bytes;
    int64_t t_submit;
    cudaEvent_t ready;  // recorded on the submitter's stream
};

struct Lane {
    tmfg_server *srv = nullptr;
    tmfg_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int *h_status = nullptr;  // pinned: the batch's status word
    std::vector<Request> reqs;
    int launch_rc = 0;
    int64_t t_launch = 0, t_done = 0;
    int seq = 0;
    bool busy = false, finished = false;
};

}  // namespace

struct tmfg_server {
    int device = 0;
    tmfg_serve_config cfg{};
    tmfg_params params{};
    std::vector<Lane> lanes;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable cv_done;  // wakes pollers
    std::deque<Request> queue;
    std::deque<tmfg_serve_result> done;
    std::vector<cudaEvent_t> event_pool;
    bool stop = false;
    int64_t next_id = 0;
    int batch_seq = 0;
    int sticky = TMFG_OK;
    std::thread worker;
};

namespace {

void CUDART_CB lane_done(void *p)
{
    Lane *l = static_cast<Lane *>(p);
    tmfg_server *s = l->srv;
    std::lock_guard<std::mutex> g(s->mu);
    l->finished = true;
    l->t_done = now_ns();
    s->cv.notify_all();
}

// Number of requests from the front of `q` that form the next batch: FIFO,
// at most max_batch, while the descriptor tables plus the requests' blocks
// fit lane_bytes.  The first request always fits (checked at submission).
int plan_batch(const std::deque<Request> &q, int max_batch, size_t lane_bytes, bool apsp)
{
    size_t acc = 0;
    int c = 0;
    for (const Request &r : q) {
        if (c == max_batch) break;
        const size_t need = acc + r.bytes + batch_table_bytes(c + 1, apsp ? c + 1 : 0);
        if (need > lane_bytes && c > 0) break;
        acc += r.bytes;
        ++c;
    }
    return c;
}

// Launch lane l's batch (no lock held).
void launch(tmfg_server *s, Lane &l)
{
    DeviceGuard g(s->device);
    std::vector<tmfg_job> jobs(l.reqs.size());
    int rc = TMFG_OK;
    for (size_t i = 0; i < l.reqs.size(); ++i) {
        jobs[i] = l.reqs[i].job;
        if (cudaStreamWaitEvent(l.stream, l.reqs[i].ready, 0) != cudaSuccess) rc = TMFG_ECUDA;
    }
    tmfg_batch_config bc{};
    bc.sssp_threads = s->cfg.sssp_threads;
    if (rc == TMFG_OK && s->cfg.pipeline) {
        std::vector<tmfg_pipeline_job> pj(l.reqs.size());
        for (size_t i = 0; i < l.reqs.size(); ++i) pj[i] = l.reqs[i].pjob;
        tmfg_pipeline_params pp{};
        pp.precision = s->cfg.precision;
        pp.tmfg = s->params;
        rc = tmfg_pipeline_run(l.ctx, pj.data(), (int)pj.size(), &pp, &bc, l.stream);
    } else if (rc == TMFG_OK) {
        rc = tmfg_batch_run(l.ctx, jobs.data(), (int)jobs.size(), &s->params, &bc, l.stream);
    }
    l.launch_rc = rc;
    *l.h_status = 0;
    cudaMemcpyAsync(l.h_status, l.ctx->status, sizeof(int), cudaMemcpyDeviceToHost, l.stream);
    cudaMemsetAsync(l.ctx->status, 0, sizeof(int), l.stream);
    if (cudaLaunchHostFunc(l.stream, lane_done, &l) != cudaSuccess) {
        // the completion cannot be signalled: wait here instead
        cudaStreamSynchronize(l.stream);
        std::lock_guard<std::mutex> gl(s->mu);
        l.finished = true;
        l.t_done = now_ns();
        if (!l.launch_rc) l.launch_rc = TMFG_ECUDA;
    }
}

void worker_main(tmfg_server *s)
{
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions
        for (Lane &l : s->lanes) {
            if (!l.busy || !l.finished) continue;
            const int st = l.launch_rc ? l.launch_rc : *l.h_status;
            for (const Request &r : l.reqs) {
                tmfg_serve_result res{};
                res.id = r.id;
                res.status = st;
                res.batch = l.seq;
                res.batch_size = (int32_t)l.reqs.size();
                res.t_submit_ns = r.t_submit;
                res.t_launch_ns = l.t_launch;
                res.t_done_ns = l.t_done;
                s->done.push_back(res);
                s->event_pool.push_back(r.ready);
            }
            l.reqs.clear();
            l.busy = l.finished = false;
            s->cv_done.notify_all();
        }
        // admissions: every free lane takes the next batch
        bool launched = false;
        for (Lane &l : s->lanes) {
            if (l.busy || s->queue.empty()) continue;
            const int c = plan_batch(s->queue, s->cfg.max_batch, s->cfg.lane_bytes,
                                     s->cfg.apsp != 0);
            l.reqs.assign(s->queue.begin(), s->queue.begin() + c);
            s->queue.erase(s->queue.begin(), s->queue.begin() + c);
            l.busy = true;
            l.finished = false;
            l.seq = s->batch_seq++;
            l.t_launch = now_ns();
            lk.unlock();
            launch(s, l);
            lk.lock();
            launched = true;
        }
        if (launched) continue;  // completions may have arrived meanwhile
        bool any_busy = false;
        for (const Lane &l : s->lanes) any_busy |= l.busy;
        if (s->stop && s->queue.empty() && !any_busy) break;
        bool ready = false;
        for (const Lane &l : s->lanes) ready |= l.busy && l.finished;
        bool free_lane = false;
        for (const Lane &l : s->lanes) free_lane |= !l.busy;
        if (ready || (free_lane && !s->queue.empty())) continue;
        // bounded wait: a lost wake-up costs at most one period
        s->cv.wait_for(lk, std::chrono::milliseconds(50));
    }
}

// Admit request r (bytes set) to the queue once the submitter's stream
// reaches this point; returns its id or minus an error code.
int64_t enqueue(tmfg_server *s, Request &r, void *stream)
{
    if (r.bytes + batch_table_bytes(1, s->cfg.apsp ? 1 : 0) > s->cfg.lane_bytes)
        return -TMFG_ENOMEM;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return -TMFG_EINVAL;
        if (!s->event_pool.empty()) {
            r.ready = s->event_pool.back();
            s->event_pool.pop_back();
        }
    }
    DeviceGuard g(s->device);
    if (!g.ok) return -TMFG_ECUDA;
    if (!r.ready && cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming) != cudaSuccess)
        return -TMFG_ECUDA;
    // the job's inputs are ready once the submitter's stream reaches here
    if (cudaEventRecord(r.ready, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaEventDestroy(r.ready);
        return -TMFG_ECUDA;
    }
    std::lock_guard<std::mutex> lg(s->mu);
    r.id = s->next_id++;
    r.t_submit = now_ns();
    s->queue.push_back(r);
    s->cv.notify_all();
    return r.id;
}

void free_lanes(tmfg_server *s)
{
    DeviceGuard g(s->device);
    for (Lane &l : s->lanes) {
        if (l.stream) {
            cudaStreamSynchronize(l.stream);
            cudaStreamDestroy(l.stream);
        }
        if (l.h_status) cudaFreeHost(l.h_status);
        if (l.ctx) tmfg_destroy(l.ctx);
    }
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    s->event_pool.clear();
}

}  // namespace

extern "C" {

size_t tmfg_serve_request_bytes(int64_t n, int32_t apsp)
{
    if (n < 4) return 0;
    return batch_request_bytes(n, apsp != 0);
}

int tmfg_serve_plan(const int64_t *n, int32_t count, int32_t apsp, int32_t max_batch,
                    size_t lane_bytes, int32_t *batch_of)
{
    if (!n || !batch_of || count < 0 || max_batch < 1) return TMFG_EINVAL;
    std::deque<Request> q;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 4) return TMFG_EINVAL;
        Request r{};
        r.id = i;
        r.bytes = batch_request_bytes(n[i], apsp != 0);
        if (r.bytes + batch_table_bytes(1, apsp ? 1 : 0) > lane_bytes) return TMFG_ENOMEM;
        q.push_back(r);
    }
    int b = 0;
    while (!q.empty()) {
        const int c = plan_batch(q, max_batch, lane_bytes, apsp != 0);
        for (int i = 0; i < c; ++i) batch_of[q[i].id] = b;
        q.erase(q.begin(), q.begin() + c);
        ++b;
    }
    return TMFG_OK;
}

int tmfg_serve_start(tmfg_server **out, int device, const tmfg_serve_config *cfg)
{
    if (!out || !cfg) return TMFG_EINVAL;
    *out = nullptr;
    const tmfg_params &p = cfg->params;
    if (p.dtype != TMFG_F32 && p.dtype != TMFG_F64) return TMFG_EINVAL;
    if (p.mode != TMFG_CORR && p.mode != TMFG_HEAP) return TMFG_EINVAL;
    if (p.prefix < 1 || (p.mode == TMFG_HEAP && p.prefix != 1)) return TMFG_EINVAL;
    if (cfg->lanes < 0 || cfg->lanes > 16 || cfg->max_batch < 0 || cfg->max_batch > 4096)
        return TMFG_EINVAL;
    if (cfg->sssp_threads && cfg->sssp_threads != 256 && cfg->sssp_threads != 512)
        return TMFG_EINVAL;
    if (cfg->pipeline && (p.dtype != TMFG_F32 || cfg->precision < TMFG_SIM_F64 ||
                          cfg->precision > TMFG_SIM_TF32X3))
        return TMFG_EINVAL;
    tmfg_server *s = new (std::nothrow) tmfg_server();
    if (!s) return TMFG_ENOMEM;
    s->device = device;
    s->cfg = *cfg;
    if (!s->cfg.lanes) s->cfg.lanes = 3;
    if (!s->cfg.max_batch) s->cfg.max_batch = 256;
    if (!s->cfg.lane_bytes) s->cfg.lane_bytes = (size_t)4 << 30;
    s->params = p;
    if (s->cfg.pipeline) s->cfg.apsp = 1;  // the dendrogram needs the distances
    s->lanes.resize(s->cfg.lanes);
    int rc = TMFG_OK;
    {
        DeviceGuard g(device);
        if (!g.ok) rc = TMFG_ECUDA;
        for (Lane &l : s->lanes) {
            if (rc) break;
            l.srv = s;
            rc = tmfg_create(&l.ctx, device, 0);
            if (rc) break;
            if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaHostAlloc(reinterpret_cast<void **>(&l.h_status), sizeof(int),
                              cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                rc = TMFG_ECUDA;
                break;
            }
            // every admitted batch fits this workspace: no allocation (and no
            // device-wide synchronisation) once serving
            rc = ensure_work(l.ctx, s->cfg.lane_bytes, l.stream);
            if (!rc)
                rc = ensure_stage(l.ctx, batch_table_bytes(s->cfg.max_batch, s->cfg.max_batch));
        }
        if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = TMFG_ECUDA;
    }
    if (rc) {
        free_lanes(s);
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return TMFG_OK;
}

int64_t tmfg_serve_submit(tmfg_server *s, const tmfg_job *job, void *stream)
{
    if (!s || !job) return -TMFG_EINVAL;
    const tmfg_job &J = *job;
    if (!J.S || J.n < 4 || J.ld < J.n || !J.order || !J.edges || !J.bubble_parent ||
        (J.n > 4 && !J.ins_face) || (J.D && J.ldd < J.n) || (s->cfg.apsp && !J.D))
        return -TMFG_EINVAL;
    if (J.n > tmfg_max_n_mode(s->params.dtype, s->params.mode, s->params.prefix)) return -TMFG_ETOOBIG;
    Request r{};
    r.job = J;
    if (!s->cfg.apsp) r.job.D = nullptr;
    r.bytes = batch_request_bytes(J.n, s->cfg.apsp != 0);
    return enqueue(s, r, stream);
}

int64_t tmfg_serve_submit_pipeline(tmfg_server *s, const tmfg_pipeline_job *job, void *stream)
{
    if (!s || !job || !s->cfg.pipeline) return -TMFG_EINVAL;
    const tmfg_pipeline_job &J = *job;
    if (!J.X || !J.S || !J.order || !J.edges || !J.bubble_parent || !J.D || !J.Z || J.n < 4 ||
        J.T < 2 || J.ldx < J.T || (J.n > 4 && !J.ins_face) || J.k < 0 || J.k > J.n ||
        (J.k > 0 && !J.labels))
        return -TMFG_EINVAL;
    if (J.n > tmfg_max_n_mode(s->params.dtype, s->params.mode, s->params.prefix) ||
        J.n > DBHT_MAX_N)
        return -TMFG_ETOOBIG;
    Request r{};
    r.pjob = J;
    r.job.n = J.n;
    r.bytes = tmfg_pipeline_request_bytes(J.n, J.T, s->cfg.precision);
    return enqueue(s, r, stream);
}

int tmfg_serve_poll(tmfg_server *s, tmfg_serve_result *out, int32_t max, int32_t wait_us)
{
    if (!s || !out || max < 0) return -TMFG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us),
                            [s] { return !s->done.empty(); });
    int c = 0;
    while (c < max && !s->done.empty()) {
        out[c++] = s->done.front();
        s->done.pop_front();
    }
    return c;
}

int64_t tmfg_serve_now_ns(void) { return now_ns(); }

int tmfg_serve_stop(tmfg_server *s)
{
    if (!s) return TMFG_EINVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Request &r : s->queue) s->event_pool.push_back(r.ready);
    const int rc = s->sticky;
    free_lanes(s);
    delete s;
    return rc;
}

}  // extern "C"
