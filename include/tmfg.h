/*
 * tmfg.h -- C ABI of libtmfg.so: GB300 (sm_103a) TMFG construction and
 * all-pairs shortest paths over the TMFG, after Raphael & Shun, "Faster
 * Parallel Triangular Maximally Filtered Graphs and Hierarchical Clustering"
 * (arXiv 2408.09399).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller (for example
 *    torch tensors on the context's device).  The library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are stream-ordered and asynchronous: they enqueue work
 *    and return.
 *  - The library allocates device memory only inside a tmfg_ctx (its
 *    workspace), never more than the budget given to tmfg_create.  A context
 *    may be used by one stream at a time.
 *  - Argument errors are returned at once.  Errors found in the data (NaN,
 *    |S| too large, asymmetry) are found on the device, recorded in the
 *    context's status word, and returned by tmfg_sync_status.  Kernels that
 *    run after a recorded error skip their work.
 *  - No C++ exception crosses this interface; there is no CPU fallback.
 *
 * Matrix layout: S is n x n, row-major, with leading dimension ld >= n
 * (elements), float (TMFG_F32) or double (TMFG_F64); the diagonal is never
 * read for arithmetic; -0.0 and +0.0 are the same value.  Off-diagonal
 * entries must be finite with |S| <= 64 (row sums are exact int64 sums of
 * S*2^40).  Vertex ids are 0..n-1.
 */
#ifndef TMFG_H
#define TMFG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
    TMFG_OK = 0,
    TMFG_EINVAL = 1,      /* bad argument (n < 4, ld < n, HEAP with prefix != 1, ...) */
    TMFG_ENOMEM = 2,      /* workspace budget or device memory exhausted */
    TMFG_ENONFINITE = 3,  /* S holds a NaN or an infinity off the diagonal */
    TMFG_EASYMMETRIC = 4, /* S[i,j] != S[j,i] (only with TMFG_CHECK_SYMMETRY) */
    TMFG_ETIMEOUT = 5,    /* a device loop reached its time limit and stopped */
    TMFG_ECUDA = 6,       /* a CUDA runtime call failed */
    TMFG_ERANGE = 7,      /* an off-diagonal |S| > 64 */
    TMFG_ETOOBIG = 8,     /* n above what this build supports for the dtype */
    TMFG_EINTERNAL = 9    /* an internal consistency check failed */
};

enum { TMFG_F32 = 0, TMFG_F64 = 1 };
enum { TMFG_CORR = 0, TMFG_HEAP = 1 };

/* tmfg_params.flags */
#define TMFG_CHECK_SYMMETRY 1u /* verify S == S^T (bitwise, -0 == +0) first */

typedef struct tmfg_ctx tmfg_ctx;

/* Create a context on CUDA device `device` whose workspace may grow to
 * `workspace_budget_bytes` (0 = no limit beyond free memory).  The context
 * holds the device status word and the workspace.  Returns TMFG_OK and sets
 * *out, or an error code (then *out is NULL). */
int tmfg_create(tmfg_ctx **out, int device, size_t workspace_budget_bytes);

/* Release the context's device memory.  Synchronises the device first. */
void tmfg_destroy(tmfg_ctx *ctx);

/* Largest n that tmfg_build supports for `dtype` in this build with
 * corr-tmfg and prefix 1 (the sorted rows, the loop's per-vertex state and
 * one APSP distance row each fit one CTA's shared memory; face ids are 16
 * bits). */
int64_t tmfg_max_n(int dtype);

/* The same for a given mode and prefix: heap-tmfg and prefixes above 1 keep
 * more per-vertex state in shared memory and stop at a smaller n. */
int64_t tmfg_max_n_mode(int dtype, int mode, int prefix);

/* Workspace bytes that tmfg_build (what = 0), tmfg_apsp exact (what = 1)
 * or approximate (what = 2, with n_hubs = 0 meaning ceil(sqrt n)), or
 * dbht_cluster (what = 3) needs. */
size_t tmfg_workspace_bytes(int64_t n, int dtype, int what, int n_hubs);

typedef struct {
    int32_t mode;   /* TMFG_CORR (Algorithm 1) or TMFG_HEAP (Algorithm 2) */
    int32_t prefix; /* prefix size P >= 1 for TMFG_CORR; must be 1 for TMFG_HEAP */
    int32_t dtype;  /* TMFG_F32 or TMFG_F64: element type of S */
    uint32_t flags; /* TMFG_CHECK_SYMMETRY or 0 */
} tmfg_params;

/* TMFG construction (Section 4.1, Algorithm 1 "corr-tmfg" and Section 4.2,
 * Algorithm 2 "heap-tmfg"; lazily advanced sorted-row pointers of Section
 * 4.3).  One up-front sort of every row of S, the initial 4-clique of the
 * largest row sums, then n-4 greedy insertions of a vertex into a face.
 *
 * Outputs (device, int32, caller-owned):
 *   order[n]            order[0..3] = the initial clique v1..v4 (row-sum
 *                       rank order), order[4+k] = the k-th inserted vertex.
 *   edges[(3n-6)*2]     the 6 clique edges (v1,v2),(v1,v3),(v1,v4),(v2,v3),
 *                       (v2,v4),(v3,v4), then (v,x),(v,y),(v,z) for each
 *                       insertion of v into face x<y<z.
 *   ins_face[(n-4)*3]   the face x<y<z used by each insertion.
 *   bubble_parent[n-3]  bubble tree: bubble 0 is the clique (parent -1);
 *                       bubble k>=1 is insertion k-1; its parent is the
 *                       bubble that created the face it used.
 * Ties: a face's best vertex is the candidate of largest gain, then smallest
 * id; pairs rank by (gain desc, vertex asc, face id asc).  The result is
 * deterministic and does not depend on the GPU or the launch. */
int tmfg_build(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, const tmfg_params *params,
               int32_t *order, int32_t *edges, int32_t *ins_face, int32_t *bubble_parent,
               void *stream);

/* The per-row sort step alone (Algorithm 1, sort loop), for inspection and
 * tests: idx[v*ldi + j] (uint16, ldi >= n-1) = the j-th vertex of row v
 * sorted by (S[v,u] desc, u asc) over u != v; rowsum[v] (int64, may be
 * NULL) = sum over u != v of S[v,u]*2^40 rounded to nearest-even.  n must be
 * <= tmfg_max_n(dtype). */
int tmfg_row_sort(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                  uint16_t *idx, int64_t ldi, int64_t *rowsum, void *stream);

typedef struct {
    int32_t approx;      /* 0: exact APSP; 1: hub-based approximate APSP */
    int32_t n_hubs;      /* approximate only; 0 = ceil(sqrt(n)) */
    float radius_factor; /* approximate only; 0 = 2.0 */
} tmfg_apsp_params;

/* All-pairs shortest paths over the TMFG (Section 2: the distances DBHT
 * uses; approximate form of Section 4.3).  Edge (a,b) of `edges` (3n-6 of
 * them, as written by tmfg_build) has length sqrt(max(0, 2(1 - S[a,b])))
 * computed in the dtype of S and rounded to float.  D[s*ldd + t] (float,
 * ldd >= n) = the smallest left-to-right float sum of the lengths along a
 * path from s to t.  Approximate: hubs = the n_hubs vertices of largest
 * degree (ties to the smaller id); for each vertex s, d_s = distance to its
 * nearest hub h(s) (ties to the lower hub rank) and r_s = radius_factor*d_s;
 * D[s,t] = min(d_s + D(h(s),t), d_t + D(h(t),s), and the exact distance if
 * it is <= r_s or <= r_t).  The approximate D is exactly symmetric. */
int tmfg_apsp(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
              const int32_t *edges, const tmfg_apsp_params *params, float *D, int64_t ldd,
              void *stream);

/* One instance of a batched run (all pointers device, caller-owned). */
typedef struct {
    const void *S;          /* n x n similarity matrix, leading dimension ld */
    int64_t n, ld;
    int32_t *order;         /* [n]        as for tmfg_build */
    int32_t *edges;         /* [(3n-6)*2] */
    int32_t *ins_face;      /* [(n-4)*3]  (may be NULL when n == 4) */
    int32_t *bubble_parent; /* [n-3] */
    float *D;               /* exact APSP output (n x n, ldd), or NULL to skip */
    int64_t ldd;
} tmfg_job;

/* Launch shape of the insertion loop of corr-tmfg with prefix 1 (no paper
 * counterpart: a tuning knob); 0 fields take the defaults.  Every shape gives
 * the same TMFG. */
typedef struct {
    int32_t threads;       /* threads of the loop's CTA: 256 (default) or 512 */
    int32_t probe_lanes;   /* lanes per sorted-row refresh: 4, 8 (default) or 16;
                              with 512 threads 8 or 16; the cluster kernel:
                              8, 16 or 32 (default) */
    int32_t stage_groups;  /* index groups of 32 face keys a round copies to
                              shared memory (default 128; fewer if they do not fit;
                              -1 = none) */
    int32_t kernel;        /* 0 = automatic (default: corr-tmfg with prefix 1
                              takes the cluster kernel with 16 CTAs and 32 lanes
                              in single builds with n >= 256 where the device
                              can place it, else the prefix-1 kernel; every
                              other mode the general kernel), 1 = the prefix-1
                              loop kernel, 2 = the
                              general loop kernel that every mode runs, 3 = the
                              cluster kernel (one build on a thread-block
                              cluster of `cluster` SMs; single builds with
                              n <= 32770 only: TMFG_EINVAL in a batch,
                              TMFG_ETOOBIG above that n) */
    int32_t cluster;       /* CTAs (SMs) of the cluster kernel: 8 (default) or 16 */
} tmfg_loop_shape;

/* Stage times (ms from the start of the call, on the device clock) of the
 * last tmfg_solve_host on this context, after waiting for it: [0] start,
 * [1] every block of S uploaded, [2] TMFG built, [3..6] the four pieces of
 * the exact distances downloaded, [7] the approximate distances downloaded;
 * -1 for a stage the call did not have.  count <= 8 entries are written. */
int tmfg_solve_host_stages(tmfg_ctx *ctx, float *ms, int32_t count);

/* Set the loop shape that later tmfg_build and tmfg_solve_host calls on this
 * context use (NULL = defaults).  TMFG_EINVAL for an unsupported shape. */
int tmfg_set_loop_shape(tmfg_ctx *ctx, const tmfg_loop_shape *shape);

/* Launch shapes of a batched run; 0 fields take the defaults.  Chosen by an
 * autotuner on the Python side (paper_2408_09399_gb300.autotune). */
typedef struct {
    int32_t sssp_threads;   /* threads per search CTA: 256 or 512 (default) */
    tmfg_loop_shape loop;   /* the loop's shape (corr-tmfg, prefix 1) */
} tmfg_batch_config;

/* Many TMFG constructions (and optionally exact APSPs) in one launch per
 * stage: one persistent grid sorts the rows of every matrix, one CTA per
 * instance runs its insertion loop, and one persistent grid runs every
 * (instance, source) search.  Every instance gets exactly the result
 * tmfg_build (and tmfg_apsp) gives it alone.  `jobs` is a HOST array of
 * `count` descriptors; all instances share `params` (same dtype and mode);
 * each n must satisfy 4 <= n <= tmfg_max_n(dtype).  Asynchronous; the
 * descriptors are copied through the context's pinned staging buffer, so
 * the host array may be reused once the call returns.  The loop runs in one
 * segment per instance (no row compaction), which suits small instances.
 * The call may be captured into a CUDA graph once the same batch has run
 * uncaptured on the context (nothing is allocated or awaited under capture;
 * TMFG_ENOMEM if it would have to); the captured descriptor copy reads the
 * context's staging buffer at each replay, so a context that serves a
 * captured graph must not run other batches in between. */
int tmfg_batch_run(tmfg_ctx *ctx, const tmfg_job *jobs, int32_t count, const tmfg_params *params,
                   const tmfg_batch_config *cfg, void *stream);

/* Largest n accepted by dbht_cluster (its bubble-tree pass keeps 10 bytes
 * per bubble in one CTA's shared memory). */
#define DBHT_MAX_N 23247

/* Optional per-vertex and per-bubble results of dbht_cluster_detail (device
 * pointers, each may be NULL). */
typedef struct {
    int32_t *direction;  /* [n-4] bubble-tree edge k = 1..n-4 (entry k-1):
                            1 = points from parent(k) into bubble k's side */
    int32_t *converging; /* [n-3] 1 = bubble has no outgoing edge */
    int32_t *group;      /* [n] converging bubble of each vertex */
    int32_t *bubble;     /* [n] bubble of each vertex */
} dbht_outputs;

/* DBHT dendrogram (Section 2, "PMFG, TMFG, and DBHT": directed bubble tree,
 * converging bubbles, vertex assignment, complete linkage inside bubbles,
 * then within groups, then across groups) from a TMFG written by tmfg_build
 * and its distances written by tmfg_apsp.  The paper sketches DBHT without
 * fixing its rules; the reading implemented (identically by the test
 * oracle) is:
 *  - bubble 0 = the initial clique order[0..3]; bubble k >= 1 = {order[k+3]}
 *    plus the face ins_face[k-1]; the bubble-tree edge (bubble_parent[k], k)
 *    crosses that face t_k;
 *  - edge k points toward bubble k's side iff the sum of q(S[a,b]) over the
 *    TMFG edges (a,b) with a in t_k and b inside exceeds the sum over those
 *    with b outside, where inside = vertices introduced by bubbles of k's
 *    subtree and q(x) = x*2^40 rounded to the nearest integer, ties to even
 *    (exact int64 sums); otherwise (ties too) it points to the parent;
 *  - converging bubbles have no outgoing edge.  A vertex's group is the
 *    converging bubble of least mean D to its 4 vertices; a non-converging
 *    bubble's home is the converging bubble of least mean D over the 16
 *    vertex pairs; a vertex's bubble is the bubble of least mean D to its
 *    4 vertices among those whose home is the vertex's group.  Means are
 *    double sums in vertex order divided by 4 or 16; ties to the smaller
 *    bubble id;
 *  - complete linkage over D inside each (group, bubble) cell (bubbles in
 *    id order), then over the cells of each group (groups in converging
 *    bubble order), then over the groups; each merge takes the pair of least
 *    complete-linkage distance, ties to the pair whose (smaller, larger)
 *    least leaf ids are lexicographically smallest.
 * D is read as D[min(i,j)*ldd + max(i,j)] and must hold non-negative,
 * non-NaN floats (as tmfg_apsp writes them).  linkage: (n-1) x 4 doubles in
 * the scipy layout (id_lo, id_hi, height, size; leaves 0..n-1, merge r
 * creates cluster n + r).  Order/edges/face/parent indices are checked on
 * the device (TMFG_EINVAL in the status word if out of range or if order is
 * not a permutation).  Workspace: tmfg_workspace_bytes(n, dtype, 3, 0)
 * (about 4 n^2 bytes).  TMFG_ETOOBIG for n > DBHT_MAX_N. */
int dbht_cluster(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                 const int32_t *order, const int32_t *edges, const int32_t *ins_face,
                 const int32_t *bubble_parent, const float *D, int64_t ldd, double *linkage,
                 void *stream);

/* dbht_cluster that also writes the intermediate results named in `out`
 * (NULL: none). */
int dbht_cluster_detail(tmfg_ctx *ctx, const void *S, int64_t n, int64_t ld, int32_t dtype,
                        const int32_t *order, const int32_t *edges, const int32_t *ins_face,
                        const int32_t *bubble_parent, const float *D, int64_t ldd,
                        double *linkage, const dbht_outputs *out, void *stream);

/* Options of tmfg_solve_host; 0 fields take the defaults. */
typedef struct {
    int32_t n_hubs;       /* approximate APSP: 0 = ceil(sqrt(n)) */
    float radius_factor;  /* approximate APSP: 0 = 2.0 */
    int32_t row_blocks;   /* S is moved and sorted in this many row blocks; 0 = 8, at most 32 */
} tmfg_solve_params;

/* The whole step from HOST memory: S (host, n x n, leading dimension ld)
 * is copied to the device in row blocks, each block's rows sorted as soon as
 * it has arrived (Algorithm 1's sort overlaps the transfer); then the
 * insertion loop; then the approximate APSP (into D_approx) and the exact
 * APSP (into D_exact, in four pieces of sources), each optional (NULL skips
 * it), with leading dimension ldd.  The TMFG (order, edges, ins_face,
 * bubble_parent) and the distances are written to HOST memory, each copied
 * back while the next stage computes (a second, internal stream carries the
 * copies).  Results
 * are those of tmfg_build and tmfg_apsp.  Asynchronous and ordered on
 * `stream` like every call: the host buffers are complete once the stream
 * has reached the end of the call (tmfg_sync_status).  Host buffers should
 * be page-locked (cudaHostAlloc or cudaHostRegister) for the copies to
 * overlap; other host memory works but serialises them.  The device copies
 * live in a second context block of about n*n*(4 + 4 + 4) bytes, within the
 * context budget. */
int tmfg_solve_host(tmfg_ctx *ctx, const void *S_host, int64_t n, int64_t ld,
                    const tmfg_params *params, const tmfg_solve_params *sp, int32_t *order,
                    int32_t *edges, int32_t *ins_face, int32_t *bubble_parent, float *D_exact,
                    float *D_approx, int64_t ldd, void *stream);

/* Precision of tmfg_similarity. */
enum { TMFG_SIM_F64 = 0, TMFG_SIM_F32 = 1, TMFG_SIM_BF16X3 = 2, TMFG_SIM_TF32X3 = 3 };

/* Pearson similarity matrix of n series (the input of the method, Section 5
 * "Datasets": the Pearson correlation of every pair of time series).
 *   X: n x T float32, row-major, contiguous (series i = X[i*T .. i*T+T-1]).
 *   S: n x n float32 output, leading dimension ld >= n; S[i,j] = rho_ij,
 *      exactly symmetric, diagonal exactly 1.
 * Each series is centred and scaled to unit norm in double on the device;
 * the products are then taken in the requested precision:
 *   TMFG_SIM_F64     double dot products (CUDA cores; the accurate reference);
 *   TMFG_SIM_F32     float dot products of the float-rounded series;
 *   TMFG_SIM_BF16X3  y = hi + lo with bf16 halves, rho = hi.hi + hi.lo + lo.hi
 *                    on the tensor cores (tcgen05, FP32 accumulation);
 *   TMFG_SIM_TF32X3  the same with TF32 halves.
 * A series that is constant or holds a NaN/infinity has no correlation:
 * TMFG_ENONFINITE is recorded in the status word.  Workspace: about
 * n*T*4 bytes (n*T*8 for F64 and TF32X3). */
int tmfg_similarity(tmfg_ctx *ctx, const float *X, int64_t n, int64_t T, int32_t precision,
                    float *S, int64_t ld, void *stream);

/* ------------------------------------------------------------ pipeline
 * The whole clustering of many instances from their raw series (no
 * counterpart in the paper: the request shape of a clustering service).
 * For every job, in stream order: the Pearson similarity of its series into
 * S (tmfg_similarity at `precision`); then the TMFG and exact APSP of all
 * jobs through tmfg_batch_run (one launch per stage for all of them); then
 * each job's DBHT dendrogram into Z (dbht_cluster) and, when k > 0, its cut
 * at k clusters into labels (tmfg_cut_labels).  Every job gets exactly what
 * those calls give it alone.  All pointers are caller-owned device memory. */
typedef struct {
    const float *X;         /* n x T series, row-major, row stride ldx >= T */
    int64_t n, T, ldx;
    float *S;               /* n x n similarity (written; ld = n) */
    int32_t *order;         /* [n] */
    int32_t *edges;         /* [(3n-6)*2] */
    int32_t *ins_face;      /* [(n-4)*3] (may be NULL when n == 4) */
    int32_t *bubble_parent; /* [n-3] */
    float *D;               /* n x n exact APSP (written; ldd = n) */
    double *Z;              /* (n-1) x 4 linkage, scipy layout (written) */
    int32_t k;              /* clusters of the cut; 0 = no cut */
    int32_t *labels;        /* [n] cluster of each series at k (k > 0) */
} tmfg_pipeline_job;

typedef struct {
    int32_t precision;      /* TMFG_SIM_* of the similarity */
    tmfg_params tmfg;       /* TMFG parameters (dtype must be TMFG_F32) */
} tmfg_pipeline_params;

/* Run the pipeline over `count` jobs (a HOST array of descriptors).
 * TMFG_ETOOBIG if an n exceeds DBHT_MAX_N or tmfg_max_n_mode; data errors
 * go to the status word (tmfg_sync_status).  Asynchronous. */
int tmfg_pipeline_run(tmfg_ctx *ctx, const tmfg_pipeline_job *jobs, int32_t count,
                      const tmfg_pipeline_params *params, const tmfg_batch_config *cfg,
                      void *stream);

/* Workspace one pipeline job of size n, length T needs in a lane. */
size_t tmfg_pipeline_request_bytes(int64_t n, int64_t T, int32_t precision);

/* Labels of the cut of a linkage Z ((n-1) x 4, device, scipy layout) at k
 * clusters (Section 5: the clusters the ARI scores): the first n - k merges
 * are applied; clusters are numbered 0..k-1 in the order of their smallest
 * member.  labels: [n] device int32.  Asynchronous. */
int tmfg_cut_labels(tmfg_ctx *ctx, const double *Z, int64_t n, int32_t k, int32_t *labels,
                    void *stream);

/* ------------------------------------------------------------ serving
 * A request server with continuous batching (no counterpart in the paper).
 * Jobs (tmfg_job, buffers resident in device memory, caller-owned) are
 * submitted one by one; a host worker thread groups the waiting jobs, first
 * come first served, into batches that run through tmfg_batch_run on one of
 * `lanes` lanes.  Each lane is a context with its own non-blocking stream and
 * a workspace of lane_bytes allocated at start, so batches on different lanes
 * overlap on the GPU and nothing is allocated while serving.  A batch takes
 * as many queued jobs as fit its lane's memory (tmfg_serve_request_bytes
 * each, plus the descriptor tables) and max_batch; a job that does not fit
 * an empty lane is refused at submission.  Every job gets exactly the result
 * tmfg_build (and tmfg_apsp, exact) give it alone, whatever it is batched
 * with.  A data error in a batch is reported for every job of that batch. */
typedef struct tmfg_server tmfg_server;

typedef struct {
    int32_t lanes;         /* concurrent batches; 0 = 3 (at most 16) */
    int32_t max_batch;     /* jobs per batch; 0 = 256 (at most 4096) */
    size_t lane_bytes;     /* workspace per lane; 0 = 4 GiB */
    tmfg_params params;    /* TMFG parameters of every job */
    int32_t apsp;          /* 1: also the exact APSP into each job's D */
    int32_t sssp_threads;  /* as in tmfg_batch_config; 0 = default */
    int32_t pipeline;      /* 1: jobs are whole pipelines (tmfg_serve_submit_pipeline,
                              run by tmfg_pipeline_run; apsp is implied) */
    int32_t precision;     /* TMFG_SIM_* of the pipelines' similarity */
} tmfg_serve_config;

typedef struct {
    int64_t id;            /* as returned by tmfg_serve_submit */
    int32_t status;        /* TMFG_OK or the error of the job's batch */
    int32_t batch;         /* sequence number of the batch that ran it */
    int32_t batch_size;    /* jobs in that batch */
    int32_t reserved;
    int64_t t_submit_ns;   /* tmfg_serve_now_ns clock: submission, */
    int64_t t_launch_ns;   /*   launch of its batch, */
    int64_t t_done_ns;     /*   completion seen by the host */
} tmfg_serve_result;

/* Start a server on `device` (creates the lanes and the worker thread). */
int tmfg_serve_start(tmfg_server **out, int device, const tmfg_serve_config *cfg);

/* Queue one job; returns its id (>= 0) or minus an error code.  The job's
 * inputs count as ready once `stream` (the submitter's cudaStream_t as
 * void*, NULL = legacy default) reaches the point of this call.  The
 * descriptor is copied; its buffers must stay valid until the job's result
 * has been polled. */
int64_t tmfg_serve_submit(tmfg_server *s, const tmfg_job *job, void *stream);

/* Queue one whole pipeline (a server started with pipeline = 1): the job
 * runs through tmfg_pipeline_run with the other jobs of its batch, and gets
 * exactly what that call gives it alone.  Admission counts
 * tmfg_pipeline_request_bytes.  Returns its id or minus an error code. */
int64_t tmfg_serve_submit_pipeline(tmfg_server *s, const tmfg_pipeline_job *job, void *stream);

/* Move up to `max` finished jobs' results into out[] (waiting up to wait_us
 * microseconds for the first); returns the count, or minus an error code.
 * A job's outputs are complete on the device when its result is returned. */
int tmfg_serve_poll(tmfg_server *s, tmfg_serve_result *out, int32_t max, int32_t wait_us);

/* Finish every submitted job, stop the worker and free the server.
 * Results not yet polled are discarded. */
int tmfg_serve_stop(tmfg_server *s);

/* The server's clock (steady, nanoseconds). */
int64_t tmfg_serve_now_ns(void);

/* Workspace bytes one job of size n needs in a lane (its admission unit). */
size_t tmfg_serve_request_bytes(int64_t n, int32_t apsp);

/* The batching rule alone, for inspection: the batch (0, 1, ...) that each
 * of `count` jobs of sizes n[] queued together would fall into when lanes
 * take them in order.  TMFG_ENOMEM if a job cannot fit an empty lane. */
int tmfg_serve_plan(const int64_t *n, int32_t count, int32_t apsp, int32_t max_batch,
                    size_t lane_bytes, int32_t *batch_of);

/* Largest n accepted by tmfg_apsp_exact_noalloc. */
#define TMFG_NOALLOC_MAX_N 21581

/* Exact APSP (same result, bit for bit, as tmfg_apsp with approx = 0) that
 * allocates no device memory and needs no tmfg_ctx.  The paper has no
 * counterpart: it is for callers that cannot call cudaMalloc -- a process
 * whose device memory is all owned by its own pool or caching allocator,
 * or a code path that must not take an allocator's locks and device
 * synchronisation.  Its scratch (about 1.3 MB: the TMFG's adjacency in CSR
 * form) is one static device array inside libtmfg.so, which every GPU that
 * loads the library holds until the process exits.
 *   S, n, ld, dtype, edges, D, ldd: as for tmfg_apsp.
 *   status: caller-owned device int32; the call sets it to 0 and the
 *           kernels record the first data error in it (read it after the
 *           stream reaches this call).
 * Runs on the current CUDA device, in the context current on the calling
 * thread: every call looks up the scratch array's device address in that
 * context (so a device reset or another current context is handled); the
 * first call on a device also reads its SM count.  Make the first call on
 * a device before any stream capture.  Device loops stop after the time
 * limit that tmfg_create uses (60 s, or TMFG_TIMEOUT_MS milliseconds from
 * the environment).  All calls share the one array and it keeps the last call's
 * contents (the call clears what must start at zero): calls whose kernels
 * overlap on the GPU, on different streams or threads, race and corrupt
 * each other's results -- order them on one stream.
 * Returns TMFG_ETOOBIG for n > TMFG_NOALLOC_MAX_N, TMFG_EINVAL for bad
 * arguments, TMFG_ECUDA if the set-up or a launch fails. */
int tmfg_apsp_exact_noalloc(const void *S, int64_t n, int64_t ld, int32_t dtype,
                            const int32_t *edges, float *D, int64_t ldd, int32_t *status,
                            void *stream);

/* Synchronise `stream`, then return the status word recorded by the
 * context's kernels since the last call (TMFG_OK if none) and clear it. */
int tmfg_sync_status(tmfg_ctx *ctx, void *stream);

/* Counters of the last tmfg_build, valid after tmfg_sync_status:
 * out[0] = face evaluations, out[1] = stale heap pops, out[2] = pointer
 * scan chunks loaded, out[3] = insertion rounds, out[4] = loop time in ns
 * (device clock), out[5..7] = SM cycles spent recomputing faces, updating
 * the max indexes, and selecting pairs (heap: resolving the stale pops);
 * out[8..10] = a finer split of those cycles (push, refresh, gains);
 * out[11..13] = heap: cycles of extraction, validation and resolution;
 * corr: pointer probes (64 sorted ids each), the warp refreshes that
 * followed a probe that found nothing, and their 256-id steps; out[14] =
 * heap: stale
 * scan cycles; out[15] = heap: epoch iterations.  `count` <= 16 entries are
 * written. */
int tmfg_last_stats(tmfg_ctx *ctx, int64_t *out, int count);

/* Latency of dependent device-memory loads (no counterpart in the paper: a
 * diagnostic for the insertion loop, whose bound is a chain of dependent
 * round trips).  Allocates a buffer of `bytes` (rounded down to a power of
 * two of 128-byte lines, at least 4096 bytes), links its lines into one
 * scattered full-period cycle, follows `warm` links untimed and then `hops`
 * links timed by the device clock, one thread with L1-bypassing loads, and
 * frees the buffer.  A buffer well inside L2 after a warm pass of one period
 * gives the L2 hit latency; a multi-gigabyte buffer, cold, gives the DRAM
 * miss latency with its address-translation misses.  Synchronous (legacy
 * default stream).  *ns_per_hop: host double.  Returns TMFG_EINVAL,
 * TMFG_ENOMEM (the buffer does not fit) or TMFG_ECUDA on failure. */
int tmfg_memory_latency(tmfg_ctx *ctx, int64_t bytes, int32_t hops, int32_t warm,
                        double *ns_per_hop);

/* Diagnostic (no paper counterpart): nanoseconds per exchange of one
 * thread-block cluster of `cluster` (8 or 16) CTAs, each exchange being what
 * the cluster loop kernel does once per insertion -- every CTA stores a
 * 16-byte record into a slot of every CTA's shared memory, then the cluster
 * passes a barrier (release / acquire) -- averaged over `iters` exchanges.
 * Synchronous (waits for the device); allocates 8 bytes of device memory.
 * TMFG_EINVAL for a bad argument, TMFG_ECUDA if the launch fails. */
int tmfg_cluster_exchange_latency(tmfg_ctx *ctx, int32_t cluster, int32_t iters,
                                  double *ns_per_exchange);

/* Static description of a return code. */
const char *tmfg_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TMFG_H */
