// internal.cuh -- declarations shared by the translation units of libtmfg.
#pragma once

#include "common.cuh"

namespace tmfg {

// api.cu: the time limit of every device loop, 60 s unless the environment
// variable TMFG_TIMEOUT_MS gives a positive number of milliseconds
unsigned long long device_timeout_ns();

// rowsort.cu
struct SortJob {  // the rows of one matrix, for the batched sort
    const void *S;
    long long ld;
    int n;
    bool vec_in, vec_out;
    uint16_t *idx;
    long long ldi;
    long long *rowsum;
};
int64_t rowsort_max_n(int dtype);
size_t rowsort_smem(int n, int dtype);
int launch_rowsort_batch(const SortJob *d_jobs, const int *d_row_begin, int njobs, int max_n,
                         int dtype, int *status, int grid, cudaStream_t stream);
// rows [row0, row1) of the matrix (row1 < 0: to the last row)
int launch_rowsort(const void *S, int n, long long ld, int dtype, uint16_t *idx, long long ldi,
                   long long *rowsum, int *status, int num_sms, cudaStream_t stream,
                   int row0 = 0, int row1 = -1);

// tmfg_loop.cu
struct LoopArgs {
    const void *S;
    long long ld;
    int n;
    int mode;
    int P;
    const uint16_t *idx;
    long long ldi;
    const long long *rowsum;
    int *order;
    int *edges;
    int *ins_face;
    int *parent;
    int4 *face;                      // [2n-4] {a<b<c, owner bubble}
    void *leaf_fresh;                // [2n-4] 16-byte slots: face keys, FRESH index
    void *leaf_stale;                // [2n-4] 16-byte slots: face keys, STALE index (heap)
    void *pend_key;                  // [2n-4] 16-byte slots: pending recomputed keys (heap)
    unsigned long long *pend_cand;   // [2n-4] the 3 candidates a pending key used
    int *fu_buf;                     // [2n-4] face update lists
    int *status;
    long long *stats;             // [16]
    unsigned long long timeout_ns;
    void *state;                  // loop state between segments (loop_state_bytes)
    int k_stop;                   // a segment stops once k >= k_stop
    int resume;                   // 0: first segment; 1: continue from state
};
// Launch shape of the corr-tmfg prefix-1 loop kernel (loop_corr1.cu):
// threads per CTA (256 or 512), lanes per sorted-row refresh (4, 8 or 16;
// 512 threads: 8 or 16), and the index groups whose keys a round copies to
// shared memory (fewer when the shared memory does not hold them).
struct LoopShape {
    int threads = 256;
    int lanes = 8;
    int groups = 128;
    // which kernel runs corr-tmfg prefix 1: -1 automatic (single builds from
    // kClusterAutoMinN on: the cluster kernel where the device can place it;
    // otherwise the general kernel where its shared memory holds n, else the
    // prefix-1 kernel), 0 the prefix-1 kernel, 1 the general kernel, 2 the
    // cluster kernel
    int general = -1;
    int cluster = 8;          // CTAs of the cluster kernel: 8 or 16
    int cluster_lanes = 32;   // its lanes per row refresh: 8, 16 or 32
};
// LoopShape from the ABI's tmfg_loop_shape (NULL or 0 fields: defaults);
// false for an unsupported shape
bool loop_shape_from(const tmfg_loop_shape *in, LoopShape *out);
size_t loop_smem_bytes(int n, int dtype, int mode);
size_t loop_state_bytes(int n);
int launch_loop(const LoopArgs &args, int dtype, cudaStream_t stream,
                const LoopShape &shape = LoopShape{});
int launch_loop_batch(const LoopArgs *d_args, int count, int max_n, int dtype, int mode, int P,
                      cudaStream_t stream, const LoopShape &shape = LoopShape{});
// the smallest shared-memory carve-out (percent) that holds `ctas` CTAs of
// `smem` dynamic bytes each
int carveout_percent(size_t smem, int ctas);

// loop_corr1.cu
// gp: the layout whose row pointers live in global memory (large n)
size_t corr1_smem_bytes(int n, int dtype, int groups, bool gp);
// the copy groups (at most `want`) that fit `limit` bytes, or -1 if nothing fits
int corr1_fit_groups(int n, int dtype, int want, size_t limit, bool gp);
bool corr1_shape_ok(int threads, int lanes);
int launch_corr1(const LoopArgs &a, const LoopShape &shape, int dtype, size_t smem, bool gp,
                 cudaStream_t stream);
// the largest n the loop of (mode, prefix) holds, for dtype
int64_t loop_max_n(int dtype, int mode, int prefix);
int launch_corr1_batch(const LoopArgs *d_args, int count, const LoopShape &shape, int dtype,
                       size_t smem, cudaStream_t stream);

// loop_cluster.cu: corr-tmfg prefix 1 on a cluster of C CTAs (single builds)
size_t cluster_smem_bytes(int n, int dtype, int C);
// C CTAs (8 or 16), lanes per row refresh (8, 16 or 32)
bool cluster_shape_ok(int C, int lanes);
int launch_cluster_loop(const LoopArgs &a, int dtype, int C, int lanes, cudaStream_t stream);
// whether the device can run the cluster kernel of C CTAs for n
bool cluster_placeable(int n, int dtype, int C, int lanes);
// the automatic choice takes the cluster kernel (16 CTAs, a warp per row
// refresh) from this n on, where it is placeable: measured on GB300 it is at
// least as fast as the one-CTA kernels from n = 300 on (4.5 vs 5.1 ms at
// n = 1000, 51 vs 65 ms at 10000, 117 vs 194 ms at 20000)
constexpr int kClusterAutoMinN = 256;

// apsp.cu
struct SsspArgs {
    int n;
    const int *rowptr;
    const uint2 *arcs;
    const int *src;      // sources (null: source i = src0 + i)
    int src0;
    int nsrc;
    float *out;          // row i of the output = source src[i]
    long long ldo;
    // approximate form
    const float *dnear;  // [n] distance to the nearest hub
    const int *near;     // [n] rank of the nearest hub
    const float *DH;     // [h x n] exact hub rows
    float rf;            // radius factor
    int *status;
    unsigned long long timeout_ns;
};
struct ApspJob {  // one graph of a batched exact APSP
    const void *S;
    long long ld;
    int n;
    const int *edges;
    int *deg, *rowptr, *cursor;
    uint2 *arcs;
};
int launch_apsp_batch(const ApspJob *d_jobs, const SsspArgs *d_sargs, const int *d_edge_begin,
                      const int *d_src_begin, int njobs, int total_edges, int max_n, int dtype,
                      int sssp_threads, int *status, int num_sms, cudaStream_t stream);
size_t apsp_work_bytes(int n, int approx, int h);
size_t sssp_smem_bytes(int n);
int launch_apsp(const void *S, int n, long long ld, int dtype, const int *edges, int approx,
                int h, float rf, float *D, long long ldd, void *work, int *status, int num_sms,
                unsigned long long timeout_ns, cudaStream_t stream);
// The exact APSP in pieces: the CSR of the TMFG once, then the rows of the
// sources [s0, s1) (row s of D), so that finished rows can be moved while
// the next piece computes.
int launch_apsp_csr(const void *S, int n, long long ld, int dtype, const int *edges, void *work,
                    int *status, cudaStream_t stream);
int launch_apsp_exact_rows(int n, void *work, float *D, long long ldd, int s0, int s1, int *status,
                           int num_sms, unsigned long long timeout_ns, cudaStream_t stream);

constexpr size_t kSmemLimit = 232448;  // 227 KB opt-in shared memory per CTA

// similarity.cu
long long sim_ldy(int T, int prec);
size_t sim_work_bytes(int n, int T, int prec);
int launch_similarity(const float *X, int n, int T, long long ldx, int prec, float *S, long long ld,
                      void *work, int *status, unsigned long long timeout_ns, cudaStream_t stream);

// dbht.cu
size_t dbht_smem_bytes(int n);
size_t dbht_work_bytes(int n);
int launch_dbht(const void *S, int n, long long ld, int dtype, const int *order, const int *edges,
                const int *ins_face, const int *parent, const float *D, long long ldd, double *Z,
                int *direction, int *converging, int *group, int *bubble, void *work, int *status,
                int num_sms, cudaStream_t stream);

}  // namespace tmfg
