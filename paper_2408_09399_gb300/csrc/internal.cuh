// internal.cuh -- declarations shared by the translation units of libtmfg.
#pragma once

#include "common.cuh"

namespace tmfg {

// rowsort.cu
int64_t rowsort_max_n(int dtype);
int launch_rowsort(const void *S, int n, long long ld, int dtype, uint16_t *idx, long long ldi,
                   long long *rowsum, int *status, int num_sms, cudaStream_t stream);

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
size_t loop_smem_bytes(int n, int dtype, int mode);
size_t loop_state_bytes(int n);
int launch_loop(const LoopArgs &args, int dtype, cudaStream_t stream);

// apsp.cu
size_t apsp_work_bytes(int n, int approx, int h);
size_t sssp_smem_bytes(int n);
int launch_apsp(const void *S, int n, long long ld, int dtype, const int *edges, int approx,
                int h, float rf, float *D, long long ldd, void *work, int *status, int num_sms,
                unsigned long long timeout_ns, cudaStream_t stream);

constexpr size_t kSmemLimit = 232448;  // 227 KB opt-in shared memory per CTA

}  // namespace tmfg
