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
    int4 *face;                   // [2n-4] {a<b<c, owner bubble}
    unsigned long long *leaf_gk;  // [2n-4] order-preserving gain key (0 = empty)
    int *leaf_v;                  // [2n-4] stored best vertex
    int *fu_buf;                  // [2n-4] corr-mode update list
    int *status;
    long long *stats;             // [8]
    unsigned long long timeout_ns;
};
size_t loop_smem_bytes(int n);
int launch_loop(const LoopArgs &args, int dtype, cudaStream_t stream);

// apsp.cu
size_t apsp_work_bytes(int n, int approx, int h);
size_t sssp_smem_bytes(int n);
int launch_apsp(const void *S, int n, long long ld, int dtype, const int *edges, int approx,
                int h, float rf, float *D, long long ldd, void *work, int *status, int num_sms,
                unsigned long long timeout_ns, cudaStream_t stream);

constexpr size_t kSmemLimit = 232448;  // 227 KB opt-in shared memory per CTA

}  // namespace tmfg
