// dsoa_internal.cuh -- host-side heap object and launch helpers shared by the
// library's translation units (not installed; user code uses dsoa.h and
// dsoa_device.cuh).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>

#include "dsoa.h"
#include "dsoa_apps.h"
#include "dsoa_device.cuh"

struct dsoa_type_info {
    int nfields;
    uint32_t field_bytes[DSOA_MAX_FIELDS];
    uint32_t col_off[DSOA_MAX_FIELDS];
    uint32_t data_bytes;  // 64-slot data segment of this type
};

struct dsoa_heap {
    // configuration
    void* base = nullptr;
    size_t bytes = 0;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int ntypes = 0;
    dsoa_type_info types[DSOA_MAX_TYPES];
    bool frozen = false;

    // frozen layout
    dsoa_ctx ctx;
    uint64_t tiles = 0;              // level-1 containers of one bitmap (scan tiles)
    uint32_t* R = nullptr;           // [M] compacted block list
    unsigned long long* Rocc = nullptr;  // [M] occupied-slot snapshot per R entry
    uint32_t* r_dev = nullptr;       // number of valid R entries
    uint32_t* tile_cnt = nullptr;    // [tiles]
    uint32_t* tile_off = nullptr;    // [tiles]
    uint32_t* done = nullptr;        // last-CTA ticket of the tile-count kernel
    unsigned long long* scratch64 = nullptr;  // [16] reductions for synchronous queries
    uint64_t meta_bytes = 0;

    // launch shapes
    int doall_tpb = 256;
    int doall_ctas_per_sm = 8;
    int slots_per_thread = 1;        // generic do-all: 1 (64 threads/block) or 2 (a warp/block);
                                     // vectorised microbench kernel: 1, 2 or 4
    int vec_slots_per_thread = 4;    // vectorised kernels: slots per thread (1, 2 or 4)
    int scan_tiles_per_cta = 1;

    uint32_t launch_seq = 0;
    uint64_t launches = 0;
    int enumerated_type = -1;        // type of the block list currently in R
    bool skip_enumeration = false;   // set by dsoa_parallel_do_enumerated
};

struct dsoa_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// ---- helpers implemented in heap.cu ----
int dsoa_ensure_frozen(dsoa_heap* h);
int dsoa_check_launch(dsoa_heap* h);                 // after a kernel launch
dsoa_ctx dsoa_launch_ctx(dsoa_heap* h);              // ctx with a fresh rotation seed
int dsoa_enumerate_internal(dsoa_heap* h, int type); // scan + compaction into R / Rocc
int dsoa_prepare_doall(dsoa_heap* h, int type);      // enumerate unless told to reuse R
unsigned dsoa_doall_grid(dsoa_heap* h);              // persistent do-all grid
unsigned dsoa_new_grid(dsoa_heap* h, uint64_t n, int tpb);

// ---- per-application dispatchers (return DSOA_ERR_UNKNOWN_METHOD if not theirs) ----
int dsoa_micro_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb);
int dsoa_micro_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_gol_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb);
int dsoa_gol_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_gol_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_wator_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_wator_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_traffic_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_traffic_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);

#define DSOA_CUDA_TRY(expr)                              \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return DSOA_ERR_CUDA;     \
    } while (0)

// Launch a do-all of method M over `type` (enumeration + persistent kernel).
template <class M>
int dsoa_run_doall(dsoa_heap* h, int type, const typename M::Args& args) {
    int rc = dsoa_prepare_doall(h, type);
    if (rc) return rc;
    if (h->slots_per_thread >= 2)
        dsoa_doall_kernel<M, 2><<<dsoa_doall_grid(h), h->doall_tpb, 0, h->stream>>>(
            dsoa_launch_ctx(h), (uint32_t)type, h->R, h->Rocc, h->r_dev, args);
    else
        dsoa_doall_kernel<M, 1><<<dsoa_doall_grid(h), h->doall_tpb, 0, h->stream>>>(
            dsoa_launch_ctx(h), (uint32_t)type, h->R, h->Rocc, h->r_dev, args);
    return dsoa_check_launch(h);
}

// parallel_new kernel: logical thread i allocates one object and constructs it.
template <class C>
__global__ void dsoa_new_kernel(dsoa_ctx c, uint32_t t, uint64_t n, typename C::Args a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const dsoa_obj o = dsoa_new(c, t);
        if (o) C::ctor(c, o, i, a);
    }
}

template <class C>
int dsoa_run_new(dsoa_heap* h, int type, uint64_t n, const typename C::Args& args) {
    if (n == 0) return DSOA_OK;
    const int tpb = 256;
    dsoa_new_kernel<C><<<dsoa_new_grid(h, n, tpb), tpb, 0, h->stream>>>(dsoa_launch_ctx(h),
                                                                      (uint32_t)type, n, args);
    return dsoa_check_launch(h);
}

template <class A>
int dsoa_copy_args(A* dst, const void* src, size_t nb) {
    if (nb != sizeof(A) || src == nullptr) return DSOA_ERR_INVALID_ARG;
    std::memcpy(dst, src, sizeof(A));
    return DSOA_OK;
}
