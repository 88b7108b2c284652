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
    uint32_t capacity;    // slots per block (64, or N_T in the per-type capacity mode)
    int base;             // the type this one extends (its fields first), or -1
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
    int capacity_mode = DSOA_CAPACITY_UNIFORM;

    // frozen layout
    dsoa_ctx ctx;
    uint64_t tiles = 0;              // level-1 containers of one bitmap (scan tiles)
    // per registered type: block list of its last enumeration, the occupancy
    // snapshot of each listed block, and the list length (device)
    uint32_t* R[DSOA_MAX_TYPES] = {nullptr};
    unsigned long long* Rocc[DSOA_MAX_TYPES] = {nullptr};
    uint32_t* r_dev[DSOA_MAX_TYPES] = {nullptr};
    uint32_t* tile_cnt = nullptr;    // [tiles]
    uint32_t* tile_off = nullptr;    // [tiles]
    uint32_t* done = nullptr;        // last-CTA ticket of the tile-count kernel
    unsigned long long* scratch64 = nullptr;  // [16] reductions for synchronous queries
    uint64_t meta_bytes = 0;

    // launch shapes
    int doall_tpb = 256;
    int doall_ctas_per_sm = 8;
    int doall_waves = 4;             // generic do-all grid = resident CTAs x waves
    int slots_per_thread = 1;        // generic do-all: 1 (64 threads/block) or 2 (a warp/block);
                                     // vectorised microbench kernel: 1, 2 or 4
    int vec_slots_per_thread = 4;    // vectorised kernels: slots per thread (1, 2 or 4)
    int scan_tiles_per_cta = 0;      // 0 = single-pass look-back; 1, 2 = tile-count + compaction kernels
    bool stream_enum = false;        // enumerate inside methods that create no objects of their own type
    bool cluster_enum = false;       // enumerate with a thread-block cluster per type (heaps up to 4 M blocks)
    uint32_t* stream_ctl = nullptr;  // ticket, finished CTAs, R length of the streamed do-all
    unsigned long long* count_acc = nullptr;  // [DSOA_MAX_TYPES] partial counts of k_count_many (zero between launches)
    uint32_t* count_ticket = nullptr;         // finished CTAs of k_count_many (zero between launches)
    unsigned long long* lb_state = nullptr;  // [ntypes][tiles] look-back state words (epoch, status, value)
    uint32_t* lb_ctl = nullptr;              // [ntypes][4]: ticket, done counter, epoch of the look-back kernel
    int lb_fits = -1;                        // look-back CTAs resident per SM (-1: not queried yet)

    uint32_t flags = 0;              // DSOA_FLAG_* applied to every launch
    uint32_t lookups = DSOA_LOOKUP_ATTEMPTS;  // r: active-block lookups before the slow path
    uint32_t launch_seq = 0;
    uint64_t launches = 0;
    bool enumerated[DSOA_MAX_TYPES] = {false};  // R[t] holds an enumeration of type t
    bool skip_enumeration = false;   // set by dsoa_parallel_do_enumerated
    bool skip_prologue = false;      // launches after the first of a family's do-all
};

struct dsoa_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// ---- helpers implemented in heap.cu ----
int dsoa_resident_ctas(const void* kernel, int tpb);   // CTAs of `kernel` per SM (cached)
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
int dsoa_micro_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_gol_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb);
int dsoa_gol_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_gol_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_wator_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_wator_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_traffic_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);
int dsoa_traffic_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb);
int dsoa_nbody_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb);
int dsoa_nbody_do(dsoa_heap* h, int type, int method, const void* a, size_t nb);

#define DSOA_CUDA_TRY(expr)                              \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return DSOA_ERR_CUDA;     \
    } while (0)

// Persistent grid of `kernel`: CTAs per SM = min(requested, resident), so that
// the whole grid is one resident wave (no tail of late CTAs).
template <typename K>
unsigned dsoa_persistent_grid(dsoa_heap* h, K* kernel, int tpb) {
    int per_sm = dsoa_resident_ctas(reinterpret_cast<const void*>(kernel), tpb);
    if (per_sm > h->doall_ctas_per_sm) per_sm = h->doall_ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    return (unsigned)(per_sm * h->num_sms);
}

// Grid of the generic (method) do-all: `doall_waves` times the resident grid.
// Methods differ in work per object (allocation, conflicts), so with one
// resident wave the slowest warps set the kernel's duration; several waves let
// the CTA scheduler hand the remaining work to SMs that finished early.
template <typename K>
unsigned dsoa_doall_grid(dsoa_heap* h, K* kernel, int tpb) {
    return dsoa_persistent_grid(h, kernel, tpb) * (unsigned)h->doall_waves;
}

// Launch of a step kernel on the heap's stream; with DSOA_FLAG_PDL it carries
// the programmatic-serialization attribute (the kernel calls dsoa_pdl_wait()
// before touching global memory).  Counts the launch; DSOA_ERR_CUDA on failure.
template <typename... KArgs, typename... Args>
int dsoa_launch_step(dsoa_heap* h, void (*kernel)(KArgs...), unsigned grid, unsigned tpb, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tpb);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = (h->flags & DSOA_FLAG_PDL) ? 1u : 0u;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    h->launches++;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DSOA_ERR_CUDA;
    }
    return DSOA_OK;
}

// Cooperative launch (every CTA co-resident) of a kernel that uses grid barriers.
template <typename... KArgs, typename... Args>
cudaError_t dsoa_launch_cooperative(void (*kernel)(KArgs...), unsigned grid, unsigned tpb, cudaStream_t s,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(tpb);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Fused enumeration + do-all of method M in one cooperative persistent launch.
template <class M, int G>
int dsoa_run_doall_fused(dsoa_heap* h, int type, const typename M::Args& args) {
    const int tpb = h->doall_tpb;
    auto* k = &dsoa_doall_fused_kernel<M, G>;
    unsigned grid = dsoa_persistent_grid(h, k, tpb);
    if (grid > DSOA_FUSED_MAX_CTAS) grid = DSOA_FUSED_MAX_CTAS;
    /* barrier counter and generation start from zero (a launch whose barrier
     * wait gave up leaves them mid-generation) */
    if (cudaMemsetAsync(h->ctx.grid_scratch + DSOA_FUSED_MAX_CTAS, 0, 2 * sizeof(uint32_t), h->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return DSOA_ERR_CUDA;
    }
    const cudaError_t e = dsoa_launch_cooperative(k, grid, (unsigned)tpb, h->stream, dsoa_launch_ctx(h),
                                                  (uint32_t)type, h->R[type], h->Rocc[type], h->r_dev[type], args);
    h->launches++;
    if (e != cudaSuccess) { cudaGetLastError(); return DSOA_ERR_CUDA; }
    h->enumerated[type] = true;
    return DSOA_OK;
}

// Launch a do-all of method M over `type` (enumeration + persistent kernel).
template <class M>
int dsoa_run_doall(dsoa_heap* h, int type, const typename M::Args& args) {
    if (!h->skip_enumeration && (h->flags & DSOA_FLAG_FUSED)) {
        if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
        if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
        return h->slots_per_thread >= 2 ? dsoa_run_doall_fused<M, 2>(h, type, args)
                                        : dsoa_run_doall_fused<M, 1>(h, type, args);
    }
    if constexpr (dsoa_streamable<M>::value) {
        if (!h->skip_enumeration && h->stream_enum) {
            if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
            if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
            const int tpb = h->doall_tpb;
            if (h->slots_per_thread >= 2) {
                auto* k = &dsoa_doall_stream_kernel<M, 2>;
                k<<<dsoa_persistent_grid(h, k, tpb), tpb, 0, h->stream>>>(
                    dsoa_launch_ctx(h), (uint32_t)type, h->R[type], h->Rocc[type], h->r_dev[type], h->stream_ctl,
                    args);
            } else {
                auto* k = &dsoa_doall_stream_kernel<M, 1>;
                k<<<dsoa_persistent_grid(h, k, tpb), tpb, 0, h->stream>>>(
                    dsoa_launch_ctx(h), (uint32_t)type, h->R[type], h->Rocc[type], h->r_dev[type], h->stream_ctl,
                    args);
            }
            const int rc = dsoa_check_launch(h);
            if (rc == DSOA_OK) h->enumerated[type] = true;
            return rc;
        }
    }
    int rc = dsoa_prepare_doall(h, type);
    if (rc) return rc;
    const int tpb = h->doall_tpb;
    const uint32_t* R = h->R[type];
    const unsigned long long* occ = h->Rocc[type];
    const uint32_t* r = h->r_dev[type];
    if (h->slots_per_thread >= 2) {
        auto* k = &dsoa_doall_kernel<M, 2>;
        return dsoa_launch_step(h, k, dsoa_doall_grid(h, k, tpb), (unsigned)tpb, dsoa_launch_ctx(h), (uint32_t)type,
                                R, occ, r, args);
    }
    auto* k = &dsoa_doall_kernel<M, 1>;
    return dsoa_launch_step(h, k, dsoa_doall_grid(h, k, tpb), (unsigned)tpb, dsoa_launch_ctx(h), (uint32_t)type,
                            R, occ, r, args);
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
