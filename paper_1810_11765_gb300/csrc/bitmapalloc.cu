// bitmapalloc.cu -- BitmapAlloc, the paper's second allocator (Sec. 6,
// "BitmapAlloc"): the whole heap is ONE array of equal-size object records in
// array-of-structures layout (no blocks, no SOA columns, no fake pointers),
// whose slots are managed by hierarchical bitmaps: one free-slot bitmap and
// one allocation bitmap per type.  The allocation bitmaps also drive the
// do-all.  It isolates the cost of pure bitmap allocation from DynaSOAr's
// block structure and SOA layout; its drawback is internal fragmentation (one
// record size for every type).
//
// The bitmaps are the library's hierarchical bitmaps (Sec. 4.1: rotated
// top-down try_find_set, clear/set with propagation) over object slots instead
// of blocks: bitmap 0 = free slots, 1 + 2t = allocated slots of type t,
// 2 + 2t = the iteration snapshot of type t taken at the start of a do-all.
//
//   new     take a set bit of the free bitmap (find + try-clear, bounded
//           retries), set it in allocated[t], run the constructor on the record
//   delete  clear the bit in allocated[t], then set it in the free bitmap
//   do-all  copy allocated[t] to the snapshot, then one thread per snapshot
//           bit of each level-0 word runs the method on its record
//
// Built-in constructors / methods: the microbench's (dsoa_apps.h ids 100-107),
// with the same semantics as on the DynaSOAr heap.
#include <algorithm>
#include <new>

#include "dsoa_internal.cuh"
#include "rng.cuh"

struct dsoa_bitmap_heap {
    void* base = nullptr;
    size_t bytes = 0;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int ntypes = 0;
    int nfields[DSOA_MAX_TYPES] = {0};
    uint32_t field_bytes[DSOA_MAX_TYPES][DSOA_MAX_FIELDS] = {{0}};
    uint32_t field_off[DSOA_MAX_TYPES][DSOA_MAX_FIELDS] = {{0}};  // byte offset inside a record
    uint32_t rec_bytes = 0;
    bool frozen = false;
    dsoa_ctx ctx;                       // bitmaps over object slots; ctx.M = slots, data = records
    unsigned long long* scratch = nullptr;  // [8] reductions of synchronous queries
    uint32_t launch_seq = 0;
    uint64_t launches = 0;
};

namespace {

constexpr uint64_t kAlignB = 256;
uint64_t up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct BLayout {
    uint64_t N = 0, bm_stride = 0, off_bm = 0, off_small = 0, total = 0;
    uint32_t nlevels = 0;
    uint64_t lvl_off[DSOA_MAX_LEVELS] = {0}, lvl_words[DSOA_MAX_LEVELS] = {0};
};

bool layout(uint64_t N, uint32_t rec, int ntypes, BLayout* L) {
    if (N == 0) return false;
    L->N = N;
    uint64_t words = (N + 63) / 64, off = 0;
    uint32_t nl = 0;
    for (;;) {
        if (nl >= DSOA_MAX_LEVELS) return false;
        L->lvl_off[nl] = off;
        L->lvl_words[nl] = words;
        off += words;
        ++nl;
        if (words == 1) break;
        words = (words + 63) / 64;
    }
    L->nlevels = nl;
    L->bm_stride = up(off, kAlignB / 8);
    uint64_t p = up(N * rec, kAlignB);
    L->off_bm = p;
    p = up(p + (uint64_t)(1 + 2 * ntypes) * L->bm_stride * 8, kAlignB);
    L->off_small = p;
    p = up(p + 16 * 8, kAlignB);
    L->total = p;
    return true;
}

// every slot free: bit i of level l set iff i < (bits at level l)
__global__ void kb_init_free(dsoa_ctx c) {
    uint64_t total = 0;
    for (uint32_t l = 0; l < c.nlevels; ++l) total += c.lvl_words[l];
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = g;
        uint32_t l = 0;
        while (i >= c.lvl_words[l]) { i -= c.lvl_words[l]; ++l; }
        const uint64_t nbits = l == 0 ? c.M : c.lvl_words[l - 1];
        const uint64_t k = std::min<uint64_t>(64, nbits - i * 64);
        c.bm[c.lvl_off[l] + i] = k >= 64 ? DSOA_ALL : ((1ull << k) - 1ull);
    }
}

__device__ __forceinline__ char* rec_of(const dsoa_ctx& c, uint64_t slot, uint32_t rec) {
    return c.data + slot * rec;
}

// per-type record field offsets, passed by value to every kernel
struct Fields {
    uint32_t rec;
    uint32_t off[DSOA_MAX_FIELDS];
};

__device__ __forceinline__ void bitmap_delete(const dsoa_ctx& c, uint32_t t, uint64_t slot) {
    if (!dsoa_bm_clear(c, dsoa_bm_alloc(t), slot, false)) {   // not allocated: double free
        dsoa_raise(c, DSOA_DEV_DOUBLE_FREE);
        return;
    }
    dsoa_bm_set(c, dsoa_bm_free(), slot);
}

// ---- the microbench's constructor and methods on records ----
struct BMicroCtor {
    static __device__ void ctor(const dsoa_ctx& c, char* r, const Fields& f, uint64_t i, const dsoa_micro_args& a) {
        const uint32_t id = a.id_base + (uint32_t)i;
        *reinterpret_cast<int32_t*>(r + f.off[0]) = (int32_t)id;
        *reinterpret_cast<float*>(r + f.off[1]) = 0.0f;
        *reinterpret_cast<unsigned long long*>(r + f.off[2]) = dsoa_sm2(a.seed, id);
    }
};
struct BMicroScale {
    static __device__ void run(const dsoa_ctx&, uint32_t, uint64_t, char* r, const Fields& f, const dsoa_micro_args&) {
        const int32_t id = *reinterpret_cast<const int32_t*>(r + f.off[0]);
        float* x = reinterpret_cast<float*>(r + f.off[1]);
        *x = __fadd_rn(__fmul_rn(*x, 1.5f), __int2float_rn(id));
    }
};
struct BMicroDelete {
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t slot, char* r, const Fields& f,
                               const dsoa_micro_args& a) {
        const uint32_t id = (uint32_t)*reinterpret_cast<const int32_t*>(r + f.off[0]);
        if (dsoa_sm3(a.seed, id, a.round) & 1ull) bitmap_delete(c, t, slot);
    }
};
struct BMicroDeleteAll {
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t slot, char*, const Fields&,
                               const dsoa_micro_args&) {
        bitmap_delete(c, t, slot);
    }
};
struct BMicroGather {
    static __device__ void run(const dsoa_ctx&, uint32_t, uint64_t, char* r, const Fields& f, const dsoa_micro_args& a) {
        const uint32_t id = (uint32_t)*reinterpret_cast<const int32_t*>(r + f.off[0]);
        if (id < a.n_ids) {
            a.x_out[id] = *reinterpret_cast<const float*>(r + f.off[1]);
            a.live_out[id] = 1;
        }
    }
};

// parallel_new: thread i takes a free slot and constructs object i there.
template <class C>
__global__ void kb_new(dsoa_ctx c, uint32_t t, uint64_t n, Fields f, dsoa_micro_args a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t slot = dsoa_bm_take(c, dsoa_bm_free(), dsoa_hash((uint32_t)i * 0x9E3779B9u ^ c.seed));
        if (slot < 0) {
            dsoa_raise(c, slot == -1 ? DSOA_DEV_OOM : DSOA_DEV_SPIN);
            continue;
        }
        C::ctor(c, rec_of(c, (uint64_t)slot, f.rec), f, i, a);
        __threadfence();
        dsoa_bm_set(c, dsoa_bm_alloc(t), (uint64_t)slot);
    }
}

// snapshot: allocated[t] -> iteration bitmap of t, every level
__global__ void kb_snapshot(dsoa_ctx c, uint32_t t) {
    const unsigned long long* src = c.bm + (uint64_t)dsoa_bm_alloc(t) * c.bm_stride;
    unsigned long long* dst = c.bm + (uint64_t)dsoa_bm_active(t) * c.bm_stride;
    uint64_t total = 0;
    for (uint32_t l = 0; l < c.nlevels; ++l) total += c.lvl_words[l];
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x)
        dst[g] = src[g];
}

// do-all: 64 threads per level-0 word of the snapshot; thread j serves bit j.
// Words whose level-1 bit is clear are skipped without reading them.
template <class M>
__global__ void kb_doall(dsoa_ctx c, uint32_t t, Fields f, dsoa_micro_args a) {
    const uint32_t b = dsoa_bm_active(t);
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / 64u;
    const uint32_t j = threadIdx.x & 63u;
    for (uint64_t wi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 64u; wi < c.lvl_words[0]; wi += groups) {
        if (L1 && !((__ldg(&L1[wi >> 6]) >> (wi & 63u)) & 1ull)) continue;
        const unsigned long long w = __ldg(&L0[wi]);
        if ((w >> j) & 1ull) {
            const uint64_t slot = wi * 64u + j;
            M::run(c, t, slot, rec_of(c, slot, f.rec), f, a);
        }
    }
}

// microbench statistics over the snapshot (same reduction as on the DynaSOAr heap)
__global__ void kb_stats(dsoa_ctx c, uint32_t t, Fields f, dsoa_micro_stats* out) {
    const uint32_t b = dsoa_bm_active(t);
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / 64u;
    const uint32_t j = threadIdx.x & 63u;
    unsigned long long live = 0, sid = 0, stag = 0, xtag = 0;
    double sx = 0.0;
    for (uint64_t wi = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 64u; wi < c.lvl_words[0]; wi += groups) {
        if ((__ldg(&L0[wi]) >> j) & 1ull) {
            const char* r = rec_of(c, wi * 64u + j, f.rec);
            const int32_t id = *reinterpret_cast<const int32_t*>(r + f.off[0]);
            const unsigned long long tag = *reinterpret_cast<const unsigned long long*>(r + f.off[2]);
            live += 1;
            sid += (unsigned long long)(long long)id;
            stag += tag;
            xtag ^= tag;
            sx += (double)*reinterpret_cast<const float*>(r + f.off[1]);
        }
    }
    for (int o = 16; o; o >>= 1) {
        live += __shfl_xor_sync(0xFFFFFFFFu, live, o);
        sid += __shfl_xor_sync(0xFFFFFFFFu, sid, o);
        stag += __shfl_xor_sync(0xFFFFFFFFu, stag, o);
        xtag ^= __shfl_xor_sync(0xFFFFFFFFu, xtag, o);
        sx += __shfl_xor_sync(0xFFFFFFFFu, sx, o);
    }
    if ((threadIdx.x & 31u) == 0 && live) {
        atomicAdd(&out->live, live);
        atomicAdd(&out->sum_id, sid);
        atomicAdd(&out->sum_tag, stag);
        atomicXor(&out->xor_tag, xtag);
        atomicAdd(&out->sum_x, sx);
    }
}

__global__ void kb_popc(dsoa_ctx c, uint32_t b, unsigned long long* out) {
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    unsigned long long cnt = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.lvl_words[0];
         i += (uint64_t)gridDim.x * blockDim.x)
        cnt += (unsigned long long)__popcll(L0[i]);
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    if ((threadIdx.x & 31u) == 0 && cnt) atomicAdd(out, cnt);
}

// Invariants at quiescence: out[0] containers whose upper bit disagrees with
// (container != 0) in any bitmap, out[1] slots neither free nor allocated or
// both (or allocated to two types), out[2] set bits beyond the last slot.
__global__ void kb_check(dsoa_ctx c, unsigned long long* out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nbm = 1u + 2u * c.ntypes;
    unsigned long long hier = 0, xr = 0, tail = 0;
    for (uint64_t wi = g0; wi < c.lvl_words[0]; wi += stride) {
        const uint64_t nbits = std::min<uint64_t>(64, c.M - wi * 64);
        const unsigned long long valid = nbits >= 64 ? DSOA_ALL : ((1ull << nbits) - 1ull);
        const unsigned long long fr = dsoa_level(c, dsoa_bm_free(), 0)[wi];
        unsigned long long any = 0, twice = 0;
        for (uint32_t t = 0; t < c.ntypes; ++t) {
            const unsigned long long a = dsoa_level(c, dsoa_bm_alloc(t), 0)[wi];
            twice |= any & a;
            any |= a;
        }
        xr += (unsigned long long)__popcll(((fr ^ any) ^ valid) & valid) + (unsigned long long)__popcll(twice | (fr & any));
        tail += (unsigned long long)__popcll((fr | any) & ~valid);
    }
    for (uint32_t b = 0; b < nbm; ++b) {
        if (b >= 1 && (b & 1u) == 0) continue;               // snapshots are not maintained
        for (uint32_t l = 1; l < c.nlevels; ++l) {
            const unsigned long long* lo = dsoa_level(c, b, l - 1);
            const unsigned long long* hi = dsoa_level(c, b, l);
            for (uint64_t i = g0; i < c.lvl_words[l - 1]; i += stride) {
                const bool bit = (hi[i >> 6] >> (i & 63u)) & 1ull;
                if (bit != (lo[i] != 0ull)) ++hier;
            }
        }
    }
    if (hier) atomicAdd(&out[0], hier);
    if (xr) atomicAdd(&out[1], xr);
    if (tail) atomicAdd(&out[2], tail);
}

int launch_ok(dsoa_bitmap_heap* h) {
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? DSOA_OK : DSOA_ERR_CUDA;
}

dsoa_ctx launch_ctx(dsoa_bitmap_heap* h) {
    dsoa_ctx c = h->ctx;
    c.seed = 0x9E3779B9u * (++h->launch_seq);
    return c;
}

Fields fields_of(const dsoa_bitmap_heap* h, int t) {
    Fields f;
    f.rec = h->rec_bytes;
    for (int i = 0; i < DSOA_MAX_FIELDS; ++i) f.off[i] = h->field_off[t][i];
    return f;
}

unsigned grid_for(dsoa_bitmap_heap* h, uint64_t threads, int tpb) {
    const uint64_t want = (threads + tpb - 1) / tpb;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)h->num_sms * 16));
}

bool is_micro_type(const dsoa_bitmap_heap* h, int t) {
    return h->nfields[t] == 3 && h->field_bytes[t][0] == 4 && h->field_bytes[t][1] == 4 && h->field_bytes[t][2] == 8;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

template <class M>
int run_doall(dsoa_bitmap_heap* h, int t, const dsoa_micro_args& a) {
    const dsoa_ctx c = launch_ctx(h);
    kb_snapshot<<<grid_for(h, h->ctx.bm_stride, 256), 256, 0, h->stream>>>(c, (uint32_t)t);
    int rc = launch_ok(h);
    if (rc) return rc;
    kb_doall<M><<<grid_for(h, h->ctx.lvl_words[0] * 64, 256), 256, 0, h->stream>>>(c, (uint32_t)t,
                                                                                    fields_of(h, t), a);
    return launch_ok(h);
}

}  // namespace

extern "C" {

int dsoa_bitmap_heap_create(size_t bytes, void* stream, dsoa_bitmap_heap** out) {
    if (!out || bytes < 4096) return DSOA_ERR_INVALID_ARG;
    *out = nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return DSOA_ERR_CUDA; }
    dsoa_bitmap_heap* h = new (std::nothrow) dsoa_bitmap_heap();
    if (!h) { cudaFree(p); return DSOA_ERR_OOM; }
    h->base = p;
    h->bytes = bytes;
    h->owns = true;
    h->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    std::memset(&h->ctx, 0, sizeof(h->ctx));
    *out = h;
    return DSOA_OK;
}

int dsoa_bitmap_register_type(dsoa_bitmap_heap* h, const uint32_t* field_bytes, int nfields, int* type_out) {
    if (!h || !field_bytes || !type_out || nfields < 1 || nfields > DSOA_MAX_FIELDS) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_ERR_FROZEN;
    if (h->ntypes >= DSOA_MAX_TYPES) return DSOA_ERR_TOO_MANY_TYPES;
    const int t = h->ntypes;
    uint32_t off = 0, align = 1;
    for (int f = 0; f < nfields; ++f) {
        const uint32_t b = field_bytes[f];
        if (b != 1 && b != 2 && b != 4 && b != 8 && b != 16) return DSOA_ERR_INVALID_ARG;
        off = (off + b - 1) / b * b;               // natural alignment inside the record
        h->field_off[t][f] = off;
        h->field_bytes[t][f] = b;
        off += b;
        align = std::max(align, b);
    }
    h->nfields[t] = nfields;
    h->rec_bytes = std::max(h->rec_bytes, (off + align - 1) / align * align);
    h->ntypes = t + 1;
    *type_out = t;
    return DSOA_OK;
}

int dsoa_bitmap_heap_freeze(dsoa_bitmap_heap* h) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_OK;
    if (h->ntypes == 0) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    // records of the largest type, aligned to 16 bytes when larger than 8
    uint32_t rec = h->rec_bytes;
    if (rec > 8) rec = (rec + 15) / 16 * 16;
    h->rec_bytes = rec;
    uint64_t lo = 0, hi = h->bytes / rec + 1;
    BLayout L;
    while (lo + 1 < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (layout(mid, rec, h->ntypes, &L) && L.total <= h->bytes) lo = mid; else hi = mid;
    }
    if (lo == 0 || !layout(lo, rec, h->ntypes, &L)) return DSOA_ERR_OOM;
    char* base = (char*)h->base;
    dsoa_ctx& c = h->ctx;
    c.data = base;
    c.bm = (unsigned long long*)(base + L.off_bm);
    uint64_t* small = (uint64_t*)(base + L.off_small);
    c.err = (int*)small;
    h->scratch = (unsigned long long*)(small + 8);
    c.M = L.N;
    c.bm_stride = L.bm_stride;
    for (int l = 0; l < DSOA_MAX_LEVELS; ++l) { c.lvl_off[l] = L.lvl_off[l]; c.lvl_words[l] = L.lvl_words[l]; }
    c.nlevels = L.nlevels;
    c.block_bytes = rec;
    c.ntypes = (uint32_t)h->ntypes;
    DSOA_CUDA_TRY(cudaMemsetAsync(c.bm, 0, (uint64_t)(1 + 2 * h->ntypes) * L.bm_stride * 8, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(small, 0, 16 * 8, h->stream));
    kb_init_free<<<std::max(1, h->num_sms * 4), 256, 0, h->stream>>>(c);
    const int rc = launch_ok(h);
    if (rc) return rc;
    h->frozen = true;
    return DSOA_OK;
}

int dsoa_bitmap_heap_info(dsoa_bitmap_heap* h, uint64_t* num_slots, uint32_t* record_bytes, uint32_t* num_levels) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    if (num_slots) *num_slots = h->ctx.M;
    if (record_bytes) *record_bytes = h->rec_bytes;
    if (num_levels) *num_levels = h->ctx.nlevels;
    return DSOA_OK;
}

int dsoa_bitmap_parallel_new(dsoa_bitmap_heap* h, int type, uint64_t n, int ctor_id, const void* args, size_t nb) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    int rc = dsoa_bitmap_heap_freeze(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    if (ctor_id != DSOA_C_MICRO) return DSOA_ERR_UNKNOWN_METHOD;
    if (!is_micro_type(h, type)) return DSOA_ERR_INVALID_ARG;
    dsoa_micro_args a;
    rc = dsoa_copy_args(&a, args, nb);
    if (rc) return rc;
    if (n == 0) return DSOA_OK;
    kb_new<BMicroCtor><<<grid_for(h, n, 256), 256, 0, h->stream>>>(launch_ctx(h), (uint32_t)type, n,
                                                                   fields_of(h, type), a);
    return launch_ok(h);
}

int dsoa_bitmap_parallel_do(dsoa_bitmap_heap* h, int type, int method_id, const void* args, size_t nb) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    int rc = dsoa_bitmap_heap_freeze(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    dsoa_micro_args a;
    rc = dsoa_copy_args(&a, args, nb);
    if (rc) return rc;
    if (method_id < 100 || method_id >= 200) return DSOA_ERR_UNKNOWN_METHOD;
    if (!is_micro_type(h, type)) return DSOA_ERR_INVALID_ARG;
    switch (method_id) {
        case DSOA_M_MICRO_SCALE:
        case DSOA_M_MICRO_SCALE_SCALAR:
        case DSOA_M_MICRO_SCALE_TMA: return run_doall<BMicroScale>(h, type, a);
        case DSOA_M_MICRO_DELETE: return run_doall<BMicroDelete>(h, type, a);
        case DSOA_M_MICRO_DELETE_ALL: return run_doall<BMicroDeleteAll>(h, type, a);
        case DSOA_M_MICRO_GATHER:
            if (!a.x_out || !a.live_out) return DSOA_ERR_INVALID_ARG;
            return run_doall<BMicroGather>(h, type, a);
        case DSOA_M_MICRO_STATS: {
            if (!a.stats) return DSOA_ERR_INVALID_ARG;
            const dsoa_ctx c = launch_ctx(h);
            kb_snapshot<<<grid_for(h, h->ctx.bm_stride, 256), 256, 0, h->stream>>>(c, (uint32_t)type);
            rc = launch_ok(h);
            if (rc) return rc;
            kb_stats<<<grid_for(h, h->ctx.lvl_words[0] * 64, 256), 256, 0, h->stream>>>(
                c, (uint32_t)type, fields_of(h, type), (dsoa_micro_stats*)a.stats);
            return launch_ok(h);
        }
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}

int dsoa_bitmap_count(dsoa_bitmap_heap* h, int type, uint64_t* out_host) {
    if (!h || !out_host || type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    int rc = dsoa_bitmap_heap_freeze(h);
    if (rc) return rc;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    DSOA_CUDA_TRY(cudaMemsetAsync(h->scratch, 0, 8, h->stream));
    kb_popc<<<grid_for(h, h->ctx.lvl_words[0], 256), 256, 0, h->stream>>>(h->ctx, dsoa_bm_alloc((uint32_t)type),
                                                                         h->scratch);
    rc = launch_ok(h);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemcpyAsync(out_host, h->scratch, 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_bitmap_check(dsoa_bitmap_heap* h, uint64_t* out_host) {
    if (!h || !out_host) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    DSOA_CUDA_TRY(cudaMemsetAsync(h->scratch, 0, 3 * 8, h->stream));
    kb_check<<<grid_for(h, h->ctx.lvl_words[0], 256), 256, 0, h->stream>>>(h->ctx, h->scratch);
    const int rc = launch_ok(h);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemcpyAsync(out_host, h->scratch, 3 * 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_bitmap_get_error(dsoa_bitmap_heap* h, int* bits_out) {
    if (!h || !bits_out) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) { *bits_out = 0; return DSOA_OK; }
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    DSOA_CUDA_TRY(cudaMemcpyAsync(bits_out, h->ctx.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(h->ctx.err, 0, sizeof(int), h->stream));
    return DSOA_OK;
}

int dsoa_bitmap_heap_destroy(dsoa_bitmap_heap* h) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->owns && h->base) cudaFree(h->base);
    delete h;
    return DSOA_OK;
}

}  // extern "C"
