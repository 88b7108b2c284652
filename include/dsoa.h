/*
 * dsoa.h -- C ABI of the GB300 SMMO runtime: a lock-free device object
 * allocator over a heap of 64-slot SOA blocks managed by hierarchical 64-bit
 * bitmaps, plus the parallel do-all (DynaSOAr, Springer & Masuhara, ECOOP 2019).
 *
 * Conventions for every entry point below:
 *   - Return value: DSOA_OK (0) or a negative DSOA_ERR_* code.  Nothing throws.
 *   - Pointers named *_host are host memory; *_dev are device memory of the
 *     heap's GPU.  The caller owns every buffer it passes in.
 *   - All GPU work is stream-ordered on the heap's stream (a cudaStream_t passed
 *     as void*, 0 = legacy default stream) and asynchronous, unless the
 *     description says "synchronous".
 *   - Device-side failures (out of memory inside a kernel, a spin limit reached,
 *     a double free, a bad handle) never trap: they set bits in a sticky device
 *     error word that dsoa_get_error() reads and clears.
 *   - A heap is not thread-safe: one host thread drives it at a time.
 */
#ifndef DSOA_H
#define DSOA_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSOA_OK 0
#define DSOA_ERR_INVALID_ARG (-1)
#define DSOA_ERR_FROZEN (-2)          /* type registration after the layout froze */
#define DSOA_ERR_TOO_MANY_TYPES (-3)
#define DSOA_ERR_OOM (-4)             /* heap too small for its own metadata      */
#define DSOA_ERR_CUDA (-5)            /* a CUDA runtime call failed               */
#define DSOA_ERR_NOT_FROZEN (-6)      /* operation needs a frozen layout          */
#define DSOA_ERR_UNKNOWN_METHOD (-7)  /* method / constructor id not built in     */
#define DSOA_ERR_CAPTURE (-8)         /* synchronous call during stream capture   */

/* bits of the sticky device error word (dsoa_get_error) */
#define DSOA_DEV_OOM 1          /* an allocation found no free block: handle 0      */
#define DSOA_DEV_SPIN 2         /* a bounded retry loop gave up                     */
#define DSOA_DEV_DOUBLE_FREE 4  /* a slot was freed twice                           */
#define DSOA_DEV_BAD_HANDLE 8   /* a handle did not decode to a valid type/block    */
#define DSOA_DEV_BAD_INDEX 16   /* a method read an instance / cell index out of range
                                   from an object field and skipped the object        */

#define DSOA_MAX_TYPES 16       /* registered types per heap                        */
#define DSOA_MAX_FIELDS 12      /* fields per type                                  */
#define DSOA_SLOTS 64           /* object slots per block (Sec. 3.1, 64-bit bitmap) */

/* Object handle (the paper's "fake pointer", Sec. 3.3, with the 35-bit address
 * trick replaced by a block index): [63:56] type id + 1, [55:6] block index,
 * [5:0] slot.  0 is the null handle. */
typedef uint64_t dsoa_obj;
typedef struct dsoa_heap dsoa_heap;
typedef struct dsoa_graph dsoa_graph;

/* Create a heap of `bytes` device bytes allocated with cudaMalloc, driven on
 * `stream`.  The byte budget covers blocks and all metadata (bitmaps, block
 * list, scratch).  Blocks are carved when the layout freezes (first allocation
 * or dsoa_heap_freeze).  Sec. 3 ("the heap is divided into M blocks"). */
int dsoa_heap_create(size_t bytes, void* stream, dsoa_heap** out);

/* Same over caller-owned device memory `dev_ptr` (256-byte aligned, `bytes`
 * long, e.g. a torch tensor); dsoa_heap_destroy does not free it. */
int dsoa_heap_create_from(void* dev_ptr, size_t bytes, void* stream, dsoa_heap** out);

/* Register an object type with `nfields` fields of `field_bytes[i]` bytes each
 * (1, 2, 4, 8 or 16).  Each field becomes one 64-element SOA column inside a
 * block, 128-byte aligned (Sec. 2.2 "clustered layout", Sec. 3.1).  Writes the
 * new type id (0, 1, ...) to *type_out.  Fails with DSOA_ERR_FROZEN after the
 * layout froze. */
int dsoa_register_type(dsoa_heap* h, const uint32_t* field_bytes, int nfields, int* type_out);

/* Register a subtype of `base` (Sec. 1 "Subclassing/Inheritance", Sec. 3.1):
 * its fields are base's fields followed by `n_extra` new ones of
 * `extra_field_bytes[i]` bytes (n_extra may be 0), so the data segment of its
 * blocks begins with the inherited SOA columns at the same field indices and a
 * method written for base reads and writes them unchanged (the handle carries
 * the runtime type, which fixes the column offsets and, in the per-type
 * capacity mode, the block capacity: Sec. 3.3).  The subtype has its own
 * blocks and its own allocated / active bitmaps: blocks of a subtype are not in
 * the bitmaps of its base (Sec. 3.4).  dsoa_parallel_do on base also visits
 * the objects of every subtype (Sec. 2.1).  Errors: DSOA_ERR_INVALID_ARG (unknown base, more than
 * DSOA_MAX_FIELDS fields in all, a bad field size), DSOA_ERR_FROZEN,
 * DSOA_ERR_TOO_MANY_TYPES. */
int dsoa_register_subtype(dsoa_heap* h, int base, const uint32_t* extra_field_bytes, int n_extra, int* type_out);

/* The type `type` extends (-1 for a type registered by dsoa_register_type). */
int dsoa_type_base(dsoa_heap* h, int type, int* base_out);

/* Freeze the layout.  Uniform capacity (the default): every type has 64 slots
 * per block and block bytes = the largest registered type's 64-slot data
 * segment.  Per-type capacity (dsoa_set_capacity_mode): see below.  M = blocks
 * that fit with their metadata.  Initialises the bitmaps (every block free,
 * Sec. 3.4).  Called implicitly by the first allocating call. */
int dsoa_heap_freeze(dsoa_heap* h);

/* Query the frozen layout (any pointer may be NULL). */
int dsoa_heap_info(dsoa_heap* h, uint64_t* num_blocks, uint32_t* block_bytes,
                   uint32_t* num_levels, uint64_t* metadata_bytes);

/* Column byte offset of field `field` of `type` inside a block's data segment
 * (final once the layout froze; before that, the uniform-capacity offset). */
int dsoa_field_offset(dsoa_heap* h, int type, int field, uint32_t* offset_out);

/* Block capacity mode, before the layout freezes (DSOA_ERR_FROZEN after).
 * DSOA_CAPACITY_PER_TYPE follows Sec. 3.2 "Block Capacity": a block holds 64
 * objects of the smallest type T_s (by summed field bytes), so its data
 * segment is T_s's 64 128-byte-aligned columns, and every type T gets
 * N_T = floor(64 size(T_s) / size(T)) slots, lowered until its columns
 * (16-byte aligned when N_T < 64) fit.  Smaller blocks for small types; larger
 * types trade slots for bytes.  A type more than 64 times larger than T_s
 * makes the freeze fail with DSOA_ERR_INVALID_ARG.  Slots at or above N_T stay
 * marked free in the block's slot word and are never reserved. */
#define DSOA_CAPACITY_UNIFORM 0
#define DSOA_CAPACITY_PER_TYPE 1
int dsoa_set_capacity_mode(dsoa_heap* h, int mode);

/* Slots per block of `type` (64, or N_T), after the freeze. */
int dsoa_type_capacity(dsoa_heap* h, int type, uint32_t* n_out);

/* parallel_new<T>(n) (Sec. 2.1): one kernel, n logical threads; thread i
 * allocates one object of `type` and runs built-in constructor `ctor_id` with
 * index i and the `args_bytes` bytes at `args_host` (copied at launch).  A
 * thread whose allocation fails (heap full) gets a null handle and sets
 * DSOA_DEV_OOM.  Constructor ids and argument structs: dsoa_apps.h. */
int dsoa_parallel_new(dsoa_heap* h, int type, uint64_t n, int ctor_id,
                      const void* args_host, size_t args_bytes);

/* parallel_do<T, f> (Sec. 2.1, Sec. 3.7): snapshot the allocation bitmaps of
 * every block of `type`, compact the block list R from the type's allocated-
 * block bitmap (hierarchical bitmap scan + prefix sum, Sec. 4.1.5, Fig. 7),
 * then run built-in method `method_id` on every object in the snapshot.
 * Objects created by the method are not visited; the method may delete `this`
 * and objects of other types.  A type with subtypes (dsoa_register_subtype)
 * covers their objects too: one enumeration launch snapshots the type and all
 * its subtypes, then the method runs in one launch per type (Sec. 2.1). */
int dsoa_parallel_do(dsoa_heap* h, int type, int method_id, const void* args_host,
                     size_t args_bytes);

/* ---- user methods (Sec. 2.1: parallel_do<T, &T::func> for any member
 * function).  A user translation unit includes dsoa_device.cuh, writes a
 * method struct (see dsoa_doall_kernel there) and names it with
 * DSOA_METHOD(id, launcher, Method): that instantiates the do-all kernel for
 * the method in the user's own library, and a static initializer registers the
 * launcher under `id` when that library is loaded.  dsoa_parallel_do(h, type,
 * id, args) then enumerates as for a built-in method and calls the launcher
 * with the prepared launch; the launch runs on the heap's stream and counts as
 * one of the heap's launches. */
#define DSOA_USER_METHOD_MIN 1000
#define DSOA_USER_METHOD_MAX 1999
typedef struct {
    const void* ctx;              /* host copy of this launch's struct dsoa_ctx          */
    size_t ctx_bytes;             /* sizeof(struct dsoa_ctx) in the library              */
    int32_t type;                 /* the type the do-all runs on                         */
    uint32_t tpb;                 /* threads per CTA (multiple of 64)                    */
    uint32_t max_ctas_per_sm;     /* resident CTAs per SM the grid may assume            */
    uint32_t num_sms;
    uint32_t waves;               /* grid = waves x resident grid                         */
    uint32_t slots_per_thread;    /* 1 or 2                                              */
    uint32_t pdl;                 /* 1: launch with programmatic stream serialization    */
    uint32_t reserved;
    const uint32_t* R;            /* device: block list of the snapshot                  */
    const uint64_t* occ;          /* device: occupancy snapshot per listed block         */
    const uint32_t* r_dev;        /* device: number of listed blocks                     */
    void* stream;                 /* cudaStream_t of the heap                            */
} dsoa_doall_launch;
/* Launches the method's do-all kernel; DSOA_OK, or DSOA_ERR_INVALID_ARG (args
 * of the wrong size, ctx of another library build), DSOA_ERR_CUDA. */
typedef int (*dsoa_method_fn)(const dsoa_doall_launch* launch, const void* args_host, size_t args_bytes);
/* Process-wide registration of `fn` under method id DSOA_USER_METHOD_MIN ..
 * DSOA_USER_METHOD_MAX.  Registering the same fn again is a no-op; another fn
 * under a taken id, a null fn or an id out of range give DSOA_ERR_INVALID_ARG.
 * An unregistered id in dsoa_parallel_do gives DSOA_ERR_UNKNOWN_METHOD. */
int dsoa_register_method(int method_id, dsoa_method_fn fn);

/* The method kernel of dsoa_parallel_do alone, over the snapshot and block
 * list of the latest enumeration of `type` (dsoa_enumerate or a previous
 * dsoa_parallel_do of the same type).  Valid only while no object of `type`
 * was created or deleted since that enumeration, except by methods run this
 * way on the same snapshot.  Used to time or to repeat the do-all kernel. */
int dsoa_parallel_do_enumerated(dsoa_heap* h, int type, int method_id, const void* args_host,
                                size_t args_bytes);

/* Run built-in plain kernel `kernel_id` (dsoa_apps.h) with n logical threads:
 * an ordinary CUDA kernel that may call device new/delete (Sec. 2.1, "new and
 * destroy are device functions callable from GPU code"). */
int dsoa_run_kernel(dsoa_heap* h, int kernel_id, uint64_t n, const void* args_host,
                    size_t args_bytes);

/* destroy() (Sec. 2.1, Alg. 2) for n handles in device memory, one kernel:
 * frees of the same block in a warp are combined.  Null handles are skipped;
 * a handle whose type or block is out of range sets DSOA_DEV_BAD_HANDLE, a slot
 * that is already free in a block that still exists sets DSOA_DEV_DOUBLE_FREE
 * (both leave the heap unchanged for that handle).  Freeing a slot of a block
 * that was already emptied and deleted violates Alg. 8's precondition and is
 * not detected; every retry loop stays bounded, so it cannot hang. */
int dsoa_delete_handles(dsoa_heap* h, const dsoa_obj* handles_dev, uint64_t n);

/* Enumerate only (the first two kernels of dsoa_parallel_do): after the call,
 * R_dev[0..*r_dev) lists the blocks of `type` in increasing order and
 * occ_dev[i] their occupied-slot masks.  The three pointers are library-owned
 * and valid until the next enumeration on this heap.  Used by user do-all
 * kernels written against dsoa_device.cuh. */
int dsoa_enumerate(dsoa_heap* h, int type, const uint32_t** R_dev,
                   const uint64_t** occ_dev, const uint32_t** r_dev);

/* Enumerate several types at once (`ntypes` distinct ids at types_host): the
 * same result as one dsoa_enumerate per type issued back to back, but the
 * single-pass enumeration serves all of them with one launch (each type keeps
 * its own block list and snapshot).  Meant for step loops whose later do-alls
 * (dsoa_parallel_do_enumerated) visit types that the earlier methods of the
 * step do not create or delete.  Asynchronous. */
int dsoa_enumerate_many(dsoa_heap* h, const int* types_host, int ntypes);

/* Number of live objects of `type` (popcounts of the slot bitmaps of the
 * blocks in the type's allocated-block bitmap).  Synchronous: waits for the
 * heap's stream.  Not allowed during stream capture. */
int dsoa_count(dsoa_heap* h, int type, uint64_t* out_host);

/* Same, stored to `out_dev` (uint64) by the kernel; graph-capturable.  out_dev
 * is any address the device may write: device memory, or pinned host memory
 * mapped into the device's address space (the value then reaches the host
 * without a copy); it needs no initialisation. */
int dsoa_count_async(dsoa_heap* h, int type, uint64_t* out_dev);

/* Live objects of `ntypes` distinct types (ids at types_host) in one launch:
 * out_dev[q] (uint64) = live objects of types_host[q], stored as by
 * dsoa_count_async.  Graph-capturable. */
int dsoa_count_many_async(dsoa_heap* h, const int* types_host, int ntypes, uint64_t* out_dev);

/* Number of free blocks (popcount of the free-block bitmap) to `out_dev`
 * (uint64); graph-capturable.  Used for admission control. */
int dsoa_free_blocks_async(dsoa_heap* h, uint64_t* out_dev);

/* Read and clear the sticky device error word (DSOA_DEV_* bits).  Synchronous. */
int dsoa_get_error(dsoa_heap* h, int* bits_out);

/* Check the allocator invariants at quiescence (Sec. 3.4, App. A.4
 * "container consistency"): writes DSOA_CHECK_COUNT counters to out_host, all
 * zero when the heap is consistent.  Synchronous. */
#define DSOA_CHECK_HIER 0          /* upper bit != (lower container != 0)          */
#define DSOA_CHECK_FREE_XOR 1      /* block neither free nor allocated, or both    */
#define DSOA_CHECK_MULTI_TYPE 2    /* block in two types' allocated bitmaps        */
#define DSOA_CHECK_ACTIVE_SUBSET 3 /* active bit without allocated bit             */
#define DSOA_CHECK_TYPE 4          /* allocated[T] block whose type id is not T    */
#define DSOA_CHECK_FREE_WORD 5     /* free block whose slot word is not all-taken  */
#define DSOA_CHECK_EMPTY_ALLOC 6   /* allocated block with no object               */
#define DSOA_CHECK_ACTIVE_EXACT 7  /* active != (allocated and not full)           */
#define DSOA_CHECK_TAIL_BITS 8     /* bits beyond M set                            */
#define DSOA_CHECK_CAP_BITS 9      /* allocated block with a slot beyond its type's
                                      capacity not marked free                      */
#define DSOA_CHECK_COUNT 10
int dsoa_check(dsoa_heap* h, uint64_t* out_host);

/* Copy the raw allocator state to host memory (synchronous), for external
 * checkers: slot words (M x u64, 1 = free slot), block types (M x u32), then
 * every hierarchical bitmap (free, then allocated[T], active[T] per type; each
 * bitmap is its levels from level 0 upward, bitmap_words u64 in total).
 * *bytes_needed receives the size; pass out_host = NULL to query it. */
int dsoa_export_state(dsoa_heap* h, void* out_host, size_t capacity, size_t* bytes_needed,
                      uint64_t* bitmap_words);

/* Checkpoint / resume (the paper has no counterpart).  dsoa_heap_save copies
 * the whole heap -- blocks, slot words, type ids, bitmaps, block lists -- behind
 * a header that records the layout into host memory `out_host` (capacity bytes,
 * at least *bytes_needed = header + heap bytes; pass out_host = NULL to query).
 * dsoa_heap_load copies such an image into a heap created with the same byte
 * size and the same registered types and capacity mode (the layout must match
 * exactly, else DSOA_ERR_INVALID_ARG); it freezes the heap first if needed.
 * References inside the heap are indices, so the image is valid at any device
 * address; object handles saved elsewhere (e.g. cell maps) stay valid.  Both
 * are synchronous and not allowed during stream capture.  Work still queued on
 * other streams must be finished by the caller. */
int dsoa_heap_save(dsoa_heap* h, void* out_host, size_t capacity, size_t* bytes_needed);
int dsoa_heap_load(dsoa_heap* h, const void* in_host, size_t bytes);

/* Device-side view of the heap for user kernels built with dsoa_device.cuh:
 * copies the struct dsoa_ctx (size ctx_bytes must match) to ctx_out_host. */
int dsoa_get_ctx(dsoa_heap* h, void* ctx_out_host, size_t ctx_bytes);

/* Stream capture of the heap's stream into a CUDA graph, for step loops. */
int dsoa_graph_begin(dsoa_heap* h);
int dsoa_graph_end(dsoa_heap* h, dsoa_graph** out);
int dsoa_graph_launch(dsoa_graph* g, void* stream);
int dsoa_graph_destroy(dsoa_graph* g);

/* Launch shape of do-all and scan kernels (0 keeps the current value):
 * threads per CTA of the do-all (multiple of 64, at most 512; default 256), CTAs
 * per SM of the resident do-all grid (1..32, capped by what fits; default 8),
 * slots handled per thread (1 or 2 for method do-alls, 1, 2 or 4 for vectorised
 * ones), the enumeration (1 or 2 = tile-count kernel + compaction kernel with
 * that many level-1 tiles per CTA, 3 = single-pass decoupled look-back kernel,
 * the default, 4 = as 3, but methods that create no objects of their own type
 * enumerate inside their own kernel, tile by tile, 5 = a thread-block cluster
 * of 8 CTAs per type scans the bitmap in shared memory and exchanges its CTAs'
 * totals through distributed shared memory, for heaps of at most 65,536
 * level-0 words (4,194,304 blocks; larger heaps use 3)), and the waves of the
 * method do-all grid (1..DSOA_MAX_WAVES, default
 * 4): its grid is `waves` times the resident grid, so that SMs that finish their
 * share early take over the rest (streaming do-alls keep one resident wave).
 * Returns DSOA_ERR_INVALID_ARG at the first value out of range (the values before
 * it in the argument list are applied). */
#define DSOA_MAX_WAVES 16
int dsoa_set_launch(dsoa_heap* h, int doall_tpb, int doall_ctas_per_sm,
                    int slots_per_thread, int scan_tiles_per_cta, int doall_waves);

/* Ablation switches of Sec. 6.4 (Fig. 10c): DSOA_FLAG_NO_COALESCE (1) turns
 * off allocation request coalescing, DSOA_FLAG_NO_ROTATE (2) turns off bitmap
 * rotation, DSOA_FLAG_NO_HINT (4) turns off the per-warp last-block hint and
 * DSOA_FLAG_FUSED (8) runs dsoa_parallel_do as ONE cooperative launch
 * (enumeration and method separated by grid barriers) instead of the
 * enumeration and do-all kernels, and DSOA_FLAG_PDL (16) launches the
 * enumeration, do-all and step-counter kernels with programmatic dependent
 * launch, so that each may be scheduled while its predecessor finishes (the
 * last three are not in the paper); DSOA_FLAG_ENUM_TICKETS (32) makes the
 * single-pass enumeration hand tiles out by a ticket counter instead of
 * ordering them by CTA index (which relies on every CTA of the launch being
 * resident: true on an otherwise idle GPU).  Two experiment switches change
 * the allocation policy (measured in the fragmentation analysis of Sec. 6.4):
 * DSOA_FLAG_NO_FRESH_GROUP (128) keeps groups of 16 or more requests searching
 * active blocks after a lost round instead of taking a fresh block, and
 * DSOA_FLAG_PAPER_R (256) counts every active-block attempt of an allocation
 * toward r, lost reservations included, and takes a fresh block after r of
 * them (Alg. 1's reading of r), and DSOA_FLAG_R_PER_ROUND (512) restores an
 * earlier policy in which r bounds the failed finds of one round and small
 * groups search again in every round.  DSOA_FLAG_DRAIN (1024) lets blocks that
 * fell to an eighth of their capacity drain: a search passes over them (at most
 * 4 times per allocation) and a warp drops its hint to one, so that they empty
 * instead of being refilled (not in the paper; it lowers fragmentation).
 * Returns DSOA_ERR_INVALID_ARG for an unknown bit.  Takes effect for launches
 * issued after the call. */
int dsoa_set_flags(dsoa_heap* h, uint32_t flags);

/* r of Sec. 4.2 / Fig. 11: an allocation's attempts on active blocks
 * (try_find_set on the active bitmap; a reservation that lost its race counts
 * as one) before it initialises a new block; 1..64, default 32 (the paper's
 * default is 5; with lost reservations counted, 5 takes fresh blocks so often
 * that a 64 MiB heap holds a Wa-Tor torus of 1344^2 instead of 1600^2 at r = 32,
 * at the same speed).  Takes effect for launches issued after the call. */
int dsoa_set_lookups(dsoa_heap* h, int r);

/* Blocks of `type` (popcount of its allocated-block bitmap) and its live
 * objects, to out_host[0] and out_host[1]; fragmentation of Sec. 6.4 is
 * F = 1 - out[1] / (64 * out[0]).  Synchronous. */
int dsoa_type_stats(dsoa_heap* h, int type, uint64_t* out_host);

/* Number of kernels this heap has launched so far (host-side counter). */
int dsoa_launch_count(dsoa_heap* h, uint64_t* out_host);

/* Destroy the heap (synchronous); frees library-allocated device memory. */
int dsoa_heap_destroy(dsoa_heap* h);

/* Human-readable name of an error code. */
const char* dsoa_error_string(int code);

/* ---- BitmapAlloc: the paper's second allocator (Sec. 6, "BitmapAlloc") ----
 * The heap is one array of equal-size object records in array-of-structures
 * layout (no blocks, no SOA columns), whose slots are managed by hierarchical
 * bitmaps like DynaSOAr's blocks: one free-slot bitmap and one allocation
 * bitmap per type (Sec. 4.1 operations over object slots).  new takes a free
 * bit and sets it in the type's allocation bitmap; delete clears it and frees
 * the slot; a do-all copies the allocation bitmap to an iteration snapshot and
 * runs one thread per snapshot bit.  It measures pure bitmap allocation
 * without DynaSOAr's block structure and SOA layout; every type occupies a
 * record of the largest type's size (internal fragmentation).
 *
 * Same conventions as the DynaSOAr heap (return codes, stream order, sticky
 * device error word).  Built in: the microbench's constructor and methods
 * (dsoa_apps.h ids 100-107 except the handle-map method; the SCALE variants all
 * run the plain per-object method) on types with fields {4, 4, 8}; any other
 * id returns DSOA_ERR_UNKNOWN_METHOD. */
typedef struct dsoa_bitmap_heap dsoa_bitmap_heap;
/* cudaMalloc'd heap of `bytes`, records and bitmaps carved at freeze. */
int dsoa_bitmap_heap_create(size_t bytes, void* stream, dsoa_bitmap_heap** out);
/* A type of `nfields` fields (1, 2, 4, 8 or 16 bytes), laid out in declaration
 * order at natural alignment inside a record; before the first allocation. */
int dsoa_bitmap_register_type(dsoa_bitmap_heap* h, const uint32_t* field_bytes, int nfields, int* type_out);
/* Freeze: record bytes = largest type (16-byte aligned above 8 bytes); slots =
 * as many records as fit beside the bitmaps; every slot free. */
int dsoa_bitmap_heap_freeze(dsoa_bitmap_heap* h);
int dsoa_bitmap_heap_info(dsoa_bitmap_heap* h, uint64_t* num_slots, uint32_t* record_bytes,
                          uint32_t* num_levels);
/* parallel_new<T>(n): thread i takes a free slot (DSOA_DEV_OOM when none) and
 * runs constructor `ctor_id` with index i. */
int dsoa_bitmap_parallel_new(dsoa_bitmap_heap* h, int type, uint64_t n, int ctor_id,
                             const void* args_host, size_t args_bytes);
/* parallel_do<T, f>: snapshot of the allocation bitmap, then method `method_id`
 * on every object of the snapshot. */
int dsoa_bitmap_parallel_do(dsoa_bitmap_heap* h, int type, int method_id, const void* args_host,
                            size_t args_bytes);
/* Live objects of `type` (popcount of its allocation bitmap).  Synchronous. */
int dsoa_bitmap_count(dsoa_bitmap_heap* h, int type, uint64_t* out_host);
/* Invariants at quiescence into out_host[3]: hierarchy mismatches, slots not
 * exactly one of {free, allocated to one type}, bits past the last slot.
 * All zero when consistent.  Synchronous. */
int dsoa_bitmap_check(dsoa_bitmap_heap* h, uint64_t* out_host);
/* Read and clear the sticky device error word.  Synchronous. */
int dsoa_bitmap_get_error(dsoa_bitmap_heap* h, int* bits_out);
/* Waits for the heap's stream, frees the heap memory and the handle. */
int dsoa_bitmap_heap_destroy(dsoa_bitmap_heap* h);

/* ---- Enumeration without allocation (the paper has no counterpart) ----
 * For callers that cannot allocate device memory while they run: a host
 * program whose own allocator owns the GPU's memory under a fixed budget, a
 * latency-critical loop in which cudaMalloc / cudaFree would synchronise the
 * device, or code that keeps several enumerations alive in buffers it manages
 * itself.  Computes what dsoa_enumerate computes -- the blocks of `type` in
 * increasing order and the occupied-slot mask of each -- into caller-owned
 * device buffers R_out_dev[capacity] (u32), occ_out_dev[capacity] (u64) and
 * *r_out_dev (u32, the number of entries written).  capacity must be at least
 * the heap's block count (dsoa_heap_info), else DSOA_ERR_INVALID_ARG.
 *
 * The scan's working memory (per-tile counts and offsets, a completion ticket)
 * is a fixed array of 2 * DSOA_NOALLOC_MAX_TILES + 64 u32 (about 33 KB) inside
 * this library, which every GPU that loads the library holds until the
 * process exits.  The call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.  Limits and rules:
 *   - heaps of at most DSOA_NOALLOC_MAX_TILES * 4096 = 16,777,216 blocks; a
 *     larger heap returns DSOA_ERR_SCRATCH_LIMIT;
 *   - the heap must be frozen (DSOA_ERR_NOT_FROZEN otherwise; not frozen
 *     implicitly) and its device must be the current device;
 *   - every call made outside stream capture looks up the array's device
 *     address (cudaGetSymbolAddress) with the heap's device current; a call
 *     made while the heap's stream is capturing uses the address of the
 *     latest call outside capture on that device.  So make one call before
 *     any stream capture, and again after a device reset (cudaDeviceReset
 *     reloads the library's module, which may move the array); a call under
 *     capture with no earlier call returns DSOA_ERR_CAPTURE;
 *   - every call shares the one array, which keeps the last call's contents;
 *     the ticket is cleared at the start of each call, counts and offsets are
 *     overwritten.  Calls that overlap on the GPU (two streams, two heaps at
 *     once) race on the array: serialise them;
 *   - asynchronous, ordered on the heap's stream. */
#define DSOA_NOALLOC_MAX_TILES 4096
#define DSOA_ERR_SCRATCH_LIMIT (-9)   /* heap larger than the fixed scratch allows */
int dsoa_enumerate_noalloc(dsoa_heap* h, int type, uint32_t* R_out_dev, uint64_t* occ_out_dev,
                           uint32_t* r_out_dev, uint64_t capacity);

#ifdef __cplusplus
}
#endif
#endif
