/*
 * dsoa_device.cuh -- device side of the GB300 SMMO runtime (header only).
 *
 * The lock-free allocator of DynaSOAr (Springer & Masuhara, ECOOP 2019,
 * Sec. 3-4 and App. A) for sm_103a, usable from any CUDA kernel:
 *
 *   dsoa_new(ctx, type)       -> handle or 0          Alg. 1 (+ Sec. 4.2 coalescing)
 *   dsoa_delete(ctx, handle)                          Alg. 2
 *   dsoa_field<F>(ctx, h, i)  -> F&  (SOA column)      Sec. 3.3, App. B
 *
 * Heap layout (one GPU, frozen at the first allocation):
 *   data[M * block_bytes]  per block 64 slots in SOA: column i of type T at
 *                          byte col_off[T][i], 64 * field_bytes long, 128 B
 *                          aligned (Sec. 2.2 clustered layout)
 *   slot[M]   u64 per block, bit s = 1 iff slot s is FREE.  The paper keeps
 *             1 = allocated; the complement lets a reservation be one
 *             atomicAnd and a free one atomicOr.  Every rule of Alg. 7-10 is
 *             restated in this polarity below.
 *   btype[M]  u32 block type id
 *   bm        hierarchical bitmaps (Sec. 4.1): free-block, and per type the
 *             allocated-block and active-block bitmaps; each is its levels,
 *             level 0 first, ceil(n/64) u64 containers per level.
 *
 * Every spin of the paper (set/clear "retry until changed", the allocation
 * retry loop, invalidation retries) is bounded; on the bound the thread sets
 * DSOA_DEV_SPIN in the sticky error word and gives up.  Nothing traps.
 */
#ifndef DSOA_DEVICE_CUH
#define DSOA_DEVICE_CUH

#include <stdint.h>
#include <string.h>

#include "dsoa.h"

#define DSOA_MAX_LEVELS 6
#define DSOA_ALL ((unsigned long long)~0ull)

/* Bounds of every retry loop (legal workloads stay far below them; a thread
 * that reaches one sets DSOA_DEV_SPIN and gives up, so no kernel can hang):
 * one blocking bitmap op or invalidation waits at most ~16 ms, one
 * allocation makes at most DSOA_ALLOC_ROUNDS block selections, each with at
 * most DSOA_TAKE_ATTEMPTS find-and-clear attempts on the free-block bitmap. */
#ifndef DSOA_SPIN_LIMIT
#define DSOA_SPIN_LIMIT (1u << 16)
#endif
#ifndef DSOA_ALLOC_ROUNDS
#define DSOA_ALLOC_ROUNDS (1u << 12)
#endif
/* Without bitmap rotation (the NoShift ablation of Sec. 6.4) every leader
 * searches from the same first bit and most rounds are lost to the same few
 * blocks; lost rounds then back off exponentially (64 ns .. 4 us, jittered) and
 * the bound is larger, so that legal workloads finish, as Alg. 1's unbounded
 * retry loop does, only slower (about a second per allocation at most). */
#ifndef DSOA_ALLOC_ROUNDS_NO_ROTATE
#define DSOA_ALLOC_ROUNDS_NO_ROTATE (1u << 18)
#endif
#ifndef DSOA_TAKE_ATTEMPTS
#define DSOA_TAKE_ATTEMPTS 256u
#endif
#ifndef DSOA_OOM_ROUNDS
#define DSOA_OOM_ROUNDS 16u               /* rounds with an empty free bitmap = OOM */
#endif
#ifndef DSOA_LOOKUP_ATTEMPTS
#define DSOA_LOOKUP_ATTEMPTS 32           /* r: an allocation's active-block attempts
                                             (lost reservations included) before it
                                             takes a fresh block; 32 keeps Wa-Tor's
                                             speed of r = 5 and packs a nearly full
                                             heap like the per-round rule or better */
#endif

/* Entry of the per-warp block hint table: a block of the type that still had
 * free slots when this warp slot last reserved in it, and the free-slot word
 * that reservation left; and the level-0 word of the free-block bitmap this
 * warp slot last took a block from, with the free bits that take left.
 * Advisory only (any value is safe). */
struct __align__(16) dsoa_hint {
    unsigned long long free;             /* free slots as last seen (1 = free)     */
    uint64_t block;                      /* block id, DSOA_NO_HINT_BLOCK if none   */
    unsigned long long fword;            /* free blocks of level-0 word fidx as
                                            last seen (1 = free)                   */
    uint64_t fidx;                       /* level-0 word index of the free-block
                                            bitmap, >= its word count if none      */
};
#define DSOA_NO_HINT_BLOCK (~0ull)
#ifdef __CUDACC__
/* the block half {free, block} of a hint entry, one 16-byte store */
__device__ __forceinline__ void dsoa_hint_put(dsoa_hint* hp, unsigned long long free, uint64_t block) {
    *reinterpret_cast<ulonglong2*>(hp) = make_ulonglong2(free, (unsigned long long)block);
}
#endif

/* Device view of a heap.  Plain data, passed to kernels by value. */
struct dsoa_ctx {
    char* data;                          /* block b at data + b * block_bytes      */
    unsigned long long* slot;            /* [M] free-slot bitmaps                  */
    uint32_t* btype;                     /* [M] block type ids                     */
    unsigned long long* bm;              /* all hierarchical bitmaps               */
    int* err;                            /* sticky DSOA_DEV_* bits                 */
    dsoa_hint* hint;                     /* [hint_mask + 1][ntypes] last block with
                                            free slots per warp slot (advisory)       */
    uint8_t* drain;                      /* [M] 1 = the block fell to few objects and
                                            is left to drain (advisory)               */
    uint32_t* grid_scratch;              /* [DSOA_GRID_SCRATCH] per-CTA aggregates and
                                            grid-barrier words of the fused do-all    */
    uint64_t M;                          /* number of blocks                       */
    uint64_t bm_stride;                  /* u64 words per hierarchical bitmap      */
    uint64_t lvl_off[DSOA_MAX_LEVELS];   /* word offset of level l in a bitmap     */
    uint64_t lvl_words[DSOA_MAX_LEVELS]; /* containers at level l                  */
    uint32_t nlevels;
    uint32_t block_bytes;
    uint32_t ntypes;
    uint32_t seed;                       /* rotation seed of this launch           */
    uint32_t flags;                      /* DSOA_FLAG_*                            */
    uint32_t hint_mask;                  /* hint-table warp slots - 1 (power of 2)  */
    uint32_t lookups;                    /* active-block lookups before the slow path
                                            (r of Sec. 4.2 / Fig. 11), >= 1           */
    uint16_t col_off[DSOA_MAX_TYPES][DSOA_MAX_FIELDS];
    unsigned long long cap[DSOA_MAX_TYPES];  /* usable slots of a block of type t (Sec. 3.2
                                            block capacity N_T): the low N_T bits.  The
                                            slots above stay marked free in the slot word
                                            and are never reserved, so occupancy (~word),
                                            EMPTY and invalidation need no mask        */
};

/* Register cap of the generic do-all kernel.  Methods that allocate are chains
 * of dependent L2 round trips; at 48 registers five 256-thread CTAs fit on an
 * SM instead of four at 64 (Wa-Tor fish move: 67 -> 61 us per step).  Any
 * block size up to 512 threads still fits. */
#ifndef DSOA_DOALL_MAXNREG
#define DSOA_DOALL_MAXNREG 48
#endif
#ifndef DSOA_FRESH_GROUP
#define DSOA_FRESH_GROUP 16u              /* group size that takes a fresh block
                                             after a lost race (leader_reserve)    */
#endif
#define DSOA_FLAG_NO_COALESCE 1u          /* ablation: one request per leader       */
#define DSOA_FLAG_NO_ROTATE 2u            /* ablation: plain find-first-set         */
#define DSOA_FLAG_NO_HINT 4u              /* ablation: no per-warp block hint       */
#define DSOA_HINT_SLOTS 8192u             /* max hint-table warp slots per type     */
#define DSOA_FLAG_FUSED 8u                /* one cooperative enumerate+do-all launch */
#define DSOA_FUSED_MAX_CTAS 2048u         /* grid limit of the fused do-all         */
#define DSOA_FLAG_ENUM_TICKETS 32u        /* single-pass enumeration: hand tiles out by a
                                             ticket counter instead of relying on every
                                             CTA of the launch being resident (for heaps
                                             enumerated while other kernels occupy the
                                             GPU); slower on large heaps                */
#define DSOA_FLAG_PDL 16u                 /* programmatic dependent launch of the
                                             enumeration, do-all and step kernels  */
#define DSOA_FLAG_NO_FRESH_GROUP 128u     /* experiment: large groups keep searching
                                             active blocks after a lost round, like
                                             small ones (no fresh-block shortcut)   */
#define DSOA_FLAG_PAPER_R 256u            /* experiment: Alg. 1's reading of r alone:
                                             every group, large ones too, searches
                                             until r attempts (lost reservations
                                             included) failed, then takes a fresh
                                             block (no fresh-group shortcut)        */
#define DSOA_FLAG_R_PER_ROUND 512u        /* experiment: the earlier policy: r bounds
                                             the failed finds of one round, and a
                                             group below DSOA_FRESH_GROUP searches
                                             again in every round                   */
#define DSOA_FLAG_DRAIN 1024u             /* let blocks that fell to few objects
                                             drain: searches pass over them and a
                                             warp drops its hint to one
                                             (dsoa_drain_mark)                      */
#ifndef DSOA_DRAIN_SKIPS
#define DSOA_DRAIN_SKIPS 4u               /* draining blocks one allocation passes
                                             over at most                           */
#endif
#ifndef DSOA_DRAIN_SHIFT
#define DSOA_DRAIN_SHIFT 3u               /* a block drains at or below
                                             capacity >> DSOA_DRAIN_SHIFT objects   */
#endif
#define DSOA_GRID_SCRATCH (DSOA_FUSED_MAX_CTAS + 64u)
#define DSOA_CTX_NO_PROLOGUE (1u << 30)   /* set by the library in the context of the
                                             do-all launches that follow the first one
                                             of a family (a type with subtypes), so a
                                             method's prologue runs once per do-all */

/* Programmatic dependent launch (sm_90 and later).  A kernel launched with the
 * programmatic-serialization attribute may be scheduled while its predecessor
 * in the stream still runs; dsoa_pdl_wait() (griddepcontrol.wait) blocks until
 * that predecessor has completed and its memory operations are visible to this
 * grid, and returns at once for a kernel launched without the attribute.  The
 * kernels the library launches that way call it before their first global
 * memory access, so each of them also completes after its predecessor and the
 * chain stays ordered.  dsoa_pdl_release() (griddepcontrol.launch_dependents)
 * lets the next kernel be scheduled once every CTA of this one has started. */
__device__ __forceinline__ void dsoa_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dsoa_pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

/* bitmap ids inside ctx.bm */
__host__ __device__ __forceinline__ uint32_t dsoa_bm_free() { return 0u; }
__host__ __device__ __forceinline__ uint32_t dsoa_bm_alloc(uint32_t t) { return 1u + 2u * t; }
__host__ __device__ __forceinline__ uint32_t dsoa_bm_active(uint32_t t) { return 2u + 2u * t; }

/* ---- handles (Sec. 3.3 object pointers, App. B address computation) ---- */
__host__ __device__ __forceinline__ dsoa_obj dsoa_make_handle(uint32_t t, uint64_t bid, uint32_t s) {
    return ((uint64_t)(t + 1u) << 56) | (bid << 6) | (uint64_t)s;
}
__host__ __device__ __forceinline__ uint32_t dsoa_h_type(dsoa_obj h) { return (uint32_t)(h >> 56) - 1u; }
__host__ __device__ __forceinline__ uint64_t dsoa_h_block(dsoa_obj h) { return (h >> 6) & ((1ull << 50) - 1ull); }
__host__ __device__ __forceinline__ uint32_t dsoa_h_slot(dsoa_obj h) { return (uint32_t)(h & 63u); }

#ifdef __CUDACC__

/* ---- memory-model helpers: bitmap words are read at device scope, never
 * through the non-coherent L1 (App. A: "volatile or atomic") ---- */
__device__ __forceinline__ unsigned long long dsoa_ld(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t dsoa_ld32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dsoa_st(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void dsoa_st32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t dsoa_ld8(const uint8_t* p) {
    unsigned short v;
    asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dsoa_st8(uint8_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "h"((unsigned short)v) : "memory");
}
/* atomicAnd with acquire semantics at device scope: loads after it observe
 * what was written before the release (fence + store) whose value it read. */
__device__ __forceinline__ unsigned long long dsoa_and_acquire(unsigned long long* p, unsigned long long m) {
    unsigned long long old;
    asm volatile("atom.acquire.gpu.global.and.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(m) : "memory");
    return old;
}
/* atomicOr with release semantics at device scope: stores before it (the
 * freed object's last field writes) are visible before the freed slot can be
 * observed -- and reserved -- by another thread. */
__device__ __forceinline__ unsigned long long dsoa_or_release(unsigned long long* p, unsigned long long m) {
    unsigned long long old;
    asm volatile("atom.release.gpu.global.or.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(m) : "memory");
    return old;
}
__device__ __forceinline__ uint32_t dsoa_lane() {
    uint32_t l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}
__device__ __forceinline__ void dsoa_raise(const dsoa_ctx& c, int bits) { atomicOr(c.err, bits); }
__device__ __forceinline__ uint32_t dsoa_smid() {
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

/* Release fence before the store that publishes a block initialisation (the
 * slot word): with the acquire RMW that reserves slots it orders the block's
 * type store before any reservation that sees the slot word (a release
 * pattern: fence.acq_rel, then a strong store). */
__device__ __forceinline__ void dsoa_fence_release() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

/* An index that a method read from an object field (an instance, a grid cell,
 * a ring), checked before it addresses an application array: out of range
 * raises DSOA_DEV_BAD_INDEX and the method skips the object.  In a consistent
 * heap no index is ever out of range; the check keeps a method in bounds after
 * a bounded wait gave up (DSOA_DEV_SPIN) and left a stale bitmap bit that lists
 * a block under a type it no longer holds. */
__device__ __forceinline__ bool dsoa_index_ok(const dsoa_ctx& c, uint64_t i, uint64_t n) {
    if (i < n) return true;
    dsoa_raise(c, DSOA_DEV_BAD_INDEX);
    return false;
}

/* One wait step of a bounded spin; false once the bound is reached (error set). */
__device__ __forceinline__ bool dsoa_backoff(const dsoa_ctx& c, uint32_t& spins) {
    if (++spins >= DSOA_SPIN_LIMIT) { dsoa_raise(c, DSOA_DEV_SPIN); return false; }
    if (spins > 8) __nanosleep(spins < 64 ? 32u : 256u);
    return true;
}

__device__ __forceinline__ uint32_t dsoa_hash(uint32_t x) {
    /* integer finaliser (xor-shift / multiply, "lowbias32" constants) */
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned long long dsoa_rotr(unsigned long long w, uint32_t r) {
    r &= 63u;
    return r ? (w >> r) | (w << (64u - r)) : w;
}
__device__ __forceinline__ unsigned long long dsoa_rotl(unsigned long long w, uint32_t r) {
    r &= 63u;
    return r ? (w << r) | (w >> (64u - r)) : w;
}
/* position of the (n+1)-th lowest set bit of w (n < popc(w)), Sec. 4.3 */
__device__ __forceinline__ uint32_t dsoa_nth_set(unsigned long long w, uint32_t n) {
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
    const uint32_t plo = __popc(lo);
    if (n < plo) return __fns(lo, 0u, (int)n + 1);
    return 32u + __fns(hi, 0u, (int)(n - plo) + 1);
}
/* mask of the lowest k set bits of w */
__device__ __forceinline__ unsigned long long dsoa_lowest_k(unsigned long long w, uint32_t k) {
    if (k == 1u) return w & (0ull - w);               /* the lowest set bit (0 if none) */
    if ((uint32_t)__popcll(w) <= k) return w;
    if (k == 0) return 0ull;
    const uint32_t p = dsoa_nth_set(w, k - 1u);
    return p == 63u ? w : (w & ((2ull << p) - 1ull));
}

__device__ __forceinline__ unsigned long long* dsoa_level(const dsoa_ctx& c, uint32_t b, uint32_t l) {
    return c.bm + (uint64_t)b * c.bm_stride + c.lvl_off[l];
}

/* ------------------------------------------------------------------------
 * Hierarchical bitmap operations (Sec. 4.1, Alg. 3-4, App. A.4).
 * clear/set at level l; `blocking` = the paper's clear(pos)/set(pos) that
 * retries until this thread changed the bit; otherwise the try_ variant.
 * A thread that empties a container (clear-last) or fills an empty one
 * (set-first) propagates to the next level with the blocking variant.
 * Returns whether this thread changed the level-l bit.
 * ------------------------------------------------------------------------ */
__device__ inline bool dsoa_bm_clear(const dsoa_ctx& c, uint32_t b, uint64_t pos,
                                     bool blocking, uint32_t l = 0,
                                     unsigned long long* first_prev = nullptr) {
    bool first = true, changed = false;
    for (; l < c.nlevels; ++l) {
        unsigned long long* w = dsoa_level(c, b, l) + (pos >> 6);
        const unsigned long long m = 1ull << (pos & 63u);
        unsigned long long prev;
        uint32_t spins = 0;
        for (;;) {
            prev = atomicAnd(w, ~m);
            if (first && first_prev) *first_prev = prev;
            if (prev & m) break;
            if (!blocking) return false;
            if (!dsoa_backoff(c, spins)) return changed;
        }
        if (first) { changed = true; first = false; }
        if (prev != m) break;          /* container still has set bits */
        pos >>= 6;
        blocking = true;
    }
    return changed;
}

__device__ inline bool dsoa_bm_set(const dsoa_ctx& c, uint32_t b, uint64_t pos, uint32_t l = 0) {
    bool first = true, changed = false;
    for (; l < c.nlevels; ++l) {
        unsigned long long* w = dsoa_level(c, b, l) + (pos >> 6);
        const unsigned long long m = 1ull << (pos & 63u);
        unsigned long long prev;
        uint32_t spins = 0;
        for (;;) {
            prev = atomicOr(w, m);
            if (!(prev & m)) break;
            if (!dsoa_backoff(c, spins)) return changed;
        }
        if (first) { changed = true; first = false; }
        if (prev != 0ull) break;       /* container was already non-empty */
        pos >>= 6;
    }
    return changed;
}

/* try_find_set (Alg. 4) with bitmap rotation (Sec. 4.2): top-down; at every
 * level the container is rotated by a hash-derived amount before ffs, so
 * different warps start at different bits.  -1 = FAIL (possibly spurious
 * while levels are transiently inconsistent).  w0, if given, receives the
 * level-0 word the search ended in. */
__device__ inline int64_t dsoa_bm_find(const dsoa_ctx& c, uint32_t b, uint32_t h,
                                       unsigned long long* w0 = nullptr) {
    uint64_t idx = 0;
    const bool rot = !(c.flags & DSOA_FLAG_NO_ROTATE);
    for (int l = (int)c.nlevels - 1; l >= 0; --l) {
        const unsigned long long w = dsoa_ld(dsoa_level(c, b, (uint32_t)l) + idx);
        if (!w) return -1;
        if (l == 0 && w0) *w0 = w;
        const uint32_t r = rot ? ((h >> ((uint32_t)l * 5u)) ^ (h >> 27)) & 63u : 0u;
        const uint32_t bit = ((uint32_t)__ffsll((long long)dsoa_rotr(w, r)) - 1u + r) & 63u;
        idx = idx * 64u + bit;
    }
    return (int64_t)idx;
}

/* clear() = find-and-clear an arbitrary set bit (Sec. 4.1.2).  -1 when the
 * bitmap is empty at the top (OOM for the free-block bitmap), -2 when
 * DSOA_TAKE_ATTEMPTS attempts lost every race (the caller retries).
 * prev0, if given, receives the level-0 word as the successful clear found it. */
static __device__ __noinline__ int64_t dsoa_bm_take(const dsoa_ctx& c, uint32_t b, uint32_t h,
                                                    unsigned long long* prev0 = nullptr) {
    for (uint32_t a = 0; a < DSOA_TAKE_ATTEMPTS; ++a) {
        const int64_t pos = dsoa_bm_find(c, b, dsoa_hash(h + a * 0x9E3779B9u));
        if (pos >= 0) {
            if (dsoa_bm_clear(c, b, (uint64_t)pos, false, 0, prev0)) return pos;
        } else if (dsoa_ld(dsoa_level(c, b, c.nlevels - 1)) == 0ull) {
            return -1;
        }
        if (a > 8) __nanosleep(64u);
    }
    return -2;
}

/* ------------------------------------------------------------------------
 * Block operations (App. A.1-A.2), free-slot polarity.
 * ------------------------------------------------------------------------ */

/* initialize_block<T> (Alg. 9): type first, fence, then all 64 slots free. */
__device__ inline void dsoa_block_init(const dsoa_ctx& c, uint64_t bid, uint32_t t) {
    dsoa_st32(&c.btype[bid], t);
    dsoa_fence_release();
    dsoa_st(&c.slot[bid], DSOA_ALL);
}

/* invalidate + delete an emptied block (Alg. 2's deletion branch with Alg. 10):
 * take every slot with one atomicAnd(0).  Success iff all 64 were free; then
 * the block leaves active[t] and allocated[t] and returns to the free bitmap.
 * Otherwise give back exactly the slots taken (atomicOr(before)); if another
 * thread freed a slot meanwhile it saw a "first free" and will set the active
 * bit, so the deferred deactivation is done here; retry if the block is empty
 * again. */
static __device__ __noinline__ void dsoa_block_invalidate(const dsoa_ctx& c, uint64_t bid) {
    for (uint32_t it = 0; it < DSOA_SPIN_LIMIT; ++it) {
        const unsigned long long before = atomicAnd(&c.slot[bid], 0ull);
        if (before == DSOA_ALL) {
            const uint32_t t = dsoa_ld32(&c.btype[bid]);
            dsoa_bm_clear(c, dsoa_bm_active(t), bid, true);
            dsoa_bm_clear(c, dsoa_bm_alloc(t), bid, true);
            dsoa_bm_set(c, dsoa_bm_free(), bid);
            return;
        }
        if (before == 0ull) return;    /* nothing taken: someone else owns it */
        const unsigned long long rb = atomicOr(&c.slot[bid], before);
        if (rb != 0ull) {
            const uint32_t t = dsoa_ld32(&c.btype[bid]);
            dsoa_bm_clear(c, dsoa_bm_active(t), bid, true);
        }
        if ((rb | before) != DSOA_ALL) return;
    }
    dsoa_raise(c, DSOA_DEV_SPIN);
}

/* Rare transitions of a block, kept out of line so that the hot paths of
 * allocation and deallocation stay small in registers. */
static __device__ __noinline__ void dsoa_block_first_free(const dsoa_ctx& c, uint32_t t, uint64_t bid) {
    dsoa_bm_set(c, dsoa_bm_active(t), bid);                 /* was full: active again */
}
static __device__ __noinline__ void dsoa_block_deactivate(const dsoa_ctx& c, uint32_t t, uint64_t bid) {
    dsoa_bm_clear(c, dsoa_bm_active(t), bid, true);         /* now full: inactive */
}

/* Draining (DSOA_FLAG_DRAIN; a policy of this runtime, not of the paper).
 * Objects never move, so a block stays in use while it holds one object, and
 * when allocations land on blocks at random, as the rotated search makes them,
 * a population that shrinks leaves many blocks holding a few objects each.  A
 * free that leaves a block's live objects at or below an eighth of its
 * capacity (DSOA_DRAIN_SHIFT; having been above) marks the block draining: a search that finds
 * it passes over it, at most DSOA_DRAIN_SKIPS times per allocation, and a warp
 * that reserved in it drops its hint to it, so that it empties and returns to
 * the free bitmap instead of being refilled.  The mark is cleared when the
 * block is taken fresh or filled.  Advisory: the bitmaps and their invariants
 * are the same with the flag and without it. */
__device__ __forceinline__ void dsoa_drain_mark(const dsoa_ctx& c, uint32_t t, uint64_t bid,
                                                unsigned long long before, unsigned long long bits) {
    const uint32_t d = (uint32_t)__popcll(c.cap[t]) >> DSOA_DRAIN_SHIFT;
    const uint32_t live_before = (uint32_t)__popcll(~before & c.cap[t]);
    const uint32_t live_after = (uint32_t)__popcll(~(before | bits) & c.cap[t]);
    if (live_after <= d && live_before > d && live_after != 0u) dsoa_st8(&c.drain[bid], 1u);
}

/* Block::deallocate for a set of slots (Alg. 8, multi-slot form used by
 * request coalescing and by rollback).  `t` is the block's type. */
__device__ __forceinline__ void dsoa_block_release(const dsoa_ctx& c, uint32_t t, uint64_t bid,
                                                   unsigned long long bits) {
    const unsigned long long before = dsoa_or_release(&c.slot[bid], bits);
    if (before & bits) {
        dsoa_raise(c, DSOA_DEV_DOUBLE_FREE);
        bits &= ~before;
        if (!bits) return;
    }
    if (c.flags & DSOA_FLAG_DRAIN) dsoa_drain_mark(c, t, bid, before, bits);
    /* FIRST: real slots (below the capacity) freed in a block that had none free;
     * a rollback that only returns slots beyond the capacity changes nothing */
    if ((before & c.cap[t]) == 0ull && (bits & c.cap[t]) != 0ull) dsoa_block_first_free(c, t, bid);
    if ((before | bits) == DSOA_ALL) dsoa_block_invalidate(c, bid);          /* EMPTY */
}

/* Slow path of Alg. 1 (a new block) with the reservation folded in: take a free
 * block and initialise it for type t with the `mask` slots already taken (type first,
 * fence, then the slot word), enter it into allocated[t], and into active[t]
 * unless the reservation filled it.  Slots are only ever taken from the word,
 * so nobody can take these, and a block with reserved slots cannot be emptied,
 * invalidated or retyped: no reservation atomic and no type re-check are needed.
 * The free block comes, when it can, from the level-0 free-bitmap word this
 * warp slot took its previous block from (the hint's fword / fidx): one
 * atomicAnd on a bit the hint still shows free, instead of the top-down find
 * (one dependent load per level) and its clear; a hint that is stale costs that
 * one atomic, then the find runs.  Emptying the word propagates as in clear().
 * -1 = no free block, -2 = every attempt lost its race. */
static __device__ __noinline__ int64_t dsoa_block_new_reserved(const dsoa_ctx& c, uint32_t t, uint32_t h,
                                                               unsigned long long mask, dsoa_hint* hp) {
    int64_t bid = -1;
    unsigned long long* L0f = dsoa_level(c, dsoa_bm_free(), 0);
    if (hp) {
        const ulonglong2 fh = *reinterpret_cast<const ulonglong2*>(&hp->fword);
        if (fh.y < c.lvl_words[0] && fh.x) {
            const uint32_t r = h & 63u;
            const uint32_t bit = ((uint32_t)__ffsll((long long)dsoa_rotr(fh.x, r)) - 1u + r) & 63u;
            const unsigned long long m = 1ull << bit;
            const unsigned long long prev = atomicAnd(L0f + fh.y, ~m);
            *reinterpret_cast<ulonglong2*>(&hp->fword) = make_ulonglong2(prev & ~m, fh.y);
            if (prev & m) {
                bid = (int64_t)(fh.y * 64u + bit);
                if (prev == m && c.nlevels > 1) dsoa_bm_clear(c, dsoa_bm_free(), fh.y, true, 1);
            }
        }
    }
    if (bid < 0) {
        unsigned long long prev = 0ull;
        bid = dsoa_bm_take(c, dsoa_bm_free(), h, &prev);
        if (bid < 0) return bid;
        if (hp)
            *reinterpret_cast<ulonglong2*>(&hp->fword) =
                make_ulonglong2(prev & ~(1ull << ((uint64_t)bid & 63u)), (unsigned long long)bid >> 6);
    }
    /* allocated[t] is read by enumerations of later launches only, so its
     * level-0 RMW goes out with the type store and its latency overlaps the
     * release fence; active[t] and the slot word, which publish the block to
     * allocations in flight, follow the fence.  Each RMW falls back to
     * dsoa_bm_set's retry loop if its bit was already set, and propagates
     * upwards if its container was empty. */
    const unsigned long long m = 1ull << ((uint64_t)bid & 63u);
    const bool act = (c.cap[t] & ~mask) != 0ull;
    unsigned long long* wa = dsoa_level(c, dsoa_bm_alloc(t), 0) + ((uint64_t)bid >> 6);
    unsigned long long* wv = dsoa_level(c, dsoa_bm_active(t), 0) + ((uint64_t)bid >> 6);
    dsoa_st32(&c.btype[bid], t);
    if (c.flags & DSOA_FLAG_DRAIN) dsoa_st8(&c.drain[bid], 0u);
    const unsigned long long pa = atomicOr(wa, m);
    dsoa_fence_release();
    dsoa_st(&c.slot[bid], DSOA_ALL & ~mask);
    const unsigned long long pv = act ? atomicOr(wv, m) : m;
    if (pa & m) dsoa_bm_set(c, dsoa_bm_alloc(t), (uint64_t)bid);
    else if (pa == 0ull && c.nlevels > 1) dsoa_bm_set(c, dsoa_bm_alloc(t), (uint64_t)bid >> 6, 1);
    if (act) {
        if (pv & m) dsoa_bm_set(c, dsoa_bm_active(t), (uint64_t)bid);
        else if (pv == 0ull && c.nlevels > 1) dsoa_bm_set(c, dsoa_bm_active(t), (uint64_t)bid >> 6, 1);
    }
    return bid;
}

/* Roll back slots reserved in a block whose type changed (Alg. 1's type check). */
static __device__ __noinline__ void dsoa_rollback(const dsoa_ctx& c, uint32_t bt, uint64_t bid, unsigned long long got) {
    dsoa_block_release(c, bt, bid, got);
}

/* Leader part of allocate<T> (Alg. 1 with request coalescing, Sec. 4.2):
 * reserve up to `want` slots of type t in ONE block.  Block selection tries
 * the active bitmap DSOA_LOOKUP_ATTEMPTS times with rotated starts, else takes
 * a free block (slow path).  A reservation is one atomicAnd of the chosen
 * slot bits; the thread whose reservation empties the free-slot word marks
 * the block inactive; a type change is rolled back.  Returns the reserved
 * slot mask (0 on OOM or spin bound) and the block in *bid_out. */
__device__ __forceinline__ unsigned long long dsoa_leader_reserve(const dsoa_ctx& c, uint32_t t, uint32_t want,
                                                         uint32_t h, uint64_t* bid_out) {
    const uint32_t act = dsoa_bm_active(t);
    const bool rot = !(c.flags & DSOA_FLAG_NO_ROTATE);
    /* Per-warp hint: the block this warp (slot of the hint table) last reserved
     * in while it still had free slots, with the free-slot word that
     * reservation left behind.  Trying it first skips the top-down bitmap
     * search and the read of the slot word: the reservation mask is taken from
     * the remembered word, and a stale word only costs slots (an atomicAnd of
     * a slot that is no longer free reserves nothing).  A stale block is just
     * another "Block Full / Deallocated / Replaced" case of App. A.3 and is
     * caught by the same checks as a stale try_find_set. */
    dsoa_hint* hp = nullptr;
    if (c.hint && !(c.flags & DSOA_FLAG_NO_HINT)) {
        const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        hp = c.hint + (gwarp & c.hint_mask) * c.ntypes + t;
    }
    uint32_t empty_free = 0;   /* rounds that found the free-block bitmap empty */
    const uint32_t max_rounds = rot ? DSOA_ALLOC_ROUNDS : DSOA_ALLOC_ROUNDS_NO_ROTATE;
    const bool per_round = (c.flags & DSOA_FLAG_R_PER_ROUND) != 0u;
    const bool fresh_group = want >= DSOA_FRESH_GROUP &&
                             !(c.flags & (DSOA_FLAG_NO_FRESH_GROUP | DSOA_FLAG_PAPER_R));
    uint32_t tries = 0;        /* active-block attempts so far, lost reservations included */
    const bool drain = (c.flags & DSOA_FLAG_DRAIN) != 0u;
    uint32_t skips = 0;        /* draining blocks passed over so far */
    for (uint32_t round = 0; round < max_rounds; ++round) {
        if (!rot && round) {           /* NoShift: thin out the races on the first bits */
            const uint32_t span = 32u << (round < 7u ? round : 7u);
            __nanosleep(span / 2u + (dsoa_hash(h ^ (round * 0x9E3779B9u)) & (span / 2u - 1u)));
        }
        int64_t bid = -1;
        unsigned long long w = 0ull;   /* free slots of bid, if already known */
        unsigned long long w0 = 0ull;  /* active blocks of the level-0 word the search ended in */
        if (round == 0 && hp) {
            const ulonglong2 hv = *reinterpret_cast<const ulonglong2*>(hp);   /* {free, block} */
            if (hv.y < c.M && hv.x) { bid = (int64_t)hv.y; w = hv.x; }
            else if (fresh_group && !per_round) tries = c.lookups;   /* no hinted block: fresh at once */
        }
        /* r of Alg. 1 (Sec. 4.2): an allocation makes at most r attempts on
         * active blocks, a reservation that lost its race counting as one, and
         * then takes a fresh block.  A group of DSOA_FRESH_GROUP or more requests
         * takes a fresh block after a lost race, and at once when its warp slot
         * has no hinted block: when far more warps allocate together than there
         * are active blocks with room (an allocation burst) they would otherwise
         * converge on the same few blocks, whose other slots the owners' hints
         * are about to take.  An empty free bitmap always searches (at most r
         * finds per round). */
        const bool search = per_round ? (round == 0 || empty_free || !fresh_group)
                                      : (empty_free != 0u || (tries < c.lookups && (round == 0 || !fresh_group)));
        if (per_round) {
            for (uint32_t a = 0; search && a < c.lookups && bid < 0; ++a)
                bid = dsoa_bm_find(c, act, dsoa_hash(h ^ (round * DSOA_LOOKUP_ATTEMPTS + a) * 0x9E3779B9u), &w0);
        } else {
            for (uint32_t a = 0; search && bid < 0 && a < c.lookups && (tries < c.lookups || empty_free); ++a, ++tries)
                bid = dsoa_bm_find(c, act, dsoa_hash(h ^ (round * DSOA_LOOKUP_ATTEMPTS + tries) * 0x9E3779B9u), &w0);
        }
        if (bid < 0) {
            const unsigned long long fmask = dsoa_lowest_k(c.cap[t], want);
            bid = dsoa_block_new_reserved(c, t, h ^ round, fmask, hp);
            if (bid == -2) continue;
            if (bid < 0) {
                /* No free block.  Blocks that other warps initialised in the
                 * same burst may still have free slots once their active bits
                 * are set: look again before reporting OOM (Alg. 1 retries
                 * forever; here a bounded number of times). */
                if (++empty_free >= DSOA_OOM_ROUNDS) { dsoa_raise(c, DSOA_DEV_OOM); return 0ull; }
                __nanosleep(256u);
                continue;
            }
            const unsigned long long left = c.cap[t] & ~fmask;    /* fresh block: reserved on init */
            if (hp) dsoa_hint_put(hp, left, left ? (uint64_t)bid : DSOA_NO_HINT_BLOCK);
            *bid_out = (uint64_t)bid;
            return fmask;
        }
        if (!w) {                      /* a block the search found: its slot word */
            unsigned long long sw = dsoa_ld(&c.slot[bid]);
            uint32_t dr = drain ? dsoa_ld8(&c.drain[bid]) : 0u;
            /* a draining block: the other active blocks of the same level-0 word
             * (one load each, no new search); when none is left, a new search */
            bool again = false;
            while (dr && skips < DSOA_DRAIN_SKIPS) {
                ++skips;
                w0 &= ~(1ull << ((uint64_t)bid & 63u));
                const uint32_t r0 = dsoa_hash(h + skips * 0x9E3779B9u) & 63u;
                const uint64_t nb = ((uint64_t)bid & ~63ull) |
                                    (((uint32_t)__ffsll((long long)dsoa_rotr(w0, r0)) - 1u + r0) & 63u);
                if (!w0 || nb >= c.M) { again = true; break; }
                bid = (int64_t)nb;
                sw = dsoa_ld(&c.slot[bid]);
                dr = dsoa_ld8(&c.drain[bid]);
            }
            if (again) continue;
            w = sw & c.cap[t];
            if (!w) continue;
        }
        const uint32_t r = rot ? (dsoa_hash(h + round) & 63u) : 0u;
        const unsigned long long mask = dsoa_rotl(dsoa_lowest_k(dsoa_rotr(w, r), want), r);
        /* acquire: the type read below sees the type written before the
         * fence of dsoa_block_init whose slot-word store this RMW follows */
        const unsigned long long before = dsoa_and_acquire(&c.slot[bid], ~mask);
        const unsigned long long got = before & mask;
        if (!got) {
            const unsigned long long left = before & c.cap[t];
            if (hp) dsoa_hint_put(hp, left, left ? (uint64_t)bid : DSOA_NO_HINT_BLOCK);
            continue;
        }
        const uint32_t bt = dsoa_ld32(&c.btype[bid]);
        const uint32_t drn = drain ? dsoa_ld8(&c.drain[bid]) : 0u;
        /* FULL: this reservation took the last free real slots of the block's type
         * (a reservation of another type may take only slots beyond that type's
         * capacity, which leaves the block's state unchanged) */
        const unsigned long long capb = c.cap[bt < c.ntypes ? bt : t];
        const unsigned long long left = before & ~mask & capb;
        const bool full = left == 0ull && (before & capb) != 0ull;
        if (full) {
            dsoa_block_deactivate(c, bt, (uint64_t)bid);
            if (drn) dsoa_st8(&c.drain[bid], 0u);
        }
        if (bt != t) {                 /* block replaced by another type: roll back */
            if (hp) dsoa_hint_put(hp, 0ull, DSOA_NO_HINT_BLOCK);
            dsoa_rollback(c, bt, (uint64_t)bid, got);
            continue;
        }
        if (hp) dsoa_hint_put(hp, left, (full || drn) ? DSOA_NO_HINT_BLOCK : (uint64_t)bid);
        *bid_out = (uint64_t)bid;
        return got;
    }
    dsoa_raise(c, DSOA_DEV_SPIN);
    return 0ull;
}

/* Prefetch into L1 the warp's block hint for type t (advisory: a method that
 * may allocate calls it early, so that the leader's hint load in dsoa_new
 * overlaps with the method's own loads instead of starting its chain). */
__device__ __forceinline__ void dsoa_prefetch_hint(const dsoa_ctx& c, uint32_t t) {
    if (!c.hint || (c.flags & DSOA_FLAG_NO_HINT)) return;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const dsoa_hint* hp = c.hint + (gwarp & c.hint_mask) * c.ntypes + t;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(hp));
}

/* new(d_allocator) T (Sec. 2.1; Alg. 1): callable from any kernel, any
 * divergence.  Same-type requests of a warp are coalesced (__match_any_sync):
 * the lowest lane of each group reserves slots for the whole group, block by
 * block, and lane k of the group takes the k-th reserved slot.  Returns the
 * handle, or 0 if the heap is out of blocks (DSOA_DEV_OOM set). */
__device__ inline dsoa_obj dsoa_new(const dsoa_ctx& c, uint32_t t) {
    const uint32_t lane = dsoa_lane();
    const uint32_t active = __activemask();
    const uint32_t peers = (c.flags & DSOA_FLAG_NO_COALESCE) ? (1u << lane) : __match_any_sync(active, t);
    const uint32_t leader = (uint32_t)__ffs((int)peers) - 1u;
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    const uint32_t want = (uint32_t)__popc(peers);
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t h0 = dsoa_hash(gwarp * 0x85EBCA6Bu ^ c.seed ^ (lane << 26));
    dsoa_obj out = 0;
    uint32_t served = 0;
    for (uint32_t round = 0; served < want; ++round) {
        unsigned long long got = 0ull;
        uint64_t bid = 0;
        if (lane == leader) got = dsoa_leader_reserve(c, t, want - served, h0 + round * 0x632BE5ABu, &bid);
        got = __shfl_sync(peers, got, (int)leader);
        bid = __shfl_sync(peers, bid, (int)leader);
        const uint32_t k = (uint32_t)__popcll(got);
        if (k == 0) break;
        if (rank >= served && rank < served + k)
            out = dsoa_make_handle(t, bid, dsoa_nth_set(got, rank - served));
        served += k;
    }
    /* Memory ordering across the group: the leader's acquire reservation
     * happens-before every lane's constructor stores into its new slot, so a
     * slot freed by another thread (release) cannot receive its old owner's
     * late stores after the new owner's. */
    __syncwarp(peers);
    return out;
}

/* destroy(d_allocator, ptr) (Sec. 2.1; Alg. 2): frees of the same block in a
 * warp are combined into one atomicOr by the group's lowest lane. */
__device__ inline void dsoa_delete(const dsoa_ctx& c, dsoa_obj h) {
    const uint32_t active = __activemask();
    const bool ok = h != 0 && dsoa_h_type(h) < c.ntypes && dsoa_h_block(h) < c.M;
    if (h != 0 && !ok) dsoa_raise(c, DSOA_DEV_BAD_HANDLE);
    const unsigned long long key = ok ? (h >> 6) : ~0ull;
    const uint32_t lane = dsoa_lane();
    const uint32_t peers = (c.flags & DSOA_FLAG_NO_COALESCE) ? (1u << lane) : __match_any_sync(active, key);
    const unsigned long long bit = ok ? (1ull << dsoa_h_slot(h)) : 0ull;
    const uint32_t lo = __reduce_or_sync(peers, (uint32_t)bit);
    const uint32_t hi = __reduce_or_sync(peers, (uint32_t)(bit >> 32));
    /* every lane's last stores to its object happen-before the leader's
     * release of the slots (dsoa_block_release) */
    __syncwarp(peers);
    if (ok && lane == (uint32_t)__ffs((int)peers) - 1u)
        dsoa_block_release(c, dsoa_h_type(h), dsoa_h_block(h), ((unsigned long long)hi << 32) | lo);
}

/* ---- field access (Sec. 3.3 / App. B, without pointer tagging) ---- */
__device__ __forceinline__ char* dsoa_block_data(const dsoa_ctx& c, uint64_t bid) {
    return c.data + bid * (uint64_t)c.block_bytes;
}
template <typename F>
__device__ __forceinline__ F* dsoa_column(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t field) {
    return reinterpret_cast<F*>(dsoa_block_data(c, bid) + c.col_off[t][field]);
}
template <typename F>
__device__ __forceinline__ F& dsoa_field(const dsoa_ctx& c, dsoa_obj h, uint32_t field) {
    return dsoa_column<F>(c, dsoa_h_type(h), dsoa_h_block(h), field)[dsoa_h_slot(h)];
}

/* A method may carry per-launch work that reads nothing the do-all writes:
 *   static __device__ void prologue(const dsoa_ctx&, const Args&);
 * CTA 0 of its do-all runs it (all threads of that CTA) before taking objects,
 * which spares the step a launch of its own (e.g. advancing the instances' step
 * counters in a kernel that does not read them).  A do-all on a type with
 * subtypes launches the method once per member type; the prologue runs in the
 * first of those launches only (the library marks the others with
 * DSOA_CTX_NO_PROLOGUE), so it runs once per dsoa_parallel_do. */
template <class M, class = void>
struct dsoa_has_prologue { static constexpr bool value = false; };
template <class M>
struct dsoa_has_prologue<M, decltype((void)&M::prologue, void())> { static constexpr bool value = true; };
template <class M>
__device__ __forceinline__ void dsoa_run_prologue(const dsoa_ctx& c, const typename M::Args& a) {
    if constexpr (dsoa_has_prologue<M>::value) {
        if (blockIdx.x == 0 && !(c.flags & DSOA_CTX_NO_PROLOGUE)) M::prologue(c, a);
    }
}

/* ------------------------------------------------------------------------
 * Parallel do-all kernel (Sec. 3.7, Fig. 6-7).  With G = 1 (the paper's
 * assignment) 64 consecutive threads serve one block of R: thread tid serves
 * slot tid % 64 of blocks R[(tid + k n) / 64].  With G = 2 one warp serves a
 * block, lane l taking slots l and l + 32 (two coalesced 128-byte rows).
 * Persistent: the grid is sized to the GPU and reads r from device memory,
 * so the launch does not depend on r (graph-capturable).  M provides
 *   static __device__ void run(const dsoa_ctx&, uint32_t type, uint64_t bid,
 *                              uint32_t slot, const Args&);
 * ------------------------------------------------------------------------ */
template <class M, int G = 1>
__global__ void __maxnreg__(DSOA_DOALL_MAXNREG) dsoa_doall_kernel(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                  const unsigned long long* __restrict__ occ,
                                  const uint32_t* __restrict__ r_dev, typename M::Args args) {
    constexpr uint32_t TPB = 64u / G;                          /* threads per block */
    dsoa_pdl_wait();
    dsoa_pdl_release();
    dsoa_run_prologue<M>(c, args);
    const uint64_t n = (uint64_t)gridDim.x * blockDim.x;      /* multiple of 64 */
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t s0 = (uint32_t)(tid % TPB);
    /* Under programmatic dependent launch R, the snapshot and r may have been
     * written while this grid was already resident: read them coherently then;
     * otherwise through the read-only path. */
    const bool pdl = (c.flags & DSOA_FLAG_PDL) != 0u;
    const uint64_t total = (uint64_t)(pdl ? dsoa_ld32(r_dev) : __ldg(r_dev)) * TPB;
    for (uint64_t g = tid; g < total; g += n) {
        const uint64_t i = g / TPB;
        const unsigned long long o = pdl ? dsoa_ld(&occ[i]) : __ldg(&occ[i]);
        const uint64_t bid = (uint64_t)(pdl ? dsoa_ld32(&R[i]) : __ldg(&R[i]));
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const uint32_t s = s0 + (uint32_t)k * TPB;
            if ((o >> s) & 1ull) M::run(c, t, bid, s, args);
        }
    }
}

/* ------------------------------------------------------------------------
 * User methods.  A user translation unit writes a method struct M like the
 * built-in ones (typedef Args; static __device__ run(ctx, type, block, slot,
 * args)) and names it once:
 *     DSOA_METHOD(1000, my_launcher, M)
 * which defines the extern "C" launcher (it instantiates dsoa_doall_kernel<M>
 * in the user's library and launches it with the shape the library prepared)
 * and registers it under the id when the library is loaded (the user library
 * links against libdsoa).  The registration's return code is kept in
 * `launcher##_dsoa_registered` (file scope): an id already taken by another
 * launcher stays with the first one.  The method may allocate (dsoa_new), delete `this`
 * and objects of other types, and read / write any field (dsoa_field,
 * dsoa_column), as the built-in methods do (Sec. 2.1).
 * ------------------------------------------------------------------------ */
template <class M>
inline int dsoa_launch_user_doall(const dsoa_doall_launch* L, const void* args_host, size_t args_bytes) {
    typedef typename M::Args A;
    if (!L || !L->ctx || L->ctx_bytes != sizeof(dsoa_ctx) || !args_host || args_bytes != sizeof(A))
        return DSOA_ERR_INVALID_ARG;
    dsoa_ctx c;
    memcpy(&c, L->ctx, sizeof(c));
    A a;
    memcpy(&a, args_host, sizeof(A));
    void (*k)(dsoa_ctx, uint32_t, const uint32_t*, const unsigned long long*, const uint32_t*, A) =
        L->slots_per_thread >= 2 ? &dsoa_doall_kernel<M, 2> : &dsoa_doall_kernel<M, 1>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)L->tpb, 0) != cudaSuccess)
        return DSOA_ERR_CUDA;
    if (per_sm > (int)L->max_ctas_per_sm) per_sm = (int)L->max_ctas_per_sm;
    if (per_sm < 1) per_sm = 1;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)per_sm * L->num_sms * (L->waves ? L->waves : 1u));
    cfg.blockDim = dim3(L->tpb);
    cfg.stream = (cudaStream_t)L->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = L->pdl ? 1u : 0u;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, c, (uint32_t)L->type, L->R,
                                             (const unsigned long long*)L->occ, L->r_dev, a);
    return e == cudaSuccess ? DSOA_OK : DSOA_ERR_CUDA;
}

#define DSOA_METHOD(method_id, launcher, M)                                                        \
    extern "C" int launcher(const dsoa_doall_launch* launch, const void* args, size_t args_bytes) { \
        return dsoa_launch_user_doall<M>(launch, args, args_bytes);                                 \
    }                                                                                               \
    static const int launcher##_dsoa_registered = dsoa_register_method((method_id), &launcher);

/* ------------------------------------------------------------------------
 * Streamed do-all: the enumeration of Sec. 3.7 done inside the method kernel.
 * The snapshot of a block only has to be taken before that block's objects
 * run, so a method that never creates objects of its own type (it may delete
 * `this`, and create or delete objects of other types) can enumerate and run
 * tile by tile: each CTA takes tiles of DSOA_STREAM_TILE_WORDS level-0 words
 * of allocated[t] by ticket, stages the tile's block ids and free-slot words
 * (its part of the snapshot) in shared memory, appends them to R / the
 * snapshot at a position reserved with one atomicAdd, and runs the method on
 * them.  R is not sorted (nothing depends on its order, Sec. 4.1.5 only needs
 * a list).  An object is visited only by the CTA holding its tile, so a
 * deletion of `this` cannot race with the snapshot of another tile.
 * ctl = {ticket, finished CTAs, length of R}: the last CTA to finish writes r
 * and resets ctl, so a replayed graph starts from zero.  No waits.
 * A method opts in with  static constexpr bool kNoNewOfOwnType = true;
 * ------------------------------------------------------------------------ */
#define DSOA_STREAM_TILE_WORDS 8u               /* 512 blocks per tile */

template <class M, class = void>
struct dsoa_streamable { static constexpr bool value = false; };
template <class M>
struct dsoa_streamable<M, decltype((void)M::kNoNewOfOwnType, void())> {
    static constexpr bool value = M::kNoNewOfOwnType;
};


template <class M, int G = 1>
__global__ void __maxnreg__(DSOA_DOALL_MAXNREG) dsoa_doall_stream_kernel(dsoa_ctx c, uint32_t t,
                                  uint32_t* __restrict__ R, unsigned long long* __restrict__ occ,
                                  uint32_t* __restrict__ r_dev, uint32_t* __restrict__ ctl,
                                  typename M::Args args) {
    constexpr uint32_t TW = DSOA_STREAM_TILE_WORDS, TB = 64u * TW;
    constexpr uint32_t TPB = 64u / G;                          /* threads per block */
    __shared__ uint32_t s_list[TB];
    __shared__ unsigned long long s_occ[TB];
    __shared__ unsigned long long s_word[TW];
    __shared__ uint32_t s_off[TW + 1];
    __shared__ uint32_t s_tile, s_base;
    const uint32_t b = dsoa_bm_alloc(t);
    const uint64_t w0 = c.lvl_words[0];
    const uint64_t ntiles = (w0 + TW - 1) / TW;
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint32_t tid = threadIdx.x;
    const uint32_t grp = tid / TPB, ngrp = blockDim.x / TPB, s0 = tid % TPB;
    dsoa_run_prologue<M>(c, args);
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(&ctl[0], 1u);
        __syncthreads();
        const uint64_t q = s_tile;
        if (q >= ntiles) break;                                 /* uniform */
        if (tid < TW) {
            const uint64_t wi = q * TW + tid;
            unsigned long long w = 0ull;
            if (wi < w0 && (!L1 || ((dsoa_ld(&L1[wi >> 6]) >> (wi & 63u)) & 1ull))) w = dsoa_ld(&L0[wi]);
            s_word[tid] = w;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
            for (uint32_t k = 0; k < TW; ++k) { s_off[k] = acc; acc += (uint32_t)__popcll(s_word[k]); }
            s_off[TW] = acc;
            if (acc) s_base = atomicAdd(&ctl[2], acc);
        }
        __syncthreads();
        const uint32_t n = s_off[TW];
        for (uint32_t k = tid; k < TB; k += blockDim.x) {     /* stage the tile's part of the snapshot */
            const unsigned long long w = s_word[k >> 6];
            const uint32_t bit = k & 63u;
            if ((w >> bit) & 1ull) {
                const uint32_t pos = s_off[k >> 6] + (uint32_t)__popcll(w & ((1ull << bit) - 1ull));
                const uint32_t bid = (uint32_t)(q * TB + k);
                const unsigned long long o = ~dsoa_ld(&c.slot[bid]);
                s_list[pos] = bid;
                s_occ[pos] = o;
                R[s_base + pos] = bid;
                occ[s_base + pos] = o;
            }
        }
        __syncthreads();
        for (uint32_t i = grp; i < n; i += ngrp) {
            const uint64_t bid = s_list[i];
            const unsigned long long o = s_occ[i];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const uint32_t s = s0 + (uint32_t)k * TPB;
                if ((o >> s) & 1ull) M::run(c, t, bid, s, args);
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctl[1], 1u) == gridDim.x - 1u) {      /* last CTA: publish r, reset */
            __threadfence();
            *r_dev = dsoa_ld32(&ctl[2]);
            dsoa_st32(&ctl[0], 0u);
            dsoa_st32(&ctl[2], 0u);
            dsoa_st32(&ctl[1], 0u);
        }
    }
}

/* device_do<T, f> (Sec. 2.1): run f(handle) on every object of type t, one
 * after another, in the calling thread -- the sequential for-each that n-body
 * style methods use to visit all pairs.  Walks the allocated-block bitmap of t
 * top-down (level-1 containers select level-0 containers, Sec. 4.1) and the
 * occupied slots of each block, one bit per object.  Objects created or
 * deleted concurrently may or may not be visited. */
template <typename F>
__device__ inline void dsoa_device_do(const dsoa_ctx& c, uint32_t t, F&& f) {
    const uint32_t b = dsoa_bm_alloc(t);
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint64_t w1n = L1 ? c.lvl_words[1] : 1u;
    for (uint64_t j = 0; j < w1n; ++j) {
        unsigned long long sel = L1 ? dsoa_ld(&L1[j]) : 1ull;
        for (; sel; sel &= sel - 1ull) {
            const uint64_t i = j * 64 + (uint64_t)(__ffsll((long long)sel) - 1);
            if (i >= c.lvl_words[0]) break;
            for (unsigned long long w = dsoa_ld(&L0[i]); w; w &= w - 1ull) {
                const uint64_t bid = i * 64 + (uint64_t)(__ffsll((long long)w) - 1);
                for (unsigned long long o = ~dsoa_ld(&c.slot[bid]); o; o &= o - 1ull)
                    f(dsoa_make_handle(t, bid, (uint32_t)(__ffsll((long long)o) - 1)));
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * Fused persistent do-all: enumeration and method in ONE cooperative launch.
 *   phase 1  CTA b counts the allocated blocks of its contiguous range of
 *            level-1 tiles (hierarchical skip) -> aggregate agg[b]
 *   barrier
 *   phase 2  exclusive prefix of agg below b and the total r; CTA b writes
 *            R / occupancy snapshot for its tiles (sorted, Fig. 7)
 *   barrier  (the snapshot is complete before any method runs: objects
 *            created by the method are never visited, Sec. 3.1)
 *   phase 3  the do-all loop of dsoa_doall_kernel over R
 * The grid must be co-resident (cooperative launch).  Barrier waits are
 * bounded; on the bound every CTA sets DSOA_DEV_SPIN and returns, having
 * stored r = 0 (an empty snapshot).  r is published only once the second
 * barrier shows every CTA's part of R written, so a give-up never leaves a
 * snapshot with unwritten entries for a later method to reuse.  The launcher
 * zeroes the barrier words before each launch: a give-up leaves them
 * mid-generation. 
 * ------------------------------------------------------------------------ */
__device__ inline bool dsoa_grid_sync(const dsoa_ctx& c, uint32_t nblocks) {
    uint32_t* count = c.grid_scratch + DSOA_FUSED_MAX_CTAS;
    uint32_t* gen = count + 1;
    __shared__ uint32_t s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1u;
        const uint32_t g = dsoa_ld32(gen);
        __threadfence();
        if (atomicAdd(count, 1u) == nblocks - 1u) {
            dsoa_st32(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            uint32_t spins = 0;
            while (dsoa_ld32(gen) == g) {
                if (++spins >= (DSOA_SPIN_LIMIT << 4)) { s_ok = 0u; dsoa_raise(c, DSOA_DEV_SPIN); break; }
                if (spins > 16) __nanosleep(64u);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0u;
}

template <class M, int G = 1>
__global__ void __launch_bounds__(512) dsoa_doall_fused_kernel(dsoa_ctx c, uint32_t t, uint32_t* __restrict__ R,
                                                               unsigned long long* __restrict__ occ,
                                                               uint32_t* __restrict__ r_dev, typename M::Args args) {
    __shared__ uint32_t list[4096];
    __shared__ uint32_t red[32];
    __shared__ uint32_t wsum[2];
    const uint32_t b = dsoa_bm_alloc(t);
    const uint32_t nb = gridDim.x, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    const uint64_t tiles = c.nlevels >= 2 ? c.lvl_words[1] : 1u;
    const uint64_t w0 = c.lvl_words[0];
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint64_t t_lo = tiles * blockIdx.x / nb, t_hi = tiles * (blockIdx.x + 1) / nb;
    uint32_t* agg = c.grid_scratch;
    dsoa_run_prologue<M>(c, args);
    /* phase 1: count this CTA's tiles (warp per tile) */
    uint32_t mine = 0;
    for (uint64_t tt = t_lo + warp; tt < t_hi; tt += nwarps) {
        const unsigned long long sel = L1 ? L1[tt] : 1ull;
        const uint64_t a = tt * 64 + lane, a2 = a + 32;
        uint32_t n = 0;
        if (((sel >> lane) & 1ull) && a < w0) n += __popcll(L0[a]);
        if (((sel >> (lane + 32)) & 1ull) && a2 < w0) n += __popcll(L0[a2]);
        for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
        mine += n;
    }
    if (lane == 0) red[warp] = mine;
    __syncthreads();
    if (tid == 0) {
        uint32_t sum = 0;
        for (uint32_t w = 0; w < nwarps; ++w) sum += red[w];
        dsoa_st32(&agg[blockIdx.x], sum);
    }
    if (!dsoa_grid_sync(c, nb)) {            /* gave up: publish an empty snapshot */
        if (tid == 0) dsoa_st32(r_dev, 0u);
        return;
    }
    /* phase 2: prefix of the aggregates below this CTA and the total */
    uint32_t below = 0, total = 0;
    for (uint32_t i = tid; i < nb; i += blockDim.x) {
        const uint32_t v = dsoa_ld32(&agg[i]);
        total += v;
        if (i < blockIdx.x) below += v;
    }
    for (int o = 16; o; o >>= 1) {
        below += __shfl_xor_sync(0xffffffffu, below, o);
        total += __shfl_xor_sync(0xffffffffu, total, o);
    }
    __syncthreads();
    if (lane == 0) { red[warp] = below; red[16 + warp] = total; }
    __syncthreads();
    if (tid == 0) {
        uint32_t sb = 0, st = 0;
        for (uint32_t w = 0; w < nwarps; ++w) { sb += red[w]; st += red[16 + w]; }
        red[0] = sb;
        red[1] = st;
    }
    __syncthreads();
    uint32_t base = red[0];
    const uint32_t r = red[1];
    /* compaction of this CTA's tiles, one tile at a time */
    for (uint64_t tt = t_lo; tt < t_hi; ++tt) {
        unsigned long long w = 0ull;
        if (tid < 64) {
            const unsigned long long sel = L1 ? L1[tt] : 1ull;
            const uint64_t wi = tt * 64 + tid;
            if (((sel >> tid) & 1ull) && wi < w0) w = L0[wi];
        }
        const uint32_t cnt = __popcll(w);
        uint32_t incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += v;
        }
        if (tid < 64 && lane == 31) wsum[tid >> 5] = incl;
        __syncthreads();
        const uint32_t tile_total = wsum[0] + wsum[1];
        if (tid < 64) {
            uint32_t k = incl - cnt + ((tid >= 32) ? wsum[0] : 0u);
            const uint64_t bid0 = (tt * 64 + tid) * 64;
            for (unsigned long long x = w; x; x &= x - 1ull)
                list[k++] = (uint32_t)(bid0 + (uint32_t)(__ffsll((long long)x) - 1));
        }
        __syncthreads();
        for (uint32_t i = tid; i < tile_total; i += blockDim.x) {
            const uint32_t bid = list[i];
            R[base + i] = bid;
            occ[base + i] = ~c.slot[bid];
        }
        base += tile_total;
        __syncthreads();
    }
    if (!dsoa_grid_sync(c, nb)) {
        if (tid == 0) dsoa_st32(r_dev, 0u);
        return;
    }
    /* every CTA wrote its part of R before the barrier: R is complete */
    if (blockIdx.x == 0 && tid == 0) dsoa_st32(r_dev, r);
    /* phase 3: the do-all over the snapshot */
    constexpr uint32_t TPB = 64u / G;
    const uint64_t n = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + tid;
    const uint32_t s0 = (uint32_t)(gtid % TPB);
    const uint64_t work = (uint64_t)r * TPB;
    for (uint64_t g = gtid; g < work; g += n) {
        const uint64_t i = g / TPB;
        const unsigned long long o = dsoa_ld(&occ[i]);
        const uint64_t bid = (uint64_t)dsoa_ld32(&R[i]);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const uint32_t s = s0 + (uint32_t)k * TPB;
            if ((o >> s) & 1ull) M::run(c, t, bid, s, args);
        }
    }
}

#endif /* __CUDACC__ */
#endif /* DSOA_DEVICE_CUH */
