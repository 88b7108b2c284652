// heap.cu -- heap lifecycle, layout, enumeration (bitmap scan + compaction),
// counting, invariant checking and CUDA-graph capture of the SMMO runtime.
//
// Paper map: heap of M equal blocks (Sec. 3), block bitmaps (Sec. 3.4),
// hierarchical bitmaps (Sec. 4.1), indices()/compaction into R (Sec. 3.7,
// Sec. 4.1.5, Fig. 7), fragmentation accounting (Sec. 6.4).
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include <cooperative_groups.h>

#include "dsoa_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr uint64_t kAlign = 256;
constexpr int kSmallWords = 64;  // small device scalars: err, r, done, ...

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct Layout {
    uint64_t M = 0, tiles = 0, bm_stride = 0;
    uint32_t nlevels = 0;
    uint64_t lvl_off[DSOA_MAX_LEVELS] = {0}, lvl_words[DSOA_MAX_LEVELS] = {0};
    uint64_t off_data = 0, off_slot = 0, off_btype = 0, off_drain = 0, off_bm = 0, off_R = 0, off_Rocc = 0,
             off_tcnt = 0, off_toff = 0, off_lb = 0, off_hint = 0, off_grid = 0, off_small = 0, total = 0;
    uint64_t hint_slots = 0;
};

// Hint-table slots (warp slots) per type: DSOA_HINT_SLOTS, or fewer for a heap
// of few blocks (at least 64, a power of two, about M / 4).
uint64_t hint_slots_for(uint64_t M) {
    uint64_t s = 64;
    while (s < DSOA_HINT_SLOTS && s < M / 4) s <<= 1;
    return s;
}

// Block capacity per type (Sec. 3.2): the block holds 64 objects of the
// smallest type T_s (128-byte columns), and a type T gets
// N_T = floor(64 size(T_s) / size(T)) slots, lowered until its columns (each
// 16-byte aligned, so that vector loads stay aligned) fit in that block.
// Writes the block's data bytes; fails for a type more than 64 times larger
// than T_s (the limitation the paper states).
int per_type_capacity(dsoa_heap* h, uint32_t* block_bytes_out) {
    int s = 0;
    uint32_t size_s = ~0u;
    for (int t = 0; t < h->ntypes; ++t) {
        uint32_t size = 0;
        for (int f = 0; f < h->types[t].nfields; ++f) size += h->types[t].field_bytes[f];
        if (size < size_s || (size == size_s && h->types[t].data_bytes < h->types[s].data_bytes)) {
            size_s = size;
            s = t;
        }
    }
    const uint32_t block = std::max<uint32_t>(128, h->types[s].data_bytes);
    for (int t = 0; t < h->ntypes; ++t) {
        dsoa_type_info& ti = h->types[t];
        uint32_t size = 0;
        for (int f = 0; f < ti.nfields; ++f) size += ti.field_bytes[f];
        uint32_t n = std::min<uint32_t>(64, 64u * size_s / size);
        for (; n > 0; --n) {
            uint32_t off = 0;
            for (int f = 0; f < ti.nfields; ++f)
                off += (uint32_t)(n == 64 ? align_up(64ull * ti.field_bytes[f], 128)
                                          : align_up((uint64_t)n * ti.field_bytes[f], 16));
            if (off <= block) break;
        }
        if (n == 0) return DSOA_ERR_INVALID_ARG;
        uint32_t off = 0;
        for (int f = 0; f < ti.nfields; ++f) {
            ti.col_off[f] = off;
            off += (uint32_t)(n == 64 ? align_up(64ull * ti.field_bytes[f], 128)
                                      : align_up((uint64_t)n * ti.field_bytes[f], 16));
        }
        ti.data_bytes = off;
        ti.capacity = n;
    }
    *block_bytes_out = block;
    return DSOA_OK;
}

bool make_layout(uint64_t M, uint32_t block_bytes, int ntypes, Layout* L) {
    const int nbm = 1 + 2 * ntypes;
    if (M == 0) return false;
    L->M = M;
    uint64_t words = (M + 63) / 64;
    uint32_t nl = 0;
    uint64_t off = 0;
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
    L->bm_stride = align_up(off, kAlign / 8);
    L->tiles = nl >= 2 ? L->lvl_words[1] : 1;
    uint64_t p = 0;
    L->off_data = p;  p = align_up(p + M * block_bytes, kAlign);
    L->off_slot = p;  p = align_up(p + M * 8, kAlign);
    L->off_btype = p; p = align_up(p + M * 4, kAlign);
    L->off_drain = p; p = align_up(p + M, kAlign);
    L->off_bm = p;    p = align_up(p + (uint64_t)nbm * L->bm_stride * 8, kAlign);
    L->off_R = p;     p = align_up(p + M * 4 * (uint64_t)ntypes, kAlign);
    L->off_Rocc = p;  p = align_up(p + M * 8 * (uint64_t)ntypes, kAlign);
    L->off_tcnt = p;  p = align_up(p + L->tiles * 4, kAlign);
    L->off_toff = p;  p = align_up(p + L->tiles * 4, kAlign);
    L->off_lb = p;    p = align_up(p + L->tiles * 8 * (uint64_t)ntypes + 16 * (uint64_t)ntypes, kAlign);
    L->hint_slots = hint_slots_for(M);
    L->off_hint = p;  p = align_up(p + L->hint_slots * (uint64_t)ntypes * sizeof(dsoa_hint), kAlign);
    L->off_grid = p;  p = align_up(p + (uint64_t)DSOA_GRID_SCRATCH * 4, kAlign);
    L->off_small = p; p = align_up(p + kSmallWords * 8, kAlign);
    L->total = p;
    return true;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Consistent "every block free" state of the free-block bitmap: bit i of level
// l is set iff i < (number of bits at level l).
__global__ void k_init_free(dsoa_ctx c) {
    uint64_t total = 0;
    for (uint32_t l = 0; l < c.nlevels; ++l) total += c.lvl_words[l];
    unsigned long long* bm = c.bm;  // bitmap 0 = free
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = g;
        uint32_t l = 0;
        while (i >= c.lvl_words[l]) { i -= c.lvl_words[l]; ++l; }
        const uint64_t nbits = l == 0 ? c.M : c.lvl_words[l - 1];
        const uint64_t lo = i * 64, hi = std::min<uint64_t>(lo + 64, nbits);
        const uint64_t k = hi - lo;
        bm[c.lvl_off[l] + i] = k >= 64 ? DSOA_ALL : ((1ull << k) - 1ull);
    }
}

// Enumeration, kernel 1 (Alg. 5 "indices", counting half): one warp per
// level-1 container ("tile" of 64 level-0 containers = 4096 blocks).  Only
// level-0 containers whose level-1 bit is set are read (hierarchical skip,
// Sec. 4.1.5).  The last CTA to finish turns the tile counts into exclusive
// offsets (prefix sum, Fig. 7) and writes r.
__global__ void k_tile_count(dsoa_ctx c, uint32_t b, uint64_t tiles, uint32_t* __restrict__ tcnt,
                             uint32_t* __restrict__ toff, uint32_t* __restrict__ r_dev,
                             uint32_t* __restrict__ done) {
    dsoa_pdl_wait();
    dsoa_pdl_release();
    const uint32_t lane = threadIdx.x & 31u, wpc = blockDim.x >> 5;
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint64_t w0 = c.lvl_words[0];
    for (uint64_t t = (uint64_t)blockIdx.x * wpc + (threadIdx.x >> 5); t < tiles;
         t += (uint64_t)gridDim.x * wpc) {
        const unsigned long long sel = L1 ? L1[t] : 1ull;
        uint32_t cnt = 0;
        const uint64_t a = t * 64 + lane, bb = a + 32;
        if (((sel >> lane) & 1ull) && a < w0) cnt += __popcll(L0[a]);
        if (((sel >> (lane + 32)) & 1ull) && bb < w0) cnt += __popcll(L0[bb]);
        cnt = warp_sum(cnt);
        if (lane == 0) tcnt[t] = cnt;
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of tcnt[0..tiles) by this CTA
    __shared__ uint32_t part[1024];
    const uint64_t per = (tiles + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = threadIdx.x * per, hi = std::min<uint64_t>(lo + per, tiles);
    uint32_t s = 0;
    for (uint64_t i = lo; i < hi; ++i) s += __ldcg(&tcnt[i]);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t i = 0; i < blockDim.x; ++i) { const uint32_t v = part[i]; part[i] = run; run += v; }
        *r_dev = run;
        *done = 0u;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) { toff[i] = run; run += __ldcg(&tcnt[i]); }
}

// Enumeration, kernel 2 (compaction + iteration-bitmap snapshot, Sec. 3.1 and
// Fig. 7): 64 threads per tile; thread j owns level-0 container 64t+j; a
// CTA-local prefix sum gives each set bit its rank; block ids are staged in
// shared memory and written out coalesced together with the snapshot of the
// block's occupied slots (the complement of its free-slot word).
template <int TPC>
__global__ void __launch_bounds__(64 * TPC) k_compact(dsoa_ctx c, uint32_t b, uint64_t tiles,
                                                      const uint32_t* __restrict__ toff,
                                                      uint32_t* __restrict__ R,
                                                      unsigned long long* __restrict__ Rocc) {
    dsoa_pdl_wait();
    dsoa_pdl_release();
    __shared__ uint32_t list[TPC][4096];
    __shared__ uint32_t wsum[TPC][2];
    const uint32_t tl = threadIdx.x >> 6, j = threadIdx.x & 63u, lane = threadIdx.x & 31u;
    const uint64_t t = (uint64_t)blockIdx.x * TPC + tl;
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    unsigned long long w = 0ull;
    if (t < tiles) {
        const unsigned long long sel = c.nlevels >= 2 ? dsoa_level(c, b, 1)[t] : 1ull;
        const uint64_t wi = t * 64 + j;
        if (((sel >> j) & 1ull) && wi < c.lvl_words[0]) w = L0[wi];
    }
    const uint32_t cnt = __popcll(w);
    uint32_t incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    if (lane == 31) wsum[tl][j >> 5] = incl;
    __syncthreads();
    const uint32_t excl = incl - cnt + ((j >= 32) ? wsum[tl][0] : 0u);
    const uint32_t tile_total = wsum[tl][0] + wsum[tl][1];
    const uint64_t bid0 = (t * 64 + j) * 64;
    uint32_t k = excl;
    for (unsigned long long x = w; x; x &= x - 1ull) list[tl][k++] = (uint32_t)(bid0 + (uint32_t)(__ffsll((long long)x) - 1));
    __syncthreads();
    if (t >= tiles) return;
    const uint32_t base = toff[t];
    for (uint32_t i = j; i < tile_total; i += 64) {
        const uint32_t bid = list[tl][i];
        R[base + i] = bid;
        Rocc[base + i] = ~c.slot[bid];
    }
}

// Single-pass enumeration (decoupled look-back, Merrill & Garland 2016): one
// 64-thread CTA per level-1 tile (64 level-0 words).  The CTA reads its tile's
// level-0 words (the enumeration runs between kernels, when a level-0 word is
// non-zero iff its level-1 bit is set, so the level-1 word need not be read
// first), publishes the tile's aggregate, and then warp 0 walks back over its
// predecessors' published aggregates / inclusive prefixes 32 at a time while
// warp 1 reads the tile's free-slot words (the snapshot, up to 2048 of them)
// into shared memory.
// The CTA publishes its inclusive prefix and writes R and the snapshot.
// Tile order: when every tile's CTA fits on the GPU at once, the tile is
// blockIdx.x (CTAs are dispatched in index order, so a CTA only waits on
// tiles of CTAs that already run); otherwise a ticket counter hands tiles out
// in the order the CTAs start.  State words carry the enumeration's epoch, so
// nothing is reset between launches (safe in graph replays); the last CTA to
// finish advances the epoch and resets the ticket.  A published value is only
// ever read as itself, so no fence precedes it.  Every wait is bounded
// (DSOA_DEV_SPIN).  A tile whose look-back gives up still finishes (its
// under-counted prefix keeps every write below the true end of R, so all
// writes stay in bounds) and marks the epoch failed; the CTA that closes a
// failed epoch publishes r = 0, so no method ever runs on, or later reuses,
// a block list with misplaced entries.
constexpr unsigned long long kLbA = 1ull, kLbP = 2ull;
__device__ __forceinline__ unsigned long long lb_word(uint32_t ep, unsigned long long st, unsigned long long v) {
    return ((unsigned long long)(ep & 0xFFFFFFu) << 40) | (st << 38) | (v & ((1ull << 38) - 1ull));
}

// Several types can be enumerated by one launch (each type's snapshot taken at
// the same point): CTAs [q * tiles, (q + 1) * tiles) serve the q-th type of the
// batch, with that type's own look-back state, ticket and epoch.
struct EnumBatch {
    uint32_t n;                                   // types in the batch
    uint32_t b[DSOA_MAX_TYPES];                   // allocated-bitmap index of each
    uint32_t* R[DSOA_MAX_TYPES];
    unsigned long long* Rocc[DSOA_MAX_TYPES];
    uint32_t* r_dev[DSOA_MAX_TYPES];
    unsigned long long* state[DSOA_MAX_TYPES];    // [tiles] look-back state words
    uint32_t* ctl[DSOA_MAX_TYPES];                // ticket, done, epoch, failed
};

__global__ void __launch_bounds__(64) k_enum_lookback(dsoa_ctx c, uint64_t tiles, EnumBatch eb,
                                                      uint32_t use_ticket) {
    __shared__ uint32_t list[4096];
    const uint32_t qt = (uint32_t)(blockIdx.x / tiles);          /* the batch's type slot */
    const uint32_t b = eb.b[qt];
    unsigned long long* __restrict__ state = eb.state[qt];
    uint32_t* __restrict__ ctl = eb.ctl[qt];
    uint32_t* __restrict__ R = eb.R[qt];
    unsigned long long* __restrict__ Rocc = eb.Rocc[qt];
    uint32_t* __restrict__ r_dev = eb.r_dev[qt];
    constexpr uint32_t kSnap = 2048;                 /* snapshot words staged by warp 1 */
    __shared__ unsigned long long snap[kSnap];
    __shared__ uint32_t wsum[2];
    __shared__ uint32_t s_tile, s_ep;
    __shared__ unsigned long long s_prefix;
    uint32_t* ticket = ctl;
    uint32_t* done = ctl + 1;
    uint32_t* epoch = ctl + 2;
    uint32_t* failed = ctl + 3;
    const uint32_t j = threadIdx.x, lane = j & 31u;
    dsoa_pdl_wait();
    dsoa_pdl_release();
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const uint64_t w0 = c.lvl_words[0];
    uint64_t t;
    unsigned long long w = 0ull;
    if (use_ticket) {
        if (j == 0) {
            s_tile = atomicAdd(ticket, 1u);
            s_ep = dsoa_ld32(epoch) + 1u;
        }
        __syncthreads();
        t = s_tile;
        if (t * 64 + j < w0) w = L0[t * 64 + j];
    } else {
        t = blockIdx.x - (uint64_t)qt * tiles;
        if (t * 64 + j < w0) w = L0[t * 64 + j];              /* in flight with the epoch read */
        if (j == 0) s_ep = dsoa_ld32(epoch) + 1u;
        __syncthreads();
    }
    const uint32_t ep = s_ep;
    const uint64_t wi = t * 64 + j;
    const uint32_t cnt = __popcll(w);
    uint32_t incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    if (lane == 31) wsum[j >> 5] = incl;
    __syncthreads();
    const uint32_t total = wsum[0] + wsum[1];
    /* publish this tile's aggregate (or its prefix, for tile 0) as early as possible */
    if (j == 0) dsoa_st(&state[t], lb_word(ep, t == 0 ? kLbP : kLbA, total));
    /* stage this tile's block ids */
    {
        uint32_t k = incl - cnt + ((j >= 32) ? wsum[0] : 0u);
        const uint64_t bid0 = wi * 64;
        for (unsigned long long x = w; x; x &= x - 1ull)
            list[k++] = (uint32_t)(bid0 + (uint32_t)(__ffsll((long long)x) - 1));
    }
    __syncthreads();
    if (j < 32) {
        /* warp 0: look back over the predecessors */
        unsigned long long prefix = 0ull;
        bool ok = true;
        if (t > 0) {
            int64_t base = (int64_t)t - 1;
            for (;;) {
                const int64_t q = base - (int64_t)lane;
                unsigned long long sw = 0ull;
                uint32_t spins = 0;
                if (q >= 0) {
                    for (;;) {
                        sw = dsoa_ld(&state[q]);
                        if ((uint32_t)(sw >> 40) == (ep & 0xFFFFFFu) && ((sw >> 38) & 3ull)) break;
                        if (++spins >= DSOA_SPIN_LIMIT) { ok = false; break; }
                        if (spins > 8) __nanosleep(32u);
                    }
                }
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                const bool isP = q >= 0 && ((sw >> 38) & 3ull) == kLbP;
                const uint32_t pmask = __ballot_sync(0xffffffffu, isP);
                const uint32_t stop = pmask ? (uint32_t)(__ffs((int)pmask) - 1) : 32u;   /* nearest P */
                unsigned long long v = (q >= 0 && lane <= stop) ? (sw & ((1ull << 38) - 1ull)) : 0ull;
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                prefix += v;
                if (pmask || base - 32 < 0) break;
                base -= 32;
            }
        }
        if (j == 0) {
            if (!ok) {
                dsoa_raise(c, DSOA_DEV_SPIN);
                atomicOr(failed, 1u);
            }
            s_prefix = prefix;
            if (t > 0) dsoa_st(&state[t], lb_word(ep, kLbP, prefix + total));
            if (t == tiles - 1) *r_dev = (uint32_t)(prefix + total);
        }
    } else {
        /* warp 1, meanwhile: the tile's part of the snapshot */
        for (uint32_t i = lane; i < total && i < kSnap; i += 32) snap[i] = ~c.slot[list[i]];
    }
    __syncthreads();
    const unsigned long long base = s_prefix;
    for (uint32_t i = j; i < total; i += 64) {
        const uint32_t bid = list[i];
        R[base + i] = bid;
        Rocc[base + i] = i < kSnap ? snap[i] : ~c.slot[bid];
    }
    /* the last CTA to finish closes the epoch */
    __syncthreads();
    if (j == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == (uint32_t)tiles - 1u) {
            __threadfence();
            if (dsoa_ld32(failed)) {         /* a tile gave up: empty snapshot */
                dsoa_st32(r_dev, 0u);
                dsoa_st32(failed, 0u);
            }
            dsoa_st32(ticket, 0u);
            dsoa_st32(done, 0u);
            __threadfence();
            dsoa_st32(epoch, ep);
        }
    }
}

// The same enumeration for heaps whose tiles do not fit on the GPU as one
// resident wave of CTAs: each CTA takes G consecutive level-1 tiles (G <=
// kEnumGMax), publishes the aggregate of all of them and looks back over the
// preceding CTAs of its type (so every CTA of the launch is resident and the
// CTA index orders the chain); it then writes its tiles' blocks in order, one
// tile of block ids staged in shared memory at a time.  R stays sorted.
constexpr uint32_t kEnumGMax = 16;

__global__ void __launch_bounds__(64) k_enum_lookback_multi(dsoa_ctx c, uint64_t tiles, uint32_t G, uint32_t ctas,
                                                            EnumBatch eb) {
    __shared__ uint32_t list[4096];
    __shared__ uint32_t tsum[kEnumGMax][2];
    __shared__ uint32_t s_ep;
    __shared__ unsigned long long s_prefix;
    const uint32_t qt = blockIdx.x / ctas;
    const uint32_t cta = blockIdx.x - qt * ctas;
    const uint32_t b = eb.b[qt];
    unsigned long long* __restrict__ state = eb.state[qt];
    uint32_t* __restrict__ ctl = eb.ctl[qt];
    uint32_t* __restrict__ R = eb.R[qt];
    unsigned long long* __restrict__ Rocc = eb.Rocc[qt];
    uint32_t* __restrict__ r_dev = eb.r_dev[qt];
    uint32_t* ticket = ctl;
    uint32_t* done = ctl + 1;
    uint32_t* epoch = ctl + 2;
    uint32_t* failed = ctl + 3;
    const uint32_t j = threadIdx.x, lane = j & 31u, warp = j >> 5;
    dsoa_pdl_wait();
    dsoa_pdl_release();
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const uint64_t w0 = c.lvl_words[0];
    const uint64_t t0 = (uint64_t)cta * G;
    unsigned long long w[kEnumGMax];
#pragma unroll
    for (uint32_t g = 0; g < kEnumGMax; ++g) {
        const uint64_t wi = (t0 + g) * 64 + j;
        w[g] = (g < G && t0 + g < tiles && wi < w0) ? L0[wi] : 0ull;
    }
    if (j == 0) s_ep = dsoa_ld32(epoch) + 1u;
    uint32_t excl[kEnumGMax];
#pragma unroll
    for (uint32_t g = 0; g < kEnumGMax; ++g) {
        const uint32_t cnt = (uint32_t)__popcll(w[g]);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += v;
        }
        excl[g] = incl - cnt;
        if (lane == 31u && g < G) tsum[g][warp] = incl;
    }
    __syncthreads();
    const uint32_t ep = s_ep;
    unsigned long long agg = 0ull;
    for (uint32_t g = 0; g < G; ++g) agg += tsum[g][0] + tsum[g][1];
    if (j == 0) dsoa_st(&state[cta], lb_word(ep, cta == 0 ? kLbP : kLbA, agg));
    if (j < 32) {
        /* warp 0: look back over the preceding CTAs of this type */
        unsigned long long prefix = 0ull;
        bool ok = true;
        if (cta > 0) {
            int64_t base = (int64_t)cta - 1;
            for (;;) {
                const int64_t q = base - (int64_t)lane;
                unsigned long long sw = 0ull;
                uint32_t spins = 0;
                if (q >= 0) {
                    for (;;) {
                        sw = dsoa_ld(&state[q]);
                        if ((uint32_t)(sw >> 40) == (ep & 0xFFFFFFu) && ((sw >> 38) & 3ull)) break;
                        if (++spins >= DSOA_SPIN_LIMIT) { ok = false; break; }
                        if (spins > 8) __nanosleep(32u);
                    }
                }
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                const bool isP = q >= 0 && ((sw >> 38) & 3ull) == kLbP;
                const uint32_t pmask = __ballot_sync(0xffffffffu, isP);
                const uint32_t stop = pmask ? (uint32_t)(__ffs((int)pmask) - 1) : 32u;
                unsigned long long v = (q >= 0 && lane <= stop) ? (sw & ((1ull << 38) - 1ull)) : 0ull;
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                prefix += v;
                if (pmask || base - 32 < 0) break;
                base -= 32;
            }
        }
        if (j == 0) {
            if (!ok) {
                dsoa_raise(c, DSOA_DEV_SPIN);
                atomicOr(failed, 1u);
            }
            s_prefix = prefix;
            if (cta > 0) dsoa_st(&state[cta], lb_word(ep, kLbP, prefix + agg));
            if (cta == ctas - 1) *r_dev = (uint32_t)(prefix + agg);
        }
    }
    __syncthreads();
    unsigned long long base = s_prefix;
#pragma unroll
    for (uint32_t g = 0; g < kEnumGMax; ++g) {
        if (g >= G) break;                                   /* uniform */
        const uint32_t total = tsum[g][0] + tsum[g][1];
        uint32_t k = excl[g] + (warp ? tsum[g][0] : 0u);
        const uint64_t bid0 = ((t0 + g) * 64 + j) * 64;
        for (unsigned long long x = w[g]; x; x &= x - 1ull)
            list[k++] = (uint32_t)(bid0 + (uint32_t)(__ffsll((long long)x) - 1));
        __syncthreads();
        for (uint32_t i = j; i < total; i += 64) {
            const uint32_t bid = list[i];
            R[base + i] = bid;
            Rocc[base + i] = ~c.slot[bid];
        }
        base += total;
        __syncthreads();
    }
    /* the last CTA of the type to finish closes the epoch */
    if (j == 0) {
        __threadfence();
        if (atomicAdd(done, 1u) == ctas - 1u) {
            __threadfence();
            if (dsoa_ld32(failed)) {         /* a CTA gave up: empty snapshot */
                dsoa_st32(r_dev, 0u);
                dsoa_st32(failed, 0u);
            }
            dsoa_st32(ticket, 0u);
            dsoa_st32(done, 0u);
            __threadfence();
            dsoa_st32(epoch, ep);
        }
    }
}

// Enumeration by a thread-block cluster per type (scan_tiles = 5; not in the
// paper): kEnumCl CTAs of 1024 threads split the level-0 words of the type's
// allocated-block bitmap into contiguous ranges, in order.  Each CTA scans the
// popcounts of its range in shared memory; after a cluster barrier every CTA
// reads the totals of the CTAs before it from their shared memory
// (distributed shared memory), which gives its first position in R; a second
// barrier keeps every CTA's shared memory alive until all have read it.  The
// CTA then stages its block ids in shared memory and writes them with the
// snapshot words, four per thread in flight.  The cluster is co-scheduled by
// the hardware, so no CTA waits on one that has not started, and nothing
// spins.  For heaps of at most kEnumCl * 1024 * kEnumClK level-0 words.
constexpr uint32_t kEnumCl = 8, kEnumClThreads = 1024, kEnumClK = 8;
constexpr uint64_t kEnumClWords = (uint64_t)kEnumCl * kEnumClThreads * kEnumClK;   // 65,536 words
constexpr uint32_t kEnumClChunk = 4096;

__global__ void __launch_bounds__(1024, 1) k_enum_cluster(dsoa_ctx c, EnumBatch eb) {
    __shared__ uint32_t list[kEnumClChunk];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_tot;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t rank = cl.block_rank();
    const uint32_t q = blockIdx.x / kEnumCl;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t b = eb.b[q];
    uint32_t* __restrict__ R = eb.R[q];
    unsigned long long* __restrict__ Rocc = eb.Rocc[q];
    dsoa_pdl_wait();
    dsoa_pdl_release();
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const uint64_t w0 = c.lvl_words[0];
    const uint64_t per_cta = (w0 + kEnumCl - 1) / kEnumCl;
    const uint64_t lo = (uint64_t)rank * per_cta;
    const uint64_t hi = lo + per_cta < w0 ? lo + per_cta : w0;
    const uint64_t per_thr = (per_cta + kEnumClThreads - 1) / kEnumClThreads;   /* <= kEnumClK */
    const uint64_t first = lo + (uint64_t)tid * per_thr;
    unsigned long long w[kEnumClK];
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t k = 0; k < kEnumClK; ++k) {
        const uint64_t i = first + k;
        w[k] = (k < per_thr && i < hi) ? L0[i] : 0ull;
        cnt += (uint32_t)__popcll(w[k]);
    }
    uint32_t incl = cnt;                                    /* CTA-wide exclusive scan */
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    if (lane == 31u) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = wsum[lane];
        uint32_t y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= (uint32_t)o) y += v;
        }
        wsum[lane] = y - x;
        if (lane == 31u) s_tot = y;                         /* this CTA's blocks */
    }
    cl.sync();                                              /* every CTA's total is in place */
    __shared__ uint32_t s_base;
    if (tid == 0) {
        uint32_t base = 0;
        for (uint32_t r = 0; r < rank; ++r) base += *cl.map_shared_rank(&s_tot, r);
        s_base = base;
        if (rank == kEnumCl - 1u) *eb.r_dev[q] = base + s_tot;
    }
    cl.sync();                                              /* remote reads done before any CTA leaves */
    const uint32_t cta_base = s_base, cta_n = s_tot;
    const uint32_t mine = wsum[warp] + incl - cnt;          /* position within this CTA's part */
    for (uint32_t chunk0 = 0; chunk0 < cta_n; chunk0 += kEnumClChunk) {
        if (cnt && mine < chunk0 + kEnumClChunk && mine + cnt > chunk0) {
            uint32_t pos = mine;
#pragma unroll
            for (uint32_t k = 0; k < kEnumClK; ++k) {
                const uint64_t bid0 = (first + k) * 64u;
                for (unsigned long long x = w[k]; x; x &= x - 1ull, ++pos)
                    if (pos >= chunk0 && pos < chunk0 + kEnumClChunk)
                        list[pos - chunk0] = (uint32_t)(bid0 + (uint32_t)(__ffsll((long long)x) - 1));
            }
        }
        __syncthreads();
        const uint32_t n = cta_n - chunk0 < kEnumClChunk ? cta_n - chunk0 : kEnumClChunk;
        for (uint32_t i0 = 0; i0 < n; i0 += 4u * kEnumClThreads) {
            uint32_t id[4];
            unsigned long long o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {                   /* four snapshot loads in flight */
                const uint32_t i = i0 + (uint32_t)u * kEnumClThreads + tid;
                id[u] = i < n ? list[i] : 0u;
                o[u] = i < n ? ~c.slot[id[u]] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t i = i0 + (uint32_t)u * kEnumClThreads + tid;
                if (i < n) {
                    R[cta_base + chunk0 + i] = id[u];
                    Rocc[cta_base + chunk0 + i] = o[u];
                }
            }
        }
        __syncthreads();
    }
}

// Live objects of one type: warp per tile; for every non-empty level-0
// container the warp reads the 64 slot words coalesced.
// Live objects of several types in one launch, stored to out[q]: one warp per
// level-0 word of a type's allocated-block bitmap (a word that is zero costs one
// load), its lanes popcount the slot words of the word's blocks (two each) in
// parallel, so the two dependent loads of every word run concurrently across the
// grid.  Counts meet in shared memory, then in acc (one atomic per CTA and
// type); the CTA that finishes last stores the totals to out and leaves acc and
// the ticket at zero for the next launch.  Plain stores to out, no pre-zeroing:
// out may be device memory or mapped pinned host memory.
struct CountBatch {
    uint32_t n;
    uint32_t b[DSOA_MAX_TYPES];
};
__global__ void k_count_many(dsoa_ctx c, CountBatch cb, unsigned long long* out, unsigned long long* acc,
                             uint32_t* ticket) {
    __shared__ unsigned long long s_cnt[DSOA_MAX_TYPES];
    __shared__ bool s_last;
    const uint32_t lane = threadIdx.x & 31u, wpc = blockDim.x >> 5;
    if (threadIdx.x < DSOA_MAX_TYPES) s_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    const uint64_t words = c.lvl_words[0], total = words * cb.n;
    uint32_t q_cur = 0, cnt = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * wpc + (threadIdx.x >> 5); g < total; g += (uint64_t)gridDim.x * wpc) {
        const uint32_t q = (uint32_t)(g / words);
        const uint64_t wi = g - (uint64_t)q * words;
        if (q != q_cur) {                          /* warp-uniform */
            cnt = warp_sum(cnt);
            if (lane == 0 && cnt) atomicAdd(&s_cnt[q_cur], (unsigned long long)cnt);
            q_cur = q;
            cnt = 0;
        }
        const unsigned long long w = dsoa_level(c, cb.b[q], 0)[wi];
        const uint64_t bid = wi * 64 + lane;
        if ((w >> lane) & 1ull) cnt += __popcll(~c.slot[bid]);
        if ((w >> (lane + 32)) & 1ull) cnt += __popcll(~c.slot[bid + 32]);
    }
    cnt = warp_sum(cnt);
    if (lane == 0 && cnt) atomicAdd(&s_cnt[q_cur], (unsigned long long)cnt);
    __syncthreads();
    if (threadIdx.x < cb.n && s_cnt[threadIdx.x]) atomicAdd(&acc[threadIdx.x], s_cnt[threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < cb.n) out[threadIdx.x] = atomicExch(&acc[threadIdx.x], 0ull);
    if (threadIdx.x == 0) atomicExch(ticket, 0u);
}

__global__ void k_popc_level0(dsoa_ctx c, uint32_t b, unsigned long long* out) {
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    uint32_t cnt = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.lvl_words[0];
         i += (uint64_t)gridDim.x * blockDim.x)
        cnt += __popcll(L0[i]);
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31u) == 0 && cnt) atomicAdd(out, (unsigned long long)cnt);
}

__device__ __forceinline__ bool bit_at(const unsigned long long* L, uint64_t i) {
    return (L[i >> 6] >> (i & 63u)) & 1ull;
}

// Invariant checker (Sec. 3.4 bitmap semantics, App. A.4 consistency).
__global__ void k_check(dsoa_ctx c, unsigned long long* v) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nbm = 1u + 2u * c.ntypes;
    unsigned long long loc[DSOA_CHECK_COUNT] = {0};
    // per-block state
    for (uint64_t bid = tid; bid < c.M; bid += stride) {
        const bool f = bit_at(dsoa_level(c, dsoa_bm_free(), 0), bid);
        uint32_t nalloc = 0, talloc = 0;
        for (uint32_t t = 0; t < c.ntypes; ++t) {
            const bool a = bit_at(dsoa_level(c, dsoa_bm_alloc(t), 0), bid);
            const bool act = bit_at(dsoa_level(c, dsoa_bm_active(t), 0), bid);
            if (a) { ++nalloc; talloc = t; }
            if (act && !a) loc[DSOA_CHECK_ACTIVE_SUBSET]++;
        }
        const unsigned long long w = c.slot[bid];
        if (nalloc > 1) loc[DSOA_CHECK_MULTI_TYPE]++;
        if (f == (nalloc > 0)) loc[DSOA_CHECK_FREE_XOR]++;
        if (f && w != 0ull) loc[DSOA_CHECK_FREE_WORD]++;
        if (nalloc == 1) {
            if (c.btype[bid] != talloc) loc[DSOA_CHECK_TYPE]++;
            if (w == DSOA_ALL) loc[DSOA_CHECK_EMPTY_ALLOC]++;
            const bool act = bit_at(dsoa_level(c, dsoa_bm_active(talloc), 0), bid);
            if (act != ((w & c.cap[talloc]) != 0ull)) loc[DSOA_CHECK_ACTIVE_EXACT]++;
            if (~w & ~c.cap[talloc]) loc[DSOA_CHECK_CAP_BITS]++;
        }
    }
    // hierarchy consistency and tail bits, every bitmap and level
    for (uint32_t b = 0; b < nbm; ++b) {
        for (uint32_t l = 0; l < c.nlevels; ++l) {
            const unsigned long long* Ll = dsoa_level(c, b, l);
            const uint64_t nbits = l == 0 ? c.M : c.lvl_words[l - 1];
            for (uint64_t i = tid; i < c.lvl_words[l]; i += stride) {
                const unsigned long long w = Ll[i];
                const uint64_t lo = i * 64;
                if (lo + 64 > nbits) {
                    const uint64_t k = nbits - lo;
                    if (w & ~((1ull << k) - 1ull)) loc[DSOA_CHECK_TAIL_BITS]++;
                }
                if (l > 0) {
                    const unsigned long long* Lb = dsoa_level(c, b, l - 1);
                    for (uint32_t k = 0; k < 64 && lo + k < nbits; ++k) {
                        const bool up = (w >> k) & 1ull;
                        if (up != (Lb[lo + k] != 0ull)) loc[DSOA_CHECK_HIER]++;
                    }
                }
            }
        }
    }
    for (int i = 0; i < DSOA_CHECK_COUNT; ++i)
        if (loc[i]) atomicAdd(&v[i], loc[i]);
}

__global__ void k_delete_handles(dsoa_ctx c, const dsoa_obj* __restrict__ hs, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dsoa_delete(c, hs[i]);
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

int init_heap(dsoa_heap* h, void* base, size_t bytes, bool owns, void* stream) {
    h->base = base;
    h->bytes = bytes;
    h->owns = owns;
    h->stream = (cudaStream_t)stream;
    DSOA_CUDA_TRY(cudaGetDevice(&h->device));
    DSOA_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    std::memset(&h->ctx, 0, sizeof(h->ctx));
    return DSOA_OK;
}

}  // namespace

// ------------------------------------------------------------------------
// helpers used by the application translation units
// ------------------------------------------------------------------------
int dsoa_check_launch(dsoa_heap* h) {
    h->launches++;
    return cudaGetLastError() == cudaSuccess ? DSOA_OK : DSOA_ERR_CUDA;
}

dsoa_ctx dsoa_launch_ctx(dsoa_heap* h) {
    dsoa_ctx c = h->ctx;
    c.seed = 0x9E3779B9u * (++h->launch_seq);
    c.flags = h->flags | (h->skip_prologue ? DSOA_CTX_NO_PROLOGUE : 0u);
    c.lookups = h->lookups;
    return c;
}

int dsoa_resident_ctas(const void* kernel, int tpb) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(kernel, tpb * 1024 + dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, tpb, 0) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

unsigned dsoa_doall_grid(dsoa_heap* h) {
    return (unsigned)std::max(1, h->num_sms * h->doall_ctas_per_sm);
}

unsigned dsoa_new_grid(dsoa_heap* h, uint64_t n, int tpb) {
    const uint64_t need = (n + tpb - 1) / tpb;
    const uint64_t cap = (uint64_t)h->num_sms * (2048 / tpb);
    return (unsigned)std::max<uint64_t>(1, std::min(need, cap));
}

int dsoa_ensure_frozen(dsoa_heap* h) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_OK;
    return dsoa_heap_freeze(h);
}

// One look-back launch for n types (validated by the caller).
static int enumerate_lookback(dsoa_heap* h, const int* types, int n) {
    if (h->lb_fits < 0) {              // CTAs of k_enum_lookback resident per SM
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_enum_lookback, 64, 0);
        h->lb_fits = per_sm;
    }
    // tile = blockIdx when every CTA of the launch is resident at once
    const uint64_t cap = (uint64_t)h->lb_fits * (uint64_t)h->num_sms;
    const bool fits = cap >= h->tiles * (uint64_t)n;
    EnumBatch eb;
    std::memset(&eb, 0, sizeof(eb));
    eb.n = (uint32_t)n;
    for (int q = 0; q < n; ++q) {
        const int t = types[q];
        eb.b[q] = dsoa_bm_alloc((uint32_t)t);
        eb.R[q] = h->R[t];
        eb.Rocc[q] = h->Rocc[t];
        eb.r_dev[q] = h->r_dev[t];
        eb.state[q] = h->lb_state + (uint64_t)t * h->tiles;
        eb.ctl[q] = h->lb_ctl + 4 * t;
    }
    int rc;
    const bool tickets = (h->flags & DSOA_FLAG_ENUM_TICKETS) != 0u;
    if (h->cluster_enum && h->ctx.lvl_words[0] <= kEnumClWords) {
        // a cluster of kEnumCl CTAs per type (scan_tiles = 5)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)n * kEnumCl);
        cfg.blockDim = dim3(kEnumClThreads);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kEnumCl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = (h->flags & DSOA_FLAG_PDL) ? 2u : 1u;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_enum_cluster, h->ctx, eb);
        h->launches++;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return DSOA_ERR_CUDA;
        }
        for (int q = 0; q < n; ++q) h->enumerated[types[q]] = true;
        return DSOA_OK;
    }
    if (!fits && !tickets) {
        // several tiles per CTA, so that the whole launch is resident (else tickets)
        static int multi_per_sm = -1;
        if (multi_per_sm < 0) {
            int ps = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_enum_lookback_multi, 64, 0);
            multi_per_sm = ps;
        }
        const uint64_t mcap = (uint64_t)multi_per_sm * (uint64_t)h->num_sms;
        if (mcap > (uint64_t)n) {
            const uint64_t G = (h->tiles * (uint64_t)n + (mcap - n) - 1) / (mcap - n);
            if (G <= kEnumGMax) {
                const uint64_t ctas = (h->tiles + G - 1) / G;
                rc = dsoa_launch_step(h, k_enum_lookback_multi, (unsigned)(ctas * (uint64_t)n), 64u, h->ctx,
                                      h->tiles, (uint32_t)G, (uint32_t)ctas, eb);
                if (rc == DSOA_OK)
                    for (int q = 0; q < n; ++q) h->enumerated[types[q]] = true;
                return rc;
            }
        }
    }
    rc = dsoa_launch_step(h, k_enum_lookback, (unsigned)(h->tiles * (uint64_t)n), 64u, h->ctx, h->tiles,
                          eb, (fits && !tickets) ? 0u : 1u);
    if (rc == DSOA_OK)
        for (int q = 0; q < n; ++q) h->enumerated[types[q]] = true;
    return rc;
}

int dsoa_enumerate_internal(dsoa_heap* h, int type) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    const uint32_t b = dsoa_bm_alloc((uint32_t)type);
    if (h->scan_tiles_per_cta == 0)        // single-pass look-back enumeration (default)
        return enumerate_lookback(h, &type, 1);
    const int tpb = 256;
    const uint64_t warps = h->tiles;
    const unsigned g1 = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((warps + 7) / 8, (uint64_t)h->num_sms * 8));
    rc = dsoa_launch_step(h, k_tile_count, g1, (unsigned)tpb, h->ctx, b, h->tiles, h->tile_cnt, h->tile_off,
                          h->r_dev[type], h->done);
    if (rc) return rc;
    const uint32_t* toff = h->tile_off;
    if (h->scan_tiles_per_cta == 2)
        rc = dsoa_launch_step(h, k_compact<2>, (unsigned)((h->tiles + 1) / 2), 128u, h->ctx, b, h->tiles, toff,
                              h->R[type], h->Rocc[type]);
    else
        rc = dsoa_launch_step(h, k_compact<1>, (unsigned)h->tiles, 64u, h->ctx, b, h->tiles, toff, h->R[type],
                              h->Rocc[type]);
    if (rc == DSOA_OK) h->enumerated[type] = true;
    return rc;
}

int dsoa_prepare_doall(dsoa_heap* h, int type) {
    if (h->skip_enumeration) return h->enumerated[type] ? DSOA_OK : DSOA_ERR_INVALID_ARG;
    return dsoa_enumerate_internal(h, type);
}

// ------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------
extern "C" {

int dsoa_heap_create(size_t bytes, void* stream, dsoa_heap** out) {
    if (!out || bytes < 4096) return DSOA_ERR_INVALID_ARG;
    *out = nullptr;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return DSOA_ERR_CUDA; }
    dsoa_heap* h = new (std::nothrow) dsoa_heap();
    if (!h) { cudaFree(p); return DSOA_ERR_OOM; }
    int rc = init_heap(h, p, bytes, true, stream);
    if (rc) { cudaFree(p); delete h; return rc; }
    *out = h;
    return DSOA_OK;
}

int dsoa_heap_create_from(void* dev_ptr, size_t bytes, void* stream, dsoa_heap** out) {
    if (!out || !dev_ptr || bytes < 4096 || ((uintptr_t)dev_ptr % kAlign) != 0) return DSOA_ERR_INVALID_ARG;
    *out = nullptr;
    dsoa_heap* h = new (std::nothrow) dsoa_heap();
    if (!h) return DSOA_ERR_OOM;
    int rc = init_heap(h, dev_ptr, bytes, false, stream);
    if (rc) { delete h; return rc; }
    *out = h;
    return DSOA_OK;
}

int dsoa_register_type(dsoa_heap* h, const uint32_t* field_bytes, int nfields, int* type_out) {
    if (!h || !field_bytes || !type_out || nfields < 1 || nfields > DSOA_MAX_FIELDS) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_ERR_FROZEN;
    if (h->ntypes >= DSOA_MAX_TYPES) return DSOA_ERR_TOO_MANY_TYPES;
    dsoa_type_info ti;
    std::memset(&ti, 0, sizeof(ti));
    ti.nfields = nfields;
    uint32_t off = 0;
    for (int i = 0; i < nfields; ++i) {
        const uint32_t fb = field_bytes[i];
        if (fb != 1 && fb != 2 && fb != 4 && fb != 8 && fb != 16) return DSOA_ERR_INVALID_ARG;
        ti.field_bytes[i] = fb;
        ti.col_off[i] = off;
        off += (uint32_t)align_up((uint64_t)DSOA_SLOTS * fb, 128);
    }
    ti.data_bytes = off;
    ti.capacity = DSOA_SLOTS;
    ti.base = -1;
    h->types[h->ntypes] = ti;
    *type_out = h->ntypes++;
    return DSOA_OK;
}

int dsoa_register_subtype(dsoa_heap* h, int base, const uint32_t* extra_field_bytes, int n_extra, int* type_out) {
    if (!h || !type_out || base < 0 || base >= h->ntypes || n_extra < 0 || (n_extra > 0 && !extra_field_bytes))
        return DSOA_ERR_INVALID_ARG;
    const dsoa_type_info& b = h->types[base];
    if (b.nfields + n_extra > DSOA_MAX_FIELDS) return DSOA_ERR_INVALID_ARG;
    uint32_t fb[DSOA_MAX_FIELDS];
    for (int f = 0; f < b.nfields; ++f) fb[f] = b.field_bytes[f];       // inherited columns first
    for (int f = 0; f < n_extra; ++f) fb[b.nfields + f] = extra_field_bytes[f];
    const int rc = dsoa_register_type(h, fb, b.nfields + n_extra, type_out);
    if (rc) return rc;
    h->types[*type_out].base = base;
    return DSOA_OK;
}

int dsoa_type_base(dsoa_heap* h, int type, int* base_out) {
    if (!h || !base_out || type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    *base_out = h->types[type].base;
    return DSOA_OK;
}

int dsoa_heap_freeze(dsoa_heap* h) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_OK;
    if (h->ntypes == 0) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    uint32_t block_bytes = 128;
    if (h->capacity_mode == DSOA_CAPACITY_PER_TYPE) {
        const int rc = per_type_capacity(h, &block_bytes);
        if (rc) return rc;
    } else {
        for (int t = 0; t < h->ntypes; ++t) block_bytes = std::max(block_bytes, h->types[t].data_bytes);
    }
    const int nbm = 1 + 2 * h->ntypes;
    (void)nbm;
    // largest M whose layout fits in the byte budget
    uint64_t lo = 0, hi = h->bytes / block_bytes + 1;
    Layout L;
    while (lo + 1 < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (make_layout(mid, block_bytes, h->ntypes, &L) && L.total <= h->bytes) lo = mid; else hi = mid;
    }
    if (lo == 0 || lo > (1ull << 32) - 1 || !make_layout(lo, block_bytes, h->ntypes, &L)) return DSOA_ERR_OOM;
    char* base = (char*)h->base;
    dsoa_ctx& c = h->ctx;
    std::memset(&c, 0, sizeof(c));
    c.data = base + L.off_data;
    c.slot = (unsigned long long*)(base + L.off_slot);
    c.btype = (uint32_t*)(base + L.off_btype);
    c.drain = (uint8_t*)(base + L.off_drain);
    c.bm = (unsigned long long*)(base + L.off_bm);
    uint64_t* small = (uint64_t*)(base + L.off_small);
    c.err = (int*)(small + 0);
    c.hint = (dsoa_hint*)(base + L.off_hint);
    c.hint_mask = (uint32_t)(L.hint_slots - 1);
    h->lb_state = (unsigned long long*)(base + L.off_lb);              // [ntypes][tiles]
    h->lb_ctl = (uint32_t*)(h->lb_state + L.tiles * (uint64_t)h->ntypes);  // [ntypes][4]: ticket, done, epoch, failed
    c.grid_scratch = (uint32_t*)(base + L.off_grid);
    h->done = (uint32_t*)(small + 1);
    h->scratch64 = (unsigned long long*)(small + 32);
    h->stream_ctl = (uint32_t*)(small + 44);  // [3] of the streamed do-all
    h->count_acc = (unsigned long long*)(small + 46);  // [16] words 46..61
    h->count_ticket = (uint32_t*)(small + 62);
    c.M = L.M;
    c.bm_stride = L.bm_stride;
    for (int l = 0; l < DSOA_MAX_LEVELS; ++l) { c.lvl_off[l] = L.lvl_off[l]; c.lvl_words[l] = L.lvl_words[l]; }
    c.nlevels = L.nlevels;
    c.block_bytes = block_bytes;
    c.ntypes = (uint32_t)h->ntypes;
    for (int t = 0; t < h->ntypes; ++t) {
        for (int f = 0; f < h->types[t].nfields; ++f) c.col_off[t][f] = (uint16_t)h->types[t].col_off[f];
        const uint32_t n = h->types[t].capacity;
        c.cap[t] = n >= 64 ? DSOA_ALL : ((1ull << n) - 1ull);
    }
    h->tiles = L.tiles;
    for (int t = 0; t < h->ntypes; ++t) {
        h->R[t] = (uint32_t*)(base + L.off_R) + (uint64_t)t * L.M;
        h->Rocc[t] = (unsigned long long*)(base + L.off_Rocc) + (uint64_t)t * L.M;
        h->r_dev[t] = (uint32_t*)(small + 8 + t);
        h->enumerated[t] = false;
    }
    h->tile_cnt = (uint32_t*)(base + L.off_tcnt);
    h->tile_off = (uint32_t*)(base + L.off_toff);
    h->meta_bytes = L.total - L.M * block_bytes;
    DSOA_CUDA_TRY(cudaMemsetAsync(c.slot, 0, L.M * 8, h->stream));            // all slots taken
    DSOA_CUDA_TRY(cudaMemsetAsync(c.btype, 0xFF, L.M * 4, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(c.drain, 0, L.M, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(c.bm, 0, (uint64_t)nbm * L.bm_stride * 8, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(small, 0, kSmallWords * 8, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(c.hint, 0xFF, ((uint64_t)c.hint_mask + 1) * (uint64_t)h->ntypes * sizeof(dsoa_hint),
                                  h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(c.grid_scratch, 0, (uint64_t)DSOA_GRID_SCRATCH * 4, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(h->lb_state, 0, L.tiles * 8 * (uint64_t)h->ntypes + 16 * (uint64_t)h->ntypes,
                                  h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(h->R[0], 0, L.M * 4 * (uint64_t)h->ntypes, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(h->Rocc[0], 0, L.M * 8 * (uint64_t)h->ntypes, h->stream));
    k_init_free<<<std::max(1, h->num_sms * 4), 256, 0, h->stream>>>(c);
    int rc = dsoa_check_launch(h);
    if (rc) return rc;
    h->frozen = true;
    return DSOA_OK;
}

int dsoa_heap_info(dsoa_heap* h, uint64_t* num_blocks, uint32_t* block_bytes, uint32_t* num_levels,
                   uint64_t* metadata_bytes) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    if (num_blocks) *num_blocks = h->ctx.M;
    if (block_bytes) *block_bytes = h->ctx.block_bytes;
    if (num_levels) *num_levels = h->ctx.nlevels;
    if (metadata_bytes) *metadata_bytes = h->meta_bytes;
    return DSOA_OK;
}

int dsoa_field_offset(dsoa_heap* h, int type, int field, uint32_t* offset_out) {
    if (!h || !offset_out || type < 0 || type >= h->ntypes || field < 0 || field >= h->types[type].nfields)
        return DSOA_ERR_INVALID_ARG;
    *offset_out = h->types[type].col_off[field];
    return DSOA_OK;
}

int dsoa_parallel_new(dsoa_heap* h, int type, uint64_t n, int ctor_id, const void* args, size_t nb) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    if (ctor_id >= 100 && ctor_id < 200) return dsoa_micro_new(h, type, n, ctor_id, args, nb);
    if (ctor_id >= 200 && ctor_id < 300) return dsoa_gol_new(h, type, n, ctor_id, args, nb);
    if (ctor_id >= 500 && ctor_id < 600) return dsoa_nbody_new(h, type, n, ctor_id, args, nb);
    return DSOA_ERR_UNKNOWN_METHOD;
}

// ---- user methods: launchers registered by user libraries (process-wide)
static std::mutex g_user_mu;
static dsoa_method_fn g_user[DSOA_USER_METHOD_MAX - DSOA_USER_METHOD_MIN + 1];

static dsoa_method_fn user_method(int id) {
    std::lock_guard<std::mutex> lock(g_user_mu);
    return g_user[id - DSOA_USER_METHOD_MIN];
}

// Enumerate as for a built-in method, then hand the prepared launch to the
// user's launcher (which instantiates dsoa_doall_kernel for its method).
static int user_do(dsoa_heap* h, int type, int method_id, const void* args, size_t nb) {
    const dsoa_method_fn fn = user_method(method_id);
    if (!fn) return DSOA_ERR_UNKNOWN_METHOD;
    int rc = dsoa_prepare_doall(h, type);
    if (rc) return rc;
    const dsoa_ctx c = dsoa_launch_ctx(h);
    dsoa_doall_launch L;
    std::memset(&L, 0, sizeof(L));
    L.ctx = &c;
    L.ctx_bytes = sizeof(c);
    L.type = type;
    L.tpb = (uint32_t)h->doall_tpb;
    L.max_ctas_per_sm = (uint32_t)h->doall_ctas_per_sm;
    L.num_sms = (uint32_t)h->num_sms;
    L.waves = (uint32_t)h->doall_waves;
    L.slots_per_thread = h->slots_per_thread >= 2 ? 2u : 1u;
    L.pdl = (h->flags & DSOA_FLAG_PDL) ? 1u : 0u;
    L.R = h->R[type];
    L.occ = (const uint64_t*)h->Rocc[type];
    L.r_dev = h->r_dev[type];
    L.stream = (void*)h->stream;
    rc = fn(&L, args, nb);
    if (rc == DSOA_OK) h->launches++;
    return rc;
}

static int parallel_do_one(dsoa_heap* h, int type, int method_id, const void* args, size_t nb) {
    if (method_id >= DSOA_USER_METHOD_MIN && method_id <= DSOA_USER_METHOD_MAX)
        return user_do(h, type, method_id, args, nb);
    if (method_id >= 100 && method_id < 200) return dsoa_micro_do(h, type, method_id, args, nb);
    if (method_id >= 200 && method_id < 300) return dsoa_gol_do(h, type, method_id, args, nb);
    if (method_id >= 300 && method_id < 400) return dsoa_wator_do(h, type, method_id, args, nb);
    if (method_id >= 400 && method_id < 500) return dsoa_traffic_do(h, type, method_id, args, nb);
    if (method_id >= 500 && method_id < 600) return dsoa_nbody_do(h, type, method_id, args, nb);
    return DSOA_ERR_UNKNOWN_METHOD;
}

// type and every type that extends it, directly or not (subtypes are registered
// after their base, so they follow it in id order)
static int type_family(const dsoa_heap* h, int type, int* out) {
    int n = 0;
    for (int u = type; u < h->ntypes; ++u) {
        int a = u;
        while (a > type) a = h->types[a].base;
        if (a == type) out[n++] = u;
    }
    return n;
}

int dsoa_register_method(int method_id, dsoa_method_fn fn) {
    if (!fn || method_id < DSOA_USER_METHOD_MIN || method_id > DSOA_USER_METHOD_MAX) return DSOA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_user_mu);
    dsoa_method_fn& slot = g_user[method_id - DSOA_USER_METHOD_MIN];
    if (slot && slot != fn) return DSOA_ERR_INVALID_ARG;
    slot = fn;
    return DSOA_OK;
}

int dsoa_parallel_do(dsoa_heap* h, int type, int method_id, const void* args, size_t nb) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    int fam[DSOA_MAX_TYPES];
    const int n = type_family(h, type, fam);
    if (n == 1) return parallel_do_one(h, type, method_id, args, nb);
    // The objects of the type and of its subtypes existing at entry: one
    // enumeration launch snapshots every member, then one do-all launch per
    // member type runs on its snapshot.
    if (!h->skip_enumeration) {
        rc = dsoa_enumerate_many(h, fam, n);
        if (rc) return rc;
    }
    const bool skip = h->skip_enumeration;
    h->skip_enumeration = true;
    for (int q = 0; q < n && rc == DSOA_OK; ++q) {
        h->skip_prologue = q > 0;      // a method's prologue runs once per do-all
        rc = parallel_do_one(h, fam[q], method_id, args, nb);
    }
    h->skip_prologue = false;
    h->skip_enumeration = skip;
    return rc;
}

int dsoa_parallel_do_enumerated(dsoa_heap* h, int type, int method_id, const void* args, size_t nb) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    h->skip_enumeration = true;
    const int rc = dsoa_parallel_do(h, type, method_id, args, nb);
    h->skip_enumeration = false;
    return rc;
}

int dsoa_run_kernel(dsoa_heap* h, int kernel_id, uint64_t n, const void* args, size_t nb) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (kernel_id >= 100 && kernel_id < 200) return dsoa_micro_kernel(h, kernel_id, n, args, nb);
    if (kernel_id >= 200 && kernel_id < 300) return dsoa_gol_kernel(h, kernel_id, n, args, nb);
    if (kernel_id >= 300 && kernel_id < 400) return dsoa_wator_kernel(h, kernel_id, n, args, nb);
    if (kernel_id >= 400 && kernel_id < 500) return dsoa_traffic_kernel(h, kernel_id, n, args, nb);
    return DSOA_ERR_UNKNOWN_METHOD;
}

int dsoa_delete_handles(dsoa_heap* h, const dsoa_obj* handles_dev, uint64_t n) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (n == 0) return DSOA_OK;
    if (!handles_dev) return DSOA_ERR_INVALID_ARG;
    k_delete_handles<<<dsoa_new_grid(h, n, 256), 256, 0, h->stream>>>(dsoa_launch_ctx(h), handles_dev, n);
    return dsoa_check_launch(h);
}

int dsoa_enumerate(dsoa_heap* h, int type, const uint32_t** R_dev, const uint64_t** occ_dev,
                   const uint32_t** r_dev) {
    int rc = dsoa_enumerate_internal(h, type);
    if (rc) return rc;
    if (R_dev) *R_dev = h->R[type];
    if (occ_dev) *occ_dev = (const uint64_t*)h->Rocc[type];
    if (r_dev) *r_dev = h->r_dev[type];
    return DSOA_OK;
}

int dsoa_enumerate_many(dsoa_heap* h, const int* types_host, int ntypes) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (!types_host || ntypes < 1 || ntypes > h->ntypes) return DSOA_ERR_INVALID_ARG;
    for (int q = 0; q < ntypes; ++q) {
        if (types_host[q] < 0 || types_host[q] >= h->ntypes) return DSOA_ERR_INVALID_ARG;
        for (int p = 0; p < q; ++p)
            if (types_host[p] == types_host[q]) return DSOA_ERR_INVALID_ARG;
    }
    if (h->scan_tiles_per_cta == 0) return enumerate_lookback(h, types_host, ntypes);
    for (int q = 0; q < ntypes; ++q) {
        rc = dsoa_enumerate_internal(h, types_host[q]);
        if (rc) return rc;
    }
    return DSOA_OK;
}

int dsoa_count_async(dsoa_heap* h, int type, uint64_t* out_dev) {
    return dsoa_count_many_async(h, &type, 1, out_dev);
}

int dsoa_count_many_async(dsoa_heap* h, const int* types_host, int ntypes, uint64_t* out_dev) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (!types_host || !out_dev || ntypes < 1 || ntypes > h->ntypes) return DSOA_ERR_INVALID_ARG;
    CountBatch cb;
    std::memset(&cb, 0, sizeof(cb));
    cb.n = (uint32_t)ntypes;
    for (int q = 0; q < ntypes; ++q) {
        if (types_host[q] < 0 || types_host[q] >= h->ntypes) return DSOA_ERR_INVALID_ARG;
        cb.b[q] = dsoa_bm_alloc((uint32_t)types_host[q]);
    }
    const uint64_t warps = h->ctx.lvl_words[0] * (uint64_t)ntypes;
    const unsigned g = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((warps + 7) / 8, (uint64_t)h->num_sms * 8));
    k_count_many<<<g, 256, 0, h->stream>>>(h->ctx, cb, (unsigned long long*)out_dev, h->count_acc, h->count_ticket);
    return dsoa_check_launch(h);
}

int dsoa_count(dsoa_heap* h, int type, uint64_t* out_host) {
    if (!h || !out_host) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    rc = dsoa_count_async(h, type, (uint64_t*)h->scratch64);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemcpyAsync(out_host, h->scratch64, 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_free_blocks_async(dsoa_heap* h, uint64_t* out_dev) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (!out_dev) return DSOA_ERR_INVALID_ARG;
    DSOA_CUDA_TRY(cudaMemsetAsync(out_dev, 0, 8, h->stream));
    const unsigned g = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((h->ctx.lvl_words[0] + 255) / 256, (uint64_t)h->num_sms * 8));
    k_popc_level0<<<g, 256, 0, h->stream>>>(h->ctx, dsoa_bm_free(), (unsigned long long*)out_dev);
    return dsoa_check_launch(h);
}

int dsoa_get_error(dsoa_heap* h, int* bits_out) {
    if (!h || !bits_out) return DSOA_ERR_INVALID_ARG;
    *bits_out = 0;
    if (!h->frozen) return DSOA_OK;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    DSOA_CUDA_TRY(cudaMemcpyAsync(bits_out, h->ctx.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaMemsetAsync(h->ctx.err, 0, sizeof(int), h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_check(dsoa_heap* h, uint64_t* out_host) {
    if (!h || !out_host) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemsetAsync(h->scratch64, 0, DSOA_CHECK_COUNT * 8, h->stream));
    k_check<<<std::max(1, h->num_sms * 4), 256, 0, h->stream>>>(h->ctx, h->scratch64);
    rc = dsoa_check_launch(h);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemcpyAsync(out_host, h->scratch64, DSOA_CHECK_COUNT * 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_export_state(dsoa_heap* h, void* out_host, size_t capacity, size_t* bytes_needed,
                      uint64_t* bitmap_words) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    const uint64_t M = h->ctx.M, nbm = 1 + 2 * (uint64_t)h->ntypes;
    const size_t need = M * 8 + M * 4 + nbm * h->ctx.bm_stride * 8;
    if (bytes_needed) *bytes_needed = need;
    if (bitmap_words) *bitmap_words = h->ctx.bm_stride;
    if (!out_host) return DSOA_OK;
    if (capacity < need) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    char* o = (char*)out_host;
    DSOA_CUDA_TRY(cudaMemcpyAsync(o, h->ctx.slot, M * 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaMemcpyAsync(o + M * 8, h->ctx.btype, M * 4, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaMemcpyAsync(o + M * 12, h->ctx.bm, nbm * h->ctx.bm_stride * 8, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

// Checkpoint image: a header that pins the layout, then the heap's bytes.  Every
// reference inside the heap (handles, block lists, bitmaps) is an index, not an
// address, so the bytes are valid in any heap with the same layout.
struct dsoa_image_header {
    uint64_t magic, version, bytes, M, meta;
    uint32_t block_bytes, nlevels, ntypes, capacity_mode;
    uint32_t nfields[DSOA_MAX_TYPES];
    uint32_t field_bytes[DSOA_MAX_TYPES][DSOA_MAX_FIELDS];
    uint32_t capacity[DSOA_MAX_TYPES];
    int32_t base[DSOA_MAX_TYPES];
};
static const uint64_t kImageMagic = 0x31304D4941534F44ull;   // "DOSAIM01"

static void image_header(const dsoa_heap* h, dsoa_image_header* H) {
    std::memset(H, 0, sizeof(*H));
    H->magic = kImageMagic;
    H->version = 3;
    H->bytes = h->bytes;
    H->M = h->ctx.M;
    H->meta = h->meta_bytes;
    H->block_bytes = h->ctx.block_bytes;
    H->nlevels = h->ctx.nlevels;
    H->ntypes = (uint32_t)h->ntypes;
    H->capacity_mode = (uint32_t)h->capacity_mode;
    for (int t = 0; t < h->ntypes; ++t) {
        H->nfields[t] = (uint32_t)h->types[t].nfields;
        for (int f = 0; f < h->types[t].nfields; ++f) H->field_bytes[t][f] = h->types[t].field_bytes[f];
        H->capacity[t] = h->types[t].capacity;
        H->base[t] = h->types[t].base;
    }
}

int dsoa_heap_save(dsoa_heap* h, void* out_host, size_t capacity, size_t* bytes_needed) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    const size_t need = sizeof(dsoa_image_header) + h->bytes;
    if (bytes_needed) *bytes_needed = need;
    if (!out_host) return DSOA_OK;
    if (capacity < need) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    image_header(h, (dsoa_image_header*)out_host);
    DSOA_CUDA_TRY(cudaMemcpyAsync((char*)out_host + sizeof(dsoa_image_header), h->base, h->bytes,
                                  cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_heap_load(dsoa_heap* h, const void* in_host, size_t bytes) {
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (!in_host || bytes != sizeof(dsoa_image_header) + h->bytes) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    dsoa_image_header mine;
    image_header(h, &mine);
    if (std::memcmp(&mine, in_host, sizeof(mine)) != 0) return DSOA_ERR_INVALID_ARG;
    DSOA_CUDA_TRY(cudaMemcpyAsync(h->base, (const char*)in_host + sizeof(dsoa_image_header), h->bytes,
                                  cudaMemcpyHostToDevice, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int t = 0; t < h->ntypes; ++t) h->enumerated[t] = false;   // enumerate again before reuse
    return DSOA_OK;
}

int dsoa_get_ctx(dsoa_heap* h, void* out, size_t nb) {
    if (!h || !out || nb != sizeof(dsoa_ctx)) return DSOA_ERR_INVALID_ARG;
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    std::memcpy(out, &h->ctx, sizeof(dsoa_ctx));
    return DSOA_OK;
}

int dsoa_graph_begin(dsoa_heap* h) {
    if (!h || h->stream == nullptr) return DSOA_ERR_INVALID_ARG;  // legacy stream cannot be captured
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    return DSOA_OK;
}

int dsoa_graph_end(dsoa_heap* h, dsoa_graph** out) {
    if (!h || !out) return DSOA_ERR_INVALID_ARG;
    *out = nullptr;
    dsoa_graph* g = new (std::nothrow) dsoa_graph();
    if (!g) return DSOA_ERR_OOM;
    if (cudaStreamEndCapture(h->stream, &g->graph) != cudaSuccess) { delete g; return DSOA_ERR_CUDA; }
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        delete g;
        return DSOA_ERR_CUDA;
    }
    *out = g;
    return DSOA_OK;
}

int dsoa_graph_launch(dsoa_graph* g, void* stream) {
    if (!g) return DSOA_ERR_INVALID_ARG;
    DSOA_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return DSOA_OK;
}

int dsoa_graph_destroy(dsoa_graph* g) {
    if (!g) return DSOA_ERR_INVALID_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return DSOA_OK;
}

int dsoa_set_launch(dsoa_heap* h, int tpb, int ctas_per_sm, int slots_per_thread, int scan_tiles, int waves) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    if (tpb) {
        if (tpb < 64 || tpb > 512 || tpb % 64) return DSOA_ERR_INVALID_ARG;
        h->doall_tpb = tpb;
    }
    if (ctas_per_sm) {
        if (ctas_per_sm < 1 || ctas_per_sm > 32) return DSOA_ERR_INVALID_ARG;
        h->doall_ctas_per_sm = ctas_per_sm;
    }
    if (slots_per_thread) {
        if (slots_per_thread != 1 && slots_per_thread != 2 && slots_per_thread != 4) return DSOA_ERR_INVALID_ARG;
        h->slots_per_thread = slots_per_thread;
        h->vec_slots_per_thread = slots_per_thread;
    }
    if (scan_tiles) {
        if (scan_tiles < 1 || scan_tiles > 5) return DSOA_ERR_INVALID_ARG;
        h->scan_tiles_per_cta = scan_tiles >= 3 ? 0 : scan_tiles;   // 3, 4, 5 = single pass
        h->stream_enum = scan_tiles == 4;                           // 4 = + streamed do-alls
        h->cluster_enum = scan_tiles == 5;                          // 5 = a cluster per type
    }
    if (waves) {
        if (waves < 1 || waves > DSOA_MAX_WAVES) return DSOA_ERR_INVALID_ARG;
        h->doall_waves = waves;
    }
    return DSOA_OK;
}

int dsoa_set_flags(dsoa_heap* h, uint32_t flags) {
    if (!h || (flags & ~(DSOA_FLAG_NO_COALESCE | DSOA_FLAG_NO_ROTATE | DSOA_FLAG_NO_HINT | DSOA_FLAG_FUSED |
                         DSOA_FLAG_PDL | DSOA_FLAG_ENUM_TICKETS | DSOA_FLAG_NO_FRESH_GROUP |
                         DSOA_FLAG_PAPER_R | DSOA_FLAG_R_PER_ROUND | DSOA_FLAG_DRAIN)))
        return DSOA_ERR_INVALID_ARG;
    h->flags = flags;
    return DSOA_OK;
}

int dsoa_set_lookups(dsoa_heap* h, int r) {
    if (!h || r < 1 || r > 64) return DSOA_ERR_INVALID_ARG;
    h->lookups = (uint32_t)r;
    return DSOA_OK;
}

int dsoa_type_stats(dsoa_heap* h, int type, uint64_t* out_host) {
    if (!h || !out_host) return DSOA_ERR_INVALID_ARG;
    if (capturing(h->stream)) return DSOA_ERR_CAPTURE;
    int rc = dsoa_ensure_frozen(h);
    if (rc) return rc;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    unsigned long long* sc = h->scratch64;
    DSOA_CUDA_TRY(cudaMemsetAsync(sc + 8, 0, 8, h->stream));
    const unsigned g = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((h->ctx.lvl_words[0] + 255) / 256, (uint64_t)h->num_sms * 8));
    k_popc_level0<<<g, 256, 0, h->stream>>>(h->ctx, dsoa_bm_alloc((uint32_t)type), sc + 8);
    rc = dsoa_check_launch(h);
    if (rc) return rc;
    rc = dsoa_count_async(h, type, (uint64_t*)(sc + 9));
    if (rc) return rc;
    DSOA_CUDA_TRY(cudaMemcpyAsync(out_host, sc + 8, 16, cudaMemcpyDeviceToHost, h->stream));
    DSOA_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return DSOA_OK;
}

int dsoa_set_capacity_mode(dsoa_heap* h, int mode) {
    if (!h || (mode != DSOA_CAPACITY_UNIFORM && mode != DSOA_CAPACITY_PER_TYPE)) return DSOA_ERR_INVALID_ARG;
    if (h->frozen) return DSOA_ERR_FROZEN;
    h->capacity_mode = mode;
    return DSOA_OK;
}

int dsoa_type_capacity(dsoa_heap* h, int type, uint32_t* n_out) {
    if (!h || !n_out || type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    *n_out = h->types[type].capacity;
    return DSOA_OK;
}

int dsoa_launch_count(dsoa_heap* h, uint64_t* out) {
    if (!h || !out) return DSOA_ERR_INVALID_ARG;
    *out = h->launches;
    return DSOA_OK;
}

int dsoa_heap_destroy(dsoa_heap* h) {
    if (!h) return DSOA_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    if (h->owns && h->base) cudaFree(h->base);
    delete h;
    return DSOA_OK;
}

const char* dsoa_error_string(int code) {
    switch (code) {
        case DSOA_OK: return "ok";
        case DSOA_ERR_INVALID_ARG: return "invalid argument";
        case DSOA_ERR_FROZEN: return "heap layout already frozen";
        case DSOA_ERR_TOO_MANY_TYPES: return "too many types";
        case DSOA_ERR_OOM: return "heap too small";
        case DSOA_ERR_CUDA: return "CUDA runtime error";
        case DSOA_ERR_NOT_FROZEN: return "heap layout not frozen";
        case DSOA_ERR_UNKNOWN_METHOD: return "unknown built-in method, constructor or kernel";
        case DSOA_ERR_CAPTURE: return "synchronous call during stream capture";
        default: return "unknown error";
    }
}

}  // extern "C"
