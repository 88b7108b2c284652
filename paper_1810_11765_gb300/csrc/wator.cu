// wator.cu -- Wa-Tor predator-prey as an SMMO application (Table 1 "wa-tor";
// Dewdney 1984).  Fish {0 inst, 1 cell, 2 age, 3 target} and Shark {0 inst,
// 1 cell, 2 age, 3 energy, 4 target, 5 eat} agents on a torus with a per-cell
// occupancy grid (0 empty, 1 fish, 2 shark), an agent-handle map and a claim
// word per cell.  One step is four do-alls:
//   Fish.choose   pick an empty N/E/S/W neighbour with Philox(seed; t, c, 1, 0),
//                 claim it with atomicMin(source cell)
//   Fish.move     age + 1; the lowest claimant moves; a mover of age >= 3
//                 leaves a newborn fish and restarts its age (allocated in place,
//                 or marked and allocated afterwards by the births kernel)
//   Shark.choose  prefer fish neighbours, else empty ones, Philox(seed; t, c, 2, 0)
//   Shark.move    age + 1; a winner eats (deletes the Fish object: cross-type
//                 delete) and refills energy to 3, else loses 1; breeds at 10;
//                 a shark at energy 0 deletes itself
// Every decision depends only on cell indices and the step index, so the
// result does not depend on thread scheduling or object placement.
#include "dsoa_internal.cuh"
#include "rng.cuh"

namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kFishBreed = 3u, kSharkBreed = 10u, kSharkEnergy = 3u;
constexpr uint32_t kFishThr = 1288490188u;   // floor(0.30 * 2^32)
constexpr uint32_t kSharkThr = 1503238553u;  // floor(0.35 * 2^32): fish or shark

// Torus neighbours of cell c: one division for the coordinates, wrap-around
// by compare-and-select (the same cells as the modular formulas).
__device__ __forceinline__ void neighbours(uint32_t c, uint32_t w, uint32_t h, uint32_t nb[4]) {
    const uint32_t y = c / w, x = c - y * w;
    const uint32_t row = y * w;
    nb[0] = (y == 0u ? h - 1u : y - 1u) * w + x;        // N
    nb[1] = row + (x + 1u == w ? 0u : x + 1u);          // E
    nb[2] = (y + 1u == h ? 0u : y + 1u) * w + x;        // S
    nb[3] = row + (x == 0u ? w - 1u : x - 1u);          // W
}

// Cells of instance I: every cell index read from an object field is checked
// against it before it addresses the instance's grids (dsoa_index_ok).
__device__ __forceinline__ uint64_t cells_of(const dsoa_inst& I) { return (uint64_t)I.w * I.h; }

// Index of the chosen candidate among k >= 1: Philox word 0 modulo k.  With
// one candidate the draw cannot matter, so it is not computed.
__device__ __forceinline__ uint32_t pick(uint32_t k, uint64_t seed, uint32_t t, uint32_t cell, uint32_t stream) {
    if (k == 1u) return 0u;
    const uint32_t u = dsoa_philox_w0(seed, t, cell, stream, 0u);
    return k == 2u ? (u & 1u) : (k == 4u ? (u & 3u) : u % 3u);
}

// The p-th neighbour (in N, E, S, W order) among those whose bit is set in
// `m`, by an unrolled scan: the candidate list stays in registers instead of
// a dynamically indexed local array.
__device__ __forceinline__ uint32_t nth_candidate(const uint32_t nb[4], uint32_t m, uint32_t p) {
    uint32_t tg = kNone, seen = 0u;
#pragma unroll
    for (int d = 0; d < 4; ++d)
        if ((m >> d) & 1u) {
            if (seen == p) tg = nb[d];
            ++seen;
        }
    return tg;
}

struct FishChoose {
    using Args = dsoa_wator_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t ik = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, ik, a.n_inst)) return;
        const dsoa_inst I = a.inst[ik];
        if (I.state != DSOA_INST_RUN) return;
        const uint32_t cell = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (!dsoa_index_ok(c, cell, cells_of(I))) return;
        uint32_t nb[4], empty = 0u;
        neighbours(cell, I.w, I.h, nb);
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (I.occ[nb[d]] == 0) empty |= 1u << d;
        uint32_t tg = kNone;
        if (empty) {
            tg = nth_candidate(nb, empty, pick((uint32_t)__popc(empty), I.seed, I.t, cell, 1u));
            atomicMin(&I.claim[tg], cell);
        }
        dsoa_column<uint32_t>(c, t, bid, 3)[s] = tg;
    }
};

struct FishMove {
    using Args = dsoa_wator_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        dsoa_prefetch_hint(c, t);
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        const dsoa_inst I = a.inst[k];
        if (I.state != DSOA_INST_RUN) return;
        uint32_t* cellp = dsoa_column<uint32_t>(c, t, bid, 1) + s;
        uint32_t* agep = dsoa_column<uint32_t>(c, t, bid, 2) + s;
        const uint32_t tg = dsoa_column<uint32_t>(c, t, bid, 3)[s];
        const uint32_t age = *agep + 1u;
        *agep = age;
        const uint32_t old = *cellp;
        if (tg == kNone) return;
        if (!dsoa_index_ok(c, tg, cells_of(I)) || !dsoa_index_ok(c, old, cells_of(I))) return;
        if (I.claim[tg] != old) return;
        I.claim[tg] = kNone;
        I.occ[tg] = 1;
        I.cellmap[tg] = dsoa_make_handle(t, bid, s);
        *cellp = tg;
        dsoa_obj nf = 0;
        if (age >= kFishBreed) {
            *agep = 0u;
            nf = dsoa_new(c, t);
            if (nf) {
                dsoa_field<uint32_t>(c, nf, 0) = k;
                dsoa_field<uint32_t>(c, nf, 1) = old;
                dsoa_field<uint32_t>(c, nf, 2) = 0u;
                dsoa_field<uint32_t>(c, nf, 3) = kNone;
            }
        }
        I.occ[old] = nf ? 1 : 0;
        I.cellmap[old] = nf;
    }
};

// Fish.move with deferred births: a mover of breeding age marks its old cell
// kBirth ("fish to be born") instead of allocating the newborn in place; the
// births kernel below creates all newborns of the step in full warps.  Nothing
// reads the old cell before that kernel: no fish can have claimed it, since it
// was occupied when the claims were made.
constexpr uint8_t kBirth = 3;

struct FishMoveDeferred {
    using Args = dsoa_wator_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        const dsoa_inst I = a.inst[k];
        if (I.state != DSOA_INST_RUN) return;
        uint32_t* cellp = dsoa_column<uint32_t>(c, t, bid, 1) + s;
        uint32_t* agep = dsoa_column<uint32_t>(c, t, bid, 2) + s;
        const uint32_t tg = dsoa_column<uint32_t>(c, t, bid, 3)[s];
        uint32_t age = *agep + 1u;
        const uint32_t old = *cellp;
        if (tg != kNone && (!dsoa_index_ok(c, tg, cells_of(I)) || !dsoa_index_ok(c, old, cells_of(I)))) return;
        if (tg != kNone && I.claim[tg] == old) {
            I.claim[tg] = kNone;
            I.occ[tg] = 1;
            I.cellmap[tg] = dsoa_make_handle(t, bid, s);
            *cellp = tg;
            const bool breed = age >= kFishBreed;
            if (breed) age = 0u;
            I.occ[old] = breed ? kBirth : 0;
            I.cellmap[old] = 0;
        }
        *agep = age;
    }
};

struct SharkChoose {
    using Args = dsoa_wator_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t ik = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, ik, a.n_inst)) return;
        const dsoa_inst I = a.inst[ik];
        if (I.state != DSOA_INST_RUN) return;
        const uint32_t cell = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (!dsoa_index_ok(c, cell, cells_of(I))) return;
        uint32_t nb[4], fish = 0u, empty = 0u;
        neighbours(cell, I.w, I.h, nb);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const uint8_t o = I.occ[nb[d]];
            fish |= (o == 1 ? 1u : 0u) << d;
            empty |= (o == 0 ? 1u : 0u) << d;
        }
        const uint32_t eat = fish ? 1u : 0u;
        const uint32_t m = fish ? fish : empty;          /* fish first, else empty cells */
        uint32_t tg = kNone;
        if (m) {
            tg = nth_candidate(nb, m, pick((uint32_t)__popc(m), I.seed, I.t, cell, 2u));
            atomicMin(&I.claim[tg], cell);
        }
        dsoa_column<uint32_t>(c, t, bid, 4)[s] = tg;
        dsoa_column<uint32_t>(c, t, bid, 5)[s] = eat;
    }
};

struct SharkMove {
    using Args = dsoa_wator_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        dsoa_prefetch_hint(c, t);
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        const dsoa_inst I = a.inst[k];
        if (I.state != DSOA_INST_RUN) return;
        uint32_t* cellp = dsoa_column<uint32_t>(c, t, bid, 1) + s;
        uint32_t* agep = dsoa_column<uint32_t>(c, t, bid, 2) + s;
        uint32_t* enp = dsoa_column<uint32_t>(c, t, bid, 3) + s;
        const uint32_t tg = dsoa_column<uint32_t>(c, t, bid, 4)[s];
        if (!dsoa_index_ok(c, *cellp, cells_of(I))) return;
        if (tg != kNone && !dsoa_index_ok(c, tg, cells_of(I))) return;
        const dsoa_obj me = dsoa_make_handle(t, bid, s);
        const uint32_t age = *agep + 1u;
        *agep = age;
        uint32_t energy = *enp;
        uint32_t cell = *cellp;
        if (tg != kNone && I.claim[tg] == cell) {
            const uint32_t old = cell;
            I.claim[tg] = kNone;
            if (dsoa_column<uint32_t>(c, t, bid, 5)[s]) {
                dsoa_delete(c, I.cellmap[tg]);
                energy = kSharkEnergy;
            } else {
                energy -= 1u;
            }
            I.occ[tg] = 2;
            I.cellmap[tg] = me;
            cell = tg;
            *cellp = tg;
            dsoa_obj ns = 0;
            if (age >= kSharkBreed) {
                *agep = 0u;
                ns = dsoa_new(c, t);
                if (ns) {
                    dsoa_field<uint32_t>(c, ns, 0) = k;
                    dsoa_field<uint32_t>(c, ns, 1) = old;
                    dsoa_field<uint32_t>(c, ns, 2) = 0u;
                    dsoa_field<uint32_t>(c, ns, 3) = kSharkEnergy;
                    dsoa_field<uint32_t>(c, ns, 4) = kNone;
                    dsoa_field<uint32_t>(c, ns, 5) = 0u;
                }
            }
            I.occ[old] = ns ? 2 : 0;
            I.cellmap[old] = ns;
        } else {
            energy -= 1u;
        }
        *enp = energy;
        if (energy == 0u) {
            I.occ[cell] = 0;
            I.cellmap[cell] = 0;
            dsoa_delete(c, me);
        }
    }
};

// Shark.move that also advances the step counter of every running instance: the
// step's last kernel reads no counter (only the choose methods draw), so CTA 0
// advances them in its prologue and the step needs no launch of its own for it.
struct SharkMoveAdvance : SharkMove {
    static __device__ void prologue(const dsoa_ctx&, const Args& a) {
        for (uint32_t i = threadIdx.x; i < a.n_inst; i += blockDim.x)
            if (a.inst[i].state == DSOA_INST_RUN) a.inst[i].t += 1u;
    }
};

struct Kill {
    using Args = dsoa_wator_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        if (a.inst[k].state == DSOA_INST_KILL) dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

// Agents of instance `target` from an explicit grid or from Philox draws.  Every
// CTA takes tiles of kInitTile cells: each thread draws the kinds of 8
// consecutive cells, the tile's fish cells and shark cells are compacted into
// two lists in shared memory, and the agents are then allocated list by list,
// so that the warps of one allocation request one type only (full warps, one
// leader reservation per up to 32 agents) instead of a few agents of each type.
// Every cell is written once: its claim word by the thread that drew it, its
// occupancy and handle by that thread if empty, else by the thread that
// allocated its agent (0 if the heap was full).
constexpr uint32_t kInitTile = 2048;

__device__ __forceinline__ uint32_t init_kind(const dsoa_wator_args& a, const dsoa_inst& I, uint32_t cell) {
    if (a.init) return a.init[cell];
    const uint32_t u = dsoa_philox_w0(I.seed, 0xFFFFFFFFu, cell, 0u, 0u);
    return u < kFishThr ? 1u : (u < kSharkThr ? 2u : 0u);
}

__device__ __forceinline__ void init_agent(const dsoa_ctx& c, const dsoa_wator_args& a, const dsoa_inst& I,
                                           uint32_t kind, uint32_t cell) {
    const dsoa_obj o = dsoa_new(c, (uint32_t)(kind == 1u ? a.fish_type : a.shark_type));
    if (o) {
        dsoa_field<uint32_t>(c, o, 0) = a.target;
        dsoa_field<uint32_t>(c, o, 1) = cell;
        dsoa_field<uint32_t>(c, o, 2) = 0u;
        if (kind == 1u) {
            dsoa_field<uint32_t>(c, o, 3) = kNone;
        } else {
            dsoa_field<uint32_t>(c, o, 3) = kSharkEnergy;
            dsoa_field<uint32_t>(c, o, 4) = kNone;
            dsoa_field<uint32_t>(c, o, 5) = 0u;
        }
    }
    I.occ[cell] = o ? (uint8_t)kind : 0;
    I.cellmap[cell] = o;
}

__global__ void __launch_bounds__(256) k_init(dsoa_ctx c, dsoa_wator_args a, uint64_t n) {
    __shared__ uint32_t fl[kInitTile], sl[kInitTile];
    __shared__ uint32_t wcount[8];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const dsoa_inst I = a.inst[a.target];
    const uint64_t tiles = (n + kInitTile - 1) / kInitTile;
    for (uint64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
        const uint64_t c0 = tl * kInitTile + (uint64_t)tid * 8u;
        uint32_t kinds = 0, own = 0;                /* 2 bits per cell; fish | sharks << 16 */
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint64_t cell = c0 + i;
            uint32_t k = 0;
            if (cell < n) {
                k = init_kind(a, I, (uint32_t)cell);
                I.claim[cell] = kNone;
                if (k != 1u && k != 2u) { I.occ[cell] = 0; I.cellmap[cell] = 0; k = 0; }
            }
            kinds |= k << (2 * i);
            own += k == 1u ? 1u : (k == 2u ? 0x10000u : 0u);
        }
        uint32_t x = own;                           /* inclusive warp scan of both counts */
#pragma unroll
        for (uint32_t o = 1; o < 32u; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31u) wcount[warp] = x;
        __syncthreads();
        uint32_t pos = x - own, total = 0;
        for (uint32_t w = 0; w < 8u; ++w) {
            if (w < warp) pos += wcount[w];
            total += wcount[w];
        }
        uint32_t pf = pos & 0xFFFFu, ps = pos >> 16;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t k = (kinds >> (2 * i)) & 3u;
            if (k == 1u) fl[pf++] = (uint32_t)(c0 + i);
            else if (k == 2u) sl[ps++] = (uint32_t)(c0 + i);
        }
        __syncthreads();
        const uint32_t nf = total & 0xFFFFu, ns = total >> 16;
        for (uint32_t i = tid; i < nf; i += blockDim.x) init_agent(c, a, I, 1u, fl[i]);
        for (uint32_t i = tid; i < ns; i += blockDim.x) init_agent(c, a, I, 2u, sl[i]);
        __syncthreads();                            /* lists and counts reused */
    }
}

// Births of the step: every CTA scans tiles of 2048 cells of each running
// instance for kBirth marks, compacts them in shared memory and allocates the
// newborn fish with full warps (so one warp leader reserves up to 32 slots at
// once), then writes the handle map and the occupancy (0 if the heap is full).
constexpr uint32_t kBirthTile = 2048;

__global__ void __launch_bounds__(256) k_births(dsoa_ctx c, dsoa_wator_args a) {
    __shared__ uint32_t list[kBirthTile];
    __shared__ uint32_t wcount[8];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    dsoa_pdl_wait();                 /* under programmatic dependent launch: Fish.move done */
    dsoa_pdl_release();
    for (uint32_t k = 0; k < a.n_inst; ++k) {
        const dsoa_inst I = a.inst[k];
        if (I.state != DSOA_INST_RUN) continue;                    /* uniform */
        const uint64_t cells = (uint64_t)I.w * I.h;
        const uint64_t tiles = (cells + kBirthTile - 1) / kBirthTile;
        for (uint64_t tl = blockIdx.x; tl < tiles; tl += gridDim.x) {
            const uint64_t c0 = tl * kBirthTile + (uint64_t)tid * 8u;
            uint8_t b[8];
            if (c0 + 8 <= cells) {
                const uint2 v = *reinterpret_cast<const uint2*>(I.occ + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) { b[i] = (uint8_t)(v.x >> (8 * i)); b[4 + i] = (uint8_t)(v.y >> (8 * i)); }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) b[i] = c0 + i < cells ? I.occ[c0 + i] : 0;
            }
            uint32_t own = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) own += b[i] == kBirth;
            uint32_t x = own;                                     /* inclusive warp scan */
#pragma unroll
            for (uint32_t o = 1; o < 32u; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31u) wcount[warp] = x;
            __syncthreads();
            uint32_t pos = x - own, total = 0;
            for (uint32_t w = 0; w < 8u; ++w) {
                if (w < warp) pos += wcount[w];
                total += wcount[w];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (b[i] == kBirth) list[pos++] = (uint32_t)(c0 + i);
            __syncthreads();
            for (uint32_t i = tid; i < total; i += blockDim.x) {
                const uint32_t cell = list[i];
                const dsoa_obj o = dsoa_new(c, (uint32_t)a.fish_type);
                if (o) {
                    dsoa_field<uint32_t>(c, o, 0) = k;
                    dsoa_field<uint32_t>(c, o, 1) = cell;
                    dsoa_field<uint32_t>(c, o, 2) = 0u;
                    dsoa_field<uint32_t>(c, o, 3) = kNone;
                }
                I.cellmap[cell] = o;
                I.occ[cell] = o ? 1 : 0;
            }
            __syncthreads();                                      /* list and counts reused */
        }
    }
}

__global__ void k_advance(dsoa_inst* inst, uint32_t n) {
    dsoa_pdl_wait();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && inst[i].state == DSOA_INST_RUN) inst[i].t += 1u;
}

}  // namespace

int dsoa_wator_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_wator_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (!args.inst) return DSOA_ERR_INVALID_ARG;
    const bool fish = type == args.fish_type, shark = type == args.shark_type;
    switch (method) {
        case DSOA_M_WATOR_FISH_CHOOSE: return fish ? dsoa_run_doall<FishChoose>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_FISH_MOVE: return fish ? dsoa_run_doall<FishMove>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_FISH_MOVE_DEFER:
            return fish ? dsoa_run_doall<FishMoveDeferred>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_SHARK_CHOOSE: return shark ? dsoa_run_doall<SharkChoose>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_SHARK_MOVE: return shark ? dsoa_run_doall<SharkMove>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_SHARK_MOVE_ADVANCE:
            return shark ? dsoa_run_doall<SharkMoveAdvance>(h, type, args) : DSOA_ERR_INVALID_ARG;
        case DSOA_M_WATOR_KILL: return (fish || shark) ? dsoa_run_doall<Kill>(h, type, args) : DSOA_ERR_INVALID_ARG;
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}

int dsoa_wator_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb) {
    dsoa_wator_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (!args.inst) return DSOA_ERR_INVALID_ARG;
    if (n == 0) return DSOA_OK;
    switch (kernel) {
        case DSOA_K_WATOR_INIT: {
            if (args.target >= args.n_inst || args.fish_type < 0 || args.fish_type >= h->ntypes ||
                args.shark_type < 0 || args.shark_type >= h->ntypes)
                return DSOA_ERR_INVALID_ARG;
            const uint64_t tiles = (n + kInitTile - 1) / kInitTile;
            const uint64_t resident = (uint64_t)std::max(1, dsoa_resident_ctas(reinterpret_cast<const void*>(&k_init), 256)) *
                                      (uint64_t)h->num_sms;
            k_init<<<(unsigned)std::min(tiles, resident), 256, 0, h->stream>>>(dsoa_launch_ctx(h), args, n);
            return dsoa_check_launch(h);
        }
        case DSOA_K_WATOR_BIRTHS: {
            if (n > args.n_inst || args.fish_type < 0 || args.fish_type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
            args.n_inst = (uint32_t)n;
            auto* k = &k_births;
            const unsigned grid = (unsigned)(std::max(1, dsoa_resident_ctas(reinterpret_cast<const void*>(k), 256)) *
                                             h->num_sms);
            return dsoa_launch_step(h, k, grid, 256u, dsoa_launch_ctx(h), args);
        }
        case DSOA_K_WATOR_ADVANCE:
            if (n > args.n_inst) return DSOA_ERR_INVALID_ARG;
            return dsoa_launch_step(h, k_advance, (unsigned)((n + 255) / 256), 256u, args.inst, (uint32_t)n);
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}
