// gol.cu -- Game of Life as an SMMO application (Table 1 "game-of-life"):
// one Cell object per site {0 inst, 1 cell, 2 count, 3 alive:u8} and one Alive
// agent {0 inst, 1 cell} per live cell, allocated on birth and deleted on death.
// A generation is three do-alls: Alive.spread, Alive.reap, Cell.decide.
// B3/S23 on a torus; every instance of a batch is served by the same launches.
#include "dsoa_internal.cuh"
#include "rng.cuh"

namespace {

// The 8 torus neighbours of cell c (Moore neighbourhood): one division for the
// coordinates, wrap-around by compare-and-select (the same cells as the
// modular formulas, also on 1- and 2-wide tori).
__device__ __forceinline__ void moore(uint32_t c, uint32_t w, uint32_t h, uint32_t nb[8]) {
    const uint32_t y = c / w, x = c - y * w;
    const uint32_t xs[3] = {x == 0u ? w - 1u : x - 1u, x, x + 1u == w ? 0u : x + 1u};
    const uint32_t rs[3] = {(y == 0u ? h - 1u : y - 1u) * w, y * w, (y + 1u == h ? 0u : y + 1u) * w};
    uint32_t k = 0;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
            if (dx != 1 || dy != 1) nb[k++] = rs[dy] + xs[dx];
}

// Cells of instance I: every cell index read from an object field is checked
// against it before it addresses the instance's grids (dsoa_index_ok).
__device__ __forceinline__ uint64_t cells_of(const dsoa_inst& I) { return (uint64_t)I.w * I.h; }

struct CellCtor {
    using Args = dsoa_gol_args;
    static __device__ void ctor(const dsoa_ctx& c, dsoa_obj o, uint64_t i, const Args& a) {
        const dsoa_inst& I = a.inst[a.target];
        const uint32_t cell = (uint32_t)i;
        dsoa_field<uint32_t>(c, o, 0) = a.target;
        dsoa_field<uint32_t>(c, o, 1) = cell;
        dsoa_field<uint32_t>(c, o, 2) = 0u;
        const bool alive = a.init ? (a.init[cell] != 0)
                                  : (dsoa_philox_w0(I.seed, 0xFFFFFFFFu, cell, 0u, 0u) < (1u << 30));
        dsoa_field<uint8_t>(c, o, 3) = (uint8_t)alive;
        I.cellmap[cell] = o;
        if (alive) {
            const dsoa_obj ag = dsoa_new(c, (uint32_t)a.alive_type);
            if (ag) {
                dsoa_field<uint32_t>(c, ag, 0) = a.target;
                dsoa_field<uint32_t>(c, ag, 1) = cell;
            }
        }
    }
};

// Alive.spread: one atomic increment of each of the 8 neighbours' counts.
struct Spread {
    using Args = dsoa_gol_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        const dsoa_inst I = a.inst[k];
        if (I.state != DSOA_INST_RUN) return;
        const uint32_t cell = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (!dsoa_index_ok(c, cell, cells_of(I))) return;
        uint32_t nc[8];
        moore(cell, I.w, I.h, nc);
        dsoa_obj nb[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) nb[k] = I.cellmap[nc[k]];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (nb[k]) atomicAdd(&dsoa_field<uint32_t>(c, nb[k], 2), 1u);
    }
};

// Alive.reap: a live cell survives with 2 or 3 live neighbours; otherwise the
// cell dies and the agent deletes itself.
struct Reap {
    using Args = dsoa_gol_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        const dsoa_inst& I = a.inst[k];
        if (I.state != DSOA_INST_RUN) return;
        const uint32_t cell = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (!dsoa_index_ok(c, cell, cells_of(I))) return;
        const dsoa_obj co = I.cellmap[cell];
        if (!co) return;
        const uint32_t n = dsoa_field<uint32_t>(c, co, 2);
        if (n != 2u && n != 3u) {
            dsoa_field<uint8_t>(c, co, 3) = 0;
            dsoa_delete(c, dsoa_make_handle(t, bid, s));
        }
    }
};

// Cell.decide: a dead cell with exactly 3 live neighbours is born (new Alive).
struct Decide {
    using Args = dsoa_gol_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        if (a.inst[k].state != DSOA_INST_RUN) return;
        uint32_t* cnt = dsoa_column<uint32_t>(c, t, bid, 2) + s;
        uint8_t* alive = dsoa_column<uint8_t>(c, t, bid, 3) + s;
        if (!*alive && *cnt == 3u) {
            const dsoa_obj ag = dsoa_new(c, (uint32_t)a.alive_type);
            if (ag) {
                dsoa_field<uint32_t>(c, ag, 0) = k;
                dsoa_field<uint32_t>(c, ag, 1) = dsoa_column<uint32_t>(c, t, bid, 1)[s];
                *alive = 1;
            }
        }
        *cnt = 0u;
    }
};

// Cell.decide that also advances the step counter of every running instance
// (no method of a generation reads it): CTA 0 does it in its prologue, so the
// generation needs no launch of its own for it.
struct DecideAdvance : Decide {
    static __device__ void prologue(const dsoa_ctx&, const Args& a) {
        for (uint32_t i = threadIdx.x; i < a.n_inst; i += blockDim.x)
            if (a.inst[i].state == DSOA_INST_RUN) a.inst[i].t += 1u;
    }
};

struct Read {
    using Args = dsoa_gol_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        uint8_t* occ = a.inst[k].occ;
        const uint32_t cell = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (occ && dsoa_index_ok(c, cell, cells_of(a.inst[k]))) occ[cell] = dsoa_column<uint8_t>(c, t, bid, 3)[s];
    }
};

struct Kill {
    using Args = dsoa_gol_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t k = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, k, a.n_inst)) return;
        if (a.inst[k].state == DSOA_INST_KILL) dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

__global__ void k_advance(dsoa_inst* inst, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && inst[i].state == DSOA_INST_RUN) inst[i].t += 1u;
}

}  // namespace

int dsoa_gol_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb) {
    dsoa_gol_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (ctor != DSOA_C_GOL_CELL) return DSOA_ERR_UNKNOWN_METHOD;
    if (!args.inst || args.target >= args.n_inst || type != args.cell_type || args.alive_type < 0 ||
        args.alive_type >= h->ntypes)
        return DSOA_ERR_INVALID_ARG;
    return dsoa_run_new<CellCtor>(h, type, n, args);
}

int dsoa_gol_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_gol_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (!args.inst) return DSOA_ERR_INVALID_ARG;
    switch (method) {
        case DSOA_M_GOL_SPREAD: return dsoa_run_doall<Spread>(h, type, args);
        case DSOA_M_GOL_REAP: return dsoa_run_doall<Reap>(h, type, args);
        case DSOA_M_GOL_DECIDE: return dsoa_run_doall<Decide>(h, type, args);
        case DSOA_M_GOL_DECIDE_ADVANCE: return dsoa_run_doall<DecideAdvance>(h, type, args);
        case DSOA_M_GOL_READ: return dsoa_run_doall<Read>(h, type, args);
        case DSOA_M_GOL_KILL: return dsoa_run_doall<Kill>(h, type, args);
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}

int dsoa_gol_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb) {
    dsoa_gol_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (kernel != DSOA_K_GOL_ADVANCE) return DSOA_ERR_UNKNOWN_METHOD;
    if (!args.inst || n > args.n_inst) return DSOA_ERR_INVALID_ARG;
    if (n == 0) return DSOA_OK;
    k_advance<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(args.inst, (uint32_t)n);
    return dsoa_check_launch(h);
}
