/*
 * dsoa_oracle.h -- sequential CPU oracle for the Single-Method Multiple-Objects
 * (SMMO) runtime of DynaSOAr (Springer & Masuhara, ECOOP 2019).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the package
 * smoke check and the benchmark's CPU-baseline leg may load this library.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * What it models: the SMMO semantics of Sec. 2.1 -- `new`, `delete`,
 * `parallel_new`, and `parallel_do` (run one method on every object of a type
 * that existed when the do-all started) -- over a plain free-list object store.
 * Placement is not modelled: the paper's allocator may put an object in any
 * free slot, and every workload result here is a function of logical ids only.
 *
 * Parity status per function (see the test files under tests/ for the pins):
 *   orc_philox4x32      pinned: published known-answer vectors (Salmon et al. SC'11)
 *   orc_splitmix64      pinned: published first outputs of SplitMix64 from state 0
 *   orc_micro_run       pinned: closed forms (x recurrence, expected live counts),
 *                       brute-force recomputation per object, order independence
 *   orc_gol_run         pinned: blinker, glider, block still-life, numpy roll-sum,
 *                       initial cells from the Philox known answers
 *   orc_wator_run       pinned: a cell-indexed brute force on 4x4..6x6 tori
 *                       (random grids, shark breeding, high seed words, step
 *                       offsets), hand-derived picks with 2, 3 and 4 candidates
 *                       from the Philox known answers, hand-derived single- and
 *                       two-agent cases, conservation, order independence; 21
 *                       planted mistakes each fail at least three pins
 *   orc_wator_frag      (frag_model.c, analysis) pinned: populations equal
 *                       orc_wator_run's at every record; block accounting
 *   orc_traffic_run     pinned: deterministic (p=0) closed forms of Nagel &
 *                       Schreckenberg 1992, conservation, brute force on L=16
 *   orc_nbody_run       pinned: two-body closed forms (first step of a pair at
 *                       rest, circular orbit), free motion, Newton's third law
 *                       exactly, hand-derived merges and merge chains, mass
 *                       conservation, order independence
 */
#ifndef DSOA_ORACLE_H
#define DSOA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based generators (published definitions, own code) ---- */
void     orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds,
                        uint32_t out[4]);
uint64_t orc_splitmix64(uint64_t state);             /* one output for `state` */
uint64_t orc_sm2(uint64_t a, uint64_t b);            /* sm(sm(a) ^ b)          */
uint64_t orc_sm3(uint64_t a, uint64_t b, uint64_t c);/* sm(sm2(a,b) ^ c)       */

/* ---- microbench: 1 type {int32 id, float x, int64 tag} ---- */
typedef struct {
    uint64_t live;      /* objects alive at the end of the round           */
    int64_t  sum_id;    /* sum of id over live objects                      */
    uint64_t sum_tag;   /* wrapping sum of tag                              */
    uint64_t xor_tag;   /* xor of tag                                       */
    double   sum_x;     /* sum of (double)x                                 */
    uint64_t news;      /* allocations this round                           */
    uint64_t deletes;   /* deallocations this round                         */
} orc_micro_round;

/* Runs `rounds` rounds of {parallel_new n_per_round; do x=x*1.5f+id; delete
 * where sm3(seed,id,round)&1}.  x_by_id / live_by_id (length rounds*n_per_round,
 * nullable) receive the final per-object state.  order_seed != 0 visits every
 * do-all snapshot in a shuffled order.  Returns 0, or -1 on allocation failure. */
int orc_micro_run(uint64_t seed, uint32_t n_per_round, uint32_t rounds,
                  uint64_t order_seed, orc_micro_round* out_rounds,
                  float* x_by_id, uint8_t* live_by_id);

/* ---- Game of Life as SMMO: Cell per site + Alive agent per live cell ---- */
/* init: nullable w*h bytes (0/1); when NULL the grid is drawn from `seed`.
 * out_grid: w*h bytes after `gens` generations.  alive_per_gen: gens+1 counts of
 * live cells (index 0 = initial); alive_objs_per_gen: gens+1 counts of Alive
 * objects in the store (must equal the former).  Returns 0 or -1. */
int orc_gol_run(uint32_t w, uint32_t h, const uint8_t* init, uint64_t seed,
                uint32_t gens, uint64_t order_seed, uint8_t* out_grid,
                uint32_t* alive_per_gen, uint32_t* alive_objs_per_gen);

/* ---- Wa-Tor predator-prey ---- */
typedef struct {
    uint32_t fish, sharks;              /* populations after the step       */
    uint32_t fish_births, shark_births; /* objects created during the step  */
    uint32_t eaten, starved;            /* fish eaten / sharks starved      */
    uint32_t fish_moves, shark_moves;   /* successful moves                 */
} orc_wator_step;

/* init: nullable w*h bytes (0 empty, 1 fish, 2 shark; agents start at age 0,
 * sharks with energy 3).  When NULL the grid is drawn from `seed`.  Step t uses
 * Philox counters with step index t0 + t.  out_occ: final w*h grid.  stats:
 * `steps` entries.  Returns 0 or -1. */
int orc_wator_run(uint32_t w, uint32_t h, const uint8_t* init, uint64_t seed,
                  uint32_t steps, uint32_t t0, uint64_t order_seed,
                  uint8_t* out_occ, orc_wator_step* stats);

/* Fragmentation of an idealised sequential allocator on the Wa-Tor run drawn
 * from `seed` (frag_model.c; analysis of Sec. 6.4, not a model of the GPU
 * allocator): policy 0 first fit, 1 best fit, 2 random fit, 3 random fit with
 * 8192 per-slot block hints, 4 the same with draining (a block fallen to 8
 * objects or fewer is left out until filled or emptied) over 64-slot blocks.
 * Every `every` steps one record: F = 1 - objects / (64 x blocks in use), fish,
 * sharks and blocks (arrays of steps / every entries; any may be NULL).
 * Returns 0 or -1. */
int orc_wator_frag(uint32_t w, uint32_t h, uint64_t seed, uint32_t steps, int policy, uint32_t every,
                   double* F_out, uint32_t* fish_out, uint32_t* sharks_out, uint32_t* blocks_out);

/* ---- batched Nagel-Schreckenberg rings ---- */
/* L[i], thr[i]: ring lengths and initial-density thresholds (u32 compare).
 * init_occ / init_v: nullable sum(L) bytes each; when init_occ is NULL the rings
 * are drawn from `seed`.  slow_thr / ramp_thr: u32 thresholds of the random
 * slow-down and of the ramp events (0.2 and 0.05 in the configured workload).
 * out_occ / out_v: sum(L) bytes (final occupancy and speed per cell).
 * cars_per_step: nullable (steps+1)*n_inst counts.  first_ring is the batch
 * index of ring 0 in the Philox counters, so that one ring of a batch can be
 * replayed alone.  Returns 0 or -1. */
int orc_traffic_run(uint32_t n_inst, uint32_t first_ring, const uint32_t* L, const uint32_t* thr,
                    uint64_t seed, uint32_t steps, uint32_t slow_thr,
                    uint32_t ramp_thr, const uint8_t* init_occ,
                    const uint8_t* init_v, uint64_t order_seed,
                    uint8_t* out_occ, uint8_t* out_v, uint32_t* cars_per_step);

/* ---- n-body and particle collisions (one type, Body) ---- */
typedef struct {
    float    G;         /* gravitational constant (a power of two)              */
    float    dt;        /* time step                                            */
    float    eps2;      /* softening added to the squared distance in FORCE (>0)*/
    float    rc2;       /* collisions: merge below this squared distance        */
    float    fscale;    /* fixed-point scale S of the force sums (a power of 2) */
    float    vscale;    /* initial velocities in [-vscale/2, vscale/2)          */
    uint32_t mass_max;  /* initial masses are the integers 1..mass_max          */
    uint32_t collide;   /* 0: n-body (FORCE, MOVE); 1: + FIND, CLAIM, MERGE, DELETE */
} orc_nbody_params;

/* n bodies with ids 0..n-1, initial state from `init` (nullable, n x 5 floats
 * px, py, vx, vy, m) or drawn from `seed`; `steps` steps.  out: n x 5 floats
 * of the final state by id (zeros for merged bodies), out_alive: n bytes,
 * count_per_step: steps+1 body counts, force_sum: 2*steps wrapped sums of the
 * fixed-point forces of each FORCE do-all (all nullable).  Returns 0 or -1. */
int orc_nbody_run(uint32_t n, const float* init, uint64_t seed, const orc_nbody_params* p,
                  uint32_t steps, uint64_t order_seed, float* out, uint8_t* out_alive,
                  uint32_t* count_per_step, int64_t* force_sum);

/* The fixed-point force of one FORCE do-all on body i of a state (n x 5 floats
 * px, py, vx, vy, m by id), summed over every other body j with alive[j]
 * (alive nullable: all).  Used to check single bodies of large runs.
 * Returns 0 or -1. */
int orc_nbody_force_on(uint32_t n, const float* state, const uint8_t* alive,
                       const orc_nbody_params* p, uint32_t i, int64_t out[2]);

#ifdef __cplusplus
}
#endif
#endif
