/*
 * dsoa_apps.h -- built-in constructors, do-all methods and plain kernels of the
 * workloads, addressed by id through dsoa_parallel_new / dsoa_parallel_do /
 * dsoa_run_kernel (dsoa.h).  Each id takes one argument struct, copied by value
 * at launch (args_bytes must equal its sizeof).  Device pointers inside the
 * structs are caller-owned and must stay valid until the work has run.
 *
 * Workloads (Table 1 of the paper; rules as stated per section below):
 *   microbench  one type {int32 id, float x, int64 tag}
 *   game of life  Cell per site + Alive agent per live cell, B3/S23 torus
 *   wa-tor      Fish / Shark agents on a torus with per-cell occupancy
 *   traffic     Nagel-Schreckenberg cars on batched rings
 *   n-body / collisions  Body objects under pairwise gravity (device_do), merged
 *               by perfectly inelastic collisions
 */
#ifndef DSOA_APPS_H
#define DSOA_APPS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- microbench (type fields: 0 id i32, 1 x f32, 2 tag u64) ---------- */
#define DSOA_C_MICRO 100              /* ctor i: id = id_base + i, x = 0, tag = sm2(seed,id) */
#define DSOA_M_MICRO_SCALE 101        /* x = x * 1.5f + (float)id, 128-bit vectorised       */
#define DSOA_M_MICRO_SCALE_SCALAR 102 /* same, one slot per thread (generic do-all kernel)  */
#define DSOA_M_MICRO_DELETE 103       /* delete this where sm3(seed, id, round) is odd     */
#define DSOA_M_MICRO_GATHER 104       /* x_out[id] = x, live_out[id] = 1                   */
#define DSOA_M_MICRO_STATS 105        /* accumulate dsoa_micro_stats                        */
#define DSOA_M_MICRO_SCALE_TMA 106    /* same as SCALE, columns staged by bulk async copies */
#define DSOA_M_MICRO_DELETE_ALL 107   /* delete this (every object of the snapshot)         */
#define DSOA_M_MICRO_HANDLES 108      /* handles_out[id] = handle of the object with that id */
#define DSOA_K_MICRO_DEVICE_DO 150    /* n threads; thread i visits every object with device_do
                                         and writes (count, sum of id) to stats[i] as two u64 */
#define DSOA_K_MICRO_ATOMIC_PEAK 151  /* n threads; thread i issues `round` 64-bit atomics with
                                         return (atomicAnd / atomicOr alternating) on the words
                                         handles_out[0 .. n_ids), word (i + k n) * 17 mod n_ids
                                         at its k-th op, so that every lane's op is its own L2
                                         request (n_ids a power of two >= 32, caller-owned
                                         device buffer).  The XOR of the returned words is
                                         stored to *(u64*)stats only when it equals seed.  It
                                         measures the L2 ceiling of single-lane bitmap atomics,
                                         the operation the allocator is built from (Sec. 4). */
#define DSOA_K_MICRO_NEW_EACH 152     /* n threads; thread i creates `round` microbench objects
                                         one after another (a loop of device new, the
                                         per-thread allocation pattern of the Linux
                                         scalability benchmark, Sec. 6.5); object j of
                                         thread i gets id = id_base + i * round + j.  n_ids
                                         holds the type to allocate (the microbench type or
                                         a type extending it).  A full heap leaves the
                                         remaining objects unallocated (DSOA_DEV_OOM). */
typedef struct {
    uint64_t seed;       /* SplitMix64 key                                   */
    uint32_t id_base;    /* constructor: first id                            */
    uint32_t round;      /* delete: round index                              */
    float* x_out;        /* gather: [n_ids] (device)                         */
    uint8_t* live_out;   /* gather: [n_ids] (device)                         */
    uint64_t n_ids;      /* gather: bound of id                              */
    void* stats;         /* stats: dsoa_micro_stats* (device, pre-zeroed)    */
    uint64_t* handles_out; /* handles: [n_ids] (device)                      */
} dsoa_micro_args;
typedef struct {
    unsigned long long live, sum_id, sum_tag, xor_tag;
    double sum_x;
} dsoa_micro_stats;

/* ---------------- instances of the grid workloads (game of life, wa-tor) ----------- */
/* One entry per instance slot; the table lives in device memory.  Objects keep
 * (inst, cell) so that one launch serves every instance of a batch. */
#define DSOA_INST_IDLE 0u    /* slot unused / finished: methods leave it alone     */
#define DSOA_INST_RUN 1u     /* stepping                                           */
#define DSOA_INST_KILL 2u    /* KILL methods delete its objects                    */
typedef struct {
    uint64_t* cellmap;   /* [w*h] game of life: Cell handle; wa-tor: agent handle  */
    uint8_t* occ;        /* [w*h] game of life: READ output; wa-tor: 0/1/2 grid    */
    uint32_t* claim;     /* [w*h] wa-tor: move claims, all 0xFFFFFFFF between steps */
    uint64_t seed;       /* Philox key of the instance                             */
    uint32_t w, h;       /* torus size                                             */
    uint32_t t;          /* the instance's own step index                          */
    uint32_t state;      /* DSOA_INST_*                                            */
} dsoa_inst;

/* ---------------- game of life: Cell {0 inst u32, 1 cell u32, 2 count u32, 3 alive u8};
 *                  Alive {0 inst u32, 1 cell u32} ------------------------------------ */
#define DSOA_C_GOL_CELL 200      /* ctor i = cell of instance `target`; initial state from
                                    `init` (nullable) or Philox(seed; 0xFFFFFFFF, i, 0, 0)
                                    < 2^30; creates the Alive agent of a live cell        */
#define DSOA_M_GOL_SPREAD 201    /* Alive: add 1 to the 8 neighbours' counts              */
#define DSOA_M_GOL_REAP 202      /* Alive: die (delete this) unless count is 2 or 3       */
#define DSOA_M_GOL_DECIDE 203    /* Cell: dead with count 3 -> new Alive; count = 0       */
#define DSOA_M_GOL_READ 204      /* Cell: occ[cell] = alive                               */
#define DSOA_M_GOL_KILL 205      /* Cell or Alive of a KILL instance: delete this         */
#define DSOA_M_GOL_DECIDE_ADVANCE 206 /* DECIDE, and t += 1 for RUN instances (the same as
                                        K_GOL_ADVANCE after it, without its launch)        */
#define DSOA_K_GOL_ADVANCE 250   /* n = n_inst: t += 1 for RUN instances                  */
typedef struct {
    dsoa_inst* inst;     /* [n_inst] device table                                   */
    const uint8_t* init; /* ctor: nullable [w*h] of `target`                        */
    uint32_t n_inst;
    uint32_t target;     /* ctor: instance slot being populated                     */
    int32_t cell_type, alive_type;
} dsoa_gol_args;

/* ---------------- wa-tor: Fish {0 inst, 1 cell, 2 age, 3 target};
 *                  Shark {0 inst, 1 cell, 2 age, 3 energy, 4 target, 5 eat} (u32) ---- */
#define DSOA_M_WATOR_FISH_CHOOSE 301   /* pick an empty neighbour, atomicMin claim       */
#define DSOA_M_WATOR_FISH_MOVE 302     /* winners move; breeding age 3 leaves a newborn  */
#define DSOA_M_WATOR_SHARK_CHOOSE 303  /* prefer a fish neighbour, else an empty one     */
#define DSOA_M_WATOR_SHARK_MOVE 304    /* eat (energy 3) or lose 1; breed at 10; starve  */
#define DSOA_M_WATOR_KILL 305          /* agent of a KILL instance: delete this          */
#define DSOA_M_WATOR_FISH_MOVE_DEFER 306 /* FISH_MOVE whose newborns are only marked (occ 3
                                          at the old cell); K_WATOR_BIRTHS creates them  */
#define DSOA_M_WATOR_SHARK_MOVE_ADVANCE 307 /* SHARK_MOVE, and t += 1 for RUN instances (the
                                               same as K_WATOR_ADVANCE after it, without
                                               its launch)                                 */
#define DSOA_K_WATOR_INIT 350          /* n = w*h of `target`: agents from `init` (nullable,
                                          0/1/2) or Philox(seed; 0xFFFFFFFF, c, 0, 0) vs
                                          0.30 / 0.35 thresholds                          */
#define DSOA_K_WATOR_ADVANCE 351       /* n = n_inst: t += 1 for RUN instances            */
#define DSOA_K_WATOR_BIRTHS 352        /* n = n_inst: a Fish (age 0) at every cell marked
                                          3 by FISH_MOVE_DEFER in RUN instances; the cell
                                          becomes 1 (0 if the heap is full)              */
typedef struct {
    dsoa_inst* inst;
    const uint8_t* init;
    uint32_t n_inst;
    uint32_t target;
    int32_t fish_type, shark_type;
} dsoa_wator_args;

/* ---------------- traffic: Car {0 ring u32, 1 pos u32, 2 v u32} --------------------- */
#define DSOA_M_TRAFFIC_MOVE 401    /* accelerate, brake to gap, random slow-down, move,
                                      leave at the off-ramp L/2 with prob ramp_thr/2^32 */
#define DSOA_M_TRAFFIC_READ 402    /* vel_out[base+pos] = v                              */
#define DSOA_K_TRAFFIC_INIT 450    /* n = total cells: cars from `init_occ` (nullable) or
                                      Philox(seed; 0xFFFFFFFF, j, ring, 0) < thr          */
#define DSOA_K_TRAFFIC_CLEAR 451   /* n = total cells: next occupancy buffer = 0         */
#define DSOA_K_TRAFFIC_ONRAMP 452  /* n = rings: new car at an empty cell 0              */
#define DSOA_K_TRAFFIC_ADVANCE 453 /* n = 1: t += 1                                      */
#define DSOA_K_TRAFFIC_ONRAMP_ADVANCE 454 /* ONRAMP, then ADVANCE, in one launch (n = rings) */
typedef struct {
    uint8_t* occ0;               /* [total] occupancy, even steps read occ0           */
    uint8_t* occ1;               /* [total] occupancy, odd steps read occ1            */
    uint8_t* vel_out;            /* [total] READ output (pre-zeroed)                   */
    const uint64_t* ring_base;   /* [n_rings+1] first cell of each ring               */
    const uint32_t* ring_thr;    /* [n_rings] initial density threshold               */
    const uint8_t* init_occ;     /* nullable [total]                                   */
    const uint8_t* init_v;       /* nullable [total]                                   */
    uint32_t* t_dev;             /* [1] step index                                     */
    uint64_t seed;
    uint32_t n_rings;
    uint32_t slow_thr;           /* 858993459 = floor(0.2 * 2^32)                      */
    uint32_t ramp_thr;           /* 214748364 = floor(0.05 * 2^32)                     */
    int32_t car_type;
} dsoa_traffic_args;

/* ---------------- n-body / particle collisions (Table 1 "nbody", "collision"):
 *   Body {0 id u32, 1 px f32, 2 py f32, 3 vx f32, 4 vy f32, 5 m f32, 6 fx i64,
 *         7 fy i64, 8 target u32, 9 incoming u32, 10 merged u32}
 * Arithmetic: every float op is one binary32 op rounded to nearest (no FMA);
 * a pair term k (x_j - x_i), k = ((G S m_i) m_j) (1/d)^3, d = sqrt(|x_j - x_i|^2
 * + eps2), is clamped to +-2^62, rounded to an integer and summed in wrapping
 * 64-bit arithmetic, so a force does not depend on the order bodies are visited
 * in.  G and the fixed-point scale S are powers of two; masses are integers.
 * The force fields are zero between steps (the constructor and MOVE clear them).
 * n-body step: FORCE (or FORCE_TILED), MOVE.  Collision step: FORCE, MOVE,
 * FIND, CLAIM, MERGE, DELETE (one enumeration; the others reuse its snapshot),
 * or with DSOA_NBODY_KEYED_FIND: FORCE_TILED, MOVE, FIND_TILED, CLAIM, MERGE,
 * DELETE. */
#define DSOA_C_NBODY 500              /* ctor i: body id i from `init` (nullable, 5 floats
                                         px py vx vy m per id) or Philox(seed; 0xFFFFFFFF, i,
                                         k, 0) word 0, k = 0..4; handle_of[i] = handle      */
#define DSOA_M_NBODY_FORCE 501        /* F = sum of pair terms over every other body, by a
                                         device_do in the calling thread (Sec. 2.1)        */
#define DSOA_M_NBODY_MOVE 502         /* v += ((F / S) / m) dt; x += v dt; F = 0            */
#define DSOA_M_COLL_FIND 503          /* target = id of the nearest body with squared
                                         distance < rc2 that is heavier, or as heavy with a
                                         lower id (ties of distance: lower id), by device_do;
                                         incoming = none, merged = 0                         */
#define DSOA_M_COLL_CLAIM 504         /* atomicMin(incoming of the target, own id)          */
#define DSOA_M_COLL_MERGE 505         /* incoming and no target: absorb the winner (mass,
                                         momentum, centre of mass); mark it merged           */
#define DSOA_M_COLL_DELETE 506        /* merged: handle_of[id] = 0, delete this              */
#define DSOA_M_NBODY_READ 507         /* out[5 id + 0..4] = px py vx vy m; alive_out[id] = 1;
                                         force_out[2 id + 0..1] = fx fy when non-null         */
#define DSOA_M_NBODY_FORCE_TILED 508  /* FORCE's result (bit for bit) from a pairwise kernel
                                         over the enumerated snapshot: CTAs take tiles of
                                         bodies staged in shared memory and add their integer
                                         partial sums atomically.  By default each unordered
                                         pair is evaluated once and gives both bodies their
                                         terms (Newton's third law, exact in fixed point);
                                         with DSOA_NBODY_ALL_PAIRS every ordered pair is
                                         evaluated for its first body only.  Needs
                                         eps2 >= 2^-80 (else DSOA_ERR_INVALID_ARG)           */
#define DSOA_M_COLL_FIND_TILED 509    /* FIND's result by the pairwise kernel, in two halves:
                                         with DSOA_NBODY_KEYED_FIND, MOVE resets target,
                                         incoming, merged and sets fx to all ones; this
                                         method leaves min(bits(d2) << 32 | id) in fx; CLAIM
                                         turns it into the target and clears fx.  By
                                         default each unordered pair is evaluated once (the
                                         smaller body gets the candidate); with
                                         DSOA_NBODY_ALL_PAIRS every ordered pair           */
#define DSOA_NBODY_NONE 0xFFFFFFFFu   /* no target / no incoming proposal                    */
#define DSOA_NBODY_KEYED_FIND 1u      /* flags: the step uses FIND_TILED                     */
#define DSOA_NBODY_ALL_PAIRS 2u       /* flags: FORCE_TILED / FIND_TILED over ordered pairs   */
typedef struct {
    uint64_t* handle_of;  /* [n_ids] id -> handle; needed by collisions (CLAIM, MERGE read
                             it, the ctor writes it, DELETE clears it); nullable for n-body */
    const float* init;    /* ctor: nullable [n_ids * 5] (device)                          */
    float* out;           /* READ: [n_ids * 5] (device, pre-zeroed)                       */
    uint8_t* alive_out;   /* READ: [n_ids] (device, pre-zeroed)                           */
    int64_t* force_out;   /* READ: nullable [n_ids * 2] fixed-point forces (device)         */
    uint64_t seed;        /* Philox key of the initial draw                               */
    uint32_t n_ids;       /* bodies created by the ctor (ids 0 .. n_ids-1)                */
    uint32_t mass_max;    /* initial masses 1 .. mass_max                                 */
    float G;              /* gravitational constant (power of two)                        */
    float dt;             /* time step                                                    */
    float eps2;           /* softening added to the squared distance (> 0)                */
    float rc2;            /* squared merge distance                                       */
    float fscale;         /* fixed-point scale S (power of two)                           */
    float vscale;         /* initial velocities in [-vscale/2, vscale/2)                  */
    int32_t body_type;
    uint32_t flags;       /* DSOA_NBODY_KEYED_FIND (MOVE and CLAIM for FIND_TILED),
                             DSOA_NBODY_ALL_PAIRS (FORCE_TILED, FIND_TILED)               */
} dsoa_nbody_args;

#ifdef __cplusplus
}
#endif
#endif
