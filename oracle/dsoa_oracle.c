/*
 * dsoa_oracle.c -- sequential CPU oracle for the SMMO runtime (DynaSOAr,
 * Springer & Masuhara, ECOOP 2019).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Loaded only by tests/, by the package
 * smoke check and by the benchmark's CPU-baseline leg.  It shares nothing with
 * the CUDA path.  Build: plain C11, -O2 -ffp-contract=off (the microbench's
 * fp32 update is a multiply followed by a separately rounded add).
 *
 * Semantics follow Sec. 2.1 of the paper: `parallel_new<T>(n)` runs a
 * constructor with ids 0..n-1; `parallel_do<T,f>` runs f on every object of T
 * that existed when the do-all began (objects created meanwhile are not
 * visited, Sec. 3.1 "iteration bitmap"); f may delete `this` and objects of
 * other types.  The object store is a free-list heap: placement is not the
 * paper's, and no result below depends on placement or visiting order.
 */
#include "dsoa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy  */
/* as 1, 2, 3", SC'11, Sec. 4.2).  Each round multiplies the two "right"    */
/* words by fixed odd constants, keeps both halves of the 64-bit products,  */
/* xors the high halves with the "left" words and the round key, and        */
/* permutes the four words; the two key words advance by Weyl increments    */
/* (golden ratio and sqrt(3)-1) between rounds.                              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds,
                    uint32_t out[4]) {
    const uint32_t MUL_A = 0xD2511F53u, MUL_B = 0xCD9E8D57u;
    const uint32_t WEYL_A = 0x9E3779B9u, WEYL_B = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) { k0 += WEYL_A; k1 += WEYL_B; }
        uint64_t pa = (uint64_t)MUL_A * (uint64_t)x0;
        uint64_t pb = (uint64_t)MUL_B * (uint64_t)x2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t n0 = pb_hi ^ x1 ^ k0;
        uint32_t n1 = pb_lo;
        uint32_t n2 = pa_hi ^ x3 ^ k1;
        uint32_t n3 = pa_lo;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t philox_w0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                          uint32_t c3) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32(ctr, key, 10, out);
    return out[0];
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, "Fast Splittable Pseudorandom Number     */
/* Generators", OOPSLA'14): the state advances by the odd "golden gamma"   */
/* and each output is a 64-bit finaliser of the new state.  The finaliser   */
/* constants are those of the JDK 8 SplittableRandom / public-domain C      */
/* splitmix64 (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31).*/
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
uint64_t orc_sm2(uint64_t a, uint64_t b) { return orc_splitmix64(orc_splitmix64(a) ^ b); }
uint64_t orc_sm3(uint64_t a, uint64_t b, uint64_t c) { return orc_splitmix64(orc_sm2(a, b) ^ c); }

/* ------------------------------------------------------------------------ */
/* Object store: a free-list heap of fixed-size records for one type.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    size_t    rec;
    uint8_t*  data;
    uint8_t*  live;
    uint32_t* freelist;
    uint32_t  cap, hw, nfree, nlive;
    int       failed;
} store_t;

static void store_init(store_t* s, size_t rec) {
    memset(s, 0, sizeof(*s));
    s->rec = rec;
}
static void store_free(store_t* s) {
    free(s->data); free(s->live); free(s->freelist);
    memset(s, 0, sizeof(*s));
}
static int store_grow(store_t* s) {
    uint32_t ncap = s->cap ? s->cap * 2u : 1024u;
    uint8_t* d = (uint8_t*)realloc(s->data, (size_t)ncap * s->rec);
    if (!d) return -1;
    s->data = d;
    uint8_t* l = (uint8_t*)realloc(s->live, ncap);
    if (!l) return -1;
    s->live = l;
    uint32_t* f = (uint32_t*)realloc(s->freelist, (size_t)ncap * sizeof(uint32_t));
    if (!f) return -1;
    s->freelist = f;
    s->cap = ncap;
    return 0;
}
/* `new`: returns the index of a zero-initialised record, or UINT32_MAX. */
static uint32_t store_new(store_t* s) {
    uint32_t idx;
    if (s->nfree) {
        idx = s->freelist[--s->nfree];
    } else {
        if (s->hw == s->cap && store_grow(s) != 0) { s->failed = 1; return UINT32_MAX; }
        idx = s->hw++;
    }
    s->live[idx] = 1;
    memset(s->data + (size_t)idx * s->rec, 0, s->rec);
    s->nlive++;
    return idx;
}
/* `delete`: deleting a dead record is a usage error and marks the store. */
static void store_delete(store_t* s, uint32_t idx) {
    if (idx >= s->hw || !s->live[idx]) { s->failed = 1; return; }
    s->live[idx] = 0;
    s->freelist[s->nfree++] = idx;
    s->nlive--;
}
static void* store_get(store_t* s, uint32_t idx) { return s->data + (size_t)idx * s->rec; }

/* The do-all snapshot: every live index at entry, in increasing index order,
 * or shuffled (Fisher-Yates driven by SplitMix64) when order_seed != 0.
 * The caller frees the returned array. */
static uint32_t* store_snapshot(const store_t* s, uint64_t order_seed, uint32_t* n_out) {
    uint32_t n = 0;
    uint32_t* out = (uint32_t*)malloc((size_t)(s->nlive ? s->nlive : 1) * sizeof(uint32_t));
    if (!out) { *n_out = 0; return NULL; }
    for (uint32_t i = 0; i < s->hw; ++i)
        if (s->live[i]) out[n++] = i;
    if (order_seed) {
        uint64_t st = order_seed;
        for (uint32_t i = n; i > 1; --i) {
            st += 1;
            uint32_t j = (uint32_t)(orc_splitmix64(st) % i);
            uint32_t t = out[i - 1]; out[i - 1] = out[j]; out[j] = t;
        }
    }
    *n_out = n;
    return out;
}

/* ------------------------------------------------------------------------ */
/* Microbench (allocator + do-all).  One type {int32 id, float x, int64 tag}. */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t id; float x; uint64_t tag; } micro_obj;

int orc_micro_run(uint64_t seed, uint32_t n_per_round, uint32_t rounds,
                  uint64_t order_seed, orc_micro_round* out_rounds,
                  float* x_by_id, uint8_t* live_by_id) {
    store_t st;
    store_init(&st, sizeof(micro_obj));
    int rc = 0;
    for (uint32_t rd = 0; rd < rounds && rc == 0; ++rd) {
        orc_micro_round stat;
        memset(&stat, 0, sizeof(stat));
        /* parallel_new<T>(n): constructor id i -> global id rd*n + i */
        for (uint32_t i = 0; i < n_per_round; ++i) {
            uint32_t k = store_new(&st);
            if (k == UINT32_MAX) { rc = -1; break; }
            micro_obj* o = (micro_obj*)store_get(&st, k);
            o->id = (int32_t)(rd * n_per_round + i);
            o->x = 0.0f;
            o->tag = orc_sm2(seed, (uint64_t)(uint32_t)o->id);
            stat.news++;
        }
        /* parallel_do: x = x * 1.5f + (float)id, two separate fp32 roundings */
        uint32_t n;
        uint32_t* snap = store_snapshot(&st, order_seed ? order_seed + 2u * rd + 1u : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            micro_obj* o = (micro_obj*)store_get(&st, snap[j]);
            float prod = o->x * 1.5f;
            o->x = prod + (float)o->id;
        }
        free(snap);
        /* parallel_do: delete this where sm3(seed, id, round) is odd */
        snap = store_snapshot(&st, order_seed ? order_seed + 2u * rd + 2u : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            micro_obj* o = (micro_obj*)store_get(&st, snap[j]);
            if (orc_sm3(seed, (uint64_t)(uint32_t)o->id, rd) & 1u) {
                store_delete(&st, snap[j]);
                stat.deletes++;
            }
        }
        free(snap);
        for (uint32_t i = 0; i < st.hw; ++i) {
            if (!st.live[i]) continue;
            micro_obj* o = (micro_obj*)store_get(&st, i);
            stat.live++;
            stat.sum_id += o->id;
            stat.sum_tag += o->tag;
            stat.xor_tag ^= o->tag;
            stat.sum_x += (double)o->x;
        }
        if (out_rounds) out_rounds[rd] = stat;
    }
    if (rc == 0 && (x_by_id || live_by_id)) {
        uint64_t total = (uint64_t)rounds * n_per_round;
        if (x_by_id) memset(x_by_id, 0, total * sizeof(float));
        if (live_by_id) memset(live_by_id, 0, total);
        for (uint32_t i = 0; i < st.hw; ++i) {
            if (!st.live[i]) continue;
            micro_obj* o = (micro_obj*)store_get(&st, i);
            if (x_by_id) x_by_id[o->id] = o->x;
            if (live_by_id) live_by_id[o->id] = 1;
        }
    }
    if (st.failed) rc = -1;
    store_free(&st);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Game of Life (Table 1 "game-of-life"), B3/S23 on a torus.                 */
/* Cell objects, one per site (parallel_new with id = site index); an Alive  */
/* object exists exactly while its cell is alive.  One generation is three   */
/* do-alls: Alive.spread (add 1 to the 8 neighbours' counts), Alive.reap     */
/* (die unless count is 2 or 3), Cell.decide (birth on count 3; reset).      */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t cell; uint32_t count; uint8_t alive; } gol_cell;
typedef struct { uint32_t cell; } gol_alive;

static uint32_t torus_nb(uint32_t c, uint32_t w, uint32_t h, int dx, int dy) {
    uint32_t x = c % w, y = c / w;
    uint32_t nx = (uint32_t)(((int64_t)x + dx + (int64_t)w) % (int64_t)w);
    uint32_t ny = (uint32_t)(((int64_t)y + dy + (int64_t)h) % (int64_t)h);
    return ny * w + nx;
}

int orc_gol_run(uint32_t w, uint32_t h, const uint8_t* init, uint64_t seed,
                uint32_t gens, uint64_t order_seed, uint8_t* out_grid,
                uint32_t* alive_per_gen, uint32_t* alive_objs_per_gen) {
    if (w == 0 || h == 0) return -1;
    uint32_t ncell = w * h;
    store_t cells, alives;
    store_init(&cells, sizeof(gol_cell));
    store_init(&alives, sizeof(gol_alive));
    uint32_t* cellmap = (uint32_t*)malloc((size_t)ncell * sizeof(uint32_t));
    if (!cellmap) return -1;
    int rc = 0;
    /* parallel_new<Cell>(w*h): the constructor draws the initial state */
    for (uint32_t c = 0; c < ncell; ++c) {
        uint32_t k = store_new(&cells);
        if (k == UINT32_MAX) { rc = -1; break; }
        cellmap[c] = k;
        gol_cell* cc = (gol_cell*)store_get(&cells, k);
        cc->cell = c;
        cc->count = 0;
        int alive = init ? (init[c] != 0)
                         : (philox_w0(seed, 0xFFFFFFFFu, c, 0, 0) < (1u << 30));
        cc->alive = (uint8_t)alive;
        if (alive) {
            uint32_t a = store_new(&alives);
            if (a == UINT32_MAX) { rc = -1; break; }
            ((gol_alive*)store_get(&alives, a))->cell = c;
        }
    }
    static const int DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    static const int DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    for (uint32_t g = 0; g <= gens && rc == 0; ++g) {
        if (alive_per_gen || alive_objs_per_gen) {
            uint32_t cnt = 0;
            for (uint32_t c = 0; c < ncell; ++c)
                cnt += ((gol_cell*)store_get(&cells, cellmap[c]))->alive;
            if (alive_per_gen) alive_per_gen[g] = cnt;
            if (alive_objs_per_gen) alive_objs_per_gen[g] = alives.nlive;
        }
        if (g == gens) break;
        uint64_t os = order_seed ? order_seed + 3ull * g : 0;
        uint32_t n;
        /* do-all Alive.spread */
        uint32_t* snap = store_snapshot(&alives, os ? os + 1 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t c = ((gol_alive*)store_get(&alives, snap[j]))->cell;
            for (int d = 0; d < 8; ++d) {
                uint32_t nb = torus_nb(c, w, h, DX[d], DY[d]);
                ((gol_cell*)store_get(&cells, cellmap[nb]))->count += 1;
            }
        }
        free(snap);
        /* do-all Alive.reap: a live cell survives with 2 or 3 live neighbours */
        snap = store_snapshot(&alives, os ? os + 2 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t c = ((gol_alive*)store_get(&alives, snap[j]))->cell;
            gol_cell* cc = (gol_cell*)store_get(&cells, cellmap[c]);
            if (cc->count != 2 && cc->count != 3) {
                cc->alive = 0;
                store_delete(&alives, snap[j]);
            }
        }
        free(snap);
        /* do-all Cell.decide: a dead cell with exactly 3 live neighbours is born */
        snap = store_snapshot(&cells, os ? os + 3 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            gol_cell* cc = (gol_cell*)store_get(&cells, snap[j]);
            if (!cc->alive && cc->count == 3) {
                uint32_t a = store_new(&alives);
                if (a == UINT32_MAX) { rc = -1; break; }
                ((gol_alive*)store_get(&alives, a))->cell = cc->cell;
                cc->alive = 1;
            }
            cc->count = 0;
        }
        free(snap);
    }
    if (rc == 0 && out_grid)
        for (uint32_t c = 0; c < ncell; ++c)
            out_grid[c] = ((gol_cell*)store_get(&cells, cellmap[c]))->alive;
    if (cells.failed || alives.failed) rc = -1;
    free(cellmap);
    store_free(&cells);
    store_free(&alives);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Wa-Tor (Table 1 "wa-tor"; Dewdney 1984).  Grid cells 0 empty, 1 fish,    */
/* 2 shark; von Neumann neighbourhood visited in the order N, E, S, W.       */
/* Per step t: Fish.choose, Fish.move, Shark.choose, Shark.move (four        */
/* do-alls).  A mover claims its target with min(source cell), so the       */
/* lowest source index wins; a mover whose age reaches the breeding age      */
/* leaves a newborn (age 0) behind and restarts its own age.  A shark that   */
/* eats refills its energy to 3, otherwise loses 1, and dies at 0.           */
/* ------------------------------------------------------------------------ */
#define WT_NONE 0xFFFFFFFFu
#define WT_FISH_BREED 3u
#define WT_SHARK_BREED 10u
#define WT_SHARK_ENERGY 3u
#define WT_FISH_THR 1288490188u   /* floor(0.30 * 2^32) */
#define WT_SHARK_THR 1503238553u  /* floor(0.35 * 2^32): fish or shark */

typedef struct { uint32_t cell, age, target; } wt_fish;
typedef struct { uint32_t cell, age, energy, target, eat; } wt_shark;

static void wt_neighbours(uint32_t c, uint32_t w, uint32_t h, uint32_t nb[4]) {
    nb[0] = torus_nb(c, w, h, 0, -1); /* N */
    nb[1] = torus_nb(c, w, h, 1, 0);  /* E */
    nb[2] = torus_nb(c, w, h, 0, 1);  /* S */
    nb[3] = torus_nb(c, w, h, -1, 0); /* W */
}

int orc_wator_run(uint32_t w, uint32_t h, const uint8_t* init, uint64_t seed,
                  uint32_t steps, uint32_t t0, uint64_t order_seed,
                  uint8_t* out_occ, orc_wator_step* stats) {
    if (w == 0 || h == 0) return -1;
    uint32_t ncell = w * h;
    uint8_t* occ = (uint8_t*)calloc(ncell, 1);
    uint32_t* agent = (uint32_t*)malloc((size_t)ncell * sizeof(uint32_t));
    uint32_t* claim = (uint32_t*)malloc((size_t)ncell * sizeof(uint32_t));
    if (!occ || !agent || !claim) { free(occ); free(agent); free(claim); return -1; }
    store_t fish, sharks;
    store_init(&fish, sizeof(wt_fish));
    store_init(&sharks, sizeof(wt_shark));
    int rc = 0;
    for (uint32_t c = 0; c < ncell; ++c) {
        agent[c] = WT_NONE;
        claim[c] = WT_NONE;
        uint8_t kind;
        if (init) {
            kind = init[c];
        } else {
            uint32_t u = philox_w0(seed, 0xFFFFFFFFu, c, 0, 0);
            kind = u < WT_FISH_THR ? 1 : (u < WT_SHARK_THR ? 2 : 0);
        }
        if (kind == 1) {
            uint32_t k = store_new(&fish);
            if (k == UINT32_MAX) { rc = -1; break; }
            wt_fish* f = (wt_fish*)store_get(&fish, k);
            f->cell = c; f->age = 0; f->target = WT_NONE;
            occ[c] = 1; agent[c] = k;
        } else if (kind == 2) {
            uint32_t k = store_new(&sharks);
            if (k == UINT32_MAX) { rc = -1; break; }
            wt_shark* s = (wt_shark*)store_get(&sharks, k);
            s->cell = c; s->age = 0; s->energy = WT_SHARK_ENERGY; s->target = WT_NONE;
            occ[c] = 2; agent[c] = k;
        }
    }
    for (uint32_t step = 0; step < steps && rc == 0; ++step) {
        uint32_t t = t0 + step;
        orc_wator_step ev;
        memset(&ev, 0, sizeof(ev));
        uint64_t os = order_seed ? order_seed + 4ull * step : 0;
        uint32_t n, nb[4], cand[4];
        /* do-all Fish.choose: pick an empty neighbour, claim it */
        uint32_t* snap = store_snapshot(&fish, os ? os + 1 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            wt_fish* f = (wt_fish*)store_get(&fish, snap[j]);
            wt_neighbours(f->cell, w, h, nb);
            uint32_t k = 0;
            for (int d = 0; d < 4; ++d) if (occ[nb[d]] == 0) cand[k++] = nb[d];
            f->target = WT_NONE;
            if (k) {
                uint32_t u = philox_w0(seed, t, f->cell, 1, 0);
                uint32_t tg = cand[u % k];
                f->target = tg;
                if (f->cell < claim[tg]) claim[tg] = f->cell;
            }
        }
        free(snap);
        /* do-all Fish.move: winners move, movers of breeding age leave a newborn */
        snap = store_snapshot(&fish, os ? os + 2 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            wt_fish* f = (wt_fish*)store_get(&fish, snap[j]);
            f->age += 1;
            if (f->target != WT_NONE && claim[f->target] == f->cell) {
                uint32_t tg = f->target, old = f->cell;
                claim[tg] = WT_NONE;
                occ[tg] = 1; agent[tg] = snap[j];
                f->cell = tg;
                ev.fish_moves++;
                if (f->age >= WT_FISH_BREED) {
                    f->age = 0;
                    uint32_t k = store_new(&fish);
                    if (k == UINT32_MAX) { rc = -1; break; }
                    f = NULL; /* the store may have moved */
                    wt_fish* nf = (wt_fish*)store_get(&fish, k);
                    nf->cell = old; nf->age = 0; nf->target = WT_NONE;
                    occ[old] = 1; agent[old] = k;
                    ev.fish_births++;
                } else {
                    occ[old] = 0; agent[old] = WT_NONE;
                }
            }
        }
        free(snap);
        if (rc) break;
        /* do-all Shark.choose: prefer a fish neighbour, else an empty one */
        snap = store_snapshot(&sharks, os ? os + 3 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            wt_shark* s = (wt_shark*)store_get(&sharks, snap[j]);
            wt_neighbours(s->cell, w, h, nb);
            uint32_t k = 0;
            for (int d = 0; d < 4; ++d) if (occ[nb[d]] == 1) cand[k++] = nb[d];
            s->eat = k ? 1u : 0u;
            if (!k)
                for (int d = 0; d < 4; ++d) if (occ[nb[d]] == 0) cand[k++] = nb[d];
            s->target = WT_NONE;
            if (k) {
                uint32_t u = philox_w0(seed, t, s->cell, 2, 0);
                uint32_t tg = cand[u % k];
                s->target = tg;
                if (s->cell < claim[tg]) claim[tg] = s->cell;
            }
        }
        free(snap);
        /* do-all Shark.move: eat or lose energy, breed, starve */
        snap = store_snapshot(&sharks, os ? os + 4 : 0, &n);
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t me = snap[j];
            wt_shark* s = (wt_shark*)store_get(&sharks, me);
            s->age += 1;
            if (s->target != WT_NONE && claim[s->target] == s->cell) {
                uint32_t tg = s->target, old = s->cell;
                claim[tg] = WT_NONE;
                if (s->eat) {
                    store_delete(&fish, agent[tg]);
                    ev.eaten++;
                    s->energy = WT_SHARK_ENERGY;
                } else {
                    s->energy -= 1;
                }
                occ[tg] = 2; agent[tg] = me;
                s->cell = tg;
                ev.shark_moves++;
                if (s->age >= WT_SHARK_BREED) {
                    s->age = 0;
                    uint32_t k = store_new(&sharks);
                    if (k == UINT32_MAX) { rc = -1; break; }
                    s = (wt_shark*)store_get(&sharks, me); /* the store may have moved */
                    wt_shark* ns = (wt_shark*)store_get(&sharks, k);
                    ns->cell = old; ns->age = 0; ns->energy = WT_SHARK_ENERGY;
                    ns->target = WT_NONE; ns->eat = 0;
                    occ[old] = 2; agent[old] = k;
                    ev.shark_births++;
                } else {
                    occ[old] = 0; agent[old] = WT_NONE;
                }
            } else {
                s->energy -= 1;
            }
            if (s->energy == 0) {
                occ[s->cell] = 0; agent[s->cell] = WT_NONE;
                store_delete(&sharks, me);
                ev.starved++;
            }
        }
        free(snap);
        ev.fish = fish.nlive;
        ev.sharks = sharks.nlive;
        if (stats) stats[step] = ev;
    }
    if (rc == 0 && out_occ) memcpy(out_occ, occ, ncell);
    if (fish.failed || sharks.failed) rc = -1;
    free(occ); free(agent); free(claim);
    store_free(&fish);
    store_free(&sharks);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Batched Nagel-Schreckenberg rings (Nagel & Schreckenberg 1992; Table 1    */
/* "traffic").  Per step t, on the occupancy at step start: accelerate by 1  */
/* up to vmax = 5, brake to the number of free cells ahead, slow down by 1   */
/* with a Philox draw, move.  A car that lands on the off-ramp cell L/2 may  */
/* leave; afterwards an empty on-ramp cell 0 may receive a new car (v = 0).  */
/* ------------------------------------------------------------------------ */
#define NS_VMAX 5u
typedef struct { uint32_t inst, pos, v; } ns_car;

int orc_traffic_run(uint32_t n_inst, uint32_t first_ring, const uint32_t* L, const uint32_t* thr,
                    uint64_t seed, uint32_t steps, uint32_t slow_thr,
                    uint32_t ramp_thr, const uint8_t* init_occ,
                    const uint8_t* init_v, uint64_t order_seed,
                    uint8_t* out_occ, uint8_t* out_v, uint32_t* cars_per_step) {
    if (n_inst == 0) return -1;
    uint64_t* off = (uint64_t*)malloc(((size_t)n_inst + 1) * sizeof(uint64_t));
    if (!off) return -1;
    off[0] = 0;
    for (uint32_t i = 0; i < n_inst; ++i) {
        if (L[i] < 2) { free(off); return -1; }
        off[i + 1] = off[i] + L[i];
    }
    uint64_t total = off[n_inst];
    uint8_t* cur = (uint8_t*)calloc(total, 1);
    uint8_t* nxt = (uint8_t*)calloc(total, 1);
    uint32_t* cars = (uint32_t*)calloc(n_inst, sizeof(uint32_t));
    if (!cur || !nxt || !cars) { free(off); free(cur); free(nxt); free(cars); return -1; }
    store_t st;
    store_init(&st, sizeof(ns_car));
    int rc = 0;
    for (uint32_t i = 0; i < n_inst && rc == 0; ++i) {
        for (uint32_t j = 0; j < L[i]; ++j) {
            int present = init_occ ? (init_occ[off[i] + j] != 0)
                                   : (philox_w0(seed, 0xFFFFFFFFu, j, first_ring + i, 0) < thr[i]);
            if (!present) continue;
            uint32_t k = store_new(&st);
            if (k == UINT32_MAX) { rc = -1; break; }
            ns_car* car = (ns_car*)store_get(&st, k);
            car->inst = i; car->pos = j;
            car->v = init_v ? init_v[off[i] + j] : 0u;
            cur[off[i] + j] = 1;
            cars[i]++;
        }
    }
    if (cars_per_step && rc == 0) memcpy(cars_per_step, cars, n_inst * sizeof(uint32_t));
    for (uint32_t t = 0; t < steps && rc == 0; ++t) {
        memset(nxt, 0, total);
        uint32_t n;
        uint32_t* snap = store_snapshot(&st, order_seed ? order_seed + t + 1 : 0, &n);
        /* do-all Car.move */
        for (uint32_t j = 0; j < n; ++j) {
            ns_car* car = (ns_car*)store_get(&st, snap[j]);
            uint32_t i = car->inst, len = L[i];
            uint32_t v = car->v + 1 < NS_VMAX ? car->v + 1 : NS_VMAX;
            uint32_t gap = 0;
            while (gap < v && !cur[off[i] + (car->pos + gap + 1) % len]) gap++;
            if (gap < v) v = gap;
            if (v > 0 && philox_w0(seed, t, car->pos, first_ring + i, 1) < slow_thr) v -= 1;
            uint32_t np = (car->pos + v) % len;
            uint32_t ramp_off = len / 2;
            if (np == ramp_off && philox_w0(seed, t, ramp_off, first_ring + i, 2) < ramp_thr) {
                store_delete(&st, snap[j]);
                cars[i]--;
                continue;
            }
            car->pos = np;
            car->v = v;
            nxt[off[i] + np] = 1;
        }
        free(snap);
        /* on-ramp: one possible arrival per ring at cell 0 */
        for (uint32_t i = 0; i < n_inst; ++i) {
            if (nxt[off[i]] == 0 && philox_w0(seed, t, 0, first_ring + i, 3) < ramp_thr) {
                uint32_t k = store_new(&st);
                if (k == UINT32_MAX) { rc = -1; break; }
                ns_car* car = (ns_car*)store_get(&st, k);
                car->inst = i; car->pos = 0; car->v = 0;
                nxt[off[i]] = 1;
                cars[i]++;
            }
        }
        uint8_t* tmp = cur; cur = nxt; nxt = tmp;
        if (cars_per_step) memcpy(cars_per_step + (size_t)(t + 1) * n_inst, cars, n_inst * sizeof(uint32_t));
    }
    if (rc == 0 && (out_occ || out_v)) {
        if (out_occ) memcpy(out_occ, cur, total);
        if (out_v) {
            memset(out_v, 0, total);
            for (uint32_t k = 0; k < st.hw; ++k) {
                if (!st.live[k]) continue;
                ns_car* car = (ns_car*)store_get(&st, k);
                out_v[off[car->inst] + car->pos] = (uint8_t)car->v;
            }
        }
    }
    if (st.failed) rc = -1;
    store_free(&st);
    free(off); free(cur); free(nxt); free(cars);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* N-body and particle collisions (Table 1 "nbody", "collision"; Sec. 2's   */
/* running example).  One type, Body {id, pos, vel, mass, force, target,    */
/* incoming, merged}.  Every body of the current set acts on every other    */
/* one through a device_do (Sec. 2.1, the sequential for-each over a type), */
/* so a force do-all is O(n^2).                                             */
/*                                                                          */
/* Arithmetic (our reading, chosen so that the result does not depend on    */
/* the order in which the for-each or the do-all visits bodies): every      */
/* float operation is one IEEE binary32 operation rounded to nearest, never */
/* contracted; the pairwise force is rounded to an integer of the fixed-    */
/* point scale S and summed in 64-bit two's complement arithmetic, which is */
/* associative, so the force on a body is exact whatever the visit order.   */
/* Because x_j - x_i == -(x_i - x_j) exactly and G S is a power of two, the */
/* pair (j, i) yields exactly the negated integers of (i, j): the forces of */
/* one FORCE do-all sum to zero exactly (Newton's third law).               */
/*                                                                          */
/* n-body step (2 do-alls): FORCE, MOVE.                                    */
/*   FORCE  F_i = sum over j != i of fix(((G S m_i) m_j) d^-3 (x_j - x_i)), */
/*          d2 = |x_j - x_i|^2 + eps2, d = sqrt(d2), d^-3 = (1/d)(1/d)(1/d) */
/*          (the paper's G m_i m_j / d^2 along the unit vector, softened,  */
/*          with the scale S folded into G; G and S are powers of two, so  */
/*          (G S m_i) is exact and m_i, m_j enter symmetrically)           */
/*   MOVE   v += (F S^-1 / m) dt;  x += v dt   (velocity first)             */
/* collision step (6 do-alls): FORCE, MOVE, then                            */
/*   FIND   target = nearest body j with |x_j - x_i|^2 < rc2 that is bigger */
/*          (heavier, or as heavy with a lower id); ties of distance go to  */
/*          the lower id.  Resets incoming and merged.                      */
/*   CLAIM  a body with a target proposes itself: incoming of the target    */
/*          = min(incoming, own id)  (lowest id wins, as in Wa-Tor)         */
/*   MERGE  a body with an incoming proposal that has no target itself      */
/*          absorbs the winner: perfectly inelastic, mass and momentum      */
/*          added, position at the centre of mass; the winner is marked     */
/*   DELETE a marked body deletes itself                                    */
/* A proposer whose target is itself merging waits for a later step, so     */
/* chains resolve one link per step and no body is absorbed twice.          */
/* ------------------------------------------------------------------------ */
#define NB_NONE 0xFFFFFFFFu
#define NB_FIX_MAX 0x1p62f

typedef struct {
    uint32_t id;
    float px, py, vx, vy, m;
    int64_t fx, fy;
    uint32_t target, incoming, merged;
} nb_body;

/* u in [0, 1) from the top 24 bits of a Philox word, exact in binary32 */
static float nb_unit(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

/* Initial state of body i: Philox(seed; 0xFFFFFFFF, i, k, 0) word 0 for
 * k = 0..4 gives pos x, pos y in [-1, 1), vel x, vel y in
 * [-vscale/2, vscale/2) and the integer mass 1 + w mod mass_max. */
static void nb_draw(uint64_t seed, uint32_t i, const orc_nbody_params* p, float st[5]) {
    st[0] = nb_unit(philox_w0(seed, 0xFFFFFFFFu, i, 0, 0)) * 2.0f - 1.0f;
    st[1] = nb_unit(philox_w0(seed, 0xFFFFFFFFu, i, 1, 0)) * 2.0f - 1.0f;
    st[2] = (nb_unit(philox_w0(seed, 0xFFFFFFFFu, i, 2, 0)) - 0.5f) * p->vscale;
    st[3] = (nb_unit(philox_w0(seed, 0xFFFFFFFFu, i, 3, 0)) - 0.5f) * p->vscale;
    st[4] = (float)(1u + philox_w0(seed, 0xFFFFFFFFu, i, 4, 0) % p->mass_max);
}

/* one pair term, already scaled by S, clamped to +-2^62 and rounded to the
 * nearest integer (ties to even) */
static int64_t nb_fix(float s) {
    if (s > NB_FIX_MAX) s = NB_FIX_MAX;
    if (s < -NB_FIX_MAX) s = -NB_FIX_MAX;
    return (int64_t)llrintf(s);
}

/* The pair term of body j (qx, qy, qm) on body i (px, py; gsm = G S m_i),
 * added to the two's complement force words. */
static void nb_pair(float px, float py, float gsm, float qx, float qy, float qm, float eps2,
                    uint64_t* fx, uint64_t* fy) {
    float dx = qx - px;
    float dy = qy - py;
    float dxx = dx * dx, dyy = dy * dy;
    float d2 = (dxx + dyy) + eps2;
    float d = sqrtf(d2);
    float inv = 1.0f / d;
    float inv2 = inv * inv;
    float inv3 = inv2 * inv;
    float k = (gsm * qm) * inv3;
    *fx += (uint64_t)nb_fix(k * dx);
    *fy += (uint64_t)nb_fix(k * dy);
}

int orc_nbody_force_on(uint32_t n, const float* state, const uint8_t* alive,
                       const orc_nbody_params* p, uint32_t i, int64_t out[2]) {
    if (!p || !state || i >= n || !(p->eps2 > 0.0f)) return -1;
    const float* si = state + (size_t)5 * i;
    const float gsm = (p->G * p->fscale) * si[4];
    uint64_t fx = 0, fy = 0;
    for (uint32_t j = 0; j < n; ++j) {
        if (j == i || (alive && !alive[j])) continue;
        const float* sj = state + (size_t)5 * j;
        nb_pair(si[0], si[1], gsm, sj[0], sj[1], sj[4], p->eps2, &fx, &fy);
    }
    out[0] = (int64_t)fx;
    out[1] = (int64_t)fy;
    return 0;
}

int orc_nbody_run(uint32_t n, const float* init, uint64_t seed, const orc_nbody_params* p,
                  uint32_t steps, uint64_t order_seed, float* out, uint8_t* out_alive,
                  uint32_t* count_per_step, int64_t* force_sum) {
    if (!p || !(p->eps2 > 0.0f) || !(p->fscale > 0.0f) || p->mass_max == 0) return -1;
    store_t st;
    store_init(&st, sizeof(nb_body));
    uint32_t* of_id = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!of_id) return -1;
    int rc = 0;
    /* parallel_new<Body>(n): constructor index i is the body id */
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t k = store_new(&st);
        if (k == UINT32_MAX) { rc = -1; break; }
        nb_body* b = (nb_body*)store_get(&st, k);
        float s[5];
        if (init) memcpy(s, init + (size_t)5 * i, sizeof(s)); else nb_draw(seed, i, p, s);
        b->id = i; b->px = s[0]; b->py = s[1]; b->vx = s[2]; b->vy = s[3]; b->m = s[4];
        b->target = NB_NONE; b->incoming = NB_NONE; b->merged = 0;
        of_id[i] = k;
    }
    if (count_per_step && rc == 0) count_per_step[0] = st.nlive;
    const float GS = p->G * p->fscale, Sinv = 1.0f / p->fscale;
    for (uint32_t step = 0; step < steps && rc == 0; ++step) {
        uint64_t os = order_seed ? order_seed + 8ull * step : 0;
        uint32_t n_snap, n_all;
        /* do-all FORCE, each body running device_do over every body */
        uint32_t* snap = store_snapshot(&st, os ? os + 1 : 0, &n_snap);
        uint32_t* all = store_snapshot(&st, os ? os + 7 : 0, &n_all);
        uint64_t sx = 0, sy = 0;
        for (uint32_t a = 0; a < n_snap; ++a) {
            nb_body* bi = (nb_body*)store_get(&st, snap[a]);
            uint64_t fx = 0, fy = 0;
            const float gsm = GS * bi->m;
            for (uint32_t c = 0; c < n_all; ++c) {
                if (all[c] == snap[a]) continue;
                const nb_body* bj = (const nb_body*)store_get(&st, all[c]);
                nb_pair(bi->px, bi->py, gsm, bj->px, bj->py, bj->m, p->eps2, &fx, &fy);
            }
            bi->fx = (int64_t)fx;
            bi->fy = (int64_t)fy;
            sx += fx; sy += fy;
        }
        free(all);
        if (force_sum) { force_sum[2 * step] = (int64_t)sx; force_sum[2 * step + 1] = (int64_t)sy; }
        /* do-all MOVE */
        for (uint32_t a = 0; a < n_snap; ++a) {
            nb_body* b = (nb_body*)store_get(&st, snap[a]);
            float ax = ((float)b->fx * Sinv) / b->m;
            float ay = ((float)b->fy * Sinv) / b->m;
            b->vx = b->vx + ax * p->dt;
            b->vy = b->vy + ay * p->dt;
            b->px = b->px + b->vx * p->dt;
            b->py = b->py + b->vy * p->dt;
        }
        if (p->collide) {
            /* do-all FIND (device_do over every body) */
            for (uint32_t a = 0; a < n_snap; ++a) {
                nb_body* bi = (nb_body*)store_get(&st, snap[a]);
                uint32_t best = NB_NONE;
                float bestd = 0.0f;
                for (uint32_t c = 0; c < n_snap; ++c) {
                    if (c == a) continue;
                    const nb_body* bj = (const nb_body*)store_get(&st, snap[c]);
                    float dx = bj->px - bi->px;
                    float dy = bj->py - bi->py;
                    float dxx = dx * dx, dyy = dy * dy;
                    float d2 = dxx + dyy;
                    int bigger = bj->m > bi->m || (bj->m == bi->m && bj->id < bi->id);
                    if (d2 < p->rc2 && bigger &&
                        (best == NB_NONE || d2 < bestd || (d2 == bestd && bj->id < best))) {
                        best = bj->id;
                        bestd = d2;
                    }
                }
                bi->target = best;
                bi->incoming = NB_NONE;
                bi->merged = 0;
            }
            /* do-all CLAIM */
            for (uint32_t a = 0; a < n_snap; ++a) {
                nb_body* b = (nb_body*)store_get(&st, snap[a]);
                if (b->target == NB_NONE) continue;
                nb_body* tb = (nb_body*)store_get(&st, of_id[b->target]);
                if (b->id < tb->incoming) tb->incoming = b->id;
            }
            /* do-all MERGE */
            for (uint32_t a = 0; a < n_snap; ++a) {
                nb_body* b = (nb_body*)store_get(&st, snap[a]);
                if (b->incoming == NB_NONE || b->target != NB_NONE) continue;
                nb_body* s = (nb_body*)store_get(&st, of_id[b->incoming]);
                float M = b->m + s->m;
                float mvx = b->m * b->vx, svx = s->m * s->vx;
                float mvy = b->m * b->vy, svy = s->m * s->vy;
                float mpx = b->m * b->px, spx = s->m * s->px;
                float mpy = b->m * b->py, spy = s->m * s->py;
                b->vx = (mvx + svx) / M;
                b->vy = (mvy + svy) / M;
                b->px = (mpx + spx) / M;
                b->py = (mpy + spy) / M;
                b->m = M;
                s->merged = 1;
            }
            /* do-all DELETE */
            for (uint32_t a = 0; a < n_snap; ++a) {
                nb_body* b = (nb_body*)store_get(&st, snap[a]);
                if (!b->merged) continue;
                of_id[b->id] = NB_NONE;
                store_delete(&st, snap[a]);
            }
        }
        free(snap);
        if (st.failed) rc = -1;
        if (count_per_step && rc == 0) count_per_step[step + 1] = st.nlive;
    }
    if (rc == 0) {
        if (out) memset(out, 0, (size_t)n * 5 * sizeof(float));
        if (out_alive) memset(out_alive, 0, n);
        for (uint32_t k = 0; k < st.hw; ++k) {
            if (!st.live[k]) continue;
            const nb_body* b = (const nb_body*)store_get(&st, k);
            if (out) {
                float* o = out + (size_t)5 * b->id;
                o[0] = b->px; o[1] = b->py; o[2] = b->vx; o[3] = b->vy; o[4] = b->m;
            }
            if (out_alive) out_alive[b->id] = 1;
        }
    }
    free(of_id);
    store_free(&st);
    return rc;
}
