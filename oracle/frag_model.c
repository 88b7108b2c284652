/*
 * frag_model.c -- fragmentation of idealised sequential allocators on a Wa-Tor
 * run (the analysis of Sec. 6.4 / Fig. 10d): how many 64-slot blocks would an
 * allocator that places every object by a fixed policy, one allocation after
 * another, keep in use for the same object lifetimes?
 *
 * TEST AND ANALYSIS INFRASTRUCTURE, NOT PRODUCT CODE.  Shares nothing with the
 * CUDA path.  The Wa-Tor rules are those of orc_wator_run (Table 1 "wa-tor";
 * readings: N, E, S, W candidates, word 0 of Philox4x32-10 at counter
 * (t, cell, 1|2, 0) modulo the candidate count, lowest source cell wins a
 * claim, every agent of a phase ages, fish breed at 3 and sharks at 10 on a
 * move, eating refills energy to 3, a shark at 0 dies), kept here per cell:
 * an object keeps its (block, slot) while it moves; a birth allocates a slot
 * by the policy, a death frees it, a block whose last object dies is released.
 * Allocations run in the order the oracle's snapshot visits agents (cell order
 * within a phase).  Its populations are pinned to orc_wator_run's by
 * tests/test_oracle_frag_model.py.
 *
 * Policies (per type, blocks of 64 slots, a fresh block is the lowest released
 * or never used one):
 *   0 first fit   the lowest-numbered block with a free slot
 *   1 best fit    a fullest block with a free slot (lowest-numbered among them)
 *   2 random fit  a block with a free slot chosen uniformly (xorshift64, fixed seed)
 *   3 hinted random fit   FM_HINTS hint slots (standing for the warps of a GPU
 *                 allocator); each allocation draws a slot uniformly and takes
 *                 the slot's block if that still has a free slot, else a block
 *                 with a free slot chosen uniformly, else a fresh block; the
 *                 slot then names the block taken
 *   4 hinted random fit with draining   as 3, but a block whose objects fall
 *                 (by a death) to FM_DRAIN or fewer is draining until it is
 *                 filled or emptied: the uniform choice leaves it out and a
 *                 hint that names it is not taken
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dsoa_oracle.h"

/* three-level bitmap over block numbers: set, clear, lowest set bit */
typedef struct { uint64_t *l0, *l1, *l2; uint32_t n2; } fm_bits;

static int fm_bits_init(fm_bits* m, uint32_t n) {
    uint32_t n0 = (n + 63) / 64, n1 = (n0 + 63) / 64;
    m->n2 = (n1 + 63) / 64;
    m->l0 = calloc(n0, 8); m->l1 = calloc(n1, 8); m->l2 = calloc(m->n2, 8);
    return m->l0 && m->l1 && m->l2 ? 0 : -1;
}
static void fm_bits_free(fm_bits* m) { free(m->l0); free(m->l1); free(m->l2); }
static void fm_set(fm_bits* m, uint32_t b) {
    m->l0[b >> 6] |= 1ull << (b & 63);
    m->l1[b >> 12] |= 1ull << ((b >> 6) & 63);
    m->l2[b >> 18] |= 1ull << ((b >> 12) & 63);
}
static void fm_clr(fm_bits* m, uint32_t b) {
    m->l0[b >> 6] &= ~(1ull << (b & 63));
    if (m->l0[b >> 6]) return;
    m->l1[b >> 12] &= ~(1ull << ((b >> 6) & 63));
    if (m->l1[b >> 12]) return;
    m->l2[b >> 18] &= ~(1ull << ((b >> 12) & 63));
}
static int64_t fm_first(const fm_bits* m) {
    for (uint32_t i = 0; i < m->n2; ++i)
        if (m->l2[i]) {
            uint32_t j = i * 64 + (uint32_t)__builtin_ctzll(m->l2[i]);
            uint32_t k = j * 64 + (uint32_t)__builtin_ctzll(m->l1[j]);
            return (int64_t)k * 64 + __builtin_ctzll(m->l0[k]);
        }
    return -1;
}
static int fm_empty(const fm_bits* m) {
    for (uint32_t i = 0; i < m->n2; ++i) if (m->l2[i]) return 0;
    return 1;
}

#define FM_HINTS 8192u
#define FM_DRAIN 8u

typedef struct {
    int policy;
    uint32_t cap, nblocks, used, live;
    uint32_t* cnt;          /* objects per block */
    uint64_t* freebits;     /* free slots per block (1 = free) */
    fm_bits released;       /* blocks that were used and are empty again */
    fm_bits* level;         /* policy 0: level[1] = partly used; policy 1: level[n] = n objects */
    uint64_t level_mask;    /* policy 1: counts with a non-empty set */
    uint32_t *pool, *pos, npool;   /* policies 2-4: partly used blocks (4: not draining), swap-remove */
    uint32_t* hint;         /* policies 3-4: block + 1 per hint slot, 0 = none */
    uint8_t* drain;         /* policy 4: 1 = draining */
    uint64_t rng;
} fm_pool;

static uint64_t fm_next(fm_pool* p) {
    p->rng ^= p->rng << 13; p->rng ^= p->rng >> 7; p->rng ^= p->rng << 17;
    return p->rng;
}

static int fm_pool_init(fm_pool* p, int policy, uint32_t cap) {
    memset(p, 0, sizeof(*p));
    p->policy = policy;
    p->cap = cap;
    p->rng = 0x9E3779B97F4A7C15ull;
    p->cnt = calloc(cap, 4);
    p->freebits = calloc(cap, 8);
    p->pool = calloc(cap, 4);
    p->pos = calloc(cap, 4);
    p->level = calloc(64, sizeof(fm_bits));
    p->hint = calloc(FM_HINTS, 4);
    p->drain = calloc(cap, 1);
    if (!p->cnt || !p->freebits || !p->pool || !p->pos || !p->level || !p->hint || !p->drain) return -1;
    if (fm_bits_init(&p->released, cap)) return -1;
    for (int q = 0; q < 64; ++q)
        if ((policy == 0 && q == 1) || (policy == 1 && q > 0))
            if (fm_bits_init(&p->level[q], cap)) return -1;
    return 0;
}
static void fm_pool_free(fm_pool* p) {
    free(p->cnt); free(p->freebits); free(p->pool); free(p->pos); free(p->hint); free(p->drain);
    fm_bits_free(&p->released);
    if (p->level) {
        for (int q = 0; q < 64; ++q)
            if (p->level[q].l0) fm_bits_free(&p->level[q]);
        free(p->level);
    }
}
/* the policy's set of partly used blocks (1..63 objects) */
static void fm_enter(fm_pool* p, uint32_t b, uint32_t n) {
    if (n == 0 || n >= 64) return;
    if (p->policy >= 2) {
        if (p->policy == 4 && p->drain[b]) return;
        p->pos[b] = p->npool; p->pool[p->npool++] = b;
        return;
    }
    uint32_t q = p->policy == 0 ? 1 : n;
    fm_set(&p->level[q], b);
    p->level_mask |= 1ull << q;
}
static void fm_leave(fm_pool* p, uint32_t b, uint32_t n) {
    if (n == 0 || n >= 64) return;
    if (p->policy >= 2) {
        if (p->policy == 4 && p->drain[b]) return;
        uint32_t i = p->pos[b], last = p->pool[--p->npool];
        p->pool[i] = last;
        p->pos[last] = i;
        return;
    }
    uint32_t q = p->policy == 0 ? 1 : n;
    fm_clr(&p->level[q], b);
    if (fm_empty(&p->level[q])) p->level_mask &= ~(1ull << q);
}
static void fm_count(fm_pool* p, uint32_t b, uint32_t n) {
    fm_leave(p, b, p->cnt[b]);
    if (p->policy == 4) {
        if (n < p->cnt[b] && n <= FM_DRAIN) p->drain[b] = 1;   /* fell to few objects */
        if (n == 64 || n == 0) p->drain[b] = 0;               /* filled or emptied */
    }
    p->cnt[b] = n;
    fm_enter(p, b, n);
}
static int64_t fm_alloc(fm_pool* p) {
    int64_t b = -1;
    uint32_t hs = FM_HINTS;
    if (p->policy >= 3) {
        hs = (uint32_t)(fm_next(p) % FM_HINTS);
        const int64_t hb = (int64_t)p->hint[hs] - 1;
        if (hb >= 0 && p->cnt[hb] > 0 && p->cnt[hb] < 64 && !(p->policy == 4 && p->drain[hb])) b = hb;
    }
    if (p->policy >= 2) {
        if (b < 0 && p->npool) b = p->pool[fm_next(p) % p->npool];
    } else if (p->level_mask) {
        uint32_t q = 63u - (uint32_t)__builtin_clzll(p->level_mask);   /* first fit: the one set */
        b = fm_first(&p->level[q]);
    }
    if (b < 0) {
        b = fm_first(&p->released);
        if (b >= 0) fm_clr(&p->released, (uint32_t)b);
        else if (p->nblocks < p->cap) b = p->nblocks++;
        else return -1;
        p->freebits[b] = ~0ull;
        p->drain[b] = 0;
        p->used++;
    }
    if (hs < FM_HINTS) p->hint[hs] = (uint32_t)b + 1u;
    uint32_t s = (uint32_t)__builtin_ctzll(p->freebits[b]);
    p->freebits[b] &= ~(1ull << s);
    fm_count(p, (uint32_t)b, p->cnt[b] + 1);
    p->live++;
    return b * 64 + s;
}
static void fm_release(fm_pool* p, int64_t h) {
    uint32_t b = (uint32_t)(h / 64), s = (uint32_t)(h % 64);
    p->freebits[b] |= 1ull << s;
    fm_count(p, b, p->cnt[b] - 1);
    p->live--;
    if (p->cnt[b] == 0) { p->used--; fm_set(&p->released, b); }
}

static uint32_t fm_w0(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2) {
    uint32_t ctr[4] = {c0, c1, c2, 0}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, out[4];
    orc_philox4x32(ctr, key, 10, out);
    return out[0];
}

int orc_wator_frag(uint32_t w, uint32_t h, uint64_t seed, uint32_t steps, int policy, uint32_t every,
                   double* F_out, uint32_t* fish_out, uint32_t* sharks_out, uint32_t* blocks_out) {
    if (w == 0 || h == 0 || policy < 0 || policy > 4 || every == 0) return -1;
    const uint32_t n = w * h, cap = n + 2;   /* a block in use holds an object: blocks <= objects <= n */
    uint8_t* kind = calloc(n, 1);
    uint8_t* eats = calloc(n, 1);
    uint32_t *age = calloc(n, 4), *en = calloc(n, 4), *movers = malloc((size_t)n * 4);
    int64_t *slot = calloc(n, 8), *target = malloc((size_t)n * 8), *best = malloc((size_t)n * 8);
    fm_pool P[2];
    int rc = (kind && eats && age && en && movers && slot && target && best) ? 0 : -1;
    if (!rc) rc = fm_pool_init(&P[0], policy, cap);
    if (!rc) rc = fm_pool_init(&P[1], policy, cap);
    for (uint32_t c = 0; c < n && !rc; ++c) {
        uint32_t u = fm_w0(seed, 0xFFFFFFFFu, c, 0);
        kind[c] = u < 1288490188u ? 1 : (u < 1503238553u ? 2 : 0);
        if (kind[c]) slot[c] = fm_alloc(&P[kind[c] - 1]);
        if (kind[c] == 2) en[c] = 3;
    }
    uint32_t rec = 0;
    for (uint32_t t = 0; t < steps && !rc; ++t) {
        for (int phase = 1; phase <= 2; ++phase) {
            uint32_t nm = 0;
            for (uint32_t c = 0; c < n; ++c) { best[c] = n; if (kind[c] == phase) movers[nm++] = c; }
            for (uint32_t i = 0; i < nm; ++i) {      /* choose */
                uint32_t c = movers[i], x = c % w, y = c / w, cand[4], k = 0;
                uint32_t nb[4] = {((y + h - 1) % h) * w + x, y * w + (x + 1) % w,
                                  ((y + 1) % h) * w + x, y * w + (x + w - 1) % w};
                if (phase == 2)
                    for (int d = 0; d < 4; ++d) if (kind[nb[d]] == 1) cand[k++] = nb[d];
                eats[c] = k > 0;
                if (!k)
                    for (int d = 0; d < 4; ++d) if (kind[nb[d]] == 0) cand[k++] = nb[d];
                target[c] = -1;
                if (k) {
                    uint32_t tg = cand[fm_w0(seed, t, c, (uint32_t)phase) % k];
                    target[c] = tg;
                    if (c < best[tg]) best[tg] = c;
                }
            }
            for (uint32_t i = 0; i < nm && !rc; ++i) {   /* move */
                uint32_t c = movers[i], a = age[c] + 1, e = en[c], here = c;
                int64_t tg = target[c];
                const uint32_t breed = phase == 1 ? 3u : 10u;
                if (tg >= 0 && best[tg] == c) {
                    if (phase == 2) {
                        if (eats[c]) { fm_release(&P[0], slot[tg]); e = 3; } else e -= 1;
                    }
                    kind[tg] = (uint8_t)phase;
                    slot[tg] = slot[c];
                    here = (uint32_t)tg;
                    if (a >= breed) {
                        a = 0;
                        age[c] = 0; en[c] = 3;
                        slot[c] = fm_alloc(&P[phase - 1]);
                        if (slot[c] < 0) rc = -1;
                    } else {
                        kind[c] = 0; age[c] = 0; en[c] = 0;
                    }
                } else if (phase == 2) {
                    e -= 1;
                }
                age[here] = a;
                if (phase == 2) {
                    en[here] = e;
                    if (e == 0) {
                        fm_release(&P[1], slot[here]);
                        kind[here] = 0; age[here] = 0; en[here] = 0;
                    }
                }
            }
        }
        if ((t + 1) % every == 0) {
            uint32_t blocks = P[0].used + P[1].used, live = P[0].live + P[1].live;
            if (F_out) F_out[rec] = blocks ? 1.0 - (double)live / (64.0 * blocks) : 0.0;
            if (fish_out) fish_out[rec] = P[0].live;
            if (sharks_out) sharks_out[rec] = P[1].live;
            if (blocks_out) blocks_out[rec] = blocks;
            ++rec;
        }
    }
    fm_pool_free(&P[0]);
    fm_pool_free(&P[1]);
    free(kind); free(eats); free(age); free(en); free(movers); free(slot); free(target); free(best);
    return rc;
}
