// nbody.cu -- n-body and particle collisions as SMMO applications (Table 1
// "nbody" and "collision"; the n-body listing of Sec. 2).  One type, Body.
// FORCE and FIND are all-pairs methods: in the paper's form every body runs a
// device_do (Sec. 2.1) over all bodies in its own thread; FORCE_TILED and
// FIND_TILED compute the same integers with a pairwise kernel over the
// enumerated snapshot whose CTAs stage chunks of bodies in shared memory.
//
// Arithmetic: every float operation is one IEEE binary32 operation rounded to
// nearest (the __f*_rn intrinsics, which the compiler never contracts into
// FMAs); each pair term is rounded to an integer of the fixed-point scale S and
// summed in wrapping 64-bit arithmetic.  Integer addition is associative, so
// the force on a body is the same whatever order (and whatever partition) the
// pairs are visited in, and the pair (j, i) yields exactly the negated
// integers of (i, j).
#include "dsoa_internal.cuh"
#include "rng.cuh"
#include "rn_math.cuh"

namespace {

enum : uint32_t { kId = 0, kPx, kPy, kVx, kVy, kM, kFx, kFy, kTarget, kIncoming, kMerged };
constexpr uint32_t kNone = DSOA_NBODY_NONE;

template <typename F>
__device__ __forceinline__ F& fld(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, uint32_t f) {
    return dsoa_column<F>(c, t, bid, f)[s];
}

// u in [0, 1) from the top 24 bits of a Philox word (exact in binary32)
__device__ __forceinline__ float unit24(uint32_t w) { return __fmul_rn((float)(w >> 8), 0x1p-24f); }

// A pair term already scaled by S: clamped to +-2^62, rounded to the nearest
// integer (ties to even), returned as a two's complement word.  A 64-bit
// float-to-integer conversion is slow here, so the word comes from 32-bit work:
// below 2^31 in magnitude (nearly every term) a 32-bit round-to-nearest-even
// conversion is exact; from 2^31 on a binary32 value is an integer,
// mantissa * 2^(exponent - 23), which shifts give exactly (a rare branch).
__device__ __noinline__ unsigned long long fix_large(float s) {
    s = fminf(fmaxf(s, -0x1p62f), 0x1p62f);
    const uint32_t u = __float_as_uint(s);
    const unsigned long long mag = (unsigned long long)((u & 0x7FFFFFu) | 0x800000u) << (((u >> 23) & 0xFFu) - 150u);
    return (u >> 31) ? 0ull - mag : mag;
}
__device__ __forceinline__ unsigned long long fix(float s) {
    if (fabsf(s) < 0x1p31f) return (unsigned long long)(long long)__float2int_rn(s);
    return fix_large(s);
}

// Adds the pair term of body (px, py) with gsm = G S m_i under body (qx, qy, qm).
__device__ __forceinline__ void pair_term(float px, float py, float gsm, float qx, float qy, float qm,
                                          float eps2, unsigned long long& fx, unsigned long long& fy) {
    const float dx = __fsub_rn(qx, px), dy = __fsub_rn(qy, py);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), eps2);
    const float inv = __frcp_rn(__fsqrt_rn(d2));
    const float k = __fmul_rn(__fmul_rn(gsm, qm), __fmul_rn(__fmul_rn(inv, inv), inv));
    fx += fix(__fmul_rn(k, dx));
    fy += fix(__fmul_rn(k, dy));
}

struct Ctor {
    using Args = dsoa_nbody_args;
    static __device__ void ctor(const dsoa_ctx& c, dsoa_obj o, uint64_t i, const Args& a) {
        const uint32_t id = (uint32_t)i;
        float s[5];
        if (a.init) {
#pragma unroll
            for (int k = 0; k < 5; ++k) s[k] = a.init[(uint64_t)5 * i + k];
        } else {
            s[0] = __fsub_rn(__fmul_rn(unit24(dsoa_philox_w0(a.seed, 0xFFFFFFFFu, id, 0u, 0u)), 2.0f), 1.0f);
            s[1] = __fsub_rn(__fmul_rn(unit24(dsoa_philox_w0(a.seed, 0xFFFFFFFFu, id, 1u, 0u)), 2.0f), 1.0f);
            s[2] = __fmul_rn(__fsub_rn(unit24(dsoa_philox_w0(a.seed, 0xFFFFFFFFu, id, 2u, 0u)), 0.5f), a.vscale);
            s[3] = __fmul_rn(__fsub_rn(unit24(dsoa_philox_w0(a.seed, 0xFFFFFFFFu, id, 3u, 0u)), 0.5f), a.vscale);
            s[4] = (float)(1u + dsoa_philox_w0(a.seed, 0xFFFFFFFFu, id, 4u, 0u) % a.mass_max);
        }
        dsoa_field<uint32_t>(c, o, kId) = id;
        dsoa_field<float>(c, o, kPx) = s[0];
        dsoa_field<float>(c, o, kPy) = s[1];
        dsoa_field<float>(c, o, kVx) = s[2];
        dsoa_field<float>(c, o, kVy) = s[3];
        dsoa_field<float>(c, o, kM) = s[4];
        dsoa_field<unsigned long long>(c, o, kFx) = 0ull;
        dsoa_field<unsigned long long>(c, o, kFy) = 0ull;
        dsoa_field<uint32_t>(c, o, kTarget) = kNone;
        dsoa_field<uint32_t>(c, o, kIncoming) = kNone;
        dsoa_field<uint32_t>(c, o, kMerged) = 0u;
        if (a.handle_of) a.handle_of[i] = o;
    }
};

// FORCE: the body adds the pair terms of every other body to its force, walking
// all bodies with device_do (the paper's structure: one sequential for-each per
// thread, neighbouring threads reading the same body at the same time).
struct Force {
    using Args = dsoa_nbody_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const dsoa_obj self = dsoa_make_handle(t, bid, s);
        const float px = fld<float>(c, t, bid, s, kPx), py = fld<float>(c, t, bid, s, kPy);
        const float gsm = __fmul_rn(__fmul_rn(a.G, a.fscale), fld<float>(c, t, bid, s, kM));
        unsigned long long fx = 0ull, fy = 0ull;
        dsoa_device_do(c, t, [&](dsoa_obj o) {
            if (o == self) return;
            const uint64_t ob = dsoa_h_block(o);
            const uint32_t os = dsoa_h_slot(o);
            pair_term(px, py, gsm, fld<float>(c, t, ob, os, kPx), fld<float>(c, t, ob, os, kPy),
                      fld<float>(c, t, ob, os, kM), a.eps2, fx, fy);
        });
        fld<unsigned long long>(c, t, bid, s, kFx) += fx;
        fld<unsigned long long>(c, t, bid, s, kFy) += fy;
    }
};

// MOVE: velocity first, then position (the listing's order); clears the force.
struct Move {
    using Args = dsoa_nbody_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        unsigned long long& fx = fld<unsigned long long>(c, t, bid, s, kFx);
        unsigned long long& fy = fld<unsigned long long>(c, t, bid, s, kFy);
        const float m = fld<float>(c, t, bid, s, kM);
        const float sinv = __frcp_rn(a.fscale);
        const float ax = __fdiv_rn(__fmul_rn(__ll2float_rn((long long)fx), sinv), m);
        const float ay = __fdiv_rn(__fmul_rn(__ll2float_rn((long long)fy), sinv), m);
        float& vx = fld<float>(c, t, bid, s, kVx);
        float& vy = fld<float>(c, t, bid, s, kVy);
        vx = __fadd_rn(vx, __fmul_rn(ax, a.dt));
        vy = __fadd_rn(vy, __fmul_rn(ay, a.dt));
        float& px = fld<float>(c, t, bid, s, kPx);
        float& py = fld<float>(c, t, bid, s, kPy);
        px = __fadd_rn(px, __fmul_rn(vx, a.dt));
        py = __fadd_rn(py, __fmul_rn(vy, a.dt));
        fy = 0ull;
        if (a.flags & DSOA_NBODY_KEYED_FIND) {     // prepare FIND_TILED and CLAIM
            fx = ~0ull;
            fld<uint32_t>(c, t, bid, s, kTarget) = kNone;
            fld<uint32_t>(c, t, bid, s, kIncoming) = kNone;
            fld<uint32_t>(c, t, bid, s, kMerged) = 0u;
        } else {
            fx = 0ull;
        }
    }
};

// FIND: the nearest bigger body within reach (device_do over all bodies).
struct Find {
    using Args = dsoa_nbody_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const dsoa_obj self = dsoa_make_handle(t, bid, s);
        const float px = fld<float>(c, t, bid, s, kPx), py = fld<float>(c, t, bid, s, kPy);
        const float m = fld<float>(c, t, bid, s, kM);
        const uint32_t id = fld<uint32_t>(c, t, bid, s, kId);
        uint32_t best = kNone;
        float bestd = 0.0f;
        dsoa_device_do(c, t, [&](dsoa_obj o) {
            if (o == self) return;
            const uint64_t ob = dsoa_h_block(o);
            const uint32_t os = dsoa_h_slot(o);
            const float dx = __fsub_rn(fld<float>(c, t, ob, os, kPx), px);
            const float dy = __fsub_rn(fld<float>(c, t, ob, os, kPy), py);
            const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            if (!(d2 < a.rc2)) return;
            const float qm = fld<float>(c, t, ob, os, kM);
            const uint32_t qid = fld<uint32_t>(c, t, ob, os, kId);
            const bool bigger = qm > m || (qm == m && qid < id);
            if (bigger && (best == kNone || d2 < bestd || (d2 == bestd && qid < best))) {
                best = qid;
                bestd = d2;
            }
        });
        fld<uint32_t>(c, t, bid, s, kTarget) = best;
        fld<uint32_t>(c, t, bid, s, kIncoming) = kNone;
        fld<uint32_t>(c, t, bid, s, kMerged) = 0u;
    }
};

// CLAIM: propose to the target; the lowest id wins.
struct Claim {
    using Args = dsoa_nbody_args;
    static constexpr bool kNoNewOfOwnType = true;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        uint32_t target = fld<uint32_t>(c, t, bid, s, kTarget);
        if (a.flags & DSOA_NBODY_KEYED_FIND) {     // the key FIND_TILED left in fx
            unsigned long long& key = fld<unsigned long long>(c, t, bid, s, kFx);
            target = key == ~0ull ? kNone : (uint32_t)key;
            fld<uint32_t>(c, t, bid, s, kTarget) = target;
            key = 0ull;
        }
        if (target == kNone || target >= a.n_ids) return;
        const dsoa_obj h = a.handle_of[target];
        if (!h) return;
        atomicMin(&dsoa_field<uint32_t>(c, h, kIncoming), fld<uint32_t>(c, t, bid, s, kId));
    }
};

// MERGE: a body with a proposal and no target of its own absorbs the winner
// (perfectly inelastic: mass and momentum add, position at the centre of mass)
// and marks it.  A winner has a target, so no body both absorbs and is absorbed.
struct Merge {
    using Args = dsoa_nbody_args;
    static constexpr bool kNoNewOfOwnType = true;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t inc = fld<uint32_t>(c, t, bid, s, kIncoming);
        if (inc == kNone || inc >= a.n_ids || fld<uint32_t>(c, t, bid, s, kTarget) != kNone) return;
        const dsoa_obj h = a.handle_of[inc];
        if (!h) return;
        const uint64_t sb = dsoa_h_block(h);
        const uint32_t ss = dsoa_h_slot(h);
        const float sm = fld<float>(c, t, sb, ss, kM);
        float& m = fld<float>(c, t, bid, s, kM);
        float& vx = fld<float>(c, t, bid, s, kVx);
        float& vy = fld<float>(c, t, bid, s, kVy);
        float& px = fld<float>(c, t, bid, s, kPx);
        float& py = fld<float>(c, t, bid, s, kPy);
        const float M = __fadd_rn(m, sm);
        vx = __fdiv_rn(__fadd_rn(__fmul_rn(m, vx), __fmul_rn(sm, fld<float>(c, t, sb, ss, kVx))), M);
        vy = __fdiv_rn(__fadd_rn(__fmul_rn(m, vy), __fmul_rn(sm, fld<float>(c, t, sb, ss, kVy))), M);
        px = __fdiv_rn(__fadd_rn(__fmul_rn(m, px), __fmul_rn(sm, fld<float>(c, t, sb, ss, kPx))), M);
        py = __fdiv_rn(__fadd_rn(__fmul_rn(m, py), __fmul_rn(sm, fld<float>(c, t, sb, ss, kPy))), M);
        m = M;
        fld<uint32_t>(c, t, sb, ss, kMerged) = 1u;
    }
};

// DELETE: a marked body deletes itself.
struct Delete {
    using Args = dsoa_nbody_args;
    static constexpr bool kNoNewOfOwnType = true;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        if (!fld<uint32_t>(c, t, bid, s, kMerged)) return;
        const uint32_t id = fld<uint32_t>(c, t, bid, s, kId);
        if (a.handle_of && id < a.n_ids) a.handle_of[id] = 0ull;
        dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

struct Read {
    using Args = dsoa_nbody_args;
    static constexpr bool kNoNewOfOwnType = true;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = fld<uint32_t>(c, t, bid, s, kId);
        if (id >= a.n_ids) return;
        float* o = a.out + (uint64_t)5 * id;
        o[0] = fld<float>(c, t, bid, s, kPx);
        o[1] = fld<float>(c, t, bid, s, kPy);
        o[2] = fld<float>(c, t, bid, s, kVx);
        o[3] = fld<float>(c, t, bid, s, kVy);
        o[4] = fld<float>(c, t, bid, s, kM);
        a.alive_out[id] = 1;
        if (a.force_out) {
            a.force_out[2 * (uint64_t)id] = (int64_t)fld<unsigned long long>(c, t, bid, s, kFx);
            a.force_out[2 * (uint64_t)id + 1] = (int64_t)fld<unsigned long long>(c, t, bid, s, kFy);
        }
    }
};

// ---------------------------------------------------------------------------
// Pairwise do-alls over the enumerated snapshot (FORCE and FIND of every body
// against every other body).  Bodies get a dense index: every CTA first builds,
// in shared memory, the exclusive prefix of the occupied-slot counts of the
// listed blocks (pre[q] bodies precede block R[q]), so dense index d is the
// (d - pre[q])-th occupied slot of the block q found by binary search.  A work
// item is (256 bodies, one per thread) x (a chunk of 1024 bodies): the CTA
// stages the chunk's (px, py, m, id) as float4 in shared memory and every thread
// folds the chunk into its register state; all threads of a warp read the same
// body, so the shared loads are broadcasts, and no thread computes an empty
// slot however sparse the blocks are.  Each CTA takes a contiguous range of
// items (mostly one i tile) and folds its partial state into the body's fields
// with one atomic per body and i tile.  The fold is an integer sum (FORCE) or
// an integer minimum (FIND), so the partition does not change the result.
// Lists longer than kDenseMaxR blocks fall back to indexing slots (64 per
// listed block; empty ones stage as mass 0, which adds exactly 0 and is never
// bigger than a body).
// ---------------------------------------------------------------------------
constexpr uint32_t kTile = 256;          // i bodies per item: one per thread
constexpr uint32_t kChunkBodies = 1024;  // j bodies per item: 16 KB of float4
constexpr uint32_t kDenseMaxR = 4096;    // listed blocks indexed densely (16 KB prefix)

// (block list position, slot) of index d; false when d names an empty slot
__device__ __forceinline__ bool locate(bool dense, const uint32_t* pre, uint32_t r,
                                       const unsigned long long* __restrict__ occ, uint32_t d,
                                       uint32_t& q, uint32_t& slot) {
    if (!dense) {
        q = d >> 6;
        slot = d & 63u;
        return (__ldg(&occ[q]) >> slot) & 1ull;
    }
    uint32_t lo = 0, hi = r;             // pre[lo] <= d < pre[hi]
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= d) lo = mid; else hi = mid;
    }
    q = lo;
    slot = dsoa_nth_set(__ldg(&occ[lo]), d - pre[lo]);
    return true;
}

// FORCE: integer sums of the pair terms, added to the force fields.
struct ForceOp {
    float px, py, gsm;
    uint32_t id;
    unsigned long long fx, fy;
    __device__ void begin(const dsoa_ctx& c, uint32_t t, uint64_t b, uint32_t s, const dsoa_nbody_args& a) {
        px = fld<float>(c, t, b, s, kPx);
        py = fld<float>(c, t, b, s, kPy);
        gsm = __fmul_rn(__fmul_rn(a.G, a.fscale), fld<float>(c, t, b, s, kM));
        id = fld<uint32_t>(c, t, b, s, kId);
        fx = fy = 0ull;
    }
    __device__ __forceinline__ void pair(const float4 q, const dsoa_nbody_args& a) {
        if (__float_as_uint(q.w) != id) pair_term(px, py, gsm, q.x, q.y, q.z, a.eps2, fx, fy);
    }
    __device__ void end(const dsoa_ctx& c, uint32_t t, uint64_t b, uint32_t s) {
        if (fx) atomicAdd(&fld<unsigned long long>(c, t, b, s, kFx), fx);
        if (fy) atomicAdd(&fld<unsigned long long>(c, t, b, s, kFy), fy);
    }
};

// FIND (keyed): the nearest bigger body within reach as the minimum of the key
// (bits of d2 << 32 | id) -- the bits of a non-negative float order like its
// value, so the minimum key is the smallest distance, ties to the lower id.
// The key lives in the fx field, which MOVE set to all ones for this purpose;
// CLAIM turns it into the target and clears the field.
struct FindOp {
    float px, py, m;
    uint32_t id;
    unsigned long long key;
    __device__ void begin(const dsoa_ctx& c, uint32_t t, uint64_t b, uint32_t s, const dsoa_nbody_args&) {
        px = fld<float>(c, t, b, s, kPx);
        py = fld<float>(c, t, b, s, kPy);
        m = fld<float>(c, t, b, s, kM);
        id = fld<uint32_t>(c, t, b, s, kId);
        key = ~0ull;
    }
    __device__ __forceinline__ void pair(const float4 q, const dsoa_nbody_args& a) {
        const uint32_t qid = __float_as_uint(q.w);
        const float dx = __fsub_rn(q.x, px), dy = __fsub_rn(q.y, py);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        const bool bigger = q.z > m || (q.z == m && qid < id);
        const unsigned long long k = ((unsigned long long)__float_as_uint(d2) << 32) | qid;
        if (qid != id && d2 < a.rc2 && bigger && k < key) key = k;
    }
    __device__ void end(const dsoa_ctx& c, uint32_t t, uint64_t b, uint32_t s) {
        if (key != ~0ull) atomicMin(&fld<unsigned long long>(c, t, b, s, kFx), key);
    }
};

// Dense mode (r <= kDenseMaxR): writes pre[] (the exclusive prefix of the
// occupied-slot counts of the listed blocks, and the total at pre[r]) and
// returns the number of bodies; otherwise returns the number of listed slots.
// Called by every thread of the CTA.
__device__ uint32_t index_space(bool dense, uint32_t r, const unsigned long long* __restrict__ occ,
                                uint32_t* pre, uint32_t* wsum) {
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (!dense) return r * 64u;
    const uint32_t per = (r + 255u) / 256u;
    const uint32_t q0 = min(r, tid * per), q1 = min(r, q0 + per);
    uint32_t own = 0;
    for (uint32_t q = q0; q < q1; ++q) own += (uint32_t)__popcll(__ldg(&occ[q]));
    uint32_t x = own;                                       // inclusive scan over the warp
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31u) wsum[warp] = x;
    __syncthreads();
    uint32_t run = x - own, total = 0;
    for (uint32_t w = 0; w < 8u; ++w) {
        if (w < warp) run += wsum[w];
        total += wsum[w];
    }
    for (uint32_t q = q0; q < q1; ++q) {
        pre[q] = run;
        run += (uint32_t)__popcll(__ldg(&occ[q]));
    }
    if (tid == 0) pre[r] = total;
    __syncthreads();
    return total;
}

template <class Op>
__global__ void __launch_bounds__(256) k_pairs_tiled(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                     const unsigned long long* __restrict__ occ,
                                                     const uint32_t* __restrict__ r_dev, dsoa_nbody_args a) {
    __shared__ float4 sj[kChunkBodies];
    __shared__ uint32_t pre[kDenseMaxR + 1];
    __shared__ uint32_t wsum[8];
    const uint32_t r = __ldg(r_dev);
    const uint32_t tid = threadIdx.x;
    const bool dense = r <= kDenseMaxR;
    const uint32_t nb = index_space(dense, r, occ, pre, wsum);   // indices: bodies (dense) or slots
    const uint64_t n_i = (nb + kTile - 1) / kTile, n_j = (nb + kChunkBodies - 1) / kChunkBodies;
    const uint64_t items = n_i * n_j;
    const uint64_t wb = items * blockIdx.x / gridDim.x, we = items * (blockIdx.x + 1) / gridDim.x;
    uint64_t cur = ~0ull, bi = 0;
    bool mine = false;
    uint32_t si = 0;
    Op op;
    for (uint64_t w = wb; w < we; ++w) {
        const uint64_t it = w / n_j, jt = w % n_j;
        if (it != cur) {
            if (mine) op.end(c, t, bi, si);
            cur = it;
            const uint32_t d = (uint32_t)(it * kTile) + tid;
            uint32_t q = 0;
            mine = d < nb && locate(dense, pre, r, occ, d, q, si);
            if (mine) {
                bi = __ldg(&R[q]);
                op.begin(c, t, bi, si, a);
            }
        }
        const uint32_t j0 = (uint32_t)(jt * kChunkBodies);
        const uint32_t jn = min(kChunkBodies, nb - j0);     // same for the whole CTA
        __syncthreads();                                    // readers of the previous chunk are done
        for (uint32_t k = tid; k < jn; k += blockDim.x) {
            float4 v = make_float4(0.f, 0.f, 0.f, __uint_as_float(kNone));
            uint32_t q = 0, sl = 0;
            if (locate(dense, pre, r, occ, j0 + k, q, sl)) {
                const uint64_t bj = __ldg(&R[q]);
                v.x = fld<float>(c, t, bj, sl, kPx);
                v.y = fld<float>(c, t, bj, sl, kPy);
                v.z = fld<float>(c, t, bj, sl, kM);
                v.w = __uint_as_float(fld<uint32_t>(c, t, bj, sl, kId));
            }
            sj[k] = v;
        }
        __syncthreads();
        if (mine) {
#pragma unroll 4
            for (uint32_t k = 0; k < jn; ++k) op.pair(sj[k], a);
        }
    }
    if (mine) op.end(c, t, bi, si);
}

// ---------------------------------------------------------------------------
// FORCE over unordered pairs (Newton's third law in the fixed-point sums).  The
// terms of j on i and of i on j share dx, dy, d2 and the inverse cube: with
// k_ij = ((G S m_i) m_j) / d^3 and k_ji = ((G S m_j) m_i) / d^3, i gets
// fix(k_ij dx) and j gets fix(k_ji (-dx)) = -fix(k_ji dx), because rounding to
// nearest commutes with negation (x_i - x_j is exactly -(x_j - x_i)).  So one
// evaluation per unordered pair gives the very integers of the all-pairs sum.
//
// Work: square tiles of kTile indices on both sides; the items are the tile
// pairs (I, J) with J >= I, row-major, split evenly over the CTAs.  Warp w holds
// i group 8 I + w (one body per lane) and pairs it with the 8 groups of 32 j
// bodies of tile J in shared memory.  Within a group the pairs go round a
// rotation: at step s lane l pairs its i with j = (l + s) mod 32, adds the i
// term to its register sum and subtracts the j term from a running j sum that
// moves one lane down after the step, so after the 32 steps lane l holds a
// whole warp's sum for j = l.  Warps take the groups in rotated order, their j
// sums meet in shared memory (64-bit shared atomics) and leave with one global
// atomic per body and item; the i sums leave when the CTA moves to the next
// row.  In a diagonal tile (I = J) warp w pairs its group only with the groups
// after it and, within its own group, takes the 31 other bodies for its i side
// alone.  Every j group is staged twice in a row, so step s reads entry
// lane + s without wrapping.  Indices past the last body (and, beyond
// kDenseMaxR listed blocks, empty slots) stage as mass 0, whose terms are
// exactly 0 either way (the inverse cube is finite for eps2 >= 2^-80).
// ---------------------------------------------------------------------------
constexpr uint32_t kSymGroups = kTile / 32u;

__device__ __forceinline__ float4 stage_body(const dsoa_ctx& c, uint32_t t, bool dense, const uint32_t* pre,
                                             uint32_t r, const unsigned long long* __restrict__ occ,
                                             const uint32_t* __restrict__ R, uint32_t nb, uint64_t d, float gs,
                                             bool& ok, uint64_t& b, uint32_t& slot) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t q = 0;
    slot = 0;
    ok = d < nb && locate(dense, pre, r, occ, (uint32_t)d, q, slot);
    if (ok) {
        b = __ldg(&R[q]);
        v.x = fld<float>(c, t, b, slot, kPx);
        v.y = fld<float>(c, t, b, slot, kPy);
        v.z = fld<float>(c, t, b, slot, kM);
        v.w = __fmul_rn(gs, v.z);
    }
    return v;
}

// items in the rows before row I of the triangle (I + 1 .. nt items per row)
__device__ __forceinline__ uint64_t tri_start(uint64_t I, uint64_t nt) { return I * nt - I * (I - 1) / 2; }

// One 32-step rotation of warp group `g` (see above).  Terms below 2^25 in
// magnitude (nearly all) are summed in 32 bits over the 32 steps (at most 2^30,
// no overflow) and folded into the 64-bit sums once; a step with a larger term
// adds its terms in 64 bits directly (the j terms by shared atomics).  kSame:
// the two coefficients of every pair are known to be equal, (G S m_i) m_j =
// (G S m_j) m_i exactly, so the j term is the negated i term, and every
// coordinate is below 2^62 in magnitude, so d2 is finite and in [eps2, FLT_MAX]
// where dsoa_rcp_sqrt_rn gives the very bits of the two rounded intrinsics.
template <bool kSame>
__device__ __forceinline__ void sym_group(const float4* col, float px, float py, float m, float gsm, float eps2,
                                          uint32_t g, uint32_t lane, uint32_t src, unsigned long long& fx,
                                          unsigned long long& fy, unsigned long long* sx, unsigned long long* sy) {
    int fx32 = 0, fy32 = 0, gx32 = 0, gy32 = 0;
#pragma unroll 8
    for (uint32_t s = 0; s < 32u; ++s) {
        const float4 q = col[s];
        const float dx = __fsub_rn(q.x, px), dy = __fsub_rn(q.y, py);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), eps2);
        const float inv = kSame ? dsoa_rcp_sqrt_rn(d2) : __frcp_rn(__fsqrt_rn(d2));
        const float inv3 = __fmul_rn(__fmul_rn(inv, inv), inv);
        const float kij = __fmul_rn(__fmul_rn(gsm, q.z), inv3);
        const float ax = __fmul_rn(kij, dx), ay = __fmul_rn(kij, dy);
        if (kSame) {
            if ((fabsf(ax) < 0x1p25f) & (fabsf(ay) < 0x1p25f)) {
                const int vx = __float2int_rn(ax), vy = __float2int_rn(ay);
                fx32 += vx;
                fy32 += vy;
                gx32 -= vx;
                gy32 -= vy;
            } else {
                const uint32_t j = 32u * g + ((lane + s) & 31u);
                const unsigned long long ux = fix(ax), uy = fix(ay);
                fx += ux;
                fy += uy;
                if (ux) atomicAdd(&sx[j], 0ull - ux);
                if (uy) atomicAdd(&sy[j], 0ull - uy);
            }
        } else {
            const float kji = __fmul_rn(__fmul_rn(q.w, m), inv3);
            const float bx = __fmul_rn(kji, dx), by = __fmul_rn(kji, dy);
            if ((fabsf(ax) < 0x1p25f) & (fabsf(ay) < 0x1p25f) & (fabsf(bx) < 0x1p25f) & (fabsf(by) < 0x1p25f)) {
                fx32 += __float2int_rn(ax);
                fy32 += __float2int_rn(ay);
                gx32 -= __float2int_rn(bx);
                gy32 -= __float2int_rn(by);
            } else {
                const uint32_t j = 32u * g + ((lane + s) & 31u);
                fx += fix(ax);
                fy += fix(ay);
                const unsigned long long ux = 0ull - fix(bx), uy = 0ull - fix(by);
                if (ux) atomicAdd(&sx[j], ux);
                if (uy) atomicAdd(&sy[j], uy);
            }
        }
        gx32 = __shfl_sync(0xFFFFFFFFu, gx32, src);
        gy32 = __shfl_sync(0xFFFFFFFFu, gy32, src);
    }
    fx += (unsigned long long)(long long)fx32;               // after 32 moves lane l holds j = l
    fy += (unsigned long long)(long long)fy32;
    if (gx32) atomicAdd(&sx[32u * g + lane], (unsigned long long)(long long)gx32);
    if (gy32) atomicAdd(&sy[32u * g + lane], (unsigned long long)(long long)gy32);
}

// an integer mass in [0, 2^12]: products of two are exact in binary32
__device__ __forceinline__ bool small_integer(float m) { return m >= 0.0f && m <= 0x1p12f && m == truncf(m); }
// coordinates below 2^62 in magnitude: squared differences stay finite
__device__ __forceinline__ bool bounded(float4 v) { return fabsf(v.x) < 0x1p62f && fabsf(v.y) < 0x1p62f; }

__global__ void __launch_bounds__(256, 5) k_force_sym(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                   const unsigned long long* __restrict__ occ,
                                                   const uint32_t* __restrict__ r_dev, dsoa_nbody_args a) {
    __shared__ float4 sj[2 * kTile];                 // group g at [64 g, 64 g + 64): its 32 bodies twice
    __shared__ unsigned long long sacc[2][kTile];    // j sums of the item
    __shared__ uint32_t pre[kDenseMaxR + 1];
    __shared__ uint32_t wsum[8];
    const uint32_t r = __ldg(r_dev);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const bool dense = r <= kDenseMaxR;
    const uint32_t nb = index_space(dense, r, occ, pre, wsum);
    const float gs = __fmul_rn(a.G, a.fscale), eps2 = a.eps2;
    const bool gs_pow2 = (__float_as_uint(gs) & 0x807FFFFFu) == 0u && gs >= 0x1p-100f && gs <= 0x1p100f;
    const uint64_t nt = (nb + kTile - 1) / kTile, items = nt * (nt + 1) / 2;
    const uint64_t wb = items * blockIdx.x / gridDim.x, we = items * (blockIdx.x + 1) / gridDim.x;
    sacc[0][tid] = 0ull;
    sacc[1][tid] = 0ull;
    uint64_t I = 0, J = 0;
    if (wb < we) {                                   // the row holding item wb
        uint64_t lo = 0, hi = nt;                    // tri_start(lo) <= wb < tri_start(hi)
        while (hi - lo > 1u) {
            const uint64_t mid = (lo + hi) >> 1;
            if (tri_start(mid, nt) <= wb) lo = mid; else hi = mid;
        }
        I = lo;
        J = I + (wb - tri_start(I, nt));
    }
    uint64_t cur = ~0ull, bi = 0;
    uint32_t si = 0;
    bool imine = false;
    float px = 0.f, py = 0.f, m = 0.f, gsm = 0.f;
    unsigned long long fx = 0ull, fy = 0ull;
    const uint32_t src = (lane + 1u) & 31u;
    for (uint64_t w = wb; w < we; ++w) {
        if (I != cur) {
            if (imine) {
                if (fx) atomicAdd(&fld<unsigned long long>(c, t, bi, si, kFx), fx);
                if (fy) atomicAdd(&fld<unsigned long long>(c, t, bi, si, kFy), fy);
            }
            cur = I;
            const float4 v = stage_body(c, t, dense, pre, r, occ, R, nb, I * kTile + tid, gs, imine, bi, si);
            px = v.x;
            py = v.y;
            m = v.z;
            gsm = v.w;
            fx = fy = 0ull;
        }
        bool jmine;
        uint64_t bj = 0;
        uint32_t sl;
        const float4 v = stage_body(c, t, dense, pre, r, occ, R, nb, J * kTile + tid, gs, jmine, bj, sl);
        __syncthreads();                             // readers of the previous tile are done
        sj[2u * tid - lane] = v;                     // = 64 warp + lane
        sj[2u * tid - lane + 32u] = v;
        // G S a power of two and every mass of both tiles a small integer: the
        // products (G S m_i) m_j and (G S m_j) m_i are exact, hence equal; with
        // all coordinates of both tiles bounded, d2 is finite
        const bool same = __syncthreads_and(small_integer(m) && small_integer(v.z) &&
                                            bounded(make_float4(px, py, 0.f, 0.f)) && bounded(v)) && gs_pow2;
        const bool diag = I == J;
#pragma unroll 1
        for (uint32_t k = 0; k < kSymGroups; ++k) {
            const uint32_t g = (warp + k) & (kSymGroups - 1u);
            if (diag && g < warp) continue;
            const float4* col = sj + 64u * g + lane;
            if (diag && g == warp) {
#pragma unroll 4
                for (uint32_t s = 1; s < 32u; ++s) {
                    const float4 q = col[s];
                    pair_term(px, py, gsm, q.x, q.y, q.z, eps2, fx, fy);
                }
                continue;
            }
            if (same)
                sym_group<true>(col, px, py, m, gsm, eps2, g, lane, src, fx, fy, sacc[0], sacc[1]);
            else
                sym_group<false>(col, px, py, m, gsm, eps2, g, lane, src, fx, fy, sacc[0], sacc[1]);
        }
        __syncthreads();                             // every j sum of the item is in
        const unsigned long long jx = sacc[0][tid], jy = sacc[1][tid];
        sacc[0][tid] = 0ull;
        sacc[1][tid] = 0ull;
        if (jmine) {
            if (jx) atomicAdd(&fld<unsigned long long>(c, t, bj, sl, kFx), jx);
            if (jy) atomicAdd(&fld<unsigned long long>(c, t, bj, sl, kFy), jy);
        }
        if (++J == nt) {
            ++I;
            J = I;
        }
    }
    if (imine) {
        if (fx) atomicAdd(&fld<unsigned long long>(c, t, bi, si, kFx), fx);
        if (fy) atomicAdd(&fld<unsigned long long>(c, t, bi, si, kFy), fy);
    }
}

// ---------------------------------------------------------------------------
// FIND over unordered pairs.  Of two distinct bodies exactly one is "bigger"
// (heavier, or as heavy with the lower id), and both see the same d2 (the
// differences of the pair are exact negations), so one evaluation per pair
// decides whose candidate it is and with which key: the smaller body's, with
// key bits(d2) << 32 | id of the bigger one.  Pairs farther apart than the merge
// distance are the rule and cost a distance and a compare; a pair within reach
// updates the i body's key in a register or the j body's key by a shared
// atomicMin, folded into the fx field with one global atomicMin per body and
// item (i keys when the CTA moves to the next row).  Tiles, items and staging
// as in k_force_sym; no running sums move between lanes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 stage_find(const dsoa_ctx& c, uint32_t t, bool dense, const uint32_t* pre,
                                             uint32_t r, const unsigned long long* __restrict__ occ,
                                             const uint32_t* __restrict__ R, uint32_t nb, uint64_t d, bool& ok,
                                             uint64_t& b, uint32_t& slot) {
    float4 v = make_float4(0.f, 0.f, 0.f, __uint_as_float(kNone));
    uint32_t q = 0;
    slot = 0;
    ok = d < nb && locate(dense, pre, r, occ, (uint32_t)d, q, slot);
    if (ok) {
        b = __ldg(&R[q]);
        v.x = fld<float>(c, t, b, slot, kPx);
        v.y = fld<float>(c, t, b, slot, kPy);
        v.z = fld<float>(c, t, b, slot, kM);
        v.w = __uint_as_float(fld<uint32_t>(c, t, b, slot, kId));
    }
    return v;
}

__global__ void __launch_bounds__(256) k_find_sym(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                  const unsigned long long* __restrict__ occ,
                                                  const uint32_t* __restrict__ r_dev, dsoa_nbody_args a) {
    __shared__ float4 sj[2 * kTile];                 // group g at [64 g, 64 g + 64): its 32 bodies twice
    __shared__ unsigned long long smin[kTile];       // j keys of the item
    __shared__ uint32_t pre[kDenseMaxR + 1];
    __shared__ uint32_t wsum[8];
    const uint32_t r = __ldg(r_dev);
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const bool dense = r <= kDenseMaxR;
    const uint32_t nb = index_space(dense, r, occ, pre, wsum);
    const float rc2 = a.rc2;
    const uint64_t nt = (nb + kTile - 1) / kTile, items = nt * (nt + 1) / 2;
    const uint64_t wb = items * blockIdx.x / gridDim.x, we = items * (blockIdx.x + 1) / gridDim.x;
    smin[tid] = ~0ull;
    uint64_t I = 0, J = 0;
    if (wb < we) {
        uint64_t lo = 0, hi = nt;
        while (hi - lo > 1u) {
            const uint64_t mid = (lo + hi) >> 1;
            if (tri_start(mid, nt) <= wb) lo = mid; else hi = mid;
        }
        I = lo;
        J = I + (wb - tri_start(I, nt));
    }
    uint64_t cur = ~0ull, bi = 0;
    uint32_t si = 0, id = kNone;
    bool imine = false;
    float px = 0.f, py = 0.f, m = 0.f;
    unsigned long long key = ~0ull;
    for (uint64_t w = wb; w < we; ++w) {
        if (I != cur) {
            if (imine && key != ~0ull) atomicMin(&fld<unsigned long long>(c, t, bi, si, kFx), key);
            cur = I;
            const float4 v = stage_find(c, t, dense, pre, r, occ, R, nb, I * kTile + tid, imine, bi, si);
            px = v.x;
            py = v.y;
            m = v.z;
            id = __float_as_uint(v.w);
            key = ~0ull;
        }
        bool jmine;
        uint64_t bj = 0;
        uint32_t sl;
        const float4 v = stage_find(c, t, dense, pre, r, occ, R, nb, J * kTile + tid, jmine, bj, sl);
        __syncthreads();                             // readers of the previous tile are done
        sj[2u * tid - lane] = v;
        sj[2u * tid - lane + 32u] = v;
        __syncthreads();
        const bool diag = I == J;
#pragma unroll 1
        for (uint32_t k = 0; k < kSymGroups; ++k) {
            const uint32_t g = (warp + k) & (kSymGroups - 1u);
            if (diag && g < warp) continue;
            const float4* col = sj + 64u * g + lane;
            const bool own = diag && g == warp;      // own group: the i side of each ordered pair
#pragma unroll 8
            for (uint32_t s = own ? 1u : 0u; s < 32u; ++s) {
                const float4 q = col[s];
                const float dx = __fsub_rn(q.x, px), dy = __fsub_rn(q.y, py);
                const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                if (d2 < rc2) {                      // rare: a pair within reach
                    const uint32_t qid = __float_as_uint(q.w);
                    const unsigned long long hi = (unsigned long long)__float_as_uint(d2) << 32;
                    if (q.z > m || (q.z == m && qid < id)) {
                        const unsigned long long kk = hi | qid;
                        if (kk < key) key = kk;
                    } else if (!own) {
                        atomicMin(&smin[32u * g + ((lane + s) & 31u)], hi | id);
                    }
                }
            }
        }
        __syncthreads();                             // every j key of the item is in
        const unsigned long long jk = smin[tid];
        smin[tid] = ~0ull;
        if (jmine && jk != ~0ull) atomicMin(&fld<unsigned long long>(c, t, bj, sl, kFx), jk);
        if (++J == nt) {
            ++I;
            J = I;
        }
    }
    if (imine && key != ~0ull) atomicMin(&fld<unsigned long long>(c, t, bi, si, kFx), key);
}

// Body's field sizes in bytes (id, px, py, vx, vy, m, fx, fy, target, incoming, merged)
constexpr uint32_t kFieldBytes[11] = {4, 4, 4, 4, 4, 4, 8, 8, 4, 4, 4};

int check_args(dsoa_heap* h, int type, const dsoa_nbody_args& a) {
    if (type != a.body_type || h->types[type].nfields != 11) return DSOA_ERR_INVALID_ARG;
    for (int f = 0; f < 11; ++f)
        if (h->types[type].field_bytes[f] != kFieldBytes[f]) return DSOA_ERR_INVALID_ARG;
    if (!(a.eps2 > 0.0f) || !(a.fscale > 0.0f)) return DSOA_ERR_INVALID_ARG;
    return DSOA_OK;
}

}  // namespace

int dsoa_nbody_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb) {
    dsoa_nbody_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (ctor != DSOA_C_NBODY) return DSOA_ERR_UNKNOWN_METHOD;
    rc = check_args(h, type, args);
    if (rc) return rc;
    if (n > args.n_ids || n > 0xFFFFFFFFull || (!args.init && args.mass_max == 0)) return DSOA_ERR_INVALID_ARG;
    return dsoa_run_new<Ctor>(h, type, n, args);
}

int dsoa_nbody_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_nbody_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    rc = check_args(h, type, args);
    if (rc) return rc;
    switch (method) {
        case DSOA_M_NBODY_FORCE: return dsoa_run_doall<Force>(h, type, args);
        case DSOA_M_NBODY_MOVE: return dsoa_run_doall<Move>(h, type, args);
        case DSOA_M_COLL_FIND: return dsoa_run_doall<Find>(h, type, args);
        case DSOA_M_COLL_CLAIM:
            if (!args.handle_of) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<Claim>(h, type, args);
        case DSOA_M_COLL_MERGE:
            if (!args.handle_of) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<Merge>(h, type, args);
        case DSOA_M_COLL_DELETE: return dsoa_run_doall<Delete>(h, type, args);
        case DSOA_M_NBODY_READ:
            if (!args.out || !args.alive_out) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<Read>(h, type, args);
        case DSOA_M_NBODY_FORCE_TILED:
        case DSOA_M_COLL_FIND_TILED: {
            if (h->ctx.M * 64ull >= 0xFFFFFFFFull) return DSOA_ERR_INVALID_ARG;  // 32-bit slot indices
            // mass-0 placeholders add exactly 0 only while the inverse cube is finite
            if (method == DSOA_M_NBODY_FORCE_TILED && !(args.eps2 >= 0x1p-80f)) return DSOA_ERR_INVALID_ARG;
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            const bool all_pairs = (args.flags & DSOA_NBODY_ALL_PAIRS) != 0u;
            auto* k = method == DSOA_M_COLL_FIND_TILED ? (all_pairs ? &k_pairs_tiled<FindOp> : &k_find_sym)
                                                       : (all_pairs ? &k_pairs_tiled<ForceOp> : &k_force_sym);
            const unsigned grid = (unsigned)(dsoa_resident_ctas(reinterpret_cast<const void*>(k), 256) * h->num_sms);
            k<<<grid ? grid : 1u, 256, 0, h->stream>>>(dsoa_launch_ctx(h), (uint32_t)type, h->R[type], h->Rocc[type],
                                                     h->r_dev[type], args);
            return dsoa_check_launch(h);
        }
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}
