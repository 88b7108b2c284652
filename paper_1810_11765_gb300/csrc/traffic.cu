// traffic.cu -- batched Nagel-Schreckenberg rings as an SMMO application
// (Table 1 "traffic"; Nagel & Schreckenberg 1992).  Car {0 ring, 1 pos, 2 v}
// objects of all rings share one heap and one launch per step.  Occupancy is
// double-buffered (step t reads buffer t&1, writes the other), so a step is
// CLEAR(next) -> Car.move (do-all) -> ONRAMP -> ADVANCE(t); ONRAMP_ADVANCE does the
// last two in one launch.
#include "dsoa_internal.cuh"
#include "rng.cuh"

namespace {

constexpr uint32_t kVmax = 5u;

__device__ __forceinline__ uint32_t ring_of(const uint64_t* base, uint32_t n, uint64_t g) {
    uint32_t lo = 0, hi = n;  // base[lo] <= g < base[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

struct Move {
    using Args = dsoa_traffic_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t step = *a.t_dev;
        const uint8_t* cur = (step & 1u) ? a.occ1 : a.occ0;
        uint8_t* nxt = (step & 1u) ? a.occ0 : a.occ1;
        const uint32_t i = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, i, a.n_rings)) return;
        uint32_t* posp = dsoa_column<uint32_t>(c, t, bid, 1) + s;
        uint32_t* vp = dsoa_column<uint32_t>(c, t, bid, 2) + s;
        const uint64_t b = a.ring_base[i];
        const uint32_t L = (uint32_t)(a.ring_base[i + 1] - b);
        const uint32_t pos = *posp;
        if (!dsoa_index_ok(c, pos, L)) return;
        uint32_t v = min(*vp + 1u, kVmax);                 // accelerate
        // free cells ahead: the kVmax cells in front are read at once (independent
        // loads, one round trip) and scanned in registers, instead of one load per
        // cell that waits for the previous one
        uint8_t ahead[kVmax];
#pragma unroll
        for (uint32_t k = 0; k < kVmax; ++k) {
            uint32_t q = pos + 1u + k;
            if (q >= L) q %= L;
            ahead[k] = cur[b + q];
        }
        uint32_t gap = v;
#pragma unroll
        for (uint32_t k = kVmax; k-- > 0;)
            if (k < v && ahead[k]) gap = k;
        v = min(v, gap);                                   // brake
        if (v > 0u && dsoa_philox_w0(a.seed, step, pos, i, 1u) < a.slow_thr) v -= 1u;  // dawdle
        const uint32_t np = (pos + v) % L;                 // move
        const uint32_t off = L / 2u;
        if (np == off && dsoa_philox_w0(a.seed, step, off, i, 2u) < a.ramp_thr) {
            dsoa_delete(c, dsoa_make_handle(t, bid, s));   // leaves at the off-ramp
            return;
        }
        *posp = np;
        *vp = v;
        nxt[b + np] = 1;
    }
};

struct Read {
    using Args = dsoa_traffic_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t i = dsoa_column<uint32_t>(c, t, bid, 0)[s];
        if (!dsoa_index_ok(c, i, a.n_rings)) return;
        const uint32_t pos = dsoa_column<uint32_t>(c, t, bid, 1)[s];
        if (!dsoa_index_ok(c, pos, a.ring_base[i + 1] - a.ring_base[i])) return;
        a.vel_out[a.ring_base[i] + pos] = (uint8_t)dsoa_column<uint32_t>(c, t, bid, 2)[s];
    }
};

__global__ void k_init(dsoa_ctx c, dsoa_traffic_args a, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
        const uint32_t i = ring_of(a.ring_base, a.n_rings, g);
        const uint32_t j = (uint32_t)(g - a.ring_base[i]);
        const bool present = a.init_occ ? (a.init_occ[g] != 0)
                                        : (dsoa_philox_w0(a.seed, 0xFFFFFFFFu, j, i, 0u) < a.ring_thr[i]);
        dsoa_obj o = 0;
        if (present) {
            o = dsoa_new(c, (uint32_t)a.car_type);
            if (o) {
                dsoa_field<uint32_t>(c, o, 0) = i;
                dsoa_field<uint32_t>(c, o, 1) = j;
                dsoa_field<uint32_t>(c, o, 2) = a.init_v ? (uint32_t)a.init_v[g] : 0u;
            }
        }
        a.occ0[g] = o ? 1 : 0;
        a.occ1[g] = 0;
    }
}

__global__ void k_clear(dsoa_traffic_args a, uint64_t n) {
    const uint32_t step = *a.t_dev;
    uint8_t* nxt = (step & 1u) ? a.occ0 : a.occ1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 16;
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; g < n; g += stride) {
        if (g + 16 <= n && ((reinterpret_cast<uintptr_t>(nxt + g) & 15u) == 0)) {
            *reinterpret_cast<uint4*>(nxt + g) = make_uint4(0, 0, 0, 0);
        } else {
            for (uint64_t k = g; k < g + 16 && k < n; ++k) nxt[k] = 0;
        }
    }
}

__global__ void k_onramp(dsoa_ctx c, dsoa_traffic_args a) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_rings) return;
    const uint32_t step = *a.t_dev;
    uint8_t* nxt = (step & 1u) ? a.occ0 : a.occ1;
    const uint64_t b = a.ring_base[i];
    if (nxt[b] == 0 && dsoa_philox_w0(a.seed, step, 0u, i, 3u) < a.ramp_thr) {
        const dsoa_obj o = dsoa_new(c, (uint32_t)a.car_type);
        if (o) {
            dsoa_field<uint32_t>(c, o, 0) = i;
            dsoa_field<uint32_t>(c, o, 1) = 0u;
            dsoa_field<uint32_t>(c, o, 2) = 0u;
            nxt[b] = 1;
        }
    }
}

__global__ void k_advance(uint32_t* t_dev) { *t_dev += 1u; }

// ONRAMP and ADVANCE in one launch: one CTA takes every ring (nothing else reads
// t during the kernel), then advances t once all its threads have read it.
__global__ void k_onramp_advance(dsoa_ctx c, dsoa_traffic_args a) {
    const uint32_t step = *a.t_dev;
    uint8_t* nxt = (step & 1u) ? a.occ0 : a.occ1;
    for (uint32_t i = threadIdx.x; i < a.n_rings; i += blockDim.x) {
        const uint64_t b = a.ring_base[i];
        if (nxt[b] == 0 && dsoa_philox_w0(a.seed, step, 0u, i, 3u) < a.ramp_thr) {
            const dsoa_obj o = dsoa_new(c, (uint32_t)a.car_type);
            if (o) {
                dsoa_field<uint32_t>(c, o, 0) = i;
                dsoa_field<uint32_t>(c, o, 1) = 0u;
                dsoa_field<uint32_t>(c, o, 2) = 0u;
                nxt[b] = 1;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.t_dev = step + 1u;
}

}  // namespace

int dsoa_traffic_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_traffic_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (type != args.car_type || !args.ring_base || !args.t_dev) return DSOA_ERR_INVALID_ARG;
    switch (method) {
        case DSOA_M_TRAFFIC_MOVE: return dsoa_run_doall<Move>(h, type, args);
        case DSOA_M_TRAFFIC_READ:
            if (!args.vel_out) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<Read>(h, type, args);
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}

int dsoa_traffic_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb) {
    dsoa_traffic_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (!args.ring_base || !args.t_dev || !args.occ0 || !args.occ1 || args.n_rings == 0) return DSOA_ERR_INVALID_ARG;
    switch (kernel) {
        case DSOA_K_TRAFFIC_INIT: {
            if (n == 0) return DSOA_OK;
            if (args.car_type < 0 || args.car_type >= h->ntypes || !args.ring_thr) return DSOA_ERR_INVALID_ARG;
            k_init<<<dsoa_new_grid(h, n, 256), 256, 0, h->stream>>>(dsoa_launch_ctx(h), args, n);
            return dsoa_check_launch(h);
        }
        case DSOA_K_TRAFFIC_CLEAR: {
            if (n == 0) return DSOA_OK;
            const uint64_t chunks = (n + 15) / 16;
            const unsigned g = (unsigned)std::min<uint64_t>((chunks + 255) / 256, (uint64_t)h->num_sms * 8);
            k_clear<<<g ? g : 1, 256, 0, h->stream>>>(args, n);
            return dsoa_check_launch(h);
        }
        case DSOA_K_TRAFFIC_ONRAMP:
            k_onramp<<<(args.n_rings + 63) / 64, 64, 0, h->stream>>>(dsoa_launch_ctx(h), args);
            return dsoa_check_launch(h);
        case DSOA_K_TRAFFIC_ADVANCE:
            k_advance<<<1, 1, 0, h->stream>>>(args.t_dev);
            return dsoa_check_launch(h);
        case DSOA_K_TRAFFIC_ONRAMP_ADVANCE:
            k_onramp_advance<<<1, 256, 0, h->stream>>>(dsoa_launch_ctx(h), args);
            return dsoa_check_launch(h);
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}
