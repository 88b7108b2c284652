// micro.cu -- allocator + do-all microbench: one type {int32 id, float x,
// int64 tag} (fields 0, 1, 2).  Constructor, the fp32 update
// x = x * 1.5f + (float)id as a generic one-slot-per-thread do-all and as a
// 128-bit vectorised SOA kernel, the parity-driven delete, and read-back
// methods (per-object gather, warp-reduced statistics).
#include "dsoa_internal.cuh"
#include "rng.cuh"

namespace {

struct MicroCtor {
    using Args = dsoa_micro_args;
    static __device__ void ctor(const dsoa_ctx& c, dsoa_obj o, uint64_t i, const Args& a) {
        const uint32_t id = a.id_base + (uint32_t)i;
        dsoa_field<int32_t>(c, o, 0) = (int32_t)id;
        dsoa_field<float>(c, o, 1) = 0.0f;
        dsoa_field<unsigned long long>(c, o, 2) = dsoa_sm2(a.seed, id);
    }
};

// x * 1.5f rounded, then + (float)id rounded: never contracted to an FMA.
__device__ __forceinline__ float micro_update(float x, int32_t id) {
    return __fadd_rn(__fmul_rn(x, 1.5f), __int2float_rn(id));
}

struct MicroScale {
    using Args = dsoa_micro_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args&) {
        const int32_t id = dsoa_column<int32_t>(c, t, bid, 0)[s];
        float* x = dsoa_column<float>(c, t, bid, 1) + s;
        *x = micro_update(*x, id);
    }
};

struct MicroDelete {
    using Args = dsoa_micro_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = (uint32_t)dsoa_column<int32_t>(c, t, bid, 0)[s];
        if (dsoa_sm3(a.seed, id, a.round) & 1ull) dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

struct MicroDeleteAll {
    using Args = dsoa_micro_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args&) {
        dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

struct MicroGather {
    using Args = dsoa_micro_args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = (uint32_t)dsoa_column<int32_t>(c, t, bid, 0)[s];
        if (id < a.n_ids) {
            a.x_out[id] = dsoa_column<float>(c, t, bid, 1)[s];
            a.live_out[id] = 1;
        }
    }
};

// 128-bit vectorised do-all (Sec. 2.2: 128-byte SOA clusters served by vector
// loads).  SPT consecutive slots per thread, 64/SPT threads per heap block;
// a 64-slot int32/float column is 256 B = 16 threads x 16 B.  Loads of U
// grid-stride iterations are issued before any arithmetic to keep enough bytes
// in flight per SM; stores of partially occupied vectors fall back to
// per-element stores so that slots outside the snapshot are never written.
template <int SPT, int U>
__global__ void __launch_bounds__(512) k_micro_scale_vec(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                         const unsigned long long* __restrict__ occ,
                                                         const uint32_t* __restrict__ r_dev) {
    constexpr uint32_t TPB = 64 / SPT;
    using IV = typename std::conditional<SPT == 4, int4, typename std::conditional<SPT == 2, int2, int>::type>::type;
    using FV = typename std::conditional<SPT == 4, float4, typename std::conditional<SPT == 2, float2, float>::type>::type;
    const uint64_t n = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t q = (uint32_t)(tid % TPB);
    const uint64_t total = (uint64_t)(*r_dev) * TPB;
    const uint32_t off_id = c.col_off[t][0] + q * SPT * 4, off_x = c.col_off[t][1] + q * SPT * 4;
    const unsigned long long full = (SPT == 64) ? ~0ull : ((1ull << SPT) - 1ull);
    for (uint64_t g0 = tid; g0 < total; g0 += n * U) {
        IV idv[U];
        FV xv[U];
        uint32_t nib[U];
        char* base[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t g = g0 + (uint64_t)u * n;
            nib[u] = 0;
            if (g < total) {
                const uint64_t i = g / TPB;
                nib[u] = (uint32_t)((__ldg(&occ[i]) >> (q * SPT)) & full);
                base[u] = c.data + (uint64_t)__ldg(&R[i]) * c.block_bytes;
                if (nib[u]) {
                    idv[u] = __ldcs(reinterpret_cast<const IV*>(base[u] + off_id));
                    xv[u] = __ldcs(reinterpret_cast<const FV*>(base[u] + off_x));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!nib[u]) continue;
            const int32_t* ip = reinterpret_cast<const int32_t*>(&idv[u]);
            float* xp = reinterpret_cast<float*>(&xv[u]);
#pragma unroll
            for (int k = 0; k < SPT; ++k) xp[k] = micro_update(xp[k], ip[k]);
            FV* dst = reinterpret_cast<FV*>(base[u] + off_x);
            if (nib[u] == (uint32_t)full) {
                __stcs(dst, xv[u]);
            } else {
                float* d = reinterpret_cast<float*>(dst);
#pragma unroll
                for (int k = 0; k < SPT; ++k)
                    if ((nib[u] >> k) & 1u) d[k] = xp[k];
            }
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_xor64(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Statistics over the snapshot: whole warps read 32 slots of one block each;
// unoccupied lanes contribute zero; one set of atomics per warp.
__global__ void __launch_bounds__(512) k_micro_stats(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                     const unsigned long long* __restrict__ occ,
                                                     const uint32_t* __restrict__ r_dev, dsoa_micro_stats* out) {
    const uint64_t n = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t s = (uint32_t)(tid & 63u);
    const uint64_t total = (uint64_t)(*r_dev) * 64u;
    unsigned long long live = 0, sid = 0, stag = 0, xtag = 0;
    double sx = 0.0;
    for (uint64_t g = tid; g < total; g += n) {
        const uint64_t i = g >> 6;
        if ((occ[i] >> s) & 1ull) {
            const uint64_t bid = R[i];
            const int32_t id = dsoa_column<int32_t>(c, t, bid, 0)[s];
            const unsigned long long tag = dsoa_column<unsigned long long>(c, t, bid, 2)[s];
            live += 1;
            sid += (unsigned long long)(long long)id;
            stag += tag;
            xtag ^= tag;
            sx += (double)dsoa_column<float>(c, t, bid, 1)[s];
        }
    }
    live = warp_sum64(live); sid = warp_sum64(sid); stag = warp_sum64(stag);
    xtag = warp_xor64(xtag); sx = warp_sumd(sx);
    if ((threadIdx.x & 31u) == 0 && live) {
        atomicAdd(&out->live, live);
        atomicAdd(&out->sum_id, sid);
        atomicAdd(&out->sum_tag, stag);
        atomicXor(&out->xor_tag, xtag);
        atomicAdd(&out->sum_x, sx);
    }
}

}  // namespace

int dsoa_micro_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb) {
    dsoa_micro_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (ctor != DSOA_C_MICRO) return DSOA_ERR_UNKNOWN_METHOD;
    if (h->types[type].nfields != 3 || h->types[type].field_bytes[0] != 4 || h->types[type].field_bytes[1] != 4 ||
        h->types[type].field_bytes[2] != 8)
        return DSOA_ERR_INVALID_ARG;
    return dsoa_run_new<MicroCtor>(h, type, n, args);
}

int dsoa_micro_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_micro_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    switch (method) {
        case DSOA_M_MICRO_SCALE: {
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            const dsoa_ctx c = dsoa_launch_ctx(h);
            const unsigned g = dsoa_doall_grid(h);
            const int tpb = h->doall_tpb;
            switch (h->vec_slots_per_thread) {
                case 1: k_micro_scale_vec<1, 4><<<g, tpb, 0, h->stream>>>(c, type, h->R, h->Rocc, h->r_dev); break;
                case 2: k_micro_scale_vec<2, 2><<<g, tpb, 0, h->stream>>>(c, type, h->R, h->Rocc, h->r_dev); break;
                default: k_micro_scale_vec<4, 2><<<g, tpb, 0, h->stream>>>(c, type, h->R, h->Rocc, h->r_dev); break;
            }
            return dsoa_check_launch(h);
        }
        case DSOA_M_MICRO_SCALE_SCALAR: return dsoa_run_doall<MicroScale>(h, type, args);
        case DSOA_M_MICRO_DELETE: return dsoa_run_doall<MicroDelete>(h, type, args);
        case DSOA_M_MICRO_DELETE_ALL: return dsoa_run_doall<MicroDeleteAll>(h, type, args);
        case DSOA_M_MICRO_GATHER:
            if (!args.x_out || !args.live_out) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<MicroGather>(h, type, args);
        case DSOA_M_MICRO_STATS: {
            if (!args.stats) return DSOA_ERR_INVALID_ARG;
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            k_micro_stats<<<dsoa_doall_grid(h), 256, 0, h->stream>>>(h->ctx, type, h->R, h->Rocc, h->r_dev,
                                                                   (dsoa_micro_stats*)args.stats);
            return dsoa_check_launch(h);
        }
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}
