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
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args&) {
        const int32_t id = dsoa_column<int32_t>(c, t, bid, 0)[s];
        float* x = dsoa_column<float>(c, t, bid, 1) + s;
        *x = micro_update(*x, id);
    }
};

struct MicroDelete {
    using Args = dsoa_micro_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = (uint32_t)dsoa_column<int32_t>(c, t, bid, 0)[s];
        if (dsoa_sm3(a.seed, id, a.round) & 1ull) dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

struct MicroDeleteAll {
    using Args = dsoa_micro_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args&) {
        dsoa_delete(c, dsoa_make_handle(t, bid, s));
    }
};

struct MicroHandles {
    using Args = dsoa_micro_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = (uint32_t)dsoa_column<int32_t>(c, t, bid, 0)[s];
        if (id < a.n_ids) a.handles_out[id] = dsoa_make_handle(t, bid, s);
    }
};

struct MicroGather {
    using Args = dsoa_micro_args;
    static constexpr bool kNoNewOfOwnType = true;   /* streamable */
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

// ---- bulk-copy staged do-all (Blackwell async copy engine) ----------------
// The id and x columns of CH consecutive blocks of R (2 x 256 B each) are
// copied into shared memory by cp.async.bulk, S chunks ahead, completing on a
// per-stage mbarrier by transaction bytes; 128 threads then update 4 slots
// each and store x straight to global (16-byte stores; per-slot stores where
// the snapshot has holes).  Bytes in flight per SM are bounded by shared
// memory (S x CH x 512 B per CTA), not by registers.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

constexpr uint32_t kBulkWaitLimit = 1u << 26;   // try_wait polls before giving up (error)

template <int CH, int S>
__global__ void __launch_bounds__(128) k_micro_scale_bulk(dsoa_ctx c, uint32_t t, const uint32_t* __restrict__ R,
                                                         const unsigned long long* __restrict__ occ,
                                                         const uint32_t* __restrict__ r_dev) {
    __shared__ __align__(128) int32_t s_id[S][CH][64];
    __shared__ __align__(128) float s_x[S][CH][64];
    __shared__ __align__(8) uint64_t bar[S];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t r = *r_dev;
    const uint32_t nchunks = (r + CH - 1) / CH;
    const uint32_t off_id = c.col_off[t][0], off_x = c.col_off[t][1];
    if (tid == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // producer: warp 0, lane i copies block i of the chunk
    auto issue = [&](uint32_t chunk, int stage) {
        const uint32_t first = chunk * CH;
        const uint32_t nb = min((uint32_t)CH, r - first);
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_tx(&bar[stage], nb * 512u);
        }
        __syncwarp();
        if (lane < nb) {
            const char* blk = c.data + (uint64_t)__ldg(&R[first + lane]) * c.block_bytes;
            bulk_g2s(&s_id[stage][lane][0], blk + off_id, 256u, &bar[stage]);
            bulk_g2s(&s_x[stage][lane][0], blk + off_x, 256u, &bar[stage]);
        }
    };
    __shared__ uint32_t s_abort;
    if (tid == 0) s_abort = 0u;
    __syncthreads();
    uint32_t j = 0;
    if (warp == 0)
        for (int k = 0; k < S; ++k) {
            const uint32_t ch = blockIdx.x + (uint32_t)k * gridDim.x;
            if (ch < nchunks) issue(ch, k);
        }
    for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++j) {
        const int stage = (int)(j % S);
        const uint32_t parity = (j / S) & 1u;
        bool ready = true;
        for (uint32_t polls = 0; !mbar_try_wait(&bar[stage], parity);) {
            if (++polls >= kBulkWaitLimit) { ready = false; break; }
        }
        if (!ready) {
            atomicOr(&s_abort, 1u);
        } else {
            const uint32_t first = ch * CH;
            const uint32_t bi = tid >> 4, q = tid & 15u;       // block in chunk, slot quad
            if (first + bi < r) {
                const uint32_t nib = (uint32_t)(__ldg(&occ[first + bi]) >> (q * 4)) & 0xFu;
                if (nib) {
                    const int4 id4 = *reinterpret_cast<const int4*>(&s_id[stage][bi][q * 4]);
                    float4 x4 = *reinterpret_cast<const float4*>(&s_x[stage][bi][q * 4]);
                    x4.x = micro_update(x4.x, id4.x);
                    x4.y = micro_update(x4.y, id4.y);
                    x4.z = micro_update(x4.z, id4.z);
                    x4.w = micro_update(x4.w, id4.w);
                    float* dst = reinterpret_cast<float*>(c.data + (uint64_t)__ldg(&R[first + bi]) * c.block_bytes +
                                                          off_x) + q * 4;
                    if (nib == 0xFu) {
                        __stcs(reinterpret_cast<float4*>(dst), x4);
                    } else {
                        if (nib & 1u) dst[0] = x4.x;
                        if (nib & 2u) dst[1] = x4.y;
                        if (nib & 4u) dst[2] = x4.z;
                        if (nib & 8u) dst[3] = x4.w;
                    }
                }
            }
        }
        __syncthreads();                                   // stage consumed by every thread
        if (s_abort) {
            // A copy did not land within the bound: report, then give the copies
            // still in flight into this CTA's shared memory a bounded time to land
            // before the CTA exits.  Uniform exit: every thread saw s_abort.
            if (tid == 0) {
                dsoa_raise(c, DSOA_DEV_SPIN);
                for (uint32_t k = 1; k <= (uint32_t)S; ++k) {
                    const uint32_t jj = j + k - 1;          // uses issued but not consumed
                    const uint32_t chk = blockIdx.x + jj * gridDim.x;
                    if (chk >= nchunks) break;
                    for (uint32_t polls = 0; polls < kBulkWaitLimit; ++polls)
                        if (mbar_try_wait(&bar[jj % S], (jj / S) & 1u)) break;
                }
            }
            return;
        }
        const uint32_t next = ch + (uint32_t)S * gridDim.x;
        if (warp == 0 && next < nchunks) issue(next, stage);
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

__global__ void k_micro_device_do(dsoa_ctx c, uint32_t t, uint64_t n, unsigned long long* out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long cnt = 0, sid = 0;
    dsoa_device_do(c, t, [&](dsoa_obj o) {
        cnt += 1;
        sid += (unsigned long long)(long long)dsoa_field<int32_t>(c, o, 0);
    });
    out[2 * i] = cnt;
    out[2 * i + 1] = sid;
}

/* Each thread allocates k objects one after another; the lanes of a warp
 * allocate together in every iteration, so each of the k rounds is one
 * warp-coalesced request of up to 32 slots. */
__global__ void k_micro_new_each(dsoa_ctx c, uint32_t t, uint64_t n, uint32_t k, dsoa_micro_args a) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        for (uint32_t j = 0; j < k; ++j) {
            const dsoa_obj o = dsoa_new(c, t);
            if (o) MicroCtor::ctor(c, o, i * k + j, a);
        }
}

/* L2 ceiling of single-lane 64-bit bitmap atomics (the allocator's building
 * block, Sec. 4): consecutive lanes hit words 17 apart (136 bytes), so each
 * lane's op is a separate L2 request, as a warp leader's reservation is. */
__global__ void k_micro_atomic_peak(unsigned long long* __restrict__ w, uint64_t mask, uint64_t n, uint32_t iters,
                                    unsigned long long key, unsigned long long* __restrict__ sink) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long acc = 0ull;
    for (uint32_t k = 0; k < iters; ++k) {
        const uint64_t idx = ((i + (uint64_t)k * n) * 17u) & mask;
        const unsigned long long bit = 1ull << (k & 63u);
        acc ^= (k & 1u) ? atomicOr(w + idx, bit) : atomicAnd(w + idx, ~bit);
    }
    if (acc == key) *sink = acc;
}

}  // namespace

int dsoa_micro_kernel(dsoa_heap* h, int kernel, uint64_t n, const void* a, size_t nb) {
    dsoa_micro_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (kernel == DSOA_K_MICRO_ATOMIC_PEAK) {
        const uint64_t nw = args.n_ids;
        if (!args.handles_out || !args.stats || n == 0 || args.round == 0 || nw < 32 || (nw & (nw - 1)))
            return DSOA_ERR_INVALID_ARG;
        k_micro_atomic_peak<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(
            (unsigned long long*)args.handles_out, nw - 1, n, args.round, (unsigned long long)args.seed,
            (unsigned long long*)args.stats);
        return dsoa_check_launch(h);
    }
    if (kernel == DSOA_K_MICRO_NEW_EACH) {
        const uint64_t type = args.n_ids;
        if (n == 0 || args.round == 0 || type >= (uint64_t)h->ntypes || h->types[type].nfields < 3 ||
            h->types[type].field_bytes[0] != 4 || h->types[type].field_bytes[1] != 4 ||
            h->types[type].field_bytes[2] != 8 || n * (uint64_t)args.round + args.id_base > 0xFFFFFFFFull)
            return DSOA_ERR_INVALID_ARG;
        const int tpb = 256;
        k_micro_new_each<<<dsoa_new_grid(h, n, tpb), tpb, 0, h->stream>>>(dsoa_launch_ctx(h), (uint32_t)type, n,
                                                                         args.round, args);
        return dsoa_check_launch(h);
    }
    if (kernel != DSOA_K_MICRO_DEVICE_DO) return DSOA_ERR_UNKNOWN_METHOD;
    if (!args.stats || n == 0 || h->ntypes < 1) return DSOA_ERR_INVALID_ARG;
    const int type = (int)args.round;    /* the type to visit */
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    k_micro_device_do<<<(unsigned)((n + 127) / 128), 128, 0, h->stream>>>(dsoa_launch_ctx(h), (uint32_t)type, n,
                                                                       (unsigned long long*)args.stats);
    return dsoa_check_launch(h);
}

int dsoa_micro_new(dsoa_heap* h, int type, uint64_t n, int ctor, const void* a, size_t nb) {
    dsoa_micro_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    if (ctor != DSOA_C_MICRO) return DSOA_ERR_UNKNOWN_METHOD;
    // the microbench type, or a type extending it (its first three columns)
    if (h->types[type].nfields < 3 || h->types[type].field_bytes[0] != 4 || h->types[type].field_bytes[1] != 4 ||
        h->types[type].field_bytes[2] != 8)
        return DSOA_ERR_INVALID_ARG;
    return dsoa_run_new<MicroCtor>(h, type, n, args);
}

int dsoa_micro_do(dsoa_heap* h, int type, int method, const void* a, size_t nb) {
    dsoa_micro_args args;
    int rc = dsoa_copy_args(&args, a, nb);
    if (rc) return rc;
    // The column kernels stream whole 64-slot columns; a type with fewer slots
    // per block (per-type capacity mode) runs the per-object method instead.
    if ((method == DSOA_M_MICRO_SCALE || method == DSOA_M_MICRO_SCALE_TMA) && type >= 0 && type < h->ntypes &&
        h->types[type].capacity != DSOA_SLOTS)
        method = DSOA_M_MICRO_SCALE_SCALAR;
    switch (method) {
        case DSOA_M_MICRO_SCALE: {
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            const dsoa_ctx c = dsoa_launch_ctx(h);
            const int tpb = h->doall_tpb;
            auto* k = &k_micro_scale_vec<4, 2>;
            if (h->vec_slots_per_thread == 1) k = &k_micro_scale_vec<1, 4>;
            if (h->vec_slots_per_thread == 2) k = &k_micro_scale_vec<2, 2>;
            k<<<dsoa_persistent_grid(h, k, tpb), tpb, 0, h->stream>>>(c, type, h->R[type], h->Rocc[type],
                                                                     h->r_dev[type]);
            return dsoa_check_launch(h);
        }
        case DSOA_M_MICRO_SCALE_TMA: {
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            auto* k = &k_micro_scale_bulk<8, 4>;
            k<<<dsoa_persistent_grid(h, k, 128), 128, 0, h->stream>>>(dsoa_launch_ctx(h), type, h->R[type],
                                                                    h->Rocc[type], h->r_dev[type]);
            return dsoa_check_launch(h);
        }
        case DSOA_M_MICRO_SCALE_SCALAR: return dsoa_run_doall<MicroScale>(h, type, args);
        case DSOA_M_MICRO_DELETE: return dsoa_run_doall<MicroDelete>(h, type, args);
        case DSOA_M_MICRO_DELETE_ALL: return dsoa_run_doall<MicroDeleteAll>(h, type, args);
        case DSOA_M_MICRO_HANDLES:
            if (!args.handles_out) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<MicroHandles>(h, type, args);
        case DSOA_M_MICRO_GATHER:
            if (!args.x_out || !args.live_out) return DSOA_ERR_INVALID_ARG;
            return dsoa_run_doall<MicroGather>(h, type, args);
        case DSOA_M_MICRO_STATS: {
            if (!args.stats) return DSOA_ERR_INVALID_ARG;
            rc = dsoa_prepare_doall(h, type);
            if (rc) return rc;
            k_micro_stats<<<dsoa_persistent_grid(h, &k_micro_stats, 256), 256, 0, h->stream>>>(
                h->ctx, type, h->R[type], h->Rocc[type], h->r_dev[type],
                                                                   (dsoa_micro_stats*)args.stats);
            return dsoa_check_launch(h);
        }
        default: return DSOA_ERR_UNKNOWN_METHOD;
    }
}
