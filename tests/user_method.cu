// A user library of do-all methods, built against the public device header
// only (include/dsoa_device.cuh) and linked against libdsoa: the path a user of
// the runtime takes for methods that are not built in (Sec. 2.1).
//
// Methods over the microbench type {0 id i32, 1 x f32, 2 tag u64}:
//   1000 scale   x = x * 1.5 + id (every operation rounded to nearest)
//   1001 spawn   allocate one object of args.other_type holding this id
//   1002 mark    out[id] = 1 for a live object of a type whose field 0 is an id
//   1003 tally   a prologue that adds 1 to *(uint32_t*)out once per launch that
//                runs it (CTA 0, thread 0); the per-object method does nothing
#include "dsoa_device.cuh"

struct UserArgs {
    uint32_t other_type;
    uint32_t n_ids;
    uint8_t* out;
};

struct UserScale {
    typedef UserArgs Args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args&) {
        float& x = dsoa_column<float>(c, t, bid, 1)[s];
        const int32_t id = dsoa_column<int32_t>(c, t, bid, 0)[s];
        x = __fadd_rn(__fmul_rn(x, 1.5f), (float)id);
    }
};

struct UserSpawn {
    typedef UserArgs Args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const dsoa_obj o = dsoa_new(c, a.other_type);
        if (o) dsoa_field<int32_t>(c, o, 0) = dsoa_column<int32_t>(c, t, bid, 0)[s];
    }
};

struct UserMark {
    typedef UserArgs Args;
    static __device__ void run(const dsoa_ctx& c, uint32_t t, uint64_t bid, uint32_t s, const Args& a) {
        const uint32_t id = (uint32_t)dsoa_column<int32_t>(c, t, bid, 0)[s];
        if (id < a.n_ids) a.out[id] = 1;
    }
};

struct UserTally {
    typedef UserArgs Args;
    static __device__ void prologue(const dsoa_ctx&, const Args& a) {
        if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned int*>(a.out), 1u);
    }
    static __device__ void run(const dsoa_ctx&, uint32_t, uint64_t, uint32_t, const Args&) {}
};

DSOA_METHOD(1000, user_scale, UserScale)
DSOA_METHOD(1001, user_spawn, UserSpawn)
DSOA_METHOD(1002, user_mark, UserMark)
DSOA_METHOD(1003, user_tally, UserTally)
