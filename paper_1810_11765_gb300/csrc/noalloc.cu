// noalloc.cu -- enumeration (block list of one type + occupancy snapshot) into
// caller-provided buffers, with its working memory in a fixed device array of
// this library instead of memory that anyone allocates at call time.
//
// Who needs it: code that must not allocate device memory while it runs --
// a host program whose allocator owns every byte of the GPU under a fixed
// budget, a latency-critical loop where cudaMalloc / cudaFree would
// synchronise the device, or a caller that wants several enumerations alive
// at once in buffers it manages itself.  Such a caller passes its own output
// buffers; the per-tile counts, offsets and completion ticket of the scan live
// in `s_enum_scratch` below, a static array every GPU that loads this library
// holds until the process exits.
#include <mutex>

#include "dsoa_internal.cuh"

namespace {

constexpr uint32_t kMaxTiles = DSOA_NOALLOC_MAX_TILES;  // level-1 containers = blocks / 4096
constexpr int kMaxDevices = 64;

// [0, kMaxTiles) tile counts, [kMaxTiles, 2 kMaxTiles) tile offsets,
// [2 kMaxTiles] completion ticket of the counting kernel, rest padding.
static __device__ __align__(256) uint32_t s_enum_scratch[2 * kMaxTiles + 64];

uint32_t* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

__device__ __forceinline__ uint32_t warp_sum_na(uint32_t v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Counting half of the scan: one warp per level-1 container (4096 blocks);
// only level-0 containers whose level-1 bit is set are read.  The last CTA
// turns counts into exclusive offsets and writes r.
__global__ void k_tile_count_na(dsoa_ctx c, uint32_t b, uint64_t tiles, uint32_t* __restrict__ scratch,
                                uint32_t* __restrict__ r_out) {
    uint32_t* tcnt = scratch;
    uint32_t* toff = scratch + kMaxTiles;
    uint32_t* ticket = scratch + 2 * kMaxTiles;
    const uint32_t lane = threadIdx.x & 31u, wpc = blockDim.x >> 5;
    const unsigned long long* L0 = dsoa_level(c, b, 0);
    const unsigned long long* L1 = c.nlevels >= 2 ? dsoa_level(c, b, 1) : nullptr;
    const uint64_t w0 = c.lvl_words[0];
    for (uint64_t t = (uint64_t)blockIdx.x * wpc + (threadIdx.x >> 5); t < tiles; t += (uint64_t)gridDim.x * wpc) {
        const unsigned long long sel = L1 ? L1[t] : 1ull;
        uint32_t cnt = 0;
        const uint64_t a = t * 64 + lane, bb = a + 32;
        if (((sel >> lane) & 1ull) && a < w0) cnt += __popcll(L0[a]);
        if (((sel >> (lane + 32)) & 1ull) && bb < w0) cnt += __popcll(L0[bb]);
        cnt = warp_sum_na(cnt);
        if (lane == 0) tcnt[t] = cnt;
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ uint32_t part[1024];
    const uint64_t per = (tiles + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = threadIdx.x * per, hi = lo + per < tiles ? lo + per : tiles;
    uint32_t s = 0;
    for (uint64_t i = lo; i < hi; ++i) s += __ldcg(&tcnt[i]);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (uint32_t i = 0; i < blockDim.x; ++i) { const uint32_t v = part[i]; part[i] = run; run += v; }
        *r_out = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (uint64_t i = lo; i < hi; ++i) { toff[i] = run; run += __ldcg(&tcnt[i]); }
}

// Compaction half: 64 threads per tile, CTA-local prefix sum of popcounts,
// block ids staged in shared memory, written coalesced with the snapshot of
// each block's occupied slots.
__global__ void __launch_bounds__(64) k_compact_na(dsoa_ctx c, uint32_t b, uint64_t tiles,
                                                   const uint32_t* __restrict__ scratch,
                                                   uint32_t* __restrict__ R_out,
                                                   unsigned long long* __restrict__ occ_out) {
    __shared__ uint32_t list[4096];
    __shared__ uint32_t wsum[2];
    const uint32_t j = threadIdx.x, lane = threadIdx.x & 31u;
    const uint64_t t = blockIdx.x;
    unsigned long long w = 0ull;
    const unsigned long long sel = c.nlevels >= 2 ? dsoa_level(c, b, 1)[t] : 1ull;
    const uint64_t wi = t * 64 + j;
    if (((sel >> j) & 1ull) && wi < c.lvl_words[0]) w = dsoa_level(c, b, 0)[wi];
    const uint32_t cnt = __popcll(w);
    uint32_t incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    if (lane == 31) wsum[j >> 5] = incl;
    __syncthreads();
    const uint32_t excl = incl - cnt + ((j >= 32) ? wsum[0] : 0u);
    const uint32_t total = wsum[0] + wsum[1];
    uint32_t k = excl;
    for (unsigned long long x = w; x; x &= x - 1ull)
        list[k++] = (uint32_t)(wi * 64 + (uint32_t)(__ffsll((long long)x) - 1));
    __syncthreads();
    const uint32_t base = scratch[kMaxTiles + t];
    for (uint32_t i = j; i < total; i += 64) {
        const uint32_t bid = list[i];
        R_out[base + i] = bid;
        occ_out[base + i] = ~c.slot[bid];
    }
}

// Device address of s_enum_scratch on `dev` (the current device).  Outside
// stream capture it is looked up on every call, so an address made stale by a
// device reset (which reloads this library's module) is never used; a call
// under capture takes the address of the latest call outside capture on that
// device (nullptr if there was none).
uint32_t* scratch_address(int dev, bool capturing) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!capturing) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, s_enum_scratch) != cudaSuccess) {
            cudaGetLastError();
            g_scratch_addr[dev] = nullptr;
            return nullptr;
        }
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    }
    return g_scratch_addr[dev];
}

}  // namespace

extern "C" int dsoa_enumerate_noalloc(dsoa_heap* h, int type, uint32_t* R_out_dev, uint64_t* occ_out_dev,
                                      uint32_t* r_out_dev, uint64_t capacity) {
    if (!h || !R_out_dev || !occ_out_dev || !r_out_dev) return DSOA_ERR_INVALID_ARG;
    if (!h->frozen) return DSOA_ERR_NOT_FROZEN;
    if (type < 0 || type >= h->ntypes) return DSOA_ERR_INVALID_ARG;
    if (capacity < h->ctx.M) return DSOA_ERR_INVALID_ARG;
    if (h->tiles > kMaxTiles) return DSOA_ERR_SCRATCH_LIMIT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device || dev < 0 || dev >= kMaxDevices)
        return DSOA_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return DSOA_ERR_CUDA;
    }
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    uint32_t* scratch = scratch_address(dev, capturing);
    if (!scratch) return capturing ? DSOA_ERR_CAPTURE : DSOA_ERR_CUDA;
    // the ticket must start at zero; counts and offsets are overwritten
    if (cudaMemsetAsync(scratch + 2 * kMaxTiles, 0, sizeof(uint32_t), h->stream) != cudaSuccess)
        return DSOA_ERR_CUDA;
    const uint32_t b = dsoa_bm_alloc((uint32_t)type);
    const uint64_t warps = h->tiles;
    uint64_t g1 = (warps + 7) / 8;
    const uint64_t cap = (uint64_t)h->num_sms * 8;
    if (g1 > cap) g1 = cap;
    if (g1 == 0) g1 = 1;
    k_tile_count_na<<<(unsigned)g1, 256, 0, h->stream>>>(h->ctx, b, h->tiles, scratch, r_out_dev);
    if (cudaGetLastError() != cudaSuccess) return DSOA_ERR_CUDA;
    k_compact_na<<<(unsigned)h->tiles, 64, 0, h->stream>>>(h->ctx, b, h->tiles, scratch, R_out_dev,
                                                           (unsigned long long*)occ_out_dev);
    if (cudaGetLastError() != cudaSuccess) return DSOA_ERR_CUDA;
    return DSOA_OK;
}
