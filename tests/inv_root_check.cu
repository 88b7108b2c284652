// Exhaustive check of dsoa_rcp_sqrt_rn (csrc/rn_math.cuh) against the correctly
// rounded intrinsics RN(1 / RN(sqrt x)) over every binary32 bit pattern in
// [lo, hi): the number of inputs whose result bits differ.
#include <cstdint>

#include "rn_math.cuh"

__global__ void k_count(uint32_t lo, uint32_t hi, unsigned long long* out) {
    unsigned long long bad = 0;
    const uint32_t n = hi - lo;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(lo + i);
        bad += __float_as_uint(dsoa_rcp_sqrt_rn(x)) != __float_as_uint(__frcp_rn(__fsqrt_rn(x)));
    }
    if (bad) atomicAdd(out, bad);
}

extern "C" long long inv_root_mismatches(uint32_t lo, uint32_t hi) {
    unsigned long long* d = nullptr;
    if (hi <= lo || cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return -1;
    unsigned long long h = 0;
    cudaMemset(d, 0, sizeof(*d));
    k_count<<<4096, 256>>>(lo, hi, d);
    const bool ok = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    return ok ? (long long)h : -1;
}
