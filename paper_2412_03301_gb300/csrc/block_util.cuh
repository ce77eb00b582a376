// block_util.cuh -- small block-wide helpers used by several kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bvss {

// Exclusive prefix sum of v over the block, in thread order.  sh must hold
// THREADS/32 + 1 ints.  Every thread of the block must call it.
template <int THREADS>
__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? sh[lane] : 0;
        int s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) sh[lane] = s - w;
        if (lane == NW - 1) sh[NW] = s;
    }
    __syncthreads();
    const int res = sh[warp] + x - v;
    *total = sh[NW];
    __syncthreads();
    return res;
}

// Order-preserving map of an FP32 value to uint32 (larger value -> larger
// key).  -0.0 and +0.0 map to the same key, so they tie as values do.
__device__ __forceinline__ uint32_t order_key(float a) {
    if (a == 0.0f) a = 0.0f;
    const uint32_t u = __float_as_uint(a);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace bvss
