// Device helpers shared by the kernels of libsmcgm.so.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace smcgm {

// Sum over the block; the result is valid in thread 0.  `sh` holds >= 32 doubles.
__device__ inline double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__device__ inline double block_max(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = -1.0 / 0.0;
    if (wid == 0) {
        v = lane < nw ? sh[lane] : -1.0 / 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

// Reciprocal of a positive double by Newton-Raphson iteration y <- y (2 - x y)
// from a single-precision seed: each step squares the relative error, so two
// steps take the ~2^-23 seed error below 2^-53.  Used where a correctly rounded
// division is not required (coefficients known to ~1 ulp suffice).
__device__ inline double recip_nr(double x) {
    double y = (double)(1.0f / (float)x);
    y = y * fma(-x, y, 2.0);
    y = y * fma(-x, y, 2.0);
    return y;
}

// Asynchronous copy of one element from global to shared memory (cp.async,
// 4 or 8 bytes; both addresses aligned to the element).  A block issues all
// its copies and then waits once, instead of one DRAM round trip per copy:
// an ordinary load into a shared array cannot pass the preceding shared
// store, because the compiler cannot rule out that the two alias.
template <typename T>
__device__ inline void cp_async_elem(T* shared_dst, const T* global_src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async copies 4 or 8 bytes here");
    const unsigned d = (unsigned)__cvta_generic_to_shared(shared_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(global_src), "n"((int)sizeof(T)) : "memory");
}

// Waits for every cp.async this thread issued; a __syncthreads() after it
// makes the copies of all threads visible to the block.
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace smcgm
