// Device helpers shared by the CUDA kernels of liblaker (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "laker_internal.h"

namespace lk {

constexpr int WARP = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum; every thread receives the result.  `red` needs
// blockDim.x / 32 slots.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
    if (wid == 0) s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Last-block-done ticket.  Call after thread 0 has written this block's
// partial; returns true in exactly one block, which may then read every
// block's partial (with ld.cg) and must reset the ticket.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x * gridDim.y * gridDim.z - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Sum of partials[0..count) in a fixed order by one block.
__device__ __forceinline__ double sum_partials(const double* partials, int count, double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += __ldcg(partials + i);
    return block_sum(s, red);
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// Grid-wide barrier of a cooperative launch (every CTA resident).  The wait is
// bounded: after ~2 s it raises LAKER_ERR_TIMEOUT in *err, and once *err is
// set every CTA leaves at its next barrier.  Returns false in that case.
struct GridSync {
    unsigned int count;
    unsigned int gen;
};
constexpr long long GRID_SPIN_CYCLES = 4000000000ll;
// Arrival is one acq_rel atomic on the counter (release: everything the CTA
// wrote before the bar.sync that precedes it; acquire: the arrivals before
// it), the last arrival resets the counter and publishes the next generation
// with a release store, and the others poll it with acquire loads; no full
// fences.  The generation is read before arriving, so it is this barrier's.
__device__ __forceinline__ bool grid_sync(GridSync* gs, int* err, long long budget = GRID_SPIN_CYCLES) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int g, prev;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&gs->gen) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&gs->count) : "memory");
        if (prev == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(&gs->count), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&gs->gen), "r"(g + 1u) : "memory");
        } else {
            const long long t0 = clock64();
            for (unsigned int spins = 1;; ++spins) {
                unsigned int cur;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(&gs->gen) : "memory");
                if (cur != g) break;
                if ((spins & 63u) == 0) {
                    if (*(volatile int*)err) break;
                    if (clock64() - t0 > budget) {
                        atomicExch(err, LAKER_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
        ok_s = (*(volatile int*)err == 0);
    }
    __syncthreads();
    return ok_s != 0;
}

// Block pairs (I, J) of an upper triangle, I <= J < nb, restricted to J >= j0
// (j0 = 0: all of them).  An operator extended by new points recomputes only
// the pairs whose column block reaches them.  Order: the rectangle I < j0 row
// by row, then the triangle j0 <= I <= J row by row.
__host__ __device__ __forceinline__ int64_t upper_pairs(int nb, int j0) {
    const int64_t w = nb - j0;
    return (int64_t)j0 * w + w * (w + 1) / 2;
}
__host__ __device__ __forceinline__ void upper_pair(int64_t t, int nb, int j0, int& I, int& J) {
    const int64_t w = nb - j0;
    if (t < (int64_t)j0 * w) {
        I = (int)(t / w);
        J = j0 + (int)(t % w);
        return;
    }
    t -= (int64_t)j0 * w;
    int i = j0;
    while (t >= nb - i) { t -= nb - i; ++i; }
    I = i;
    J = i + (int)t;
}

}  // namespace lk
