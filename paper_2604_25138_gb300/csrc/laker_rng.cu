// Random directions z_k ~ N(0, I_n) drawn on the device (Sec. IV-B,
// Eq. random_directions) from a counter-based generator, so that a fit can be
// driven by a seed instead of an n x N_r host array.
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011).  A 128-bit counter (c0..c3) and a
// 64-bit key (k0, k1) go through ten rounds; each round multiplies c0 and c2
// by the constants 0xD2511F53 and 0xCD9E8D57, keeps both halves of the
// 64-bit products and mixes them with c1, c3 and the key:
//     (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// and the key is bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85) before
// every round but the first.
//
// Normals: pair g of the n x N_r row-major array (elements 2g and 2g + 1)
// uses the block of counter (g mod 2^32, g div 2^32, 0, 0) under the key
// (seed mod 2^32, seed div 2^32).  Its words x0..x3 give two 53-bit uniforms
// u = ((x_a >> 6) 2^27 + (x_b >> 5) + 1/2) 2^-53 in (0, 1), from (x0, x1) and
// (x2, x3), and the Box-Muller transform turns them into
// r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 ln u1).
#include <cmath>

#include "laker_internal.h"

namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
    const uint64_t m = ((uint64_t)(a >> 6) << 27) | (uint64_t)(b >> 5);
    return ((double)m + 0.5) * 0x1.0p-53;
}

__global__ void k_philox_words(uint2 key, uint64_t ctr0, int64_t count, uint32_t* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const uint64_t g = ctr0 + (uint64_t)j;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0u, 0u), key);
    out[4 * j] = x.x;
    out[4 * j + 1] = x.y;
    out[4 * j + 2] = x.z;
    out[4 * j + 3] = x.w;
}

__global__ void k_gauss(uint2 key, int64_t count, double* __restrict__ Z) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * g >= count) return;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)((uint64_t)g >> 32), 0u, 0u), key);
    const double u1 = uniform53(x.x, x.y), u2 = uniform53(x.z, x.w);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    Z[2 * g] = r * c;
    if (2 * g + 1 < count) Z[2 * g + 1] = r * s;
}

}  // namespace

laker_status random_directions(laker_ctx* ctx, uint64_t seed, int64_t count, double* Z) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t pairs = (count + 1) / 2;
    k_gauss<<<(unsigned)((pairs + 255) / 256), 256, 0, ctx->stream>>>(key, count, Z);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

extern "C" laker_status laker_philox4x32_10(laker_ctx* ctx, uint64_t key, uint64_t counter0, int64_t count,
                                            uint32_t* out) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!out || count < 0) return set_error(ctx, LAKER_ERR_ARG, "philox: bad arguments");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    if (count == 0) return LAKER_OK;
    k_philox_words<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(
        make_uint2((uint32_t)key, (uint32_t)(key >> 32)), counter0, count, out);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

extern "C" laker_status laker_random_directions(laker_ctx* ctx, uint64_t seed, int64_t n, int n_r, double* Z) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!Z || n < 1 || n_r < 1) return set_error(ctx, LAKER_ERR_ARG, "random directions: bad arguments");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    return random_directions(ctx, seed, n * (int64_t)n_r, Z);
}
