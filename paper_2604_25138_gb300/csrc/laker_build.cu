// Kernel construction: G_ij = exp(scale <q_i, q_j>)  (Sec. III-A,
// Eq. sc-exp-kernel; Algorithm 1, kernel-construction stage).
//
// G is symmetric, so only tiles (bi <= bj) are evaluated and each off-diagonal
// tile is written twice (direct and, through a shared-memory transpose,
// mirrored), halving the float64 exponentials -- the dominant cost on GB300,
// whose float64 pipe runs at ~1/74 of the float32 rate.  Float64 operators
// store G in float64; mixed operators store the float32 pair (hi, lo) with
// hi = fl32(G), lo = fl32(G - hi): hi alone is the float32 operator, hi + lo is
// G to ~2^-48 for the double-float true residual, in the same 8 bytes/entry.
#include <cuda_bf16.h>

#include <cmath>

#include "laker_device.cuh"

namespace {

constexpr int BT = 64;   // output tile edge
constexpr int BD = 32;   // embedding-dimension chunk

// Position of the 128 x 128 tile (I, J), I <= J, of the packed upper triangle
// of nb blocks (row-major over I).
__device__ __forceinline__ int64_t pk_tile(int I, int J, int nb) {
    return (int64_t)I * nb - (int64_t)I * (I - 1) / 2 + (J - I);
}

// MODE 0: float64 G, full n x ldk; MODE 1: float32 pair (hi, lo), full; MODE 2:
// float32 pair in the packed upper triangle of 128 x 128 tiles (K32 is the
// packed array; ldk is the number of 128-blocks), padding entries zero.
template <int MODE>
__global__ void __launch_bounds__(256)
k_build_sym(const double* __restrict__ Q, int64_t n, int d, double scale,
            double* __restrict__ K64, float* __restrict__ K32, float* __restrict__ K32lo, int64_t ldk, int nt, int j0) {
    constexpr bool PAIR = MODE != 0;
    // blockIdx.x enumerates the upper-triangular tile pairs with bj >= j0
    int bi, bj;
    lk::upper_pair(blockIdx.x, nt, j0, bi, bj);

    __shared__ double sm[2 * BD * (BT + 1)];
    double (*Qi)[BT + 1] = reinterpret_cast<double (*)[BT + 1]>(sm);
    double (*Qj)[BT + 1] = reinterpret_cast<double (*)[BT + 1]>(sm + BD * (BT + 1));
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

    for (int k0 = 0; k0 < d; k0 += BD) {
        for (int idx = threadIdx.x; idx < BT * BD; idx += blockDim.x) {
            const int r = idx / BD, k = idx % BD;
            const int64_t gi = (int64_t)bi * BT + r, gj = (int64_t)bj * BT + r;
            const bool kin = (k0 + k) < d;
            Qi[k][r] = (gi < n && kin) ? Q[gi * d + k0 + k] : 0.0;
            Qj[k][r] = (gj < n && kin) ? Q[gj * d + k0 + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < BD; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = Qi[k][ty + 16 * u]; b[u] = Qj[k][tx + 16 * u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }

    // exp, direct store, stage for the mirrored store
    double (*T)[BT + 1] = reinterpret_cast<double (*)[BT + 1]>(sm);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = ty + 16 * u;
        const int64_t i = (int64_t)bi * BT + r;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = tx + 16 * v;
            const int64_t j = (int64_t)bj * BT + c;
            const double g = exp(scale * acc[u][v]);
            T[r][c] = g;
            if (MODE == 2) {
                const double gz = (i < n && j < n) ? g : 0.0;
                const float h = (float)gz;
                float* tile = K32 + pk_tile(bi >> 1, bj >> 1, (int)ldk) * (2 * 128 * 128);
                const int row = (bi & 1) * BT + r, col = (bj & 1) * BT + c;
                tile[row * 128 + col] = h;
                tile[128 * 128 + row * 128 + col] = (float)(gz - (double)h);
            } else if (i < n && j < n) {
                if (PAIR) {
                    const float h = (float)g;
                    K32[i * ldk + j] = h;
                    K32lo[i * ldk + j] = (float)(g - (double)h);
                } else {
                    K64[i * ldk + j] = g;
                }
            }
        }
    }
    if (bi == bj) return;
    // packed: only a diagonal 128-tile needs its lower 64 x 64 block mirrored
    if (MODE == 2 && (bi >> 1) != (bj >> 1)) return;
    __syncthreads();
    for (int idx = threadIdx.x; idx < BT * BT; idx += blockDim.x) {
        const int c = idx / BT, r = idx % BT;   // output row bj*BT + c, column bi*BT + r
        const int64_t oi = (int64_t)bj * BT + c, oj = (int64_t)bi * BT + r;
        if (MODE == 2) {
            const double gz = (oi < n && oj < n) ? T[r][c] : 0.0;
            const float h = (float)gz;
            float* tile = K32 + pk_tile(bi >> 1, bj >> 1, (int)ldk) * (2 * 128 * 128);
            tile[(BT + c) * 128 + r] = h;
            tile[128 * 128 + (BT + c) * 128 + r] = (float)(gz - (double)h);
        } else if (oi < n && oj < n) {
            const double g = T[r][c];
            if (PAIR) {
                const float h = (float)g;
                K32[oi * ldk + oj] = h;
                K32lo[oi * ldk + oj] = (float)(g - (double)h);
            } else {
                K64[oi * ldk + oj] = g;
            }
        }
    }
}

__global__ void k_diag(const double* __restrict__ Q, int64_t n, int d, double scale, double lambda,
                       double* __restrict__ diag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < d; ++k) s = fma(Q[i * d + k], Q[i * d + k], s);
    diag[i] = exp(scale * s) + lambda;
}

// Split q * sqrt(scale * log2(e)) into bf16 high and low parts (zero-padded to
// dpad columns).  Folding the scale and log2(e) into the operands lets the
// matrix-free kernels feed the tensor-core logits straight into ex2.
__global__ void k_split_bf16(const double* __restrict__ Q, int64_t n, int d, int dpad, double fold,
                             uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                             float* __restrict__ q32) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * dpad) return;
    const int64_t i = idx / dpad;
    const int k = (int)(idx % dpad);
    const double q = (k < d) ? Q[i * d + k] * fold : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(q);
    const __nv_bfloat16 l = __double2bfloat16(q - (double)__bfloat162float(h));
    hi[idx] = __bfloat16_as_ushort(h);
    lo[idx] = __bfloat16_as_ushort(l);
    if (k < d) q32[i * d + k] = (float)Q[i * d + k];
}

}  // namespace

// Copy the 128 x 128 packed tiles (I, J), I <= J < J0, of an operator over
// fewer blocks into the packed layout of nb blocks: row I's run of tiles is
// contiguous in both layouts.
laker_status copy_packed_tiles(laker_ctx* ctx, const float* src, int nb_src, float* dst, int nb, int J0) {
    const size_t tile = (size_t)2 * 128 * 128 * sizeof(float);
    for (int I = 0; I < J0; ++I) {
        const int64_t a = (int64_t)I * nb_src - (int64_t)I * (I - 1) / 2;
        const int64_t b = (int64_t)I * nb - (int64_t)I * (I - 1) / 2;
        LK_CUDA(ctx, cudaMemcpyAsync((char*)dst + b * tile, (const char*)src + a * tile, (size_t)(J0 - I) * tile,
                                     cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return LAKER_OK;
}

laker_status build_operator(laker_ctx* ctx, laker_op* op, const laker_op* prev) {
    const int64_t n = op->n;
    const int d = op->d;
    op->ldk = (n + 3) / 4 * 4;
    op->dpad = (d + 15) / 16 * 16;
    // prev: the same operator over the first prev->n points; its stored
    // entries are copied and only the tile pairs whose column block reaches
    // the new points are evaluated (the same kernels on the same tiles, so the
    // result equals a fresh build bit for bit)
    const int64_t n0 = prev ? prev->n : 0;
    // FP64: float64 G; FP32: the float32 pair, full (its float32 product
    // streams rows of hi); BF16X3: the pair packed in the upper triangle, read
    // only by the float64-accurate product (the operator is matrix-free)
    const int mode = op->precision == LAKER_FP64 ? 0 : op->precision == LAKER_FP32 ? 1 : 2;
    laker_status st;
    float* Kp = nullptr;
    if (mode == 1) {
        if ((st = lk_malloc(ctx, (void**)&op->K32, (size_t)n * op->ldk * sizeof(float))) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&op->K32lo, (size_t)n * op->ldk * sizeof(float))) != LAKER_OK) return st;
    } else if (mode == 0) {
        if ((st = lk_malloc(ctx, (void**)&op->K64, (size_t)n * op->ldk * sizeof(double))) != LAKER_OK) return st;
    } else {
        if ((st = resid_prepare(ctx, op, &Kp)) != LAKER_OK) return st;
    }
    if ((st = lk_malloc(ctx, (void**)&op->diagA, (size_t)n * sizeof(double))) != LAKER_OK) return st;
    if (op->ldk > n && mode != 2) {
        if (mode == 1) {
            LK_CUDA(ctx, cudaMemset2DAsync(op->K32 + n, op->ldk * sizeof(float), 0, (op->ldk - n) * sizeof(float), n,
                                           ctx->stream));
            LK_CUDA(ctx, cudaMemset2DAsync(op->K32lo + n, op->ldk * sizeof(float), 0, (op->ldk - n) * sizeof(float),
                                           n, ctx->stream));
        } else {
            LK_CUDA(ctx, cudaMemset2DAsync(op->K64 + n, op->ldk * sizeof(double), 0, (op->ldk - n) * sizeof(double), n,
                                           ctx->stream));
        }
    }
    if (prev && mode != 2) {
        if (mode == 1) {
            LK_CUDA(ctx, cudaMemcpy2DAsync(op->K32, op->ldk * sizeof(float), prev->K32, prev->ldk * sizeof(float),
                                           n0 * sizeof(float), n0, cudaMemcpyDeviceToDevice, ctx->stream));
            LK_CUDA(ctx, cudaMemcpy2DAsync(op->K32lo, op->ldk * sizeof(float), prev->K32lo, prev->ldk * sizeof(float),
                                           n0 * sizeof(float), n0, cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            LK_CUDA(ctx, cudaMemcpy2DAsync(op->K64, op->ldk * sizeof(double), prev->K64, prev->ldk * sizeof(double),
                                           n0 * sizeof(double), n0, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    if (mode == 2 && d <= 64) {
        if ((st = resid_build_df(ctx, op, prev)) != LAKER_OK) return st;
    } else if (mode == 2) {
        const int nb128 = (int)((n + 127) / 128);
        const int nt = 2 * nb128;   // 64-blocks, padded so that every packed tile is written
        const int J0 = prev ? (int)(n0 / 128) : 0;   // whole 128-blocks of the previous operator
        if (prev && (st = copy_packed_tiles(ctx, resid_packed(prev), (int)((n0 + 127) / 128), Kp, nb128, J0)) !=
                        LAKER_OK)
            return st;
        const int64_t pairs = lk::upper_pairs(nt, 2 * J0);
        if (pairs > 0)
            k_build_sym<2><<<(unsigned)pairs, 256, 0, ctx->stream>>>(op->Q64, n, d, op->scale, nullptr, Kp, nullptr,
                                                                     nb128, nt, 2 * J0);
    } else {
        const int nt = (int)((n + BT - 1) / BT);
        const int j0 = prev ? (int)(n0 / BT) : 0;   // whole tiles of the previous operator
        const int64_t pairs = lk::upper_pairs(nt, j0);
        if (pairs > 0) {
            if (mode == 1)
                k_build_sym<1><<<(unsigned)pairs, 256, 0, ctx->stream>>>(op->Q64, n, d, op->scale, nullptr, op->K32,
                                                                         op->K32lo, op->ldk, nt, j0);
            else
                k_build_sym<0><<<(unsigned)pairs, 256, 0, ctx->stream>>>(op->Q64, n, d, op->scale, op->K64, nullptr,
                                                                         nullptr, op->ldk, nt, j0);
        }
    }
    if (!(mode == 2 && d <= 64)) LK_LAUNCHED(ctx);
    k_diag<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(op->Q64, n, d, op->scale, op->lambda,
                                                                 op->diagA);
    LK_LAUNCHED(ctx);
    if (op->precision == LAKER_BF16X3 && !(op->scale > 0.0))
        return set_error(ctx, LAKER_ERR_ARG, "BF16X3 operator needs scale > 0");
    // split-bf16 operands: the matrix-free product (BF16X3) and the
    // tensor-core random directions of the fit (FP32 and BF16X3, d <= 64)
    if (op->precision != LAKER_FP64 && op->scale > 0.0 && op->dpad <= 64) {
        const size_t e = (size_t)n * op->dpad;
        if ((st = lk_malloc(ctx, (void**)&op->Qhi, e * 2)) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&op->Qlo, e * 2)) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&op->Q32, (size_t)n * d * sizeof(float))) != LAKER_OK) return st;
        const double fold = std::sqrt(op->scale * 1.4426950408889634);
        k_split_bf16<<<(unsigned)((e + 255) / 256), 256, 0, ctx->stream>>>(op->Q64, n, d, op->dpad, fold,
                                                                           op->Qhi, op->Qlo, op->Q32);
        LK_LAUNCHED(ctx);
        if (op->precision == LAKER_BF16X3 && (st = mf_prepare(ctx, op)) != LAKER_OK) return st;
    }
    return LAKER_OK;
}
