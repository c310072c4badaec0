// Radio-map reconstruction  r(x_m) = sum_i exp(scale <q(x_m), q_i>) alpha_i
// (Sec. III-A, Eq. sc-radio-map-reconstruction; Algorithm 1, reconstruction stage).
//
// Block = 64 query rows x one slice of the training points; logits in float64,
// float64 exp, per-row sums across the 16 column threads by shuffles, slices
// summed afterwards in a fixed order.
#include <algorithm>

#include "laker_device.cuh"

namespace {

constexpr int BT = 64;
constexpr int BD = 32;

__global__ void __launch_bounds__(256)
k_map_fp64(const double* __restrict__ Qg, int64_t m, const double* __restrict__ Q, int64_t n, int d,
           double scale, const double* __restrict__ alpha, int64_t tiles_per_slice, double* __restrict__ part) {
    __shared__ double A[BD][BT + 1];
    __shared__ double B[BD][BT + 1];
    __shared__ double al[BT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t g0 = (int64_t)blockIdx.x * BT;
    const int64_t nt = (n + BT - 1) / BT;
    const int64_t t0 = (int64_t)blockIdx.y * tiles_per_slice, t1 = min(nt, t0 + tiles_per_slice);
    double rows[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t j0 = tile * BT;
        double acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
        for (int k0 = 0; k0 < d; k0 += BD) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < BT * BD; idx += blockDim.x) {
                const int r = idx / BD, k = idx % BD;
                const bool kin = (k0 + k) < d;
                const int64_t gi = g0 + r, gj = j0 + r;
                A[k][r] = (gi < m && kin) ? Qg[gi * d + k0 + k] : 0.0;
                B[k][r] = (gj < n && kin) ? Q[gj * d + k0 + k] : 0.0;
            }
            if (k0 == 0 && threadIdx.x < BT) al[threadIdx.x] = (j0 + threadIdx.x < n) ? alpha[j0 + threadIdx.x] : 0.0;
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < BD; ++k) {
                double a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) { a[u] = A[k][ty + 16 * u]; b[u] = B[k][tx + 16 * u]; }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const double av = al[tx + 16 * v];
                if (av != 0.0) rows[u] = fma(exp(scale * acc[u][v]), av, rows[u]);
            }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        double s = rows[u];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t gi = g0 + ty + 16 * u;
        if (tx == 0 && gi < m) part[(int64_t)blockIdx.y * m + gi] = s;
    }
}

__global__ void k_sum_slices(int64_t m, int ns, const double* __restrict__ part, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int z = 0; z < ns; ++z) s += part[(int64_t)z * m + i];
    out[i] = s;
}

}  // namespace

laker_status eval_map(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m, const double* alpha,
                      double* out) {
    const int64_t n = op->n;
    const int64_t mt = (m + BT - 1) / BT, nt = (n + BT - 1) / BT;
    int64_t slices = std::max<int64_t>(1, std::min<int64_t>(nt, (2 * ctx->num_sms + mt - 1) / mt));
    const int64_t per = (nt + slices - 1) / slices;
    slices = (nt + per - 1) / per;
    double* part = nullptr;
    laker_status st = lk_malloc(ctx, (void**)&part, (size_t)slices * m * sizeof(double));
    if (st != LAKER_OK) return st;
    dim3 grid((unsigned)mt, (unsigned)slices);
    k_map_fp64<<<grid, 256, 0, ctx->stream>>>(Qg, m, op->Q64, n, op->d, op->scale, alpha, per, part);
    LK_LAUNCHED(ctx);
    k_sum_slices<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, (int)slices, part, out);
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(part);
    return LAKER_OK;
}
