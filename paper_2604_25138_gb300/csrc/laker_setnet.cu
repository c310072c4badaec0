// Learned set-to-parameters network (an extension beyond the paper, whose
// only learning is the CCCP fit of Sec. IV-B..D): predicts log c and the
// per-direction log(D_k N_r / n) of Sigma_* = c I + U diag(D) U^T for a new
// measurement set, to replace or start the CCCP fit.
//
//   per point:     h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), h3 = tanh(h2 W3 + b3)
//                  with x = [location / L, q, y]
//   set code:      z = mean over the points of h3
//   log c:         g = tanh(z Wg1 + bg1), log c = g . wg2 + bg2
//   direction k:   e_k = tanh([z, f_k] Wd1 + bd1), log(D_k N_r / n) = e_k . wd2 + bd2,
//                  f_k = [log(|u_k| / n), (1/N_r) sum_j M_kj^2] from the fit's first stage
//                  (every input and target free of the instance size)
//   loss:          (1/B) sum_b [(log c_b - t_b)^2 + (1/K_b) sum_k (log D_bk - T_bk)^2]
//
// Weights are used in bf16 (the rounding of float32 master weights, refreshed
// after every Adam step); activations and sums are float32.  The dense
// layers run through one tiled GEMM kernel with fused bias + tanh or
// tanh-derivative epilogues; every reduction is in a fixed order.
#include <cuda_bf16.h>
#include <string>
#include <cstring>
#include <cstdio>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "laker_device.cuh"

struct laker_setnet {
    laker_ctx* ctx = nullptr;
    int in_dim = 0, H = 0, Hd = 0;
    int64_t np = 0;
    int64_t off[14] = {};            // W1 b1 W2 b2 W3 b3 Wg1 bg1 wg2 bg2 Wd1 bd1 wd2 bd2
    float* theta = nullptr;          // float32 master weights
    __nv_bfloat16* wbf = nullptr;    // bf16 compute copy
    float* m = nullptr;              // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    int step = 0;
    // activations of the last forward pass (grown on demand)
    int64_t cap_p = 0, cap_b = 0, cap_k = 0;
    float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dh = nullptr, *dh2 = nullptr;
    float *z = nullptr, *g = nullptr, *dz = nullptr, *dg = nullptr;
    float *V = nullptr, *E = nullptr, *dV = nullptr, *dE = nullptr;
    float *logc = nullptr, *logD = nullptr, *dlogc = nullptr, *dlogD = nullptr, *loss = nullptr;
    int *poff = nullptr, *koff = nullptr, *pinst = nullptr, *kinst = nullptr;
    const float* X = nullptr;        // point features of the last forward pass (caller's buffer)
    int B = 0;
    int64_t P = 0, K = 0;
};

namespace {

enum { W1 = 0, B1, W2, B2, W3, B3, WG1, BG1, WG2, BG2, WD1, BD1, WD2, BD2 };

constexpr int GT = 64, GK = 16;
enum { EPI_STORE = 0, EPI_TANH = 1, EPI_DTANH = 2, EPI_ADD = 3 };

__device__ __forceinline__ float ldv(const float* p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[M x N] = epi(op(A) op(B)): op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k],
// op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n].  EPI_TANH: tanh(acc + bias[n]);
// EPI_DTANH: acc * (1 - Y[m][n]^2) with Y at C's layout; EPI_ADD: C += acc.
template <bool TA, bool TB, typename BT_, int EPI>
__global__ void __launch_bounds__(256)
k_sn_gemm(int M, int N, int K, const float* __restrict__ A, int lda, const BT_* __restrict__ B, int ldb,
          const BT_* __restrict__ bias, const float* __restrict__ Y, float* __restrict__ C, int ldc) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int idx = tid + r * 256;
            if (!TA) {
                const int ml = idx / GK, kl = idx % GK, m = m0 + ml, k = k0 + kl;
                As[kl][ml] = (m < M && k < K) ? A[(int64_t)m * lda + k] : 0.f;
            } else {
                const int kl = idx / GT, ml = idx % GT, m = m0 + ml, k = k0 + kl;
                As[kl][ml] = (m < M && k < K) ? A[(int64_t)k * lda + m] : 0.f;
            }
            if (!TB) {
                const int kl = idx / GT, nl = idx % GT, n = n0 + nl, k = k0 + kl;
                Bs[kl][nl] = (n < N && k < K) ? ldv(B + (int64_t)k * ldb + n) : 0.f;
            } else {
                const int nl = idx / GK, kl = idx % GK, n = n0 + nl, k = k0 + kl;
                Bs[kl][nl] = (n < N && k < K) ? ldv(B + (int64_t)n * ldb + k) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float* c = C + (int64_t)m * ldc + n;
            if (EPI == EPI_TANH) *c = tanhf(acc[i][j] + ldv(bias + n));
            else if (EPI == EPI_DTANH) { const float y = Y[(int64_t)m * ldc + n]; *c = acc[i][j] * (1.f - y * y); }
            else if (EPI == EPI_ADD) *c += acc[i][j];
            else *c = acc[i][j];
        }
    }
}

// z[b] = mean of h3 over the points of instance b (one block per instance).
__global__ void k_sn_pool(int H, const float* __restrict__ h3, const int* __restrict__ poff, float* __restrict__ z) {
    const int b = blockIdx.x;
    const int p0 = poff[b], p1 = poff[b + 1];
    const float inv = 1.f / (float)max(1, p1 - p0);
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        float s = 0.f;
        for (int i = p0; i < p1; ++i) s += h3[(int64_t)i * H + j];
        z[(int64_t)b * H + j] = s * inv;
    }
}

// V[k] = [z[b(k)], f_k]
__global__ void k_sn_dirin(int64_t K, int H, const float* __restrict__ z, const float* __restrict__ F,
                           const int* __restrict__ kinst, float* __restrict__ V) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * (H + 2)) return;
    const int64_t k = idx / (H + 2);
    const int j = (int)(idx % (H + 2));
    V[idx] = (j < H) ? z[(int64_t)kinst[k] * H + j] : F[k * 2 + (j - H)];
}

// out[r] = X[r] . w + b0 for r < R (one warp per row)
template <typename WT>
__global__ void k_sn_dot(int64_t R, int Hc, const float* __restrict__ X, const WT* __restrict__ w,
                         const WT* __restrict__ b0, float* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    float s = 0.f;
    for (int j = lane; j < Hc; j += 32) s = fmaf(X[r * Hc + j], ldv(w + j), s);
    s = lk::warp_sum(s);
    if (lane == 0) out[r] = s + ldv(b0);
}

// loss and its derivative with respect to the outputs (one block, fixed order)
__global__ void k_sn_loss(int B, const int* __restrict__ koff, const float* __restrict__ logc,
                          const float* __restrict__ tc, const float* __restrict__ logD, const float* __restrict__ tD,
                          float* __restrict__ dlogc, float* __restrict__ dlogD, float* loss) {
    __shared__ double red[32];
    double L = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const int k0 = koff[b], k1 = koff[b + 1];
        const float Kb = (float)max(1, k1 - k0);
        const float ec = logc[b] - tc[b];
        dlogc[b] = 2.f * ec / B;
        double s = 0.0;
        for (int k = k0; k < k1; ++k) {
            const float e = logD[k] - tD[k];
            dlogD[k] = 2.f * e / (Kb * B);
            s += (double)e * e;
        }
        L += ((double)ec * ec + s / Kb) / B;
    }
    L = lk::block_sum(L, red);
    if (threadIdx.x == 0) *loss = (float)L;
}

// dE = dlogD[k] wd2 (1 - E^2);  dG = dlogc[b] wg2 (1 - g^2)
__global__ void k_sn_head_back(int64_t R, int Hc, const float* __restrict__ dout, const __nv_bfloat16* __restrict__ w,
                               const float* __restrict__ Y, float* __restrict__ dY) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * Hc) return;
    const int64_t r = idx / Hc;
    const int j = (int)(idx % Hc);
    const float y = Y[idx];
    dY[idx] = dout[r] * __bfloat162float(w[j]) * (1.f - y * y);
}

// grad_w[j] = sum_r dout[r] X[r][j] (j < Hc), grad_b = sum_r dout[r]; one block.
__global__ void k_sn_head_wgrad(int64_t R, int Hc, const float* __restrict__ dout, const float* __restrict__ X,
                                float* __restrict__ gw, float* __restrict__ gb) {
    for (int j = threadIdx.x; j <= Hc; j += blockDim.x) {
        float s = 0.f;
        for (int64_t r = 0; r < R; ++r) s = fmaf(dout[r], j < Hc ? X[r * Hc + j] : 1.f, s);
        if (j < Hc) gw[j] = s;
        else *gb = s;
    }
}

// column sums of an R x C matrix (bias gradients), fixed order per column
__global__ void k_sn_colsum(int64_t R, int C, const float* __restrict__ X, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int64_t r = 0; r < R; ++r) s += X[r * C + c];
    out[c] = s;
}

// dz[b][j] += sum_{k in b} dV[k][j] (j < H)
__global__ void k_sn_dz_dir(int H, const int* __restrict__ koff, const float* __restrict__ dV, float* __restrict__ dz) {
    const int b = blockIdx.x;
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        float s = 0.f;
        for (int k = koff[b]; k < koff[b + 1]; ++k) s += dV[(int64_t)k * (H + 2) + j];
        dz[(int64_t)b * H + j] += s;
    }
}

// dA3[i] = dz[b(i)] / n_b * (1 - h3^2)
__global__ void k_sn_unpool(int64_t P, int H, const float* __restrict__ dz, const int* __restrict__ pinst,
                            const int* __restrict__ poff, const float* __restrict__ h3, float* __restrict__ da3) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * H) return;
    const int64_t i = idx / H;
    const int j = (int)(idx % H);
    const int b = pinst[i];
    const float y = h3[idx];
    da3[idx] = dz[(int64_t)b * H + j] / (float)(poff[b + 1] - poff[b]) * (1.f - y * y);
}

__global__ void k_sn_adam(int64_t n, float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                          const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2,
                          __nv_bfloat16* __restrict__ wbf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[i] = t;
    wbf[i] = __float2bfloat16_rn(t);
}

__global__ void k_sn_to_bf16(int64_t n, const float* __restrict__ th, __nv_bfloat16* __restrict__ wbf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wbf[i] = __float2bfloat16_rn(th[i]);
}

// point features x_i = [loc_i (2), q_i (d), y_i] as float32
__global__ void k_sn_point_features(int64_t n, int d, const double* __restrict__ loc, const double* __restrict__ Q,
                                    const double* __restrict__ y, float* __restrict__ X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = d + 3;
    if (idx >= n * w) return;
    const int64_t i = idx / w;
    const int j = (int)(idx % w);
    X[idx] = (float)(j < 2 ? loc[i * 2 + j] : (j < 2 + d ? Q[i * d + (j - 2)] : y[i]));
}

unsigned gsz(int64_t c, int b = 256) { return (unsigned)((c + b - 1) / b); }

template <bool TA, bool TB, typename BT_, int EPI>
laker_status sn_gemm(laker_ctx* ctx, int M, int N, int K, const float* A, int lda, const BT_* B, int ldb,
                     const BT_* bias, const float* Y, float* C, int ldc) {
    if (M <= 0 || N <= 0) return LAKER_OK;
    dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT));
    k_sn_gemm<TA, TB, BT_, EPI><<<grid, 256, 0, ctx->stream>>>(M, N, K, A, lda, B, ldb, bias, Y, C, ldc);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

laker_status grow(laker_ctx* ctx, laker_setnet* s, int B, int64_t P, int64_t K) {
    const int H = s->H, Hd = s->Hd;
    laker_status st;
    if (P > s->cap_p) {
        for (float** p : {&s->h1, &s->h2, &s->h3, &s->dh, &s->dh2}) { cudaFree(*p); *p = nullptr; }
        cudaFree(s->pinst);
        s->pinst = nullptr;
        for (float** p : {&s->h1, &s->h2, &s->h3, &s->dh, &s->dh2})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * P * H)) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&s->pinst, sizeof(int) * P)) != LAKER_OK) return st;
        s->cap_p = P;
    }
    if (B > s->cap_b) {
        for (float** p : {&s->z, &s->g, &s->dz, &s->dg}) { cudaFree(*p); *p = nullptr; }
        for (float** p : {&s->logc, &s->dlogc}) { cudaFree(*p); *p = nullptr; }
        cudaFree(s->poff);
        cudaFree(s->koff);
        for (float** p : {&s->z, &s->g, &s->dz, &s->dg})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * B * H)) != LAKER_OK) return st;
        for (float** p : {&s->logc, &s->dlogc})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * B)) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&s->poff, sizeof(int) * (B + 1))) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&s->koff, sizeof(int) * (B + 1))) != LAKER_OK) return st;
        s->cap_b = B;
    }
    if (K > s->cap_k) {
        for (float** p : {&s->V, &s->dV}) { cudaFree(*p); *p = nullptr; }
        for (float** p : {&s->E, &s->dE}) { cudaFree(*p); *p = nullptr; }
        for (float** p : {&s->logD, &s->dlogD}) { cudaFree(*p); *p = nullptr; }
        cudaFree(s->kinst);
        for (float** p : {&s->V, &s->dV})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * K * (H + 2))) != LAKER_OK) return st;
        for (float** p : {&s->E, &s->dE})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * K * Hd)) != LAKER_OK) return st;
        for (float** p : {&s->logD, &s->dlogD})
            if ((st = lk_malloc(ctx, (void**)p, sizeof(float) * K)) != LAKER_OK) return st;
        if ((st = lk_malloc(ctx, (void**)&s->kinst, sizeof(int) * K)) != LAKER_OK) return st;
        s->cap_k = K;
    }
    if (!s->loss && (st = lk_malloc(ctx, (void**)&s->loss, sizeof(float))) != LAKER_OK) return st;
    return LAKER_OK;
}

}  // namespace

// ---- internal entry points --------------------------------------------------

laker_status setnet_create(laker_ctx* ctx, int in_dim, int H, int Hd, uint64_t seed, laker_setnet** out) {
    laker_setnet* s = new laker_setnet();
    s->ctx = ctx;
    s->in_dim = in_dim;
    s->H = H;
    s->Hd = Hd;
    const int64_t sizes[14] = {(int64_t)in_dim * H, H, (int64_t)H * H, H, (int64_t)H * H, H, (int64_t)H * H, H,
                               H, 1, (int64_t)(H + 2) * Hd, Hd, Hd, 1};
    int64_t o = 0;
    for (int i = 0; i < 14; ++i) { s->off[i] = o; o += sizes[i]; }
    s->np = o;
    // Glorot-uniform weights, zero biases (seeded, host side)
    std::vector<float> th((size_t)o, 0.f);
    std::mt19937_64 rng(seed);
    auto init = [&](int idx, int fan_in, int fan_out) {
        const float a = std::sqrt(6.f / (float)(fan_in + fan_out));
        std::uniform_real_distribution<float> U(-a, a);
        for (int64_t i = 0; i < sizes[idx]; ++i) th[(size_t)(s->off[idx] + i)] = U(rng);
    };
    init(W1, in_dim, H);
    init(W2, H, H);
    init(W3, H, H);
    init(WG1, H, H);
    init(WG2, H, 1);
    init(WD1, H + 2, Hd);
    init(WD2, Hd, 1);
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&s->theta, sizeof(float) * o)) != LAKER_OK) { delete s; return st; }
    if ((st = lk_malloc(ctx, (void**)&s->wbf, sizeof(__nv_bfloat16) * o)) != LAKER_OK) { delete s; return st; }
    if ((st = lk_malloc(ctx, (void**)&s->m, sizeof(float) * o)) != LAKER_OK) { delete s; return st; }
    if ((st = lk_malloc(ctx, (void**)&s->v, sizeof(float) * o)) != LAKER_OK) { delete s; return st; }
    if ((st = lk_malloc(ctx, (void**)&s->grad, sizeof(float) * o)) != LAKER_OK) { delete s; return st; }
    LK_CUDA(ctx, cudaMemcpyAsync(s->theta, th.data(), sizeof(float) * o, cudaMemcpyHostToDevice, ctx->stream));
    LK_CUDA(ctx, cudaMemsetAsync(s->m, 0, sizeof(float) * o, ctx->stream));
    LK_CUDA(ctx, cudaMemsetAsync(s->v, 0, sizeof(float) * o, ctx->stream));
    k_sn_to_bf16<<<gsz(o), 256, 0, ctx->stream>>>(o, s->theta, s->wbf);
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *out = s;
    return LAKER_OK;
}

void setnet_destroy(laker_setnet* s) {
    if (!s) return;
    for (void* p : {(void*)s->theta, (void*)s->wbf, (void*)s->m, (void*)s->v, (void*)s->grad, (void*)s->h1,
                    (void*)s->h2, (void*)s->h3, (void*)s->dh, (void*)s->dh2, (void*)s->z, (void*)s->g, (void*)s->dz,
                    (void*)s->dg, (void*)s->V, (void*)s->E, (void*)s->dV, (void*)s->dE, (void*)s->logc,
                    (void*)s->logD, (void*)s->dlogc, (void*)s->dlogD, (void*)s->loss, (void*)s->poff,
                    (void*)s->koff, (void*)s->pinst, (void*)s->kinst})
        cudaFree(p);
    delete s;
}

laker_status setnet_set_params(laker_ctx* ctx, laker_setnet* s, const float* host) {
    LK_CUDA(ctx, cudaMemcpyAsync(s->theta, host, sizeof(float) * s->np, cudaMemcpyHostToDevice, ctx->stream));
    k_sn_to_bf16<<<gsz(s->np), 256, 0, ctx->stream>>>(s->np, s->theta, s->wbf);
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaMemsetAsync(s->m, 0, sizeof(float) * s->np, ctx->stream));
    LK_CUDA(ctx, cudaMemsetAsync(s->v, 0, sizeof(float) * s->np, ctx->stream));
    s->step = 0;
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

laker_status setnet_get_params(laker_ctx* ctx, const laker_setnet* s, float* host) {
    LK_CUDA(ctx, cudaMemcpyAsync(host, s->theta, sizeof(float) * s->np, cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

laker_status setnet_point_features(laker_ctx* ctx, int64_t n, int d, const double* loc, const double* Q,
                                   const double* y, float* X) {
    k_sn_point_features<<<gsz(n * (d + 3)), 256, 0, ctx->stream>>>(n, d, loc, Q, y, X);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

// Forward pass over a batch: B instances, points X (P x in_dim, instance b owns
// rows poff[b]..poff[b+1]), directions F (K x 2, rows koff[b]..koff[b+1]).
// Outputs stay in the network's buffers (s->logc, s->logD).
laker_status setnet_forward(laker_ctx* ctx, laker_setnet* s, int B, const float* X, const int* poff_h,
                            const float* F, const int* koff_h) {
    const int64_t P = poff_h[B], K = koff_h[B];
    laker_status st;
    if ((st = grow(ctx, s, B, P, K)) != LAKER_OK) return st;
    s->B = B;
    s->P = P;
    s->K = K;
    s->X = X;
    std::vector<int> pinst((size_t)P), kinst((size_t)std::max<int64_t>(1, K));
    for (int b = 0; b < B; ++b) {
        for (int i = poff_h[b]; i < poff_h[b + 1]; ++i) pinst[(size_t)i] = b;
        for (int k = koff_h[b]; k < koff_h[b + 1]; ++k) kinst[(size_t)k] = b;
    }
    cudaStream_t st_ = ctx->stream;
    LK_CUDA(ctx, cudaMemcpyAsync(s->poff, poff_h, sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st_));
    LK_CUDA(ctx, cudaMemcpyAsync(s->koff, koff_h, sizeof(int) * (B + 1), cudaMemcpyHostToDevice, st_));
    LK_CUDA(ctx, cudaMemcpyAsync(s->pinst, pinst.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st_));
    if (K > 0) LK_CUDA(ctx, cudaMemcpyAsync(s->kinst, kinst.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st_));
    const int H = s->H, Hd = s->Hd, D0 = s->in_dim;
    const __nv_bfloat16* w = s->wbf;
    if ((st = sn_gemm<false, false, __nv_bfloat16, EPI_TANH>(ctx, (int)P, H, D0, X, D0, w + s->off[W1], H,
                                                            w + s->off[B1], nullptr, s->h1, H)) != LAKER_OK) return st;
    if ((st = sn_gemm<false, false, __nv_bfloat16, EPI_TANH>(ctx, (int)P, H, H, s->h1, H, w + s->off[W2], H,
                                                            w + s->off[B2], nullptr, s->h2, H)) != LAKER_OK) return st;
    if ((st = sn_gemm<false, false, __nv_bfloat16, EPI_TANH>(ctx, (int)P, H, H, s->h2, H, w + s->off[W3], H,
                                                            w + s->off[B3], nullptr, s->h3, H)) != LAKER_OK) return st;
    k_sn_pool<<<B, 256, 0, st_>>>(H, s->h3, s->poff, s->z);
    LK_LAUNCHED(ctx);
    if ((st = sn_gemm<false, false, __nv_bfloat16, EPI_TANH>(ctx, B, H, H, s->z, H, w + s->off[WG1], H,
                                                            w + s->off[BG1], nullptr, s->g, H)) != LAKER_OK) return st;
    k_sn_dot<__nv_bfloat16><<<gsz(B, 8), 256, 0, st_>>>(B, H, s->g, w + s->off[WG2], w + s->off[BG2], s->logc);
    LK_LAUNCHED(ctx);
    if (K > 0) {
        k_sn_dirin<<<gsz(K * (H + 2)), 256, 0, st_>>>(K, H, s->z, F, s->kinst, s->V);
        LK_LAUNCHED(ctx);
        if ((st = sn_gemm<false, false, __nv_bfloat16, EPI_TANH>(ctx, (int)K, Hd, H + 2, s->V, H + 2,
                                                                w + s->off[WD1], Hd, w + s->off[BD1], nullptr, s->E,
                                                                Hd)) != LAKER_OK)
            return st;
        k_sn_dot<__nv_bfloat16><<<gsz(K, 8), 256, 0, st_>>>(K, Hd, s->E, w + s->off[WD2], w + s->off[BD2], s->logD);
        LK_LAUNCHED(ctx);
    }
    return LAKER_OK;
}

// Loss against targets (tc: B, tD: K) and the gradient of the loss with
// respect to the float32 parameters (evaluated at the bf16 weights) into
// s->grad; *loss_h receives the loss.  Requires setnet_forward on the batch.
laker_status setnet_backward(laker_ctx* ctx, laker_setnet* s, const float* tc, const float* tD, float* loss_h) {
    const int B = s->B, H = s->H, Hd = s->Hd, D0 = s->in_dim;
    const int64_t P = s->P, K = s->K;
    const __nv_bfloat16* w = s->wbf;
    float* gr = s->grad;
    cudaStream_t st_ = ctx->stream;
    laker_status st;
    k_sn_loss<<<1, 256, 0, st_>>>(B, s->koff, s->logc, tc, s->logD, tD, s->dlogc, s->dlogD, s->loss);
    LK_LAUNCHED(ctx);
    // direction head
    LK_CUDA(ctx, cudaMemsetAsync(s->dz, 0, sizeof(float) * B * H, st_));
    if (K > 0) {
        k_sn_head_wgrad<<<1, 256, 0, st_>>>(K, Hd, s->dlogD, s->E, gr + s->off[WD2], gr + s->off[BD2]);
        LK_LAUNCHED(ctx);
        k_sn_head_back<<<gsz(K * Hd), 256, 0, st_>>>(K, Hd, s->dlogD, w + s->off[WD2], s->E, s->dE);
        LK_LAUNCHED(ctx);
        if ((st = sn_gemm<true, false, float, EPI_STORE>(ctx, H + 2, Hd, (int)K, s->V, H + 2, s->dE, Hd, nullptr,
                                                         nullptr, gr + s->off[WD1], Hd)) != LAKER_OK)
            return st;
        k_sn_colsum<<<gsz(Hd), 256, 0, st_>>>(K, Hd, s->dE, gr + s->off[BD1]);
        LK_LAUNCHED(ctx);
        if ((st = sn_gemm<false, true, __nv_bfloat16, EPI_STORE>(ctx, (int)K, H + 2, Hd, s->dE, Hd, w + s->off[WD1],
                                                                 Hd, nullptr, nullptr, s->dV, H + 2)) != LAKER_OK)
            return st;
        k_sn_dz_dir<<<B, 256, 0, st_>>>(H, s->koff, s->dV, s->dz);
        LK_LAUNCHED(ctx);
    } else {
        LK_CUDA(ctx, cudaMemsetAsync(gr + s->off[WD1], 0, sizeof(float) * (s->off[BD2] + 1 - s->off[WD1]), st_));
    }
    // log c head
    k_sn_head_wgrad<<<1, 256, 0, st_>>>(B, H, s->dlogc, s->g, gr + s->off[WG2], gr + s->off[BG2]);
    LK_LAUNCHED(ctx);
    k_sn_head_back<<<gsz((int64_t)B * H), 256, 0, st_>>>(B, H, s->dlogc, w + s->off[WG2], s->g, s->dg);
    LK_LAUNCHED(ctx);
    if ((st = sn_gemm<true, false, float, EPI_STORE>(ctx, H, H, B, s->z, H, s->dg, H, nullptr, nullptr,
                                                     gr + s->off[WG1], H)) != LAKER_OK)
        return st;
    k_sn_colsum<<<gsz(H), 256, 0, st_>>>(B, H, s->dg, gr + s->off[BG1]);
    LK_LAUNCHED(ctx);
    if ((st = sn_gemm<false, true, __nv_bfloat16, EPI_ADD>(ctx, B, H, H, s->dg, H, w + s->off[WG1], H, nullptr,
                                                          nullptr, s->dz, H)) != LAKER_OK)
        return st;
    // pooling and the point MLP
    k_sn_unpool<<<gsz(P * H), 256, 0, st_>>>(P, H, s->dz, s->pinst, s->poff, s->h3, s->dh);
    LK_LAUNCHED(ctx);
    float* dA = s->dh;     // dA3
    float* dB = s->dh2;
    if ((st = sn_gemm<true, false, float, EPI_STORE>(ctx, H, H, (int)P, s->h2, H, dA, H, nullptr, nullptr,
                                                     gr + s->off[W3], H)) != LAKER_OK)
        return st;
    k_sn_colsum<<<gsz(H), 256, 0, st_>>>(P, H, dA, gr + s->off[B3]);
    LK_LAUNCHED(ctx);
    if ((st = sn_gemm<false, true, __nv_bfloat16, EPI_DTANH>(ctx, (int)P, H, H, dA, H, w + s->off[W3], H, nullptr,
                                                            s->h2, dB, H)) != LAKER_OK)
        return st;   // dA2
    if ((st = sn_gemm<true, false, float, EPI_STORE>(ctx, H, H, (int)P, s->h1, H, dB, H, nullptr, nullptr,
                                                     gr + s->off[W2], H)) != LAKER_OK)
        return st;
    k_sn_colsum<<<gsz(H), 256, 0, st_>>>(P, H, dB, gr + s->off[B2]);
    LK_LAUNCHED(ctx);
    if ((st = sn_gemm<false, true, __nv_bfloat16, EPI_DTANH>(ctx, (int)P, H, H, dB, H, w + s->off[W2], H, nullptr,
                                                            s->h1, dA, H)) != LAKER_OK)
        return st;   // dA1
    if ((st = sn_gemm<true, false, float, EPI_STORE>(ctx, D0, H, (int)P, s->X, D0, dA, H, nullptr, nullptr,
                                                     gr + s->off[W1], H)) != LAKER_OK)
        return st;
    k_sn_colsum<<<gsz(H), 256, 0, st_>>>(P, H, dA, gr + s->off[B1]);
    LK_LAUNCHED(ctx);
    if (loss_h) {
        LK_CUDA(ctx, cudaMemcpyAsync(loss_h, s->loss, sizeof(float), cudaMemcpyDeviceToHost, st_));
        LK_CUDA(ctx, cudaStreamSynchronize(st_));
    }
    return LAKER_OK;
}

laker_status setnet_adam(laker_ctx* ctx, laker_setnet* s, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    s->step += 1;
    const float c1 = 1.f - std::pow(b1, (float)s->step), c2 = 1.f - std::pow(b2, (float)s->step);
    k_sn_adam<<<gsz(s->np), 256, 0, ctx->stream>>>(s->np, s->theta, s->m, s->v, s->grad, lr, b1, b2, eps, c1, c2,
                                                   s->wbf);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

// Prediction for one instance of n points and nr directions: device pointers
// to log c (1) and log D (nr) in the network's buffers.
laker_status setnet_predict(laker_ctx* ctx, laker_setnet* s, int64_t n, const float* X, int nr, const float* F,
                            const float** logc, const float** logD) {
    const int poff[2] = {0, (int)n}, koff[2] = {0, nr};
    laker_status st = setnet_forward(ctx, s, 1, X, poff, F, koff);
    if (st != LAKER_OK) return st;
    *logc = s->logc;
    *logD = s->logD;
    return LAKER_OK;
}

// ---- C ABI -------------------------------------------------------------------

static laker_status sn_check_batch(laker_ctx* ctx, const laker_setnet* s, int B, const float* X, const int* poff,
                                   const float* F, const int* koff) {
    if (!s || !X || !poff || !koff || B < 1) return set_error(ctx, LAKER_ERR_ARG, "set network: bad batch");
    if (poff[0] != 0 || koff[0] != 0) return set_error(ctx, LAKER_ERR_ARG, "set network: offsets start at 0");
    for (int b = 0; b < B; ++b)
        if (poff[b + 1] <= poff[b] || koff[b + 1] < koff[b])
            return set_error(ctx, LAKER_ERR_ARG, "set network: every instance needs points");
    if (koff[B] > 0 && !F) return set_error(ctx, LAKER_ERR_ARG, "set network: null direction features");
    return LAKER_OK;
}

extern "C" {

laker_status laker_setnet_create(laker_ctx* ctx, int in_dim, int hidden, int dir_hidden, uint64_t seed,
                                 laker_setnet** net) {
    if (!ctx || !net) return LAKER_ERR_ARG;
    if (in_dim < 1 || hidden < 1 || dir_hidden < 1) return set_error(ctx, LAKER_ERR_ARG, "set network: bad sizes");
    return setnet_create(ctx, in_dim, hidden, dir_hidden, seed, net);
}

laker_status laker_setnet_destroy(laker_setnet* net) {
    setnet_destroy(net);
    return LAKER_OK;
}

int64_t laker_setnet_num_params(const laker_setnet* net) { return net ? net->np : 0; }

laker_status laker_setnet_get_params(laker_ctx* ctx, const laker_setnet* net, float* host) {
    if (!ctx || !net || !host) return LAKER_ERR_ARG;
    return setnet_get_params(ctx, net, host);
}

laker_status laker_setnet_set_params(laker_ctx* ctx, laker_setnet* net, const float* host) {
    if (!ctx || !net || !host) return LAKER_ERR_ARG;
    return setnet_set_params(ctx, net, host);
}

laker_status laker_setnet_point_features(laker_ctx* ctx, int64_t n, int d, const double* loc, const double* Q,
                                         const double* y, float* X) {
    if (!ctx || !loc || !Q || !y || !X || n < 1 || d < 1) return ctx ? set_error(ctx, LAKER_ERR_ARG, "bad features") : LAKER_ERR_ARG;
    return setnet_point_features(ctx, n, d, loc, Q, y, X);
}

laker_status laker_setnet_forward(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                  const float* F, const int* koff, float* logc, float* logD) {
    if (!ctx) return LAKER_ERR_ARG;
    laker_status st = sn_check_batch(ctx, net, B, X, poff, F, koff);
    if (st != LAKER_OK) return st;
    if ((st = setnet_forward(ctx, net, B, X, poff, F, koff)) != LAKER_OK) return st;
    if (logc) LK_CUDA(ctx, cudaMemcpyAsync(logc, net->logc, sizeof(float) * B, cudaMemcpyDeviceToDevice, ctx->stream));
    if (logD && koff[B] > 0)
        LK_CUDA(ctx, cudaMemcpyAsync(logD, net->logD, sizeof(float) * koff[B], cudaMemcpyDeviceToDevice, ctx->stream));
    return LAKER_OK;
}

laker_status laker_setnet_gradient(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                   const float* F, const int* koff, const float* tc, const float* tD, float* grad,
                                   float* loss) {
    if (!ctx || !tc || (koff && koff[B] > 0 && !tD)) return ctx ? set_error(ctx, LAKER_ERR_ARG, "null targets") : LAKER_ERR_ARG;
    laker_status st = sn_check_batch(ctx, net, B, X, poff, F, koff);
    if (st != LAKER_OK) return st;
    if ((st = setnet_forward(ctx, net, B, X, poff, F, koff)) != LAKER_OK) return st;
    if ((st = setnet_backward(ctx, net, tc, tD, loss)) != LAKER_OK) return st;
    if (grad) LK_CUDA(ctx, cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->np, cudaMemcpyDeviceToDevice, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

laker_status laker_setnet_train_step(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                     const float* F, const int* koff, const float* tc, const float* tD, float lr,
                                     float* loss) {
    if (!ctx || !tc || (koff && koff[B] > 0 && !tD)) return ctx ? set_error(ctx, LAKER_ERR_ARG, "null targets") : LAKER_ERR_ARG;
    if (!(lr > 0.f)) return set_error(ctx, LAKER_ERR_ARG, "set network: learning rate must be > 0");
    laker_status st = sn_check_batch(ctx, net, B, X, poff, F, koff);
    if (st != LAKER_OK) return st;
    if ((st = setnet_forward(ctx, net, B, X, poff, F, koff)) != LAKER_OK) return st;
    if ((st = setnet_backward(ctx, net, tc, tD, loss)) != LAKER_OK) return st;
    return setnet_adam(ctx, net, lr);
}

// Checkpoint file: 8-byte magic "LAKERSN1", int32 in_dim, hidden,
// dir_hidden, Adam step, int64 parameter count, then float32 weights, Adam
// first and second moments (parameter count each), little-endian as written
// by the host.
static const char kSnMagic[8] = {'L', 'A', 'K', 'E', 'R', 'S', 'N', '1'};

laker_status laker_setnet_save(laker_ctx* ctx, const laker_setnet* net, const char* path) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!net || !path) return set_error(ctx, LAKER_ERR_ARG, "set network save: null argument");
    std::vector<float> buf((size_t)3 * net->np);
    LK_CUDA(ctx, cudaMemcpyAsync(buf.data(), net->theta, sizeof(float) * net->np, cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaMemcpyAsync(buf.data() + net->np, net->m, sizeof(float) * net->np, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    LK_CUDA(ctx, cudaMemcpyAsync(buf.data() + 2 * net->np, net->v, sizeof(float) * net->np, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(ctx, LAKER_ERR_ARG, std::string("set network save: cannot open ") + path);
    const int32_t hdr[4] = {net->in_dim, net->H, net->Hd, net->step};
    const int64_t np = net->np;
    bool ok = std::fwrite(kSnMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(&np, sizeof(np), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LAKER_OK : set_error(ctx, LAKER_ERR_ARG, std::string("set network save: write failed: ") + path);
}

laker_status laker_setnet_load(laker_ctx* ctx, const char* path, laker_setnet** net) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!net || !path) return set_error(ctx, LAKER_ERR_ARG, "set network load: null argument");
    *net = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(ctx, LAKER_ERR_ARG, std::string("set network load: cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    int64_t np = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kSnMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && std::fread(&np, sizeof(np), 1, f) == 1 &&
              hdr[0] >= 1 && hdr[1] >= 1 && hdr[2] >= 1 && hdr[3] >= 0 && np >= 1;
    std::vector<float> buf;
    if (ok) {
        buf.resize((size_t)3 * np);
        ok = std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    }
    std::fclose(f);
    if (!ok) return set_error(ctx, LAKER_ERR_ARG, std::string("set network load: not a set-network checkpoint: ") + path);
    laker_setnet* s = nullptr;
    laker_status st = setnet_create(ctx, hdr[0], hdr[1], hdr[2], 0, &s);
    if (st != LAKER_OK) return st;
    if (s->np != np) {
        setnet_destroy(s);
        return set_error(ctx, LAKER_ERR_ARG, "set network load: parameter count does not match the sizes");
    }
    cudaError_t e = cudaMemcpyAsync(s->theta, buf.data(), sizeof(float) * np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->m, buf.data() + np, sizeof(float) * np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->v, buf.data() + 2 * np, sizeof(float) * np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        k_sn_to_bf16<<<gsz(np), 256, 0, ctx->stream>>>(np, s->theta, s->wbf);
        ctx->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        setnet_destroy(s);
        return set_error(ctx, LAKER_ERR_CUDA, std::string("set network load: ") + cudaGetErrorString(e));
    }
    s->step = hdr[3];
    *net = s;
    return LAKER_OK;
}

}  // extern "C"

int setnet_in_dim(const laker_setnet* s) { return s->in_dim; }
