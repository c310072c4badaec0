// Radio-map reconstruction  r(x_m) = sum_i exp(scale <q(x_m), q_i>) alpha_i
// (Sec. III-A, Eq. sc-radio-map-reconstruction; Algorithm 1, reconstruction stage).
//
// This file holds the float64 kernel (float64 operators) and the double-float
// kernel (mixed operators whose logits exceed the tensor-core form's bound, see
// laker_map_tc.cu), and the dispatch between the methods.  Float64 kernel:
// block = 64 query rows x one slice of the training points; logits in float64,
// float64 exp, per-row sums across the 16 column threads by shuffles, slices
// summed afterwards in a fixed order.
#include <algorithm>
#include <mutex>

#include "laker_device.cuh"
#include "laker_df.cuh"

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

// ---------------------------------------------------------------------------
// Double-float variant (float32 pipes): every kernel value exp(s <qg, q>) is
// accurate to ~1e-14 relative.  The map sums alpha_i G(x, x_i) with |alpha| up to
// ~|y| / lambda, so per-entry errors of float32 size (~1e-7) would reach tenths
// of a dB; double-float keeps them far below 0.01 dB.
// Thread = one query row (its embedding, pre-scaled by s, in registers);
// block = 128 rows x one slice of training points staged 32 at a time.
// ---------------------------------------------------------------------------
constexpr int DF_ROWS = 128;
constexpr int DF_TILE = 32;

template <int DM>
__global__ void __launch_bounds__(DF_ROWS)
k_map_df(const float2* __restrict__ Qg_df, int64_t m, const float2* __restrict__ Q_df, int64_t n, int d,
         const float2* __restrict__ alpha_df, int64_t tiles_per_slice, double* __restrict__ part) {
    __shared__ float2 qs[DF_TILE][DM];
    __shared__ float2 as[DF_TILE];
    __shared__ float e2tab[128];
    lk::df_exp_table_init(e2tab);   // ordered before its first use by the tile loop's barriers
    const int64_t row = (int64_t)blockIdx.x * DF_ROWS + threadIdx.x;
    lk::df2 g[DM];
#pragma unroll
    for (int t = 0; t < DM; ++t) {
        float2 v = make_float2(0.f, 0.f);
        if (row < m && t < d) v = Qg_df[row * d + t];
        g[t] = {v.x, v.y};
    }
    lk::df2 acc{0.f, 0.f};
    const int64_t nt = (n + DF_TILE - 1) / DF_TILE;
    const int64_t t0 = (int64_t)blockIdx.y * tiles_per_slice, t1 = min(nt, t0 + tiles_per_slice);
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t j0 = tile * DF_TILE;
        __syncthreads();
        for (int idx = threadIdx.x; idx < DF_TILE * DM; idx += DF_ROWS) {
            const int r = idx / DM, t = idx % DM;
            const int64_t j = j0 + r;
            qs[r][t] = (j < n && t < d) ? Q_df[j * d + t] : make_float2(0.f, 0.f);
        }
        if (threadIdx.x < DF_TILE) {
            const int64_t j = j0 + threadIdx.x;
            as[threadIdx.x] = (j < n) ? alpha_df[j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int jmax = (n - j0 < DF_TILE) ? (int)(n - j0) : DF_TILE;
        for (int r = 0; r < jmax; ++r) {
            lk::Dot2 dot;
#pragma unroll
            for (int t = 0; t < DM; ++t) {
                if (t < d) {
                    const float2 q = qs[r][t];
                    dot.add(g[t], lk::df2{q.x, q.y});
                }
            }
            const lk::df2 e = lk::df_exp(dot.value(), e2tab);
            const float2 a = as[r];
            acc = lk::df_add(acc, lk::df_mul(e, lk::df2{a.x, a.y}));
        }
    }
    if (row < m) part[(int64_t)blockIdx.y * m + row] = lk::df_to(acc);
}

// x (float64, count) -> double-float pairs of scale * x
__global__ void k_to_df(int64_t count, const double* __restrict__ x, double scale, float2* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const lk::df2 v = lk::df_from(x[i] * scale);
    y[i] = make_float2(v.hi, v.lo);
}

}  // namespace

static laker_status eval_map_df(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m, const double* alpha,
                                double* out) {
    const int64_t n = op->n;
    const int d = op->d;
    float2 *qg = nullptr, *q = nullptr, *a = nullptr;
    double* part = nullptr;
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&qg, (size_t)m * d * sizeof(float2))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&q, (size_t)n * d * sizeof(float2))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&a, (size_t)n * sizeof(float2))) != LAKER_OK) return st;
    k_to_df<<<(unsigned)((m * d + 255) / 256), 256, 0, ctx->stream>>>(m * d, Qg, op->scale, qg);
    LK_LAUNCHED(ctx);
    k_to_df<<<(unsigned)((n * d + 255) / 256), 256, 0, ctx->stream>>>(n * d, op->Q64, 1.0, q);
    LK_LAUNCHED(ctx);
    k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, alpha, 1.0, a);
    LK_LAUNCHED(ctx);
    const int64_t mt = (m + DF_ROWS - 1) / DF_ROWS, nt = (n + DF_TILE - 1) / DF_TILE;
    int64_t slices = std::max<int64_t>(1, std::min<int64_t>(nt, (4 * ctx->num_sms + mt - 1) / mt));
    const int64_t per = (nt + slices - 1) / slices;
    slices = (nt + per - 1) / per;
    if ((st = lk_malloc(ctx, (void**)&part, (size_t)slices * m * sizeof(double))) != LAKER_OK) return st;
    dim3 grid((unsigned)mt, (unsigned)slices);
    if (d <= 16) k_map_df<16><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
    else if (d <= 32) k_map_df<32><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
    else if (d <= 64) k_map_df<64><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
    else return set_error(ctx, LAKER_ERR_UNSUPPORTED, "double-float map supports d <= 64");
    LK_LAUNCHED(ctx);
    k_sum_slices<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, (int)slices, part, out);
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(qg);
    cudaFree(q);
    cudaFree(a);
    cudaFree(part);
    return LAKER_OK;
}

laker_status eval_map(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m, const double* alpha,
                      double* out, int method) {
    if (method == LAKER_MAP_TENSOR || (method == LAKER_MAP_AUTO && op->precision != LAKER_FP64)) {
        bool applied = false;
        const laker_status st = eval_map_tc(ctx, op, Qg, m, alpha, out, &applied);
        if (st != LAKER_OK || applied) return st;
        if (method == LAKER_MAP_TENSOR)
            return set_error(ctx, LAKER_ERR_UNSUPPORTED, "tensor-core map: d > 64 or scale max|qg| max|q| > 1/2");
    }
    if (op->precision != LAKER_FP64) return eval_map_df(ctx, op, Qg, m, alpha, out);
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

// ---------------------------------------------------------------------------
// Radio map without device allocation.
//
// Some callers cannot call cudaMalloc: services whose device memory is owned
// and fully pre-reserved by another allocator (a framework's caching
// allocator, a fixed-budget real-time process), or loops that must not
// synchronise the device, which cudaMalloc and cudaFree do.  This variant
// launches the same map kernels as the double-float / float64 method of
// laker_eval_map_method but takes its scratch (the
// double-float copies of the inputs and the per-slice partial sums) from the
// static device array below instead of allocating it.
//
// * The array is LAKER_MAP_SCRATCH_BYTES (32 MiB) per device, resident on every
//   GPU that loads this library until the process exits.
// * Host code cannot use the array's name as a device address; its address is
//   looked up once per device with cudaGetSymbolAddress, with that device
//   current, on the first call for that device.  Make that first call before
//   any stream capture.
// * Every call on a device shares the array and leaves its contents behind.
//   Each kernel writes every scratch element it later reads, so nothing has
//   to start at zero.  Calls whose work overlaps on the GPU (other streams,
//   other threads) race on the array: serialise them.
// ---------------------------------------------------------------------------
#define LAKER_MAP_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_map_scratch[LAKER_MAP_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;   // first calls on a device from several host threads
}  // namespace

static laker_status noalloc_setup(laker_ctx* ctx, void** scratch) {
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return set_error(ctx, LAKER_ERR_ARG, "device index out of range for the static scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_ptr[ctx->device] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_map_scratch);
        if (e != cudaSuccess)
            return set_error(ctx, LAKER_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[ctx->device] = p;
    }
    *scratch = g_scratch_ptr[ctx->device];
    return LAKER_OK;
}

extern "C" laker_status laker_eval_map_noalloc(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                                               const double* alpha, double* out) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!op || !Qg || !alpha || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (m < 1) return set_error(ctx, LAKER_ERR_ARG, "need m >= 1");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = op->n;
    const int d = op->d;
    const bool df = op->precision != LAKER_FP64;
    if (df && d > 64) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "double-float map supports d <= 64");
    // fixed part of the scratch: double-float copies of Qg, Q and alpha
    const size_t fixed = df ? ((size_t)m * d + (size_t)n * d + (size_t)n) * sizeof(float2) : 0;
    const size_t fixed_al = (fixed + 255) / 256 * 256;
    if (fixed_al + (size_t)m * sizeof(double) > LAKER_MAP_SCRATCH_BYTES)
        return set_error(ctx, LAKER_ERR_ARG,
                         "laker_eval_map_noalloc: " + std::to_string(fixed_al + (size_t)m * sizeof(double)) +
                             " bytes of scratch needed, the static scratch holds " +
                             std::to_string(LAKER_MAP_SCRATCH_BYTES) + "; use laker_eval_map");
    void* base = nullptr;
    laker_status st = noalloc_setup(ctx, &base);
    if (st != LAKER_OK) return st;
    unsigned char* sb = static_cast<unsigned char*>(base);
    const int64_t rows = df ? DF_ROWS : BT;
    const int64_t tile = df ? DF_TILE : BT;
    const int64_t mt = (m + rows - 1) / rows, nt = (n + tile - 1) / tile;
    const int64_t want = df ? 4 * ctx->num_sms : 2 * ctx->num_sms;
    int64_t slices = std::max<int64_t>(1, std::min<int64_t>(nt, (want + mt - 1) / mt));
    const int64_t fit = (int64_t)((LAKER_MAP_SCRATCH_BYTES - fixed_al) / ((size_t)m * sizeof(double)));
    slices = std::min(slices, fit);
    const int64_t per = (nt + slices - 1) / slices;
    slices = (nt + per - 1) / per;
    double* part = reinterpret_cast<double*>(sb + fixed_al);
    dim3 grid((unsigned)mt, (unsigned)slices);
    if (df) {
        float2* qg = reinterpret_cast<float2*>(sb);
        float2* q = qg + (size_t)m * d;
        float2* a = q + (size_t)n * d;
        k_to_df<<<(unsigned)((m * d + 255) / 256), 256, 0, ctx->stream>>>(m * d, Qg, op->scale, qg);
        LK_LAUNCHED(ctx);
        k_to_df<<<(unsigned)((n * d + 255) / 256), 256, 0, ctx->stream>>>(n * d, op->Q64, 1.0, q);
        LK_LAUNCHED(ctx);
        k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, alpha, 1.0, a);
        LK_LAUNCHED(ctx);
        if (d <= 16) k_map_df<16><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
        else if (d <= 32) k_map_df<32><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
        else k_map_df<64><<<grid, DF_ROWS, 0, ctx->stream>>>(qg, m, q, n, d, a, per, part);
    } else {
        k_map_fp64<<<grid, 256, 0, ctx->stream>>>(Qg, m, op->Q64, n, d, op->scale, alpha, per, part);
    }
    LK_LAUNCHED(ctx);
    k_sum_slices<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(m, (int)slices, part, out);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}
