// Radio-map reconstruction on the tensor cores
//   r(x) = sum_i alpha_i exp(L_i(x)),  L_i(x) = s <q(x), q_i>
// (Sec. III-A, Eq. sc-radio-map-reconstruction; Algorithm 1, reconstruction).
//
// The exponential is split at second order, an identity in exact arithmetic:
//   exp(L) = 1 + L + L^2/2 + L^3 g(L),   g(L) = sum_{k>=0} L^k / (k+3)!,
// so that
//   r(x) = m0 + s q(x).m1 + (s^2/2) q(x)^T M2 q(x) + sum_i alpha_i L_i^3 g(L_i)
// with the alpha-weighted moments m0 = sum_i alpha_i, m1 = sum_i alpha_i q_i
// and M2 = sum_i alpha_i q_i q_i^T.  alpha of a strongly regularised kernel
// system is large and cancels (|alpha| ~ |y| / lambda while r ~ |y|), so the
// first three terms, which carry that cancellation, are float64 (moments over
// the training points, then a d x d quadratic form per grid point).  The
// remainder term is small wherever |L| is (|L^3 g(L)| <= 0.03 for |L| <= 1/2),
// so relative float32 errors in it cost ~1e-3 of what they would cost on
// exp(L) itself: its logits come from tcgen05 MMAs of a three-piece bf16
// split of q sqrt(s) (six cross products: float32-accurate logits), g is a
// degree-5 polynomial (interpolant at Chebyshev nodes of [-1/2, 1/2], relative
// error < 1e-8), and the per-row sums are float32 over 64 columns, then
// double-float.  The path applies when s max|q(x)| max|q_i| <= 1/2 (Cauchy-
// Schwarz bounds every |L|); otherwise the caller uses the double-float kernel.
//
// Kernel layout (one CTA per SM, persistent over work items): an item is 256
// grid points (two 128-row A operands held in shared memory) against one
// slice of the training points, streamed by TMA as 128-point B tiles through a
// ring; one thread issues the MMAs into a double-buffered pair of 128 x 128
// float32 accumulators (all 512 tensor-memory columns); sixteen epilogue warps
// read the logits with tcgen05.ld and accumulate alpha_j L^3 g(L) per row with
// packed float32x2 arithmetic.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "laker_device.cuh"
#include "laker_tc.cuh"

namespace {

constexpr int MT_B = 128;                 // rows of an A operand = columns of a B tile
constexpr int MT_NA = 2;                  // A operands per item (256 grid points)
constexpr int MT_ROWS = MT_NA * MT_B;
constexpr int MT_EPI_WARPS = 16;          // 4 per tensor-memory lane quadrant
constexpr int MT_THREADS = (MT_EPI_WARPS + 2) * 32;
constexpr int MT_COLS = 64;               // columns of a B tile per epilogue warp
constexpr uint32_t MT_TMEM_COLS = 2 * MT_NA * MT_B;   // two accumulator sets: 512 columns
constexpr int MT_PIECES = 3;
constexpr int MT_DEG = 5;                 // degree of the polynomial for g

template <int DPAD>
struct MtCfg {
    static constexpr int TILE = MT_B * DPAD * 2;                       // one bf16 piece, 128 rows
    static constexpr int STAGES = DPAD >= 64 ? 2 : DPAD >= 32 ? 4 : 8;
    static constexpr int SWZ = DPAD * 2;
};

struct MtSmem {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t afull;
    uint64_t aempty;
    uint32_t tmem_base;
};

struct MtSched {
    int64_t mpad;    // grid rows, padded to a multiple of 256
    int ntiles;      // training tiles of 128 points
    int slices;      // training slices per 256-row block
    int per;         // tiles per slice
    int items;       // (m / 256) x slices
};

struct MtPoly {
    float c[MT_DEG + 1];
};

__device__ __forceinline__ void mt_item(int it, const MtSched& s, int& sb, int& t0, int& t1) {
    sb = it / s.slices;
    const int z = it % s.slices;
    t0 = z * s.per;
    t1 = min(s.ntiles, t0 + s.per);
}

// One 16-column chunk: part += alpha_j L^3 g(L) over the chunk's columns.
__device__ __forceinline__ void mt_chunk(const uint32_t* v, const float4* a4, const MtPoly& P, float2& part) {
    float2 al[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 t = __ldg(a4 + u);
        al[2 * u] = make_float2(t.x, t.y);
        al[2 * u + 1] = make_float2(t.z, t.w);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 L = make_float2(__uint_as_float(v[2 * k]), __uint_as_float(v[2 * k + 1]));
        float2 g = make_float2(P.c[MT_DEG], P.c[MT_DEG]);
#pragma unroll
        for (int e = MT_DEG - 1; e >= 0; --e) g = __ffma2_rn(g, L, make_float2(P.c[e], P.c[e]));
        const float2 L2 = __fmul2_rn(L, L);
        const float2 aL = __fmul2_rn(al[k], L);
        part = __ffma2_rn(__fmul2_rn(aL, L2), g, part);
    }
}

template <int DPAD>
__global__ void __launch_bounds__(MT_THREADS, 1)
k_map_tc(const __grid_constant__ CUtensorMap g_h, const __grid_constant__ CUtensorMap g_m,
         const __grid_constant__ CUtensorMap g_l, const __grid_constant__ CUtensorMap t_h,
         const __grid_constant__ CUtensorMap t_m, const __grid_constant__ CUtensorMap t_l,
         const float* __restrict__ alpha32, MtSched sch, MtPoly poly, double* __restrict__ part,
         int* __restrict__ err) {
    using C = MtCfg<DPAD>;
    constexpr int TILE = C::TILE;
    extern __shared__ __align__(1024) unsigned char mt_smem_raw[];
    unsigned char* base = mt_smem_raw;
    {
        const uint32_t a = smem_u32(base);
        base += (1024 - (a & 1023)) & 1023;
    }
    unsigned char* sA = base;                                    // [a][piece]
    unsigned char* sB = base + MT_NA * MT_PIECES * TILE;         // [stage][piece]
    MtSmem* S = reinterpret_cast<MtSmem*>(sB + C::STAGES * MT_PIECES * TILE);
    const CUtensorMap* gm[3] = {&g_h, &g_m, &g_l};
    const CUtensorMap* tm[3] = {&t_h, &t_m, &t_l};

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(&S->full[s], 1); mbar_init(&S->empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&S->tfull[a], 1); mbar_init(&S->tempty[a], MT_EPI_WARPS); }
        mbar_init(&S->afull, 1);
        mbar_init(&S->aempty, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MT_EPI_WARPS + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(MT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == MT_EPI_WARPS) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int issued = 0, nitem = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < sch.items && ok; it += G) {
                int sb, t0, t1;
                mt_item(it, sch, sb, t0, t1);
                if (nitem > 0 && !mbar_wait(&S->aempty, (nitem - 1) & 1, err)) break;
                mbar_expect_tx(&S->afull, MT_NA * MT_PIECES * TILE);
                for (int a = 0; a < MT_NA; ++a)
                    for (int p = 0; p < MT_PIECES; ++p)
                        tma_load_2d(sA + (a * MT_PIECES + p) * TILE, gm[p], &S->afull, 0, sb * MT_ROWS + a * MT_B);
                ++nitem;
                for (int t = t0; t < t1; ++t) {
                    const int st = issued % C::STAGES;
                    const uint32_t ph = (issued / C::STAGES) & 1;
                    if (!mbar_wait(&S->empty[st], ph ^ 1, err)) { ok = false; break; }
                    mbar_expect_tx(&S->full[st], MT_PIECES * TILE);
                    for (int p = 0; p < MT_PIECES; ++p)
                        tma_load_2d(sB + (st * MT_PIECES + p) * TILE, tm[p], &S->full[st], 0, t * MT_B);
                    ++issued;
                }
            }
            // drain: every copy this CTA issued has landed before it may exit
            if (nitem > 0) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->afull, (nitem - 1) & 1) && clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
            for (int i = max(0, issued - C::STAGES); i < issued; ++i) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->full[i % C::STAGES], (i / C::STAGES) & 1) && clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
        }
    } else if (warp == MT_EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc_bf16(MT_B, MT_B);
            // the six cross products of the pieces (h, m, l) whose orders add to at most 2
            constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
            constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
            int nitem = 0, seq = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < sch.items && ok; it += G) {
                int sb, t0, t1;
                mt_item(it, sch, sb, t0, t1);
                if (nitem > 0) umma_commit(&S->aempty);   // the previous item's MMAs release the A operands
                if (!mbar_wait(&S->afull, nitem & 1, err)) break;
                ++nitem;
                for (int t = t0; t < t1; ++t) {
                    const int st = seq % C::STAGES;
                    const uint32_t ph = (seq / C::STAGES) & 1;
                    const int ab = seq & 1;
                    const uint32_t aph = (seq >> 1) & 1;
                    if (!mbar_wait(&S->tempty[ab], aph ^ 1, err)) { ok = false; break; }
                    tc_fence_after();
                    if (!mbar_wait(&S->full[st], ph, err)) { ok = false; break; }
                    tc_fence_after();
                    for (int a = 0; a < MT_NA; ++a) {
                        const uint32_t d = tmem + (uint32_t)((ab * MT_NA + a) * MT_B);
                        uint32_t accum = 0;
#pragma unroll
                        for (int kk = 0; kk < DPAD / 16; ++kk) {
                            const int kb = kk * 32;
#pragma unroll
                            for (int x = 0; x < 6; ++x) {
                                umma_bf16(d, smem_desc(sA + (a * MT_PIECES + pa[x]) * TILE, C::SWZ, kb),
                                          smem_desc(sB + (st * MT_PIECES + pb[x]) * TILE, C::SWZ, kb), idesc, accum);
                                accum = 1;
                            }
                        }
                    }
                    umma_commit(&S->empty[st]);
                    umma_commit(&S->tfull[ab]);
                    ++seq;
                }
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3, h = warp >> 2;
        const int a = h >> 1, ch = h & 1;
        const int row_in_item = a * MT_B + q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        int seq = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < sch.items && ok; it += G) {
            int sb, t0, t1;
            mt_item(it, sch, sb, t0, t1);
            float hi = 0.f, lo = 0.f;   // double-float row sum over the item's tiles
            for (int t = t0; t < t1; ++t) {
                const int ab = seq & 1;
                const uint32_t aph = (seq >> 1) & 1;
                int w = (lane == 0) ? (int)mbar_wait(&S->tfull[ab], aph, err) : 0;
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) { ok = false; break; }
                tc_fence_after();
                const uint32_t tcol = tmem + lane_addr + (uint32_t)((ab * MT_NA + a) * MT_B + ch * MT_COLS);
                const float4* a4 = reinterpret_cast<const float4*>(alpha32 + (int64_t)t * MT_B + ch * MT_COLS);
                float2 p2 = make_float2(0.f, 0.f);
                uint32_t v[16];
#pragma unroll
                for (int c = 0; c < MT_COLS / 16; ++c) {
                    tmem_ld16(tcol + c * 16, v);
                    tmem_wait(v);
                    if (c == MT_COLS / 16 - 1) {   // last read of this accumulator: release it
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&S->tempty[ab]);
                    }
                    mt_chunk(v, a4 + c * 4, poly, p2);
                }
                const float sv = p2.x + p2.y;
                const float sum = hi + sv;   // two-sum
                const float bp = sum - hi;
                lo += (hi - (sum - bp)) + (sv - bp);
                hi = sum;
                ++seq;
            }
            if (!ok) break;
            const int z = it % sch.slices;
            part[((int64_t)z * 2 + ch) * sch.mpad + (int64_t)sb * MT_ROWS + row_in_item] = (double)hi + (double)lo;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MT_EPI_WARPS + 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT_TMEM_COLS)
                     : "memory");
    }
}

// Three-piece bf16 split of x = q sqrt(s):  h = bf16(x), m = bf16(x - h),
// l = bf16(x - h - m)  (rows x dpad, zero padding in columns >= d and rows >=
// rows_valid), and the largest |q_i|^2 (atomic max on the float64 bits, which
// order like the values for non-negative numbers).
__global__ void k_map_split3(int64_t rows_valid, int64_t rows_pad, int d, int dpad, const double* __restrict__ Q,
                             double sq, __nv_bfloat16* __restrict__ ph, __nv_bfloat16* __restrict__ pm,
                             __nv_bfloat16* __restrict__ pl, unsigned long long* __restrict__ maxnorm2) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows_pad) return;
    double nrm = 0.0;
    for (int k = lane; k < dpad; k += 32) {
        double x = 0.0;
        if (r < rows_valid && k < d) {
            const double qv = Q[r * d + k];
            nrm = fma(qv, qv, nrm);
            x = qv * sq;
        }
        const __nv_bfloat16 h = __double2bfloat16(x);
        const double r1 = x - (double)__bfloat162float(h);
        const __nv_bfloat16 m = __double2bfloat16(r1);
        const double r2 = r1 - (double)__bfloat162float(m);
        ph[r * dpad + k] = h;
        pm[r * dpad + k] = m;
        pl[r * dpad + k] = __double2bfloat16(r2);
    }
    nrm = lk::warp_sum(nrm);
    if (lane == 0 && r < rows_valid) atomicMax(maxnorm2, (unsigned long long)__double_as_longlong(nrm));
}

__global__ void k_map_alpha32(int64_t n, int64_t npad, const double* __restrict__ alpha, float* __restrict__ a32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npad) a32[i] = (i < n) ? (float)alpha[i] : 0.f;
}

// alpha-weighted moments, one block per entry in a fixed order:
// entry 0 = sum alpha_i, 1 + a = sum alpha_i q_ia, then for a <= b the pair
// (a, b) of sum alpha_i q_ia q_ib (stored at 1 + d + a d + b and mirrored).
__global__ void k_map_moments(int64_t n, int d, const double* __restrict__ Q, const double* __restrict__ alpha,
                              double* __restrict__ mom) {
    __shared__ double red[8];
    int e = blockIdx.x, a = -1, b = -1;
    if (e >= 1 && e <= d) a = e - 1;
    else if (e > d) {
        int t = e - 1 - d;
        a = 0;
        while (t >= d - a) { t -= d - a; ++a; }
        b = a + t;
    }
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double v = alpha[i];
        if (a >= 0) v *= Q[i * d + a];
        if (b >= 0) v *= Q[i * d + b];
        s += v;
    }
    s = lk::block_sum(s, red);
    if (threadIdx.x == 0) {
        if (a < 0) mom[0] = s;
        else if (b < 0) mom[1 + a] = s;
        else {
            mom[1 + d + a * d + b] = s;
            mom[1 + d + b * d + a] = s;
        }
    }
}

// r(x) = m0 + s q.m1 + (s^2/2) q^T M2 q + the remainder partial sums (slices
// and column halves added in a fixed order); thread per grid point.
__global__ void __launch_bounds__(256) k_map_finish(int64_t m, int d, int64_t mpad, int slices, double s,
                                                    const double* __restrict__ Qg, const double* __restrict__ mom,
                                                    const double* __restrict__ part, double* __restrict__ out) {
    extern __shared__ double msh[];   // 1 + d + d * d
    const int E = 1 + d + d * d;
    for (int i = threadIdx.x; i < E; i += blockDim.x) msh[i] = mom[i];
    __syncthreads();
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= m) return;
    const double* q = Qg + x * d;
    const double* M2 = msh + 1 + d;
    double lin = 0.0, quad = 0.0;
    for (int a = 0; a < d; ++a) {
        const double qa = q[a];
        lin = fma(qa, msh[1 + a], lin);
        double t = 0.5 * M2[a * d + a] * qa;
        for (int b = a + 1; b < d; ++b) t = fma(M2[a * d + b], q[b], t);
        quad = fma(qa, t, quad);
    }
    double r = 0.0;
    for (int z = 0; z < slices; ++z) r += part[(int64_t)(2 * z) * mpad + x] + part[(int64_t)(2 * z + 1) * mpad + x];
    out[x] = msh[0] + s * lin + s * s * quad + r;
}

// Coefficients of the degree-5 interpolant of g(L) = sum_k L^k / (k+3)! at the
// six Chebyshev nodes of [-1/2, 1/2] (long double series and elimination).
MtPoly remainder_poly() {
    constexpr int N = MT_DEG + 1;
    long double V[N][N + 1];
    for (int i = 0; i < N; ++i) {
        const long double x = 0.5L * std::cos((2.0L * i + 1.0L) * 3.14159265358979323846264338327950288L / (2.0L * N));
        long double g = 0.0L, term = 1.0L / 6.0L;
        for (int k = 0; k < 40; ++k) {   // term = x^k / (k + 3)!
            g += term;
            term *= x / (long double)(k + 4);
        }
        long double p = 1.0L;
        for (int j = 0; j < N; ++j) { V[i][j] = p; p *= x; }
        V[i][N] = g;
    }
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r)
            if (std::fabs(V[r][c]) > std::fabs(V[piv][c])) piv = r;
        for (int j = 0; j <= N; ++j) std::swap(V[c][j], V[piv][j]);
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            const long double f = V[r][c] / V[c][c];
            for (int j = c; j <= N; ++j) V[r][j] -= f * V[c][j];
        }
    }
    MtPoly P;
    for (int j = 0; j < N; ++j) P.c[j] = (float)(V[j][N] / V[j][j]);
    return P;
}

size_t mt_smem_bytes(int dpad) {
    const size_t tile = (size_t)MT_B * dpad * 2;
    const int stages = dpad >= 64 ? MtCfg<64>::STAGES : dpad >= 32 ? MtCfg<32>::STAGES : MtCfg<16>::STAGES;
    // at least 120 KB so that one CTA holds an SM and its 512 tensor-memory columns
    return std::max<size_t>(120 * 1024, 1024 + (size_t)(MT_NA + stages) * MT_PIECES * tile + sizeof(MtSmem));
}

}  // namespace

// Largest s max|q(x)| max|q_i| for which the split form is used.
constexpr double MT_LOGIT_BOUND = 0.5;

laker_status eval_map_tc(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m, const double* alpha,
                         double* out, bool* applied) {
    *applied = false;
    const int d = op->d;
    if (d > 64) return LAKER_OK;
    const int dpad = d <= 16 ? 16 : d <= 32 ? 32 : 64;   // operand row = one swizzle span
    auto encode = get_encode(ctx);
    if (!encode) return LAKER_ERR_CUDA;
    const int64_t n = op->n;
    cudaStream_t s = ctx->stream;
    const int64_t nsb = (m + MT_ROWS - 1) / MT_ROWS;
    const int64_t mpad = nsb * MT_ROWS;
    const int ntiles = (int)((n + MT_B - 1) / MT_B);
    const int64_t npad = (int64_t)ntiles * MT_B;
    MtSched sch;
    sch.mpad = mpad;
    sch.ntiles = ntiles;
    int slices = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (ctx->num_sms + nsb - 1) / nsb));
    sch.per = (ntiles + slices - 1) / slices;
    sch.slices = (ntiles + sch.per - 1) / sch.per;
    if (nsb * sch.slices > (int64_t)1 << 30) return set_error(ctx, LAKER_ERR_ARG, "map: too many grid points");
    sch.items = (int)(nsb * sch.slices);

    std::vector<void*> bufs;
    auto alloc = [&](void** p, size_t bytes) {
        laker_status st = lk_malloc(ctx, p, bytes);
        if (st == LAKER_OK) bufs.push_back(*p);
        return st;
    };
    auto release = [&]() {
        for (void* p : bufs) cudaFree(p);
    };
    __nv_bfloat16 *gp = nullptr, *tp = nullptr;
    float* a32 = nullptr;
    unsigned long long* norms = nullptr;
    double *mom = nullptr, *part = nullptr;
    int* err = nullptr;
    const int E = 1 + d + d * d;
    laker_status st;
    if ((st = alloc((void**)&gp, (size_t)3 * mpad * dpad * sizeof(__nv_bfloat16))) != LAKER_OK ||
        (st = alloc((void**)&tp, (size_t)3 * npad * dpad * sizeof(__nv_bfloat16))) != LAKER_OK ||
        (st = alloc((void**)&a32, (size_t)npad * sizeof(float))) != LAKER_OK ||
        (st = alloc((void**)&norms, 2 * sizeof(unsigned long long))) != LAKER_OK ||
        (st = alloc((void**)&mom, (size_t)E * sizeof(double))) != LAKER_OK ||
        (st = alloc((void**)&part, (size_t)2 * sch.slices * mpad * sizeof(double))) != LAKER_OK ||
        (st = alloc((void**)&err, sizeof(int))) != LAKER_OK) {
        release();
        return st;
    }
#define MT_TRY(call)                                                                           \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            release();                                                                         \
            return set_error(ctx, LAKER_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                      \
    } while (0)
    MT_TRY(cudaMemsetAsync(norms, 0, 2 * sizeof(unsigned long long), s));
    MT_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    const double sq = std::sqrt(op->scale);
    k_map_split3<<<(unsigned)((mpad + 7) / 8), 256, 0, s>>>(m, mpad, d, dpad, Qg, sq, gp, gp + mpad * dpad,
                                                            gp + 2 * mpad * dpad, norms);
    ctx->launches++;
    k_map_split3<<<(unsigned)((npad + 7) / 8), 256, 0, s>>>(n, npad, d, dpad, op->Q64, sq, tp, tp + npad * dpad,
                                                            tp + 2 * npad * dpad, norms + 1);
    ctx->launches++;
    MT_TRY(cudaGetLastError());
    unsigned long long hn[2] = {0, 0};
    MT_TRY(cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s));
    MT_TRY(cudaStreamSynchronize(s));
    double ng, nt;
    std::memcpy(&ng, &hn[0], sizeof(double));
    std::memcpy(&nt, &hn[1], sizeof(double));
    const double bound = op->scale * std::sqrt(ng) * std::sqrt(nt);
    if (!(bound <= MT_LOGIT_BOUND)) {   // also NaN
        release();
        return LAKER_OK;
    }
    k_map_alpha32<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(n, npad, alpha, a32);
    ctx->launches++;
    k_map_moments<<<(unsigned)E - (unsigned)(d * (d - 1) / 2), 256, 0, s>>>(n, d, op->Q64, alpha, mom);
    ctx->launches++;
    MT_TRY(cudaGetLastError());

    CUtensorMap maps[6];
    const CUtensorMapSwizzle swz = dpad == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : dpad == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                : CU_TENSOR_MAP_SWIZZLE_32B;
    for (int k = 0; k < 6; ++k) {
        const bool grid = k < 3;
        const int64_t rows = grid ? mpad : npad;
        void* ptr = grid ? (void*)(gp + k * mpad * dpad) : (void*)(tp + (k - 3) * npad * dpad);
        const cuuint64_t dims[2] = {(cuuint64_t)dpad, (cuuint64_t)rows};
        const cuuint64_t strides[1] = {(cuuint64_t)dpad * 2};
        const cuuint32_t box[2] = {(cuuint32_t)dpad, (cuuint32_t)MT_B};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            release();
            return set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled failed (map)");
        }
    }
    static const MtPoly poly = remainder_poly();
    const size_t smem = mt_smem_bytes(dpad);
    const unsigned grid = (unsigned)std::min<int64_t>(sch.items, ctx->num_sms);
#define MT_LAUNCH(D)                                                                                        \
    do {                                                                                                    \
        MT_TRY(cudaFuncSetAttribute(k_map_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_map_tc<D><<<grid, MT_THREADS, smem, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], a32, \
                                                   sch, poly, part, err);                                  \
    } while (0)
    if (dpad == 16) MT_LAUNCH(16);
    else if (dpad == 32) MT_LAUNCH(32);
    else MT_LAUNCH(64);
#undef MT_LAUNCH
    ctx->launches++;
    MT_TRY(cudaGetLastError());
    const size_t fsm = (size_t)E * sizeof(double);
    if (fsm > 48 * 1024) MT_TRY(cudaFuncSetAttribute(k_map_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
    k_map_finish<<<(unsigned)((m + 255) / 256), 256, fsm, s>>>(m, d, mpad, sch.slices, op->scale, Qg, mom, part, out);
    ctx->launches++;
    MT_TRY(cudaGetLastError());
    int herr = 0;
    MT_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MT_TRY(cudaStreamSynchronize(s));
    release();
#undef MT_TRY
    if (herr) return set_error(ctx, (laker_status)herr, "tensor-core map: bounded wait expired");
    *applied = true;
    return LAKER_OK;
}
