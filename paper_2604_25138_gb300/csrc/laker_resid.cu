// Float64-accurate product w = (lambda I + G) x for split-bf16 operators, the
// true residual of mixed-precision PCG (residual replacement every k
// products; Sec. IV-E PCG with reliable updates).
//
// Near convergence the terms G_ij alpha_j are ~1e4 and cancel to O(1) sums, so
// each kernel value must be right to ~2^-45: it is stored, once per unordered
// pair, as a float32 pair (hi, lo) with hi + lo = G_ij to ~2^-48.  G is
// symmetric, so only the upper triangle of 128 x 128 tiles is kept, tile
// (I, J), I <= J, at position I nb - I (I - 1)/2 + (J - I) of a packed array,
// hi tile then lo tile, row-major: half the bytes of the full pair, and each
// stored value serves both its row sum (sum_j G_ij x_j, i in block I) and,
// off the diagonal, its column sum (sum_i G_ij x_i, j in block J).
//
// k_df_sym: one CTA per SM on a contiguous range of the tiles (row-major over
// I); 16 warps, warp w takes rows 8w .. 8w + 7 of a tile and lane l the
// columns 4l .. 4l + 3 (16-byte streaming loads, all eight rows' loads issued
// before the arithmetic).  Products are accumulated with the K = 3 dot product
// of Ogita, Rump and Oishi (Dot3 in laker_df.cuh) in float32 arithmetic:
// rows in registers for the CTA's whole segment of block row I, columns per
// tile (reduced over the 16 warps in shared memory in a fixed order).
// k_df_sym_finish adds lambda x_i, the row partials of the segments of block
// I and the column partials of the tiles (I', I), I' < I, in a fixed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "laker_device.cuh"
#include "laker_df.cuh"
#include "laker_tc.cuh"

namespace {

constexpr int RT = 128;              // tile edge
constexpr int RW = 16;               // warps per CTA
constexpr int RR = RT / RW;          // rows per warp

struct RSched {
    int nb;        // blocks of 128
    int64_t T;     // tiles nb (nb + 1) / 2
    int G;         // CTAs
    int slots;     // max CTAs sharing one block row
};

__host__ __device__ __forceinline__ int64_t r_row_start(int I, int nb) {
    return (int64_t)I * nb - (int64_t)I * (I - 1) / 2;
}
__host__ __device__ __forceinline__ int64_t r_begin(int64_t g, const RSched& s) { return g * s.T / s.G; }
__host__ __device__ __forceinline__ int r_owner(int64_t t, const RSched& s) {
    int g = (int)((t * s.G) / s.T);
    while (g + 1 < s.G && r_begin(g + 1, s) <= t) ++g;
    while (g > 0 && r_begin(g, s) > t) --g;
    return g;
}
__host__ __device__ __forceinline__ int r_row_of(int64_t t, int nb) {
    int I = 0;
    while (I + 1 < nb && r_row_start(I + 1, nb) <= t) ++I;
    return I;
}

__device__ __forceinline__ bool r_gated(const PcgScalars* sc, int gate) {
    if (sc == nullptr || gate == 0) return false;
    if (*(volatile const int*)&sc->converged != 0) return true;
    return *(volatile const int*)&sc->need_true == 0;
}

__device__ __forceinline__ lk::df2 shfl_df(lk::df2 v, int o) {
    lk::df2 u;
    u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    return u;
}

constexpr int RQ = 32;                       // rows of a quarter tile (one pipeline stage)
constexpr int RSTAGES = 5;
constexpr uint32_t RQ_BYTES = RQ * RT * 4;   // one quarter of hi (or lo): 16 KB
constexpr int R_THREADS = (RW + 1) * 32;     // 16 compute warps + one copy warp

struct RSmem {
    uint64_t full[RSTAGES];
    uint64_t empty[RSTAGES];
};

size_t r_smem_bytes() { return 128 + (size_t)RSTAGES * 2 * RQ_BYTES + sizeof(RSmem); }

// One CTA per SM over a contiguous range of the tiles.  A copy warp streams
// each tile as four quarters (32 rows of hi, then of lo: 2 x 16 KB contiguous
// bulk copies) through a 5-stage shared-memory ring; 16 compute warps take 2
// rows of each quarter (warp w: rows 2w, 2w + 1 of the quarter, i.e. rows
// 32 q + 2w + {0, 1} of the tile) and lane l the columns 4l .. 4l + 3.
__global__ void __launch_bounds__(R_THREADS, 1)
k_df_sym(const float* __restrict__ Kp, RSched sch, int64_t n, const double* __restrict__ x,
         float2* __restrict__ rowpart, float2* __restrict__ colpart, const PcgScalars* sc, int gate,
         int* __restrict__ err) {
    if (r_gated(sc, gate)) return;
    __shared__ float2 xI[RT], xJ[RT];
    __shared__ float2 cred[RW][RT];
    extern __shared__ __align__(128) unsigned char r_smem_raw[];
    unsigned char* base = r_smem_raw;
    {
        const uint32_t a = smem_u32(base);
        base += (128 - (a & 127)) & 127;
    }
    float* ring = reinterpret_cast<float*>(base);                          // [stage][hi 32 x 128][lo 32 x 128]
    RSmem* S = reinterpret_cast<RSmem*>(base + (size_t)RSTAGES * 2 * RQ_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x;
    const int64_t t0 = r_begin(g, sch), t1 = r_begin(g + 1, sch);
    if (t0 >= t1) return;
    if (threadIdx.x == 0) {
        for (int st = 0; st < RSTAGES; ++st) { mbar_init(&S->full[st], 1); mbar_init(&S->empty[st], RW); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int64_t nq = (t1 - t0) * 4;    // quarters this CTA streams
    if (warp == RW) {
        // ---------------- copy warp ----------------
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t q = 0; q < nq; ++q) {
                const int st = (int)(q % RSTAGES);
                if (!mbar_wait(&S->empty[st], (uint32_t)((q / RSTAGES) & 1) ^ 1, err)) break;
                const int64_t t = t0 + q / 4;
                const int part = (int)(q % 4);
                const float* hi = Kp + t * (2 * RT * RT) + part * RQ * RT;
                float* dst = ring + (size_t)st * 2 * RQ * RT;
                mbar_expect_tx(&S->full[st], 2 * RQ_BYTES);
                bulk_load(dst, hi, RQ_BYTES, &S->full[st]);
                bulk_load(dst + RQ * RT, hi + RT * RT, RQ_BYTES, &S->full[st]);
                issued = q + 1;
            }
            for (int64_t q = (issued > RSTAGES ? issued - RSTAGES : 0); q < issued; ++q) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->full[q % RSTAGES], (uint32_t)((q / RSTAGES) & 1)) &&
                       clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
        }
        // the copy warp joins no further barrier: compute warps sync with named barrier 1
        return;
    }
    // ---------------- compute warps ----------------
    auto csync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(RW * 32) : "memory"); };
    int I = r_row_of(t0, sch.nb);
    int J = I + (int)(t0 - r_row_start(I, sch.nb));
    lk::Dot3 row[8];   // rows 32 qq + 2 warp + e of block I, qq = 0..3, e = 0..1
    auto load_x = [&](float2* dst, int blk) {
        if (threadIdx.x < RT) {
            const int64_t i = (int64_t)blk * RT + threadIdx.x;
            const lk::df2 v = lk::df_from(i < n ? x[i] : 0.0);
            dst[threadIdx.x] = make_float2(v.hi, v.lo);
        }
    };
    auto flush = [&](int blk) {
        const int slot = g - r_owner(r_row_start(blk, sch.nb), sch);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            lk::df2 v = row[k].value();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = lk::df_add(v, shfl_df(v, o));
            if (lane == 0) {
                const int r = (k >> 1) * RQ + 2 * warp + (k & 1);
                rowpart[((int64_t)blk * sch.slots + slot) * RT + r] = make_float2(v.hi, v.lo);
            }
            row[k] = lk::Dot3();
        }
    };
    load_x(xI, I);
    bool dirty = false;
    // once a bounded wait has expired (the error word is set) a warp skips its
    // waits and arithmetic but keeps reaching every named barrier, so that all
    // compute warps leave the loop together
    bool ok = true;
    int64_t q = 0;
    for (int64_t t = t0; t < t1; ++t) {
        load_x(xJ, J);
        csync();
        lk::df2 xj[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) { const float2 v = xJ[4 * lane + c]; xj[c] = {v.x, v.y}; }
        const bool diag = (I == J);
        lk::Dot3 col[4];
#pragma unroll
        for (int part = 0; part < 4; ++part, ++q) {
            const int st = (int)(q % RSTAGES);
            if (ok) {
                int w = (lane == 0) ? (int)mbar_wait(&S->full[st], (uint32_t)((q / RSTAGES) & 1), err) : 0;
                ok = __shfl_sync(0xffffffffu, w, 0) != 0;
            }
            if (!ok) continue;
            const float* hq = ring + (size_t)st * 2 * RQ * RT;
            const float* lq = hq + RQ * RT;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int rr = 2 * warp + e;                       // row within the quarter
                const float4 h = reinterpret_cast<const float4*>(hq + rr * RT)[lane];
                const float4 l = reinterpret_cast<const float4*>(lq + rr * RT)[lane];
                const float gh[4] = {h.x, h.y, h.z, h.w};
                const float gl[4] = {l.x, l.y, l.z, l.w};
                const float2 xv = xI[part * RQ + rr];
                const lk::df2 xi = {xv.x, xv.y};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const lk::df2 gv = {gh[c], gl[c]};
                    row[2 * part + e].add(gv, xj[c]);
                    if (!diag) col[c].add(gv, xi);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->empty[st]);
        }
        dirty = true;
        if (!diag) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const lk::df2 v = col[c].value();
                cred[warp][4 * lane + c] = make_float2(v.hi, v.lo);
            }
        }
        csync();
        if (!diag && threadIdx.x < RT) {
            lk::df2 s = {cred[0][threadIdx.x].x, cred[0][threadIdx.x].y};
#pragma unroll
            for (int w = 1; w < RW; ++w) s = lk::df_add(s, lk::df2{cred[w][threadIdx.x].x, cred[w][threadIdx.x].y});
            colpart[t * RT + threadIdx.x] = make_float2(s.hi, s.lo);
        }
        if (++J == sch.nb) {
            flush(I);
            dirty = false;
            ++I;
            J = I;
            if (t + 1 < t1) load_x(xI, I);
        }
    }
    if (ok && dirty) flush(I);
}

// w_i = lambda x_i + (row partials of block I's segments) + (column partials of
// the tiles (I', I), I' < I), all in double-float, in a fixed order.
__global__ void k_df_sym_finish(RSched sch, int64_t n, double lambda, const double* __restrict__ x,
                                const float2* __restrict__ rowpart, const float2* __restrict__ colpart,
                                const int* __restrict__ nslots, double* __restrict__ w, const PcgScalars* sc,
                                int gate) {
    if (r_gated(sc, gate)) return;
    const int I = blockIdx.x;
    const int r = threadIdx.x;
    const int64_t i = (int64_t)I * RT + r;
    if (i >= n) return;
    lk::df2 s = {0.f, 0.f};
    const int ns = nslots[I];
    for (int k = 0; k < ns; ++k) {
        const float2 v = rowpart[((int64_t)I * sch.slots + k) * RT + r];
        s = lk::df_add(s, lk::df2{v.x, v.y});
    }
    for (int Ip = 0; Ip < I; ++Ip) {
        const float2 v = colpart[(r_row_start(Ip, sch.nb) + (I - Ip)) * RT + r];
        s = lk::df_add(s, lk::df2{v.x, v.y});
    }
    w[i] = fma(lambda, x[i], lk::df_to(s));
}

// Packed pair (hi, lo) of the upper-triangular tiles in double-float on the
// float32 pipes (GB300's float64 rate is ~1/64 of float32): each thread takes
// one column j of a tile (its embedding row, pre-scaled by sqrt(scale), in
// registers) and half of the rows i (from shared memory); the logit is a
// compensated dot product (Dot3, error ~2^-70 of the sum of |terms|) and the
// exponential Tang's double-float exp (~1e-14 relative), so hi + lo is G_ij
// to ~2^-46.  Stores are coalesced along j.  Entries with i or j >= n are 0.
template <int DM>
__global__ void __launch_bounds__(256)
k_build_packed_df(const float2* __restrict__ Qs, int64_t n, int d, int nb, int j0, float* __restrict__ Kp) {
    extern __shared__ float2 qi_s[];             // 128 rows x DM df values of block I
    __shared__ float e2tab[128];
    lk::df_exp_table_init(e2tab);
    int I, J;                                    // tiles with J >= j0 (all: j0 = 0)
    lk::upper_pair(blockIdx.x, nb, j0, I, J);
    const int64_t t = r_row_start(I, nb) + (J - I);
    for (int idx = threadIdx.x; idx < RT * DM; idx += blockDim.x) {
        const int r = idx / DM, k = idx % DM;
        const int64_t i = (int64_t)I * RT + r;
        qi_s[idx] = (i < n && k < d) ? Qs[i * d + k] : make_float2(0.f, 0.f);
    }
    const int c = threadIdx.x & (RT - 1), half = threadIdx.x >> 7;
    const int64_t j = (int64_t)J * RT + c;
    lk::df2 qj[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) {
        const float2 v = (j < n && k < d) ? Qs[j * d + k] : make_float2(0.f, 0.f);
        qj[k] = {v.x, v.y};
    }
    __syncthreads();
    float* hi = Kp + t * (2 * RT * RT);
    float* lo = hi + RT * RT;
    // four rows at a time: four independent compensated dot products in flight
    for (int r0 = half * (RT / 2); r0 < (half + 1) * (RT / 2); r0 += 4) {
        lk::Dot3 dot[4];
#pragma unroll
        for (int k = 0; k < DM; ++k) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 q = qi_s[(r0 + u) * DM + k];
                dot[u].add(lk::df2{q.x, q.y}, qj[k]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u;
            const int64_t i = (int64_t)I * RT + r;
            float h = 0.f, l = 0.f;
            if (i < n && j < n) {
                const lk::df2 e = lk::df_exp(dot[u].value(), e2tab);
                h = e.hi;
                l = e.lo;
            }
            hi[r * RT + c] = h;
            lo[r * RT + c] = l;
        }
    }
}

__global__ void k_q_df(int64_t count, const double* __restrict__ x, double scale, float2* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const lk::df2 v = lk::df_from(x[i] * scale);
    y[i] = make_float2(v.hi, v.lo);
}

}  // namespace

struct ResidWork {
    RSched sch;
    float* Kp = nullptr;          // packed (hi, lo) tiles of the upper triangle
    float2* rowpart = nullptr;
    float2* colpart = nullptr;
    int* nslots = nullptr;
    int* err = nullptr;           // status word of the bounded waits
};

void resid_release(laker_op* op) {
    ResidWork* rw = static_cast<ResidWork*>(op->rw);
    if (!rw) return;
    cudaFree(rw->Kp);
    cudaFree(rw->rowpart);
    cudaFree(rw->colpart);
    cudaFree(rw->nslots);
    cudaFree(rw->err);
    delete rw;
    op->rw = nullptr;
}

// Packed storage and the tile schedule of an operator (built by the caller).
laker_status resid_prepare(laker_ctx* ctx, laker_op* op, float** Kp) {
    ResidWork* rw = new ResidWork();
    RSched& s = rw->sch;
    s.nb = (int)((op->n + RT - 1) / RT);
    s.T = (int64_t)s.nb * (s.nb + 1) / 2;
    s.G = (int)std::min<int64_t>(s.T, (int64_t)ctx->num_sms);
    s.slots = 1;
    std::vector<int> ns((size_t)s.nb);
    for (int I = 0; I < s.nb; ++I) {
        const int64_t a = r_row_start(I, s.nb), b = a + (s.nb - I) - 1;
        ns[(size_t)I] = r_owner(b, s) - r_owner(a, s) + 1;
        s.slots = std::max(s.slots, ns[(size_t)I]);
    }
    op->rw = rw;
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&rw->Kp, (size_t)s.T * 2 * RT * RT * sizeof(float))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&rw->rowpart, (size_t)s.nb * s.slots * RT * sizeof(float2))) != LAKER_OK)
        return st;
    if ((st = lk_malloc(ctx, (void**)&rw->colpart, (size_t)s.T * RT * sizeof(float2))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&rw->nslots, (size_t)s.nb * sizeof(int))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&rw->err, sizeof(int))) != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMemsetAsync(rw->err, 0, sizeof(int), ctx->stream));
    LK_CUDA(ctx, cudaFuncSetAttribute(k_df_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)r_smem_bytes()));
    LK_CUDA(ctx, cudaMemcpyAsync(rw->nslots, ns.data(), sizeof(int) * s.nb, cudaMemcpyHostToDevice, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *Kp = rw->Kp;
    return LAKER_OK;
}

// w = (lambda I + G) x from the packed pair; gate 1 skips the launch's work
// unless a true residual is due (PCG residual replacement).
laker_status resid_matvec(laker_ctx* ctx, const laker_op* op, const double* x, double* w, const PcgScalars* sc,
                          int gate) {
    const ResidWork* rw = static_cast<const ResidWork*>(op->rw);
    if (!rw) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "packed float64-accurate operator not built");
    k_df_sym<<<(unsigned)rw->sch.G, R_THREADS, r_smem_bytes(), ctx->stream>>>(rw->Kp, rw->sch, op->n, x, rw->rowpart,
                                                                              rw->colpart, sc, gate, rw->err);
    LK_LAUNCHED(ctx);
    k_df_sym_finish<<<(unsigned)rw->sch.nb, RT, 0, ctx->stream>>>(rw->sch, op->n, op->lambda, x, rw->rowpart,
                                                                    rw->colpart, rw->nslots, w, sc, gate);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

const float* resid_packed(const laker_op* op) {
    const ResidWork* rw = static_cast<const ResidWork*>(op->rw);
    return rw ? rw->Kp : nullptr;
}

// Fill the packed pair of a split-bf16 operator (d <= 64) in double-float.
// prev: the same operator over the first prev->n points; its tiles (I, J)
// with J below the first block that reaches a new point are copied, the rest
// are evaluated.
laker_status resid_build_df(laker_ctx* ctx, const laker_op* op, const laker_op* prev) {
    const ResidWork* rw = static_cast<const ResidWork*>(op->rw);
    if (!rw) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "packed pair not allocated");
    const int64_t n = op->n;
    const int d = op->d;
    const int J0 = prev ? (int)(prev->n / RT) : 0;
    if (prev) {
        const ResidWork* pw = static_cast<const ResidWork*>(prev->rw);
        if (!pw) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "previous operator has no packed pair");
        laker_status s2 = copy_packed_tiles(ctx, pw->Kp, pw->sch.nb, rw->Kp, rw->sch.nb, J0);
        if (s2 != LAKER_OK) return s2;
    }
    const int64_t tiles = lk::upper_pairs(rw->sch.nb, J0);
    float2* Qs = nullptr;
    laker_status st = lk_malloc(ctx, (void**)&Qs, (size_t)n * d * sizeof(float2));
    if (st != LAKER_OK) return st;
    k_q_df<<<(unsigned)((n * d + 255) / 256), 256, 0, ctx->stream>>>(n * d, op->Q64, std::sqrt(op->scale), Qs);
    LK_LAUNCHED(ctx);
    const int dm = d <= 16 ? 16 : d <= 32 ? 32 : 64;
    const size_t smem = (size_t)RT * dm * sizeof(float2);
    cudaError_t e = cudaSuccess;
#define LK_PB(D)                                                                                                  \
    e = cudaFuncSetAttribute(k_build_packed_df<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    if (e == cudaSuccess && tiles > 0)                                                                            \
        k_build_packed_df<D><<<(unsigned)tiles, 256, smem, ctx->stream>>>(Qs, n, d, rw->sch.nb, J0, rw->Kp)
    if (dm == 16) { LK_PB(16); } else if (dm == 32) { LK_PB(32); } else { LK_PB(64); }
#undef LK_PB
    if (e != cudaSuccess) { cudaFree(Qs); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(Qs);
    return LAKER_OK;
}

// Status of the bounded waits of the float64-accurate product (synchronises
// the stream); LAKER_ERR_TIMEOUT if one expired, and the word is cleared.
laker_status resid_status(laker_ctx* ctx, const laker_op* op) {
    const ResidWork* rw = static_cast<const ResidWork*>(op->rw);
    if (!rw) return LAKER_OK;
    int h = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(&h, rw->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!h) return LAKER_OK;
    LK_CUDA(ctx, cudaMemsetAsync(rw->err, 0, sizeof(int), ctx->stream));
    return set_error(ctx, (laker_status)h, "float64-accurate product: bounded wait expired");
}
