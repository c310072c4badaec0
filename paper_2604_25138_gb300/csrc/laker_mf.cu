// Matrix-free operator  w = (lambda I + G) p,  G_ij = 2^(q'_i . q'_j)  with
// q' = q sqrt(scale log2 e)  (Sec. III-A Eq. sc-exp-kernel; the matvec-only
// access of Sec. IV-D, remark after Eq. kernel_shrinkage_cccp_normalization).
//
// Blackwell (sm_103a) kernel over the symmetric tile schedule (each unordered
// pair of 128-index blocks once, n(n+1)/2 pairs), one persistent CTA per SM
// on an equal contiguous range of the tiles:
//   * a TMA (cp.async.bulk.tensor) warp streams the 128-row tiles of block J
//     (split-bf16 operands q' = hi + lo) through an 8-stage shared-memory ring
//     (4 stages for d > 32) and reloads the fixed block I once per segment;
//   * one elected thread issues tcgen05.mma (kind::f16, bf16 in, f32 out) for
//     the split product  hi_i.hi_j + hi_i.lo_j + lo_i.hi_j + lo_i.lo_j  into a
//     ring of four 128 x 128 float32 accumulators (all 512 tensor-memory
//     columns).  The fourth product makes the logits the exact Gram matrix of
//     the rounded embedding hi + lo, so the computed kernel is exp of a Gram
//     matrix and stays positive semidefinite (Schur product theorem): without
//     it the operator error (~1e-6 n) exceeds lambda at n = 16384 and CG
//     breaks down;
//   * sixteen epilogue warps read the logits with tcgen05.ld, apply ex2.approx
//     (the MUFU unit, 32 results/clk/SM on GB300) and accumulate e * p_j into
//     block I's row sums and e * p_i into block J's column sums with packed
//     float32x2 FMAs, overlapping the tensor-core work of the next tiles.
// Row sums go to a per-segment partial buffer and column sums to a per-tile
// one; a finishing kernel adds lambda p, sums a row's partials in a fixed
// order and performs the PCG p^T w reduction.
// Every mbarrier wait is bounded; on timeout the kernel raises an error word,
// drains its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>
#include <cstring>

#include "laker_device.cuh"
#include "laker_tc.cuh"

namespace {

constexpr int MF_B = 128;            // block edge: tensor-memory lanes (j) = MMA N (i)
constexpr int MF_EPW = 4;            // epilogue warps per tensor-memory lane quadrant
constexpr int MF_EPI_WARPS = 4 * MF_EPW;
constexpr int MF_WCOLS = MF_B / MF_EPW;   // i columns per epilogue warp
constexpr int MF_THREADS = (MF_EPI_WARPS + 2) * 32;
constexpr int MF_NACC = 4;           // accumulator ring in tensor memory
constexpr uint32_t MF_TMEM_COLS = MF_NACC * MF_B;   // all 512 columns: one CTA per SM

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int DPAD>
struct MfCfg {
    static constexpr int STAGES = DPAD >= 64 ? 4 : 8;      // ring of streamed j-block operand tiles
    static constexpr int TILE_BYTES = MF_B * DPAD * 2;     // one bf16 operand tile (128 rows)
    static constexpr int SWZ = DPAD * 2;                    // swizzle span = row bytes
    // add the four epilogue parts of a column sum in shared memory (one
    // partial per column and tile) or write them apart (four): with d = 64 the
    // tensor cores leave the epilogue slack for the extra barrier and the
    // partials shrink 4x (n = 65536: 0.54 GB of partial writes and reads per
    // product; the product measured 934 -> 900 us); at d <= 32 the epilogue is
    // the bottleneck and the barrier made the main kernel 16 % slower
    static constexpr bool REDUCE = DPAD >= 64;
};

struct MfSmem {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t tfull[MF_NACC];
    uint64_t tempty[MF_NACC];
    uint64_t bfull;
    uint64_t bempty;
    uint32_t tmem_base;
    // column sums of the four epilogue parts of a lane quadrant, two buffers
    float cred[2][4][MF_EPW][32];
};

// Symmetric tile schedule.  With nb blocks of 128 indices, block row I owns
// the tiles (I, J = (I + k) mod nb) for k = 0 .. len(I) - 1: k = 0 is the
// diagonal tile and every unordered pair of distinct blocks appears exactly
// once (distances 1 .. (nb - 1) / 2 for every row, and distance nb / 2 only
// for rows I < nb / 2 when nb is even).  The T tiles, row-major in (I, k),
// are split into G equal contiguous ranges, one per CTA (one per SM); a range
// crossing block rows is processed as segments, one per block row.
struct MfSched {
    int64_t T;
    int nb;
    int base;    // len(I) = base + (I < half)
    int half;
    int G;
    int slots;   // max CTAs sharing one block row
};
__host__ __device__ __forceinline__ int mf_row_len(int I, const MfSched& s) { return s.base + (I < s.half ? 1 : 0); }
__host__ __device__ __forceinline__ int64_t mf_row_start(int I, const MfSched& s) {
    return I < s.half ? (int64_t)I * (s.base + 1)
                      : (int64_t)s.half * (s.base + 1) + (int64_t)(I - s.half) * s.base;
}
__host__ __device__ __forceinline__ void mf_tile(int64_t x, const MfSched& s, int& I, int& k) {
    const int64_t x0 = (int64_t)s.half * (s.base + 1);
    if (x < x0) {
        I = (int)(x / (s.base + 1));
        k = (int)(x % (s.base + 1));
    } else {
        I = s.half + (int)((x - x0) / s.base);
        k = (int)((x - x0) % s.base);
    }
}
__host__ __device__ __forceinline__ int64_t mf_tile_begin(int64_t g, const MfSched& s) { return g * s.T / s.G; }
__host__ __device__ __forceinline__ int mf_owner(int64_t x, const MfSched& s) {
    int g = (int)((x * s.G) / s.T);
    while (g + 1 < s.G && mf_tile_begin(g + 1, s) <= x) ++g;
    while (g > 0 && mf_tile_begin(g, s) > x) --g;
    return g;
}

// One 16-column chunk of the epilogue: e = 2^logit; the fixed block's row
// sums take e * p_j (j = this lane), the streamed block's sums take e * p_i.
// Pairs of columns go through the packed float32x2 FMA.
template <bool DIAG>
__device__ __forceinline__ void mf_chunk(const uint32_t* v, float2* acc, const float4* pI4, float pj, float2* sJ) {
    const float2 pjj = make_float2(pj, pj);
    float2 pI[8];
    if (!DIAG) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 t = __ldg(pI4 + u);
            pI[2 * u] = make_float2(t.x, t.y);
            pI[2 * u + 1] = make_float2(t.z, t.w);
        }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const float2 e = make_float2(ex2_approx(__uint_as_float(v[2 * m])), ex2_approx(__uint_as_float(v[2 * m + 1])));
        acc[m] = __ffma2_rn(e, pjj, acc[m]);
        if (!DIAG) sJ[m & 1] = __ffma2_rn(e, pI[m], sJ[m & 1]);
    }
}

// Sum of a[c] over the 32 lanes for the 32 columns c, by recursive halving:
// afterwards lane L holds the sum of column L in a[0].
__device__ __forceinline__ void mf_lane_reduce(float* a, int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s, H = 16 >> s;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float send = up ? a[m] : a[m + H];
            const float keep = up ? a[m + H] : a[m];
            a[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// Both 16-column loads are issued before one wait, so a tile exposes one
// tensor-memory read latency.
template <bool DIAG>
__device__ __forceinline__ void mf_tile_epilogue(uint32_t tcol, float2* acc, const float4* pI4, float pj, float2* sJ) {
    static_assert(MF_WCOLS == 32, "two 16-column chunks per warp");
    uint32_t v[32];
    tmem_ld16(tcol, v);
    tmem_ld16(tcol + 16, v + 16);
    tmem_wait(v);
    tmem_wait(v + 16);
    mf_chunk<DIAG>(v, acc, pI4, pj, sJ);
    mf_chunk<DIAG>(v + 16, acc + 8, pI4 + 4, pj, sJ);
}

// Tile (I, J): logits D[j][i] = q'_j . q'_i for the 128 j of block J
// (tensor-memory lanes, MMA M) and the 128 i of block I (columns, MMA N).
// Epilogue warp (quadrant q, part h) owns lanes 32q..32q+31 and columns
// 32h..32h+31: it accumulates the block-I row sums over its lanes in
// registers for the whole segment, and writes the block-J sums of an
// off-diagonal tile to colpart: added over the four parts h in shared memory
// to colpart[x * 128 + j] (d = 64), or apart to colpart[(x * 128 + j) * 4 + h].  At the end of a
// segment the row sums are reduced over the lanes and stored to
// rowpart[((I * slots + slot) * 4 + q) * 128 + i].
template <int DPAD>
__global__ void __launch_bounds__(MF_THREADS, 1)
k_mf_bf16x3(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
            const float* __restrict__ pf, MfSched sch, float* __restrict__ rowpart, float* __restrict__ colpart,
            int* __restrict__ err, const PcgScalars* sc) {
    if (sc != nullptr && *(volatile const int*)&sc->converged) return;   // uniform: fixed during the kernel
    using C = MfCfg<DPAD>;
    constexpr int TILE = C::TILE_BYTES;
    extern __shared__ __align__(1024) unsigned char mf_smem_raw[];
    unsigned char* base = mf_smem_raw;
    {   // align the dynamic window to 1024 bytes (swizzle-pattern repeat)
        const uint32_t a = smem_u32(base);
        base += (1024 - (a & 1023)) & 1023;
    }
    unsigned char* sB_hi = base;                  // fixed block I
    unsigned char* sB_lo = base + TILE;
    unsigned char* sA = base + 2 * TILE;          // stage s: hi at 2s, lo at 2s + 1 (streamed block J)
    MfSmem* S = reinterpret_cast<MfSmem*>(base + (2 + 2 * C::STAGES) * TILE);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x;
    const int64_t t0 = mf_tile_begin(g, sch);
    const int ntiles = (int)(mf_tile_begin(g + 1, sch) - t0);
    int I0 = 0, k0 = 0;
    mf_tile(t0, sch, I0, k0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(&S->full[s], 1); mbar_init(&S->empty[s], 1); }
        for (int a = 0; a < MF_NACC; ++a) { mbar_init(&S->tfull[a], 1); mbar_init(&S->tempty[a], MF_EPI_WARPS); }
        mbar_init(&S->bfull, 1);
        mbar_init(&S->bempty, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MF_EPI_WARPS + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(MF_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == MF_EPI_WARPS) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int issued = 0, seg = 0, I = I0, k = k0;
            for (int it = 0; it < ntiles; ++it) {
                if (it == 0 || k == 0) {   // new segment: reload the fixed block once the MMAs released it
                    if (seg > 0 && !mbar_wait(&S->bempty, (seg - 1) & 1, err)) break;
                    mbar_expect_tx(&S->bfull, 2 * TILE);
                    tma_load_2d(sB_hi, &map_hi, &S->bfull, 0, I * MF_B);
                    tma_load_2d(sB_lo, &map_lo, &S->bfull, 0, I * MF_B);
                    ++seg;
                }
                const int st = it % C::STAGES;
                const uint32_t ph = (it / C::STAGES) & 1;
                if (!mbar_wait(&S->empty[st], ph ^ 1, err)) break;
                const int J = (I + k) % sch.nb;
                unsigned char* a = sA + 2 * st * TILE;
                mbar_expect_tx(&S->full[st], 2 * TILE);
                tma_load_2d(a, &map_hi, &S->full[st], 0, J * MF_B);
                tma_load_2d(a + TILE, &map_lo, &S->full[st], 0, J * MF_B);
                issued = it + 1;
                if (++k == mf_row_len(I, sch)) { ++I; k = 0; }
            }
            // drain: every copy this CTA issued has landed before it may exit
            if (seg > 0) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->bfull, (seg - 1) & 1) && clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
            for (int it = max(0, issued - C::STAGES); it < issued; ++it) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->full[it % C::STAGES], (it / C::STAGES) & 1) &&
                       clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
        }
    } else if (warp == MF_EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc_bf16(MF_B, MF_B);
            // shared-memory descriptors built once: the start-address field is
            // the byte address / 16, so tile q of the ring is dA0 + q TILE / 16
            // and the K step kk (32 bytes) adds 2 (all addresses < 256 KB)
            const uint64_t dA0 = smem_desc(sA, C::SWZ, 0);
            const uint64_t dBh = smem_desc(sB_hi, C::SWZ, 0), dBl = smem_desc(sB_lo, C::SWZ, 0);
            int seg = 0, I = I0, k = k0;
            for (int it = 0; it < ntiles; ++it) {
                if (it == 0 || k == 0) {
                    if (seg > 0) umma_commit(&S->bempty);       // previous segment's MMAs release block I
                    if (!mbar_wait(&S->bfull, seg & 1, err)) break;
                    ++seg;
                }
                const int st = it % C::STAGES;
                const uint32_t ph = (it / C::STAGES) & 1;
                const int acc = it % MF_NACC;
                const uint32_t aph = (it / MF_NACC) & 1;
                if (!mbar_wait(&S->tempty[acc], aph ^ 1, err)) break;
                tc_fence_after();
                if (!mbar_wait(&S->full[st], ph, err)) break;
                tc_fence_after();
                const uint64_t dAh = dA0 + (uint64_t)((2 * st * TILE) >> 4), dAl = dAh + (uint64_t)(TILE >> 4);
                const uint32_t d = tmem + acc * MF_B;
#pragma unroll
                for (int kk = 0; kk < DPAD / 16; ++kk) {
                    const uint64_t o = 2 * kk;   // 16 bf16 = 32 bytes along K
                    umma_bf16(d, dAh + o, dBh + o, idesc, kk > 0 ? 1u : 0u);
                    umma_bf16(d, dAh + o, dBl + o, idesc, 1u);
                    umma_bf16(d, dAl + o, dBh + o, idesc, 1u);
                    umma_bf16(d, dAl + o, dBl + o, idesc, 1u);
                }
                umma_commit(&S->empty[st]);
                umma_commit(&S->tfull[acc]);
                if (++k == mf_row_len(I, sch)) { ++I; k = 0; }
            }
        }
    } else {
        // ---------------- epilogue: exp, row sums and column sums ----------------
        const int q = warp & 3, h = warp >> 2;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        float2 acc[MF_WCOLS / 2];
        const float4* pI4 = nullptr;   // p of this warp's 32 columns of block I (L1-resident)
        int I = I0, k = k0, segI = I0;
        auto load_seg = [&](int blk) {
            pI4 = reinterpret_cast<const float4*>(pf + (int64_t)blk * MF_B + h * MF_WCOLS);
#pragma unroll
            for (int c = 0; c < MF_WCOLS / 2; ++c) acc[c] = make_float2(0.f, 0.f);
        };
        auto flush = [&](int blk) {
            float a[MF_WCOLS];
#pragma unroll
            for (int c = 0; c < MF_WCOLS / 2; ++c) { a[2 * c] = acc[c].x; a[2 * c + 1] = acc[c].y; }
            mf_lane_reduce(a, lane);
            const int slot = g - mf_owner(mf_row_start(blk, sch), sch);
            rowpart[(((int64_t)blk * sch.slots + slot) * 4 + q) * MF_B + h * MF_WCOLS + lane] = a[0];
        };
        // once a bounded wait has expired (the error word is set) a warp skips
        // its waits and tensor-memory reads but runs on through the tiles, so
        // that the four warps of a quadrant still meet at every named barrier
        bool live = true;
        int noff = 0;   // off-diagonal tiles so far (the same in every warp)
        if (ntiles > 0) load_seg(I0);
        float pj_next = ntiles > 0 ? __ldg(pf + (int64_t)((I0 + k0) % sch.nb) * MF_B + q * 32 + lane) : 0.f;
        for (int it = 0; it < ntiles; ++it) {
            if (it > 0 && k == 0) {
                flush(segI);
                segI = I;
                load_seg(I);
            }
            const bool diag = (k == 0);
            const float pj = pj_next;
            int In = I, kn = k + 1;
            if (kn == mf_row_len(I, sch)) { ++In; kn = 0; }
            if (it + 1 < ntiles) pj_next = __ldg(pf + (int64_t)((In + kn) % sch.nb) * MF_B + q * 32 + lane);
            const int accb = it % MF_NACC;
            const uint32_t aph = (it / MF_NACC) & 1;
            if (live) {
                // one lane waits, the warp follows: tcgen05.ld below must run converged
                const int w = (lane == 0) ? (int)mbar_wait(&S->tfull[accb], aph, err) : 0;
                live = __shfl_sync(0xffffffffu, w, 0) != 0;
            }
            float2 sJ[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (live) {
                tc_fence_after();
                const uint32_t tcol = tmem + lane_addr + accb * MF_B + h * MF_WCOLS;
                if (diag) mf_tile_epilogue<true>(tcol, acc, pI4, pj, sJ);
                else mf_tile_epilogue<false>(tcol, acc, pI4, pj, sJ);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->tempty[accb]);
            }
            if (!diag) {
                const float part = (sJ[0].x + sJ[0].y) + (sJ[1].x + sJ[1].y);
                if (MfCfg<DPAD>::REDUCE) {
                    // the quadrant's four parts of a column are added in shared
                    // memory, in a fixed order, and written once: a quarter of
                    // the partial traffic of writing them apart.  The buffer
                    // alternates per off-diagonal tile, so that the barrier of
                    // the tile between two uses of a buffer orders part 0's
                    // reads before the next writes
                    float(*cr)[32] = S->cred[noff & 1][q];
                    ++noff;
                    cr[h][lane] = part;
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + q), "r"(32 * MF_EPW) : "memory");
                    if (h == 0)
                        colpart[(t0 + it) * MF_B + q * 32 + lane] =
                            (cr[0][lane] + cr[1][lane]) + (cr[2][lane] + cr[3][lane]);
                } else {
                    colpart[((t0 + it) * MF_B + q * 32 + lane) * MF_EPW + h] = part;
                }
            }
            I = In;
            k = kn;
        }
        if (ntiles > 0) flush(segI);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MF_EPI_WARPS + 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MF_TMEM_COLS)
                     : "memory");
    }
}

// p = z + beta p_old (or p = x), float64 copy to pout and zero-padded float32 copy.
__global__ void k_mf_prep(int64_t n, int64_t npad, const double* __restrict__ pin, const double* __restrict__ z,
                          double* __restrict__ pout, float* __restrict__ pf, const PcgScalars* sc, int fuse) {
    if (sc != nullptr && *(volatile const int*)&sc->converged) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) { pf[i] = 0.f; return; }
    // beta = 0 starts a new direction; p_old is not read (it may hold what a
    // broken-down step left)
    const double b = fuse ? sc->beta : 0.0;
    const double p = !fuse ? pin[i] : (b == 0.0 ? z[i] : fma(b, pin[i], z[i]));
    if (fuse) pout[i] = p;
    pf[i] = (float)p;
}

// w_i = lambda p_i + (block row I's segment partials over slots and lane
// quadrants) + (column sums of the off-diagonal tiles (I', I)).  CTA (I, cq)
// takes the 32 columns 32cq..32cq+31 of block row I with 16 groups of 32
// threads: group g adds the distances kk = 1 + g, 17 + g, ... and a share of
// the row partials; the groups are added in a fixed order.  p^T w -> delta in
// the last CTA.
constexpr int MF_FIN_COLS = 32;
static_assert(MF_EPW == 4, "the epilogue adds the four parts of a column in shared memory");
constexpr int MF_FIN_GROUPS = 16;
__global__ void __launch_bounds__(MF_FIN_GROUPS * MF_FIN_COLS)
k_mf_finish(int64_t n, MfSched sch, double lambda, const float* __restrict__ rowpart,
            const float* __restrict__ colpart, int parts, const int* __restrict__ nslots,
            const double* __restrict__ p, double* __restrict__ w, PcgScalars* sc, double* __restrict__ partials,
            const int* err) {
    if (sc != nullptr && *(volatile const int*)&sc->converged) return;
    __shared__ double red[MF_FIN_GROUPS * MF_FIN_COLS / 32];
    __shared__ float gsum[MF_FIN_GROUPS][MF_FIN_COLS];
    const int I = blockIdx.x;
    const int c = blockIdx.y * MF_FIN_COLS + (threadIdx.x % MF_FIN_COLS);
    const int grp = threadIdx.x / MF_FIN_COLS;
    // row partials: the (slot, quadrant) entries are spread over the groups
    float s = 0.f;
    {
        const int nslot = nslots[I];   // CTAs that own a segment of block row I
        for (int e = grp; e < 4 * nslot; e += MF_FIN_GROUPS)
            s += __ldg(rowpart + (((int64_t)I * sch.slots + e / 4) * 4 + (e % 4)) * MF_B + c);
    }
    // column sums of the tiles (I - kk, I): four independent loads in flight;
    // parts = 4: the epilogue's four parts of a column are one 16-byte load,
    // added in the epilogue's order
    float t[2] = {0.f, 0.f};
    const float4* cp4 = reinterpret_cast<const float4*>(colpart);
    for (int kb = 1 + grp; kb <= sch.base; kb += 4 * MF_FIN_GROUPS) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int kk = kb + u * MF_FIN_GROUPS;
            int Ip = I - kk;
            if (Ip < 0) Ip += sch.nb;
            const bool ok = kk <= sch.base && kk < mf_row_len(Ip, sch);
            const int64_t x = (mf_row_start(Ip, sch) + kk) * MF_B + c;
            if (!ok) {
                v[u] = 0.f;
            } else if (parts == 1) {
                v[u] = __ldg(colpart + x);
            } else {
                const float4 q4 = __ldg(cp4 + x);
                v[u] = (q4.x + q4.y) + (q4.z + q4.w);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u & 1] += v[u];
    }
    gsum[grp][threadIdx.x % MF_FIN_COLS] = s + (t[0] + t[1]);
    __syncthreads();
    const int64_t i = (int64_t)I * MF_B + c;
    double pw = 0.0;
    if (grp == 0 && i < n) {
        // four independent chains of four, added in a fixed order
        double q4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int gq = 0; gq < MF_FIN_GROUPS; ++gq) q4[gq & 3] += (double)gsum[gq][threadIdx.x];
        const double tot = (q4[0] + q4[1]) + (q4[2] + q4[3]);
        const double wi = fma(lambda, p[i], tot);
        w[i] = wi;
        pw = p[i] * wi;
    }
    if (sc == nullptr) return;
    // only group 0 (warp 0) holds nonzero terms: one warp reduces them
    if (grp == 0) pw = lk::warp_sum(pw);
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) partials[bid] = pw;
    if (lk::last_block(&sc->ticket[0])) {
        const double pAp = lk::sum_partials(partials, gridDim.x * gridDim.y, red);
        if (threadIdx.x == 0) {
            sc->pAp = pAp;
            if (*(volatile const int*)err != 0) {
                sc->converged = 2;
                sc->delta = 0.0;
            } else if (!(pAp > 0.0) || !isfinite(pAp)) {
                // mixed forms: the guard replaces the residual and rolls back
                if (sc->refine_every > 0) sc->breakdown = 1;
                else sc->converged = 2;
                sc->delta = 0.0;
            } else {
                sc->delta = sc->rz / pAp;
            }
            sc->iters += 1;
            sc->ticket[0] = 0;
        }
    }
}

// Dynamic shared memory per CTA; at least 120 KB so that one CTA holds an SM
// and its 512 tensor-memory columns never wait in alloc.
size_t mf_smem_bytes(int dpad) {
    const size_t tile = (size_t)MF_B * dpad * 2;
    const int stages = dpad >= 64 ? MfCfg<64>::STAGES : MfCfg<32>::STAGES;
    return std::max<size_t>(120 * 1024, 1024 + (2 + 2 * (size_t)stages) * tile + sizeof(MfSmem));
}

}  // namespace

// Workspace of the matrix-free operator, allocated at build time.
struct MfWork {
    CUtensorMap map_hi, map_lo;
    float* pf = nullptr;        // padded float32 p
    float* rowpart = nullptr;   // segment row sums (see k_mf_bf16x3)
    float* colpart = nullptr;   // column sums of off-diagonal tiles
    int* err = nullptr;         // device error word
    int* nslots = nullptr;      // per block row: number of CTAs owning a segment of it
    MfSched sch;
};

static void mf_release_work(MfWork* wk);

namespace {

laker_status mf_launch_main(laker_ctx* ctx, const laker_op* op, const MfWork* wk, const PcgScalars* sc) {
    const size_t smem = mf_smem_bytes(op->dpad);
    const unsigned grid = (unsigned)wk->sch.G;
#define LK_MF_LAUNCH(D)                                                                                        \
    k_mf_bf16x3<D><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch, wk->rowpart, \
                                                             wk->colpart, wk->err, sc)
    if (op->dpad == 16) LK_MF_LAUNCH(16);
    else if (op->dpad == 32) LK_MF_LAUNCH(32);
    else LK_MF_LAUNCH(64);
#undef LK_MF_LAUNCH
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

}  // namespace

laker_status mf_prepare(laker_ctx* ctx, laker_op* op) {
    if (!(op->dpad == 16 || op->dpad == 32 || op->dpad == 64))
        return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator supports d <= 64");
    auto encode = get_encode(ctx);
    if (!encode) return LAKER_ERR_CUDA;
    MfWork* wk = new MfWork();
    const int64_t n = op->n;
    MfSched& sc = wk->sch;
    sc.nb = (int)((n + MF_B - 1) / MF_B);
    sc.base = (sc.nb - 1) / 2 + 1;
    sc.half = (sc.nb % 2 == 0) ? sc.nb / 2 : 0;
    sc.T = (int64_t)sc.half * (sc.base + 1) + (int64_t)(sc.nb - sc.half) * sc.base;
    sc.G = (int)std::min<int64_t>(sc.T, (int64_t)ctx->num_sms);
    sc.slots = 1;
    for (int I = 0; I < sc.nb; ++I) {
        const int64_t x0 = mf_row_start(I, sc);
        sc.slots = std::max(sc.slots, mf_owner(x0 + mf_row_len(I, sc) - 1, sc) - mf_owner(x0, sc) + 1);
    }
    const int64_t npad = (int64_t)sc.nb * MF_B;
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&wk->pf, (size_t)npad * sizeof(float))) != LAKER_OK) { delete wk; return st; }
    if ((st = lk_malloc(ctx, (void**)&wk->rowpart, (size_t)sc.nb * sc.slots * 4 * MF_B * sizeof(float))) !=
        LAKER_OK) { mf_release_work(wk); return st; }
    if ((st = lk_malloc(ctx, (void**)&wk->colpart, (size_t)sc.T * (op->dpad >= 64 ? 1 : MF_EPW) * MF_B * sizeof(float))) != LAKER_OK) {
        mf_release_work(wk);
        return st;
    }
    if ((st = lk_malloc(ctx, (void**)&wk->err, sizeof(int))) != LAKER_OK) { mf_release_work(wk); return st; }
    {
        std::vector<int> ns((size_t)sc.nb);
        for (int I = 0; I < sc.nb; ++I) {
            const int64_t x0 = mf_row_start(I, sc);
            ns[(size_t)I] = mf_owner(x0 + mf_row_len(I, sc) - 1, sc) - mf_owner(x0, sc) + 1;
        }
        if ((st = lk_malloc(ctx, (void**)&wk->nslots, sizeof(int) * sc.nb)) != LAKER_OK) { mf_release_work(wk); return st; }
        LK_CUDA(ctx, cudaMemcpy(wk->nslots, ns.data(), sizeof(int) * sc.nb, cudaMemcpyHostToDevice));
    }
    LK_CUDA(ctx, cudaMemsetAsync(wk->err, 0, sizeof(int), ctx->stream));
    const cuuint64_t dims[2] = {(cuuint64_t)op->dpad, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)op->dpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)op->dpad, (cuuint32_t)MF_B};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle swz = op->dpad == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : op->dpad == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                    : CU_TENSOR_MAP_SWIZZLE_32B;
    for (int which = 0; which < 2; ++which) {
        CUresult r = encode(which == 0 ? &wk->map_hi : &wk->map_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                            which == 0 ? (void*)op->Qhi : (void*)op->Qlo, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            mf_release_work(wk);
            return set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled failed");
        }
    }
    const size_t smem = mf_smem_bytes(op->dpad);
    cudaError_t e;
    if (op->dpad == 16) e = cudaFuncSetAttribute(k_mf_bf16x3<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (op->dpad == 32) e = cudaFuncSetAttribute(k_mf_bf16x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(k_mf_bf16x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { mf_release_work(wk); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    op->mf = wk;
    return LAKER_OK;
}

static void mf_release_work(MfWork* wk) {
    if (!wk) return;
    cudaFree(wk->pf);
    cudaFree(wk->rowpart);
    cudaFree(wk->colpart);
    cudaFree(wk->err);
    cudaFree(wk->nslots);
    delete wk;
}

void mf_release(laker_op* op) {
    mf_release_work(static_cast<MfWork*>(op->mf));
    op->mf = nullptr;
}

laker_status mf_status(laker_ctx* ctx, const laker_op* op) {
    const MfWork* wk = static_cast<const MfWork*>(op->mf);
    if (!wk) return LAKER_OK;
    int h = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(&h, wk->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return h ? set_error(ctx, (laker_status)h, "matrix-free kernel: bounded wait expired") : LAKER_OK;
}

laker_status mf_matvec_launch(laker_ctx* ctx, const laker_op* op, const double* pin, const double* z, double* pout,
                              double* w, PcgScalars* sc, double* partials, int fuse, float*, float*) {
    const MfWork* wk = static_cast<const MfWork*>(op->mf);
    if (!wk) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator not prepared");
    const int64_t n = op->n;
    const int64_t npad = (int64_t)wk->sch.nb * MF_B;
    const double* p = fuse ? pout : pin;
    k_mf_prep<<<(unsigned)((npad + 255) / 256), 256, 0, ctx->stream>>>(n, npad, pin, z, pout, wk->pf, sc, fuse);
    LK_LAUNCHED(ctx);
    laker_status st = mf_launch_main(ctx, op, wk, sc);
    if (st != LAKER_OK) return st;
    k_mf_finish<<<dim3(wk->sch.nb, MF_B / MF_FIN_COLS), MF_FIN_GROUPS * MF_FIN_COLS, 0, ctx->stream>>>(n, wk->sch, op->lambda, wk->rowpart, wk->colpart, op->dpad >= 64 ? 1 : MF_EPW, wk->nslots, p, w, sc, partials,
                                             wk->err);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

laker_status mf_time_main(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    const MfWork* wk = static_cast<const MfWork*>(op->mf);
    if (!wk) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator not prepared");
    const int64_t n = op->n;
    const int64_t npad = (int64_t)wk->sch.nb * MF_B;
    k_mf_prep<<<(unsigned)((npad + 255) / 256), 256, 0, ctx->stream>>>(n, npad, x, nullptr, nullptr, wk->pf, nullptr,
                                                                       0);
    LK_LAUNCHED(ctx);
    cudaEvent_t e0, e1;
    LK_CUDA(ctx, cudaEventCreate(&e0));
    LK_CUDA(ctx, cudaEventCreate(&e1));
    laker_status st = LAKER_OK;
    for (int rep = -1; rep < reps && st == LAKER_OK; ++rep) {
        if (rep == 0) LK_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        st = mf_launch_main(ctx, op, wk, nullptr);
    }
    if (st == LAKER_OK) LK_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    if (st == LAKER_OK) LK_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0.f;
    if (st == LAKER_OK) LK_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LAKER_OK) return st;
    *ms = (double)t / reps;
    return mf_status(ctx, op);
}
