// Matrix-free operator  w = (lambda I + G) p,  G_ij = 2^(q'_i . q'_j)  with
// q' = q sqrt(scale log2 e)  (Sec. III-A Eq. sc-exp-kernel; the matvec-only
// access of Sec. IV-D, remark after Eq. kernel_shrinkage_cccp_normalization).
//
// Blackwell (sm_103a) kernel, one CTA per (128-row block, slice of columns):
//   * TMA (cp.async.bulk.tensor) streams 128-row tiles of the split-bf16
//     operands q' = hi + lo into a 4-stage shared-memory ring;
//   * one elected thread issues tcgen05.mma (kind::f16, bf16 in, f32 out) for
//     the split product  hi_i.hi_j + hi_i.lo_j + lo_i.hi_j + lo_i.lo_j  into a
//     double-buffered 128 x 128 float32 accumulator in tensor memory.  The
//     fourth product makes the logits the exact Gram matrix of the rounded
//     embedding hi + lo, so the computed kernel is exp of a Gram matrix and
//     stays positive semidefinite (Schur product theorem): without it the
//     operator error (~1e-6 n) exceeds lambda at n = 16384 and CG breaks down;
//   * eight epilogue warps read the logits with tcgen05.ld, apply ex2.approx
//     (the MUFU unit, 32 results/clk/SM on GB300) and accumulate e * p_j in
//     registers, overlapping the tensor-core work of the next tile.
// The grid is one wave of persistent CTAs (two per SM) over equal contiguous
// ranges of the row-block-major tile order; per-segment row sums go to a
// partial buffer and a finishing kernel adds lambda p, sums a row's partials
// in a fixed order and performs the PCG p^T w reduction.
// Every mbarrier wait is bounded; on timeout the kernel raises an error word,
// drains its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "laker_device.cuh"

namespace {

constexpr int MF_ROWS = 128;        // rows per CTA = tensor-memory lanes
constexpr int MF_COLS = 128;        // columns per tile = MMA N
constexpr int MF_STAGES = 4;
constexpr int MF_EPI_WARPS = 8;
constexpr int MF_THREADS = (MF_EPI_WARPS + 2) * 32;
constexpr uint32_t MF_TMEM_COLS = 2 * MF_COLS;
constexpr long long MF_SPIN_CYCLES = 4000000000ll;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after MF_SPIN_CYCLES or once another thread raised *err.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > MF_SPIN_CYCLES) {
            atomicExch(err, LAKER_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor, K-major operand with a swizzle of
// `swz_bytes` (32/64/128) per row: SBO = 8 rows, LBO unused for swizzled
// K-major layouts, fixed version bits 46..48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(const void* tile, int swz_bytes, int kbyte_offset) {
    const uint32_t addr = smem_u32(tile) + kbyte_offset;
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);                 // start address
    d |= (uint64_t)1 << 16;                                   // leading byte offset (unused)
    d |= (uint64_t)((8 * swz_bytes) >> 4) << 32;              // stride byte offset
    d |= (uint64_t)1 << 46;                                   // version
    const uint64_t mode = (swz_bytes == 128) ? 2 : (swz_bytes == 64) ? 4 : 6;
    d |= mode << 61;
    return d;
}

// Instruction descriptor for kind::f16: D f32, A/B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive float32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct MfSmem {
    // operand tiles first (1024-byte aligned by construction)
    // [A_hi][A_lo][stage0 B_hi][stage0 B_lo]...[stage S-1 B_lo]
    uint64_t full[MF_STAGES];
    uint64_t empty[MF_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t afull;
    uint64_t aempty;
    uint32_t tmem_base;
};

// Static schedule: the T = row_blocks x col_tiles tiles, in row-block-major
// order, are split into G equal contiguous ranges, one per CTA (2 CTAs per SM,
// one wave).  A range crossing a row-block boundary is processed as segments;
// each segment's row sums go to part[((rb * slots + slot) * 2 + half) * 128 + r]
// with slot = CTA index - first CTA touching row block rb.
struct MfSched {
    int64_t T;
    int G;
    int CT;      // column tiles per row block
    int slots;   // max CTAs touching one row block
};
__host__ __device__ __forceinline__ int64_t mf_tile_begin(int64_t g, const MfSched& s) { return g * s.T / s.G; }
__host__ __device__ __forceinline__ int mf_owner(int64_t x, const MfSched& s) {
    int g = (int)((x * s.G) / s.T);
    while (g + 1 < s.G && mf_tile_begin(g + 1, s) <= x) ++g;
    while (g > 0 && mf_tile_begin(g, s) > x) --g;
    return g;
}

template <int DPAD>
__global__ void __launch_bounds__(MF_THREADS, 2)
k_mf_bf16x3(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
            const float* __restrict__ pf, MfSched sch, float* __restrict__ part, int* __restrict__ err,
            const PcgScalars* sc) {
    if (sc != nullptr && *(volatile const int*)&sc->converged) return;   // uniform: fixed during the kernel
    constexpr int TILE_BYTES = MF_ROWS * DPAD * 2;             // one bf16 operand tile
    constexpr int SWZ = DPAD * 2;                              // swizzle span = row bytes
    extern __shared__ __align__(1024) unsigned char mf_smem_raw[];
    unsigned char* base = mf_smem_raw;
    {   // align the dynamic window to 1024 bytes (swizzle-pattern repeat)
        const uint32_t a = smem_u32(base);
        base += (1024 - (a & 1023)) & 1023;
    }
    unsigned char* sA_hi = base;
    unsigned char* sA_lo = base + TILE_BYTES;
    unsigned char* sB = base + 2 * TILE_BYTES;                 // stage s: hi at 2s, lo at 2s+1
    MfSmem* S = reinterpret_cast<MfSmem*>(base + (2 + 2 * MF_STAGES) * TILE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x;
    const int64_t t0 = mf_tile_begin(g, sch);
    const int ntiles = (int)(mf_tile_begin(g + 1, sch) - t0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < MF_STAGES; ++s) { mbar_init(&S->full[s], 1); mbar_init(&S->empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&S->tfull[a], 1); mbar_init(&S->tempty[a], MF_EPI_WARPS); }
        mbar_init(&S->afull, 1);
        mbar_init(&S->aempty, 1);
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
            int issued = 0, seg = 0, cur_rb = -1;
            bool ok = true;
            for (int it = 0; ok && it < ntiles; ++it) {
                const int64_t x = t0 + it;
                const int rb = (int)(x / sch.CT), ct = (int)(x % sch.CT);
                if (rb != cur_rb) {   // new segment: reload the row-block operand once it is free
                    if (seg > 0 && !mbar_wait(&S->aempty, (seg - 1) & 1, err)) { ok = false; break; }
                    mbar_expect_tx(&S->afull, 2 * TILE_BYTES);
                    tma_load_2d(sA_hi, &map_hi, &S->afull, 0, rb * MF_ROWS);
                    tma_load_2d(sA_lo, &map_lo, &S->afull, 0, rb * MF_ROWS);
                    cur_rb = rb;
                    ++seg;
                }
                const int st = it % MF_STAGES;
                const uint32_t ph = (it / MF_STAGES) & 1;
                if (!mbar_wait(&S->empty[st], ph ^ 1, err)) { ok = false; break; }
                unsigned char* b = sB + 2 * st * TILE_BYTES;
                mbar_expect_tx(&S->full[st], 2 * TILE_BYTES);
                tma_load_2d(b, &map_hi, &S->full[st], 0, ct * MF_COLS);
                tma_load_2d(b + TILE_BYTES, &map_lo, &S->full[st], 0, ct * MF_COLS);
                issued = it + 1;
            }
            // drain: every copy this CTA issued has landed before it may exit
            if (seg > 0) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->afull, (seg - 1) & 1) && clock64() - c0 < MF_SPIN_CYCLES) {
                }
            }
            for (int it = max(0, issued - MF_STAGES); it < issued; ++it) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->full[it % MF_STAGES], (it / MF_STAGES) & 1) &&
                       clock64() - c0 < MF_SPIN_CYCLES) {
                }
            }
        }
    } else if (warp == MF_EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc_bf16(MF_ROWS, MF_COLS);
            int seg = 0, cur_rb = -1;
            for (int it = 0; it < ntiles; ++it) {
                const int rb = (int)((t0 + it) / sch.CT);
                if (rb != cur_rb) {
                    if (seg > 0) umma_commit(&S->aempty);       // previous segment's MMAs release A
                    if (!mbar_wait(&S->afull, seg & 1, err)) break;
                    cur_rb = rb;
                    ++seg;
                }
                const int st = it % MF_STAGES;
                const uint32_t ph = (it / MF_STAGES) & 1;
                const int acc = it & 1;
                const uint32_t aph = (it >> 1) & 1;
                if (!mbar_wait(&S->tempty[acc], aph ^ 1, err)) break;
                tc_fence_after();
                if (!mbar_wait(&S->full[st], ph, err)) break;
                const unsigned char* bh = sB + 2 * st * TILE_BYTES;
                const unsigned char* bl = bh + TILE_BYTES;
                const uint32_t d = tmem + acc * MF_COLS;
#pragma unroll
                for (int k = 0; k < DPAD / 16; ++k) {
                    const int kb = k * 32;   // 16 bf16 = 32 bytes along K
                    umma_bf16(d, smem_desc(sA_hi, SWZ, kb), smem_desc(bh, SWZ, kb), idesc, k > 0 ? 1u : 0u);
                    umma_bf16(d, smem_desc(sA_hi, SWZ, kb), smem_desc(bl, SWZ, kb), idesc, 1u);
                    umma_bf16(d, smem_desc(sA_lo, SWZ, kb), smem_desc(bh, SWZ, kb), idesc, 1u);
                    umma_bf16(d, smem_desc(sA_lo, SWZ, kb), smem_desc(bl, SWZ, kb), idesc, 1u);
                }
                umma_commit(&S->empty[st]);
                umma_commit(&S->tfull[acc]);
            }
        }
    } else {
        // ---------------- epilogue: exp and row sums ----------------
        const int quad = warp & 3, half = warp >> 2;
        const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
        const int r = quad * 32 + lane;
        float acc4[4] = {0.f, 0.f, 0.f, 0.f};   // four independent FMA chains
        int cur_rb = ntiles > 0 ? (int)(t0 / sch.CT) : 0;
        auto flush = [&](int rb) {   // no barrier: each column half writes its own partial
            const int slot = g - mf_owner((int64_t)rb * sch.CT, sch);
            part[(((int64_t)rb * sch.slots + slot) * 2 + half) * MF_ROWS + r] =
                (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
            acc4[0] = acc4[1] = acc4[2] = acc4[3] = 0.f;
        };
        for (int it = 0; it < ntiles; ++it) {
            const int64_t x = t0 + it;
            const int rb = (int)(x / sch.CT), ct = (int)(x % sch.CT);
            if (rb != cur_rb) {
                flush(cur_rb);
                cur_rb = rb;
            }
            const int acc = it & 1;
            const uint32_t aph = (it >> 1) & 1;
            // one lane waits, the warp follows: tcgen05.ld below must run converged
            int ok = (lane == 0) ? (int)mbar_wait(&S->tfull[acc], aph, err) : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int jbase = ct * MF_COLS + half * 64;
#pragma unroll
            for (int c = 0; c < 64; c += 32) {
                float v[32];
                tmem_ld32(tmem + lane_addr + acc * MF_COLS + half * 64 + c, v);
                const float4* pp = reinterpret_cast<const float4*>(pf + jbase + c);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 p4 = __ldg(pp + u);
                    acc4[0] = fmaf(ex2_approx(v[4 * u + 0]), p4.x, acc4[0]);
                    acc4[1] = fmaf(ex2_approx(v[4 * u + 1]), p4.y, acc4[1]);
                    acc4[2] = fmaf(ex2_approx(v[4 * u + 2]), p4.z, acc4[2]);
                    acc4[3] = fmaf(ex2_approx(v[4 * u + 3]), p4.w, acc4[3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->tempty[acc]);
        }
        if (ntiles > 0) flush(cur_rb);
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
    const double p = fuse ? fma(sc->beta, pin[i], z[i]) : pin[i];
    if (fuse) pout[i] = p;
    pf[i] = (float)p;
}

// w = lambda p + the row's segment partials (fixed order); p^T w -> delta in the last block.
__global__ void __launch_bounds__(256)
k_mf_finish(int64_t n, MfSched sch, double lambda, const float* __restrict__ part, const double* __restrict__ p,
            double* __restrict__ w, PcgScalars* sc, double* __restrict__ partials, const int* err) {
    if (sc != nullptr && *(volatile const int*)&sc->converged) return;
    __shared__ double red[8];
    const int64_t R = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = min(n, (int64_t)blockIdx.x * R), r1 = min(n, r0 + R);
    double pw = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const int rb = (int)(i / MF_ROWS), r = (int)(i % MF_ROWS);
        const int64_t x0 = (int64_t)rb * sch.CT;
        const int g0 = mf_owner(x0, sch), g1 = mf_owner(x0 + sch.CT - 1, sch);
        double s = 0.0;
        for (int slot = 0; slot <= g1 - g0; ++slot)
            for (int h = 0; h < 2; ++h)
                s += (double)part[(((int64_t)rb * sch.slots + slot) * 2 + h) * MF_ROWS + r];
        const double wi = fma(lambda, p[i], s);
        w[i] = wi;
        pw = fma(p[i], wi, pw);
    }
    if (sc == nullptr) return;
    pw = lk::block_sum(pw, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = pw;
    if (lk::last_block(&sc->ticket[0])) {
        const double pAp = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->pAp = pAp;
            if (*(volatile const int*)err != 0 || !(pAp > 0.0) || !isfinite(pAp)) {
                sc->converged = 2;
                sc->delta = 0.0;
            } else {
                sc->delta = sc->rz / pAp;
            }
            sc->iters += 1;
            sc->ticket[0] = 0;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode(laker_ctx* ctx) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || p == nullptr) {
        set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled not available");
        return nullptr;
    }
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return fn;
}

// Dynamic shared memory per CTA; at least 80 KB so that at most two CTAs
// share an SM and their 2 x 256 tensor-memory columns never wait in alloc.
size_t mf_smem_bytes(int dpad) {
    const size_t tile = (size_t)MF_ROWS * dpad * 2;
    return std::max<size_t>(80 * 1024, 1024 + (2 + 2 * MF_STAGES) * tile + sizeof(MfSmem));
}

}  // namespace

// Workspace of the matrix-free operator, allocated at build time.
struct MfWork {
    CUtensorMap map_hi, map_lo;
    float* pf = nullptr;       // padded float32 p
    float* part = nullptr;     // segment partial row sums (see MfSched)
    int* err = nullptr;        // device error word
    MfSched sch;
    int col_tiles = 0;
};

laker_status mf_prepare(laker_ctx* ctx, laker_op* op) {
    if (!(op->dpad == 16 || op->dpad == 32 || op->dpad == 64))
        return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator supports d <= 64");
    auto encode = get_encode(ctx);
    if (!encode) return LAKER_ERR_CUDA;
    MfWork* wk = new MfWork();
    const int64_t n = op->n;
    const int64_t npad = (n + MF_COLS - 1) / MF_COLS * MF_COLS;
    wk->col_tiles = (int)(npad / MF_COLS);
    const int row_blocks = (int)((n + MF_ROWS - 1) / MF_ROWS);
    MfSched& sc = wk->sch;
    sc.CT = wk->col_tiles;
    sc.T = (int64_t)row_blocks * sc.CT;
    sc.G = (int)std::min<int64_t>(sc.T, 2 * (int64_t)ctx->num_sms);
    sc.slots = 1;
    for (int rb = 0; rb < row_blocks; ++rb) {
        const int64_t x0 = (int64_t)rb * sc.CT;
        sc.slots = std::max(sc.slots, mf_owner(x0 + sc.CT - 1, sc) - mf_owner(x0, sc) + 1);
    }
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&wk->pf, (size_t)npad * sizeof(float))) != LAKER_OK) { delete wk; return st; }
    if ((st = lk_malloc(ctx, (void**)&wk->part, (size_t)row_blocks * sc.slots * 2 * MF_ROWS * sizeof(float))) !=
        LAKER_OK) { delete wk; return st; }
    if ((st = lk_malloc(ctx, (void**)&wk->err, sizeof(int))) != LAKER_OK) { delete wk; return st; }
    LK_CUDA(ctx, cudaMemsetAsync(wk->err, 0, sizeof(int), ctx->stream));
    const cuuint64_t dims[2] = {(cuuint64_t)op->dpad, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)op->dpad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)op->dpad, (cuuint32_t)MF_ROWS};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle swz = op->dpad == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : op->dpad == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                    : CU_TENSOR_MAP_SWIZZLE_32B;
    for (int which = 0; which < 2; ++which) {
        CUresult r = encode(which == 0 ? &wk->map_hi : &wk->map_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                            which == 0 ? (void*)op->Qhi : (void*)op->Qlo, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) { delete wk; return set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled failed"); }
    }
    const size_t smem = mf_smem_bytes(op->dpad);
    cudaError_t e;
    if (op->dpad == 16) e = cudaFuncSetAttribute(k_mf_bf16x3<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (op->dpad == 32) e = cudaFuncSetAttribute(k_mf_bf16x3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(k_mf_bf16x3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { delete wk; return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    op->mf = wk;
    return LAKER_OK;
}

void mf_release(laker_op* op) {
    MfWork* wk = static_cast<MfWork*>(op->mf);
    if (!wk) return;
    cudaFree(wk->pf);
    cudaFree(wk->part);
    cudaFree(wk->err);
    delete wk;
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
    const int64_t npad = (int64_t)wk->col_tiles * MF_COLS;
    const double* p = fuse ? pout : pin;
    k_mf_prep<<<(unsigned)((npad + 255) / 256), 256, 0, ctx->stream>>>(n, npad, pin, z, pout, wk->pf, sc, fuse);
    LK_LAUNCHED(ctx);
    const size_t smem = mf_smem_bytes(op->dpad);
    const unsigned grid = (unsigned)wk->sch.G;
    if (op->dpad == 16)
        k_mf_bf16x3<16><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch, wk->part,
                                                                 wk->err, sc);
    else if (op->dpad == 32)
        k_mf_bf16x3<32><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch, wk->part,
                                                                 wk->err, sc);
    else
        k_mf_bf16x3<64><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch, wk->part,
                                                                 wk->err, sc);
    LK_LAUNCHED(ctx);
    const int fb = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 2 * ctx->num_sms);
    k_mf_finish<<<fb, 256, 0, ctx->stream>>>(n, wk->sch, op->lambda, wk->part, p, w, sc, partials, wk->err);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

laker_status mf_time_main(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    const MfWork* wk = static_cast<const MfWork*>(op->mf);
    if (!wk) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matrix-free operator not prepared");
    const int64_t n = op->n;
    const int64_t npad = (int64_t)wk->col_tiles * MF_COLS;
    k_mf_prep<<<(unsigned)((npad + 255) / 256), 256, 0, ctx->stream>>>(n, npad, x, nullptr, nullptr, wk->pf, nullptr,
                                                                       0);
    LK_LAUNCHED(ctx);
    const size_t smem = mf_smem_bytes(op->dpad);
    const unsigned grid = (unsigned)wk->sch.G;
    cudaEvent_t e0, e1;
    LK_CUDA(ctx, cudaEventCreate(&e0));
    LK_CUDA(ctx, cudaEventCreate(&e1));
    for (int rep = -1; rep < reps; ++rep) {
        if (rep == 0) LK_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        if (op->dpad == 16)
            k_mf_bf16x3<16><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch,
                                                                     wk->part, wk->err, nullptr);
        else if (op->dpad == 32)
            k_mf_bf16x3<32><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch,
                                                                     wk->part, wk->err, nullptr);
        else
            k_mf_bf16x3<64><<<grid, MF_THREADS, smem, ctx->stream>>>(wk->map_hi, wk->map_lo, wk->pf, wk->sch,
                                                                     wk->part, wk->err, nullptr);
        LK_LAUNCHED(ctx);
    }
    LK_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    LK_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0.f;
    LK_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / reps;
    return mf_status(ctx, op);
}
