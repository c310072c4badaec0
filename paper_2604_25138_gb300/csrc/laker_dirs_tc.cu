// Random directions u_k = (lambda I + G) z_k (Sec. IV-B, Eq. random_directions)
// for mixed-precision operators, matrix-free on the tensor cores: G is never
// formed, each 128 x 128 tile of it is recomputed from the embeddings and used
// at once for all the directions of a chunk.
//
//   S_IJ = Q'_I Q'_J^T                (split-bf16 logits in log2 units, tcgen05)
//   P_IJ = 2^S_IJ                     (ex2, float32; P = G_IJ)
//   O_I += P_IJ Z~_J                  (P split as bf16 hi + lo, tcgen05)
//   U_I  = O_I + lambda Z~_I          (float64)
//
// Z~ is Z rounded to bf16 (round to nearest even): the directions are still
// standard-normal random vectors to 2^-9, and U is A Z~ for exactly those
// vectors, to ~1e-5 relative (the hi + lo split of P keeps 16 bits of it;
// the logits use the products hi.hi + hi.lo + lo.hi).  The caller normalises
// the columns.
//
// Kernel layout: one CTA per (block I of 128 rows, chunk of 128 directions),
// looping over every block J of 128 columns (one CTA per SM: 224 KB of shared
// memory at d = 64 and 512 tensor-memory columns).  Roles:
//   * a TMA warp streams Q'_J (hi, lo) and the tile of Z~^T (128 directions x
//     128 columns, two 64-column swizzled halves) through a 2-stage ring, after
//     loading Q'_I once;
//   * one thread issues the MMAs: S(t + 1) into the other half of a
//     double-buffered logit accumulator, then O += P_hi Z~ + P_lo Z~ for
//     step t once the epilogue has written P(t);
//   * eight epilogue warps (two per tensor-memory lane quadrant, 64 columns
//     each) read S with tcgen05.ld, take ex2, split P into bf16 hi / lo and
//     store them into shared memory in the 128-byte-swizzled K-major layout
//     the MMA reads (row i, 16-byte chunk c of a 64-column half at chunk
//     c xor (i mod 8)), then release them to the MMA through an mbarrier
//     after a generic-to-async proxy fence.  At the end they read O and write
//     U = O + lambda Z~ in float64.
// Every mbarrier wait is bounded: on timeout the kernel raises an error word,
// drains its own copies and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "laker_device.cuh"
#include "laker_tc.cuh"

namespace {

constexpr int DT_B = 128;                       // rows per block, columns per step, directions per chunk
constexpr int DT_EPI_WARPS = 8;                 // two per tensor-memory lane quadrant
constexpr int DT_THREADS = (DT_EPI_WARPS + 2) * 32;
constexpr int DT_STAGES = 2;
constexpr uint32_t DT_TMEM_COLS = 512;          // S[0], S[1], O (128 columns each)
constexpr int DT_HALF = DT_B * 64 * 2;          // 128 rows x 64 bf16 (128-byte rows): 16 KB

template <int DPAD>
struct DtCfg {
    static constexpr int QTILE = DT_B * DPAD * 2;     // one bf16 piece of 128 rows of Q'
    static constexpr int SWZ = DPAD * 2;
    static constexpr int STAGE = 2 * QTILE + 2 * DT_HALF;   // Q'_J hi, lo + Z~ tile
};

struct DtSmem {
    uint64_t full[DT_STAGES];
    uint64_t empty[DT_STAGES];
    uint64_t qfull;
    uint64_t sfull[2];
    uint64_t sempty[2];
    uint64_t pfull;
    uint64_t pempty;
    uint64_t ofull;
    uint32_t tmem_base;
};

size_t dt_smem_bytes(int dpad) {
    const size_t q = (size_t)DT_B * dpad * 2;
    return 1024 + 2 * q + DT_STAGES * (2 * q + 2 * DT_HALF) + 4 * DT_HALF + sizeof(DtSmem);
}

__device__ __forceinline__ float dt_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Byte offset of the 16-byte chunk c (0..7) of row r in a 128-row x 64-column
// bf16 half stored K-major with the 128-byte swizzle.
__device__ __forceinline__ uint32_t dt_swz(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

template <int DPAD>
__global__ void __launch_bounds__(DT_THREADS, 1)
k_dirs_tc(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
          const __grid_constant__ CUtensorMap map_zt, int64_t n, int nr, int nb, double lambda,
          const double* __restrict__ Z, double* __restrict__ U, int* __restrict__ err) {
    using C = DtCfg<DPAD>;
    extern __shared__ __align__(1024) unsigned char dt_smem_raw[];
    unsigned char* base = dt_smem_raw;
    {
        const uint32_t a = smem_u32(base);
        base += (1024 - (a & 1023)) & 1023;
    }
    unsigned char* sQI = base;                                   // hi, lo
    unsigned char* sStage = base + 2 * C::QTILE;                 // [stage]: Q'_J hi, lo, Z~ halves 0, 1
    unsigned char* sP = sStage + DT_STAGES * C::STAGE;           // P hi halves 0, 1; P lo halves 0, 1
    DtSmem* S = reinterpret_cast<DtSmem*>(sP + 4 * DT_HALF);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x;
    const int chunk = blockIdx.y;
    const int T = nb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < DT_STAGES; ++s) { mbar_init(&S->full[s], 1); mbar_init(&S->empty[s], 1); }
        mbar_init(&S->qfull, 1);
        for (int b = 0; b < 2; ++b) { mbar_init(&S->sfull[b], 1); mbar_init(&S->sempty[b], DT_EPI_WARPS); }
        mbar_init(&S->pfull, DT_EPI_WARPS);
        mbar_init(&S->pempty, 1);
        mbar_init(&S->ofull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == DT_EPI_WARPS + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S->tmem_base)),
                     "r"(DT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;
    const uint32_t tO = tmem + 2 * DT_B;

    if (warp == DT_EPI_WARPS) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int issued = 0;
            mbar_expect_tx(&S->qfull, 2 * C::QTILE);
            tma_load_2d(sQI, &map_hi, &S->qfull, 0, I * DT_B);
            tma_load_2d(sQI + C::QTILE, &map_lo, &S->qfull, 0, I * DT_B);
            for (int t = 0; t < T; ++t) {
                const int st = t % DT_STAGES;
                if (!mbar_wait(&S->empty[st], ((t / DT_STAGES) & 1) ^ 1, err)) break;
                unsigned char* g = sStage + st * C::STAGE;
                mbar_expect_tx(&S->full[st], C::STAGE);
                tma_load_2d(g, &map_hi, &S->full[st], 0, t * DT_B);
                tma_load_2d(g + C::QTILE, &map_lo, &S->full[st], 0, t * DT_B);
                tma_load_2d(g + 2 * C::QTILE, &map_zt, &S->full[st], t * DT_B, chunk * DT_B);
                tma_load_2d(g + 2 * C::QTILE + DT_HALF, &map_zt, &S->full[st], t * DT_B + 64, chunk * DT_B);
                issued = t + 1;
            }
            // drain: every copy this CTA issued has landed before it may exit
            {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->qfull, 0) && clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
            for (int t = max(0, issued - DT_STAGES); t < issued; ++t) {
                const long long c0 = clock64();
                while (!mbar_try_wait(&S->full[t % DT_STAGES], (t / DT_STAGES) & 1) && clock64() - c0 < TC_SPIN_CYCLES) {
                }
            }
        }
    } else if (warp == DT_EPI_WARPS + 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc_bf16(DT_B, DT_B);
            bool ok = mbar_wait(&S->qfull, 0, err);
            auto issue_S = [&](int t) -> bool {
                const int st = t % DT_STAGES;
                if (!mbar_wait(&S->full[st], (t / DT_STAGES) & 1, err)) return false;
                if (!mbar_wait(&S->sempty[t & 1], ((t >> 1) & 1) ^ 1, err)) return false;
                tc_fence_after();
                const unsigned char* qh = sStage + st * C::STAGE;
                const unsigned char* ql = qh + C::QTILE;
                const uint32_t d = tmem + (t & 1) * DT_B;
#pragma unroll
                for (int kk = 0; kk < DPAD / 16; ++kk) {
                    const int kb = kk * 32;
                    umma_bf16(d, smem_desc(sQI, C::SWZ, kb), smem_desc(qh, C::SWZ, kb), idesc, kk > 0 ? 1u : 0u);
                    umma_bf16(d, smem_desc(sQI, C::SWZ, kb), smem_desc(ql, C::SWZ, kb), idesc, 1u);
                    umma_bf16(d, smem_desc(sQI + C::QTILE, C::SWZ, kb), smem_desc(qh, C::SWZ, kb), idesc, 1u);
                }
                umma_commit(&S->sfull[t & 1]);
                return true;
            };
            if (ok && T > 0) ok = issue_S(0);
            for (int t = 0; ok && t < T; ++t) {
                if (t + 1 < T && !(ok = issue_S(t + 1))) break;
                if (!(ok = mbar_wait(&S->pfull, t & 1, err))) break;
                tc_fence_after();
                const unsigned char* zt = sStage + (t % DT_STAGES) * C::STAGE + 2 * C::QTILE;
#pragma unroll
                for (int piece = 0; piece < 2; ++piece) {
                    const unsigned char* pp = sP + piece * 2 * DT_HALF;
#pragma unroll
                    for (int kk = 0; kk < DT_B / 16; ++kk) {
                        const int half = kk >> 2, kb = (kk & 3) * 32;
                        umma_bf16(tO, smem_desc(pp + half * DT_HALF, 128, kb), smem_desc(zt + half * DT_HALF, 128, kb),
                                  idesc, (t > 0 || piece > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                umma_commit(&S->pempty);
                umma_commit(&S->empty[t % DT_STAGES]);
            }
            if (ok) umma_commit(&S->ofull);
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3, h = warp >> 2;      // lane quadrant, 64-column half
        const int r = q * 32 + lane;                 // row i within the block (tensor-memory lane)
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        const uint32_t pbase = smem_u32(sP) + h * DT_HALF;   // this warp's half of P hi; lo at + 2 halves
        bool ok = true;
        for (int t = 0; t < T; ++t) {
            int w = (lane == 0) ? (int)mbar_wait(&S->sfull[t & 1], (t >> 1) & 1, err) : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) { ok = false; break; }
            tc_fence_after();
            uint32_t v[64];
            const uint32_t ta = tmem + lane_addr + (t & 1) * DT_B + h * 64;
            tmem_ld16(ta, v);
            tmem_ld16(ta + 16, v + 16);
            tmem_ld16(ta + 32, v + 32);
            tmem_ld16(ta + 48, v + 48);
            tmem_wait(v);
            tmem_wait(v + 16);
            tmem_wait(v + 32);
            tmem_wait(v + 48);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->sempty[t & 1]);
            uint32_t hi[32], lo[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const float p0 = dt_ex2(__uint_as_float(v[2 * e])), p1 = dt_ex2(__uint_as_float(v[2 * e + 1]));
                hi[e] = pack_bf16(p0, p1);
                const float h0 = __uint_as_float(hi[e] << 16), h1 = __uint_as_float(hi[e] & 0xFFFF0000u);
                lo[e] = pack_bf16(p0 - h0, p1 - h1);
            }
            // P(t - 1) must have been read by its MMAs before it is overwritten
            w = (lane == 0) ? (int)mbar_wait(&S->pempty, (t & 1) ^ 1, err) : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) { ok = false; break; }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t off = dt_swz(r, c);
                sts128(pbase + off, hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
                sts128(pbase + 2 * DT_HALF + off, lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&S->pfull);
        }
        if (ok) {
            int w = (lane == 0) ? (int)mbar_wait(&S->ofull, 0, err) : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            if (w) {
                tc_fence_after();
                const int64_t i = (int64_t)I * DT_B + r;
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    uint32_t o[16];
                    tmem_ld16(tO + lane_addr + h * 64 + c4 * 16, o);
                    tmem_wait(o);
                    if (i < n) {
                        const int k0 = chunk * DT_B + h * 64 + c4 * 16;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int k = k0 + e;
                            if (k < nr) {
                                const double z = (double)__bfloat162float(__double2bfloat16(Z[i * nr + k]));
                                U[i * nr + k] = fma(lambda, z, (double)__uint_as_float(o[e]));
                            }
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == DT_EPI_WARPS + 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(DT_TMEM_COLS) : "memory");
    }
}

// Z (n x nr float64, row-major) -> Z~^T (nr x ldz bf16), rounded to nearest even
__global__ void k_zt_bf16(int64_t n, int nr, int64_t ldz, const double* __restrict__ Z, uint16_t* __restrict__ Zt) {
    __shared__ uint16_t tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
    for (int e = threadIdx.y; e < 32; e += blockDim.y) {
        const int64_t i = i0 + e, k = k0 + threadIdx.x;
        tile[e][threadIdx.x] = (i < n && k < nr) ? __bfloat16_as_ushort(__double2bfloat16(Z[i * nr + k])) : 0;
    }
    __syncthreads();
    for (int e = threadIdx.y; e < 32; e += blockDim.y) {
        const int64_t k = k0 + e, i = i0 + threadIdx.x;
        if (k < nr && i < ldz) Zt[k * ldz + i] = tile[threadIdx.x][e];
    }
}

}  // namespace

bool dirs_tc_supported(const laker_op* op) {
    return op->Qhi != nullptr && op->Qlo != nullptr && (op->dpad == 16 || op->dpad == 32 || op->dpad == 64) &&
           op->scale > 0.0;
}

// U (n x nr float64) = (lambda I + G) Z~ on the tensor cores (see the file header).
laker_status dirs_tc(laker_ctx* ctx, const laker_op* op, const double* Z, int nr, double* U) {
    if (!dirs_tc_supported(op)) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "tensor-core directions need d <= 64");
    auto encode = get_encode(ctx);
    if (!encode) return LAKER_ERR_CUDA;
    const int64_t n = op->n;
    const int nb = (int)((n + DT_B - 1) / DT_B);
    const int nch = (nr + DT_B - 1) / DT_B;
    const int64_t ldz = (n + 7) / 8 * 8;                       // 16-byte rows
    uint16_t* Zt = nullptr;
    int* err = nullptr;
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&Zt, (size_t)nr * ldz * 2)) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&err, sizeof(int))) != LAKER_OK) { cudaFree(Zt); return st; }
    struct Free { void* a; void* b; ~Free() { cudaFree(a); cudaFree(b); } } fr{Zt, err};
    LK_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    k_zt_bf16<<<dim3((unsigned)((ldz + 31) / 32), (unsigned)((nr + 31) / 32)), dim3(32, 8), 0, ctx->stream>>>(n, nr, ldz,
                                                                                                           Z, Zt);
    LK_LAUNCHED(ctx);
    CUtensorMap mh, ml, mz;
    const cuuint32_t estr[2] = {1, 1};
    {
        const cuuint64_t dims[2] = {(cuuint64_t)op->dpad, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)op->dpad * 2};
        const cuuint32_t box[2] = {(cuuint32_t)op->dpad, (cuuint32_t)DT_B};
        const CUtensorMapSwizzle swz = op->dpad == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                       : op->dpad == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                        : CU_TENSOR_MAP_SWIZZLE_32B;
        for (int which = 0; which < 2; ++which) {
            CUresult r = encode(which == 0 ? &mh : &ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                which == 0 ? (void*)op->Qhi : (void*)op->Qlo, dims, strides, box, estr,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled (Q) failed");
        }
    }
    {
        // Z~^T: inner dimension j (n columns, zero fill beyond), outer k (nr rows)
        const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)nr};
        const cuuint64_t strides[1] = {(cuuint64_t)ldz * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)DT_B};
        CUresult r = encode(&mz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Zt, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return set_error(ctx, LAKER_ERR_CUDA, "cuTensorMapEncodeTiled (Z) failed");
    }
    const size_t smem = dt_smem_bytes(op->dpad);
    const dim3 grid((unsigned)nb, (unsigned)nch);
#define LK_DT_LAUNCH(D)                                                                                            \
    do {                                                                                                           \
        cudaError_t e_ = cudaFuncSetAttribute(k_dirs_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e_ != cudaSuccess) return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e_));                     \
        k_dirs_tc<D><<<grid, DT_THREADS, smem, ctx->stream>>>(mh, ml, mz, n, nr, nb, op->lambda, Z, U, err);       \
    } while (0)
    if (op->dpad == 16) LK_DT_LAUNCH(16);
    else if (op->dpad == 32) LK_DT_LAUNCH(32);
    else LK_DT_LAUNCH(64);
#undef LK_DT_LAUNCH
    LK_LAUNCHED(ctx);
    int herr = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_error(ctx, (laker_status)herr, "tensor-core directions: bounded wait expired");
    return LAKER_OK;
}
