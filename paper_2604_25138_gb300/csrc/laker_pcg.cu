// Preconditioned conjugate gradient on GB300 (Sec. IV-E, Algorithm 1, PCG stage).
//
// One PCG iteration is a fixed sequence of kernels, all reading their scalars
// from device memory so that a block of iterations is captured once into a
// CUDA graph and replayed; the host only polls a convergence word between
// replays:
//
//   MV   p = z + beta p_old (fused prologue), w = (lambda I + G) p,
//        p^T w  -> last block: delta = r.z / p^T A p
//        (materialised: a stream of G; matrix-free: prep, tcgen05 kernel, finish)
//   UPD  alpha += delta p, r -= delta w, |r|^2 -> last block: stop test
//   [TR1, TR2]  only when a float64-accurate residual is due (mixed forms):
//        w2 = (lambda I + G) alpha in compensated double-float, r = y - w2
//        replaces the recursive residual (reliable updates), stop test on |r|
//   UTR  t = U^T r as partial sums over row chunks (CCCP preconditioner)
//   PRE  z = P r, r^T z -> last block: beta = r.z_new / r.z_old
//
// The replaced residual must be accurate well below the tolerance: near
// convergence |G_ij alpha_j| ~ 1e4 terms cancel to O(1) sums, and a residual
// with ~1e-7 noise (plain double-float Dot2) was observed to make the
// replacements diverge at kappa ~ 1e8; the Dot3 evaluation keeps it ~1e-8.
//
// All cross-block sums go through per-block partials reduced in a fixed order
// by the last block to finish (atomic ticket), so results are deterministic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "laker_device.cuh"
#include "laker_df.cuh"

namespace {

constexpr int MV_THREADS = 512;
constexpr int VEC_THREADS = 256;

enum Gate { GATE_NONE = 0, GATE_RUNNING = 1, GATE_TRUE = 2 };

__device__ __forceinline__ bool gated_out(const PcgScalars* sc, int gate) {
    if (gate == GATE_NONE || sc == nullptr) return false;
    const int conv = *(volatile const int*)&sc->converged;
    if (conv != 0) return true;
    if (gate == GATE_TRUE) return *(volatile const int*)&sc->need_true == 0;
    return false;
}

// ---------------------------------------------------------------------------
// MV: materialised operator.  Block b owns rows [r0, r1); p is staged in
// shared memory column chunk by column chunk (converted to the storage type of
// G), each warp streams whole rows of G with 16-byte loads and keeps the
// running row sums in shared memory across chunks.
// ---------------------------------------------------------------------------
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int N = 2; };

template <typename T>
__device__ __forceinline__ T dot16(const typename Vec16<T>::type& a, const T* p);
template <>
__device__ __forceinline__ float dot16<float>(const float4& a, const float* p) {
    const float4 b = *reinterpret_cast<const float4*>(p);
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
template <>
__device__ __forceinline__ double dot16<double>(const double2& a, const double* p) {
    const double2 b = *reinterpret_cast<const double2*>(p);
    return fma(a.x, b.x, a.y * b.y);
}

template <typename T, bool STREAM>
__device__ __forceinline__ typename Vec16<T>::type ldk16(const typename Vec16<T>::type* p) {
    if (STREAM) return __ldcs(p);   // G larger than L2: evict-first
    return __ldg(p);                // G L2-resident across iterations
}

// gate: skip when converged (GATE_RUNNING) or when no true residual is due
// (GATE_TRUE); reduce: p^T w -> delta in the last block.
template <typename T, bool STREAM>
__global__ void __launch_bounds__(MV_THREADS)
k_matvec_mat(const T* __restrict__ K, int64_t ldk, int64_t n, double lambda, int64_t chunk,
             const double* __restrict__ pin, const double* __restrict__ z, double* __restrict__ pout,
             int fuse, double* __restrict__ w, PcgScalars* sc, double* __restrict__ partials, int gate,
             int reduce) {
    if (gated_out(sc, gate)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
    T* ps = reinterpret_cast<T*>(smraw);
    double* acc = reinterpret_cast<double*>(smraw + chunk * sizeof(T));
    __shared__ double red[MV_THREADS / 32];
    const double beta = fuse ? sc->beta : 0.0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) acc[i] = 0.0;

    constexpr int VN = Vec16<T>::N;
    using V = typename Vec16<T>::type;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t clen = min(chunk, n - c0);
        const int64_t cpad = (clen + VN - 1) / VN * VN;   // ldk padding is zero in G
        __syncthreads();
        for (int64_t j = threadIdx.x; j < cpad; j += blockDim.x) {
            const int64_t gj = c0 + j;
            double v = 0.0;
            if (gj < n) v = fuse ? fma(beta, pin[gj], z[gj]) : pin[gj];
            ps[j] = (T)v;
        }
        __syncthreads();
        const int64_t nv = cpad / VN;
        for (int rr = wid; rr < nrows; rr += nw) {
            const V* row = reinterpret_cast<const V*>(K + (r0 + rr) * ldk + c0);
            T s = T(0);
            int64_t v = lane;
            for (; v + 3 * 32 < nv; v += 4 * 32) {
                const V a0 = ldk16<T, STREAM>(row + v), a1 = ldk16<T, STREAM>(row + v + 32);
                const V a2 = ldk16<T, STREAM>(row + v + 64), a3 = ldk16<T, STREAM>(row + v + 96);
                s += dot16<T>(a0, ps + v * VN) + dot16<T>(a1, ps + (v + 32) * VN) +
                     dot16<T>(a2, ps + (v + 64) * VN) + dot16<T>(a3, ps + (v + 96) * VN);
            }
            for (; v < nv; v += 32) s += dot16<T>(ldk16<T, STREAM>(row + v), ps + v * VN);
            s = lk::warp_sum(s);
            if (lane == 0) acc[rr] += (double)s;
        }
    }
    __syncthreads();
    // epilogue: w = G p + lambda p, p^T w, and p_new for the owned rows
    double pw = 0.0;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        const int64_t gi = r0 + i;
        const double pi = !fuse ? pin[gi] : (beta == 0.0 ? z[gi] : fma(beta, pin[gi], z[gi]));
        const double wi = fma(lambda, pi, acc[i]);
        w[gi] = wi;
        if (fuse) pout[gi] = pi;
        pw = fma(pi, wi, pw);
    }
    if (sc == nullptr || !reduce) return;
    pw = lk::block_sum(pw, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = pw;
    if (lk::last_block(&sc->ticket[0])) {
        const double pAp = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->pAp = pAp;
            if (!(pAp > 0.0) || !isfinite(pAp)) {
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

// ---------------------------------------------------------------------------
// Float64-accurate product with G stored as the float32 pair (hi, lo):
// w = lambda x + (hi + lo) x in compensated (Dot3) arithmetic on the float32
// pipes.  8 bytes of G per entry, like float64, but HBM-bound instead of
// float64-FMA-bound on GB300.  Used for the true residual of mixed solves.
// ---------------------------------------------------------------------------
__device__ __forceinline__ lk::df2 warp_sum_df(lk::df2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lk::df2 u;
        u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = lk::df_add(v, u);
    }
    return v;
}

__global__ void __launch_bounds__(MV_THREADS)
k_matvec_df(const float* __restrict__ Khi, const float* __restrict__ Klo, int64_t ldk, int64_t n, double lambda,
            int64_t chunk, const double* __restrict__ x, double* __restrict__ w, const PcgScalars* sc, int gate) {
    if (gated_out(sc, gate)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    const int nrows = r1 > r0 ? (int)(r1 - r0) : 0;
    float2* xs = reinterpret_cast<float2*>(smraw);
    double* acc = reinterpret_cast<double*>(smraw + chunk * sizeof(float2));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) acc[i] = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int64_t clen = min(chunk, n - c0);
        const int64_t cpad = (clen + 3) / 4 * 4;
        __syncthreads();
        for (int64_t j = threadIdx.x; j < cpad; j += blockDim.x) {
            const int64_t gj = c0 + j;
            const lk::df2 v = lk::df_from(gj < n ? x[gj] : 0.0);
            xs[j] = make_float2(v.hi, v.lo);
        }
        __syncthreads();
        const int64_t nv = cpad / 4;
        for (int rr = wid; rr < nrows; rr += nw) {
            const float4* rh = reinterpret_cast<const float4*>(Khi + (r0 + rr) * ldk + c0);
            const float4* rl = reinterpret_cast<const float4*>(Klo + (r0 + rr) * ldk + c0);
            lk::Dot3 d0, d1;
            int64_t v = lane;
            for (; v + 32 < nv; v += 64) {
                const float4 a0 = __ldcs(rh + v), b0 = __ldcs(rl + v);
                const float4 a1 = __ldcs(rh + v + 32), b1 = __ldcs(rl + v + 32);
                const float2* p0 = xs + 4 * v;
                const float2* p1 = xs + 4 * (v + 32);
                d0.add({a0.x, b0.x}, {p0[0].x, p0[0].y});
                d1.add({a1.x, b1.x}, {p1[0].x, p1[0].y});
                d0.add({a0.y, b0.y}, {p0[1].x, p0[1].y});
                d1.add({a1.y, b1.y}, {p1[1].x, p1[1].y});
                d0.add({a0.z, b0.z}, {p0[2].x, p0[2].y});
                d1.add({a1.z, b1.z}, {p1[2].x, p1[2].y});
                d0.add({a0.w, b0.w}, {p0[3].x, p0[3].y});
                d1.add({a1.w, b1.w}, {p1[3].x, p1[3].y});
            }
            for (; v < nv; v += 32) {
                const float4 a0 = __ldcs(rh + v), b0 = __ldcs(rl + v);
                const float2* p0 = xs + 4 * v;
                d0.add({a0.x, b0.x}, {p0[0].x, p0[0].y});
                d0.add({a0.y, b0.y}, {p0[1].x, p0[1].y});
                d0.add({a0.z, b0.z}, {p0[2].x, p0[2].y});
                d0.add({a0.w, b0.w}, {p0[3].x, p0[3].y});
            }
            const lk::df2 sum = warp_sum_df(lk::df_add(d0.value(), d1.value()));
            if (lane == 0) acc[rr] += lk::df_to(sum);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        const int64_t gi = r0 + i;
        w[gi] = fma(lambda, x[gi], acc[i]);
    }
}

// ---------------------------------------------------------------------------
// Vector kernels.  Block b owns the contiguous rows [b*R, (b+1)*R).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void row_range(int64_t n, int64_t& r0, int64_t& r1) {
    const int64_t R = (n + gridDim.x - 1) / gridDim.x;
    r0 = min(n, (int64_t)blockIdx.x * R);
    r1 = min(n, r0 + R);
}

struct PrecView {
    int kind;
    int n_r;
    int nch;          // row chunks of U^T r: t holds nch partial vectors of n_r
    int ldw;          // row pitch of W (n_r rounded up to 4 for float32 W, n_r for float64)
    int64_t ldu;
    double cinv;
    const void* UT;   // n_r x ldu, U transposed
    const void* W;    // n x n_r
    const double* dinv;
};

// INIT: alpha = 0, r = y, p = 0, |y|^2.
__global__ void __launch_bounds__(VEC_THREADS)
k_pcg_init(int64_t n, const double* __restrict__ y, double* __restrict__ alpha, double* __restrict__ r,
           double* __restrict__ p0, double* __restrict__ abest, double* __restrict__ rbest, PcgScalars* sc,
           double* __restrict__ partials, double tol) {
    __shared__ double red[VEC_THREADS / 32];
    int64_t r0, r1;
    row_range(n, r0, r1);
    double yy = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double yi = y[i];
        alpha[i] = 0.0;
        r[i] = yi;
        p0[i] = 0.0;
        abest[i] = 0.0;   // the guard's fallback before its first replacement: alpha = 0
        rbest[i] = yi;
        yy = fma(yi, yi, yy);
    }
    yy = lk::block_sum(yy, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = yy;
    if (lk::last_block(&sc->ticket[1])) {
        const double tot = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->yy = tot;
            sc->rr = tot;
            sc->tol2yy = tol * tol * tot;
            sc->rz = 0.0;
            sc->beta = 0.0;
            sc->delta = 0.0;
            sc->iters = 0;
            sc->true_count = 0;
            sc->need_true = 0;
            sc->converged = (tot == 0.0) ? 1 : (isfinite(tot) ? 0 : 2);
            sc->ticket[1] = 0;
        }
    }
}

// Warm start: alpha holds the caller's start alpha^0 and w2 = (lambda I + G)
// alpha^0 (float64-accurate); r^0 = y - w2.  A start that already meets the
// tolerance ends the solve before the first product.
__global__ void __launch_bounds__(VEC_THREADS)
k_pcg_init_warm(int64_t n, const double* __restrict__ y, const double* __restrict__ alpha,
                const double* __restrict__ w2, double* __restrict__ r, double* __restrict__ p0,
                double* __restrict__ abest, double* __restrict__ rbest, PcgScalars* sc,
                double* __restrict__ partials, double tol) {
    __shared__ double red[VEC_THREADS / 32];
    int64_t r0, r1;
    row_range(n, r0, r1);
    double yy = 0.0, rr = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double yi = y[i];
        const double ri = yi - w2[i];
        r[i] = ri;
        p0[i] = 0.0;
        abest[i] = alpha[i];   // the guard's fallback before its first replacement
        rbest[i] = ri;
        yy = fma(yi, yi, yy);
        rr = fma(ri, ri, rr);
    }
    yy = lk::block_sum(yy, red);
    rr = lk::block_sum(rr, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = yy;
        partials[gridDim.x + blockIdx.x] = rr;
    }
    if (lk::last_block(&sc->ticket[1])) {
        const double tyy = lk::sum_partials(partials, gridDim.x, red);
        const double trr = lk::sum_partials(partials + gridDim.x, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->yy = tyy;
            sc->rr = trr;
            sc->rr_true = trr;
            sc->tol2yy = tol * tol * tyy;
            sc->rz = 0.0;
            sc->beta = 0.0;
            sc->delta = 0.0;
            sc->iters = 0;
            sc->true_count = 0;
            sc->need_true = 0;
            sc->converged = (!isfinite(tyy) || !isfinite(trr)) ? 2 : (trr <= sc->tol2yy ? 1 : 0);
            sc->ticket[1] = 0;
        }
    }
}

// UPD: alpha += delta p, r -= delta w, |r|^2; stop / refinement decisions.
__global__ void __launch_bounds__(VEC_THREADS)
k_pcg_update(int64_t n, const double* __restrict__ p, const double* __restrict__ w, double* __restrict__ alpha,
             double* __restrict__ r, PcgScalars* sc, double* __restrict__ partials, const double* __restrict__ y,
             double lambda) {
    if (gated_out(sc, GATE_RUNNING)) return;
    __shared__ double red[VEC_THREADS / 32];
    int64_t r0, r1;
    row_range(n, r0, r1);
    const double delta = sc->delta;
    double* trace = sc->trace;   // uniform: the trace also needs r.alpha and y.alpha
    const bool gap = sc->gap_tol > 0.0;   // uniform: so does the objective-gap stop
    const bool objective = trace != nullptr || gap;
    double rr = 0.0, ra = 0.0, ya = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ai = fma(delta, p[i], alpha[i]);
        alpha[i] = ai;
        const double ri = fma(-delta, w[i], r[i]);
        r[i] = ri;
        rr = fma(ri, ri, rr);
        if (objective) {
            ra = fma(ri, ai, ra);
            ya = fma(y[i], ai, ya);
        }
    }
    rr = lk::block_sum(rr, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = rr;
    if (objective) {
        ra = lk::block_sum(ra, red);
        ya = lk::block_sum(ya, red);
        if (threadIdx.x == 0) {
            partials[gridDim.x + blockIdx.x] = ra;
            partials[2 * gridDim.x + blockIdx.x] = ya;
        }
    }
    if (lk::last_block(&sc->ticket[2])) {
        const double tot = lk::sum_partials(partials, gridDim.x, red);
        double tra = 0.0, tya = 0.0;
        if (objective) {
            tra = lk::sum_partials(partials + gridDim.x, gridDim.x, red);
            tya = lk::sum_partials(partials + 2 * gridDim.x, gridDim.x, red);
        }
        if (threadIdx.x == 0) {
            sc->rr = tot;
            const int it = sc->iters;
            // R(alpha) = |G alpha - y|^2 + lambda alpha^T G alpha with G alpha = y - r - lambda alpha
            // (Eq. simu-R-definition) is |r|^2 + lambda (r.alpha + y.alpha)
            const double R = fma(lambda, tra + tya, tot);
            if (trace && it >= 1 && it <= sc->trace_cap) {
                trace[4 * (it - 1)] = delta;
                trace[4 * (it - 1) + 1] = tot / sc->yy;
                trace[4 * (it - 1) + 2] = R;
            }
            const bool small = tot <= sc->tol2yy;
            if (sc->refine_every > 0) {
                // mixed forms: a non-finite recursive residual or a breakdown
                // is handled by the guard at the replacement it forces
                sc->since_true += 1;
                if (!isfinite(tot)) sc->breakdown = 1;
                if (isfinite(tot) && gap && fabs(R - sc->R_ref) <= sc->gap_tol * fabs(sc->R_ref))
                    sc->converged = 1;   // objective gap reached (Eq. iterations, TAR.TOL)
                else if (small || sc->breakdown || sc->since_true >= sc->interval || it >= sc->max_iter)
                    sc->need_true = 1;
            } else if (!isfinite(tot)) {
                sc->converged = 2;
            } else if (gap && fabs(R - sc->R_ref) <= sc->gap_tol * fabs(sc->R_ref)) {
                sc->converged = 1;   // objective gap reached (Eq. iterations, TAR.TOL)
            } else if (small) {
                sc->converged = 1;
            } else if (it >= sc->max_iter) {
                sc->converged = 3;
            }
            sc->ticket[2] = 0;
        }
    }
}

// TR2: r = y - w2 with w2 = (lambda I + G) alpha; stop test on the true
// residual, and the guard of the mixed forms.
//
// Between replacements the recursion runs on the inexact operator A~.  Where
// A~ is within its own rounding of losing definiteness (split-bf16 products
// at n = 65536, lambda = 1e-4: the float32 accumulation and ex2.approx errors
// are of order lambda along the bottom of the spectrum), long intervals let
// CG build directions along which p^T A~ p is wrong or <= 0, and the true
// residual grows without bound: measured, a replacement every 30 products
// diverged on that instance after reaching 1.2e-6, every 20 converged.  The
// recursive residual itself stays within ~1e-3 of the true one at every
// replacement, so the guard watches the true residual: the lowest one seen is
// saved with its iterate; a non-finite residual, or two replacements in a row
// more than 30 times above the best, roll back to the saved iterate, restart
// the direction and halve the interval.  (CG's residual is not monotone: its
// early transient stays within ~4 times of the first replacement's value, and
// near the accuracy floor single spikes above 30 times recover -- a float32
// solve at lambda = 1.1e-5, n = 7633 that rolled back on each spike ended as
// stagnated, where the unguarded iteration converged -- while divergence
// grows at every replacement.)  A breakdown p^T A~ p <= 0 only makes the
// direction useless: it forces a replacement and restarts the direction from
// the current iterate, or rolls back at once if that replacement is more than
// 30 times above the best.  At the smallest
// interval a further roll-back ends the solve (stagnation).  (The true energy
// phi(alpha), exact CG's monotone quantity, cannot serve: near convergence its
// changes are below the cancellation of y^T alpha in float64.)
constexpr int GUARD_MIN_INTERVAL = 4;
constexpr double GUARD_GROWTH2 = 900.0;   // (30x)^2 in |r|^2
constexpr int GUARD_RISES = 2;             // ... at that many replacements in a row

__global__ void __launch_bounds__(VEC_THREADS)
k_true_residual(int64_t n, const double* __restrict__ y, const double* __restrict__ w2, double* __restrict__ r,
                PcgScalars* sc, double* __restrict__ partials) {
    if (gated_out(sc, GATE_TRUE)) return;
    __shared__ double red[VEC_THREADS / 32];
    int64_t r0, r1;
    row_range(n, r0, r1);
    double rr = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ri = y[i] - w2[i];
        r[i] = ri;
        rr = fma(ri, ri, rr);
    }
    rr = lk::block_sum(rr, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = rr;
    if (lk::last_block(&sc->ticket[3])) {
        const double tot = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->rr = tot;
            sc->rr_true = tot;
            sc->true_count += 1;
            sc->need_true = 0;
            sc->since_true = 0;
            const bool bad = !isfinite(tot);
            int action = 0;
            if (!bad && tot <= sc->tol2yy) {
                sc->converged = 1;
            } else if (!bad && tot < sc->rr_best) {
                sc->rr_best = tot;
                sc->grow = 0;
                action = 1;
                if (sc->breakdown) {   // keep the iterate, drop the direction
                    sc->restart_dir = 1;
                    sc->restarts += 1;
                }
            } else if (bad || (tot > GUARD_GROWTH2 * sc->rr_best && (++sc->grow >= GUARD_RISES || sc->breakdown))) {
                action = 2;
                sc->grow = 0;
                if (sc->interval <= GUARD_MIN_INTERVAL) {
                    sc->converged = 4;   // stagnated: the saved iterate is returned
                } else {
                    sc->interval = max(GUARD_MIN_INTERVAL, sc->interval / 2);
                    sc->restarts += 1;
                    sc->restart_dir = 1;
                }
            } else {
                if (tot <= GUARD_GROWTH2 * sc->rr_best) sc->grow = 0;
                if (sc->breakdown) {   // no roll-back due: drop only the direction
                    sc->restart_dir = 1;
                    sc->restarts += 1;
                }
            }
            sc->breakdown = 0;
            if (sc->converged == 0 && sc->iters >= sc->max_iter) {
                sc->converged = 3;
                if (action == 0) action = 2;   // return the lowest-residual iterate
            }
            sc->guard_action = action;
            sc->ticket[3] = 0;
        }
    }
}

// Guard copies: action 1 saves (alpha, r) as the best iterate, action 2
// restores them.  Every block reads the action before it counts itself done,
// so the last block to finish can clear it for the next replacement.
__global__ void __launch_bounds__(VEC_THREADS)
k_pcg_guard(int64_t n, double* __restrict__ alpha, double* __restrict__ r, double* __restrict__ abest,
            double* __restrict__ rbest, PcgScalars* sc) {
    const int action = *(volatile const int*)&sc->guard_action;
    if (action == 0) return;
    int64_t r0, r1;
    row_range(n, r0, r1);
    if (action == 1) {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            abest[i] = alpha[i];
            rbest[i] = r[i];
        }
    } else {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            alpha[i] = abest[i];
            r[i] = rbest[i];
        }
    }
    if (lk::last_block(&sc->ticket[6])) {
        if (threadIdx.x == 0) {
            sc->guard_action = 0;
            sc->ticket[6] = 0;
        }
    }
}

// UTR: t_k = sum_i U_ik r_i.  One block per k streams row k of U^T (padded
// pitch ldu, zeros past n) with 16-byte loads; the block's threads stride over
// the row, keep two independent sums each, and reduce in a fixed order.
template <typename PT> struct UtrVec;
template <> struct UtrVec<float> { using type = float4; static constexpr int N = 4; };
template <> struct UtrVec<double> { using type = double2; static constexpr int N = 2; };

__device__ __forceinline__ float dot_vec(const float4& u, const double* r) {
    const double2 r01 = *reinterpret_cast<const double2*>(r);
    const double2 r23 = *reinterpret_cast<const double2*>(r + 2);
    return fmaf(u.x, (float)r01.x, fmaf(u.y, (float)r01.y, fmaf(u.z, (float)r23.x, u.w * (float)r23.y)));
}
__device__ __forceinline__ double dot_vec(const double2& u, const double* r) {
    const double2 rr = *reinterpret_cast<const double2*>(r);
    return fma(u.x, rr.x, u.y * rr.y);
}

template <typename PT> __device__ __forceinline__ void load_r(const double* r, int64_t e, PT* rv);
template <> __device__ __forceinline__ void load_r<float>(const double* r, int64_t e, float* rv) {
    const double2 a = *reinterpret_cast<const double2*>(r + e), b = *reinterpret_cast<const double2*>(r + e + 2);
    rv[0] = (float)a.x; rv[1] = (float)a.y; rv[2] = (float)b.x; rv[3] = (float)b.y;
}
template <> __device__ __forceinline__ void load_r<double>(const double* r, int64_t e, double* rv) {
    const double2 a = *reinterpret_cast<const double2*>(r + e);
    rv[0] = a.x; rv[1] = a.y;
}
__device__ __forceinline__ float dot_v(const float4& u, const float* rv) {
    return fmaf(u.x, rv[0], fmaf(u.y, rv[1], fmaf(u.z, rv[2], u.w * rv[3])));
}
__device__ __forceinline__ double dot_v(const double2& u, const double* rv) { return fma(u.x, rv[0], u.y * rv[1]); }

// UTR: t_k = sum_i U_ik r_i for four directions k0..k0+3 per block and one
// chunk of the rows per blockIdx.y (partial sums t[chunk * n_r + k], added in
// chunk order by the apply): every load of r serves the four rows of U^T
// (padded pitch ldu, zeros past n), 16-byte loads, two steps in flight; each
// block reduces its four sums in a fixed order.
template <typename PT>
__global__ void __launch_bounds__(256)
k_utr(int64_t n, PrecView pv, const double* __restrict__ r, PT* __restrict__ t, const PcgScalars* sc, int gate) {
    if (gated_out(sc, gate)) return;
    __shared__ PT red[4][8];
    constexpr int VN = UtrVec<PT>::N;
    using V = typename UtrVec<PT>::type;
    const int k0 = blockIdx.x * 4;
    const int nk = min(4, pv.n_r - k0);
    const V* u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = reinterpret_cast<const V*>((const PT*)pv.UT + (int64_t)(k0 + (q < nk ? q : 0)) * pv.ldu);
    const int64_t nfull = n / VN;                 // vectors entirely inside [0, n)
    const int64_t per = (nfull + gridDim.y - 1) / gridDim.y;
    const int64_t v_lo = min(nfull, (int64_t)blockIdx.y * per), v_hi = min(nfull, v_lo + per);
    PT a[4] = {PT(0), PT(0), PT(0), PT(0)}, b[4] = {PT(0), PT(0), PT(0), PT(0)};
    int64_t v = v_lo + threadIdx.x;
    for (; v + 256 < v_hi; v += 512) {
        PT ra[VN], rb[VN];
        load_r<PT>(r, v * VN, ra);
        load_r<PT>(r, (v + 256) * VN, rb);
        V ua[4], ub[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { ua[q] = __ldg(u[q] + v); ub[q] = __ldg(u[q] + v + 256); }
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] += dot_v(ua[q], ra); b[q] += dot_v(ub[q], rb); }
    }
    for (; v < v_hi; v += 256) {
        PT ra[VN];
        load_r<PT>(r, v * VN, ra);
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] += dot_v(__ldg(u[q] + v), ra);
    }
    if (blockIdx.y == gridDim.y - 1)
        for (int64_t i = nfull * VN + threadIdx.x; i < n; i += 256)
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] += reinterpret_cast<const PT*>(u[q])[i] * (PT)r[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const PT s = lk::warp_sum(a[q] + b[q]);
        if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < nk) {
        PT s = PT(0);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        t[(int64_t)blockIdx.y * pv.n_r + k0 + threadIdx.x] = s;
    }
}

// PRE: z = P r, r^T z, beta.  CCCP: z_i = c^-1/2 r_i + sum_k W_ik t_k, four
// rows per warp in flight.
template <typename PT>
__global__ void __launch_bounds__(VEC_THREADS)
k_precond(int64_t n, const double* __restrict__ r, double* __restrict__ z, PcgScalars* sc,
          double* __restrict__ partials, PrecView pv, const PT* __restrict__ t, int gate) {
    if (gated_out(sc, gate)) return;
    __shared__ double red[VEC_THREADS / 32];
    __shared__ __align__(16) PT ts[LK_MAX_NR];
    int64_t r0, r1;
    row_range(n, r0, r1);
    double rz = 0.0;
    if (pv.kind == PRECOND_CCCP && sizeof(PT) == 4) {
        // float32 W with a 16-byte row pitch: four rows per warp, float4 loads
        for (int k = threadIdx.x; k < pv.ldw; k += blockDim.x) {
            PT v = PT(0);
            if (k < pv.n_r)
                for (int c = 0; c < pv.nch; ++c) v += __ldcg(t + (int64_t)c * pv.n_r + k);
            ts[k] = v;
        }
        __syncthreads();
        const float4* W4 = reinterpret_cast<const float4*>(pv.W);
        const float4* t4 = reinterpret_cast<const float4*>(ts);
        const int nk4 = pv.ldw / 4;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int64_t i = r0 + 4 * wid; i < r1; i += 4 * nw) {
            const int nrow = (r1 - i < 4) ? (int)(r1 - i) : 4;
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            int k4 = lane;
            for (; k4 + 96 < nk4; k4 += 128) {   // 16 independent 16-byte loads in flight
                float4 w[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        w[q][u] = (q < nrow) ? __ldg(W4 + (i + q) * nk4 + k4 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 tk = t4[k4 + 32 * u];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        acc[q] = fmaf(w[q][u].x, tk.x, fmaf(w[q][u].y, tk.y, fmaf(w[q][u].z, tk.z, fmaf(w[q][u].w, tk.w, acc[q]))));
                }
            }
            for (; k4 < nk4; k4 += 32) {
                const float4 tk = t4[k4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 w = (q < nrow) ? __ldg(W4 + (i + q) * nk4 + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
                    acc[q] = fmaf(w.x, tk.x, fmaf(w.y, tk.y, fmaf(w.z, tk.z, fmaf(w.w, tk.w, acc[q]))));
                }
            }
            // every lane holds the four sums; lane q finishes row i + q, so the
            // float64 tail is one warp instruction per step for all four rows
            float aq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) aq[q] = lk::warp_sum(acc[q]);
            if (lane < nrow) {
                const float a = (lane == 0) ? aq[0] : (lane == 1) ? aq[1] : (lane == 2) ? aq[2] : aq[3];
                const double ri = r[i + lane];
                const double zi = fma(pv.cinv, ri, (double)a);
                z[i + lane] = zi;
                rz = fma(ri, zi, rz);
            }
        }
    } else if (pv.kind == PRECOND_CCCP) {
        for (int k = threadIdx.x; k < pv.n_r; k += blockDim.x) {
            PT v = PT(0);
            for (int c = 0; c < pv.nch; ++c) v += __ldcg(t + (int64_t)c * pv.n_r + k);
            ts[k] = v;
        }
        __syncthreads();
        const PT* W = (const PT*)pv.W;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int64_t i = r0 + 4 * wid; i < r1; i += 4 * nw) {
            const int nrow = (r1 - i < 4) ? (int)(r1 - i) : 4;
            PT acc[4] = {PT(0), PT(0), PT(0), PT(0)};
            for (int k = lane; k < pv.n_r; k += 32) {
                const PT tk = ts[k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < nrow) acc[q] += W[(i + q) * pv.n_r + k] * tk;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const PT a = lk::warp_sum(acc[q]);
                if (lane == 0 && q < nrow) {
                    const double zi = fma(pv.cinv, r[i + q], (double)a);
                    z[i + q] = zi;
                    rz = fma(r[i + q], zi, rz);
                }
            }
        }
    } else {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double ri = r[i];
            const double zi = (pv.kind == PRECOND_JACOBI) ? ri * pv.dinv[i] : ri;
            z[i] = zi;
            rz = fma(ri, zi, rz);
        }
    }
    if (sc == nullptr) return;
    rz = lk::block_sum(rz, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = rz;
    if (lk::last_block(&sc->ticket[4])) {
        const double tot = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            const double old = sc->rz;
            if (!isfinite(tot) || tot < 0.0) sc->converged = 2;
            else if (tot == 0.0) sc->converged = 1;
            sc->beta = (old > 0.0 && sc->restart_dir == 0) ? tot / old : 0.0;
            sc->restart_dir = 0;
            sc->rz = tot;
            const int it = sc->iters;
            if (sc->trace && it >= 1 && it <= sc->trace_cap) sc->trace[4 * (it - 1) + 3] = sc->beta;
            sc->ticket[4] = 0;
        }
    }
}

// |y - w|^2 -> sc->rr_true (final report only)
__global__ void __launch_bounds__(VEC_THREADS)
k_resid_norm(int64_t n, const double* __restrict__ y, const double* __restrict__ w, PcgScalars* sc,
             double* __restrict__ partials) {
    __shared__ double red[VEC_THREADS / 32];
    int64_t r0, r1;
    row_range(n, r0, r1);
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double e = y[i] - w[i];
        s = fma(e, e, s);
    }
    s = lk::block_sum(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
    if (lk::last_block(&sc->ticket[5])) {
        const double tot = lk::sum_partials(partials, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->rr_true = tot;
            sc->ticket[5] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct Workspace {
    double *r, *z, *p[2], *w, *w2, *abest, *rbest, *partials;
    void* t;
    PcgScalars* sc;
    unsigned int* ticket;
    int vec_blocks;
    int pre_blocks;
    int mv_blocks;
    bool borrowed;   // buffers belong to a PcgArena: nothing to free
};

// Elementwise vector kernels with a scalar reduction.
int vec_blocks_for(const laker_ctx* ctx, int64_t n) {
    int64_t b = (n + 255) / 256;
    b = std::min<int64_t>(b, 2 * ctx->num_sms);
    return (int)std::max<int64_t>(1, b);
}
// The preconditioner apply streams W (n x n_r): many blocks.
int pre_blocks_for(const laker_ctx* ctx, int64_t n) {
    int64_t b = (n + 31) / 32;                     // >= 32 rows: every warp has four rows
    b = std::min<int64_t>(b, 8 * ctx->num_sms);
    return (int)std::max<int64_t>(1, b);
}
int mv_blocks_for(const laker_ctx* ctx, int64_t n) {
    int64_t b = std::min<int64_t>((n + 7) / 8, ctx->num_sms);
    return (int)std::max<int64_t>(1, b);
}

constexpr size_t MV_SMEM_MAX = 200 * 1024;
constexpr int64_t STREAM_BYTES = 48ll << 20;   // G above this size is streamed evict-first

template <typename T>
laker_status launch_mv(laker_ctx* ctx, const laker_op* op, const T* K, const double* pin, const double* z,
                       double* pout, int fuse, double* w, PcgScalars* sc, double* partials, int gate,
                       int reduce, int blocks) {
    const int64_t n = op->n;
    int64_t chunk = std::min<int64_t>((n + 3) / 4 * 4, (int64_t)(160 * 1024 / sizeof(T)));
    chunk = chunk / 4 * 4;
    const int64_t rows_per = (n + blocks - 1) / blocks;
    const size_t smem = chunk * sizeof(T) + rows_per * sizeof(double);
    if (smem > MV_SMEM_MAX) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matvec row block too large");
    const bool stream = (int64_t)(n * op->ldk * sizeof(T)) > STREAM_BYTES;
    if (stream)
        k_matvec_mat<T, true><<<blocks, MV_THREADS, smem, ctx->stream>>>(K, op->ldk, n, op->lambda, chunk, pin, z,
                                                                        pout, fuse, w, sc, partials, gate, reduce);
    else
        k_matvec_mat<T, false><<<blocks, MV_THREADS, smem, ctx->stream>>>(K, op->ldk, n, op->lambda, chunk, pin, z,
                                                                         pout, fuse, w, sc, partials, gate, reduce);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

laker_status launch_mv_df(laker_ctx* ctx, const laker_op* op, const double* x, double* w, const PcgScalars* sc,
                          int gate, int blocks) {
    const int64_t n = op->n;
    int64_t chunk = std::min<int64_t>((n + 3) / 4 * 4, (int64_t)(160 * 1024 / sizeof(float2)));
    chunk = chunk / 4 * 4;
    const int64_t rows_per = (n + blocks - 1) / blocks;
    const size_t smem = chunk * sizeof(float2) + rows_per * sizeof(double);
    if (smem > MV_SMEM_MAX) return set_error(ctx, LAKER_ERR_UNSUPPORTED, "matvec row block too large");
    k_matvec_df<<<blocks, MV_THREADS, smem, ctx->stream>>>(op->K32, op->K32lo, op->ldk, n, op->lambda, chunk, x, w,
                                                           sc, gate);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

// Row chunks of U^T r: enough blocks for ~3 per SM, each chunk >= 1024 rows.
int utr_chunks(const laker_ctx* ctx, int64_t n, int n_w) {
    const int64_t nb = std::max(1, (n_w + 3) / 4);
    const int64_t want = (3 * ctx->num_sms + nb - 1) / nb;
    const int64_t cap = std::max<int64_t>(1, n / 1024);
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, cap), 32));
}

PrecView make_view(const laker_ctx* ctx, const laker_precond* P, bool use32) {
    PrecView v{};
    v.nch = 1;
    if (P == nullptr) { v.kind = PRECOND_IDENTITY; return v; }
    v.kind = P->kind;
    v.n_r = P->n_w;
    if (v.kind == PRECOND_CCCP) v.nch = utr_chunks(ctx, P->n, v.n_r);
    v.ldu = P->ldu;
    v.cinv = P->cinvsqrt;
    v.UT = use32 ? (const void*)P->UT32 : (const void*)P->UT64;
    v.W = use32 ? (const void*)P->W32 : (const void*)P->W64;
    v.ldw = use32 ? P->ldw : P->n_w;
    v.dinv = P->dinv;
    return v;
}

template <typename PT>
laker_status launch_utr(laker_ctx* ctx, int64_t n, const PrecView& pv, const double* r, PT* t, const PcgScalars* sc,
                        int gate) {
    if (pv.kind != PRECOND_CCCP) return LAKER_OK;
    k_utr<PT><<<dim3((unsigned)((pv.n_r + 3) / 4), (unsigned)pv.nch), 256, 0, ctx->stream>>>(n, pv, r, t, sc, gate);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

laker_status ws_alloc(laker_ctx* ctx, const laker_op* op, int n_r, Workspace& ws) {
    const int64_t n = op->n;
    ws.vec_blocks = vec_blocks_for(ctx, n);
    ws.pre_blocks = pre_blocks_for(ctx, n);
    ws.mv_blocks = mv_blocks_for(ctx, n);
    laker_status st;
    double* base = nullptr;
    if ((st = lk_malloc(ctx, (void**)&base, (size_t)8 * n * sizeof(double))) != LAKER_OK) return st;
    ws.r = base; ws.z = base + n; ws.p[0] = base + 2 * n; ws.p[1] = base + 3 * n; ws.w = base + 4 * n;
    ws.w2 = base + 5 * n; ws.abest = base + 6 * n; ws.rbest = base + 7 * n;
    // per-block partials of any of the kernels (the matrix-free finish runs one block per 128 rows)
    const int64_t nb = std::max<int64_t>(8 * ctx->num_sms + 8, 4 * ((n + 127) / 128) + 8);
    if ((st = lk_malloc(ctx, (void**)&ws.partials, (size_t)nb * sizeof(double))) != LAKER_OK) return st;
    const int nr = std::max(1, n_r);
    if ((st = lk_malloc(ctx, &ws.t, (size_t)nr * utr_chunks(ctx, n, nr) * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&ws.sc, sizeof(PcgScalars))) != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMemsetAsync(ws.sc, 0, sizeof(PcgScalars), ctx->stream));
    ws.ticket = ws.sc->ticket + 7;
    return LAKER_OK;
}
// Workspace on an arena's buffers (no allocation); LAKER_ERR_ARG if the solve
// does not fit the arena's capacities.
laker_status ws_borrow(laker_ctx* ctx, const laker_op* op, int n_r, const PcgArena& a, Workspace& ws) {
    const int64_t n = op->n;
    const int64_t nb = std::max<int64_t>(8 * ctx->num_sms + 8, 4 * ((n + 127) / 128) + 8);
    const int nr = std::max(1, n_r);
    const int64_t tneed = (int64_t)nr * utr_chunks(ctx, n, nr);
    if (n > a.n_cap || nb > a.partials_cap || tneed > a.t_cap)
        return set_error(ctx, LAKER_ERR_ARG, "solve larger than the workspace arena");
    ws.vec_blocks = vec_blocks_for(ctx, n);
    ws.pre_blocks = pre_blocks_for(ctx, n);
    ws.mv_blocks = mv_blocks_for(ctx, n);
    double* base = a.base;
    ws.r = base; ws.z = base + n; ws.p[0] = base + 2 * n; ws.p[1] = base + 3 * n; ws.w = base + 4 * n;
    ws.w2 = base + 5 * n; ws.abest = base + 6 * n; ws.rbest = base + 7 * n;
    ws.partials = a.partials;
    ws.t = a.t;
    ws.sc = a.sc;
    LK_CUDA(ctx, cudaMemsetAsync(ws.sc, 0, sizeof(PcgScalars), ctx->stream));
    ws.ticket = ws.sc->ticket + 7;
    ws.borrowed = true;
    return LAKER_OK;
}

void ws_free(Workspace& ws) {
    if (ws.borrowed) return;
    cudaFree(ws.r);
    cudaFree(ws.partials);
    cudaFree(ws.t);
    cudaFree(ws.sc);
}

template <typename PT>
laker_status enqueue_iteration(laker_ctx* ctx, const laker_op* op, const PrecView& pv, Workspace& ws,
                               const double* y, double* alpha, int parity, bool mixed) {
    const int64_t n = op->n;
    double* pin = ws.p[parity];
    double* pout = ws.p[parity ^ 1];
    laker_status st;
    // MV with the operator's inner precision
    if (op->variant == LAKER_MATRIX_FREE) {
        st = mf_matvec_launch(ctx, op, pin, ws.z, pout, ws.w, ws.sc, ws.partials, 1, nullptr, nullptr);
    } else if (op->precision == LAKER_FP64) {
        st = launch_mv<double>(ctx, op, op->K64, pin, ws.z, pout, 1, ws.w, ws.sc, ws.partials, GATE_RUNNING, 1,
                               ws.mv_blocks);
    } else {
        st = launch_mv<float>(ctx, op, op->K32, pin, ws.z, pout, 1, ws.w, ws.sc, ws.partials, GATE_RUNNING, 1,
                              ws.mv_blocks);
    }
    if (st != LAKER_OK) return st;
    k_pcg_update<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, pout, ws.w, alpha, ws.r, ws.sc, ws.partials, y,
                                                                  op->lambda);
    LK_LAUNCHED(ctx);
    if (mixed) {
        // TR1: w2 = (lambda I + G) alpha in double-float, only when a true residual is due
        st = op->rw ? resid_matvec(ctx, op, alpha, ws.w2, ws.sc, 1)
                    : launch_mv_df(ctx, op, alpha, ws.w2, ws.sc, GATE_TRUE, ws.mv_blocks);
        if (st != LAKER_OK) return st;
        k_true_residual<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, y, ws.w2, ws.r, ws.sc, ws.partials);
        LK_LAUNCHED(ctx);
        k_pcg_guard<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, alpha, ws.r, ws.abest, ws.rbest, ws.sc);
        LK_LAUNCHED(ctx);
    }
    if ((st = launch_utr<PT>(ctx, n, pv, ws.r, (PT*)ws.t, ws.sc, GATE_RUNNING)) != LAKER_OK) return st;
    k_precond<PT><<<ws.pre_blocks, VEC_THREADS, 0, ctx->stream>>>(n, ws.r, ws.z, ws.sc, ws.partials, pv,
                                                                   (const PT*)ws.t, GATE_RUNNING);
    LK_LAUNCHED(ctx);
    return LAKER_OK;
}

}  // namespace

laker_status op_matvec_inner(laker_ctx* ctx, const laker_op* op, const double* x, double* w) {
    if (op->variant == LAKER_MATRIX_FREE) {
        laker_status st = mf_matvec_launch(ctx, op, x, nullptr, nullptr, w, nullptr, nullptr, 0, nullptr, nullptr);
        return st != LAKER_OK ? st : mf_status(ctx, op);
    }
    if (op->precision == LAKER_FP64)
        return launch_mv<double>(ctx, op, op->K64, x, nullptr, nullptr, 0, w, nullptr, nullptr, GATE_NONE, 0,
                                 mv_blocks_for(ctx, op->n));
    return launch_mv<float>(ctx, op, op->K32, x, nullptr, nullptr, 0, w, nullptr, nullptr, GATE_NONE, 0,
                            mv_blocks_for(ctx, op->n));
}

laker_status op_matvec_fp64(laker_ctx* ctx, const laker_op* op, const double* x, double* w) {
    if (op->rw) {
        const laker_status st = resid_matvec(ctx, op, x, w, nullptr, 0);
        return st != LAKER_OK ? st : resid_status(ctx, op);
    }
    if (op->precision != LAKER_FP64) return launch_mv_df(ctx, op, x, w, nullptr, GATE_NONE, mv_blocks_for(ctx, op->n));
    return launch_mv<double>(ctx, op, op->K64, x, nullptr, nullptr, 0, w, nullptr, nullptr, GATE_NONE, 0,
                             mv_blocks_for(ctx, op->n));
}

laker_status op_time_materialised(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    double* w = nullptr;
    laker_status st = lk_malloc(ctx, (void**)&w, (size_t)op->n * sizeof(double));
    if (st != LAKER_OK) return st;
    cudaEvent_t e0, e1;
    LK_CUDA(ctx, cudaEventCreate(&e0));
    LK_CUDA(ctx, cudaEventCreate(&e1));
    for (int rep = -1; rep < reps && st == LAKER_OK; ++rep) {
        if (rep == 0) LK_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        st = op_matvec_inner(ctx, op, x, w);
    }
    LK_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    LK_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0.f;
    LK_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(w);
    *ms = (double)t / reps;
    return st;
}

// Average device time of one whole product w = (lambda I + G) x as a solve
// issues it (matrix-free: prep, tensor-core kernel and finish; materialised:
// the streamed matvec), over `reps` back-to-back launches after one warm-up,
// with CUDA events on the context's stream and no synchronisation between
// the launches.
laker_status op_time_product(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    double* w = nullptr;
    laker_status st = lk_malloc(ctx, (void**)&w, (size_t)op->n * sizeof(double));
    if (st != LAKER_OK) return st;
    cudaEvent_t e0, e1;
    LK_CUDA(ctx, cudaEventCreate(&e0));
    LK_CUDA(ctx, cudaEventCreate(&e1));
    const bool mf = op->variant == LAKER_MATRIX_FREE;
    for (int rep = -1; rep < reps && st == LAKER_OK; ++rep) {
        if (rep == 0) LK_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
        st = mf ? mf_matvec_launch(ctx, op, x, nullptr, nullptr, w, nullptr, nullptr, 0, nullptr, nullptr)
                : op_matvec_inner(ctx, op, x, w);
    }
    LK_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    LK_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0.f;
    LK_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(w);
    if (st != LAKER_OK) return st;
    *ms = (double)t / reps;
    return mf ? mf_status(ctx, op) : LAKER_OK;
}

laker_status pcg_arena_alloc(laker_ctx* ctx, int64_t n_max, int nw_max, PcgArena* a) {
    *a = PcgArena{};
    a->n_cap = std::max<int64_t>(1, n_max);
    a->partials_cap = std::max<int64_t>(8 * ctx->num_sms + 8, 4 * ((a->n_cap + 127) / 128) + 8);
    a->t_cap = (int64_t)std::max(1, nw_max) * 32;   // utr_chunks() <= 32
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&a->base, (size_t)8 * a->n_cap * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&a->partials, (size_t)a->partials_cap * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, &a->t, (size_t)a->t_cap * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&a->sc, sizeof(PcgScalars))) != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMallocHost(&a->flag_host, sizeof(int)));
    return LAKER_OK;
}

void pcg_arena_free(PcgArena* a) {
    cudaFree(a->base);
    cudaFree(a->partials);
    cudaFree(a->t);
    cudaFree(a->sc);
    if (a->flag_host) cudaFreeHost(a->flag_host);
    *a = PcgArena{};
}

laker_status pcg_prepare(laker_ctx* ctx) {
    LK_CUDA(ctx, cudaFuncSetAttribute(k_matvec_mat<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)MV_SMEM_MAX));
    LK_CUDA(ctx, cudaFuncSetAttribute(k_matvec_mat<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)MV_SMEM_MAX));
    LK_CUDA(ctx, cudaFuncSetAttribute(k_matvec_mat<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)MV_SMEM_MAX));
    LK_CUDA(ctx, cudaFuncSetAttribute(k_matvec_mat<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)MV_SMEM_MAX));
    LK_CUDA(ctx, cudaFuncSetAttribute(k_matvec_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MV_SMEM_MAX));
    return LAKER_OK;
}

laker_status precond_apply(laker_ctx* ctx, const laker_precond* P, const double* r, double* z) {
    const int64_t n = P->n;
    const int vb = pre_blocks_for(ctx, n);
    PrecView pv = make_view(ctx, P, P->use32);
    if (P->kind != PRECOND_CCCP) {
        k_precond<double><<<vb, VEC_THREADS, 0, ctx->stream>>>(n, r, z, nullptr, nullptr, pv, nullptr, GATE_NONE);
        LK_LAUNCHED(ctx);
        return LAKER_OK;
    }
    void* t = nullptr;
    double* ra = nullptr;
    laker_status st;
    if ((st = lk_malloc(ctx, &t, (size_t)P->n_w * pv.nch * sizeof(double))) != LAKER_OK) return st;
    if (reinterpret_cast<uintptr_t>(r) & 15) {   // the U^T r kernel reads r with 16-byte loads
        if ((st = lk_malloc(ctx, (void**)&ra, (size_t)n * sizeof(double))) != LAKER_OK) { cudaFree(t); return st; }
        LK_CUDA(ctx, cudaMemcpyAsync(ra, r, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        r = ra;
    }
    if (P->use32) {
        st = launch_utr<float>(ctx, n, pv, r, (float*)t, nullptr, GATE_NONE);
        k_precond<float><<<vb, VEC_THREADS, 0, ctx->stream>>>(n, r, z, nullptr, nullptr, pv, (const float*)t, GATE_NONE);
    } else {
        st = launch_utr<double>(ctx, n, pv, r, (double*)t, nullptr, GATE_NONE);
        k_precond<double><<<vb, VEC_THREADS, 0, ctx->stream>>>(n, r, z, nullptr, nullptr, pv, (const double*)t,
                                                               GATE_NONE);
    }
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(t);
    cudaFree(ra);
    return st;
}

laker_status pcg_solve(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                       double* alpha, double tol, int max_iter, int refine_every, laker_solve_info* info,
                       double* trace, int trace_cap, double R_ref, double gap_tol, bool warm,
                       const PcgArena* arena) {
    const int64_t n = op->n;
    const bool mixed = (op->precision != LAKER_FP64) && refine_every > 0;
    const bool use32 = (op->precision != LAKER_FP64);
    Workspace ws{};
    laker_status st = arena ? ws_borrow(ctx, op, P ? P->n_w : 0, *arena, ws) : ws_alloc(ctx, op, P ? P->n_w : 0, ws);
    if (st != LAKER_OK) return st;
    PrecView pv = make_view(ctx, P, use32);
    if (P && P->kind == PRECOND_CCCP && ((use32 && (P->UT32 == nullptr || P->W32 == nullptr)) ||
                                          (!use32 && P->UT64 == nullptr))) {
        ws_free(ws);
        return set_error(ctx, LAKER_ERR_ARG, "preconditioner has no float32 factors for this operator");
    }
    PcgScalars init{};
    init.max_iter = max_iter;
    init.refine_every = mixed ? refine_every : 0;
    init.interval = init.refine_every;
    init.rr_best = HUGE_VAL;   // the first replacement sets it
    init.R_ref = R_ref;
    init.gap_tol = gap_tol;
    struct TraceBuf {
        double* p = nullptr;
        ~TraceBuf() { cudaFree(p); }
    } tb;
    double*& dtrace = tb.p;
    if (trace && trace_cap > 0) {
        if ((st = lk_malloc(ctx, (void**)&dtrace, (size_t)4 * trace_cap * sizeof(double))) != LAKER_OK) {
            ws_free(ws);
            return st;
        }
        LK_CUDA(ctx, cudaMemsetAsync(dtrace, 0, (size_t)4 * trace_cap * sizeof(double), ctx->stream));
        init.trace = dtrace;
        init.trace_cap = trace_cap;
    }
    LK_CUDA(ctx, cudaMemcpyAsync(ws.sc, &init, sizeof(init), cudaMemcpyHostToDevice, ctx->stream));

    auto run_init = [&]() -> laker_status {
        laker_status s2;
        if (warm) {
            if ((s2 = op_matvec_fp64(ctx, op, alpha, ws.w2)) != LAKER_OK) return s2;
            k_pcg_init_warm<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, y, alpha, ws.w2, ws.r, ws.p[0],
                                                                            ws.abest, ws.rbest, ws.sc, ws.partials,
                                                                            tol);
        } else {
            k_pcg_init<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, y, alpha, ws.r, ws.p[0], ws.abest,
                                                                       ws.rbest, ws.sc, ws.partials, tol);
        }
        LK_LAUNCHED(ctx);
        if (use32) {
            if ((s2 = launch_utr<float>(ctx, n, pv, ws.r, (float*)ws.t, ws.sc, GATE_RUNNING)) != LAKER_OK) return s2;
            k_precond<float><<<ws.pre_blocks, VEC_THREADS, 0, ctx->stream>>>(n, ws.r, ws.z, ws.sc, ws.partials, pv,
                                                                              (const float*)ws.t, GATE_RUNNING);
        } else {
            if ((s2 = launch_utr<double>(ctx, n, pv, ws.r, (double*)ws.t, ws.sc, GATE_RUNNING)) != LAKER_OK) return s2;
            k_precond<double><<<ws.pre_blocks, VEC_THREADS, 0, ctx->stream>>>(n, ws.r, ws.z, ws.sc, ws.partials, pv,
                                                                               (const double*)ws.t, GATE_RUNNING);
        }
        LK_LAUNCHED(ctx);
        return LAKER_OK;
    };
    if ((st = run_init()) != LAKER_OK) { ws_free(ws); return st; }

    // capture a block of 2*H iterations (even/odd p buffers) into a graph
    const int H = 8;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t launches_before = ctx->launches;
    LK_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    for (int h = 0; h < H && st == LAKER_OK; ++h) {
        for (int parity = 0; parity < 2 && st == LAKER_OK; ++parity) {
            st = use32 ? enqueue_iteration<float>(ctx, op, pv, ws, y, alpha, parity, mixed)
                       : enqueue_iteration<double>(ctx, op, pv, ws, y, alpha, parity, mixed);
        }
    }
    cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != LAKER_OK) { if (graph) cudaGraphDestroy(graph); ws_free(ws); return st; }
    if (ce != cudaSuccess) { ws_free(ws); return set_error(ctx, LAKER_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce)); }
    const int64_t per_replay = ctx->launches - launches_before;
    ctx->launches = launches_before;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); ws_free(ws); return set_error(ctx, LAKER_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ce)); }

    int* flag_host = nullptr;
    if (arena) flag_host = arena->flag_host;
    else LK_CUDA(ctx, cudaMallocHost(&flag_host, sizeof(int)));
    const int max_replays = max_iter / (2 * H) + 2;
    for (int rep = 0; rep < max_replays; ++rep) {
        LK_CUDA(ctx, cudaGraphLaunch(exec, ctx->stream));
        ctx->launches += per_replay;
        LK_CUDA(ctx, cudaMemcpyAsync(flag_host, &ws.sc->converged, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (*flag_host != 0) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (!arena) cudaFreeHost(flag_host);
    if (op->variant == LAKER_MATRIX_FREE && (st = mf_status(ctx, op)) != LAKER_OK) { ws_free(ws); return st; }
    if ((st = resid_status(ctx, op)) != LAKER_OK) { ws_free(ws); return st; }

    // final report: float64-accurate residual of the returned alpha
    if ((st = op_matvec_fp64(ctx, op, alpha, ws.w2)) != LAKER_OK) { ws_free(ws); return st; }
    k_resid_norm<<<ws.vec_blocks, VEC_THREADS, 0, ctx->stream>>>(n, y, ws.w2, ws.sc, ws.partials);
    LK_LAUNCHED(ctx);
    PcgScalars out{};
    LK_CUDA(ctx, cudaMemcpyAsync(&out, ws.sc, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ws_free(ws);
    if (dtrace) {
        const int rows = std::min(out.iters, trace_cap);
        for (int i = rows; i < trace_cap; ++i)
            for (int q = 0; q < 4; ++q) trace[4 * i + q] = 0.0;
        cudaError_t ce2 = rows > 0 ? cudaMemcpy(trace, dtrace, (size_t)4 * rows * sizeof(double), cudaMemcpyDeviceToHost)
                                   : cudaSuccess;
        if (ce2 != cudaSuccess) return set_error(ctx, LAKER_ERR_CUDA, std::string("trace copy: ") + cudaGetErrorString(ce2));
    }
    laker_status result = LAKER_OK;
    if (out.converged == 2) result = LAKER_ERR_BREAKDOWN;
    else if (out.converged != 1) result = LAKER_ERR_MAXITER;
    if (info) {
        info->iterations = out.iters;
        info->true_residuals = out.true_count;
        info->converged = out.converged == 1;
        info->rel_res = out.yy > 0 ? std::sqrt(out.rr / out.yy) : 0.0;
        info->rel_res_true = out.yy > 0 ? std::sqrt(out.rr_true / out.yy) : 0.0;
        info->status = result;
        info->restarts = out.restarts;
    }
    if (result != LAKER_OK)
        return set_error(ctx, result, result == LAKER_ERR_BREAKDOWN ? "PCG breakdown"
                                      : out.converged == 4 ? "mixed PCG stagnated at the operator's accuracy floor "
                                                             "(the lowest-residual iterate is returned)"
                                                           : "PCG reached max_iter");
    return LAKER_OK;
}
