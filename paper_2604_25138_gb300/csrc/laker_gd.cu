// Numerical-layer baseline and metric of Sec. V-A on the GPU:
//
//  * Gradient descent on R(alpha) = |G alpha - y|^2 + lambda alpha^T G alpha
//    (Eq. simu-R-definition), the paper's first-order baseline:
//        alpha^{k+1} = alpha^k - eta grad R(alpha^k),
//        grad R = 2 G (G alpha + lambda alpha - y) = -2 G r,  r = y - (lambda I + G) alpha,
//    i.e. alpha^{k+1} = alpha^k + 2 eta (A r - lambda r) with A = lambda I + G:
//    two operator products per step.  The paper picks eta by grid search; an
//    eta <= 0 here selects 1/L with L = 2 mu (mu + lambda), mu = lambda_max(G)
//    from a power iteration, the largest step for which every eigen-component
//    of the error contracts (the caller's grid search scales it).
//  * The prediction discrepancy |G alpha - G alpha_ref| / |G alpha_ref|
//    (Eq. prediction-discrepancy), with the float64-accurate operator.
//
// Reductions use per-block partials summed in a fixed order by the last block.
#include <algorithm>
#include <cmath>
#include <vector>

#include "laker_device.cuh"

namespace {

constexpr int GT = 256;

struct GdScal {
    double rr;          // |r|^2 of the current iterate
    double R;           // R(alpha) of the current iterate
    double yy;
    unsigned int ticket[2];
};

// r = y - w (w = A alpha); |r|^2 and R(alpha) = |r + lambda alpha|^2 + lambda alpha.(y - r - lambda alpha)
__global__ void __launch_bounds__(GT)
k_gd_resid(int64_t n, const double* __restrict__ y, const double* __restrict__ w, const double* __restrict__ alpha,
           double lambda, double* __restrict__ r, GdScal* sc, double* __restrict__ part, double* trace_row) {
    __shared__ double red[GT / 32];
    double rr = 0.0, fit = 0.0, reg = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * GT + threadIdx.x; i < n; i += (int64_t)gridDim.x * GT) {
        const double ri = y[i] - w[i];
        r[i] = ri;
        const double ai = alpha[i];
        const double e = fma(lambda, ai, ri);          // -(G alpha - y)_i
        rr = fma(ri, ri, rr);
        fit = fma(e, e, fit);
        reg = fma(ai, y[i] - e, reg);                  // alpha_i (G alpha)_i
    }
    rr = lk::block_sum(rr, red);
    fit = lk::block_sum(fit, red);
    reg = lk::block_sum(reg, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rr;
        part[gridDim.x + blockIdx.x] = fit;
        part[2 * gridDim.x + blockIdx.x] = reg;
    }
    if (lk::last_block(&sc->ticket[0])) {
        const double a = lk::sum_partials(part, gridDim.x, red);
        const double b = lk::sum_partials(part + gridDim.x, gridDim.x, red);
        const double c = lk::sum_partials(part + 2 * gridDim.x, gridDim.x, red);
        if (threadIdx.x == 0) {
            sc->rr = a;
            sc->R = fma(lambda, c, b);
            if (trace_row) {
                trace_row[0] = a / sc->yy;
                trace_row[1] = sc->R;
            }
            sc->ticket[0] = 0;
        }
    }
}

// alpha += 2 eta (s - lambda r), s = A r
__global__ void k_gd_step(int64_t n, const double* __restrict__ s, const double* __restrict__ r, double lambda,
                          double two_eta, double* __restrict__ alpha) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) alpha[i] = fma(two_eta, fma(-lambda, r[i], s[i]), alpha[i]);
}

// sum of x_i^2 (and of (a_i - b_i)^2 when b is given) into out[0..1] by one pass + last block
__global__ void __launch_bounds__(GT)
k_sqnorm(int64_t n, const double* __restrict__ x, const double* __restrict__ u, double cu, GdScal* sc,
         double* __restrict__ part, double* out) {
    __shared__ double red[GT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * GT + threadIdx.x; i < n; i += (int64_t)gridDim.x * GT) {
        const double v = u ? fma(cu, u[i], x[i]) : x[i];
        s = fma(v, v, s);
    }
    s = lk::block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (lk::last_block(&sc->ticket[1])) {
        const double t = lk::sum_partials(part, gridDim.x, red);
        if (threadIdx.x == 0) {
            *out = t;
            sc->ticket[1] = 0;
        }
    }
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ z,
                        double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fma(a, x[i], b * z[i]);
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

unsigned gblocks(int64_t n) { return (unsigned)std::min<int64_t>((n + GT - 1) / GT, 1024); }
unsigned eblocks(int64_t n) { return (unsigned)((n + 255) / 256); }

struct GdWork {
    double* buf = nullptr;    // r, w, s, v: 4 n
    double* part = nullptr;   // 3 * 1024
    GdScal* sc = nullptr;
    double* norms = nullptr;  // 4
    ~GdWork() { cudaFree(buf); cudaFree(part); cudaFree(sc); cudaFree(norms); }
};

laker_status gd_alloc(laker_ctx* ctx, int64_t n, GdWork& g) {
    laker_status st;
    if ((st = lk_malloc(ctx, (void**)&g.buf, (size_t)4 * n * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&g.part, (size_t)3 * 1024 * sizeof(double))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&g.sc, sizeof(GdScal))) != LAKER_OK) return st;
    if ((st = lk_malloc(ctx, (void**)&g.norms, 4 * sizeof(double))) != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMemsetAsync(g.sc, 0, sizeof(GdScal), ctx->stream));
    return LAKER_OK;
}

laker_status sqnorm(laker_ctx* ctx, int64_t n, const double* x, const double* u, double cu, GdWork& g, double* host) {
    k_sqnorm<<<gblocks(n), GT, 0, ctx->stream>>>(n, x, u, cu, g.sc, g.part, g.norms);
    LK_LAUNCHED(ctx);
    LK_CUDA(ctx, cudaMemcpyAsync(host, g.norms, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

}  // namespace

// lambda_max(G) by `iters` power-iteration steps on A from the all-ones vector
// (for an entrywise-positive G its Perron vector has positive entries, so the
// start has a component along it).
laker_status gd_lambda_max(laker_ctx* ctx, const laker_op* op, int iters, double* mu) {
    const int64_t n = op->n;
    GdWork g;
    laker_status st = gd_alloc(ctx, n, g);
    if (st != LAKER_OK) return st;
    double* v = g.buf;
    double* w = g.buf + n;
    k_fill<<<eblocks(n), 256, 0, ctx->stream>>>(n, 1.0 / std::sqrt((double)n), v);
    LK_LAUNCHED(ctx);
    double lam = 0.0;
    for (int k = 0; k < iters; ++k) {
        if ((st = op_matvec_inner(ctx, op, v, w)) != LAKER_OK) return st;
        double h = 0.0;
        if ((st = sqnorm(ctx, n, w, nullptr, 0.0, g, &h)) != LAKER_OK) return st;
        lam = std::sqrt(h);   // |A v| with |v| = 1
        if (!(lam > 0.0) || !std::isfinite(lam)) return set_error(ctx, LAKER_ERR_NONFINITE, "power iteration failed");
        k_axpby<<<eblocks(n), 256, 0, ctx->stream>>>(n, 1.0 / lam, w, 0.0, w, v);
        LK_LAUNCHED(ctx);
    }
    *mu = lam - op->lambda;
    return LAKER_OK;
}

extern "C" laker_status laker_gd_solve(laker_ctx* ctx, const laker_op* op, const double* y, double* alpha, double eta,
                                       double tol, int max_iter, double* eta_used, laker_solve_info* info,
                                       double* trace, int trace_cap) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!op || !y || !alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (max_iter < 0 || !(tol >= 0.0) || (trace && trace_cap < 1))
        return set_error(ctx, LAKER_ERR_ARG, "gradient descent: bad arguments");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = op->n;
    laker_status st;
    if (!(eta > 0.0)) {
        double mu = 0.0;
        if ((st = gd_lambda_max(ctx, op, 50, &mu)) != LAKER_OK) return st;
        eta = 1.0 / (2.0 * mu * (mu + op->lambda));
    }
    if (eta_used) *eta_used = eta;
    GdWork g;
    if ((st = gd_alloc(ctx, n, g)) != LAKER_OK) return st;
    double* r = g.buf;
    double* w = g.buf + n;
    double* s = g.buf + 2 * n;
    double* dtrace = nullptr;
    struct Free { double*& p; ~Free() { cudaFree(p); } } ft{dtrace};
    if (trace) {
        if ((st = lk_malloc(ctx, (void**)&dtrace, (size_t)2 * trace_cap * sizeof(double))) != LAKER_OK) return st;
        LK_CUDA(ctx, cudaMemsetAsync(dtrace, 0, (size_t)2 * trace_cap * sizeof(double), ctx->stream));
    }
    double yy = 0.0;
    if ((st = sqnorm(ctx, n, y, nullptr, 0.0, g, &yy)) != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMemcpyAsync(&g.sc->yy, &yy, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    LK_CUDA(ctx, cudaMemsetAsync(alpha, 0, (size_t)n * sizeof(double), ctx->stream));
    const double tol2 = tol * tol * yy;
    int it = 0;
    int converged = 0;
    GdScal hs{};
    // iterate k: r = y - A alpha_k (the residual of the current iterate), then
    // the step; the test on |r| is read back every 16 steps
    for (; it <= max_iter; ++it) {
        if ((st = op_matvec_inner(ctx, op, alpha, w)) != LAKER_OK) return st;
        k_gd_resid<<<gblocks(n), GT, 0, ctx->stream>>>(n, y, w, alpha, op->lambda, r, g.sc, g.part,
                                                     (dtrace && it >= 1 && it <= trace_cap) ? dtrace + 2 * (it - 1)
                                                                                            : nullptr);
        LK_LAUNCHED(ctx);
        if ((it & 15) == 0 || it == max_iter) {
            LK_CUDA(ctx, cudaMemcpyAsync(&hs, g.sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
            LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            if (!std::isfinite(hs.rr)) return set_error(ctx, LAKER_ERR_BREAKDOWN, "gradient descent diverged");
            if (hs.rr <= tol2) { converged = 1; break; }
        }
        if (it == max_iter) break;
        if ((st = op_matvec_inner(ctx, op, r, s)) != LAKER_OK) return st;
        k_gd_step<<<eblocks(n), 256, 0, ctx->stream>>>(n, s, r, op->lambda, 2.0 * eta, alpha);
        LK_LAUNCHED(ctx);
    }
    LK_CUDA(ctx, cudaMemcpyAsync(&hs, g.sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (dtrace) {
        const int rows = std::min(it, trace_cap);
        for (int i = 0; i < 2 * trace_cap; ++i) trace[i] = 0.0;
        if (rows > 0)
            LK_CUDA(ctx, cudaMemcpy(trace, dtrace, (size_t)2 * rows * sizeof(double), cudaMemcpyDeviceToHost));
    }
    // float64-accurate residual of the returned alpha
    if ((st = op_matvec_fp64(ctx, op, alpha, w)) != LAKER_OK) return st;
    double rt = 0.0;
    if ((st = sqnorm(ctx, n, y, w, -1.0, g, &rt)) != LAKER_OK) return st;
    const laker_status result = converged ? LAKER_OK : LAKER_ERR_MAXITER;
    if (info) {
        info->iterations = it;
        info->true_residuals = 0;
        info->converged = converged;
        info->rel_res = yy > 0 ? std::sqrt(hs.rr / yy) : 0.0;
        info->rel_res_true = yy > 0 ? std::sqrt(rt / yy) : 0.0;
        info->status = result;
        info->restarts = 0;
    }
    return result == LAKER_OK ? LAKER_OK : set_error(ctx, result, "gradient descent reached max_iter");
}

extern "C" laker_status laker_op_lambda_max(laker_ctx* ctx, const laker_op* op, int iters, double* mu) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!op || !mu || iters < 1) return set_error(ctx, LAKER_ERR_ARG, "power iteration: bad arguments");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    return gd_lambda_max(ctx, op, iters, mu);
}

extern "C" laker_status laker_prediction_discrepancy(laker_ctx* ctx, const laker_op* op, const double* alpha,
                                                     const double* alpha_ref, double* out) {
    if (!ctx) return LAKER_ERR_ARG;
    if (!op || !alpha || !alpha_ref || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    LK_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = op->n;
    GdWork g;
    laker_status st = gd_alloc(ctx, n, g);
    if (st != LAKER_OK) return st;
    double* dlt = g.buf;
    double* w = g.buf + n;
    // G x = (lambda I + G) x - lambda x with the float64-accurate operator
    k_axpby<<<eblocks(n), 256, 0, ctx->stream>>>(n, 1.0, alpha, -1.0, alpha_ref, dlt);
    LK_LAUNCHED(ctx);
    if ((st = op_matvec_fp64(ctx, op, dlt, w)) != LAKER_OK) return st;
    double num = 0.0, den = 0.0;
    if ((st = sqnorm(ctx, n, w, dlt, -op->lambda, g, &num)) != LAKER_OK) return st;
    if ((st = op_matvec_fp64(ctx, op, alpha_ref, w)) != LAKER_OK) return st;
    if ((st = sqnorm(ctx, n, w, alpha_ref, -op->lambda, g, &den)) != LAKER_OK) return st;
    if (!(den > 0.0)) return set_error(ctx, LAKER_ERR_ARG, "prediction discrepancy: G alpha_ref is zero");
    *out = std::sqrt(num / den);
    return LAKER_OK;
}
