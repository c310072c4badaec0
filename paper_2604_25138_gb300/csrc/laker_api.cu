// C ABI of liblaker: argument checks, handle lifetime, dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "laker_internal.h"

laker_status pcg_prepare(laker_ctx* ctx);

laker_status set_error(laker_ctx* ctx, laker_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

laker_status lk_malloc(laker_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, LAKER_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                                 "): " + cudaGetErrorString(e));
    }
    return LAKER_OK;
}

namespace {

laker_status check_ctx(laker_ctx* ctx) {
    if (!ctx) return LAKER_ERR_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e));
    return LAKER_OK;
}

void free_op(laker_op* op) {
    if (!op) return;
    mf_release(op);
    resid_release(op);
    cudaFree(op->Q64);
    cudaFree(op->Qhi);
    cudaFree(op->Qlo);
    cudaFree(op->Q32);
    cudaFree(op->K64);
    cudaFree(op->K32);
    cudaFree(op->K32lo);
    cudaFree(op->diagA);
    delete op;
}

void free_precond(laker_precond* P) {
    if (!P) return;
    cudaFree(P->D);
    cudaFree(P->U64);
    cudaFree(P->W64);
    cudaFree(P->UT32);
    cudaFree(P->UT64);
    cudaFree(P->W32);
    cudaFree(P->dinv);
    cudaFree(P->feat);
    delete P;
}

__global__ void k_recip(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = 1.0 / x[i];
}

__global__ void k_nonfinite(int64_t count, const double* __restrict__ x, int* flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count && !isfinite(x[i])) atomicExch(flag, 1);
}

}  // namespace

// Returns LAKER_ERR_NONFINITE if any of x[0..count) is NaN/Inf.
laker_status scan_finite(laker_ctx* ctx, const double* x, int64_t count) {
    int* flag = nullptr;
    laker_status st = lk_malloc(ctx, (void**)&flag, sizeof(int));
    if (st != LAKER_OK) return st;
    LK_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    k_nonfinite<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(count, x, flag);
    LK_LAUNCHED(ctx);
    int h = 0;
    LK_CUDA(ctx, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(flag);
    return h ? set_error(ctx, LAKER_ERR_NONFINITE, "non-finite value in input") : LAKER_OK;
}


extern "C" {

laker_status laker_create(laker_ctx** out, int device, void* stream) {
    if (!out) return LAKER_ERR_ARG;
    *out = nullptr;
    laker_ctx* ctx = new (std::nothrow) laker_ctx();
    if (!ctx) return LAKER_ERR_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete ctx; return LAKER_ERR_CUDA; }
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete ctx; return LAKER_ERR_CUDA; }
        ctx->owns_stream = true;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (ctx->num_sms <= 0) ctx->num_sms = 1;
    laker_status st = pcg_prepare(ctx);
    if (st != LAKER_OK) { laker_destroy(ctx); return st; }
    *out = ctx;
    return LAKER_OK;
}

laker_status laker_destroy(laker_ctx* ctx) {
    if (!ctx) return LAKER_ERR_ARG;
    if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LAKER_OK;
}

const char* laker_last_error(const laker_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

const char* laker_status_string(int status) {
    switch (status) {
        case LAKER_OK: return "ok";
        case LAKER_ERR_ARG: return "invalid argument";
        case LAKER_ERR_CUDA: return "CUDA error";
        case LAKER_ERR_NOT_SPD: return "matrix not positive definite";
        case LAKER_ERR_BREAKDOWN: return "PCG breakdown";
        case LAKER_ERR_MAXITER: return "maximum iterations reached";
        case LAKER_ERR_NONFINITE: return "non-finite input";
        case LAKER_ERR_TIMEOUT: return "device wait timed out";
        case LAKER_ERR_OOM: return "out of device memory";
        case LAKER_ERR_UNSUPPORTED: return "unsupported option combination";
        default: return "unknown status";
    }
}

int64_t laker_launch_count(const laker_ctx* ctx) { return ctx ? ctx->launches : -1; }

laker_status laker_build_kernel(laker_ctx* ctx, const double* Q, int64_t n, int d, double scale, double lambda,
                                int precision, int variant, laker_op** out) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!out || !Q) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n < 1 || d < 1 || d > 256) return set_error(ctx, LAKER_ERR_ARG, "need n >= 1 and 1 <= d <= 256");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return set_error(ctx, LAKER_ERR_ARG, "need lambda > 0");
    if (!std::isfinite(scale)) return set_error(ctx, LAKER_ERR_ARG, "scale not finite");
    if (precision < LAKER_FP64 || precision > LAKER_BF16X3) return set_error(ctx, LAKER_ERR_ARG, "bad precision");
    if (variant < LAKER_AUTO || variant > LAKER_MATRIX_FREE) return set_error(ctx, LAKER_ERR_ARG, "bad variant");
    // split-bf16 operators are matrix-free; float64 operators are materialised;
    // float32 operators (d <= 64, scale > 0) have both variants, and AUTO
    // times one product of each after the build and keeps the faster
    const int dpad = (d + 15) / 16 * 16;   // the tensor-core kernels take dpad = 16, 32 or 64
    const bool fp32_mf_ok = precision == LAKER_FP32 && (dpad == 16 || dpad == 32 || dpad == 64) && scale > 0.0;
    const bool autotune = variant == LAKER_AUTO && fp32_mf_ok;
    if (variant == LAKER_AUTO)
        variant = (precision == LAKER_BF16X3) ? LAKER_MATRIX_FREE : LAKER_MATERIALISED;
    if (precision == LAKER_BF16X3) variant = LAKER_MATRIX_FREE;
    if (precision == LAKER_FP64 && variant == LAKER_MATRIX_FREE)
        return set_error(ctx, LAKER_ERR_UNSUPPORTED, "float64 operators are materialised only");
    if (precision == LAKER_FP32 && variant == LAKER_MATRIX_FREE && !fp32_mf_ok)
        return set_error(ctx, LAKER_ERR_UNSUPPORTED, "the matrix-free float32 operator needs d <= 32 or 49 <= d <= 64, and scale > 0");
    if ((st = scan_finite(ctx, Q, n * d)) != LAKER_OK) return st;
    laker_op* op = new (std::nothrow) laker_op();
    if (!op) return LAKER_ERR_OOM;
    op->ctx = ctx;
    op->device = ctx->device;
    op->n = n;
    op->d = d;
    op->scale = scale;
    op->lambda = lambda;
    op->precision = precision;
    op->variant = variant;
    if ((st = lk_malloc(ctx, (void**)&op->Q64, (size_t)n * d * sizeof(double))) != LAKER_OK) { free_op(op); return st; }
    cudaError_t e = cudaMemcpyAsync(op->Q64, Q, (size_t)n * d * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) { free_op(op); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    if ((st = build_operator(ctx, op)) != LAKER_OK) { free_op(op); return st; }
    if (precision == LAKER_FP32 && (variant == LAKER_MATRIX_FREE || autotune)) {
        if ((st = mf_prepare(ctx, op)) != LAKER_OK) { free_op(op); return st; }
    }
    if (autotune) {
        // one product of each variant on y = 1 (after a warm-up each), CUDA events
        double* x = nullptr;
        if ((st = lk_malloc(ctx, (void**)&x, (size_t)n * sizeof(double))) != LAKER_OK) { free_op(op); return st; }
        std::vector<double> ones((size_t)n, 1.0);
        e = cudaMemcpyAsync(x, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        double tm = 0.0, tf = 0.0;
        if (e == cudaSuccess) {
            op->variant = LAKER_MATERIALISED;
            st = op_time_product(ctx, op, x, 3, &tm);
            op->variant = LAKER_MATRIX_FREE;
            if (st == LAKER_OK) st = op_time_product(ctx, op, x, 3, &tf);
        }
        cudaFree(x);
        if (e != cudaSuccess) { free_op(op); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
        if (st != LAKER_OK) { free_op(op); return st; }
        op->t_mat_ms = tm;
        op->t_mf_ms = tf;
        op->variant = (tf < tm) ? LAKER_MATRIX_FREE : LAKER_MATERIALISED;
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free_op(op); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    *out = op;
    return LAKER_OK;
}

laker_status laker_op_append(laker_ctx* ctx, const laker_op* op, const double* Q_new, int64_t m, laker_op** out) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !Q_new || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (m < 1) return set_error(ctx, LAKER_ERR_ARG, "need m >= 1");
    if (op->device != ctx->device) return set_error(ctx, LAKER_ERR_ARG, "operator belongs to another device");
    if ((st = scan_finite(ctx, Q_new, m * op->d)) != LAKER_OK) return st;
    laker_op* nop = new (std::nothrow) laker_op();
    if (!nop) return LAKER_ERR_OOM;
    nop->ctx = ctx;
    nop->device = ctx->device;
    nop->n = op->n + m;
    nop->d = op->d;
    nop->scale = op->scale;
    nop->lambda = op->lambda;
    nop->precision = op->precision;
    nop->variant = op->variant;   // the variant the operator resolved to
    const size_t qb = (size_t)op->n * op->d * sizeof(double);
    if ((st = lk_malloc(ctx, (void**)&nop->Q64, qb + (size_t)m * op->d * sizeof(double))) != LAKER_OK) {
        free_op(nop);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(nop->Q64, op->Q64, qb, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)nop->Q64 + qb, Q_new, (size_t)m * op->d * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream);
    if (e != cudaSuccess) { free_op(nop); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    if ((st = build_operator(ctx, nop, op)) != LAKER_OK) { free_op(nop); return st; }
    if (nop->precision == LAKER_FP32 && nop->variant == LAKER_MATRIX_FREE) {
        if ((st = mf_prepare(ctx, nop)) != LAKER_OK) { free_op(nop); return st; }
    }
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free_op(nop); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    *out = nop;
    return LAKER_OK;
}

laker_status laker_op_describe(const laker_op* op, int* precision, int* variant, double* t_materialised_ms,
                               double* t_matrix_free_ms) {
    if (!op) return LAKER_ERR_ARG;
    if (precision) *precision = op->precision;
    if (variant) *variant = op->variant;
    if (t_materialised_ms) *t_materialised_ms = op->t_mat_ms;
    if (t_matrix_free_ms) *t_matrix_free_ms = op->t_mf_ms;
    return LAKER_OK;
}

// Destroy calls do not touch the context, which the caller may have destroyed
// first; a handle keeps its own device.
laker_status laker_op_destroy(laker_op* op) {
    if (!op) return LAKER_ERR_ARG;
    if (cudaSetDevice(op->device) != cudaSuccess) cudaGetLastError();
    free_op(op);
    return LAKER_OK;
}

laker_status laker_op_matvec(laker_ctx* ctx, const laker_op* op, const double* x, double* w) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !x || !w) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    return op_matvec_inner(ctx, op, x, w);
}

laker_status laker_op_matvec_fp64(laker_ctx* ctx, const laker_op* op, const double* x, double* w) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !x || !w) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    return op_matvec_fp64(ctx, op, x, w);
}

laker_status laker_op_time_operator(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !x || !ms || reps < 1) return set_error(ctx, LAKER_ERR_ARG, "bad arguments");
    if (op->variant == LAKER_MATRIX_FREE) return mf_time_main(ctx, op, x, reps, ms);
    return op_time_materialised(ctx, op, x, reps, ms);
}

laker_status laker_op_time_product(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !x || !ms || reps < 1) return set_error(ctx, LAKER_ERR_ARG, "bad arguments");
    return op_time_product(ctx, op, x, reps, ms);
}

laker_status laker_fit_preconditioner(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r, double gamma,
                                      double rho, double eps, int max_iter, double tol, laker_precond** out,
                                      laker_fit_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !Z || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n_r < 1 || n_r > LK_MAX_NR) return set_error(ctx, LAKER_ERR_ARG, "need 1 <= n_r <= 2048");
    if (!(gamma >= 0.0) || !(eps > 0.0) || rho > 1.0 || max_iter < 1 || !(tol >= 0.0))
        return set_error(ctx, LAKER_ERR_ARG, "bad CCCP parameters");
    if ((st = scan_finite(ctx, Z, op->n * (int64_t)n_r)) != LAKER_OK) return st;
    laker_precond* P = new (std::nothrow) laker_precond();
    if (!P) return LAKER_ERR_OOM;
    P->ctx = ctx;
    P->device = ctx->device;
    P->use32 = op->precision != LAKER_FP64;
    st = fit_cccp(ctx, op, Z, n_r, gamma, rho, eps, max_iter, tol, P, info);
    if (st != LAKER_OK) { free_precond(P); return st; }
    *out = P;
    return LAKER_OK;
}

laker_status laker_fit_preconditioner_warm(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r,
                                           double gamma, double rho, double eps, int max_iter, double tol,
                                           const laker_precond* prev, laker_precond** out, laker_fit_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !Z || !out || !prev) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n_r < 1 || n_r > LK_MAX_NR) return set_error(ctx, LAKER_ERR_ARG, "need 1 <= n_r <= 2048");
    if (prev->kind != PRECOND_CCCP || prev->n_r != n_r || !prev->D)
        return set_error(ctx, LAKER_ERR_ARG, "warm start needs a CCCP preconditioner over the same n_r directions");
    if (prev->device != ctx->device || op->device != ctx->device)
        return set_error(ctx, LAKER_ERR_ARG, "operator or previous preconditioner belongs to another device");
    if (!(gamma >= 0.0) || !(eps > 0.0) || rho > 1.0 || max_iter < 1 || !(tol >= 0.0))
        return set_error(ctx, LAKER_ERR_ARG, "bad CCCP parameters");
    if ((st = scan_finite(ctx, Z, op->n * (int64_t)n_r)) != LAKER_OK) return st;
    laker_precond* P = new (std::nothrow) laker_precond();
    if (!P) return LAKER_ERR_OOM;
    P->ctx = ctx;
    P->device = ctx->device;
    P->use32 = op->precision != LAKER_FP64;
    st = fit_cccp(ctx, op, Z, n_r, gamma, rho, eps, max_iter, tol, P, info, nullptr, nullptr, 0, prev);
    if (st != LAKER_OK) { free_precond(P); return st; }
    *out = P;
    return LAKER_OK;
}

laker_status laker_fit_preconditioner_seeded(laker_ctx* ctx, const laker_op* op, uint64_t seed, int n_r,
                                             double gamma, double rho, double eps, int max_iter, double tol,
                                             laker_precond** out, laker_fit_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n_r < 1 || n_r > LK_MAX_NR) return set_error(ctx, LAKER_ERR_ARG, "need 1 <= n_r <= 2048");
    if (!(gamma >= 0.0) || !(eps > 0.0) || rho > 1.0 || max_iter < 1 || !(tol >= 0.0))
        return set_error(ctx, LAKER_ERR_ARG, "bad CCCP parameters");
    double* Z = nullptr;
    if ((st = lk_malloc(ctx, (void**)&Z, (size_t)op->n * n_r * sizeof(double))) != LAKER_OK) return st;
    if ((st = random_directions(ctx, seed, op->n * (int64_t)n_r, Z)) != LAKER_OK) { cudaFree(Z); return st; }
    laker_precond* P = new (std::nothrow) laker_precond();
    if (!P) { cudaFree(Z); return LAKER_ERR_OOM; }
    P->ctx = ctx;
    P->device = ctx->device;
    P->use32 = op->precision != LAKER_FP64;
    st = fit_cccp(ctx, op, Z, n_r, gamma, rho, eps, max_iter, tol, P, info);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(Z);
    if (st != LAKER_OK) { free_precond(P); return st; }
    *out = P;
    return LAKER_OK;
}

laker_status laker_fit_preconditioner_learned(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r,
                                              double gamma, double rho, double eps, int max_iter, double tol,
                                              laker_setnet* net, const float* X, int mode, laker_precond** out,
                                              laker_fit_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !Z || !out || !net || !X) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    *out = nullptr;
    if (mode != 0 && mode != 1) return set_error(ctx, LAKER_ERR_ARG, "mode must be 0 (warm start) or 1 (direct)");
    if (setnet_in_dim(net) != op->d + 3) return set_error(ctx, LAKER_ERR_ARG, "set network input size is not d + 3");
    if (n_r < 1 || n_r > LK_MAX_NR) return set_error(ctx, LAKER_ERR_ARG, "need 1 <= n_r <= 2048");
    if (!(gamma >= 0.0) || !(eps > 0.0) || rho > 1.0 || max_iter < 1 || !(tol >= 0.0))
        return set_error(ctx, LAKER_ERR_ARG, "bad CCCP parameters");
    if ((st = scan_finite(ctx, Z, op->n * (int64_t)n_r)) != LAKER_OK) return st;
    laker_precond* P = new (std::nothrow) laker_precond();
    if (!P) return LAKER_ERR_OOM;
    P->ctx = ctx;
    P->device = ctx->device;
    P->use32 = op->precision != LAKER_FP64;
    st = fit_cccp(ctx, op, Z, n_r, gamma, rho, eps, max_iter, tol, P, info, net, X, mode);
    if (st != LAKER_OK) { free_precond(P); return st; }
    *out = P;
    return LAKER_OK;
}

laker_status laker_precond_direction_features(laker_ctx* ctx, const laker_precond* P, float* F) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!P || !F) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (P->kind != PRECOND_CCCP || !P->feat) return set_error(ctx, LAKER_ERR_ARG, "not a CCCP preconditioner");
    LK_CUDA(ctx, cudaMemcpyAsync(F, P->feat, sizeof(float) * 2 * P->n_r, cudaMemcpyDeviceToDevice, ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

laker_status laker_precond_jacobi(laker_ctx* ctx, const laker_op* op, laker_precond** out) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    laker_precond* P = new (std::nothrow) laker_precond();
    if (!P) return LAKER_ERR_OOM;
    P->ctx = ctx;
    P->device = ctx->device;
    P->kind = PRECOND_JACOBI;
    P->n = op->n;
    if ((st = lk_malloc(ctx, (void**)&P->dinv, (size_t)op->n * sizeof(double))) != LAKER_OK) { free_precond(P); return st; }
    k_recip<<<(unsigned)((op->n + 255) / 256), 256, 0, ctx->stream>>>(op->n, op->diagA, P->dinv);
    ctx->launches++;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free_precond(P); return set_error(ctx, LAKER_ERR_CUDA, cudaGetErrorString(e)); }
    *out = P;
    return LAKER_OK;
}

laker_status laker_precond_destroy(laker_precond* P) {
    if (!P) return LAKER_ERR_ARG;
    if (cudaSetDevice(P->device) != cudaSuccess) cudaGetLastError();
    free_precond(P);
    return LAKER_OK;
}

laker_status laker_precond_apply(laker_ctx* ctx, const laker_precond* P, const double* r, double* z) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!P || !r || !z) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    return precond_apply(ctx, P, r, z);
}

laker_status laker_precond_export(laker_ctx* ctx, const laker_precond* P, double* c, double* D, double* Ubar) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!P) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (P->kind != PRECOND_CCCP) return set_error(ctx, LAKER_ERR_ARG, "not a CCCP preconditioner");
    if (c) LK_CUDA(ctx, cudaMemcpyAsync(c, &P->c, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if (D) LK_CUDA(ctx, cudaMemcpyAsync(D, P->D, P->n_r * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    if (Ubar)
        LK_CUDA(ctx, cudaMemcpyAsync(Ubar, P->U64, (size_t)P->n * P->n_r * sizeof(double), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    LK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LAKER_OK;
}

laker_status laker_pcg_solve(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                             double* alpha, double tol, int max_iter, int refine_every, laker_solve_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !y || !alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    if (P && P->n != op->n) return set_error(ctx, LAKER_ERR_ARG, "preconditioner size mismatch");
    if ((st = scan_finite(ctx, y, op->n)) != LAKER_OK) return st;
    return pcg_solve(ctx, op, P, y, alpha, tol, max_iter, refine_every, info);
}

laker_status laker_pcg_solve_warm(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                                  double* alpha, double tol, int max_iter, int refine_every, laker_solve_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !y || !alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    if (P && P->n != op->n) return set_error(ctx, LAKER_ERR_ARG, "preconditioner size mismatch");
    if ((st = scan_finite(ctx, y, op->n)) != LAKER_OK) return st;
    if ((st = scan_finite(ctx, alpha, op->n)) != LAKER_OK) return st;
    return pcg_solve(ctx, op, P, y, alpha, tol, max_iter, refine_every, info, nullptr, 0, 0.0, 0.0, true);
}

laker_status laker_pcg_solve_trace(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                                   double* alpha, double tol, int max_iter, int refine_every, laker_solve_info* info,
                                   double* trace, int trace_cap) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !y || !alpha || !trace) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (trace_cap < 1) return set_error(ctx, LAKER_ERR_ARG, "need trace_cap >= 1");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    if (P && P->n != op->n) return set_error(ctx, LAKER_ERR_ARG, "preconditioner size mismatch");
    if ((st = scan_finite(ctx, y, op->n)) != LAKER_OK) return st;
    return pcg_solve(ctx, op, P, y, alpha, tol, max_iter, refine_every, info, trace, trace_cap);
}

laker_status laker_pcg_solve_gap(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                                 double* alpha, double R_ref, double gap, double tol, int max_iter, int refine_every,
                                 laker_solve_info* info) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !y || !alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (!(gap > 0.0) || !std::isfinite(R_ref) || R_ref == 0.0)
        return set_error(ctx, LAKER_ERR_ARG, "need gap > 0 and a finite, nonzero R_ref");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    if (P && P->n != op->n) return set_error(ctx, LAKER_ERR_ARG, "preconditioner size mismatch");
    if ((st = scan_finite(ctx, y, op->n)) != LAKER_OK) return st;
    return pcg_solve(ctx, op, P, y, alpha, tol, max_iter, refine_every, info, nullptr, 0, R_ref, gap);
}

laker_status laker_set_wait_budget(laker_ctx* ctx, int64_t cycles) {
    if (!ctx) return LAKER_ERR_ARG;
    if (cycles < 0) return set_error(ctx, LAKER_ERR_ARG, "wait budget must be >= 0");
    ctx->wait_cycles = cycles;
    return LAKER_OK;
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x: the
// negative pivots of the LDL^T factorisation of T - x I (Sturm count).
static int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int count = 0;
    double q = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        q = (a[i] - x) - (i > 0 ? b[i - 1] * b[i - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++count;
    }
    return count;
}

laker_status laker_lanczos_extremes(const double* trace, int k, double* lmin, double* lmax) {
    if (!trace || !lmin || !lmax || k < 1) return LAKER_ERR_ARG;
    std::vector<double> a((size_t)k), b((size_t)std::max(0, k - 1));
    for (int j = 0; j < k; ++j) {
        const double d = trace[4 * j], bp = (j > 0) ? trace[4 * (j - 1) + 3] : 0.0, dp = (j > 0) ? trace[4 * (j - 1)] : 1.0;
        if (!(d > 0.0) || !(bp >= 0.0)) return LAKER_ERR_ARG;
        a[(size_t)j] = 1.0 / d + bp / dp;
        if (j + 1 < k) {
            const double bj = trace[4 * j + 3];
            if (!(bj >= 0.0)) return LAKER_ERR_ARG;
            b[(size_t)j] = std::sqrt(bj) / d;
        }
    }
    double lo = a[0], hi = a[0];
    for (int j = 0; j < k; ++j) {   // Gershgorin interval
        const double r = (j > 0 ? std::fabs(b[(size_t)j - 1]) : 0.0) + (j + 1 < k ? std::fabs(b[(size_t)j]) : 0.0);
        lo = std::min(lo, a[(size_t)j] - r);
        hi = std::max(hi, a[(size_t)j] + r);
    }
    auto kth = [&](int idx) {   // idx-th smallest eigenvalue by bisection
        double l = lo, h = hi;
        for (int it = 0; it < 400 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
            const double mid = 0.5 * (l + h);
            if (sturm_below(a, b, mid) > idx) h = mid;
            else l = mid;
        }
        return 0.5 * (l + h);
    };
    *lmin = kth(0);
    *lmax = kth(k - 1);
    return LAKER_OK;
}

int laker_trace_gap_iterations(const double* trace, int k_max, double R_ref, double gap) {
    if (!trace || k_max < 1 || !(R_ref != 0.0)) return -1;
    for (int k = 0; k < k_max; ++k)
        if (std::fabs(trace[4 * k + 2] - R_ref) <= gap * std::fabs(R_ref)) return k + 1;
    return -1;
}

laker_status laker_pcg_solve_batched(laker_ctx* ctx, int count, const laker_batch_item* items, double tol,
                                     int max_iter, int refine_every, laker_solve_info* infos, double* done_ms) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (count < 1 || !items) return set_error(ctx, LAKER_ERR_ARG, "need count >= 1 and items");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    for (int i = 0; i < count; ++i) {
        if (!items[i].op || !items[i].y || !items[i].alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
        if ((st = scan_finite(ctx, items[i].y, items[i].op->n)) != LAKER_OK) return st;
    }
    return pcg_solve_batched(ctx, count, items, tol, max_iter, refine_every, infos, done_ms);
}

laker_status laker_eval_map_method(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                                   const double* alpha, double* out, int method) {
    laker_status st = check_ctx(ctx);
    if (st != LAKER_OK) return st;
    if (!op || !Qg || !alpha || !out) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
    if (m < 1) return set_error(ctx, LAKER_ERR_ARG, "need m >= 1");
    if (method < LAKER_MAP_AUTO || method > LAKER_MAP_TENSOR) return set_error(ctx, LAKER_ERR_ARG, "unknown map method");
    return eval_map(ctx, op, Qg, m, alpha, out, method);
}

laker_status laker_eval_map(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m, const double* alpha,
                            double* out) {
    return laker_eval_map_method(ctx, op, Qg, m, alpha, out, LAKER_MAP_AUTO);
}

}  // extern "C"
