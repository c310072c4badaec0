// Host-side internals shared by the CUDA translation units of liblaker.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/laker.h"

// Device-resident PCG scalars.  All reductions that feed them are done in a
// fixed order, so a solve is bit-reproducible for a given launch shape.
struct PcgScalars {
    double rz;          // r^T z of the current iterate
    double pAp;         // p^T (lambda I + G) p
    double delta;       // step length
    double beta;        // conjugation coefficient
    double rr;          // |r|^2 of the recursive residual
    double yy;          // |y|^2
    double tol2yy;      // tol^2 |y|^2
    double rr_true;     // |y - A alpha|^2 at the last true-residual step
    int converged;      // 0 running, 1 converged, 2 breakdown, 3 max iterations, 4 stagnated
    int iters;          // operator products so far
    int need_true;      // the next true-residual step must run
    int true_count;     // true residuals computed
    int max_iter;
    int refine_every;   // 0 = never replace the residual
    int pad0, pad1;
    unsigned int ticket[8];
    double* trace;      // per product k: delta, |r|^2/|y|^2, R(alpha), beta (4 doubles), or null
    int trace_cap;      // products the trace holds
    int pad2;
    double R_ref;       // reference objective of the gap stop
    double gap_tol;     // > 0: stop once |R(alpha) - R_ref| <= gap_tol |R_ref|
    // Guard of the mixed forms (residual replacement with an inexact operator)
    double rr_best;     // lowest true |r|^2 seen at a replacement (HUGE_VAL before the first)
    int interval;       // current replacement interval (starts at refine_every)
    int since_true;     // products since the last replacement
    int restarts;       // roll-backs to the best iterate
    int guard_action;   // 1: save alpha, r as the best iterate; 2: restore them
    int restart_dir;    // 1: the next direction is the preconditioned residual (beta = 0)
    int breakdown;      // p^T A p <= 0 in a mixed solve: replace and roll back
    int grow;           // replacements in a row more than 30x above the best
    int pad3;
};

struct laker_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int num_sms = 0;
    int64_t launches = 0;
    int64_t wait_cycles = 0;    // budget of bounded device waits (0 = the default, ~2 s)
    std::string last_error;
};

struct laker_op {
    laker_ctx* ctx = nullptr;
    int device = 0;           // the context's device, kept for destroy
    int64_t n = 0;
    int d = 0;
    int dpad = 0;             // d rounded up to a multiple of 16 (bf16 operands)
    int64_t ldk = 0;          // leading dimension of materialised G (multiple of 4)
    double scale = 1.0;
    double lambda = 0.0;
    int precision = LAKER_FP64;
    int variant = LAKER_MATERIALISED;
    double* Q64 = nullptr;    // n x d
    uint16_t* Qhi = nullptr;  // n x dpad bf16, high part of Q * sqrt(scale * log2 e)
    uint16_t* Qlo = nullptr;  // n x dpad bf16, low part
    float* Q32 = nullptr;     // n x d float copy
    double* K64 = nullptr;    // n x ldk, G in float64 (float64 operators)
    float* K32 = nullptr;     // n x ldk, G rounded to float (mixed operators)
    float* K32lo = nullptr;   // n x ldk, G - K32 rounded to float: K32 + K32lo is G to ~2^-48
    double* diagA = nullptr;  // n, lambda + G_ii
    void* mf = nullptr;       // matrix-free operator workspace (tensor maps, buffers)
    void* rw = nullptr;       // packed float32 pair and schedule of the float64-accurate product (BF16X3)
    double t_mat_ms = 0.0;    // product times measured by the AUTO variant choice (0 if not measured)
    double t_mf_ms = 0.0;
};

// Largest number of random directions N_r (a preconditioner apply keeps the
// N_r-vector U^T r in shared memory).
constexpr int LK_MAX_NR = 2048;

enum PrecondKind { PRECOND_IDENTITY = 0, PRECOND_JACOBI = 1, PRECOND_CCCP = 2 };

struct laker_precond {
    laker_ctx* ctx = nullptr;
    int device = 0;           // the context's device, kept for destroy
    int kind = PRECOND_IDENTITY;
    int64_t n = 0;
    int n_r = 0;
    int n_w = 0;              // columns of the apply form (UT, W): n_r, or the kept eigen-directions
    double c = 1.0;           // Sigma_* = c I + U diag(D) U^T
    double cinvsqrt = 1.0;    // c^{-1/2}
    double* D = nullptr;      // n_r
    double* U64 = nullptr;    // n x n_r, unit columns u_bar_k
    double* W64 = nullptr;    // n x n_r, W = U B with P = c^{-1/2} I + W U^T
    float* W32 = nullptr;     // n x ldw (zero padding), float32 applies
    int ldw = 0;              // row pitch of W32: n_r rounded up to 4
    int64_t ldu = 0;          // row pitch of UT (n rounded up to 4)
    double* UT64 = nullptr;   // n_r x ldu, U transposed (float64 applies)
    float* UT32 = nullptr;    // n_r x ldu, U transposed (float32 applies)
    double* dinv = nullptr;   // Jacobi: 1/diag(A)
    bool use32 = false;       // apply in float32 (mixed solves)
    float* feat = nullptr;    // n_r x 2: [log |u_k|, sum_j M_kj^2] (inputs of the learned start)
};

// ---- error plumbing ------------------------------------------------------
laker_status set_error(laker_ctx* ctx, laker_status st, const std::string& msg);
#define LK_CUDA(ctx, call)                                                          \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return set_error((ctx), LAKER_ERR_CUDA,                                 \
                             std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)
#define LK_LAUNCHED(ctx)                                                            \
    do {                                                                            \
        (ctx)->launches++;                                                          \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess)                                                      \
            return set_error((ctx), LAKER_ERR_CUDA,                                 \
                             std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

laker_status lk_malloc(laker_ctx* ctx, void** p, size_t bytes);

// ---- translation-unit entry points ---------------------------------------
// laker_build.cu
// prev (may be null): the same operator over the first prev->n points, whose
// stored entries are reused (streaming append)
laker_status build_operator(laker_ctx* ctx, laker_op* op, const laker_op* prev = nullptr);
laker_status copy_packed_tiles(laker_ctx* ctx, const float* src, int nb_src, float* dst, int nb, int J0);
laker_status op_matvec_inner(laker_ctx* ctx, const laker_op* op, const double* x, double* w);
laker_status op_matvec_fp64(laker_ctx* ctx, const laker_op* op, const double* x, double* w);
// laker_pcg.cu
// Preallocated buffers for solves that must not allocate (concurrent solves
// on several streams: an allocation or free would synchronise the device).
struct PcgArena {
    double* base = nullptr;        // 8 n_cap doubles
    int64_t n_cap = 0;
    double* partials = nullptr;
    int64_t partials_cap = 0;
    void* t = nullptr;             // t_cap doubles
    int64_t t_cap = 0;
    PcgScalars* sc = nullptr;
    int* flag_host = nullptr;      // pinned
};
// LAKER_ERR_NONFINITE if any of x[0..count) (device) is NaN or Inf
laker_status scan_finite(laker_ctx* ctx, const double* x, int64_t count);
laker_status pcg_arena_alloc(laker_ctx* ctx, int64_t n_max, int nw_max, PcgArena* a);
void pcg_arena_free(PcgArena* a);
laker_status pcg_solve(laker_ctx* ctx, const laker_op* op, const laker_precond* P,
                       const double* y, double* alpha, double tol, int max_iter,
                       int refine_every, laker_solve_info* info, double* trace = nullptr,
                       int trace_cap = 0, double R_ref = 0.0, double gap_tol = 0.0, bool warm = false,
                       const PcgArena* arena = nullptr);
laker_status precond_apply(laker_ctx* ctx, const laker_precond* P, const double* r, double* z);
// laker_fit.cu
laker_status fit_cccp(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r,
                      double gamma, double rho, double eps, int max_iter, double tol,
                      laker_precond* P, laker_fit_info* info,
                      laker_setnet* net = nullptr, const float* X = nullptr, int mode = 0,
                      const laker_precond* warm = nullptr);
// laker_map.cu
laker_status eval_map(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                      const double* alpha, double* out, int method);
// laker_map_tc.cu (tensor-core map; *applied = false when its logit bound fails)
laker_status eval_map_tc(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                         const double* alpha, double* out, bool* applied);
// laker_mf.cu (matrix-free operator)
laker_status mf_prepare(laker_ctx* ctx, laker_op* op);
void mf_release(laker_op* op);
laker_status mf_status(laker_ctx* ctx, const laker_op* op);
laker_status mf_time_main(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms);
laker_status op_time_materialised(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms);
laker_status op_time_product(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms);
// laker_dirs_tc.cu (tensor-core random directions (lambda I + G) Z~, Z~ = bf16(Z))
bool dirs_tc_supported(const laker_op* op);
laker_status dirs_tc(laker_ctx* ctx, const laker_op* op, const double* Z, int nr, double* U);
// laker_resid.cu (float64-accurate product from the packed upper-triangular pair)
laker_status resid_prepare(laker_ctx* ctx, laker_op* op, float** Kp);
void resid_release(laker_op* op);
laker_status resid_build_df(laker_ctx* ctx, const laker_op* op, const laker_op* prev = nullptr);
const float* resid_packed(const laker_op* op);   // the packed pair of a split-bf16 operator
laker_status resid_status(laker_ctx* ctx, const laker_op* op);
laker_status resid_matvec(laker_ctx* ctx, const laker_op* op, const double* x, double* w, const PcgScalars* sc,
                          int gate);
// laker_rng.cu (Philox4x32-10 Gaussian directions, n_r-major rows)
laker_status random_directions(laker_ctx* ctx, uint64_t seed, int64_t count, double* Z);
// laker_setnet.cu
laker_status setnet_predict(laker_ctx* ctx, laker_setnet* s, int64_t n, const float* X, int nr, const float* F,
                            const float** logc, const float** logD);
int setnet_in_dim(const laker_setnet* s);
// laker_batch.cu
laker_status pcg_solve_batched(laker_ctx* ctx, int count, const laker_batch_item* items, double tol, int max_iter,
                               int refine_every, laker_solve_info* infos, double* done_ms);
laker_status mf_matvec_launch(laker_ctx* ctx, const laker_op* op, const double* pin,
                              const double* z, double* pout, double* w, PcgScalars* sc,
                              double* partials, int fuse_p, float* pbuf, float* wbuf);
