// Many independent PCG solves at once (the PCG stage of Algorithm 1 per
// instance), as concurrent single-instance solves on separate CUDA streams.
//
// The persistent batched solver (laker_batch.cu) advances every instance in
// lock step behind grid-wide barriers: each iteration pays ~45 us of
// barriers and phase latencies whatever the number of active instances, and
// a small instance cannot fill the GPU.  Here each of `streams` host threads
// takes the next instance from a shared counter and runs the single-instance
// solver on its own stream (graph-captured iterations, residual-replacement
// guard), so small instances overlap on the GPU and a finished instance frees
// its stream for the next at once.  The solves allocate nothing: every worker
// owns a preallocated workspace sized for the largest instance, because an
// allocation or a free synchronises the device and would serialise the
// streams.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "laker_internal.h"

extern "C" laker_status laker_pcg_solve_concurrent(laker_ctx* ctx, int count, const laker_batch_item* items,
                                                   double tol, int max_iter, int refine_every, int streams,
                                                   laker_solve_info* infos, double* done_ms) {
    if (!ctx) return LAKER_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, LAKER_ERR_CUDA, "cudaSetDevice failed");
    if (count < 1 || !items) return set_error(ctx, LAKER_ERR_ARG, "need count >= 1 and items");
    if (!(tol >= 0.0) || max_iter < 1 || refine_every < 0) return set_error(ctx, LAKER_ERR_ARG, "bad PCG parameters");
    if (streams < 1 || streams > 64) return set_error(ctx, LAKER_ERR_ARG, "need 1 <= streams <= 64");
    int64_t n_max = 1;
    int nw_max = 1;
    for (int i = 0; i < count; ++i) {
        const laker_batch_item& it = items[i];
        if (!it.op || !it.y || !it.alpha) return set_error(ctx, LAKER_ERR_ARG, "null pointer");
        if (it.P && it.P->n != it.op->n) return set_error(ctx, LAKER_ERR_ARG, "preconditioner size mismatch");
        if (it.op->device != ctx->device) return set_error(ctx, LAKER_ERR_ARG, "operator belongs to another device");
        n_max = std::max(n_max, it.op->n);
        if (it.P) nw_max = std::max(nw_max, it.P->n_w);
        laker_status st = scan_finite(ctx, it.y, it.op->n);
        if (st != LAKER_OK) return st;
    }
    {   // an operator with its own product workspace (matrix-free or packed pair) serves one item only
        std::vector<const laker_op*> ws_ops;
        for (int i = 0; i < count; ++i)
            if (items[i].op->mf || items[i].op->rw) ws_ops.push_back(items[i].op);
        std::sort(ws_ops.begin(), ws_ops.end());
        if (std::adjacent_find(ws_ops.begin(), ws_ops.end()) != ws_ops.end())
            return set_error(ctx, LAKER_ERR_ARG, "a matrix-free or split-bf16 operator appears in two items");
    }
    streams = std::min(streams, count);

    // worker contexts (own stream each) and workspaces, before any worker runs
    std::vector<laker_ctx> wctx((size_t)streams);
    std::vector<PcgArena> arena((size_t)streams);
    cudaEvent_t ready = nullptr;
    laker_status st = LAKER_OK;
    auto cleanup = [&]() {
        for (int w = 0; w < streams; ++w) {
            pcg_arena_free(&arena[(size_t)w]);
            if (wctx[(size_t)w].stream) cudaStreamDestroy(wctx[(size_t)w].stream);
        }
        if (ready) cudaEventDestroy(ready);
    };
    for (int w = 0; w < streams && st == LAKER_OK; ++w) {
        laker_ctx& c = wctx[(size_t)w];
        c.device = ctx->device;
        c.num_sms = ctx->num_sms;
        c.wait_cycles = ctx->wait_cycles;
        if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
            c.stream = nullptr;
            st = set_error(ctx, LAKER_ERR_CUDA, "stream creation failed");
            break;
        }
        c.owns_stream = true;
        st = pcg_arena_alloc(ctx, n_max, nw_max, &arena[(size_t)w]);
    }
    // the inputs were produced on the caller's stream: every worker stream waits for it
    if (st == LAKER_OK && cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess)
        st = set_error(ctx, LAKER_ERR_CUDA, "event creation failed");
    if (st == LAKER_OK && cudaEventRecord(ready, ctx->stream) != cudaSuccess)
        st = set_error(ctx, LAKER_ERR_CUDA, "event record failed");
    for (int w = 0; w < streams && st == LAKER_OK; ++w)
        if (cudaStreamWaitEvent(wctx[(size_t)w].stream, ready, 0) != cudaSuccess)
            st = set_error(ctx, LAKER_ERR_CUDA, "stream wait failed");
    if (st != LAKER_OK) { cleanup(); return st; }

    // an instance no worker took (none could select the device) reports an error, not success
    std::vector<laker_status> status((size_t)count, LAKER_ERR_CUDA);
    std::vector<laker_solve_info> info((size_t)count);
    std::vector<double> done((size_t)count, 0.0);
    std::vector<std::string> why((size_t)count, "not run: no worker thread could select the device");
    std::atomic<int> next{0};
    const auto t0 = std::chrono::steady_clock::now();
    auto worker = [&](int w) {
        laker_ctx& c = wctx[(size_t)w];
        if (cudaSetDevice(c.device) != cudaSuccess) return;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= count) break;
            const laker_batch_item& it = items[i];
            laker_solve_info fi{};
            why[(size_t)i].clear();
            status[(size_t)i] = pcg_solve(&c, it.op, it.P, it.y, it.alpha, tol, max_iter, refine_every, &fi, nullptr,
                                          0, 0.0, 0.0, false, &arena[(size_t)w]);
            if (status[(size_t)i] != LAKER_OK) {
                fi.status = status[(size_t)i];
                why[(size_t)i] = c.last_error;
            }
            info[(size_t)i] = fi;
            done[(size_t)i] =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    };
    // the threads that started take every instance between them; if none
    // could be started the calling thread runs worker 0 itself
    std::vector<std::thread> pool;
    try {
        pool.reserve((size_t)streams);
        for (int w = 0; w < streams; ++w) pool.emplace_back(worker, w);
    } catch (...) {
    }
    for (std::thread& t : pool) t.join();
    if (pool.empty()) worker(0);

    // the worst status: hard errors, then breakdown, then max_iter
    const auto rank = [](laker_status x) {
        return x == LAKER_OK ? 0 : x == LAKER_ERR_MAXITER ? 1 : x == LAKER_ERR_BREAKDOWN ? 2 : 3;
    };
    laker_status worst = LAKER_OK;
    std::string msg;
    for (int i = 0; i < count; ++i) {
        if (infos) {
            infos[i] = info[(size_t)i];
            if (status[(size_t)i] != LAKER_OK) infos[i].status = status[(size_t)i];
        }
        if (done_ms) done_ms[i] = done[(size_t)i];
        if (rank(status[(size_t)i]) > rank(worst)) {
            worst = status[(size_t)i];
            msg = "instance " + std::to_string(i) + ": " + why[(size_t)i];
        }
    }
    for (int w = 0; w < streams; ++w) ctx->launches += wctx[(size_t)w].launches;
    cleanup();
    if (worst != LAKER_OK) return set_error(ctx, worst, "concurrent PCG: " + msg);
    return LAKER_OK;
}
