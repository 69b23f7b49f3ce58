// Batched implicit steps over ensemble members of uneven grids and orders.
//
// Each member is a jfnk context with its own non-blocking stream.  A pool of
// host threads takes members from a shared counter, largest first, and drives
// each member's implicit step (Newton, FGMRES, preconditioner graph) on the
// member's stream, so the GPU runs the members' kernels concurrently: small
// members fill the SMs that large members leave idle between their launches
// and synchronisations.  Members share nothing on the device (own buffers,
// fixed-order reductions), so a member's result is bit-identical alone and in
// any batch.
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

struct jfnk_batch {
    int n;
    std::vector<jfnk_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<int> order;      // members, largest first
    int threads;
    void *desc;                  // device room for the grouped-operator descriptors
};

extern "C" {

int jfnk_batch_create(jfnk_ctx *const *ctxs, int n, int max_threads, jfnk_batch **out) {
    if (!out || !ctxs || n < 1) return JFNK_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return JFNK_EINVAL;
    jfnk_batch *b = new (std::nothrow) jfnk_batch();
    if (!b) return JFNK_ENOMEM;
    b->n = n;
    b->ctx.assign(ctxs, ctxs + n);
    b->streams.assign(n, nullptr);
    for (int i = 0; i < n; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) cudaStreamDestroy(b->streams[j]);
            delete b;
            return JFNK_ECUDA;
        }
    }
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->ctx[x]->N > b->ctx[y]->N; });
    b->threads = max_threads > 0 ? std::min(max_threads, n) : std::min(n, 16);
    b->desc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_jf_device_mu);   // no allocation during another thread's capture
        if (cudaMalloc(&b->desc, dg_member_bytes() * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
            delete b;
            return JFNK_ENOMEM;
        }
    }
    *out = b;
    return JFNK_OK;
}

void jfnk_batch_destroy(jfnk_batch *b) {
    if (!b) return;
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    if (b->desc) {
        std::lock_guard<std::mutex> lock(g_jf_device_mu);
        cudaFree(b->desc);
    }
    delete b;
}

int jfnk_batch_step(jfnk_batch *b, double *const *U, const double *dt, const int *scheme, int *status,
                    jfnk_stats *stats) {
    if (!b || !U || !dt || !scheme) return JFNK_EINVAL;
    for (int i = 0; i < b->n; ++i)
        if (!U[i]) return JFNK_EINVAL;
    std::atomic<int> next(0);
    std::vector<int> rc(b->n, JFNK_OK);
    auto worker = [&]() {
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= b->n) return;
            const int i = b->order[q];
            jfnk_stats st;
            rc[i] = implicit_step(b->ctx[i], U[i], dt[i], scheme[i], &st, b->streams[i]);
            if (stats) stats[i] = st;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < b->threads; ++t) pool.emplace_back(worker);
    worker();
    for (auto &t : pool) t.join();
    int first = JFNK_OK;
    for (int i = 0; i < b->n; ++i) {
        if (status) status[i] = rc[i];
        if (rc[i] != JFNK_OK && first == JFNK_OK) first = rc[i];
    }
    return first;
}

int jfnk_batch_dg_residual(jfnk_batch *b, const double *const *U, double *const *f, void *stream) {
    if (!b) return JFNK_EINVAL;
    return dg_residual_grouped(b->ctx.data(), b->n, U, f, b->desc, (cudaStream_t)stream);
}

}  // extern "C"
