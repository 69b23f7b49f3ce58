// Batched implicit steps over ensemble members of uneven grids and orders.
//
// Two modes.  Streams: each member is a jfnk context with its own non-blocking
// stream; a pool of host threads takes members from a shared counter, largest
// first, and drives each member's implicit step (Newton, FGMRES, preconditioner
// graph) on the member's stream, so the GPU runs the members' kernels
// concurrently.  Lock-step: one host thread per member runs the same solver
// code, but its launches and stream operations are recorded, not issued
// (t_jf_rec); whenever every unfinished member waits at a synchronisation
// point (a norm or a Hessenberg column read back), the recorded operations of
// all members are replayed on one stream, and at each step of the replay the
// members whose next operation is the same kernel (same body and argument
// types, block shape and shared memory) run it in ONE grouped launch
// (k_grouped): each block finds its member in a table of argument records.
// Members share nothing on the device (own buffers, fixed-order reductions) and
// a grouped block runs the body with its member's arguments, block index and
// block count, so in both modes a member's result is bit-identical alone and in
// any batch.
#include <limits.h>
#include <linux/futex.h>
#include <sys/syscall.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <memory>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "internal.h"

thread_local JfRecorder *t_jf_rec = nullptr;

// ---- stream operations of the solver path (recorded while t_jf_rec is set) ----
cudaError_t jf_memcpy(void *dst, const void *src, size_t n, cudaMemcpyKind kind, cudaStream_t s) {
    if (!t_jf_rec) return cudaMemcpyAsync(dst, src, n, kind, s);
    JfOp op;
    op.glaunch = nullptr;
    op.kernel = false;
    if (kind == cudaMemcpyHostToDevice) {   // the source may be the caller's stack: keep a copy
        auto buf = std::make_shared<std::vector<unsigned char>>((const unsigned char *)src,
                                                                (const unsigned char *)src + n);
        op.run = [=](cudaStream_t st) { return cudaMemcpyAsync(dst, buf->data(), n, kind, st); };
    } else {
        op.run = [=](cudaStream_t st) { return cudaMemcpyAsync(dst, src, n, kind, st); };
    }
    t_jf_rec->ops.push_back(std::move(op));
    return cudaSuccess;
}

cudaError_t jf_memset(void *dst, int v, size_t n, cudaStream_t s) {
    if (!t_jf_rec) return cudaMemsetAsync(dst, v, n, s);
    JfOp op;
    op.glaunch = nullptr;
    op.kernel = false;
    op.run = [=](cudaStream_t st) { return cudaMemsetAsync(dst, v, n, st); };
    t_jf_rec->ops.push_back(std::move(op));
    return cudaSuccess;
}

// Shared state of one lock-step batch step: member states, their recorders and
// the replay's table memory (device tables filled from pinned staging).
// Members and coordinator meet through two futex words, so that a round's
// members wake in parallel instead of one by one through a mutex:
// `pending` counts the members still running in this round (the last to reach
// a synchronisation point or to finish wakes the coordinator), `gen` is bumped
// by the coordinator when the round's replay is complete.
struct JfLockstep {
    std::vector<int> state;   // 0 running, 1 waiting at a synchronisation, 2 finished
    std::vector<JfRecorder> rec;
    std::atomic<int> pending{0};
    std::atomic<int> gen{0};
    cudaError_t err = cudaSuccess;
    cudaStream_t s = nullptr;
    char *dtab = nullptr;
    unsigned char *htab = nullptr;
    size_t cap = 0;
    unsigned long long launches = 0, grouped = 0, member_launches = 0, rounds = 0;
    double ms_members = 0, ms_issue = 0, ms_device = 0;   // host wall clock per phase of the rounds
    bool group = true;   // false: every recorded launch replays alone (the same order)
};

namespace {

static_assert(sizeof(std::atomic<int>) == sizeof(int), "futex word");

void futex_wait(std::atomic<int> *w, int expected) {
    syscall(SYS_futex, reinterpret_cast<int *>(w), FUTEX_WAIT_PRIVATE, expected, nullptr, nullptr, 0);
}
void futex_wake(std::atomic<int> *w) {
    syscall(SYS_futex, reinterpret_cast<int *>(w), FUTEX_WAKE_PRIVATE, INT_MAX, nullptr, nullptr, 0);
}

// A member leaves the running set (state 1: at a synchronisation point, 2: finished).
void member_arrive(JfLockstep *L, int member, int state) {
    L->state[member] = state;
    if (L->pending.fetch_sub(1) == 1) futex_wake(&L->pending);
}

}  // namespace

cudaError_t jf_sync(cudaStream_t s) {
    JfRecorder *r = t_jf_rec;
    if (!r) return cudaStreamSynchronize(s);
    JfLockstep *L = r->ls;
    const int g = L->gen.load();
    member_arrive(L, r->member, 1);
    for (int v = L->gen.load(); v == g; v = L->gen.load()) futex_wait(&L->gen, v);
    return L->err;
}

namespace {

constexpr size_t TAB_ALIGN = 256;

// Replay every member's recorded operations on L->s.  The round is planned
// first: operations that are not launches are taken as soon as they reach the
// head of their member's queue; then one launch kind at the heads is taken once
// for all the members it heads (see the choice below), its argument table
// staged, until every queue is empty.  Then the staged tables go to the device
// in one copy and the planned operations are issued in order.
// One step of a planned round: a member's operation replayed as is (m >= 0), or a
// grouped launch whose table was staged at `off` (m < 0).
struct Action {
    int m;
    size_t i;
    const JfOp *op;
    size_t off;
    int nmem;
    unsigned total;
};

// Issue planned actions: one copy of the staged tables, then the operations in order.
cudaError_t issue(JfLockstep *L, const std::vector<Action> &acts, size_t staged) {
    if (staged) {
        const cudaError_t e = cudaMemcpyAsync(L->dtab, L->htab, staged, cudaMemcpyHostToDevice, L->s);
        if (e != cudaSuccess) return e;
    }
    for (const Action &a : acts) {
        const cudaError_t e = a.m >= 0 ? a.op->run(L->s)
                                       : a.op->glaunch(L->dtab + a.off, a.nmem, a.total, a.op->block, a.op->smem, L->s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t replay(JfLockstep *L) {
    using Key = std::tuple<const void *, unsigned, unsigned, unsigned, size_t>;
    auto key_of = [](const JfOp &o) {
        return Key{(const void *)o.glaunch, o.block.x, o.block.y, o.block.z, o.smem};
    };
    const int n = (int)L->rec.size();
    std::vector<size_t> h(n, 0);
    // the groupable launches each member has still to make in this round, by kind
    std::vector<std::map<Key, int>> left(n);
    for (int m = 0; m < n; ++m)
        for (const JfOp &o : L->rec[m].ops)
            if (o.glaunch) ++left[m][key_of(o)];
    size_t off = 0;
    std::vector<int> sel;
    std::vector<Action> acts;
    for (;;) {
        bool any = false;
        for (int m = 0; m < n; ++m) {
            std::vector<JfOp> &ops = L->rec[m].ops;
            while (h[m] < ops.size() && !ops[h[m]].glaunch) {
                acts.push_back(Action{m, h[m], &ops[h[m]], 0, 0, 0});
                if (ops[h[m]].kernel) {
                    ++L->launches;
                    ++L->member_launches;
                }
                ++h[m];
            }
            if (h[m] < ops.size()) any = true;
        }
        if (!any) return issue(L, acts, off);
        // Choose the kind to launch: a kind at some heads that no other member will
        // still need later in this round (launching it now loses no member), the one
        // whose members have the most operations left; if every kind at the heads is
        // still needed by members behind, the kind whose members have the most
        // operations left (members that are behind advance first)
        std::map<Key, size_t> weight;
        std::map<Key, int> heads;
        for (int m = 0; m < n; ++m) {
            if (h[m] >= L->rec[m].ops.size()) continue;
            const Key k = key_of(L->rec[m].ops[h[m]]);
            weight[k] += L->rec[m].ops.size() - h[m];
            ++heads[k];
        }
        const Key *best = nullptr;
        bool best_free = false;
        size_t best_w = 0;
        for (const auto &kv : weight) {
            int later = 0;   // members not at this kind now that still need it
            for (int m = 0; m < n; ++m) {
                if (h[m] >= L->rec[m].ops.size()) continue;
                auto it = left[m].find(kv.first);
                const int need = it == left[m].end() ? 0 : it->second;
                if (need > 0 && !(key_of(L->rec[m].ops[h[m]]) == kv.first)) ++later;
            }
            const bool free = later == 0;
            if (!best || (free && !best_free) || (free == best_free && kv.second > best_w)) {
                best = &kv.first;
                best_free = free;
                best_w = kv.second;
            }
        }
        const Key k = *best;
        sel.clear();
        for (int m = 0; m < n; ++m)
            if (h[m] < L->rec[m].ops.size() && key_of(L->rec[m].ops[h[m]]) == k) sel.push_back(m);
        L->member_launches += sel.size();
        ++L->launches;
        for (int m : sel) --left[m][k];
        const JfOp &o0 = L->rec[sel[0]].ops[h[sel[0]]];
        if (!L->group) {   // every member alone, in member order
            for (int m : sel) {
                acts.push_back(Action{m, h[m], &L->rec[m].ops[h[m]], 0, 0, 0});
                ++h[m];
            }
            L->launches += sel.size() - 1;
            continue;
        }
        if (sel.size() == 1) {   // alone: the member's own launch
            acts.push_back(Action{sel[0], h[sel[0]], &o0, 0, 0, 0});
            ++h[sel[0]];
            continue;
        }
        const size_t es = o0.ent.size(), bytes = es * sel.size();
        if (bytes > L->cap) return cudaErrorInvalidValue;
        if (off + bytes > L->cap) {   // staging full: issue what is planned and let it drain
            cudaError_t e = issue(L, acts, off);
            if (e == cudaSuccess) e = cudaStreamSynchronize(L->s);
            if (e != cudaSuccess) return e;
            acts.clear();
            off = 0;
        }
        unsigned total = 0;
        for (size_t q = 0; q < sel.size(); ++q) {
            const JfOp &o = L->rec[sel[q]].ops[h[sel[q]]];
            unsigned char *dst = L->htab + off + q * es;
            memcpy(dst, o.ent.data(), es);
            memcpy(dst, &total, sizeof(unsigned));   // JfEnt::b0
            total += o.nb;
        }
        acts.push_back(Action{-1, 0, &o0, off, (int)sel.size(), total});
        ++L->grouped;
        off += (bytes + TAB_ALIGN - 1) / TAB_ALIGN * TAB_ALIGN;
        for (int m : sel) ++h[m];
    }
}

}  // namespace

struct jfnk_batch {
    int n;
    std::vector<jfnk_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<int> order;      // members, largest first
    int threads;
    void *desc;                  // device room for the grouped-operator descriptors
    int mode;                    // JFNK_BATCH_STREAMS / JFNK_BATCH_LOCKSTEP
    char *dtab;                  // lock-step replay tables (device) and their pinned staging
    unsigned char *htab;
    size_t tab_cap;
    unsigned long long last_launches, last_grouped, last_member_launches, last_rounds;
    double last_ms[3];
};

namespace {

// One class of members (one order k) in lock-step: wait until none of them is
// running, replay what they recorded, wait for the device, release them.
void coordinate(JfLockstep &L) {
    using clk = std::chrono::steady_clock;
    auto ms = [](clk::time_point a, clk::time_point b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
    for (;;) {
        const auto t0 = clk::now();
        for (int v = L.pending.load(); v != 0; v = L.pending.load()) futex_wait(&L.pending, v);
        bool done = true;
        for (int x : L.state)
            if (x != 2) done = false;
        const auto t1 = clk::now();
        cudaError_t e = L.err == cudaSuccess ? replay(&L) : L.err;
        const auto t2 = clk::now();
        const cudaError_t es = cudaStreamSynchronize(L.s);
        const auto t3 = clk::now();
        L.ms_members += ms(t0, t1);
        L.ms_issue += ms(t1, t2);
        L.ms_device += ms(t2, t3);
        if (e == cudaSuccess) e = es;
        ++L.rounds;
        for (auto &r : L.rec) r.ops.clear();
        L.err = e;
        if (done) return;
        int run = 0;
        for (int &x : L.state)
            if (x == 1) {
                x = 0;
                ++run;
            }
        L.pending.store(run);
        L.gen.fetch_add(1);
        futex_wake(&L.gen);
    }
}

// Members of the same order share the grouped launches of their class; the
// classes run concurrently, each replayed on its own stream by its own
// coordinator thread (the stream of its first member).
int lockstep_step(jfnk_batch *b, double *const *U, const double *dt, const int *scheme, std::vector<int> &rc,
                  jfnk_stats *stats) {
    const int n = b->n;
    std::vector<int> cls_of(n);
    std::vector<std::vector<int>> cls;
    for (int np1 = 2; np1 <= 5; ++np1) {
        std::vector<int> m;
        for (int i = 0; i < n; ++i)
            if (b->ctx[i]->np1 == np1) m.push_back(i);
        if (m.empty()) continue;
        for (int i : m) cls_of[i] = (int)cls.size();
        cls.push_back(m);
    }
    const int nc = (int)cls.size();
    const size_t cap = b->tab_cap / (size_t)nc / 256 * 256;
    std::vector<std::unique_ptr<JfLockstep>> Ls;
    for (int q = 0; q < nc; ++q) {
        Ls.emplace_back(new JfLockstep());
        JfLockstep &L = *Ls.back();
        const int nm = (int)cls[q].size();
        L.state.assign(nm, 0);
        L.pending.store(nm);
        L.rec.resize(nm);
        L.s = b->streams[cls[q][0]];
        L.dtab = b->dtab + (size_t)q * cap;
        L.htab = b->htab + (size_t)q * cap;
        L.cap = cap;
        L.group = b->mode == JFNK_BATCH_LOCKSTEP;
        for (int j = 0; j < nm; ++j) {
            L.rec[j].ls = &L;
            L.rec[j].member = j;
        }
    }
    std::vector<std::thread> pool;
    for (int i = 0; i < n; ++i) {
        JfLockstep &L = *Ls[cls_of[i]];
        const int j = (int)(std::find(cls[cls_of[i]].begin(), cls[cls_of[i]].end(), i) - cls[cls_of[i]].begin());
        pool.emplace_back([&, i, j]() {
            t_jf_rec = &L.rec[j];
            jfnk_stats st;
            rc[i] = implicit_step(b->ctx[i], U[i], dt[i], scheme[i], &st, b->streams[i]);
            t_jf_rec = nullptr;
            if (stats) stats[i] = st;
            member_arrive(&L, j, 2);
        });
    }
    std::vector<std::thread> coords;
    for (int q = 1; q < nc; ++q) coords.emplace_back([&, q]() { coordinate(*Ls[q]); });
    coordinate(*Ls[0]);
    for (auto &t : coords) t.join();
    for (auto &t : pool) t.join();
    b->last_launches = b->last_grouped = b->last_member_launches = b->last_rounds = 0;
    b->last_ms[0] = b->last_ms[1] = b->last_ms[2] = 0.0;
    int rcode = JFNK_OK;
    for (auto &Lp : Ls) {
        const JfLockstep &L = *Lp;
        b->last_launches += L.launches;
        b->last_grouped += L.grouped;
        b->last_member_launches += L.member_launches;
        b->last_rounds = std::max(b->last_rounds, L.rounds);
        b->last_ms[0] = std::max(b->last_ms[0], L.ms_members);
        b->last_ms[1] = std::max(b->last_ms[1], L.ms_issue);
        b->last_ms[2] = std::max(b->last_ms[2], L.ms_device);
        if (L.err != cudaSuccess) rcode = JFNK_ECUDA;
    }
    __atomic_fetch_add(&g_jf_launches, b->last_launches, __ATOMIC_RELAXED);
    return rcode;
}

}  // namespace

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
    b->mode = JFNK_BATCH_STREAMS;
    b->dtab = nullptr;
    b->htab = nullptr;
    b->tab_cap = 0;
    b->last_launches = b->last_grouped = b->last_member_launches = b->last_rounds = 0;
    b->last_ms[0] = b->last_ms[1] = b->last_ms[2] = 0.0;
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
    {
        std::lock_guard<std::mutex> lock(g_jf_device_mu);
        if (b->desc) cudaFree(b->desc);
        if (b->dtab) cudaFree(b->dtab);
        if (b->htab) cudaFreeHost(b->htab);
    }
    delete b;
}

int jfnk_batch_set_mode(jfnk_batch *b, int mode) {
    if (!b || mode < JFNK_BATCH_STREAMS || mode > JFNK_BATCH_LOCKSTEP_UNGROUPED) return JFNK_EINVAL;
    if (mode != JFNK_BATCH_STREAMS && !b->dtab) {
        // room for the argument tables of one replay round: every member's
        // recorded launches between two synchronisation points
        const size_t cap = (size_t)64 << 20;
        std::lock_guard<std::mutex> lock(g_jf_device_mu);
        if (cudaMalloc(&b->dtab, cap) != cudaSuccess) {
            cudaGetLastError();
            b->dtab = nullptr;
            return JFNK_ENOMEM;
        }
        if (cudaMallocHost(&b->htab, cap) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(b->dtab);
            b->dtab = nullptr;
            b->htab = nullptr;
            return JFNK_ENOMEM;
        }
        b->tab_cap = cap;
    }
    b->mode = mode;
    return JFNK_OK;
}

int jfnk_batch_last_launches(const jfnk_batch *b, unsigned long long *launches, unsigned long long *grouped,
                             unsigned long long *member_launches, unsigned long long *rounds) {
    if (!b) return JFNK_EINVAL;
    if (launches) *launches = b->last_launches;
    if (grouped) *grouped = b->last_grouped;
    if (member_launches) *member_launches = b->last_member_launches;
    if (rounds) *rounds = b->last_rounds;
    return JFNK_OK;
}

int jfnk_batch_last_times(const jfnk_batch *b, double *ms3) {
    if (!b || !ms3) return JFNK_EINVAL;
    for (int i = 0; i < 3; ++i) ms3[i] = b->last_ms[i];
    return JFNK_OK;
}

int jfnk_batch_step(jfnk_batch *b, double *const *U, const double *dt, const int *scheme, int *status,
                    jfnk_stats *stats) {
    if (!b || !U || !dt || !scheme) return JFNK_EINVAL;
    for (int i = 0; i < b->n; ++i)
        if (!U[i]) return JFNK_EINVAL;
    std::vector<int> rc(b->n, JFNK_OK);
    if (b->mode != JFNK_BATCH_STREAMS) {
        const int lr = lockstep_step(b, U, dt, scheme, rc, stats);
        int first = lr;
        for (int i = 0; i < b->n; ++i) {
            if (status) status[i] = rc[i];
            if (rc[i] != JFNK_OK && first == JFNK_OK) first = rc[i];
        }
        return first;
    }
    std::atomic<int> next(0);
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
