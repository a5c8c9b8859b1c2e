// serve.cu -- the serving loop: force requests of many independent systems (the
// concurrent cluster simulations of a served stream) are queued as they arrive and
// evaluated by a few slots with continuous batching.  A slot that becomes free takes
// every queued request that fits its share of the memory budget and evaluates them
// together as one forest (fmm_evaluate_batch), so small requests share launches and
// requests arriving while other batches run go into the next free slot; slots run
// on their own streams, so their work overlaps on the device.  A result is the one
// the system gets alone: the forest evaluation keeps every system's tree, lists and
// summation order (checked bit for bit by the tests).
//
// Memory: a registered system has a footprint (fmm_footprint_bytes for its N and the
// context's parameters); registration is refused (FMM_E_ADMISSION) when that is more
// than one slot's share of the budget, and a batch never holds more than one share.
// Every slot keeps its workspace (tree, expansions, lists, staging) allocated between
// batches, so a steady stream of requests allocates nothing.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "serve.cuh"

namespace gb3 {

using clk = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int sys = -1;
    int64_t n = 0;
    const double* x = nullptr;
    const double* mu = nullptr;
    double G = 1.0;
    double* psi = nullptr;
    double* acc = nullptr;
    clk::time_point t_submit, t_done;
    int rc = 0;
    bool done = false;
    char err[200] = {0};
};

struct System {
    int64_t n = 0;
    uint64_t footprint = 0;
    bool live = false;
    bool in_flight = false;
};

struct Slot {
    std::thread th;
    cudaStream_t stream = nullptr;
    fmm_ctx* sub = nullptr;
    // staging of a multi-request batch: x [n][3], mu, psi, acc [n][3]
    double *sx = nullptr, *smu = nullptr, *spsi = nullptr, *sacc = nullptr;
    int64_t cap = 0;
};

struct Serve {
    fmm_params prm;
    int device = 0;
    uint64_t budget = 0, share = 0;
    int nslots = 2;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    std::vector<System> systems;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<Slot> slots;
};

static void free_staging(Slot& sl) {
    double** ps[] = {&sl.sx, &sl.smu, &sl.spsi, &sl.sacc};
    for (double** p : ps) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    sl.cap = 0;
}

static int grow_staging(Slot& sl, int64_t n) {
    if (n <= sl.cap) return 0;
    free_staging(sl);
    const int64_t want = n + n / 4 + 1024;
    if (cudaMalloc(&sl.sx, sizeof(double) * 3 * want) != cudaSuccess ||
        cudaMalloc(&sl.smu, sizeof(double) * want) != cudaSuccess ||
        cudaMalloc(&sl.spsi, sizeof(double) * want) != cudaSuccess ||
        cudaMalloc(&sl.sacc, sizeof(double) * 3 * want) != cudaSuccess) {
        cudaGetLastError();
        free_staging(sl);
        return FMM_E_OOM;
    }
    sl.cap = want;
    return 0;
}

static void fail_all(std::vector<Request*>& batch, int rc, const char* msg) {
    for (Request* r : batch) {
        r->rc = rc;
        snprintf(r->err, sizeof r->err, "%s", msg ? msg : fmm_strerror(rc));
    }
}

#define SLOT_CU(expr)                                                   \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) {                                        \
            fail_all(batch, FMM_E_CUDA, cudaGetErrorString(_e));        \
            return;                                                     \
        }                                                               \
    } while (0)

static void run_batch(Slot& sl, std::vector<Request*>& batch) {
    if (batch.size() == 1) {  // one request: evaluate in place
        Request* r = batch[0];
        int rc = fmm_evaluate(sl.sub, r->n, r->x, r->mu, r->G, nullptr, r->psi, r->acc, sl.stream, nullptr);
        if (rc) {
            fail_all(batch, rc, fmm_last_error(sl.sub));
            return;
        }
        SLOT_CU(cudaStreamSynchronize(sl.stream));
        return;
    }
    const int k = (int)batch.size();
    std::vector<int64_t> off(k + 1, 0);
    std::vector<double> G(k);
    for (int i = 0; i < k; ++i) {
        off[i + 1] = off[i] + batch[i]->n;
        G[i] = batch[i]->G;
    }
    int rc = grow_staging(sl, off[k]);
    if (rc) {
        fail_all(batch, rc, "staging allocation failed");
        return;
    }
    for (int i = 0; i < k; ++i) {
        const Request* r = batch[i];
        if (!r->n) continue;
        SLOT_CU(cudaMemcpyAsync(sl.sx + 3 * off[i], r->x, sizeof(double) * 3 * r->n, cudaMemcpyDeviceToDevice, sl.stream));
        SLOT_CU(cudaMemcpyAsync(sl.smu + off[i], r->mu, sizeof(double) * r->n, cudaMemcpyDeviceToDevice, sl.stream));
    }
    rc = fmm_evaluate_batch(sl.sub, k, off.data(), sl.sx, sl.smu, G.data(), sl.spsi, sl.sacc, sl.stream, nullptr);
    if (rc) {
        fail_all(batch, rc, fmm_last_error(sl.sub));
        return;
    }
    for (int i = 0; i < k; ++i) {
        const Request* r = batch[i];
        if (!r->n) continue;
        SLOT_CU(cudaMemcpyAsync(r->psi, sl.spsi + off[i], sizeof(double) * r->n, cudaMemcpyDeviceToDevice, sl.stream));
        SLOT_CU(cudaMemcpyAsync(r->acc, sl.sacc + 3 * off[i], sizeof(double) * 3 * r->n, cudaMemcpyDeviceToDevice,
                                sl.stream));
    }
    SLOT_CU(cudaStreamSynchronize(sl.stream));
}

static void slot_loop(Serve* S, int w) {
    Slot& sl = S->slots[w];
    cudaSetDevice(S->device);
    std::vector<Request*> batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
            if (S->queue.empty()) return;  // stopping, and nothing left to do
            batch.clear();
            uint64_t fp = 0;
            while (!S->queue.empty()) {
                Request* r = S->queue.front();
                const uint64_t f = S->systems[r->sys].footprint;
                if (!batch.empty() && fp + f > S->share) break;
                batch.push_back(r);
                fp += f;
                S->queue.pop_front();
            }
        }
        run_batch(sl, batch);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const clk::time_point now = clk::now();
            for (Request* r : batch) {
                r->done = true;
                r->t_done = now;
                S->systems[r->sys].in_flight = false;
            }
        }
        S->cv_done.notify_all();
    }
}

// start the slots (first registration); the caller holds S->mu
static int start_slots(fmm_ctx* ctx, Serve* S) {
    if (!S->slots.empty()) return 0;
    if (S->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, FMM_E_CUDA, "cudaMemGetInfo failed");
        }
        S->budget = (uint64_t)(0.8 * (double)fr);
    }
    S->share = S->budget / (uint64_t)S->nslots;
    S->slots.resize(S->nslots);
    for (Slot& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return ctx_fail(ctx, FMM_E_CUDA, "cudaStreamCreate failed");
        }
        int rc = fmm_create(&sl.sub, &S->prm, S->device);
        if (rc) return ctx_fail(ctx, rc, "creating a slot context failed");
    }
    for (int w = 0; w < S->nslots; ++w) S->slots[w].th = std::thread(slot_loop, S, w);
    return 0;
}

static Serve* serve_of(fmm_ctx* ctx, bool create) {
    Serve*& s = ctx_serve(ctx);
    if (!s && create) {
        s = new (std::nothrow) Serve();
        if (s) {
            s->prm = *ctx_params(ctx);
            s->device = ctx_device(ctx);
        }
    }
    return s;
}

void serve_destroy(Serve* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (Slot& sl : S->slots)
        if (sl.th.joinable()) sl.th.join();
    for (Slot& sl : S->slots) {
        free_staging(sl);
        if (sl.sub) fmm_destroy(sl.sub);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

uint64_t serve_workspace_bytes(Serve* S) {
    if (!S) return 0;
    uint64_t b = 0;
    for (Slot& sl : S->slots) b += fmm_workspace_bytes(sl.sub) + (uint64_t)sl.cap * 8 * sizeof(double);
    return b;
}

}  // namespace gb3

using namespace gb3;

extern "C" {

int fmm_serve_config(fmm_ctx* ctx, uint64_t budget_bytes, int slots) {
    if (!ctx || slots < 0 || slots > 16) return FMM_E_INVALID;
    Serve* S = serve_of(ctx, true);
    if (!S) return FMM_E_OOM;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->slots.empty()) return ctx_fail(ctx, FMM_E_BUSY, "the serving loop is already running");
    S->budget = budget_bytes;
    S->nslots = slots ? slots : 2;
    return 0;
}

int fmm_system_register(fmm_ctx* ctx, int64_t n, int* sys_id) {
    if (!ctx || !sys_id || n < 0 || n > 0x7fffffffLL) return FMM_E_INVALID;
    *sys_id = -1;
    Serve* S = serve_of(ctx, true);
    if (!S) return FMM_E_OOM;
    std::lock_guard<std::mutex> lk(S->mu);
    int rc = start_slots(ctx, S);
    if (rc) return rc;
    const uint64_t f = (uint64_t)fmm_footprint_bytes(&S->prm, n);
    if (f > S->share) {
        char msg[160];
        snprintf(msg, sizeof msg, "footprint %llu bytes above the slot budget %llu", (unsigned long long)f,
                 (unsigned long long)S->share);
        return ctx_fail(ctx, FMM_E_ADMISSION, msg);
    }
    System sy;
    sy.n = n;
    sy.footprint = f;
    sy.live = true;
    for (size_t i = 0; i < S->systems.size(); ++i)
        if (!S->systems[i].live) {
            S->systems[i] = sy;
            *sys_id = (int)i;
            return 0;
        }
    S->systems.push_back(sy);
    *sys_id = (int)S->systems.size() - 1;
    return 0;
}

int fmm_submit(fmm_ctx* ctx, int sys_id, const double* x, const double* mu, double G, double* psi, double* acc,
               uint64_t* ticket) {
    if (!ctx || !ticket) return FMM_E_INVALID;
    *ticket = 0;
    Serve* S = serve_of(ctx, false);
    if (!S) return ctx_fail(ctx, FMM_E_NOTFOUND, "no system registered");
    if (!std::isfinite(G)) return ctx_fail(ctx, FMM_E_INVALID, "G is not finite");
    Request* r = new (std::nothrow) Request();
    if (!r) return FMM_E_OOM;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (sys_id < 0 || sys_id >= (int)S->systems.size() || !S->systems[sys_id].live) {
            delete r;
            return ctx_fail(ctx, FMM_E_NOTFOUND, "unknown system id");
        }
        System& sy = S->systems[sys_id];
        if (sy.n > 0 && (!x || !mu || !psi || !acc)) {
            delete r;
            return ctx_fail(ctx, FMM_E_INVALID, "NULL buffer");
        }
        if (sy.in_flight) {
            delete r;
            return ctx_fail(ctx, FMM_E_BUSY, "the system has a request in flight");
        }
        sy.in_flight = true;
        r->ticket = S->next_ticket++;
        r->sys = sys_id;
        r->n = sy.n;
        r->x = x;
        r->mu = mu;
        r->G = G;
        r->psi = psi;
        r->acc = acc;
        r->t_submit = clk::now();
        S->reqs[r->ticket] = r;
        S->queue.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return 0;
}

int fmm_poll(fmm_ctx* ctx, uint64_t ticket, int timeout_ms, double* latency_s) {
    if (!ctx) return FMM_E_INVALID;
    Serve* S = serve_of(ctx, false);
    if (!S) return ctx_fail(ctx, FMM_E_NOTFOUND, "unknown ticket");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return ctx_fail(ctx, FMM_E_NOTFOUND, "unknown ticket");
    Request* r = it->second;
    if (!r->done && timeout_ms != 0) {
        auto pred = [&] { return r->done; };
        if (timeout_ms < 0) S->cv_done.wait(lk, pred);
        else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    }
    if (!r->done) return FMM_E_BUSY;
    const int rc = r->rc;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (rc) ctx_fail(ctx, rc, r->err);
    S->reqs.erase(it);
    delete r;
    return rc;
}

int fmm_system_release(fmm_ctx* ctx, int sys_id) {
    if (!ctx) return FMM_E_INVALID;
    Serve* S = serve_of(ctx, false);
    if (!S) return ctx_fail(ctx, FMM_E_NOTFOUND, "unknown system id");
    std::lock_guard<std::mutex> lk(S->mu);
    if (sys_id < 0 || sys_id >= (int)S->systems.size() || !S->systems[sys_id].live)
        return ctx_fail(ctx, FMM_E_NOTFOUND, "unknown system id");
    if (S->systems[sys_id].in_flight) return ctx_fail(ctx, FMM_E_BUSY, "the system has a request in flight");
    S->systems[sys_id].live = false;
    return 0;
}

}  // extern "C"
