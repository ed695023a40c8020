// Serving form: a request loop with continuous batching over one index.
//
// Requests (one query each, with its own k and nprobe) are queued by
// fa_server_submit. A dispatcher thread closes a batch when it holds
// max_batch requests or when its oldest request has waited window_us, takes
// a free slot of the device memory pool (the paper's per-query working blocks
// of §5, here one block per batch: query, per-query k / nprobe and results in
// HBM plus pinned host staging), and launches the search on the slot's stream
// without waiting. Up to `slots` batches are in flight at once, so requests
// that arrive while others run are admitted as soon as a slot (memory) frees
// up and their kernels overlap on the device. Completions are found by polling
// each slot's event; every request is stamped with its latency from submit to
// completion.
#include <string.h>

#include <chrono>
#include <deque>
#include <thread>
#include <vector>

#include "fa_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id;
    int32_t k, nprobe;
    Clock::time_point t0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    float *q = nullptr;        // device [max_batch][d]
    int32_t *kq = nullptr;     // device [max_batch]
    int32_t *npq = nullptr;    // device [max_batch]
    int64_t *ids = nullptr;    // device [max_batch][kmax]
    float *dist = nullptr;     // device [max_batch][kmax]
    float *h_q = nullptr;      // pinned staging
    int32_t *h_k = nullptr, *h_np = nullptr;
    int64_t *h_ids = nullptr;
    float *h_dist = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
    fa_status status = FA_OK;
    std::string error;
};

struct Done {
    int64_t id;
    int32_t k;
    double latency_us;
    fa_status status;
    std::vector<int64_t> ids;
    std::vector<float> dist;
};

}  // namespace

struct fa_server {
    fa_index *ix = nullptr;
    fa_server_params p{};
    fa_search_params sp{};
    int32_t d = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<std::vector<float>> pending_q;
    std::deque<Done> done;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 0;
    int64_t batches = 0, batched_requests = 0;
    int64_t device_bytes = 0;
};

namespace fa {

static void slot_free(Slot &s) {
    if (s.st) cudaStreamSynchronize(s.st);
    void *dp[] = {s.q, s.kq, s.npq, s.ids, s.dist};
    for (void *x : dp)
        if (x) cudaFree(x);
    void *hp[] = {s.h_q, s.h_k, s.h_np, s.h_ids, s.h_dist};
    for (void *x : hp)
        if (x) cudaFreeHost(x);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.st) cudaStreamDestroy(s.st);
    s = Slot{};
}

template <class T>
static void srv_dalloc(T *&p, size_t n, int64_t &bytes) {
    if (alloc_fault() || cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        throw Error{FA_ERR_OOM, "server slot allocation failed"};
    }
    bytes += (int64_t)(sizeof(T) * n);
}

template <class T>
static void srv_halloc(T *&p, size_t n) {
    FA_CHECK_CUDA(cudaHostAlloc((void **)&p, sizeof(T) * (n ? n : 1), cudaHostAllocDefault));
}

// Completed slots -> per-request results. Caller holds sv->mu.
static bool harvest(fa_server *sv) {
    bool any = false;
    for (Slot &s : sv->slots) {
        if (!s.busy) continue;
        const cudaError_t q = cudaEventQuery(s.ev);
        if (q == cudaErrorNotReady) continue;
        const auto now = Clock::now();
        if (q != cudaSuccess && s.status == FA_OK) {
            s.status = FA_ERR_CUDA;
            cudaGetLastError();
        }
        const int32_t kmax = sv->p.kmax;
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            const Request &r = s.reqs[i];
            Done dn;
            dn.id = r.id;
            dn.k = r.k;
            dn.status = s.status;
            dn.latency_us = std::chrono::duration<double, std::micro>(now - r.t0).count();
            dn.ids.assign(s.h_ids + i * kmax, s.h_ids + i * kmax + r.k);
            dn.dist.assign(s.h_dist + i * kmax, s.h_dist + i * kmax + r.k);
            sv->done.push_back(std::move(dn));
        }
        s.reqs.clear();
        s.busy = false;
        any = true;
    }
    if (any) sv->cv_done.notify_all();
    return any;
}

// Launches one batch on slot s (copies and search enqueued, no wait).
static void launch_batch(fa_server *sv, Slot &s) {
    const int64_t nb = (int64_t)s.reqs.size();
    const int32_t d = sv->d, kmax = sv->p.kmax, npmax = sv->p.nprobe_max;
    for (int64_t i = 0; i < nb; ++i) {
        s.h_k[i] = s.reqs[i].k;
        s.h_np[i] = s.reqs[i].nprobe;
    }
    s.status = FA_OK;
    FA_CHECK_CUDA(cudaMemcpyAsync(s.q, s.h_q, sizeof(float) * nb * d, cudaMemcpyHostToDevice, s.st));
    FA_CHECK_CUDA(cudaMemcpyAsync(s.kq, s.h_k, 4 * nb, cudaMemcpyHostToDevice, s.st));
    FA_CHECK_CUDA(cudaMemcpyAsync(s.npq, s.h_np, 4 * nb, cudaMemcpyHostToDevice, s.st));
    fa_search_params sp = sv->sp;
    // the tiled persistent scan: one query with a long probe set spreads over
    // many CTAs instead of holding its whole batch back
    sp.flags |= FA_QUERIES_ON_DEVICE | FA_OUTPUTS_ON_DEVICE | FA_NO_SYNC | FA_PERSISTENT;
    sp.k_per_query = s.kq;
    sp.nprobe_per_query = s.npq;
    sp.probes = nullptr;
    sp.stats = nullptr;
    sp.trace = nullptr;
    sp.stream = s.st;
    const fa_status st = fa_search_ex(sv->ix, s.q, nb, d, kmax, npmax, &sp, s.ids, s.dist);
    if (st != FA_OK) {
        s.status = st;
        s.error = fa_last_error();
    }
    FA_CHECK_CUDA(cudaMemcpyAsync(s.h_ids, s.ids, sizeof(int64_t) * nb * kmax, cudaMemcpyDeviceToHost, s.st));
    FA_CHECK_CUDA(cudaMemcpyAsync(s.h_dist, s.dist, sizeof(float) * nb * kmax, cudaMemcpyDeviceToHost, s.st));
    FA_CHECK_CUDA(cudaEventRecord(s.ev, s.st));
    s.busy = true;
}

static void worker_loop(fa_server *sv) {
    cudaSetDevice(sv->ix->device);
    const auto window = std::chrono::microseconds(sv->p.window_us);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        harvest(sv);
        if (sv->stop && sv->pending.empty()) {
            bool busy = false;
            for (Slot &s : sv->slots) busy |= s.busy;
            if (!busy) break;
        }
        if (sv->pending.empty()) {
            sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
            continue;
        }
        // continuous batching: close the batch when full or when its oldest
        // request has waited a window
        const bool full = (int64_t)sv->pending.size() >= sv->p.max_batch;
        const bool due = Clock::now() - sv->pending.front().t0 >= window;
        if (!full && !due && !sv->stop) {
            sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            continue;
        }
        // admission: a free slot (its block of device memory)
        Slot *free_slot = nullptr;
        for (Slot &s : sv->slots)
            if (!s.busy) {
                free_slot = &s;
                break;
            }
        if (!free_slot) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(10));
            lk.lock();
            continue;
        }
        const int64_t nb = std::min<int64_t>((int64_t)sv->pending.size(), sv->p.max_batch);
        Slot &s = *free_slot;
        s.reqs.clear();
        for (int64_t i = 0; i < nb; ++i) {
            s.reqs.push_back(sv->pending.front());
            memcpy(s.h_q + i * sv->d, sv->pending_q.front().data(), sizeof(float) * sv->d);
            sv->pending.pop_front();
            sv->pending_q.pop_front();
        }
        sv->batches += 1;
        sv->batched_requests += nb;
        try {
            launch_batch(sv, s);
        } catch (const Error &e) {
            s.status = e.st;
            s.error = e.msg;
            cudaEventRecord(s.ev, s.st);
            s.busy = true;
        }
    }
}

}  // namespace fa

using namespace fa;

extern "C" {

void fa_server_params_init(fa_server_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->max_batch = 1024;
    p->window_us = 200;
    p->slots = 4;
    p->kmax = 100;
    p->nprobe_max = 256;
    p->mem_budget_bytes = 0;
}

fa_status fa_server_create(fa_index *ix, const fa_server_params *p, const fa_search_params *sp,
                           fa_server **out) {
    if (!ix || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    *out = nullptr;
    fa_server *sv = new fa_server();
    try {
        if (p) sv->p = *p;
        else fa_server_params_init(&sv->p);
        if (sp) sv->sp = *sp;
        else fa_search_params_init(&sv->sp);
        FA_REQUIRE(sv->p.max_batch >= 1 && sv->p.slots >= 1 && sv->p.slots <= 64, FA_ERR_ARG,
                   "max_batch >= 1 and slots in 1..64");
        FA_REQUIRE(sv->p.kmax >= 1 && sv->p.kmax <= 256, FA_ERR_ARG, "kmax must be in 1..256");
        FA_REQUIRE(sv->p.nprobe_max >= 1 && sv->p.nprobe_max <= 512, FA_ERR_ARG,
                   "nprobe_max must be in 1..512");
        FA_REQUIRE(sv->sp.rerank_n == 0 || sv->p.kmax <= 128, FA_ERR_ARG, "re-rank supports k <= 128");
        sv->ix = ix;
        sv->d = ix->d;
        FA_CHECK_CUDA(cudaSetDevice(ix->device));
        // admission by memory: the slot count is cut to what the budget holds
        const int64_t per_req = (int64_t)sv->d * 4 + 8 + (int64_t)sv->p.kmax * 12 +
                                (int64_t)ix->dev.Mp * 256 * 4 + (int64_t)std::max(sv->p.kmax, sv->sp.rerank_n) * 8;
        int nslots = sv->p.slots;
        if (sv->p.mem_budget_bytes > 0) {
            const int64_t per_slot = per_req * sv->p.max_batch;
            nslots = (int)std::max<int64_t>(1, std::min<int64_t>(nslots, sv->p.mem_budget_bytes / per_slot));
        }
        sv->slots.resize(nslots);
        const int64_t B = sv->p.max_batch, K = sv->p.kmax;
        for (Slot &s : sv->slots) {
            FA_CHECK_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
            FA_CHECK_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
            srv_dalloc(s.q, B * sv->d, sv->device_bytes);
            srv_dalloc(s.kq, B, sv->device_bytes);
            srv_dalloc(s.npq, B, sv->device_bytes);
            srv_dalloc(s.ids, B * K, sv->device_bytes);
            srv_dalloc(s.dist, B * K, sv->device_bytes);
            srv_halloc(s.h_q, B * sv->d);
            srv_halloc(s.h_k, B);
            srv_halloc(s.h_np, B);
            srv_halloc(s.h_ids, B * K);
            srv_halloc(s.h_dist, B * K);
        }
        // enough search workspaces for every slot to run at once
        {
            std::lock_guard<std::mutex> lk(ix->mu);
            ix->max_ws = std::max(ix->max_ws, nslots + 2);
        }
        sv->worker = std::thread(worker_loop, sv);
    } catch (const Error &e) {
        set_error("%s", e.msg.c_str());
        for (Slot &s : sv->slots) slot_free(s);
        delete sv;
        return e.st;
    }
    *out = sv;
    return FA_OK;
}

fa_status fa_server_submit(fa_server *sv, const float *queries, int64_t n, const int32_t *k,
                           const int32_t *nprobe, int64_t *out_request_ids) {
    if (!sv || (n > 0 && (!queries || !k || !nprobe))) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            set_error("server is stopping");
            return FA_ERR_STATE;
        }
        for (int64_t i = 0; i < n; ++i) {
            if (k[i] < 1 || k[i] > sv->p.kmax || nprobe[i] < 1) {
                set_error("request %lld: k must be in 1..kmax and nprobe >= 1", (long long)i);
                return FA_ERR_ARG;
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            Request r;
            r.id = sv->next_id++;
            r.k = k[i];
            r.nprobe = std::min(nprobe[i], sv->p.nprobe_max);
            r.t0 = now;
            sv->pending.push_back(r);
            sv->pending_q.emplace_back(queries + i * sv->d, queries + (i + 1) * sv->d);
            if (out_request_ids) out_request_ids[i] = r.id;
        }
    }
    sv->cv_work.notify_one();
    return FA_OK;
}

int64_t fa_server_poll(fa_server *sv, int64_t max_results, int32_t timeout_us, int64_t *request_ids,
                       int64_t *ids, float *dist, int32_t kstride, double *latency_us,
                       int32_t *status) {
    if (!sv || max_results < 1) return 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && timeout_us > 0)
        sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us));
    int64_t n = 0;
    while (n < max_results && !sv->done.empty()) {
        Done &dn = sv->done.front();
        if (request_ids) request_ids[n] = dn.id;
        if (latency_us) latency_us[n] = dn.latency_us;
        if (status) status[n] = dn.status;
        for (int32_t j = 0; j < kstride; ++j) {
            if (ids) ids[n * kstride + j] = j < dn.k ? dn.ids[j] : -1;
            if (dist) dist[n * kstride + j] = j < dn.k ? dn.dist[j] : INFINITY;
        }
        sv->done.pop_front();
        ++n;
    }
    return n;
}

fa_status fa_server_stats(fa_server *sv, fa_server_stats_t *out) {
    if (!sv || !out) {
        set_error("null argument");
        return FA_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof *out);
    out->batches = sv->batches;
    out->requests = sv->batched_requests;
    out->pending = (int64_t)sv->pending.size();
    int inflight = 0;
    for (Slot &s : sv->slots) inflight += s.busy;
    out->inflight_batches = inflight;
    out->slots = (int32_t)sv->slots.size();
    out->device_bytes = sv->device_bytes;
    return FA_OK;
}

void fa_server_destroy(fa_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->ix->device);
    for (Slot &s : sv->slots) slot_free(s);
    delete sv;
}

}  // extern "C"
