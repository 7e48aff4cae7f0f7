// Continuous-batching server for actor queries (batched inference for the parallel
// environments of Alg. 1, "Sample a_t ~ pi(f(o~_t), s_t)").
//
// A host scheduler thread keeps up to `slots` inference batches in flight.  Each slot
// owns an activation arena, a high-priority stream and a pair of timing events.  Whenever
// a slot is free and requests are queued, it admits them in arrival order up to the
// slot's rows (the arenas are sized from the memory budget, checked against the device's
// free memory at start) and launches them as one ragged batch; it polls the in-flight
// batches' completion events and completes their requests.  Requests that arrive while
// batches run are admitted as soon as a slot frees, so their work overlaps the batches
// still on the GPU, and the serving streams run ahead of the update graph's stream.
// A request's latency is its queueing time on the host (submit to its batch's launch)
// plus its batch's device time (launch marker to completion event), so the scheduler's
// own polling delay is not part of it.
#include "sq_internal.h"

#include <algorithm>
#include <chrono>
#include <cstdlib>

namespace sq {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = 4;

struct ServeSlot {
    struct Item { uint64_t ticket; squint_act_request req; Clock::time_point t0; };
    ActArena arena;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    bool busy = false;
    std::vector<Item> batch;
    Clock::time_point t_launch;
    int64_t version = 0;
    int rows = 0;
};

struct ServeState {
    struct Done { int rc; double latency_us; int64_t version; double begin_us, end_us; int slot, rows; };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeSlot::Item> queue;
    std::unordered_map<uint64_t, Done> done;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    int slot_rows = 0;
    size_t row_bytes = 0;
    size_t max_queue = 1 << 16;
    int max_reqs = 0;
    int64_t arena_bytes = 0;
    std::vector<ServeSlot> slots;
    cudaEvent_t epoch = nullptr;     // device times are reported from this event
};

// Requests of one finished (or failed) slot: latency, device interval, completion.
static void complete_slot(ServeState* st, ServeSlot& sl, int si, int rc) {
    float b_ms = 0.f, e_ms = 0.f;
    if (rc == SQUINT_OK && (cudaEventElapsedTime(&b_ms, st->epoch, sl.ev_begin) != cudaSuccess ||
                            cudaEventElapsedTime(&e_ms, st->epoch, sl.ev_end) != cudaSuccess))
        rc = SQUINT_ECUDA;
    const double dev_us = 1000.0 * ((double)e_ms - (double)b_ms);
    {
        std::lock_guard<std::mutex> lk(st->mu);
        for (const auto& it : sl.batch) {
            const double queued = std::chrono::duration<double, std::micro>(sl.t_launch - it.t0).count();
            st->done[it.ticket] = ServeState::Done{rc, queued + dev_us, sl.version, 1000.0 * b_ms, 1000.0 * e_ms, si,
                                                   sl.rows};
        }
    }
    sl.batch.clear();
    sl.busy = false;
    st->cv_done.notify_all();
}

static void serve_loop(squint_handle* h, ServeState* st) {
    cudaSetDevice(h->device);
    std::vector<squint_act_request> reqs;
    for (;;) {
        // ---- complete the batches that finished
        int busy = 0;
        for (int si = 0; si < (int)st->slots.size(); ++si) {
            ServeSlot& sl = st->slots[si];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev_end);
            if (q == cudaSuccess) complete_slot(st, sl, si, SQUINT_OK);
            else if (q != cudaErrorNotReady) complete_slot(st, sl, si, SQUINT_ECUDA);
            else ++busy;
        }
        // ---- admit queued requests into every free slot
        for (int si = 0; si < (int)st->slots.size(); ++si) {
            ServeSlot& sl = st->slots[si];
            if (sl.busy) continue;
            {
                std::lock_guard<std::mutex> lk(st->mu);
                int rows = 0;
                while (!st->queue.empty()) {
                    const auto& p = st->queue.front();
                    if (rows + p.req.n > st->slot_rows || (int)sl.batch.size() >= st->max_reqs) break;
                    rows += p.req.n;
                    sl.batch.push_back(p);
                    st->queue.pop_front();
                }
                sl.rows = rows;
            }
            if (sl.batch.empty()) break;
            reqs.clear();
            for (const auto& p : sl.batch) reqs.push_back(p.req);
            sl.t_launch = Clock::now();
            int rc = cudaEventRecord(sl.ev_begin, sl.stream) == cudaSuccess ? SQUINT_OK : SQUINT_ECUDA;
            if (rc == SQUINT_OK) rc = h->act(sl.arena, reqs.data(), (int)reqs.size(), sl.stream, &sl.version);
            if (rc == SQUINT_OK && cudaEventRecord(sl.ev_end, sl.stream) != cudaSuccess) rc = SQUINT_ECUDA;
            sl.busy = true;
            if (rc != SQUINT_OK) complete_slot(st, sl, si, rc);
            else ++busy;
        }
        // ---- wait for work: a submit, or (with batches in flight) a short poll interval
        std::unique_lock<std::mutex> lk(st->mu);
        if (busy == 0) {
            if (st->queue.empty() && st->stop) return;
            st->cv_work.wait(lk, [&] { return st->stop || !st->queue.empty(); });
        } else if (st->queue.empty() || busy == (int)st->slots.size()) {
            st->cv_work.wait_for(lk, std::chrono::microseconds(10));
        }
    }
}

}  // namespace sq

using namespace sq;

namespace {

std::shared_ptr<ServeState> serve_of(squint_handle* h) {
    std::lock_guard<std::mutex> lk(h->serve_mu);
    return h->serve;
}

}  // namespace

extern "C" {

int squint_serve_start(squint_handle* h, int max_rows, size_t mem_budget_bytes) {
    if (!h || max_rows < 1) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    std::lock_guard<std::mutex> slk(h->serve_mu);
    if (h->serve) return SQUINT_ESTATE;
    const size_t rb = h->act_row_bytes();
    // admission by memory: the slots' arenas (allocated now) stay within the budget and
    // within the device memory that is free
    size_t free_b = 0, total_b = 0;
    SQ_CK(h, cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = std::min(mem_budget_bytes, free_b / 10 * 9);
    if (budget < rb) {
        g_last_error = "memory budget (or free device memory) below one row of activations";
        return SQUINT_ENOMEM;
    }
    int slots = 3;
    if (const char* e = std::getenv("SQUINT_SERVE_SLOTS")) slots = std::max(1, std::min(kMaxSlots, std::atoi(e)));
    // arena rows are rounded up to 256, so the budget is checked on the rounded size
    auto arena_rows = [](int r) { return std::max((r + 255) / 256 * 256, 256); };
    int rows = std::min(max_rows, (int)std::min<size_t>(budget / rb, (size_t)INT32_MAX));
    while (slots > 1 && (size_t)slots * arena_rows(rows) * rb > budget) --slots;
    while (rows > 1 && (size_t)slots * arena_rows(rows) * rb > budget) rows = std::max(1, rows / 2);
    auto st = std::make_shared<ServeState>();
    st->slot_rows = rows;
    st->row_bytes = rb;
    st->max_reqs = std::max(rows, 64);
    st->slots.resize(slots);
    int lo = 0, hi = 0;
    SQ_CK(h, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    int rc = SQUINT_OK;
    for (auto& sl : st->slots) {
        if (cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreate(&sl.ev_begin) != cudaSuccess || cudaEventCreate(&sl.ev_end) != cudaSuccess) {
            rc = SQUINT_ECUDA;
            break;
        }
        std::lock_guard<std::mutex> lk(h->act_mu);
        rc = h->alloc_arena(sl.arena, rows, st->max_reqs);
        if (rc != SQUINT_OK) break;
        st->arena_bytes += (int64_t)sl.arena.bytes;
        h->arenas.push_back(&sl.arena);
    }
    if (rc == SQUINT_OK && (cudaEventCreate(&st->epoch) != cudaSuccess ||
                            cudaEventRecord(st->epoch, st->slots[0].stream) != cudaSuccess ||
                            cudaEventSynchronize(st->epoch) != cudaSuccess))
        rc = SQUINT_ECUDA;
    if (rc != SQUINT_OK) {
        std::lock_guard<std::mutex> lk(h->act_mu);
        for (auto& sl : st->slots) {
            h->arenas.erase(std::remove(h->arenas.begin(), h->arenas.end(), &sl.arena), h->arenas.end());
            h->free_arena(sl.arena);
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.ev_begin) cudaEventDestroy(sl.ev_begin);
            if (sl.ev_end) cudaEventDestroy(sl.ev_end);
        }
        if (st->epoch) cudaEventDestroy(st->epoch);
        return rc;
    }
    h->serve = st;
    st->th = std::thread(serve_loop, h, st.get());
    return SQUINT_OK;
}

int squint_serve_submit(squint_handle* h, const squint_act_request* req, uint64_t* ticket) {
    if (!h || !req || !ticket) return SQUINT_EINVAL;
    std::shared_ptr<ServeState> st = serve_of(h);
    if (!st) return SQUINT_ESTATE;
    if (req->n < 1 || req->n > st->slot_rows) {
        g_last_error = "request larger than the admission limits";
        return SQUINT_EINVAL;
    }
    if ((!req->obs && !h->L.conv.empty()) || !req->proprio || !req->actions || (req->mode != 0 && req->mode != 1))
        return SQUINT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        if (st->stop) return SQUINT_ESTATE;
        if (st->queue.size() >= st->max_queue) return SQUINT_EAGAIN;
        *ticket = st->next_ticket++;
        st->queue.push_back(ServeSlot::Item{*ticket, *req, Clock::now()});
    }
    st->cv_work.notify_one();
    return SQUINT_OK;
}

int squint_serve_poll_ex(squint_handle* h, uint64_t ticket, int64_t timeout_us, squint_serve_result* out) {
    if (!h) return SQUINT_EINVAL;
    std::shared_ptr<ServeState> st = serve_of(h);
    if (!st) return SQUINT_ESTATE;
    std::unique_lock<std::mutex> lk(st->mu);
    auto ready = [&] { return st->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_us <= 0) return st->stop ? SQUINT_ESTATE : SQUINT_EAGAIN;
        // a stop wakes the waiters; a ticket the stopped server never completes is ESTATE
        st->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return ready() || st->stop; });
        if (!ready()) return st->stop ? SQUINT_ESTATE : SQUINT_EAGAIN;
    }
    const auto d = st->done[ticket];
    st->done.erase(ticket);
    if (d.rc != SQUINT_OK) return d.rc;
    if (out) {
        out->latency_us = d.latency_us;
        out->policy_version = d.version;
        out->device_begin_us = d.begin_us;
        out->device_end_us = d.end_us;
        out->slot = d.slot;
        out->batch_rows = d.rows;
    }
    return SQUINT_OK;
}

int squint_serve_poll(squint_handle* h, uint64_t ticket, int64_t timeout_us, double* latency_us,
                      int64_t* policy_version) {
    squint_serve_result r{};
    const int rc = squint_serve_poll_ex(h, ticket, timeout_us, &r);
    if (rc != SQUINT_OK) return rc;
    if (latency_us) *latency_us = r.latency_us;
    if (policy_version) *policy_version = r.policy_version;
    return SQUINT_OK;
}

int squint_serve_info(squint_handle* h, int* slots, int* slot_rows, int64_t* arena_bytes) {
    if (!h) return SQUINT_EINVAL;
    std::shared_ptr<ServeState> st = serve_of(h);
    if (!st) return SQUINT_ESTATE;
    if (slots) *slots = (int)st->slots.size();
    if (slot_rows) *slot_rows = st->slot_rows;
    if (arena_bytes) *arena_bytes = st->arena_bytes;
    return SQUINT_OK;
}

int squint_serve_stop(squint_handle* h) {
    if (!h) return SQUINT_OK;
    std::shared_ptr<ServeState> st;
    {
        std::lock_guard<std::mutex> lk(h->serve_mu);
        st = std::move(h->serve);
        h->serve.reset();
    }
    if (!st) return SQUINT_OK;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->stop = true;
    }
    st->cv_work.notify_all();
    if (st->th.joinable()) st->th.join();   // the queued and in-flight work completes first
    st->cv_done.notify_all();
    std::lock_guard<std::mutex> lk(h->act_mu);
    for (auto& sl : st->slots) {
        cudaStreamSynchronize(sl.stream);
        h->arenas.erase(std::remove(h->arenas.begin(), h->arenas.end(), &sl.arena), h->arenas.end());
        h->free_arena(sl.arena);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.ev_begin);
        cudaEventDestroy(sl.ev_end);
    }
    cudaEventDestroy(st->epoch);
    return SQUINT_OK;
}

}  // extern "C"
