// Continuous-batching server for actor queries (batched inference for the
// parallel environments of Alg. 1, "Sample a_t ~ pi(f(o~_t), s_t)").
//
// A host scheduler thread owns one act stream.  Requests queue on submit; each
// scheduling round admits queued requests in arrival order while the rows of the
// batch stay within max_rows and their activation memory within the budget,
// launches them as one ragged batch, and completes them when the batch's event
// fires.  Requests that arrive while a batch is on the GPU wait for the next
// round, so the GPU always works on everything that has arrived and fits.
#include "sq_internal.h"

#include <chrono>

namespace sq {

using Clock = std::chrono::steady_clock;

struct ServeState {
    struct Pending { uint64_t ticket; squint_act_request req; Clock::time_point t0; };
    struct Done { double latency_us; int64_t version; };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Done> done;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    int max_rows = 0;
    size_t budget = 0;
    size_t row_bytes = 0;
    size_t max_queue = 1 << 16;
    int max_reqs = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int error = SQUINT_OK;
};

static void serve_loop(squint_handle* h, ServeState* st) {
    cudaSetDevice(h->device);
    std::vector<ServeState::Pending> batch;
    std::vector<squint_act_request> reqs;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(st->mu);
            st->cv_work.wait(lk, [&] { return st->stop || !st->queue.empty(); });
            if (st->queue.empty() && st->stop) return;
            batch.clear();
            int rows = 0;
            while (!st->queue.empty()) {
                const auto& p = st->queue.front();
                const int nr = rows + p.req.n;
                if (nr > st->max_rows || (size_t)nr * st->row_bytes > st->budget ||
                    (int)batch.size() >= st->max_reqs)
                    break;
                rows = nr;
                batch.push_back(p);
                st->queue.pop_front();
            }
        }
        reqs.clear();
        for (const auto& p : batch) reqs.push_back(p.req);
        int64_t version = 0;
        int rc = h->act(reqs.data(), (int)reqs.size(), st->stream, &version);
        if (rc == SQUINT_OK && cudaEventRecord(st->ev, st->stream) != cudaSuccess) rc = SQUINT_ECUDA;
        if (rc == SQUINT_OK && cudaEventSynchronize(st->ev) != cudaSuccess) rc = SQUINT_ECUDA;
        const auto t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lk(st->mu);
            if (rc != SQUINT_OK) st->error = rc;
            for (const auto& p : batch) {
                const double us = std::chrono::duration<double, std::micro>(t1 - p.t0).count();
                st->done[p.ticket] = ServeState::Done{rc == SQUINT_OK ? us : -1.0, version};
            }
        }
        st->cv_done.notify_all();
    }
}

}  // namespace sq

using namespace sq;

extern "C" {

int squint_serve_start(squint_handle* h, int max_rows, size_t mem_budget_bytes) {
    if (!h || max_rows < 1) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (h->serve) return SQUINT_ESTATE;
    const size_t rb = h->act_row_bytes();
    if (mem_budget_bytes < rb) {
        g_last_error = "memory budget below one row of activations";
        return SQUINT_ENOMEM;
    }
    const int rows = (int)std::min<size_t>((size_t)max_rows, mem_budget_bytes / rb);
    const int max_reqs = std::max(rows, 64);
    {
        std::lock_guard<std::mutex> lk(h->act_mu);
        int rc = h->ensure_act_capacity(rows, max_reqs);
        if (rc != SQUINT_OK) return rc;
    }
    auto* st = new ServeState();
    st->max_rows = rows;
    st->budget = mem_budget_bytes;
    st->row_bytes = rb;
    st->max_reqs = max_reqs;
    if (cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&st->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete st;
        return SQUINT_ECUDA;
    }
    h->serve = st;
    st->th = std::thread(serve_loop, h, st);
    return SQUINT_OK;
}

int squint_serve_submit(squint_handle* h, const squint_act_request* req, uint64_t* ticket) {
    if (!h || !req || !ticket) return SQUINT_EINVAL;
    ServeState* st = h->serve;
    if (!st) return SQUINT_ESTATE;
    if (req->n < 1 || req->n > st->max_rows || (size_t)req->n * st->row_bytes > st->budget) {
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
        st->queue.push_back(ServeState::Pending{*ticket, *req, Clock::now()});
    }
    st->cv_work.notify_one();
    return SQUINT_OK;
}

int squint_serve_poll(squint_handle* h, uint64_t ticket, int64_t timeout_us, double* latency_us,
                      int64_t* policy_version) {
    if (!h) return SQUINT_EINVAL;
    ServeState* st = h->serve;
    if (!st) return SQUINT_ESTATE;
    std::unique_lock<std::mutex> lk(st->mu);
    auto ready = [&] { return st->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_us <= 0) return SQUINT_EAGAIN;
        if (!st->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return SQUINT_EAGAIN;
    }
    const auto d = st->done[ticket];
    st->done.erase(ticket);
    if (d.latency_us < 0) return st->error ? st->error : SQUINT_ECUDA;
    if (latency_us) *latency_us = d.latency_us;
    if (policy_version) *policy_version = d.version;
    return SQUINT_OK;
}

int squint_serve_stop(squint_handle* h) {
    if (!h || !h->serve) return SQUINT_OK;
    ServeState* st = h->serve;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->stop = true;
    }
    st->cv_work.notify_all();
    if (st->th.joinable()) st->th.join();
    cudaStreamSynchronize(st->stream);
    cudaStreamDestroy(st->stream);
    cudaEventDestroy(st->ev);
    delete st;
    h->serve = nullptr;
    return SQUINT_OK;
}

}  // extern "C"
