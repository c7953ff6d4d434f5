// serve.cu -- continuous batching of aperture-mass requests on one GPU.
//
// A server owns one host thread and `max_slots` CUDA streams.  Requests are
// queued by fm_serve_submit; the thread admits them in arrival order as soon
// as a stream slot is free and their scratch fits in the memory budget minus
// the scratch of the requests still running.  Each admitted request runs its
// whole pipeline (KS + starlet, then the noise maps when R >= 2) on its own
// stream, so requests that arrive while others run overlap on the device.
// Completion is seen through one CUDA event per request; the thread then
// frees the slot and the budget and stamps the finish time.  Results are
// read (once) with fm_serve_poll / fm_serve_wait.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fm {

static int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

namespace {

struct Req {
    fm_request r{};
    int status = FM_PENDING;
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    int slot = -1;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
};

struct Server {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<char> slot_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    std::vector<uint64_t> running;
    size_t in_use = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    static constexpr size_t kMaxQueue = 1u << 20;

    void finish(Req &q, int status)
    {
        q.status = status;
        q.t_done = now_ns();
        if (q.slot >= 0) {
            slot_busy[q.slot] = 0;
            q.slot = -1;
            in_use -= q.bytes;
        }
        if (q.ev) {
            cudaEventDestroy(q.ev);
            q.ev = nullptr;
        }
    }

    static int run(const fm_request &r, cudaStream_t s)
    {
        fm_config cfg{};
        cfg.precision = r.precision;
        int st = map_starlet_run(r.g1, r.g2, r.out_pyramid, r.n, r.J, 1, cfg, s);
        if (st == FM_OK && r.R >= 2 && r.out_var)
            st = map_noise_run(r.g1, r.g2, r.out_var, nullptr, r.n, r.J, r.R, r.seed, cfg, s, false);
        return st;
    }

    void loop()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            bool progress = false;
            // completions
            for (size_t i = 0; i < running.size();) {
                Req &q = reqs[running[i]];
                const cudaError_t e = cudaEventQuery(q.ev);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                if (e != cudaSuccess) set_error(std::string("request failed: ") + cudaGetErrorString(e));
                finish(q, e == cudaSuccess ? FM_OK : FM_ECUDA);
                running[i] = running.back();
                running.pop_back();
                progress = true;
            }
            if (stop && running.empty()) break;
            // admissions, in arrival order
            while (!stop && !queue.empty()) {
                const uint64_t t = queue.front();
                Req &q = reqs[t];
                if (q.bytes > budget) {
                    queue.pop_front();
                    finish(q, FM_EBUDGET);
                    progress = true;
                    continue;
                }
                int slot = -1;
                for (int k = 0; k < max_slots; ++k)
                    if (!slot_busy[k]) {
                        slot = k;
                        break;
                    }
                if (slot < 0 || in_use + q.bytes > budget) break;
                queue.pop_front();
                slot_busy[slot] = 1;
                q.slot = slot;
                in_use += q.bytes;
                q.t_admit = now_ns();
                const fm_request r = q.r;
                cudaStream_t s = streams[slot];
                lk.unlock();
                int st = run(r, s);
                cudaEvent_t ev = nullptr;
                if (st == FM_OK) {
                    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                    if (e == cudaSuccess) e = cudaEventRecord(ev, s);
                    if (e != cudaSuccess) st = cuda_fail(e, "request completion event");
                }
                lk.lock();
                Req &q2 = reqs[t];
                if (st != FM_OK) {
                    if (ev) cudaEventDestroy(ev);
                    // the stream may still hold part of the request's work
                    lk.unlock();
                    cudaStreamSynchronize(s);
                    lk.lock();
                    finish(q2, st);
                } else {
                    q2.ev = ev;
                    running.push_back(t);
                }
                progress = true;
            }
            if (stop && queue.empty() && running.empty()) break;
            if (!progress) cv.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 50));
        }
    }
};

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" {

size_t fm_request_scratch_bytes(const fm_request *req)
{
    if (!req) return 0;
    fm_config cfg{};
    cfg.precision = req->precision;
    size_t a = map_starlet_scratch_bytes(req->n, req->J, 1, cfg);
    size_t b = (req->R >= 2 && req->out_var) ? noise_scratch_bytes(req->n, req->J, req->R, cfg, false) : 0;
    return a > b ? a : b;  // stream-ordered frees let the noise pass reuse the first pass's scratch
}

int fm_serve_create(size_t mem_budget_bytes, int max_slots, void **server)
{
    if (!server || max_slots < 1 || max_slots > 64 || mem_budget_bytes == 0) {
        set_error("fm_serve_create: need server != NULL, 1 <= max_slots <= 64, budget > 0");
        return FM_EINVAL;
    }
    Server *sv = new Server();
    sv->budget = mem_budget_bytes;
    sv->max_slots = max_slots;
    cudaError_t e = cudaGetDevice(&sv->device);
    for (int k = 0; e == cudaSuccess && k < max_slots; ++k) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) sv->streams.push_back(s);
    }
    if (e != cudaSuccess) {
        for (auto s : sv->streams) cudaStreamDestroy(s);
        delete sv;
        return cuda_fail(e, "fm_serve_create");
    }
    sv->slot_busy.assign(max_slots, 0);
    sv->th = std::thread([sv] { sv->loop(); });
    *server = sv;
    return FM_OK;
}

int fm_serve_submit(void *server, const fm_request *req, uint64_t *ticket)
{
    Server *sv = static_cast<Server *>(server);
    if (!sv || !req || !ticket) {
        set_error("fm_serve_submit: null argument");
        return FM_EINVAL;
    }
    const fm_request &r = *req;
    if (r.n < 4 || r.n > 8192 || !is_pow2(r.n) || r.J < 2 || (long)r.n < (1L << r.J) ||
        (r.precision != FM_F32 && r.precision != FM_F64) || !r.g1 || !r.g2 || !r.out_pyramid || r.R < 0 ||
        r.R == 1 || (r.R >= 2 && !r.out_var)) {
        set_error("fm_serve_submit: invalid request");
        return FM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->queue.size() >= Server::kMaxQueue) {
        set_error("fm_serve_submit: queue full");
        return FM_EBUSY;
    }
    const uint64_t t = sv->next_ticket++;
    Req q;
    q.r = r;
    q.bytes = fm_request_scratch_bytes(&r);
    q.t_submit = now_ns();
    sv->reqs.emplace(t, q);
    sv->queue.push_back(t);
    *ticket = t;
    sv->cv.notify_one();
    return FM_OK;
}

int fm_serve_poll(void *server, uint64_t ticket, fm_result *result)
{
    Server *sv = static_cast<Server *>(server);
    if (!sv || !result) {
        set_error("fm_serve_poll: null argument");
        return FM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("fm_serve_poll: unknown ticket");
        return FM_ENOTFOUND;
    }
    const Req &q = it->second;
    result->status = q.status;
    result->t_submit_ns = q.t_submit;
    result->t_admit_ns = q.t_admit;
    result->t_done_ns = q.t_done;
    if (q.status != FM_PENDING) {
        sv->reqs.erase(it);  // a finished result is handed out once
        return FM_OK;
    }
    return FM_PENDING;
}

int fm_serve_wait(void *server, uint64_t ticket, fm_result *result, double timeout_s)
{
    const int64_t deadline = now_ns() + (int64_t)(timeout_s * 1e9);
    for (;;) {
        int st = fm_serve_poll(server, ticket, result);
        if (st != FM_PENDING) return st;
        if (now_ns() > deadline) {
            set_error("fm_serve_wait: timed out");
            return FM_ETIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int fm_serve_destroy(void *server)
{
    Server *sv = static_cast<Server *>(server);
    if (!sv) return FM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // queued requests never start
        for (uint64_t t : sv->queue) sv->reqs[t].status = FM_EINVAL;
        sv->queue.clear();
        sv->cv.notify_one();
    }
    if (sv->th.joinable()) sv->th.join();
    for (auto s : sv->streams) cudaStreamDestroy(s);
    delete sv;
    return FM_OK;
}

}  // extern "C"
