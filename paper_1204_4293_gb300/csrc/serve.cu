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
//
// Heavy requests (at least 2^32 pixel-scales of work: large noise maps) run
// at most FM_TUNE_SERVE_HEAVY at a time (default one): several of them side
// by side stretch one another for no gain in throughput (the serving trace's
// heaviest request, 4096^2 with R = 1000, takes ~1 s alone and ~3 s beside
// others), while the light requests queued behind a waiting heavy one are
// admitted past it.
//
// Continuous batching: when the request at the head of the queue asks for the
// pyramid only (R = 0) of a map of at most 1024^2, the queued requests of the
// same (n, J, precision) join it, up to FM_TUNE_SERVE_MERGE maps and within
// the budget, and the group runs as one batched KS + starlet call on one
// slot: each input is copied into a gathered batch (one device-to-device
// copy per request), the batch runs through the chunked pipeline, and each
// pyramid is copied out.  Every map's arithmetic is the same as alone, so
// the results are bit for bit those of single runs.
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
    std::vector<uint64_t> members;  // a merged group's other requests (held by its first)
    bool heavy = false;             // counted in Server::heavy_running while it runs
};

// pyramid-only requests of maps up to 1024^2 may run merged
bool mergeable(const fm_request &r) { return r.R == 0 && r.n <= 1024; }
// heavy: at least 2^32 pixel-scales of work (n^2 J (1 + R)), e.g. noise maps
// of 4096^2 with R = 100 or 1024^2 with R = 1000
bool heavy(const fm_request &r) { return (double)r.n * r.n * r.J * (1.0 + (r.R >= 2 ? r.R : 0)) >= 4294967296.0; }
bool same_shape(const fm_request &a, const fm_request &b)
{
    return a.n == b.n && a.J == b.J && a.precision == b.precision;
}
// device bytes of a merged run of `count` maps: gathered inputs and pyramids
// plus the batched pipeline's scratch
size_t group_bytes(const fm_request &r, int count)
{
    fm_config cfg{};
    cfg.precision = r.precision;
    const size_t es = r.precision == FM_F64 ? 8 : 4, nn = (size_t)r.n * r.n;
    return (size_t)count * (2 + r.J) * nn * es + map_starlet_scratch_bytes(r.n, r.J, count, cfg) + 512;
}

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
    int heavy_running = 0;
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
            if (q.heavy) --heavy_running;
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
            // heavy requests run few at a time: their chunks take the internal streams
            st = map_noise_run(r.g1, r.g2, r.out_var, nullptr, r.n, r.J, r.R, r.seed, cfg, s, false, heavy(r));
        return st;
    }

    // one batched call over a group of same-shape pyramid-only requests
    static int run_group(const std::vector<fm_request> &rs, cudaStream_t s)
    {
        const fm_request &r0 = rs[0];
        fm_config cfg{};
        cfg.precision = r0.precision;
        const size_t es = r0.precision == FM_F64 ? 8 : 4, map_b = (size_t)r0.n * r0.n * es;
        const size_t B = rs.size();
        Scratch sc;  // freed on s after the copies out
        int st = scratch_alloc(sc, B * (2 + r0.J) * map_b, s);
        if (st) return st;
        char *g1b = static_cast<char *>(sc.p), *g2b = g1b + B * map_b, *pyb = g2b + B * map_b;
        for (size_t i = 0; i < B; ++i) {
            FM_CUDA_TRY(cudaMemcpyAsync(g1b + i * map_b, rs[i].g1, map_b, cudaMemcpyDeviceToDevice, s));
            FM_CUDA_TRY(cudaMemcpyAsync(g2b + i * map_b, rs[i].g2, map_b, cudaMemcpyDeviceToDevice, s));
        }
        if ((st = map_starlet_run(g1b, g2b, pyb, r0.n, r0.J, (int)B, cfg, s, false))) return st;
        for (size_t i = 0; i < B; ++i)
            FM_CUDA_TRY(cudaMemcpyAsync(rs[i].out_pyramid, pyb + i * r0.J * map_b, r0.J * map_b,
                                        cudaMemcpyDeviceToDevice, s));
        return FM_OK;
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
                for (uint64_t m : q.members) finish(reqs[m], e == cudaSuccess ? FM_OK : FM_ECUDA);
                q.members.clear();
                finish(q, e == cudaSuccess ? FM_OK : FM_ECUDA);
                running[i] = running.back();
                running.pop_back();
                progress = true;
            }
            if (stop && running.empty()) break;
            // admissions, in arrival order; a heavy request waits while
            // FM_TUNE_SERVE_HEAVY others run, and the light ones queued
            // behind it may go first
            for (auto it = queue.begin(); !stop && it != queue.end();) {
                const uint64_t t = *it;
                Req &q = reqs[t];
                if (q.bytes > budget) {
                    it = queue.erase(it);
                    finish(q, FM_EBUDGET);
                    progress = true;
                    continue;
                }
                const int heavy_max = g_serve_heavy.load();
                if (heavy(q.r) && heavy_max > 0 && heavy_running >= heavy_max) {
                    ++it;
                    continue;
                }
                int slot = -1;
                for (int k = 0; k < max_slots; ++k)
                    if (!slot_busy[k]) {
                        slot = k;
                        break;
                    }
                if (slot < 0 || in_use + q.bytes > budget) break;
                it = queue.erase(it);
                // later queued requests of the same shape join a mergeable one
                std::vector<uint64_t> group;
                const int merge_max = g_serve_merge.load();
                if (merge_max > 1 && mergeable(q.r)) {
                    for (auto jt = it; jt != queue.end() && (int)group.size() + 1 < merge_max;) {
                        const Req &o = reqs[*jt];
                        if (mergeable(o.r) && same_shape(o.r, q.r) &&
                            in_use + group_bytes(q.r, (int)group.size() + 2) <= budget) {
                            group.push_back(*jt);
                            jt = queue.erase(jt);
                        } else {
                            ++jt;
                        }
                    }
                }
                const size_t bytes = group.empty() ? q.bytes : group_bytes(q.r, (int)group.size() + 1);
                slot_busy[slot] = 1;
                q.slot = slot;
                q.bytes = bytes;
                in_use += bytes;
                q.heavy = heavy(q.r);
                if (q.heavy) ++heavy_running;
                q.t_admit = now_ns();
                std::vector<fm_request> rs{q.r};
                for (uint64_t m : group) {
                    reqs[m].t_admit = q.t_admit;
                    rs.push_back(reqs[m].r);
                }
                q.members = group;
                const fm_request r = q.r;
                cudaStream_t s = streams[slot];
                lk.unlock();
                int st = group.empty() ? run(r, s) : run_group(rs, s);
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
                    for (uint64_t m : q2.members) finish(reqs[m], st);
                    q2.members.clear();
                    finish(q2, st);
                } else {
                    q2.ev = ev;
                    running.push_back(t);
                }
                progress = true;
                it = queue.begin();  // submissions may have changed the queue meanwhile
            }
            if (stop && queue.empty() && running.empty()) break;
            if (!progress) cv.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 50));
        }
    }
};

}  // namespace
}  // namespace fm

namespace fm {
std::atomic<int> g_serve_merge{16};
std::atomic<int> g_serve_heavy{1};
}

using namespace fm;

extern "C" {

size_t fm_request_scratch_bytes(const fm_request *req)
{
    if (!req) return 0;
    fm_config cfg{};
    cfg.precision = req->precision;
    size_t a = map_starlet_scratch_bytes(req->n, req->J, 1, cfg);
    size_t b = (req->R >= 2 && req->out_var) ? noise_scratch_bytes(req->n, req->J, req->R, cfg, false, heavy(*req)) : 0;
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
