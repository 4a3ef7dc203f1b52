// Continuous-batching server for SSQA anneals (ssqa_server_* / ssqa_submit /
// ssqa_poll).  The paper runs one anneal at a time; serving many GI / Ising
// solves of different sizes is this library's addition around the same
// per-request computation (Eq. 6).
//
// Requests queue on the host.  `max_slots` worker threads each own a CUDA
// stream.  A worker admits the oldest queued request whose device footprint
// fits in what is left of the HBM budget; a request may be passed over only a
// bounded number of times (2 x max_slots), after which nothing behind it is
// admitted until it fits, so that a large request cannot starve.  When the
// admitted request runs on the resident tensor-core kernel with a batched
// variant, the worker also takes the queued requests of the same variant and
// cycle count that fit (up to one wave of CTAs) and runs them all in one
// launch (ssqa_anneal_batch); other requests run alone (ssqa_anneal).  All
// state stays on the device for the whole anneal; requests admitted while
// others run overlap on the GPU.  Results are identical to a lone
// ssqa_anneal call: every random draw is keyed by the request's own seed and
// trial indices.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ssqa_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const ssqa_ising *ising = nullptr;
    ssqa_params params{};
    size_t bytes = 0;
    int key = -1;     // batched launch variant (-1: runs alone)
    int ctas = 0;     // column groups = CTAs on the resident kernel
    int bypass = 0;   // times a later request was admitted while this one was the oldest
    int state = 0;  // 0 queued, 1 running, 2 done
    int rc = SSQA_OK;
    std::string err;
    std::vector<int8_t> sigma, hist;
    std::vector<int32_t> is;
    std::vector<int64_t> e_final, e_best;
    std::vector<int32_t> best_cycle;
    Clock::time_point t_submit, t_done;
};

size_t footprint(const ssqa_ising *I, const ssqa_params &p) {
    const size_t N = size_t(I->N), cols = size_t(p.trials) * p.R, Np = (N + 15) / 16 * 16;
    const size_t state = cols * N * (1 + 4 + size_t(p.delay)) + cols * 24;
    // the larger of the CUDA-core scratch and the streamed path's operand slots
    const size_t scratch_cc = size_t(p.delay + 2) * cols * Np + cols * N * 8 + cols * 32;
    const size_t groups = (size_t(p.trials) + 128 / p.R - 1) / (128 / p.R);
    const size_t scratch_s = groups * size_t(p.delay + 2) * size_t(I->tc.KB) * 4096 + cols * Np + cols * 32 + 1024;
    const size_t scratch = scratch_cc > scratch_s ? scratch_cc : scratch_s;
    const size_t instance = N * N * 2 + N * 12 + I->tc.b.size() + I->tc.bs.size();
    return state + scratch + instance;
}

}  // namespace

struct ssqa_server {
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> workers;

    int nsm = 148;
    int max_bypass = 8;

    // Under mu: the requests to run next (oldest first, bounded bypass), or
    // none.  A batch shares one launch: same variant and cycle count, at most
    // one wave of CTAs, at most ssqa's batch size.
    std::vector<std::shared_ptr<Request>> admit() {
        std::vector<std::shared_ptr<Request>> out;
        if (queue.empty()) return out;
        size_t free = budget - used;
        int ctas = 0;
        const uint64_t head_ticket = queue.front()->ticket;
        for (auto it = queue.begin(); it != queue.end();) {
            Request &q = **it;
            const bool head = q.ticket == head_ticket;
            bool take = q.bytes <= free;
            if (take && !out.empty()) {
                const Request &first = *out.front();
                take = first.key >= 0 && q.key == first.key && q.params.cycles == first.params.cycles &&
                       ctas + q.ctas <= nsm && out.size() < 48;
            }
            if (take) {
                free -= q.bytes;
                ctas += q.ctas;
                out.push_back(*it);
                it = queue.erase(it);
                if (out.front()->key < 0) break;  // runs alone
                continue;
            }
            if (head && out.empty()) {
                // the oldest request does not fit: later ones may pass it a bounded number of times
                if (q.bypass >= max_bypass) break;
            }
            ++it;
        }
        if (!out.empty() && !queue.empty()) {
            // the oldest request left was passed over if anything newer was admitted
            uint64_t newest = 0;
            for (const auto &r : out) newest = r->ticket > newest ? r->ticket : newest;
            if (queue.front()->ticket < newest) ++queue.front()->bypass;
        }
        return out;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t st = nullptr;
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        for (;;) {
            std::vector<std::shared_ptr<Request>> rs;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    if (stop && queue.empty()) break;
                    rs = admit();
                    if (!rs.empty()) break;
                    cv_work.wait(lk);
                }
                if (rs.empty()) break;
                for (auto &r : rs) {
                    used += r->bytes;
                    r->state = 1;
                }
            }
            if (rs.size() == 1 && rs[0]->key < 0)
                run(rs[0].get(), st);
            else
                run_batch(rs, st);
            {
                std::lock_guard<std::mutex> lk(mu);
                const auto now = Clock::now();
                for (auto &r : rs) {
                    used -= r->bytes;
                    r->state = 2;
                    r->t_done = now;
                }
            }
            cv_done.notify_all();
            cv_work.notify_all();
        }
        if (st) cudaStreamDestroy(st);
    }

    static bool alloc_results(Request *r) {
        const ssqa_params &p = r->params;
        const size_t N = size_t(r->ising->N), cols = size_t(p.trials) * p.R;
        try {
            r->sigma.assign(cols * N, 0);
            r->is.assign(cols * N, 0);
            r->e_final.assign(cols, 0);
            if (p.delay) r->hist.assign(cols * N * size_t(p.delay), 0);
            if (p.flags & SSQA_FLAG_TRACK_BEST) {
                r->e_best.assign(cols, 0);
                r->best_cycle.assign(cols, 0);
            }
        } catch (...) {
            r->rc = SSQA_ERR_OOM;
            r->err = "server: out of host memory for results";
            return false;
        }
        return true;
    }

    static void run(Request *r, cudaStream_t st) {
        if (!alloc_results(r)) return;
        const ssqa_params &p = r->params;
        ssqa_result res{};
        res.sigma = r->sigma.data();
        res.is_state = r->is.data();
        res.e_final = r->e_final.data();
        res.sigma_hist = p.delay ? r->hist.data() : nullptr;
        if (p.flags & SSQA_FLAG_TRACK_BEST) {
            res.e_best = r->e_best.data();
            res.best_cycle = r->best_cycle.data();
        }
        r->rc = ssqa_anneal(r->ising, &p, &res, st);
        if (r->rc) r->err = ssqa_last_error();
    }

    // Several requests in one ssqa_anneal_batch call: device result buffers
    // per request, one launch, then the results back into each request.
    static void run_batch(const std::vector<std::shared_ptr<Request>> &rs, cudaStream_t st) {
        const size_t n = rs.size();
        std::vector<const ssqa_ising *> isings(n);
        std::vector<ssqa_params> ps(n);
        std::vector<ssqa_result> outs(n);
        std::vector<void *> bufs;
        auto fail_all = [&](int rc, const std::string &msg) {
            for (auto &r : rs) {
                r->rc = rc;
                r->err = msg;
            }
        };
        auto dalloc = [&](size_t bytes) -> void * {
            void *q = nullptr;
            if (ssqa::dev_alloc(&q, bytes ? bytes : 1, st) != cudaSuccess) return nullptr;
            bufs.push_back(q);
            return q;
        };
        bool ok = true;
        for (size_t k = 0; k < n && ok; ++k) {
            Request *r = rs[k].get();
            if (!alloc_results(r)) {
                fail_all(r->rc, r->err);
                ok = false;
                break;
            }
            const ssqa_params &p = r->params;
            const size_t N = size_t(r->ising->N), cols = size_t(p.trials) * p.R;
            isings[k] = r->ising;
            ps[k] = p;
            ps[k].flags |= SSQA_FLAG_DEVICE_PTRS;
            ssqa_result &o = outs[k];
            o = ssqa_result{};
            o.sigma = static_cast<int8_t *>(dalloc(cols * N));
            o.is_state = static_cast<int32_t *>(dalloc(cols * N * 4));
            o.e_final = static_cast<int64_t *>(dalloc(cols * 8));
            if (p.delay) o.sigma_hist = static_cast<int8_t *>(dalloc(cols * N * size_t(p.delay)));
            if (p.flags & SSQA_FLAG_TRACK_BEST) {
                o.e_best = static_cast<int64_t *>(dalloc(cols * 8));
                o.best_cycle = static_cast<int32_t *>(dalloc(cols * 4));
            }
            if (!o.sigma || !o.is_state || !o.e_final || (p.delay && !o.sigma_hist) ||
                ((p.flags & SSQA_FLAG_TRACK_BEST) && (!o.e_best || !o.best_cycle))) {
                cudaGetLastError();
                fail_all(SSQA_ERR_OOM, "server: device memory for results");
                ok = false;
            }
        }
        if (ok) {
            const int rc = ssqa_anneal_batch(int32_t(n), isings.data(), ps.data(), outs.data(), nullptr, st);
            if (rc) {
                fail_all(rc, ssqa_last_error());
                ok = false;
            }
        }
        if (ok) {
            cudaError_t e = cudaSuccess;
            for (size_t k = 0; k < n && !e; ++k) {
                Request *r = rs[k].get();
                const ssqa_result &o = outs[k];
                if (!e) e = cudaMemcpyAsync(r->sigma.data(), o.sigma, r->sigma.size(), cudaMemcpyDeviceToHost, st);
                if (!e) e = cudaMemcpyAsync(r->is.data(), o.is_state, r->is.size() * 4, cudaMemcpyDeviceToHost, st);
                if (!e) e = cudaMemcpyAsync(r->e_final.data(), o.e_final, r->e_final.size() * 8, cudaMemcpyDeviceToHost, st);
                if (!e && o.sigma_hist)
                    e = cudaMemcpyAsync(r->hist.data(), o.sigma_hist, r->hist.size(), cudaMemcpyDeviceToHost, st);
                if (!e && o.e_best) {
                    e = cudaMemcpyAsync(r->e_best.data(), o.e_best, r->e_best.size() * 8, cudaMemcpyDeviceToHost, st);
                    if (!e)
                        e = cudaMemcpyAsync(r->best_cycle.data(), o.best_cycle, r->best_cycle.size() * 4,
                                            cudaMemcpyDeviceToHost, st);
                }
            }
            if (!e) e = cudaStreamSynchronize(st);
            if (e) {
                cudaGetLastError();
                fail_all(SSQA_ERR_DEVICE, std::string("server: result download: ") + cudaGetErrorString(e));
            }
        }
        for (void *q : bufs) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
    }
};

extern "C" {

int ssqa_server_create(size_t hbm_budget, int32_t max_slots, int32_t device, ssqa_server **out) {
    if (!out) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_server_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64 || hbm_budget == 0)
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_server_create: max_slots in 1..64 and a nonzero budget");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ssqa::fail(SSQA_ERR_DEVICE, "ssqa_server_create: no such CUDA device");
    }
    ssqa_server *s = new (std::nothrow) ssqa_server();
    if (!s) return ssqa::fail(SSQA_ERR_OOM, "ssqa_server_create: out of host memory");
    s->device = device;
    s->budget = hbm_budget;
    s->max_bypass = 2 * max_slots;
    if (cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        s->nsm = 148;
    }
    try {
        for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s] { s->worker(); });
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->workers) t.join();
        delete s;
        return ssqa::fail(SSQA_ERR_OOM, "ssqa_server_create: cannot start worker threads");
    }
    *out = s;
    return SSQA_OK;
}

void ssqa_server_destroy(ssqa_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    delete s;
}

int ssqa_submit(ssqa_server *s, const ssqa_ising *ising, const ssqa_params *params, uint64_t *ticket) {
    if (!s || !ising || !params || !ticket) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_submit: NULL argument");
    if (params->flags & SSQA_FLAG_DEVICE_PTRS)
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_submit: results are returned in host memory");
    if (params->init_mode == SSQA_INIT_FROM_STATE)
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_submit: resuming from a state is not served");
    if (params->R < 1 || params->R > 128 || params->trials < 1 || params->cycles < 0 || params->delay < 0 ||
        params->delay > 3)
        return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_submit: bad R, trials, cycles or delay");
    auto r = std::make_shared<Request>();
    r->ising = ising;
    r->params = *params;
    r->bytes = footprint(ising, *params);
    r->key = ssqa::batch_key(ising, params);
    r->ctas = int((int64_t(params->trials) + 128 / params->R - 1) / (128 / params->R));
    if (r->bytes > s->budget)
        return ssqa::fail(SSQA_ERR_BUDGET, "ssqa_submit: request needs more device memory than the whole budget");
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_submit: server is shutting down");
        r->ticket = s->next_ticket++;
        s->queue.push_back(r);
        s->all.emplace(r->ticket, r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return SSQA_OK;
}

int ssqa_poll(ssqa_server *s, uint64_t ticket, ssqa_result *out, int32_t timeout_ms, double *latency_us) {
    if (!s) return ssqa::fail(SSQA_ERR_INVALID_ARG, "ssqa_poll: NULL server");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return ssqa::fail(SSQA_ERR_NOT_FOUND, "ssqa_poll: unknown ticket");
        r = it->second;
        auto done = [&] { return r->state == 2; };
        if (timeout_ms < 0)
            s->cv_done.wait(lk, done);
        else if (!done())
            s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
        if (r->state != 2) return SSQA_PENDING;
        s->all.erase(ticket);
    }
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    if (r->rc) return ssqa::fail(r->rc, r->err);
    if (out) {
        const ssqa_params &p = r->params;
        if (out->sigma) std::memcpy(out->sigma, r->sigma.data(), r->sigma.size());
        if (out->is_state) std::memcpy(out->is_state, r->is.data(), r->is.size() * 4);
        if (out->e_final) std::memcpy(out->e_final, r->e_final.data(), r->e_final.size() * 8);
        if (out->sigma_hist && p.delay) std::memcpy(out->sigma_hist, r->hist.data(), r->hist.size());
        if ((p.flags & SSQA_FLAG_TRACK_BEST) && out->e_best && out->best_cycle) {
            std::memcpy(out->e_best, r->e_best.data(), r->e_best.size() * 8);
            std::memcpy(out->best_cycle, r->best_cycle.data(), r->best_cycle.size() * 4);
        }
    }
    return SSQA_OK;
}

}  // extern "C"
