// Continuous-batching solve server: a request loop on one GPU that admits solves of
// different grids and wavenumbers as worker slots and device memory free up, runs the
// admitted ones concurrently on their own CUDA streams (their kernels overlap on the
// device), and keeps each solve's hierarchy and Krylov basis on the device for its whole
// life.  Built only on the public C ABI of hh.h.
//
// Admission: a request is taken from the queue in arrival order by the first free worker.
// It runs on an idle pooled problem of the same shape (grid, boundary tags), retargeted
// to its k, delta, delta_hat, or on a new problem if the device budget has room for its
// footprint; otherwise idle problems of other shapes are destroyed, least recently used
// first, until it fits, and if nothing can be freed the worker waits for a running solve
// to return its problem.  Problem creation, destruction and preconditioner-graph capture
// are serialised by one lock, so that no allocation or free runs while a graph is being
// captured; solves run without it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hh.h"
#include "internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
    long long id = 0;
    hh_request r{};
    const void* rhs = nullptr;
    void* u = nullptr;
    hh_status st = HH_OK;
    hh_info info{};
    clk::time_point t_submit, t_start, t_end;
    bool done = false;
    std::string err;
};

struct Slot {
    hh_problem* p = nullptr;
    cudaStream_t stream = nullptr;  // the problem's caller stream, used by nobody else
    hh_grid grid{};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    size_t bytes = 0;
    bool busy = false;
    long long last_use = 0;
};

bool same_shape(const Slot& s, const hh_request& r) {
    if (s.grid.dim != r.grid.dim || s.grid.n != r.grid.n) return false;
    for (int i = 0; i < 2 * r.grid.dim; ++i)
        if (s.bc[i] != r.bc[i]) return false;
    return true;
}

double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

}  // namespace

struct hh_server {
    int device = 0;
    int slots = 1;
    size_t budget = 0;
    hh_options opts{};
    std::mutex mu;                   // queue, pool, accounting
    std::condition_variable cv;      // work queued, problem returned, request done
    std::mutex dev_mu;               // create / destroy / graph capture
    std::deque<Req*> queue;
    std::map<long long, std::unique_ptr<Req>> reqs;
    std::vector<std::unique_ptr<Slot>> pool;
    std::vector<std::thread> workers;
    size_t held = 0;                 // device bytes of pooled problems (busy or idle)
    size_t reserved = 0;             // bytes promised to problems being created
    hh_server_stats st{};
    long long next_id = 1, tick = 0;
    int running = 0;
    bool stop = false;
};

namespace {

void drop_problem(hh_server* S, hh_problem* p, cudaStream_t stream) {
    std::lock_guard<std::mutex> g(S->dev_mu);
    if (p) hh_destroy(p);
    if (stream) cudaStreamDestroy(stream);
}

// Take a problem for request q (lock held on entry and exit; may release it while waiting).
// Returns the slot, or nullptr with *create_bytes set when a new problem must be created
// (its bytes already reserved).
Slot* acquire(hh_server* S, std::unique_lock<std::mutex>& lk, const Req* q, size_t need, size_t* create_bytes) {
    *create_bytes = 0;
    for (;;) {
        for (auto& s : S->pool)
            if (!s->busy && s->p && same_shape(*s, q->r)) {
                s->busy = true;
                ++S->st.problems_reused;
                return s.get();
            }
        if (S->held + S->reserved + need <= S->budget) {
            S->reserved += need;
            *create_bytes = need;
            return nullptr;
        }
        // evict the least recently used idle problem of another shape
        Slot* victim = nullptr;
        for (auto& s : S->pool)
            if (!s->busy && s->p && (!victim || s->last_use < victim->last_use)) victim = s.get();
        if (victim) {
            hh_problem* p = victim->p;
            cudaStream_t sv = victim->stream;
            const size_t b = victim->bytes;
            victim->p = nullptr;
            victim->stream = nullptr;
            victim->busy = true;  // being destroyed
            lk.unlock();
            drop_problem(S, p, sv);
            lk.lock();
            S->held -= b;
            ++S->st.problems_evicted;
            S->pool.erase(std::remove_if(S->pool.begin(), S->pool.end(),
                                         [&](const std::unique_ptr<Slot>& s) { return s.get() == victim; }),
                          S->pool.end());
            continue;
        }
        S->cv.wait(lk);  // a running solve returns its problem
    }
}

void worker(hh_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
        if (S->queue.empty()) return;  // stopping and drained
        Req* q = S->queue.front();
        S->queue.pop_front();
        const size_t need = hh_footprint_bytes(&q->r.grid, &S->opts);
        size_t create = 0;
        Slot* slot = acquire(S, lk, q, need, &create);
        q->t_start = clk::now();
        ++S->running;
        S->st.max_concurrent = std::max(S->st.max_concurrent, S->running);
        lk.unlock();

        hh_status st = HH_OK;
        std::string err;
        const double k = q->r.k, delta = q->r.delta, dh = q->r.delta_hat;
        if (!slot) {
            hh_problem* p = nullptr;
            cudaStream_t stream = nullptr;
            {
                std::lock_guard<std::mutex> g(S->dev_mu);
                if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
                    stream = nullptr;
                    st = HH_ERR_CUDA;
                    err = "stream creation failed";
                } else {
                    st = hh_create_problem(&q->r.grid, k, delta, dh, q->r.bc, &S->opts, stream, &p);
                    if (st == HH_OK) st = hh_prepare(p);
                    if (st != HH_OK) err = hh_last_error();
                }
            }
            lk.lock();
            S->reserved -= create;
            if (st == HH_OK) {
                auto s = std::make_unique<Slot>();
                s->p = p;
                s->stream = stream;
                s->grid = q->r.grid;
                std::memcpy(s->bc, q->r.bc, sizeof(s->bc));
                s->bytes = create;
                s->busy = true;
                slot = s.get();
                S->pool.push_back(std::move(s));
                S->held += create;
                ++S->st.problems_created;
                S->st.peak_bytes = std::max(S->st.peak_bytes, S->held);
                lk.unlock();
            } else {
                lk.unlock();
                drop_problem(S, p, stream);
            }
        } else {
            std::lock_guard<std::mutex> g(S->dev_mu);
            st = hh_set_params(slot->p, &k, &delta, &dh);
            if (st == HH_OK) st = hh_prepare(slot->p);
            if (st != HH_OK) err = hh_last_error();
        }
        if (st == HH_OK) {
            st = q->r.rhs_kind == 1 ? hh_solve_host_nodal(slot->p, q->rhs, q->r.tol, q->u, &q->info)
                                    : hh_solve_host(slot->p, q->rhs, q->r.tol, q->u, &q->info);
            if (st != HH_OK && st != HH_NOT_CONVERGED) err = hh_last_error();
        }

        lk.lock();
        q->st = st;
        q->err = err;
        q->t_end = clk::now();
        q->done = true;
        --S->running;
        if (st == HH_OK || st == HH_NOT_CONVERGED)
            ++S->st.completed;
        else
            ++S->st.failed;
        if (slot) {
            slot->busy = false;
            slot->last_use = ++S->tick;
            if (st != HH_OK && st != HH_NOT_CONVERGED && slot->p) {
                // a failed problem is not reused
                hh_problem* p = slot->p;
                cudaStream_t sv = slot->stream;
                S->held -= slot->bytes;
                S->pool.erase(std::remove_if(S->pool.begin(), S->pool.end(),
                                             [&](const std::unique_ptr<Slot>& s) { return s.get() == slot; }),
                              S->pool.end());
                lk.unlock();
                drop_problem(S, p, sv);
                lk.lock();
            }
        }
        S->cv.notify_all();
    }
}

}  // namespace

extern "C" {

hh_status invalid(const char* msg) {
    hh::set_last_error(msg);
    return HH_ERR_INVALID;
}

hh_status hh_server_create(int slots, size_t device_budget, const hh_options* opts, hh_server** out) {
    if (!out) return invalid("null out");
    *out = nullptr;
    if (slots < 1 || slots > 64) return invalid("slots must be in 1..64");
    if (device_budget == 0 || !opts) return invalid("zero budget or null options");
    if (opts->levels < 1 || opts->levels > 16) return invalid("levels must be in 1..16");
    if (opts->formulation != HH_FORM_PRIMAL) return invalid("the server solves primal problems");
    const hh_grid g{2, std::max(2, 1 << (opts->levels - 1))};
    if (hh_footprint_bytes(&g, opts) == 0) return HH_ERR_INVALID;  // options rejected, message set
    auto* S = new hh_server();
    cudaGetDevice(&S->device);
    S->slots = slots;
    S->budget = device_budget;
    S->opts = *opts;
    S->st.budget = device_budget;
    for (int w = 0; w < slots; ++w) S->workers.emplace_back(worker, S);
    *out = S;
    return HH_OK;
}

hh_status hh_server_submit(hh_server* S, const hh_request* r, const void* rhs_host, void* u_host, long long* ticket) {
    if (!S || !r || !rhs_host || !u_host || !ticket) return invalid("null argument");
    if (!(r->tol > 0)) return invalid("tol must be > 0");
    if (r->rhs_kind != 0 && r->rhs_kind != 1) return invalid("rhs_kind must be 0 (load vector) or 1 (nodal source)");
    const size_t need = hh_footprint_bytes(&r->grid, &S->opts);
    if (need == 0) return HH_ERR_INVALID;  // grid rejected, message set
    if (need > S->budget) return invalid("request footprint exceeds the server's device budget");
    if (!(r->k > 0) || !(r->delta >= 0) || !(r->delta_hat > 0) || !std::isfinite(r->k) ||
        !std::isfinite(r->delta) || !std::isfinite(r->delta_hat))
        return invalid("need k > 0, delta >= 0, delta_hat > 0 (finite)");
    for (int i = 0; i < 2 * r->grid.dim; ++i)
        if (r->bc[i] != HH_BC_SOMMERFELD && r->bc[i] != HH_BC_DIRICHLET) return invalid("bad boundary tag");
    auto q = std::make_unique<Req>();
    q->r = *r;
    q->rhs = rhs_host;
    q->u = u_host;
    q->t_submit = clk::now();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) return invalid("server is stopping");
    q->id = S->next_id++;
    *ticket = q->id;
    S->queue.push_back(q.get());
    S->reqs[q->id] = std::move(q);
    ++S->st.submitted;
    S->cv.notify_all();
    return HH_OK;
}

hh_status hh_server_wait(hh_server* S, long long ticket, hh_info* info, double* latency_s, double* queue_s) {
    if (!S) return invalid("null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return invalid("unknown ticket (never issued, or already waited for)");
    Req* q = it->second.get();
    S->cv.wait(lk, [&] { return q->done; });
    if (info) *info = q->info;
    if (latency_s) *latency_s = secs(q->t_submit, q->t_end);
    if (queue_s) *queue_s = secs(q->t_submit, q->t_start);
    const hh_status st = q->st;
    if (st != HH_OK && st != HH_NOT_CONVERGED) hh::set_last_error(q->err.c_str());
    S->reqs.erase(it);
    return st;
}

hh_status hh_server_get_stats(hh_server* S, hh_server_stats* out) {
    if (!S || !out) return invalid("null argument");
    std::lock_guard<std::mutex> g(S->mu);
    *out = S->st;
    out->held_bytes = S->held;
    out->queued = (long long)S->queue.size();
    out->running = S->running;
    return HH_OK;
}

void hh_server_destroy(hh_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    for (auto& t : S->workers) t.join();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    for (auto& s : S->pool) {
        if (s->p) hh_destroy(s->p);
        if (s->stream) cudaStreamDestroy(s->stream);
    }
    cudaSetDevice(cur);
    delete S;
}

}  // extern "C"
