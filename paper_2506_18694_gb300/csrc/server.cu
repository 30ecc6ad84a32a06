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
    bool fallback = false;   // solve again with fb_opts / fb_dh if the first solve does not converge
    bool packed = false;     // the pack dispatcher runs its first solve
    bool fallback_pending = false;  // left the pack unconverged: a worker runs the fallback
    hh_options fb_opts{};
    double fb_dh = 0.0;
    const void* rhs = nullptr;
    void* u = nullptr;
    hh_status st = HH_OK;
    hh_info info{};
    clk::time_point t_submit, t_start, t_end;
    bool done = false;
    std::string err;
};

struct Slot {
    int kind = 0;                   // 0: built with the server's options, 1: with the fallback's
    hh_problem* p = nullptr;
    cudaStream_t stream = nullptr;  // the problem's caller stream, used by nobody else
    hh_grid grid{};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    size_t bytes = 0;
    bool busy = false;
    long long last_use = 0;
};

bool same_shape(const Slot& s, const hh_request& r, int kind) {
    if (s.kind != kind || s.grid.dim != r.grid.dim || s.grid.n != r.grid.n) return false;
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
    bool has_fallback = false;       // see hh_server_set_fallback
    int pack_capacity = 0;           // > 0: 2D requests run in a pack (hh_server_set_pack)
    int pack_max_hss = 0;            // only those with at most this many HSS steps (0: all)
    std::thread pack_thread;
    hh_options fb_opts{};
    double fb_dh = 0.0;
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

void release(hh_server* S, std::unique_lock<std::mutex>& lk, Slot* slot, hh_status st);

// Take a problem for request q (lock held on entry and exit; may release it while waiting).
// Returns the slot, or nullptr with *create_bytes set when a new problem must be created
// (its bytes already reserved).  wait = false: returns nullptr with *create_bytes = 0 instead
// of waiting for a running solve to return its problem.
Slot* acquire(hh_server* S, std::unique_lock<std::mutex>& lk, const Req* q, int kind, size_t need,
              size_t* create_bytes, bool wait = true) {
    *create_bytes = 0;
    for (;;) {
        for (auto& s : S->pool)
            if (!s->busy && s->p && same_shape(*s, q->r, kind)) {
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
        if (!wait) return nullptr;
        S->cv.wait(lk);  // a running solve returns its problem
    }
}

// A problem for request q built with opts (kind 0: the server's, 1: the fallback's) and shift
// dh, taken from the pool (retargeted) or created, busy; nullptr with *st set on failure, or
// with *st = HH_OK when wait = false and no memory is free now.  Lock held on entry and exit.
Slot* obtain(hh_server* S, std::unique_lock<std::mutex>& lk, Req* q, int kind, const hh_options& opts, double dh,
             bool wait, hh_status* st, std::string* err) {
    *st = HH_OK;
    const size_t need = hh_footprint_bytes(&q->r.grid, &opts);
    size_t create = 0;
    Slot* slot = acquire(S, lk, q, kind, need, &create, wait);
    if (!slot && create == 0) return nullptr;  // nothing free now (wait = false)
    lk.unlock();
    const double k = q->r.k, delta = q->r.delta;
    if (!slot) {
        hh_problem* p = nullptr;
        cudaStream_t stream = nullptr;
        {
            std::lock_guard<std::mutex> g(S->dev_mu);
            if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
                stream = nullptr;
                *st = HH_ERR_CUDA;
                *err = "stream creation failed";
            } else {
                *st = hh_create_problem(&q->r.grid, k, delta, dh, q->r.bc, &opts, stream, &p);
                if (*st == HH_OK) *st = hh_prepare(p);
                if (*st != HH_OK) *err = hh_last_error();
            }
        }
        lk.lock();
        S->reserved -= create;
        if (*st == HH_OK) {
            auto sl = std::make_unique<Slot>();
            sl->kind = kind;
            sl->p = p;
            sl->stream = stream;
            sl->grid = q->r.grid;
            std::memcpy(sl->bc, q->r.bc, sizeof(sl->bc));
            sl->bytes = create;
            sl->busy = true;
            slot = sl.get();
            S->pool.push_back(std::move(sl));
            S->held += create;
            ++S->st.problems_created;
            S->st.peak_bytes = std::max(S->st.peak_bytes, S->held);
            return slot;
        }
        lk.unlock();
        drop_problem(S, p, stream);
        lk.lock();
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> g(S->dev_mu);
        *st = hh_set_params(slot->p, &k, &delta, &dh);
        if (*st == HH_OK) *st = hh_prepare(slot->p);
        if (*st != HH_OK) *err = hh_last_error();
    }
    lk.lock();
    if (*st != HH_OK) {
        release(S, lk, slot, *st);
        return nullptr;
    }
    return slot;
}

// Return a problem to the pool after a solve that ended with status st (a failed problem is
// destroyed, not reused).  Lock held on entry and exit.
void release(hh_server* S, std::unique_lock<std::mutex>& lk, Slot* slot, hh_status st) {
    slot->busy = false;
    slot->last_use = ++S->tick;
    if (st != HH_OK && st != HH_NOT_CONVERGED && slot->p) {
        hh_problem* p = slot->p;
        cudaStream_t sv = slot->stream;
        S->held -= slot->bytes;
        S->pool.erase(std::remove_if(S->pool.begin(), S->pool.end(),
                                     [&](const std::unique_ptr<Slot>& x) { return x.get() == slot; }),
                      S->pool.end());
        lk.unlock();
        drop_problem(S, p, sv);
        lk.lock();
    }
    S->cv.notify_all();  // a problem went back to the pool
}

// One solve of request q (obtain a problem, solve, release).  Lock held on entry and exit.
hh_status attempt(hh_server* S, std::unique_lock<std::mutex>& lk, Req* q, int kind, const hh_options& opts,
                  double dh, hh_info* info, std::string* err) {
    hh_status st;
    Slot* slot = obtain(S, lk, q, kind, opts, dh, true, &st, err);
    if (!slot) return st;
    lk.unlock();
    st = q->r.rhs_kind == 1 ? hh_solve_host_nodal(slot->p, q->rhs, q->r.tol, q->u, info)
                            : hh_solve_host(slot->p, q->rhs, q->r.tol, q->u, info);
    if (st != HH_OK && st != HH_NOT_CONVERGED) *err = hh_last_error();
    lk.lock();
    release(S, lk, slot, st);
    return st;
}

// Record the outcome of request q (lock held).
void complete(hh_server* S, Req* q, hh_status st, const hh_info& info, const std::string& err) {
    q->st = st;
    q->err = err;
    q->info = info;
    q->t_end = clk::now();
    q->done = true;
    --S->running;
    if (st == HH_OK || st == HH_NOT_CONVERGED)
        ++S->st.completed;
    else
        ++S->st.failed;
    S->cv.notify_all();
}

bool fallback_fits(hh_server* S, const Req* q) {
    const size_t need = q->fallback ? hh_footprint_bytes(&q->r.grid, &q->fb_opts) : 0;
    return q->fallback && need > 0 && need <= S->budget;
}

// the next request a worker runs: the first that the pack does not take, or one that left the
// pack unconverged and waits for its fallback solve
Req* worker_job(hh_server* S) {
    for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if (!(*it)->packed || (*it)->fallback_pending) {
            Req* q = *it;
            S->queue.erase(it);
            return q;
        }
    return nullptr;
}

void worker(hh_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        Req* q = nullptr;
        S->cv.wait(lk, [&] { return (q = worker_job(S)) != nullptr || (S->stop && S->queue.empty()); });
        if (!q) return;  // stopping and drained
        std::string err;
        hh_info info{};
        hh_status st = HH_NOT_CONVERGED;
        if (!q->fallback_pending) {
            q->t_start = clk::now();
            ++S->running;
            S->st.max_concurrent = std::max(S->st.max_concurrent, S->running);
            st = attempt(S, lk, q, 0, S->opts, q->r.delta_hat, &info, &err);
        } else {
            info = q->info;  // the first (packed) solve
        }
        if (st == HH_NOT_CONVERGED && fallback_fits(S, q)) {
            hh_info info2{};
            st = attempt(S, lk, q, 1, q->fb_opts, q->fb_dh, &info2, &err);
            info2.outer_its += info.outer_its;
            info2.hss_its += info.hss_its;
            info2.vcycles += info.vcycles;
            info2.seconds += info.seconds;
            info2.kernel_launches += info.kernel_launches;
            info2.fallback = 1;
            info = info2;
        }
        complete(S, q, st, info, err);
    }
}

// The pack dispatcher: requests the pack can run join it as slots and device memory allow,
// between rounds; finished members leave at once (their slot is refilled in the next round).
void dispatcher(hh_server* S) {
    cudaSetDevice(S->device);
    hh_pack* pk = nullptr;
    const hh_status cst = hh_pack_create(S->pack_capacity, &pk);
    std::vector<int> done(S->pack_capacity);
    std::map<int, std::pair<Req*, Slot*>> members;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // admit
        while ((int)members.size() < S->pack_capacity) {
            Req* q = nullptr;
            for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
                if ((*it)->packed && !(*it)->fallback_pending) {
                    q = *it;
                    break;
                }
            if (!q) break;
            hh_status st;
            std::string err;
            Slot* slot = nullptr;
            if (cst == HH_OK) {
                slot = obtain(S, lk, q, 0, S->opts, q->r.delta_hat, members.empty(), &st, &err);
                if (!slot && st == HH_OK) break;  // no memory now: wait for members to finish
            } else {
                st = cst;
                err = "pack creation failed";
            }
            S->queue.erase(std::find(S->queue.begin(), S->queue.end(), q));
            q->t_start = clk::now();
            ++S->running;
            S->st.max_concurrent = std::max(S->st.max_concurrent, S->running);
            if (!slot) {
                complete(S, q, st, hh_info{}, err);
                continue;
            }
            int ps = -1;
            lk.unlock();
            st = hh_pack_add(pk, slot->p, q->rhs, q->r.rhs_kind == 1 ? 2 : 1, q->r.tol, q->u, &ps);
            if (st != HH_OK) err = hh_last_error();
            lk.lock();
            if (st != HH_OK) {
                release(S, lk, slot, st);
                complete(S, q, st, hh_info{}, err);
                continue;
            }
            members[ps] = {q, slot};
        }
        if (members.empty()) {
            const bool more = std::any_of(S->queue.begin(), S->queue.end(),
                                          [](const Req* q) { return q->packed && !q->fallback_pending; });
            if (S->stop && !more) break;
            if (!more) S->cv.wait(lk);
            continue;
        }
        // one round (new requests join before the next one)
        int nd = 0;
        lk.unlock();
        hh_status rs;
        {
            std::lock_guard<std::mutex> g(S->dev_mu);  // a round may capture the pack's graph
            rs = hh_pack_run(pk, 1, done.data(), &nd);
        }
        const std::string rerr = rs == HH_OK ? std::string() : std::string(hh_last_error());
        lk.lock();
        if (rs != HH_OK) {  // the pack failed: every member fails
            for (auto& [ps, qs] : members) {
                hh_info none{};
                hh_pack_take(pk, ps, &none);
                release(S, lk, qs.second, rs);
                complete(S, qs.first, rs, none, rerr);
            }
            members.clear();
            continue;
        }
        for (int i = 0; i < nd; ++i) {
            auto it = members.find(done[i]);
            if (it == members.end()) continue;
            Req* q = it->second.first;
            Slot* slot = it->second.second;
            members.erase(it);
            hh_info info{};
            const hh_status st = hh_pack_take(pk, done[i], &info);
            const std::string err = (st == HH_OK || st == HH_NOT_CONVERGED) ? std::string() : hh_last_error();
            release(S, lk, slot, st);
            if (st == HH_NOT_CONVERGED && fallback_fits(S, q)) {
                q->info = info;
                q->fallback_pending = true;  // a worker solves it again with the fallback settings
                S->queue.push_front(q);
                S->cv.notify_all();
                continue;
            }
            complete(S, q, st, info, err);
        }
    }
    lk.unlock();
    if (pk) hh_pack_destroy(pk);
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
    q->fallback = S->has_fallback;
    q->fb_opts = S->fb_opts;
    q->fb_dh = S->fb_dh;
    // HSS steps of the request (ceil(k^theta), an integer power counted exactly)
    const double v = std::pow(r->k, S->opts.theta), vr = std::round(v);
    const int steps = std::fabs(v - vr) <= 1e-9 * std::max(1.0, v) ? (int)vr : (int)std::ceil(v);
    q->packed = S->pack_capacity > 0 && r->grid.dim == 2 && (S->pack_max_hss == 0 || steps <= S->pack_max_hss);
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

hh_status hh_server_set_fallback(hh_server* S, const hh_options* opts, double delta_hat) {
    if (!S) return invalid("null server");
    if (opts) {
        if (!(delta_hat > 0) || !std::isfinite(delta_hat)) return invalid("fallback delta_hat must be > 0 (finite)");
        if (opts->formulation != HH_FORM_PRIMAL) return invalid("the server solves primal problems");
        const hh_grid g{2, std::max(2, 1 << (std::max(1, std::min(16, opts->levels)) - 1))};
        if (opts->levels < 1 || opts->levels > 16 || hh_footprint_bytes(&g, opts) == 0)
            return invalid("fallback options rejected");
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->has_fallback = opts != nullptr;
    if (opts) {
        S->fb_opts = *opts;
        S->fb_dh = delta_hat;
    }
    return HH_OK;
}

hh_status hh_server_set_pack(hh_server* S, int capacity, int max_hss_steps) {
    if (!S) return invalid("null server");
    if (capacity < 1 || capacity > 256) return invalid("pack capacity must be in 1..256");
    if (max_hss_steps < 0) return invalid("max_hss_steps must be >= 0");
    const hh_options& o = S->opts;
    if (o.smoother != HH_SMOOTH_JACOBI || o.cycle_gamma != 1 || o.cycles_per_hss != 1 || o.nu_pre != 2 ||
        o.nu_post != 2 || o.precision != HH_C64 || o.outer != HH_OUTER_FGMRES || o.levels < 2 || o.levels > 5)
        return invalid("the server's options cannot be packed (V(2,2) scaled Jacobi, one cycle per HSS step, "
                       "complex64 cycles, FGMRES, 2..5 levels)");
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->pack_capacity > 0) return invalid("the server already packs its requests");
    if (S->st.submitted > 0) return invalid("set the pack before the first request");
    S->pack_capacity = capacity;
    S->pack_max_hss = max_hss_steps;
    S->pack_thread = std::thread(dispatcher, S);
    return HH_OK;
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
    if (S->pack_thread.joinable()) S->pack_thread.join();
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
