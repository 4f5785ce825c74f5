// Continuous-batching solve server (host code): requests of many grid sizes and accuracy
// classes arrive at any time and are admitted onto the GPU as stream slots and device
// memory free up, so that their work overlaps on the device.  See superpot.h (sp_server_*)
// for the contract.
//
// One scheduler thread owns every CUDA call of the server except the completion callbacks:
//   - requests wait in per-key queues (key = grid size and precision);
//   - a key is served by resident plans (with their multiplier, workspace and batch
//     buffers), created on first use within the device-memory budget, evicting idle plans
//     of other keys least recently used first;
//   - the key whose oldest request has waited longest is served first; its waiting
//     requests form one batch (at most max_batch, at most max_batch_points grid points);
//   - a batch runs on a free slot stream: host-to-device copies, one batched solve
//     (Alg. 2 for each right-hand side), device-to-host copies, then a host callback
//     (cudaLaunchHostFunc) that stamps completion on the monotonic clock and hands the
//     slot back to the scheduler; small batches take the high-priority slots first;
//   - the callback runs on a thread of the CUDA driver, which must never wait for the
//     scheduler (the scheduler may itself be waiting inside a CUDA call for the device,
//     which waits for the callback): it only appends to a list under a lock of its own that
//     no one holds across a CUDA call, and the scheduler, waking at least every 100
//     microseconds while batches are in flight, finishes the requests;
//   - a request that cannot be served (a plan that cannot be created, a budget that can
//     never hold it) fails alone.
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "sp_internal.h"

namespace {

double now_s()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

void sleep_until_s(double t)
{
    for (;;) {
        const double d = t - now_s();
        if (d <= 0.0) return;
        if (d > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds((long long)((d - 1e-4) * 1e6)));
        // the last 100 microseconds are spun, for an arrival on time
    }
}

size_t io_size(sp_precision p) { return p == SP_FP32 ? 4 : 8; }

struct Req {
    long long id;
    int n;
    sp_precision prec;
    const void* in;
    void* out;
    double arrival, launched, done;
    sp_status status;
};

struct Entry {
    int n;
    sp_precision prec;
    sp_plan plan;
    void* d_in;
    void* d_out;
    size_t bytes;
    bool busy;
    double last_used;
};

struct Slot {
    sp_server_s* srv;
    cudaStream_t st;
    bool busy;
    Entry* entry;
    std::vector<Req*> reqs;
};

using Key = std::pair<int, int>;  // (n, precision)

}  // namespace

struct sp_server_s {
    sp_server_config cfg;
    int device;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::map<Key, std::deque<Req*>> pending;
    std::map<Key, std::vector<Entry*>> entries;
    std::vector<Slot*> slots;
    std::deque<Req*> done_queue;
    std::vector<sp_server_record> records;
    std::unordered_map<long long, Req*> live;
    double used_bytes = 0, peak_bytes = 0;
    long long batches = 0, next_id = 1;
    int in_flight = 0;  // batches launched and not yet finished (under mu)
    // completion callbacks' hand-over (under cb_mu only; never held across a CUDA call)
    std::mutex cb_mu;
    std::vector<std::pair<void*, double>> cb_done;  // (slot, completion time)
    bool stopping = false, stopped = false;
    cudaStream_t mem_st = nullptr;
    std::thread sched, feeder;
};

namespace {
using Srv = sp_server_s;

size_t entry_bytes(const Srv* s, int n, sp_precision p)
{
    const size_t c = (p == SP_FP64 || p == SP_DF32) ? 16 : 8, r = io_size(p);
    const size_t ldz = (size_t)(n + 1 + 7) / 8 * 8, nn = (size_t)n;
    const size_t work = (size_t)s->cfg.max_batch * c * nn * 2 * nn * ldz;
    const size_t tables = (nn + 1) * (nn + 1) * ldz * (8 + (p == SP_DF32 ? 8 : 4)) + 3 * 2 * nn * 32;
    const size_t io = 2 * (size_t)s->cfg.max_batch * nn * nn * nn * r;
    return work + tables + io + (1u << 20);
}

int batch_cap(const Srv* s, int n)
{
    const long long pts = (long long)n * n * n;
    long long cap = s->cfg.max_batch_points / pts;
    if (cap > s->cfg.max_batch) cap = s->cfg.max_batch;
    return cap < 1 ? 1 : (int)cap;
}

// Finish a request (any status), with the lock held.
void finish(Srv* s, Req* r, sp_status st, double t)
{
    r->status = st;
    r->done = t;
    if (st == SP_OK) {
        sp_server_record rec;
        rec.arrival = r->arrival;
        rec.launched = r->launched;
        rec.done = t;
        rec.n = r->n;
        rec.precision = (int)r->prec;
        s->records.push_back(rec);
    }
    s->done_queue.push_back(r);
}

void destroy_entry(Srv* s, Entry* e)
{
    sp_plan_destroy(e->plan);
    cudaFreeAsync(e->d_in, s->mem_st);
    cudaFreeAsync(e->d_out, s->mem_st);
    s->used_bytes -= (double)e->bytes;
    delete e;
}

// Free idle plans of other keys, least recently used first, until `need` fits.
bool evict_for(Srv* s, size_t need, Key keep)
{
    std::vector<std::pair<double, Entry*>> idle;
    for (auto& kv : s->entries)
        if (kv.first != keep)
            for (Entry* e : kv.second)
                if (!e->busy) idle.emplace_back(e->last_used, e);
    std::sort(idle.begin(), idle.end(), [](const std::pair<double, Entry*>& a, const std::pair<double, Entry*>& b) {
        return a.first < b.first;
    });
    for (auto& ie : idle) {
        if (s->used_bytes + (double)need <= s->cfg.budget_bytes) break;
        Entry* e = ie.second;
        auto& lst = s->entries[{e->n, (int)e->prec}];
        lst.erase(std::find(lst.begin(), lst.end(), e));
        destroy_entry(s, e);
    }
    return s->used_bytes + (double)need <= s->cfg.budget_bytes;
}

// A free resident plan of the key, a new one within the budget, or NULL (wait).  On a
// failure to create one, *err is set.
Entry* get_entry(Srv* s, Key key, sp_status* err)
{
    *err = SP_OK;
    auto& lst = s->entries[key];
    for (Entry* e : lst)
        if (!e->busy) return e;
    if ((int)lst.size() >= s->cfg.plans_per_key) return nullptr;
    const int n = key.first;
    const sp_precision prec = (sp_precision)key.second;
    const size_t need = entry_bytes(s, n, prec);
    if (s->used_bytes + (double)need > s->cfg.budget_bytes && !evict_for(s, need, key)) return nullptr;
    Entry* e = new (std::nothrow) Entry();
    if (!e) {
        *err = SP_ERR_OOM;
        return nullptr;
    }
    e->n = n;
    e->prec = prec;
    const int nn[3] = {n, n, n};
    const double lo[3] = {s->cfg.lo, s->cfg.lo, s->cfg.lo}, hi[3] = {s->cfg.hi, s->cfg.hi, s->cfg.hi};
    sp_status rc = sp_plan_create(&e->plan, nn, lo, hi, 2, nullptr, nullptr, 0, 1e-4, prec, s->cfg.max_batch);
    if (rc == SP_OK) rc = sp_kernel_precompute(e->plan, s->mem_st);
    const size_t io = (size_t)s->cfg.max_batch * (size_t)n * n * n * io_size(prec);
    if (rc == SP_OK) rc = sp_cuda_check(cudaMallocAsync(&e->d_in, io, s->mem_st), "server batch buffer");
    if (rc == SP_OK) rc = sp_cuda_check(cudaMallocAsync(&e->d_out, io, s->mem_st), "server batch buffer");
    // the slot streams are not ordered after mem_st: publish the plan once it is ready
    if (rc == SP_OK) rc = sp_cuda_check(cudaStreamSynchronize(s->mem_st), "server plan setup");
    if (rc != SP_OK) {
        sp_plan_destroy(e->plan);
        if (e->d_in) cudaFreeAsync(e->d_in, s->mem_st);
        if (e->d_out) cudaFreeAsync(e->d_out, s->mem_st);
        delete e;
        *err = rc;
        return nullptr;
    }
    e->bytes = need;
    e->last_used = now_s();
    lst.push_back(e);
    s->used_bytes += (double)need;
    s->peak_bytes = std::max(s->peak_bytes, s->used_bytes);
    return e;
}

void CUDART_CB on_batch_done(void* ud)
{
    Slot* sl = static_cast<Slot*>(ud);
    Srv* s = sl->srv;
    const double t = now_s();
    {
        std::lock_guard<std::mutex> g(s->cb_mu);
        s->cb_done.emplace_back(ud, t);
    }
    s->cv_sched.notify_one();
}

// Finish the batches whose callbacks have run (mu held).  Returns true if there were any.
bool drain_completions(Srv* s)
{
    std::vector<std::pair<void*, double>> done;
    {
        std::lock_guard<std::mutex> g(s->cb_mu);
        done.swap(s->cb_done);
    }
    for (auto& d : done) {
        Slot* sl = static_cast<Slot*>(d.first);
        for (Req* r : sl->reqs) finish(s, r, SP_OK, d.second);
        sl->reqs.clear();
        sl->entry->busy = false;
        sl->entry->last_used = d.second;
        sl->entry = nullptr;
        sl->busy = false;
        --s->in_flight;
    }
    if (!done.empty()) s->cv_done.notify_all();
    return !done.empty();
}

// Launch one batch on slot `sl` (lock held; the CUDA calls only enqueue work).
void launch(Srv* s, Slot* sl, Entry* e, std::vector<Req*>& reqs)
{
    const size_t io = (size_t)e->n * e->n * e->n * io_size(e->prec);
    const double t = now_s();
    sl->busy = true;
    sl->entry = e;
    sl->reqs = reqs;
    e->busy = true;
    const int b = (int)reqs.size();
    sp_status rc = SP_OK;
    for (int i = 0; i < b && rc == SP_OK; ++i) {
        reqs[i]->launched = t;
        rc = sp_cuda_check(cudaMemcpyAsync((char*)e->d_in + i * io, reqs[i]->in, io, cudaMemcpyHostToDevice, sl->st),
                           "server input copy");
    }
    if (rc == SP_OK) rc = sp_solve_batched(e->plan, e->d_in, e->d_out, b, sl->st);
    for (int i = 0; i < b && rc == SP_OK; ++i)
        rc = sp_cuda_check(cudaMemcpyAsync(reqs[i]->out, (char*)e->d_out + i * io, io, cudaMemcpyDeviceToHost, sl->st),
                           "server output copy");
    if (rc == SP_OK) rc = sp_cuda_check(cudaLaunchHostFunc(sl->st, on_batch_done, sl), "server completion callback");
    if (rc == SP_OK) ++s->in_flight;
    if (rc != SP_OK) {  // the batch fails alone; the slot and plan are released after its stream drains
        cudaStreamSynchronize(sl->st);
        const double td = now_s();
        for (Req* r : sl->reqs) finish(s, r, rc, td);
        sl->reqs.clear();
        sl->busy = false;
        sl->entry = nullptr;
        e->busy = false;
        s->cv_done.notify_all();
        return;
    }
    ++s->batches;
}

// One scheduling step (lock held): launch at most one batch.  Returns true if it did.
bool schedule_one(Srv* s)
{
    std::vector<Slot*> free_hi, free_lo;
    for (int i = 0; i < (int)s->slots.size(); ++i)
        if (!s->slots[i]->busy) (i < s->cfg.priority_slots ? free_hi : free_lo).push_back(s->slots[i]);
    if (free_hi.empty() && free_lo.empty()) return false;
    std::vector<std::pair<double, Key>> keys;
    for (auto& kv : s->pending)
        if (!kv.second.empty()) keys.emplace_back(kv.second.front()->arrival, kv.first);
    std::sort(keys.begin(), keys.end());
    for (auto& k : keys) {
        const Key key = k.second;
        auto& q = s->pending[key];
        const sp_precision prec = (sp_precision)key.second;
        if ((double)entry_bytes(s, key.first, prec) > s->cfg.budget_bytes) {  // can never be admitted
            const double t = now_s();
            while (!q.empty()) {
                finish(s, q.front(), SP_ERR_OOM, t);
                q.pop_front();
            }
            s->cv_done.notify_all();
            continue;
        }
        sp_status err;
        Entry* e = get_entry(s, key, &err);
        if (!e) {
            if (err != SP_OK) {  // the plan cannot be created: this key's requests fail
                const double t = now_s();
                while (!q.empty()) {
                    finish(s, q.front(), err, t);
                    q.pop_front();
                }
                s->cv_done.notify_all();
            }
            continue;
        }
        const int cap = batch_cap(s, key.first);
        std::vector<Req*> reqs;
        while (!q.empty() && (int)reqs.size() < cap) {
            reqs.push_back(q.front());
            q.pop_front();
        }
        const bool small = (long long)reqs.size() * key.first * key.first * key.first <= s->cfg.small_points;
        Slot* sl = small ? (!free_hi.empty() ? free_hi[0] : free_lo[0]) : (!free_lo.empty() ? free_lo[0] : free_hi[0]);
        launch(s, sl, e, reqs);
        return true;
    }
    return false;
}

void scheduler(Srv* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stopping) {
        drain_completions(s);
        if (schedule_one(s)) continue;
        // callbacks notify without mu, so a wakeup can be missed: poll while work is in flight
        if (s->in_flight > 0) s->cv_sched.wait_for(lk, std::chrono::microseconds(100));
        else s->cv_sched.wait(lk);
    }
}

sp_status enqueue(Srv* s, long long id, int n, sp_precision prec, const void* in, void* out, double arrival)
{
    Req* r = new (std::nothrow) Req();
    if (!r) return sp_fail(SP_ERR_OOM, "host allocation failed");
    r->id = id;
    r->n = n;
    r->prec = prec;
    r->in = in;
    r->out = out;
    r->arrival = arrival;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stopping) {
        delete r;
        return sp_fail(SP_ERR_INVALID, "server is stopping");
    }
    s->live[id] = r;
    s->pending[{n, (int)prec}].push_back(r);
    s->cv_sched.notify_one();
    return SP_OK;
}

sp_status check_request(int n, sp_precision prec, const void* in, const void* out)
{
    if (n < 2) return sp_fail(SP_ERR_INVALID, "n must be >= 2 (got %d)", n);
    if (prec != SP_FP64 && prec != SP_FP32 && prec != SP_MIXED && prec != SP_DF32)
        return sp_fail(SP_ERR_INVALID, "unknown precision %d", (int)prec);
    if (!in || !out) return sp_fail(SP_ERR_INVALID, "rho_host and u_host must be non-NULL");
    return SP_OK;
}

}  // namespace

extern "C" double sp_monotonic_seconds(void) { return now_s(); }

extern "C" size_t sp_server_entry_bytes(const sp_server_config* cfg, int n, sp_precision prec)
{
    if (!cfg || n < 1) return 0;
    Srv tmp;
    tmp.cfg = *cfg;
    return entry_bytes(&tmp, n, prec);
}

extern "C" sp_status sp_server_create(sp_server* out, const sp_server_config* cfg)
{
    sp_clear_error();
    if (!out || !cfg) return sp_fail(SP_ERR_INVALID, "out and cfg must be non-NULL");
    *out = nullptr;
    if (!(cfg->hi > cfg->lo) || cfg->max_batch < 1 || cfg->slots < 1 || cfg->plans_per_key < 1 ||
        cfg->priority_slots < 0 || cfg->max_batch_points < 1 || !(cfg->budget_bytes > 0))
        return sp_fail(SP_ERR_INVALID, "bad server configuration");
    Srv* s = new (std::nothrow) Srv();
    if (!s) return sp_fail(SP_ERR_OOM, "host allocation failed");
    s->cfg = *cfg;
    if (s->cfg.priority_slots > s->cfg.slots - 1) s->cfg.priority_slots = s->cfg.slots - 1;
    cudaGetDevice(&s->device);
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    sp_status rc = sp_cuda_check(cudaStreamCreateWithFlags(&s->mem_st, cudaStreamNonBlocking), "server stream");
    for (int i = 0; i < cfg->slots && rc == SP_OK; ++i) {
        Slot* sl = new (std::nothrow) Slot();
        if (!sl) {
            rc = sp_fail(SP_ERR_OOM, "host allocation failed");
            break;
        }
        sl->srv = s;
        s->slots.push_back(sl);
        rc = sp_cuda_check(cudaStreamCreateWithPriority(&sl->st, cudaStreamNonBlocking,
                                                        i < s->cfg.priority_slots ? greatest : least),
                           "server slot stream");
    }
    if (rc != SP_OK) {
        for (Slot* sl : s->slots) {
            if (sl->st) cudaStreamDestroy(sl->st);
            delete sl;
        }
        if (s->mem_st) cudaStreamDestroy(s->mem_st);
        delete s;
        return rc;
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    return SP_OK;
}

extern "C" sp_status sp_server_prepare(sp_server s, int n, sp_precision prec)
{
    sp_clear_error();
    if (!s) return sp_fail(SP_ERR_INVALID, "server is NULL");
    if (n < 2) return sp_fail(SP_ERR_INVALID, "n must be >= 2");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != s->device)
        return sp_fail(SP_ERR_INVALID, "the server's device (%d) must be current (current: %d)", s->device, cur);
    std::lock_guard<std::mutex> g(s->mu);
    const Key key{n, (int)prec};
    auto& lst = s->entries[key];
    // plans_per_key plans while the budget holds them (more are built on demand)
    std::vector<Entry*> held;
    for (Entry* e : lst) {
        if (!e->busy) {
            e->busy = true;
            held.push_back(e);
        }
    }
    sp_status rc = SP_OK;
    while ((int)lst.size() < s->cfg.plans_per_key &&
           s->used_bytes + (double)entry_bytes(s, n, prec) <= s->cfg.budget_bytes) {
        sp_status err;
        Entry* e = get_entry(s, key, &err);
        if (!e) {
            rc = err != SP_OK ? err : sp_fail(SP_ERR_OOM, "no room for another plan");
            break;
        }
        e->busy = true;
        held.push_back(e);
    }
    for (Entry* e : held) e->busy = false;
    return rc;
}

extern "C" sp_status sp_server_submit(sp_server s, int n, sp_precision prec, const void* rho_host, void* u_host,
                                      double arrival, long long* ticket)
{
    sp_clear_error();
    if (!s || !ticket) return sp_fail(SP_ERR_INVALID, "server and ticket must be non-NULL");
    sp_status rc = check_request(n, prec, rho_host, u_host);
    if (rc) return rc;
    long long id;
    {
        std::lock_guard<std::mutex> g(s->mu);
        id = s->next_id++;
    }
    if ((rc = enqueue(s, id, n, prec, rho_host, u_host, arrival < 0 ? now_s() : arrival))) return rc;
    *ticket = id;
    return SP_OK;
}

extern "C" sp_status sp_server_replay(sp_server s, int count, const double* arrival, const int* n, const int* prec,
                                      const void* const* rho_host, void* const* u_host, long long* tickets)
{
    sp_clear_error();
    if (!s || count < 0 || (count > 0 && (!arrival || !n || !prec || !rho_host || !u_host || !tickets)))
        return sp_fail(SP_ERR_INVALID, "bad replay arguments");
    for (int i = 0; i < count; ++i) {
        sp_status rc = check_request(n[i], (sp_precision)prec[i], rho_host[i], u_host[i]);
        if (rc) return rc;
        if (i > 0 && arrival[i] < arrival[i - 1]) return sp_fail(SP_ERR_INVALID, "arrival times must not decrease");
    }
    if (s->feeder.joinable()) s->feeder.join();  // a previous replay has finished submitting
    long long first;
    {
        std::lock_guard<std::mutex> g(s->mu);
        first = s->next_id;
        s->next_id += count;
    }
    for (int i = 0; i < count; ++i) tickets[i] = first + i;
    std::vector<Req> plan(count);
    for (int i = 0; i < count; ++i) {
        plan[i].id = first + i;
        plan[i].n = n[i];
        plan[i].prec = (sp_precision)prec[i];
        plan[i].in = rho_host[i];
        plan[i].out = u_host[i];
        plan[i].arrival = arrival[i];
    }
    s->feeder = std::thread([s, plan]() {
        for (const Req& r : plan) {
            sleep_until_s(r.arrival);
            if (enqueue(s, r.id, r.n, r.prec, r.in, r.out, r.arrival) != SP_OK) return;
        }
    });
    return SP_OK;
}

extern "C" sp_status sp_server_next_done(sp_server s, double timeout_s, long long* ticket, double* times)
{
    sp_clear_error();
    if (!s || !ticket) return sp_fail(SP_ERR_INVALID, "server and ticket must be non-NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto pred = [s] { return !s->done_queue.empty() || s->stopped; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
    if (s->done_queue.empty()) {
        if (s->stopped) return sp_fail(SP_ERR_INVALID, "server stopped and drained");
        return SP_ERR_NOT_READY;  // timeout, nothing finished
    }
    Req* r = s->done_queue.front();
    s->done_queue.pop_front();
    *ticket = r->id;
    if (times) {
        times[0] = r->arrival;
        times[1] = r->launched;
        times[2] = r->done;
    }
    const sp_status st = r->status;
    s->live.erase(r->id);
    delete r;
    if (st != SP_OK) return sp_fail(st, "request %lld failed (status %d)", *ticket, (int)st);
    return SP_OK;
}

extern "C" sp_status sp_server_stats(sp_server s, long long* batches, double* peak_bytes, double* used_bytes)
{
    sp_clear_error();
    if (!s) return sp_fail(SP_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    if (batches) *batches = s->batches;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    if (used_bytes) *used_bytes = s->used_bytes;
    return SP_OK;
}

extern "C" int sp_server_records(sp_server s, int max, sp_server_record* out)
{
    sp_clear_error();
    if (!s) {
        sp_fail(SP_ERR_INVALID, "server is NULL");
        return -1;
    }
    std::lock_guard<std::mutex> g(s->mu);
    const int total = (int)s->records.size();
    for (int i = 0; out && i < max && i < total; ++i) out[i] = s->records[i];
    return total;
}

extern "C" sp_status sp_server_shutdown(sp_server s)
{
    sp_clear_error();
    if (!s) return SP_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stopped) return SP_OK;
        s->stopping = true;  // a replay's feeder stops at its next arrival
        s->cv_sched.notify_all();
    }
    if (s->feeder.joinable()) s->feeder.join();
    if (s->sched.joinable()) s->sched.join();
    // batches in flight complete (their callbacks hand them over)
    for (Slot* sl : s->slots) cudaStreamSynchronize(sl->st);
    std::lock_guard<std::mutex> g(s->mu);
    drain_completions(s);
    const double t = now_s();
    for (auto& kv : s->pending) {
        for (Req* r : kv.second) finish(s, r, SP_ERR_INVALID, t);
        kv.second.clear();
    }
    s->stopped = true;
    s->cv_done.notify_all();
    return SP_OK;
}

extern "C" sp_status sp_server_destroy(sp_server s)
{
    sp_clear_error();
    if (!s) return SP_OK;
    sp_server_shutdown(s);
    const int dev = s->device;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != dev) cudaSetDevice(dev);
    for (auto& kv : s->entries)
        for (Entry* e : kv.second) destroy_entry(s, e);
    s->entries.clear();
    cudaStreamSynchronize(s->mem_st);
    cudaStreamDestroy(s->mem_st);
    for (Slot* sl : s->slots) {
        cudaStreamDestroy(sl->st);
        delete sl;
    }
    for (Req* r : s->done_queue) delete r;
    delete s;
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    return SP_OK;
}
