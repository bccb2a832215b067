// Serving loop: continuous batching of independent Ewald evaluations (ewald_server_*).
//
// The paper evaluates one system per time step (Section 4); a serving deployment instead
// receives many independent systems of uneven size.  A server owns:
//   * a FIFO of submitted requests,
//   * `max_slots` slots, each with a reusable plan (re-parameterised per request, so its
//     cell lists, k tables and workspaces stay resident and are only regrown when a request
//     needs more), a CUDA stream and a completion event,
//   * a scheduler thread that, whenever a slot is free, admits queued requests first-fit in
//     arrival order while the device memory held by all slots (estimated per request from its
//     parameters and N) stays within the HBM budget, hands each admitted request to its
//     slot, and retires requests whose completion event has fired;
//   * one launcher thread per slot, which re-parameterises the slot's plan and launches the
//     request's whole pipeline on the slot's stream (the host work of a launch, ~0.1-0.3 ms
//     for a request of a few thousand particles, runs for several slots at once).
// Requests admitted while others are running execute concurrently on separate streams.
// Every wait on the host is bounded (ewald_wait takes a time limit); no kernel waits on
// another request.
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ewald_internal.cuh"

using namespace ew;

namespace {

struct Pending {
    uint64_t ticket;
    ewald_request req;
    double t_submit;
    size_t footprint;
    cudaEvent_t ready;   // recorded on the producer stream at submit
};

struct Slot {
    ewald_plan *plan = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    double *energy_d = nullptr;
    double *energy_h = nullptr;   // pinned [4]
    int *status_h = nullptr;      // pinned [1]
    bool busy = false;
    uint64_t ticket = 0;
    size_t held = 0;              // device bytes attributed to this slot's plan
    double t_admit = 0;
    double t_submit = 0;
    size_t footprint = 0;
    int launch_status = EWALD_OK;
    // hand-over to the slot's launcher thread (under the server's mutex)
    bool has_work = false;        // a request waits for its launch
    bool launched = true;         // the request's pipeline (or its failure) has been issued
    Pending work{};
};

constexpr int kMaxBypass = 64;   // requests admitted past a waiting head before it blocks them

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int cuda_st(cudaError_t e)
{
    if (e == cudaSuccess) return EWALD_OK;
    return e == cudaErrorMemoryAllocation ? EWALD_E_NOMEM : EWALD_E_CUDA;
}

// One step of the admission policy for the queued request at the front of the scan (pure
// host logic: the scheduler and ewald_server_simulate share it).  The request (footprint
// fp, is_head when it is the first in the queue) would run on the idle slot that holds the
// most memory (the first such slot); if the held total with it exceeds the budget, the
// idle slots other than that one give back their workspaces, in slot order, until it fits
// (they are reclaimed even if it still does not).  Returns kAdmitStop, with nothing to
// reclaim, when no slot is idle, or when the request is not the head and the head has
// already been passed over max_bypass times (then nothing behind the head may run, so no
// idle workspace is given up for it); kAdmitSkip when it does not fit (the scan goes on with
// the next request); kAdmitTake when it is admitted on *slot.
enum AdmitAction { kAdmitStop = 0, kAdmitSkip = 1, kAdmitTake = 2 };
struct AdmitSlot {
    bool busy;
    int64_t held;
};
int admit_step(int64_t fp, bool is_head, const std::vector<AdmitSlot> &slots, int64_t held_total,
               int64_t budget, int head_bypass, int max_bypass, int *slot,
               std::vector<int> *reclaim)
{
    reclaim->clear();
    int fs = -1;
    for (int i = 0; i < (int)slots.size(); ++i)
        if (!slots[i].busy && (fs < 0 || slots[i].held > slots[fs].held)) fs = i;
    if (fs < 0) return kAdmitStop;
    if (!is_head && head_bypass >= max_bypass) return kAdmitStop;
    int64_t after = held_total - slots[fs].held + fp;
    for (int i = 0; i < (int)slots.size() && after > budget; ++i) {
        if (slots[i].busy || i == fs || slots[i].held == 0) continue;
        reclaim->push_back(i);
        after -= slots[i].held;
    }
    if (after > budget) return kAdmitSkip;
    *slot = fs;
    return kAdmitTake;
}

}  // namespace

struct ewald_server {
    int device = 0;
    size_t budget = 0;
    std::vector<Slot> slots;
    std::deque<Pending> queue;
    size_t max_queue = 1 << 16;
    std::unordered_map<uint64_t, ewald_result> results;   // finished, not yet polled
    std::unordered_map<uint64_t, int> state;              // 0 queued, 1 running, 2 done
    std::mutex mu;
    std::condition_variable cv;      // wakes the scheduler
    std::condition_variable wcv;     // wakes the launcher threads
    std::thread th;
    std::vector<std::thread> launchers;
    bool stop = false;
    bool quit_launchers = false;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0;
    int64_t held_total = 0, peak_held = 0, peak_running = 0;
    int head_bypass = 0;             // admissions that passed over the head of the queue
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

size_t request_footprint(const ewald_request &r)
{
    Plan probe;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (plan_setup_host(probe, r.L, r.beta, r.r_c, r.k_max, r.precision) != EWALD_OK) return 0;
    return plan_footprint(probe, r.n);
}

// Launch one request on a slot (scheduler thread, no lock held).
int launch(ewald_server *s, Slot &sl, const Pending &pd)
{
    const ewald_request &r = pd.req;
    int st;
    if (!sl.plan) {
        st = ewald_create(r.L, r.beta, r.r_c, r.k_max, r.precision, &sl.plan);
    } else {
        const Plan &p = sl.plan->p;
        if (p.L != r.L || p.beta != r.beta || p.rc != r.r_c || p.kmax != r.k_max ||
            p.precision != r.precision)
            st = plan_reconfigure(sl.plan, r.L, r.beta, r.r_c, r.k_max, r.precision);
        else
            st = EWALD_OK;
    }
    if (st != EWALD_OK) return st;
    cudaError_t e;
    if (pd.ready && (e = cudaStreamWaitEvent(sl.stream, pd.ready, 0)) != cudaSuccess) return cuda_st(e);
    st = ewald_compute_async(sl.plan, r.n, r.pos, r.q, r.forces, sl.energy_d, EWALD_PART_ALL,
                             sl.stream);
    if (st != EWALD_OK) return st;
    if ((e = cudaMemcpyAsync(sl.energy_h, sl.energy_d, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                             sl.stream)) != cudaSuccess)
        return cuda_st(e);
    if ((e = cudaMemcpyAsync(sl.status_h, sl.plan->p.d_status, sizeof(int), cudaMemcpyDeviceToHost,
                             sl.stream)) != cudaSuccess)
        return cuda_st(e);
    if ((e = cudaEventRecord(sl.done, sl.stream)) != cudaSuccess) return cuda_st(e);
    return EWALD_OK;
}

int bits_to_status(int bits)
{
    if (bits & kStNonFinite) return EWALD_E_NONFINITE;
    if (bits & kStTimeout) return EWALD_E_TIMEOUT;
    if (bits & kStNonNeutral) return EWALD_E_NONNEUTRAL;
    return EWALD_OK;
}

void finish(ewald_server *s, Slot &sl, int status)
{
    ewald_result res;
    res.status = status;
    for (int i = 0; i < 4; ++i) res.energy[i] = status == EWALD_OK ? sl.energy_h[i] : 0.0;
    res.t_submit = sl.t_submit;
    res.t_admit = sl.t_admit;
    res.t_done = now_s(s->t0);
    res.footprint_bytes = (int64_t)sl.footprint;
    s->results[sl.ticket] = res;
    s->state[sl.ticket] = 2;
    sl.busy = false;
    s->completed++;
}

// Launcher thread of slot idx: launches every request the scheduler hands to the slot.
void launcher(ewald_server *s, int idx)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        Slot &sl = s->slots[idx];
        s->wcv.wait(lk, [&] { return sl.has_work || s->quit_launchers; });
        if (!sl.has_work) break;
        const Pending pd = sl.work;
        sl.has_work = false;
        lk.unlock();
        const int st = launch(s, sl, pd);
        if (pd.ready) cudaEventDestroy(pd.ready);
        lk.lock();
        sl.launch_status = st;
        sl.launched = true;
        s->cv.notify_one();
    }
}

void scheduler(ewald_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        int running = 0;
        // retire finished requests
        for (Slot &sl : s->slots) {
            if (!sl.busy) continue;
            if (!sl.launched) { ++running; continue; }
            if (sl.launch_status != EWALD_OK) {
                finish(s, sl, sl.launch_status);
                progress = true;
                continue;
            }
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) { ++running; continue; }
            finish(s, sl, q == cudaSuccess ? bits_to_status(*sl.status_h) : EWALD_E_CUDA);
            progress = true;
        }
        if (s->stop && running == 0) break;
        // admit: first fit over the queue, in arrival order.  A request that does not fit
        // first reclaims the workspaces of idle slots; once the head of the queue has been
        // passed over kMaxBypass times, nothing behind it is admitted before it.
        if (!s->stop) {
            std::vector<AdmitSlot> view(s->slots.size());
            std::vector<int> reclaim;
            for (auto it = s->queue.begin(); it != s->queue.end();) {
                for (size_t i = 0; i < s->slots.size(); ++i)
                    view[i] = AdmitSlot{s->slots[i].busy, (int64_t)s->slots[i].held};
                const bool is_head = it == s->queue.begin();
                int si = -1;
                const int act = admit_step((int64_t)it->footprint, is_head, view, s->held_total,
                                           (int64_t)s->budget, s->head_bypass, kMaxBypass, &si,
                                           &reclaim);
                for (int r : reclaim) {
                    Slot &sl = s->slots[r];
                    lk.unlock();
                    if (sl.plan) { ewald_destroy(sl.plan); sl.plan = nullptr; }
                    lk.lock();
                    s->held_total -= (int64_t)sl.held;
                    sl.held = 0;
                }
                if (act == kAdmitStop) break;
                if (act == kAdmitSkip) {   // does not fit now: try the next one
                    ++it;
                    continue;
                }
                if (is_head) s->head_bypass = 0;
                else ++s->head_bypass;
                Pending pd = *it;
                it = s->queue.erase(it);
                Slot &sl = s->slots[si];
                sl.busy = true;
                sl.ticket = pd.ticket;
                sl.t_submit = pd.t_submit;
                sl.footprint = pd.footprint;
                s->held_total += (int64_t)pd.footprint - (int64_t)sl.held;
                sl.held = pd.footprint;
                if (s->held_total > s->peak_held) s->peak_held = s->held_total;
                s->state[pd.ticket] = 1;
                ++running;
                if (running > s->peak_running) s->peak_running = running;
                sl.t_admit = now_s(s->t0);
                sl.work = pd;
                sl.has_work = true;
                sl.launched = false;
                s->wcv.notify_all();
                progress = true;
                // (the reclaims above unlock the mutex: restart from the queue's head)
                it = s->queue.begin();
            }
        }
        if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
    // cancel whatever is still queued
    for (Pending &pd : s->queue) {
        if (pd.ready) cudaEventDestroy(pd.ready);
        s->state.erase(pd.ticket);
    }
    s->queue.clear();
}

}  // namespace

extern "C" int ewald_server_create(int max_slots, size_t hbm_budget_bytes, ewald_server_t *out)
{
    if (!out || max_slots < 1 || max_slots > 64) return EWALD_E_INVAL;
    *out = nullptr;
    ewald_server *s = new (std::nothrow) ewald_server();
    if (!s) return EWALD_E_NOMEM;
    cudaGetDevice(&s->device);
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return EWALD_E_CUDA; }
        hbm_budget_bytes = (size_t)(0.8 * (double)fr);
    }
    s->budget = hbm_budget_bytes;
    s->slots.resize(max_slots);
    for (Slot &sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc((void **)&sl.energy_d, 4 * sizeof(double));
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sl.energy_h, 4 * sizeof(double), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sl.status_h, sizeof(int), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            *out = s;
            ewald_server_destroy(s);
            *out = nullptr;
            return cuda_st(e);
        }
    }
    for (int i = 0; i < max_slots; ++i) s->launchers.emplace_back(launcher, s, i);
    s->th = std::thread(scheduler, s);
    *out = s;
    return EWALD_OK;
}

extern "C" int ewald_submit(ewald_server_t s, const ewald_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return EWALD_E_INVAL;
    if (req->n < 1 || !req->pos || !req->q || !req->forces) return EWALD_E_INVAL;
    Plan probe;
    int st = plan_setup_host(probe, req->L, req->beta, req->r_c, req->k_max, req->precision);
    if (st != EWALD_OK) return st;
    const size_t fp = request_footprint(*req);
    if (fp > s->budget) return EWALD_E_INVAL;
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return EWALD_E_CUDA;
    if (cudaEventRecord(ready, (cudaStream_t)req->stream) != cudaSuccess) {
        cudaEventDestroy(ready);
        return EWALD_E_CUDA;
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) { cudaEventDestroy(ready); return EWALD_E_INVAL; }
    if (s->queue.size() >= s->max_queue) { cudaEventDestroy(ready); return EWALD_E_BUSY; }
    Pending pd;
    pd.ticket = s->next_ticket++;
    pd.req = *req;
    pd.t_submit = now_s(s->t0);
    pd.footprint = fp;
    pd.ready = ready;
    s->queue.push_back(pd);
    s->state[pd.ticket] = 0;
    s->submitted++;
    *ticket = pd.ticket;
    s->cv.notify_one();
    return EWALD_OK;
}

extern "C" int ewald_poll(ewald_server_t s, uint64_t ticket, ewald_result *out)
{
    if (!s || !out) return EWALD_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto st = s->state.find(ticket);
    if (st == s->state.end()) return EWALD_E_NOTFOUND;
    if (st->second != 2) return EWALD_PENDING;
    *out = s->results[ticket];
    s->results.erase(ticket);
    s->state.erase(st);
    return EWALD_OK;
}

extern "C" int ewald_wait(ewald_server_t s, uint64_t ticket, double timeout_s, ewald_result *out)
{
    if (!s || !out || !(timeout_s >= 0)) return EWALD_E_INVAL;
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (true) {
        int r = ewald_poll(s, ticket, out);
        if (r != EWALD_PENDING) return r;
        if (std::chrono::steady_clock::now() >= t_end) return EWALD_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" int ewald_server_stats(ewald_server_t s, int64_t stats[5])
{
    if (!s || !stats) return EWALD_E_INVAL;
    std::lock_guard<std::mutex> g(s->mu);
    stats[0] = s->submitted;
    stats[1] = s->completed;
    stats[2] = s->held_total;
    stats[3] = s->peak_held;
    stats[4] = s->peak_running;
    return EWALD_OK;
}

extern "C" int ewald_server_destroy(ewald_server_t s)
{
    if (!s) return EWALD_E_INVAL;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_one();
    }
    if (s->th.joinable()) s->th.join();
    {
        // (the scheduler has exited with no request running or waiting for its launch)
        std::lock_guard<std::mutex> g(s->mu);
        s->quit_launchers = true;
        s->wcv.notify_all();
    }
    for (std::thread &t : s->launchers)
        if (t.joinable()) t.join();
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.plan) ewald_destroy(sl.plan);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFree(sl.energy_d);
        if (sl.energy_h) cudaFreeHost(sl.energy_h);
        if (sl.status_h) cudaFreeHost(sl.status_h);
    }
    delete s;
    return EWALD_OK;
}

// Host-only replay of the admission policy with a simulated executor (no device work): the
// requests arrive at t_arrive (in index order at equal times), each runs for its duration
// once admitted, a finished slot keeps its memory until reclaimed, and after every event the
// scheduler's admission pass runs (first fit in arrival order, restarted from the head after
// every admission) with the same admit_step.  Writes the admission order (request indices)
// and times, and the peak of the held total.
extern "C" int ewald_server_simulate(int max_slots, int64_t budget, int n,
                                     const int64_t *footprint, const double *t_arrive,
                                     const double *duration, int64_t *order, double *t_admit,
                                     int64_t *peak_held)
{
    if (max_slots < 1 || max_slots > 64 || budget < 0 || n < 0 || (n > 0 && (!footprint ||
        !t_arrive || !duration || !order || !t_admit)) || !peak_held)
        return EWALD_E_INVAL;
    for (int i = 0; i < n; ++i)
        if (footprint[i] < 0 || footprint[i] > budget || !(duration[i] >= 0) ||
            !(t_arrive[i] >= 0) || (i > 0 && t_arrive[i] < t_arrive[i - 1]))
            return EWALD_E_INVAL;
    std::vector<AdmitSlot> slots(max_slots, AdmitSlot{false, 0});
    std::vector<double> ends(max_slots, 0.0);
    std::deque<int> queue;
    std::vector<int> reclaim;
    int64_t held = 0, peak = 0;
    int bypass = 0, next = 0, admitted = 0;
    double t = 0.0;
    while (admitted < n) {
        // next event: an arrival or the end of a running request
        double tn = next < n ? t_arrive[next] : 1e300;
        for (int i = 0; i < max_slots; ++i)
            if (slots[i].busy && ends[i] < tn) tn = ends[i];
        if (tn >= 1e300) return EWALD_E_INVAL;   // nothing can ever be admitted
        t = tn;
        for (int i = 0; i < max_slots; ++i)
            if (slots[i].busy && ends[i] <= t) slots[i].busy = false;
        while (next < n && t_arrive[next] <= t) queue.push_back(next++);
        for (size_t k = 0; k < queue.size();) {
            int si = -1;
            const int act = admit_step(footprint[queue[k]], k == 0, slots, held, budget, bypass,
                                       kMaxBypass, &si, &reclaim);
            for (int r : reclaim) {
                held -= slots[r].held;
                slots[r].held = 0;
            }
            if (act == kAdmitStop) break;
            if (act == kAdmitSkip) { ++k; continue; }
            bypass = k == 0 ? 0 : bypass + 1;
            const int i = queue[k];
            queue.erase(queue.begin() + k);
            held += footprint[i] - slots[si].held;
            slots[si].held = footprint[i];
            slots[si].busy = true;
            ends[si] = t + duration[i];
            if (held > peak) peak = held;
            order[admitted] = i;
            t_admit[i] = t;
            ++admitted;
            k = 0;
        }
    }
    *peak_held = peak;
    return EWALD_OK;
}
