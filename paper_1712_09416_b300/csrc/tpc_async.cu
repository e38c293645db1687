// Asynchronous long-running side tasks for the event loop (Sect. 3, item 4;
// Sect. 5.1), and one built-in accumulate-then-fit task.
//
// A tpc_async object owns one host thread.  The event loop hands it a job
// when processing an event (tpc_async_start, which never waits), checks at
// every event whether a job has finished (tpc_async_poll with timeout 0) and
// uses the result as soon as it has; events keep flowing while the job runs,
// so the event queue does not fill up behind it (Sect. 3, Fig. 4 against
// Sect. 5.1, Fig. 5).  The thread runs an optional initialisation callback
// once before any job, and passes caller pointers both ways (job in, result
// out).
//
// The built-in task (tpc_chi2_calib) accumulates the chi^2 and ndf of every
// track of every event and, every n-th event, fits the scale s^2 by which the
// tracker's cluster error underestimates the observed scatter (the ratio of
// the tracks' summed chi^2 to their summed ndf, with tracks above trim times
// the current scale removed until the kept set is stable).  It stands in for
// the calibration fits of Sect. 3 without their physics.  Its result is fed
// back event-synchronously (Sect. 5.2, 5.3) through tpc_track_set_params.
//
// Host code only: no device work, no CUDA calls.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/tpctrack.h"

struct tpc_async {
    tpc_async_init_fn init = nullptr;
    tpc_async_run_fn run = nullptr;
    tpc_async_drop_fn drop = nullptr;
    void* user = nullptr;
    int max_unfinished = 1;
    struct Job {
        uint64_t id;
        void* job;
    };
    struct Done {
        uint64_t id;
        void* result;
        int status;
    };
    std::mutex mu;
    std::condition_variable cv_job, cv_done;
    std::deque<Job> queue;   // started, not yet running
    std::deque<Done> done;   // finished, not yet polled (start order)
    bool running = false;
    bool stop = false;
    uint64_t next_id = 1;
    bool init_done = false;
    int init_status = TPC_OK;
    tpc_async_stats stats{};
    std::thread th;
};

namespace {

void async_main(tpc_async* a)
{
    const int st = a->init ? a->init(a->user) : TPC_OK;
    {
        std::lock_guard<std::mutex> lk(a->mu);
        a->init_status = st;
        a->init_done = true;
    }
    a->cv_done.notify_all();
    if (st != TPC_OK) return;
    for (;;) {
        tpc_async::Job j;
        {
            std::unique_lock<std::mutex> lk(a->mu);
            a->cv_job.wait(lk, [&] { return a->stop || !a->queue.empty(); });
            if (a->stop) return;  // queued jobs are dropped by tpc_async_destroy
            j = a->queue.front();
            a->queue.pop_front();
            a->running = true;
        }
        const auto t0 = std::chrono::steady_clock::now();
        void* result = nullptr;
        const int rc = a->run(a->user, j.job, &result);
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(a->mu);
            a->running = false;
            a->done.push_back({j.id, result, rc});
            a->stats.finished += 1;
            a->stats.busy_ms += ms;
            a->stats.max_task_ms = std::max(a->stats.max_task_ms, ms);
        }
        a->cv_done.notify_all();
    }
}

// ---------------------------------------------------------------------------
// built-in task: chi^2 / ndf scale of the tracks of a run of events
// ---------------------------------------------------------------------------
struct Chi2Job {
    std::vector<double> chi2, ndf;  // tracks with ndf > 0
    uint64_t first_event = 0, last_event = 0, n_events = 0;
    uint64_t params_version = 0;
};

int chi2_fit(void* user, void* job, void** result)
{
    const double trim = *(const double*)user;
    std::unique_ptr<Chi2Job> J((Chi2Job*)job);
    auto* F = new tpc_chi2_fit{};
    F->first_event = J->first_event;
    F->last_event = J->last_event;
    F->n_events = J->n_events;
    F->params_version = J->params_version;
    F->n_tracks = (int64_t)J->chi2.size();
    *result = F;
    const size_t n = J->chi2.size();
    if (n == 0) {
        F->scale2 = NAN;
        return TPC_OK;
    }
    // start from all tracks, then keep those with chi2 <= trim * ndf * s2
    // until the kept set repeats
    double sc = 0.0, sn = 0.0;
    for (size_t i = 0; i < n; ++i) {
        sc += J->chi2[i];
        sn += J->ndf[i];
    }
    double s2 = sc / sn;
    int64_t kept = (int64_t)n;
    std::vector<unsigned char> keep(n, 1), next(n);
    int it = 0;
    for (; it < 100; ++it) {
        sc = sn = 0.0;
        int64_t k = 0;
        const double cut = trim * s2;
        for (size_t i = 0; i < n; ++i) {
            next[i] = J->chi2[i] <= cut * J->ndf[i];
            if (next[i]) {
                sc += J->chi2[i];
                sn += J->ndf[i];
                ++k;
            }
        }
        if (k == 0) break;  // nothing below the cut: keep the last estimate
        const bool same = next == keep;
        keep.swap(next);
        kept = k;
        s2 = sc / sn;
        if (same) break;
    }
    F->scale2 = s2;
    F->n_kept = kept;
    F->n_iter = it < 100 ? it + 1 : 100;
    return TPC_OK;
}

void chi2_drop(void*, void* job, void* result)
{
    delete (Chi2Job*)job;
    delete (tpc_chi2_fit*)result;
}

}  // namespace

struct tpc_chi2_calib {
    double trim = 3.0;
    int every_n = 1;
    tpc_async* task = nullptr;
    std::unique_ptr<Chi2Job> acc;  // events accumulated since the last start
    uint64_t n_added = 0;
    std::mutex mu;
};

extern "C" {

int tpc_async_create(tpc_async_init_fn init, tpc_async_run_fn run, tpc_async_drop_fn drop,
                     void* user, int max_unfinished, tpc_async** out)
{
    if (!out) return TPC_EINVAL;
    *out = nullptr;
    if (!run || max_unfinished < 1 || max_unfinished > 1024) return TPC_EINVAL;
    auto a = std::make_unique<tpc_async>();
    a->init = init;
    a->run = run;
    a->drop = drop;
    a->user = user;
    a->max_unfinished = max_unfinished;
    try {
        a->th = std::thread(async_main, a.get());
    } catch (...) {
        return TPC_ENOMEM;
    }
    int st;
    {
        std::unique_lock<std::mutex> lk(a->mu);
        a->cv_done.wait(lk, [&] { return a->init_done; });
        st = a->init_status;
    }
    if (st != TPC_OK) {
        a->th.join();
        return st;
    }
    *out = a.release();
    return TPC_OK;
}

int tpc_async_start(tpc_async* a, void* job, uint64_t* task)
{
    if (!a) return TPC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(a->mu);
        const int unfinished = (int)a->queue.size() + (a->running ? 1 : 0);
        if (unfinished >= a->max_unfinished) {
            a->stats.refused += 1;
            return TPC_EBUSY;
        }
        const uint64_t id = a->next_id++;
        a->queue.push_back({id, job});
        a->stats.started += 1;
        if (task) *task = id;
    }
    a->cv_job.notify_one();
    return TPC_OK;
}

int tpc_async_poll(tpc_async* a, int timeout_us, uint64_t* task, void** result, int* task_status)
{
    if (!a) return TPC_EINVAL;
    std::unique_lock<std::mutex> lk(a->mu);
    auto ready = [&] { return !a->done.empty(); };
    if (timeout_us < 0) {
        // waiting forever on an idle runner would never end: wait only while
        // something is queued or running
        a->cv_done.wait(lk, [&] { return ready() || (a->queue.empty() && !a->running); });
    } else if (timeout_us > 0) {
        a->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    if (!ready()) return TPC_EBUSY;
    const tpc_async::Done d = a->done.front();
    a->done.pop_front();
    if (task) *task = d.id;
    if (result) *result = d.result;
    if (task_status) *task_status = d.status;
    return TPC_OK;
}

int tpc_async_get_stats(tpc_async* a, tpc_async_stats* out)
{
    if (!a || !out) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(a->mu);
    *out = a->stats;
    out->queued = (int64_t)a->queue.size();
    out->running = a->running ? 1 : 0;
    out->unpolled = (int64_t)a->done.size();
    return TPC_OK;
}

void tpc_async_destroy(tpc_async* a)
{
    if (!a) return;
    {
        std::lock_guard<std::mutex> lk(a->mu);
        a->stop = true;
    }
    a->cv_job.notify_all();
    if (a->th.joinable()) a->th.join();  // the running job, if any, completes
    if (a->drop) {
        for (auto& j : a->queue) a->drop(a->user, j.job, nullptr);
        for (auto& d : a->done) a->drop(a->user, nullptr, d.result);
    }
    delete a;
}

// ---------------------------------------------------------------------------

int tpc_chi2_calib_create(int every_n_events, double trim, int max_unfinished, tpc_chi2_calib** out)
{
    if (!out) return TPC_EINVAL;
    *out = nullptr;
    if (every_n_events < 1 || !(trim > 1.0) || !std::isfinite(trim)) return TPC_EINVAL;
    auto c = std::make_unique<tpc_chi2_calib>();
    c->trim = trim;
    c->every_n = every_n_events;
    const int rc = tpc_async_create(nullptr, chi2_fit, chi2_drop, &c->trim, max_unfinished, &c->task);
    if (rc != TPC_OK) return rc;
    *out = c.release();
    return TPC_OK;
}

int tpc_chi2_calib_add(tpc_chi2_calib* c, const tpc_tracks* t, uint64_t params_version)
{
    if (!c || !t || t->n_tracks < 0 || (t->n_tracks > 0 && (!t->chi2 || !t->ndf)))
        return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    const uint64_t ev = c->n_added++;
    if (c->acc && c->acc->params_version != params_version) c->acc.reset();  // one parameter set per fit
    if (!c->acc) {
        c->acc = std::make_unique<Chi2Job>();
        c->acc->first_event = ev;
        c->acc->params_version = params_version;
    }
    Chi2Job& J = *c->acc;
    for (int64_t i = 0; i < t->n_tracks; ++i) {
        if (t->ndf[i] <= 0) continue;
        J.chi2.push_back((double)t->chi2[i]);
        J.ndf.push_back((double)t->ndf[i]);
    }
    J.last_event = ev;
    J.n_events += 1;
    if ((int64_t)J.n_events < c->every_n) return TPC_OK;
    Chi2Job* job = c->acc.release();
    const int rc = tpc_async_start(c->task, job, nullptr);
    if (rc == TPC_EBUSY) {  // the side thread is still busy: keep accumulating
        c->acc.reset(job);
        return TPC_OK;
    }
    if (rc != TPC_OK) {
        delete job;
        return rc;
    }
    return TPC_OK;
}

int tpc_chi2_calib_poll(tpc_chi2_calib* c, int timeout_us, tpc_chi2_fit* out)
{
    if (!c) return TPC_EINVAL;
    void* r = nullptr;
    int st = TPC_OK;
    const int rc = tpc_async_poll(c->task, timeout_us, nullptr, &r, &st);
    if (rc != TPC_OK) return rc;
    std::unique_ptr<tpc_chi2_fit> F((tpc_chi2_fit*)r);
    if (out && F) *out = *F;
    return st;
}

int tpc_chi2_calib_stats(tpc_chi2_calib* c, tpc_async_stats* out)
{
    if (!c) return TPC_EINVAL;
    return tpc_async_get_stats(c->task, out);
}

void tpc_chi2_calib_destroy(tpc_chi2_calib* c)
{
    if (!c) return;
    tpc_async_destroy(c->task);
    delete c;
}

}  // extern "C"
