// tpc_dispatch.cu -- round-robin dispatcher of whole events over tracker
// instances (host code only).
//
// The paper balances load by running several instances of a component and
// handing them events in turn (Sect. 2: round robin over the instances of a
// component; each instance processes one event after another).  Here an
// instance is a tracker context on one GPU (or any object with the submit /
// poll / release calls of tpc_instance_ops): tpc_dispatch_submit gives each
// event to the next healthy instance, the caller polls its tickets in any
// order and gets every event's tracks, whichever instance ran it.  Events are
// independent (no exchange step), so nothing is communicated between the
// instances.  An instance whose calls fail with a device or timeout error
// (TPC_ECUDA, TPC_ETIMEOUT, TPC_ENOMEM) is taken out of the rotation and the
// events it still holds are submitted again to the others; an event's own
// invalid clusters (TPC_EINVAL) fail its ticket only.
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/tpctrack.h"

namespace {

struct Pending {
    tpc_clusters ev;       // the caller's inputs, kept until the ticket is released
    tpc_geometry geom;
    float bz = 0.0f;
    int inst = -1;         // instance that holds the event
    uint64_t inner = 0;    // that instance's ticket
    bool polled = false;   // results handed out (released by tpc_dispatch_release)
};

bool instance_failure(int rc)
{
    return rc == TPC_ECUDA || rc == TPC_ETIMEOUT || rc == TPC_ENOMEM;
}

}  // namespace

struct tpc_dispatch {
    tpc_instance_ops ops;
    std::vector<void*> inst;
    std::vector<bool> healthy;
    std::vector<tpc_track_ctx*> owned;   // contexts created by tpc_dispatch_create
    std::vector<int64_t> n_events;       // events submitted to each instance
    std::map<uint64_t, Pending> tickets;
    uint64_t next_ticket = 1;
    int next_inst = 0;
    int64_t reissued = 0;
    std::mutex mu;
};

namespace {

int ctx_submit(void* inst, const tpc_clusters* ev, const tpc_geometry* g, float bz,
               uint64_t* ticket)
{
    return tpc_track_submit((tpc_track_ctx*)inst, ev, g, bz, ticket);
}
int ctx_poll(void* inst, uint64_t ticket, int timeout_us, tpc_tracks* out)
{
    return tpc_track_poll((tpc_track_ctx*)inst, ticket, timeout_us, out);
}
int ctx_release(void* inst, uint64_t ticket)
{
    return tpc_track_release((tpc_track_ctx*)inst, ticket);
}

// Submit p to the healthy instances in turn, starting at the round-robin
// position; an instance that fails with a device error leaves the rotation.
// Caller holds d->mu.
int place(tpc_dispatch* d, Pending& p)
{
    const int n = (int)d->inst.size();
    for (int tries = 0; tries < n; ++tries) {
        const int k = d->next_inst;
        d->next_inst = (d->next_inst + 1) % n;
        if (!d->healthy[k]) continue;
        uint64_t inner = 0;
        const int rc = d->ops.submit(d->inst[k], &p.ev, &p.geom, p.bz, &inner);
        if (rc == TPC_OK) {
            p.inst = k;
            p.inner = inner;
            ++d->n_events[k];
            return TPC_OK;
        }
        if (!instance_failure(rc)) return rc;  // the event itself is at fault
        d->healthy[k] = false;
    }
    return TPC_ECUDA;  // no healthy instance left
}

// Take instance k out of the rotation and hand its events to the others.
// Caller holds d->mu.
int fail_instance(tpc_dispatch* d, int k)
{
    d->healthy[k] = false;
    int rc_all = TPC_OK;
    for (auto& kv : d->tickets) {
        Pending& p = kv.second;
        if (p.inst != k || p.polled) continue;
        d->ops.release(d->inst[k], p.inner);  // best effort on a failed instance
        p.inst = -1;
        const int rc = place(d, p);
        if (rc == TPC_OK) ++d->reissued;
        else rc_all = rc;
    }
    return rc_all;
}

}  // namespace

extern "C" {

int tpc_dispatch_create_custom(const tpc_instance_ops* ops, void* const* instances, int n,
                               tpc_dispatch** out)
{
    if (!ops || !ops->submit || !ops->poll || !ops->release || !instances || n < 1 || n > 1024 ||
        !out)
        return TPC_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!instances[k]) return TPC_EINVAL;
    auto d = std::make_unique<tpc_dispatch>();
    d->ops = *ops;
    d->inst.assign(instances, instances + n);
    d->healthy.assign(n, true);
    d->n_events.assign(n, 0);
    *out = d.release();
    return TPC_OK;
}

int tpc_dispatch_create(const int* devices, int n_dev, const tpc_track_config* cfg,
                        tpc_dispatch** out)
{
    if (!devices || n_dev < 1 || n_dev > 1024 || !cfg || !out) return TPC_EINVAL;
    std::vector<tpc_track_ctx*> ctxs;
    for (int k = 0; k < n_dev; ++k) {
        tpc_track_config c = *cfg;
        c.device = devices[k];
        c.cuda_stream = nullptr;  // every instance works on streams of its own
        tpc_track_ctx* ctx = nullptr;
        const int rc = tpc_track_create(&c, &ctx);
        if (rc != TPC_OK) {
            for (auto* x : ctxs) tpc_track_destroy(x);
            return rc;
        }
        ctxs.push_back(ctx);
    }
    static const tpc_instance_ops kCtxOps = {ctx_submit, ctx_poll, ctx_release};
    std::vector<void*> inst(ctxs.begin(), ctxs.end());
    const int rc = tpc_dispatch_create_custom(&kCtxOps, inst.data(), n_dev, out);
    if (rc != TPC_OK) {
        for (auto* x : ctxs) tpc_track_destroy(x);
        return rc;
    }
    (*out)->owned = ctxs;
    return TPC_OK;
}

int tpc_dispatch_submit(tpc_dispatch* d, const tpc_clusters* ev, const tpc_geometry* geom,
                        float bz_tesla, uint64_t* ticket)
{
    if (!d || !ev || !geom || !ticket) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(d->mu);
    Pending p;
    p.ev = *ev;
    p.geom = *geom;
    p.bz = bz_tesla;
    const int rc = place(d, p);
    if (rc != TPC_OK) return rc;
    *ticket = d->next_ticket++;
    d->tickets.emplace(*ticket, p);
    return TPC_OK;
}

int tpc_dispatch_poll(tpc_dispatch* d, uint64_t ticket, int timeout_us, tpc_tracks* out)
{
    if (!d || !out) return TPC_EINVAL;
    std::unique_lock<std::mutex> lk(d->mu);
    for (int round = 0; round <= (int)d->inst.size(); ++round) {
        auto it = d->tickets.find(ticket);
        if (it == d->tickets.end()) return TPC_EINVAL;
        Pending& p = it->second;
        if (p.inst < 0) return TPC_ECUDA;  // no healthy instance could take it
        const int k = p.inst;
        const uint64_t inner = p.inner;
        void* inst = d->inst[k];
        lk.unlock();  // the wait for the device runs without the lock
        const int rc = d->ops.poll(inst, inner, timeout_us, out);
        lk.lock();
        it = d->tickets.find(ticket);
        if (it == d->tickets.end()) return TPC_EINVAL;  // released meanwhile
        if (rc == TPC_OK) {
            it->second.polled = true;
            return TPC_OK;
        }
        if (!instance_failure(rc)) return rc;  // TPC_EBUSY, or the event's own error
        if (it->second.inst == k) fail_instance(d, k);  // (else already moved)
    }
    return TPC_ECUDA;
}

int tpc_dispatch_release(tpc_dispatch* d, uint64_t ticket)
{
    if (!d) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(d->mu);
    auto it = d->tickets.find(ticket);
    if (it == d->tickets.end()) return TPC_EINVAL;
    if (it->second.inst >= 0) d->ops.release(d->inst[it->second.inst], it->second.inner);
    d->tickets.erase(it);
    return TPC_OK;
}

int tpc_dispatch_fail_instance(tpc_dispatch* d, int instance)
{
    if (!d) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(d->mu);
    if (instance < 0 || instance >= (int)d->inst.size()) return TPC_EINVAL;
    if (!d->healthy[instance]) return TPC_OK;
    return fail_instance(d, instance);
}

int tpc_dispatch_stats(tpc_dispatch* d, int cap, int64_t* events_per_instance,
                       int32_t* healthy, int64_t* reissued)
{
    if (!d) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(d->mu);
    const int n = (int)d->inst.size();
    for (int k = 0; k < n && k < cap; ++k) {
        if (events_per_instance) events_per_instance[k] = d->n_events[k];
        if (healthy) healthy[k] = d->healthy[k] ? 1 : 0;
    }
    if (reissued) *reissued = d->reissued;
    return n;
}

void tpc_dispatch_destroy(tpc_dispatch* d)
{
    if (!d) return;
    {
        std::lock_guard<std::mutex> lk(d->mu);
        for (auto& kv : d->tickets)
            if (kv.second.inst >= 0) d->ops.release(d->inst[kv.second.inst], kv.second.inner);
        d->tickets.clear();
    }
    for (auto* x : d->owned) tpc_track_destroy(x);
    delete d;
}

}  // extern "C"
