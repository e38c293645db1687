// tpctrack.cu -- host side of libtpctrack.so: contexts, device arenas, launch
// orchestration, result collection, debug dumps and the served form.
//
// Memory: every slot owns one device arena sized at creation for
// max_clusters_per_event clusters, max_events_per_launch events and
// max_rows rows; no allocation happens while tracking.  Slot 0 serves the
// direct calls (tpc_track_event/batch/launch); with tpc_track_submit, one
// worker thread per slot pulls every queued event that fits its arena into
// its next launch (continuous batching), so launches of different slots run
// concurrently on the device while the next requests queue up.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tpctrack.h"
#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr double kKappa = 0.299792458e-2;  // cm^-1 per (GeV/c)^-1 per tesla
constexpr int kMaxEventsPerLaunch = 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Capacities of one arena.
struct Caps {
    long long n;   // clusters
    int e;         // events
    int s;         // sectors
    int r;         // rows per sector
    long long rs;  // s * r
    long long bins;
    int t;         // tracklet slots
    long long row_tiles, hit_tiles;
};

struct HostOut {  // pinned host copies of one launch's results
    int32_t* sector = nullptr;
    float* x = nullptr;
    float* param = nullptr;
    float* cov = nullptr;
    float* chi2 = nullptr;
    int32_t* ndf = nullptr;
    int32_t* hit_off = nullptr;
    int32_t* hit_cid = nullptr;
    int32_t* sec_trk_off = nullptr;
    int32_t* sec_hit_off = nullptr;
    int32_t* ev_hit_off = nullptr;  // per-event rebased hit offsets, concatenated
};

struct LaunchInfo {
    int n_ev = 0;
    std::vector<long long> ev_n;     // clusters per event
    std::vector<int> ev_sec_base, ev_n_sec;
    int S = 0, R = 0;
    Launch L;
    bool pending = false;
    bool done = false;
    tpc_track_counters counters{};
};

struct Slot {
    int id = 0;
    Caps caps{};
    char* dev = nullptr;
    size_t dev_bytes = 0;
    // fixed device buffers
    float *in_y, *in_z;
    uint16_t *in_row, *in_sec;
    void* desc_dev;      // EventDesc[e] | ev_off[e+1] | sec_event[s]
    char* zero_dev;      // counters | row_cnt | sec_first | sec_end | tile_state
    size_t zero_cap = 0;
    int *row_off, *big_rows;
    RowGrid* grid;
    float4* tmp_rec;
    int* rank;
    float2* hyz;
    int *hcid, *hrow, *bin_start;
    int16_t *up, *dn, *upc, *dnc;
    unsigned long long* weight;
    unsigned char* mark;
    int* crowded;
    int* starts;
    TrackletHdr* tl;
    int4* tl_chain;
    int* tl_rowhit;
    int* tl_list;
    int* upg;
    unsigned long long* tl_key;
    int *tl_nown, *tl_out, *tl_hitoff, *sec_trk_off, *sec_hit_off;
    unsigned* tl_own;
    int *k_sector, *k_ndf, *k_hit_off, *k_hit_cid, *k_gsec;
    float *k_x, *k_param, *k_cov, *k_chi2;
    // merger scratch and merged outputs
    MgState* mg_st;
    MgFit* mg_fit;
    unsigned long long* mg_key;
    int *mg_best, *mg_link, *mg_in, *mg_absorbed, *mg_oidx, *mg_ohoff;
    float4* mg_hxyz;
    float* mg_xs;
    int* mg_xi;
    float4* mg_pre;
    int *m_sector, *m_ndf, *m_hit_off, *m_hit_cid, *m_sec_trk_off, *m_sec_hit_off;
    float *m_x, *m_param, *m_cov, *m_chi2;
    // host side
    void* desc_ring[2] = {nullptr, nullptr};  // pinned mirrors of desc_dev, used in turn
    cudaEvent_t desc_done[2] = {nullptr, nullptr};
    bool desc_used[2] = {false, false};
    int desc_turn = 0;
    void* desc_host = nullptr;  // the mirror of the current launch
    size_t desc_bytes = 0;
    // profiling: one event after every kernel of every launch while enabled
    bool prof = false;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
    std::vector<std::pair<std::string, std::pair<size_t, size_t>>> prof_marks;  // name, (ev0, ev1)
    size_t prof_last = 0;
    Counters* cnt_host = nullptr;
    HostOut out;
    cudaStream_t stream = nullptr;  // the stream of the slot's current launch
    bool own_stream = false;
    // home: the slot's stream for served launches and single-stream direct
    // launches (the context's stream for slot 0); pipe: its stream for
    // direct launches spread over several slots (a stream of its own, also
    // for slot 0)
    cudaStream_t home = nullptr, pipe = nullptr;
    bool own_pipe = false;
    bool launched = false;  // done_ev has been recorded
    cudaEvent_t done_ev = nullptr;
    LaunchInfo info;
    std::vector<tpc_tracks> tracks;  // per event of the last results
    // the kernel sequence of the last launch shape, captured as a CUDA graph
    cudaGraphExec_t graph = nullptr;
    Launch graph_L{};
    Schedule graph_sched{};
};

struct Request {
    uint64_t ticket;
    tpc_clusters ev;
    std::vector<float> row_x;
    tpc_geometry geom;
    float bz;
    tpc_track_params prm;   // the parameter set current when the event was submitted
    uint64_t prm_version;
    std::chrono::steady_clock::time_point t_submit;
};

// A served ticket's tracks live in a pinned host buffer of the context's
// pool, written by device-to-host copies; the buffer goes back to the pool
// when the ticket is released.
struct PinnedBuf {
    char* p = nullptr;
    size_t cap = 0;
};

struct TicketResult {
    int status = TPC_EBUSY;
    tpc_track_params prm{};  // the parameter set the event is tracked with
    uint64_t prm_version = 0;
    PinnedBuf buf;
    tpc_tracks view{};
};

}  // namespace
}  // namespace tpc

struct tpc_track_ctx {
    tpc_track_config cfg;
    std::vector<std::unique_ptr<tpc::Slot>> slots;
    std::string err;
    mutable std::mutex err_mu;  // err is written by worker threads too
    // served form
    std::mutex mu;
    std::condition_variable cv_req, cv_done;
    std::deque<tpc::Request> queue;
    std::map<uint64_t, std::unique_ptr<tpc::TicketResult>> results;
    std::vector<std::thread> workers;
    std::mutex pool_mu;
    std::vector<tpc::PinnedBuf> pool;  // free pinned result buffers
    bool stop = false;
    uint64_t next_ticket = 1;
    uint64_t prm_version = 0;  // bumped by every tpc_track_set_params (cfg.params under mu)
    std::atomic<int> direct_busy{0};
    long long dbg_spin = 0;   // look-back poll limit of the next launches (0 = default)
    int dbg_stall = 0;        // 1 + hit tile that never publishes (test hook), 0 = none
    bool graphs = true;  // TPC_NO_GRAPH=1: launch the kernels one by one
    tpc::Schedule sched;
    // direct launches: spread over `streams` slots in turn; the launches not
    // yet collected, oldest first
    int streams = 1;
    int next_slot = 0;
    int last_slot = 0;  // slot of the last collected launch
    std::deque<int> direct;
    cudaEvent_t fork_ev = nullptr;
};

namespace tpc {
namespace {

int fail(tpc_track_ctx* ctx, int code, const std::string& msg)
{
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->err = msg;
    }
    return code;
}

#define CUDA_TRY(ctx, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((ctx), TPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

Caps make_caps(const tpc_track_config& c)
{
    Caps k;
    k.n = std::max<long long>(1, c.max_clusters_per_event);
    k.e = c.max_events_per_launch > 0 ? c.max_events_per_launch : 64;
    k.r = c.max_rows > 0 ? c.max_rows : 159;
    k.s = k.e * 36;
    k.rs = (long long)k.s * k.r;
    k.bins = k.n * kBinsPerHitX2 / 2 + 2 * k.rs + 16;
    k.t = (int)std::min<long long>(k.n / 8 + 4096, 0x7fffffffLL / 256);
    k.row_tiles = k.rs / kRowTile + 2;
    k.hit_tiles = k.n / kHitTile + 2;
    return k;
}

// Lay out (or, with base == nullptr, just size) the arena of a slot.
size_t layout(Slot& s, char* base)
{
    const Caps& k = s.caps;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = align_up(off, 256);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    s.in_y = (float*)take(4 * k.n);
    s.in_z = (float*)take(4 * k.n);
    s.in_row = (uint16_t*)take(2 * k.n);
    s.in_sec = (uint16_t*)take(2 * k.n);
    s.desc_bytes = sizeof(EventDesc) * k.e + sizeof(long long) * (k.e + 1) + sizeof(int) * k.s +
                   sizeof(float) * kMaxRows + 64;
    s.desc_dev = take(s.desc_bytes);
    s.zero_cap = align_up(sizeof(Counters), 256) + 4 * (k.rs * kCntPad + 2 * k.s + k.e) +
                 8 * (k.row_tiles + k.hit_tiles + k.s + ((long long)k.t + kMgTile - 1) / kMgTile) + 4096;
    s.zero_dev = take(s.zero_cap);
    s.row_off = (int*)take(4 * (k.rs + 1));
    s.big_rows = (int*)take(4 * k.rs);
    s.grid = (RowGrid*)take(sizeof(RowGrid) * k.rs);
    s.tmp_rec = (float4*)take(16 * k.n);
    s.rank = (int*)take(4 * k.n);
    s.hyz = (float2*)take(8 * k.n);
    s.hcid = (int*)take(4 * k.n);
    s.hrow = (int*)take(4 * k.n);
    s.bin_start = (int*)take(4 * k.bins);
    s.up = (int16_t*)take(2 * k.n);
    s.dn = (int16_t*)take(2 * k.n);
    s.upc = (int16_t*)take(2 * k.n);
    s.dnc = (int16_t*)take(2 * k.n);
    s.weight = (unsigned long long*)take(8 * k.n);
    s.mark = (unsigned char*)take(k.n);
    s.crowded = (int*)take(4 * k.n);
    s.starts = (int*)take(4 * (size_t)k.t);
    s.tl = (TrackletHdr*)take(sizeof(TrackletHdr) * (size_t)k.t);
    s.tl_chain = (int4*)take(16 * (size_t)k.t);
    s.tl_rowhit = (int*)take(4 * (size_t)k.t * k.r);
    s.tl_list = (int*)take(4 * (size_t)k.t);
    s.upg = (int*)take(4 * k.n);
    s.tl_key = (unsigned long long*)take(8 * (size_t)k.t);
    s.tl_nown = (int*)take(4 * (size_t)k.t);
    s.tl_own = (unsigned*)take(4 * (size_t)kOwnWords * k.t);
    s.tl_out = (int*)take(4 * (size_t)k.t);
    s.tl_hitoff = (int*)take(4 * (size_t)k.t);
    s.sec_trk_off = (int*)take(4 * (k.s + 1));
    s.sec_hit_off = (int*)take(4 * (k.s + 1));
    s.k_sector = (int*)take(4 * (size_t)k.t);
    s.k_ndf = (int*)take(4 * (size_t)k.t);
    s.k_hit_off = (int*)take(4 * ((size_t)k.t + 1));
    s.k_hit_cid = (int*)take(4 * k.n);
    s.k_x = (float*)take(4 * (size_t)k.t);
    s.k_param = (float*)take(20 * (size_t)k.t);
    s.k_cov = (float*)take(60 * (size_t)k.t);
    s.k_chi2 = (float*)take(4 * (size_t)k.t);
    s.k_gsec = (int*)take(4 * (size_t)k.t);
    s.mg_st = (MgState*)take(sizeof(MgState) * (size_t)k.t);
    s.mg_fit = (MgFit*)take(sizeof(MgFit) * (size_t)k.t);
    s.mg_key = (unsigned long long*)take(8 * (size_t)k.t);
    s.mg_best = (int*)take(4 * (size_t)k.t);
    s.mg_link = (int*)take(4 * (size_t)k.t);
    s.mg_in = (int*)take(4 * (size_t)k.t);
    s.mg_absorbed = (int*)take(4 * (size_t)k.t);
    s.mg_oidx = (int*)take(4 * (size_t)k.t);
    s.mg_ohoff = (int*)take(4 * (size_t)k.t);
    s.mg_hxyz = (float4*)take(16 * k.n);
    s.mg_xs = (float*)take(4 * (size_t)k.t);
    s.mg_xi = (int*)take(4 * (size_t)k.t);
    s.mg_pre = (float4*)take(32 * (size_t)k.t);
    s.m_sector = (int*)take(4 * (size_t)k.t);
    s.m_ndf = (int*)take(4 * (size_t)k.t);
    s.m_hit_off = (int*)take(4 * ((size_t)k.t + 1));
    s.m_hit_cid = (int*)take(4 * k.n);
    s.m_sec_trk_off = (int*)take(4 * (k.s + 1));
    s.m_sec_hit_off = (int*)take(4 * (k.s + 1));
    s.m_x = (float*)take(4 * (size_t)k.t);
    s.m_param = (float*)take(20 * (size_t)k.t);
    s.m_cov = (float*)take(60 * (size_t)k.t);
    s.m_chi2 = (float*)take(4 * (size_t)k.t);
    return align_up(off, 256);
}

int alloc_slot(tpc_track_ctx* ctx, Slot& s)
{
    s.dev_bytes = layout(s, nullptr);
    char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, s.dev_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TPC_ENOMEM, "cudaMalloc of a " + std::to_string(s.dev_bytes >> 20) +
                                         " MiB arena failed: " + cudaGetErrorString(e));
    }
    s.dev = base;
    layout(s, base);
    const Caps& k = s.caps;
    for (int i = 0; i < 2; ++i) {
        CUDA_TRY(ctx, cudaMallocHost(&s.desc_ring[i], s.desc_bytes));
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&s.desc_done[i], cudaEventDisableTiming));
    }
    s.desc_host = s.desc_ring[0];
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.cnt_host, sizeof(Counters)));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.sector, 4 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.x, 4 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.param, 20 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.cov, 60 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.chi2, 4 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.ndf, 4 * (size_t)k.t));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.hit_off, 4 * ((size_t)k.t + 1)));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.hit_cid, 4 * (size_t)k.n));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.sec_trk_off, 4 * ((size_t)k.s + 1)));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.sec_hit_off, 4 * ((size_t)k.s + 1)));
    CUDA_TRY(ctx, cudaMallocHost((void**)&s.out.ev_hit_off, 4 * ((size_t)k.t + k.e + 1)));
    CUDA_TRY(ctx, cudaEventCreateWithFlags(&s.done_ev, cudaEventDisableTiming));
    return TPC_OK;
}

void free_slot(Slot& s)
{
    if (s.home) cudaStreamSynchronize(s.home);
    if (s.dev) cudaFree(s.dev);
    for (int i = 0; i < 2; ++i) {
        if (s.desc_ring[i]) cudaFreeHost(s.desc_ring[i]);
        if (s.desc_done[i]) cudaEventDestroy(s.desc_done[i]);
    }
    for (cudaEvent_t e : s.prof_pool) cudaEventDestroy(e);
    if (s.cnt_host) cudaFreeHost(s.cnt_host);
    void* hp[] = {s.out.sector, s.out.x, s.out.param, s.out.cov, s.out.chi2, s.out.ndf,
                  s.out.hit_off, s.out.hit_cid, s.out.sec_trk_off, s.out.sec_hit_off,
                  s.out.ev_hit_off};
    for (void* p : hp)
        if (p) cudaFreeHost(p);
    if (s.done_ev) cudaEventDestroy(s.done_ev);
    if (s.graph) cudaGraphExecDestroy(s.graph);
    if (s.pipe) cudaStreamSynchronize(s.pipe);
    if (s.own_pipe && s.pipe) cudaStreamDestroy(s.pipe);
    if (s.own_stream && s.home) cudaStreamDestroy(s.home);
    s = Slot();
}

int check_geometry(tpc_track_ctx* ctx, const Slot& s, const tpc_geometry* g)
{
    if (!g || !g->row_x) return fail(ctx, TPC_EINVAL, "geometry or row_x is NULL");
    if (g->n_rows < 3 || g->n_rows > kMaxRows || g->n_rows > s.caps.r)
        return fail(ctx, TPC_EINVAL, "n_rows out of range (3.." + std::to_string(std::min(kMaxRows, s.caps.r)) + ")");
    for (int r = 0; r < g->n_rows; ++r) {
        if (!std::isfinite(g->row_x[r])) return fail(ctx, TPC_EINVAL, "row_x not finite");
        if (r > 0 && !(g->row_x[r] > g->row_x[r - 1]))
            return fail(ctx, TPC_EINVAL, "row_x not strictly ascending");
    }
    if (g->n_sectors_phi < 1 || g->n_sectors_phi > 36)
        return fail(ctx, TPC_EINVAL, "n_sectors_phi out of range (1..36)");
    if (!(g->half_angle_rad > 0.0f && g->half_angle_rad < 1.5f) || !(g->z_max > 0.0f))
        return fail(ctx, TPC_EINVAL, "half_angle_rad or z_max out of range");
    return TPC_OK;
}

// Record the next profiling event on the slot's stream; returns its index.
size_t prof_event(Slot& s)
{
    if (s.prof_used == s.prof_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        s.prof_pool.push_back(e);
    }
    cudaEventRecord(s.prof_pool[s.prof_used], s.stream);
    return s.prof_used++;
}

void launch_all(const Launch& L, const Schedule& S, cudaStream_t st, const KernelHook* hk)
{
    launch_binning(L, S, st, hk);
    launch_finder(L, S, st, hk);
    launch_constructor(L, S, st, hk);
    launch_selector(L, S, st, hk);
    if (L.merge) launch_merger(L, S, st, hk);
}

// The kernel sequence as one CUDA graph launch.  The graph of the slot is
// captured again only when the launch record or the schedule changed (a new
// event shape), and then updated in place when its topology allows.
int launch_graph(tpc_track_ctx* ctx, Slot& s, const Launch& L)
{
    const bool same = s.graph && std::memcmp(&s.graph_L, &L, sizeof(Launch)) == 0 &&
                      std::memcmp(&s.graph_sched, &ctx->sched, sizeof(Schedule)) == 0;
    if (!same) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();  // stream cannot be captured: launch directly
            launch_all(L, ctx->sched, s.stream, nullptr);
            return TPC_OK;
        }
        launch_all(L, ctx->sched, s.stream, nullptr);
        if (cudaStreamEndCapture(s.stream, &g) != cudaSuccess || !g) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return fail(ctx, TPC_ECUDA, "graph capture of the kernel sequence failed");
        }
        bool ok = false;
        if (s.graph) {
            cudaGraphExecUpdateResultInfo info;
            ok = cudaGraphExecUpdate(s.graph, g, &info) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                cudaGraphExecDestroy(s.graph);
                s.graph = nullptr;
            }
        }
        if (!ok && cudaGraphInstantiate(&s.graph, g, 0) != cudaSuccess) {
            cudaGetLastError();
            s.graph = nullptr;
            cudaGraphDestroy(g);
            return fail(ctx, TPC_ECUDA, "graph instantiation failed");
        }
        cudaGraphDestroy(g);
        s.graph_L = L;
        s.graph_sched = ctx->sched;
    }
    CUDA_TRY(ctx, cudaGraphLaunch(s.graph, s.stream));
    return TPC_OK;
}

// Enqueue the whole device pipeline of one launch on the slot's stream.
int enqueue(tpc_track_ctx* ctx, Slot& s, int n_ev, const tpc_clusters* ev, const tpc_geometry* g,
            float bz, const tpc_track_params& P)
{
    if (n_ev < 1 || n_ev > s.caps.e || n_ev > kMaxEventsPerLaunch)
        return fail(ctx, TPC_EINVAL, "n_ev out of range (1.." + std::to_string(s.caps.e) + ")");
    if (!ev) return fail(ctx, TPC_EINVAL, "events pointer is NULL");
    if (int rc = check_geometry(ctx, s, g)) return rc;
    if (!std::isfinite(bz)) return fail(ctx, TPC_EINVAL, "bz not finite");
    const int n_sec = g->n_sectors_phi * (g->split_z ? 2 : 1);
    long long n_total = 0;
    for (int i = 0; i < n_ev; ++i) {
        if (ev[i].n < 0) return fail(ctx, TPC_EINVAL, "negative cluster count");
        if (ev[i].n > 0 && (!ev[i].y || !ev[i].z || !ev[i].row || !ev[i].sector))
            return fail(ctx, TPC_EINVAL, "NULL cluster array");
        n_total += ev[i].n;
    }
    if (n_total > s.caps.n)
        return fail(ctx, TPC_EINVAL, "clusters in the launch exceed max_clusters_per_event");
    const int S = n_sec * n_ev;
    if (S > s.caps.s) return fail(ctx, TPC_EINVAL, "sectors in the launch exceed the arena");
    // descriptor mirror of this launch: wait until its previous copy is done
    s.desc_turn ^= 1;
    if (s.desc_used[s.desc_turn]) CUDA_TRY(ctx, cudaEventSynchronize(s.desc_done[s.desc_turn]));
    s.desc_host = s.desc_ring[s.desc_turn];
    LaunchInfo& I = s.info;
    I = LaunchInfo();
    I.n_ev = n_ev;
    I.S = S;
    I.R = g->n_rows;
    // descriptor tables
    EventDesc* dh = (EventDesc*)s.desc_host;
    long long* offh = (long long*)((char*)s.desc_host + sizeof(EventDesc) * s.caps.e);
    int* sech = (int*)((char*)offh + sizeof(long long) * (s.caps.e + 1));
    float* xrh = (float*)(sech + s.caps.s);
    for (int r = 0; r < g->n_rows; ++r) xrh[r] = g->row_x[r];
    long long off = 0;
    for (int i = 0; i < n_ev; ++i) {
        EventDesc d;
        if (ev[i].on_device || ev[i].n == 0) {
            d.y = ev[i].y;
            d.z = ev[i].z;
            d.row = ev[i].row;
            d.sec = ev[i].sector;
        } else {
            d.y = s.in_y + off;
            d.z = s.in_z + off;
            d.row = s.in_row + off;
            d.sec = s.in_sec + off;
        }
        d.n = ev[i].n;
        d.cl_off = off;
        d.sec_base = i * n_sec;
        d.n_sec = n_sec;
        dh[i] = d;
        offh[i] = off;
        I.ev_n.push_back(ev[i].n);
        I.ev_sec_base.push_back(i * n_sec);
        I.ev_n_sec.push_back(n_sec);
        for (int k = 0; k < n_sec; ++k) sech[i * n_sec + k] = i;
        off += ev[i].n;
    }
    offh[n_ev] = off;
    // launch record
    Launch& L = I.L;
    std::memset(&L, 0, sizeof(L));
    L.n_total = n_total;
    L.n_events = n_ev;
    L.R = g->n_rows;
    L.S = S;
    L.RS = S * g->n_rows;
    L.n_sectors_phi = g->n_sectors_phi;
    L.split_z = g->split_z ? 1 : 0;
    L.t_cap = s.caps.t;
    L.tan_half = tanf(g->half_angle_rad);
    L.z_max = g->z_max;
    L.kB = (float)(kKappa * (double)bz);
    L.sy2 = P.meas_sigma_y * P.meas_sigma_y;
    L.sz2 = P.meas_sigma_z * P.meas_sigma_z;
    L.slope_win_y = P.slope_win_y;
    L.slope_win_z = P.slope_win_z;
    L.d_max = P.d_max;
    L.chi2_hit = P.chi2_hit;
    L.sin_max = P.sin_max;
    L.edge_margin = P.edge_margin;
    L.seed_var_s = P.seed_var_s;
    L.seed_var_t = P.seed_var_t;
    L.seed_var_q = P.seed_var_q;
    L.sy = std::fabs(P.meas_sigma_y);
    L.sz = std::fabs(P.meas_sigma_z);
    L.seed_sd_s = std::sqrt(P.seed_var_s);
    L.seed_sd_t = std::sqrt(P.seed_var_t);
    L.seed_sd_q = std::sqrt(P.seed_var_q);
    L.max_gap = P.max_gap;
    L.min_chain = P.min_chain;
    L.min_tracklet_hits = P.min_tracklet_hits;
    L.min_track_hits = P.min_track_hits;
    L.merge = P.merge ? 1 : 0;
    L.mg_chi2 = P.merge_chi2;
    L.mg_dx_lo = P.merge_dx_lo;
    L.mg_dx_hi = P.merge_dx_hi;
    {
        const double d = 2.0 * (double)g->half_angle_rad;
        L.mg_cd = (float)std::cos(d);
        L.mg_sd = (float)std::sin(d);
        L.mg_ring = g->n_sectors_phi * d > 2.0 * M_PI - 1e-6 ? 1 : 0;
    }
    L.n_mg_tiles = (int)(((long long)s.caps.t + kMgTile - 1) / kMgTile);
    L.spin_limit = ctx->dbg_spin;
    L.stall_hit_tile = ctx->dbg_stall;
    L.ev = (EventDesc*)s.desc_dev;
    L.ev_off = (long long*)((char*)s.desc_dev + sizeof(EventDesc) * s.caps.e);
    L.sec_event = (int*)((char*)L.ev_off + sizeof(long long) * (s.caps.e + 1));
    L.xr = (const float*)(L.sec_event + s.caps.s);
    // zero region laid out for this launch
    {
        size_t zo = 0;
        auto take = [&](size_t bytes) {
            zo = align_up(zo, 16);
            char* p = s.zero_dev + zo;
            zo += bytes;
            return p;
        };
        L.cnt = (Counters*)take(sizeof(Counters));
        L.row_cnt = (int*)take(4 * (size_t)L.RS * kCntPad);
        L.ev_invalid = (int*)take(4 * (size_t)n_ev);
        L.sec_first = (int*)take(4 * (size_t)S);
        L.sec_end = (int*)take(4 * (size_t)S);
        L.n_row_tiles = (int)((L.RS + kRowTile - 1) / kRowTile);
        if (L.n_row_tiles < 1) L.n_row_tiles = 1;
        L.n_hit_tiles = (int)((n_total + kHitTile - 1) / kHitTile);
        if (L.n_hit_tiles < 1) L.n_hit_tiles = 1;
        L.tile_state = (unsigned long long*)take(8 * ((size_t)L.n_row_tiles + L.n_hit_tiles + S +
                                                     (L.merge ? L.n_mg_tiles : 0)));
        zo = align_up(zo, 16);
        if (zo > s.zero_cap) return fail(ctx, TPC_EINVAL, "internal: zero region too small");
        CUDA_TRY(ctx, cudaMemsetAsync(s.zero_dev, 0, zo, s.stream));
    }
    L.row_off = s.row_off;
    L.big_rows = s.big_rows;
    L.grid = s.grid;
    L.tmp_rec = s.tmp_rec;
    L.rank = s.rank;
    L.hyz = s.hyz;
    L.hcid = s.hcid;
    L.hrow = s.hrow;
    L.bin_start = s.bin_start;
    L.up = s.up;
    L.dn = s.dn;
    L.upc = s.upc;
    L.dnc = s.dnc;
    L.weight = s.weight;
    L.mark = s.mark;
    L.crowded = s.crowded;
    L.starts = s.starts;
    L.tl = s.tl;
    L.tl_chain = s.tl_chain;
    L.tl_rowhit = s.tl_rowhit;
    L.tl_list = s.tl_list;
    L.upg = s.upg;
    L.tl_key = s.tl_key;
    L.tl_nown = s.tl_nown;
    L.tl_own = s.tl_own;
    L.tl_out = s.tl_out;
    L.tl_hitoff = s.tl_hitoff;
    L.sec_trk_off = s.sec_trk_off;
    L.sec_hit_off = s.sec_hit_off;
    L.k_sector = s.k_sector;
    L.k_x = s.k_x;
    L.k_param = s.k_param;
    L.k_cov = s.k_cov;
    L.k_chi2 = s.k_chi2;
    L.k_ndf = s.k_ndf;
    L.k_hit_off = s.k_hit_off;
    L.k_hit_cid = s.k_hit_cid;
    L.k_gsec = s.k_gsec;
    L.mg_st = s.mg_st;
    L.mg_fit = s.mg_fit;
    L.mg_key = s.mg_key;
    L.mg_best = s.mg_best;
    L.mg_link = s.mg_link;
    L.mg_in = s.mg_in;
    L.mg_absorbed = s.mg_absorbed;
    L.mg_oidx = s.mg_oidx;
    L.mg_ohoff = s.mg_ohoff;
    L.mg_hxyz = s.mg_hxyz;
    L.mg_xs = s.mg_xs;
    L.mg_xi = s.mg_xi;
    L.mg_pre = s.mg_pre;
    L.m_sector = s.m_sector;
    L.m_x = s.m_x;
    L.m_param = s.m_param;
    L.m_cov = s.m_cov;
    L.m_chi2 = s.m_chi2;
    L.m_ndf = s.m_ndf;
    L.m_hit_off = s.m_hit_off;
    L.m_hit_cid = s.m_hit_cid;
    L.m_sec_trk_off = s.m_sec_trk_off;
    L.m_sec_hit_off = s.m_sec_hit_off;
    // inputs
    CUDA_TRY(ctx, cudaMemcpyAsync(s.desc_dev, s.desc_host, s.desc_bytes, cudaMemcpyHostToDevice, s.stream));
    CUDA_TRY(ctx, cudaEventRecord(s.desc_done[s.desc_turn], s.stream));
    s.desc_used[s.desc_turn] = true;
    for (int i = 0; i < n_ev; ++i) {
        if (ev[i].on_device || ev[i].n == 0) continue;
        const size_t n = (size_t)ev[i].n;
        const long long o = dh[i].cl_off;
        CUDA_TRY(ctx, cudaMemcpyAsync(s.in_y + o, ev[i].y, 4 * n, cudaMemcpyHostToDevice, s.stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.in_z + o, ev[i].z, 4 * n, cudaMemcpyHostToDevice, s.stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.in_row + o, ev[i].row, 2 * n, cudaMemcpyHostToDevice, s.stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.in_sec + o, ev[i].sector, 2 * n, cudaMemcpyHostToDevice, s.stream));
    }
    KernelHook hook{nullptr, nullptr};
    if (s.prof) {
        hook.after = [](void* user, const char* name) {
            Slot& sl = *(Slot*)user;
            const size_t i0 = sl.prof_last;
            const size_t i1 = prof_event(sl);
            sl.prof_marks.push_back({name, {i0, i1}});
            sl.prof_last = i1;
        };
        hook.user = &s;
        s.prof_last = prof_event(s);
    }
    const KernelHook* hk = s.prof ? &hook : nullptr;
    if (s.prof || !ctx->graphs) launch_all(L, ctx->sched, s.stream, hk);
    else if (int rc = launch_graph(ctx, s, L)) return rc;
    CUDA_TRY(ctx, cudaGetLastError());
    CUDA_TRY(ctx, cudaMemcpyAsync(s.cnt_host, L.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s.stream));
    CUDA_TRY(ctx, cudaEventRecord(s.done_ev, s.stream));
    s.launched = true;
    I.pending = true;
    return TPC_OK;
}

// Wait for the slot's launch and turn its device status into a code.
// Invalid clusters fail the launch unless per_event (the served form, where
// they fail only their own event's ticket: they are never binned, so the
// other events of the launch are unaffected).
int launch_status(tpc_track_ctx* ctx, Slot& s, bool per_event = false)
{
    LaunchInfo& I = s.info;
    if (!I.pending) return fail(ctx, TPC_EINVAL, "no launch pending");
    I.pending = false;
    CUDA_TRY(ctx, cudaEventSynchronize(s.done_ev));
    CUDA_TRY(ctx, cudaGetLastError());
    const Counters& c = *s.cnt_host;
    if (c.n_invalid && !per_event)
        return fail(ctx, TPC_EINVAL, std::to_string(c.n_invalid) + " invalid clusters (row, sector or coordinate)");
    if (c.timeout) return fail(ctx, TPC_ETIMEOUT, "a bounded device wait gave up");
    if (c.ovf_row) return fail(ctx, TPC_ECAPACITY, "a pad row holds more than 4096 clusters");
    if (c.ovf_tracklets || c.n_starts > s.caps.t)
        return fail(ctx, TPC_ECAPACITY, "start hits exceed the tracklet slots");
    if (c.ovf_sector) return fail(ctx, TPC_ECAPACITY, "a sector emits more than 4096 tracks");
    return TPC_OK;
}

void fill_counters(Slot& s)
{
    LaunchInfo& I = s.info;
    const Counters& c = *s.cnt_host;
    tpc_track_counters& K = I.counters;
    K.n_clusters = 0;
    for (long long n : I.ev_n) K.n_clusters += n;
    K.n_rows_total = (int64_t)I.S * I.R;
    K.n_bins = c.n_bins;
    K.n_links = c.n_links;
    K.n_starts = c.n_starts;
    K.n_tracklets = c.n_tracklets;
    K.n_valid_tracklets = c.n_valid;
    K.n_tracklet_hits = c.n_tracklet_hits;
    K.n_tracks = c.n_tracks;
    K.n_track_hits = c.n_track_hits;
    K.n_chain_hits = c.n_chain_hits;
    K.n_dominated_chains = c.n_dominated;
    K.n_sector_tracks = c.n_tracks;
    K.max_row_hits = c.max_row_hits;
    K.max_sector_tracks = c.max_sector_tracks;
    K.n_crowded_hits = c.n_crowded;
    if (I.L.merge) {
        K.n_tracks = c.n_mg_tracks;
        K.n_merge_links = c.n_mg_links;
        K.n_merge_chains = c.n_mg_chains;
    }
    I.done = true;
}

// The device arrays of a launch's final tracks: the selector's, or the
// merger's when the launch merged.
struct DevOut {
    const int* sector;
    const float *x, *param, *cov, *chi2;
    const int *ndf, *hit_off, *hit_cid, *sec_trk_off, *sec_hit_off;
    int nt, nh;
};
DevOut dev_out(const Slot& s)
{
    const Counters& c = *s.cnt_host;
    if (s.info.L.merge)
        return {s.m_sector, s.m_x, s.m_param, s.m_cov, s.m_chi2, s.m_ndf, s.m_hit_off, s.m_hit_cid,
                s.m_sec_trk_off, s.m_sec_hit_off, c.n_mg_tracks, c.n_track_hits};
    return {s.k_sector, s.k_x, s.k_param, s.k_cov, s.k_chi2, s.k_ndf, s.k_hit_off, s.k_hit_cid,
            s.sec_trk_off, s.sec_hit_off, c.n_tracks, c.n_track_hits};
}

// Wait for the slot's launch, check the device status, copy the results.
int collect(tpc_track_ctx* ctx, Slot& s)
{
    LaunchInfo& I = s.info;
    s.tracks.assign(I.n_ev, tpc_tracks{});
    if (int rc = launch_status(ctx, s)) return rc;
    const DevOut D = dev_out(s);
    const int nt = D.nt, nh = D.nh;
    cudaStream_t st = s.stream;
    if (nt > 0) {
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.sector, D.sector, 4 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.x, D.x, 4 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.param, D.param, 20 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.cov, D.cov, 60 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.chi2, D.chi2, 4 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.ndf, D.ndf, 4 * (size_t)nt, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.hit_off, D.hit_off, 4 * ((size_t)nt + 1), cudaMemcpyDeviceToHost, st));
    }
    if (nh > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(s.out.hit_cid, D.hit_cid, 4 * (size_t)nh, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s.out.sec_trk_off, D.sec_trk_off, 4 * ((size_t)I.S + 1), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    // split per event (sectors of an event are contiguous, so are its tracks)
    int32_t* eho = s.out.ev_hit_off;
    for (int e = 0; e < I.n_ev; ++e) {
        const int t0 = nt > 0 ? s.out.sec_trk_off[I.ev_sec_base[e]] : 0;
        const int t1 = nt > 0 ? s.out.sec_trk_off[I.ev_sec_base[e] + I.ev_n_sec[e]] : 0;
        const int h0 = nt > 0 ? s.out.hit_off[t0] : 0;
        tpc_tracks& T = s.tracks[e];
        T.n_tracks = t1 - t0;
        T.sector = s.out.sector + t0;
        T.x = s.out.x + t0;
        T.param = s.out.param + 5 * (size_t)t0;
        T.cov = s.out.cov + 15 * (size_t)t0;
        T.chi2 = s.out.chi2 + t0;
        T.ndf = s.out.ndf + t0;
        T.hit_cid = s.out.hit_cid + h0;
        for (int j = t0; j <= t1; ++j) eho[j - t0] = (nt > 0 ? s.out.hit_off[j] : 0) - h0;
        T.hit_off = eho;
        eho += (t1 - t0) + 1;
    }
    fill_counters(s);
    return TPC_OK;
}

}  // namespace

void prepare_kernels(Schedule* s)
{
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n_sm > 0)
        s->n_sm = n_sm;
    prepare_binning();
    prepare_selector();
    prepare_merger();
    s->tl_max_per_sm = constructor_occupancy();
    s->tl_blocks_per_sm = s->tl_max_per_sm;
    s->nr_max_per_sm = neighbour_rows_occupancy();
}

namespace {

PinnedBuf pool_get(tpc_track_ctx* ctx, size_t need)
{
    {
        std::lock_guard<std::mutex> lk(ctx->pool_mu);
        for (size_t i = 0; i < ctx->pool.size(); ++i)
            if (ctx->pool[i].cap >= need) {
                PinnedBuf b = ctx->pool[i];
                ctx->pool[i] = ctx->pool.back();
                ctx->pool.pop_back();
                return b;
            }
    }
    // twice the size asked for (at least 4 MB): later, larger events reuse
    // the buffer instead of pinning new host memory in the middle of a run
    PinnedBuf b;
    const size_t cap = align_up(std::max<size_t>(2 * need, 4u << 20), 1 << 20);
    if (cudaHostAlloc((void**)&b.p, cap, cudaHostAllocDefault) == cudaSuccess) b.cap = cap;
    else b.p = nullptr;
    return b;
}

void pool_put(tpc_track_ctx* ctx, PinnedBuf b)
{
    if (!b.p) return;
    std::lock_guard<std::mutex> lk(ctx->pool_mu);
    ctx->pool.push_back(b);
}

// Served form: wait for the slot's launch and copy every event's tracks from
// the device straight into a pinned buffer of its ticket (no host copy).
int collect_to_tickets(tpc_track_ctx* ctx, Slot& s, std::vector<std::unique_ptr<TicketResult>>& out)
{
    LaunchInfo& I = s.info;
    if (int rc = launch_status(ctx, s, true)) return rc;
    const Counters& c = *s.cnt_host;
    const DevOut D = dev_out(s);
    const int nt = D.nt;
    cudaStream_t st = s.stream;
    std::vector<int> inv(I.n_ev, 0);
    CUDA_TRY(ctx, cudaMemcpyAsync(s.out.sec_trk_off, D.sec_trk_off, 4 * ((size_t)I.S + 1), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(s.out.sec_hit_off, D.sec_hit_off, 4 * ((size_t)I.S + 1), cudaMemcpyDeviceToHost, st));
    if (c.n_invalid)
        CUDA_TRY(ctx, cudaMemcpyAsync(inv.data(), I.L.ev_invalid, 4 * (size_t)I.n_ev, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::vector<int> h0s(I.n_ev);
    for (int e = 0; e < I.n_ev; ++e) {
        const int sb = I.ev_sec_base[e], se = sb + I.ev_n_sec[e];
        const int t0 = nt > 0 ? s.out.sec_trk_off[sb] : 0, t1 = nt > 0 ? s.out.sec_trk_off[se] : 0;
        const int h0 = nt > 0 ? s.out.sec_hit_off[sb] : 0, h1 = nt > 0 ? s.out.sec_hit_off[se] : 0;
        const size_t m = (size_t)(t1 - t0), mh = (size_t)(h1 - h0);
        size_t off = 0;
        auto place = [&](size_t bytes) {
            const size_t o = off;
            off = align_up(off + bytes, 16);
            return o;
        };
        const size_t o_sec = place(4 * m), o_x = place(4 * m), o_par = place(20 * m),
                     o_cov = place(60 * m), o_chi = place(4 * m), o_ndf = place(4 * m),
                     o_ho = place(4 * (m + 1)), o_hc = place(4 * mh);
        TicketResult& R = *out[e];
        if (inv[e]) {  // this event had invalid clusters: no result for it
            R.status = fail(ctx, TPC_EINVAL, std::to_string(inv[e]) +
                                                 " invalid clusters (row, sector or coordinate)");
            continue;
        }
        R.status = TPC_OK;
        R.buf = pool_get(ctx, off);
        if (!R.buf.p) return fail(ctx, TPC_ENOMEM, "pinned result buffer");
        char* b = R.buf.p;
        if (m > 0) {
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_sec, D.sector + t0, 4 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_x, D.x + t0, 4 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_par, D.param + 5 * (size_t)t0, 20 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_cov, D.cov + 15 * (size_t)t0, 60 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_chi, D.chi2 + t0, 4 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_ndf, D.ndf + t0, 4 * m, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_ho, D.hit_off + t0, 4 * (m + 1), cudaMemcpyDeviceToHost, st));
        }
        if (mh > 0)
            CUDA_TRY(ctx, cudaMemcpyAsync(b + o_hc, D.hit_cid + h0, 4 * mh, cudaMemcpyDeviceToHost, st));
        tpc_tracks& V = R.view;
        V.n_tracks = (int64_t)m;
        V.sector = (const int32_t*)(b + o_sec);
        V.x = (const float*)(b + o_x);
        V.param = (const float*)(b + o_par);
        V.cov = (const float*)(b + o_cov);
        V.chi2 = (const float*)(b + o_chi);
        V.ndf = (const int32_t*)(b + o_ndf);
        V.hit_off = (const int32_t*)(b + o_ho);
        V.hit_cid = (const int32_t*)(b + o_hc);
        h0s[e] = h0;
        if (m == 0) *(int32_t*)(b + o_ho) = 0;
    }
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int e = 0; e < I.n_ev; ++e) {  // hit offsets relative to the event
        TicketResult& R = *out[e];
        if (R.status != TPC_OK) continue;
        int32_t* ho = (int32_t*)R.view.hit_off;
        if (R.view.n_tracks > 0)
            for (int64_t j = 0; j <= R.view.n_tracks; ++j) ho[j] -= h0s[e];
    }
    fill_counters(s);
    return TPC_OK;
}

// --------------------------------------------------------------------------
// debug dumps (event 0 of the last completed launch)
// --------------------------------------------------------------------------
int dump(tpc_track_ctx* ctx, Slot& s, int stage, int event, void* buf, size_t cap, size_t* used)
{
    LaunchInfo& I = s.info;
    if (!I.done) return fail(ctx, TPC_EINVAL, "no completed launch to dump");
    if (event < 0 || event >= I.n_ev) return fail(ctx, TPC_EINVAL, "no such event in the last launch");
    const int R = I.R;
    // an event's sectors are consecutive in the launch's (sector, row) list,
    // and so are its sorted hits
    const int RSb = I.ev_sec_base[event] * R;
    const int RSe = RSb + I.ev_n_sec[event] * R;
    const long long n0 = I.ev_n[event];
    std::vector<int> row_all(RSe + 2);
    CUDA_TRY(ctx, cudaMemcpy(row_all.data(), s.row_off, 4 * (size_t)(RSe + 1), cudaMemcpyDeviceToHost));
    const int hb = row_all[RSb];   // first sorted hit of the event
    const int nh = row_all[RSe] - hb;  // its sorted hits
    std::vector<int> row_off(row_all.begin() + RSb, row_all.begin() + RSe + 1);
    for (int& v : row_off) v -= hb;
    std::vector<int> hcid(nh), hrow(nh);
    if (nh) {
        CUDA_TRY(ctx, cudaMemcpy(hcid.data(), s.hcid + hb, 4 * (size_t)nh, cudaMemcpyDeviceToHost));
        CUDA_TRY(ctx, cudaMemcpy(hrow.data(), s.hrow + hb, 4 * (size_t)nh, cudaMemcpyDeviceToHost));
    }
    const int sb = I.ev_sec_base[event];
    // row index within the event's rows (hrow holds the launch-wide sector)
    auto row_of = [&](int i) { return ((hrow[i] >> 8) - sb) * R + (hrow[i] & 255); };
    std::vector<char> out;
    auto put = [&](const void* p, size_t b) {
        const char* c = (const char*)p;
        out.insert(out.end(), c, c + b);
    };
    if (stage == TPC_DUMP_SORTED) {
        put(hcid.data(), 4 * (size_t)nh);
    } else if (stage == TPC_DUMP_LINKS || stage == TPC_DUMP_CLEAN) {
        std::vector<int16_t> u(nh), d(nh);
        if (nh) {
            CUDA_TRY(ctx, cudaMemcpy(u.data(), (stage == TPC_DUMP_LINKS ? s.up : s.upc) + hb, 2 * (size_t)nh, cudaMemcpyDeviceToHost));
            CUDA_TRY(ctx, cudaMemcpy(d.data(), (stage == TPC_DUMP_LINKS ? s.dn : s.dnc) + hb, 2 * (size_t)nh, cudaMemcpyDeviceToHost));
        }
        std::vector<int32_t> uc(n0, -1), dc(n0, -1);
        for (int i = 0; i < nh; ++i) {
            const int g = row_of(i);
            if (u[i] >= 0) uc[hcid[i]] = hcid[row_off[g + 1] + u[i]];
            if (d[i] >= 0) dc[hcid[i]] = hcid[row_off[g - 1] + d[i]];
        }
        put(uc.data(), 4 * (size_t)n0);
        put(dc.data(), 4 * (size_t)n0);
    } else if (stage == TPC_DUMP_STARTS || stage == TPC_DUMP_TRACKLETS) {
        const int ns = std::min<int>(s.cnt_host->n_starts, s.caps.t);
        std::vector<int> st(ns);
        std::vector<TrackletHdr> tl(ns);
        if (ns) {
            CUDA_TRY(ctx, cudaMemcpy(st.data(), s.starts, 4 * (size_t)ns, cudaMemcpyDeviceToHost));
            CUDA_TRY(ctx, cudaMemcpy(tl.data(), s.tl, sizeof(TrackletHdr) * (size_t)ns, cudaMemcpyDeviceToHost));
        }
        std::vector<std::pair<int, int>> order;  // (start cid, tracklet) of the event
        for (int t = 0; t < ns; ++t)
            if (st[t] >= hb && st[t] < hb + nh) order.push_back({hcid[st[t] - hb], t});
        std::sort(order.begin(), order.end());
        if (stage == TPC_DUMP_STARTS) {
            for (auto& o : order) put(&o.first, 4);
        } else {
            // the rowhit rows of every start at once (global sorted indices)
            std::vector<int32_t> rh_all((size_t)ns * R);
            if (ns) CUDA_TRY(ctx, cudaMemcpy(rh_all.data(), s.tl_rowhit, 4 * (size_t)ns * R, cudaMemcpyDeviceToHost));
            int32_t count = 0;
            for (auto& o : order)
                if (tl[o.second].chain_len >= s.info.L.min_chain && !tl[o.second].dominated) ++count;
            put(&count, 4);
            for (auto& o : order) {
                const TrackletHdr& H = tl[o.second];
                if (H.chain_len < s.info.L.min_chain || H.dominated) continue;
                tpc_dump_tracklet D;
                std::memset(&D, 0, sizeof(D));
                D.start_cid = o.first;
                D.sector = (hrow[H.start - hb] >> 8) - sb;
                D.valid = H.valid;
                D.nhits = H.nhits;
                D.first_row = H.first;
                D.last_row = H.last;
                D.ndf = H.ndf;
                D.x = H.x;
                std::memcpy(D.param, H.p, sizeof(D.param));
                std::memcpy(D.cov, H.C, sizeof(D.cov));
                D.chi2 = H.chi2;
                put(&D, sizeof(D));
                const int32_t* rh = rh_all.data() + (size_t)o.second * R;
                std::vector<int32_t> rc(R, -1);
                for (int r = H.first; r <= H.last && r >= 0; ++r)
                    if (rh[r] >= hb && rh[r] < hb + nh) rc[r] = hcid[rh[r] - hb];
                put(rc.data(), 4 * (size_t)R);
            }
        }
    } else if (stage == TPC_DUMP_WEIGHTS) {
        std::vector<unsigned long long> w(nh);
        if (nh) CUDA_TRY(ctx, cudaMemcpy(w.data(), s.weight + hb, 8 * (size_t)nh, cudaMemcpyDeviceToHost));
        std::vector<unsigned long long> wc(n0, 0ULL);
        for (int i = 0; i < nh; ++i) wc[hcid[i]] = w[i];
        put(wc.data(), 8 * (size_t)n0);
    } else {
        return fail(ctx, TPC_EINVAL, "unknown dump stage");
    }
    if (used) *used = out.size();
    if (buf && cap > 0) std::memcpy(buf, out.data(), std::min(cap, out.size()));
    return TPC_OK;
}

// Make st the slot's stream, ordered after the slot's previous launch.
int use_stream(tpc_track_ctx* ctx, Slot& s, cudaStream_t st)
{
    if (s.stream != st && s.launched) CUDA_TRY(ctx, cudaStreamWaitEvent(st, s.done_ev, 0));
    s.stream = st;
    return TPC_OK;
}

// --------------------------------------------------------------------------
// served form: one worker per slot pulls what fits into its next launch
// --------------------------------------------------------------------------
void worker(tpc_track_ctx* ctx, Slot* s)
{
    cudaSetDevice(ctx->cfg.device);
    for (;;) {
        std::vector<Request> batch;
        {
            std::unique_lock<std::mutex> lk(ctx->mu);
            ctx->cv_req.wait(lk, [&] { return ctx->stop || !ctx->queue.empty(); });
            if (ctx->stop && ctx->queue.empty()) return;
            long long sum = 0;
            while (!ctx->queue.empty() && (int)batch.size() < s->caps.e) {
                Request& q = ctx->queue.front();
                if (!batch.empty()) {
                    const Request& b0 = batch.front();
                    const bool same = q.bz == b0.bz && q.geom.n_rows == b0.geom.n_rows &&
                                      q.geom.n_sectors_phi == b0.geom.n_sectors_phi &&
                                      q.geom.split_z == b0.geom.split_z &&
                                      q.geom.half_angle_rad == b0.geom.half_angle_rad &&
                                      q.geom.z_max == b0.geom.z_max && q.row_x == b0.row_x &&
                                      q.prm_version == b0.prm_version;
                    if (!same || sum + q.ev.n > s->caps.n) break;
                }
                sum += q.ev.n;
                batch.push_back(std::move(q));
                ctx->queue.pop_front();
            }
        }
        std::vector<tpc_clusters> evs;
        for (auto& q : batch) evs.push_back(q.ev);
        tpc_geometry g = batch.front().geom;
        g.row_x = batch.front().row_x.data();
        const auto t0 = std::chrono::steady_clock::now();
        std::vector<std::unique_ptr<TicketResult>> done(batch.size());
        for (auto& d : done) d = std::make_unique<TicketResult>();
        int rc = enqueue(ctx, *s, (int)evs.size(), evs.data(), &g, batch.front().bz, batch.front().prm);
        const auto t1 = std::chrono::steady_clock::now();
        if (rc == TPC_OK) rc = collect_to_tickets(ctx, *s, done);
        const auto t2 = std::chrono::steady_clock::now();
        for (auto& d : done) {
            if (rc != TPC_OK) d->status = rc;  // launch-wide error
            if (d->status != TPC_OK) {  // no partial result: buffers back to the pool
                pool_put(ctx, d->buf);
                d->buf = PinnedBuf{};
                d->view = tpc_tracks{};
            }
        }
        // fill the tickets' own result objects in place (pollers hold pointers
        // to them); the swapped-out placeholders are freed outside the lock
        std::unique_lock<std::mutex> lk(ctx->mu);
        for (size_t i = 0; i < batch.size(); ++i) {
            auto it = ctx->results.find(batch[i].ticket);
            if (it == ctx->results.end()) continue;
            done[i]->prm = it->second->prm;
            done[i]->prm_version = it->second->prm_version;
            std::swap(*it->second, *done[i]);
        }
        ctx->cv_done.notify_all();
        lk.unlock();
        for (auto& d : done) pool_put(ctx, d->buf);  // tickets released meanwhile
        done.clear();
    }
}

}  // namespace
}  // namespace tpc

using namespace tpc;

extern "C" {

void tpc_track_default_params(tpc_track_params* p)
{
    if (!p) return;
    p->meas_sigma_y = 0.1f;
    p->meas_sigma_z = 0.1f;
    p->slope_win_y = 2.0f;
    p->slope_win_z = 2.0f;
    p->d_max = 0.6f;
    p->chi2_hit = 16.0f;
    p->max_gap = 5;
    p->min_chain = 3;
    p->min_tracklet_hits = 10;
    p->min_track_hits = 10;
    p->sin_max = 0.99f;
    p->edge_margin = 2.0f;
    p->seed_var_s = 1.0f;
    p->seed_var_t = 1.0f;
    p->seed_var_q = 100.0f;
    p->merge = 0;
    p->merge_chi2 = 30.0f;
    p->merge_dx_lo = -5.0f;
    p->merge_dx_hi = 30.0f;
}

static bool params_ok(const tpc_track_params& P)
{
    return P.meas_sigma_y > 0 && P.meas_sigma_z > 0 && std::isfinite(P.meas_sigma_y) &&
           std::isfinite(P.meas_sigma_z) && P.d_max >= 0 && P.chi2_hit > 0 && P.max_gap >= 1 &&
           P.min_chain >= 2 && P.min_tracklet_hits >= 1 && P.min_track_hits >= 1 &&
           P.sin_max > 0 && P.sin_max < 1 && P.seed_var_s > 0 && P.seed_var_t > 0 &&
           P.seed_var_q > 0 && (P.merge == 0 || P.merge == 1) && P.merge_chi2 > 0 &&
           std::isfinite(P.merge_chi2) && std::isfinite(P.merge_dx_lo) &&
           std::isfinite(P.merge_dx_hi) && P.merge_dx_lo <= P.merge_dx_hi;
}

int tpc_track_create(const tpc_track_config* cfg, tpc_track_ctx** out)
{
    if (!out) return TPC_EINVAL;
    *out = nullptr;
    if (!cfg) return TPC_EINVAL;
    if (cfg->max_clusters_per_event <= 0 || cfg->max_clusters_per_event > (1LL << 29) ||
        cfg->max_events_in_flight < 1 || cfg->max_events_in_flight > 16 ||
        cfg->max_rows < 0 || cfg->max_rows > kMaxRows || cfg->max_events_per_launch < 0 ||
        cfg->max_events_per_launch > kMaxEventsPerLaunch)
        return TPC_EINVAL;
    if (!params_ok(cfg->params)) return TPC_EINVAL;
    auto ctx = std::make_unique<tpc_track_ctx>();
    ctx->cfg = *cfg;
    const char* ng = std::getenv("TPC_NO_GRAPH");
    ctx->graphs = !(ng && ng[0] == '1');
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        return TPC_ECUDA;
    }
    prepare_kernels(&ctx->sched);
    if (cudaGetLastError() != cudaSuccess) return TPC_ECUDA;
    const int n_slots = cfg->max_events_in_flight;
    size_t total = 0;
    for (int i = 0; i < n_slots; ++i) {
        auto s = std::make_unique<Slot>();
        s->id = i;
        s->caps = make_caps(*cfg);
        total += layout(*s, nullptr);
        ctx->slots.push_back(std::move(s));
    }
    if (cfg->mem_budget && total > cfg->mem_budget) return TPC_ENOMEM;
    for (auto& s : ctx->slots) {
        int rc = alloc_slot(ctx.get(), *s);
        if (rc == TPC_OK) {
            if (s->id == 0 && cfg->cuda_stream) {
                s->stream = (cudaStream_t)cfg->cuda_stream;
            } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess) {
                s->own_stream = true;
            } else {
                rc = TPC_ECUDA;
            }
            s->home = s->pipe = s->stream;
            if (rc == TPC_OK && s->id == 0) {
                if (cudaStreamCreateWithFlags(&s->pipe, cudaStreamNonBlocking) == cudaSuccess)
                    s->own_pipe = true;
                else
                    rc = TPC_ECUDA;
            }
        }
        if (rc != TPC_OK) {
            for (auto& t : ctx->slots) free_slot(*t);
            return rc;
        }
    }
    if (cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
        for (auto& t : ctx->slots) free_slot(*t);
        return TPC_ECUDA;
    }
    *out = ctx.release();
    return TPC_OK;
}

int tpc_track_launch(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev, const tpc_geometry* geom,
                     float bz)
{
    if (!ctx) return TPC_EINVAL;
    if (!ctx->workers.empty()) return fail(ctx, TPC_EBUSY, "context is serving submitted events");
    cudaSetDevice(ctx->cfg.device);
    Slot& s0 = *ctx->slots[0];
    if (s0.prof && s0.prof_used > 60000) return fail(ctx, TPC_EINVAL, "profiling buffer full");
    // while profiling, launches run one at a time on the context's stream
    const int K = s0.prof ? 1 : ctx->streams;
    const int j = K == 1 ? 0 : ctx->next_slot % K;
    ctx->next_slot = K == 1 ? 0 : (j + 1) % K;
    Slot& s = *ctx->slots[j];
    // results of this slot's uncollected launch are dropped
    s.info.pending = false;
    ctx->direct.erase(std::remove(ctx->direct.begin(), ctx->direct.end(), j), ctx->direct.end());
    cudaStream_t st = K == 1 ? s.home : s.pipe;
    if (int rc = use_stream(ctx, s, st)) return rc;
    if (st != s0.home) {  // fork: after the caller's work on the context's stream
        CUDA_TRY(ctx, cudaEventRecord(ctx->fork_ev, s0.home));
        CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->fork_ev, 0));
    }
    tpc_track_params P;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        P = ctx->cfg.params;
    }
    const int rc = enqueue(ctx, s, n_ev, ev, geom, bz, P);
    if (rc == TPC_OK) ctx->direct.push_back(j);
    return rc;
}

int tpc_track_join(tpc_track_ctx* ctx)
{
    if (!ctx) return TPC_EINVAL;
    cudaSetDevice(ctx->cfg.device);
    cudaStream_t home = ctx->slots[0]->home;
    for (auto& s : ctx->slots)
        if (s->launched && s->stream != home) CUDA_TRY(ctx, cudaStreamWaitEvent(home, s->done_ev, 0));
    return TPC_OK;
}

int tpc_track_results(tpc_track_ctx* ctx, int cap, tpc_tracks* outs)
{
    if (!ctx) return TPC_EINVAL;
    cudaSetDevice(ctx->cfg.device);
    if (ctx->direct.empty()) return fail(ctx, TPC_EINVAL, "no launch pending");
    const int j = ctx->direct.front();
    if (outs && cap < ctx->slots[j]->info.n_ev)
        return fail(ctx, TPC_EINVAL, "outs holds fewer entries than the launch has events (" +
                                         std::to_string(ctx->slots[j]->info.n_ev) + ")");
    ctx->direct.pop_front();
    ctx->last_slot = j;
    Slot& s = *ctx->slots[j];
    const int n_ev = s.info.n_ev;
    int rc = collect(ctx, s);
    if (outs)
        for (int e = 0; e < n_ev; ++e) outs[e] = rc == TPC_OK ? s.tracks[e] : tpc_tracks{};
    return rc;
}

int tpc_track_batch(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev, const tpc_geometry* geom,
                    float bz, tpc_tracks* outs)
{
    if (ctx && ctx->workers.empty()) {  // uncollected direct launches are dropped
        for (int j : ctx->direct) ctx->slots[j]->info.pending = false;
        ctx->direct.clear();
    }
    int rc = tpc_track_launch(ctx, n_ev, ev, geom, bz);
    if (rc != TPC_OK) {
        if (outs && ctx)
            for (int e = 0; e < n_ev; ++e) outs[e] = tpc_tracks{};
        return rc;
    }
    return tpc_track_results(ctx, n_ev, outs);
}

int tpc_track_event(tpc_track_ctx* ctx, const tpc_clusters* ev, const tpc_geometry* geom, float bz,
                    tpc_tracks* out)
{
    return tpc_track_batch(ctx, 1, ev, geom, bz, out);
}

int tpc_track_submit(tpc_track_ctx* ctx, const tpc_clusters* ev, const tpc_geometry* geom, float bz,
                     uint64_t* ticket)
{
    if (!ctx || !ev || !ticket) return TPC_EINVAL;
    if (int rc = check_geometry(ctx, *ctx->slots[0], geom)) return rc;
    if (ev->n < 0 || ev->n > ctx->slots[0]->caps.n)
        return fail(ctx, TPC_EINVAL, "event larger than one slot");
    if (ev->n > 0 && (!ev->y || !ev->z || !ev->row || !ev->sector))
        return fail(ctx, TPC_EINVAL, "NULL cluster array");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->workers.empty()) {
        for (auto& s : ctx->slots) {
            if (s->info.pending) {
                cudaEventSynchronize(s->done_ev);
                s->info.pending = false;
            }
            use_stream(ctx, *s, s->home);
            ctx->workers.emplace_back(worker, ctx, s.get());
        }
        ctx->direct.clear();
    }
    Request q;
    q.ticket = ctx->next_ticket++;
    q.ev = *ev;
    q.row_x.assign(geom->row_x, geom->row_x + geom->n_rows);
    q.geom = *geom;
    q.bz = bz;
    q.prm = ctx->cfg.params;
    q.prm_version = ctx->prm_version;
    q.t_submit = std::chrono::steady_clock::now();
    auto R = std::make_unique<TicketResult>();
    R->prm = q.prm;
    R->prm_version = q.prm_version;
    ctx->results[q.ticket] = std::move(R);
    *ticket = q.ticket;
    ctx->queue.push_back(std::move(q));
    ctx->cv_req.notify_one();
    return TPC_OK;
}

int tpc_track_poll(tpc_track_ctx* ctx, uint64_t ticket, int timeout_us, tpc_tracks* out)
{
    if (!ctx) return TPC_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->results.find(ticket);
    if (it == ctx->results.end()) return fail(ctx, TPC_EINVAL, "unknown ticket");
    TicketResult* R = it->second.get();
    auto ready = [&] { return R->status != TPC_EBUSY; };
    if (timeout_us < 0) ctx->cv_done.wait(lk, ready);
    else if (timeout_us > 0) ctx->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (!ready()) return TPC_EBUSY;
    if (out) *out = R->status == TPC_OK ? R->view : tpc_tracks{};
    return R->status;
}

int tpc_track_release(tpc_track_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return TPC_EINVAL;
    std::unique_ptr<TicketResult> gone;  // freed after the lock is released
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->results.find(ticket);
    if (it == ctx->results.end()) return fail(ctx, TPC_EINVAL, "unknown ticket");
    if (it->second->status == TPC_EBUSY) return fail(ctx, TPC_EBUSY, "ticket still in flight");
    gone = std::move(it->second);
    ctx->results.erase(it);
    pool_put(ctx, gone->buf);
    return TPC_OK;
}

int tpc_track_set_params(tpc_track_ctx* ctx, const tpc_track_params* p, uint64_t* first_ticket,
                         uint64_t* version)
{
    if (!ctx || !p) return TPC_EINVAL;
    if (!params_ok(*p)) return fail(ctx, TPC_EINVAL, "parameter out of range");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->cfg.params = *p;
    ++ctx->prm_version;
    if (first_ticket) *first_ticket = ctx->next_ticket;
    if (version) *version = ctx->prm_version;
    return TPC_OK;
}

int tpc_track_get_params(tpc_track_ctx* ctx, tpc_track_params* p, uint64_t* version)
{
    if (!ctx || !p) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *p = ctx->cfg.params;
    if (version) *version = ctx->prm_version;
    return TPC_OK;
}

int tpc_track_ticket_params(tpc_track_ctx* ctx, uint64_t ticket, tpc_track_params* p, uint64_t* version)
{
    if (!ctx) return TPC_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->results.find(ticket);
    if (it == ctx->results.end()) return fail(ctx, TPC_EINVAL, "unknown ticket");
    if (p) *p = it->second->prm;
    if (version) *version = it->second->prm_version;
    return TPC_OK;
}

int tpc_track_set_profiling(tpc_track_ctx* ctx, int on)
{
    if (!ctx) return TPC_EINVAL;
    if (!ctx->workers.empty()) return fail(ctx, TPC_EBUSY, "context is serving submitted events");
    cudaSetDevice(ctx->cfg.device);
    for (auto& t : ctx->slots)
        if (t->stream) CUDA_TRY(ctx, cudaStreamSynchronize(t->stream));
    Slot& s = *ctx->slots[0];
    if (int rc = use_stream(ctx, s, s.home)) return rc;
    s.prof = on != 0;
    s.prof_used = 0;
    s.prof_marks.clear();
    return TPC_OK;
}

int tpc_track_kernel_times(tpc_track_ctx* ctx, tpc_kernel_time* out, int cap, int* n)
{
    if (!ctx || !n) return TPC_EINVAL;
    Slot& s = *ctx->slots[0];
    cudaSetDevice(ctx->cfg.device);
    CUDA_TRY(ctx, cudaStreamSynchronize(s.stream));
    std::vector<tpc_kernel_time> acc;
    for (auto& m : s.prof_marks) {
        float ms = 0.0f;
        CUDA_TRY(ctx, cudaEventElapsedTime(&ms, s.prof_pool[m.second.first], s.prof_pool[m.second.second]));
        tpc_kernel_time* t = nullptr;
        for (auto& a : acc)
            if (m.first == a.name) t = &a;
        if (!t) {
            tpc_kernel_time z;
            std::memset(&z, 0, sizeof(z));
            std::snprintf(z.name, sizeof(z.name), "%s", m.first.c_str());
            acc.push_back(z);
            t = &acc.back();
        }
        t->total_ms += ms;
        t->launches += 1;
    }
    *n = (int)acc.size();
    for (int i = 0; i < (int)acc.size() && i < cap; ++i) out[i] = acc[i];
    return TPC_OK;
}

int tpc_track_get_schedule(const tpc_track_ctx* ctx, tpc_track_schedule* out)
{
    if (!ctx || !out) return TPC_EINVAL;
    const Schedule& S = ctx->sched;
    out->n_sm = S.n_sm;
    out->tl_max_per_sm = S.tl_max_per_sm;
    out->bin_blocks_per_sm = S.bin_blocks_per_sm;
    out->sort_threads = S.sort_threads;
    out->nb_threads = S.nb_threads;
    out->tl_blocks_per_sm = S.tl_blocks_per_sm;
    out->max_streams = (int)ctx->slots.size();
    out->streams = ctx->streams;
    out->nb_mode = S.nb_mode;
    return TPC_OK;
}

int tpc_track_set_schedule(tpc_track_ctx* ctx, const tpc_track_schedule* q)
{
    if (!ctx || !q) return TPC_EINVAL;
    if (!ctx->workers.empty()) return fail(ctx, TPC_EBUSY, "context is serving submitted events");
    const Schedule& S = ctx->sched;
    if (q->bin_blocks_per_sm < 1 || q->bin_blocks_per_sm > 32 ||
        (q->sort_threads != 256 && q->sort_threads != 512) ||
        (q->nb_threads != 64 && q->nb_threads != 128 && q->nb_threads != 256) ||
        q->tl_blocks_per_sm < 1 || q->tl_blocks_per_sm > S.tl_max_per_sm || q->streams < 1 ||
        q->streams > (int)ctx->slots.size() || (q->nb_mode != 0 && q->nb_mode != 1))
        return fail(ctx, TPC_EINVAL, "schedule value out of range");
    ctx->streams = q->streams;
    ctx->next_slot = 0;
    ctx->sched.bin_blocks_per_sm = q->bin_blocks_per_sm;
    ctx->sched.sort_threads = q->sort_threads;
    ctx->sched.nb_threads = q->nb_threads;
    ctx->sched.tl_blocks_per_sm = q->tl_blocks_per_sm;
    ctx->sched.nb_mode = q->nb_mode;
    return TPC_OK;
}

int tpc_track_autotune(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev,
                       const tpc_geometry* geom, float bz, int reps, tpc_track_schedule* out)
{
    if (!ctx) return TPC_EINVAL;
    if (!ctx->workers.empty()) return fail(ctx, TPC_EBUSY, "context is serving submitted events");
    if (reps < 1 || reps > 50) return fail(ctx, TPC_EINVAL, "reps out of range (1..50)");
    cudaSetDevice(ctx->cfg.device);
    for (auto& t : ctx->slots)
        if (t->stream) CUDA_TRY(ctx, cudaStreamSynchronize(t->stream));
    ctx->direct.clear();
    for (auto& t : ctx->slots) t->info.pending = false;
    Slot& s = *ctx->slots[0];
    if (int rc = use_stream(ctx, s, s.home)) return rc;
    const Schedule start = ctx->sched;
    tpc_track_params P;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        P = ctx->cfg.params;
    }
    // median over reps launches (after one warm-up) of the summed device time
    // of the named kernels under schedule S
    auto time_kernels = [&](const Schedule& S, const std::vector<std::string>& names,
                            double* ms) -> int {
        if (s.stream) CUDA_TRY(ctx, cudaStreamSynchronize(s.stream));
        ctx->sched = S;
        s.prof = true;
        std::vector<double> t;
        int rc = TPC_OK;
        for (int r = 0; r <= reps && rc == TPC_OK; ++r) {
            s.prof_used = 0;
            s.prof_marks.clear();
            s.info.pending = false;
            rc = enqueue(ctx, s, n_ev, ev, geom, bz, P);
            if (rc == TPC_OK) rc = launch_status(ctx, s);
            if (rc != TPC_OK || r == 0) continue;
            double sum = 0.0;
            for (auto& m : s.prof_marks) {
                bool want = false;
                for (auto& nm : names) want = want || m.first == nm;
                if (!want) continue;
                float x = 0.0f;
                if (cudaEventElapsedTime(&x, s.prof_pool[m.second.first], s.prof_pool[m.second.second]) != cudaSuccess) {
                    cudaGetLastError();
                    rc = fail(ctx, TPC_ECUDA, "autotune timing event");
                }
                sum += x;
            }
            t.push_back(sum);
        }
        s.prof = false;
        s.prof_used = 0;
        s.prof_marks.clear();
        ctx->sched = start;
        if (rc != TPC_OK) return rc;
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return TPC_OK;
    };
    Schedule best = start;
    auto tune = [&](int Schedule::*field, std::vector<int> cands, std::vector<std::string> names) -> int {
        double best_ms = 1e30;
        int best_v = best.*field;
        for (int v : cands) {
            Schedule S = best;
            S.*field = v;
            double ms = 0.0;
            if (int rc = time_kernels(S, names, &ms)) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best_v = v;
            }
        }
        best.*field = best_v;
        return TPC_OK;
    };
    const int mx = start.tl_max_per_sm;
    std::vector<int> tl = {mx};
    for (int v : {mx * 3 / 4, mx / 2})
        if (v >= 1 && std::find(tl.begin(), tl.end(), v) == tl.end()) tl.push_back(v);
    int rc = tune(&Schedule::tl_blocks_per_sm, tl, {"k_constructor_fwd", "k_constructor_bwd"});
    if (!rc) rc = tune(&Schedule::nb_threads, {64, 128, 256}, {"k_neighbours", "k_neighbours_crowded"});
    if (!rc) rc = tune(&Schedule::nb_mode, {0, 1}, {"k_neighbours", "k_neighbours_crowded"});
    if (!rc) rc = tune(&Schedule::sort_threads, {256, 512}, {"k_rowsort_big", "k_rowsort_big4k"});
    if (!rc) rc = tune(&Schedule::bin_blocks_per_sm, {2, 4, 8, 16}, {"k_count", "k_scatter"});
    if (rc) return rc;
    ctx->sched = best;
    // streams: rounds of 8 launches per stream spread over K slots, timed on
    // the context's stream from the first fork to the join, each K with the
    // constructor block counts above (concurrent launches share the SMs, so
    // the best count alone need not be the best together); a larger K must
    // win by 1% to be taken
    const int kmax = std::min(8, (int)ctx->slots.size());
    std::vector<int> ks;
    for (int K : {1, 2, 3, 4, 6, 8})
        if (K <= kmax) ks.push_back(K);
    if (kmax > 1) {
        const Schedule tuned = ctx->sched;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        CUDA_TRY(ctx, cudaEventCreate(&e0));
        CUDA_TRY(ctx, cudaEventCreate(&e1));
        double best_per = 1e30;
        int best_k = 1, best_tl = tuned.tl_blocks_per_sm;
        for (int K : ks)
        for (int tlv : (K == 1 ? std::vector<int>{tuned.tl_blocks_per_sm} : tl)) {
            if (rc != TPC_OK) break;
            ctx->streams = K;
            ctx->next_slot = 0;
            ctx->sched.tl_blocks_per_sm = tlv;
            std::vector<double> t;
            for (int r = 0; r <= std::max(reps, 7) && rc == TPC_OK; ++r) {
                const int nl = 8 * K;
                rc = cudaEventRecord(e0, s.home) == cudaSuccess ? TPC_OK : TPC_ECUDA;
                for (int l = 0; l < nl && rc == TPC_OK; ++l) rc = tpc_track_launch(ctx, n_ev, ev, geom, bz);
                if (rc == TPC_OK) rc = tpc_track_join(ctx);
                if (rc == TPC_OK && cudaEventRecord(e1, s.home) != cudaSuccess) rc = TPC_ECUDA;
                if (rc == TPC_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = TPC_ECUDA;
                // each slot's last launch holds the status of its launches
                while (rc == TPC_OK && !ctx->direct.empty()) {
                    Slot& q = *ctx->slots[ctx->direct.front()];
                    ctx->direct.pop_front();
                    rc = launch_status(ctx, q);
                }
                float ms = 0.0f;
                if (rc == TPC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = TPC_ECUDA;
                if (rc == TPC_OK && r > 0) t.push_back(ms / nl);
            }
            if (rc != TPC_OK) break;
            std::sort(t.begin(), t.end());
            const double per = t[t.size() / 2];
            if (per < best_per * (K > best_k ? 0.99 : 1.0)) {
                best_per = per;
                best_k = K;
                best_tl = tlv;
            }
        }
        ctx->sched.tl_blocks_per_sm = best_tl;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->direct.clear();
        ctx->streams = best_k;
        ctx->next_slot = 0;
        if (rc != TPC_OK) {
            cudaGetLastError();
            ctx->streams = 1;
            ctx->sched = tuned;
            return rc == TPC_ECUDA ? fail(ctx, TPC_ECUDA, "autotune stream timing") : rc;
        }
    }
    for (auto& t : ctx->slots) t->info.done = false;  // the tuning launches' results are not offered
    return out ? tpc_track_get_schedule(ctx, out) : TPC_OK;
}

int tpc_track_get_counters(const tpc_track_ctx* ctx, tpc_track_counters* c)
{
    if (!ctx || !c) return TPC_EINVAL;
    *c = ctx->slots[ctx->last_slot]->info.counters;
    return TPC_OK;
}

void* tpc_track_stream(const tpc_track_ctx* ctx) { return ctx ? (void*)ctx->slots[0]->home : nullptr; }

int tpc_track_debug_dump(tpc_track_ctx* ctx, int stage, void* host_buf, size_t cap, size_t* used)
{
    if (!ctx) return TPC_EINVAL;
    cudaSetDevice(ctx->cfg.device);
    return dump(ctx, *ctx->slots[ctx->last_slot], stage, 0, host_buf, cap, used);
}

int tpc_track_set_debug_waits(tpc_track_ctx* ctx, int64_t spin_limit, int32_t stall_hit_tile)
{
    if (!ctx) return TPC_EINVAL;
    if (spin_limit < 0 || spin_limit > (1LL << 40) || stall_hit_tile < -1)
        return fail(ctx, TPC_EINVAL, "debug wait settings out of range");
    if (!ctx->workers.empty()) return fail(ctx, TPC_EBUSY, "context is serving submitted events");
    ctx->dbg_spin = (long long)spin_limit;
    ctx->dbg_stall = stall_hit_tile + 1;
    return TPC_OK;
}

int tpc_track_debug_dump_event(tpc_track_ctx* ctx, int stage, int event, void* host_buf,
                               size_t cap, size_t* used)
{
    if (!ctx) return TPC_EINVAL;
    cudaSetDevice(ctx->cfg.device);
    return dump(ctx, *ctx->slots[ctx->last_slot], stage, event, host_buf, cap, used);
}

const char* tpc_track_last_error(const tpc_track_ctx* ctx)
{
    if (!ctx) return "NULL context";
    // a copy owned by the calling thread: stays valid while workers report
    thread_local std::string copy;
    std::lock_guard<std::mutex> lk(ctx->err_mu);
    copy = ctx->err;
    return copy.c_str();
}

void tpc_track_destroy(tpc_track_ctx* ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv_req.notify_all();
    for (auto& t : ctx->workers) t.join();
    cudaSetDevice(ctx->cfg.device);
    for (auto& s : ctx->slots) free_slot(*s);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    for (auto& r : ctx->results)
        if (r.second->buf.p) cudaFreeHost(r.second->buf.p);
    for (auto& b : ctx->pool) cudaFreeHost(b.p);
    delete ctx;
}

}  // extern "C"
