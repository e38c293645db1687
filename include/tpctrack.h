/*
 * tpctrack.h -- C ABI of the B300 TPC sector tracker (libtpctrack.so).
 *
 * The library reconstructs particle tracks in the TPC sectors of one or more
 * events: cellular-automaton track finding followed by a Kalman-filter track
 * fit, the two parts of the ALICE HLT TPC tracker (paper, Abstract and
 * Sect. 4).  The tracker consumes the clusters of all TPC links of an event
 * (Sect. 2: the track reconstruction subscribes to all TPC links), events are
 * reconstructed one after another or many at a time (Sect. 2: the chain works
 * as a pipeline with many events in flight), and the tracks with their
 * parameters and covariances feed the calibration (Sect. 3, item 1).  The
 * paper's `FitTracks()` wraps one device launch over all tracks (Sect. 4.1,
 * Listing 2); here every entry point wraps the device pipeline of binning,
 * neighbour finding and cleaning, start hits, tracklet construction and
 * selection, all hand-written CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point:
 *   - Sector frame: x along the pad-row normal (outward), y along the row,
 *     z along the beam.  Pad row r is the plane x = row_x[r].  Sector s_phi
 *     has its centre at alpha = (s_phi + 0.5) * 2 * half_angle.  With split_z
 *     the sectors are doubled at z = 0: sector s_phi + n_sectors_phi holds
 *     z < 0.
 *   - Track state at x: (y, z, sin(phi), tan(lambda), q/pT), with phi the
 *     angle of the momentum to the x axis in the xy plane, lambda the dip
 *     angle, q/pT in (GeV/c)^-1.  Covariance: 15 floats, lower triangle in
 *     row order (C00, C10, C11, C20, C21, C22, ..., C44).
 *   - Cluster id (cid): the index of a cluster in its event's input arrays.
 *   - Every call returns a status code; nothing aborts or prints.  On error
 *     tpc_track_last_error() gives a one-line reason.
 *   - Thread safety: one context is driven by one host thread at a time,
 *     except tpc_track_submit, tpc_track_poll, tpc_track_release,
 *     tpc_track_set_params, tpc_track_get_params, tpc_track_ticket_params
 *     and tpc_track_last_error, which may be called from several threads at
 *     once (a submitting thread and a polling thread, say).
 */
#ifndef TPCTRACK_H
#define TPCTRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    TPC_OK = 0,
    TPC_EINVAL = -1,     /* invalid argument or input cluster (bad row/sector, NaN/Inf) */
    TPC_ENOMEM = -2,     /* device or host allocation failed */
    TPC_ECUDA = -3,      /* a CUDA call failed */
    TPC_ECAPACITY = -4,  /* a device buffer would overflow; no partial result is returned */
    TPC_ETIMEOUT = -5,   /* a bounded device wait gave up */
    TPC_EBUSY = -6       /* served ticket not finished yet */
};

/* Detector geometry.  row_x is host memory, read during the call. */
typedef struct {
    int n_rows;            /* pad rows, 3..256 (159 for the ALICE TPC) */
    const float* row_x;    /* [n_rows] cm, strictly ascending */
    int n_sectors_phi;     /* sectors around phi (18), or 1 for a single wedge */
    int split_z;           /* 1: sectors doubled at the z = 0 membrane */
    float half_angle_rad;  /* half opening of a sector (10 deg) */
    float z_max;           /* drift length, cm (250) */
} tpc_geometry;

/* One event's clusters, structure of arrays.  With on_device = 1 the four
 * pointers are device pointers on the context's device (e.g. a torch
 * tensor's data_ptr); otherwise host memory (pinned memory gives the fastest
 * copies).  The caller keeps them valid for the duration of the call (for
 * tpc_track_launch: until tpc_track_results returns; for tpc_track_submit:
 * until tpc_track_poll has returned TPC_OK for the ticket). */
typedef struct {
    int64_t n;
    const float* y;           /* [n] cm, sector frame */
    const float* z;           /* [n] cm */
    const uint16_t* row;      /* [n] pad row, < n_rows */
    const uint16_t* sector;   /* [n] sector, < n_sectors_phi * (split_z ? 2 : 1) */
    int on_device;
} tpc_clusters;

/* Reconstructed tracks of one event, ordered by (sector, row of the first
 * hit, cid of the start hit).  All arrays are host memory owned by the
 * context, valid until the next tpc_track_event / tpc_track_batch /
 * tpc_track_results call on the context, or for served tickets until
 * tpc_track_release(ticket). */
typedef struct {
    int64_t n_tracks;
    const int32_t* sector;    /* [n_tracks] */
    const float* x;           /* [n_tracks] cm, plane of the innermost tracklet hit */
    const float* param;       /* [n_tracks][5] state at x */
    const float* cov;         /* [n_tracks][15] */
    const float* chi2;        /* [n_tracks] */
    const int32_t* ndf;       /* [n_tracks] 2 * (tracklet hits) - 5 */
    const int32_t* hit_off;   /* [n_tracks + 1] offsets into hit_cid */
    const int32_t* hit_cid;   /* input cluster indices, ascending row within a track */
} tpc_tracks;

/* Tracker parameters; tpc_track_default_params() fills the defaults. */
typedef struct {
    float meas_sigma_y, meas_sigma_z;  /* cluster errors, cm (0.1, 0.1) */
    float slope_win_y, slope_win_z;    /* neighbour windows |dy| <= w |dx| (2.0, 2.0) */
    float d_max;                       /* neighbour kink cut (0.6) */
    float chi2_hit;                    /* searched-hit chi2 cut (16) */
    int max_gap;                       /* consecutive missed rows ending a search (5) */
    int min_chain;                     /* hits of a chain to build a tracklet (3) */
    int min_tracklet_hits;             /* hits of a valid tracklet (10) */
    int min_track_hits;                /* owned hits of an emitted track (10) */
    float sin_max;                     /* transport fails at |sin phi| >= sin_max (0.99) */
    float edge_margin;                 /* cm beyond the sector edge ending a search (2) */
    float seed_var_s;                  /* seed variance of the slope dy/dx (1); sin(phi) gets it x cos^6(phi) */
    float seed_var_t;                  /* seed variance of the slope dz/dx (1); tan(lambda) gets it x cos^2(phi) */
    float seed_var_q;                  /* seed variance of q/pT (100) */
    /* Sector track merger and global refit (0 = off, the default).  With
     * merge = 1 the tracks of neighbouring phi sectors (same z half) and of
     * the two halves of one phi sector are joined where one continues the
     * other, and each joined chain is refitted over all its hits:
     *   - a track's state is carried to its outermost hit, turned into the
     *     other sector's frame and carried to the other track's state;
     *   - the pair is admissible if the gap between the two (along x of the
     *     outer track's frame) lies in [merge_dx_lo, merge_dx_hi] cm and the
     *     5-parameter chi2 of the two states is <= merge_chi2;
     *   - tracks are linked when each is the other's admissible partner of
     *     least chi2; a chain (of any length) is refitted from its
     *     outermost hit inward (Kalman filter, frames turned between tracks).
     * A merged track takes the place (and sector) of its innermost track;
     * its state is at the innermost hit, ndf = 2 * hits - 5, and its hit list
     * is the tracks' lists, innermost track first.  Tracks not merged are
     * unchanged. */
    int merge;
    float merge_chi2;                  /* (30) */
    float merge_dx_lo, merge_dx_hi;    /* (-5, 30) cm */
} tpc_track_params;

/* Context configuration. */
typedef struct {
    int device;                       /* CUDA device ordinal */
    size_t mem_budget;                /* bytes of device memory the context may hold; 0 = derive */
    int64_t max_clusters_per_event;   /* capacity of one launch (sum over a batch), > 0 */
    int max_events_in_flight;         /* served slots (device arenas); >= 1 */
    void* cuda_stream;                /* cudaStream_t for the launches, NULL = own stream */
    int max_rows;                     /* largest n_rows of any geometry used (0 = 159) */
    int max_events_per_launch;        /* events in one batch launch (0 = 64), <= 1024 */
    tpc_track_params params;
} tpc_track_config;

typedef struct tpc_track_ctx tpc_track_ctx;

/* Fill p with the default parameters listed above. */
void tpc_track_default_params(tpc_track_params* p);

/* Create a context: allocates every device arena up front (no allocation
 * happens on the tracking path).  Passage: the tracker is one component
 * instance of the chain that processes one event after another (Sect. 2);
 * the context is that instance's state on one GPU.  Returns TPC_EINVAL for a bad config,
 * TPC_ENOMEM if the arenas do not fit the device or mem_budget, TPC_ECUDA
 * for other CUDA failures.  *out is NULL on failure. */
int tpc_track_create(const tpc_track_config* cfg, tpc_track_ctx** out);

/* Track one event: stage inputs (host->device copy unless on_device), run
 * the device pipeline, copy the tracks back.  Blocks until done.  Passage:
 * the tracker takes the clusters of all TPC links of one event (Sect. 2) and
 * finds tracks with a cellular automaton and fits them with a Kalman filter
 * (Abstract); the call wraps the device launch the way FitTracks() wraps
 * FitTracksGPU (Sect. 4.1, Listings 2-3).  Inputs are
 * checked on the device before any result is produced: an invalid cluster
 * gives TPC_EINVAL, an overflow TPC_ECAPACITY; in both cases out->n_tracks = 0. */
int tpc_track_event(tpc_track_ctx* ctx, const tpc_clusters* ev, const tpc_geometry* geom,
                    float bz_tesla, tpc_tracks* out);

/* Track n_ev events in one device pass (sectors of all events side by side,
 * one launch per stage).  Passage: many events are in flight in the chain at
 * once (Sect. 2) and different kernels run concurrently (Sect. 4.2, last
 * paragraph); a batch fills the GPU with the work of many events.  outs[i] receives event i.  The cluster counts
 * summed over the batch must not exceed max_clusters_per_event.  Each
 * event's tracks are identical to those of tpc_track_event on it alone. */
int tpc_track_batch(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev,
                    const tpc_geometry* geom, float bz_tesla, tpc_tracks* outs);

/* Asynchronous form of tpc_track_batch: enqueue the device pipeline and
 * return.  With host inputs the copies are enqueued too (the inputs must
 * stay valid until tpc_track_results).  The tracks stay in device memory
 * until tpc_track_results, which waits for the oldest launch not yet
 * collected, checks its device status and copies its tracks out.
 * With the schedule's streams = 1 (the default) every launch runs on the
 * context's stream and a launch first discards the results of a pending
 * one.  With streams = K > 1, consecutive launches go to K slots in turn,
 * each on a stream of its own, so that the kernels of up to K launches run
 * concurrently (Sect. 4.2: several different kernels in parallel); each
 * launch starts after the work enqueued on the context's stream before the
 * call (inputs written there are seen), a launch discards the uncollected
 * results of the launch K before it (same slot), and the context's stream
 * does not wait for the launches until tpc_track_join.  While profiling is on
 * (tpc_track_set_profiling), launches run one at a time on the context's
 * stream.  tpc_track_batch drops every uncollected launch first.
 * tpc_track_results writes one tpc_tracks per event of the collected launch
 * into outs[0 .. cap-1]: a launch of more than cap events returns TPC_EINVAL
 * and stays pending (outs may be NULL with any cap, to collect the status
 * only). */
int tpc_track_launch(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev,
                     const tpc_geometry* geom, float bz_tesla);
int tpc_track_results(tpc_track_ctx* ctx, int cap, tpc_tracks* outs);

/* Make the context's stream wait for every launch enqueued so far (on all
 * slots); never blocks the host.  Work the caller enqueues on the context's
 * stream afterwards (a timing event, a copy of inputs into reused buffers)
 * runs after those launches. */
int tpc_track_join(tpc_track_ctx* ctx);

/* Served form: queue one event.  Passage: events arrive one after another
 * and a component must keep up without its input queue filling (Sect. 2,
 * Sect. 3 item 4, Fig. 4); continuous batching over slots keeps several
 * events in flight.  Every slot (a device arena, all of them
 * allocated at creation within mem_budget) has a worker thread that takes
 * the queued events, as many as fit the slot, into its next launch;
 * launches on different slots overlap on the device.  The caller's input
 * buffers must stay valid until the ticket is polled done.  An event with
 * invalid clusters fails its own ticket (TPC_EINVAL) and no other.  *ticket
 * identifies the request.  Returns TPC_EINVAL for an event larger than one
 * slot. */
int tpc_track_submit(tpc_track_ctx* ctx, const tpc_clusters* ev, const tpc_geometry* geom,
                     float bz_tesla, uint64_t* ticket);

/* Wait up to timeout_us (0 = just test, < 0 = forever) for a ticket.
 * Passage: the consumer checks for finished work at each event without
 * waiting (Sect. 5.1, the asynchronous pattern of Fig. 5).
 * TPC_OK fills *out (valid until tpc_track_release); TPC_EBUSY if not done;
 * the ticket's own error code if its launch failed. */
int tpc_track_poll(tpc_track_ctx* ctx, uint64_t ticket, int timeout_us, tpc_tracks* out);

/* Free the host memory of a finished ticket (the ticket's results are the
 * tracks handed on to calibration, Sect. 3; the caller keeps them until this
 * call). */
int tpc_track_release(tpc_track_ctx* ctx, uint64_t ticket);

/* Event-synchronous parameter updates (Sect. 3, item 2; Sect. 5.2, 5.3: new
 * calibration data enter the chain in step with an event, and it is known
 * which event was processed with which data).
 *
 * tpc_track_set_params makes *p the context's parameter set (the same range
 * checks as tpc_track_create; TPC_EINVAL leaves the current set).  Every
 * event submitted afterwards, and every later direct call, uses it; events
 * already submitted keep the set they were submitted with, and no launch mixes
 * two sets.  *first_ticket (may be NULL) receives the first ticket tracked
 * with the new set, *version (may be NULL) its version number (the count of
 * tpc_track_set_params calls on the context; 0 is the creation set).
 * tpc_track_get_params returns the current set and its version.
 * tpc_track_ticket_params returns the set and version a submitted ticket is
 * tracked with (until the ticket is released), for reproducing the event. */
int tpc_track_set_params(tpc_track_ctx* ctx, const tpc_track_params* p, uint64_t* first_ticket,
                         uint64_t* version);
int tpc_track_get_params(tpc_track_ctx* ctx, tpc_track_params* p, uint64_t* version);
int tpc_track_ticket_params(tpc_track_ctx* ctx, uint64_t ticket, tpc_track_params* p,
                            uint64_t* version);

/* Asynchronous long-running side tasks (Sect. 3, item 4; Sect. 5.1).
 *
 * A runner owns one host thread.  It calls init(user) once on that thread
 * before any job (init may be NULL; a non-zero return is returned by
 * tpc_async_create, which then creates nothing), then run(user, job, &result)
 * for every started job, one at a time, in start order.  The event loop
 * starts a job while processing an event and checks at every event whether a
 * job has finished, so no event waits for the job (the event queue does not
 * fill up behind a long fit: Fig. 4 against Fig. 5).
 *   tpc_async_create   max_unfinished (1..1024) bounds the jobs started and
 *                      not yet finished; drop (may be NULL) is called by
 *                      tpc_async_destroy with (user, job, NULL) for every job
 *                      never run and (user, NULL, result) for every result
 *                      never polled, so that their memory can be freed.
 *   tpc_async_start    queues job (owned by the runner until run returns)
 *                      and never waits: TPC_EBUSY when max_unfinished jobs
 *                      are unfinished.  *task (may be NULL) gets its id
 *                      (1, 2, ... in start order).
 *   tpc_async_poll     the oldest finished job not yet polled: its id, the
 *                      result pointer run produced (now the caller's) and the
 *                      status run returned.  Waits up to timeout_us (0 = just
 *                      test; < 0 = while any job is queued or running).
 *                      TPC_EBUSY if none has finished.
 *   tpc_async_destroy  lets the running job finish (jobs are not cancelled),
 *                      runs no queued job, joins the thread.
 * Every function may be called from any thread; one runner's jobs never run
 * concurrently with each other. */
typedef struct tpc_async tpc_async;
typedef int (*tpc_async_init_fn)(void* user);
typedef int (*tpc_async_run_fn)(void* user, void* job, void** result);
typedef void (*tpc_async_drop_fn)(void* user, void* job, void* result);
typedef struct {
    int64_t started, finished, refused;  /* refused: tpc_async_start returned TPC_EBUSY */
    int64_t queued, running, unpolled;   /* now */
    double busy_ms, max_task_ms;         /* summed and longest run time of finished jobs */
} tpc_async_stats;
int tpc_async_create(tpc_async_init_fn init, tpc_async_run_fn run, tpc_async_drop_fn drop,
                     void* user, int max_unfinished, tpc_async** out);
int tpc_async_start(tpc_async* a, void* job, uint64_t* task);
int tpc_async_poll(tpc_async* a, int timeout_us, uint64_t* task, void** result, int* task_status);
int tpc_async_get_stats(tpc_async* a, tpc_async_stats* out);
void tpc_async_destroy(tpc_async* a);

/* Built-in accumulate-then-fit side task: the chi^2 scale of the tracks.
 * tpc_chi2_calib_add (called once per event, never waits) appends the chi2
 * and ndf of the event's tracks with ndf > 0 (of *t it reads n_tracks, chi2
 * and ndf only); once every_n_events events
 * tracked with one parameter version have been added it hands them to its
 * runner's thread as one fit (if max_unfinished fits are still unfinished it
 * keeps accumulating and tries again at the next event).  Adding an event of
 * another parameter version drops the partial accumulation: every fit covers
 * events tracked with one parameter set.  Events are numbered 0, 1, ... in
 * the order added.
 * The fit: s2 = sum chi2 / sum ndf over all tracks; then repeatedly keep the
 * tracks with chi2 <= trim * s2 * ndf and set s2 = sum chi2 / sum ndf over the
 * kept ones, until the kept set repeats (at most 100 rounds).  s2 estimates
 * (true cluster error / assumed cluster error)^2 when the assumed error is
 * wrong, so sigma * sqrt(s2) is the corrected cluster error to feed back
 * with tpc_track_set_params.  trim > 1.  A fit of no track gives s2 = NaN.
 * tpc_chi2_calib_poll returns the oldest finished fit as tpc_async_poll does. */
typedef struct tpc_chi2_calib tpc_chi2_calib;
typedef struct {
    uint64_t first_event, last_event, n_events, params_version;
    int64_t n_tracks, n_kept;
    int32_t n_iter, pad;
    double scale2;
} tpc_chi2_fit;
int tpc_chi2_calib_create(int every_n_events, double trim, int max_unfinished,
                          tpc_chi2_calib** out);
int tpc_chi2_calib_add(tpc_chi2_calib* c, const tpc_tracks* t, uint64_t params_version);
int tpc_chi2_calib_poll(tpc_chi2_calib* c, int timeout_us, tpc_chi2_fit* out);
int tpc_chi2_calib_stats(tpc_chi2_calib* c, tpc_async_stats* out);
void tpc_chi2_calib_destroy(tpc_chi2_calib* c);

/* Per-launch counters of the last tpc_track_results (for the byte model
 * of the benchmark and for tests).  n_chain_hits is the number of hits on
 * the chains of all start hits (every start hit included); n_tracklets
 * counts the chains that got a tracklet, n_dominated_chains those that did
 * not because other tracklets' forward extensions took all their hits. */
typedef struct {
    int64_t n_clusters, n_rows_total, n_bins, n_links, n_starts, n_tracklets,
            n_valid_tracklets, n_tracklet_hits, n_tracks, n_track_hits, n_chain_hits;
    int64_t n_dominated_chains;
    int64_t n_merge_links, n_merge_chains;  /* merger: links, refitted chains (0 without merge) */
    int64_t n_sector_tracks;                /* tracks before merging (= n_tracks without merge) */
    int64_t max_row_hits;       /* high-water marks: clusters of the fullest (sector, row) of the */
    int64_t max_sector_tracks;  /* launch and tracks of its fullest sector (each limited to 4096) */
    int64_t n_crowded_hits;     /* hits whose neighbour windows held more than four candidates a side */
} tpc_track_counters;
int tpc_track_get_counters(const tpc_track_ctx* ctx, tpc_track_counters* c);

/* Stream the context launches on (a cudaStream_t). */
void* tpc_track_stream(const tpc_track_ctx* ctx);

/* Kernel timing for benchmarks.  tpc_track_set_profiling(ctx, 1) waits for
 * the context's stream, clears the record, and makes every later direct
 * launch record a CUDA event after each of its kernels on the launch stream
 * (0 turns it off).  tpc_track_kernel_times waits for the stream and writes,
 * per kernel name in launch order, the summed device time and the number of
 * launches recorded (up to cap entries; *n receives the count). */
typedef struct {
    char name[32];
    double total_ms;
    int64_t launches;
} tpc_kernel_time;
int tpc_track_set_profiling(tpc_track_ctx* ctx, int on);
int tpc_track_kernel_times(tpc_track_ctx* ctx, tpc_kernel_time* out, int cap, int* n);

/* Launch schedule: grid and block shapes of the kernels.  It changes the
 * speed only, never the results.  n_sm and tl_max_per_sm describe the device
 * and the constructor's occupancy limit (read-only); the others are:
 *   bin_blocks_per_sm  blocks per SM of the count and scatter kernels (1..32)
 *   sort_threads       threads of a block of the large-row sort (rows above 1024 hits; 256 or 512)
 *   nb_threads         threads of a neighbour-finder block (64, 128 or 256)
 *   tl_blocks_per_sm   persistent constructor blocks per SM (1..tl_max_per_sm)
 *   streams            slots that consecutive direct launches go to in turn,
 *                      each on its own stream (1..max_streams, the context's
 *                      max_events_in_flight; see tpc_track_launch)
 *   nb_mode            neighbour finder: 0 one thread per hit, 1 one block
 *                      per pad row with the two adjacent rows staged in
 *                      shared memory; both give the same links
 * tpc_track_set_schedule rejects other values with TPC_EINVAL and returns
 * TPC_EBUSY while the context serves submitted events. */
typedef struct {
    int n_sm, tl_max_per_sm;
    int bin_blocks_per_sm, sort_threads, nb_threads, tl_blocks_per_sm;
    int max_streams, streams;
    int nb_mode;
} tpc_track_schedule;
int tpc_track_get_schedule(const tpc_track_ctx* ctx, tpc_track_schedule* out);
int tpc_track_set_schedule(tpc_track_ctx* ctx, const tpc_track_schedule* s);

/* Autotuner: runs the launch of n_ev events (arguments as for
 * tpc_track_batch) with each candidate value of every schedule field, reps
 * times each (1..50), times the kernel that the field shapes with CUDA
 * events, and keeps the fastest value per field (fields shape different
 * kernels, so they are tuned one after the other).  Last it times rounds
 * (at least 7) of 8K back-to-back launches spread over K = 1, 2, 3, 4, 6, 8
 * streams (up to max_streams)
 * (from the context's stream to tpc_track_join), for K > 1 with each of the
 * constructor block counts tried before (launches running together share the
 * SMs), and takes the pair with the shortest time per launch (a larger K
 * must win by 1%).  Writes the chosen
 * schedule to *out (may be NULL) and makes it the context's schedule.  The
 * results of the tuning launches are discarded.  Same errors as
 * tpc_track_batch, TPC_EBUSY while serving submitted events. */
int tpc_track_autotune(tpc_track_ctx* ctx, int n_ev, const tpc_clusters* ev,
                       const tpc_geometry* geom, float bz_tesla, int reps,
                       tpc_track_schedule* out);

/* Debug dump of an intermediate stage of event 0 of the last completed
 * launch, for parity tests.  Passage: the paper checks its device code by
 * running the same algorithm on the CPU and comparing (one common source
 * for CPU and GPU, Sect. 4.1); here every stage is compared with the
 * independent CPU oracle.  Writes at most cap bytes to host_buf and the
 * size needed to *used (call with cap = 0 to query).  Stages:
 *   TPC_DUMP_LINKS      int32 [2][n]: up, down link as cid (or -1), by cid
 *   TPC_DUMP_CLEAN      int32 [2][n]: links after cleaning, by cid
 *   TPC_DUMP_STARTS     int32 [n_starts]: start-hit cids, ascending
 *   TPC_DUMP_TRACKLETS  int32 count, then count records of
 *                       tpc_dump_tracklet followed by int32 rowhit[n_rows]
 *                       (cid or -1), ordered by start cid
 *   TPC_DUMP_WEIGHTS    uint64 [n]: hit weight by cid (0 = none)
 *   TPC_DUMP_SORTED     int32 [n]: cids in the device's (sector, row, bin) order
 * Returns TPC_EINVAL for an unknown stage or no completed launch. */
enum { TPC_DUMP_LINKS = 1, TPC_DUMP_CLEAN = 2, TPC_DUMP_STARTS = 3, TPC_DUMP_TRACKLETS = 4,
       TPC_DUMP_WEIGHTS = 5, TPC_DUMP_SORTED = 6 };
typedef struct {
    int32_t start_cid, sector, valid, nhits, first_row, last_row, ndf, pad;
    float x, param[5], cov[15], chi2;
} tpc_dump_tracklet;
int tpc_track_debug_dump(tpc_track_ctx* ctx, int stage, void* host_buf, size_t cap,
                         size_t* used);

/* Test hook of the bounded device waits (the decoupled look-back scans that
 * order binning, start hits, the selector's output and the merger's output
 * wait on their predecessor tiles; a component that stalls must not stall
 * the event stream, paper Sect. 3 item 4 and Sect. 5.1).  For the launches
 * that follow on this context: a wait gives up after spin_limit polls
 * (0 = the default, 2^22), and with stall_hit_tile >= 0 the hit tile of that
 * index (tiles of 2048 sorted hits in the start-hit compaction) never
 * publishes its state, so that every tile after it gives up.  A launch whose
 * wait gave up runs none of its later kernels and fails with TPC_ETIMEOUT and
 * no result; the context stays usable.  (0, -1) restores normal launches.
 * TPC_EINVAL for spin_limit outside [0, 2^40] or stall_hit_tile < -1,
 * TPC_EBUSY while the context serves submitted events. */
int tpc_track_set_debug_waits(tpc_track_ctx* ctx, int64_t spin_limit, int32_t stall_hit_tile);

/* The same dump for event `event` (0 .. n_ev - 1) of the last completed
 * launch, so that each event of a batch can be compared stage by stage; cids,
 * rows and sectors are those of that event.  TPC_EINVAL for an event index
 * outside the launch. */
int tpc_track_debug_dump_event(tpc_track_ctx* ctx, int stage, int event, void* host_buf,
                               size_t cap, size_t* used);

/* Neighbour links of one event without any allocation (this entry point has
 * no counterpart in the paper; it serves callers that cannot allocate device
 * memory: code running inside a framework that owns the device allocator,
 * code under a hard memory budget where a cudaMalloc may fail at any moment,
 * and callers that must avoid the device-wide synchronisation cudaMalloc and
 * cudaFree can imply).  It runs the tracker's binning and neighbour-finding
 * kernels on ev's clusters and writes, for every cluster id c, the cid of its
 * up and down neighbour (or -1) to up_cid[c] and dn_cid[c]: the same links as
 * TPC_DUMP_LINKS after tpc_track_event.
 *   ev        device clusters (on_device must be 1), at most 131072 of them;
 *             more gives TPC_EINVAL before any device work
 *   geom      as for tpc_track_event, at most 36 sectors in total
 *   params    slope windows and d_max are used
 *   up_cid, dn_cid  device arrays of ev->n int32 each, written by the call
 *   cuda_stream     stream for the work (NULL = legacy default stream)
 * Scratch memory is a static device array of this library, about 11.2 MB,
 * held on every device that loads the library until the process exits.  No
 * context, cudaMalloc or cudaFree is involved.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that
 * device current) and sets up the kernels.  Every call copies its small
 * descriptor from the host and synchronises cuda_stream before it returns
 * (it reads the status back), so no call can be made while that stream is
 * being captured into a CUDA graph.  Every call on a device shares the array
 * and clears what must start at zero, so calls whose work overlaps on the
 * GPU (other threads, other streams) race: serialise them.  Returns after the
 * work has completed: TPC_OK, TPC_EINVAL (bad argument or invalid cluster),
 * TPC_ECAPACITY (a row above 4096 clusters), TPC_ETIMEOUT or TPC_ECUDA (also
 * when a launch error from earlier work is pending on the calling thread; it
 * is left pending). */
int tpc_track_links_noalloc(const tpc_clusters* ev, const tpc_geometry* geom,
                            const tpc_track_params* params, int32_t* up_cid, int32_t* dn_cid,
                            void* cuda_stream);

/* ------------------------------------------------------------------------
 * Round-robin dispatcher over tracker instances.  The paper runs several
 * instances of a component and hands them whole events in turn to balance
 * the load (Sect. 2); events are independent, so the instances exchange
 * nothing.  An instance is any object with these three calls (with the
 * meaning of tpc_track_submit / poll / release); tpc_dispatch_create makes
 * one tracker context per listed device and uses those.
 * ------------------------------------------------------------------------ */
typedef struct {
    int (*submit)(void* instance, const tpc_clusters* ev, const tpc_geometry* geom,
                  float bz_tesla, uint64_t* ticket);
    int (*poll)(void* instance, uint64_t ticket, int timeout_us, tpc_tracks* out);
    int (*release)(void* instance, uint64_t ticket);
} tpc_instance_ops;

typedef struct tpc_dispatch tpc_dispatch;

/* One context per entry of devices[n_dev] (a device may be listed more than
 * once), each created with *cfg (device and cuda_stream replaced), owned and
 * destroyed by the dispatcher.  Errors of tpc_track_create are returned;
 * nothing is left allocated then. */
int tpc_dispatch_create(const int* devices, int n_dev, const tpc_track_config* cfg,
                        tpc_dispatch** out);

/* A dispatcher over n caller-owned instances (1..1024) driven through ops;
 * the instances must outlive the dispatcher.  TPC_EINVAL for a NULL call or
 * instance. */
int tpc_dispatch_create_custom(const tpc_instance_ops* ops, void* const* instances, int n,
                               tpc_dispatch** out);

/* Hand one event to the next healthy instance in turn.  *ticket numbers the
 * events 1, 2, ... in submission order.  The caller keeps ev's buffers (and
 * geom's row_x) valid until the ticket is released: an event is submitted
 * again to another instance when the one holding it fails.  An instance whose
 * submit, or a later poll of one of its tickets, fails with TPC_ECUDA,
 * TPC_ETIMEOUT or TPC_ENOMEM leaves the rotation and its events go to the
 * others; any other error (TPC_EINVAL: the event's own invalid clusters)
 * fails that ticket only.  TPC_ECUDA when no healthy instance is left. */
int tpc_dispatch_submit(tpc_dispatch* d, const tpc_clusters* ev, const tpc_geometry* geom,
                        float bz_tesla, uint64_t* ticket);

/* Wait up to timeout_us for a ticket (as tpc_track_poll); *out stays valid
 * until tpc_dispatch_release.  Tickets may be polled in any order and from
 * several threads. */
int tpc_dispatch_poll(tpc_dispatch* d, uint64_t ticket, int timeout_us, tpc_tracks* out);

/* Release a ticket's results (and the caller's input buffers). */
int tpc_dispatch_release(tpc_dispatch* d, uint64_t ticket);

/* Take an instance out of the rotation as if it had failed (host-side fault
 * injection for tests and for an operator who drains a device); its
 * unreleased events not yet polled go to the other instances. */
int tpc_dispatch_fail_instance(tpc_dispatch* d, int instance);

/* Events submitted to each instance (re-issued ones included), whether it is
 * healthy, and the number of re-issued events; returns the instance count. */
int tpc_dispatch_stats(tpc_dispatch* d, int cap, int64_t* events_per_instance,
                       int32_t* healthy, int64_t* reissued);

/* Release everything; contexts made by tpc_dispatch_create are destroyed. */
void tpc_dispatch_destroy(tpc_dispatch* d);

/* One-line description of the last error on the context (never NULL).  The
 * string belongs to the calling thread and stays valid until its next call
 * of tpc_track_last_error. */
const char* tpc_track_last_error(const tpc_track_ctx* ctx);

/* Release every resource of the context (waits for its device work). */
void tpc_track_destroy(tpc_track_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TPCTRACK_H */
