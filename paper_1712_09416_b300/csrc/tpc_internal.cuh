// tpc_internal.cuh -- device-side records shared by the tracker's kernels and
// the host orchestrator of libtpctrack.so.  Not part of the public ABI.
//
// Data layout in HBM (one arena per slot, allocated at context creation):
//   inputs      per-event pointers (EventDesc), host inputs staged as SoA
//   rows        (global sector, row) records: counts, offsets, y-z grids;
//               a batch is its events' sectors side by side, so every kernel
//               sees one flat list of sectors
//   hits        sorted by (sector, row, bin, cid): hyz (f32 pairs), hcid (event
//               cid), hrow (sector << 8 | row); bins hold row-local offsets
//   links       up/dn/upc/dnc as int16 row-local indices into the adjacent row,
//               upg the cleaned up link as a global hit index
//   tracklets   one per start hit: header + rowhit[R] (global hit index)
//   outputs     tracks in canonical order, hit cids
#pragma once
#include <cstdint>
#include <vector_types.h>

namespace tpc {

constexpr int kMaxRows = 256;          // pad rows per sector (row index fits 8 bits)
constexpr int kOwnWords = kMaxRows / 32;
constexpr int kMaxRowHits = 4096;      // hits of one (sector,row) handled in shared memory
constexpr int kMaxSectorTracks = 4096; // emitted tracks per sector sorted in shared memory
constexpr int kMaxBinsPerDim = 512;
// y-z bins of a row with cnt hits: max(1, cnt * kBinsPerHitX2 / 2)
constexpr int kBinsPerHitX2 = 4;
constexpr int kMaxRowBins = kMaxRowHits * kBinsPerHitX2 / 2;
// rows up to kSmallRowHits hits are sorted with a small shared-memory
// footprint (more rows in flight); larger rows go to a second pass
constexpr int kSmallRowHits = 1024;
constexpr long long kSpinLimit = 1LL << 22;  // bounded look-back waits
constexpr int kRowTile = 512;    // (sector, row) records per look-back tile of k_rowscan
constexpr int kHitTile = 2048;   // sorted hits per look-back tile of k_clean_starts
// Row counters one per 32-byte sector: the clusters of an event hit a few
// thousand counters with atomics, and counters sharing a sector serialise.
constexpr int kCntPad = 8;

struct EventDesc {
    const float* y;
    const float* z;
    const uint16_t* row;
    const uint16_t* sec;
    long long n;
    long long cl_off;   // first global cluster index of the event
    int sec_base;       // first global sector of the event
    int n_sec;
};

struct RowGrid {        // y-z bin grid of one (sector,row)
    float y0, z0, idy, idz;
    int ny, nz, bin_off, pad;
};

struct TrackletHdr {
    float x, p[5], C[15], chi2;
    int start;          // global sorted index of the chain start h0
    int nhits, first, last, ndf, valid, chain_len;
    int dominated;      // every chain hit taken by other tracklets' forward extensions
};

// Device counters and status, zeroed before every launch.
struct Counters {
    int n_invalid;        // clusters failing the input checks
    int ovf_row;          // a row above kMaxRowHits
    int ovf_tracklets;    // more start hits than tracklet slots
    int ovf_sector;       // more emitted tracks in a sector than kMaxSectorTracks
    int timeout;          // a bounded look-back wait gave up
    int n_links;
    int n_starts;
    int n_tracklets;      // chains long enough for a tracklet
    int n_valid;
    int n_tracklet_hits;
    int n_tracks;
    int n_track_hits;
    int n_bins;
    int ticket_rows, ticket_hits, ticket_sectors;
    int n_crowded;        // hits whose neighbour windows overflow the register lists
    int tl_next;          // work counters of the persistent constructor passes
    int tl_next2;
    int n_dominated;      // chains whose tracklet is not built (dominated)
    int n_bwd;            // chains listed for the backward pass: long forward ranges
    int n_bwd_short;      // ... and short ones (listed from the back of tl_list)
    int n_chain_hits;     // hits on the chains of all start hits
    int n_big_rows;       // rows above kSmallRowHits hits (listed for the large row sort)
    int n_mid_rows;       // rows for the block row sort of k_rowsort
    int mid_next;         // its work counter
    int n_mg_links;       // merger: links between sector tracks
    int n_mg_chains;      // merger: refitted chains of two or more tracks
    int n_mg_tracks;      // merger: tracks after merging
    int max_row_hits;     // high-water marks: hits of the fullest (sector, row)
    int max_sector_tracks;  // ... and emitted tracks of the fullest sector
    int pad[2];
};

// Merger scratch: a sector track's outer state, and the refit of a chain
// stored at its first (innermost) track.
struct MgState {
    float x, p[5], C[15];
    int ok;
};
struct MgFit {
    float x, p[5], C[15], chi2;
    int ndf, ok, nhits, pad;
};

// Everything a kernel needs, passed by value.
struct Launch {
    // sizes
    long long n_total;   // clusters in the launch
    int n_events;
    int R;               // rows per sector
    int S;               // global sectors in the launch
    int RS;              // S * R
    int n_sectors_phi, split_z;
    int t_cap;           // tracklet slots
    // geometry and field
    float tan_half, z_max, kB;   // kB = KAPPA * bz
    // pad-row radii live in device memory (indexing a kernel-parameter array
    // with a lane-dependent row serialises on the constant cache)
    const float* xr;            // [R]
    // parameters
    float sy2, sz2;              // measurement variances
    float slope_win_y, slope_win_z, d_max, chi2_hit, sin_max, edge_margin;
    float seed_var_s, seed_var_t, seed_var_q;
    float sy, sz, seed_sd_s, seed_sd_t, seed_sd_q;  // square roots of the above
    int max_gap, min_chain, min_tracklet_hits, min_track_hits;
    // arena
    EventDesc* ev;              // [n_events]
    long long* ev_off;          // [n_events + 1] cluster offsets
    int* sec_event;             // [S] event of a global sector
    int* row_cnt;               // [RS * kCntPad] hit count of row g at g * kCntPad
    int* ev_invalid;            // [n_events] invalid clusters per event
    int* big_rows;              // [RS] rows for the block row sorts (from the front) and the large row sort (from the back)
    int* row_off;               // [RS + 1]
    RowGrid* grid;              // [RS]
    unsigned long long* tile_state;  // look-back states (rows | hits | sectors)
    int n_row_tiles, n_hit_tiles;
    int* rank;                  // [n_total] arrival rank of a cluster in its row
    float4* tmp_rec;            // row-scattered (y, z, cid bits, unused): one 16-byte store each
    float2* hyz; int* hcid; int* hrow; // sorted (y, z), cid, sector << 8 | row
    int* bin_start;
    int16_t* up; int16_t* dn; int16_t* upc; int16_t* dnc;
    int* upg;                   // [N] cleaned up link, global index or -1
    unsigned long long* weight;
    unsigned char* mark;        // [N] hit taken by a forward extension search (or null)
    int* crowded;               // [N] hits for the chunked neighbour search
    int* starts;                // [t_cap] global sorted index
    TrackletHdr* tl;            // [t_cap]
    int4* tl_chain;             // [t_cap] start hit, its sector << 8 | row, chain end hit, end row
    int* tl_rowhit;             // [t_cap * R] global hit index or -1
    int* tl_list;               // [t_cap] work order of the backward pass: long chains from
                                // the front, short ones from the back (list_at)
    unsigned long long* tl_key; // [t_cap] sector-local sort key or ~0
    int* tl_nown;               // [t_cap]
    unsigned* tl_own;           // [t_cap * kOwnWords] owned-row bits, 32 rows per word from first
    int* tl_out;                // [t_cap] output track index or -1
    int* tl_hitoff;             // [t_cap] output hit offset
    int* sec_first;             // [S] first tracklet of a sector
    int* sec_end;               // [S]
    int* sec_trk_off;           // [S + 1] output track offset of a sector
    int* sec_hit_off;           // [S + 1]
    // outputs
    int* k_sector; float* k_x; float* k_param; float* k_cov; float* k_chi2; int* k_ndf;
    int* k_hit_off; int* k_hit_cid;
    int* k_gsec;                // [t_cap] global sector of an output track
    // sector track merger (run when merge != 0)
    int merge, mg_ring;         // ring: the phi sectors close around the beam axis
    float mg_chi2, mg_dx_lo, mg_dx_hi;
    float mg_cd, mg_sd;         // cos, sin of the angle between neighbouring sectors
    int n_mg_tiles;             // look-back tiles of the compaction (after the sectors')
    MgState* mg_st;             // [t_cap]
    MgFit* mg_fit;              // [t_cap]
    unsigned long long* mg_key; // [t_cap] ~(chi2 bits << 32 | a) of b's best a, 0 = none
    int* mg_best; int* mg_link; int* mg_in; int* mg_absorbed;  // [t_cap]
    int* mg_oidx; int* mg_ohoff;    // [t_cap] output index / hit offset before a track
    float4* mg_hxyz;            // [clusters] (x, y, z) of the hits of linked tracks, as k_hit_cid
    float* mg_xs; int* mg_xi;   // [t_cap] each sector's tracks by ascending x: x, track index
    float4* mg_pre;             // [2 t_cap] the same order: (x, t, q/pT, C33), (C43, C44, index, 0)
    int* m_sector; float* m_x; float* m_param; float* m_cov; float* m_chi2; int* m_ndf;
    int* m_hit_off; int* m_hit_cid; int* m_sec_trk_off; int* m_sec_hit_off;
    Counters* cnt;
    // bounded waits: polls of a look-back before it gives up (0 = kSpinLimit);
    // test hook: 1 + the index of a hit tile whose look-back state is never
    // published, so that the tiles after it give up (0 = none)
    long long spin_limit;
    int stall_hit_tile;
    int pad_dbg;
};

// ---------------------------------------------------------------------------
// ordered prefix across thread blocks (decoupled look-back), one warp calls.
// The 64-bit state holds a 2-bit status (1 aggregate, 2 inclusive) over a
// 62-bit payload; payloads are two packed 31-bit counts (a << 31 | b) whose
// sums never carry.  Waits are bounded; on timeout cnt->timeout is set.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr unsigned long long kPayload = (1ULL << 62) - 1;

__device__ __forceinline__ unsigned long long pack2(unsigned a, unsigned b)
{
    return ((unsigned long long)a << 31) | (unsigned long long)b;
}
__device__ __forceinline__ unsigned unpack_a(unsigned long long v) { return (unsigned)(v >> 31); }
__device__ __forceinline__ unsigned unpack_b(unsigned long long v)
{
    return (unsigned)(v & 0x7FFFFFFFULL);
}

// Called by all 32 lanes of one warp (the same arguments on every lane);
// returns the exclusive prefix of `tile` on every lane.  Each round reads the
// states of the 32 nearest unread predecessors at once (lane j reads tile
// base - j): when every state up to the nearest inclusive one is published,
// their payloads are summed; the walk ends at an inclusive state.  After
// `limit` polls without progress the wait gives up: cnt->timeout is set (the
// kernels after it return at once and the launch reports TPC_ETIMEOUT).
__device__ inline unsigned long long lookback_warp(unsigned long long* state, int tile,
                                                   unsigned long long aggregate, Counters* cnt,
                                                   long long limit, bool stall = false)
{
    const int lane = threadIdx.x & 31;
    if (limit <= 0) limit = kSpinLimit;
    if (stall) return 0;  // test hook: publish nothing, the tiles after this one give up
    if (tile == 0) {
        if (lane == 0) st_release(&state[0], (2ULL << 62) | aggregate);
        return 0;
    }
    if (lane == 0) st_release(&state[tile], (1ULL << 62) | aggregate);
    unsigned long long excl = 0;
    int base = tile - 1;
    long long spins = 0;
    for (;;) {
        const int t = base - lane;
        const unsigned long long v = t >= 0 ? ld_acquire(&state[t]) : (2ULL << 62);
        const unsigned f = (unsigned)(v >> 62);
        const unsigned pm = __ballot_sync(0xffffffffu, f == 2);
        const unsigned zm = __ballot_sync(0xffffffffu, f == 0);
        const int first_p = pm ? __ffs(pm) - 1 : 31;
        const unsigned upto = first_p == 31 ? 0xffffffffu : ((2u << first_p) - 1u);
        if (zm & upto) {
            if (++spins > limit) {
                if (lane == 0) atomicExch(&cnt->timeout, 1);
                break;
            }
            __nanosleep(20);
            continue;
        }
        unsigned long long part = (lane <= first_p) ? (v & kPayload) : 0ULL;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        excl += part;
        if (pm) break;
        base -= 32;
    }
    if (lane == 0) st_release(&state[tile], (2ULL << 62) | (excl + aggregate));
    return excl;
}

// Asynchronous global -> shared copies of one 8- or 4-byte element
// (cp.async, completed by cp_async_wait_all and made visible to the block by
// the barrier after it).
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Bin of a coordinate in a row grid, clamped to the edge bins.  The same
// monotone arithmetic sorts the hits and bounds every window query, so a
// window [lo, hi] maps onto bins [bin(lo), bin(hi)] that hold all its hits.
__device__ __forceinline__ int bin_y(const RowGrid& G, float y)
{
    const int b = (int)floorf((y - G.y0) * G.idy);
    return min(max(b, 0), G.ny - 1);
}
__device__ __forceinline__ int bin_z(const RowGrid& G, float z)
{
    const int b = (int)floorf((z - G.z0) * G.idz);
    return min(max(b, 0), G.nz - 1);
}

// Position i of the backward pass's work order in tl_list (written by
// k_dominance): the n_long chains with long forward ranges first (from the
// front), then the others (from the back); a longest-first hand-out keeps
// fewer lanes idle at the end of the persistent pass.
__device__ __forceinline__ int list_at(const Launch& L, int i, int n_long)
{
    return i < n_long ? L.tl_list[i] : L.tl_list[L.t_cap - 1 - (i - n_long)];
}

// Profiling hook: called on the host right after each kernel is enqueued.
struct KernelHook {
    void (*after)(void* user, const char* name);
    void* user;
};
inline void hook_after(const KernelHook* h, const char* name)
{
    if (h && h->after) h->after(h->user, name);
}

// Launch schedule of the kernels on one device: grid and block shapes that
// do not change the results, only the speed (the autotuner picks them).
struct Schedule {
    int n_sm = 148;            // multiprocessors of the device
    int bin_blocks_per_sm = 4; // k_count / k_scatter grid
    int sort_threads = 512;    // k_rowsort_big block (256 or 512)
    int nb_threads = 128;      // k_neighbours block (64, 128 or 256)
    int tl_blocks_per_sm = 0;  // persistent k_constructor blocks per SM (<= tl_max_per_sm)
    int tl_max_per_sm = 0;     // occupancy limit of k_constructor
    int nb_mode = 0;           // 0 one thread per hit, 1 row blocks with staged rows (same results)
    int nr_max_per_sm = 0;     // occupancy limit of the row-block neighbour kernel
};

// Once per device (current device): kernel attributes and the default
// schedule.  Launchers make no other runtime calls than kernel launches, so
// a launch sequence can be captured into a CUDA graph.
void prepare_kernels(Schedule* s);
void prepare_binning();
void prepare_selector();
void prepare_merger();
int constructor_occupancy();
int neighbour_rows_occupancy();

// host-side launchers (one translation unit each)
void launch_binning(const Launch& L, const Schedule& S, void* stream, const KernelHook* hook);
void launch_finder(const Launch& L, const Schedule& S, void* stream, const KernelHook* hook);
void launch_constructor(const Launch& L, const Schedule& S, void* stream, const KernelHook* hook);
void launch_merger(const Launch& L, const Schedule& S, void* stream, const KernelHook* hook);
constexpr int kMgTile = 1024;  // tracks per look-back tile of the merger's compaction
void launch_selector(const Launch& L, const Schedule& S, void* stream, const KernelHook* hook);

}  // namespace tpc
