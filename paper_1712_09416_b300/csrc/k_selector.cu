// k_selector.cu -- shared-hit resolution and output of the tracks.
//
// A hit belongs to the valid tracklet with the largest weight key
// (nHits << 32 | ~cid(h0)), which the constructor left in weight[] with
// atomicMax.  A tracklet becomes a track when it owns at least
// min_track_hits hits and at least half of its hits; the track keeps the
// owned hits and the tracklet's parameters.  Tracks are emitted in the order
// (sector, row of the first owned hit, cid of h0).
//   k_sel_decide  one warp per tracklet: owned hits (kept as one bit per
//                 row), decision, sort key; also marks the tracklet range of
//                 every sector (tracklets are ordered by sector because start
//                 hits are)
//   k_sel_sort    one block per sector, in sector order: compacts the
//                 emitted tracklets, sorts their keys in shared memory (rank
//                 sort up to 2048 keys, else bitonic), scans their hit counts and takes
//                 the sector's output offsets from a decoupled look-back
//   k_sel_write   one warp per emitted tracklet: header and owned hit cids
//                 (from the owned-row bits, no second read of the weights)
// Bytes per cluster: rowhit 2 + weight 8 per assigned hit (decide), about
// 100 B per track header and 4 B per output hit (write).
#include <cuda_runtime.h>

#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr unsigned long long kNone = ~0ULL;

// Two parts in one kernel.  One thread per tracklet slot: the tracklet
// range of every sector (slots are ordered by sector because start hits
// are; the sector comes from the chain record), and the "no track" result
// of every slot without a valid tracklet.  One warp per valid tracklet
// (those of the backward pass's list), lanes over its rows: owned hits,
// decision, sort key.  The two parts write disjoint slots.
__global__ void k_sel_decide(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int n_long = L.cnt->n_bwd;
    const int n_list = min(n_long + L.cnt->n_bwd_short, L.t_cap);
    const int lane = threadIdx.x & 31;
    const int threads = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_st; t += threads) {
        const int gs = L.tl_chain[t].y >> 8;
        if (t == 0 || (L.tl_chain[t - 1].y >> 8) != gs) L.sec_first[gs] = t;
        if (t == n_st - 1 || (L.tl_chain[t + 1].y >> 8) != gs) L.sec_end[gs] = t + 1;
        if (!L.tl[t].valid) {
            L.tl_key[t] = kNone;
            L.tl_nown[t] = 0;
            L.tl_out[t] = -1;
        }
    }
    const int warps = threads >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_list; i += warps) {
        const int t = list_at(L, i, n_long);
        const TrackletHdr& H = L.tl[t];
        if (!H.valid) continue;
        unsigned long long out = kNone;
        int nown = 0;
        const unsigned long long key = ((unsigned long long)H.nhits << 32) |
                                       (unsigned long long)(0xFFFFFFFFu - (unsigned)L.hcid[H.start]);
        const int* rowhit = L.tl_rowhit + (size_t)t * L.R;
        int first_own = -1;
        for (int r0 = H.first; r0 <= H.last; r0 += 32) {
            const int r = r0 + lane;
            bool own = false;
            if (r <= H.last) {
                const int h = rowhit[r];
                own = h >= 0 && L.weight[h] == key;
            }
            const unsigned b = __ballot_sync(0xffffffffu, own);
            if (lane == 0) L.tl_own[(size_t)t * kOwnWords + (r0 - H.first) / 32] = b;
            if (b && first_own < 0) first_own = r0 + __ffs(b) - 1;
            nown += __popc(b);
        }
        if (nown >= L.min_track_hits && 2 * nown >= H.nhits)
            out = ((unsigned long long)first_own << 32) | (unsigned long long)(unsigned)L.hcid[H.start];
        if (lane == 0) {
            L.tl_key[t] = out;
            L.tl_nown[t] = nown;
            L.tl_out[t] = -1;
        }
    }
}

constexpr int kSortThreads = 512;
// sectors with at most this many emitted tracks are rank-sorted
constexpr int kRankSortMax = kMaxSectorTracks / 2;

__global__ void __launch_bounds__(kSortThreads) k_sel_sort(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ unsigned long long keys[];         // [kMaxSectorTracks]
    int* idx = reinterpret_cast<int*>(keys + kMaxSectorTracks);  // [kMaxSectorTracks]
    __shared__ int m_s, tile_s;
    __shared__ unsigned long long prefix_s;
    __shared__ int warp_sum[kSortThreads / 32];
    if (threadIdx.x == 0) {
        tile_s = atomicAdd(&L.cnt->ticket_sectors, 1);
        m_s = 0;
    }
    __syncthreads();
    const int g = tile_s;  // sectors are processed in ticket order
    const int t0 = L.sec_first[g], t1 = L.sec_end[g];
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const unsigned long long k = L.tl_key[t];
        if (k != kNone) {
            const int pos = atomicAdd(&m_s, 1);
            if (pos < kMaxSectorTracks) {
                keys[pos] = k;
                idx[pos] = t;
            }
        }
    }
    __syncthreads();
    int m = m_s;
    if (threadIdx.x == 0 && m > 0) atomicMax(&L.cnt->max_sector_tracks, m);
    if (m > kMaxSectorTracks) {
        if (threadIdx.x == 0) atomicExch(&L.cnt->ovf_sector, 1);
        m = kMaxSectorTracks;
    }
    if (m <= kRankSortMax) {
        // rank sort (keys are unique): the rank of a key is the number of
        // smaller keys; the sorted copy goes to the upper half and back
        unsigned long long* k2 = keys + kRankSortMax;
        int* i2 = idx + kRankSortMax;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const unsigned long long a = keys[i];
            int rank = 0;
            for (int j = 0; j < m; ++j) rank += keys[j] < a ? 1 : 0;
            k2[rank] = a;
            i2[rank] = idx[i];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            keys[i] = k2[i];
            idx[i] = i2[i];
        }
        __syncthreads();
    }
    int P = 1;
    while (P < m) P <<= 1;
    if (m <= kRankSortMax) P = 1;  // sorted already: no bitonic stage runs
    for (int i = m + threadIdx.x; i < P; i += blockDim.x) {
        keys[i] = kNone;
        idx[i] = -1;
    }
    __syncthreads();
    // bitonic sort, ascending keys (unique)
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = keys[i], b = keys[l];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                        const int ti = idx[i];
                        idx[i] = idx[l];
                        idx[l] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    // hit offsets: each thread handles a contiguous chunk of the sorted tracks
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int lo = min(m, (int)threadIdx.x * per), hi = min(m, lo + per);
    int hsum = 0;
    for (int i = lo; i < hi; ++i) hsum += L.tl_nown[idx[i]];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = hsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        int run = 0;
        if (threadIdx.x == 0) {
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const int v = warp_sum[w];
                warp_sum[w] = run;
                run += v;
            }
        }
        run = __shfl_sync(0xffffffffu, run, 0);
        const unsigned long long p = lookback_warp(L.tile_state + L.n_row_tiles + L.n_hit_tiles,
                                                   g, pack2((unsigned)m, (unsigned)run), L.cnt,
                                                   L.spin_limit);
        if (threadIdx.x == 0) {
            prefix_s = p;
            const int tb = (int)unpack_a(p), hb = (int)unpack_b(p);
            L.sec_trk_off[g] = tb;
            L.sec_hit_off[g] = hb;
            if (g == L.S - 1) {
                L.sec_trk_off[L.S] = tb + m;
                L.sec_hit_off[L.S] = hb + run;
                L.cnt->n_tracks = tb + m;
                L.cnt->n_track_hits = hb + run;
                L.k_hit_off[tb + m] = hb + run;
            }
        }
    }
    __syncthreads();
    const int tb = (int)unpack_a(prefix_s), hb = (int)unpack_b(prefix_s);
    int off = hb + warp_sum[wid] + incl - hsum;
    for (int i = lo; i < hi; ++i) {
        const int t = idx[i];
        L.tl_out[t] = tb + i;
        L.tl_hitoff[t] = off;
        off += L.tl_nown[t];
    }
}

// one warp per tracklet: header by lane 0, owned hits by all lanes in row order
__global__ void k_sel_write(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_st; t += warps) {
        const int j = L.tl_out[t];
        if (j < 0) continue;
        const TrackletHdr& H = L.tl[t];
        const int off0 = L.tl_hitoff[t];
        if (lane < 5) L.k_param[(size_t)j * 5 + lane] = H.p[lane];
        if (lane < 15) L.k_cov[(size_t)j * 15 + lane] = H.C[lane];
        if (lane == 0) {
            const int gs = L.hrow[H.start] >> 8;
            const int e = L.sec_event[gs];
            L.k_sector[j] = gs - L.ev[e].sec_base;
            L.k_x[j] = H.x;
            L.k_chi2[j] = H.chi2;
            L.k_ndf[j] = H.ndf;
            L.k_hit_off[j] = off0;
            L.k_gsec[j] = gs;
        }
        // owned rows from the bits k_sel_decide left (no weight reads here)
        const int* rowhit = L.tl_rowhit + (size_t)t * L.R;
        const unsigned* ownw = L.tl_own + (size_t)t * kOwnWords;
        int off = off0;
        for (int r0 = H.first, c = 0; r0 <= H.last; r0 += 32, ++c) {
            const unsigned b = ownw[c];
            if ((b >> lane) & 1u)
                L.k_hit_cid[off + __popc(b & ((1u << lane) - 1))] = L.hcid[rowhit[r0 + lane]];
            off += __popc(b);
        }
    }
}

}  // namespace

constexpr size_t kSelSortSmem = kMaxSectorTracks * (sizeof(unsigned long long) + sizeof(int));

void prepare_selector()
{
    cudaFuncSetAttribute(k_sel_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSelSortSmem);
}

void launch_selector(const Launch& L, const Schedule& S, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    int blocks = (L.t_cap + 7) / 8;  // one warp per tracklet, 8 warps per block
    if (blocks > S.n_sm * 16) blocks = S.n_sm * 16;
    if (blocks < 1) blocks = 1;
    k_sel_decide<<<blocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_sel_decide");
    k_sel_sort<<<L.S, kSortThreads, kSelSortSmem, stream>>>(L);
    hook_after(hook, "k_sel_sort");
    k_sel_write<<<blocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_sel_write");
}

}  // namespace tpc
