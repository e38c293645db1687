// k_binning.cu -- input checks and row-grid binning of the clusters.
//
// The cellular automaton of the sector tracker (paper, Abstract) looks for
// neighbours in the adjacent pad rows and the fit picks up hits row by row,
// so every hit is kept sorted by (sector, row, y-z bin, cid) with per-bin
// offsets: a window query on a row touches a few contiguous ranges.
//   k_count    checks every cluster (row, sector in range, y and z finite),
//              counts the clusters of each (sector, row) and keeps each
//              cluster's arrival rank in its row
//   k_rowscan  exclusive scan of the row counts and of the per-row bin
//              counts (single pass, decoupled look-back), and the y-z grid
//              of each row sized for about two hits per bin
//   k_scatter  moves every cluster to row offset + rank
//   k_rowsort  counting sort of each row by bin in shared memory, cid order
//              inside a bin; writes the sorted hits and the bin offsets (and
//              clears the hit weights for the fit).  Rows of up to 384 hits
//              (most rows of central and peripheral events) take one warp each, with no
//              block barriers; rows of up to 1024 hits, listed by k_rowscan,
//              one block each, taken in turn from the list by the same
//              blocks first; larger rows are sorted by k_rowsort_big with
//              larger shared-memory footprints (up to 2048 hits, and up to
//              4096)
// Bytes per cluster (read + write): count 12, scatter 12 + 12, rowsort 12 +
// 16 + 8 (weights), plus the row and bin tables.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr int kEvSmem = 1024;

// Row sorts: rows of up to kWarpRowHits hits take one warp, rows of up to
// kSmallRowHits one block of k_rowsort, larger rows one block of
// k_rowsort_big.
// (384: most pad rows of a central event take a warp; rows of up to 512 or
// only 256 hits per warp were slower on the B300)
constexpr int kWarpRowHits = 384;
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kWsHist = kWarpRowHits * kBinsPerHitX2 / 2 + 4;  // >= nb + 1, keeps 16-byte regions

__device__ __forceinline__ int find_event(const long long* off, int n_ev, long long i)
{
    int lo = 0, hi = n_ev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool cluster_of(const Launch& L, const long long* off_s, long long i,
                                           float& y, float& z, int& g, int& cid, int& e)
{
    e = find_event(off_s, L.n_events, i);
    const EventDesc d = L.ev[e];
    const long long j = i - d.cl_off;
    y = d.y[j];
    z = d.z[j];
    const int r = d.row[j];
    const int s = d.sec[j];
    cid = (int)j;
    if (r >= L.R || s >= d.n_sec || !isfinite(y) || !isfinite(z)) return false;
    g = (d.sec_base + s) * L.R + r;
    return true;
}

__device__ __forceinline__ void load_offsets(const Launch& L, long long* off_s)
{
    for (int e = threadIdx.x; e <= L.n_events; e += blockDim.x) off_s[e] = L.ev_off[e];
    __syncthreads();
}

// Clusters per thread and loop step: their loads, and then their atomics,
// are issued together.
constexpr int kBinIlp = 4;

__global__ void k_count(Launch L)
{
    __shared__ long long off_s[kEvSmem + 1];
    load_offsets(L, off_s);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < L.n_total;
         i0 += kBinIlp * stride) {
        int g[kBinIlp], e[kBinIlp];
        bool ok[kBinIlp];
#pragma unroll
        for (int k = 0; k < kBinIlp; ++k) {
            const long long i = i0 + k * stride;
            float y, z;
            int cid;
            g[k] = 0;
            e[k] = 0;
            ok[k] = i < L.n_total && cluster_of(L, off_s, i, y, z, g[k], cid, e[k]);
        }
#pragma unroll
        for (int k = 0; k < kBinIlp; ++k) {
            const long long i = i0 + k * stride;
            if (i >= L.n_total) break;
            if (ok[k]) {
                L.rank[i] = atomicAdd(&L.row_cnt[g[k] * kCntPad], 1);
            } else {  // skipped (never binned); counted for its event
                atomicAdd(&L.cnt->n_invalid, 1);
                atomicAdd(&L.ev_invalid[e[k]], 1);
            }
        }
    }
}

// y-z grid of row g holding cnt hits: about two hits per bin over the row's
// extent (sector width plus 2 cm, z range of the sector side plus 2 cm).
__device__ __forceinline__ RowGrid make_grid(const Launch& L, int g, int cnt)
{
    const int gs = g / L.R;
    const int r = g - gs * L.R;
    const int e = L.sec_event[gs];
    const int s = gs - L.ev[e].sec_base;
    const float x = __ldg(&L.xr[r]);
    const float yh = x * L.tan_half + 2.0f;
    float zlo = -L.z_max, zhi = L.z_max;
    if (L.split_z) {
        if (s < L.n_sectors_phi) zlo = 0.0f;
        else zhi = 0.0f;
    }
    zlo -= 2.0f;
    zhi += 2.0f;
    const float W = 2.0f * yh, H = zhi - zlo;
    const int nb = max(1, cnt * kBinsPerHitX2 / 2);
    int ny = (int)(sqrtf((float)nb * W / H) + 0.5f);
    ny = min(max(ny, 1), min(nb, kMaxBinsPerDim));   // ny * nz <= nb always
    int nz = min(max(nb / ny, 1), kMaxBinsPerDim);
    RowGrid G;
    G.y0 = -yh;
    G.z0 = zlo;
    G.idy = (float)ny / W;
    G.idz = (float)nz / H;
    G.ny = ny;
    G.nz = nz;
    G.bin_off = 0;
    G.pad = 0;
    return G;
}

constexpr int kScanThreads = 256;
constexpr int kScanItems = kRowTile / kScanThreads;
constexpr int kScanTile = kRowTile;
static_assert(kScanItems * kScanThreads == kRowTile, "row tile");

// block-wide exclusive scan of one packed value per thread; returns the
// exclusive prefix of this thread and the block total in *total
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* total)
{
    __shared__ unsigned long long warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long w = lane < nw ? warp_tot[lane] : 0ULL;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) warp_tot[lane] = wi - w;   // exclusive prefix of warp
        if (lane == nw - 1) warp_tot[31] = wi;    // block total (nw <= 31 here)
    }
    __syncthreads();
    const unsigned long long res = warp_tot[wid] + incl - v;
    *total = warp_tot[31];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_rowscan(Launch L)
{
    __shared__ int tile_s;
    __shared__ unsigned long long prefix_s;
    if (threadIdx.x == 0) tile_s = atomicAdd(&L.cnt->ticket_rows, 1);
    __syncthreads();
    const int tile = tile_s;
    const int g0 = tile * kScanTile + threadIdx.x * kScanItems;
    unsigned long long loc[kScanItems];
    unsigned long long sum = 0;
    int cmax = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int g = g0 + k;
        unsigned long long v = 0;
        if (g < L.RS) {
            const int c = L.row_cnt[g * kCntPad];
            cmax = max(cmax, c);
            // rows for the block sorts: from the front of big_rows the rows
            // for k_rowsort, from the back those for k_rowsort_big
            if (c > kWarpRowHits) {
                if (c <= kSmallRowHits) L.big_rows[atomicAdd(&L.cnt->n_mid_rows, 1)] = g;
                else L.big_rows[L.RS - 1 - atomicAdd(&L.cnt->n_big_rows, 1)] = g;
            }
            RowGrid G = make_grid(L, g, c);
            L.grid[g] = G;
            v = pack2((unsigned)c, (unsigned)(G.ny * G.nz + 1));
        }
        loc[k] = sum;
        sum += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    if ((threadIdx.x & 31) == 0 && cmax > 0) atomicMax(&L.cnt->max_row_hits, cmax);
    unsigned long long total;
    const unsigned long long excl = block_excl_scan(sum, &total);
    if (threadIdx.x < 32) {
        const unsigned long long p = lookback_warp(L.tile_state, tile, total, L.cnt, L.spin_limit);
        if (threadIdx.x == 0) prefix_s = p;
    }
    __syncthreads();
    const unsigned long long base = prefix_s + excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int g = g0 + k;
        if (g < L.RS) {
            const unsigned long long v = base + loc[k];
            L.row_off[g] = (int)unpack_a(v);
            L.grid[g].bin_off = (int)unpack_b(v);
            if (g == L.RS - 1) {
                const int c = L.row_cnt[g * kCntPad];
                const RowGrid G = L.grid[g];
                L.row_off[L.RS] = (int)unpack_a(v) + c;
                L.cnt->n_bins = (int)unpack_b(v) + G.ny * G.nz + 1;
            }
        }
    }
}

__global__ void k_scatter(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    __shared__ long long off_s[kEvSmem + 1];
    load_offsets(L, off_s);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < L.n_total;
         i0 += kBinIlp * stride) {
        float y[kBinIlp], z[kBinIlp];
        int pos[kBinIlp], cid[kBinIlp];
#pragma unroll
        for (int k = 0; k < kBinIlp; ++k) {
            const long long i = i0 + k * stride;
            int g = 0, e = 0;
            pos[k] = -1;
            if (i < L.n_total && cluster_of(L, off_s, i, y[k], z[k], g, cid[k], e))
                pos[k] = L.row_off[g] + L.rank[i];
        }
#pragma unroll
        for (int k = 0; k < kBinIlp; ++k) {
            if (pos[k] < 0) continue;
            L.tmp_rec[pos[k]] = make_float4(y[k], z[k], __int_as_float(cid[k]), 0.0f);
        }
    }
}

// Shared memory of a block row sort for rows of up to cap hits, and of a
// warp row sort.
constexpr size_t sort_smem(int cap)
{
    return sizeof(int) * (cap * kBinsPerHitX2 / 2 + 2) + sizeof(int) * cap +
           3 * sizeof(int16_t) * cap;
}
constexpr size_t kWarpSortSmem = sizeof(int) * kWsHist + sizeof(int) * kWarpRowHits +
                                 3 * sizeof(int16_t) * kWarpRowHits;
constexpr size_t kRowsortSmem = sort_smem(kSmallRowHits) > kRsWarps * kWarpSortSmem
                                    ? sort_smem(kSmallRowHits)
                                    : kRsWarps * kWarpSortSmem;
static_assert(kWarpSortSmem % 16 == 0, "warp regions stay aligned");

// Write the sorted row: hit p of the row is input hit order[p]; every bin's
// start offset (and the row's end in bin nb).
__device__ __forceinline__ void write_row(const Launch& L, int base, int n, int nb, int bin_off,
                                          int hrow, const int16_t* order, const int* cid,
                                          const int* hist, int t0, int dt)
{
    for (int p = t0; p < n; p += dt) {
        const int i = order[p];
        const float4 c = L.tmp_rec[base + i];
        L.hyz[base + p] = make_float2(c.x, c.y);
        L.hcid[base + p] = cid[i];
        L.hrow[base + p] = hrow;
        L.weight[base + p] = 0ULL;
        if (L.mark) L.mark[base + p] = 0;
    }
    for (int b = t0; b <= nb; b += dt) L.bin_start[bin_off + b] = hist[b];
}

// Insertion sort by cid inside each bin (bins hold a few hits); threads t0,
// t0 + dt, ... take bins in turn.
__device__ __forceinline__ void cid_order(int nb, const int* hist, const int* scid,
                                          int16_t* sorder, int t0, int dt)
{
    for (int b = t0; b < nb; b += dt) {
        const int lo = hist[b], hi = hist[b + 1];
        for (int a = lo + 1; a < hi; ++a) {
            const int16_t v = sorder[a];
            const int key = scid[v];
            int c = a - 1;
            while (c >= lo && scid[sorder[c]] > key) {
                sorder[c + 1] = sorder[c];
                --c;
            }
            sorder[c + 1] = v;
        }
    }
}

// Counting sort of row g (up to CAP hits) by the whole block; every thread
// calls it.  A row above kMaxRowHits is a capacity error: its hits are
// copied unsorted and every bin left empty, so that the later stages stay in
// bounds, and the launch fails.
template <int CAP>
__device__ void sort_row_block(const Launch& L, int g, unsigned char* smem)
{
    int* hist = reinterpret_cast<int*>(smem);                // [nb + 1]
    int* scid = hist + (CAP * kBinsPerHitX2 / 2 + 2);        // [n]
    int16_t* sbin = reinterpret_cast<int16_t*>(scid + CAP);  // [n]
    int16_t* sslot = sbin + CAP;                             // [n]
    int16_t* sorder = sslot + CAP;                           // [n]
    const int base = L.row_off[g];
    const int n = L.row_off[g + 1] - base;
    const RowGrid G = L.grid[g];
    const int nb = G.ny * G.nz;
    const int gs = g / L.R;
    const int hrow = (gs << 8) | (g - gs * L.R);
    if (n > CAP) {
        if (threadIdx.x == 0) atomicExch(&L.cnt->ovf_row, 1);
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const float4 c = L.tmp_rec[base + p];
            L.hyz[base + p] = make_float2(c.x, c.y);
            L.hcid[base + p] = __float_as_int(c.z);
            L.hrow[base + p] = hrow;
            L.weight[base + p] = 0ULL;
            if (L.mark) L.mark[base + p] = 0;
        }
        for (int b = threadIdx.x; b <= nb; b += blockDim.x) L.bin_start[G.bin_off + b] = 0;
        return;
    }
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 c = L.tmp_rec[base + i];
        const int b = bin_z(G, c.y) * G.ny + bin_y(G, c.x);
        sbin[i] = (int16_t)b;
        scid[i] = __float_as_int(c.z);
        sslot[i] = (int16_t)atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    // exclusive scan of hist[0..nb] (hist[nb] = 0 -> becomes n)
    {
        const int per = (nb + 1 + blockDim.x - 1) / blockDim.x;
        const int lo = threadIdx.x * per;
        const int hi = min(lo + per, nb + 1);
        int sum = 0;
        for (int b = lo; b < hi; ++b) sum += hist[b];
        unsigned long long tot;
        int run = (int)block_excl_scan((unsigned long long)sum, &tot);
        for (int b = lo; b < hi; ++b) {
            const int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) sorder[hist[sbin[i]] + sslot[i]] = (int16_t)i;
    __syncthreads();
    cid_order(nb, hist, scid, sorder, threadIdx.x, blockDim.x);
    __syncthreads();
    write_row(L, base, n, nb, G.bin_off, hrow, sorder, scid, hist, threadIdx.x, blockDim.x);
    __syncthreads();
}

// The same counting sort of row g (base, n <= kWarpRowHits hits) by one
// warp, with warp-synchronous steps.
__device__ void sort_row_warp(const Launch& L, int g, int base, int n, unsigned char* ws, int lane)
{
    int* hist = reinterpret_cast<int*>(ws);                          // [kWsHist]
    int* scid = hist + kWsHist;                                      // [n]
    int16_t* sbin = reinterpret_cast<int16_t*>(scid + kWarpRowHits);  // [n]
    int16_t* sslot = sbin + kWarpRowHits;                            // [n]
    int16_t* sorder = sslot + kWarpRowHits;                          // [n]
    const RowGrid G = L.grid[g];
    const int nb = G.ny * G.nz;  // <= max(1, 2n) < kWsHist
    const int gs = g / L.R;
    const int hrow = (gs << 8) | (g - gs * L.R);
    for (int b = lane; b <= nb; b += 32) hist[b] = 0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const float4 c = L.tmp_rec[base + i];
        const int b = bin_z(G, c.y) * G.ny + bin_y(G, c.x);
        sbin[i] = (int16_t)b;
        scid[i] = __float_as_int(c.z);
        sslot[i] = (int16_t)atomicAdd(&hist[b], 1);
    }
    __syncwarp();
    // exclusive scan of hist[0..nb], one contiguous chunk of bins per lane
    {
        const int per = (nb + 1 + 31) >> 5;
        const int lo = lane * per;
        const int hi = min(lo + per, nb + 1);
        int sum = 0;
        for (int b = lo; b < hi; ++b) sum += hist[b];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - sum;
        for (int b = lo; b < hi; ++b) {
            const int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) sorder[hist[sbin[i]] + sslot[i]] = (int16_t)i;
    __syncwarp();
    cid_order(nb, hist, scid, sorder, lane, 32);
    __syncwarp();
    write_row(L, base, n, nb, G.bin_off, hrow, sorder, scid, hist, lane, 32);
    __syncwarp();
}

// Every row of up to kSmallRowHits hits.  The blocks first take the listed
// rows of kWarpRowHits + 1 to kSmallRowHits hits one at a time from the
// list (a work counter), then their warps sort the rows of up to
// kWarpRowHits hits, one row per warp, so that the many small rows of a
// batch of peripheral events are not each paid for with a block's barriers,
// and the two kinds of row overlap on the GPU.
__global__ void __launch_bounds__(kRsThreads) k_rowsort(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ __align__(16) unsigned char smem[];  // kRowsortSmem bytes
    __shared__ int item_s;
    const int n_mid = min(L.cnt->n_mid_rows, L.RS);
    for (;;) {
        __syncthreads();  // the last item read by every thread
        if (threadIdx.x == 0) item_s = atomicAdd(&L.cnt->mid_next, 1);
        __syncthreads();
        const int it = item_s;
        if (it >= n_mid) break;
        sort_row_block<kSmallRowHits>(L, L.big_rows[it], smem);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ws = smem + w * kWarpSortSmem;
    const int stride = gridDim.x * kRsWarps;
    int g = blockIdx.x * kRsWarps + w;
    // the next row's offsets are read while this one is sorted
    int nx0 = 0, nx1 = 0;
    if (g < L.RS) {
        nx0 = L.row_off[g];
        nx1 = L.row_off[g + 1];
    }
    for (; g < L.RS; g += stride) {
        const int base = nx0;
        const int n = nx1 - base;
        const int gn = g + stride;
        if (gn < L.RS) {
            nx0 = L.row_off[gn];
            nx1 = L.row_off[gn + 1];
        }
        if (n <= kWarpRowHits) sort_row_warp(L, g, base, n, ws, lane);
    }
}

// The rows above kSmallRowHits hits, one block each: CAP = kMidRowHits
// sorts those of up to kMidRowHits hits (the pad rows of a pile-up event)
// with half the shared memory, so twice as many blocks fit on an SM; CAP =
// kMaxRowHits the larger ones.
constexpr int kMidRowHits = 2048;

template <int CAP>
__global__ void __launch_bounds__(512) k_rowsort_big(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ __align__(16) unsigned char smem_big[];
    const int n_big = min(L.cnt->n_big_rows, L.RS);
    for (int it = blockIdx.x; it < n_big; it += gridDim.x) {
        const int g = L.big_rows[L.RS - 1 - it];
        const int n = L.row_off[g + 1] - L.row_off[g];
        if ((n <= kMidRowHits) == (CAP == kMidRowHits)) sort_row_block<CAP>(L, g, smem_big);
    }
}

}  // namespace

int g_rowsort_per_sm = 1;       // resident k_rowsort blocks per SM
int g_big_per_sm[2][2] = {{1, 1}, {1, 1}};  // k_rowsort_big<mid, max> x (256, 512 threads)

void prepare_binning()
{
    cudaFuncSetAttribute(k_rowsort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowsortSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_rowsort_per_sm, k_rowsort, kRsThreads,
                                                  kRowsortSmem);
    if (g_rowsort_per_sm < 1) g_rowsort_per_sm = 1;
    cudaFuncSetAttribute(k_rowsort_big<kMidRowHits>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem(kMidRowHits));
    cudaFuncSetAttribute(k_rowsort_big<kMaxRowHits>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem(kMaxRowHits));
    for (int t = 0; t < 2; ++t) {
        const int th = t ? 512 : 256;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_big_per_sm[0][t], k_rowsort_big<kMidRowHits>,
                                                      th, sort_smem(kMidRowHits));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_big_per_sm[1][t], k_rowsort_big<kMaxRowHits>,
                                                      th, sort_smem(kMaxRowHits));
        for (int k = 0; k < 2; ++k)
            if (g_big_per_sm[k][t] < 1) g_big_per_sm[k][t] = 1;
    }
}

void launch_binning(const Launch& L, const Schedule& S, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const int blocks = S.n_sm * S.bin_blocks_per_sm;
    k_count<<<blocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_count");
    k_rowscan<<<L.n_row_tiles, kScanThreads, 0, stream>>>(L);
    hook_after(hook, "k_rowscan");
    k_scatter<<<blocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_scatter");
    {
        // every block resident at once (the loop over small rows is grid-strided)
        long long rb = (long long)S.n_sm * g_rowsort_per_sm;
        if (rb > L.RS) rb = L.RS;
        if (rb < 1) rb = 1;
        k_rowsort<<<(int)rb, kRsThreads, kRowsortSmem, stream>>>(L);
        hook_after(hook, "k_rowsort");
    }
    // the rows above kSmallRowHits hits, listed by k_rowscan (every block
    // resident at once)
    const int t = S.sort_threads == 256 ? 0 : 1;
    const int threads = t ? 512 : 256;
    k_rowsort_big<kMidRowHits><<<S.n_sm * g_big_per_sm[0][t], threads, sort_smem(kMidRowHits),
                                 stream>>>(L);
    hook_after(hook, "k_rowsort_big");
    k_rowsort_big<kMaxRowHits><<<S.n_sm * g_big_per_sm[1][t], threads, sort_smem(kMaxRowHits),
                                 stream>>>(L);
    hook_after(hook, "k_rowsort_big4k");
}

}  // namespace tpc
