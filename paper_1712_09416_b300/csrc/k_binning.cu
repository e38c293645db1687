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
//   k_rowsort  one block per row: counting sort by bin in shared memory,
//              cid order inside a bin, writes the sorted hits and the bin
//              offsets (and clears the hit weights for the fit); rows above
//              1024 hits are listed and sorted by a second launch with a
//              larger shared-memory footprint
// Bytes per cluster (read + write): count 12, scatter 12 + 12, rowsort 12 +
// 16 + 8 (weights), plus the row and bin tables.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr int kEvSmem = 1024;

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
            L.tmp_yz[pos[k]] = make_float2(y[k], z[k]);
            L.tmp_cid[pos[k]] = cid[k];
        }
    }
}

constexpr int kSortThreads = 512;

// Shared memory of a row sort for rows of up to cap hits.
constexpr size_t sort_smem(int cap)
{
    return sizeof(int) * (cap * kBinsPerHitX2 / 2 + 2) + sizeof(int) * cap +
           3 * sizeof(int16_t) * cap;
}

// One block per row: counting sort by bin, cid order inside a bin.  BIG =
// false sorts the rows of up to kSmallRowHits hits and lists the larger ones
// in big_rows; BIG = true sorts the listed rows (up to kMaxRowHits each).
template <bool BIG>
__global__ void __launch_bounds__(kSortThreads) k_rowsort(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    constexpr int CAP = BIG ? kMaxRowHits : kSmallRowHits;
    extern __shared__ unsigned char smem[];
    int* hist = reinterpret_cast<int*>(smem);                           // [nb + 1]
    int* scid = hist + (CAP * kBinsPerHitX2 / 2 + 2);                   // [n]
    int16_t* sbin = reinterpret_cast<int16_t*>(scid + CAP);             // [n]
    int16_t* sslot = sbin + CAP;                                        // [n]
    int16_t* sorder = sslot + CAP;                                      // [n]
    const int n_items = BIG ? min(L.cnt->n_big_rows, L.RS) : L.RS;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int g = BIG ? L.big_rows[it] : it;
        const int base = L.row_off[g];
        const int n = L.row_off[g + 1] - base;
        if (!BIG && n > CAP) {
            if (threadIdx.x == 0) L.big_rows[atomicAdd(&L.cnt->n_big_rows, 1)] = g;
            continue;
        }
        const RowGrid G = L.grid[g];
        const int nb = G.ny * G.nz;
        const int gs = g / L.R;
        const int hrow = (gs << 8) | (g - gs * L.R);
        if (n > kMaxRowHits) {
            // capacity error: keep the row in bounds for the later stages
            // (hits copied unsorted, every bin empty); the launch fails.
            if (threadIdx.x == 0) atomicExch(&L.cnt->ovf_row, 1);
            for (int p = threadIdx.x; p < n; p += blockDim.x) {
                L.hyz[base + p] = L.tmp_yz[base + p];
                L.hcid[base + p] = L.tmp_cid[base + p];
                L.hrow[base + p] = hrow;
                L.weight[base + p] = 0ULL;
                if (L.mark) L.mark[base + p] = 0;
            }
            for (int b = threadIdx.x; b <= nb; b += blockDim.x) L.bin_start[G.bin_off + b] = 0;
            continue;
        }
        for (int b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float2 c = L.tmp_yz[base + i];
            const int b = bin_z(G, c.y) * G.ny + bin_y(G, c.x);
            sbin[i] = (int16_t)b;
            scid[i] = L.tmp_cid[base + i];
            sslot[i] = (int16_t)atomicAdd(&hist[b], 1);
        }
        __syncthreads();
        // exclusive scan of hist[0..nb] (hist[nb] = 0 -> becomes n)
        {
            const int per = (nb + 1 + blockDim.x - 1) / blockDim.x;
            const int lo = threadIdx.x * per;
            const int hi = min(lo + per, nb + 1);
            int s = 0;
            for (int b = lo; b < hi; ++b) s += hist[b];
            unsigned long long tot;
            const int ex = (int)block_excl_scan((unsigned long long)s, &tot);
            int run = ex;
            for (int b = lo; b < hi; ++b) {
                const int c = hist[b];
                hist[b] = run;
                run += c;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) sorder[hist[sbin[i]] + sslot[i]] = (int16_t)i;
        __syncthreads();
        // cid order inside each bin (bins hold a few hits)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
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
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int i = sorder[p];
            L.hyz[base + p] = L.tmp_yz[base + i];
            L.hcid[base + p] = scid[i];
            L.hrow[base + p] = hrow;
            L.weight[base + p] = 0ULL;
            if (L.mark) L.mark[base + p] = 0;
        }
        for (int b = threadIdx.x; b <= nb; b += blockDim.x) L.bin_start[G.bin_off + b] = hist[b];
        __syncthreads();
    }
}

}  // namespace

void prepare_binning()
{
    cudaFuncSetAttribute(k_rowsort<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem(kSmallRowHits));
    cudaFuncSetAttribute(k_rowsort<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sort_smem(kMaxRowHits));
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
    const int rows_blocks = L.RS < S.n_sm * 16 ? L.RS : S.n_sm * 16;
    const int threads = S.sort_threads == 256 ? 256 : kSortThreads;
    k_rowsort<false><<<rows_blocks > 0 ? rows_blocks : 1, threads, sort_smem(kSmallRowHits),
                       stream>>>(L);
    hook_after(hook, "k_rowsort");
    // the rows above kSmallRowHits hits, listed by the first pass
    k_rowsort<true><<<S.n_sm * 2, kSortThreads, sort_smem(kMaxRowHits), stream>>>(L);
    hook_after(hook, "k_rowsort_big");
}

}  // namespace tpc
