// k_finder.cu -- the cellular-automaton part of the sector tracker (paper,
// Abstract): neighbour finding, mutual-link cleaning and start hits.
//
//   k_neighbours   one thread per hit h on row r.  Candidates on rows r +- 1 inside the slope windows
//                  |dy| <= SY |dx|, |dz| <= SZ |dx| are taken from the y-z bins
//                  that cover the window; every (down, up) pair is scored by
//                  the straight-line kink D = (sy_u - sy_d)^2 + (sz_u - sz_d)^2;
//                  the least D wins (exact ties to the lower cid of up, then of
//                  down) and links are kept when D <= D_MAX.  The decision is
//                  taken in binary32 with one rounding per operation (no fused
//                  multiply-add, IEEE division), so it is reproducible exactly.
//   k_clean_starts tiles of consecutive sorted hits: keep a link only if the
//                  partner links back, mark start hits (up link, no down link)
//                  and compact them in (sector, row, bin, cid) order with a
//                  single-pass decoupled look-back scan.
// Bytes per cluster: neighbours read y, z (8) + bins, write up/dn (4);
// cleaning reads links (4) and gathers partners (4), writes 4, starts 4/hit.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr int kNbThreads = 256;  // largest block; the schedule picks 64, 128 or 256

struct RowView {      // one adjacent row
    const float2* yz;
    const int* cid;
    const int* bins;
    RowGrid G;
};

// Admissible candidates of one side, kept in registers (at most kList); the
// insert is a chain of predicated moves so that the list never spills.
constexpr int kList = 4;
struct CandList {
    float sy[kList], sz[kList];
    int cid[kList], k[kList];
    int n;
};

__device__ __forceinline__ void push(CandList& c, float sy, float sz, int k)
{
#pragma unroll
    for (int j = 0; j < kList; ++j) {
        if (c.n == j) {
            c.sy[j] = sy;
            c.sz[j] = sz;
            c.k[j] = k;
        }
    }
    ++c.n;
}

// Scan one side's window: admissible candidates and their slopes.  up = true
// gives slopes (c - h) * inv, up = false gives (h - c) * inv.  The hit ranges
// of the window's z-bins (up to four) are walked as one flat index space so
// that lanes with different bin counts stay together, four candidates per
// step with their loads issued together; the cids of the kept candidates are
// read at the end.
__device__ __forceinline__ void collect(const RowView& V, float yh, float zh, float inv, float wy,
                                       float wz, bool up, CandList& c)
{
    const float my = 1e-3f * (1.0f + fabsf(yh)), mz = 1e-3f * (1.0f + fabsf(zh));
    const int y0 = bin_y(V.G, yh - wy - my), y1 = bin_y(V.G, yh + wy + my);
    const int z0 = bin_z(V.G, zh - wz - mz), z1 = bin_z(V.G, zh + wz + mz);
    c.n = 0;
    auto test = [&](int k, float2 v) {
        const float ddy = up ? __fsub_rn(v.x, yh) : __fsub_rn(yh, v.x);
        const float ddz = up ? __fsub_rn(v.y, zh) : __fsub_rn(zh, v.y);
        if (fabsf(ddy) <= wy && fabsf(ddz) <= wz)
            push(c, __fmul_rn(ddy, inv), __fmul_rn(ddz, inv), k);
    };
    if (z1 - z0 < 4) {
        int a[4], n[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int bz = z0 + j;
            a[j] = 0;
            n[j] = 0;
            if (bz <= z1) {
                a[j] = V.bins[bz * V.G.ny + y0];
                n[j] = V.bins[bz * V.G.ny + y1 + 1] - a[j];
            }
        }
        const int c1 = n[0], c2 = c1 + n[1], c3 = c2 + n[2], tot = c3 + n[3];
        for (int q = 0; q < tot; q += 4) {
            int kk[4];
            float2 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qj = q + j < tot ? q + j : q;
                kk[j] = qj < c1 ? a[0] + qj : qj < c2 ? a[1] + (qj - c1)
                                          : qj < c3 ? a[2] + (qj - c2) : a[3] + (qj - c3);
                v[j] = V.yz[kk[j]];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (q + j < tot) test(kk[j], v[j]);
        }
    } else {
        for (int bz = z0; bz <= z1; ++bz) {
            const int ka = V.bins[bz * V.G.ny + y0], kb = V.bins[bz * V.G.ny + y1 + 1];
            for (int k = ka; k < kb; ++k) test(k, V.yz[k]);
        }
    }
#pragma unroll
    for (int j = 0; j < kList; ++j)
        if (j < c.n) c.cid[j] = V.cid[c.k[j]];
}

__device__ __forceinline__ void consider(float syu, float szu, int cu, int ku, float syd, float szd,
                                         int cd, int kd, float& bestD, int& bcu, int& bcd,
                                         int& biu, int& bid)
{
    const float ey = __fsub_rn(syu, syd), ez = __fsub_rn(szu, szd);
    const float Dv = __fadd_rn(__fmul_rn(ey, ey), __fmul_rn(ez, ez));
    const bool better = bcu < 0 || Dv < bestD || (Dv == bestD && (cu < bcu || (cu == bcu && cd < bcd)));
    if (better) {
        bestD = Dv;
        bcu = cu;
        bcd = cd;
        biu = ku;
        bid = kd;
    }
}

// The candidates of one side lie in the window's y-z bins: for each z-bin
// from z0 to z1 the sorted hits [bins[bz*ny + y0], bins[bz*ny + y1 + 1]).
// BinWalk enumerates them bin after bin, four indices at a time, so that the
// loads of a batch are issued together.
struct BinWalk {
    int bz, z1, k, kb;
};

__device__ __forceinline__ void walk_open(const RowView& V, int y0, int y1, int z0, int z1,
                                          BinWalk& w)
{
    w.bz = z0;
    w.z1 = z1;
    w.k = V.bins[z0 * V.G.ny + y0];
    w.kb = V.bins[z0 * V.G.ny + y1 + 1];
}

// next candidate index, or -1 when the window is exhausted
__device__ __forceinline__ int walk_next(const RowView& V, int y0, int y1, BinWalk& w)
{
    while (w.k >= w.kb) {
        if (++w.bz > w.z1) return -1;
        w.k = V.bins[w.bz * V.G.ny + y0];
        w.kb = V.bins[w.bz * V.G.ny + y1 + 1];
    }
    return w.k++;
}

// Crowded windows: admissible up candidates are gathered in registers in chunks of up to
// kUpChunk (slopes, cid, index; batches of four loads until the chunk holds
// more than kUpChunk - 4); for each chunk every down candidate is streamed
// from the bins and scored against the whole chunk.  Any number of
// candidates on either side takes this path (a further chunk re-streams the
// down side).
constexpr int kUpChunk = 8;

// Best (down, up) pair when a window holds more admissible candidates than
// the register lists of best_pair (run by k_neighbours_crowded, a kernel of
// its own, so that its registers do not weigh on the common path).
__device__ __forceinline__ void best_pair_crowded(const RowView& U, const RowView& D, float yh, float zh,
                                          float iu, float id, float wyu, float wzu, float wyd,
                                          float wzd, float& bestD, int& bcu, int& bcd, int& biu,
                                          int& bid)
{
    const float my = 1e-3f * (1.0f + fabsf(yh)), mz = 1e-3f * (1.0f + fabsf(zh));
    const int uy0 = bin_y(U.G, yh - wyu - my), uy1 = bin_y(U.G, yh + wyu + my);
    const int uz0 = bin_z(U.G, zh - wzu - mz), uz1 = bin_z(U.G, zh + wzu + mz);
    const int dy0 = bin_y(D.G, yh - wyd - my), dy1 = bin_y(D.G, yh + wyd + my);
    const int dz0 = bin_z(D.G, zh - wzd - mz), dz1 = bin_z(D.G, zh + wzd + mz);
    BinWalk wu;
    walk_open(U, uy0, uy1, uz0, uz1, wu);
    bool up_left = true;
    while (up_left) {
        // the next chunk of admissible up candidates
        float csy[kUpChunk], csz[kUpChunk];
        int ccid[kUpChunk], ck[kUpChunk];
        int n = 0;
        while (n <= kUpChunk - 4) {  // a batch of four always fits
            int kk[4];
            float2 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                kk[j] = walk_next(U, uy0, uy1, wu);
                if (kk[j] >= 0) v[j] = U.yz[kk[j]];
            }
            bool any = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (kk[j] < 0) continue;
                any = true;
                const float ddy = __fsub_rn(v[j].x, yh), ddz = __fsub_rn(v[j].y, zh);
                if (fabsf(ddy) <= wyu && fabsf(ddz) <= wzu) {
#pragma unroll
                    for (int q = 0; q < kUpChunk; ++q) {
                        if (q == n) {
                            csy[q] = __fmul_rn(ddy, iu);
                            csz[q] = __fmul_rn(ddz, iu);
                            ck[q] = kk[j];
                        }
                    }
                    ++n;
                }
            }
            if (!any) {
                up_left = false;
                break;
            }
        }
        if (n == 0) break;
#pragma unroll
        for (int q = 0; q < kUpChunk; ++q)
            if (q < n) ccid[q] = U.cid[ck[q]];
        // stream the down side against this chunk
        BinWalk wd;
        walk_open(D, dy0, dy1, dz0, dz1, wd);
        for (;;) {
            int kk[4];
            float2 v[4];
            int cdv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                kk[j] = walk_next(D, dy0, dy1, wd);
                if (kk[j] >= 0) {
                    v[j] = D.yz[kk[j]];
                    cdv[j] = D.cid[kk[j]];
                }
            }
            if (kk[0] < 0) break;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (kk[j] < 0) break;
                const float ddy = __fsub_rn(yh, v[j].x), ddz = __fsub_rn(zh, v[j].y);
                if (!(fabsf(ddy) <= wyd) || !(fabsf(ddz) <= wzd)) continue;
                const float syd = __fmul_rn(ddy, id), szd = __fmul_rn(ddz, id);
#pragma unroll
                for (int q = 0; q < kUpChunk; ++q)
                    if (q < n)
                        consider(csy[q], csz[q], ccid[q], ck[q], syd, szd, cdv[j], kk[j], bestD,
                                 bcu, bcd, biu, bid);
            }
        }
    }
}

// Best (down, up) pair of hit (yh, zh): least D over all admissible pairs.
// Returns false, with nothing decided, when a side has more admissible
// candidates than its list holds (the hit goes to k_neighbours_crowded).
__device__ __forceinline__ bool best_pair(const RowView& U, const RowView& D, float yh, float zh,
                                          float iu, float id, float wyu, float wzu, float wyd,
                                          float wzd, float& bestD, int& bcu, int& bcd, int& biu,
                                          int& bid)
{
    CandList cu, cd;
    collect(U, yh, zh, iu, wyu, wzu, true, cu);
    collect(D, yh, zh, id, wyd, wzd, false, cd);
    if (cu.n <= kList && cd.n <= kList) {
#pragma unroll
        for (int a = 0; a < kList; ++a) {
            if (a >= cu.n) break;
#pragma unroll
            for (int b = 0; b < kList; ++b) {
                if (b >= cd.n) break;
                consider(cu.sy[a], cu.sz[a], cu.cid[a], cu.k[a], cd.sy[b], cd.sz[b], cd.cid[b],
                         cd.k[b], bestD, bcu, bcd, biu, bid);
            }
        }
        return true;
    }
    return false;  // more candidates than the lists hold
}

// Hand hit i to k_neighbours_crowded (warp-aggregated append).
__device__ __forceinline__ void push_crowded(const Launch& L, int i)
{
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int b = 0;
    if (lane == leader) b = atomicAdd(&L.cnt->n_crowded, __popc(m));
    b = __shfl_sync(m, b, leader);
    L.crowded[b + __popc(m & ((1u << lane) - 1))] = i;
}

// One thread per sorted hit; the adjacent rows' hits, bins and grids are read
// through the L1 cache (the hits of a block share one or two rows).  Capped
// at 64 registers (a few bytes of spills): eight 128-thread blocks per SM
// instead of six hide more of the gathers' latency (8% faster on a launch of
// eight central events).
__global__ void __launch_bounds__(kNbThreads, 4) k_neighbours(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_hits = L.row_off[L.RS];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_hits; i += gridDim.x * blockDim.x) {
        const int hr = __ldg(&L.hrow[i]);
        const int gs = hr >> 8, r = hr & 255;
        if (r == 0 || r == L.R - 1) {
            L.up[i] = -1;
            L.dn[i] = -1;
            continue;
        }
        const int g = gs * L.R + r;
        const float xh = __ldg(&L.xr[r]), xu = __ldg(&L.xr[r + 1]), xd = __ldg(&L.xr[r - 1]);
        const float iu = __frcp_rn(__fsub_rn(xu, xh)), id = __frcp_rn(__fsub_rn(xh, xd));
        const float wyu = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xu, xh)));
        const float wzu = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xu, xh)));
        const float wyd = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xd, xh)));
        const float wzd = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xd, xh)));
        RowView U, D;
        U.G = L.grid[g + 1];
        D.G = L.grid[g - 1];
        const int bu = __ldg(&L.row_off[g + 1]), bd = __ldg(&L.row_off[g - 1]);
        U.yz = L.hyz + bu;
        U.cid = L.hcid + bu;
        U.bins = L.bin_start + U.G.bin_off;
        D.yz = L.hyz + bd;
        D.cid = L.hcid + bd;
        D.bins = L.bin_start + D.G.bin_off;
        const float2 ch = L.hyz[i];
        const float yh = ch.x, zh = ch.y;
        float bestD = 0.0f;
        int bcu = -1, bcd = -1, biu = -1, bid = -1;
        if (!best_pair(U, D, yh, zh, iu, id, wyu, wzu, wyd, wzd, bestD, bcu, bcd, biu, bid)) {
            push_crowded(L, i);
            continue;
        }
        const bool link = bcu >= 0 && bestD <= L.d_max;
        L.up[i] = link ? (int16_t)biu : (int16_t)-1;
        L.dn[i] = link ? (int16_t)bid : (int16_t)-1;
    }
}

// The hits whose windows held more admissible candidates than the lists of
// best_pair: the same decision with the chunked search (one thread per hit).
__global__ void __launch_bounds__(kNbThreads) k_neighbours_crowded(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n = min(L.cnt->n_crowded, L.n_total > 0x7fffffff ? 0x7fffffff : (int)L.n_total);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int i = L.crowded[q];
        const int hr = L.hrow[i];
        const int gs = hr >> 8, r = hr & 255;
        const int g = gs * L.R + r;
        const float xh = __ldg(&L.xr[r]), xu = __ldg(&L.xr[r + 1]), xd = __ldg(&L.xr[r - 1]);
        const float iu = __frcp_rn(__fsub_rn(xu, xh)), id = __frcp_rn(__fsub_rn(xh, xd));
        const float wyu = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xu, xh)));
        const float wzu = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xu, xh)));
        const float wyd = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xd, xh)));
        const float wzd = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xd, xh)));
        RowView U, D;
        U.G = L.grid[g + 1];
        D.G = L.grid[g - 1];
        const int bu = L.row_off[g + 1], bd = L.row_off[g - 1];
        U.yz = L.hyz + bu;
        U.cid = L.hcid + bu;
        U.bins = L.bin_start + U.G.bin_off;
        D.yz = L.hyz + bd;
        D.cid = L.hcid + bd;
        D.bins = L.bin_start + D.G.bin_off;
        const float2 ch = L.hyz[i];
        float bestD = 0.0f;
        int bcu = -1, bcd = -1, biu = -1, bid = -1;
        best_pair_crowded(U, D, ch.x, ch.y, iu, id, wyu, wzu, wyd, wzd, bestD, bcu, bcd, biu, bid);
        const bool link = bcu >= 0 && bestD <= L.d_max;
        L.up[i] = link ? (int16_t)biu : (int16_t)-1;
        L.dn[i] = link ? (int16_t)bid : (int16_t)-1;
    }
}

// Row blocks (schedule nb_mode = 1): a block takes one (sector, row) at a
// time, stages the hits, cids and bin offsets of the two adjacent rows in
// shared memory (cp.async; a row above kNrCap hits is read from global
// memory instead), then its threads run the same per-hit search as
// k_neighbours over the row's hits.  Identical links; the candidates come
// from shared memory instead of L1/L2.
constexpr int kNrThreads = 128;
constexpr int kNrCap = 1024;              // staged hits of one adjacent row
constexpr int kNrBinCap = 2 * kNrCap + 2; // its bin offsets (2 bins per hit, + 1)

constexpr size_t nr_smem()
{
    return 2 * (sizeof(float2) * kNrCap + sizeof(int) * kNrCap + sizeof(int) * kNrBinCap);
}

__device__ __forceinline__ void nr_stage(const Launch& L, int g, float2* syz, int* scid,
                                         int* sbins, RowView& V)
{
    const int a = L.row_off[g], n = L.row_off[g + 1] - a;
    V.G = L.grid[g];
    const int nb = V.G.ny * V.G.nz + 1;
    const int* gb = L.bin_start + V.G.bin_off;
    if (n <= kNrCap && nb <= kNrBinCap) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            cp_async8(syz + i, L.hyz + a + i);
            cp_async4(scid + i, L.hcid + a + i);
        }
        for (int i = threadIdx.x; i < nb; i += blockDim.x) cp_async4(sbins + i, gb + i);
        V.yz = syz;
        V.cid = scid;
        V.bins = sbins;
    } else {
        V.yz = L.hyz + a;
        V.cid = L.hcid + a;
        V.bins = gb;
    }
}

__global__ void __launch_bounds__(kNrThreads) k_neighbours_rows(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ __align__(16) unsigned char nr_sm[];
    float2* syz = reinterpret_cast<float2*>(nr_sm);  // [2][kNrCap]: up row, down row
    int* scid = reinterpret_cast<int*>(syz + 2 * kNrCap);
    int* sbins = scid + 2 * kNrCap;                  // [2][kNrBinCap]
    for (int g = blockIdx.x; g < L.RS; g += gridDim.x) {
        const int r = g % L.R;
        const int a = L.row_off[g], n = L.row_off[g + 1] - a;
        if (n == 0) continue;
        if (r == 0 || r == L.R - 1) {
            for (int i = a + threadIdx.x; i < a + n; i += blockDim.x) {
                L.up[i] = -1;
                L.dn[i] = -1;
            }
            continue;
        }
        RowView U, D;
        nr_stage(L, g + 1, syz, scid, sbins, U);
        nr_stage(L, g - 1, syz + kNrCap, scid + kNrCap, sbins + kNrBinCap, D);
        const float xh = __ldg(&L.xr[r]), xu = __ldg(&L.xr[r + 1]), xd = __ldg(&L.xr[r - 1]);
        const float iu = __frcp_rn(__fsub_rn(xu, xh)), id = __frcp_rn(__fsub_rn(xh, xd));
        const float wyu = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xu, xh)));
        const float wzu = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xu, xh)));
        const float wyd = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xd, xh)));
        const float wzd = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xd, xh)));
        cp_async_wait_all();
        __syncthreads();
        for (int i = a + threadIdx.x; i < a + n; i += blockDim.x) {
            const float2 ch = L.hyz[i];
            float bestD = 0.0f;
            int bcu = -1, bcd = -1, biu = -1, bid = -1;
            if (!best_pair(U, D, ch.x, ch.y, iu, id, wyu, wzu, wyd, wzd, bestD, bcu, bcd, biu, bid)) {
                push_crowded(L, i);
                continue;
            }
            const bool link = bcu >= 0 && bestD <= L.d_max;
            L.up[i] = link ? (int16_t)biu : (int16_t)-1;
            L.dn[i] = link ? (int16_t)bid : (int16_t)-1;
        }
        __syncthreads();  // the staged rows are overwritten by the next row
    }
}

constexpr int kCsThreads = 256;
constexpr int kCsItems = kHitTile / kCsThreads;
constexpr int kCsTile = kHitTile;
static_assert(kCsItems * kCsThreads == kHitTile, "hit tile");

__global__ void __launch_bounds__(kCsThreads) k_clean_starts(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    __shared__ int tile_s;
    __shared__ unsigned long long prefix_s;
    __shared__ int warp_links[kCsThreads / 32];
    if (threadIdx.x == 0) tile_s = atomicAdd(&L.cnt->ticket_hits, 1);
    __syncthreads();
    const int tile = tile_s;
    const int n_hits = L.row_off[L.RS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // items are strided by the block size so that the loads coalesce; the
    // compaction order is item-major, i.e. hit order inside the tile
    bool is_start[kCsItems];
    int n_start = 0, n_link = 0;
#pragma unroll
    for (int k = 0; k < kCsItems; ++k) {
        const int i = tile * kCsTile + k * kCsThreads + threadIdx.x;
        is_start[k] = false;
        if (i < n_hits) {
            const int hr = L.hrow[i];
            const int g = (hr >> 8) * L.R + (hr & 255);
            const int li = i - L.row_off[g];
            const int u = L.up[i], d = L.dn[i];
            int16_t uc = -1, dc = -1;
            int ug = -1;
            if (u >= 0) {
                n_link++;
                const int gu = L.row_off[g + 1] + u;
                if (L.dn[gu] == li) {
                    uc = (int16_t)u;
                    ug = gu;
                }
            }
            if (d >= 0 && L.up[L.row_off[g - 1] + d] == li) dc = (int16_t)d;
            L.upc[i] = uc;
            L.dnc[i] = dc;
            L.upg[i] = ug;
            is_start[k] = uc >= 0 && dc < 0;
        }
    }
    // count starts per item slot across the block in item-major order:
    // position = prefix over (k, thread) pairs
    int cnt_k[kCsItems];
#pragma unroll
    for (int k = 0; k < kCsItems; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, is_start[k]);
        cnt_k[k] = __popc(b);
        n_start += is_start[k] ? 1 : 0;
    }
    (void)n_start;
    // per (k, warp) counts -> exclusive offsets in (k, warp, lane) order
    __shared__ int kw_cnt[kCsItems][kCsThreads / 32];
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kCsItems; ++k) kw_cnt[k][wid] = cnt_k[k];
    }
    {
        int lk = n_link;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lk += __shfl_down_sync(0xffffffffu, lk, o);
        if (lane == 0) warp_links[wid] = lk;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int run = 0;
        if (threadIdx.x == 0) {
            for (int k = 0; k < kCsItems; ++k)
                for (int w = 0; w < kCsThreads / 32; ++w) {
                    const int c = kw_cnt[k][w];
                    kw_cnt[k][w] = run;
                    run += c;
                }
            int links = 0;
            for (int w = 0; w < kCsThreads / 32; ++w) links += warp_links[w];
            if (links) atomicAdd(&L.cnt->n_links, links);
        }
        run = __shfl_sync(0xffffffffu, run, 0);
        const unsigned long long p =
            lookback_warp(L.tile_state + L.n_row_tiles, tile, (unsigned long long)run, L.cnt,
                          L.spin_limit, L.stall_hit_tile == tile + 1);
        if (threadIdx.x == 0) {
            prefix_s = p;
            if (tile == (int)gridDim.x - 1) L.cnt->n_starts = (int)(p + run);
        }
    }
    __syncthreads();
    const int pre = (int)prefix_s;
#pragma unroll
    for (int k = 0; k < kCsItems; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, is_start[k]);
        if (is_start[k]) {
            const int pos = pre + kw_cnt[k][wid] + __popc(b & ((1u << lane) - 1));
            if (pos < L.t_cap) L.starts[pos] = tile * kCsTile + k * kCsThreads + threadIdx.x;
            else atomicExch(&L.cnt->ovf_tracklets, 1);
        }
    }
}

}  // namespace

int neighbour_rows_occupancy()
{
    cudaFuncSetAttribute(k_neighbours_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)nr_smem());
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_neighbours_rows, kNrThreads, nr_smem());
    return per_sm < 1 ? 1 : per_sm;
}

void launch_finder(const Launch& L, const Schedule& S, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    if (S.nb_mode == 1) {
        long long nb = (long long)S.n_sm * (S.nr_max_per_sm > 0 ? S.nr_max_per_sm : 1);
        if (nb > L.RS) nb = L.RS;
        if (nb < 1) nb = 1;
        k_neighbours_rows<<<(int)nb, kNrThreads, nr_smem(), stream>>>(L);
    } else {
        const int th = (S.nb_threads == 64 || S.nb_threads == 256) ? S.nb_threads : 128;
        long long nb = (L.n_total + th - 1) / th;
        if (nb > (long long)S.n_sm * 64) nb = (long long)S.n_sm * 64;
        if (nb < 1) nb = 1;
        k_neighbours<<<(int)nb, th, 0, stream>>>(L);
    }
    hook_after(hook, "k_neighbours");
    {
        long long nc = (L.n_total + 255) / 256;
        if (nc > (long long)S.n_sm * 8) nc = (long long)S.n_sm * 8;
        if (nc < 1) nc = 1;
        k_neighbours_crowded<<<(int)nc, 256, 0, stream>>>(L);
    }
    hook_after(hook, "k_neighbours_crowded");
    k_clean_starts<<<L.n_hit_tiles, kCsThreads, 0, stream>>>(L);
    hook_after(hook, "k_clean_starts");
}

}  // namespace tpc
