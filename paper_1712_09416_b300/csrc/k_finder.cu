// k_finder.cu -- the cellular-automaton part of the sector tracker (paper,
// Abstract): neighbour finding, mutual-link cleaning and start hits.
//
//   k_neighbours   one block per (sector, row r), one thread per hit h of the
//                  row.  Candidates on rows r +- 1 inside the slope windows
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

constexpr int kNbThreads = 128;

__global__ void __launch_bounds__(kNbThreads) k_neighbours(Launch L)
{
    for (int g = blockIdx.x; g < L.RS; g += gridDim.x) {
        const int gs = g / L.R;
        const int r = g - gs * L.R;
        const int base = L.row_off[g];
        const int n = L.row_off[g + 1] - base;
        if (r == 0 || r == L.R - 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                L.up[base + i] = -1;
                L.dn[base + i] = -1;
            }
            continue;
        }
        const float xh = L.row_x[r], xu = L.row_x[r + 1], xd = L.row_x[r - 1];
        const float dxu = __fsub_rn(xu, xh), dxd = __fsub_rn(xh, xd);
        const float wyu = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xu, xh)));
        const float wzu = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xu, xh)));
        const float wyd = __fmul_rn(L.slope_win_y, fabsf(__fsub_rn(xd, xh)));
        const float wzd = __fmul_rn(L.slope_win_z, fabsf(__fsub_rn(xd, xh)));
        const RowGrid Gu = L.grid[g + 1], Gd = L.grid[g - 1];
        const int bu = L.row_off[g + 1], bd = L.row_off[g - 1];
        const int* binu = L.bin_start + Gu.bin_off;
        const int* bind = L.bin_start + Gd.bin_off;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float yh = L.hy[base + i], zh = L.hz[base + i];
            // bins covering the windows, widened by a margin so that rounding
            // of the bounds can never drop an admissible candidate
            const float my = 1e-3f * (1.0f + fabsf(yh)), mz = 1e-3f * (1.0f + fabsf(zh));
            const int uy0 = bin_y(Gu, yh - wyu - my), uy1 = bin_y(Gu, yh + wyu + my);
            const int uz0 = bin_z(Gu, zh - wzu - mz), uz1 = bin_z(Gu, zh + wzu + mz);
            const int dy0 = bin_y(Gd, yh - wyd - my), dy1 = bin_y(Gd, yh + wyd + my);
            const int dz0 = bin_z(Gd, zh - wzd - mz), dz1 = bin_z(Gd, zh + wzd + mz);
            float bestD = 0.0f;
            int bcu = -1, bcd = -1, biu = -1, bid = -1;
            for (int bzu = uz0; bzu <= uz1; ++bzu) {
                const int ua = binu[bzu * Gu.ny + uy0], ub = binu[bzu * Gu.ny + uy1 + 1];
                for (int ku = ua; ku < ub; ++ku) {
                    const float ddyu = __fsub_rn(L.hy[bu + ku], yh);
                    const float ddzu = __fsub_rn(L.hz[bu + ku], zh);
                    if (!(fabsf(ddyu) <= wyu) || !(fabsf(ddzu) <= wzu)) continue;
                    const float syu = __fdiv_rn(ddyu, dxu), szu = __fdiv_rn(ddzu, dxu);
                    const int cu = L.hcid[bu + ku];
                    for (int bzd = dz0; bzd <= dz1; ++bzd) {
                        const int da = bind[bzd * Gd.ny + dy0], db = bind[bzd * Gd.ny + dy1 + 1];
                        for (int kd = da; kd < db; ++kd) {
                            const float ddyd = __fsub_rn(yh, L.hy[bd + kd]);
                            const float ddzd = __fsub_rn(zh, L.hz[bd + kd]);
                            if (!(fabsf(ddyd) <= wyd) || !(fabsf(ddzd) <= wzd)) continue;
                            const float syd = __fdiv_rn(ddyd, dxd), szd = __fdiv_rn(ddzd, dxd);
                            const float ey = __fsub_rn(syu, syd), ez = __fsub_rn(szu, szd);
                            const float D = __fadd_rn(__fmul_rn(ey, ey), __fmul_rn(ez, ez));
                            const int cd = L.hcid[bd + kd];
                            const bool better = bcu < 0 || D < bestD ||
                                                (D == bestD && (cu < bcu || (cu == bcu && cd < bcd)));
                            if (better) {
                                bestD = D;
                                bcu = cu;
                                bcd = cd;
                                biu = ku;
                                bid = kd;
                            }
                        }
                    }
                }
            }
            const bool link = bcu >= 0 && bestD <= L.d_max;
            L.up[base + i] = link ? (int16_t)biu : (int16_t)-1;
            L.dn[base + i] = link ? (int16_t)bid : (int16_t)-1;
        }
    }
}

constexpr int kCsThreads = 256;
constexpr int kCsItems = 8;
constexpr int kCsTile = kCsThreads * kCsItems;

__global__ void __launch_bounds__(kCsThreads) k_clean_starts(Launch L)
{
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
            if (u >= 0) {
                n_link++;
                if (L.dn[L.row_off[g + 1] + u] == li) uc = (int16_t)u;
            }
            if (d >= 0 && L.up[L.row_off[g - 1] + d] == li) dc = (int16_t)d;
            L.upc[i] = uc;
            L.dnc[i] = dc;
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
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < kCsItems; ++k)
            for (int w = 0; w < kCsThreads / 32; ++w) {
                const int c = kw_cnt[k][w];
                kw_cnt[k][w] = run;
                run += c;
            }
        int links = 0;
        for (int w = 0; w < kCsThreads / 32; ++w) links += warp_links[w];
        if (links) atomicAdd(&L.cnt->n_links, links);
        prefix_s = lookback_exclusive(L.tile_state + L.n_row_tiles, tile,
                                      (unsigned long long)run, L.cnt);
        if (tile == (int)gridDim.x - 1) L.cnt->n_starts = (int)(prefix_s + run);
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

void launch_finder(const Launch& L, void* stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const int blocks = L.RS < 148 * 16 ? L.RS : 148 * 16;
    k_neighbours<<<blocks > 0 ? blocks : 1, kNbThreads, 0, stream>>>(L);
    k_clean_starts<<<L.n_hit_tiles, kCsThreads, 0, stream>>>(L);
}

}  // namespace tpc
