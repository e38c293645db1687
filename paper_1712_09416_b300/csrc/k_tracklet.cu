// k_tracklet.cu -- tracklet construction: the Kalman-filter part of the
// sector tracker (paper, Abstract), one thread per chain like the paper's
// one-thread-per-track fit (Sect. 4.1, Listing 2).
//
// k_chains follows, for every start hit, the chain of cleaned up-links (one
// thread per start hit).  k_constructor then, one lane per chain, seeds a
// state (y, z, sin phi, tan lambda, q/pT) from the chord of the chain, fits
// the chain forward, extends it outward row by row (transport to the pad-row
// plane, least-chi2 hit in the box that bounds the chi2 ellipse, update), then
// refits backward from the last hit with the covariance reset to the seed,
// picking up hits below the chain the same way.  The result is the state and
// covariance at the innermost hit.  The 5-vector and the 15 covariance
// entries live in registers; the forward hit list lives in the tracklet's
// rowhit slot and the inputs of the next row are loaded one step ahead.
// k_weights: valid tracklets raise the weight of their hits to the key
// (nHits << 32 | ~cid(h0)) with atomicMax.
//
// Arithmetic is binary32.  Transport between planes x0 -> x1 (dx = x1 - x0):
//   s1 = s0 + C_k dx, C_k = -kB q/pT;  y1 = y0 + dx (s0 + s1)/(c0 + c1);
//   dS = chord * asin(h)/h (h = |C_k| chord / 2), signed like dx;  z1 = z0 + t dS,
// with the exact Jacobian; d(dS)/dC_k is evaluated as
//   dS^2 [ (s1/c1) sinc^2(dphi/2) / 2 + (sin dphi - dphi)/dphi^2 ],  dphi = C_k dS,
// a form without cancellation as C_k -> 0.
// Bytes: k_chains 8 per chain hit (link read, rowhit write) + 32 per start;
// k_constructor per assigned hit y z 8 (forward) + 8 (backward), rowhit 4
// (written) + 4 (read back), about 116 per tracklet (chain record, header);
// k_weights per assigned hit rowhit 4 + weight read-modify-write 16.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"
#include "tpc_fit.cuh"

namespace tpc {

namespace {

constexpr int kTlThreads = 64;

__device__ __forceinline__ bool outside(const Fit& f, float yref, float zref, const Launch& L)
{
    return fabsf(f.p[0] + yref) > f.x * L.tan_half + L.edge_margin ||
           fabsf(f.p[1] + zref) > L.z_max + L.edge_margin;
}

// Candidates ka..kb-1 (global sorted indices) in batches of four loads.
__device__ __forceinline__ void scan_range(const Fit& f, float yref, float zref, int ka, int kb,
                                           float S00, float S01, float S11, float id,
                                           const Launch& L, float& best, int& bk, float& by,
                                           float& bzv)
{
    for (int k = ka; k < kb; k += 4) {
        float2 c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            c[j] = L.hyz[k + j < kb ? k + j : ka];
            c[j].x -= yref;
            c[j].y -= zref;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k + j >= kb) break;
            const float r0 = c[j].x - f.p[0];
            const float r1 = c[j].y - f.p[1];
            const float chi2 = (S11 * r0 * r0 - 2.0f * S01 * r0 * r1 + S00 * r1 * r1) * id;
            // exact ties (rare) go to the lower cid; the cid is read only then
            if (chi2 < best || (chi2 == best && L.hcid[k + j] < L.hcid[bk])) {
                best = chi2;
                bk = k + j;
                by = c[j].x;
                bzv = c[j].y;
            }
        }
    }
}

// Least-chi2 hit of a row (grid G, hits from base) with chi2 <= chi2_hit,
// exact ties to the lower cid; returns its global index or -1 and its
// coordinates relative to (yref, zref) in (my, mz).  Every hit in the bins covering the box that
// bounds the chi2 ellipse is tried.  When the box spans at most two z-bins
// (nearly always: bins are several cm wide, the box a few mm) the four bin
// offsets are read at once and the two hit ranges walked as one list.
__device__ __forceinline__ int search(const Fit& f, float yref, float zref, const RowGrid& G,
                                      int base, const Launch& L, float& my, float& mz)
{
    const float* C = f.C;
    const float S00 = C[0] + L.sy2, S01 = C[1], S11 = C[2] + L.sz2;
    const float id = __fdividef(1.0f, S00 * S11 - S01 * S01);
    const float wy = 1.01f * sqrtf(L.chi2_hit * S00) + 1e-3f;
    const float wz = 1.01f * sqrtf(L.chi2_hit * S11) + 1e-3f;
    const float ya = f.p[0] + yref, za = f.p[1] + zref;  // absolute window centre
    const int y0 = bin_y(G, ya - wy), y1 = bin_y(G, ya + wy);
    const int z0 = bin_z(G, za - wz), z1 = bin_z(G, za + wz);
    const int* bins = L.bin_start + G.bin_off;
    float best = 3.0e38f, by = 0.0f, bzv = 0.0f;
    int bk = -1;
    if (z1 - z0 <= 1) {
        const int a0 = bins[z0 * G.ny + y0], b0 = bins[z0 * G.ny + y1 + 1];
        int a1 = 0, b1 = 0;
        if (z1 > z0) {
            a1 = bins[z1 * G.ny + y0];
            b1 = bins[z1 * G.ny + y1 + 1];
        }
        const int n0 = b0 - a0, tot = n0 + (b1 - a1);
        for (int q = 0; q < tot; q += 4) {
            int kk[4];
            float2 c[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qj = q + j < tot ? q + j : 0;
                kk[j] = base + (qj < n0 ? a0 + qj : a1 + (qj - n0));
                c[j] = L.hyz[kk[j]];
                c[j].x -= yref;
                c[j].y -= zref;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (q + j >= tot) break;
                const float r0 = c[j].x - f.p[0];
                const float r1 = c[j].y - f.p[1];
                const float chi2 = (S11 * r0 * r0 - 2.0f * S01 * r0 * r1 + S00 * r1 * r1) * id;
                if (chi2 < best || (chi2 == best && L.hcid[kk[j]] < L.hcid[bk])) {
                    best = chi2;
                    bk = kk[j];
                    by = c[j].x;
                    bzv = c[j].y;
                }
            }
        }
    } else {
        for (int bz = z0; bz <= z1; ++bz) {
            const int ka = base + bins[bz * G.ny + y0], kb = base + bins[bz * G.ny + y1 + 1];
            scan_range(f, yref, zref, ka, kb, S00, S01, S11, id, L, best, bk, by, bzv);
        }
    }
    my = by;
    mz = bzv;
    return (bk >= 0 && best <= L.chi2_hit) ? bk : -1;
}

// Seed covariance at the current direction: diagonal, cluster variances for
// (y, z), slope variances of dy/dx and dz/dx carried over to sin(phi) and
// tan(lambda) (factors cos^6 phi and cos^2 phi), seed_var_q for q/pT.

// One thread per start hit: follow its chain of cleaned up-links, record the
// chain's hits in the tracklet's rowhit slot and the chain in tl_chain
// (start hit, sector << 8 | row, end hit, end row).  Chains shorter than
// min_chain get their final (empty) header here.  Every lane walks a chain
// of its own at the same time, so the serial link loads overlap across the
// grid instead of stalling a warp of the constructor.
constexpr int kChThreads = 256;

__global__ void __launch_bounds__(kChThreads) k_chains(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    int my_tl = 0, my_hits = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_st; t += gridDim.x * blockDim.x) {
        const int s = L.starts[t];
        const int hr = L.hrow[s];
        const int r0 = hr & 255;
        int* rowhit = L.tl_rowhit + (size_t)t * L.R;
        rowhit[r0] = s;
        int cur = s, rr = r0;
        while (rr < L.R - 1) {
            const int u = L.upg[cur];
            if (u < 0) break;
            ++rr;
            cur = u;
            rowhit[rr] = u;
        }
        const int len = rr - r0 + 1;
        L.tl_chain[t] = make_int4(s, hr, cur, rr);
        TrackletHdr& H = L.tl[t];
        H.start = s;
        H.chain_len = len;
        my_hits += len;
        if (len < L.min_chain) {
            H.valid = 0;
            H.nhits = 0;
            H.first = -1;
            H.last = -1;
            H.ndf = 0;
        } else {
            ++my_tl;
        }
    }
    __shared__ int red[2];
    if (threadIdx.x == 0) red[0] = red[1] = 0;
    __syncthreads();
    if (my_tl) atomicAdd(&red[0], my_tl);
    if (my_hits) atomicAdd(&red[1], my_hits);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (red[0]) atomicAdd(&L.cnt->n_tracklets, red[0]);
        if (red[1]) atomicAdd(&L.cnt->n_chain_hits, red[1]);
    }
}

// Persistent lanes: every lane owns one tracklet at a time and advances it by
// one pad row per loop iteration, forward (chain hits, then search) and then
// backward (assigned hits, then search below the chain).  Lanes of a warp run
// the same row-step code whatever the pass, and a lane whose tracklet is done
// takes the next start hit at once, so the warp stays converged.
__global__ void __launch_bounds__(kTlThreads) k_constructor(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    __shared__ float best_s[21][kTlThreads];  // state + covariance at the innermost backward hit
    __shared__ float pl_s[5][kTlThreads];     // forward state at the last assigned hit
    __shared__ float xs[kMaxRows];            // pad-row radii
    for (int i = threadIdx.x; i < L.R; i += blockDim.x) xs[i] = L.xr[i];
    __syncthreads();
#define BEST(i) best_s[i][threadIdx.x]
#define PL(i) pl_s[i][threadIdx.x]
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int lane = threadIdx.x & 31;
    int t = -1;
    int phase = 0;  // 1 forward, 2 backward
    int r = 0, r0 = 0, rk = 0, last = 0, first = 0, gap = 0, nupd = 0, gbase = 0;
    float chi2 = 0.0f;
    // y and z of the state are kept relative to the start hit (yref, zref):
    // small numbers carry the per-step rounding of binary32 far below the
    // resolution; measurements are shifted by the same reference
    float yref = 0.0f, zref = 0.0f;
    Fit f;
    // The tracklet's rowhit slot holds the hit of every row the forward pass
    // visits (global index, -1 none); the backward pass reads it ahead and
    // rewrites it in place.
    int* rowhit = nullptr;
    // Inputs of the next row, loaded one step ahead: for a row whose hit is
    // known (chain rows forward, rows of the forward range backward) the hit
    // and its coordinates, for a row to search its hit offset and grid.  The
    // rowhit entry of the row after next is read one step earlier still, so
    // that the coordinate load never waits on it.
    bool pknown = false;
    int pb = 0, ph = -1, ph2 = -1;
    float2 pyz = make_float2(0.0f, 0.0f);
    RowGrid pG;
    int my_valid = 0, my_hits = 0;

    // stage row rn of the pass (requires ph2 = rowhit[rn] if rn is known)
    auto stage = [&](int rn, bool fwdp) {
        pknown = fwdp ? rn <= rk : rn >= r0;
        if (pknown) {
            ph = ph2;
            if (ph >= 0) pyz = L.hyz[ph];
        } else {
            pb = L.row_off[gbase + rn];
            pG = L.grid[gbase + rn];
        }
        const int rn2 = fwdp ? rn + 1 : rn - 1;
        if (fwdp ? rn2 <= rk : rn2 >= r0) ph2 = rowhit[rn2];
    };

    bool exhausted = false;  // no start hit left for this lane
    for (;;) {
        // every lane stays in the loop until the whole warp is done, and the
        // warp reconverges here at the top of each row step
        __syncwarp();
        const bool need = t < 0 && !exhausted;
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (m) {
            // warp-aggregated fetch of the next start hits
            const int leader = __ffs(m) - 1;
            int b = 0;
            if (lane == leader) b = atomicAdd(&L.cnt->tl_next, __popc(m));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (need) {
                t = b + __popc(m & ((1u << lane) - 1));
                if (t >= n_st) {
                    t = -1;
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, t >= 0)) {
            if (__all_sync(0xffffffffu, exhausted)) break;
            continue;
        }
        if (t < 0) continue;
        if (phase == 0) {
            // the chain, followed by k_chains: start hit, row, end hit, end row
            const int4 ch = L.tl_chain[t];
            gbase = (ch.y >> 8) * L.R;
            r0 = ch.y & 255;
            rk = ch.w;
            if (rk - r0 + 1 < L.min_chain) {  // header already written
                t = -1;
                continue;
            }
            rowhit = L.tl_rowhit + (size_t)t * L.R;
            const int h1 = rk > r0 ? rowhit[r0 + 1] : -1;
            const float2 c0 = L.hyz[ch.x];
            // seed from the chord h0 -> hk, update at h0
            const float2 ck = L.hyz[ch.z];
            const float x0 = xs[r0], x1 = xs[rk];
            const float tphi = (ck.x - c0.x) / (x1 - x0);
            const float dzdx = (ck.y - c0.y) / (x1 - x0);
            const float cphi = rsqrtf(1.0f + tphi * tphi);
            yref = c0.x;
            zref = c0.y;
            f.x = x0;
            f.p[0] = 0.0f;
            f.p[1] = 0.0f;
            f.p[2] = tphi * cphi;
            f.p[3] = dzdx * cphi;
            f.p[4] = 0.0f;
            seed_cov(f, L);
            update(f, 0.0f, 0.0f, L);
#pragma unroll
            for (int i = 0; i < 5; ++i) PL(i) = f.p[i];
            last = r0;
            gap = 0;
            r = r0 + 1;
            phase = 1;
            ph2 = h1;
            if (r < L.R) stage(r, true);
        }
        // ---- one row step of the current pass ----
        const bool fwd = phase == 1;
        bool end_pass = fwd ? r >= L.R : r < 0;
        if (!end_pass) {
            const bool known = pknown;
            const int base = pb;
            const RowGrid G = pG;
            float my = pyz.x - yref, mz = pyz.y - zref;
            int h = known ? ph : -1;
            const int rn = fwd ? r + 1 : r - 1;
            if (fwd ? rn < L.R : rn >= 0) stage(rn, fwd);
            if (!transport(f, xs[r], L)) {
                end_pass = true;
            } else {
                if (!known) {
                    if (outside(f, yref, zref, L)) end_pass = true;
                    else h = search(f, yref, zref, G, base, L, my, mz);
                }
                if (!end_pass) {
                    if (h >= 0) {
                        const float dchi2 = update(f, my, mz, L);
                        if (fwd) {
                            if (!known) rowhit[r] = h;
                            last = r;
#pragma unroll
                            for (int i = 0; i < 5; ++i) PL(i) = f.p[i];
                        } else {
                            chi2 += dchi2;
                            ++nupd;
                            rowhit[r] = h;
                            first = r;
                            BEST(0) = f.x;
#pragma unroll
                            for (int i = 0; i < 5; ++i) BEST(1 + i) = f.p[i];
#pragma unroll
                            for (int i = 0; i < 15; ++i) BEST(6 + i) = f.C[i];
                        }
                        if (!known) gap = 0;
                    } else {
                        // a row without a hit: searched and missed, or a row
                        // of the forward range that the forward pass missed
                        if (!known) {
                            rowhit[r] = -1;
                            if (++gap >= L.max_gap) end_pass = true;
                        }
                    }
                    r = rn;
                }
            }
        }
        if (!end_pass) continue;
        if (fwd) {
            // backward from the last hit with the covariance reset to the seed
#pragma unroll
            for (int i = 0; i < 5; ++i) f.p[i] = PL(i);
            seed_cov(f, L);
            f.x = xs[last];
            const float2 c = L.hyz[rowhit[last]];
            chi2 = update(f, c.x - yref, c.y - zref, L);
            nupd = 1;
            first = last;
            BEST(0) = f.x;
#pragma unroll
            for (int i = 0; i < 5; ++i) BEST(1 + i) = f.p[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) BEST(6 + i) = f.C[i];
            gap = 0;
            phase = 2;
            r = last - 1;
            if (r >= 0) {
                ph2 = r >= r0 ? rowhit[r] : -1;
                stage(r, false);
            }
            continue;
        }
        // tracklet done: header (the hit weights are raised by k_weights)
        bool fin = isfinite(chi2);
#pragma unroll
        for (int i = 0; i < 20; ++i) fin = fin && isfinite(BEST(1 + i));
#pragma unroll
        for (int i = 0; i < 5; ++i) fin = fin && BEST(6 + CI(i, i)) > 0.0f;
        const bool valid = nupd >= L.min_tracklet_hits && fin;
        TrackletHdr& H = L.tl[t];
        H.x = BEST(0);
#pragma unroll
        for (int i = 0; i < 5; ++i) H.p[i] = BEST(1 + i);
        H.p[0] += yref;
        H.p[1] += zref;
#pragma unroll
        for (int i = 0; i < 15; ++i) H.C[i] = BEST(6 + i);
        H.chi2 = chi2;
        H.nhits = nupd;
        H.first = first;
        H.last = last;
        H.ndf = 2 * nupd - 5;
        H.valid = valid ? 1 : 0;
        if (valid) {
            ++my_valid;
            my_hits += nupd;
        }
        t = -1;
        phase = 0;
    }
#undef BEST
#undef PL
    // block totals of the counters
    __shared__ int red[2];
    if (threadIdx.x == 0) red[0] = red[1] = 0;
    __syncthreads();
    if (my_valid) atomicAdd(&red[0], my_valid);
    if (my_hits) atomicAdd(&red[1], my_hits);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (red[0]) atomicAdd(&L.cnt->n_valid, red[0]);
        if (red[1]) atomicAdd(&L.cnt->n_tracklet_hits, red[1]);
    }
}

// Hit weights: one warp per tracklet, lanes over its rows; every hit of a
// valid tracklet gets atomicMax(weight, (nHits << 32) | (0xFFFFFFFF - cid(h0))).
__global__ void k_weights(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_st; t += warps) {
        const TrackletHdr& H = L.tl[t];
        if (H.chain_len < L.min_chain || !H.valid) continue;
        const unsigned long long key = ((unsigned long long)H.nhits << 32) |
                                       (unsigned long long)(0xFFFFFFFFu - (unsigned)L.hcid[H.start]);
        const int* rowhit = L.tl_rowhit + (size_t)t * L.R;
        for (int r = H.first + lane; r <= H.last; r += 32) {
            const int h = rowhit[r];
            if (h >= 0) atomicMax(&L.weight[h], key);
        }
    }
}

// ---------------------------------------------------------------------------
// Row-synchronous constructor (schedule tl_mode = 1): a block takes a chunk of
// kSwThreads consecutive start hits (one tracklet per thread; consecutive
// starts lie in few sectors and a narrow band of rows) and sweeps the pad rows
// once outward (every forward pass of the chunk advances by one row per
// step) and once inward (every backward pass).  The hits and bin offsets of
// the row being swept are staged in shared memory for up to kSwSecs sectors
// of the chunk (one copy warp each, cp.async, one row ahead), so the window
// searches and the known-hit reads hit shared memory instead of L2.  A sector
// row that does not fit, or a sector beyond the first kSwSecs, is read from
// global memory.  Every tracklet does exactly the arithmetic of k_constructor,
// so the results are identical; only the schedule differs.
constexpr int kSwThreads = 128;
constexpr int kSwSecs = kSwThreads / 32;  // staged sectors: one copy warp each
constexpr int kSwCap = 1024;              // staged hits of one row step, all slots
constexpr int kSwBinCap = 2 * kSwCap + 2 * kSwSecs;

struct SwDesc {          // one (sector, row) of a row step
    const float2* yz;    // its hits (shared memory when staged)
    const int* bins;     // its bin offsets (shared memory when staged)
    RowGrid G;
    int base;            // global sorted index of the row's first hit
    int pad[3];
};

constexpr size_t sweep_smem()
{
    return sizeof(float2) * 2 * kSwCap + sizeof(int) * 2 * kSwBinCap +
           sizeof(SwDesc) * 2 * kSwSecs + sizeof(float) * 26 * kSwThreads +
           sizeof(float) * kMaxRows;
}

// Least-chi2 hit of a row described by D (same rule and arithmetic as search()).
__device__ __forceinline__ int search_sw(const Fit& f, float yref, float zref, const SwDesc& D,
                                         const Launch& L, float& my, float& mz)
{
    const RowGrid& G = D.G;
    const float* C = f.C;
    const float S00 = C[0] + L.sy2, S01 = C[1], S11 = C[2] + L.sz2;
    const float id = __fdividef(1.0f, S00 * S11 - S01 * S01);
    const float wy = 1.01f * sqrtf(L.chi2_hit * S00) + 1e-3f;
    const float wz = 1.01f * sqrtf(L.chi2_hit * S11) + 1e-3f;
    const float ya = f.p[0] + yref, za = f.p[1] + zref;
    const int y0 = bin_y(G, ya - wy), y1 = bin_y(G, ya + wy);
    const int z0 = bin_z(G, za - wz), z1 = bin_z(G, za + wz);
    const int* bins = D.bins;
    const float2* yz = D.yz;
    float best = 3.0e38f, by = 0.0f, bzv = 0.0f;
    int bk = -1;
    for (int bz = z0; bz <= z1; bz += 2) {
        // two z-bins per pass, their hit ranges walked as one list
        const int a0 = bins[bz * G.ny + y0], b0 = bins[bz * G.ny + y1 + 1];
        int a1 = 0, b1 = 0;
        if (bz + 1 <= z1) {
            a1 = bins[(bz + 1) * G.ny + y0];
            b1 = bins[(bz + 1) * G.ny + y1 + 1];
        }
        const int n0 = b0 - a0, tot = n0 + (b1 - a1);
        for (int q = 0; q < tot; q += 4) {
            int kk[4];
            float2 c[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int qj = q + j < tot ? q + j : 0;
                kk[j] = qj < n0 ? a0 + qj : a1 + (qj - n0);
                c[j] = yz[kk[j]];
                c[j].x -= yref;
                c[j].y -= zref;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (q + j >= tot) break;
                const float r0 = c[j].x - f.p[0];
                const float r1 = c[j].y - f.p[1];
                const float chi2 = (S11 * r0 * r0 - 2.0f * S01 * r0 * r1 + S00 * r1 * r1) * id;
                if (chi2 < best ||
                    (chi2 == best && bk >= 0 && L.hcid[D.base + kk[j]] < L.hcid[D.base + bk])) {
                    best = chi2;
                    bk = kk[j];
                    by = c[j].x;
                    bzv = c[j].y;
                }
            }
        }
    }
    my = by;
    mz = bzv;
    return (bk >= 0 && best <= L.chi2_hit) ? D.base + bk : -1;
}

// Copy warp of slot w: stage (sector sec, row rr) into buffer b of the row
// slabs, or point the descriptor at global memory when it does not fit.
// (a, n, G) are the row's offset, hit count and grid, loaded a step ahead.
__device__ __forceinline__ void sw_stage(const Launch& L, float2* s_yz, int* s_bins,
                                         SwDesc* s_desc, int b, int w, int nslot, int a, int n,
                                         const RowGrid& G)
{
    const int lane = threadIdx.x & 31;
    const int cap_h = kSwCap / nslot, cap_b = kSwBinCap / nslot;
    const int nb = G.ny * G.nz + 1;
    const int* gbins = L.bin_start + G.bin_off;
    SwDesc d;
    d.G = G;
    d.base = a;
    if (n <= cap_h && nb <= cap_b) {
        float2* dy = s_yz + b * kSwCap + w * cap_h;
        int* db = s_bins + b * kSwBinCap + w * cap_b;
        for (int i = lane; i < n; i += 32) cp_async8(dy + i, L.hyz + a + i);
        for (int i = lane; i < nb; i += 32) cp_async4(db + i, gbins + i);
        d.yz = dy;
        d.bins = db;
    } else {
        d.yz = L.hyz + a;
        d.bins = gbins;
    }
    if (lane == 0) s_desc[b * kSwSecs + w] = d;
}

__global__ void __launch_bounds__(kSwThreads) k_sweep(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ __align__(16) unsigned char sw_smem[];
    float2* s_yz = reinterpret_cast<float2*>(sw_smem);                  // [2][kSwCap]
    int* s_bins = reinterpret_cast<int*>(s_yz + 2 * kSwCap);            // [2][kSwBinCap]
    SwDesc* s_desc = reinterpret_cast<SwDesc*>(s_bins + 2 * kSwBinCap); // [2][kSwSecs]
    float* s_best = reinterpret_cast<float*>(s_desc + 2 * kSwSecs);     // [21][threads]
    float* s_pl = s_best + 21 * kSwThreads;                             // [5][threads]
    float* xs = s_pl + 5 * kSwThreads;                                  // [kMaxRows]
    __shared__ int s_sec[kSwThreads];
    __shared__ int s_slot_sec[kSwSecs];
    __shared__ int s_nslot, s_chunk, s_rlo, s_rhi;
#define SBEST(i) s_best[(i) * kSwThreads + threadIdx.x]
#define SPL(i) s_pl[(i) * kSwThreads + threadIdx.x]
    for (int i = threadIdx.x; i < L.R; i += blockDim.x) xs[i] = L.xr[i];
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int n_chunks = (n_st + kSwThreads - 1) / kSwThreads;
    const int wid = threadIdx.x >> 5;
    int my_valid = 0, my_hits = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_chunk = atomicAdd(&L.cnt->tl_next, 1);
            s_rlo = L.R;
            s_rhi = -1;
        }
        __syncthreads();
        const int chunk = s_chunk;
        if (chunk >= n_chunks) break;
        // ---- set-up of the chunk's tracklets (as k_constructor's phase 0)
        int t = chunk * kSwThreads + threadIdx.x;
        int r0 = 0, rk = 0, last = 0, first = 0, gap = 0, nupd = 0, gs = -1;
        float chi2 = 0.0f, yref = 0.0f, zref = 0.0f, mly = 0.0f, mlz = 0.0f;
        int* rowhit = nullptr;
        int hk = -1;  // hit of the next known row, read a step ahead
        Fit f;
        bool fwd_on = false;
        if (t < n_st) {
            const int4 ch = L.tl_chain[t];
            gs = ch.y >> 8;
            r0 = ch.y & 255;
            rk = ch.w;
            if (rk - r0 + 1 < L.min_chain) {
                t = -1;
                gs = -1;
            } else {
                rowhit = L.tl_rowhit + (size_t)t * L.R;
                const float2 c0 = L.hyz[ch.x];
                const float2 ckk = L.hyz[ch.z];
                const float x0 = xs[r0], x1 = xs[rk];
                const float tphi = (ckk.x - c0.x) / (x1 - x0);
                const float dzdx = (ckk.y - c0.y) / (x1 - x0);
                const float cphi = rsqrtf(1.0f + tphi * tphi);
                yref = c0.x;
                zref = c0.y;
                f.x = x0;
                f.p[0] = 0.0f;
                f.p[1] = 0.0f;
                f.p[2] = tphi * cphi;
                f.p[3] = dzdx * cphi;
                f.p[4] = 0.0f;
                seed_cov(f, L);
                update(f, 0.0f, 0.0f, L);
#pragma unroll
                for (int i = 0; i < 5; ++i) SPL(i) = f.p[i];
                mly = 0.0f;
                mlz = 0.0f;
                last = r0;
                fwd_on = r0 + 1 < L.R;
                hk = rk > r0 ? rowhit[r0 + 1] : -1;
                if (fwd_on) atomicMin(&s_rlo, r0 + 1);
                else atomicMax(&s_rhi, last);
            }
        } else {
            t = -1;
        }
        s_sec[threadIdx.x] = gs;
        __syncthreads();
        if (threadIdx.x == 0) {
            // distinct sectors of the chunk in order (starts are sorted by
            // sector); the first kSwSecs are staged
            int ns = 0, prev = -1;
            for (int i = 0; i < kSwThreads; ++i) {
                const int v = s_sec[i];
                if (v >= 0 && v != prev) {
                    if (ns < kSwSecs) s_slot_sec[ns] = v;
                    ++ns;
                    prev = v;
                }
            }
            s_nslot = min(ns, kSwSecs);
        }
        __syncthreads();
        const int nslot = s_nslot;
        int slot = -1;
        for (int j = 0; j < nslot; ++j)
            if (s_slot_sec[j] == gs) slot = j;
        const int gbase = gs * L.R;

        // ---- the two sweeps: dir = +1 (forward passes), then -1 (backward)
        for (int dir = 1; dir >= -1; dir -= 2) {
            int r = dir > 0 ? s_rlo : s_rhi;
            if (dir > 0 ? r >= L.R : r < 0) {
                __syncthreads();
                if (dir > 0) continue;
                break;
            }
            // copy warps: row r now, the next row's offsets and grid ahead
            int na = 0, nn = 0;
            RowGrid nG;
            const bool copier = wid < nslot;
            if (copier) {
                const int g = s_slot_sec[wid] * L.R + r;
                const int a = L.row_off[g];
                sw_stage(L, s_yz, s_bins, s_desc, r & 1, wid, nslot, a, L.row_off[g + 1] - a,
                         L.grid[g]);
                const int rn = r + dir;
                if (rn >= 0 && rn < L.R) {
                    na = L.row_off[g + dir];
                    nn = L.row_off[g + dir + 1] - na;
                    nG = L.grid[g + dir];
                }
            }
            cp_async_wait_all();
            __syncthreads();
            bool bwd_wait = dir < 0 && t >= 0;   // backward pass not yet begun
            bool bwd_on = false;
            for (;;) {
                const int rn = r + dir;
                // (A) stage the next row
                if (copier && rn >= 0 && rn < L.R) {
                    sw_stage(L, s_yz, s_bins, s_desc, rn & 1, wid, nslot, na, nn, nG);
                    const int rnn = rn + dir;
                    if (rnn >= 0 && rnn < L.R) {
                        const int g = s_slot_sec[wid] * L.R + rnn;
                        na = L.row_off[g];
                        nn = L.row_off[g + 1] - na;
                        nG = L.grid[g];
                    }
                }
                // (B) one row step of every tracklet in its pass
                SwDesc D;
                const bool stepping = dir > 0 ? (fwd_on && r > r0) : (bwd_on && r < last);
                if (stepping || (bwd_wait && r == last)) {
                    if (slot >= 0) {
                        D = s_desc[(r & 1) * kSwSecs + slot];
                    } else {
                        const int g = gbase + r;
                        D.base = L.row_off[g];
                        D.G = L.grid[g];
                        D.yz = L.hyz + D.base;
                        D.bins = L.bin_start + D.G.bin_off;
                    }
                }
                if (dir > 0) {
                    int hk_next = -1;
                    if (fwd_on && rn > r0 && rn <= rk) hk_next = rowhit[rn];
                    if (stepping) {
                        const bool known = r <= rk;
                        bool end_pass = false;
                        int h = known ? hk : -1;
                        float my = 0.0f, mz = 0.0f;
                        if (!transport(f, xs[r], L)) {
                            end_pass = true;
                        } else {
                            if (known) {
                                const float2 c = D.yz[h - D.base];
                                my = c.x - yref;
                                mz = c.y - zref;
                            } else if (outside(f, yref, zref, L)) {
                                end_pass = true;
                            } else {
                                h = search_sw(f, yref, zref, D, L, my, mz);
                            }
                            if (!end_pass) {
                                if (h >= 0) {
                                    update(f, my, mz, L);
                                    if (!known) rowhit[r] = h;
                                    last = r;
                                    mly = my;
                                    mlz = mz;
#pragma unroll
                                    for (int i = 0; i < 5; ++i) SPL(i) = f.p[i];
                                    if (!known) gap = 0;
                                } else if (!known) {
                                    rowhit[r] = -1;
                                    if (++gap >= L.max_gap) end_pass = true;
                                }
                            }
                        }
                        if (end_pass || r == L.R - 1) fwd_on = false;
                        if (!fwd_on) atomicMax(&s_rhi, last);
                    }
                    hk = hk_next;
                } else {
                    int hk_next = hk;
                    if (bwd_wait && r == last) {
                        // backward from the last hit, covariance reset to the seed
#pragma unroll
                        for (int i = 0; i < 5; ++i) f.p[i] = SPL(i);
                        seed_cov(f, L);
                        f.x = xs[last];
                        chi2 = update(f, mly, mlz, L);
                        nupd = 1;
                        first = last;
                        SBEST(0) = f.x;
#pragma unroll
                        for (int i = 0; i < 5; ++i) SBEST(1 + i) = f.p[i];
#pragma unroll
                        for (int i = 0; i < 15; ++i) SBEST(6 + i) = f.C[i];
                        gap = 0;
                        bwd_wait = false;
                        bwd_on = last > 0;
                        hk_next = (rn >= r0 && rn >= 0) ? rowhit[rn] : -1;
                    } else if (stepping) {
                        const bool known = r >= r0;
                        bool end_pass = false;
                        int h = known ? hk : -1;
                        float my = 0.0f, mz = 0.0f;
                        if (rn >= r0 && rn >= 0) hk_next = rowhit[rn];
                        if (!transport(f, xs[r], L)) {
                            end_pass = true;
                        } else {
                            if (!known) {
                                if (outside(f, yref, zref, L)) end_pass = true;
                                else h = search_sw(f, yref, zref, D, L, my, mz);
                            } else if (h >= 0) {
                                const float2 c = D.yz[h - D.base];
                                my = c.x - yref;
                                mz = c.y - zref;
                            }
                            if (!end_pass) {
                                if (h >= 0) {
                                    chi2 += update(f, my, mz, L);
                                    ++nupd;
                                    rowhit[r] = h;
                                    first = r;
                                    SBEST(0) = f.x;
#pragma unroll
                                    for (int i = 0; i < 5; ++i) SBEST(1 + i) = f.p[i];
#pragma unroll
                                    for (int i = 0; i < 15; ++i) SBEST(6 + i) = f.C[i];
                                    if (!known) gap = 0;
                                } else if (!known) {
                                    if (++gap >= L.max_gap) end_pass = true;
                                }
                            }
                        }
                        if (end_pass || r == 0) bwd_on = false;
                    }
                    hk = hk_next;
                    if (t >= 0 && !bwd_wait && !bwd_on) {
                        // tracklet done: header (weights are raised by k_weights)
                        bool fin = isfinite(chi2);
#pragma unroll
                        for (int i = 0; i < 20; ++i) fin = fin && isfinite(SBEST(1 + i));
#pragma unroll
                        for (int i = 0; i < 5; ++i) fin = fin && SBEST(6 + CI(i, i)) > 0.0f;
                        const bool valid = nupd >= L.min_tracklet_hits && fin;
                        TrackletHdr& H = L.tl[t];
                        H.x = SBEST(0);
#pragma unroll
                        for (int i = 0; i < 5; ++i) H.p[i] = SBEST(1 + i);
                        H.p[0] += yref;
                        H.p[1] += zref;
#pragma unroll
                        for (int i = 0; i < 15; ++i) H.C[i] = SBEST(6 + i);
                        H.chi2 = chi2;
                        H.nhits = nupd;
                        H.first = first;
                        H.last = last;
                        H.ndf = 2 * nupd - 5;
                        H.valid = valid ? 1 : 0;
                        if (valid) {
                            ++my_valid;
                            my_hits += nupd;
                        }
                        t = -1;
                    }
                }
                // (C) the next row is staged and every step of this row done
                cp_async_wait_all();
                const bool more = dir > 0 ? fwd_on : (bwd_wait || bwd_on);
                if (!__syncthreads_or(more ? 1 : 0)) break;
                r = rn;
                if (r < 0 || r >= L.R) break;  // (a pass ends at the last row)
            }
        }
    }
#undef SBEST
#undef SPL
    __shared__ int red[2];
    if (threadIdx.x == 0) red[0] = red[1] = 0;
    __syncthreads();
    if (my_valid) atomicAdd(&red[0], my_valid);
    if (my_hits) atomicAdd(&red[1], my_hits);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (red[0]) atomicAdd(&L.cnt->n_valid, red[0]);
        if (red[1]) atomicAdd(&L.cnt->n_tracklet_hits, red[1]);
    }
}

}  // namespace

int constructor_occupancy()
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_constructor, kTlThreads, 0);
    return per_sm < 1 ? 1 : per_sm;
}

int sweep_occupancy()
{
    cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem());
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep, kSwThreads, sweep_smem());
    return per_sm < 1 ? 1 : per_sm;
}

void launch_constructor(const Launch& L, const Schedule& S, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const int n_sm = S.n_sm;
    // persistent: up to as many blocks as fit on the GPU at once
    int per_sm = S.tl_blocks_per_sm;
    if (per_sm < 1 || (S.tl_max_per_sm > 0 && per_sm > S.tl_max_per_sm)) per_sm = S.tl_max_per_sm;
    if (per_sm < 1) per_sm = 1;
    {
        long long cb = ((long long)L.t_cap + kChThreads - 1) / kChThreads;
        if (cb > (long long)n_sm * 8) cb = (long long)n_sm * 8;
        if (cb < 1) cb = 1;
        k_chains<<<(int)cb, kChThreads, 0, stream>>>(L);
        hook_after(hook, "k_chains");
    }
    if (S.tl_mode == 1) {
        int sb = (S.sw_max_per_sm > 0 ? S.sw_max_per_sm : 1) * n_sm;
        const int chunks = (L.t_cap + kSwThreads - 1) / kSwThreads;
        if (sb > chunks) sb = chunks;
        if (sb < 1) sb = 1;
        k_sweep<<<sb, kSwThreads, sweep_smem(), stream>>>(L);
        hook_after(hook, "k_constructor");
    } else {
        int blocks = per_sm * n_sm;
        const int need = (L.t_cap + kTlThreads - 1) / kTlThreads;
        if (blocks > need) blocks = need;
        if (blocks < 1) blocks = 1;
        k_constructor<<<blocks, kTlThreads, 0, stream>>>(L);
        hook_after(hook, "k_constructor");
    }
    int wblocks = (L.t_cap + 7) / 8;
    if (wblocks > n_sm * 16) wblocks = n_sm * 16;
    if (wblocks < 1) wblocks = 1;
    k_weights<<<wblocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_weights");
}

}  // namespace tpc
