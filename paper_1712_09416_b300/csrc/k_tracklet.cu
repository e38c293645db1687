// k_tracklet.cu -- tracklet construction: the Kalman-filter part of the
// sector tracker (paper, Abstract), one thread per chain like the paper's
// one-thread-per-track fit (Sect. 4.1, Listing 2).
//
// k_chains follows, for every start hit, the chain of cleaned up-links (one
// thread per start hit).  k_constructor<1> then, one lane per chain, seeds a
// state (y, z, sin phi, tan lambda, q/pT) from the chord of the chain, fits
// the chain forward and extends it outward row by row (transport to the
// pad-row plane, least-chi2 hit in the box that bounds the chi2 ellipse,
// update), marking every hit its extension search takes.  k_dominance drops
// the chains all of whose hits were taken so (other tracklets already follow
// their track outward).  k_constructor<2> refits the remaining chains
// backward from the last hit with the covariance reset to the seed, picking
// up hits below the chain the same way; the result is the state and
// covariance at the innermost hit.  The 5-vector and the covariance live in
// registers: the forward pass carries the 15 entries of C, the backward pass
// a square-root factor U (C = U U^T, 25 entries; tpc_fit.cuh), which keeps
// the binary32 result within a small fraction of the parity bars where the
// update of C itself loses the digits the innermost state depends on.  The
// forward hit list lives in the tracklet's rowhit slot and the inputs of the
// next row are loaded one step ahead; the first update of a pass runs inside
// the common row step, with no transport.
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
// k_dominance 16 per chain + 5 per chain hit read (rowhit, mark);
// forward pass per hit y z 8 + rowhit 4 (+ a mark byte per extension hit),
// backward pass per hit y z 8 + rowhit 4 (read) + 4 (written), about 116 per
// tracklet (chain record, header); k_weights per assigned hit rowhit 4 +
// weight read-modify-write 16.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "tpc_internal.cuh"
#include "tpc_fit.cuh"

namespace tpc {

namespace {

constexpr int kTlThreads = 64;

template <class FitT>
__device__ __forceinline__ bool outside(const FitT& f, float yref, float zref, const Launch& L)
{
    return fabsf(f.p[0] + yref) > f.x * L.tan_half + L.edge_margin ||
           fabsf(f.p[1] + zref) > L.z_max + L.edge_margin;
}

// Candidates ka..kb-1 (global sorted indices) in batches of four loads.
template <class FitT>
__device__ __forceinline__ void scan_range(const FitT& f, float yref, float zref, int ka, int kb,
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
            if (chi2 < best || (chi2 == best && bk >= 0 && L.hcid[k + j] < L.hcid[bk])) {
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
template <class FitT>
__device__ __forceinline__ int search(const FitT& f, float yref, float zref, const RowGrid& G,
                                      int base, const Launch& L, float& my, float& mz)
{
    float S00, S01, S11;
    meas_cov(f, L, S00, S01, S11);
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
                if (chi2 < best || (chi2 == best && bk >= 0 && L.hcid[kk[j]] < L.hcid[bk])) {
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

// Result of the backward pass: x, state and covariance (C = U U^T, lower
// triangle) into the lane's column of the shared array best[21][blockDim].
template <class FitT>
__device__ __forceinline__ void save_best(const FitT& f, float (*best)[kTlThreads])
{
    float C[15];
    cov_of(f, C);
    best[0][threadIdx.x] = f.x;
#pragma unroll
    for (int i = 0; i < 5; ++i) best[1 + i][threadIdx.x] = f.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) best[6 + i][threadIdx.x] = C[i];
}

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
        H.dominated = 0;
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
// one pad row per loop iteration; a lane whose tracklet is done takes the
// next start hit at once, so the warp stays converged.  PASS 1 runs the
// forward passes (chain hits, then search) of every chain, marks the hits its
// extension search takes and leaves the forward state at the last hit in the
// header; PASS 2 (after k_dominance) runs the backward passes (assigned hits,
// then search below the chain) of the chains k_dominance listed (those not
// dominated).
// Minimum resident blocks per SM the register allocation aims at, per pass
// (the forward pass fits ten 64-thread blocks per SM without spills).
#ifndef TPC_TL_MINB1
#define TPC_TL_MINB1 10
#endif
#ifndef TPC_TL_MINB2
#define TPC_TL_MINB2 1
#endif

template <int PASS>
__global__ void __launch_bounds__(kTlThreads, PASS == 1 ? TPC_TL_MINB1 : TPC_TL_MINB2)
    k_constructor(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    __shared__ float best_s[21][kTlThreads];  // state + covariance at the innermost backward hit
    __shared__ float pl_s[5][kTlThreads];     // forward state at the last assigned hit
    __shared__ float xs[kMaxRows];            // pad-row radii
    for (int i = threadIdx.x; i < L.R; i += blockDim.x) xs[i] = L.xr[i];
    __syncthreads();
#define BEST(i) best_s[i][threadIdx.x]
#define PL(i) pl_s[i][threadIdx.x]
    // PASS 1 takes every chain, PASS 2 the chains k_dominance listed
    // PASS 1 takes the chains in start-list order (handed out inner-first
    // they kept more lanes busy but ran slower), PASS 2 longest-first
    const int n_long = L.cnt->n_bwd;
    const int n_st = min(PASS == 1 ? L.cnt->n_starts : n_long + L.cnt->n_bwd_short, L.t_cap);
    const int lane = threadIdx.x & 31;
    int t = -1;
    int phase = 0;  // 1 forward, 2 backward
    int r = 0, r0 = 0, rk = 0, last = 0, first = 0, gap = 0, nupd = 0, gbase = 0;
    float chi2 = 0.0f;
    // y and z of the state are kept relative to the start hit (yref, zref):
    // small numbers carry the per-step rounding of binary32 far below the
    // resolution; measurements are shifted by the same reference
    float yref = 0.0f, zref = 0.0f;
    // The forward pass carries the covariance itself; the backward pass, whose
    // state is the result, carries a square-root factor (C = U U^T): for
    // short tracklets whose seed variances collapse by orders of magnitude
    // the binary32 update of C itself loses the digits that the parameters
    // at the innermost hit depend on.
    typename std::conditional<PASS == 1, Fit, FitSR>::type f;
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
    // The first step of a pass (row r0 forward, row `last` backward) is an
    // update at a known hit without a transport; it runs inside the common
    // row step, so that the warp stays converged through the update.
    bool skip_tr = false;
    // f is the state right after the latest update (no transport since).
    // The result of a pass is that state: it is stored (PL forward, BEST
    // backward) only before a step that may leave it without an update (a
    // row to search, or a known row without a hit), and at the end.
    bool fresh = false;
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
            if (lane == leader) b = atomicAdd(PASS == 1 ? &L.cnt->tl_next : &L.cnt->tl_next2, __popc(m));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (need) {
                t = b + __popc(m & ((1u << lane) - 1));
                if (t >= n_st) {
                    t = -1;
                    exhausted = true;
                } else if (PASS == 2) {
                    t = list_at(L, t, n_long);
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
            const float2 c0 = L.hyz[ch.x];
            yref = c0.x;
            zref = c0.y;
            gap = 0;
            fresh = false;
            skip_tr = true;
            pknown = true;
            if (PASS == 2) {
                // backward from the last hit with the covariance reset to the
                // seed, starting from the forward state left in the header;
                // the first step updates at the last hit
                const TrackletHdr& H = L.tl[t];
                last = H.last;
#pragma unroll
                for (int i = 0; i < 5; ++i) f.p[i] = H.p[i];
                seed_cov(f, L);
                f.x = xs[last];
                ph = rowhit[last];
                pyz = L.hyz[ph];
                ph2 = last - 1 >= r0 ? rowhit[last - 1] : -1;
                chi2 = 0.0f;
                nupd = 0;
                first = last;
                phase = 2;
                r = last;
            } else {
                // seed from the chord h0 -> hk; the first step updates at h0
                const int h1 = rk > r0 ? rowhit[r0 + 1] : -1;
                const float2 ck = L.hyz[ch.z];
                const float x0 = xs[r0], x1 = xs[rk];
                const float tphi = (ck.x - c0.x) / (x1 - x0);
                const float dzdx = (ck.y - c0.y) / (x1 - x0);
                const float cphi = rsqrtf(1.0f + tphi * tphi);
                f.x = x0;
                f.p[0] = 0.0f;
                f.p[1] = 0.0f;
                f.p[2] = tphi * cphi;
                f.p[3] = dzdx * cphi;
                f.p[4] = 0.0f;
                seed_cov(f, L);
                ph = ch.x;
                pyz = c0;
                ph2 = h1;
                last = r0;
                phase = 1;
                r = r0;
            }
        }
        // ---- one row step of the current pass ----
        constexpr bool fwd = PASS == 1;
        bool end_pass = fwd ? r >= L.R : r < 0;
        if (!end_pass) {
            const bool known = pknown;
            const int base = pb;
            const RowGrid G = pG;
            float my = pyz.x - yref, mz = pyz.y - zref;
            int h = known ? ph : -1;
            const int rn = fwd ? r + 1 : r - 1;
            if (fwd ? rn < L.R : rn >= 0) stage(rn, fwd);
            if (!skip_tr) {
                if (fresh && !(known && h >= 0)) {
                    // the step may leave the state of the latest update
                    if (fwd) {
#pragma unroll
                        for (int i = 0; i < 5; ++i) PL(i) = f.p[i];
                    } else {
                        save_best(f, best_s);
                    }
                    fresh = false;
                }
                // a failed transport leaves f as it was
                if (!transport(f, xs[r], L)) end_pass = true;
                else fresh = false;
            }
            skip_tr = false;
            if (!end_pass) {
                if (!known) {
                    if (outside(f, yref, zref, L)) end_pass = true;
                    else h = search(f, yref, zref, G, base, L, my, mz);
                }
                if (!end_pass) {
                    if (h >= 0) {
                        const float dchi2 = update(f, my, mz, L);
                        fresh = true;
                        if (fwd) {
                            if (!known) {
                                rowhit[r] = h;
                                L.mark[h] = 1;  // taken by a forward extension search
                            }
                            last = r;
                        } else {
                            chi2 += dchi2;
                            ++nupd;
                            if (!known) rowhit[r] = h;  // a known row holds h already
                            first = r;
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
            // forward pass done: the state at the last hit (relative to the
            // start hit) and the last row wait in the header for PASS 2
            TrackletHdr& H = L.tl[t];
            if (fresh) {
#pragma unroll
                for (int i = 0; i < 5; ++i) H.p[i] = f.p[i];
            } else {
#pragma unroll
                for (int i = 0; i < 5; ++i) H.p[i] = PL(i);
            }
            H.last = last;
            t = -1;
            phase = 0;
            continue;
        }
        if (fresh) save_best(f, best_s);
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

// Chains whose forward range (last assigned row - start row) spans at least
// this many rows are handed to the backward pass first.
constexpr int kBwdLongRows = 64;

// Dominance: one thread per chain.  A chain long enough for a tracklet all
// of whose hits were taken by forward extension searches (of other
// tracklets: a tracklet's own extension starts above its chain) gets no
// tracklet and its header is made final; the others are listed for the
// backward pass (warp-aggregated), whose warps then hold only tracklets to
// refit.  The hits are read four rows at a time (independent loads) and the
// scan stops at the first hit no extension took.
__global__ void k_dominance(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    int n_dom = 0;
    // whole warps step together (ballot below)
    for (int t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < n_st; t0 += stride) {
        const int t = t0 + lane;
        bool keep = false, longr = false;
        if (t < n_st) {
            const int4 ch = L.tl_chain[t];
            const int r0 = ch.y & 255, rk = ch.w;
            if (rk - r0 + 1 >= L.min_chain) {
                const int* rowhit = L.tl_rowhit + (size_t)t * L.R;
                for (int r = r0; r <= rk && !keep; r += 4) {
                    int h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) h[j] = r + j <= rk ? rowhit[r + j] : -1;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (h[j] >= 0 && !L.mark[h[j]]) keep = true;
                }
                if (keep) {
                    longr = L.tl[t].last - r0 >= kBwdLongRows;
                } else {
                    TrackletHdr& H = L.tl[t];
                    H.dominated = 1;
                    H.valid = 0;
                    H.nhits = 0;
                    H.first = -1;
                    H.last = -1;
                    H.ndf = 0;
                    ++n_dom;
                }
            }
        }
        const unsigned ml = __ballot_sync(0xffffffffu, keep && longr);
        const unsigned ms = __ballot_sync(0xffffffffu, keep && !longr);
        if (ml | ms) {
            int bl = 0, bs = 0;
            if (lane == 0) {
                if (ml) bl = atomicAdd(&L.cnt->n_bwd, __popc(ml));
                if (ms) bs = atomicAdd(&L.cnt->n_bwd_short, __popc(ms));
            }
            bl = __shfl_sync(0xffffffffu, bl, 0);
            bs = __shfl_sync(0xffffffffu, bs, 0);
            const unsigned below = (1u << lane) - 1;
            if (keep && longr) L.tl_list[bl + __popc(ml & below)] = t;
            if (keep && !longr) L.tl_list[L.t_cap - 1 - (bs + __popc(ms & below))] = t;
        }
    }
    // block totals
    __shared__ int red;
    if (threadIdx.x == 0) red = 0;
    __syncthreads();
    if (n_dom) atomicAdd(&red, n_dom);
    __syncthreads();
    if (threadIdx.x == 0 && red) {
        atomicAdd(&L.cnt->n_dominated, red);
        atomicSub(&L.cnt->n_tracklets, red);
    }
}

// Hit weights: one warp per tracklet, lanes over its rows; every hit of a
// valid tracklet gets atomicMax(weight, (nHits << 32) | (0xFFFFFFFF - cid(h0))).
// (Slots are taken in order: fed from the backward pass's list instead, in
// its arbitrary order, the kernel was 1.5x slower.)
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

}  // namespace

// Resident blocks per SM of each constructor pass (the passes have
// different register counts; each is capped by its own).
static int pass_occupancy(int pass)
{
    int a = 0;
    if (pass == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_constructor<1>, kTlThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_constructor<2>, kTlThreads, 0);
    return a < 1 ? 1 : a;
}

// The schedule's range of constructor blocks per SM: up to the larger of
// the two passes' occupancies.
// (Queried when a context is created, before any stream capture.)
static std::atomic<int> g_occ1{0}, g_occ2{0};

int constructor_occupancy()
{
    const int a = pass_occupancy(1), b = pass_occupancy(2);
    g_occ1 = a;
    g_occ2 = b;
    return a > b ? a : b;
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
    const int occ1 = g_occ1 > 0 ? (int)g_occ1 : per_sm, occ2 = g_occ2 > 0 ? (int)g_occ2 : per_sm;
    const int need = (L.t_cap + kTlThreads - 1) / kTlThreads;
    auto grid = [&](int occ) {
        int b = (per_sm < occ ? per_sm : occ) * n_sm;
        if (b > need) b = need;
        return b < 1 ? 1 : b;
    };
    k_constructor<1><<<grid(occ1), kTlThreads, 0, stream>>>(L);
    hook_after(hook, "k_constructor_fwd");
    {
        int db = (L.t_cap + 255) / 256;
        if (db > n_sm * 8) db = n_sm * 8;
        if (db < 1) db = 1;
        k_dominance<<<db, 256, 0, stream>>>(L);
        hook_after(hook, "k_dominance");
    }
    k_constructor<2><<<grid(occ2), kTlThreads, 0, stream>>>(L);
    hook_after(hook, "k_constructor_bwd");
    int wblocks = (L.t_cap + 7) / 8;
    if (wblocks > n_sm * 16) wblocks = n_sm * 16;
    if (wblocks < 1) wblocks = 1;
    k_weights<<<wblocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_weights");
}

}  // namespace tpc
