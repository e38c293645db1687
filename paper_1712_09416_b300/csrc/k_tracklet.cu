// k_tracklet.cu -- tracklet construction: the Kalman-filter part of the
// sector tracker (paper, Abstract), one thread per chain like the paper's
// one-thread-per-track fit (Sect. 4.1, Listing 2).
//
// For every start hit the thread follows the chain of cleaned up-links, seeds
// a state (y, z, sin phi, tan lambda, q/pT) from the chord of the chain, fits
// the chain forward, extends it outward row by row (transport to the pad-row
// plane, least-chi2 hit in the box that bounds the chi2 ellipse, update), then
// refits backward from the last hit with the covariance reset to the seed,
// picking up hits below the chain the same way.  The result is the state and
// covariance at the innermost hit.  The 5-vector and the 15 covariance
// entries live in registers; the forward hit list lives in the tracklet's
// rowhit slot and the inputs of the next row are loaded one step ahead.  Valid tracklets raise the
// weight of their hits to the key (nHits << 32 | ~cid(h0)) with atomicMax.
//
// Arithmetic is binary32.  Transport between planes x0 -> x1 (dx = x1 - x0):
//   s1 = s0 + C_k dx, C_k = -kB q/pT;  y1 = y0 + dx (s0 + s1)/(c0 + c1);
//   dS = chord * asin(h)/h (h = |C_k| chord / 2), signed like dx;  z1 = z0 + t dS,
// with the exact Jacobian; d(dS)/dC_k is evaluated as
//   dS^2 [ (s1/c1) sinc^2(dphi/2) / 2 + (sin dphi - dphi)/dphi^2 ],  dphi = C_k dS,
// a form without cancellation as C_k -> 0.
// Bytes per assigned hit: chain link 4, y z 8 (forward) + 8 (backward), rowhit
// 4, weight read-modify-write 16, header about 100 per tracklet.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"

namespace tpc {

namespace {

constexpr int kTlThreads = 64;

// lower-triangle index of (i, j), i >= j
#define CI(i, j) ((i) * ((i) + 1) / 2 + (j))

struct Fit {
    float x;
    float p[5];
    float C[15];
};

__device__ __forceinline__ float cget(const float* C, int i, int j)
{
    return i >= j ? C[CI(i, j)] : C[CI(j, i)];
}

__device__ __forceinline__ bool transport(Fit& f, float x1, const Launch& L)
{
    const float dx = x1 - f.x;
    const float ck = -L.kB * f.p[4];
    const float s0 = f.p[2];
    const float s1 = s0 + ck * dx;
    if (!(fabsf(s1) < L.sin_max) || !(fabsf(s0) < L.sin_max)) return false;
    const float q0 = (1.0f - s0) * (1.0f + s0), q1 = (1.0f - s1) * (1.0f + s1);
    const float ic0 = rsqrtf(q0), ic1 = rsqrtf(q1);
    const float c0 = q0 * ic0, c1 = q1 * ic1;
    const float cc = c0 + c1;
    const float icc = __fdividef(1.0f, cc);
    const float ss = s0 + s1;
    const float dy = dx * ss * icc;
    const float ch = sqrtf(dx * dx + dy * dy);
    const float h = 0.5f * fabsf(ck) * ch;
    float ratio;
    if (h < 0.03f) {
        const float h2 = h * h;
        ratio = 1.0f + h2 * (1.0f / 6.0f + h2 * (3.0f / 40.0f));
    } else {
        ratio = __fdividef(asinf(h), h);
    }
    float dS = ch * ratio;
    if (dx < 0.0f) dS = -dS;
    const float t = f.p[3];
    const float a = dx * (2.0f * cc + ss * (s0 * ic0 + s1 * ic1)) * (icc * icc);
    const float b = -L.kB * dx * dx * (cc + ss * s1 * ic1) * (icc * icc);
    const float c = t * dx * ss * ic0 * ic1 * icc;
    const float d = dS;
    const float dphi = ck * dS;
    const float u2 = dphi * dphi;
    float sinc2, rest;
    if (fabsf(dphi) < 0.2f) {
        sinc2 = 1.0f - u2 * (1.0f / 12.0f - u2 * (1.0f / 360.0f));
        rest = dphi * (-1.0f / 6.0f + u2 * (1.0f / 120.0f - u2 * (1.0f / 5040.0f)));
    } else {
        const float hs = __fdividef(sinf(0.5f * dphi), 0.5f * dphi);
        sinc2 = hs * hs;
        rest = __fdividef(sinf(dphi) - dphi, u2);
    }
    const float dSdC = dS * dS * (0.5f * s1 * ic1 * sinc2 + rest);
    const float e = -L.kB * t * dSdC;
    const float g = -L.kB * dx;

    f.p[0] += dy;
    f.p[1] += t * dS;
    f.p[2] = s1;
    f.x = x1;

    float* C = f.C;
    const float C00 = C[0], C10 = C[1], C11 = C[2], C20 = C[3], C21 = C[4], C22 = C[5];
    const float C30 = C[6], C31 = C[7], C32 = C[8], C33 = C[9];
    const float C40 = C[10], C41 = C[11], C42 = C[12], C43 = C[13], C44 = C[14];
    // T = J C (rows 0..2 change)
    const float T00 = C00 + a * C20 + b * C40;
    const float T02 = C20 + a * C22 + b * C42;
    const float T04 = C40 + a * C42 + b * C44;
    const float T10 = C10 + c * C20 + d * C30 + e * C40;
    const float T11 = C11 + c * C21 + d * C31 + e * C41;
    const float T12 = C21 + c * C22 + d * C32 + e * C42;
    const float T13 = C31 + c * C32 + d * C33 + e * C43;
    const float T14 = C41 + c * C42 + d * C43 + e * C44;
    const float T20 = C20 + g * C40;
    const float T21 = C21 + g * C41;
    const float T22 = C22 + g * C42;
    const float T23 = C32 + g * C43;
    const float T24 = C42 + g * C44;
    // C' = T J^T, lower triangle
    C[0] = T00 + a * T02 + b * T04;
    C[1] = T10 + a * T12 + b * T14;
    C[2] = T11 + c * T12 + d * T13 + e * T14;
    C[3] = T20 + a * T22 + b * T24;
    C[4] = T21 + c * T22 + d * T23 + e * T24;
    C[5] = T22 + g * T24;
    C[6] = C30 + a * C32 + b * C43;
    C[7] = C31 + c * C32 + d * C33 + e * C43;
    C[8] = C32 + g * C43;
    C[9] = C33;
    C[10] = C40 + a * C42 + b * C44;
    C[11] = C41 + c * C42 + d * C43 + e * C44;
    C[12] = C42 + g * C44;
    C[13] = C43;
    C[14] = C44;
    return true;
}

// Kalman update with measurement (my, mz); returns the chi2 increment.
__device__ __forceinline__ float update(Fit& f, float my, float mz, const Launch& L)
{
    float* C = f.C;
    const float S00 = C[0] + L.sy2, S01 = C[1], S11 = C[2] + L.sz2;
    const float id = __fdividef(1.0f, S00 * S11 - S01 * S01);
    const float I00 = S11 * id, I01 = -S01 * id, I11 = S00 * id;
    const float r0 = my - f.p[0], r1 = mz - f.p[1];
    float c0[5], c1[5];  // old columns 0 and 1
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        c0[i] = cget(C, i, 0);
        c1[i] = cget(C, i, 1);
    }
    float K0[5], K1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        K0[i] = c0[i] * I00 + c1[i] * I01;
        K1[i] = c0[i] * I01 + c1[i] * I11;
        f.p[i] += K0[i] * r0 + K1[i] * r1;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) C[CI(i, j)] -= K0[i] * c0[j] + K1[i] * c1[j];
    return r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
}

__device__ __forceinline__ bool outside(const Fit& f, const Launch& L)
{
    return fabsf(f.p[0]) > f.x * L.tan_half + L.edge_margin ||
           fabsf(f.p[1]) > L.z_max + L.edge_margin;
}

// Bin offsets of the search window of the next row, loaded one step ahead
// from the position predicted along the current direction (with a margin);
// used when the exact window falls inside the predicted one.
struct Spec {
    int y0, y1, z0, z1;  // predicted bin ranges (z1 <= z0 + 1)
    int a0, b0, a1, b1;  // row-local hit ranges of z-bins z0 and z0 + 1
    bool valid;
};

__device__ __forceinline__ void scan_range(const Fit& f, int ka, int kb, float S00, float S01,
                                           float S11, float id, const Launch& L, float& best,
                                           int& bk, float& by, float& bzv)
{
    for (int k = ka; k < kb; k += 4) {
        float cy[4], cz[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kk = k + j < kb ? k + j : ka;
            cy[j] = L.hy[kk];
            cz[j] = L.hz[kk];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k + j >= kb) break;
            const float r0 = cy[j] - f.p[0];
            const float r1 = cz[j] - f.p[1];
            const float chi2 = (S11 * r0 * r0 - 2.0f * S01 * r0 * r1 + S00 * r1 * r1) * id;
            // exact ties (rare) go to the lower cid; the cid is read only then
            if (chi2 < best || (chi2 == best && L.hcid[k + j] < L.hcid[bk])) {
                best = chi2;
                bk = k + j;
                by = cy[j];
                bzv = cz[j];
            }
        }
    }
}

// Least-chi2 hit of a row (grid G, hits from base) with chi2 <= chi2_hit,
// exact ties to the lower cid; returns its global index or -1 and its
// coordinates in (my, mz).  Every hit in the bins covering the box that
// bounds the chi2 ellipse is tried (a superset when the prefetched bins of
// the predicted window are used).
__device__ __forceinline__ int search(const Fit& f, const RowGrid& G, int base, const Spec& sp,
                                      const Launch& L, float& my, float& mz)
{
    const float* C = f.C;
    const float S00 = C[0] + L.sy2, S01 = C[1], S11 = C[2] + L.sz2;
    const float id = __fdividef(1.0f, S00 * S11 - S01 * S01);
    const float wy = 1.01f * sqrtf(L.chi2_hit * S00) + 1e-3f;
    const float wz = 1.01f * sqrtf(L.chi2_hit * S11) + 1e-3f;
    const int y0 = bin_y(G, f.p[0] - wy), y1 = bin_y(G, f.p[0] + wy);
    const int z0 = bin_z(G, f.p[1] - wz), z1 = bin_z(G, f.p[1] + wz);
    float best = 3.0e38f, by = 0.0f, bzv = 0.0f;
    int bk = -1;
    if (sp.valid && y0 >= sp.y0 && y1 <= sp.y1 && z0 >= sp.z0 && z1 <= sp.z1) {
        scan_range(f, base + sp.a0, base + sp.b0, S00, S01, S11, id, L, best, bk, by, bzv);
        if (sp.z1 > sp.z0)
            scan_range(f, base + sp.a1, base + sp.b1, S00, S01, S11, id, L, best, bk, by, bzv);
    } else {
        const int* bins = L.bin_start + G.bin_off;
        for (int bz = z0; bz <= z1; ++bz) {
            const int ka = base + bins[bz * G.ny + y0], kb = base + bins[bz * G.ny + y1 + 1];
            scan_range(f, ka, kb, S00, S01, S11, id, L, best, bk, by, bzv);
        }
    }
    my = by;
    mz = bzv;
    return (bk >= 0 && best <= L.chi2_hit) ? bk : -1;
}

// Predicted window of the row at xn from the current state, and the loads of
// its bin offsets.
__device__ __forceinline__ void speculate(const Fit& f, float xn, const RowGrid& G, const Launch& L,
                                          Spec& sp)
{
    const float s = f.p[2];
    const float c2 = (1.0f - s) * (1.0f + s);
    const float ic = rsqrtf(fmaxf(c2, 1e-4f));
    const float dx = xn - f.x;
    const float yp = f.p[0] + dx * s * ic, zp = f.p[1] + dx * f.p[3] * ic;
    const float wy = sqrtf(L.chi2_hit * (f.C[0] + L.sy2)) + 0.5f + 0.1f * fabsf(dx);
    const float wz = sqrtf(L.chi2_hit * (f.C[2] + L.sz2)) + 0.5f + 0.1f * fabsf(dx);
    sp.y0 = bin_y(G, yp - wy);
    sp.y1 = bin_y(G, yp + wy);
    sp.z0 = bin_z(G, zp - wz);
    sp.z1 = min(bin_z(G, zp + wz), sp.z0 + 1);
    const int* bins = L.bin_start + G.bin_off;
    sp.a0 = bins[sp.z0 * G.ny + sp.y0];
    sp.b0 = bins[sp.z0 * G.ny + sp.y1 + 1];
    if (sp.z1 > sp.z0) {
        sp.a1 = bins[sp.z1 * G.ny + sp.y0];
        sp.b1 = bins[sp.z1 * G.ny + sp.y1 + 1];
    } else {
        sp.a1 = sp.b1 = 0;
    }
    sp.valid = true;
}

// Seed covariance at the current direction: diagonal, cluster variances for
// (y, z), slope variances of dy/dx and dz/dx carried over to sin(phi) and
// tan(lambda) (factors cos^6 phi and cos^2 phi), seed_var_q for q/pT.
__device__ __forceinline__ void seed_cov(Fit& f, const Launch& L)
{
    const float c2 = (1.0f - f.p[2]) * (1.0f + f.p[2]);
#pragma unroll
    for (int i = 0; i < 15; ++i) f.C[i] = 0.0f;
    f.C[CI(0, 0)] = L.sy2;
    f.C[CI(1, 1)] = L.sz2;
    f.C[CI(2, 2)] = L.seed_var_s * c2 * c2 * c2;
    f.C[CI(3, 3)] = L.seed_var_t * c2;
    f.C[CI(4, 4)] = L.seed_var_q;
}

// Persistent lanes: every lane owns one tracklet at a time and advances it by
// one pad row per loop iteration, forward (chain hits, then search) and then
// backward (assigned hits, then search below the chain).  Lanes of a warp run
// the same row-step code whatever the pass, and a lane whose tracklet is done
// takes the next start hit at once, so the warp stays converged.
__global__ void __launch_bounds__(kTlThreads) k_constructor(Launch L)
{
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
    Fit f;
    // The tracklet's rowhit slot holds the hit of every row the forward pass
    // visits (global index, -1 none) and yz its coordinates; the backward
    // pass reads both one step ahead and rewrites rowhit in place.
    int* rowhit = nullptr;
    float2* yz = nullptr;
    // inputs of the next row to process, loaded one step ahead
    bool pknown = false;
    int pb = 0, ph = -1;
    float2 pyz = make_float2(0.0f, 0.0f);
    RowGrid pG;
    Spec sp;
    sp.valid = false;
    int my_tracklets = 0, my_valid = 0, my_hits = 0;

    auto load_row = [&](int rr, bool fwdp) {
        pknown = fwdp ? rr <= rk : rr >= r0;
        pb = L.row_off[gbase + rr];
        if (pknown) {
            ph = rowhit[rr];
            pyz = yz[rr];
        } else {
            pG = L.grid[gbase + rr];
        }
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
            const int s = L.starts[t];
            const int hr = L.hrow[s];
            gbase = (hr >> 8) * L.R;
            r0 = hr & 255;
            TrackletHdr& H = L.tl[t];
            rowhit = L.tl_rowhit + (size_t)t * L.R;
            yz = L.tl_yz + (size_t)t * L.R;
            // follow the chain, recording its hits and their coordinates
            float2 c0 = make_float2(L.hy[s], L.hz[s]);
            rowhit[r0] = s;
            yz[r0] = c0;
            float2 ck = c0;
            int cur = s, rr = r0;
            while (rr < L.R - 1) {
                const int u = L.upg[cur];
                if (u < 0) break;
                ++rr;
                cur = u;
                ck = make_float2(L.hy[u], L.hz[u]);
                rowhit[rr] = u;
                yz[rr] = ck;
            }
            rk = rr;
            const int len = rk - r0 + 1;
            H.start = s;
            H.chain_len = len;
            if (len < L.min_chain) {
                H.valid = 0;
                H.nhits = 0;
                H.first = -1;
                H.last = -1;
                H.ndf = 0;
                t = -1;
                continue;
            }
            ++my_tracklets;
            // seed from the chord h0 -> hk, update at h0
            const float x0 = xs[r0], x1 = xs[rk];
            const float tphi = (ck.x - c0.x) / (x1 - x0);
            const float dzdx = (ck.y - c0.y) / (x1 - x0);
            const float cphi = rsqrtf(1.0f + tphi * tphi);
            f.x = x0;
            f.p[0] = c0.x;
            f.p[1] = c0.y;
            f.p[2] = tphi * cphi;
            f.p[3] = dzdx * cphi;
            f.p[4] = 0.0f;
            seed_cov(f, L);
            update(f, c0.x, c0.y, L);
#pragma unroll
            for (int i = 0; i < 5; ++i) PL(i) = f.p[i];
            last = r0;
            gap = 0;
            r = r0 + 1;
            phase = 1;
            sp.valid = false;
            if (r < L.R) load_row(r, true);
        }
        // ---- one row step of the current pass ----
        const bool fwd = phase == 1;
        bool end_pass = fwd ? r >= L.R : r < 0;
        if (!end_pass) {
            const bool known = pknown;
            const int base = pb;
            const RowGrid G = pG;
            const Spec spc = sp;
            float my = pyz.x, mz = pyz.y;
            int h = known ? ph : -1;
            const int rn = fwd ? r + 1 : r - 1;
            const bool has_next = fwd ? rn < L.R : rn >= 0;
            if (has_next) load_row(rn, fwd);
            sp.valid = false;
            if (!transport(f, xs[r], L)) {
                end_pass = true;
            } else {
                if (!known) {
                    if (outside(f, L)) end_pass = true;
                    else h = search(f, G, base, spc, L, my, mz);
                }
                if (!end_pass) {
                    if (h >= 0) {
                        const float dchi2 = update(f, my, mz, L);
                        if (fwd) {
                            if (!known) {
                                rowhit[r] = h;
                                yz[r] = make_float2(my, mz);
                            }
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
                    if (!end_pass && has_next && !pknown) speculate(f, xs[rn], pG, L, sp);
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
            const float2 c = yz[last];
            chi2 = update(f, c.x, c.y, L);
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
            sp.valid = false;
            if (r >= 0) load_row(r, false);
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
    __shared__ int red[3];
    if (threadIdx.x == 0) red[0] = red[1] = red[2] = 0;
    __syncthreads();
    if (my_tracklets) atomicAdd(&red[0], my_tracklets);
    if (my_valid) atomicAdd(&red[1], my_valid);
    if (my_hits) atomicAdd(&red[2], my_hits);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (red[0]) atomicAdd(&L.cnt->n_tracklets, red[0]);
        if (red[1]) atomicAdd(&L.cnt->n_valid, red[1]);
        if (red[2]) atomicAdd(&L.cnt->n_tracklet_hits, red[2]);
    }
}

// Hit weights: one warp per tracklet, lanes over its rows; every hit of a
// valid tracklet gets atomicMax(weight, (nHits << 32) | (0xFFFFFFFF - cid(h0))).
__global__ void k_weights(Launch L)
{
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

void launch_constructor(const Launch& L, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t sm = 0;
    // persistent: as many blocks as fit on the GPU at once
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_constructor, kTlThreads, sm);
        if (per_sm < 1) per_sm = 1;
    }
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int blocks = per_sm * n_sm;
    const int need = (L.t_cap + kTlThreads - 1) / kTlThreads;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k_constructor<<<blocks, kTlThreads, sm, stream>>>(L);
    hook_after(hook, "k_constructor");
    int wblocks = (L.t_cap + 7) / 8;
    if (wblocks > n_sm * 16) wblocks = n_sm * 16;
    if (wblocks < 1) wblocks = 1;
    k_weights<<<wblocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_weights");
}

}  // namespace tpc
