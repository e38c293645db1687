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
// entries live in registers; the forward hit list of the chain lives in
// shared memory (one int16 column per thread).  Valid tracklets raise the
// weight of their hits to the key (nHits << 32 | ~cid(h0)) with atomicMax.
//
// Arithmetic is binary32.  Transport between planes x0 -> x1 (dx = x1 - x0):
//   s1 = s0 + C_k dx, C_k = -kB q/pT;  y1 = y0 + dx (s0 + s1)/(c0 + c1);
//   dS = chord * asin(h)/h (h = |C_k| chord / 2), signed like dx;  z1 = z0 + t dS,
// with the exact Jacobian; d(dS)/dC_k is evaluated as
//   dS^2 [ (s1/c1) sinc^2(dphi/2) / 2 + (sin dphi - dphi)/dphi^2 ],  dphi = C_k dS,
// a form without cancellation as C_k -> 0.
// Bytes per assigned hit: chain link 2, y z 8 (forward) + 8 (backward), rowhit
// 2, weight read-modify-write 16, header about 100 per tracklet.
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
    const float c0 = sqrtf((1.0f - s0) * (1.0f + s0));
    const float c1 = sqrtf((1.0f - s1) * (1.0f + s1));
    const float cc = c0 + c1;
    const float icc = 1.0f / cc;
    const float ss = s0 + s1;
    const float dy = dx * ss * icc;
    const float ch = sqrtf(dx * dx + dy * dy);
    const float h = 0.5f * fabsf(ck) * ch;
    float ratio;
    if (h < 0.03f) {
        const float h2 = h * h;
        ratio = 1.0f + h2 * (1.0f / 6.0f + h2 * (3.0f / 40.0f));
    } else {
        ratio = asinf(h) / h;
    }
    float dS = ch * ratio;
    if (dx < 0.0f) dS = -dS;
    const float t = f.p[3];
    const float ic0 = 1.0f / c0, ic1 = 1.0f / c1;
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
        const float hs = sinf(0.5f * dphi) / (0.5f * dphi);
        sinc2 = hs * hs;
        rest = (sinf(dphi) - dphi) / u2;
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
    const float id = 1.0f / (S00 * S11 - S01 * S01);
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

// Least-chi2 hit of row g with chi2 <= chi2_hit (exact ties to the lower
// cid); returns its row-local index or -1.
__device__ __forceinline__ int search(const Fit& f, int g, const Launch& L)
{
    const float* C = f.C;
    const float S00 = C[0] + L.sy2, S01 = C[1], S11 = C[2] + L.sz2;
    const float id = 1.0f / (S00 * S11 - S01 * S01);
    const float wy = 1.01f * sqrtf(L.chi2_hit * S00) + 1e-3f;
    const float wz = 1.01f * sqrtf(L.chi2_hit * S11) + 1e-3f;
    const RowGrid G = L.grid[g];
    const int base = L.row_off[g];
    const int* bins = L.bin_start + G.bin_off;
    const int y0 = bin_y(G, f.p[0] - wy), y1 = bin_y(G, f.p[0] + wy);
    const int z0 = bin_z(G, f.p[1] - wz), z1 = bin_z(G, f.p[1] + wz);
    float best = 3.0e38f;
    int bk = -1, bc = 0x7fffffff;
    for (int bz = z0; bz <= z1; ++bz) {
        const int ka = bins[bz * G.ny + y0], kb = bins[bz * G.ny + y1 + 1];
        for (int k = ka; k < kb; ++k) {
            const float r0 = L.hy[base + k] - f.p[0];
            const float r1 = L.hz[base + k] - f.p[1];
            const float chi2 = (S11 * r0 * r0 - 2.0f * S01 * r0 * r1 + S00 * r1 * r1) * id;
            if (chi2 < best || (chi2 == best && L.hcid[base + k] < bc)) {
                best = chi2;
                bk = k;
                bc = L.hcid[base + k];
            }
        }
    }
    return (bk >= 0 && best <= L.chi2_hit) ? bk : -1;
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

__global__ void __launch_bounds__(kTlThreads) k_constructor(Launch L)
{
    extern __shared__ int16_t fl_s[];  // [R][kTlThreads]
    const int n_st = min(L.cnt->n_starts, L.t_cap);
    int my_tracklets = 0, my_valid = 0, my_hits = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_st; t += gridDim.x * blockDim.x) {
        int16_t* fl = fl_s + threadIdx.x;
#define FL(r) fl[(r) * kTlThreads]
        const int s = L.starts[t];
        const int hr = L.hrow[s];
        const int gbase = (hr >> 8) * L.R;
        const int r0 = hr & 255;
        TrackletHdr& H = L.tl[t];
        // follow the chain of cleaned up-links
        FL(r0) = (int16_t)(s - L.row_off[gbase + r0]);
        int cur = s, r = r0;
        while (r < L.R - 1) {
            const int u = L.upc[cur];
            if (u < 0) break;
            ++r;
            cur = L.row_off[gbase + r] + u;
            FL(r) = (int16_t)u;
        }
        const int rk = r;
        const int len = rk - r0 + 1;
        H.start = s;
        H.chain_len = len;
        if (len < L.min_chain) {
            H.valid = 0;
            H.nhits = 0;
            H.first = -1;
            H.last = -1;
            H.ndf = 0;
            continue;
        }
        ++my_tracklets;
        // seed from the chord h0 -> hk
        Fit f;
        {
            const float x0 = L.row_x[r0], x1 = L.row_x[rk];
            const float y0 = L.hy[s], z0 = L.hz[s];
            const float tphi = (L.hy[cur] - y0) / (x1 - x0);
            const float dzdx = (L.hz[cur] - z0) / (x1 - x0);
            const float cphi = 1.0f / sqrtf(1.0f + tphi * tphi);
            f.x = x0;
            f.p[0] = y0;
            f.p[1] = z0;
            f.p[2] = tphi * cphi;
            f.p[3] = dzdx * cphi;
            f.p[4] = 0.0f;
            seed_cov(f, L);
            update(f, y0, z0, L);
        }
        float pL[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) pL[i] = f.p[i];
        int last = r0;
        bool stopped = false;
        // forward pass over the chain (no test)
        for (r = r0 + 1; r <= rk; ++r) {
            const int hidx = L.row_off[gbase + r] + FL(r);
            const float my = L.hy[hidx], mz = L.hz[hidx];
            if (!transport(f, L.row_x[r], L)) {
                stopped = true;
                break;
            }
            update(f, my, mz, L);
            last = r;
#pragma unroll
            for (int i = 0; i < 5; ++i) pL[i] = f.p[i];
        }
        // forward extension
        if (!stopped) {
            int gap = 0;
            for (r = rk + 1; r < L.R; ++r) {
                if (!transport(f, L.row_x[r], L)) break;
                if (outside(f, L)) break;
                const int k = search(f, gbase + r, L);
                if (k >= 0) {
                    const int hidx = L.row_off[gbase + r] + k;
                    update(f, L.hy[hidx], L.hz[hidx], L);
                    FL(r) = (int16_t)k;
                    last = r;
#pragma unroll
                    for (int i = 0; i < 5; ++i) pL[i] = f.p[i];
                    gap = 0;
                } else {
                    FL(r) = (int16_t)-1;
                    if (++gap >= L.max_gap) break;
                }
            }
        }
        // backward pass from the last hit, covariance reset to the seed
        int16_t* rowhit = L.tl_rowhit + (size_t)t * L.R;
#pragma unroll
        for (int i = 0; i < 5; ++i) f.p[i] = pL[i];
        seed_cov(f, L);
        f.x = L.row_x[last];
        float chi2;
        {
            const int hidx = L.row_off[gbase + last] + FL(last);
            chi2 = update(f, L.hy[hidx], L.hz[hidx], L);
        }
        int nupd = 1, first = last;
        rowhit[last] = FL(last);
        Fit best = f;
        bool ok = true;
        for (r = last - 1; r >= r0; --r) {
            const int k = FL(r);
            if (k < 0) {
                rowhit[r] = -1;
                continue;
            }
            const int hidx = L.row_off[gbase + r] + k;
            const float my = L.hy[hidx], mz = L.hz[hidx];
            if (!transport(f, L.row_x[r], L)) {
                ok = false;
                break;
            }
            chi2 += update(f, my, mz, L);
            ++nupd;
            rowhit[r] = (int16_t)k;
            first = r;
            best = f;
        }
        if (ok) {
            int gap = 0;
            for (r = r0 - 1; r >= 0; --r) {
                if (!transport(f, L.row_x[r], L)) break;
                if (outside(f, L)) break;
                const int k = search(f, gbase + r, L);
                if (k >= 0) {
                    const int hidx = L.row_off[gbase + r] + k;
                    chi2 += update(f, L.hy[hidx], L.hz[hidx], L);
                    ++nupd;
                    rowhit[r] = (int16_t)k;
                    first = r;
                    best = f;
                    gap = 0;
                } else {
                    rowhit[r] = -1;
                    if (++gap >= L.max_gap) break;
                }
            }
        }
#undef FL
        bool fin = isfinite(chi2);
#pragma unroll
        for (int i = 0; i < 5; ++i) fin = fin && isfinite(best.p[i]);
#pragma unroll
        for (int i = 0; i < 15; ++i) fin = fin && isfinite(best.C[i]);
#pragma unroll
        for (int i = 0; i < 5; ++i) fin = fin && best.C[CI(i, i)] > 0.0f;
        const bool valid = nupd >= L.min_tracklet_hits && fin;
        H.x = best.x;
#pragma unroll
        for (int i = 0; i < 5; ++i) H.p[i] = best.p[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) H.C[i] = best.C[i];
        H.chi2 = chi2;
        H.nhits = nupd;
        H.first = first;
        H.last = last;
        H.ndf = 2 * nupd - 5;
        H.valid = valid ? 1 : 0;
        if (valid) {
            ++my_valid;
            my_hits += nupd;
            const unsigned long long key = ((unsigned long long)nupd << 32) |
                                           (unsigned long long)(0xFFFFFFFFu - (unsigned)L.hcid[s]);
            for (int rr = first; rr <= last; ++rr) {
                const int k = rowhit[rr];
                if (k >= 0) atomicMax(&L.weight[L.row_off[gbase + rr] + k], key);
            }
        }
    }
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

}  // namespace

void launch_constructor(const Launch& L, void* stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const size_t sm = (size_t)L.R * kTlThreads * sizeof(int16_t);
    cudaFuncSetAttribute(k_constructor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int blocks = (L.t_cap + kTlThreads - 1) / kTlThreads;
    if (blocks > 148 * 12) blocks = 148 * 12;
    if (blocks < 1) blocks = 1;
    k_constructor<<<blocks, kTlThreads, sm, stream>>>(L);
}

}  // namespace tpc
