// tpc_fit.cuh -- binary32 track-fit arithmetic shared by the tracklet
// constructor and the sector track merger: the state (x; y, z, sin phi,
// tan lambda, q/pT) with its 15-entry covariance, helix transport between
// planes x0 -> x1 with its exact Jacobian, the Kalman update with a (y, z)
// measurement, and the seed covariance.
//
// Transport (dx = x1 - x0): s1 = s0 + C_k dx, C_k = -kB q/pT;
//   y1 = y0 + dx (s0 + s1)/(c0 + c1); dS = chord * asin(h)/h (h = |C_k| chord / 2),
//   signed like dx; z1 = z0 + t dS.  d(dS)/dC_k is evaluated as
//   dS^2 [ (s1/c1) sinc^2(dphi/2) / 2 + (sin dphi - dphi)/dphi^2 ], dphi = C_k dS,
//   a form without cancellation as C_k -> 0.
#pragma once
#include "tpc_internal.cuh"

namespace tpc {
namespace {

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

}  // namespace
}  // namespace tpc
