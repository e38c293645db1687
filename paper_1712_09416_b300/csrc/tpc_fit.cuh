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

// Transport of the state (x, p) to the plane x1: the new state and the
// non-trivial entries of the Jacobian J = d(p1)/d(p0), which differs from
// the identity in dy/ds = a, dy/d(q/pT) = b, dz/ds = c, dz/dt = d,
// dz/d(q/pT) = e and ds/d(q/pT) = g.  Returns false, leaving the state as it
// was, when |sin phi| would reach sin_max.
struct Jac {
    float a, b, c, d, e, g;
};

__device__ __forceinline__ bool transport_state(float& x, float* p, float x1, const Launch& L,
                                                Jac& J)
{
    const float dx = x1 - x;
    const float ck = -L.kB * p[4];
    const float s0 = p[2];
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
    const float t = p[3];
    J.a = dx * (2.0f * cc + ss * (s0 * ic0 + s1 * ic1)) * (icc * icc);
    J.b = -L.kB * dx * dx * (cc + ss * s1 * ic1) * (icc * icc);
    J.c = t * dx * ss * ic0 * ic1 * icc;
    J.d = dS;
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
    J.e = -L.kB * t * dSdC;
    J.g = -L.kB * dx;

    p[0] += dy;
    p[1] += t * dS;
    p[2] = s1;
    x = x1;
    return true;
}

__device__ __forceinline__ bool transport(Fit& f, float x1, const Launch& L)
{
    Jac J;
    if (!transport_state(f.x, f.p, x1, L, J)) return false;
    const float a = J.a, b = J.b, c = J.c, d = J.d, e = J.e, g = J.g;
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

// (S00, S01, S11) = C[0:2, 0:2] + V
__device__ __forceinline__ void meas_cov(const Fit& f, const Launch& L, float& S00, float& S01,
                                         float& S11)
{
    S00 = f.C[0] + L.sy2;
    S01 = f.C[1];
    S11 = f.C[2] + L.sz2;
}

__device__ __forceinline__ void cov_of(const Fit& f, float* C)
{
#pragma unroll
    for (int i = 0; i < 15; ++i) C[i] = f.C[i];
}

// ---- square-root form (backward pass of the tracklet constructor) ----
// The covariance is carried as a factor U with C = U U^T (5x5, row-major,
// not triangular).  In binary32 this keeps about twice the significant
// digits of C itself where the fit pins a parameter down by orders of
// magnitude from its seed variance (the q/pT variance falls from 100 to
// ~1e-2): the update C -= K C[0:2,:] cancels there, the factor form does
// not.  Transport is U <- J U (rows 0..2 change).  The (y, z) measurement
// is taken as two scalar updates (V is diagonal) in Potter's form: for the
// measured component i, a = U^T e_i, alpha = a.a + v, w = U a (= C e_i),
// p += w r / alpha, U <- U - gamma w a^T with gamma = 1 / (alpha +
// sqrt(alpha v)); the chi2 increment is the sum of r^2 / alpha of the two
// (equal to r^T S^-1 r of the joint update).
struct FitSR {
    float x;
    float p[5];
    float U[25];
};

__device__ __forceinline__ bool transport(FitSR& f, float x1, const Launch& L)
{
    Jac J;
    if (!transport_state(f.x, f.p, x1, L, J)) return false;
    float* U = f.U;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float u2 = U[10 + j], u3 = U[15 + j], u4 = U[20 + j];
        U[j] += J.a * u2 + J.b * u4;
        U[5 + j] += J.c * u2 + J.d * u3 + J.e * u4;
        U[10 + j] = u2 + J.g * u4;
    }
    return true;
}

// (S00, S01, S11) = C[0:2, 0:2] + V
__device__ __forceinline__ void meas_cov(const FitSR& f, const Launch& L, float& S00,
                                         float& S01, float& S11)
{
    const float* U = f.U;
    float a = 0.0f, b = 0.0f, c = 0.0f;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        a += U[j] * U[j];
        b += U[j] * U[5 + j];
        c += U[5 + j] * U[5 + j];
    }
    S00 = a + L.sy2;
    S01 = b;
    S11 = c + L.sz2;
}

template <int I>
__device__ __forceinline__ float update_sr_1(FitSR& f, float m, float v)
{
    float* U = f.U;
    float a[5], w[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) a[j] = U[5 * I + j];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float s = 0.0f;
#pragma unroll
        for (int j = 0; j < 5; ++j) s += U[5 * k + j] * a[j];
        w[k] = s;  // w[I] = a.a = C_II
    }
    const float al = w[I] + v;
    const float ial = __fdividef(1.0f, al);
    const float r = m - f.p[I];
    const float kr = r * ial;
#pragma unroll
    for (int k = 0; k < 5; ++k) f.p[k] += w[k] * kr;
    const float q = v * ial;  // in (0, 1]
    const float gam = __fdividef(ial, 1.0f + q * rsqrtf(q));
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float gk = gam * w[k];
#pragma unroll
        for (int j = 0; j < 5; ++j) U[5 * k + j] -= gk * a[j];
    }
    return r * kr;
}

// Kalman update with measurement (my, mz); returns the chi2 increment.
__device__ __forceinline__ float update(FitSR& f, float my, float mz, const Launch& L)
{
    const float c0 = update_sr_1<0>(f, my, L.sy2);
    return c0 + update_sr_1<1>(f, mz, L.sz2);
}

// Seed: U = diag of the seed standard deviations (the same seed covariance
// as seed_cov).
__device__ __forceinline__ void seed_cov(FitSR& f, const Launch& L)
{
    const float c2 = (1.0f - f.p[2]) * (1.0f + f.p[2]);
    const float c1 = sqrtf(c2);
#pragma unroll
    for (int i = 0; i < 25; ++i) f.U[i] = 0.0f;
    f.U[0] = L.sy;
    f.U[6] = L.sz;
    f.U[12] = L.seed_sd_s * c2 * c1;
    f.U[18] = L.seed_sd_t * c1;
    f.U[24] = L.seed_sd_q;
}

// C = U U^T, lower triangle
__device__ __forceinline__ void cov_of(const FitSR& f, float* C)
{
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int k = 0; k <= i; ++k) {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < 5; ++j) s += f.U[5 * i + j] * f.U[5 * k + j];
            C[CI(i, k)] = s;
        }
}

}  // namespace
}  // namespace tpc
