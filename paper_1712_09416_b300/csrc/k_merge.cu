// k_merge.cu -- sector track merger and global refit, run after the selector
// when the launch's merge flag is set.  The step after the sector tracker:
// the tracker sees the clusters of all TPC links of an event (paper, Sect. 2),
// so a particle cut by a sector boundary or by the z = 0 membrane can be
// joined again.  The rules (the paper gives none, so they are readings):
//
//   M0 rotation of a state at x into a frame turned by d:
//      x' = x cos d + y sin d, y' = -x sin d + y cos d, s' = s cos d - c sin d,
//      valid iff c' = c cos d + s sin d > 0 and |s'| < sin_max; covariance
//      carried to the plane x' (dy'/dy = c/c', dz'/dy = -t sin d / c',
//      ds'/dy = -C_k sin d, ds'/ds = c'/c).
//   M1 outer state: a track's state transported to its outermost hit.
//   M2 partners of a track: the tracks of the phi-neighbour sectors in the
//      same z half (d = -+ the sector angle; across phi = 0 only for a closed
//      ring) and of the same phi sector in the other half (d = 0).
//   M3 match chi2 of (a, b): a's outer state turned into b's frame and
//      transported to b's x; admissible iff the gap x_b - x_a' lies in
//      [dx_lo, dx_hi] and r^T (C_a' + C_b)^-1 r <= chi2 cut.
//   M4 link a -> b iff each is the other's admissible partner of least chi2
//      (ties to the lower index).
//   M5 refit of a chain (any length): the outermost track's outer state,
//      covariance reset to the seed covariance, every hit inward (frames
//      turned at each change of track); result at the innermost hit.
//
// Kernels: k_mg_outer (M1, one thread per track; also clears the scratch),
// k_mg_sortx (each sector's tracks ordered by x), k_mg_match (M2-M3, one
// warp per track a, lanes over the tracks of its partner sectors whose x lies
// in the gap window; b's best a by a 64-bit atomicMax of ~(chi2 bits << 32 | a)),
// k_mg_link (M4), k_mg_gather (hit coordinates of linked tracks), k_mg_refit
// (M5, one thread per chain), k_mg_scan (output
// index and hit offset of every surviving track in the original order,
// decoupled look-back over tiles of kMgTile tracks), k_mg_write (one warp per
// output track).  Arithmetic is binary32.
#include <cuda_runtime.h>

#include "tpc_internal.cuh"
#include "tpc_fit.cuh"

namespace tpc {

namespace {

constexpr int kMgThreads = 128;
constexpr int kScanThreads = 256;
constexpr int kScanPer = kMgTile / kScanThreads;

__device__ __forceinline__ void load_track(Fit& f, const Launch& L, int j)
{
    f.x = L.k_x[j];
#pragma unroll
    for (int i = 0; i < 5; ++i) f.p[i] = L.k_param[(size_t)j * 5 + i];
#pragma unroll
    for (int i = 0; i < 15; ++i) f.C[i] = L.k_cov[(size_t)j * 15 + i];
}

// M0; false (f unchanged) if the turned track would not run outward
__device__ __forceinline__ bool rotate(Fit& f, float cd, float sd, const Launch& L)
{
    const float s = f.p[2];
    const float c = sqrtf((1.0f - s) * (1.0f + s));
    const float s1 = s * cd - c * sd;
    const float c1 = c * cd + s * sd;
    if (!(c1 > 0.0f) || !(fabsf(s1) < L.sin_max)) return false;
    const float ck = -L.kB * f.p[4];
    const float j00 = c / c1, j10 = -f.p[3] * sd / c1, j20 = -ck * sd, j22 = c1 / c;
    const float x1 = f.x * cd + f.p[0] * sd;
    const float y1 = -f.x * sd + f.p[0] * cd;
    f.x = x1;
    f.p[0] = y1;
    f.p[2] = s1;
    float* C = f.C;
    const float C00 = C[0], C10 = C[1], C11 = C[2], C20 = C[3], C21 = C[4], C22 = C[5];
    const float C30 = C[6], C31 = C[7], C32 = C[8], C40 = C[10], C41 = C[11], C42 = C[12];
    // rows 0..2 of J are (j00 e0), (j10 e0 + e1), (j20 e0 + j22 e2)
    const float u2 = j20 * C00 + j22 * C20;  // row 2 of J C, column 0
    C[0] = j00 * j00 * C00;
    C[1] = j00 * (j10 * C00 + C10);
    C[2] = j10 * j10 * C00 + 2.0f * j10 * C10 + C11;
    C[3] = j00 * u2;
    C[4] = j10 * u2 + j20 * C10 + j22 * C21;
    C[5] = j20 * j20 * C00 + 2.0f * j20 * j22 * C20 + j22 * j22 * C22;
    C[6] = j00 * C30;
    C[7] = j10 * C30 + C31;
    C[8] = j20 * C30 + j22 * C32;
    C[10] = j00 * C40;
    C[11] = j10 * C40 + C41;
    C[12] = j20 * C40 + j22 * C42;
    return true;
}

// The same rotation on a square-root factor (C = U U^T): U <- J U.
__device__ __forceinline__ bool rotate(FitSR& f, float cd, float sd, const Launch& L)
{
    const float s = f.p[2];
    const float c = sqrtf((1.0f - s) * (1.0f + s));
    const float s1 = s * cd - c * sd;
    const float c1 = c * cd + s * sd;
    if (!(c1 > 0.0f) || !(fabsf(s1) < L.sin_max)) return false;
    const float ck = -L.kB * f.p[4];
    const float j00 = c / c1, j10 = -f.p[3] * sd / c1, j20 = -ck * sd, j22 = c1 / c;
    const float x1 = f.x * cd + f.p[0] * sd;
    const float y1 = -f.x * sd + f.p[0] * cd;
    f.x = x1;
    f.p[0] = y1;
    f.p[2] = s1;
    float* U = f.U;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float u0 = U[j];
        U[j] = j00 * u0;
        U[5 + j] = j10 * u0 + U[5 + j];
        U[10 + j] = j20 * u0 + j22 * U[10 + j];
    }
    return true;
}

// r^T (C_f + C_b)^-1 r with r = p_f - p_b, by Cholesky; -1 if not positive definite
__device__ __forceinline__ float match_chi2(const Fit& f, const Launch& L, int b)
{
    float r[5], A[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) r[i] = f.p[i] - L.k_param[(size_t)b * 5 + i];
#pragma unroll
    for (int i = 0; i < 15; ++i) A[i] = f.C[i] + L.k_cov[(size_t)b * 15 + i];
    float q = 0.0f, u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float a = A[CI(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) a -= A[CI(i, k)] * A[CI(j, k)];
            if (i == j) {
                if (!(a > 0.0f)) return -1.0f;
                A[CI(i, i)] = sqrtf(a);
            } else {
                A[CI(i, j)] = a / A[CI(j, j)];
            }
        }
        float v = r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= A[CI(i, k)] * u[k];
        u[i] = v / A[CI(i, i)];
        q += u[i] * u[i];
    }
    return q;
}

__device__ __forceinline__ int n_tracks(const Launch& L) { return L.cnt->n_tracks; }

// M1, and the scratch of the later kernels
__global__ void __launch_bounds__(kMgThreads) k_mg_outer(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
        const int e = L.sec_event[L.k_gsec[j]];
        const int last = L.k_hit_cid[L.k_hit_off[j + 1] - 1];
        Fit f;
        load_track(f, L, j);
        const bool ok = transport(f, L.xr[L.ev[e].row[last]], L);
        MgState& O = L.mg_st[j];
        O.x = f.x;
#pragma unroll
        for (int i = 0; i < 5; ++i) O.p[i] = f.p[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) O.C[i] = f.C[i];
        O.ok = ok;
        L.mg_key[j] = 0ULL;
        L.mg_in[j] = -1;
        L.mg_absorbed[j] = 0;
        L.mg_fit[j].ok = 0;
    }
}

// The tracks of each sector ordered by x (bitonic sort in shared memory, one
// block per sector; a sector holds at most kMaxSectorTracks tracks), so that
// the matcher scans only the tracks whose x can lie in the gap window.
constexpr int kSortXThreads = 512;
__global__ void __launch_bounds__(kSortXThreads) k_mg_sortx(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    extern __shared__ float sx[];                   // [kMaxSectorTracks]
    int* si = reinterpret_cast<int*>(sx + kMaxSectorTracks);  // [kMaxSectorTracks]
    const int g = blockIdx.x;
    // a sector over kMaxSectorTracks fails the launch (selector); stay in bounds
    const int t0 = L.sec_trk_off[g], m = min(L.sec_trk_off[g + 1] - t0, kMaxSectorTracks);
    if (m <= 0) return;
    int p2 = 1;
    while (p2 < m) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        sx[i] = i < m ? L.k_x[t0 + i] : __int_as_float(0x7f800000);  // +inf pads
        si[i] = i < m ? t0 + i : 0x7fffffff;
    }
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const float a = sx[i], b = sx[l];
                    const int ia = si[i], ib = si[l];
                    const bool gt = a > b || (a == b && ia > ib);
                    if (gt == up) {
                        sx[i] = b;
                        sx[l] = a;
                        si[i] = ib;
                        si[l] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int b = si[i];
        L.mg_xs[t0 + i] = sx[i];
        L.mg_xi[t0 + i] = b;
        // the matcher's first tests read one 32-byte record per candidate
        L.mg_pre[2 * (t0 + i)] = make_float4(sx[i], L.k_param[(size_t)b * 5 + 3],
                                             L.k_param[(size_t)b * 5 + 4], L.k_cov[(size_t)b * 15 + 9]);
        L.mg_pre[2 * (t0 + i) + 1] = make_float4(L.k_cov[(size_t)b * 15 + 13], L.k_cov[(size_t)b * 15 + 14],
                                                 __int_as_float(b), 0.0f);
    }
}

// First position in xs[0, n) whose value is >= v (xs ascending), by the
// whole warp (same arguments on every lane): each round probes 32 evenly
// spaced positions at once and keeps the bracket the ballot points to.
__device__ __forceinline__ int warp_lower_bound(const float* xs, int n, float v)
{
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int p = lo + lane * step;
        const bool valid = p < hi;
        const unsigned below = __ballot_sync(0xffffffffu, valid && xs[p] < v);
        const unsigned nvalid = __popc(__ballot_sync(0xffffffffu, valid));
        const int c = __popc(below);  // probes below v come first
        const int nlo = c > 0 ? lo + (c - 1) * step + 1 : lo;
        const int nhi = c < (int)nvalid ? lo + c * step : hi;
        lo = nlo;
        hi = nhi;
    }
    const int p = lo + lane;
    const unsigned below = __ballot_sync(0xffffffffu, p < hi && xs[p] < v);
    return lo + __popc(below);
}

// M2-M3: one warp per track a, its lanes over the candidate tracks b
__global__ void __launch_bounds__(kMgThreads) k_mg_match(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    const int N = L.n_sectors_phi;
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < T; a += warps) {
        const MgState& O = L.mg_st[a];
        int best = -1;
        float bchi = 0.0f;
        if (O.ok) {
            const int gs = L.k_gsec[a];
            const int base = L.ev[L.sec_event[gs]].sec_base;
            const int ls = gs - base, k = ls % N, half = ls / N;
            const float t_a = O.p[3], q_a = O.p[4], c33 = O.C[9], c43 = O.C[13], c44 = O.C[14];
            const float cut_pre = L.mg_chi2 * 1.001f + 1e-3f;
            for (int q = 0; q < 3; ++q) {
                int lb;
                float sd = 0.0f;
                if (q < 2) {
                    int kb = k + (q ? 1 : -1);
                    if (kb < 0 || kb >= N) {
                        if (!L.mg_ring || N < 3) continue;
                        kb = (kb + N) % N;
                    }
                    lb = half * N + kb;
                    sd = q ? L.mg_sd : -L.mg_sd;
                } else {
                    if (!L.split_z) continue;
                    lb = (1 - half) * N + k;
                }
                // a's outer state in b's frame (the same on every lane)
                Fit r;
                r.x = O.x;
#pragma unroll
                for (int i = 0; i < 5; ++i) r.p[i] = O.p[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) r.C[i] = O.C[i];
                if (q < 2 && !rotate(r, L.mg_cd, sd, L)) continue;
                // the tracks of sector gb with x in the gap window (widened by
                // 0.01 cm against rounding; the exact test follows)
                const int gb = base + lb;
                const int s0 = L.sec_trk_off[gb];
                const int ns = min(L.sec_trk_off[gb + 1] - s0, kMaxSectorTracks);
                const float* xs = L.mg_xs + s0;
                const int k0 = warp_lower_bound(xs, ns, r.x + L.mg_dx_lo - 0.01f);
                const int k1 = warp_lower_bound(xs, ns, r.x + L.mg_dx_hi + 0.01f);
                for (int kk = k0 + lane; kk < k1; kk += 32) {
                    const float4 pa = L.mg_pre[2 * (s0 + kk)], pb = L.mg_pre[2 * (s0 + kk) + 1];
                    const int b = __float_as_int(pb.z);
                    const float gap = pa.x - r.x;
                    if (!(gap >= L.mg_dx_lo && gap <= L.mg_dx_hi)) continue;
                    // tan(lambda) and q/pT and their covariance block are left
                    // as they are by transport and rotation, so their 2x2 chi2
                    // bounds the 5x5 one from below: a pair over the cut there
                    // (with a margin for rounding) is over it in full
                    {
                        const float dt = t_a - pa.y;
                        const float dq = q_a - pa.z;
                        const float s33 = c33 + pa.w;
                        const float s43 = c43 + pb.x;
                        const float s44 = c44 + pb.y;
                        const float det = s33 * s44 - s43 * s43;
                        if (det > 0.0f &&
                            dt * dt * s44 - 2.0f * dt * dq * s43 + dq * dq * s33 > cut_pre * det)
                            continue;
                    }
                    Fit t = r;
                    if (!transport(t, L.k_x[b], L)) continue;
                    const float chi2 = match_chi2(t, L, b);
                    if (!(chi2 >= 0.0f && chi2 <= L.mg_chi2)) continue;
                    if (best < 0 || chi2 < bchi || (chi2 == bchi && b < best)) {
                        bchi = chi2;
                        best = b;
                    }
                    atomicMax(&L.mg_key[b],
                              ~(((unsigned long long)__float_as_uint(chi2) << 32) | (unsigned)a));
                }
            }
        }
        // least chi2 over the lanes, ties to the lower index
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oc = __shfl_xor_sync(0xffffffffu, bchi, o);
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            if (ob >= 0 && (best < 0 || oc < bchi || (oc == bchi && ob < best))) {
                bchi = oc;
                best = ob;
            }
        }
        if (lane == 0) L.mg_best[a] = best;
    }
}

// M4
__global__ void __launch_bounds__(kMgThreads) k_mg_link(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < T; a += gridDim.x * blockDim.x) {
        const int b = L.mg_best[a];
        int lo = -1;
        if (b >= 0) {
            const unsigned long long key = ~L.mg_key[b];
            if ((unsigned)(key & 0xFFFFFFFFULL) == (unsigned)a) lo = b;
        }
        L.mg_link[a] = lo;
        if (lo >= 0) {
            L.mg_in[lo] = a;
            atomicAdd(&L.cnt->n_mg_links, 1);
        }
    }
}

// (x, y, z) of every hit of a linked track, in the order of k_hit_cid, so that
// the refit reads one float4 per hit instead of three dependent loads
__global__ void k_mg_gather(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < T; j += warps) {
        if (L.mg_link[j] < 0 && L.mg_in[j] < 0) continue;
        const EventDesc ev = L.ev[L.sec_event[L.k_gsec[j]]];
        const int k1 = L.k_hit_off[j + 1];
        for (int k = L.k_hit_off[j] + lane; k < k1; k += 32) {
            const int c = L.k_hit_cid[k];
            L.mg_hxyz[k] = make_float4(L.xr[ev.row[c]], ev.y[c], ev.z[c], 0.0f);
        }
    }
}

// M5: one thread per chain head (a track with an outgoing and no incoming link)
__global__ void __launch_bounds__(kMgThreads) k_mg_refit(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    const int N = L.n_sectors_phi;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < T; h += gridDim.x * blockDim.x) {
        if (L.mg_in[h] >= 0 || L.mg_link[h] < 0) continue;
        // every track has at most one incoming and one outgoing link, so the
        // chain from a head ends within T steps (the bound only guards reads)
        int so = h, m = 1, nh = L.k_hit_off[h + 1] - L.k_hit_off[h];
        while (L.mg_link[so] >= 0 && m <= T) {
            so = L.mg_link[so];
            nh += L.k_hit_off[so + 1] - L.k_hit_off[so];
            ++m;
        }
        if (m > T) continue;
        const MgState& O = L.mg_st[so];
        if (!O.ok) continue;
        // square-root factor of the covariance, as in the tracklet
        // constructor's backward pass (the refit restarts from the seed
        // covariance, where the binary32 update of C itself cancels)
        FitSR f;
        f.x = O.x;
#pragma unroll
        for (int i = 0; i < 5; ++i) f.p[i] = O.p[i];
        seed_cov(f, L);
        float chi2 = 0.0f;
        bool ok = true;
        int a = so;
        for (;;) {
            const int k1 = L.k_hit_off[a], k0 = L.k_hit_off[a + 1] - 1;
            float4 hit = L.mg_hxyz[k0];
            for (int kk = k0; kk >= k1; --kk) {
                // the next hit's coordinates load during this hit's arithmetic
                const float4 nxt = kk > k1 ? L.mg_hxyz[kk - 1] : hit;
                if (hit.x != f.x && !transport(f, hit.x, L)) {
                    ok = false;
                    break;
                }
                chi2 += update(f, hit.y, hit.z, L);
                hit = nxt;
            }
            if (!ok || a == h) break;
            const int inner = L.mg_in[a];
            const int ka = L.k_gsec[inner] % N, kp = L.k_gsec[a] % N;
            if (ka != kp) {  // turn into the inner track's frame
                int dk = ka - kp;
                if (dk > 1) dk -= N;  // neighbours across phi = 0
                if (dk < -1) dk += N;
                if (!rotate(f, L.mg_cd, dk > 0 ? L.mg_sd : -L.mg_sd, L)) {
                    ok = false;
                    break;
                }
            }
            a = inner;
        }
        MgFit& F = L.mg_fit[h];
        if (!ok) continue;
        F.x = f.x;
#pragma unroll
        for (int i = 0; i < 5; ++i) F.p[i] = f.p[i];
        cov_of(f, F.C);
        F.chi2 = chi2;
        F.ndf = 2 * nh - 5;
        F.nhits = nh;
        F.ok = 1;
        for (int b = L.mg_link[h]; b >= 0; b = L.mg_link[b]) L.mg_absorbed[b] = 1;
        atomicAdd(&L.cnt->n_mg_chains, 1);
    }
}

__device__ __forceinline__ int out_hits(const Launch& L, int j)
{
    return L.mg_fit[j].ok ? L.mg_fit[j].nhits : L.k_hit_off[j + 1] - L.k_hit_off[j];
}

// output index and hit offset of every track (surviving tracks keep their order)
__global__ void __launch_bounds__(kScanThreads) k_mg_scan(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    __shared__ int s_cnt[kScanThreads / 32], s_hit[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    const int T = n_tracks(L);
    const int tile = blockIdx.x;
    const int t0 = tile * kMgTile;
    if (t0 >= T && !(T == 0 && tile == 0)) return;
    const int lo = t0 + threadIdx.x * kScanPer;
    int cnt = 0, hits = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int j = lo + i;
        if (j < T && !L.mg_absorbed[j]) {
            ++cnt;
            hits += out_hits(L, j);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int ic = cnt, ih = hits;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int vc = __shfl_up_sync(0xffffffffu, ic, o);
        const int vh = __shfl_up_sync(0xffffffffu, ih, o);
        if (lane >= o) {
            ic += vc;
            ih += vh;
        }
    }
    if (lane == 31) {
        s_cnt[wid] = ic;
        s_hit[wid] = ih;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        int tc = 0, th = 0;
        if (threadIdx.x == 0) {
            for (int w = 0; w < kScanThreads / 32; ++w) {
                const int vc = s_cnt[w], vh = s_hit[w];
                s_cnt[w] = tc;
                s_hit[w] = th;
                tc += vc;
                th += vh;
            }
        }
        tc = __shfl_sync(0xffffffffu, tc, 0);
        th = __shfl_sync(0xffffffffu, th, 0);
        const unsigned long long p = lookback_warp(
            L.tile_state + L.n_row_tiles + L.n_hit_tiles + L.S, tile, pack2((unsigned)tc, (unsigned)th), L.cnt,
            L.spin_limit);
        if (threadIdx.x == 0) {
            s_prefix = p;
            if (t0 + kMgTile >= T) {  // the last tile: totals
                const int nt = (int)unpack_a(p) + tc, nhit = (int)unpack_b(p) + th;
                L.cnt->n_mg_tracks = nt;
                L.m_hit_off[nt] = nhit;
            }
        }
    }
    __syncthreads();
    int oc = (int)unpack_a(s_prefix) + s_cnt[wid] + ic - cnt;
    int oh = (int)unpack_b(s_prefix) + s_hit[wid] + ih - hits;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int j = lo + i;
        if (j >= T) break;
        L.mg_oidx[j] = oc;
        L.mg_ohoff[j] = oh;
        if (!L.mg_absorbed[j]) {
            ++oc;
            oh += out_hits(L, j);
        }
    }
}

// one warp per surviving track: header, then its hits (a chain's tracks in turn)
__global__ void k_mg_write(Launch L)
{
    if (L.cnt->timeout) return;  // an earlier bounded wait gave up
    const int T = n_tracks(L);
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = L.cnt->n_mg_tracks, total_hits = L.cnt->n_track_hits;
    for (int g = gt; g <= L.S; g += gridDim.x * blockDim.x) {  // per-sector output offsets
        const int j = L.sec_trk_off[g];
        L.m_sec_trk_off[g] = j < T ? L.mg_oidx[j] : total;
        L.m_sec_hit_off[g] = j < T ? L.mg_ohoff[j] : total_hits;
    }
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int j = gt >> 5; j < T; j += warps) {
        if (L.mg_absorbed[j]) continue;
        const int o = L.mg_oidx[j];
        const bool merged = L.mg_fit[j].ok;
        const MgFit& F = L.mg_fit[j];
        if (lane < 5) L.m_param[(size_t)o * 5 + lane] = merged ? F.p[lane] : L.k_param[(size_t)j * 5 + lane];
        if (lane < 15) L.m_cov[(size_t)o * 15 + lane] = merged ? F.C[lane] : L.k_cov[(size_t)j * 15 + lane];
        if (lane == 0) {
            L.m_sector[o] = L.k_sector[j];
            L.m_x[o] = merged ? F.x : L.k_x[j];
            L.m_chi2[o] = merged ? F.chi2 : L.k_chi2[j];
            L.m_ndf[o] = merged ? F.ndf : L.k_ndf[j];
            L.m_hit_off[o] = L.mg_ohoff[j];
        }
        int dst = L.mg_ohoff[j];
        for (int a = j; a >= 0; a = merged ? L.mg_link[a] : -1) {
            const int k0 = L.k_hit_off[a], k1 = L.k_hit_off[a + 1];
            for (int k = k0 + lane; k < k1; k += 32) L.m_hit_cid[dst + (k - k0)] = L.k_hit_cid[k];
            dst += k1 - k0;
        }
    }
}

}  // namespace

constexpr size_t kSortXSmem = kMaxSectorTracks * (sizeof(float) + sizeof(int));

void prepare_merger()
{
    cudaFuncSetAttribute(k_mg_sortx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortXSmem);
}

void launch_merger(const Launch& L, const Schedule& S, void* stream_, const KernelHook* hook)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    int blocks = (L.t_cap + kMgThreads - 1) / kMgThreads;
    if (blocks > S.n_sm * 8) blocks = S.n_sm * 8;
    if (blocks < 1) blocks = 1;
    k_mg_outer<<<blocks, kMgThreads, 0, stream>>>(L);
    hook_after(hook, "k_mg_outer");
    k_mg_sortx<<<L.S, kSortXThreads, kSortXSmem, stream>>>(L);
    hook_after(hook, "k_mg_sortx");
    int mblocks = (L.t_cap + kMgThreads / 32 - 1) / (kMgThreads / 32);  // one warp per track
    if (mblocks > S.n_sm * 16) mblocks = S.n_sm * 16;
    if (mblocks < 1) mblocks = 1;
    k_mg_match<<<mblocks, kMgThreads, 0, stream>>>(L);
    hook_after(hook, "k_mg_match");
    k_mg_link<<<blocks, kMgThreads, 0, stream>>>(L);
    hook_after(hook, "k_mg_link");
    int wblocks = (L.t_cap + 7) / 8;  // one warp per track, 8 warps per block
    if (wblocks > S.n_sm * 16) wblocks = S.n_sm * 16;
    if (wblocks < 1) wblocks = 1;
    k_mg_gather<<<wblocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_mg_gather");
    k_mg_refit<<<blocks, kMgThreads, 0, stream>>>(L);
    hook_after(hook, "k_mg_refit");
    k_mg_scan<<<L.n_mg_tiles, kScanThreads, 0, stream>>>(L);
    hook_after(hook, "k_mg_scan");
    k_mg_write<<<wblocks, 256, 0, stream>>>(L);
    hook_after(hook, "k_mg_write");
}

}  // namespace tpc
