/*
 * tpc_oracle.c -- plain, slow CPU oracle of the per-sector TPC track finder
 * (cellular automaton) and track fitter (Kalman filter).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The GPU tracker shares no
 * code, header, table or constant with it and never calls it.
 *
 * What the paper fixes: the ALICE HLT TPC tracker finds tracks with a cellular
 * automaton and fits them with a Kalman filter (Abstract; Sect. 4 intro), it
 * is the most compute-intense reconstruction step (Sect. 2), and its fit runs
 * one track per thread (Sect. 4.1, Listings 1-3).  The steps of the algorithm
 * are deferred to the paper's references, so every rule below is a stated
 * reading, written so that it can be checked by eye:
 *
 *   geometry  pad row r is the plane x = row_x[r] in the sector frame; sector
 *             s covers |y| <= x tan(half_angle); B along +z.
 *   state     p = (y, z, s = sin(phi), t = tan(lambda), q/pT) at x, with a 5x5
 *             symmetric covariance C; curvature C_k = -KAPPA * Bz * q/pT.
 *   C2        neighbours: best (down, up) pair by straight-line kink score.
 *   C3        cleaner: keep mutual links only.
 *   C4        start hits: up link and no down link; chains follow up links.
 *   C5        helix transport between planes with its analytic Jacobian.
 *   C6        Kalman update with a (y, z) measurement.
 *   C7        tracklet: seed from the chain, forward fit + extension search,
 *             backward refit + search, result at the innermost hit.
 *   C8        selector: hits go to the tracklet with the largest weight key;
 *             a track keeps its owned hits.
 *   C9        iterated backward refit on a fixed hit set (tests only).
 *
 * Floating point: everything is binary64, the neighbour decision of C2
 * included (slopes are plain quotients of binary64 differences).  Where that
 * decision could go the other way under a small rounding of D or of a window
 * test, the hit carries near-tie bits (ORC_C2_TIE_*): the best and the
 * second-best pair within tie_d, the best D within tie_d of D_MAX, or a
 * candidate within tie_win cm of a window edge.  A binary32 restatement of
 * the same rule (one rounding per operation; this file is compiled with
 * -ffp-contract=off) can be evaluated alongside as a diagnostic; it feeds
 * nothing downstream.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_KAPPA 0.299792458e-2 /* cm^-1 per (GeV/c)^-1 per tesla */

/* ------------------------------------------------------------------------ */
/* configuration and result records (mirrored by oracle.py with ctypes)       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double half_angle;  /* rad, half opening of a sector */
    double z_max;       /* cm */
    double bz;          /* tesla */
    double sigma_y, sigma_z;  /* cm, measurement errors */
    double chi2_hit;    /* acceptance of a searched hit */
    double sin_max;     /* transport fails at |s| >= sin_max */
    double edge_margin; /* cm beyond the sector edge / z range */
    double seed_var_s, seed_var_t, seed_var_q; /* seed covariance diagonal */
    double tie_chi2;    /* near-tie width on chi2 decisions */
    double tie_sin;     /* near-tie width on |s| vs sin_max */
    double tie_edge;    /* near-tie width (cm) on the edge stops */
    double tie_d;       /* near-tie width on the C2 kink score D */
    double tie_win;     /* near-tie width (cm) on the C2 slope windows */
    float slope_win_y, slope_win_z, d_max, pad0;
    int32_t n_rows, n_sectors_phi, split_z;
    int32_t max_gap, min_chain, min_tracklet_hits, min_track_hits;
    int32_t pad1;
} orc_config;

typedef struct {
    /* links by cid, -1 = none; all [n] */
    int32_t* up;     /* C2, binary64 decision */
    int32_t* dn;
    int32_t* c2_tie; /* C2 near-tie bits per hit (ORC_C2_TIE_*) */
    int32_t* up32;   /* C2, binary32 restatement (diagnostic, may be NULL) */
    int32_t* dn32;
    int32_t* fwd_mark; /* C7a: 1 if a forward extension search took the hit, | 2 if
                          one whose pass carries near-tie bits did (may be NULL) */
    int32_t* up_c;   /* C3 */
    int32_t* dn_c;
    /* tracklets (one per chain of >= min_chain hits), capacity cap_tracklets */
    int64_t cap_tracklets;
    int32_t* t_start;   /* cid of the chain start h0 */
    int32_t* t_sector;
    int32_t* t_chain_len;
    int32_t* t_valid;
    int32_t* t_nhits;
    int32_t* t_first_row;
    int32_t* t_last_row;
    int32_t* t_flags;   /* near-tie bits, see ORC_TIE_* */
    int32_t* t_ndf;
    double* t_x;
    double* t_p;        /* [cap][5] */
    double* t_C;        /* [cap][15] lower triangle, row order */
    double* t_chi2;
    int32_t* t_rowhit;  /* [cap][n_rows] cid or -1 */
    /* hit weights [n] */
    uint64_t* weight;
    /* tracks, capacity cap_tracks; hits capacity n */
    int64_t cap_tracks;
    int32_t* k_tracklet;  /* index into the tracklet arrays */
    int32_t* k_sector;
    int32_t* k_ndf;
    double* k_x;
    double* k_p;
    double* k_C;
    double* k_chi2;
    int32_t* k_hit_off;   /* [cap+1] */
    int32_t* k_hit_cid;   /* [n] */
    /* counters (out) */
    int64_t n_tracklets, n_tracks, n_track_hits;
    int64_t n_links, n_link_flips32, n_c2_ties, n_starts, n_dominated;
} orc_result;

enum {
    ORC_TIE_CHI2_CUT = 1,   /* best chi2 within tie_chi2 of chi2_hit */
    ORC_TIE_CHI2_PAIR = 2,  /* second-best chi2 within tie_chi2 of the best */
    ORC_TIE_SIN = 4,        /* |s| within tie_sin of sin_max at a transport */
    ORC_TIE_EDGE = 8,       /* |y| or |z| within tie_edge of the stop bound */
    ORC_TIE_CHAIN = 512,    /* a chain hit lies outside the chi2 acceptance */
};

enum {
    ORC_C2_TIE_PAIR = 1,    /* second-best pair within tie_d of the best D */
    ORC_C2_TIE_CUT = 2,     /* best D within tie_d of D_MAX */
    ORC_C2_TIE_WIN = 4,     /* a candidate within tie_win cm of a window edge */
};

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */
/* ------------------------------------------------------------------------ */

static int tri(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

static void cov_to_tri(double C[5][5], double* out)
{
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) out[tri(i, j)] = C[i][j];
}

static void tri_to_cov(const double* in, double C[5][5])
{
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) C[i][j] = in[tri(i, j)];
}

/* ------------------------------------------------------------------------ */
/* C5: helix transport between pad-row planes                                 */
/* ------------------------------------------------------------------------ */

/*
 * Move state p (at plane x0) to the plane x1 along the helix, and the
 * covariance with it (C <- J C J^T, no process noise).  With dx = x1 - x0 and
 * C_k = -KAPPA * bz * q/pT:
 *   s1 = s0 + C_k dx                       (fails if |s1| >= sin_max)
 *   y1 = y0 + dx (s0 + s1) / (c0 + c1)     c = sqrt(1 - s^2) > 0
 *   dS = ch * asin(h) / h, signed like dx  ch = chord length, h = |C_k| ch / 2
 *   z1 = z0 + t dS; t and q/pT unchanged.
 * J holds the exact partial derivatives of (y1, z1, s1, t1, q1) with respect
 * to (y0, z0, s0, t0, q0).  Returns 0, or -1 on failure (state untouched).
 * ORC_TIE_SIN is or-ed into *flags when |s0| or |s1| lies within tie of sin_max.
 */
int orc_transport(double x0, double x1, double bz, double sin_max, double tie,
                  double* p, double C[5][5], double J[5][5], int* flags)
{
    const double kB = ORC_KAPPA * bz;
    const double dx = x1 - x0;
    const double ck = -kB * p[4];
    const double s0 = p[2];
    const double s1 = s0 + ck * dx;
    if (flags && (fabs(fabs(s1) - sin_max) <= tie || fabs(fabs(s0) - sin_max) <= tie))
        *flags |= ORC_TIE_SIN;
    if (!(fabs(s1) < sin_max) || !(fabs(s0) < sin_max)) return -1;
    const double c0 = sqrt(1.0 - s0 * s0);
    const double c1 = sqrt(1.0 - s1 * s1);
    const double cc = c0 + c1;
    const double dy = dx * (s0 + s1) / cc;
    const double ch = sqrt(dx * dx + dy * dy);
    const double h = fabs(ck) * ch * 0.5;
    double dS = (h > 0.0) ? ch * asin(h) / h : ch;
    if (dx < 0.0) dS = -dS;
    const double t = p[3];

    double Jl[5][5];
    memset(Jl, 0, sizeof(Jl));
    for (int i = 0; i < 5; ++i) Jl[i][i] = 1.0;
    Jl[0][2] = dx * (2.0 * cc + (s0 + s1) * (s0 / c0 + s1 / c1)) / (cc * cc);
    Jl[0][4] = -kB * dx * dx * (cc + (s0 + s1) * s1 / c1) / (cc * cc);
    Jl[1][2] = t * dx * (s0 + s1) / (c0 * c1 * cc);
    Jl[1][3] = dS;
    /* d(dS)/d(C_k) = (dx/c1 - dS)/C_k; near C_k = 0 its series
     * g''/2 + g''' C_k / 3 with g(C) = asin(s0 + C dx) is used instead. */
    double dSdC;
    if (fabs(ck * dx) > 1e-5) {
        dSdC = (dx / c1 - dS) / ck;
    } else {
        const double g2 = dx * dx * s0 / (c0 * c0 * c0);
        const double g3 = dx * dx * dx * (1.0 + 2.0 * s0 * s0) / (c0 * c0 * c0 * c0 * c0);
        dSdC = 0.5 * g2 + g3 * ck / 3.0;
    }
    Jl[1][4] = -kB * t * dSdC;
    Jl[2][4] = -kB * dx;

    p[0] += dy;
    p[1] += t * dS;
    p[2] = s1;

    if (C) {
        double T[5][5], N[5][5];
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double a = 0.0;
                for (int k = 0; k < 5; ++k) a += Jl[i][k] * C[k][j];
                T[i][j] = a;
            }
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double a = 0.0;
                for (int k = 0; k < 5; ++k) a += T[i][k] * Jl[j][k];
                N[i][j] = a;
            }
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) C[i][j] = 0.5 * (N[i][j] + N[j][i]);
    }
    if (J) memcpy(J, Jl, sizeof(Jl));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* C6: Kalman update with a (y, z) measurement                                */
/* ------------------------------------------------------------------------ */

/*
 * Residual r = m - (y, z), S = C[0:2,0:2] + diag(vy, vz), K = C[:,0:2] S^-1,
 * p += K r, C -= K C[0:2,:], returns chi2 increment r^T S^-1 r.
 */
double orc_update(double* p, double C[5][5], double my, double mz, double vy, double vz)
{
    const double r0 = my - p[0], r1 = mz - p[1];
    const double S00 = C[0][0] + vy, S01 = C[0][1], S11 = C[1][1] + vz;
    const double det = S00 * S11 - S01 * S01;
    const double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
    double K[5][2];
    for (int i = 0; i < 5; ++i) {
        K[i][0] = C[i][0] * I00 + C[i][1] * I01;
        K[i][1] = C[i][0] * I01 + C[i][1] * I11;
    }
    for (int i = 0; i < 5; ++i) p[i] += K[i][0] * r0 + K[i][1] * r1;
    double N[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) N[i][j] = C[i][j] - (K[i][0] * C[0][j] + K[i][1] * C[1][j]);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) C[i][j] = 0.5 * (N[i][j] + N[j][i]);
    return r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
}

/* chi2 of a candidate hit against the predicted state, without updating */
static double predicted_chi2(const double* p, double C[5][5], double my, double mz,
                             double vy, double vz)
{
    const double r0 = my - p[0], r1 = mz - p[1];
    const double S00 = C[0][0] + vy, S01 = C[0][1], S11 = C[1][1] + vz;
    const double det = S00 * S11 - S01 * S01;
    return (S11 * r0 * r0 - 2.0 * S01 * r0 * r1 + S00 * r1 * r1) / det;
}

/* ------------------------------------------------------------------------ */
/* per-sector hit lists                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const double* y;      /* widened inputs */
    const double* z;
    const float* yf;      /* binary32 inputs for the C2 decision */
    const float* zf;
    const uint16_t* row;
    const uint16_t* sector;
    int n_rows, n_sectors;
    const double* xr;     /* widened row positions */
    const float* xrf;
    int64_t* list_off;    /* [(S*R)+1] */
    int32_t* list_cid;    /* cids grouped by (sector,row), ascending cid */
} hits_t;

static int row_list(const hits_t* H, int sec, int r, const int32_t** out)
{
    const int64_t k = (int64_t)sec * H->n_rows + r;
    *out = H->list_cid + H->list_off[k];
    return (int)(H->list_off[k + 1] - H->list_off[k]);
}

/* ------------------------------------------------------------------------ */
/* C2: neighbour finder (brute force over all hits of the adjacent rows)      */
/* ------------------------------------------------------------------------ */

/*
 * Hit h on row r (1 <= r <= R-2).  Candidate c on row r+-1 is admissible iff
 * |y_c - y_h| <= SY |x_c - x_h| and |z_c - z_h| <= SZ |x_c - x_h|.  Slopes
 * sy_u = (y_u - y_h)/(x_u - x_h), sy_d = (y_h - y_d)/(x_h - x_d), likewise z;
 * score D = (sy_u - sy_d)^2 + (sz_u - sz_d)^2, the straight-line kink.  The
 * admissible pair (d, u) with the least D wins, exact ties going to the lower
 * cid(u) and then the lower cid(d); the links are set iff D <= D_MAX.
 * Binary64 throughout.  *tie receives the near-tie bits of the decision:
 * ORC_C2_TIE_PAIR when the best D is at most D_MAX + tie_d and another
 * admissible pair lies within tie_d of it, ORC_C2_TIE_CUT when the best D
 * lies within tie_d of D_MAX, ORC_C2_TIE_WIN when a candidate lies within
 * tie_win cm of the edge of its slope window (inside the window widened by
 * tie_win and outside the window narrowed by it, in y or in z).
 */
static void best_pair_f64(const hits_t* H, const orc_config* cfg, int sec, int r, int32_t h,
                          int32_t* up, int32_t* dn, int32_t* tie)
{
    const int32_t *lu, *ld;
    const int nu = row_list(H, sec, r + 1, &lu);
    const int nd = row_list(H, sec, r - 1, &ld);
    const double xh = H->xr[r], xu = H->xr[r + 1], xd = H->xr[r - 1];
    const double wyu = cfg->slope_win_y * fabs(xu - xh), wzu = cfg->slope_win_z * fabs(xu - xh);
    const double wyd = cfg->slope_win_y * fabs(xd - xh), wzd = cfg->slope_win_z * fabs(xd - xh);
    const double tw = cfg->tie_win, dmax = cfg->d_max;
    int flags = 0;
    /* window edges: a candidate inside the widened window but not inside the
     * narrowed one sits within tie_win of an edge */
    for (int a = 0; a < nu + nd; ++a) {
        const int32_t c = a < nu ? lu[a] : ld[a - nu];
        const double wy = a < nu ? wyu : wyd, wz = a < nu ? wzu : wzd;
        const double ay = fabs(H->y[c] - H->y[h]), az = fabs(H->z[c] - H->z[h]);
        if (ay <= wy + tw && az <= wz + tw && (ay > wy - tw || az > wz - tw))
            flags |= ORC_C2_TIE_WIN;
    }
    double bestD = 0.0, second = INFINITY;
    int32_t bu = -1, bd = -1;
    for (int a = 0; a < nu; ++a) {
        const int32_t u = lu[a];
        if (!(fabs(H->y[u] - H->y[h]) <= wyu) || !(fabs(H->z[u] - H->z[h]) <= wzu)) continue;
        const double syu = (H->y[u] - H->y[h]) / (xu - xh);
        const double szu = (H->z[u] - H->z[h]) / (xu - xh);
        for (int b = 0; b < nd; ++b) {
            const int32_t d = ld[b];
            if (!(fabs(H->y[d] - H->y[h]) <= wyd) || !(fabs(H->z[d] - H->z[h]) <= wzd)) continue;
            const double syd = (H->y[h] - H->y[d]) / (xh - xd);
            const double szd = (H->z[h] - H->z[d]) / (xh - xd);
            const double D = (syu - syd) * (syu - syd) + (szu - szd) * (szu - szd);
            if (bu < 0 || D < bestD || (D == bestD && (u < bu || (u == bu && d < bd)))) {
                if (bu >= 0) second = bestD;
                bestD = D;
                bu = u;
                bd = d;
            } else if (D < second) {
                second = D;
            }
        }
    }
    if (bu >= 0 && bestD <= dmax + cfg->tie_d && second - bestD <= cfg->tie_d)
        flags |= ORC_C2_TIE_PAIR;
    if (bu >= 0 && fabs(bestD - dmax) <= cfg->tie_d) flags |= ORC_C2_TIE_CUT;
    *tie = flags;
    if (bu >= 0 && bestD <= dmax) { *up = bu; *dn = bd; }
    else { *up = -1; *dn = -1; }
}

/*
 * Diagnostic only: the same rule restated in binary32 (differences rounded,
 * slopes as differences times the rounded reciprocal of the row spacing,
 * one rounding per operation).  Its links are compared with the binary64
 * decision to show that they differ only at hits with near-tie bits; no
 * later step uses them.
 */
static void best_pair_f32(const hits_t* H, const orc_config* cfg, int sec, int r, int32_t h,
                          int32_t* up, int32_t* dn)
{
    const int32_t *lu, *ld;
    const int nu = row_list(H, sec, r + 1, &lu);
    const int nd = row_list(H, sec, r - 1, &ld);
    const float xh = H->xrf[r], xu = H->xrf[r + 1], xd = H->xrf[r - 1];
    const float iu = 1.0f / (xu - xh), id = 1.0f / (xh - xd);
    const float wyu = cfg->slope_win_y * fabsf(xu - xh), wzu = cfg->slope_win_z * fabsf(xu - xh);
    const float wyd = cfg->slope_win_y * fabsf(xd - xh), wzd = cfg->slope_win_z * fabsf(xd - xh);
    const float yh = H->yf[h], zh = H->zf[h];
    float bestD = 0.0f;
    int32_t bu = -1, bd = -1;
    for (int a = 0; a < nu; ++a) {
        const int32_t u = lu[a];
        const float ddyu = H->yf[u] - yh, ddzu = H->zf[u] - zh;
        if (!(fabsf(ddyu) <= wyu) || !(fabsf(ddzu) <= wzu)) continue;
        const float syu = ddyu * iu, szu = ddzu * iu;
        for (int b = 0; b < nd; ++b) {
            const int32_t d = ld[b];
            const float ddyd = yh - H->yf[d], ddzd = zh - H->zf[d];
            if (!(fabsf(ddyd) <= wyd) || !(fabsf(ddzd) <= wzd)) continue;
            const float syd = ddyd * id, szd = ddzd * id;
            const float ey = syu - syd, ez = szu - szd;
            const float ey2 = ey * ey, ez2 = ez * ez;
            const float D = ey2 + ez2;
            if (bu < 0 || D < bestD || (D == bestD && (u < bu || (u == bu && d < bd)))) {
                bestD = D;
                bu = u;
                bd = d;
            }
        }
    }
    if (bu >= 0 && bestD <= cfg->d_max) { *up = bu; *dn = bd; }
    else { *up = -1; *dn = -1; }
}

/* ------------------------------------------------------------------------ */
/* C7: tracklet construction from one chain                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int valid, nhits, first_row, last_row, flags, ndf;
    double x, p[5], C[5][5], chi2;
} tracklet_t;

/*
 * Seed covariance at a state with sin(phi) = s: diagonal, with the cluster
 * variances for (y, z), the variances seed_var_s and seed_var_t of the slopes
 * dy/dx and dz/dx carried over to sin(phi) and tan(lambda) at that direction
 * (d sin(phi)/d(dy/dx) = cos^3 phi, d tan(lambda)/d(dz/dx) = cos phi), and
 * seed_var_q for q/pT.
 */
static void seed_cov(const orc_config* cfg, double C[5][5], double s)
{
    const double c2 = 1.0 - s * s;
    memset(C, 0, 25 * sizeof(double));
    C[0][0] = cfg->sigma_y * cfg->sigma_y;
    C[1][1] = cfg->sigma_z * cfg->sigma_z;
    C[2][2] = cfg->seed_var_s * c2 * c2 * c2;
    C[3][3] = cfg->seed_var_t * c2;
    C[4][4] = cfg->seed_var_q;
}

/*
 * Seed of a tracklet from its first hit (x0, y0, z0) and the chain's last hit
 * (x1, y1, z1): tan(phi) = (y1 - y0)/(x1 - x0), s = tan(phi)/sqrt(1 + tan^2),
 * t = ((z1 - z0)/(x1 - x0)) cos(phi), q/pT = 0, at x0 with (y, z) of the first hit.
 */
static void seed_state(double x0, double y0, double z0, double x1, double y1, double z1,
                       double* p)
{
    const double tphi = (y1 - y0) / (x1 - x0);
    const double dzdx = (z1 - z0) / (x1 - x0);
    const double cphi = 1.0 / sqrt(1.0 + tphi * tphi);
    p[0] = y0;
    p[1] = z0;
    p[2] = tphi * cphi;
    p[3] = dzdx * cphi;
    p[4] = 0.0;
}

/*
 * Stop test of the searched rows: |y| > x tan(half_angle) + margin or
 * |z| > z_max + margin ends the pass.  Sets the edge near-tie flag.
 */
static int outside(const orc_config* cfg, double x, const double* p, int* flags)
{
    const double by = x * tan(cfg->half_angle) + cfg->edge_margin;
    const double bz = cfg->z_max + cfg->edge_margin;
    if (fabs(fabs(p[0]) - by) <= cfg->tie_edge || fabs(fabs(p[1]) - bz) <= cfg->tie_edge)
        *flags |= ORC_TIE_EDGE;
    return fabs(p[0]) > by || fabs(p[1]) > bz;
}

/*
 * Search row r of the sector for the hit of least predicted chi2 with
 * chi2 <= chi2_hit (exact ties to the lower cid).  Every hit of the row is
 * tried.  Returns the cid or -1, and sets the near-tie flags.
 */
static int32_t search_row(const hits_t* H, const orc_config* cfg, int sec, int r,
                          const double* p, double C[5][5], int* flags)
{
    const int32_t* l;
    const int n = row_list(H, sec, r, &l);
    const double vy = cfg->sigma_y * cfg->sigma_y, vz = cfg->sigma_z * cfg->sigma_z;
    double best = INFINITY, second = INFINITY;
    int32_t bc = -1;
    for (int a = 0; a < n; ++a) {
        const int32_t c = l[a];
        const double chi2 = predicted_chi2(p, C, H->y[c], H->z[c], vy, vz);
        if (chi2 < best || (chi2 == best && c < bc)) { second = best; best = chi2; bc = c; }
        else if (chi2 < second) second = chi2;
    }
    if (bc >= 0 && fabs(best - cfg->chi2_hit) <= cfg->tie_chi2) *flags |= ORC_TIE_CHI2_CUT;
    if (bc >= 0 && best <= cfg->chi2_hit + cfg->tie_chi2 && second - best <= cfg->tie_chi2)
        *flags |= ORC_TIE_CHI2_PAIR;
    if (bc >= 0 && best <= cfg->chi2_hit) return bc;
    return -1;
}

/*
 * Near-tie bits (flags): a chi2 decision within tie_chi2 of the cut or of
 * the runner-up, |s| within tie_sin of sin_max at a transport, |y| or |z|
 * within tie_edge of a stop bound, and ORC_TIE_CHAIN when a chain hit is
 * updated (without a test, as the chain prescribes) with a chi2 increment
 * above chi2_hit: such a chain is not one helix (the cellular automaton
 * joined two particles), the fit is pulled far outside its own covariance,
 * and its later decisions depend on the precision of the arithmetic.
 *
 * The tracklet of a chain h[0..k] on consecutive rows of sector sec
 * (k + 1 >= min_chain) is built in two passes.
 *
 * Forward: seed at x of h0 with (y, z) of h0, tan(phi) and dz/dx from the
 * chord h0 -> hk, s = tan(phi)/sqrt(1 + tan^2 phi), t = (dz/dx) cos(phi),
 * q/pT = 0, C = seed; update at h0, transport + update at each chain hit (no
 * test), then extend outward row by row with the chi2 search, ending after
 * max_gap misses in a row, at a transport failure or outside the sector.
 * The hits the extension search takes are the forward extension hits.
 */
typedef struct {
    int32_t* fwd;       /* [n_rows] forward hit per row (cid or -1) */
    int r0, rk, last;   /* first and last chain row, last assigned row */
    int flags;
    double pL[5];       /* state right after the update at row last */
} fwdpass_t;

static void forward_pass(const hits_t* H, const orc_config* cfg, int sec, const int32_t* chain,
                         int k1, fwdpass_t* F)
{
    const int R = H->n_rows;
    const double vy = cfg->sigma_y * cfg->sigma_y, vz = cfg->sigma_z * cfg->sigma_z;
    int32_t* fwd = F->fwd;
    for (int r = 0; r < R; ++r) fwd[r] = -1;
    int flags = 0;
    const int r0 = H->row[chain[0]];
    const int rk = H->row[chain[k1 - 1]];
    double p[5], C[5][5];
    seed_state(H->xr[r0], H->y[chain[0]], H->z[chain[0]], H->xr[rk], H->y[chain[k1 - 1]],
               H->z[chain[k1 - 1]], p);
    seed_cov(cfg, C, p[2]);
    double x = H->xr[r0];
    /* over the chain */
    orc_update(p, C, H->y[chain[0]], H->z[chain[0]], vy, vz);
    fwd[r0] = chain[0];
    int last = r0;
    memcpy(F->pL, p, sizeof(F->pL));
    int stopped = 0;
    for (int i = 1; i < k1; ++i) {
        const int r = H->row[chain[i]];
        if (orc_transport(x, H->xr[r], cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &flags)) {
            stopped = 1;
            break;
        }
        x = H->xr[r];
        if (orc_update(p, C, H->y[chain[i]], H->z[chain[i]], vy, vz) > cfg->chi2_hit)
            flags |= ORC_TIE_CHAIN;
        fwd[r] = chain[i];
        last = r;
        memcpy(F->pL, p, sizeof(F->pL));
    }
    /* extension */
    if (!stopped) {
        int gap = 0;
        for (int r = rk + 1; r < R; ++r) {
            if (orc_transport(x, H->xr[r], cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &flags))
                break;
            x = H->xr[r];
            if (outside(cfg, x, p, &flags)) break;
            const int32_t c = search_row(H, cfg, sec, r, p, C, &flags);
            if (c >= 0) {
                orc_update(p, C, H->y[c], H->z[c], vy, vz);
                fwd[r] = c;
                last = r;
                memcpy(F->pL, p, sizeof(F->pL));
                gap = 0;
            } else if (++gap >= cfg->max_gap) {
                break;
            }
        }
    }
    F->r0 = r0;
    F->rk = rk;
    F->last = last;
    F->flags = flags;
}

/*
 * Backward: from the last assigned row L with the forward state kept there
 * and C reset to the seed, update at L, then go inward: rows assigned forward
 * are updated without a test, rows below the first chain row are searched as
 * above.  The result is the state and covariance right after the last
 * backward update (the innermost hit); chi2 and ndf = 2 nUpd - 5 come from
 * the backward pass.  rowhit[] receives the backward hit set (cid per row,
 * -1 elsewhere).
 */
static void backward_pass(const hits_t* H, const orc_config* cfg, int sec, const fwdpass_t* F,
                          tracklet_t* T, int32_t* rowhit)
{
    const int R = H->n_rows;
    const double vy = cfg->sigma_y * cfg->sigma_y, vz = cfg->sigma_z * cfg->sigma_z;
    const int32_t* fwd = F->fwd;
    const int r0 = F->r0, last = F->last;
    int flags = F->flags;
    double p[5], C[5][5];
    for (int r = 0; r < R; ++r) rowhit[r] = -1;
    memcpy(p, F->pL, sizeof(p));
    seed_cov(cfg, C, p[2]);
    double x = H->xr[last];
    double chi2 = orc_update(p, C, H->y[fwd[last]], H->z[fwd[last]], vy, vz);
    int nupd = 1;
    rowhit[last] = fwd[last];
    int first = last;
    double pb[5], Cb[5][5], xb = x;
    memcpy(pb, p, sizeof(pb));
    memcpy(Cb, C, sizeof(Cb));
    int ok = 1;
    for (int r = last - 1; r >= r0 && ok; --r) {
        if (fwd[r] < 0) continue;
        if (orc_transport(x, H->xr[r], cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &flags)) {
            ok = 0;
            break;
        }
        x = H->xr[r];
        chi2 += orc_update(p, C, H->y[fwd[r]], H->z[fwd[r]], vy, vz);
        ++nupd;
        rowhit[r] = fwd[r];
        first = r;
        memcpy(pb, p, sizeof(pb));
        memcpy(Cb, C, sizeof(Cb));
        xb = x;
    }
    if (ok) {
        int gap = 0;
        for (int r = r0 - 1; r >= 0; --r) {
            if (orc_transport(x, H->xr[r], cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &flags))
                break;
            x = H->xr[r];
            if (outside(cfg, x, p, &flags)) break;
            const int32_t c = search_row(H, cfg, sec, r, p, C, &flags);
            if (c >= 0) {
                chi2 += orc_update(p, C, H->y[c], H->z[c], vy, vz);
                ++nupd;
                rowhit[r] = c;
                first = r;
                memcpy(pb, p, sizeof(pb));
                memcpy(Cb, C, sizeof(Cb));
                xb = x;
                gap = 0;
            } else if (++gap >= cfg->max_gap) {
                break;
            }
        }
    }
    T->nhits = nupd;
    T->first_row = first;
    T->last_row = last;
    T->x = xb;
    memcpy(T->p, pb, sizeof(pb));
    memcpy(T->C, Cb, sizeof(Cb));
    T->chi2 = chi2;
    T->ndf = 2 * nupd - 5;
    T->flags = flags;
    int fin = isfinite(chi2);
    for (int i = 0; i < 5; ++i) {
        fin = fin && isfinite(pb[i]) && Cb[i][i] > 0.0;
        for (int j = 0; j < 5; ++j) fin = fin && isfinite(Cb[i][j]);
    }
    T->valid = (nupd >= cfg->min_tracklet_hits) && fin;
}

/* ------------------------------------------------------------------------ */
/* whole event                                                                */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int32_t idx; } sortkey_t;

static int cmp_key(const void* a, const void* b)
{
    const uint64_t x = ((const sortkey_t*)a)->key, y = ((const sortkey_t*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Track one event: every sector on its own, C2 -> C8.  Clusters whose row or
 * sector is out of range, or whose y or z is not finite, are rejected (-1).
 * Returns 0, -1 on bad input, -4 when a capacity is exceeded.
 */
int orc_track_event(const orc_config* cfg, const float* row_x, int64_t n, const float* yf,
                    const float* zf, const uint16_t* row, const uint16_t* sector, orc_result* res)
{
    const int R = cfg->n_rows;
    const int S = cfg->n_sectors_phi * (cfg->split_z ? 2 : 1);
    if (R < 3 || R > 512 || S < 1) return -1;
    for (int64_t i = 0; i < n; ++i)
        if (row[i] >= R || sector[i] >= S || !isfinite(yf[i]) || !isfinite(zf[i])) return -1;

    hits_t H;
    H.n = n;
    H.n_rows = R;
    H.n_sectors = S;
    H.row = row;
    H.sector = sector;
    H.yf = yf;
    H.zf = zf;
    double* y = malloc(sizeof(double) * (n + 1));
    double* z = malloc(sizeof(double) * (n + 1));
    double* xr = malloc(sizeof(double) * R);
    H.list_off = calloc((size_t)S * R + 1, sizeof(int64_t));
    H.list_cid = malloc(sizeof(int32_t) * (n + 1));
    int64_t* fill = calloc((size_t)S * R, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) { y[i] = yf[i]; z[i] = zf[i]; }
    for (int r = 0; r < R; ++r) xr[r] = row_x[r];
    H.y = y; H.z = z; H.xr = xr; H.xrf = row_x;
    /* group cids by (sector, row): counting sort, ascending cid in each group */
    for (int64_t i = 0; i < n; ++i) H.list_off[(int64_t)sector[i] * R + row[i] + 1]++;
    for (int64_t k = 0; k < (int64_t)S * R; ++k) H.list_off[k + 1] += H.list_off[k];
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = (int64_t)sector[i] * R + row[i];
        H.list_cid[H.list_off[k] + fill[k]++] = (int32_t)i;
    }

    /* C2 */
    res->n_links = 0;
    res->n_link_flips32 = 0;
    res->n_c2_ties = 0;
    for (int64_t i = 0; i < n; ++i) {
        res->up[i] = res->dn[i] = -1;
        res->c2_tie[i] = 0;
        if (res->up32) res->up32[i] = res->dn32[i] = -1;
        const int r = row[i];
        if (r < 1 || r > R - 2) continue;
        best_pair_f64(&H, cfg, sector[i], r, (int32_t)i, &res->up[i], &res->dn[i], &res->c2_tie[i]);
        if (res->up[i] >= 0) res->n_links++;
        if (res->c2_tie[i]) res->n_c2_ties++;
        if (res->up32) {
            best_pair_f32(&H, cfg, sector[i], r, (int32_t)i, &res->up32[i], &res->dn32[i]);
            if (res->up32[i] != res->up[i] || res->dn32[i] != res->dn[i]) res->n_link_flips32++;
        }
    }
    /* C3: mutual links only */
    for (int64_t i = 0; i < n; ++i) {
        const int32_t u = res->up[i], d = res->dn[i];
        res->up_c[i] = (u >= 0 && res->dn[u] == (int32_t)i) ? u : -1;
        res->dn_c[i] = (d >= 0 && res->up[d] == (int32_t)i) ? d : -1;
    }
    /* C4 + C7: chains from start hits, in (sector, row, cid) order.  First
     * the forward pass of every chain, marking the hits its extension search
     * takes; then C7a: a chain all of whose hits are marked lies on a track
     * that other tracklets already follow outward, and gets no tracklet (it
     * is dominated); the others get their backward pass. */
    int status = 0;
    int64_t nt = 0;
    res->n_starts = 0;
    res->n_dominated = 0;
    int64_t cap_ch = 64, n_ch = 0, n_chain_hits = 0, cap_hits = 1024;
    int32_t* ch_start = malloc(sizeof(int32_t) * cap_ch);
    int32_t* ch_sec = malloc(sizeof(int32_t) * cap_ch);
    int64_t* ch_off = malloc(sizeof(int64_t) * (cap_ch + 1));
    int32_t* ch_hits = malloc(sizeof(int32_t) * cap_hits);
    ch_off[0] = 0;
    for (int64_t k = 0; k < (int64_t)S * R; ++k) {
        const int sec = (int)(k / R);
        for (int64_t a = H.list_off[k]; a < H.list_off[k + 1]; ++a) {
            const int32_t h = H.list_cid[a];
            if (!(res->up_c[h] >= 0 && res->dn_c[h] < 0)) continue;
            res->n_starts++;
            int len = 0;
            for (int32_t c = h; c >= 0 && len < R; c = res->up_c[c]) ++len;
            if (len < cfg->min_chain) continue;
            if (n_ch + 1 >= cap_ch) {
                cap_ch *= 2;
                ch_start = realloc(ch_start, sizeof(int32_t) * cap_ch);
                ch_sec = realloc(ch_sec, sizeof(int32_t) * cap_ch);
                ch_off = realloc(ch_off, sizeof(int64_t) * (cap_ch + 1));
            }
            while (n_chain_hits + len > cap_hits) {
                cap_hits *= 2;
                ch_hits = realloc(ch_hits, sizeof(int32_t) * cap_hits);
            }
            int q = 0;
            for (int32_t c = h; c >= 0 && q < len; c = res->up_c[c]) ch_hits[n_chain_hits + q++] = c;
            n_chain_hits += len;
            ch_start[n_ch] = h;
            ch_sec[n_ch] = sec;
            ch_off[++n_ch] = n_chain_hits;
        }
    }
    fwdpass_t* F = malloc(sizeof(fwdpass_t) * (n_ch + 1));
    int32_t* fwd_rows = malloc(sizeof(int32_t) * (size_t)(n_ch + 1) * R);
    unsigned char* marked = calloc((size_t)n + 1, 1);
    for (int64_t i = 0; i < n_ch; ++i) {
        F[i].fwd = fwd_rows + (size_t)i * R;
        forward_pass(&H, cfg, ch_sec[i], ch_hits + ch_off[i], (int)(ch_off[i + 1] - ch_off[i]), &F[i]);
        for (int r = F[i].rk + 1; r <= F[i].last; ++r)
            if (F[i].fwd[r] >= 0) marked[F[i].fwd[r]] |= F[i].flags ? 3 : 1;
    }
    if (res->fwd_mark)
        for (int64_t i = 0; i < n; ++i) res->fwd_mark[i] = marked[i];
    for (int64_t i = 0; i < n_ch && status == 0; ++i) {
        int all = 1;
        for (int64_t q = ch_off[i]; q < ch_off[i + 1]; ++q) all = all && marked[ch_hits[q]];
        if (all) {
            res->n_dominated++;
            continue;
        }
        if (nt >= res->cap_tracklets) { status = -4; break; }
        tracklet_t T;
        backward_pass(&H, cfg, ch_sec[i], &F[i], &T, res->t_rowhit + nt * R);
        res->t_start[nt] = ch_start[i];
        res->t_sector[nt] = ch_sec[i];
        res->t_chain_len[nt] = (int32_t)(ch_off[i + 1] - ch_off[i]);
        res->t_valid[nt] = T.valid;
        res->t_nhits[nt] = T.nhits;
        res->t_first_row[nt] = T.first_row;
        res->t_last_row[nt] = T.last_row;
        res->t_flags[nt] = T.flags;
        res->t_ndf[nt] = T.ndf;
        res->t_x[nt] = T.x;
        memcpy(res->t_p + nt * 5, T.p, sizeof(T.p));
        cov_to_tri(T.C, res->t_C + nt * 15);
        res->t_chi2[nt] = T.chi2;
        ++nt;
    }
    free(F); free(fwd_rows); free(marked);
    free(ch_start); free(ch_sec); free(ch_off); free(ch_hits);
    res->n_tracklets = nt;
    /* C7 weights: key = (nHits << 32) | (0xFFFFFFFF - cid(h0)), max over valid tracklets */
    for (int64_t i = 0; i < n; ++i) res->weight[i] = 0;
    for (int64_t t = 0; t < nt && status == 0; ++t) {
        if (!res->t_valid[t]) continue;
        const uint64_t key = ((uint64_t)res->t_nhits[t] << 32) |
                             (uint64_t)(0xFFFFFFFFu - (uint32_t)res->t_start[t]);
        for (int r = 0; r < R; ++r) {
            const int32_t c = res->t_rowhit[t * R + r];
            if (c >= 0 && key > res->weight[c]) res->weight[c] = key;
        }
    }
    /* C8 selector */
    int64_t nk = 0, nh = 0;
    sortkey_t* order = malloc(sizeof(sortkey_t) * (nt + 1));
    for (int64_t t = 0; t < nt && status == 0; ++t) {
        if (!res->t_valid[t]) continue;
        const uint64_t key = ((uint64_t)res->t_nhits[t] << 32) |
                             (uint64_t)(0xFFFFFFFFu - (uint32_t)res->t_start[t]);
        int own = 0, first_own = -1;
        for (int r = 0; r < R; ++r) {
            const int32_t c = res->t_rowhit[t * R + r];
            if (c >= 0 && res->weight[c] == key) {
                if (first_own < 0) first_own = r;
                ++own;
            }
        }
        if (own < cfg->min_track_hits || 2 * own < res->t_nhits[t]) continue;
        order[nk].key = ((uint64_t)res->t_sector[t] << 40) | ((uint64_t)first_own << 32) |
                        (uint64_t)(uint32_t)res->t_start[t];
        order[nk].idx = (int32_t)t;
        ++nk;
    }
    if (status == 0 && nk > res->cap_tracks) status = -4;
    if (status == 0) {
        qsort(order, (size_t)nk, sizeof(sortkey_t), cmp_key);
        res->k_hit_off[0] = 0;
        for (int64_t j = 0; j < nk; ++j) {
            const int32_t t = order[j].idx;
            const uint64_t key = ((uint64_t)res->t_nhits[t] << 32) |
                                 (uint64_t)(0xFFFFFFFFu - (uint32_t)res->t_start[t]);
            res->k_tracklet[j] = t;
            res->k_sector[j] = res->t_sector[t];
            res->k_ndf[j] = res->t_ndf[t];
            res->k_x[j] = res->t_x[t];
            memcpy(res->k_p + j * 5, res->t_p + (int64_t)t * 5, 5 * sizeof(double));
            memcpy(res->k_C + j * 15, res->t_C + (int64_t)t * 15, 15 * sizeof(double));
            res->k_chi2[j] = res->t_chi2[t];
            for (int r = 0; r < R; ++r) {
                const int32_t c = res->t_rowhit[(int64_t)t * R + r];
                if (c >= 0 && res->weight[c] == key) res->k_hit_cid[nh++] = c;
            }
            res->k_hit_off[j + 1] = (int32_t)nh;
        }
        res->n_tracks = nk;
        res->n_track_hits = nh;
    }
    free(order);
    free(y); free(z); free(xr); free(H.list_off); free(H.list_cid); free(fill);
    return status;
}

/* ------------------------------------------------------------------------ */
/* entry points for the unit checks                                           */
/* ------------------------------------------------------------------------ */

/* C5 on a packed covariance: p[5], Ct[15] in/out, J[25] out (row-major). */
int orc_transport_packed(double x0, double x1, double bz, double sin_max, double* p, double* Ct,
                         double* J)
{
    double C[5][5], Jl[5][5];
    tri_to_cov(Ct, C);
    const int rc = orc_transport(x0, x1, bz, sin_max, 0.0, p, C, Jl, NULL);
    if (rc == 0) {
        cov_to_tri(C, Ct);
        if (J) memcpy(J, Jl, sizeof(Jl));
    }
    return rc;
}

/* C6 on a packed covariance; returns the chi2 increment. */
double orc_update_packed(double* p, double* Ct, double my, double mz, double vy, double vz)
{
    double C[5][5];
    tri_to_cov(Ct, C);
    const double chi2 = orc_update(p, C, my, mz, vy, vz);
    cov_to_tri(C, Ct);
    return chi2;
}

/*
 * C7 on a given hit set (one hit per listed row, rows strictly ascending, all
 * of them used as the chain, no search), binary64 hits, then C9: n_iter more
 * backward passes, each seeded with the previous result moved to the
 * outermost hit and the covariance reset to the seed.  Outputs the state at
 * the innermost hit.  Returns 0 or -1 on a transport failure.
 */
int orc_fit_fixed(const orc_config* cfg, const double* xr, int n_hits, const int32_t* rows,
                  const double* hy, const double* hz, int n_iter, double* p_out, double* C_out,
                  double* chi2_out, int32_t* ndf_out)
{
    const double vy = cfg->sigma_y * cfg->sigma_y, vz = cfg->sigma_z * cfg->sigma_z;
    if (n_hits < 2) return -1;
    const int r0 = rows[0], rk = rows[n_hits - 1];
    double p[5], C[5][5];
    seed_state(xr[r0], hy[0], hz[0], xr[rk], hy[n_hits - 1], hz[n_hits - 1], p);
    seed_cov(cfg, C, p[2]);
    double x = xr[r0];
    orc_update(p, C, hy[0], hz[0], vy, vz);
    for (int i = 1; i < n_hits; ++i) {
        if (orc_transport(x, xr[rows[i]], cfg->bz, cfg->sin_max, 0.0, p, C, NULL, NULL)) return -1;
        x = xr[rows[i]];
        orc_update(p, C, hy[i], hz[i], vy, vz);
    }
    double chi2 = 0.0;
    for (int pass = 0; pass <= n_iter; ++pass) {
        if (pass > 0) {
            /* previous result (at the innermost hit) moved to the outermost hit */
            if (orc_transport(xr[r0], xr[rk], cfg->bz, cfg->sin_max, 0.0, p, NULL, NULL, NULL))
                return -1;
        }
        x = xr[rk];
        seed_cov(cfg, C, p[2]);
        chi2 = orc_update(p, C, hy[n_hits - 1], hz[n_hits - 1], vy, vz);
        for (int i = n_hits - 2; i >= 0; --i) {
            if (orc_transport(x, xr[rows[i]], cfg->bz, cfg->sin_max, 0.0, p, C, NULL, NULL))
                return -1;
            x = xr[rows[i]];
            chi2 += orc_update(p, C, hy[i], hz[i], vy, vz);
        }
    }
    memcpy(p_out, p, sizeof(p));
    cov_to_tri(C, C_out);
    *chi2_out = chi2;
    *ndf_out = 2 * n_hits - 5;
    return 0;
}

/* Seed state of C7 from two hits (for the unit checks). */
void orc_seed(double x0, double y0, double z0, double x1, double y1, double z1, double* p)
{
    seed_state(x0, y0, z0, x1, y1, z1, p);
}

/* ------------------------------------------------------------------------ */
/* M: sector track merger and global refit                                    */
/* ------------------------------------------------------------------------ */
/*
 * The paper places this step after the sector tracker (the tracker takes the
 * clusters of all TPC links of an event, Sect. 2) but gives no rule, so every
 * rule here is a reading:
 *
 *   M0 rotation of a state at x into a frame turned by d (d = alpha_to -
 *      alpha_from): x' = x cos d + y sin d, y' = -x sin d + y cos d,
 *      s' = s cos d - c sin d with c = sqrt(1 - s^2); the track must still
 *      move outward, c' = c cos d + s sin d > 0, and |s'| < sin_max; z, t and
 *      q/pT are unchanged.  The covariance is carried to the plane x' of the
 *      new frame (a change of y slides the point along the track back onto
 *      that plane): dy'/dy = c/c', dz'/dy = -t sin d / c', ds'/dy = -C_k sin d,
 *      ds'/ds = c'/c, the rest the identity.
 *   M1 outer state of a sector track: its state (at its innermost hit)
 *      transported to the plane of its outermost hit.
 *   M2 candidate pairs (a, b): b lies in a phi neighbour of a's sector in the
 *      same z half (frames turned by -+ 2 half_angle; across phi = 0 only
 *      when the sectors close the ring), or in a's phi sector in the other z
 *      half (same frame).
 *   M3 match of a pair: a's outer state turned into b's frame (M0), then
 *      transported to the plane x_b of b's state; admissible iff the gap
 *      x_b - x_a' lies in [dx_lo, dx_hi], M0 and the transport succeed, and
 *      chi2 = r^T (C_a' + C_b)^-1 r <= chi2_cut with r = p_a' - p_b.
 *   M4 links: a -> b iff b is the admissible partner of a with the least
 *      chi2 (ties to the lower index) and a is that of b; a chain starts at a
 *      track with an outgoing and no incoming link and follows the links.
 *   M5 refit of a chain s_1 (innermost) .. s_m: s_m's outer state, covariance
 *      reset to the seed covariance, updated with s_m's outermost hit; then
 *      every other hit inward (each segment's hits by descending row; at a
 *      change of segment the state is turned into the inner segment's frame
 *      and transported to its outermost hit).  The result is the state at
 *      s_1's innermost hit, chi2 the sum of the increments, ndf = 2 * hits - 5.
 *      A chain whose refit fails (a transport or rotation fails) is not
 *      merged; chains of any length are refitted (every track has at most
 *      one incoming and one outgoing link, so a chain from a head without an
 *      incoming link ends).
 *
 * Near-tie bits (for the parity tests) mark the tracks whose links could
 * change under rounding: a chi2 within tie_chi2 of the cut or of the next
 * candidate, and a pair that would be admissible (chi2 within the cut plus
 * tie_chi2) while its gap lies within tie_dx of the window or |s| within
 * tie_sin of sin_max at its rotation or transport.
 */

typedef struct {
    double chi2_cut, dx_lo, dx_hi;
    double tie_chi2, tie_dx;
} orc_merge_config;

enum { ORC_MTIE_CUT = 16, ORC_MTIE_PAIR = 32, ORC_MTIE_DX = 64, ORC_MTIE_SIN = 128 };

static void sandwich(const double J[5][5], double C[5][5])
{
    double T[5][5], N[5][5];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double a = 0.0;
            for (int k = 0; k < 5; ++k) a += J[i][k] * C[k][j];
            T[i][j] = a;
        }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double a = 0.0;
            for (int k = 0; k < 5; ++k) a += T[i][k] * J[j][k];
            N[i][j] = a;
        }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) C[i][j] = 0.5 * (N[i][j] + N[j][i]);
}

/* M0.  Returns 0, or -1 when the turned track would not move outward or
 * |s'| >= sin_max (nothing is changed then). */
int orc_rotate(double d, double bz, double sin_max, double tie, double* x, double* p,
               double C[5][5], double J[5][5], int* flags)
{
    const double cd = cos(d), sd = sin(d);
    const double s = p[2];
    if (!(fabs(s) < 1.0)) return -1;
    const double c = sqrt(1.0 - s * s);
    const double s1 = s * cd - c * sd;
    const double c1 = c * cd + s * sd;
    if (flags && fabs(fabs(s1) - sin_max) <= tie) *flags |= ORC_MTIE_SIN;
    if (!(c1 > 0.0) || !(fabs(s1) < sin_max)) return -1;
    const double ck = -ORC_KAPPA * bz * p[4];
    double Jr[5][5];
    memset(Jr, 0, sizeof(Jr));
    Jr[0][0] = c / c1;
    Jr[1][0] = -p[3] * sd / c1;
    Jr[1][1] = 1.0;
    Jr[2][0] = -ck * sd;
    Jr[2][2] = c1 / c;
    Jr[3][3] = 1.0;
    Jr[4][4] = 1.0;
    const double x1 = *x * cd + p[0] * sd;
    const double y1 = -*x * sd + p[0] * cd;
    *x = x1;
    p[0] = y1;
    p[2] = s1;
    if (C) sandwich(Jr, C);
    if (J) memcpy(J, Jr, sizeof(Jr));
    return 0;
}

/* M0 on a packed covariance (for the unit checks). */
int orc_rotate_packed(double d, double bz, double sin_max, double* x, double* p, double* Ct,
                      double* J)
{
    double C[5][5], Jr[5][5];
    tri_to_cov(Ct, C);
    const int rc = orc_rotate(d, bz, sin_max, 0.0, x, p, C, Jr, NULL);
    if (rc == 0) {
        cov_to_tri(C, Ct);
        if (J) memcpy(J, Jr, sizeof(Jr));
    }
    return rc;
}

/* r^T S^-1 r by Cholesky; -1 if S is not positive definite. */
static double chi2_5(const double r[5], double S[5][5])
{
    double L[5][5];
    memset(L, 0, sizeof(L));
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) {
            double a = S[i][j];
            for (int k = 0; k < j; ++k) a -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(a > 0.0)) return -1.0;
                L[i][i] = sqrt(a);
            } else {
                L[i][j] = a / L[j][j];
            }
        }
    double u[5], q = 0.0;
    for (int i = 0; i < 5; ++i) {
        double a = r[i];
        for (int k = 0; k < i; ++k) a -= L[i][k] * u[k];
        u[i] = a / L[i][i];
        q += u[i] * u[i];
    }
    return q;
}

static double sector_alpha(const orc_config* cfg, int sec)
{
    const int k = sec % cfg->n_sectors_phi;
    return (k + 0.5) * 2.0 * cfg->half_angle;
}

/* sectors whose tracks may continue a track of sector sa (M2); returns count */
static int merge_partners(const orc_config* cfg, int sa, int out[3], double d[3])
{
    const int N = cfg->n_sectors_phi;
    const int k = sa % N, half = sa / N;
    const int ring = N * 2.0 * cfg->half_angle > 4.0 * acos(0.0) - 1e-9;  /* closes the ring */
    int n = 0;
    for (int dk = -1; dk <= 1; dk += 2) {
        int kb = k + dk;
        if (kb < 0 || kb >= N) {
            if (!ring || N < 3) continue;
            kb = (kb + N) % N;
        }
        out[n] = half * N + kb;
        d[n] = dk * 2.0 * cfg->half_angle;
        ++n;
    }
    if (cfg->split_z) {
        out[n] = (1 - half) * N + k;
        d[n] = 0.0;
        ++n;
    }
    return n;
}

/*
 * M1-M5 on the sector tracks of one event (arrays as produced by
 * orc_track_event: sector, x, p[5], C[15], hit_off[T+1], hit_cid).
 * Outputs per track: link_out (index of the continuing track or -1), flags
 * (near-tie bits), match_chi2 (chi2 of its outgoing link), chain_head (the
 * first track of its merged chain, itself if not merged); per chain head with
 * m_ok = 1 the refit m_x, m_p[5], m_C[15], m_chi2, m_ndf and the chain's
 * length m_len.  Returns 0, or -1 on bad input.
 */
int orc_merge(const orc_config* cfg, const orc_merge_config* mc, const float* row_x,
              const float* yf, const float* zf, const uint16_t* row, int64_t T,
              const int32_t* sector, const double* tx, const double* tp, const double* tC,
              const int32_t* hit_off, const int32_t* hit_cid, int32_t* link_out, int32_t* flags,
              double* match_chi2, int32_t* chain_head, double* m_x, double* m_p, double* m_C,
              double* m_chi2, int32_t* m_ndf, int32_t* m_ok, int32_t* m_len)
{
    const int S = cfg->n_sectors_phi * (cfg->split_z ? 2 : 1);
    const double vy = cfg->sigma_y * cfg->sigma_y, vz = cfg->sigma_z * cfg->sigma_z;
    for (int64_t a = 0; a < T; ++a)
        if (sector[a] < 0 || sector[a] >= S || hit_off[a + 1] <= hit_off[a]) return -1;
    /* tracks grouped by sector (ascending index within a sector) */
    int64_t* soff = calloc((size_t)S + 1, sizeof(int64_t));
    int64_t* sidx = malloc(sizeof(int64_t) * (size_t)(T + 1));
    int64_t* fill = calloc((size_t)S, sizeof(int64_t));
    for (int64_t a = 0; a < T; ++a) soff[sector[a] + 1]++;
    for (int s = 0; s < S; ++s) soff[s + 1] += soff[s];
    for (int64_t a = 0; a < T; ++a) sidx[soff[sector[a]] + fill[sector[a]]++] = a;
    /* M1 */
    double* xo = malloc(sizeof(double) * (size_t)(T + 1));
    double* po = malloc(sizeof(double) * 5 * (size_t)(T + 1));
    double (*Co)[5][5] = malloc(sizeof(double[5][5]) * (size_t)(T + 1));
    int* oko = malloc(sizeof(int) * (size_t)(T + 1));
    for (int64_t a = 0; a < T; ++a) {
        const int32_t last = hit_cid[hit_off[a + 1] - 1];
        xo[a] = row_x[row[last]];
        memcpy(po + 5 * a, tp + 5 * a, 5 * sizeof(double));
        tri_to_cov(tC + 15 * a, Co[a]);
        int fl = 0;
        oko[a] = orc_transport(tx[a], xo[a], cfg->bz, cfg->sin_max, cfg->tie_sin, po + 5 * a,
                               Co[a], NULL, &fl) == 0;
        flags[a] = fl ? ORC_MTIE_SIN : 0;
    }
    /* M3: best partner per track on each side, with the runner-up for ties */
    int64_t* best_b = malloc(sizeof(int64_t) * (size_t)(T + 1));
    int64_t* best_a = malloc(sizeof(int64_t) * (size_t)(T + 1));
    double* chi_b = malloc(sizeof(double) * (size_t)(T + 1));
    double* chi_a = malloc(sizeof(double) * (size_t)(T + 1));
    double* chi_b2 = malloc(sizeof(double) * (size_t)(T + 1));
    double* chi_a2 = malloc(sizeof(double) * (size_t)(T + 1));
    for (int64_t a = 0; a < T; ++a) {
        best_b[a] = best_a[a] = -1;
        chi_b[a] = chi_a[a] = chi_b2[a] = chi_a2[a] = INFINITY;
    }
    for (int64_t a = 0; a < T; ++a) {
        if (!oko[a]) continue;
        int ps[3];
        double pd[3];
        const int np = merge_partners(cfg, sector[a], ps, pd);
        for (int q = 0; q < np; ++q) {
            /* a's outer state in the frame of sector ps[q] (independent of b);
             * a rotation that fails within the tie width is evaluated as if
             * it had passed, for the near-tie bits only */
            double xr = xo[a], pr[5], Cr[5][5];
            memcpy(pr, po + 5 * a, sizeof(pr));
            memcpy(Cr, Co[a], sizeof(Cr));
            int fr = 0, relaxed = 0;
            if (pd[q] != 0.0 &&
                orc_rotate(pd[q], cfg->bz, cfg->sin_max, cfg->tie_sin, &xr, pr, Cr, NULL, &fr)) {
                if (!fr) continue;
                xr = xo[a];
                memcpy(pr, po + 5 * a, sizeof(pr));
                memcpy(Cr, Co[a], sizeof(Cr));
                if (orc_rotate(pd[q], cfg->bz, 1.0 - 1e-9, 0.0, &xr, pr, Cr, NULL, NULL)) continue;
                relaxed = 1;
            }
            for (int64_t k = soff[ps[q]]; k < soff[ps[q] + 1]; ++k) {
                const int64_t b = sidx[k];
                double x = xr, p[5], C[5][5];
                memcpy(p, pr, sizeof(p));
                memcpy(C, Cr, sizeof(C));
                const double gap = tx[b] - x;
                const int near_dx = fabs(gap - mc->dx_lo) <= mc->tie_dx || fabs(gap - mc->dx_hi) <= mc->tie_dx;
                const int in_window = gap >= mc->dx_lo && gap <= mc->dx_hi;
                if (!in_window && !near_dx) continue;
                int ft = 0;
                int bad = orc_transport(x, tx[b], cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &ft);
                if (bad) {
                    if (!ft) continue;
                    memcpy(p, pr, sizeof(p));
                    memcpy(C, Cr, sizeof(C));
                    if (orc_transport(x, tx[b], cfg->bz, 1.0 - 1e-9, 0.0, p, C, NULL, NULL)) continue;
                }
                double r[5], Sm[5][5], Cb[5][5];
                tri_to_cov(tC + 15 * b, Cb);
                for (int i = 0; i < 5; ++i) {
                    r[i] = p[i] - tp[5 * b + i];
                    for (int j = 0; j < 5; ++j) Sm[i][j] = C[i][j] + Cb[i][j];
                }
                const double chi2 = chi2_5(r, Sm);
                if (chi2 < 0.0) continue;
                /* a bound met within its tie width matters only for a pair
                 * that could be admissible */
                if ((ft || fr || near_dx) && chi2 <= mc->chi2_cut + mc->tie_chi2) {
                    const int bit = near_dx ? ORC_MTIE_DX : ORC_MTIE_SIN;
                    flags[a] |= bit;
                    flags[b] |= bit;
                }
                if (relaxed || bad || !in_window) continue;
                if (fabs(chi2 - mc->chi2_cut) <= mc->tie_chi2) {
                    flags[a] |= ORC_MTIE_CUT;
                    flags[b] |= ORC_MTIE_CUT;
                }
                if (!(chi2 <= mc->chi2_cut)) continue;
                /* least chi2, ties to the lower index (candidates of b come in
                 * ascending a, those of a in ascending b within a sector, and
                 * sectors in the order above; compare indices explicitly) */
                if (chi2 < chi_b[a] || (chi2 == chi_b[a] && b < best_b[a])) {
                    chi_b2[a] = chi_b[a];
                    chi_b[a] = chi2;
                    best_b[a] = b;
                } else if (chi2 < chi_b2[a]) {
                    chi_b2[a] = chi2;
                }
                if (chi2 < chi_a[b] || (chi2 == chi_a[b] && a < best_a[b])) {
                    chi_a2[b] = chi_a[b];
                    chi_a[b] = chi2;
                    best_a[b] = a;
                } else if (chi2 < chi_a2[b]) {
                    chi_a2[b] = chi2;
                }
            }
        }
    }
    for (int64_t a = 0; a < T; ++a) {
        if (chi_b2[a] - chi_b[a] <= mc->tie_chi2) flags[a] |= ORC_MTIE_PAIR;
        if (chi_a2[a] - chi_a[a] <= mc->tie_chi2) flags[a] |= ORC_MTIE_PAIR;
    }
    /* M4 */
    int64_t* link_in = malloc(sizeof(int64_t) * (size_t)(T + 1));
    for (int64_t a = 0; a < T; ++a) link_in[a] = -1;
    for (int64_t a = 0; a < T; ++a) {
        link_out[a] = -1;
        match_chi2[a] = 0.0;
        chain_head[a] = (int32_t)a;
        m_ok[a] = 0;
        m_len[a] = 1;
        const int64_t b = best_b[a];
        if (b >= 0 && best_a[b] == a) {
            link_out[a] = (int32_t)b;
            match_chi2[a] = chi_b[a];
        }
    }
    for (int64_t a = 0; a < T; ++a)
        if (link_out[a] >= 0) link_in[link_out[a]] = a;
    /* M5 */
    int64_t* chain = malloc(sizeof(int64_t) * (size_t)(T + 1));
    for (int64_t h = 0; h < T; ++h) {
        if (link_in[h] >= 0 || link_out[h] < 0) continue;
        int m = 0;
        for (int64_t a = h; a >= 0 && m < T; a = link_out[a]) chain[m++] = a;
        /* start: outer state of the outermost segment, seed covariance */
        const int64_t so = chain[m - 1];
        double x = xo[so], p[5], C[5][5];
        memcpy(p, po + 5 * so, sizeof(p));
        seed_cov(cfg, C, p[2]);
        double chi2 = 0.0;
        int n_upd = 0, ok = oko[so];
        for (int g = m - 1; g >= 0 && ok; --g) {
            const int64_t a = chain[g];
            if (g < m - 1) {
                const double d = sector_alpha(cfg, sector[a]) - sector_alpha(cfg, sector[chain[g + 1]]);
                int fl = 0;
                if (d != 0.0 && orc_rotate(d, cfg->bz, cfg->sin_max, cfg->tie_sin, &x, p, C, NULL, &fl)) ok = 0;
                if (fl) flags[a] |= ORC_MTIE_SIN;
            }
            for (int32_t k = hit_off[a + 1] - 1; k >= hit_off[a] && ok; --k) {
                const int32_t c = hit_cid[k];
                const double xh = row_x[row[c]];
                if (xh != x) {
                    int ft = 0;
                    if (orc_transport(x, xh, cfg->bz, cfg->sin_max, cfg->tie_sin, p, C, NULL, &ft)) ok = 0;
                    if (ft) flags[a] |= ORC_MTIE_SIN;
                    x = xh;
                }
                if (ok) {
                    chi2 += orc_update(p, C, yf[c], zf[c], vy, vz);
                    ++n_upd;
                }
            }
        }
        if (!ok) continue;
        m_ok[h] = 1;
        m_len[h] = m;
        m_x[h] = x;
        memcpy(m_p + 5 * h, p, sizeof(p));
        cov_to_tri(C, m_C + 15 * h);
        m_chi2[h] = chi2;
        m_ndf[h] = 2 * n_upd - 5;
        for (int g = 0; g < m; ++g) chain_head[chain[g]] = (int32_t)h;
    }
    free(soff); free(sidx); free(fill); free(xo); free(po); free(Co); free(oko);
    free(best_b); free(best_a); free(chi_b); free(chi_a); free(chi_b2); free(chi_a2);
    free(link_in); free(chain);
    return 0;
}
