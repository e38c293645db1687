"""Seeded synthetic TPC events for the sector tracker.

This module only simulates events: charged helices from a vertex in a uniform
solenoidal field (B along +z) cross the planar pad rows of the TPC sectors, and
every crossing on the outgoing branch leaves one cluster, smeared in y and z.
It holds none of the tracker's arithmetic (no transport in the sector frame, no
fit, no neighbour rule); the circle geometry here works in the global frame.
Both the CUDA tracker's tests and the CPU oracle's tests draw their inputs from
here, so that the two see identical events.

The paper gives no event model (its Table 1 runs on ALICE Pb-Pb data that is
not available); these synthetic events stand in for it:

* pT = 0.1 * 100**U GeV/c, eta ~ U(-0.9, 0.9), phi0 ~ U(0, 2pi), q = +-1,
  B = 0.5 T, so the signed curvature is dphi/dS = -KAPPA * B * q / pT.
* pad row r is the plane x = row_x[r] of each 20-degree sector frame, with
  row_x = 85 + r * 162/158 cm (159 rows), held in binary32 so the tracker and
  the generator place the planes at the same positions.
* sector k of 18 in phi has its centre at alpha_k = (k + 0.5) * 20 deg; with
  ``split_z`` the sectors are doubled at the z = 0 membrane (sector k + 18 for
  z < 0).  A crossing is in the sector if |y_local| <= x * tan(10 deg).
* one cluster per row on the outgoing branch (vertex to the point of largest
  distance from the beam axis), crossing the plane with local x increasing; the
  branch ends at |z| > z_max or where it first crosses a row plane of a sector
  that is not instrumented.
* Gaussian smear sigma_y = sigma_z = 0.1 cm; noise = round(0.05 * N_signal)
  clusters uniform in sector, row, y within the row's width and z within the
  sector's range; MC label = particle index, -1 for noise.
* clusters are shuffled; the cluster id (cid) of a cluster is its input index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KAPPA = 0.299792458e-2  # cm^-1 per (GeV/c)^-1 per tesla
N_ROWS = 159
X_FIRST, X_LAST = 85.0, 247.0
HALF_ANGLE = math.radians(10.0)
Z_MAX = 250.0
BZ = 0.5
N_PHI_FULL = 18


def default_row_x(n_rows: int = N_ROWS) -> np.ndarray:
    """Pad-row radii as binary32: 85 + r * (162 / 158) cm."""
    r = np.arange(n_rows, dtype=np.float64)
    return (X_FIRST + r * ((X_LAST - X_FIRST) / (n_rows - 1))).astype(np.float32)


@dataclass
class Particles:
    q: np.ndarray
    pt: np.ndarray
    tanl: np.ndarray
    phi0: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray

    def __len__(self):
        return len(self.q)

    @staticmethod
    def concat(parts: list["Particles"]) -> "Particles":
        return Particles(*[np.concatenate([getattr(p, f) for p in parts])
                           for f in ("q", "pt", "tanl", "phi0", "vx", "vy", "vz")])


@dataclass
class Event:
    """One event: SoA clusters plus the geometry they were generated in."""
    y: np.ndarray           # float32 (float64 for noiseless fits)
    z: np.ndarray
    row: np.ndarray         # uint16
    sector: np.ndarray      # uint16
    label: np.ndarray       # int32, particle index or -1
    row_x: np.ndarray       # float32 [n_rows]
    n_sectors_phi: int
    split_z: int
    half_angle: float = HALF_ANGLE
    z_max: float = Z_MAX
    bz: float = BZ
    particles: Particles | None = None
    # per-cluster truth in the sector frame (unsmeared), for fit checks
    true_y: np.ndarray | None = None
    true_z: np.ndarray | None = None
    true_sinphi: np.ndarray | None = None
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.y)

    @property
    def n_sectors(self) -> int:
        return self.n_sectors_phi * (2 if self.split_z else 1)

    def select_sectors(self, sectors) -> "Event":
        """Sub-event holding only the clusters of the given sectors (ids kept)."""
        m = np.isin(self.sector, np.asarray(sectors))
        sub = Event(self.y[m], self.z[m], self.row[m], self.sector[m], self.label[m],
                    self.row_x, self.n_sectors_phi, self.split_z, self.half_angle,
                    self.z_max, self.bz, self.particles,
                    None if self.true_y is None else self.true_y[m],
                    None if self.true_z is None else self.true_z[m],
                    None if self.true_sinphi is None else self.true_sinphi[m],
                    dict(self.info, parent_index=np.nonzero(m)[0]))
        return sub


def draw_particles(rng: np.random.Generator, n: int, *, phi_range=(0.0, 2 * math.pi),
                   vertex_r=(0.0, 0.0), vertex_z=(0.0, 0.0)) -> Particles:
    """pT log-uniform in 0.1-10 GeV/c, |eta| < 0.9, charge +-1, vertex as given."""
    pt = 0.1 * 100.0 ** rng.random(n)
    eta = rng.uniform(-0.9, 0.9, n)
    phi0 = rng.uniform(phi_range[0], phi_range[1], n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    rv = rng.uniform(vertex_r[0], vertex_r[1], n) if vertex_r[1] > 0 else np.zeros(n)
    phv = rng.uniform(0.0, 2 * math.pi, n)
    vz = (rng.uniform(vertex_z[0], vertex_z[1], n) if vertex_z[1] > vertex_z[0]
          else np.full(n, float(vertex_z[0])))
    return Particles(q=q, pt=pt, tanl=np.sinh(eta), phi0=phi0,
                     vx=rv * np.cos(phv), vy=rv * np.sin(phv), vz=vz)


def helix_crossings(p: Particles, row_x: np.ndarray, *, instrumented_phi: np.ndarray,
                    split_z: bool, z_max: float = Z_MAX, bz: float = BZ,
                    half_angle: float = HALF_ANGLE):
    """Closed-form crossings of each helix with the row planes of all 18 phi-sectors.

    Global-frame circle: centre c = v + (1/C)(-sin phi0, cos phi0), position
    P(phi) = c + (1/C)(sin phi, -cos phi), arc length S = (phi - phi0)/C taken
    modulo one turn.  The plane of row r in sector k is n_k . P = x_r with
    n_k = (cos a_k, sin a_k); outward crossings have sin(phi - a_k) = C (x_r - n_k.c)
    with cos(phi - a_k) > 0.  Returns per-cluster arrays (particle, row, sector,
    y_local, z, sin(phi - a_k)) in float64, before smearing.
    """
    n = len(p)
    R = len(row_x)
    xr = row_x.astype(np.float64)
    C = -KAPPA * bz * p.q / p.pt
    xc = p.vx - np.sin(p.phi0) / C
    yc = p.vy + np.cos(p.phi0) / C
    two_pi = 2.0 * math.pi
    sgn = np.sign(C)
    # first maximum of the distance from the beam axis after the vertex
    beta = np.arctan2(yc, xc)
    phi_turn = beta + sgn * (math.pi / 2)
    s_turn = np.mod((phi_turn - p.phi0) * sgn, two_pi)
    s_turn = np.where(s_turn <= 0.0, two_pi, s_turn) / np.abs(C)

    alpha = (np.arange(N_PHI_FULL) + 0.5) * (2.0 * half_angle)
    ca, sa = np.cos(alpha), np.sin(alpha)
    xcl = xc[:, None] * ca[None, :] + yc[:, None] * sa[None, :]   # [n, 18]
    ycl = -xc[:, None] * sa[None, :] + yc[:, None] * ca[None, :]
    tanh_ = math.tan(half_angle)

    best_S = np.full((n, R), np.inf)
    best_k = np.full((n, R), -1, dtype=np.int64)
    best_y = np.zeros((n, R))
    best_s = np.zeros((n, R))
    for r in range(R):
        v = C[:, None] * (xr[r] - xcl)
        ok = np.abs(v) < 1.0
        vv = np.where(ok, v, 0.0)
        psi = np.arcsin(vv)
        phi = alpha[None, :] + psi
        S = np.mod((phi - p.phi0[:, None]) * sgn[:, None], two_pi) / np.abs(C)[:, None]
        yl = ycl - np.cos(psi) / C[:, None]
        ok &= S <= s_turn[:, None]
        ok &= np.abs(yl) <= xr[r] * tanh_
        S = np.where(ok, S, np.inf)
        k = np.argmin(S, axis=1)
        idx = np.arange(n)
        best_S[:, r] = S[idx, k]
        best_k[:, r] = np.where(np.isfinite(S[idx, k]), k, -1)
        best_y[:, r] = yl[idx, k]
        best_s[:, r] = vv[idx, k]
    has = np.isfinite(best_S)
    z = p.vz[:, None] + p.tanl[:, None] * np.where(has, best_S, 0.0)
    instr = np.zeros(N_PHI_FULL, dtype=bool)
    instr[instrumented_phi] = True
    bad = has & ((np.abs(z) > z_max) | ~instr[np.maximum(best_k, 0)])
    s_stop = np.where(bad, best_S, np.inf).min(axis=1)
    keep = has & (best_S < s_stop[:, None])
    pi_, ri_ = np.nonzero(keep)
    k_ = best_k[pi_, ri_]
    zz = z[pi_, ri_]
    sector = k_.copy()
    if split_z:
        sector = sector + N_PHI_FULL * (zz < 0.0)
    return pi_, ri_, sector, best_y[pi_, ri_], zz, best_s[pi_, ri_]


def make_event(rng: np.random.Generator, particles: Particles, *, n_sectors_phi: int,
               split_z: bool, sigma: float = 0.1, noise_frac: float = 0.05,
               row_x: np.ndarray | None = None, dtype=np.float32,
               shuffle: bool = True) -> Event:
    """Clusters of the given particles plus uniform noise, shuffled."""
    row_x = default_row_x() if row_x is None else row_x
    instrumented = np.arange(n_sectors_phi)
    pi_, ri_, sec, yl, zz, sl = helix_crossings(particles, row_x, instrumented_phi=instrumented,
                                                split_z=split_z)
    ns = len(pi_)
    ys = yl + (rng.normal(0.0, sigma, ns) if sigma > 0 else 0.0)
    zs = zz + (rng.normal(0.0, sigma, ns) if sigma > 0 else 0.0)
    n_noise = int(round(noise_frac * ns))
    n_sec = n_sectors_phi * (2 if split_z else 1)
    nsec = rng.integers(0, n_sec, n_noise)
    nrow = rng.integers(0, len(row_x), n_noise)
    xr = row_x.astype(np.float64)[nrow]
    ny = rng.uniform(-1.0, 1.0, n_noise) * xr * math.tan(HALF_ANGLE)
    if split_z:
        nz = np.where(nsec < n_sectors_phi, rng.uniform(0.0, Z_MAX, n_noise),
                      rng.uniform(-Z_MAX, 0.0, n_noise))
    else:
        nz = rng.uniform(-Z_MAX, Z_MAX, n_noise)
    y = np.concatenate([ys, ny])
    z = np.concatenate([zs, nz])
    row = np.concatenate([ri_, nrow]).astype(np.uint16)
    sector = np.concatenate([sec, nsec]).astype(np.uint16)
    label = np.concatenate([pi_, np.full(n_noise, -1)]).astype(np.int32)
    ty = np.concatenate([yl, np.full(n_noise, np.nan)])
    tz = np.concatenate([zz, np.full(n_noise, np.nan)])
    ts = np.concatenate([sl, np.full(n_noise, np.nan)])
    order = rng.permutation(len(y)) if shuffle else np.arange(len(y))
    return Event(y=y[order].astype(dtype), z=z[order].astype(dtype), row=row[order],
                 sector=sector[order], label=label[order], row_x=row_x,
                 n_sectors_phi=n_sectors_phi, split_z=int(split_z), particles=particles,
                 true_y=ty[order], true_z=tz[order], true_sinphi=ts[order],
                 info={"n_signal": ns, "n_noise": n_noise})


# --------------------------------------------------------------------------
# The five workloads (seeds fixed)
# --------------------------------------------------------------------------

def one_sector_event(seed: int = 1, n_tracks: int = 200, **kw) -> Event:
    """One 20-degree sector, |z| < 250 cm tracked as one sector, primaries from the origin."""
    rng = np.random.default_rng(seed)
    p = draw_particles(rng, n_tracks, phi_range=(0.0, 2 * HALF_ANGLE))
    return make_event(rng, p, n_sectors_phi=1, split_z=False, **kw)


def central_event(seed: int = 2, n_primaries: int = 10_000, secondary_frac: float = 0.1,
                  **kw) -> Event:
    """36 sectors: primaries from the origin plus secondaries from vertices with r ~ U(0, 50) cm."""
    rng = np.random.default_rng(seed)
    prim = draw_particles(rng, n_primaries)
    n_sec = int(round(secondary_frac * n_primaries))
    sec = draw_particles(rng, n_sec, vertex_r=(0.0, 50.0))
    return make_event(rng, Particles.concat([prim, sec]), n_sectors_phi=N_PHI_FULL,
                      split_z=True, **kw)


def batch_multiplicities(n_events: int = 64, seed0: int = 3000) -> list[int]:
    """n_tracks = round(20 * 500**U) per event, one seed per event."""
    return [int(round(20 * 500 ** np.random.default_rng(seed0 + i).random()))
            for i in range(n_events)]


def batch_events(n_events: int = 64, seed0: int = 3000) -> list[Event]:
    """Events of uneven multiplicity, log-uniform from 20 to 10,000 tracks."""
    out = []
    for i in range(n_events):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(20 * 500 ** rng.random()))
        prim = draw_particles(rng, n)
        sec = draw_particles(rng, int(round(0.1 * n)), vertex_r=(0.0, 50.0))
        out.append(make_event(rng, Particles.concat([prim, sec]), n_sectors_phi=N_PHI_FULL,
                              split_z=True))
    return out


def served_multiplicity(rng: np.random.Generator) -> int:
    """min(10000, max(1, round(Exp(mean 1500))))."""
    return int(min(10_000, max(1, round(rng.exponential(1500.0)))))


def served_event(rng: np.random.Generator, n_tracks: int) -> Event:
    prim = draw_particles(rng, n_tracks)
    sec = draw_particles(rng, int(round(0.1 * n_tracks)), vertex_r=(0.0, 50.0))
    return make_event(rng, Particles.concat([prim, sec]), n_sectors_phi=N_PHI_FULL, split_z=True)


def pileup_event(seed: int = 5, n_collisions: int = 50) -> Event:
    """Collisions of 200-2000 tracks with vertex z ~ U(-200, 200) cm merged into one event."""
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_collisions):
        n = int(rng.integers(200, 2001))
        vz = rng.uniform(-200.0, 200.0)
        parts.append(draw_particles(rng, n, vertex_z=(vz, vz)))
    return make_event(rng, Particles.concat(parts), n_sectors_phi=N_PHI_FULL, split_z=True)


def noiseless_track(q: float, pt: float, tanl: float, phi0: float, *, vx=0.0, vy=0.0, vz=0.0,
                    n_sectors_phi=1) -> Event:
    """One helix, no smear, no noise, float64 coordinates (for exact fit checks)."""
    p = Particles(q=np.array([q]), pt=np.array([pt]), tanl=np.array([tanl]),
                  phi0=np.array([phi0]), vx=np.array([vx]), vy=np.array([vy]), vz=np.array([vz]))
    rng = np.random.default_rng(0)
    return make_event(rng, p, n_sectors_phi=n_sectors_phi, split_z=False, sigma=0.0,
                      noise_frac=0.0, dtype=np.float64, shuffle=False)


def mc_performance(ev: Event, sector, hit_off, hit_cid, *, min_clusters: int = 30,
                   match_frac: float = 0.9, pt_min: float = 0.2) -> dict:
    """Tracks against the generator's labels, per particle segment in a sector.

    A track matches particle P when at least match_frac of its hits carry P's
    label; it then matches the segment (P, its sector).  A segment is
    reconstructable when it holds at least min_clusters clusters.  Returns
    efficiency (all segments and pT >= pt_min), fake rate (unmatched tracks)
    and clone rate (extra matches of a segment), over all tracks given.
    """
    sector = np.asarray(sector, np.int64)
    hit_off = np.asarray(hit_off, np.int64)
    hit_cid = np.asarray(hit_cid, np.int64)
    n_tr = len(sector)
    n_seg_sec = int(ev.n_sectors_phi * (2 if ev.split_z else 1))
    lab = ev.label.astype(np.int64)
    res = {"n_tracks": n_tr}
    matched = np.zeros(0, np.int64)
    fakes = n_tr
    if n_tr:
        nh = np.diff(hit_off)
        tid = np.repeat(np.arange(n_tr), nh)
        l = lab[hit_cid] + 1  # 0 = noise
        key = tid * (int(lab.max()) + 2) + l
        k, c = np.unique(key, return_counts=True)
        kt, kl = k // (int(lab.max()) + 2), k % (int(lab.max()) + 2)
        order = np.lexsort((-c, kt))  # per track, largest count first
        first = np.ones(len(order), bool)
        first[1:] = kt[order][1:] != kt[order][:-1]
        best_t, best_l, best_c = kt[order][first], kl[order][first], c[order][first]
        ok = (best_l > 0) & (best_c >= match_frac * nh[best_t])
        matched = (best_l[ok] - 1) * n_seg_sec + sector[best_t[ok]]
        fakes = n_tr - int(ok.sum())
    sig = lab >= 0
    seg = lab[sig] * n_seg_sec + ev.sector[sig].astype(np.int64)
    sk, sc = np.unique(seg, return_counts=True)
    recble = sk[sc >= min_clusters]
    mk, mc = np.unique(matched, return_counts=True)
    found = np.isin(recble, mk)
    pt = ev.particles.pt[recble // n_seg_sec]
    res["n_reconstructable"] = int(len(recble))
    res["efficiency"] = float(found.mean()) if len(recble) else float("nan")
    sel = pt >= pt_min
    res[f"efficiency_pt{pt_min:g}"] = float(found[sel].mean()) if sel.any() else float("nan")
    res["fake_rate"] = fakes / max(1, n_tr)
    res["clone_rate"] = int(np.sum(mc - 1)) / max(1, n_tr)
    return res


def particle_performance(ev: Event, hit_off, hit_cid, *, min_clusters: int = 30,
                         match_frac: float = 0.9) -> dict:
    """Tracks against the generator's labels, per particle (all its sectors
    together, unlike mc_performance).

    A track matches particle P when at least match_frac of its hits carry P's
    label.  A particle is reconstructable when it left at least min_clusters
    clusters.  Returns the efficiency (reconstructable particles with a
    matching track), the mean number of matching tracks per found particle
    (1 when no particle is split into pieces) and the fake rate (tracks that
    match no particle)."""
    hit_off = np.asarray(hit_off, np.int64)
    hit_cid = np.asarray(hit_cid, np.int64)
    n_tr = len(hit_off) - 1
    lab = ev.label.astype(np.int64)
    n_part = int(lab.max()) + 1 if len(lab) else 0
    counts = np.bincount(lab[lab >= 0], minlength=n_part)
    reco = counts >= min_clusters
    res = {"n_tracks": n_tr, "reconstructable": int(reco.sum())}
    if n_tr <= 0 or n_part == 0:
        res.update(efficiency=0.0, tracks_per_found_particle=0.0, fake_rate=0.0)
        return res
    nh = np.diff(hit_off)
    tid = np.repeat(np.arange(n_tr), nh)
    l = lab[hit_cid] + 1  # 0 = noise
    key = tid * (n_part + 1) + l
    k, c = np.unique(key, return_counts=True)
    kt, kl = k // (n_part + 1), k % (n_part + 1)
    order = np.lexsort((-c, kt))
    first = np.ones(len(order), bool)
    first[1:] = kt[order][1:] != kt[order][:-1]
    best_t, best_l, best_c = kt[order][first], kl[order][first], c[order][first]
    ok = (best_l > 0) & (best_c >= match_frac * nh[best_t])
    per_part = np.bincount(best_l[ok] - 1, minlength=n_part)
    found = reco & (per_part > 0)
    res["efficiency"] = float(found.sum() / max(1, reco.sum()))
    res["tracks_per_found_particle"] = float(per_part[found].sum() / max(1, found.sum()))
    res["fake_rate"] = float(1.0 - ok.sum() / n_tr)
    return res
