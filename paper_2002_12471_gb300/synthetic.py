"""Seeded synthetic inputs: phantoms, geometries and list-mode events.

This module is the only code shared by the CUDA path's tests and the oracle's
tests, and it holds none of the reconstruction's arithmetic: it computes no
system-model entry, no sensitivity and no EM step.  It only makes inputs.

* Phantoms are ellipse unions rasterised by 8 x 8 sub-sampling per pixel
  (area average), shaped like the 2-D DaT-scan study of the paper (Section 3:
  striatal uptake in caudate and putamen inside a head with a skull).  The
  paper's Zubal phantom is not available; these stand in for it.
* Events come from a small 2-D photon Monte-Carlo, standing in for the
  paper's Monte-Carlo list-mode simulator (Section 3): emission from the
  activity map, Woodcock (delta) tracking through the mu-map, in-plane
  Compton scattering of any order with the Klein-Nishina angular law, escape
  towards the nearest of the detector angles, then a depth-dependent Gaussian
  collimator blur on position and a Gaussian energy blur.  It is a data
  source, like a real scanner: it does not evaluate the model the
  reconstruction uses, and it includes higher scatter orders the first-order
  model leaves out.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MEC2_KEV = 510.99895


# ------------------------------------------------------------------ geometry

def geometry(n_angles, n_bins, bin_mm, radius_mm, *, angle0_rad=0.0, coll_fwhm0_mm=2.5,
             coll_fwhm_slope=0.05, e0_kev=159.0, fwhm_frac_e0=0.10, e_lo_kev=100.0,
             e_hi_kev=175.0):
    """Scanner description shared by both sides (plain numbers only)."""
    return dict(n_angles=int(n_angles), angle0_rad=float(angle0_rad), n_bins=int(n_bins),
                bin_mm=float(bin_mm), radius_mm=float(radius_mm),
                coll_fwhm0_mm=float(coll_fwhm0_mm), coll_fwhm_slope=float(coll_fwhm_slope),
                e0_kev=float(e0_kev), fwhm_frac_e0=float(fwhm_frac_e0),
                e_lo_kev=float(e_lo_kev), e_hi_kev=float(e_hi_kev))


# ------------------------------------------------------------------ phantoms

@dataclass
class Phantom:
    mu: np.ndarray          # ny x nx, per mm, at the photopeak energy
    activity: np.ndarray    # ny x nx, arbitrary units
    pixel_mm: float
    rois: dict = field(default_factory=dict)   # name -> ny x nx area fractions


def _subsample_grid(n, pixel_mm, sub=8):
    """Sub-sample coordinates (mm) of an n x n grid centred on the origin."""
    k = (np.arange(n * sub) + 0.5) / sub - 0.5 * n
    return k * pixel_mm


def _ellipse(x, y, cx, cy, ax, ay, rot_deg=0.0):
    t = math.radians(rot_deg)
    dx, dy = x - cx, y - cy
    xr = dx * math.cos(t) + dy * math.sin(t)
    yr = -dx * math.sin(t) + dy * math.cos(t)
    return (xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0


def _area_average(field_hi, n, sub=8):
    return field_hi.reshape(n, sub, n, sub).mean(axis=(1, 3))


def disk_phantom(n=16, pixel_mm=8.0, sub=8, hot_ratio=6.0):
    """Tiny case: water disk r = 56 mm (mu 0.0146/mm) whose outer 8 mm is a
    bone ring (mu 0.025/mm); two hot disks r = 8 mm at (+-16, 12) mm."""
    c = _subsample_grid(n, pixel_mm, sub)
    X, Y = np.meshgrid(c, c)
    r = np.hypot(X, Y)
    mu = np.where(r <= 56.0, np.where(r > 48.0, 0.025, 0.0146), 0.0)
    act = np.where(r <= 48.0, 1.0, 0.0)
    hot = _ellipse(X, Y, -16, 12, 8, 8) | _ellipse(X, Y, 16, 12, 8, 8)
    act = np.where(hot, hot_ratio, act)
    return Phantom(mu=_area_average(mu, n, sub), activity=_area_average(act, n, sub),
                   pixel_mm=pixel_mm, rois={"hot": _area_average(hot * 1.0, n, sub)})


def brain_phantom(n=64, pixel_mm=4.0, sub=8, uptake=8.0, jitter=None):
    """DaT-like 2-D brain: head 78 x 96 mm semi-axes with a 6 mm skull
    (mu 0.025/mm) around a brain (mu 0.0146/mm, activity 1); caudate L/R at
    (-+11, 18) mm, semi-axes 5 x 9, rotated -+15 deg; putamen L/R at (-+25, 2)
    mm, semi-axes 5.5 x 14, rotated -+10 deg; striatal activity ``uptake``.

    ``jitter`` (a numpy Generator) perturbs centres by +-2 mm, axes by a factor
    in [0.9, 1.1] and the uptake in [6, 10] (the family used to train the
    scatter surrogate)."""
    c = _subsample_grid(n, pixel_mm, sub)
    X, Y = np.meshgrid(c, c)

    def jit_c(v):
        return v + (jitter.uniform(-2, 2) if jitter is not None else 0.0)

    def jit_a(v):
        return v * (jitter.uniform(0.9, 1.1) if jitter is not None else 1.0)

    if jitter is not None:
        uptake = jitter.uniform(6.0, 10.0)
    hx, hy = jit_a(78.0), jit_a(96.0)
    head = _ellipse(X, Y, 0, 0, hx, hy)
    brain = _ellipse(X, Y, 0, 0, hx - 6.0, hy - 6.0)
    caud = (_ellipse(X, Y, jit_c(-11), jit_c(18), jit_a(5), jit_a(9), -15)
            | _ellipse(X, Y, jit_c(11), jit_c(18), jit_a(5), jit_a(9), 15))
    put = (_ellipse(X, Y, jit_c(-25), jit_c(2), jit_a(5.5), jit_a(14), -10)
           | _ellipse(X, Y, jit_c(25), jit_c(2), jit_a(5.5), jit_a(14), 10))
    mu = np.where(brain, 0.0146, np.where(head, 0.025, 0.0))
    act = np.where(brain, 1.0, 0.0)
    act = np.where(brain & (caud | put), uptake, act)
    return Phantom(mu=_area_average(mu, n, sub), activity=_area_average(act, n, sub),
                   pixel_mm=pixel_mm,
                   rois={"caudate": _area_average(caud * 1.0, n, sub),
                         "putamen": _area_average(put * 1.0, n, sub)})


# ------------------------------------------------------------------ workloads

def workload(name):
    """The named workloads: (phantom, geometry, n_events, n_subsets, n_iters)."""
    if name == "tiny16":
        ph = disk_phantom()
        g = geometry(32, 16, 8.0, 80.0)
        return ph, g, 2000, 4, 5
    if name == "dat64":
        ph = brain_phantom(64, 4.0)
        g = geometry(120, 64, 4.0, 150.0)
        return ph, g, 200_000, 8, 10
    if name == "dat128":
        ph = brain_phantom(128, 2.0)
        g = geometry(120, 128, 2.0, 150.0)
        return ph, g, 1_000_000, 8, 10
    if name == "dat32":
        # mid-size parity case: several tiles of every kernel and ragged tails
        ph = brain_phantom(32, 8.0)
        g = geometry(60, 32, 8.0, 150.0)
        return ph, g, 20_000, 6, 4
    raise KeyError(name)


# ------------------------------------------------------------------ events

@dataclass
class Events:
    angle: np.ndarray   # int32, detector angle index
    u_mm: np.ndarray    # float32, lateral position on the detector
    e_kev: np.ndarray   # float32, deposited energy
    order: np.ndarray   # int8, true scatter order (diagnostic only)

    def __len__(self):
        return len(self.angle)


def _kn_sim_total(e_kev):
    """Simulator's material law: total Klein-Nishina cross section (textbook
    form, units of 2 pi r_e^2), used only to scale mu with photon energy."""
    k = e_kev / MEC2_KEV
    l = np.log1p(2 * k)
    return ((1 + k) / k ** 2 * (2 * (1 + k) / (1 + 2 * k) - l / k) + l / (2 * k)
            - (1 + 3 * k) / (1 + 2 * k) ** 2)


def _sample_deflection(rng, e_kev):
    """In-plane Compton deflection angle psi in [0, 2 pi) with density
    proportional to the Klein-Nishina shape (which is <= 1), by rejection."""
    n = len(e_kev)
    psi = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        cand = rng.uniform(0.0, 2 * np.pi, len(todo))
        c = np.cos(cand)
        e = e_kev[todo]
        p = 1.0 / (1.0 + e / MEC2_KEV * (1.0 - c))
        shape = 0.5 * p * p * (p + 1.0 / p - (1.0 - c * c))
        acc = rng.uniform(0.0, 1.0, len(todo)) < shape
        psi[todo[acc]] = cand[acc]
        todo = todo[~acc]
    return psi


def _photon_batch(rng, ph: Phantom, g: dict, n: int, max_order: int):
    """Track ``n`` emitted photons; return (angle, u, E, order) of those
    detected inside the extent and the window."""
    ny, nx = ph.mu.shape
    dpx = ph.pixel_mm
    xmin, ymin = -0.5 * nx * dpx, -0.5 * ny * dpx
    mu0 = ph.mu.reshape(-1)
    mu_max0 = float(mu0.max())
    cdf = np.cumsum(ph.activity.reshape(-1).astype(np.float64))
    cdf /= cdf[-1]
    e0 = g["e0_kev"]
    s0 = _kn_sim_total(np.array(e0))
    half = 0.5 * g["n_bins"] * g["bin_mm"]
    dth = 2 * np.pi / g["n_angles"]
    fw2s = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    pix = np.searchsorted(cdf, rng.uniform(0.0, 1.0, n), side="right")
    pix = np.minimum(pix, nx * ny - 1)
    x = xmin + (pix % nx + rng.uniform(0, 1, n)) * dpx
    y = ymin + (pix // nx + rng.uniform(0, 1, n)) * dpx
    phi = rng.uniform(0.0, 2 * np.pi, n)
    e = np.full(n, e0)
    order = np.zeros(n, dtype=np.int8)
    lx, ly = x.copy(), y.copy()            # last emission / interaction point
    alive = np.ones(n, dtype=bool)
    escaped = np.zeros(n, dtype=bool)
    while True:
        idx = np.nonzero(alive & ~escaped)[0]
        if len(idx) == 0:
            break
        mu_max = mu_max0 * _kn_sim_total(e[idx]) / s0
        step = -np.log(rng.uniform(0.0, 1.0, len(idx)) + 1e-300) / mu_max
        x[idx] += step * np.cos(phi[idx])
        y[idx] += step * np.sin(phi[idx])
        ix = np.floor((x[idx] - xmin) / dpx).astype(np.int64)
        iy = np.floor((y[idx] - ymin) / dpx).astype(np.int64)
        inside = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
        escaped[idx[~inside]] = True
        idx, ix, iy = idx[inside], ix[inside], iy[inside]
        real = rng.uniform(0.0, 1.0, len(idx)) * mu_max0 < mu0[iy * nx + ix]
        hit = idx[real]
        if len(hit):
            psi = _sample_deflection(rng, e[hit])
            e[hit] = e[hit] / (1.0 + e[hit] / MEC2_KEV * (1.0 - np.cos(psi)))
            phi[hit] = np.mod(phi[hit] + psi, 2 * np.pi)
            order[hit] += 1
            lx[hit], ly[hit] = x[hit], y[hit]
            alive[hit[order[hit] > max_order]] = False
    det = np.nonzero(escaped & alive)[0]
    a = np.mod(np.rint((phi[det] - g["angle0_rad"]) / dth).astype(np.int64), g["n_angles"])
    th = g["angle0_rad"] + a * dth
    px, py = lx[det], ly[det]
    depth = g["radius_mm"] - (px * np.cos(th) + py * np.sin(th))
    su = (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * depth) * fw2s
    u = -px * np.sin(th) + py * np.cos(th) + su * rng.standard_normal(len(det))
    se = g["fwhm_frac_e0"] * np.sqrt(e0 * e[det]) * fw2s
    em = e[det] + se * rng.standard_normal(len(det))
    keep = (np.abs(u) <= half) & (em >= g["e_lo_kev"]) & (em <= g["e_hi_kev"])
    u32 = u[keep].astype(np.float32)
    e32 = em[keep].astype(np.float32)
    # float32 rounding must not push a value out of the acceptance region
    u32 = np.clip(u32, np.float32(-half), np.float32(half))
    e32 = np.clip(e32, np.float32(g["e_lo_kev"]), np.float32(g["e_hi_kev"]))
    return a[keep].astype(np.int32), u32, e32, order[det][keep]


def simulate_events(ph: Phantom, g: dict, n_events: int, seed: int, *, max_order=6,
                    batch=1 << 20) -> Events:
    """Exactly ``n_events`` detected events from a seeded photon Monte-Carlo
    (Philox bit generator keyed by ``seed``)."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    out = []
    got = 0
    while got < n_events:
        out.append(_photon_batch(rng, ph, g, batch, max_order))
        got += len(out[-1][0])
    A, U, E, O = (np.concatenate(c)[:n_events] for c in zip(*out))
    return Events(angle=A, u_mm=U, e_kev=E, order=O)


def simulate_emissions(ph: Phantom, g: dict, n_emitted: int, seed: int, *, max_order=6,
                       batch=1 << 20) -> Events:
    """Every detected event of exactly ``n_emitted`` emitted photons (same
    Monte-Carlo as ``simulate_events``), so that counts per scatter order can
    be compared with their expectation per emitted photon."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    out = []
    left = int(n_emitted)
    while left > 0:
        n = min(batch, left)
        out.append(_photon_batch(rng, ph, g, n, max_order))
        left -= n
    A, U, E, O = (np.concatenate(c) for c in zip(*out))
    return Events(angle=A, u_mm=U, e_kev=E, order=O)


def realisation_counts(n_real=64, seed=4, lo=50_000, hi=400_000):
    """Uneven event counts of independent noise realisations:
    lambda_r = lo + (hi - lo) U_r, J_r ~ Poisson(lambda_r)."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    lam = lo + (hi - lo) * rng.uniform(0.0, 1.0, n_real)
    return rng.poisson(lam).astype(np.int64)


def bin_events(ev: Events, g: dict, e_edges) -> np.ndarray:
    """Binned data of a list of events (the paper's binning experiment,
    Section 4): photon counts per (angle, detector position bin, energy bin)
    as a float32 array [n_angles, n_bins, len(e_edges) - 1].  Position bins
    are the detector's (n_bins of bin_mm centred on the axis); energy bin k
    is [e_edges[k], e_edges[k + 1]) (the last bin closed).  Events outside
    the extent or the edges are dropped.  A histogram: no model arithmetic."""
    edges = np.asarray(e_edges, dtype=np.float64)
    nb, K = int(g["n_bins"]), len(edges) - 1
    half = 0.5 * nb * g["bin_mm"]
    u = np.asarray(ev.u_mm, dtype=np.float64)
    e = np.asarray(ev.e_kev, dtype=np.float64)
    a = np.asarray(ev.angle, dtype=np.int64)
    b = np.floor((u + half) / g["bin_mm"]).astype(np.int64)
    b = np.where(u == half, nb - 1, b)
    k = np.searchsorted(edges, e, side="right") - 1
    k = np.where(e == edges[-1], K - 1, k)
    ok = (b >= 0) & (b < nb) & (k >= 0) & (k < K) & (a >= 0) & (a < g["n_angles"])
    counts = np.zeros((int(g["n_angles"]), nb, K), dtype=np.float64)
    np.add.at(counts, (a[ok], b[ok], k[ok]), 1.0)
    return counts.astype(np.float32)
