"""FP64 reference of the support initialiser: a crude OSEM on binned data.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper reduces the cost of the list-mode reconstruction, which grows
with the number of non-zero voxels, by first estimating the object's
boundary from a crude OSEM reconstruction of the binned sinogram (Sec. 2.2,
last paragraph).  It gives no details; the reading here (and in the
library) is:

* sinogram c[a, k]: events of angle a in position bin k = floor((u + U/2)/w)
  (U = n_bins w the detector extent; u = U/2 goes to the last bin), every
  energy of the window;
* crude projector, no attenuation, no scatter, no energy: the collimator
  response integrated over the bin,
      A[a, k, n] = 1/2 [erf((hi_k - u_a(p_n)) / (sqrt 2 sigma)) - erf((lo_k - u_a(p_n)) / (sqrt 2 sigma))],
  sigma = sigma_u(d_a(p_n)), over every pixel n of the grid;
* ordered subsets by angle (a mod N_s), subset sensitivity
  s^i_n = sum_{a in A_i} sum_k A[a, k, n], uniform start f_n = sum c / sum_n s_n,
  update f_n <- f_n / s^i_n sum_{a in A_i, k} A[a, k, n] c[a, k] / y[a, k] with
  y = A f (bins with y = 0 contribute nothing; s^i_n = 0 gives f_n = 0);
* support = {n : f_n >= tau max f}, dilated by r pixels (square neighbourhood).
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def geometry_arrays(g: dict, nx: int, ny: int, pixel_mm: float):
    """u_a(p_n) and sigma_u(d_a(p_n)) of every angle a and grid pixel n."""
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    x = ((ix.reshape(-1) + 0.5 - 0.5 * nx) * pixel_mm).astype(np.float64)
    y = ((iy.reshape(-1) + 0.5 - 0.5 * ny) * pixel_mm).astype(np.float64)
    th = g["angle0_rad"] + 2.0 * np.pi * np.arange(g["n_angles"]) / g["n_angles"]
    u = -np.outer(np.sin(th), x) + np.outer(np.cos(th), y)
    depth = g["radius_mm"] - (np.outer(np.cos(th), x) + np.outer(np.sin(th), y))
    sigma = (g["coll_fwhm0_mm"] + g["coll_fwhm_slope"] * depth) / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    return u, sigma


def projector(g: dict, nx: int, ny: int, pixel_mm: float):
    """A[a, k, n] of the crude projector (FP64, erf of the bin edges)."""
    u, sigma = geometry_arrays(g, nx, ny, pixel_mm)
    w = g["bin_mm"]
    edges = -0.5 * g["n_bins"] * w + w * np.arange(g["n_bins"] + 1)
    z = (edges[None, :, None] - u[:, None, :]) / (math.sqrt(2.0) * sigma[:, None, :])
    E = _erf(z)
    return 0.5 * (E[:, 1:, :] - E[:, :-1, :])


def sinogram(g: dict, angle, u_mm):
    """Event counts per (angle, position bin)."""
    w = g["bin_mm"]
    k = np.floor((np.asarray(u_mm, dtype=np.float64) + 0.5 * g["n_bins"] * w) / w).astype(np.int64)
    k = np.clip(k, 0, g["n_bins"] - 1)
    c = np.zeros((g["n_angles"], g["n_bins"]), dtype=np.float64)
    np.add.at(c, (np.asarray(angle, dtype=np.int64), k), 1.0)
    return c


def osem(A, c, n_subsets: int, n_iters: int):
    """Crude OSEM on the sinogram; returns the image and its per-sub-iteration
    history (for the count-conservation pin)."""
    n_angles = A.shape[0]
    sens = np.stack([A[i::n_subsets].sum(axis=(0, 1)) for i in range(n_subsets)])
    f = np.full(A.shape[2], c.sum() / sens.sum(), dtype=np.float64)
    hist = []
    for _ in range(n_iters):
        for i in range(n_subsets):
            Ai = A[i::n_subsets]                      # angles a with a mod N_s == i
            ci = c[i::n_subsets]
            y = np.einsum("akn,n->ak", Ai, f)
            r = np.where(y > 0, ci / np.where(y > 0, y, 1.0), 0.0)
            back = np.einsum("akn,ak->n", Ai, r)
            f = np.where(sens[i] > 0, f * back / np.where(sens[i] > 0, sens[i], 1.0), 0.0)
            hist.append((i, f.copy(), y))
    return f, sens, hist


def support_mask(f, nx: int, ny: int, threshold: float, dilate: int):
    """{f >= threshold max f}, dilated by `dilate` pixels (square neighbourhood)."""
    core = (f >= threshold * f.max()).reshape(ny, nx)
    out = np.zeros_like(core)
    for dy in range(-dilate, dilate + 1):
        for dx in range(-dilate, dilate + 1):
            src = core[max(0, -dy):ny - max(0, dy), max(0, -dx):nx - max(0, dx)]
            out[max(0, dy):ny - max(0, -dy), max(0, dx):nx - max(0, -dx)] |= src
    return out.reshape(-1)
