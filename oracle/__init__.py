"""FP64 CPU oracle for list-mode OS-LM-MLEM with attenuation and scatter
compensation (Rahman, Laforest, Jha, ISBI 2020).

TEST INFRASTRUCTURE ONLY.  Tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library under
``paper_2002_12471_gb300`` never does, and shares no code with it.

The path-sum model and the sensitivity are plain C (``lmosem_oracle.c``,
compiled on first use with gcc, OpenMP over events only).  The EM update and
the log-likelihood are written here with numpy, one line per equation:

* Eq. 8  (E-step):   zbar_{j,P_q} = f_q p_jq / y_j with y_j = sum_n p_jn f_n
* Eq. 7  (OS M-step): f_q <- sum_{j in S_i} zbar_{j,P_q} / (T s^i_q)
* Eq. 3  (log-likelihood, without the constant log J!):
         l(f) = sum_j log(T y_j) - T sum_n s_n f_n

Binned attributes (the paper's binning experiment, Section 4): a row is a
bin (angle, position bin, energy bin) with a count n_i; its model is the
event model integrated over the bin, and the EM update and the likelihood
weight each row by its count (n_i identical events).

Where the paper is silent, the reading taken is stated in the docstring of
the function that uses it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmosem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblmosem_oracle.so")
_lock = threading.Lock()
_lib = None

MEC2_KEV = 510.99895


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liblmosem_oracle.so`` (gcc, -O2,
    OpenMP, IEEE arithmetic: no fast-math)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    compile_source(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_source(src, out):
    """gcc a copy of the C oracle into a shared library (same flags as
    ``build``); the tests use it for copies with a planted mistake."""
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", out, src, "-lm"])
    return out


class Geom(ctypes.Structure):
    """Mirror of ``orc_geom`` (the oracle's own copy of the problem statement)."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("pixel_mm", ctypes.c_double),
        ("n_angles", ctypes.c_int32), ("angle0_rad", ctypes.c_double),
        ("n_bins", ctypes.c_int32), ("bin_mm", ctypes.c_double),
        ("radius_mm", ctypes.c_double),
        ("coll_fwhm0_mm", ctypes.c_double), ("coll_fwhm_slope", ctypes.c_double),
        ("e0_kev", ctypes.c_double), ("fwhm_frac_e0", ctypes.c_double),
        ("e_lo_kev", ctypes.c_double), ("e_hi_kev", ctypes.c_double),
        ("pos_cut", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def load(path):
    """Load a compiled copy of ``lmosem_oracle.c`` and declare its functions
    (``lib()`` loads the one ``build()`` makes)."""
    L = ctypes.CDLL(path)
    L.orc_compton_energy.restype = ctypes.c_double
    L.orc_compton_energy.argtypes = [ctypes.c_double, ctypes.c_double]
    L.orc_kn_shape.restype = ctypes.c_double
    L.orc_kn_shape.argtypes = [ctypes.c_double, ctypes.c_double]
    L.orc_kn_mean.restype = ctypes.c_double
    L.orc_kn_mean.argtypes = [ctypes.c_double]
    L.orc_sigma_kn.restype = ctypes.c_double
    L.orc_sigma_kn.argtypes = [ctypes.c_double]
    L.orc_line_integral.restype = ctypes.c_double
    L.orc_line_integral.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double]
    L.orc_ray_to_edge.restype = ctypes.c_double
    L.orc_ray_to_edge.argtypes = L.orc_line_integral.argtypes
    L.orc_det_u.restype = ctypes.c_double
    L.orc_det_u.argtypes = [ctypes.POINTER(Geom), ctypes.c_int,
                            ctypes.c_double, ctypes.c_double]
    L.orc_det_depth.restype = ctypes.c_double
    L.orc_det_depth.argtypes = L.orc_det_u.argtypes
    L.orc_build_tables.restype = None
    L.orc_build_tables.argtypes = [ctypes.POINTER(Geom), _dp, _ip, ctypes.c_int,
                                   _ip, ctypes.c_int, _dp, _dp]
    L.orc_model.restype = None
    L.orc_model.argtypes = [ctypes.POINTER(Geom), _dp, _ip, ctypes.c_int, _ip,
                            ctypes.c_int, _dp, _dp, _ip, _dp, _dp, ctypes.c_int64, _dp,
                            ctypes.c_int]
    L.orc_model_binned.restype = None
    L.orc_model_binned.argtypes = [ctypes.POINTER(Geom), _dp, _ip, ctypes.c_int, _ip,
                                   ctypes.c_int, _dp, _dp, _ip, _ip, _ip, ctypes.c_int64,
                                   _dp, _dp, ctypes.c_int]
    L.orc_sensitivity.restype = None
    L.orc_sensitivity.argtypes = [ctypes.POINTER(Geom), _dp, _ip, ctypes.c_int, _ip,
                                  ctypes.c_int, _dp, _dp, ctypes.c_int, _dp,
                                  ctypes.c_int]
    return L


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


# ---------------------------------------------------------------- physics

def compton_energy(e_kev, cos_psi):
    return lib().orc_compton_energy(float(e_kev), float(cos_psi))


def kn_shape(e_kev, cos_psi):
    return lib().orc_kn_shape(float(e_kev), float(cos_psi))


def kn_mean(e_kev):
    return lib().orc_kn_mean(float(e_kev))


def sigma_kn(e_kev):
    return lib().orc_sigma_kn(float(e_kev))


def line_integral(mu, dpx, p0, p1):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    ny, nx = mu.shape
    return lib().orc_line_integral(_d(mu), nx, ny, float(dpx), float(p0[0]), float(p0[1]),
                                   float(p1[0]), float(p1[1]))


def ray_to_edge(mu, dpx, p0, direction):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    ny, nx = mu.shape
    return lib().orc_ray_to_edge(_d(mu), nx, ny, float(dpx), float(p0[0]), float(p0[1]),
                                 float(direction[0]), float(direction[1]))


# ---------------------------------------------------------------- problem

# 0.5 z^2 above this  <=>  the Gaussian position factor is below 1e-16 of its
# peak: terms that small cannot change an FP64 sum.
DEFAULT_POS_CUT = float(-np.log(1e-16))


class Problem:
    """The oracle's copy of one reconstruction problem: geometry, mu-map at
    E0 (per mm, ny x nx), emission support and scatter pixel lists, and the
    attenuation tables (built once, FP64).

    ``support`` defaults to {mu > 0}; scatter pixels are always {mu > 0}
    (a photon can only Compton-scatter where there is matter)."""

    def __init__(self, geom: dict, mu, support=None, pos_cut: float = DEFAULT_POS_CUT):
        self.mu = np.ascontiguousarray(mu, dtype=np.float64)
        ny, nx = self.mu.shape
        g = Geom()
        g.nx, g.ny = nx, ny
        for k in ("pixel_mm", "angle0_rad", "bin_mm", "radius_mm", "coll_fwhm0_mm",
                  "coll_fwhm_slope", "e0_kev", "fwhm_frac_e0", "e_lo_kev", "e_hi_kev"):
            setattr(g, k, float(geom[k]))
        g.n_angles = int(geom["n_angles"])
        g.n_bins = int(geom["n_bins"])
        g.pos_cut = float(pos_cut)
        self.geom = g
        flat = self.mu.reshape(-1)
        if support is None:
            sup = np.nonzero(flat > 0)[0]
        else:
            sup = np.nonzero(np.asarray(support).reshape(-1) != 0)[0]
        self.support = np.ascontiguousarray(sup, dtype=np.int32)
        self.scatter = np.ascontiguousarray(np.nonzero(flat > 0)[0], dtype=np.int32)
        self.l_edge = np.zeros((g.n_angles, nx * ny), dtype=np.float64)
        self.l_pair = np.zeros((len(self.support), len(self.scatter)), dtype=np.float64)
        lib().orc_build_tables(ctypes.byref(g), _d(self.mu), _i(self.support), len(self.support),
                               _i(self.scatter), len(self.scatter), _d(self.l_edge),
                               _d(self.l_pair))

    @property
    def n_sup(self):
        return len(self.support)

    def pixel_centres(self, pix):
        g = self.geom
        pix = np.asarray(pix)
        ix, iy = pix % g.nx, pix // g.nx
        return ((ix + 0.5 - 0.5 * g.nx) * g.pixel_mm, (iy + 0.5 - 0.5 * g.ny) * g.pixel_mm)

    def line_attenuation(self, angle, u_mm, s_mm):
        """Attenuation inputs of the scatter surrogate: the integral of mu(E0)
        along the detector line {s omega_a + u t_a} of angle a from depth s
        on, towards the detector.  Definition (the one the surrogate's
        inputs use): exact integrals (``ray_to_edge``) at nodes h = half a
        pixel apart, u_i = -U + i h (U = half the detector extent + 3h/4:
        no node line runs along a grid line at the axis angles, where the
        integral would depend on which side of it rounding falls) and
        s_k = -S + k h (S = half the grid diagonal + h, so s_0 lies before
        the grid and the node at s_0 is the whole line), interpolated
        bilinearly; u and s are clamped to [node 0, last node - 1e-3 h].
        Nodes are computed on demand and cached."""
        g = self.geom
        h = 0.5 * g.pixel_mm
        U = 0.5 * g.n_bins * g.bin_mm + 0.75 * h
        S = 0.5 * g.pixel_mm * np.hypot(g.nx, g.ny) + h
        nu, ns = int(np.ceil(2 * U / h)) + 1, int(np.ceil(2 * S / h)) + 1
        cache = self.__dict__.setdefault("_line_nodes", {})

        def node(a, i, k):
            key = (a, i, k)
            if key not in cache:
                th = g.angle0_rad + 2.0 * np.pi * a / g.n_angles
                om = (np.cos(th), np.sin(th))
                u, sk = -U + i * h, -S + k * h
                p0 = (sk * om[0] - u * om[1], sk * om[1] + u * om[0])
                cache[key] = ray_to_edge(self.mu, g.pixel_mm, p0, om)
            return cache[key]

        a_, u_, s_ = np.broadcast_arrays(np.asarray(angle), np.asarray(u_mm, dtype=np.float64),
                                         np.asarray(s_mm, dtype=np.float64))
        out = np.empty(a_.shape, dtype=np.float64)
        for idx in np.ndindex(a_.shape):
            fu = min(max((u_[idx] + U) / h, 0.0), nu - 1 - 1e-3)
            fs = min(max((s_[idx] + S) / h, 0.0), ns - 1 - 1e-3)
            i, k = int(np.floor(fu)), int(np.floor(fs))
            wu, ws = fu - i, fs - k
            a = int(a_[idx])
            lo = (1 - ws) * node(a, i, k) + ws * node(a, i, k + 1)
            hi = (1 - ws) * node(a, i + 1, k) + ws * node(a, i + 1, k + 1)
            out[idx] = (1 - wu) * lo + wu * hi
        return out

    def line_start(self):
        """Depth of the first line node (before the grid): the whole-line
        attenuation is ``line_attenuation`` there."""
        g = self.geom
        return -(0.5 * g.pixel_mm * np.hypot(g.nx, g.ny) + 0.5 * g.pixel_mm)

    def model(self, angle, u_mm, e_kev, primary=True, scatter=True):
        """p[j, q] of every event j and support pixel q (paper Eq. 2 with
        Eq. 4: pr(A_j|P) s_eff(P) summed over the primary path and every
        first-order in-plane scatter path that starts in pixel q).  The
        flags restrict the sum to the primary path or to the scatter paths."""
        angle = np.ascontiguousarray(angle, dtype=np.int32)
        u = np.ascontiguousarray(u_mm, dtype=np.float64)
        e = np.ascontiguousarray(e_kev, dtype=np.float64)
        n = len(angle)
        p = np.zeros((n, self.n_sup), dtype=np.float64)
        lib().orc_model(ctypes.byref(self.geom), _d(self.mu), _i(self.support), self.n_sup,
                        _i(self.scatter), len(self.scatter), _d(self.l_edge), _d(self.l_pair),
                        _i(angle), _d(u), _d(e), n, _d(p), int(primary) | (int(scatter) << 1))
        return p

    def model_binned(self, angle, pos_bin, e_bin, e_edges, primary=True, scatter=True):
        """p[r, q] for binned rows r = (angle, detector position bin, energy
        bin): the probability that an emission in support pixel q is detected
        at that angle with its position and energy in the bin, i.e. the event
        model of ``model`` integrated over the bin.  Position bins are the
        detector's (n_bins of bin_mm over the extent); energy bin k is
        [e_edges[k], e_edges[k + 1]]."""
        angle = np.ascontiguousarray(angle, dtype=np.int32)
        pb = np.ascontiguousarray(pos_bin, dtype=np.int32)
        eb = np.ascontiguousarray(e_bin, dtype=np.int32)
        edges = np.ascontiguousarray(e_edges, dtype=np.float64)
        n = len(angle)
        p = np.zeros((n, self.n_sup), dtype=np.float64)
        lib().orc_model_binned(ctypes.byref(self.geom), _d(self.mu), _i(self.support), self.n_sup,
                               _i(self.scatter), len(self.scatter), _d(self.l_edge),
                               _d(self.l_pair), _i(angle), _i(pb), _i(eb), n, _d(edges), _d(p),
                               int(primary) | (int(scatter) << 1))
        return p

    def sensitivity(self, n_subsets: int, primary=True, scatter=True):
        """s[i, q]: sum of s_eff over the paths from pixel q that reach the
        detector at angles of subset i (denominator of Eq. 7).  Subset i holds
        the angles a with a mod n_subsets == i (reading of 'based on the
        detector angle').  The flags restrict the sum to the primary path or
        to the first-order scatter paths."""
        s = np.zeros((n_subsets, self.n_sup), dtype=np.float64)
        lib().orc_sensitivity(ctypes.byref(self.geom), _d(self.mu), _i(self.support),
                              self.n_sup, _i(self.scatter), len(self.scatter),
                              _d(self.l_edge), _d(self.l_pair), int(n_subsets), _d(s),
                              int(primary) | (int(scatter) << 1))
        return s


# ---------------------------------------------------------------- EM

def subset_of(angle, n_subsets):
    """Subset index of each event: its detector angle modulo N_s."""
    return np.asarray(angle) % n_subsets


def initial_image(n_events, s_total, T=1.0):
    """Uniform image on the support with T sum_n s_n f_n = J (reading: the
    paper starts from a support found by a crude binned OSEM)."""
    return np.full(s_total.shape, n_events / (T * s_total.sum()), dtype=np.float64)


def osem_subiteration(p_sub, f, s_i, T=1.0, w=None):
    """One OS-LM-MLEM sub-iteration (Eqs. 7-8) on the rows of one subset.

    y_j = sum_n p_jn f_n; events with y_j = 0 contribute nothing;
    f_q <- f_q sum_j w_j p_jq / y_j / (T s^i_q), and f_q = 0 where s^i_q = 0.
    w_j = 1 for list-mode events; a binned row counts its n_j events."""
    y = p_sub @ f
    ok = y > 0
    wv = 1.0 if w is None else np.asarray(w, dtype=np.float64)[ok]
    b = p_sub[ok].T @ (wv / y[ok])
    out = np.zeros_like(f)
    pos = s_i > 0
    out[pos] = f[pos] * b[pos] / (T * s_i[pos])
    return out


def osem(p, angle, s_sub, n_iters, f0, T=1.0, weights=None):
    """N_g global iterations over N_s subsets in index order, always from the
    latest sub-iterate (reading of the iteration state eta of Eq. 9).
    ``weights``: per-row counts of binned rows (None: list-mode events).
    Returns the image after every global iteration."""
    n_subsets = s_sub.shape[0]
    sub = subset_of(angle, n_subsets)
    rows = [np.nonzero(sub == i)[0] for i in range(n_subsets)]
    f = np.array(f0, dtype=np.float64)
    hist = []
    for _ in range(n_iters):
        for i in range(n_subsets):
            w = None if weights is None else np.asarray(weights)[rows[i]]
            f = osem_subiteration(p[rows[i]], f, s_sub[i], T, w)
        hist.append(f.copy())
    return f, hist


def loglik(p, f, s_total, T=1.0, weights=None):
    """Eq. 3 without the data-only constant: sum_j w_j log(T y_j) - T sum s f
    (w_j = 1 for events, the count of a binned row)."""
    y = p @ f
    w = 1.0 if weights is None else np.asarray(weights, dtype=np.float64)
    return float(np.sum(w * np.log(T * y)) - T * np.dot(s_total, f))


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))
