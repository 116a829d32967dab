"""Python binding of the lmosem C ABI (``include/lmosem.h``).

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of ``liblmosem.so``.  Functions keep the C names; a non-OK status
raises :class:`LmosemError` with the library's message.  Device arrays are
passed as torch CUDA tensors (or raw integer addresses); torch supplies
device memory and streams and nothing else.  There is no CPU fallback: if
the shared library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblmosem.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENUMERIC, ESTATE, ENOTIMPL = range(8)
MODEL_FP32, MODEL_FP16_SCALED, MODEL_BF16_SCALED = 0, 1, 2
FORMATS = {"fp32": MODEL_FP32, "fp16": MODEL_FP16_SCALED, "bf16": MODEL_BF16_SCALED}


class LmosemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


class Object(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("pixel_mm", ctypes.c_double),
                ("h_mu_per_mm", ctypes.POINTER(ctypes.c_double)),
                ("h_support", ctypes.POINTER(ctypes.c_uint8))]


class Geometry(ctypes.Structure):
    _fields_ = [("n_angles", ctypes.c_int32), ("angle0_rad", ctypes.c_double),
                ("n_bins", ctypes.c_int32), ("bin_mm", ctypes.c_double),
                ("radius_mm", ctypes.c_double), ("coll_fwhm0_mm", ctypes.c_double),
                ("coll_fwhm_slope", ctypes.c_double)]


class Energy(ctypes.Structure):
    _fields_ = [("e0_kev", ctypes.c_double), ("fwhm_frac_e0", ctypes.c_double),
                ("e_lo_kev", ctypes.c_double), ("e_hi_kev", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("k_sigma", ctypes.c_float), ("table_budget_bytes", ctypes.c_int64),
                ("profile", ctypes.c_int32), ("wait_budget_cycles", ctypes.c_int64),
                ("pass_variant", ctypes.c_int32), ("ring_rows", ctypes.c_int32),
                ("ring_stages", ctypes.c_int32), ("surrogate_kernel", ctypes.c_int32),
                ("prefetch_groups", ctypes.c_int32), ("e_sigma", ctypes.c_float)]


KERNEL_CLASSES = ["tables", "sort", "wtable", "pathsum", "quantize", "sens", "pass", "update",
                  "other", "surrogate", "mlp"]
SURROGATE_PARAMS = 199967
SURROGATE_INPUTS = 8
SURROGATE_BASIS = 28
MODEL_SURROGATE_FP32 = 3
FORMATS["surrogate"] = MODEL_SURROGATE_FP32


class TrainOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("target_floor", ctypes.c_float), ("residual_fit", ctypes.c_int32),
                ("magnitude_power", ctypes.c_float)]


_vp = ctypes.c_void_p
_i32, _i64, _dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double

# name -> (restype, argtypes); mirrors include/lmosem.h
_GRID = {}   # context -> (ny, nx) of its grid, for the host-side outputs sized by it

SIGNATURES = {
    "lmosem_create": (ctypes.c_int, [ctypes.POINTER(Object), ctypes.POINTER(Geometry),
                                     ctypes.POINTER(Energy), ctypes.POINTER(Options), _vp,
                                     ctypes.POINTER(_vp)]),
    "lmosem_destroy": (None, [_vp]),
    "lmosem_last_error": (ctypes.c_char_p, [_vp]),
    "lmosem_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lmosem_n_support": (_i32, [_vp]),
    "lmosem_n_scatter": (_i32, [_vp]),
    "lmosem_support": (ctypes.c_int, [_vp, _vp]),
    "lmosem_sensitivity": (ctypes.c_int, [_vp, _i32, _vp]),
    "lmosem_build_model": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i32, ctypes.c_int]),
    "lmosem_init_image": (ctypes.c_int, [_vp, _dbl, _vp]),
    "lmosem_iterate": (ctypes.c_int, [_vp, _i32, _dbl, _vp, _vp]),
    "lmosem_loglik": (ctypes.c_int, [_vp, _dbl, _vp, _vp]),
    "lmosem_reconstruct": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i32, ctypes.c_int, _i32, _dbl,
                                          _vp, _vp]),
    "lmosem_model_rows": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "lmosem_model_bytes": (_i64, [_vp]),
    "lmosem_launch_count": (_i64, [_vp]),
    "lmosem_model_terms": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "lmosem_set_wait_budget": (ctypes.c_int, [_vp, _i64]),
    "lmosem_subset_totals": (ctypes.c_int, [_vp, _dbl, _vp, _vp]),
    "lmosem_profile_read": (ctypes.c_int, [_vp, _vp, _vp]),
    "lmosem_osem_subiter_noalloc": (ctypes.c_int, [_vp, _i64, _i32, _i64, _vp, _vp, _dbl, _vp]),
    "lmosem_build_model_batch": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_int]),
    "lmosem_build_model_binned": (ctypes.c_int, [_vp, _vp, _i32, _vp, _i32, ctypes.c_int]),
    "lmosem_init_image_batch": (ctypes.c_int, [_vp, _dbl, _vp]),
    "lmosem_iterate_batch": (ctypes.c_int, [_vp, _i32, _dbl, _vp]),
    "lmosem_autotune_batch": (ctypes.c_int, [_vp, _dbl, _vp, _vp]),
    "lmosem_set_batch_tiles": (ctypes.c_int, [_vp, _i32, _i32]),
    "lmosem_binned_support": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_int32, _vp, _vp]),
    "lmosem_surrogate_samples": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "lmosem_surrogate_train": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(TrainOpts), _vp, _vp]),
    "lmosem_surrogate_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "lmosem_surrogate_infer": (ctypes.c_int, [_vp, _vp, _vp, _i64, _vp]),
    "lmosem_surrogate_load": (ctypes.c_int, [_vp, _vp]),
    "lmosem_set_surrogate_check": (ctypes.c_int, [_vp, _dbl, _i32]),
    "lmosem_measure_ex2_rate": (ctypes.c_int, [_vp, _i32, _i32, _i64, _vp]),
    "lmosem_surrogate_check": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lmosem_set_surrogate_gate": (ctypes.c_int, [_vp, _dbl, _dbl]),
    "lmosem_surrogate_gate": (ctypes.c_int, [_vp, _vp, _vp]),
}

_lib = None


def load():
    """Load ``liblmosem.so`` (built in-tree by ``build.py``).  Raises when it
    is missing: the library has no other implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblmosem.so is not built; run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _status_name(st):
    try:
        return load().lmosem_status_string(st).decode()
    except Exception:  # noqa: BLE001 - message formatting only
        return "status"


def _ptr(x):
    """Device address of a torch tensor, or an integer address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(ctx, st):
    if st != OK:
        msg = load().lmosem_last_error(ctx).decode() if ctx else ""
        raise LmosemError(st, msg)


# ------------------------------------------------------------------ entry points

def lmosem_create(mu_per_mm, pixel_mm, geom: dict, support=None, k_sigma=0.0,
                  table_budget_bytes=0, stream=None, profile=False, wait_budget_cycles=0,
                  pass_variant=0, ring_rows=0, ring_stages=0, surrogate_kernel=0, prefetch_groups=0,
                  e_sigma=0.0):
    """Create a context.  ``mu_per_mm`` is an (ny, nx) host array at the
    photopeak, ``geom`` holds the scanner and energy fields of
    ``include/lmosem.h``; ``stream`` is a torch.cuda.Stream or a raw handle."""
    L = load()
    mu = np.ascontiguousarray(mu_per_mm, dtype=np.float64)
    ny, nx = mu.shape
    sup = None
    if support is not None:
        sup = np.ascontiguousarray(np.asarray(support).reshape(ny, nx) != 0, dtype=np.uint8)
    obj = Object(nx, ny, float(pixel_mm), mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 sup.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if sup is not None else None)
    g = Geometry(int(geom["n_angles"]), float(geom["angle0_rad"]), int(geom["n_bins"]),
                 float(geom["bin_mm"]), float(geom["radius_mm"]), float(geom["coll_fwhm0_mm"]),
                 float(geom["coll_fwhm_slope"]))
    e = Energy(float(geom["e0_kev"]), float(geom["fwhm_frac_e0"]), float(geom["e_lo_kev"]),
               float(geom["e_hi_kev"]))
    o = Options(float(k_sigma), int(table_budget_bytes), int(profile),
                int(wait_budget_cycles), int(pass_variant), int(ring_rows), int(ring_stages),
                int(surrogate_kernel), int(prefetch_groups), float(e_sigma))
    h = _vp()
    s = getattr(stream, "cuda_stream", stream)
    st = L.lmosem_create(ctypes.byref(obj), ctypes.byref(g), ctypes.byref(e), ctypes.byref(o),
                         s, ctypes.byref(h))
    if st != OK:
        raise LmosemError(st, "lmosem_create rejected the problem")
    _GRID[h.value] = (ny, nx)
    return h.value


def lmosem_destroy(ctx):
    _GRID.pop(ctx, None)
    load().lmosem_destroy(ctx)


def lmosem_n_support(ctx):
    return int(load().lmosem_n_support(ctx))


def lmosem_n_scatter(ctx):
    return int(load().lmosem_n_scatter(ctx))


def lmosem_support(ctx):
    out = np.zeros(lmosem_n_support(ctx), dtype=np.int32)
    _check(ctx, load().lmosem_support(ctx, out.ctypes.data))
    return out


def lmosem_sensitivity(ctx, n_subsets, d_sens=None):
    _check(ctx, load().lmosem_sensitivity(ctx, int(n_subsets), _ptr(d_sens)))


def _n_events(d_angle, d_u_mm, d_e_kev):
    """Common length of the three event arrays: the library reads that many
    entries of each, so a shorter one is refused here."""
    ns = [int(x.numel()) if hasattr(x, "numel") else int(len(x)) for x in (d_angle, d_u_mm, d_e_kev)]
    if ns[1] != ns[0] or ns[2] != ns[0]:
        raise ValueError("angle, position and energy arrays differ in length")
    return ns[0]


def lmosem_build_model(ctx, d_angle, d_u_mm, d_e_kev, n_subsets, fmt="fp32"):
    n = _n_events(d_angle, d_u_mm, d_e_kev)
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    _check(ctx, load().lmosem_build_model(ctx, _ptr(d_angle), _ptr(d_u_mm), _ptr(d_e_kev), n,
                                          int(n_subsets), f))


def lmosem_init_image(ctx, acq_time, d_f):
    _check(ctx, load().lmosem_init_image(ctx, float(acq_time), _ptr(d_f)))


def lmosem_iterate(ctx, n_iters, acq_time, d_f, d_loglik=None):
    _check(ctx, load().lmosem_iterate(ctx, int(n_iters), float(acq_time), _ptr(d_f),
                                      _ptr(d_loglik)))


def lmosem_subset_totals(ctx, acq_time, d_f, d_out):
    _check(ctx, load().lmosem_subset_totals(ctx, float(acq_time), _ptr(d_f), _ptr(d_out)))


def lmosem_loglik(ctx, acq_time, d_f, d_out):
    _check(ctx, load().lmosem_loglik(ctx, float(acq_time), _ptr(d_f), _ptr(d_out)))


def _host(x, dtype):
    """Host address of a contiguous CPU torch tensor or numpy array of the
    given numpy dtype (pinned torch tensors make the library's copies
    asynchronous)."""
    if hasattr(x, "data_ptr"):
        if (x.is_cuda or not x.is_contiguous()
                or str(x.dtype).replace("torch.", "") != np.dtype(dtype).name):
            raise ValueError("expected a contiguous host tensor of %s" % np.dtype(dtype).name)
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def lmosem_reconstruct(ctx, h_angle, h_u_mm, h_e_kev, n_subsets, n_iters, acq_time=1.0, fmt="fp32",
                       h_f=None, h_loglik=None):
    """Whole reconstruction from host event arrays; returns (image, loglik).
    ``h_f`` / ``h_loglik``: optional host outputs (N_nz float32, 1 float64),
    e.g. pinned torch tensors; numpy arrays are allocated otherwise."""
    a, ka = _host(h_angle, np.int32)
    u, ku = _host(h_u_mm, np.float32)
    e, ke = _host(h_e_kev, np.float32)
    n = _n_events(ka, ku, ke)
    if h_f is None:
        h_f = np.empty(lmosem_n_support(ctx), dtype=np.float32)
    if h_loglik is None:
        h_loglik = np.empty(1, dtype=np.float64)
    pf, kf = _host(h_f, np.float32)
    pl, kl = _host(h_loglik, np.float64)
    if len(kf) < lmosem_n_support(ctx) or len(kl) < 1:
        raise ValueError("output buffers too small")
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    _check(ctx, load().lmosem_reconstruct(ctx, a, u, e, n, int(n_subsets), f, int(n_iters),
                                          float(acq_time), pf, pl))
    return kf, kl


def lmosem_model_rows(ctx, d_event_ids, d_out):
    n = int(d_event_ids.numel())
    _check(ctx, load().lmosem_model_rows(ctx, _ptr(d_event_ids), n, _ptr(d_out)))


def lmosem_model_bytes(ctx):
    return int(load().lmosem_model_bytes(ctx))


def lmosem_launch_count(ctx):
    return int(load().lmosem_launch_count(ctx))


def lmosem_model_terms(ctx):
    """Path terms the path-sum kernels formed in the last exact model build."""
    n = ctypes.c_int64(0)
    _check(ctx, load().lmosem_model_terms(ctx, ctypes.byref(n)))
    return int(n.value)


def lmosem_set_wait_budget(ctx, cycles):
    _check(ctx, load().lmosem_set_wait_budget(ctx, int(cycles)))


def lmosem_profile_read(ctx):
    """{kernel class: (device ms, launches)} since the last read."""
    ms = np.zeros(len(KERNEL_CLASSES), dtype=np.float64)
    n = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    _check(ctx, load().lmosem_profile_read(ctx, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


def lmosem_build_model_binned(ctx, d_counts, e_edges, n_subsets, fmt="fp32"):
    """Binned form: d_counts is a device float32 tensor [n_angles, n_bins,
    n_ebins] of photon counts, e_edges the n_ebins + 1 energy bin edges."""
    edges = np.ascontiguousarray(e_edges, dtype=np.float64)
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    _check(ctx, load().lmosem_build_model_binned(ctx, _ptr(d_counts), len(edges) - 1, edges.ctypes.data,
                                                 int(n_subsets), f))


def lmosem_build_model_batch(ctx, d_angle, d_u_mm, d_e_kev, event_offsets, n_subsets, fmt="fp32"):
    off = np.ascontiguousarray(event_offsets, dtype=np.int64)
    if len(off) and off[-1] > _n_events(d_angle, d_u_mm, d_e_kev):
        raise ValueError("the last event offset lies beyond the event arrays")
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    _check(ctx, load().lmosem_build_model_batch(ctx, _ptr(d_angle), _ptr(d_u_mm), _ptr(d_e_kev),
                                                off.ctypes.data, len(off) - 1, int(n_subsets), f))


def lmosem_init_image_batch(ctx, acq_time, d_f):
    _check(ctx, load().lmosem_init_image_batch(ctx, float(acq_time), _ptr(d_f)))


def lmosem_iterate_batch(ctx, n_iters, acq_time, d_f):
    _check(ctx, load().lmosem_iterate_batch(ctx, int(n_iters), float(acq_time), _ptr(d_f)))


def lmosem_autotune_batch(ctx, acq_time, d_f):
    """Returns the chosen (chunk_rows, ctas_per_sm)."""
    out = np.zeros(2, dtype=np.int32)
    _check(ctx, load().lmosem_autotune_batch(ctx, float(acq_time), _ptr(d_f), out.ctypes.data))
    return int(out[0]), int(out[1])


def lmosem_set_batch_tiles(ctx, chunk_rows, ctas_per_sm):
    _check(ctx, load().lmosem_set_batch_tiles(ctx, int(chunk_rows), int(ctas_per_sm)))


def lmosem_binned_support(ctx, d_angle, d_u_mm, d_e_kev, n_subsets=4, n_iters=3, threshold=0.15, dilate=0,
                          d_image=None):
    """Support mask (ny * nx uint8, host) from the crude binned OSEM.  The
    defaults cover every pixel of the DaT-like phantoms' activity (at 3, 6
    and 10 iterations) and none of the air around them."""
    n = _n_events(d_angle, d_u_mm, d_e_kev)
    L = load()
    ny, nx = _GRID[ctx]
    mask = np.zeros(ny * nx, dtype=np.uint8)
    _check(ctx, L.lmosem_binned_support(ctx, _ptr(d_angle), _ptr(d_u_mm), _ptr(d_e_kev), n, int(n_subsets),
                                        int(n_iters), float(threshold), int(dilate), mask.ctypes.data,
                                        _ptr(d_image) if d_image is not None else None))
    return mask


def lmosem_surrogate_samples(ctx, d_angle, d_u_mm, d_e_kev, d_features, d_log_scatter, d_rel_log=None):
    n = _n_events(d_angle, d_u_mm, d_e_kev)
    _check(ctx, load().lmosem_surrogate_samples(ctx, _ptr(d_angle), _ptr(d_u_mm), _ptr(d_e_kev), n,
                                                _ptr(d_features), _ptr(d_log_scatter),
                                                _ptr(d_rel_log) if d_rel_log is not None else None))


def lmosem_surrogate_train(ctx, d_features, d_targets, d_weights, steps=2000, batch=4096, lr=1e-3,
                           seed=1, target_floor=0.0, residual_fit=False, d_rel_log=None, magnitude_power=0.0):
    """Trains in place; returns the per-step minibatch loss curve."""
    n = int(d_targets.numel())
    curve = np.zeros(int(steps), dtype=np.float64)
    o = TrainOpts(int(steps), int(batch), float(lr), int(seed), float(target_floor), int(bool(residual_fit)),
                  float(magnitude_power))
    _check(ctx, load().lmosem_surrogate_train(ctx, _ptr(d_features), _ptr(d_targets),
                                              _ptr(d_rel_log) if d_rel_log is not None else None, n,
                                              ctypes.byref(o), _ptr(d_weights), curve.ctypes.data))
    return curve


def lmosem_surrogate_grad(ctx, d_weights, d_features, d_targets, d_grad):
    loss = ctypes.c_double()
    n = int(d_targets.numel())
    _check(ctx, load().lmosem_surrogate_grad(ctx, _ptr(d_weights), _ptr(d_features), _ptr(d_targets), n,
                                             _ptr(d_grad), ctypes.byref(loss)))
    return loss.value


def lmosem_surrogate_infer(ctx, d_weights, d_features, d_out):
    n = int(d_out.numel())
    _check(ctx, load().lmosem_surrogate_infer(ctx, _ptr(d_weights), _ptr(d_features), n, _ptr(d_out)))


def lmosem_surrogate_load(ctx, d_weights):
    _check(ctx, load().lmosem_surrogate_load(ctx, _ptr(d_weights)))


def lmosem_set_surrogate_check(ctx, tol=1e-2, n_check_rows=0):
    """Tolerance (relative L2 of sampled rows) above which a surrogate build
    is replaced by the exact path sum (0: measure only), and the sampled row
    count (0: 512)."""
    _check(ctx, load().lmosem_set_surrogate_check(ctx, float(tol), int(n_check_rows)))


def lmosem_surrogate_check(ctx):
    """(rel_err, row_max, exact) of the exact check of the current surrogate
    model: relative L2 error of the sampled rows, largest per-row error, and
    whether the model was rebuilt with the exact path sum."""
    err, mx, ex = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(ctx, load().lmosem_surrogate_check(ctx, ctypes.byref(err), ctypes.byref(mx), ctypes.byref(ex)))
    return err.value, mx.value, bool(ex.value)


def lmosem_set_surrogate_gate(ctx, row_tol=1e-2, bin_kev=0.0):
    """Energy gate of the surrogate form (0: off): rows of the energy bins
    whose sampled mean row error exceeds row_tol, and of every lower bin,
    are rebuilt with the exact path sum (bin_kev = 0: 5 keV bins)."""
    _check(ctx, load().lmosem_set_surrogate_gate(ctx, float(row_tol), float(bin_kev)))


def lmosem_surrogate_gate(ctx):
    """(e_cut_kev, frac_exact) of the current surrogate-form model: rows
    with E below e_cut_kev hold the exact path sum, a fraction frac_exact of
    all rows."""
    cut, frac = ctypes.c_double(), ctypes.c_double()
    _check(ctx, load().lmosem_surrogate_gate(ctx, ctypes.byref(cut), ctypes.byref(frac)))
    return cut.value, frac.value


def surrogate_init(seed=0, layers=(SURROGATE_INPUTS, 256, 256, 256, 256, 1)):
    """Initial surrogate weights as a blob: He-normal weights (standard
    deviation sqrt(2 / fan_in)), zero biases, output standardisation (0, 1);
    training sets the standardisation from its targets."""
    rng = np.random.default_rng(seed)
    params = [[rng.standard_normal((fo, fi)) * np.sqrt(2.0 / fi), np.zeros(fo)]
              for fi, fo in zip(layers[:-1], layers[1:])]
    return pack_surrogate(params)


def pack_surrogate(params, mu=0.0, sigma=1.0, baseline=None):
    """Flatten [[W, b], ...] (the oracle's layout) into the library's blob;
    the baseline coefficients default to zero (the network alone)."""
    parts = [np.asarray(a, dtype=np.float64).ravel() for layer in params for a in layer]
    base = np.zeros(SURROGATE_BASIS) if baseline is None else np.asarray(baseline, dtype=np.float64)
    blob = np.concatenate(parts + [base, np.array([mu, sigma])]).astype(np.float32)
    assert blob.size == SURROGATE_PARAMS, blob.size
    return blob


def unpack_surrogate(blob, layers=(SURROGATE_INPUTS, 256, 256, 256, 256, 1)):
    blob = np.asarray(blob, dtype=np.float64)
    params, k = [], 0
    for fi, fo in zip(layers[:-1], layers[1:]):
        W = blob[k:k + fo * fi].reshape(fo, fi)
        k += fo * fi
        b = blob[k:k + fo]
        k += fo
        params.append([W, b])
    k += SURROGATE_BASIS  # the baseline coefficients
    return params, float(blob[k]), float(blob[k + 1])


def lmosem_osem_subiter_noalloc(d_rows, n_support, d_f, d_sens_i, acq_time, stream=None):
    """One sub-iteration on caller-provided FP32 rows (a 2-D tensor, row
    stride = its second dimension) without any device allocation; for
    callers that cannot allocate device memory."""
    n_rows, ld = int(d_rows.shape[0]), int(d_rows.stride(0))
    s = getattr(stream, "cuda_stream", stream)
    st = load().lmosem_osem_subiter_noalloc(_ptr(d_rows), n_rows, int(n_support), ld, _ptr(d_f),
                                            _ptr(d_sens_i), float(acq_time), s)
    if st != OK:
        raise LmosemError(st, "lmosem_osem_subiter_noalloc rejected the call")


def header_functions(header_path=None):
    """Names of the functions declared in include/lmosem.h."""
    import re
    if header_path is None:
        header_path = os.path.join(os.path.dirname(_HERE), "include", "lmosem.h")
    txt = open(header_path).read()
    return sorted(set(re.findall(r"\b(lmosem_[a-z0-9_]+)\s*\(", txt)))


def lmosem_measure_ex2_rate(stream=None, ctas_per_sm=4, threads=512, iters=1 << 16):
    """ex2.approx.ftz.f32 evaluations per second on the current device."""
    out = ctypes.c_double()
    s = getattr(stream, "cuda_stream", stream)
    st = load().lmosem_measure_ex2_rate(s, int(ctas_per_sm), int(threads), int(iters), ctypes.byref(out))
    if st != OK:
        raise LmosemError(st, "lmosem_measure_ex2_rate failed")
    return out.value
