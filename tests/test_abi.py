"""The C ABI library loads on a machine without a GPU, exports every
function include/lmosem.h declares, and rejects bad problem statements on
the host before touching the device (CPU only)."""
import ctypes

import numpy as np
import pytest

import paper_2002_12471_gb300.lmosem as L
from paper_2002_12471_gb300 import synthetic as S


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return L.load()


def test_exports_every_declared_function(lib):
    declared = L.header_functions()
    assert len(declared) >= 15
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared) == set(L.SIGNATURES), set(declared) ^ set(L.SIGNATURES)


def test_status_strings(lib):
    assert lib.lmosem_status_string(0) == b"ok"
    assert lib.lmosem_status_string(1) == b"invalid argument"
    assert lib.lmosem_status_string(6) == b"called out of order"


def _call_create(mu, g, nx=None, pixel=4.0, k_sigma=0.0, support=None, **knobs):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    ny, nx0 = mu.shape
    obj = L.Object(nx if nx is not None else nx0, ny, pixel,
                   mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), support)
    geo = L.Geometry(g["n_angles"], g["angle0_rad"], g["n_bins"], g["bin_mm"], g["radius_mm"],
                     g["coll_fwhm0_mm"], g["coll_fwhm_slope"])
    en = L.Energy(g["e0_kev"], g["fwhm_frac_e0"], g["e_lo_kev"], g["e_hi_kev"])
    opt = L.Options(k_sigma, 0)
    for k, v in knobs.items():
        setattr(opt, k, v)
    h = ctypes.c_void_p()
    st = L.load().lmosem_create(ctypes.byref(obj), ctypes.byref(geo), ctypes.byref(en),
                                ctypes.byref(opt), None, ctypes.byref(h))
    return st, h.value


@pytest.mark.parametrize("bad", [
    dict(n_angles=0), dict(n_bins=0), dict(bin_mm=-1.0), dict(radius_mm=30.0),
    dict(coll_fwhm0_mm=0.0), dict(coll_fwhm_slope=-0.1), dict(e_lo_kev=180.0),
    dict(fwhm_frac_e0=0.0), dict(e0_kev=float("nan")),
])
def test_create_rejects_bad_geometry(lib, bad):
    ph = S.disk_phantom()
    g = S.geometry(32, 16, 8.0, 80.0)
    g.update(bad)
    st, h = _call_create(ph.mu, g, pixel=ph.pixel_mm)
    assert st == L.EINVAL and not h


def test_create_rejects_bad_object(lib):
    ph = S.disk_phantom()
    g = S.geometry(32, 16, 8.0, 80.0)
    assert _call_create(ph.mu, g, nx=0, pixel=ph.pixel_mm)[0] == L.EINVAL
    assert _call_create(ph.mu, g, pixel=0.0)[0] == L.EINVAL
    assert _call_create(np.zeros((16, 16)), g, pixel=ph.pixel_mm)[0] == L.EINVAL   # empty support
    neg = ph.mu.copy()
    neg[3, 3] = -0.01
    assert _call_create(neg, g, pixel=ph.pixel_mm)[0] == L.EINVAL
    nan = ph.mu.copy()
    nan[2, 2] = np.nan
    assert _call_create(nan, g, pixel=ph.pixel_mm)[0] == L.EINVAL
    assert _call_create(ph.mu, g, pixel=ph.pixel_mm, k_sigma=-1.0)[0] == L.EINVAL
    assert _call_create(ph.mu, g, pixel=ph.pixel_mm, e_sigma=25.0)[0] == L.EINVAL
    assert _call_create(ph.mu, g, pixel=ph.pixel_mm, e_sigma=float("nan"))[0] == L.EINVAL


def test_null_context_calls_fail_cleanly(lib):
    assert lib.lmosem_sensitivity(None, 4, None) == L.EINVAL
    assert lib.lmosem_iterate(None, 1, 1.0, None, None) == L.EINVAL
    assert lib.lmosem_build_model(None, None, None, None, 10, 1, 0) == L.EINVAL
    assert lib.lmosem_n_support(None) == 0
    assert lib.lmosem_model_bytes(None) == 0
    lib.lmosem_destroy(None)


def test_every_context_call_rejects_a_null_context(lib):
    """Every status-returning entry point that takes a context returns
    EINVAL for a null one, before touching the device."""
    import ctypes
    skip = {"lmosem_create", "lmosem_status_string", "lmosem_osem_subiter_noalloc",
            "lmosem_n_support", "lmosem_n_scatter"}   # counts, 0 for a null context
    seen = 0
    for name, (res, args) in L.SIGNATURES.items():
        if name in skip or res is not ctypes.c_int or not args or args[0] is not ctypes.c_void_p:
            continue
        vals = [None]
        for t in args[1:]:
            if t in (ctypes.c_double, ctypes.c_float):
                vals.append(0.0)
            elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64):
                vals.append(0)
            else:
                vals.append(None)
        assert getattr(lib, name)(*vals) == L.EINVAL, name
        seen += 1
    assert seen >= 20


def test_host_buffer_marshalling_checks_dtype_and_device():
    """The host-buffer call's marshalling passes contiguous CPU tensors and
    numpy arrays of the declared type and refuses anything else."""
    import torch
    p, keep = L._host(torch.arange(4, dtype=torch.int32), np.int32)
    assert p == keep.data_ptr()
    p, keep = L._host(np.arange(4, dtype=np.int64), np.int32)     # converted copy, kept alive
    assert keep.dtype == np.int32 and p == keep.ctypes.data
    for bad in (torch.zeros(4, dtype=torch.float32), torch.zeros(8, dtype=torch.int32)[::2]):
        with pytest.raises(ValueError):
            L._host(bad, np.int32)


def test_host_call_rejects_mismatched_event_arrays():
    """The host-buffer call checks the three event arrays' lengths before the
    library reads them (no context is needed to reach that check)."""
    with pytest.raises(ValueError):
        L.lmosem_reconstruct(None, np.zeros(4, np.int32), np.zeros(3, np.float32),
                             np.zeros(4, np.float32), 1, 1)


def test_device_calls_reject_mismatched_event_arrays():
    """Every wrapper that passes event arrays checks their common length (and
    the batch's last offset against it) before the library reads them."""
    a, u, e = np.zeros(5, np.int32), np.zeros(4, np.float32), np.zeros(5, np.float32)
    for call in (lambda: L.lmosem_build_model(None, a, u, e, 1),
                 lambda: L.lmosem_surrogate_samples(None, a, u, e, None, None),
                 lambda: L.lmosem_build_model_batch(None, a, u, e, [0, 5], 1),
                 lambda: L.lmosem_build_model_batch(None, a, e, e, [0, 6], 1)):
        with pytest.raises(ValueError):
            call()


@pytest.mark.parametrize("bad", [
    dict(profile=3), dict(pass_variant=5), dict(pass_variant=-1), dict(ring_rows=-1),
    dict(surrogate_kernel=3), dict(prefetch_groups=-2), dict(prefetch_groups=17),
])
def test_create_rejects_bad_tuning_options(lib, bad):
    """Out-of-range tuning knobs are refused before any device work."""
    ph = S.disk_phantom()
    g = S.geometry(32, 16, 8.0, 80.0)
    st, h = _call_create(ph.mu, g, pixel=ph.pixel_mm, **bad)
    assert st == L.EINVAL and not h
