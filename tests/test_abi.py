"""Host-side checks of the C ABI: the library loads, exports every symbol its header
declares, and rejects bad arguments before touching the GPU."""
import ctypes

import numpy as np
import pytest

from paper_1908_00041_gb300 import api


@pytest.fixture(scope="module")
def lib():
    from paper_1908_00041_gb300 import build
    build.build()
    return api.lib()


def test_exports_every_header_symbol(lib):
    syms = api.header_symbols()
    assert len(syms) >= 12
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_gl_grid_host(lib):
    for n in [1, 2, 17, 512, 1024]:
        x, w = api.favest_gl_grid(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        o = np.argsort(x)
        assert np.all(np.diff(x) < 0)
        assert np.max(np.abs(x[o] - xr)) < 1e-14
        assert np.max(np.abs(w[o] - wr)) < 1e-13 * max(1, n / 100)


def test_strerror(lib):
    assert api.favest_strerror(0) == "success"
    assert "invalid" in api.favest_strerror(api.FAVEST_EINVAL)
    assert api.favest_strerror(-99) == "unknown status"


def _create(L, batch, prec=0, io=0, x=None, w=None):
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    xp = x.ctypes.data_as(dp) if x is not None else None
    wp = w.ctypes.data_as(dp) if w is not None else None
    st = api.lib().favest_plan_create(L, batch, prec, io, xp, wp, ctypes.byref(h))
    return st, h.value


def test_plan_create_rejects_bad_arguments(lib):
    assert _create(0, 1)[0] == api.FAVEST_EINVAL
    assert _create(4096, 1)[0] == api.FAVEST_EINVAL
    assert _create(16, 0)[0] == api.FAVEST_EINVAL
    assert _create(16, 1, prec=7)[0] == api.FAVEST_EINVAL
    assert _create(16, 1, io=5)[0] == api.FAVEST_EINVAL
    x, w = api.favest_gl_grid(17)
    xa = x.copy()
    xa[0] += 1e-6                       # not symmetric
    assert _create(16, 1, x=xa, w=w)[0] == api.FAVEST_EINVAL
    wa = w.copy()
    wa[3] *= 1.01
    assert _create(16, 1, x=x, w=wa)[0] == api.FAVEST_EINVAL
    xb = x.copy()
    xb[0] = 1.0                         # pole not allowed
    xb[-1] = -1.0
    assert _create(16, 1, x=xb, w=w)[0] == api.FAVEST_EINVAL
    # out pointer NULL
    assert api.lib().favest_plan_create(16, 1, 0, 0, None, None, None) == api.FAVEST_EINVAL


def test_null_plan_calls(lib):
    L = api.lib()
    nul = ctypes.c_void_p(None)
    assert L.favest_fwd(nul, nul, nul, nul, nul, nul) == api.FAVEST_EINVAL
    assert L.favest_adj(nul, nul, nul, nul, nul, nul) == api.FAVEST_EINVAL
    assert L.favest_set_weights_unit(nul, 0) == api.FAVEST_EINVAL
    assert L.favest_status(nul, nul) == api.FAVEST_EINVAL
    L.favest_plan_destroy(nul)


def test_new_entry_points_reject_bad_arguments(lib):
    """Entry points of the real-field, Clebsch-Gordan and batch forms: NULL plans and
    invalid requests come back as status codes without touching a device."""
    L = api.lib()
    nul = ctypes.c_void_p(None)
    h = ctypes.c_void_p()
    assert L.favest_fwd_cart(nul, nul, nul, nul, nul) == api.FAVEST_EINVAL
    assert L.favest_adj_cart(nul, nul, nul, nul, nul) == api.FAVEST_EINVAL
    assert L.favest_fwd_ex(nul, nul, nul, nul, nul, 0, nul) == api.FAVEST_EINVAL
    assert L.favest_adj_ex(nul, nul, nul, nul, nul, 0, nul) == api.FAVEST_EINVAL
    assert L.favest_cg_plan_create(16, 1, None, None, None) == api.FAVEST_EINVAL
    assert L.favest_cg_plan_create(0, 1, None, None, ctypes.byref(h)) == api.FAVEST_EINVAL
    assert L.favest_cg_plan_create(16, 5000, None, None, ctypes.byref(h)) == api.FAVEST_EINVAL
    # real fields with the CG route, complex128 or real double with split precision
    assert _create(16, 1, prec=api.FAVEST_BF16X6, io=api.FAVEST_IO_C128)[0] == api.FAVEST_EUNSUPPORTED
    assert _create(16, 1, prec=api.FAVEST_BF16X6, io=api.FAVEST_IO_R64)[0] == api.FAVEST_EUNSUPPORTED
    Ls = (ctypes.c_int * 2)(16, 31)
    assert L.favest_batch_create(2, Ls, None, None, api.FAVEST_BF16X6, 9, 0, ctypes.byref(h)) == api.FAVEST_EINVAL
    # real planes must start on 16 bytes: float offsets multiple of 4
    off = (ctypes.c_longlong * 2)(0, 578)
    assert L.favest_batch_create(2, Ls, off, None, api.FAVEST_BF16X6, api.FAVEST_IO_R32, 0,
                                 ctypes.byref(h)) == api.FAVEST_EINVAL
    assert L.favest_kernel_work(nul, b"fft_fwd", None, None, None) == api.FAVEST_EINVAL


def test_cg_stability_rejects_bad_arguments(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    r = np.empty(4)

    def call(L, z, ratios=True):
        z = np.ascontiguousarray(z, dtype=np.float64)
        return api.lib().favest_cg_stability(L, len(z), z.ctypes.data_as(dp) if len(z) else None, None,
                                             r.ctypes.data_as(dp) if ratios else None, ctypes.c_void_p(0))
    ok = np.array([0.1, -0.5])
    assert call(0, ok) == api.FAVEST_EINVAL
    assert call(1024, ok) == api.FAVEST_EINVAL
    assert call(5, np.array([])) == api.FAVEST_EINVAL
    assert call(5, ok, ratios=False) == api.FAVEST_EINVAL
    for bad in (1.0, -1.0, 1.5, np.nan, np.inf):
        assert call(5, np.array([0.2, bad])) == api.FAVEST_EINVAL


def test_alloc_failure_hook_host_side(lib):
    """The allocation-failure hook's host logic (no device needed): arming resets the count,
    bad arguments are refused."""
    L = api.lib()
    assert L.favest_debug_fail_alloc(-2) == api.FAVEST_EINVAL
    assert L.favest_debug_fail_alloc(3) == api.FAVEST_OK
    assert L.favest_debug_alloc_count() == 0
    assert L.favest_debug_fail_alloc(-1) == api.FAVEST_OK
    assert L.favest_debug_alloc_count() == 0
