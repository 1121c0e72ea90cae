"""Thin ctypes binding of the favest C ABI (include/favest.h).

Every function here only marshals arguments (tensor pointers, sizes, streams) and
checks the returned status; all arithmetic runs in the CUDA library.  If the
library cannot be loaded the first call raises ``FavestError`` -- there is no
fallback path.
"""
import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

FAVEST_OK = 0
FAVEST_EINVAL = -1
FAVEST_ENOMEM = -2
FAVEST_ECUDA = -3
FAVEST_EUNSUPPORTED = -4
FAVEST_ETIMEOUT = -5
FAVEST_EDEVICE = -6
FAVEST_EINTERNAL = -7

FAVEST_FP64 = 0
FAVEST_BF16X6 = 1
FAVEST_IO_C128 = 0
FAVEST_IO_C64 = 1
FAVEST_IO_R32 = 2
FAVEST_IO_R64 = 3
FAVEST_FLAG_UNIT_WEIGHTS = 1
FAVEST_FLAG_WEIGHTED = 2
FAVEST_FLAG_REAL_TRANSPOSE = 4
FAVEST_FLAG_SHARE_LAMBDA = 8
FAVEST_BATCH_AUTOTUNE = 1
FAVEST_BATCH_GRAPH = 2

_lock = threading.Lock()
_lib = None


class FavestError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = "favest error %d" % status
        if _lib is not None:
            msg += " (%s)" % _lib.favest_strerror(status).decode()
        super().__init__(msg + (": " + what if what else ""))


def library_path():
    """The in-tree library, or the file named by FAVEST_LIBRARY (an alternative build
    of the same sources, e.g. one made with different compile flags)."""
    return os.environ.get("FAVEST_LIBRARY") or _build.LIB


def lib(build_if_missing=False):
    """Load libfavest.so (built in-tree by paper_1908_00041_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                if not build_if_missing:
                    raise FavestError(FAVEST_EUNSUPPORTED,
                                      "CUDA library %s is not built (run __graft_entry__.build())" % path)
                _build.build()
            L = ctypes.CDLL(path)
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
            L.favest_gl_grid.argtypes = [i, d, d]
            L.favest_plan_create.argtypes = [i, i, i, i, d, d, ctypes.POINTER(vp)]
            L.favest_fwd.argtypes = [vp, vp, vp, vp, vp, vp]
            L.favest_adj.argtypes = [vp, vp, vp, vp, vp, vp]
            L.favest_fwd_ex.argtypes = [vp, vp, vp, vp, vp, i, vp]
            L.favest_adj_ex.argtypes = [vp, vp, vp, vp, vp, i, vp]
            L.favest_set_weights_unit.argtypes = [vp, i]
            L.favest_plan_L.argtypes = [vp]
            L.favest_plan_batch.argtypes = [vp]
            L.favest_plan_precision.argtypes = [vp]
            L.favest_plan_workspace_bytes.argtypes = [vp]
            L.favest_plan_workspace_bytes.restype = ctypes.c_size_t
            L.favest_status.argtypes = [vp, vp]
            L.favest_plan_destroy.argtypes = [vp]
            L.favest_plan_destroy.restype = None
            L.favest_strerror.argtypes = [i]
            L.favest_strerror.restype = ctypes.c_char_p
            L.favest_launches_per_call.argtypes = [vp, i]
            L.favest_probe_peaks.argtypes = [d, d]
            L.favest_kernel_work.argtypes = [vp, ctypes.c_char_p, d, d, ctypes.POINTER(ctypes.c_int)]
            pi, pll = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)
            L.favest_plan_tune.argtypes = [vp, vp]
            L.favest_selftest_wait_timeout.argtypes = [vp, ctypes.c_uint, d]
            L.favest_plan_gen_shape.argtypes = [vp, pi, pi]
            L.favest_plan_gen_chains.argtypes = [vp]
            L.favest_plan_set_gen_shape.argtypes = [vp, i, i, i]
            L.favest_batch_create.argtypes = [i, pi, pll, pll, i, i, i, ctypes.POINTER(vp)]
            L.favest_fwd_batched.argtypes = [vp, vp, vp, vp, vp, vp]
            L.favest_adj_batched.argtypes = [vp, vp, vp, vp, vp, vp]
            L.favest_batch_ngroups.argtypes = [vp]
            L.favest_batch_group.argtypes = [vp, i, pi, pi, pi, pi]
            L.favest_batch_field_elems.argtypes = [vp]
            L.favest_batch_field_elems.restype = ctypes.c_longlong
            L.favest_batch_coef_elems.argtypes = [vp]
            L.favest_batch_coef_elems.restype = ctypes.c_longlong
            L.favest_batch_status.argtypes = [vp, vp]
            L.favest_batch_destroy.argtypes = [vp]
            L.favest_fwd_fp64_noalloc.argtypes = [i, i, vp, vp, vp, vp, vp]
            L.favest_noalloc_scratch_bytes.restype = ctypes.c_size_t
            L.favest_cg_plan_create.argtypes = [i, i, d, d, ctypes.POINTER(vp)]
            L.favest_cg_plan_create_ex.argtypes = [i, i, i, d, d, ctypes.POINTER(vp)]
            L.favest_fwd_cart.argtypes = [vp, vp, vp, vp, vp]
            L.favest_adj_cart.argtypes = [vp, vp, vp, vp, vp]
            L.favest_cg_stability.argtypes = [i, i, d, d, d, vp]
            L.favest_debug_fail_alloc.argtypes = [ctypes.c_longlong]
            L.favest_debug_alloc_count.restype = ctypes.c_longlong
            L.favest_debug_check_layout.argtypes = [i, i, i, i, i, i, ctypes.c_char_p, i]
            L.favest_scatter_create.argtypes = [i, i, i, d, d, ctypes.POINTER(vp)]
            L.favest_scatter_fwd.argtypes = [vp, vp, vp, vp, vp]
            L.favest_scatter_adj.argtypes = [vp, vp, vp, vp, vp]
            L.favest_scatter_npts.argtypes = [vp]
            L.favest_scatter_destroy.argtypes = [vp]
            L.favest_scatter_destroy.restype = None
            L.favest_profile_enable.argtypes = [vp, i]
            L.favest_profile_read.argtypes = [vp, i, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_longlong)]
            _lib = L
    return _lib


def header_symbols():
    """Function names declared in include/favest.h."""
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "include", "favest.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"\b(favest_[A-Za-z0-9_]+)\s*\(", txt)))


def _check(status, what=""):
    if status != FAVEST_OK:
        raise FavestError(status, what)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def debug_check_layout(L, batch, precision=FAVEST_BF16X6, io_type=FAVEST_IO_C64, gemm_n=0, poison=0):
    """Host-only bounds check of the index tables a plan of this shape would use
    (favest_debug_check_layout; no GPU needed): returns (status, message)."""
    buf = ctypes.create_string_buffer(256)
    st = lib().favest_debug_check_layout(int(L), int(batch), int(precision), int(io_type), int(gemm_n), int(poison),
                                         buf, len(buf))
    return st, buf.value.decode()


def favest_gl_grid(nlat):
    """Gauss-Legendre nodes (descending) and weights from the library (host)."""
    x = np.empty(nlat)
    w = np.empty(nlat)
    _check(lib().favest_gl_grid(nlat, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "favest_gl_grid")
    return x, w


def favest_plan_create(L, batch, precision=FAVEST_FP64, io_type=FAVEST_IO_C128,
                       cos_theta=None, w_lat=None):
    """Returns an opaque plan handle (int)."""
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    if cos_theta is not None:
        cos_theta = np.ascontiguousarray(cos_theta, dtype=np.float64)
        w_lat = np.ascontiguousarray(w_lat, dtype=np.float64)
        xp, wp = cos_theta.ctypes.data_as(dp), w_lat.ctypes.data_as(dp)
    else:
        xp = wp = None
    _check(lib().favest_plan_create(int(L), int(batch), int(precision), int(io_type), xp, wp,
                                    ctypes.byref(h)), "favest_plan_create")
    return h.value


def favest_fwd(plan, Tth, Tph, a, b, stream=None):
    _check(lib().favest_fwd(ctypes.c_void_p(plan), _ptr(Tth), _ptr(Tph), _ptr(a), _ptr(b),
                            _stream(stream)), "favest_fwd")


def favest_adj(plan, a, b, Tth, Tph, stream=None):
    _check(lib().favest_adj(ctypes.c_void_p(plan), _ptr(a), _ptr(b), _ptr(Tth), _ptr(Tph),
                            _stream(stream)), "favest_adj")


def favest_fwd_ex(plan, Tth, Tph, a, b, flags, stream=None):
    _check(lib().favest_fwd_ex(ctypes.c_void_p(plan), _ptr(Tth), _ptr(Tph), _ptr(a), _ptr(b), int(flags),
                               _stream(stream)), "favest_fwd_ex")


def favest_adj_ex(plan, a, b, Tth, Tph, flags, stream=None):
    _check(lib().favest_adj_ex(ctypes.c_void_p(plan), _ptr(a), _ptr(b), _ptr(Tth), _ptr(Tph), int(flags),
                               _stream(stream)), "favest_adj_ex")


def favest_set_weights_unit(plan, flag):
    _check(lib().favest_set_weights_unit(ctypes.c_void_p(plan), int(flag)), "favest_set_weights_unit")


def favest_status(plan, stream=None):
    return lib().favest_status(ctypes.c_void_p(plan), _stream(stream))


def favest_plan_destroy(plan):
    lib().favest_plan_destroy(ctypes.c_void_p(plan))


def favest_plan_workspace_bytes(plan):
    return lib().favest_plan_workspace_bytes(ctypes.c_void_p(plan))


def favest_launches_per_call(plan, adjoint=0):
    return lib().favest_launches_per_call(ctypes.c_void_p(plan), int(adjoint))


def favest_profile_enable(plan, enable):
    _check(lib().favest_profile_enable(ctypes.c_void_p(plan), int(enable)), "favest_profile_enable")


def favest_profile_read(plan, max_kernels=16):
    """{kernel name: (milliseconds, launches)} accumulated since the last read."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    ms = (ctypes.c_double * max_kernels)()
    cnt = (ctypes.c_longlong * max_kernels)()
    k = lib().favest_profile_read(ctypes.c_void_p(plan), max_kernels, names, ms, cnt)
    if k < 0:
        raise FavestError(k, "favest_profile_read")
    raw = names.raw
    out = {}
    for i in range(k):
        nm = raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
        out[nm] = (ms[i], cnt[i])
    return out


def favest_fwd_fp64_noalloc(L, batch, Tth, Tph, a, b, stream=None):
    """FP64 forward transform using only the library's static 32 MB device scratch
    (no device allocation); see include/favest.h.  Tth, Tph: contiguous complex128 CUDA
    tensors [batch, L+1, 2(L+1)]; a, b: [batch, L^2+2L], all on the current device (the
    C entry point sees raw pointers only, so shapes and types are checked here)."""
    import torch
    L, batch = int(L), int(batch)
    shapes = {"Tth": (batch, L + 1, 2 * (L + 1)), "Tph": (batch, L + 1, 2 * (L + 1)),
              "a": (batch, L * L + 2 * L), "b": (batch, L * L + 2 * L)}
    dev = torch.cuda.current_device()
    for name, t in (("Tth", Tth), ("Tph", Tph), ("a", a), ("b", b)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev
                and t.dtype == torch.complex128 and t.is_contiguous() and tuple(t.shape) == shapes[name]):
            raise ValueError("%s: expected a contiguous complex128 tensor of shape %s on cuda:%d, got %s"
                             % (name, shapes[name], dev, getattr(t, "device", type(t))))
    _check(lib().favest_fwd_fp64_noalloc(L, batch, _ptr(Tth), _ptr(Tph), _ptr(a), _ptr(b),
                                         _stream(stream)), "favest_fwd_fp64_noalloc")


def favest_noalloc_scratch_bytes():
    return lib().favest_noalloc_scratch_bytes()


def favest_probe_peaks():
    """(fp64_tflops, fp32_tflops) measured on the current device."""
    f64 = ctypes.c_double()
    f32 = ctypes.c_double()
    _check(lib().favest_probe_peaks(ctypes.byref(f64), ctypes.byref(f32)), "favest_probe_peaks")
    return f64.value, f32.value


def favest_cg_stability(L, cos_theta, stream=None, per_coef=False):
    """Stability ratios of the forward CG route (Sec. 5.5, eq. r_stable) at points with the
    given cos(theta) values (host array): (r_hat, kappa_hat, r_tilde, kappa_tilde), and with
    per_coef the 4 x (L^2+2L) per-coefficient extremes as well."""
    z = np.ascontiguousarray(np.asarray(cos_theta, dtype=np.float64).ravel())
    K = L * L + 2 * L
    r = np.empty(4)
    ext = np.empty((4, K)) if per_coef else None
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().favest_cg_stability(int(L), int(z.size), z.ctypes.data_as(dp),
                                     ext.ctypes.data_as(dp) if per_coef else None, r.ctypes.data_as(dp),
                                     _stream(stream)), "favest_cg_stability")
    return (tuple(float(v) for v in r), ext) if per_coef else tuple(float(v) for v in r)


def favest_strerror(status):
    return lib().favest_strerror(int(status)).decode()


class Plan:
    """Owning wrapper around a favest plan with tensor allocation helpers."""

    def __init__(self, L, batch=1, precision=FAVEST_FP64, io_type=FAVEST_IO_C128,
                 cos_theta=None, w_lat=None):
        import torch
        self.L, self.batch, self.precision, self.io_type = int(L), int(batch), precision, io_type
        self.nlat, self.nphi = L + 1, 2 * (L + 1)
        # real fields keep orders m >= 0 only: L(L+3)/2 coefficients per family
        self.real = io_type in (FAVEST_IO_R32, FAVEST_IO_R64)
        self.K = L * (L + 3) // 2 if self.real else L * L + 2 * L
        self.cdtype = torch.complex128 if io_type in (FAVEST_IO_C128, FAVEST_IO_R64) else torch.complex64
        self.fdtype = {FAVEST_IO_R32: torch.float32, FAVEST_IO_R64: torch.float64}.get(io_type, self.cdtype)
        self.handle = favest_plan_create(L, batch, precision, io_type, cos_theta, w_lat)
        self._unit = 0

    def close(self):
        if getattr(self, "handle", None):
            favest_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t, shape, name, dtype=None):
        dtype = dtype or self.cdtype
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError("%s: expected contiguous CUDA %s tensor of shape %s, got %s %s %s"
                             % (name, dtype, shape, t.device, t.dtype, tuple(t.shape)))

    def field_shape(self):
        return (self.batch, self.nlat, self.nphi)

    def coef_shape(self):
        return (self.batch, self.K)

    def set_unit_weights(self, flag):
        if flag != self._unit:
            favest_set_weights_unit(self.handle, flag)
            self._unit = flag

    def fwd(self, Tth, Tph, a=None, b=None, stream=None, unit_weights=False, real_transpose=False,
            share_lambda=False):
        import torch
        self._check_tensor(Tth, self.field_shape(), "Tth", self.fdtype)
        self._check_tensor(Tph, self.field_shape(), "Tph", self.fdtype)
        if a is None:
            a = torch.empty(self.coef_shape(), dtype=self.cdtype, device=Tth.device)
        if b is None:
            b = torch.empty(self.coef_shape(), dtype=self.cdtype, device=Tth.device)
        self._check_tensor(a, self.coef_shape(), "a")
        self._check_tensor(b, self.coef_shape(), "b")
        flags = (FAVEST_FLAG_UNIT_WEIGHTS if unit_weights else 0) | (FAVEST_FLAG_REAL_TRANSPOSE if real_transpose else 0)
        flags |= FAVEST_FLAG_SHARE_LAMBDA if share_lambda else 0
        favest_fwd_ex(self.handle, Tth, Tph, a, b, flags, stream)
        return a, b

    def adj(self, a, b, Tth=None, Tph=None, stream=None, weighted=False, real_transpose=False,
            share_lambda=False):
        import torch
        self._check_tensor(a, self.coef_shape(), "a")
        self._check_tensor(b, self.coef_shape(), "b")
        if Tth is None:
            Tth = torch.empty(self.field_shape(), dtype=self.fdtype, device=a.device)
        if Tph is None:
            Tph = torch.empty(self.field_shape(), dtype=self.fdtype, device=a.device)
        self._check_tensor(Tth, self.field_shape(), "Tth", self.fdtype)
        self._check_tensor(Tph, self.field_shape(), "Tph", self.fdtype)
        flags = (FAVEST_FLAG_WEIGHTED if weighted else 0) | (FAVEST_FLAG_REAL_TRANSPOSE if real_transpose else 0)
        flags |= FAVEST_FLAG_SHARE_LAMBDA if share_lambda else 0
        favest_adj_ex(self.handle, a, b, Tth, Tph, flags, stream)
        return Tth, Tph

    def status(self, stream=None):
        return favest_status(self.handle, stream)

    def workspace_bytes(self):
        return favest_plan_workspace_bytes(self.handle)

    def selftest_wait_timeout(self, poll_limit=1 << 14):
        """Run the failure-path self-test (see include/favest.h): returns (status, ms)."""
        ms = ctypes.c_double()
        st = lib().favest_selftest_wait_timeout(ctypes.c_void_p(self.handle), int(poll_limit), ctypes.byref(ms))
        return st, ms.value

    def tune(self, stream=None):
        """Pick the fastest generator block shape for this plan (split precision)."""
        _check(lib().favest_plan_tune(ctypes.c_void_p(self.handle), _stream(stream)), "favest_plan_tune")
        return self.gen_shape()

    def gen_shape(self):
        lt, mb = ctypes.c_int(), ctypes.c_int()
        _check(lib().favest_plan_gen_shape(ctypes.c_void_p(self.handle), ctypes.byref(lt), ctypes.byref(mb)),
               "favest_plan_gen_shape")
        return lt.value, mb.value

    def set_gen_shape(self, lt, mb, nj):
        """Apply a generator shape the tuner offers, without timing (see tune_cache)."""
        _check(lib().favest_plan_set_gen_shape(ctypes.c_void_p(self.handle), int(lt), int(mb), int(nj)),
               "favest_plan_set_gen_shape")

    def gen_chains(self):
        """Latitude recurrences per generator thread of the shape in use (1 or 2)."""
        n = lib().favest_plan_gen_chains(ctypes.c_void_p(self.handle))
        _check(n if n < 0 else 0, "favest_plan_gen_chains")
        return n

    def launches_per_call(self, adjoint=0):
        return favest_launches_per_call(self.handle, adjoint)

    def profile(self, enable=True):
        favest_profile_enable(self.handle, 1 if enable else 0)

    def profile_read(self):
        return favest_profile_read(self.handle)

    def kernel_work(self, name):
        """(algorithmic bytes, flops, pipe) of one launch of kernel `name` (0 = HBM,
        1 = FP64 pipe, 2 = tensor pipe, 3 = FP32 pipe)."""
        nb = ctypes.c_double()
        fl = ctypes.c_double()
        pipe = ctypes.c_int()
        _check(lib().favest_kernel_work(ctypes.c_void_p(self.handle), name.encode(), ctypes.byref(nb),
                                        ctypes.byref(fl), ctypes.byref(pipe)), "favest_kernel_work")
        return nb.value, fl.value, pipe.value


class CgPlan:
    """FP64 plan of the Clebsch-Gordan route (Thm. 1, Thm. 2): fields as Cartesian
    components, T [batch, 3, L+1, 2(L+1)] complex128, coefficients [batch, L^2+2L]
    complex128; with real=True real fields, T float64, and half-spectrum coefficients
    [batch, L(L+3)/2] complex128 (m >= 0)."""

    def __init__(self, L, batch=1, cos_theta=None, w_lat=None, real=False):
        import torch
        self.L, self.batch, self.real = int(L), int(batch), bool(real)
        self.nlat, self.nphi = L + 1, 2 * (L + 1)
        self.K = L * (L + 3) // 2 if self.real else L * L + 2 * L
        self.cdtype = torch.complex128
        self.fdtype = torch.float64 if self.real else torch.complex128
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        xp = wp = None
        if cos_theta is not None:
            cos_theta = np.ascontiguousarray(cos_theta, dtype=np.float64)
            w_lat = np.ascontiguousarray(w_lat, dtype=np.float64)
            xp, wp = cos_theta.ctypes.data_as(dp), w_lat.ctypes.data_as(dp)
        io = FAVEST_IO_R64 if self.real else FAVEST_IO_C128
        _check(lib().favest_cg_plan_create_ex(self.L, self.batch, io, xp, wp, ctypes.byref(h)),
               "favest_cg_plan_create_ex")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            favest_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_shape(self):
        return (self.batch, 3, self.nlat, self.nphi)

    def coef_shape(self):
        return (self.batch, self.K)

    def _check(self, t, shape, name, dtype=None):
        dtype = self.cdtype if dtype is None else dtype
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError("%s: expected contiguous CUDA %s tensor of shape %s" % (name, dtype, shape))

    def fwd(self, T, a=None, b=None, stream=None):
        import torch
        self._check(T, self.field_shape(), "T", self.fdtype)
        a = torch.empty(self.coef_shape(), dtype=self.cdtype, device=T.device) if a is None else a
        b = torch.empty(self.coef_shape(), dtype=self.cdtype, device=T.device) if b is None else b
        self._check(a, self.coef_shape(), "a")
        self._check(b, self.coef_shape(), "b")
        _check(lib().favest_fwd_cart(ctypes.c_void_p(self.handle), _ptr(T), _ptr(a), _ptr(b), _stream(stream)),
               "favest_fwd_cart")
        return a, b

    def adj(self, a, b, T=None, stream=None):
        import torch
        self._check(a, self.coef_shape(), "a")
        self._check(b, self.coef_shape(), "b")
        T = torch.empty(self.field_shape(), dtype=self.fdtype, device=a.device) if T is None else T
        self._check(T, self.field_shape(), "T", self.fdtype)
        _check(lib().favest_adj_cart(ctypes.c_void_p(self.handle), _ptr(a), _ptr(b), _ptr(T), _stream(stream)),
               "favest_adj_cart")
        return T

    def status(self, stream=None):
        return favest_status(self.handle, stream)

    def profile(self, enable=True):
        favest_profile_enable(self.handle, 1 if enable else 0)

    def profile_read(self):
        return favest_profile_read(self.handle)


class ScatterPlan:
    """Transforms at arbitrary points (the paper's FaVeST_fwd(T, L, X, w) / FaVeST_adj(a, b, X)):
    X host [npts, 3] unit vectors, w host [npts] weights (None: unit weights); fields as
    Cartesian components T [batch, npts, 3] complex128, coefficients [batch, L^2+2L]."""

    def __init__(self, L, X, w=None, batch=1):
        import torch
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.ndim != 2 or X.shape[1] != 3:
            raise ValueError("X: expected [npts, 3] points")
        self.L, self.batch, self.npts = int(L), int(batch), int(X.shape[0])
        self.K = L * L + 2 * L
        self.cdtype = torch.complex128
        dp = ctypes.POINTER(ctypes.c_double)
        wp = None
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float64).ravel()
            if w.size != self.npts:
                raise ValueError("w: expected %d weights" % self.npts)
            wp = w.ctypes.data_as(dp)
        h = ctypes.c_void_p()
        _check(lib().favest_scatter_create(self.L, self.batch, self.npts, X.ctypes.data_as(dp), wp, ctypes.byref(h)),
               "favest_scatter_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            lib().favest_scatter_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_shape(self):
        return (self.batch, self.npts, 3)

    def coef_shape(self):
        return (self.batch, self.K)

    def _check(self, t, shape, name):
        if not (t.is_cuda and t.dtype == self.cdtype and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError("%s: expected contiguous CUDA complex128 tensor of shape %s" % (name, shape))

    def fwd(self, T, a=None, b=None, stream=None):
        import torch
        self._check(T, self.field_shape(), "T")
        a = torch.empty(self.coef_shape(), dtype=self.cdtype, device=T.device) if a is None else a
        b = torch.empty(self.coef_shape(), dtype=self.cdtype, device=T.device) if b is None else b
        self._check(a, self.coef_shape(), "a")
        self._check(b, self.coef_shape(), "b")
        _check(lib().favest_scatter_fwd(ctypes.c_void_p(self.handle), _ptr(T), _ptr(a), _ptr(b), _stream(stream)),
               "favest_scatter_fwd")
        return a, b

    def adj(self, a, b, T=None, stream=None):
        import torch
        self._check(a, self.coef_shape(), "a")
        self._check(b, self.coef_shape(), "b")
        T = torch.empty(self.field_shape(), dtype=self.cdtype, device=a.device) if T is None else T
        self._check(T, self.field_shape(), "T")
        _check(lib().favest_scatter_adj(ctypes.c_void_p(self.handle), _ptr(a), _ptr(b), _ptr(T), _stream(stream)),
               "favest_scatter_adj")
        return T


class BatchPlan:
    """Ragged batch: fields of individual degrees Ls[i] packed back to back (see
    favest_batch_create).  Grid buffers are flat complex tensors of field_elems elements
    (one per component), coefficient buffers flat tensors of coef_elems elements."""

    def __init__(self, Ls, precision=FAVEST_BF16X6, io_type=FAVEST_IO_C64, field_off=None, coef_off=None,
                 autotune=False, graph=True):
        import torch
        self.Ls = [int(x) for x in Ls]
        self.precision, self.io_type = precision, io_type
        self.real = io_type in (FAVEST_IO_R32, FAVEST_IO_R64)
        self.cdtype = torch.complex128 if io_type in (FAVEST_IO_C128, FAVEST_IO_R64) else torch.complex64
        self.fdtype = {FAVEST_IO_R32: torch.float32, FAVEST_IO_R64: torch.float64}.get(io_type, self.cdtype)
        n = len(self.Ls)
        Larr = (ctypes.c_int * n)(*self.Ls)
        fo = (ctypes.c_longlong * n)(*field_off) if field_off is not None else None
        co = (ctypes.c_longlong * n)(*coef_off) if coef_off is not None else None
        flags = (FAVEST_BATCH_AUTOTUNE if autotune else 0) | (FAVEST_BATCH_GRAPH if graph else 0)
        h = ctypes.c_void_p()
        _check(lib().favest_batch_create(n, Larr, fo, co, precision, io_type, flags, ctypes.byref(h)),
               "favest_batch_create")
        self.handle = h.value
        self.field_elems = lib().favest_batch_field_elems(ctypes.c_void_p(self.handle))
        self.coef_elems = lib().favest_batch_coef_elems(ctypes.c_void_p(self.handle))
        self.field_off, self.coef_off = [], []
        f = c = 0
        align = {FAVEST_IO_R32: 4, FAVEST_IO_C128: 1}.get(io_type, 2)   # elements per 16 bytes
        for i, L in enumerate(self.Ls):
            self.field_off.append(field_off[i] if field_off is not None else f)
            self.coef_off.append(coef_off[i] if coef_off is not None else c)
            f += -(-(L + 1) * 2 * (L + 1) // align) * align
            c += self._ncoef(L)

    def _ncoef(self, L):
        return L * (L + 3) // 2 if self.real else L * L + 2 * L

    def close(self):
        if getattr(self, "handle", None):
            lib().favest_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self):
        out = []
        for g in range(lib().favest_batch_ngroups(ctypes.c_void_p(self.handle))):
            v = [ctypes.c_int() for _ in range(4)]
            _check(lib().favest_batch_group(ctypes.c_void_p(self.handle), g, *[ctypes.byref(x) for x in v]),
                   "favest_batch_group")
            out.append({"L": v[0].value, "fields": v[1].value, "gen_lt": v[2].value, "gen_mb": v[3].value})
        return out

    def field(self, buf, i):
        """View of field i's component plane in a flat grid buffer, [L+1, 2(L+1)]."""
        L = self.Ls[i]
        o = self.field_off[i]
        return buf[o:o + (L + 1) * 2 * (L + 1)].view(L + 1, 2 * (L + 1))

    def coef(self, buf, i):
        L = self.Ls[i]
        o = self.coef_off[i]
        return buf[o:o + self._ncoef(L)]

    def fwd(self, Tth, Tph, a=None, b=None, stream=None):
        import torch
        if a is None:
            a = torch.empty(self.coef_elems, dtype=self.cdtype, device=Tth.device)
        if b is None:
            b = torch.empty(self.coef_elems, dtype=self.cdtype, device=Tth.device)
        _check(lib().favest_fwd_batched(ctypes.c_void_p(self.handle), _ptr(Tth), _ptr(Tph), _ptr(a), _ptr(b),
                                        _stream(stream)), "favest_fwd_batched")
        return a, b

    def adj(self, a, b, Tth=None, Tph=None, stream=None):
        import torch
        if Tth is None:
            Tth = torch.empty(self.field_elems, dtype=self.fdtype, device=a.device)
        if Tph is None:
            Tph = torch.empty(self.field_elems, dtype=self.fdtype, device=a.device)
        _check(lib().favest_adj_batched(ctypes.c_void_p(self.handle), _ptr(a), _ptr(b), _ptr(Tth), _ptr(Tph),
                                        _stream(stream)), "favest_adj_batched")
        return Tth, Tph

    def status(self, stream=None):
        return lib().favest_batch_status(ctypes.c_void_p(self.handle), _stream(stream))
