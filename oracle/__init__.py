"""CPU oracle for FwdVSHT / AdjVSHT (FaVeST, arXiv 1908.00041).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library and never calls it.

The arithmetic lives in ``favest_oracle.c`` (plain C, FP64), compiled on first use
into ``oracle/_build/``.  This module only marshals numpy arrays.

Forms:
  * O1 literal (Sec. 3 eqs. Blm1, Blm2, vsh2, ninecoeff; Def. FwdVSHT eq. fwdvsht2;
    Def. AdjVSHT eq. SLvec): ``fwd_literal``, ``adj_literal``, ``vsh_point``,
    ``fwd_literal_grid_coefs``, ``adj_literal_grid_points``.
  * O3 separable (same sums regrouped on a Gauss-Legendre grid): ``fwd_sep``,
    ``adj_sep``.
  * Gauss-Legendre rule (Sec. 5.1): ``gl``.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "favest_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle's C source into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i = ctypes.c_int
            d = ctypes.c_double
            L.orc_gl.argtypes = [i, dp, dp]
            L.orc_lambda_col.argtypes = [i, i, d, d, dp]
            L.orc_sh_point.argtypes = [i, d, d, dp]
            L.orc_cg9.argtypes = [i, i, dp]
            L.orc_vsh_point.argtypes = [i, d, d, dp, dp]
            L.orc_fwd_literal.argtypes = [i, i, dp, dp, dp, dp, dp, dp]
            L.orc_adj_literal.argtypes = [i, dp, dp, i, dp, dp, dp]
            L.orc_fwd_literal_grid_coefs.argtypes = [i, i, i, dp, dp, dp, dp, i, ip, ip, dp, dp]
            L.orc_adj_literal_grid_points.argtypes = [i, i, i, dp, dp, dp, i, ip, ip, dp, dp, dp]
            L.orc_fwd_sep.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp]
            L.orc_adj_sep.argtypes = [i, i, i, dp, dp, dp, dp, dp]
            L.orc_fwd_sep_orders.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp, i, i]
            L.orc_adj_sep_orders.argtypes = [i, i, i, dp, dp, dp, dp, dp, i, i]
            L.orc_num_threads.restype = i
            L.orc_set_num_threads.argtypes = [i]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def ncoef(L):
    """Coefficients per family for degrees 1..L: L^2 + 2L (l-major, m = -l..l)."""
    return L * L + 2 * L


def cidx(l, m):
    """Position of (l, m) in a coefficient sequence: l^2 + l + m - 1."""
    return l * l + l + m - 1


def gl(n):
    """Gauss-Legendre nodes x_j = cos(theta_j) (descending) and weights (sum 2)."""
    x = np.empty(n)
    w = np.empty(n)
    lib().orc_gl(n, _d(x), _d(w))
    return x, w


def lambda_col(m, lmax, theta):
    """lambda_l^m(theta), l = m..lmax (normalised associated Legendre, CS phase)."""
    out = np.empty(lmax - m + 1)
    lib().orc_lambda_col(m, lmax, float(np.cos(theta)), float(np.sin(theta)), _d(out))
    return out


def lambda_col_x(m, lmax, cost, sint):
    out = np.empty(lmax - m + 1)
    lib().orc_lambda_col(m, lmax, float(cost), float(sint), _d(out))
    return out


def sh_point(lmax, theta, phi):
    """Scalar Y_lm(theta, phi), l = 0..lmax, index l^2 + l + m."""
    out = np.empty((lmax + 1) ** 2, dtype=np.complex128)
    lib().orc_sh_point(lmax, float(theta), float(phi), _d(out.view(np.float64)))
    return out


def cg9(l, m):
    """The nine Clebsch-Gordan closed forms of eq. ninecoeff (see favest_oracle.c)."""
    out = np.empty(9)
    lib().orc_cg9(l, m, _d(out))
    return out


def vsh_point(L, theta, phi):
    """Cartesian Y^div_lm, Y^curl_lm (K x 3 complex each) at one point (eq. vsh2)."""
    K = ncoef(L)
    yd = np.empty((K, 3), dtype=np.complex128)
    yc = np.empty((K, 3), dtype=np.complex128)
    lib().orc_vsh_point(L, float(theta), float(phi), _d(yd.view(np.float64)), _d(yc.view(np.float64)))
    return yd, yc


def fwd_literal(L, theta, phi, w, T):
    """O1 FwdVSHT at arbitrary points; T: npts x 3 complex Cartesian."""
    theta, phi, w = _f64(theta), _f64(phi), _f64(w)
    T = _c128(T)
    K = ncoef(L)
    a = np.empty(K, dtype=np.complex128)
    b = np.empty(K, dtype=np.complex128)
    lib().orc_fwd_literal(L, len(theta), _d(theta), _d(phi), _d(w), _d(T.view(np.float64)),
                          _d(a.view(np.float64)), _d(b.view(np.float64)))
    return a, b


def adj_literal(L, a, b, theta, phi):
    """O1 AdjVSHT at arbitrary points; returns npts x 3 complex Cartesian."""
    a, b = _c128(a), _c128(b)
    theta, phi = _f64(theta), _f64(phi)
    T = np.empty((len(theta), 3), dtype=np.complex128)
    lib().orc_adj_literal(L, _d(a.view(np.float64)), _d(b.view(np.float64)), len(theta),
                          _d(theta), _d(phi), _d(T.view(np.float64)))
    return T


def fwd_literal_grid_coefs(L, x, W, Tth, Tph, ells, ms):
    """O1 a_lm, b_lm for listed (l, m) on an nlat x nphi grid (sampled checks)."""
    Tth, Tph = _c128(Tth), _c128(Tph)
    nlat, nphi = Tth.shape
    x, W = _f64(x), _f64(W)
    ells = np.ascontiguousarray(ells, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    a = np.empty(len(ells), dtype=np.complex128)
    b = np.empty(len(ells), dtype=np.complex128)
    lib().orc_fwd_literal_grid_coefs(L, nlat, nphi, _d(x), _d(W), _d(Tth.view(np.float64)),
                                     _d(Tph.view(np.float64)), len(ells), _i(ells), _i(ms),
                                     _d(a.view(np.float64)), _d(b.view(np.float64)))
    return a, b


def adj_literal_grid_points(L, nlat, nphi, x, a, b, js, ks):
    """O1 T_theta, T_phi (and the normal component) at listed grid points (j, k)."""
    a, b = _c128(a), _c128(b)
    x = _f64(x)
    js = np.ascontiguousarray(js, dtype=np.int32)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    n = len(js)
    tt = np.empty(n, dtype=np.complex128)
    tp = np.empty(n, dtype=np.complex128)
    nr = np.empty(n, dtype=np.complex128)
    lib().orc_adj_literal_grid_points(L, nlat, nphi, _d(x), _d(a.view(np.float64)),
                                      _d(b.view(np.float64)), n, _i(js), _i(ks),
                                      _d(tt.view(np.float64)), _d(tp.view(np.float64)),
                                      _d(nr.view(np.float64)))
    return tt, tp, nr


def fwd_sep(L, x, W, Tth, Tph):
    """O3 full FwdVSHT on an nlat x nphi grid (exact per-ring DFT + Legendre sums)."""
    Tth, Tph = _c128(Tth), _c128(Tph)
    nlat, nphi = Tth.shape
    x, W = _f64(x), _f64(W)
    K = ncoef(L)
    a = np.empty(K, dtype=np.complex128)
    b = np.empty(K, dtype=np.complex128)
    lib().orc_fwd_sep(L, nlat, nphi, _d(x), _d(W), _d(Tth.view(np.float64)),
                      _d(Tph.view(np.float64)), _d(a.view(np.float64)), _d(b.view(np.float64)))
    return a, b


def adj_sep(L, x, a, b, nphi):
    """O3 full AdjVSHT onto an len(x) x nphi grid."""
    a, b = _c128(a), _c128(b)
    x = _f64(x)
    nlat = len(x)
    tt = np.empty((nlat, nphi), dtype=np.complex128)
    tp = np.empty((nlat, nphi), dtype=np.complex128)
    lib().orc_adj_sep(L, nlat, nphi, _d(x), _d(a.view(np.float64)), _d(b.view(np.float64)),
                      _d(tt.view(np.float64)), _d(tp.view(np.float64)))
    return tt, tp


def fwd_sep_orders(L, x, W, Tth, Tph, mstart, mstep):
    """O3 forward restricted to orders m = mstart-L, mstart-L+mstep, ... (others left 0)."""
    Tth, Tph = _c128(Tth), _c128(Tph)
    nlat, nphi = Tth.shape
    x, W = _f64(x), _f64(W)
    K = ncoef(L)
    a = np.zeros(K, dtype=np.complex128)
    b = np.zeros(K, dtype=np.complex128)
    lib().orc_fwd_sep_orders(L, nlat, nphi, _d(x), _d(W), _d(Tth.view(np.float64)),
                             _d(Tph.view(np.float64)), _d(a.view(np.float64)),
                             _d(b.view(np.float64)), int(mstart), int(mstep))
    return a, b


def adj_sep_orders(L, x, a, b, nphi, mstart, mstep):
    """O3 adjoint summing only the orders m = mstart-L, mstart-L+mstep, ..."""
    a, b = _c128(a), _c128(b)
    x = _f64(x)
    nlat = len(x)
    tt = np.empty((nlat, nphi), dtype=np.complex128)
    tp = np.empty((nlat, nphi), dtype=np.complex128)
    lib().orc_adj_sep_orders(L, nlat, nphi, _d(x), _d(a.view(np.float64)), _d(b.view(np.float64)),
                             _d(tt.view(np.float64)), _d(tp.view(np.float64)), int(mstart), int(mstep))
    return tt, tp


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    lib().orc_set_num_threads(int(n))


def grid(L):
    """The (L+1) x 2(L+1) Gauss-Legendre tensor grid: x_j, W_j, theta_j, phi_k."""
    nlat, nphi = L + 1, 2 * (L + 1)
    x, W = gl(nlat)
    theta = np.arccos(np.clip(x, -1.0, 1.0))
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    return x, W, theta, phi


def sph_to_cart(theta, phi, Tth, Tph):
    """Cartesian T = T_theta e_theta + T_phi e_phi at points (theta, phi)."""
    ct, st, cp, sp = np.cos(theta), np.sin(theta), np.cos(phi), np.sin(phi)
    return np.stack([Tth * ct * cp - Tph * sp, Tth * ct * sp + Tph * cp, -Tth * st], axis=-1)
