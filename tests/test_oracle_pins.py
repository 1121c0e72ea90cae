"""Pins for the CPU oracle: each test checks the oracle against something other than
itself -- library routines (sympy, scipy, mpmath, numpy), closed forms derived from
the paper's definitions, invariants the paper states, and exactness of the
Gauss-Legendre rule.  None of these touch the CUDA library.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import sph_harm_y

from helpers import read_field_a

RNG = np.random.default_rng(12345)


def cidx(l, m):
    return l * l + l + m - 1


def rand_points(n, rng=RNG):
    z = rng.uniform(-0.98, 0.98, n)
    return np.arccos(z), rng.uniform(0, 2 * np.pi, n)


# ---------------------------------------------------------------------------
# Gauss-Legendre rule (Sec. 5.1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 255])
def test_gl_matches_numpy(orc, n):
    x, w = orc.gl(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    order = np.argsort(x)
    assert np.all(np.diff(x) < 0), "nodes must be descending (theta ascending)"
    assert np.max(np.abs(x[order] - xr)) < 1e-14
    assert np.max(np.abs(w[order] - wr)) < 1e-13


@pytest.mark.parametrize("n", [8, 33, 512, 1024])
def test_gl_exactness_and_symmetry(orc, n):
    x, w = orc.gl(n)
    assert np.all(w > 0)
    assert np.max(np.abs(x + x[::-1])) < 1e-15
    assert np.max(np.abs(w - w[::-1])) < 1e-15
    # int_{-1}^{1} x^k dx = 2/(k+1) for even k, 0 for odd k; exact for k <= 2n-1.
    # Legendre moments are better conditioned: sum_j w_j P_k(x_j) = 2 delta_k0.
    for k in [0, 1, 2, 7, 2 * n - 2, 2 * n - 1]:
        if k > 2 * n - 1:
            continue
        pk = np.polynomial.legendre.legval(x, [0] * k + [1])
        ref = 2.0 if k == 0 else 0.0
        assert abs(np.dot(w, pk) - ref) < 1e-13 * max(1, math.sqrt(n))


# ---------------------------------------------------------------------------
# Clebsch-Gordan closed forms, eq. ninecoeff vs a library routine
# ---------------------------------------------------------------------------
def test_cg9_against_sympy(orc):
    from sympy.physics.wigner import clebsch_gordan
    for l in range(1, 7):
        for m in range(-l, l + 1):
            got = orc.cg9(l, m)
            # C^{l,m}_{j1,m1,1,q} = <j1 m1; 1 q | l m>
            spec = [(l - 1, m - 1, 1), (l + 1, m - 1, 1), (l - 1, m, 0), (l + 1, m, 0),
                    (l - 1, m + 1, -1), (l + 1, m + 1, -1), (l, m - 1, 1), (l, m + 1, -1),
                    (l, m, 0)]
            for k, (j1, m1, q) in enumerate(spec):
                if abs(m1) > j1:
                    ref = 0.0
                else:
                    ref = float(clebsch_gordan(j1, 1, l, m1, q, m))
                assert abs(got[k] - ref) < 1e-14, (l, m, k, got[k], ref)


# ---------------------------------------------------------------------------
# Scalar spherical harmonics (Sec. 3) vs scipy; Legendre values at large degree
# ---------------------------------------------------------------------------
def test_sh_matches_scipy(orc):
    th, ph = rand_points(6)
    for t, p in zip(th, ph):
        y = orc.sh_point(20, t, p)
        for l in range(21):
            for m in range(-l, l + 1):
                assert abs(y[l * l + l + m] - sph_harm_y(l, m, t, p)) < 1e-13


@pytest.mark.parametrize("l", [100, 511, 1023, 2250])
def test_unsold_scalar(orc, l):
    """sum_m |Y_lm|^2 = (2l+1)/(4 pi) at any point (addition theorem).

    Near a pole the sum is carried by lambda_l^0, whose sensitivity to the rounding of
    cos(theta) grows like l^2 (1 - x) ~ l: the bound is 1e-14 * l relative."""
    for t in [1e-3, 0.02, 0.7, math.pi / 2, 2.9]:
        s = 0.0
        for m in range(0, l + 1):
            v = orc.lambda_col(m, l, t)[-1]
            s += v * v * (1 if m == 0 else 2)
        ref = (2 * l + 1) / (4 * math.pi)
        assert abs(s - ref) < 1e-14 * l * ref


def test_lambda_extended_range_against_mpmath(orc):
    """Values whose recurrence passes far below the double range (lambda_m^m ~ 1e-400)
    but which are of normal size at the evaluated degree."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    m, st = 800, 0.3
    ct = math.sqrt(1 - st * st)
    col = orc.lambda_col_x(m, 3000, ct, st)
    for l in [2700, 2850, 3000]:
        x = mpmath.mpf(ct)
        p = mpmath.legenp(l, m, x, type=2)
        norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m) / mpmath.factorial(l + m))
        ref = float(norm * p)
        assert abs(ref) > 1e-6
        assert abs(col[l - m] - ref) < 1e-10 * abs(ref), (l, col[l - m], ref)
    # Condon-Shortley phase at odd order
    assert abs(float(mpmath.legenp(1, 1, 0.3, type=2)) + math.sqrt(1 - 0.09)) < 1e-15


# ---------------------------------------------------------------------------
# Vector spherical harmonics, literal CG form (O1, eqs. Blm1, Blm2, vsh2)
# ---------------------------------------------------------------------------
def _grad_Y(l, m, t, p, h=1e-4):
    """Surface gradient of scipy's Y_lm: 4th-order central difference in theta,
    d/dphi = i m exactly.  Returns (d_theta Y, (1/sin) d_phi Y)."""
    f = lambda tt: sph_harm_y(l, m, tt, p)
    dth = (8 * (f(t + h) - f(t - h)) - (f(t + 2 * h) - f(t - 2 * h))) / (12 * h)
    dph = 1j * m * sph_harm_y(l, m, t, p) / math.sin(t)
    return dth, dph


def _basis(t, p):
    et = np.array([math.cos(t) * math.cos(p), math.cos(t) * math.sin(p), -math.sin(t)])
    ep = np.array([-math.sin(p), math.cos(p), 0.0])
    xr = np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])
    return et, ep, xr


def test_vsh_tangent_and_closed_forms(orc):
    """Y^div = grad* Y / sqrt(l(l+1)), Y^curl = x cross grad* Y / sqrt(l(l+1)), both tangent."""
    L = 6
    th, ph = rand_points(8)
    for t, p in zip(th, ph):
        yd, yc = orc.vsh_point(L, t, p)
        et, ep, xr = _basis(t, p)
        for l in range(1, L + 1):
            for m in range(-l, l + 1):
                k = cidx(l, m)
                assert abs(np.dot(xr, yd[k])) < 1e-14
                assert abs(np.dot(xr, yc[k])) < 1e-14
                gt, gp = _grad_Y(l, m, t, p)
                s = 1 / math.sqrt(l * (l + 1))
                ref_d = s * (gt * et + gp * ep)
                ref_c = s * (gt * ep - gp * et)     # x cross e_theta = e_phi, x cross e_phi = -e_theta
                assert np.max(np.abs(yd[k] - ref_d)) < 1e-10, (l, m)
                assert np.max(np.abs(yc[k] - ref_c)) < 1e-10, (l, m)


@pytest.mark.parametrize("l", [1, 7, 40])
def test_unsold_vector(orc, l):
    """sum_m |Y^div_lm|^2 = sum_m |Y^curl_lm|^2 = (2l+1)/(4 pi)."""
    th, ph = rand_points(3)
    for t, p in zip(th, ph):
        yd, yc = orc.vsh_point(l, t, p)
        sl = slice(cidx(l, -l), cidx(l, l) + 1)
        ref = (2 * l + 1) / (4 * math.pi)
        assert abs(np.sum(np.abs(yd[sl]) ** 2) - ref) < 1e-12 * ref
        assert abs(np.sum(np.abs(yc[sl]) ** 2) - ref) < 1e-12 * ref


def _vsh_matrix(orc, L, theta, phi):
    """Columns Y^div_lm, Y^curl_lm at the points, rows (point, component)."""
    cols = []
    for t, p in zip(theta, phi):
        yd, yc = orc.vsh_point(L, t, p)
        cols.append(np.concatenate([yd, yc], axis=0))   # 2K x 3
    A = np.stack(cols, axis=0)                           # npts x 2K x 3
    return A.transpose(0, 2, 1).reshape(-1, A.shape[1])  # (npts*3) x 2K


def test_orthonormality_independent_quadrature(orc):
    """<Y, Y'> = delta on the sphere (Sec. 3), integrated with numpy's GL nodes in
    cos(theta) x a trapezoid rule in phi -- both exact far beyond degree 2L."""
    L = 4
    xr, wr = np.polynomial.legendre.leggauss(24)
    nphi = 48
    t = np.repeat(np.arccos(xr), nphi)
    p = np.tile(2 * np.pi * np.arange(nphi) / nphi, len(xr))
    w = np.repeat(wr, nphi) * (2 * np.pi / nphi)
    A = _vsh_matrix(orc, L, t, p)
    G = (A.conj() * np.repeat(w, 3)[:, None]).T @ A
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-13


def test_discrete_orthonormality_on_grid(orc):
    """A^H W A = I on the (L+1) x 2(L+1) GL grid (exact for degree <= 2L+1)."""
    L = 6
    x, W, theta, phi = orc.grid(L)
    t = np.repeat(theta, len(phi))
    p = np.tile(phi, len(theta))
    w = np.repeat(W, len(phi)) * (2 * np.pi / len(phi))
    A = _vsh_matrix(orc, L, t, p)
    G = (A.conj() * np.repeat(w, 3)[:, None]).T @ A
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-13


# ---------------------------------------------------------------------------
# Transforms: roundtrip, Parseval, adjoint identity, real symmetry, O1 vs O3
# ---------------------------------------------------------------------------
def _rand_coefs(L, rng, decay=1.0):
    K = L * L + 2 * L
    ell = np.concatenate([[l] * (2 * l + 1) for l in range(1, L + 1)])
    s = (ell + 1.0) ** (-decay)
    a = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) * s
    b = (rng.standard_normal(K) + 1j * rng.standard_normal(K)) * s
    return a, b


def _grid_pts(orc, L):
    x, W, theta, phi = orc.grid(L)
    t = np.repeat(theta, len(phi))
    p = np.tile(phi, len(theta))
    w = np.repeat(W, len(phi)) * (2 * np.pi / len(phi))
    return x, W, theta, phi, t, p, w


def test_roundtrip_parseval_literal(orc):
    L = 8
    rng = np.random.default_rng(7)
    a, b = _rand_coefs(L, rng)
    x, W, theta, phi, t, p, w = _grid_pts(orc, L)
    T = orc.adj_literal(L, a, b, t, p)
    # tangent
    xr = np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], -1)
    assert np.max(np.abs(np.sum(xr * T, -1))) < 1e-13
    a2, b2 = orc.fwd_literal(L, t, p, w, T)
    assert np.max(np.abs(a2 - a)) < 1e-13 and np.max(np.abs(b2 - b)) < 1e-13
    # Parseval / truncation identity of Sec. 4.3 on the exact rule
    lhs = np.sum(w * np.sum(np.abs(T) ** 2, -1))
    rhs = np.sum(np.abs(a) ** 2) + np.sum(np.abs(b) ** 2)
    assert abs(lhs - rhs) < 1e-13 * rhs


def test_adjoint_identity_and_real_symmetry(orc):
    L = 7
    rng = np.random.default_rng(8)
    x, W, theta, phi, t, p, w = _grid_pts(orc, L)
    # random tangent field (not band-limited)
    Tth = rng.standard_normal(len(t)) + 1j * rng.standard_normal(len(t))
    Tph = rng.standard_normal(len(t)) + 1j * rng.standard_normal(len(t))
    T = orc.sph_to_cart(t, p, Tth, Tph)
    a, b = orc.fwd_literal(L, t, p, w, T)
    c1, c2 = _rand_coefs(L, rng)
    S = orc.adj_literal(L, c1, c2, t, p)
    lhs = np.sum(np.conj(S) * (w[:, None] * T))
    rhs = np.vdot(c1, a) + np.vdot(c2, b)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # real fields: a_{l,-m} = (-1)^m conj(a_{l,m})
    Tr = orc.sph_to_cart(t, p, Tth.real, Tph.real)
    ar, br = orc.fwd_literal(L, t, p, w, Tr)
    for l in range(1, L + 1):
        for m in range(1, l + 1):
            sg = (-1) ** m
            assert abs(ar[cidx(l, -m)] - sg * np.conj(ar[cidx(l, m)])) < 1e-13
            assert abs(br[cidx(l, -m)] - sg * np.conj(br[cidx(l, m)])) < 1e-13


@pytest.mark.parametrize("L", [1, 2, 4, 9])
def test_separable_equals_literal(orc, L):
    """O3 (theta/phi closed form, per-ring exact DFT) equals O1 (literal CG form)."""
    rng = np.random.default_rng(100 + L)
    x, W, theta, phi, t, p, w = _grid_pts(orc, L)
    nlat, nphi = len(theta), len(phi)
    Tth = rng.standard_normal((nlat, nphi)) + 1j * rng.standard_normal((nlat, nphi))
    Tph = rng.standard_normal((nlat, nphi)) + 1j * rng.standard_normal((nlat, nphi))
    T = orc.sph_to_cart(t, p, Tth.ravel(), Tph.ravel())
    a1, b1 = orc.fwd_literal(L, t, p, w, T)
    a3, b3 = orc.fwd_sep(L, x, W, Tth, Tph)
    sc = max(np.max(np.abs(a1)), np.max(np.abs(b1)))
    assert np.max(np.abs(a1 - a3)) < 1e-13 * sc and np.max(np.abs(b1 - b3)) < 1e-13 * sc
    # per-coefficient literal form on the grid agrees as well
    ls = [l for l in range(1, L + 1) for m in range(-l, l + 1)]
    ms = [m for l in range(1, L + 1) for m in range(-l, l + 1)]
    a4, b4 = orc.fwd_literal_grid_coefs(L, x, W, Tth, Tph, ls, ms)
    assert np.max(np.abs(a1 - a4)) < 1e-13 * sc and np.max(np.abs(b1 - b4)) < 1e-13 * sc
    # adjoint
    c1, c2 = _rand_coefs(L, rng)
    S = orc.adj_literal(L, c1, c2, t, p)
    et = np.stack([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)], -1)
    ep = np.stack([-np.sin(p), np.cos(p), np.zeros_like(p)], -1)
    Sth = np.sum(S * et, -1).reshape(nlat, nphi)
    Sph = np.sum(S * ep, -1).reshape(nlat, nphi)
    tt, tp = orc.adj_sep(L, x, c1, c2, nphi)
    sc = np.max(np.abs(Sth))
    assert np.max(np.abs(tt - Sth)) < 1e-13 * sc and np.max(np.abs(tp - Sph)) < 1e-13 * sc
    js = np.repeat(np.arange(nlat), nphi)
    ks = np.tile(np.arange(nphi), nlat)
    t5, p5, nr = orc.adj_literal_grid_points(L, nlat, nphi, x, c1, c2, js, ks)
    assert np.max(np.abs(t5 - Sth.ravel())) < 1e-13 * sc
    assert np.max(np.abs(p5 - Sph.ravel())) < 1e-13 * sc
    assert np.max(np.abs(nr)) < 1e-13 * sc


def _single_mode_field(orc, L, l0, m0, curl):
    """grad* Y_{l0 m0} (curl=False) or x cross grad* Y_{l0 m0} (curl=True) on the grid,
    built from scipy's Y_lm with a 4th-order theta difference."""
    x, W, theta, phi = orc.grid(L)
    Tth = np.empty((len(theta), len(phi)), complex)
    Tph = np.empty_like(Tth)
    for j, t in enumerate(theta):
        for k, p in enumerate(phi):
            gt, gp = _grad_Y(l0, m0, t, p)
            if curl:
                Tth[j, k], Tph[j, k] = -gp, gt
            else:
                Tth[j, k], Tph[j, k] = gt, gp
    return x, W, Tth, Tph


@pytest.mark.parametrize("l0,m0", [(1, 0), (3, -2), (5, 5)])
def test_single_mode_fields(orc, l0, m0):
    """grad* Y_{l0 m0} -> a = sqrt(l0(l0+1)) delta, b = 0 (and the curl analogue)."""
    L = 6
    for curl in (False, True):
        x, W, Tth, Tph = _single_mode_field(orc, L, l0, m0, curl)
        a, b = orc.fwd_sep(L, x, W, Tth, Tph)
        hit, other = (b, a) if curl else (a, b)
        ref = np.zeros_like(hit)
        ref[cidx(l0, m0)] = math.sqrt(l0 * (l0 + 1))
        assert np.max(np.abs(hit - ref)) < 1e-9
        assert np.max(np.abs(other)) < 1e-9


def _read_field_a():
    return read_field_a()


def _field_a(orc, L):
    """Tangent Field A of Sec. 5.2 sampled on the GL grid, from scipy's Y_lm."""
    x, W, theta, phi = orc.grid(L)
    c1, c5 = -1 / math.sqrt(3), 8 * math.sqrt(2) / (3 * math.sqrt(385))
    Tth = np.zeros((len(theta), len(phi)), complex)
    Tph = np.zeros_like(Tth)
    for j, t in enumerate(theta):
        for k, p in enumerate(phi):
            st = 0
            for (c, l, m) in [(c1, 1, 0), (c5, 5, 4)]:      # stream function: L s = x cross grad* s
                gt, gp = _grad_Y(l, m, t, p)
                Tth[j, k] += -c * gp
                Tph[j, k] += c * gt
            for (c, l, m) in [(1 / 25, 4, 0), (1 / 25, 6, -3)]:   # potential: grad* v
                gt, gp = _grad_Y(l, m, t, p)
                Tth[j, k] += c * gt
                Tph[j, k] += c * gp
    return x, W, Tth, Tph


def test_field_a_closed_form_and_paper_bounds(orc):
    coefs, t1, t2 = _read_field_a()
    L = 10
    x, W, Tth, Tph = _field_a(orc, L)
    a, b = orc.fwd_sep(L, x, W, Tth, Tph)
    ref_a = np.zeros_like(a)
    ref_b = np.zeros_like(b)
    for fam, l, m, v in coefs:
        (ref_a if fam == "a" else ref_b)[cidx(l, m)] = v
    assert np.max(np.abs(a - ref_a)) < 1e-9
    assert np.max(np.abs(b - ref_b)) < 1e-9
    # reconstruction error (Table 1, GL row): ours must not exceed the paper's
    tt, tp = orc.adj_sep(L, x, a, b, Tth.shape[1])
    w = np.repeat(W, Tth.shape[1]) * (2 * np.pi / Tth.shape[1])
    num = np.sum(w * (np.abs(tt - Tth) ** 2 + np.abs(tp - Tph) ** 2).ravel())
    den = np.sum(w * (np.abs(Tth) ** 2 + np.abs(Tph) ** 2).ravel())
    assert math.sqrt(num / den) <= t1[10]
    # Table 2 style repeated transform at L = 40 on exact coefficients
    L2 = 40
    x2, W2, theta2, phi2 = orc.grid(L2)
    A = np.zeros(L2 * L2 + 2 * L2, complex)
    B = np.zeros_like(A)
    for fam, l, m, v in coefs:
        (A if fam == "a" else B)[cidx(l, m)] = v
    T1 = orc.adj_sep(L2, x2, A, B, len(phi2))
    A1, B1 = orc.fwd_sep(L2, x2, W2, *T1)
    T2 = orc.adj_sep(L2, x2, A1, B1, len(phi2))
    d_coef = max(np.max(np.abs(A1 - A)), np.max(np.abs(B1 - B)))
    d_T = max(np.max(np.abs(T2[0] - T1[0])), np.max(np.abs(T2[1] - T1[1])))
    assert d_coef <= t2[3] and d_T <= t2[2]


@pytest.mark.parametrize("L,mstep", [(4, 2), (9, 3), (20, 7), (31, 64)])
def test_strided_order_subsets_partition_the_transforms(orc, L, mstep):
    """The order subsets the timed CPU baseline runs (orders m = mstart - L + k mstep) partition
    the separable transforms: each forward subset fills exactly its own orders with the full
    transform's values and leaves every other coefficient zero, and the adjoint subsets sum to
    the full synthesis.  So a baseline timed on one subset and scaled by mstep counts the
    work of the whole transform."""
    rng = np.random.default_rng(300 + L)
    x, W, theta, phi = orc.grid(L)
    nlat, nphi = len(theta), len(phi)
    Tth = rng.standard_normal((nlat, nphi)) + 1j * rng.standard_normal((nlat, nphi))
    Tph = rng.standard_normal((nlat, nphi)) + 1j * rng.standard_normal((nlat, nphi))
    a, b = orc.fwd_sep(L, x, W, Tth, Tph)
    ms = np.concatenate([np.arange(-l, l + 1) for l in range(1, L + 1)])
    sa = np.zeros_like(a)
    sb = np.zeros_like(b)
    for m0 in range(min(mstep, 2 * L + 1)):
        pa, pb = orc.fwd_sep_orders(L, x, W, Tth, Tph, m0, mstep)
        mine = ((ms + L - m0) % mstep) == 0
        assert np.array_equal(pa[mine], a[mine]) and np.array_equal(pb[mine], b[mine])
        assert not np.any(pa[~mine]) and not np.any(pb[~mine])
        sa += pa
        sb += pb
    assert np.array_equal(sa, a) and np.array_equal(sb, b)
    c1, c2 = _rand_coefs(L, rng)
    tt, tp = orc.adj_sep(L, x, c1, c2, nphi)
    st = np.zeros_like(tt)
    sp = np.zeros_like(tp)
    for m0 in range(min(mstep, 2 * L + 1)):
        qt, qp = orc.adj_sep_orders(L, x, c1, c2, nphi, m0, mstep)
        st += qt
        sp += qp
    sc = max(np.max(np.abs(tt)), np.max(np.abs(tp)))
    assert np.max(np.abs(st - tt)) < 1e-13 * sc and np.max(np.abs(sp - tp)) < 1e-13 * sc
