"""Pins of the oracle's Clebsch-Gordan route (Thm. 1, Thm. 2): it must reproduce the
literal O1 transforms (Cartesian Y^div, Y^curl of eqs. Blm1, Blm2, vsh2) at arbitrary,
non-quadrature points -- the theorems are identities for any point set -- and the
separable theta/phi oracle O3 on a Gauss-Legendre grid."""
import numpy as np
import pytest

from oracle import cg_route


def _rand_points(n, rng):
    return np.arccos(rng.uniform(-0.97, 0.97, n)), rng.uniform(0, 2 * np.pi, n)


@pytest.mark.parametrize("L", [1, 2, 5, 8])
def test_thm1_equals_literal_forward(orc, L):
    rng = np.random.default_rng(40 + L)
    th, ph = _rand_points(60, rng)
    w = rng.uniform(0.1, 1.0, 60)
    T = rng.standard_normal((60, 3)) + 1j * rng.standard_normal((60, 3))   # any vectors
    a1, b1 = orc.fwd_literal(L, th, ph, w, T)
    a2, b2 = cg_route.fwd_cg(L, th, ph, w, T)
    sc = max(np.max(np.abs(a1)), np.max(np.abs(b1)))
    assert np.max(np.abs(a2 - a1)) < 1e-13 * sc
    assert np.max(np.abs(b2 - b1)) < 1e-13 * sc


@pytest.mark.parametrize("L", [1, 2, 5, 8])
def test_thm2_equals_literal_adjoint(orc, L):
    rng = np.random.default_rng(50 + L)
    th, ph = _rand_points(40, rng)
    K = L * L + 2 * L
    a = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    b = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    T1 = orc.adj_literal(L, a, b, th, ph)
    T2 = cg_route.adj_cg(L, a, b, th, ph)
    assert np.max(np.abs(T2 - T1)) < 1e-13 * np.max(np.abs(T1))


def test_cg_route_on_gl_grid_equals_separable(orc):
    """On the GL grid the CG route (Cartesian components) and O3 (theta/phi components)
    give the same coefficients, and the CG adjoint reproduces O3's field."""
    L = 7
    rng = np.random.default_rng(61)
    x, W, theta, phi = orc.grid(L)
    tt = rng.standard_normal((len(theta), len(phi))) + 1j * rng.standard_normal((len(theta), len(phi)))
    tp = rng.standard_normal((len(theta), len(phi))) + 1j * rng.standard_normal((len(theta), len(phi)))
    TH, PH = np.meshgrid(theta, phi, indexing="ij")
    Tc = orc.sph_to_cart(TH.ravel(), PH.ravel(), tt.ravel(), tp.ravel())
    w = np.repeat(W, len(phi)) * (2 * np.pi / len(phi))
    a1, b1 = orc.fwd_sep(L, x, W, tt, tp)
    a2, b2 = cg_route.fwd_cg(L, TH.ravel(), PH.ravel(), w, Tc)
    sc = max(np.max(np.abs(a1)), np.max(np.abs(b1)))
    assert np.max(np.abs(a2 - a1)) < 1e-12 * sc and np.max(np.abs(b2 - b1)) < 1e-12 * sc
    K = L * L + 2 * L
    ca = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    cb = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    rt, rp = orc.adj_sep(L, x, ca, cb, len(phi))
    Tref = orc.sph_to_cart(TH.ravel(), PH.ravel(), rt.ravel(), rp.ravel())
    Tcg = cg_route.adj_cg(L, ca, cb, TH.ravel(), PH.ravel())
    assert np.max(np.abs(Tcg - Tref)) < 1e-12 * np.max(np.abs(Tref))
