"""Pins of the oracle's stability ratios (Sec. 5.5, eq. r_stable) against facts that do not
come from the oracle's own construction: the size of the sum against the theta/phi closed
form |grad* Y_lm| / sqrt(l(l+1)) (finite differences of the scalar functions), the printed
sums of term sizes for every (l, m) with l <= 3 from sympy's Clebsch-Gordan values and scipy's
associated Legendre functions, a hand-derived closed form of rho_tilde at (1, 1), the
triangle and Cauchy-Schwarz bounds, independence of the longitude and symmetry in m."""
import math

import numpy as np
import pytest

from oracle import lambda_col, stability

R2 = math.sqrt(2.0)


def _points(n, seed, lo=-0.98, hi=0.98):
    rng = np.random.default_rng(seed)
    return np.arccos(rng.uniform(lo, hi, n)), rng.uniform(0.0, 2.0 * np.pi, n)


def test_sizes_equal_gradient_closed_form(orc):
    """|Y^div_lm| = |Y^curl_lm| = sqrt((d_theta lambda)^2 + m^2 lambda^2 / sin^2) / sqrt(l(l+1))."""
    L = 6
    th, ph = _points(12, 7)
    sd, _, sc, _ = stability.point_terms(L, th, ph)
    h = 1e-5
    for k, t in enumerate(th):
        for l in range(1, L + 1):
            for m in range(-l, l + 1):
                mu = abs(m)
                lam = lambda_col(mu, l, t)[-1]
                dlam = (lambda_col(mu, l, t + h)[-1] - lambda_col(mu, l, t - h)[-1]) / (2 * h)
                ref = math.sqrt(dlam ** 2 + (m * lam / math.sin(t)) ** 2) / math.sqrt(l * (l + 1))
                i = l * l + l + m - 1
                assert abs(sd[k, i] - ref) < 1e-8 * max(1.0, ref)
                assert abs(sc[k, i] - ref) < 1e-8 * max(1.0, ref)


def test_term_sums_at_l1_m1_from_sympy_and_scipy(orc):
    sympy_cg = pytest.importorskip("sympy.physics.quantum.cg")
    special = pytest.importorskip("scipy.special")

    def cg(l1, m1, q, l, m):          # <l1 m1; 1 q | l m>
        return float(sympy_cg.CG(l1, m1, 1, q, l, m).doit())

    def ymag(l, m, t):
        m = abs(m)
        nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
        return nrm * abs(special.lpmv(m, l, math.cos(t)))

    c1, d1 = math.sqrt(2.0 / 3.0), math.sqrt(1.0 / 3.0)
    th, ph = _points(9, 8)
    _, vd, _, vc = stability.point_terms(1, th, ph)
    i = 1 * 1 + 1 + 1 - 1
    for k, t in enumerate(th):
        # terms at (l-1, m-1) = (0, 0), (l+1, m-1) = (2, 0), (l+1, m+1) = (2, 2), (l+1, m) = (2, 1);
        # (l-1, m+1) = (0, 2) and (l-1, m) = (0, 1) do not exist
        vhat = R2 * (c1 * abs(cg(0, 0, 1, 1, 1)) * ymag(0, 0, t) + d1 * abs(cg(2, 0, 1, 1, 1)) * ymag(2, 0, t)
                     + d1 * abs(cg(2, 2, -1, 1, 1)) * ymag(2, 2, t) + d1 * abs(cg(2, 1, 0, 1, 1)) * ymag(2, 1, t))
        vtil = R2 * (abs(cg(1, 0, 1, 1, 1)) * ymag(1, 0, t) + abs(cg(1, 1, 0, 1, 1)) * ymag(1, 1, t))
        assert abs(vd[k, i] - vhat) < 1e-14
        assert abs(vc[k, i] - vtil) < 1e-14


def test_term_sums_for_all_l_up_to_3_from_sympy_and_scipy(orc):
    """Vhat and Vtilde written out from the printed formula with sympy's Clebsch-Gordan values
    (<l' m'; 1 q | l m>) and scipy's associated Legendre functions, every (l, m), l <= 3."""
    sympy_cg = pytest.importorskip("sympy.physics.quantum.cg")
    special = pytest.importorskip("scipy.special")

    def ymag(l, m, t):
        if l < 0 or abs(m) > l:
            return np.zeros_like(t)
        m = abs(m)
        nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
        return nrm * np.abs(special.lpmv(m, l, np.cos(t)))

    def cg(l1, m1, q, l, m):
        if l1 < 0 or abs(m1) > l1:
            return 0.0
        return float(sympy_cg.CG(l1, m1, 1, q, l, m).doit())

    L = 3
    th, ph = _points(7, 12)
    _, vd, _, vc = stability.point_terms(L, th, ph)
    for l in range(1, L + 1):
        cl, dl = math.sqrt((l + 1.0) / (2 * l + 1)), math.sqrt(l / (2.0 * l + 1))
        for m in range(-l, l + 1):
            i = l * l + l + m - 1
            div = [(cl, l - 1, m - 1, 1), (dl, l + 1, m - 1, 1), (cl, l - 1, m + 1, -1),
                   (dl, l + 1, m + 1, -1), (cl, l - 1, m, 0), (dl, l + 1, m, 0)]
            curl = [(1.0, l, m - 1, 1), (1.0, l, m + 1, -1), (1.0, l, m, 0)]
            vhat = R2 * sum(c * abs(cg(l1, m1, q, l, m)) * ymag(l1, m1, th) for c, l1, m1, q in div)
            vtil = R2 * sum(c * abs(cg(l1, m1, q, l, m)) * ymag(l1, m1, th) for c, l1, m1, q in curl)
            assert np.max(np.abs(vd[:, i] - vhat)) < 1e-14, (l, m)
            assert np.max(np.abs(vc[:, i] - vtil)) < 1e-14, (l, m)


def test_rho_tilde_closed_form_at_l1_m1(orc):
    """mu1 = <1 0; 1 1|1 1> = -1/sqrt2, mu2 = <1 1; 1 0|1 1> = 1/sqrt2, lambda_1^0 ~ cos,
    lambda_1^1 ~ sin/sqrt2: rho_tilde = sqrt(cos^2 + sin^2/2) / (sqrt2 (|cos| + sin/sqrt2))."""
    th, ph = _points(15, 9, -0.999, 0.999)
    _, rt = stability.point_ratios(1, th, ph)
    c, s = np.abs(np.cos(th)), np.sin(th)
    ref = np.sqrt(c ** 2 + s ** 2 / 2) / (R2 * (c + s / R2))
    assert np.max(np.abs(rt[:, 2] - ref)) < 1e-15 * 10
    assert np.max(np.abs(rt[:, 0] - ref)) < 1e-15 * 10      # m = -1


def test_bounds_phi_independence_and_m_symmetry(orc):
    L = 7
    th, ph = _points(40, 10, -0.999, 0.999)
    rh, rt = stability.point_ratios(L, th, ph)
    assert np.nanmax(rh) <= 1 / R2 * (1 + 1e-14)                 # triangle inequality
    assert np.nanmax(rt) <= 1 / R2 * (1 + 1e-14)
    assert np.nanmin(rt) >= 1 / math.sqrt(6) * (1 - 1e-14)         # Cauchy-Schwarz, three terms
    rh2, rt2 = stability.point_ratios(L, th, ph + 1.234)
    assert np.nanmax(np.abs(rh2 - rh)) < 1e-14
    assert np.nanmax(np.abs(rt2 - rt)) < 1e-14
    for l in range(1, L + 1):
        for m in range(1, l + 1):
            a, b = l * l + l + m - 1, l * l + l - m - 1
            assert np.max(np.abs(rh[:, a] - rh[:, b])) < 1e-14
            assert np.max(np.abs(rt[:, a] - rt[:, b])) < 1e-14


def test_summary_ratios(orc):
    th, ph = _points(300, 11, -1.0, 1.0)
    r_hat, k_hat, r_til, k_til = stability.ratios(5, th, ph)
    assert 0.5 < r_hat <= 1 / R2 * (1 + 1e-14) and 0.5 < r_til <= 1 / R2 * (1 + 1e-14)
    assert k_hat >= R2 and R2 <= k_til <= math.sqrt(6) * (1 + 1e-14)
    ext = stability.coefficient_extremes(5, th, ph)
    assert ext.shape == (4, 35)
    assert np.all(ext[1] <= ext[0]) and np.all(ext[3] <= ext[2])
