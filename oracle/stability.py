"""CPU oracle of the stability ratios of the forward Clebsch-Gordan route (Sec. 5.5,
eq. r_stable).

TEST INFRASTRUCTURE (like the rest of ``oracle/``): only the tests, ``smoke()`` and the
CPU legs of ``bench.py`` may use it; it shares no code with the CUDA library.

At a point x_k, Thm. 1 (eq. almblmviaFlm) writes the conjugated vector harmonics as a few
terms, each a coefficient times a conjugated scalar harmonic times a constant Cartesian
vector (the T^(1), T^(2), T^(3) weights of the theorem):

    Y^div_lm(x)^*  = xi1 Y*_{l-1,m-1} u_- + xi2 Y*_{l+1,m-1} u_- + xi3 Y*_{l-1,m+1} u_+
                   + xi4 Y*_{l+1,m+1} u_+ + xi5 Y*_{l-1,m} e_3 + xi6 Y*_{l+1,m} e_3,
    Y^curl_lm(x)^* = -i mu1 Y*_{l,m-1} u_- - i mu3 Y*_{l,m+1} u_+ - i mu2 Y*_{l,m} e_3,

with u_- = (-1, i, 0)/sqrt2, u_+ = (1, i, 0)/sqrt2, e_3 = (0, 0, 1), Y_{l',m'} = 0 unless
|m'| <= l', and the xi, mu values (eqs. xi_klm, mu_klm) as products of c_l, d_l
(eq. cl,dl,betal) and the Clebsch-Gordan closed forms of eq. ninecoeff.  Section 5.5 compares
the size of each sum with the printed sums of the sizes of its terms:

    Vhat_{l,m,k}   = sqrt2 (|xi1| |Y_{l-1,m-1}(x_k)| + ... + |xi6| |Y_{l+1,m}(x_k)|),
    Vtilde_{l,m,k} = sqrt2 (|mu1| |Y_{l,m-1}(x_k)| + |mu3| |Y_{l,m+1}(x_k)| + |mu2| |Y_{l,m}(x_k)|),
    rho_hat = |Y^div_lm(x_k)^*| / Vhat,   rho_tilde = |Y^curl_lm(x_k)^*| / Vtilde.

Readings (the printed formula leaves them open): the "absolute value of an individual term"
takes |xi| (Clebsch-Gordan values can be negative); the printed factor sqrt2 multiplies all
terms; a point where V vanishes has no ratio and is left out.  Printed this way the ratio
is at most 1/sqrt2 (triangle inequality, since |u_-| = |u_+| = 1).  Section 5.5 cites the
summation analysis of Higham, whose condition number of a sum is the reciprocal
(sum of |terms|) / |sum|, unbounded where the sum cancels; both are reported:
    r_hat   = max rho_hat,     kappa_hat   = max 1/rho_hat,
    r_tilde = max rho_tilde,   kappa_tilde = max 1/rho_tilde,
over l <= L, 1 <= |m| <= l (the range of eq. r_stable) and the points.
"""
import math

import numpy as np

from . import cg9, cidx, ncoef, sh_point

_R2 = 1.0 / math.sqrt(2.0)
_UM = np.array([-1.0, 1j, 0.0]) * _R2      # u_-
_UP = np.array([1.0, 1j, 0.0]) * _R2       # u_+
_E3 = np.array([0.0, 0.0, 1.0], dtype=complex)


def _c(l):
    return math.sqrt((l + 1.0) / (2.0 * l + 1.0))


def _d(l):
    return math.sqrt(l / (2.0 * l + 1.0))


def point_terms(L, theta, phi):
    """Sizes of the sums and printed sums of term sizes at the points (theta, phi):
    |Y^div*|, Vhat, |Y^curl*|, Vtilde, each npts x (L^2+2L) for l = 1..L, |m| <= l
    (coefficient order l^2 + l + m - 1)."""
    theta = np.atleast_1d(np.asarray(theta, dtype=float))
    phi = np.atleast_1d(np.asarray(phi, dtype=float))
    Y = np.stack([sh_point(L + 1, t, p) for t, p in zip(theta, phi)], axis=0)   # npts x (L+2)^2
    npts = len(theta)

    def ys(l, m):
        if l < 0 or abs(m) > l:
            return np.zeros(npts, dtype=complex)
        return Y[:, l * l + l + m]

    K = ncoef(L)
    out = [np.empty((npts, K)) for _ in range(4)]
    for l in range(1, L + 1):
        cl, dl = _c(l), _d(l)
        for m in range(-l, l + 1):
            g = cg9(l, m)
            div = [(cl * g[0], ys(l - 1, m - 1), _UM), (dl * g[1], ys(l + 1, m - 1), _UM),
                   (cl * g[4], ys(l - 1, m + 1), _UP), (dl * g[5], ys(l + 1, m + 1), _UP),
                   (cl * g[2], ys(l - 1, m), _E3), (dl * g[3], ys(l + 1, m), _E3)]
            curl = [(-1j * g[6], ys(l, m - 1), _UM), (-1j * g[7], ys(l, m + 1), _UP),
                    (-1j * g[8], ys(l, m), _E3)]
            for q, terms in enumerate((div, curl)):
                vec = sum(c * np.conj(y)[:, None] * u[None, :] for c, y, u in terms)   # npts x 3
                out[2 * q][:, cidx(l, m)] = np.sqrt(np.sum(np.abs(vec) ** 2, axis=1))
                out[2 * q + 1][:, cidx(l, m)] = math.sqrt(2.0) * sum(abs(c) * np.abs(y) for c, y, _ in terms)
    return tuple(out)


def point_ratios(L, theta, phi):
    """rho_hat, rho_tilde (npts x (L^2+2L)); NaN where V = 0."""
    sd, vd, sc, vc = point_terms(L, theta, phi)
    with np.errstate(invalid="ignore", divide="ignore"):
        rh = np.where(vd > 0, sd / np.where(vd > 0, vd, 1.0), np.nan)
        rt = np.where(vc > 0, sc / np.where(vc > 0, vc, 1.0), np.nan)
    return rh, rt


def coefficient_extremes(L, theta, phi):
    """Per coefficient (l, m): [max_k rho_hat, min_k rho_hat, max_k rho_tilde, min_k rho_tilde]
    as a 4 x (L^2+2L) array (points without a ratio skipped)."""
    rh, rt = point_ratios(L, theta, phi)
    return np.stack([np.nanmax(rh, axis=0), np.nanmin(rh, axis=0),
                     np.nanmax(rt, axis=0), np.nanmin(rt, axis=0)])


def ratios(L, theta, phi):
    """(r_hat, kappa_hat, r_tilde, kappa_tilde) over l <= L, 1 <= |m| <= l and the points."""
    ext = coefficient_extremes(L, theta, phi)
    sel = [cidx(l, m) for l in range(1, L + 1) for m in range(-l, l + 1) if m != 0]
    e = ext[:, sel]
    return (float(np.max(e[0])), float(1.0 / np.min(e[1])),
            float(np.max(e[2])), float(1.0 / np.min(e[3])))
