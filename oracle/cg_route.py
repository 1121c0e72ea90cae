"""CPU oracle of the paper's Clebsch-Gordan route (Sec. 4, Thm. 1 and Thm. 2).

TEST INFRASTRUCTURE (like the rest of ``oracle/``): only the tests, ``smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; it shares no code with the CUDA library.

The route evaluates the vector transforms through scalar spherical harmonic transforms of
the Cartesian components T^(1), T^(2), T^(3) of a field (T = sum_c T^(c) e_c):

* FwdVSHT (Thm. 1, eq. almblmviaFlm): with the FwdSHT F_lm(f) = sum_k w_k f_k Y_lm(x_k)^*
  (eq. Flm) of the three components to degree L+1,
    a_lm = 1/sqrt2 { xi1_{l-1,m-1} [-F(T1) + i F(T2)]_{l-1,m-1} + xi2_{l+1,m-1} [..]_{l+1,m-1}
                   + xi3_{l-1,m+1} [F(T1) + i F(T2)]_{l-1,m+1} + xi4_{l+1,m+1} [..]_{l+1,m+1} }
           + xi5_{l-1,m} F(T3)_{l-1,m} + xi6_{l+1,m} F(T3)_{l+1,m},
    b_lm = -i/sqrt2 [ mu1_{l,m-1} (-F(T1) + i F(T2))_{l,m-1} + mu3_{l,m+1} (F(T1) + i F(T2))_{l,m+1} ]
           - i mu2_{l,m} F(T3)_{l,m},
  with the xi (eq. xi_klm) and mu (eq. mu_klm) products of c_l, d_l (eq. cl,dl,betal) and
  the Clebsch-Gordan values of eq. ninecoeff.  Every xi/mu at the shifted index is a CG
  value of the output index (l, m): xi1_{l-1,m-1} = c_l C^{l,m}_{l-1,m-1,1,1} and so on.
* AdjVSHT (Thm. 2, eq. SLvecviascal): the coefficient sets nu^(1..6) (eqs. nulm1, nulm2)
  and eta^(1..3) (eq. etalm) and scalar syntheses S_K(g) = sum_{l<=K} g_lm Y_lm (eq.
  SLscalar),
    T1 = -1/sqrt2 (S_{L-1}(nu1) + S_{L+1}(nu2) + S_L(eta1)),
    T2 = -1/sqrt2 (S_{L-1}(nu3) + S_{L+1}(nu4) - S_L(eta2)),
    T3 = S_{L-1}(nu5) + S_{L+1}(nu6) + S_L(eta3).
  Reading of the garbled support conditions of nu2, nu4, nu6: a_{l,m} = 0 outside
  1 <= l <= L, |m| <= l, and every nu is evaluated for all |m| <= l.

Scalar Y_lm and the nine CG closed forms come from ``favest_oracle.c`` (``sh_point``,
``cg9``), both pinned against scipy and sympy.
"""
import math

import numpy as np

from . import cg9, cidx, sh_point


def _sidx(l, m):
    return l * l + l + m


def _ytable(lmax, theta, phi):
    """Y_lm at every point: npts x (lmax+1)^2, index l^2 + l + m."""
    return np.stack([sh_point(lmax, t, p) for t, p in zip(theta, phi)], axis=0)


def _c(l):
    return math.sqrt((l + 1.0) / (2.0 * l + 1.0))


def _d(l):
    return math.sqrt(l / (2.0 * l + 1.0))


def fwd_cg(L, theta, phi, w, T):
    """Thm. 1: a_lm, b_lm (l = 1..L, |m| <= l) from Cartesian T (npts x 3 complex) at the
    points (theta, phi) with weights w, through FwdSHTs of degree L+1."""
    Y = _ytable(L + 1, theta, phi)                      # npts x (L+2)^2
    wT = np.asarray(w)[:, None] * np.asarray(T)         # npts x 3
    F = wT.T @ np.conj(Y)                               # 3 x (L+2)^2: F_lm(T^(c)) (eq. Flm)
    minus = -F[0] + 1j * F[1]                           # [-F(T1) + i F(T2)]
    plus = F[0] + 1j * F[1]                             # [ F(T1) + i F(T2)]
    F3 = F[2]

    def at(v, l, m):
        return v[_sidx(l, m)] if 0 <= l <= L + 1 and abs(m) <= l else 0.0

    K = L * L + 2 * L
    a = np.zeros(K, complex)
    b = np.zeros(K, complex)
    r2 = 1.0 / math.sqrt(2.0)
    for l in range(1, L + 1):
        cl, dl = _c(l), _d(l)
        for m in range(-l, l + 1):
            g = cg9(l, m)
            # xi1_{l-1,m-1} = c_l C^{l,m}_{l-1,m-1,1,1}; xi2_{l+1,m-1} = d_l C^{l,m}_{l+1,m-1,1,1};
            # xi3_{l-1,m+1} = c_l C^{l,m}_{l-1,m+1,1,-1}; xi4_{l+1,m+1} = d_l C^{l,m}_{l+1,m+1,1,-1};
            # xi5_{l-1,m} = c_l C^{l,m}_{l-1,m,1,0};       xi6_{l+1,m} = d_l C^{l,m}_{l+1,m,1,0}
            s = 0.0
            if abs(m - 1) <= l - 1:
                s += cl * g[0] * at(minus, l - 1, m - 1)
            s += dl * g[1] * at(minus, l + 1, m - 1)
            if abs(m + 1) <= l - 1:
                s += cl * g[4] * at(plus, l - 1, m + 1)
            s += dl * g[5] * at(plus, l + 1, m + 1)
            av = r2 * s
            if abs(m) <= l - 1:
                av += cl * g[2] * at(F3, l - 1, m)
            av += dl * g[3] * at(F3, l + 1, m)
            # mu1_{l,m-1} = C^{l,m}_{l,m-1,1,1}, mu3_{l,m+1} = C^{l,m}_{l,m+1,1,-1}, mu2_{l,m} = C^{l,m}_{l,m,1,0}
            t = 0.0
            if abs(m - 1) <= l:
                t += g[6] * at(minus, l, m - 1)
            if abs(m + 1) <= l:
                t += g[7] * at(plus, l, m + 1)
            bv = -1j * r2 * t - 1j * g[8] * at(F3, l, m)
            a[cidx(l, m)] = av
            b[cidx(l, m)] = bv
    return a, b


def adj_cg(L, a, b, theta, phi):
    """Thm. 2: Cartesian S_L(a, b) at the points (npts x 3 complex), through the nu/eta
    coefficient sets and scalar syntheses of degrees L-1, L, L+1."""
    a = np.asarray(a)
    b = np.asarray(b)

    def A(l, m):
        return a[cidx(l, m)] if 1 <= l <= L and abs(m) <= l else 0.0

    def Bc(l, m):
        return b[cidx(l, m)] if 1 <= l <= L and abs(m) <= l else 0.0

    def C(L_, M_, k):
        """The k-th closed form of eq. ninecoeff for the coupled state (L_, M_), used
        only where the uncoupled state it multiplies exists."""
        return cg9(L_, M_)[k]

    n = (L + 2) ** 2
    nu = np.zeros((6, n), complex)
    eta = np.zeros((3, n), complex)
    for l in range(0, L + 2):
        for m in range(-l, l + 1):
            k = _sidx(l, m)
            if l <= L - 1:
                # C^{l+1,m+1}_{l,m,1,1} and C^{l+1,m-1}_{l,m,1,-1}, C^{l+1,m}_{l,m,1,0}
                c1 = _c(l + 1)
                u = A(l + 1, m + 1) * C(l + 1, m + 1, 0)
                v = A(l + 1, m - 1) * C(l + 1, m - 1, 4)
                nu[0, k] = c1 * (u - v)
                nu[2, k] = 1j * c1 * (u + v)
                nu[4, k] = A(l + 1, m) * c1 * C(l + 1, m, 2)
            if 2 <= l <= L + 1:
                # C^{l-1,m+1}_{l,m,1,1}, C^{l-1,m-1}_{l,m,1,-1}, C^{l-1,m}_{l,m,1,0}
                d1 = _d(l - 1)
                u = A(l - 1, m + 1) * C(l - 1, m + 1, 1) if abs(m + 1) <= l - 1 else 0.0
                v = A(l - 1, m - 1) * C(l - 1, m - 1, 5) if abs(m - 1) <= l - 1 else 0.0
                nu[1, k] = d1 * (u - v)
                nu[3, k] = 1j * d1 * (u + v)
                if abs(m) <= l - 1:
                    nu[5, k] = A(l - 1, m) * d1 * C(l - 1, m, 3)
            if 1 <= l <= L:
                # C^{l,m+1}_{l,m,1,1}, C^{l,m-1}_{l,m,1,-1}, C^{l,m}_{l,m,1,0}
                u = Bc(l, m + 1) * C(l, m + 1, 6) if abs(m + 1) <= l else 0.0
                v = Bc(l, m - 1) * C(l, m - 1, 7) if abs(m - 1) <= l else 0.0
                eta[0, k] = 1j * (u - v)
                eta[1, k] = u + v
                eta[2, k] = 1j * Bc(l, m) * C(l, m, 8)
    Y = _ytable(L + 1, theta, phi)                      # S_K(g) = Y @ g (degrees above K are 0)
    S = lambda g: Y @ g
    r2 = 1.0 / math.sqrt(2.0)
    T1 = -r2 * (S(nu[0]) + S(nu[1]) + S(eta[0]))
    T2 = -r2 * (S(nu[2]) + S(nu[3]) - S(eta[1]))
    T3 = S(nu[4]) + S(nu[5]) + S(eta[2])
    return np.stack([T1, T2, T3], axis=-1)
