"""Seeded synthetic inputs (no transform arithmetic).

Coefficient sets are drawn with numpy's PCG64 (``numpy.random.default_rng(seed)``):
for every field in order, family a then b, l-major (l = 1..L, m = -l..l), real and
imaginary parts i.i.d. standard normal times the spectrum factor (l+1)^(-p).  This
module is shared by the tests, the benchmark and the oracle-side checks; it holds
none of the method's arithmetic.
"""
import numpy as np


def degrees(L):
    """Degree l of every coefficient position, l-major (length L^2 + 2L)."""
    return np.concatenate([np.full(2 * l + 1, l) for l in range(1, L + 1)]).astype(np.int64)


def orders(L):
    return np.concatenate([np.arange(-l, l + 1) for l in range(1, L + 1)]).astype(np.int64)


def coefficients(L, batch, seed, decay=1.0, rng=None):
    """(a, b): complex128 arrays [batch, L^2+2L], N(0,1)*(l+1)^-decay parts."""
    rng = np.random.default_rng(seed) if rng is None else rng
    K = L * L + 2 * L
    s = (degrees(L) + 1.0) ** (-float(decay))
    a = np.empty((batch, K), np.complex128)
    b = np.empty((batch, K), np.complex128)
    for f in range(batch):
        for arr in (a, b):
            z = rng.standard_normal((K, 2))
            arr[f] = (z[:, 0] + 1j * z[:, 1]) * s
    return a, b


def ragged_degrees(nfields, choices, seed):
    """Degrees of a ragged batch: rng.choice(choices, nfields) drawn first."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(choices), nfields), rng


def grid_field(L, batch, seed):
    """Random (not band-limited) tangent field components on the (L+1) x 2(L+1) grid:
    complex128 [batch, L+1, 2(L+1)] each, parts i.i.d. standard normal."""
    rng = np.random.default_rng(seed)
    shape = (batch, L + 1, 2 * (L + 1))
    tt = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    tp = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return tt, tp


def mask(L, seed_rng):
    """Positive latitude-longitude mask g ~ U[0.5, 1.5] on the grid."""
    return seed_rng.uniform(0.5, 1.5, (L + 1, 2 * (L + 1)))


def real_grid_field(L, batch, seed):
    """Random real tangent field components on the (L+1) x 2(L+1) grid: float64
    [batch, L+1, 2(L+1)] each, i.i.d. standard normal (theta plane drawn first)."""
    rng = np.random.default_rng(seed)
    shape = (batch, L + 1, 2 * (L + 1))
    return rng.standard_normal(shape), rng.standard_normal(shape)


def half_coefficients(L, batch, seed, decay=1.0, rng=None):
    """Coefficients of real fields, orders m >= 0 only: complex128 [batch, L(L+3)/2],
    l-major (l = 1..L, m = 0..l); per field a then b, (re, im) i.i.d. standard normal
    times (l+1)^-decay, with the imaginary part of every m = 0 entry set to zero."""
    rng = np.random.default_rng(seed) if rng is None else rng
    KR = L * (L + 3) // 2
    deg = np.concatenate([np.full(l + 1, l) for l in range(1, L + 1)])
    m0 = np.concatenate([np.arange(l + 1) == 0 for l in range(1, L + 1)])
    s = (deg + 1.0) ** (-float(decay))
    a = np.empty((batch, KR), np.complex128)
    b = np.empty((batch, KR), np.complex128)
    for f in range(batch):
        for arr in (a, b):
            z = rng.standard_normal((KR, 2))
            z[m0, 1] = 0.0
            arr[f] = (z[:, 0] + 1j * z[:, 1]) * s
    return a, b
