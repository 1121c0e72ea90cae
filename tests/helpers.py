"""Shared test helpers: error metrics and grid construction (no transform arithmetic)."""
import os

import numpy as np


def normwise_err(got, ref):
    """max |got - ref| / max |ref| over the last axis, maximised over leading axes."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    if ref.ndim == 1:
        ref = ref[None]
        got = got[None]
    den = np.max(np.abs(ref), axis=-1)
    num = np.max(np.abs(got - ref), axis=-1)
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den))


def rms_err(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def cidx(l, m):
    return l * l + l + m - 1


def sample_coefs(L, n, rng):
    """n distinct (l, m) positions including the corners l = 1, l = L, m = +-l, 0."""
    fixed = [(1, -1), (1, 0), (1, 1), (L, -L), (L, 0), (L, L), (L, L - 1), (max(1, L // 2), 0)]
    out = {p for p in fixed}
    while len(out) < n:
        l = int(rng.integers(1, L + 1))
        m = int(rng.integers(-l, l + 1))
        out.add((l, m))
    out = sorted(out)
    return np.array([p[0] for p in out]), np.array([p[1] for p in out])


def hidx(l, m):
    """Position of (l, m >= 0) in a half-spectrum (real-field) coefficient array."""
    return l * (l + 1) // 2 - 1 + m


def _half_positions(L):
    ls = np.concatenate([np.full(l + 1, l) for l in range(1, L + 1)])
    ms = np.concatenate([np.arange(l + 1) for l in range(1, L + 1)])
    return ls, ms


def half_of_full(c, L):
    """The m >= 0 entries of full l-major coefficient arrays [..., L^2+2L]."""
    ls, ms = _half_positions(L)
    return np.asarray(c)[..., cidx(ls, ms)]


def full_of_half(c, L):
    """Hermitian extension c_{l,-m} = (-1)^m conj(c_lm) of half-spectrum arrays
    [..., L(L+3)/2] to full l-major arrays [..., L^2+2L]."""
    c = np.asarray(c)
    ls, ms = _half_positions(L)
    out = np.zeros(c.shape[:-1] + (L * L + 2 * L,), np.result_type(c, np.complex64))
    out[..., cidx(ls, ms)] = c
    pos = ms > 0
    sg = np.where(ms[pos] % 2 == 1, -1.0, 1.0)
    out[..., cidx(ls[pos], -ms[pos])] = sg * np.conj(c[..., pos])
    return out


def read_field_a():
    """Tangent Field A fixture (tests/golden/field_a.txt): its exact coefficients
    [(family, l, m, value)], the paper's Table 1 GL row {L: error} and Table 2 GL row
    [|T1-T0|, |T2-T0|, |T2-T1|, coefficient difference] at L = 40."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "field_a.txt")
    coefs, t1, t2 = [], {}, None
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] in ("a", "b"):
            coefs.append((line[0], int(line[1]), int(line[2]), float(line[3]) + 1j * float(line[4])))
        elif line[0] == "table1":
            t1[int(line[1])] = float(line[2])
        elif line[0] == "table2":
            t2 = [float(v) for v in line[2:]]
    return coefs, t1, t2
