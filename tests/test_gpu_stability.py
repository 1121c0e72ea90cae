"""GPU parity of the stability ratios of the forward Clebsch-Gordan route (Sec. 5.5,
eq. r_stable) against the oracle: per-coefficient extremes over the points and the four
summary ratios, at several degrees, point counts with ragged warps, points close to the
poles and a single point; at the paper's largest case (L = 10, N = 100,000) through the
bounds that hold at any size and agreement on a sampled subset.  The ratios are
extremes of per-point values, so the only tolerance is the rounding of each value."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_00041_gb300 import api  # noqa: E402
from oracle import stability  # noqa: E402

TOL = 1e-12
R2 = math.sqrt(2.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    api.lib(build_if_missing=True)


def _points(n, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    z = rng.uniform(lo, hi, n)
    return z, np.arccos(z), rng.uniform(0.0, 2.0 * np.pi, n)


def _compare(L, z, th, ph):
    r, ext = api.favest_cg_stability(L, z, per_coef=True)
    ref = stability.coefficient_extremes(L, th, ph)
    assert np.max(np.abs(ext - ref)) < TOL
    rr = stability.ratios(L, th, ph)
    assert abs(r[0] - rr[0]) < TOL and abs(r[2] - rr[2]) < TOL
    assert abs(r[1] - rr[1]) < TOL * rr[1] ** 2 and abs(r[3] - rr[3]) < TOL * rr[3] ** 2
    return r, ext


@pytest.mark.parametrize("L,n", [(1, 1), (1, 33), (5, 100), (5, 257), (10, 1000), (31, 200)])
def test_stability_vs_oracle(L, n):
    z, th, ph = _points(n, 500 + L * 7 + n)
    _compare(L, z, th, ph)


def test_stability_near_poles():
    z = np.array([1 - 1e-12, -1 + 1e-12, 1 - 1e-6, -1 + 1e-9, 0.0, 0.999999])
    _compare(12, z, np.arccos(z), np.zeros_like(z))


def test_stability_high_degree_finite_and_bounded():
    z, _, ph = _points(300, 77)
    z[:3] = [1 - 1e-13, -1 + 1e-13, 1 - 1e-10]
    th = np.arccos(z)
    r, ext = api.favest_cg_stability(200, z, per_coef=True)
    assert np.all(np.isfinite(ext[[0, 2]])) and np.all(np.isfinite(ext[[1, 3]]))
    assert r[0] <= 1 / R2 * (1 + 1e-13) and r[2] <= 1 / R2 * (1 + 1e-13)
    assert r[3] <= math.sqrt(6) * (1 + 1e-13)
    # the degrees the oracle reaches quickly, at the same points
    sub = stability.coefficient_extremes(8, th, ph)
    K8 = 8 * 8 + 16
    assert np.max(np.abs(ext[:, :K8] - sub)) < TOL


def test_stability_paper_size_l10_n100000():
    z, th, ph = _points(100_000, 2019)
    r, ext = api.favest_cg_stability(10, z, per_coef=True)
    assert r[0] <= 1 / R2 * (1 + 1e-13) and r[2] <= 1 / R2 * (1 + 1e-13)
    assert R2 <= r[3] <= math.sqrt(6) * (1 + 1e-13) and r[1] >= R2
    # order of the points does not matter (extremes are exact): identical bits
    perm = np.random.default_rng(3).permutation(len(z))
    r2, ext2 = api.favest_cg_stability(10, z[perm], per_coef=True)
    assert r2 == r and np.array_equal(ext2, ext)
    # extremes over all points bracket those of a sampled subset, which match the oracle
    idx = np.random.default_rng(4).choice(len(z), 400, replace=False)
    rs, exs = api.favest_cg_stability(10, z[idx], per_coef=True)
    ref = stability.coefficient_extremes(10, th[idx], ph[idx])
    assert np.max(np.abs(exs - ref)) < TOL
    assert np.all(ext[0] >= exs[0]) and np.all(ext[1] <= exs[1])
    assert np.all(ext[2] >= exs[2]) and np.all(ext[3] <= exs[3])
