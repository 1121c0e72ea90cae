"""Host-side checks of the real-field (half-spectrum) coefficient layout used by the
FAVEST_IO_R32 tests: the half-spectrum index and the Hermitian extension
a_{l,-m} = (-1)^m conj(a_lm), against the oracle's transform of a real field."""
import numpy as np

from helpers import cidx, full_of_half, half_of_full, hidx

from paper_1908_00041_gb300 import synthetic


def test_half_index_is_dense_l_major():
    L = 9
    pos = [hidx(l, m) for l in range(1, L + 1) for m in range(l + 1)]
    assert pos == list(range(L * (L + 3) // 2))


def test_hermitian_extension_matches_oracle_real_field(orc):
    L = 12
    x, W, theta, phi = orc.grid(L)
    tt, tp = synthetic.real_grid_field(L, 1, seed=5)
    a, b = orc.fwd_sep(L, x, W, tt[0] + 0j, tp[0] + 0j)
    for c in (a, b):
        h = half_of_full(c, L)
        assert np.allclose(full_of_half(h, L), c, rtol=0, atol=1e-13 * np.max(np.abs(c)))
        assert np.max(np.abs(h[[hidx(l, 0) for l in range(1, L + 1)]].imag)) < 1e-13 * np.max(np.abs(c))
    assert cidx(L, L) == L * L + 2 * L - 1


def test_half_coefficients_recipe():
    a, b = synthetic.half_coefficients(6, 2, seed=3, decay=1.0)
    assert a.shape == (2, 27) and b.shape == (2, 27)
    m0 = [hidx(l, 0) for l in range(1, 7)]
    assert np.all(a[:, m0].imag == 0) and np.all(b[:, m0].imag == 0)
    a2, _ = synthetic.half_coefficients(6, 2, seed=3, decay=1.0)
    assert np.array_equal(a, a2)
