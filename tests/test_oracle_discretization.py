"""Pins of the Fourier pseudospectral discretization (Section 3.1,
eqs. FT_3 and laplace_approx) against textbook facts: the DFT written as an
explicit sum and numpy.fft, exact plane-wave eigenfunctions of the spectral
Laplacian (Nyquist included), Parseval, and the second derivative of a
Gaussian."""
import numpy as np
import pytest

from oracle import discretization as disc


@pytest.mark.parametrize("n", [8, 16, 64])
def test_dft_matrix_matches_explicit_sum_and_numpy(n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    explicit = np.array([sum(f[j] * np.exp(-2j * np.pi * j * k / n) for j in range(n)) / n
                         for k in range(n)])
    assert np.allclose(disc.dft_matrix(n) @ f, explicit, atol=1e-14)
    assert np.allclose(disc.dft_matrix(n) @ f, np.fft.fft(f) / n, atol=1e-14)
    assert np.allclose(disc.idft_matrix(n) @ (disc.dft_matrix(n) @ f), f, atol=1e-13)


@pytest.mark.parametrize("n,lo,hi", [(16, -4.0, 4.0), (32, -16.0, 16.0), (64, 0.0, 3.0)])
def test_plane_waves_are_exact_eigenfunctions(n, lo, hi):
    x = lo + np.arange(n) * (hi - lo) / n
    L = 0.5 * (hi - lo)
    for k in range(-n // 2, n // 2):
        mu = np.pi * k / L
        wk = np.exp(1j * mu * (x - lo))
        for lap in (disc.laplacian_fft(wk, (lo,), (hi,)), disc.laplacian_dft(wk, (lo,), (hi,)),
                    disc.laplacian_matrix_1d(n, lo, hi) @ wk):
            assert np.allclose(lap, -mu * mu * wk, atol=1e-10 * max(1.0, mu * mu))


def test_laplacian_forms_agree_2d_3d():
    rng = np.random.default_rng(0)
    for shape, lo, hi in [((8, 16), (-3.0, -5.0), (3.0, 5.0)), ((4, 8, 8), (-1.0, -2.0, -2.0), (1.0, 2.0, 2.0))]:
        f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        a = disc.laplacian_fft(f, lo, hi)
        b = disc.laplacian_dft(f, lo, hi)
        c = (disc.laplacian_matrix(shape, lo, hi) @ f.ravel()).reshape(shape)
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
        assert np.abs(a - c).max() < 1e-12 * np.abs(a).max()


def test_gaussian_second_derivative_spectral_accuracy():
    n, lo, hi = 128, -12.0, 12.0
    x = lo + np.arange(n) * (hi - lo) / n
    f = np.exp(-x * x / 2)
    exact = (x * x - 1) * f
    lap = disc.laplacian_fft(f, (lo,), (hi,)).real
    assert np.abs(lap - exact).max() < 1e-12


def test_parseval():
    rng = np.random.default_rng(3)
    n = 32
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ft = disc.dft_matrix(n) @ f
    assert np.isclose(np.sum(np.abs(f) ** 2) / n, np.sum(np.abs(ft) ** 2), rtol=1e-13)


def test_wavenumber_ordering_and_nyquist():
    mu = disc.wavenumbers(8, -2.0, 2.0)
    # L = 2: mu_k = pi k / 2, DFT order k = 0,1,2,3,-4,-3,-2,-1
    assert np.allclose(mu, np.pi * np.array([0, 1, 2, 3, -4, -3, -2, -1]) / 2.0)
