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


def test_inverse_kdiag_on_plane_waves():
    """IDFT diag(s(|mu|^2)) DFT multiplies a plane wave exp(i (mu_a x + mu_b y))
    by s(mu_a^2 + mu_b^2), with mu = pi k / L written out here from the
    definition (Nyquist included); s = 1 / (|mu|^2 / 2 + sigma), the
    preconditioner T_sigma, then inverts -Lap/2 + sigma."""
    shape, lo, hi = (8, 12), (-3.0, -4.0), (3.0, 5.0)
    xs = [a + np.arange(n) * (b - a) / n for n, a, b in zip(shape, lo, hi)]
    X, Y = np.meshgrid(*xs, indexing="ij")
    La, Lb = 0.5 * (hi[0] - lo[0]), 0.5 * (hi[1] - lo[1])
    sigma = 0.7

    def symbol(k2):
        return 1.0 / (0.5 * k2 + sigma)
    for ka, kb in ((0, 0), (1, 0), (0, -3), (2, 5), (-4, -6), (3, -6)):
        ma, mb = np.pi * ka / La, np.pi * kb / Lb
        wave = np.exp(1j * (ma * (X - lo[0]) + mb * (Y - lo[1])))
        got = disc.inverse_kdiag(wave, symbol, lo, hi)
        np.testing.assert_allclose(got, symbol(ma * ma + mb * mb) * wave, atol=1e-13)
        got = disc.inverse_kdiag(wave, lambda k2: -k2, lo, hi)
        np.testing.assert_allclose(got, -(ma * ma + mb * mb) * wave, atol=1e-11 * max(1.0, ma * ma + mb * mb))
    rng = np.random.default_rng(4)
    f = rng.standard_normal(shape)
    g = -0.5 * (disc.laplacian_matrix(shape, lo, hi) @ f.ravel()).reshape(shape) + sigma * f
    np.testing.assert_allclose(disc.inverse_kdiag(g, symbol, lo, hi), f, atol=1e-12)


def test_spectral_derivative_of_sines_and_cosines():
    """d/dx sin(mu_k (x - lo)) = mu_k cos(mu_k (x - lo)) and d/dx cos = -mu_k sin
    for |k| < N/2 along either axis of a 2-D array; the Nyquist cosine has a
    zero derivative (its coefficient is dropped), and a function constant
    along the axis differentiates to zero."""
    shape, lo, hi = (16, 10), (-2.0, 0.0), (2.0, 5.0)
    xs = [a + np.arange(n) * (b - a) / n for n, a, b in zip(shape, lo, hi)]
    grids = np.meshgrid(*xs, indexing="ij")
    for ax in (0, 1):
        n, L = shape[ax], 0.5 * (hi[ax] - lo[ax])
        t = grids[ax] - lo[ax]
        other = np.cos(0.3 * grids[1 - ax])            # constant along ax
        for k in range(1, n // 2):
            mu = np.pi * k / L
            d = disc.spectral_derivative(np.sin(mu * t) * other, ax, lo, hi)
            np.testing.assert_allclose(d, mu * np.cos(mu * t) * other, atol=1e-12 * mu)
            d = disc.spectral_derivative(np.cos(mu * t) * other, ax, lo, hi)
            np.testing.assert_allclose(d, -mu * np.sin(mu * t) * other, atol=1e-12 * mu)
        nyq = np.cos(np.pi * (n // 2) / L * t)
        assert np.abs(disc.spectral_derivative(nyq, ax, lo, hi)).max() < 1e-12
        assert np.abs(disc.spectral_derivative(np.cos(0.3 * grids[1 - ax]), ax, lo, hi)).max() < 1e-12
