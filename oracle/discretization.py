"""Fourier pseudospectral discretization (Section 3.1).

Grid: N even, nodes x_n = lo + n h, h = (hi - lo)/N, n = 0..N-1, box
half-length L = (hi - lo)/2.  Plane waves W_k(x) = exp(i mu_k (x - lo)),
mu_k = pi k / L, k = -N/2 .. N/2-1.

DFT (eq. FT_3):   F~_k = (1/N) sum_n F(x_n) exp(-2 pi i n k / N).
Interpolant (eq. laplace_approx): F(x_n) = sum_k F~_k W_k(x_n).
Laplacian (eq. laplace_approx): (Lap F)(x_n) = sum_k -mu_k^2 F~_k W_k(x_n),
the Nyquist mode k = -N/2 keeping its mu^2 (the sum runs over all k).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np


def wavenumbers(n: int, lo: float, hi: float) -> np.ndarray:
    """mu_k for k = -N/2..N/2-1, returned in DFT index order j = 0..N-1
    (j < N/2 -> k = j, j >= N/2 -> k = j - N)."""
    L = 0.5 * (hi - lo)
    k = np.arange(n)
    k = np.where(k < n // 2, k, k - n)
    return np.pi * k / L


def dft_matrix(n: int) -> np.ndarray:
    """Forward DFT of eq. FT_3 as a matrix: Ft[k, n] = exp(-2 pi i n k/N)/N,
    rows in DFT index order."""
    idx = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(idx, idx) / n) / n


def idft_matrix(n: int) -> np.ndarray:
    """Interpolant evaluation at the nodes: F(x_n) = sum_k F~_k W_k(x_n) with
    W_k(x_n) = exp(2 pi i n k / N) (the inverse of dft_matrix)."""
    idx = np.arange(n)
    return np.exp(2j * np.pi * np.outer(idx, idx) / n)


def laplacian_matrix_1d(n: int, lo: float, hi: float) -> np.ndarray:
    """The dense N x N spectral second-derivative matrix
    [[Lap]] = IDFT diag(-mu_k^2) DFT (eq. laplace_approx); real symmetric."""
    mu = wavenumbers(n, lo, hi)
    m = idft_matrix(n) @ np.diag(-mu ** 2) @ dft_matrix(n)
    return m.real


def laplacian_matrix(shape, lo, hi) -> np.ndarray:
    """Dense Laplacian on the tensor grid: Kronecker sum of the 1-D matrices."""
    mats = [laplacian_matrix_1d(nn, a, b) for nn, a, b in zip(shape, lo, hi)]
    total = None
    for ax, mat in enumerate(mats):
        term = np.ones((1, 1))
        for bx in range(len(mats)):
            term = np.kron(term, mat if bx == ax else np.eye(shape[bx]))
        total = term if total is None else total + term
    return total


def _apply_along(mat: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    f = np.moveaxis(f, axis, -1)
    out = f @ mat.T
    return np.moveaxis(out, -1, axis)


def laplacian_dft(f: np.ndarray, lo, hi) -> np.ndarray:
    """Laplacian of grid function(s) by separable DFT matrices: for each axis,
    DFT along that axis, multiply by -mu_k^2, evaluate the interpolant.
    The last len(lo) axes of f are the spatial axes."""
    d = len(lo)
    out = np.zeros(f.shape, dtype=np.result_type(f.dtype, np.complex128))
    for ax in range(d):
        axis = f.ndim - d + ax
        n = f.shape[axis]
        mu = wavenumbers(n, lo[ax], hi[ax])
        op = idft_matrix(n) @ np.diag(-mu ** 2) @ dft_matrix(n)
        out += _apply_along(op, f, axis)
    return out


def laplacian_fft(f: np.ndarray, lo, hi) -> np.ndarray:
    """Laplacian by numpy.fft: the full d-dimensional transform, multiply by
    -|mu|^2, inverse transform.  The last len(lo) axes are spatial."""
    d = len(lo)
    axes = tuple(range(f.ndim - d, f.ndim))
    spec = np.fft.fftn(f, axes=axes)
    k2 = np.zeros([f.shape[a] for a in axes])
    for i, a in enumerate(axes):
        mu = wavenumbers(f.shape[a], lo[i], hi[i])
        shape = [1] * d
        shape[i] = f.shape[a]
        k2 = k2 + (mu ** 2).reshape(shape)
    return np.fft.ifftn(-k2 * spec, axes=axes)


def spectral_derivative(f: np.ndarray, axis_index: int, lo, hi) -> np.ndarray:
    """First derivative along one spatial axis by the Fourier interpolant,
    with the Nyquist coefficient zeroed (the interpolant's derivative of the
    unpaired mode k = -N/2 is not real).  f has exactly len(lo) axes."""
    n = f.shape[axis_index]
    mu = wavenumbers(n, lo[axis_index], hi[axis_index]).astype(np.complex128)
    mu[n // 2] = 0.0
    spec = np.fft.fft(f, axis=axis_index)
    shape = [1] * f.ndim
    shape[axis_index] = n
    return np.fft.ifft(1j * mu.reshape(shape) * spec, axis=axis_index).real


def inverse_kdiag(f: np.ndarray, symbol, lo, hi) -> np.ndarray:
    """Apply IDFT diag(symbol(|mu|^2)) DFT over the last len(lo) axes."""
    d = len(lo)
    axes = tuple(range(f.ndim - d, f.ndim))
    k2 = np.zeros([f.shape[a] for a in axes])
    for i, a in enumerate(axes):
        mu = wavenumbers(f.shape[a], lo[i], hi[i])
        shape = [1] * d
        shape[i] = f.shape[a]
        k2 = k2 + (mu ** 2).reshape(shape)
    out = np.fft.ifftn(symbol(k2) * np.fft.fftn(f, axes=axes), axes=axes)
    return out if np.iscomplexobj(f) else out.real
