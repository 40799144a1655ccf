"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the BdG method itself: it defines the
workload parameters (grids, boxes, interaction constants, block sizes), the
harmonic trap sampled on the grid, and seeded random numbers (initial spinors
for the ground-state flow, initial blocks for the eigensolver, the parameter
draws of the batched workload).  Both the CPU oracle and the CUDA path take
their inputs from here; neither computes them itself.

Grid convention: an axis with N points on the half-open box [lo, hi) has
nodes x_n = lo + n*h, h = (hi-lo)/N, n = 0..N-1 (Section 3.1; the half-open
reading of the grid set).  Arrays are C-ordered with axis 0 = x, axis 1 = y,
axis 2 = z, the last axis fastest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """Parameters of one BdG problem instance."""
    name: str
    n: Tuple[int, ...]           # grid points per axis (powers of two)
    lo: Tuple[float, ...]        # box lower corner per axis
    hi: Tuple[float, ...]        # box upper corner per axis (exclusive)
    gamma: Tuple[float, ...]     # trap frequencies gamma_alpha, V = 1/2 sum gamma^2 x^2
    beta_n: float
    beta_s: float
    p: float = 0.0               # linear Zeeman
    q: float = 0.0               # quadratic Zeeman
    M: float = 0.0               # magnetization of the ground state
    k: int = 16                  # wanted eigenpairs
    m: int = 24                  # block size
    gs_seed: int = 0
    block_seed: int = 0

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def npts(self) -> int:
        return int(np.prod(self.n))

    @property
    def h(self) -> Tuple[float, ...]:
        return tuple((b - a) / nn for a, b, nn in zip(self.lo, self.hi, self.n))

    def with_grid(self, n: Sequence[int]) -> "Workload":
        return dataclasses.replace(self, n=tuple(int(v) for v in n))


# The benchmark workloads, named by dimension and points per axis: the 1-D
# FP64 case, the 2-D FP64-versus-mixed case, the 3-D mixed case and the large
# 3-D case (the batched 2-D workload is drawn by batched_workloads below).
W1D_N256 = Workload("1d_n256", (256,), (-16.0,), (16.0,), (1.0,), 10.0, -1.0, 0.0, 0.0,
                   k=16, m=24, gs_seed=101, block_seed=1001)
W2D_N256 = Workload("2d_n256", (256, 256), (-12.0, -12.0), (12.0, 12.0), (1.0, 1.0),
                   100.0, -2.0, 0.0, 0.1, k=32, m=48, gs_seed=102, block_seed=1002)
W3D_N128 = Workload("3d_n128", (128, 128, 128), (-8.0,) * 3, (8.0,) * 3, (1.0, 1.5, 2.0),
                   200.0, -4.0, 0.05, 0.2, k=32, m=48, gs_seed=103, block_seed=1003)
W3D_N256 = Workload("3d_n256", (256, 256, 256), (-10.0,) * 3, (10.0,) * 3, (1.0, 1.0, 1.0),
                   400.0, -8.0, 0.0, 0.1, k=24, m=32, gs_seed=105, block_seed=1005)
WORKLOADS = {w.name: w for w in (W1D_N256, W2D_N256, W3D_N128, W3D_N256)}


def batched_workloads(count: int = 64, seed: int = 4) -> list:
    """Parameter draws of the batched 2-D workload: per instance, in order, a
    grid from {64^2, 128^2, 256^2}, beta_n ~ U[50,200], beta_s ~ U[-5,5],
    q ~ U[0,0.5]; box [-12,12)^2, isotropic trap, p = 0, k = 16, m = 24."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        nn = int(rng.choice([64, 128, 256]))
        bn = float(rng.uniform(50.0, 200.0))
        bs = float(rng.uniform(-5.0, 5.0))
        q = float(rng.uniform(0.0, 0.5))
        out.append(Workload(f"batch{i}_n{nn}", (nn, nn), (-12.0, -12.0), (12.0, 12.0),
                            (1.0, 1.0), bn, bs, 0.0, q, k=16, m=24,
                            gs_seed=104 + i, block_seed=2004 + i))
    return out


def axes(w: Workload):
    """Node coordinates per axis, x_n = lo + n h."""
    return [lo + np.arange(nn, dtype=np.float64) * (hi - lo) / nn
            for nn, lo, hi in zip(w.n, w.lo, w.hi)]


def potential(w: Workload) -> np.ndarray:
    """Harmonic trap V(x) = 1/2 sum_alpha gamma_alpha^2 x_alpha^2 on the grid
    (eq. Vpoten), shape w.n, float64."""
    grids = np.meshgrid(*axes(w), indexing="ij")
    v = np.zeros(w.n, dtype=np.float64)
    for g, gam in zip(grids, w.gamma):
        v += 0.5 * (gam * g) ** 2
    return v


def initial_spinor(w: Workload, seed: Optional[int] = None) -> np.ndarray:
    """Seeded start of the ground-state flow: a Gaussian envelope with seeded
    positive weights per component plus a small seeded perturbation, shape
    (3,)+w.n, float64, not normalised."""
    rng = np.random.Generator(np.random.PCG64(w.gs_seed if seed is None else seed))
    grids = np.meshgrid(*axes(w), indexing="ij")
    r2 = np.zeros(w.n)
    for g, gam in zip(grids, w.gamma):
        r2 += gam * g * g
    env = np.exp(-0.5 * r2)
    wts = 0.5 + rng.uniform(0.0, 1.0, size=3)
    phi = np.stack([wts[j] * env for j in range(3)])
    phi *= 1.0 + 0.05 * rng.standard_normal(phi.shape)
    return phi


def random_block(w: Workload, nvec: int, complex_: bool = True,
                 seed: Optional[int] = None) -> np.ndarray:
    """Seeded N(0,1) block of nvec 6-component vectors, shape (nvec, 6, npts);
    complex blocks draw real and imaginary parts independently."""
    rng = np.random.Generator(np.random.PCG64(w.block_seed if seed is None else seed))
    shape = (nvec, 6, w.npts)
    if complex_:
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return rng.standard_normal(shape)


def smooth_block(w: Workload, nvec: int, seed: Optional[int] = None) -> np.ndarray:
    """Seeded smooth complex block: Gaussian-windowed random low-order
    polynomials, shape (nvec, 6, npts).  Used where the FP32 error relative to
    the operator norm is measured on resolved data."""
    rng = np.random.Generator(np.random.PCG64(w.block_seed + 7 if seed is None else seed))
    grids = np.meshgrid(*axes(w), indexing="ij")
    r2 = np.zeros(w.n)
    for g, gam in zip(grids, w.gamma):
        r2 += gam * g * g
    env = np.exp(-0.5 * r2).ravel()
    out = np.empty((nvec, 6, w.npts), dtype=np.complex128)
    flat = [g.ravel() for g in grids]
    for i in range(nvec):
        for c in range(6):
            poly = np.full(w.npts, rng.standard_normal() + 1j * rng.standard_normal())
            for g in flat:
                poly += (rng.standard_normal() + 1j * rng.standard_normal()) * g
                poly += 0.3 * (rng.standard_normal() + 1j * rng.standard_normal()) * g * g
            out[i, c] = poly * env
    return out


def small(w: Workload, n: int) -> Workload:
    """The same physics on a coarser grid with n points per axis."""
    return w.with_grid((n,) * w.dim)


def describe(w: Workload) -> dict:
    return {"workload": w.name, "grid": list(w.n), "box": [list(w.lo), list(w.hi)],
            "gamma": list(w.gamma), "beta_n": w.beta_n, "beta_s": w.beta_s,
            "p": w.p, "q": w.q, "M": w.M, "k": w.k, "m": w.m}
