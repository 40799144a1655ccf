"""The seeded input generators (shared by the oracle and the CUDA path, and
holding none of the method's arithmetic): the same seed gives bit-identical
inputs, different seeds give different ones, and the recipe stated for each
workload holds (grids, boxes, trap, parameter ranges of the batched draws)."""
import numpy as np

import synth


def test_same_seed_same_inputs():
    w = synth.W1D_N256
    for f in (lambda: synth.initial_spinor(w), lambda: synth.random_block(w, 3),
              lambda: synth.random_block(w, 2, complex_=False), lambda: synth.smooth_block(w, 2)):
        a, b = f(), f()
        assert a.dtype == b.dtype and np.array_equal(a, b)
    assert not np.array_equal(synth.random_block(w, 2, seed=1), synth.random_block(w, 2, seed=2))
    assert not np.array_equal(synth.initial_spinor(w, seed=1), synth.initial_spinor(w, seed=2))


def test_shapes_and_types():
    w = synth.W2D_N256
    assert w.npts == 256 * 256 and w.dim == 2
    assert synth.potential(w).shape == (256, 256)
    x = synth.random_block(synth.W1D_N256, 4)
    assert x.shape == (4, 6, 256) and x.dtype == np.complex128
    assert synth.initial_spinor(synth.W1D_N256).shape == (3, 256)


def test_grid_and_trap():
    """Nodes x_n = lo + n h on the half-open box and V = 1/2 sum gamma^2 x^2."""
    w = synth.W3D_N128
    ax = synth.axes(w)
    h = (w.hi[0] - w.lo[0]) / w.n[0]
    assert ax[0][0] == w.lo[0] and abs(ax[0][-1] - (w.hi[0] - h)) < 1e-12
    V = synth.potential(synth.small(w, 8))
    x = synth.axes(synth.small(w, 8))
    i, j, k = 1, 5, 6
    expect = 0.5 * sum((g * xx[n]) ** 2 for g, xx, n in zip(w.gamma, x, (i, j, k)))
    assert abs(V[i, j, k] - expect) < 1e-12


def test_batched_draws_follow_the_recipe():
    ws = synth.batched_workloads()
    assert len(ws) == 64
    for i, w in enumerate(ws):
        assert w.n[0] == w.n[1] and w.n[0] in (64, 128, 256)
        assert 50.0 <= w.beta_n <= 200.0 and -5.0 <= w.beta_s <= 5.0 and 0.0 <= w.q <= 0.5
        assert w.k == 16 and w.m == 24 and w.gs_seed == 104 + i and w.block_seed == 2004 + i
    assert len({w.n[0] for w in ws}) == 3
    assert [w.beta_n for w in synth.batched_workloads()] == [w.beta_n for w in ws]
