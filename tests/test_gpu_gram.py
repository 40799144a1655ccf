"""Parity of bdg_gram (the Gram contraction of the bi-orthogonal Gram-Schmidt
and of the Rayleigh-Ritz projected matrices, Section 3.2; Theorem
"Biorthogonality") with the oracle's pair_gram, element by element relative
to sum |a b| (the scale of the rounding):

  - tensor cores (split-BF16 slices, FP32 accumulation): 4e-6 for C64 and
    C128 blocks (FP32 accuracy);
  - CUDA cores: C128 in double-float 1e-14, C64 in FP32 1e-5;

on block shapes of the solver (48 x 48, 144 x 144 and 16 x 160 real
columns), on the row count of the 256^2 workload's f- or g-part
(3 * 65536 = 196608) and on ragged lengths (37, 1000, 20011 rows: part of one
stage, several chunks with a short tail), plus columns of very different
magnitude and bit-identical repeats."""
import numpy as np
import pytest

from gpu_util import need_torch_cuda

pytestmark = pytest.mark.gpu


def _blocks(torch, P, Q, n, dtype, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.randn((P, n), dtype=dtype, device="cuda", generator=g)
    B = torch.randn((Q, n), dtype=dtype, device="cuda", generator=g)
    # columns a thousand times smaller, and a decaying profile, as in the solver's blocks
    A[::5] *= 1e-3
    B[:, n // 2:] *= 1e-4
    return A, B


def _check(bdg, A, B, engine, tol):
    from oracle import lrep
    G = bdg.gram(A, B, engine=engine).cpu().numpy()
    S, Sabs = lrep.pair_gram(A.cpu().numpy(), B.cpu().numpy())
    err = np.abs(G - S) / np.maximum(Sabs, 1e-300)
    assert err.max() < tol, (err.max(), np.unravel_index(err.argmax(), err.shape))
    return G


@pytest.mark.parametrize("P,Q,n", [(24, 24, 196608), (72, 72, 20011), (8, 80, 1000), (24, 24, 37)])
@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_gram_tensor_cores_against_oracle(P, Q, n, dt):
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    dtype = torch.complex64 if dt == "c64" else torch.complex128
    A, B = _blocks(torch, P, Q, n, dtype, seed=P + Q + n)
    G = _check(bdg, A, B, bdg.GRAM_TENSOR, 4e-6)
    G2 = bdg.gram(A, B, engine=bdg.GRAM_TENSOR).cpu().numpy()
    assert np.array_equal(G, G2)


@pytest.mark.parametrize("dt,tol", [("c64", 1e-5), ("c128", 1e-14)])
def test_gram_cuda_cores_against_oracle(dt, tol):
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    dtype = torch.complex64 if dt == "c64" else torch.complex128
    for P, Q, n in [(72, 72, 20011), (24, 24, 196608)]:
        A, B = _blocks(torch, P, Q, n, dtype, seed=7)
        _check(bdg, A, B, bdg.GRAM_SIMT, tol)


def test_gram_edges():
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    A = torch.randn((4, 100), dtype=torch.complex128, device="cuda")
    B = torch.randn((81, 100), dtype=torch.complex128, device="cuda")
    with pytest.raises(RuntimeError, match="UNSUPPORTED"):
        bdg.gram(A, B, engine=bdg.GRAM_TENSOR)        # 162 real columns of B
    Z = torch.zeros((4, 0), dtype=torch.complex128, device="cuda")
    G = bdg.gram(Z, Z[:3], engine=bdg.GRAM_TENSOR)
    assert G.shape == (8, 6) and float(G.abs().max()) == 0.0
