"""bdg_ground_state (device flow + Newton) against the oracle's ground state
(eq. groundDef on S_M, eq. chem-formula): residual <= 1e-12, mu to 1e-10
relative, the density rho = |Phi|^2 (invariant under the spin rotations that
leave a ferromagnetic ground state degenerate) to 1e-9, and Phi itself up to
a global sign where the state is non-degenerate (q > 0)."""
import numpy as np
import pytest

import synth
from gpu_util import need_torch_cuda, oracle_problem

pytestmark = pytest.mark.gpu

CASES = [
    synth.Workload("s1d_n64", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, k=8, m=12, gs_seed=101),
    synth.Workload("s1d_n64_q", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.1, k=8, m=11, gs_seed=102),
    synth.Workload("s2d_16", (16, 16), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.4), 12.0, -1.0, 0.05, 0.3, k=10, m=14,
                   gs_seed=8),
    synth.Workload("s1d_afm", (128,), (-10.0,), (10.0,), (1.0,), 20.0, 2.0, 0.0, 0.0, k=4, m=8, gs_seed=11),
]


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_ground_state_matches_oracle(w):
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    V, phi_o, mu_o, op = oracle_problem(w)
    prm = bdg.params_from(w)
    phi, mu, res, it = bdg.ground_state(prm, w.M, V, synth.initial_spinor(w), tol=1e-12)
    assert res <= 1e-12
    assert it > 0
    np.testing.assert_allclose(mu, mu_o, rtol=1e-10, atol=1e-12)
    phi_o = phi_o.reshape(3, -1)
    rho, rho_o = np.sum(phi ** 2, 0), np.sum(phi_o ** 2, 0)
    assert np.max(np.abs(rho - rho_o)) <= 1e-9 * np.max(rho_o)
    if w.q > 0:
        err = min(np.max(np.abs(phi - phi_o)), np.max(np.abs(phi + phi_o)))
        assert err <= 1e-8 * np.max(np.abs(phi_o)), err
    # the constraint set S_M: mass 1, magnetization M (weighted l2, Section 3.3)
    cell = float(np.prod(w.h))
    n = cell * np.sum(phi ** 2, 1)
    assert abs(n.sum() - 1.0) < 1e-12 and abs(n[0] - n[2] - w.M) < 1e-12


def test_ground_state_rejects_bad_input():
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = CASES[0]
    prm = bdg.params_from(w)
    V = synth.potential(w)
    with pytest.raises(bdg.BdgError) as e:
        bdg.ground_state(prm, 1.5, V, synth.initial_spinor(w))
    assert e.value.status == bdg.ERR_INVALID
    with pytest.raises(bdg.BdgError) as e:
        bdg.ground_state(prm, 0.0, V, np.zeros((3, 64)))
    assert e.value.status in (bdg.ERR_INVALID,)
