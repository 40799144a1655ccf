"""Accuracy experiment of Section 4.1 (Example "Accuracy", Case I, both rows
of Table 1: ferromagnetic beta_n = 885.4, beta_s = -4.1 and Anti-FM
beta_n = 240.8, beta_s = 7.5; box [-16, 16), gamma_x = 1, h0 = 1, and the
magnetization M = 0.5, the reading that reproduces both printed rows) run
entirely through the device path: bdg_ground_state for Phi_g, bdg_solve
(FP64) for the 20 smallest excitations, and the Kohn mode omega = gamma_x
among them (Theorem "Analytical eigenpairs").

Checks: at h0/2 and h0/4 the errors e_omega and e_uv of the Kohn mode
reproduce the printed values (e_omega to 1 %, e_uv to 30 %; the oracle's
own pin of the same table holds e_omega to 0.5 %); for the FM row, at h0/8
e_omega lies below the printed 1.383e-9 (the device and the oracle reach
about 1e-12 there), and e_omega falls by more than three orders of magnitude
per halving of h from h0/2 on (spectral accuracy, Section 3.4).

Residuals: for the lowest pairs (omega_1 about 0.019, |H| about 140-190) the
relative residual 1e-10 lies near the FP64 floor.  The dense eigenvectors,
evaluated with the oracle's FFT product, sit at 1e-10 to 4e-10.  With a
block of m = 40 for k = 20 the device solve reached 1e-10 for all pairs at
N = 64 and 128 in 180-240 iterations; with m = 24 it was too slow to.  The
test holds the Kohn pair to 1e-9 and the block to 1e-6 and accepts
BDG_ERR_NOT_CONVERGED at maxit.  The eigenvalue error is quadratic in the
residual, far below the e_omega compared."""
import json
import os

import numpy as np
import pytest

import synth
from gpu_util import need_torch_cuda

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


ROWS = {"fm": (885.4, -4.1), "afm": (240.8, 7.5)}
TABLE1_M = 0.5


def _case(n, row):
    bn, bs = ROWS[row]
    return synth.Workload(f"t1_{row}_{n}", (n,), (-16.0,), (16.0,), (1.0,), bn, bs, M=TABLE1_M, k=20, m=40,
                          gs_seed=17, block_seed=18)


def _kohn_errors(n, row="fm"):
    from oracle import kohn
    from paper_2506_08308_gb300 import bdg
    w = _case(n, row)
    V = synth.potential(w)
    phi, mu, res, _ = bdg.ground_state(bdg.params_from(w), w.M, V, synth.initial_spinor(w), tol=1e-12)
    assert res <= 1e-12
    plan = bdg.Plan(bdg.params_from(w, prec=bdg.FP64, tol=1e-10, maxit=400, seed=w.block_seed), V,
                    phi.reshape(-1))
    om, UV, resid, nconv = plan.solve(w.k, w.m, allow_not_converged=True)
    plan.close()
    i = int(np.argmin(np.abs(om - 1.0)))
    assert resid[i] <= 1e-9, (i, resid)
    assert resid.max() <= 1e-6, resid
    uv = UV[i].cpu().numpy().real
    (gam, f, g), = kohn.kohn_modes(w, phi)
    euv = kohn.e_uv(uv[:3].ravel(), uv[3:].ravel(), (f + g).ravel()[:, None], (f - g).ravel()[:, None])
    return kohn.e_omega(om[i], gam), euv


@pytest.mark.parametrize("row", ["fm", "afm"])
def test_table1_case1_device_path(row):
    need_torch_cuda()
    with open(os.path.join(HERE, "golden", f"table1_case1_{row}.json")) as fh:
        gold = json.load(fh)
    errs = {}
    for n, key in ((64, "h0/2"), (128, "h0/4")):
        eom, euv = _kohn_errors(n, row)
        pe, pu = gold["e_omega"][key], gold["e_uv"][key]
        assert abs(eom - pe) < 0.01 * pe, (key, eom, pe)
        assert abs(euv - pu) < 0.3 * pu, (key, euv, pu)
        errs[n] = eom
    if row != "fm":
        return
    eom256, _ = _kohn_errors(256)
    assert eom256 < gold["e_omega"]["h0/8"], eom256
    assert errs[128] < 1e-3 * errs[64] and eom256 < 1e-3 * errs[128] + 1e-11
