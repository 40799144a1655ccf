"""Write tests/golden/solve_2d_n256.json: the 32 smallest excitation energies
of the 2-D benchmark instance (box [-12, 12)^2, N = 256^2, V = |x|^2/2,
beta_n = 100, beta_s = -2, p = 0, q = 0.1, M = 0) from the CPU oracle alone.

Steps (all in oracle/, FP64):
  1. ground state by the normalized gradient flow plus Newton-PCG from the
     seeded start spinor, stopped at max |H Phi - mu Phi| <= 1e-12
     (eq. groundDef, reading P18);
  2. chemical potentials by eq. chem-formula, the operator of eq. lrep-d and
     the deflation bases of reading P7;
  3. the oracle's block subspace iteration (reading P8) from the seeded real
     start block, k = 32, m = 48, relative residual <= 1e-10 (reading P9),
     preconditioned by 10 inner PCG steps on H_+ / H_- (reading P10).

The run also records the oracle's measured wall time and iteration count,
which is the CPU timing of this instance solved to convergence, and writes
the oracle's ground state Phi (3 x 256^2 FP64) to phi_2d_n256.npz beside
the JSON file, so that tests can build the oracle operator without
repeating the flow (several minutes on the host).

Usage: python tests/golden/make_solve_2d_n256.py [out.json] [--ground-state-only]
  --ground-state-only  steps 1-2 only: rewrite phi_2d_n256.npz, keep the JSON
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import apply as ap  # noqa: E402
from oracle import ground_state as gs  # noqa: E402
from oracle import lrep  # noqa: E402


def main(out_path, ground_state_only=False):
    w = synth.W2D_N256
    t0 = time.time()
    V = synth.potential(w)
    phi, mu, res_gs, it_gs = gs.ground_state(w, V, synth.initial_spinor(w), tol=1e-12)
    t_gs = time.time() - t0
    np.savez_compressed(os.path.join(os.path.dirname(out_path), "phi_2d_n256.npz"), phi=phi, mu=mu)
    if ground_state_only:
        return
    op = ap.Operator(w, phi, V, mu)
    Zf, Zg = lrep.deflation_bases(op, phi)
    X0 = synth.random_block(w, w.m, complex_=False)
    t1 = time.time()
    om, F, G, res, it = lrep.solve_iterative(op, w.k, w.m, X0, Zf, Zg, tol=1e-10, maxit=1000, inner=10,
                                             verbose=True)
    t_solve = time.time() - t1
    # a-posteriori check of the pairs through the UV operator (reading P9)
    r_uv = lrep.residual_uv(op, lrep.fg_to_uv(F, G), om)
    out = {
        "source": "oracle/ only: ground state (tol 1e-12), deflation bases, block subspace iteration "
                  "(k = 32, m = 48, tol 1e-10, 10 inner PCG steps) on the 2-D benchmark instance",
        "workload": synth.describe(w),
        "omega": [float(x) for x in om],
        "resid": [float(x) for x in res],
        "resid_uv": [float(x) for x in r_uv],
        "mu": [float(x) for x in mu],
        "ground_state_residual": float(res_gs),
        "ground_state_iterations": int(it_gs),
        "ground_state_seconds": t_gs,
        "iterations": int(it),
        "solve_seconds": t_solve,
        "cpu_threads": os.cpu_count(),
        "nzf": int(Zf.shape[1]),
        "nzg": int(Zg.shape[1]),
    }
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: out[k] for k in ("iterations", "solve_seconds", "ground_state_seconds")}))
    assert max(res) <= 1e-10, max(res)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    main(args[0] if args else os.path.join(HERE, "solve_2d_n256.json"), "--ground-state-only" in sys.argv)
