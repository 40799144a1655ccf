"""bdg_chemical_potentials_noalloc, the entry point for callers that must not
allocate device memory during a call: it works in a fixed scratch array the
library owns instead of buffers it allocates.  Its chemical potentials must
agree with the ones bdg_plan_create computes (read back with bdg_plan_mu) on
two calls in a row -- the second call sees the first call's leftovers in the
shared array -- and plans beyond its size limit must be refused.

The file sorts last so that a run stopping at the first failure has run every
other test before this one."""
import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    synth.Workload("na_1d_q", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.1, gs_seed=102),
    synth.Workload("na_2d_16", (16, 16), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.4), 12.0, -1.0, 0.05, 0.3, gs_seed=8),
    # the largest grid the fixed scratch holds: 128^2 = 16384 points
    synth.Workload("na_2d_128", (128, 128), (-8.0, -8.0), (8.0, 8.0), (1.0, 1.0), 50.0, 2.0, 0.0, 0.2, gs_seed=9),
]


def _spinor(w):
    """A normalised seeded spinor; the chemical-potential formula applies to
    any Phi, so no ground state is needed to compare the two code paths."""
    phi = synth.initial_spinor(w)
    return phi / np.sqrt(np.prod(w.h) * np.sum(phi ** 2))


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_noalloc_matches_plan_mu(w):
    need_torch_cuda()
    V = synth.potential(w)
    phi = _spinor(w)
    ref_plan = make_plan(w, V, phi)                    # mu = NaN: computed at plan creation
    mu_ref = ref_plan.mu
    other = make_plan(w, V, phi, mu=(0.0, 0.0, 0.0))   # a plan that uses given mu
    for plan in (ref_plan, other, ref_plan):           # consecutive calls share the scratch
        mu = plan.chemical_potentials_noalloc()
        np.testing.assert_allclose(mu, mu_ref, rtol=1e-12, atol=0)
    np.testing.assert_array_equal(other.mu, [0.0, 0.0, 0.0])   # the plan's own mu is untouched
    ref_plan.close()
    other.close()


def test_noalloc_allocates_nothing():
    """The entry point exists for callers that cannot let a call allocate (a
    memory budget or caching allocator that owns all device memory, a loop
    that cannot take an allocation's implicit synchronization), so the device's
    free memory must not change across its calls on a fresh plan, whose own
    lazily allocated scratch buffers are all still empty.  A first call on an
    earlier plan comes before the measurement: loading the library's device
    code (which holds the fixed array) is not an allocation by the call."""
    torch = need_torch_cuda()
    w = CASES[1]
    V = synth.potential(w)
    phi = _spinor(w)
    warm = make_plan(w, V, phi)
    mu_ref = warm.chemical_potentials_noalloc()
    fresh = make_plan(w, V, phi, mu=(1.0, 2.0, 3.0))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        np.testing.assert_allclose(fresh.chemical_potentials_noalloc(), mu_ref, rtol=1e-12, atol=0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    warm.close()
    fresh.close()


def test_noalloc_vanishing_component():
    """A polar spinor (phi_1 = phi_-1 = 0): mu_+-1 come from mu_1 + mu_-1 = 2 mu_0."""
    need_torch_cuda()
    w = CASES[0]
    V = synth.potential(w)
    phi = _spinor(w)
    phi[0] = 0.0
    phi[2] = 0.0
    plan = make_plan(w, V, phi)
    mu_ref = plan.mu
    for _ in range(2):
        np.testing.assert_allclose(plan.chemical_potentials_noalloc(), mu_ref, rtol=1e-12, atol=0)
    plan.close()


def test_noalloc_rejects_large_grid():
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = synth.Workload("na_big", (256, 128), (-8.0, -8.0), (8.0, 8.0), (1.0, 1.0), 10.0, -1.0)
    plan = make_plan(w, synth.potential(w), _spinor(w), mu=(1.0, 1.0, 1.0))
    with pytest.raises(bdg.BdgError) as e:
        plan.chemical_potentials_noalloc()
    assert e.value.status == bdg.ERR_UNSUPPORTED
    assert "16384" in str(e.value)
    plan.close()
