"""Host-side checks of the C ABI (no GPU): the library builds, loads, and
exports every function include/bdg.h declares; the Python binding's struct
matches the header's field order; argument errors that the host side
rejects before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_2506_08308_gb300 import build, bdg
    build.build()
    return bdg.load()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "bdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bdg_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert "bdg_apply" in names and "bdg_solve" in names
    for name in names:
        assert hasattr(lib, name), name
    from paper_2506_08308_gb300 import bdg
    assert sorted(bdg.EXPORTS) == names


def test_params_struct_matches_header():
    from paper_2506_08308_gb300 import bdg
    src = open(os.path.join(ROOT, "include", "bdg.h")).read()
    body = src[src.index("typedef struct {"):src.index("} bdg_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([a-z_]+)(?:\[3\])?\s*[;,]", body)
    assert [f for f, _ in bdg.Params._fields_] == fields


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2506_08308_gb300 import bdg
    import numpy as np
    # bad grid size: rejected before any device work
    prm = bdg.make_params((12,), (-1.0,), (1.0,), 1.0, 0.0)
    with pytest.raises(bdg.BdgError) as e:
        bdg.Plan(prm, np.zeros(12), np.zeros(36))
    assert e.value.status == bdg.ERR_INVALID
    prm = bdg.make_params((16,), (1.0,), (-1.0,), 1.0, 0.0)
    with pytest.raises(bdg.BdgError) as e:
        bdg.Plan(prm, np.zeros(16), np.zeros(48))
    assert e.value.status == bdg.ERR_INVALID
    prm = bdg.make_params((16,), (-1.0,), (1.0,), float("nan"), 0.0)
    with pytest.raises(bdg.BdgError) as e:
        bdg.Plan(prm, np.zeros(16), np.zeros(48))
    assert e.value.status == bdg.ERR_INVALID
    prm = bdg.make_params((2048,), (-1.0,), (1.0,), 1.0, 0.0)
    with pytest.raises(bdg.BdgError) as e:
        bdg.Plan(prm, np.zeros(2048), np.zeros(3 * 2048))
    assert e.value.status == bdg.ERR_UNSUPPORTED
    # NULL plan
    assert lib.bdg_apply(None, 0, 0, None, None, 1, None) == bdg.ERR_INVALID
    assert lib.bdg_plan_destroy(None) == bdg.OK
    assert b"plan is NULL" in lib.bdg_last_error(None)


def test_null_and_range_checks_of_every_entry_point(lib):
    """Argument checks that run before any device work, for the entry points
    added after the product: solve, bi-orthonormalisation, ground state, the
    allocation-free chemical potentials and the perturbed densities."""
    import ctypes
    from paper_2506_08308_gb300 import bdg
    import numpy as np
    nconv = ctypes.c_int(0)
    rank = ctypes.c_int(0)
    om = np.zeros(4)
    assert lib.bdg_solve(None, 4, 8, None, bdg._dptr(om), None, None, ctypes.byref(nconv), None) == bdg.ERR_INVALID
    assert lib.bdg_biortho(None, bdg.C128, None, None, 4, None, None, 0, ctypes.byref(rank), None) == bdg.ERR_INVALID
    assert lib.bdg_chemical_potentials_noalloc(None, bdg._dptr(np.zeros(3)), None) == bdg.ERR_INVALID
    t1 = np.zeros(1)
    assert lib.bdg_perturbed_density(None, bdg.C128, None, 1, bdg._dptr(t1), bdg._dptr(t1), 1, 0.1, None,
                                     None) == bdg.ERR_INVALID
    prm = bdg.make_params((16,), (-4.0,), (4.0,), 1.0, 0.0)
    V, phi0 = np.zeros(16), np.ones(48)
    out, mu, res = np.zeros(48), np.zeros(3), np.zeros(1)
    it = ctypes.c_int(0)
    # magnetisation outside (-1, 1) and a non-positive tolerance are refused on the host
    assert lib.bdg_ground_state(ctypes.byref(prm), 1.5, bdg._dptr(V), bdg._dptr(phi0), 1e-12, 10, bdg._dptr(out),
                                bdg._dptr(mu), bdg._dptr(res), ctypes.byref(it), None) == bdg.ERR_INVALID
    assert lib.bdg_ground_state(ctypes.byref(prm), 0.0, bdg._dptr(V), bdg._dptr(phi0), 0.0, 10, bdg._dptr(out),
                                bdg._dptr(mu), bdg._dptr(res), ctypes.byref(it), None) == bdg.ERR_INVALID
    assert lib.bdg_ground_state(None, 0.0, None, None, 1e-12, 10, None, None, None, None, None) == bdg.ERR_INVALID


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """The package has no CPU path: without libbdg.so every call raises."""
    from paper_2506_08308_gb300 import bdg
    monkeypatch.setattr(bdg, "LIBPATH", str(tmp_path / "libbdg.so"))
    monkeypatch.setattr(bdg, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        bdg.load()


def test_output_tensor_checks_of_the_binding():
    """The binding refuses a caller-supplied output tensor whose shape, dtype,
    device or layout differ from what the library will write."""
    torch = pytest.importorskip("torch")
    from paper_2506_08308_gb300 import bdg
    good = torch.empty((2, 1, 3, 8), dtype=torch.float64)
    bdg._check_out(good, (2, 1, 3, 8), torch.float64, good.device)
    for bad, why in ((torch.empty((2, 1, 3, 7), dtype=torch.float64), "shape"),
                     (torch.empty((2, 1, 3, 8), dtype=torch.float32), "dtype"),
                     (torch.empty((2, 1, 8, 3), dtype=torch.float64).transpose(2, 3), "layout")):
        with pytest.raises(ValueError):
            bdg._check_out(bad, (2, 1, 3, 8), torch.float64, good.device)
    with pytest.raises(ValueError):
        bdg._check_out(good, (2, 1, 3, 8), torch.float64, torch.device("meta"))


def test_binding_checks_blocks_before_the_library():
    """biortho and solve check the blocks they hand to the library (device,
    dtype, exact shape, contiguity) before any call: exercised on a plan
    object that has no library handle, so any call through would fail."""
    torch = pytest.importorskip("torch")
    from paper_2506_08308_gb300 import bdg
    p = bdg.Plan.__new__(bdg.Plan)
    p.npts, p.lib, p.handle = 8, None, None
    cpu = torch.zeros((2, 3, 8), dtype=torch.complex128)
    with pytest.raises(ValueError):
        p.biortho(cpu, cpu.clone())
    with pytest.raises(ValueError):
        p.biortho(torch.zeros((2, 3, 8), dtype=torch.float64), cpu)
    with pytest.raises(ValueError):
        p.solve(2, 4, X0=torch.zeros((4, 6, 8), dtype=torch.complex128), want_vectors=False)
    # a locked pair needs both halves: Gl alone (or Fl alone) is refused
    # rather than silently dropped
    for kw in ({"Gl": cpu}, {"Fl": cpu}):
        with pytest.raises(ValueError, match="Fl and Gl go together"):
            p.biortho(cpu, cpu.clone(), **kw)


def test_gram_and_batched_checks_on_the_host(lib):
    """bdg_gram refuses a bad dtype or engine, negative sizes, a column stride
    below the column length, NULL blocks with rows to sum and a tensor-core
    B block wider than 160 real columns, and is a no-op for empty blocks;
    bdg_solve_batched refuses NULL arrays; the binding checks the blocks'
    types and shapes before calling the library.  None of this touches a
    device."""
    import numpy as np
    import torch
    from paper_2506_08308_gb300 import bdg
    G = np.zeros(64)
    g = bdg._dptr(G)
    one = ctypes.c_void_p(1)   # never dereferenced: every case below fails before device work
    assert lib.bdg_gram(7, bdg.GRAM_SIMT, one, 10, 2, one, 10, 2, 10, g, None) == bdg.ERR_INVALID
    assert lib.bdg_gram(bdg.C128, 5, one, 10, 2, one, 10, 2, 10, g, None) == bdg.ERR_INVALID
    assert lib.bdg_gram(bdg.C128, bdg.GRAM_SIMT, one, 10, -1, one, 10, 2, 10, g, None) == bdg.ERR_INVALID
    assert lib.bdg_gram(bdg.C128, bdg.GRAM_SIMT, one, 5, 2, one, 10, 2, 10, g, None) == bdg.ERR_INVALID
    assert lib.bdg_gram(bdg.C128, bdg.GRAM_SIMT, None, 10, 2, one, 10, 2, 10, g, None) == bdg.ERR_INVALID
    assert lib.bdg_gram(bdg.C64, bdg.GRAM_TENSOR, one, 10, 2, one, 10, 81, 10, g, None) == bdg.ERR_UNSUPPORTED
    assert lib.bdg_gram(bdg.C128, bdg.GRAM_SIMT, None, 0, 0, None, 0, 3, 10, g, None) == bdg.OK
    nconv = (ctypes.c_int * 1)()
    assert lib.bdg_solve_batched(None, 1, None, None, None, None, None, nconv, None) == bdg.ERR_INVALID
    assert lib.bdg_solve_batched(None, 0, None, None, None, None, None, None, None) == bdg.OK
    A = torch.zeros((2, 8), dtype=torch.complex64)
    B = torch.zeros((2, 8), dtype=torch.complex128)
    with pytest.raises(ValueError):
        bdg.gram(A, B)                      # mixed dtypes
    with pytest.raises(ValueError):
        bdg.gram(A, A[:, :4])               # different column lengths
    with pytest.raises(ValueError):
        bdg.gram(A, A)                      # host tensors
