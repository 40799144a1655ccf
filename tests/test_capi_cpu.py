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
