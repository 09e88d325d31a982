"""CPU checks of the C ABI: the library loads, exports every entry point that
include/ddtm.h declares, and validates arguments on the host."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_02370_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ddtm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ddtm_[a-z_A-Z0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("ddtm_create", "ddtm_load_gauge", "ddtm_apply_D", "ddtm_sap", "ddtm_setup",
                 "ddtm_build_coarse", "ddtm_apply_Dc", "ddtm_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_1610_02370_gb300 import ddtm
    assert set(declared_symbols()) <= set(ddtm.SIGNATURES)


def test_create_rejects_bad_geometry_without_touching_the_gpu(lib):
    from paper_1610_02370_gb300 import ddtm
    bad = [((6, 4, 4, 4), (4, 4, 4, 4)),   # 6 not divisible by 4
           ((4, 4, 4, 4), (4, 4, 4, 4)),   # one block per direction: no red-black colouring
           ((12, 8, 8, 8), (4, 4, 4, 4)),  # 3 blocks in t: odd count
           ((8, 8, 8, 8), (3, 4, 4, 4))]   # odd block extent
    for dims, block in bad:
        with pytest.raises(ddtm.DDTMError) as e:
            ddtm.ddtm_create(dims, block)
        assert e.value.code == ddtm.ERR_ARG


def test_default_params_are_table_1(lib):
    from paper_1610_02370_gb300 import ddtm
    p = ddtm.ddtm_default_params()
    assert (p.n_setup, p.nv[0], p.post_smooth, p.nmr) == (5, 28, 4, 3)
    assert (p.kcycle_restart, p.kcycle_max_restarts, p.kcycle_tol) == (5, 2, 0.1)
    assert (p.coarse_restart, p.coarse_max_restarts, p.coarse_tol, p.delta) == (100, 5, 0.1, 5.2)
    assert list(p.block[0]) == [4, 4, 4, 4] and list(p.block[1]) == [2, 2, 2, 2]


def test_binding_rejects_bad_buffers_on_the_host(lib):
    """The Python binding passes only C-contiguous complex128 buffers, refuses read-only outputs and
    mixed host / device arguments, before any library call."""
    import numpy as np

    from paper_1610_02370_gb300 import ddtm
    good = np.zeros((2, 3), dtype=np.complex128)
    p, loc = ddtm._buf(good)
    assert p == good.ctypes.data and loc == ddtm.LOC_HOST
    for bad in (np.zeros((2, 3)), np.zeros((3, 2), dtype=np.complex128).T, [1.0 + 0j]):
        with pytest.raises(TypeError):
            ddtm._buf(bad)
    ro = np.zeros(4, dtype=np.complex128)
    ro.flags.writeable = False
    ddtm._buf(ro)  # fine as an input
    with pytest.raises(TypeError):
        ddtm._buf(ro, writable=True)
    with pytest.raises(TypeError):
        ddtm._same_loc((1, ddtm.LOC_HOST), (2, ddtm.LOC_DEVICE))
    assert ddtm._same_loc((1, ddtm.LOC_DEVICE), (2, ddtm.LOC_DEVICE)) == ddtm.LOC_DEVICE
