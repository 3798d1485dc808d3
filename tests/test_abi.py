"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every function declared in include/fsim.h (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fsim_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_24968_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fsim_basis_create", "fsim_schwarz", "fsim_fock_build", "fsim_scf"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2510_24968_gb300 import EXPORTS
    assert sorted(EXPORTS) == declared_functions()


def test_defaults_and_errors_without_gpu(lib):
    from paper_2510_24968_gb300 import fsim
    o = fsim.fsim_fock_opts_default()
    assert o.schwarz_tau == 1e-10 and o.precision == fsim.FSIM_FP64 and o.nshards == 1
    s = fsim.fsim_scf_opts_default()
    assert s.max_iter == 100 and s.diis_size == 8
    # argument validation happens before any device work
    L = fsim.load()
    assert L.fsim_fock_build(None, None, None, None, None) == fsim.FSIM_EINVAL
    assert b"null" in L.fsim_last_error()
    assert L.fsim_basis_nbf(None) == fsim.FSIM_EINVAL
