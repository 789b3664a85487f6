"""CPU checks of the library boundary: it builds for sm_103a, exports every
entry point that include/ibim.h declares, validates arguments on the host,
and shares no code with the oracle."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(ibim_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1709_08070_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("ibim_build_sphere", "ibim_matvec", "ibim_solve", "ibim_energy", "ibim_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_host_side_argument_checks(built_lib):
    from paper_1709_08070_gb300 import ibim
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_build_sphere(-1.0, (0, 0, 0), None, 0.25, 0.5, stream=0)
    assert e.value.status == 1
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_build_sphere(1.0, (0, 0, 0), None, 0.0, 0.5, stream=0)
    assert e.value.status == 1
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_build_from_nodes([[float("nan"), 0, 0]], [[0, 0, 1]], [0.1], 0.25, stream=0)
    assert e.value.status == 3
    L = ibim.lib()
    assert L.ibim_num_nodes(None, None) == 1


def test_oracle_and_cuda_path_share_no_code():
    """The product package never imports the oracle; the oracle never includes
    or imports the package or its header."""
    pkg = os.path.join(ROOT, "paper_1709_08070_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
            src = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
            assert "oracle/" not in src and "ibim_oracle" not in src, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.*")):
        if f.endswith((".py", ".c", ".h")):
            src = open(f).read()
            assert "paper_1709_08070_gb300" not in src, f
            assert "ibim.h" not in src and "csrc" not in src, f
