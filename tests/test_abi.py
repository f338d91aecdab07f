"""Host-side checks of the C ABI boundary (no GPU needed): the library builds
for sm_103a, loads, exports every function include/*.h declares, shares no
code with the oracle, and the binding refuses to import without it."""
import ctypes
import glob
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1604_05937_gb300")


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w ]*?[\s\*]+(ext_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    return __graft_entry__.build_library_only()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["ext_mesh_create", "ext_number_dofs", "ext_par_loop", "ext_batch_create", "ext_sync_check",
              "ext_last_error", "ext_space_info", "ext_mesh_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    L.ext_abi_version.restype = ctypes.c_int32
    assert L.ext_abi_version() == 1


def test_validation_needs_no_gpu(libpath):
    """Argument checks run on the host before any CUDA call."""
    sys.path.insert(0, ROOT)
    import paper_1604_05937_gb300 as E
    import numpy as np
    cells = np.array([[0, 1, 2]], dtype=np.int32)
    xy = np.array([[0, 0], [1, 0], [0, 1]], dtype=np.float64)
    with pytest.raises(E.ExtError, match="EXT_EINVAL"):
        E.ext_mesh_create(3, 3, 1, cells, xy, 0)  # layers < 1
    with pytest.raises(E.ExtError, match="out of range"):
        E.ext_mesh_create(3, 3, 1, np.array([[0, 1, 5]], dtype=np.int32), xy, 2)
    with pytest.raises(E.ExtError, match="repeats vertex"):
        E.ext_mesh_create(3, 3, 1, np.array([[0, 1, 1]], dtype=np.int32), xy, 2)
    with pytest.raises(E.ExtError, match="clockwise"):
        E.ext_mesh_create(3, 3, 1, np.array([[0, 2, 1]], dtype=np.int32), xy, 2)
    with pytest.raises(E.ExtError, match="kind"):
        E.ext_mesh_create(5, 3, 1, cells, xy, 2)
    # variable layers: every cell spans at least one layer from a level >= 0,
    # and every vertex belongs to a cell
    with pytest.raises(E.ExtError, match="layers 0"):
        E.ext_mesh_create_var(3, 3, 1, cells, xy, np.array([0]), np.array([0]))
    with pytest.raises(E.ExtError, match="first -1"):
        E.ext_mesh_create_var(3, 3, 1, cells, xy, np.array([-1]), np.array([2]))
    with pytest.raises(E.ExtError, match="belongs to no cell"):
        E.ext_mesh_create_var(3, 4, 1, cells, np.vstack([xy, [[1.0, 1.0]]]), np.array([0]), np.array([2]))
    with pytest.raises(ValueError):
        E.ext_mesh_create_var(3, 3, 1, cells, xy, np.array([0, 0]), np.array([1, 1]))


def test_cuda_path_shares_no_code_with_oracle():
    for f in glob.glob(os.path.join(PKG, "**", "*"), recursive=True):
        if f.endswith((".cu", ".cuh", ".py", ".h")):
            txt = open(f).read()
            assert "oracle" not in txt.lower(), f
    out = subprocess.run(["nm", "-D", os.path.join(PKG, "libextmesh.so")], capture_output=True, text=True).stdout
    assert "oracle_" not in out


def test_binding_fails_loudly_without_library(tmp_path):
    dst = tmp_path / "paper_1604_05937_gb300"
    shutil.copytree(PKG, dst, ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1604_05937_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0
    assert "not built" in r.stderr
