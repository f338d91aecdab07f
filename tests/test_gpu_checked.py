"""The checked build and ext_space_check.

libextmesh_checked.so (ext_api.cu compiled with EXT_CHECKED, loaded when
EXTMESH_CHECKED=1) range-checks on the device, before every ext_par_loop,
each index the launch will form from its arguments' stencil lists (and the
gather form's vertex rows), and launches nothing when one is out of range.
One parity pass runs under it.  ext_space_check runs the same check on one
space in either build; a map entry moved out of range on purpose must be
reported (EXT_EDEVICE) by ext_space_check first, and only then is a launch
tried with it, in the checked build, where it must be refused before any
kernel runs."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1604_05937_gb300 as E  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_parity_pass():
    env = dict(os.environ, EXTMESH_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "import paper_1604_05937_gb300 as E; print(E.LIB_PATH)"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("libextmesh_checked.so"), r.stdout + r.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                        os.path.join(ROOT, "tests", "test_gpu_var_facets.py"),
                        os.path.join(ROOT, "tests", "test_gpu_ragged.py"),
                        "-k", "not forced_form and not batched"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-3000:]
    assert " passed" in r.stdout


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found")


CHILD = r"""
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import meshgen
import paper_1604_05937_gb300 as E
m = meshgen.tri_mesh(8, seed=77, order="rcm")
gm = E.Mesh(m.cells, m.xy, 4)
cs = E.Space(gm, "CG1xCG1", ncomp=3)
ps = E.Space(gm, "CG1xCG1")
X = E.extrude_coords(gm, cs)
f = torch.ones(ps.ndofs, dtype=torch.float64, device="cuda")
info = E.ext_space_info(ps.handle)
ptr = info[3] + 4 * 5
rt = ctypes.CDLL(sys.argv[2])
old = ctypes.c_int32(0)
assert rt.cudaMemcpy(ctypes.byref(old), ctypes.c_void_p(ptr), ctypes.c_size_t(4), 2) == 0
bad = ctypes.c_int32(ps.ndofs + 7)
assert rt.cudaMemcpy(ctypes.c_void_p(ptr), ctypes.byref(bad), ctypes.c_size_t(4), 1) == 0
try:
    E.ext_space_check(ps.handle)
    print("CHECK-MISSED")
    sys.exit(1)
except E.ExtError as e:
    print("CHECK", e.status)
b = ps.zeros()
try:
    E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, f, E.EXT_READ), (ps, b, E.EXT_INC))
    print("LAUNCHED")
except E.ExtError as e:
    print("REFUSED", e.status)
assert rt.cudaMemcpy(ctypes.c_void_p(ptr), ctypes.byref(old), ctypes.c_size_t(4), 1) == 0
E.ext_space_check(ps.handle)
E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, f, E.EXT_READ), (ps, b, E.EXT_INC))
E.ext_sync_check()
print("SUM", float(b.sum()))
"""


def test_space_check_and_checked_launch_refuse_out_of_range_entry():
    rt = _cudart()
    name = os.path.basename(rt._name)
    env = dict(os.environ, EXTMESH_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, name], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr[-2000:]
    assert f"CHECK {E.EXT_EDEVICE}" in r.stdout
    assert f"REFUSED {E.EXT_EDEVICE}" in r.stdout
    total = float(r.stdout.split("SUM")[1].split()[0])
    assert abs(total - 1.0) < 1e-12  # int 1 v over the unit cube
