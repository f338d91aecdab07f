"""Failure path of the one bounded wait in the library: the bulk-copy vertex
pass of the P1xP1 gather form waits on an mbarrier for its own copies.  The
test hook EXTMESH_TEST_BULK_SKIP=<step> (read once per process) makes the
first such launch leave out the copy of one warp step (no arrival on its
barrier either) and lowers the poll limit, so that warp's wait runs out with
no copy in flight.  The warp sets the device error word and returns;
ext_sync_check must report EXT_ETIMEOUT, and the next launch in the same
process must run normally and match the oracle.  No kernel faults, traps or
hangs: the wait is a bounded poll loop."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import meshgen
import oracle as O
import paper_1604_05937_gb300 as E
dev = torch.device("cuda:0")
m = meshgen.tri_mesh(71, seed=951, order="rcm")
L = 100
gm = E.Mesh(m.cells, m.xy, L)
cs = E.Space(gm, "CG1xCG1", ncomp=3)
ps = E.Space(gm, "CG1xCG1")
X = E.extrude_coords(gm, cs)
f = meshgen.uniform_field(ps.ndofs, 952)
fd = torch.from_numpy(f).to(dev)
E.ext_set_option(E.EXT_OPT_P1_FORM, E.EXT_P1_GATHER)
b = ps.zeros()
E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, fd, E.EXT_READ), (ps, b, E.EXT_WRITE))
try:
    E.ext_sync_check()
    print("NO-TIMEOUT")
except E.ExtError as e:
    print("STATUS", e.status)
b = ps.zeros()
E.par_loop(gm, E.EXT_K_MASS_P1P1, (cs, X, E.EXT_READ), (ps, fd, E.EXT_READ), (ps, b, E.EXT_WRITE))
E.ext_sync_check()
csp, Xo = O.coords(m.cells, m.xy, L)
osp = O.number(m.cells, m.nverts, L, O.DELTA["CG1xCG1"])
ref, absr = np.zeros(osp.ndofs), np.zeros(osp.ndofs)
O.par_loop(O.K_MASS, m.cells, L, [(csp, Xo, 3, O.READ), (osp, f, 1, O.READ), (osp, ref, 1, O.INC, absr)])
got = b.cpu().numpy()
ok = bool(np.all(np.abs(got - ref) <= 1e-12 * absr + 1e-300))
print("RECOVERED", ok)
"""


@pytest.mark.parametrize("step", [0, 5])
def test_bulk_wait_runs_out_and_library_recovers(step):
    import paper_1604_05937_gb300 as E
    # the two-pass flat gather runs the bulk-copy vertex pass
    env = dict(os.environ, EXTMESH_TEST_BULK_SKIP=str(step), EXTMESH_P1_FLAT="split")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert f"STATUS {E.EXT_ETIMEOUT}" in r.stdout, r.stdout
    assert "RECOVERED True" in r.stdout, r.stdout
