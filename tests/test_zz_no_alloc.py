"""The batched launch that allocates no device memory (ext_batch_run_noalloc).

It exists for callers that cannot call cudaMalloc -- code running under a
device-memory budget owned by someone else, or loops that cannot take the
implicit synchronisation of an allocation.  It must give the same residual
and adjoint as the plan-based batched launch (ext_batch_create +
ext_batch_launch), within the tolerance the parity tests use, on two calls
in a row (the second call reuses the shared scratch array left by the
first).  This file is collected last on purpose."""
import numpy as np
import pytest

import meshgen
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1604_05937_gb300 as E  # noqa: E402

P1 = O.DELTA["CG1xCG1"]
dev = torch.device("cuda:0")


def test_noalloc_batch_matches_plan_two_calls():
    bp = meshgen.batched_params(count=6, seed=2100, cmin=40, cmax=2500, lmin=1, lmax=37)
    meshes, per, flat, absF, absG, keep = [], [], [], [], [], []
    for i, (n, L) in enumerate(zip(bp.n, bp.layers)):
        m = meshgen.tri_mesh(n, seed=2200 + i, order="random" if i % 2 else "rcm")
        gm = E.Mesh(m.cells, m.xy, L)
        cs = E.Space(gm, "CG1xCG1", ncomp=3)
        sp = E.Space(gm, "CG1xCG1")
        X = E.extrude_coords(gm, cs)
        u = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 2300 + i)).to(dev)
        w = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 2400 + i)).to(dev)
        Fp, Gp, Fn, Gn = (sp.zeros() for _ in range(4))
        per.append([(cs, X, E.EXT_READ), (sp, u, E.EXT_READ), (sp, w, E.EXT_READ), (sp, Fp, E.EXT_INC),
                    (sp, Gp, E.EXT_INC)])
        flat += [(cs.handle, X, E.EXT_READ), (sp.handle, u, E.EXT_READ), (sp.handle, w, E.EXT_READ),
                 (sp.handle, Fn, E.EXT_INC), (sp.handle, Gn, E.EXT_INC)]
        meshes.append(gm)
        keep.append((cs, sp, X, u, w, Fp, Gp, Fn, Gn))
        # absolute contribution sums from the oracle set the tolerance scale
        csp, Xo = O.coords(m.cells, m.xy, L)
        osp = O.number(m.cells, m.nverts, L, P1)
        uo, wo = u.cpu().numpy(), w.cpu().numpy()
        aF, aG, tF, tG = (np.zeros(osp.ndofs) for _ in range(4))
        O.par_loop(O.K_U2V, m.cells, L, [(csp, Xo, 3, O.READ), (osp, uo, 1, O.READ), (osp, tF, 1, O.INC, aF)])
        O.par_loop(O.K_U2V_ADJ, m.cells, L, [(csp, Xo, 3, O.READ), (osp, uo, 1, O.READ), (osp, wo, 1, O.READ),
                                             (osp, tG, 1, O.INC, aG)])
        absF.append(aF)
        absG.append(aG)

    params = dict(cols_per_item=4, layer_tile=0, use_atomics=1, threads=256, ctas_per_sm=4)
    plan = E.Batch(meshes, E.EXT_K_U2V_FWDADJ, per, params=params)
    for k in keep:
        k[5].zero_()
        k[6].zero_()
    plan.launch()
    torch.cuda.synchronize()
    handles = [m.handle for m in meshes]
    for call in range(2):
        for k in keep:
            k[7].zero_()
            k[8].zero_()
        E.ext_batch_run_noalloc(handles, E.EXT_K_U2V_FWDADJ, 5, flat, params=None if call else params)
        E.ext_sync_check()
        for i, k in enumerate(keep):
            Fp, Gp, Fn, Gn = (t.cpu().numpy() for t in k[5:9])
            assert np.all(np.abs(Fn - Fp) <= 1e-12 * absF[i] + 1e-300), (call, i)
            assert np.all(np.abs(Gn - Gp) <= 1e-12 * absG[i] + 1e-300), (call, i)
    assert float(torch.stack([k[7].abs().sum() for k in keep]).sum()) > 0


def test_noalloc_rejects_oversized_batch_and_colours():
    m = meshgen.tri_mesh(2, seed=1)
    gm = E.Mesh(m.cells, m.xy, 2)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, "CG1xCG1")
    X = E.extrude_coords(gm, cs)
    u, F = sp.zeros(), sp.zeros()
    args = [(cs.handle, X, E.EXT_READ), (sp.handle, u, E.EXT_READ), (sp.handle, F, E.EXT_INC)]
    n = E.EXT_NOALLOC_MAX_MESHES + 1
    with pytest.raises(E.ExtError, match="limit"):
        E.ext_batch_run_noalloc([gm.handle] * n, E.EXT_K_U2V_FWD, 3, args * n)
    with pytest.raises(E.ExtError, match="EXT_EUNSUPPORTED"):
        E.ext_batch_run_noalloc([gm.handle], E.EXT_K_U2V_FWD, 3, args,
                                params=dict(cols_per_item=32, layer_tile=0, use_atomics=0, threads=256,
                                            ctas_per_sm=2))


def test_noalloc_and_plan_reject_overlapping_outputs():
    """The batched entry points check, per mesh, that no written argument
    overlaps another one: with the forward and adjoint outputs in one buffer
    both the plan and the allocation-free launch fail with EXT_EINVAL before
    launching anything."""
    m = meshgen.tri_mesh(6, seed=2500, order="rcm")
    gm = E.Mesh(m.cells, m.xy, 3)
    cs = E.Space(gm, "CG1xCG1", ncomp=3)
    sp = E.Space(gm, "CG1xCG1")
    X = E.extrude_coords(gm, cs)
    u = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 2501)).to(dev)
    w = torch.from_numpy(meshgen.uniform_field(sp.ndofs, 2502)).to(dev)
    F = sp.zeros()
    args = [(cs.handle, X, E.EXT_READ), (sp.handle, u, E.EXT_READ), (sp.handle, w, E.EXT_READ),
            (sp.handle, F, E.EXT_INC), (sp.handle, F, E.EXT_INC)]
    with pytest.raises(E.ExtError, match="overlaps"):
        E.ext_batch_run_noalloc([gm.handle], E.EXT_K_U2V_FWDADJ, 5, args)
    with pytest.raises(E.ExtError, match="overlaps"):
        E.ext_batch_create([gm.handle], E.EXT_K_U2V_FWDADJ, 5, args, params=None)
    args[4] = (sp.handle, u, E.EXT_INC)  # the adjoint output aliasing the input u
    with pytest.raises(E.ExtError, match="overlaps"):
        E.ext_batch_run_noalloc([gm.handle], E.EXT_K_U2V_FWDADJ, 5, args)
