"""Rows longer than the row gather takes (more than 32 entries): the rest of
the mesh stays on the row gather and those rows are computed by a second,
per-row kernel, in every row-gather entry point -- the assembly, the
cached-geometry time step, the nodal outputs, the batched call, the
allocation-free call and the host-buffer call -- each against the oracle.
The meshes are unstructured (Delaunay) with one node of 49 or 81 entries."""
import ctypes

import numpy as np
import pytest

import meshgen
import oracle
from tests._common import errors, vec_scaled_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


def _oracle_u(u, precision):
    return u if precision == "fp64" else u.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module", params=[(8, 48, 6), (6, 80, 7)], ids=["hub49", "hub81"])
def hub(request):
    m, k, seed = request.param
    return meshgen.delaunay_hub(m=m, k=k, seed=seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_long_rows_assembly_step_nodal(hub, precision):
    mesh, u = hub
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    info = asm.info()
    assert asm.max_row > 32 and info.long_rows >= 1
    assert asm.scatter == nsi.SCATTERS["gather"]  # the mesh stays on the row gather
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = (x.double().cpu().numpy() for x in asm.assemble(ut))
    A_static, _ = asm.static_part()
    A2, rhs2 = (x.double().cpu().numpy() for x in asm.assemble_convective(ut, A_static))
    r3, dtr, mr = (x.double().cpu().numpy() for x in asm.nodal(ut))
    rp, ci = (x.cpu().numpy() for x in asm.pattern())
    asm.close()
    uo = _oracle_u(u, precision)
    orp, oci, oA, oG, orhs = oracle.assemble(mesh.coord, mesh.lnods, uo, None, RHO, MU, DT)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], err
    err2 = errors(rp, A2, oG, rhs2, oA, oG, orhs)
    assert max(err2.values()) <= TOL[precision], err2
    onr, ondt, onm = oracle.nodal(mesh.coord, mesh.lnods, uo, RHO, DT)
    for k in range(3):
        assert vec_scaled_err(r3[k], onr[k]) <= TOL[precision]
    assert vec_scaled_err(dtr, ondt) <= TOL[precision] and vec_scaled_err(mr, onm) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
def test_long_rows_batched_noalloc_host(hub, precision):
    """The batched call (with a Kuhn cube beside the hub mesh), the
    allocation-free call and the host-buffer call give nsi_assemble's results
    bit for bit."""
    mesh, u = hub
    cube, uc = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=93)
    asms = [nsi.Assembler(x.coord, x.lnods, precision=precision) for x in (mesh, cube)]
    us = [torch.as_tensor(v.T.copy()) for v in (u, uc)]
    singles = [[t.clone() for t in a.assemble(v)] for a, v in zip(asms, us)]
    batched = nsi.assemble_batched(asms, us)
    torch.cuda.synchronize()
    for s_, b_ in zip(singles, batched):
        for x, y in zip(s_, b_):
            assert torch.equal(x, y)
    asm = asms[0]
    lib = nsi.load_library()
    fields, keep = asm.fields(us[0], None, RHO, MU, DT)
    outs = asm.empty_outputs()
    for t in outs:
        t.fill_(float("nan"))
    o = nsi.NsiOutputs(outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.nsi_assemble_noalloc(asm.handle, ctypes.byref(fields), ctypes.byref(o), stream) == nsi.NSI_OK
    torch.cuda.synchronize()
    for x, y in zip(outs, singles[0]):
        assert torch.equal(x, y)
    vt = torch.float64 if precision == "fp64" else torch.float32
    uh = us[0].to(vt).pin_memory()
    Ah = torch.empty(asm.nnz, dtype=asm.out_dtype).pin_memory()
    Gh = torch.empty(3, asm.nnz, dtype=asm.out_dtype).pin_memory()
    rh = torch.empty(3, asm.n, dtype=asm.out_dtype).pin_memory()
    asm.assemble_host(uh, Ah, Gh, rh)
    for x, y in zip((Ah, Gh, rh), singles[0]):
        assert torch.equal(x, y.cpu())
    for a in asms:
        a.close()
