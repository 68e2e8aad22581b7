"""The allocation-free assembly entry point, through the C ABI.

Some callers cannot allocate device memory while they run (a plugin with a
fixed memory budget, a real-time loop, a host that owns every allocation).
nsi_assemble_noalloc serves them: it must give the same A, G and rhs as
nsi_assemble, call after call, without allocating, and refuse meshes whose
node records do not fit its static scratch.  This file is collected last so
that a stop-at-first-failure run has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import meshgen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}


def _noalloc(lib, asm, fields, outs, stream):
    o = nsi.NsiOutputs(outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr())
    return lib.nsi_assemble_noalloc(asm.handle, ctypes.byref(fields), ctypes.byref(o), stream)


def _close(got, ref, tol):
    scale = max(float(ref.abs().max()), 1e-300)
    return float((got.double() - ref.double()).abs().max()) <= tol * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_noalloc_matches_assemble_two_calls(precision):
    lib = nsi.load_library()
    mesh, u = meshgen.config_mesh(N=12, jitter=0.15, numbering="random", seed=61)
    u2 = meshgen.add_noise(u, 0.3, np.random.default_rng(62))
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter="gather")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, uu in enumerate((u, u2)):
        ut = torch.as_tensor(uu.T.copy())
        ref = [t.clone() for t in asm.assemble(ut, rho=1.0, mu=1e-3, dt=1e-2)]
        fields, keep = asm.fields(ut, None, 1.0, 1e-3, 1e-2)
        outs = asm.empty_outputs()
        for t in outs:
            t.fill_(float("nan"))  # every entry must be written by the call
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        status = _noalloc(lib, asm, fields, outs, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert status == nsi.NSI_OK, lib.nsi_last_error().decode()
        if call == 1:
            assert free_after == free_before  # nothing allocated on a later call
        for got, want in zip(outs, ref):
            assert not torch.isnan(got).any()
            assert _close(got, want, TOL[precision])
            assert torch.equal(got, want)  # same kernels, same order: bit-identical
    asm.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    lib = nsi.load_library()
    mesh, u = meshgen.config_mesh(N=64, jitter=0.0, numbering="natural", seed=63)  # 274,625 nodes
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="fp64", scatter="gather")
    ut = torch.as_tensor(u.T.copy())
    fields, keep = asm.fields(ut, None, 1.0, 1e-3, 1e-2)
    outs = asm.empty_outputs()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = _noalloc(lib, asm, fields, outs, stream)
    assert status == nsi.NSI_ERR_UNSUPPORTED
    msg = lib.nsi_last_error().decode()
    assert "274625 nodes" in msg and "scratch" in msg
    asm.close()


def _sliver_mesh():
    """4^3 Kuhn cube with node (2,2,2) moved by 0.499 h along (1,-1,0): two
    slivers whose rows the mixed modes recompute in double after the kernel."""
    mesh, u = meshgen.config_mesh(N=4, jitter=0.0, numbering="natural", seed=0)
    coord = mesh.coord.copy()
    coord[2 + 5 * (2 + 5 * 2)] += 0.499 * 0.25 * np.array([1.0, -1.0, 0.0])
    return meshgen.Mesh(coord=coord, lnods=mesh.lnods, N=4), u


@pytest.mark.parametrize("precision", ["mixed64", "mixed32"])
@pytest.mark.parametrize("launch", ["fan", "star-debug"])
def test_noalloc_same_kernels_and_fixup(precision, launch):
    """The allocation-free call runs whatever nsi_assemble runs for the handle:
    the edge-fan kernel when nsi_set_launch(-1) selected it, the bounds-checked
    kernels of a debug handle, and in both cases the double-precision rows of
    badly shaped elements afterwards."""
    lib = nsi.load_library()
    mesh, u = _sliver_mesh()
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter="gather",
                        debug_checks=(launch == "star-debug"))
    assert asm.info().exact_rows > 0
    if launch == "fan":
        nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_GATHER, -1)
        assert asm.info().rows_per_block == -1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    u2 = meshgen.add_noise(u, 0.3, np.random.default_rng(64))
    for uu in (u, u2):
        ut = torch.as_tensor(uu.T.copy())
        ref = [t.clone() for t in asm.assemble(ut)]
        fields, keep = asm.fields(ut, None, 1.0, 1e-3, 1e-2)
        outs = asm.empty_outputs()
        for t in outs:
            t.fill_(float("nan"))
        status = _noalloc(lib, asm, fields, outs, stream)
        torch.cuda.synchronize()
        assert status == nsi.NSI_OK, lib.nsi_last_error().decode()
        for got, want in zip(outs, ref):
            assert torch.equal(got, want)
    asm.device_status()  # raises if a device-side bounds check fired
    asm.close()
