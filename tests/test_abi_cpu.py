"""The C-ABI library loads on a host without a GPU, exports every function
declared in include/*.h, and rejects bad arguments before touching the GPU."""
import ctypes
import glob
import os
import re

import pytest

import paper_2111_05651_gb300 as nsi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(nsi_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["nsi_assemble_create", "nsi_assemble", "nsi_assemble_batched", "nsi_assemble_vjp",
                     "nsi_assemble_destroy", "nsi_csr_pattern", "nsi_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = nsi.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(nsi.exported_symbols()) <= declared_functions()


def test_abi_version():
    assert nsi.nsi_abi_version() == 2


def test_struct_layouts_match_header():
    # sizes of the ABI structs on LP64 (x86_64 and aarch64 alike)
    assert ctypes.sizeof(nsi.NsiMesh) == 48
    assert ctypes.sizeof(nsi.NsiOptions) == 32
    assert ctypes.sizeof(nsi.NsiFields) == 72
    assert ctypes.sizeof(nsi.NsiOutputs) == 24
    assert ctypes.sizeof(nsi.NsiInfo) == 72


def test_null_arguments_rejected_without_gpu():
    lib = nsi.load_library()
    h = ctypes.c_void_p()
    opts = nsi.NsiOptions(0, 0, 0, 0)
    assert lib.nsi_assemble_create(None, ctypes.byref(opts), None, ctypes.byref(h)) == nsi.NSI_ERR_INVALID_ARG
    assert "NULL" in nsi.nsi_last_error()
    assert lib.nsi_assemble_create(None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    mesh = nsi.NsiMesh(0, 0, None, None, None, None)
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(opts), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    mesh = nsi.NsiMesh(4, 1, None, None, None, None)
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(opts), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    bad = nsi.NsiOptions(7, 0, 0, 0)
    mesh = nsi.NsiMesh(4, 1, 8, 8, 8, 8)   # non-NULL dummies: options are checked first
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(bad), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    bad = nsi.NsiOptions(0, 9, 0, 0)
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(bad), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    bad = nsi.NsiOptions(0, 0, 33, 0)
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(bad), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    bad = nsi.NsiOptions(0, 0, 0, 0, (ctypes.c_int32 * 4)(0, 1, 0, 0))
    assert lib.nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(bad), None, ctypes.byref(h)) == \
        nsi.NSI_ERR_INVALID_ARG
    assert h.value is None


def test_calls_on_null_handle():
    lib = nsi.load_library()
    f = nsi.NsiFields()
    o = nsi.NsiOutputs()
    assert lib.nsi_assemble(None, ctypes.byref(f), ctypes.byref(o), None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_mode(None, ctypes.byref(f), ctypes.byref(o), 0, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_vjp(None, ctypes.byref(f), None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_residual(None, ctypes.byref(f), None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_host(None, ctypes.byref(f), ctypes.byref(o), None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_csr_pattern(None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_info(None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_device_status(None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_set_launch(None, 0, 0) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_autotune(None, ctypes.byref(f), ctypes.byref(o), 3, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_noalloc(None, ctypes.byref(f), ctypes.byref(o), None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_convective(None, ctypes.byref(f), None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_nodal(None, ctypes.byref(f), None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_stabilized(None, ctypes.byref(f), None, None, None, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_destroy(None) == nsi.NSI_OK
    hs = (ctypes.c_void_p * 1)()
    assert lib.nsi_assemble_batched(hs, None, None, -1, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_batched(hs, None, None, nsi.NSI_MAX_BATCH + 1, None) == nsi.NSI_ERR_INVALID_ARG
    assert lib.nsi_assemble_batched(None, None, None, 0, None) == nsi.NSI_OK


def test_assembler_needs_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        nsi.Assembler([[0, 0, 0]], [[0, 0, 0, 0]])
