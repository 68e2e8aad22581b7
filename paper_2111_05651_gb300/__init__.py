"""GB300-native P1 tetrahedral incompressible-flow matrix assembly.

A thin Python binding over the C ABI of ``libnsi_assemble.so`` (declared in
``include/nsi_assemble.h``).  Every step of the assembly runs in the library's
CUDA kernels; this module only marshals arguments.  PyTorch supplies device
memory and streams.  There is no CPU fallback: importing works without a GPU,
but every compute call needs the compiled library and a CUDA device and
raises otherwise.

Low-level functions keep the C names (``nsi_assemble_create``,
``nsi_assemble``, ``nsi_assemble_batched``, ``nsi_assemble_vjp``,
``nsi_assemble_destroy``, ...) and take ctypes structures; the ``Assembler``
class wraps them for torch tensors, and ``NsiResidual`` is the
``torch.autograd.Function`` of the assembled residual.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "NSI_OK", "NSI_FP64", "NSI_MIXED_F32_ACC64", "NSI_MIXED_F32_ACC32",
    "NSI_SCATTER_AUTO", "NSI_SCATTER_COLOR", "NSI_SCATTER_ATOMIC", "NSI_SCATTER_GATHER",
    "NsiMesh", "NsiOptions", "NsiFields", "NsiOutputs", "NsiInfo", "NsiError",
    "load_library", "library_path", "exported_symbols",
    "nsi_assemble_create", "nsi_assemble_destroy", "nsi_csr_pattern", "nsi_csr_pattern_copy", "nsi_info",
    "nsi_assemble", "nsi_assemble_mode", "nsi_assemble_batched", "nsi_assemble_vjp", "nsi_assemble_host",
    "nsi_assemble_convective", "nsi_assemble_nodal", "nsi_assemble_stabilized",
    "nsi_residual", "nsi_device_status", "nsi_set_timing_events", "nsi_autotune", "nsi_set_launch",
    "nsi_last_error", "nsi_abi_version",
    "Assembler", "NsiResidual", "assemble_batched",
]

# enums (include/nsi_assemble.h)
NSI_OK, NSI_ERR_INVALID_ARG, NSI_ERR_BAD_MESH, NSI_ERR_CUDA = 0, 1, 2, 3
NSI_ERR_OOM, NSI_ERR_UNSUPPORTED, NSI_ERR_TIMEOUT, NSI_ERR_DEVICE_CHECK = 4, 5, 6, 7
NSI_FP64, NSI_MIXED_F32_ACC64, NSI_MIXED_F32_ACC32 = 0, 1, 2
NSI_SCATTER_AUTO, NSI_SCATTER_COLOR, NSI_SCATTER_ATOMIC, NSI_SCATTER_GATHER = 0, 1, 2, 3
NSI_MAX_BATCH = 128
PRECISIONS = {"fp64": NSI_FP64, "mixed64": NSI_MIXED_F32_ACC64, "mixed32": NSI_MIXED_F32_ACC32}
SCATTERS = {"auto": NSI_SCATTER_AUTO, "color": NSI_SCATTER_COLOR, "atomic": NSI_SCATTER_ATOMIC,
            "gather": NSI_SCATTER_GATHER}

_STATUS = {0: "NSI_OK", 1: "NSI_ERR_INVALID_ARG", 2: "NSI_ERR_BAD_MESH", 3: "NSI_ERR_CUDA", 4: "NSI_ERR_OOM",
           5: "NSI_ERR_UNSUPPORTED", 6: "NSI_ERR_TIMEOUT", 7: "NSI_ERR_DEVICE_CHECK"}


class NsiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class NsiMesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64), ("lnods", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p)]


class NsiOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("scatter", ctypes.c_int32), ("block", ctypes.c_int32),
                ("debug_checks", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class NsiFields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p * 3), ("u_n", ctypes.c_void_p * 3), ("rho", ctypes.c_double),
                ("mu", ctypes.c_double), ("dt", ctypes.c_double)]


class NsiOutputs(ctypes.Structure):
    _fields_ = [("A_val", ctypes.c_void_p), ("G_val", ctypes.c_void_p), ("rhs", ctypes.c_void_p)]


class NsiInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_elems", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_colors", ctypes.c_int32), ("max_row", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("scatter", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("rows_per_block", ctypes.c_int32),
                ("n_plans", ctypes.c_int32), ("persistent", ctypes.c_int32), ("exact_rows", ctypes.c_int32),
                ("long_rows", ctypes.c_int32), ("fan_ok", ctypes.c_int32)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "nsi_assemble_create": [ctypes.POINTER(NsiMesh), ctypes.POINTER(NsiOptions), _P, ctypes.POINTER(_P)],
    "nsi_assemble_destroy": [_P],
    "nsi_csr_pattern": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int64)],
    "nsi_csr_pattern_copy": [_P, _P, _P, _P],
    "nsi_info": [_P, ctypes.POINTER(NsiInfo)],
    "nsi_assemble": [_P, ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs), _P],
    "nsi_assemble_mode": [_P, ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs), ctypes.c_int32, _P],
    "nsi_assemble_batched": [ctypes.POINTER(_P), ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs),
                             ctypes.c_int32, _P],
    "nsi_assemble_vjp": [_P, ctypes.POINTER(NsiFields), _P, _P, _P, _P],
    "nsi_assemble_convective": [_P, ctypes.POINTER(NsiFields), _P, _P, _P, _P],
    "nsi_assemble_nodal": [_P, ctypes.POINTER(NsiFields), _P, _P, _P, _P],
    "nsi_assemble_stabilized": [_P, ctypes.POINTER(NsiFields), _P, _P, _P, _P],
    "nsi_assemble_host": [_P, ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs), _P],
    "nsi_residual": [_P, ctypes.POINTER(NsiFields), _P, _P],
    "nsi_device_status": [_P, _P],
    "nsi_set_timing_events": [_P, _P, _P],
    "nsi_assemble_noalloc": [_P, ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs), _P],
    "nsi_autotune": [_P, ctypes.POINTER(NsiFields), ctypes.POINTER(NsiOutputs), ctypes.c_int32, _P,
                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "nsi_set_launch": [_P, ctypes.c_int32, ctypes.c_int32],
    "nsi_gather_values": [ctypes.POINTER(_P), ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int32, _P],
    "nsi_add_values": [ctypes.POINTER(_P), ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int32, _P],
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library(build: bool = True):
    """Load (building first if needed) the CUDA library; raises if it cannot be built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libnsi_assemble.so is missing ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, argt in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_int
            lib.nsi_last_error.restype = ctypes.c_char_p
            lib.nsi_last_error.argtypes = []
            lib.nsi_abi_version.restype = ctypes.c_int32
            lib.nsi_abi_version.argtypes = []
            _lib = lib
    return _lib


def exported_symbols():
    """Names of the ABI functions the binding expects the library to export."""
    return sorted(list(_SIGNATURES) + ["nsi_last_error", "nsi_abi_version"])


def _check(status):
    if status != NSI_OK:
        raise NsiError(status, load_library(build=False).nsi_last_error().decode())


# ------------------------------------------------------------ C-named calls --
def nsi_last_error() -> str:
    return load_library().nsi_last_error().decode()


def nsi_abi_version() -> int:
    return int(load_library().nsi_abi_version())


def nsi_assemble_create(mesh: NsiMesh, opts: NsiOptions, stream=None):
    h = _P()
    _check(load_library().nsi_assemble_create(ctypes.byref(mesh), ctypes.byref(opts), stream, ctypes.byref(h)))
    return h


def nsi_assemble_destroy(h):
    _check(load_library().nsi_assemble_destroy(h))


def nsi_csr_pattern(h):
    rp, ci, nnz = _P(), _P(), ctypes.c_int64()
    _check(load_library().nsi_csr_pattern(h, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz)))
    return rp.value, ci.value, nnz.value


def nsi_csr_pattern_copy(h, row_ptr_ptr, col_idx_ptr, stream=None):
    _check(load_library().nsi_csr_pattern_copy(h, row_ptr_ptr, col_idx_ptr, stream))


def nsi_info(h) -> NsiInfo:
    info = NsiInfo()
    _check(load_library().nsi_info(h, ctypes.byref(info)))
    return info


def nsi_assemble(h, fields: NsiFields, outputs: NsiOutputs, stream=None):
    _check(load_library().nsi_assemble(h, ctypes.byref(fields), ctypes.byref(outputs), stream))


def nsi_assemble_mode(h, fields: NsiFields, outputs: NsiOutputs, scatter: int, stream=None):
    _check(load_library().nsi_assemble_mode(h, ctypes.byref(fields), ctypes.byref(outputs), scatter, stream))


def nsi_assemble_batched(handles, fields, outputs, stream=None):
    count = len(handles)
    hs = (_P * max(count, 1))(*[h.value if isinstance(h, _P) else h for h in handles])
    fs = (NsiFields * max(count, 1))(*fields)
    os_ = (NsiOutputs * max(count, 1))(*outputs)
    _check(load_library().nsi_assemble_batched(hs, fs, os_, count, stream))


def nsi_assemble_vjp(h, fields: NsiFields, w_ptr, grad_u_ptr, grad_mu_ptr, stream=None):
    _check(load_library().nsi_assemble_vjp(h, ctypes.byref(fields), w_ptr, grad_u_ptr, grad_mu_ptr, stream))


def nsi_assemble_convective(h, fields: NsiFields, A_static_ptr, A_ptr, rhs_ptr, stream=None):
    _check(load_library().nsi_assemble_convective(h, ctypes.byref(fields), A_static_ptr, A_ptr, rhs_ptr, stream))


def nsi_assemble_nodal(h, fields: NsiFields, rhs_ptr, dt_rho_ptr, mass_rho_ptr, stream=None):
    _check(load_library().nsi_assemble_nodal(h, ctypes.byref(fields), rhs_ptr, dt_rho_ptr, mass_rho_ptr, stream))


def nsi_assemble_stabilized(h, fields: NsiFields, Auu_ptr, G_ptr, rhs_ptr, stream=None):
    _check(load_library().nsi_assemble_stabilized(h, ctypes.byref(fields), Auu_ptr, G_ptr, rhs_ptr, stream))


def nsi_assemble_host(h, fields: NsiFields, outputs: NsiOutputs, stream=None):
    _check(load_library().nsi_assemble_host(h, ctypes.byref(fields), ctypes.byref(outputs), stream))


def nsi_residual(h, fields: NsiFields, r_ptr, stream=None):
    _check(load_library().nsi_residual(h, ctypes.byref(fields), r_ptr, stream))


def nsi_autotune(h, fields: NsiFields, outputs: NsiOutputs, reps=5, stream=None):
    sc, rows = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().nsi_autotune(h, ctypes.byref(fields), ctypes.byref(outputs), reps, stream,
                                       ctypes.byref(sc), ctypes.byref(rows)))
    return sc.value, rows.value


def nsi_set_launch(h, scatter, rows_per_block):
    _check(load_library().nsi_set_launch(h, scatter, rows_per_block))


def nsi_set_timing_events(h, start_event_ptr, stop_event_ptr):
    _check(load_library().nsi_set_timing_events(h, start_event_ptr, stop_event_ptr))


def nsi_device_status(h, stream=None):
    _check(load_library().nsi_device_status(h, stream))


# --------------------------------------------------------------- torch layer --
def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Assembler:
    """One mesh on the GPU: CSR pattern and gather maps built once, then
    ``assemble(u)`` -> (A [nnz], G [3, nnz], rhs [3, n]) as torch tensors.

    coord: float64 tensor [n, 3] (or a tuple of three [n] tensors); lnods:
    int32 tensor [E, 4], 0-based.  Both are copied to the GPU if needed.
    precision: 'fp64' | 'mixed64' | 'mixed32'; scatter: 'auto' | 'gather' |
    'color' | 'atomic'.
    """

    def __init__(self, coord, lnods, precision="mixed64", scatter="auto", debug_checks=False, device=None,
                 stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("Assembler needs a CUDA device (no CPU fallback)")
        load_library()
        self.device = torch.device(device if device is not None else "cuda")
        if isinstance(coord, (tuple, list)):
            xyz = [torch.as_tensor(c, dtype=torch.float64).to(self.device).contiguous() for c in coord]
        else:
            c = torch.as_tensor(coord, dtype=torch.float64).to(self.device)
            xyz = [c[:, k].contiguous() for k in range(3)]
        ln = torch.as_tensor(lnods, dtype=torch.int32).to(self.device).contiguous()
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.scatter = SCATTERS[scatter] if isinstance(scatter, str) else int(scatter)
        self.vel_dtype = torch.float64 if self.precision == NSI_FP64 else torch.float32
        self.out_dtype = torch.float32 if self.precision == NSI_MIXED_F32_ACC32 else torch.float64
        mesh = NsiMesh(xyz[0].shape[0], ln.shape[0], ln.data_ptr(), xyz[0].data_ptr(), xyz[1].data_ptr(),
                       xyz[2].data_ptr())
        opts = NsiOptions(self.precision, self.scatter, 0, int(bool(debug_checks)))
        with torch.cuda.device(self.device):
            self.handle = nsi_assemble_create(mesh, opts, _stream_ptr(stream))
        info = nsi_info(self.handle)
        self.scatter = info.scatter  # the handle's default mode, resolved by the library
        self.n, self.E, self.nnz = info.n_nodes, info.n_elems, info.nnz
        self.n_colors, self.max_row, self.device_bytes = info.n_colors, info.max_row, info.device_bytes
        self._pattern = None

    def close(self):
        if getattr(self, "handle", None) is not None:
            nsi_assemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- pattern
    def pattern(self):
        """(row_ptr int32 [n+1], col_idx int32 [nnz]) as device tensors (copies)."""
        torch = _torch()
        if self._pattern is None:
            rp = torch.empty(self.n + 1, dtype=torch.int32, device=self.device)
            ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=self.device)
            nsi_csr_pattern_copy(self.handle, _ptr(rp), _ptr(ci), _stream_ptr(None))
            self._pattern = (rp, ci[: self.nnz])
        return self._pattern

    # ------------------------------------------------------------- marshal
    def _vel(self, u):
        torch = _torch()
        if isinstance(u, (tuple, list)):
            comps = [torch.as_tensor(c) for c in u]
        else:
            u = torch.as_tensor(u)
            comps = [u[k] for k in range(3)] if u.shape[0] == 3 and u.dim() == 2 else [u[:, k] for k in range(3)]
        out = []
        for c in comps:
            if c.device != self.device or c.dtype != self.vel_dtype or not c.is_contiguous():
                c = c.to(device=self.device, dtype=self.vel_dtype).contiguous()
            if c.numel() != self.n:
                raise ValueError("velocity component has the wrong length")
            out.append(c)
        return out

    def fields(self, u, u_n=None, rho=1.0, mu=1e-3, dt=1e-2):
        comps = self._vel(u)
        ncomps = self._vel(u_n) if u_n is not None else None
        f = NsiFields()
        for k in range(3):
            f.u[k] = comps[k].data_ptr()
            f.u_n[k] = ncomps[k].data_ptr() if ncomps is not None else None
        f.rho, f.mu, f.dt = float(rho), float(mu), float(dt)
        return f, (comps, ncomps)

    def empty_outputs(self):
        torch = _torch()
        A = torch.empty(self.nnz, dtype=self.out_dtype, device=self.device)
        G = torch.empty(3, self.nnz, dtype=self.out_dtype, device=self.device)
        rhs = torch.empty(3, self.n, dtype=self.out_dtype, device=self.device)
        return A, G, rhs

    # ----------------------------------------------------------------- calls
    def assemble(self, u, u_n=None, rho=1.0, mu=1e-3, dt=1e-2, out=None, scatter=None, stream=None):
        """Assemble (A, G, rhs) for nodal velocity u ([3, n], [n, 3] or 3 tensors)."""
        f, keep = self.fields(u, u_n, rho, mu, dt)
        A, G, rhs = out if out is not None else self.empty_outputs()
        o = NsiOutputs(A.data_ptr(), G.data_ptr(), rhs.data_ptr())
        mode = self.scatter if scatter is None else (SCATTERS[scatter] if isinstance(scatter, str) else scatter)
        nsi_assemble_mode(self.handle, f, o, mode, _stream_ptr(stream))
        return A, G, rhs

    def static_part(self, rho=1.0, mu=1e-3, dt=1e-2, out=None, stream=None):
        """(A_static, G): the velocity-independent assembly (A at u = 0: the viscous
        part plus the lumped mass; G), for ``assemble_convective``."""
        torch = _torch()
        zero = torch.zeros(3, self.n, dtype=self.vel_dtype, device=self.device)
        A, G, _ = self.assemble(zero, rho=rho, mu=mu, dt=dt, out=out, stream=stream)
        return A, G

    def assemble_convective(self, u, A_static, u_n=None, rho=1.0, mu=1e-3, dt=1e-2, out=None, stream=None):
        """(A, rhs) of one time step with cached geometry: A = A_static + C(u)."""
        torch = _torch()
        f, keep = self.fields(u, u_n, rho, mu, dt)
        if out is None:
            out = (torch.empty(self.nnz, dtype=self.out_dtype, device=self.device),
                   torch.empty(3, self.n, dtype=self.out_dtype, device=self.device))
        A, rhs = out
        if A_static.dtype != self.out_dtype or A_static.numel() != self.nnz or not A_static.is_contiguous():
            raise ValueError("A_static must be a contiguous [nnz] tensor of the output dtype")
        nsi_assemble_convective(self.handle, f, _ptr(A_static), _ptr(A), _ptr(rhs), _stream_ptr(stream))
        return A, rhs

    def assemble_stabilized(self, u, u_n=None, rho=1.0, mu=1e-3, dt=1e-2, out=None, stream=None):
        """(Auu [9, nnz], G [3, nnz], rhs [3, n]): the stabilised velocity block,
        Auu[3 i + j] the (i, j) entry of every CSR entry's 3x3 block."""
        torch = _torch()
        f, keep = self.fields(u, u_n, rho, mu, dt)
        if out is None:
            out = (torch.empty(9, self.nnz, dtype=self.out_dtype, device=self.device),
                   torch.empty(3, self.nnz, dtype=self.out_dtype, device=self.device),
                   torch.empty(3, self.n, dtype=self.out_dtype, device=self.device))
        Auu, G, rhs = out
        for t, shape in ((Auu, (9, self.nnz)), (G, (3, self.nnz)), (rhs, (3, self.n))):
            if t.dtype != self.out_dtype or tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"stabilised output must be a contiguous {shape} tensor of the output dtype")
        nsi_assemble_stabilized(self.handle, f, _ptr(Auu), _ptr(G), _ptr(rhs), _stream_ptr(stream))
        return Auu, G, rhs

    def nodal(self, u_n, rho=1.0, dt=1e-2, out=None, stream=None):
        """(rhs [3, n], dt_rho [n], mass_rho [n]): the paper's per-node outputs."""
        torch = _torch()
        f, keep = self.fields(u_n, None, rho, 0.0, dt)
        if out is None:
            out = (torch.empty(3, self.n, dtype=self.out_dtype, device=self.device),
                   torch.empty(self.n, dtype=self.out_dtype, device=self.device),
                   torch.empty(self.n, dtype=self.out_dtype, device=self.device))
        rhs, dtr, mr = out
        nsi_assemble_nodal(self.handle, f, _ptr(rhs), _ptr(dtr), _ptr(mr), _stream_ptr(stream))
        return rhs, dtr, mr

    def assemble_host(self, u_host, A_host, G_host, rhs_host, rho=1.0, mu=1e-3, dt=1e-2, stream=None):
        """End-to-end call on HOST tensors (pinned recommended): H2D of u, assembly, D2H of outputs."""
        f = NsiFields()
        for k in range(3):
            f.u[k] = u_host[k].data_ptr()
            f.u_n[k] = None
        f.rho, f.mu, f.dt = float(rho), float(mu), float(dt)
        o = NsiOutputs(A_host.data_ptr(), G_host.data_ptr(), rhs_host.data_ptr())
        nsi_assemble_host(self.handle, f, o, _stream_ptr(stream))

    def residual(self, u, rho=1.0, mu=1e-3, dt=1e-2, u_n=None, out=None, stream=None):
        """R = A(u) u - b, node-component layout [3, n] (matrix-free, no assembled matrix)."""
        torch = _torch()
        f, keep = self.fields(u, u_n, rho, mu, dt)
        R = out if out is not None else torch.empty(3, self.n, dtype=self.vel_dtype, device=self.device)
        nsi_residual(self.handle, f, _ptr(R), _stream_ptr(stream))
        return R

    def vjp(self, u, w, rho=1.0, mu=1e-3, dt=1e-2, stream=None):
        """(grad_u [3, n], grad_mu) of sum(w * R(u, mu))."""
        torch = _torch()
        f, keep = self.fields(u, None, rho, mu, dt)
        wc = torch.stack(self._vel(w)).contiguous()
        gu = torch.empty(3, self.n, dtype=self.vel_dtype, device=self.device)
        gmu = torch.empty(1, dtype=torch.float64, device=self.device)
        nsi_assemble_vjp(self.handle, f, _ptr(wc), _ptr(gu), _ptr(gmu), _stream_ptr(stream))
        return gu, gmu

    def device_status(self, stream=None):
        nsi_device_status(self.handle, _stream_ptr(stream))

    def info(self):
        return nsi_info(self.handle)

    def autotune(self, u, rho=1.0, mu=1e-3, dt=1e-2, reps=5, cache=None, stream=None):
        """Pick scatter mode and rows-per-block by timing them on this mesh.

        With ``cache`` (a JSON file path), a choice made before for the same GPU,
        precision and mesh size is reused without timing; new choices are added.
        Returns (scatter mode name, rows per block).
        """
        import json
        import torch

        key = "|".join([torch.cuda.get_device_name(self.device), str(self.precision), str(self.n), str(self.E),
                        str(self.nnz), str(self.max_row)])
        db = {}
        if cache and os.path.exists(cache):
            try:
                with open(cache) as fh:
                    db = json.load(fh)
            except (OSError, ValueError):
                db = {}
        names = {v: k for k, v in SCATTERS.items()}
        if key in db:
            sc, rows = db[key]["scatter"], db[key]["rows_per_block"]
            nsi_set_launch(self.handle, SCATTERS[sc], rows)
        else:
            f, keep = self.fields(u, None, rho, mu, dt)
            A, G, rhs = self.empty_outputs()
            o = NsiOutputs(A.data_ptr(), G.data_ptr(), rhs.data_ptr())
            code, rows = nsi_autotune(self.handle, f, o, reps, _stream_ptr(stream))
            sc = names[code]
            if cache:
                db[key] = {"scatter": sc, "rows_per_block": rows}
                tmp = f"{cache}.{os.getpid()}.tmp"
                with open(tmp, "w") as fh:
                    json.dump(db, fh, indent=1)
                os.replace(tmp, cache)
        self.scatter = nsi_info(self.handle).scatter
        return sc, rows

    def set_timing_events(self, start=None, stop=None):
        """Record torch.cuda.Event pair around the main assembly kernel of later calls (None: off)."""
        if start is None or stop is None:
            nsi_set_timing_events(self.handle, None, None)
            return
        for ev in (start, stop):
            if not ev.cuda_event:  # torch creates the CUDA event on first record
                ev.record()
        nsi_set_timing_events(self.handle, ctypes.c_void_p(start.cuda_event), ctypes.c_void_p(stop.cuda_event))


def _components(first, rest, stride, ncomp):
    """Device pointers of ncomp component arrays: ``first`` (or None) then the
    rows of ``rest`` (a [k, stride] tensor)."""
    ptrs = []
    if first is not None:
        ptrs.append(first.data_ptr())
    es = rest.element_size()
    while len(ptrs) < ncomp:
        ptrs.append(rest.data_ptr() + (len(ptrs) - (first is not None)) * stride * es)
    return (ctypes.c_void_p * ncomp)(*ptrs)


def gather_values(first, rest, stride, idx, ncomp=4, stream=None):
    """[count, ncomp] tensor of the values at positions idx of the component
    arrays (first, rest[0], rest[1], ...) -- e.g. A and G -- via nsi_gather_values."""
    torch = _torch()
    count = int(idx.numel())
    dst = torch.empty((count, ncomp), dtype=rest.dtype, device=rest.device)
    comps = _components(first, rest, stride, ncomp)
    _check(load_library().nsi_gather_values(comps, ncomp, _ptr(idx), count, _ptr(dst), rest.element_size(),
                                            _stream_ptr(stream)))
    return dst


def add_values(first, rest, stride, idx, vals, ncomp=4, stream=None):
    """(first, rest[0], ...)[idx[k]] += vals[k, :] via nsi_add_values (idx distinct)."""
    count = int(idx.numel())
    if count == 0:
        return
    comps = _components(first, rest, stride, ncomp)
    vals = vals.contiguous()
    _check(load_library().nsi_add_values(comps, ncomp, _ptr(idx), count, _ptr(vals), rest.element_size(),
                                         _stream_ptr(stream)))


def assemble_batched(assemblers, us, rho=1.0, mu=1e-3, dt=1e-2, outs=None, stream=None):
    """One persistent launch over several meshes; returns the list of (A, G, rhs)."""
    fields, keep, outputs, results = [], [], [], []
    for k, (asm, u) in enumerate(zip(assemblers, us)):
        f, kp = asm.fields(u, None, rho, mu, dt)
        fields.append(f)
        keep.append(kp)
        A, G, rhs = outs[k] if outs is not None else asm.empty_outputs()
        outputs.append(NsiOutputs(A.data_ptr(), G.data_ptr(), rhs.data_ptr()))
        results.append((A, G, rhs))
    nsi_assemble_batched([a.handle for a in assemblers], fields, outputs, _stream_ptr(stream))
    return results


def _make_residual_function():
    torch = _torch()

    class _NsiResidual(torch.autograd.Function):
        """R(u, mu) = A(u) u - b (b fixed) with the hand-written adjoint kernel as backward.

        forward(u [3, n], mu (0-d tensor), assembler, rho, dt) -> R [3, n]
        """

        @staticmethod
        def forward(ctx, u, mu, asm, rho=1.0, dt=1e-2):
            R = asm.residual(u.detach(), rho=rho, mu=float(mu), dt=dt)
            ctx.save_for_backward(u.detach())
            ctx.asm, ctx.rho, ctx.dt, ctx.mu = asm, rho, dt, float(mu)
            return R

        @staticmethod
        def backward(ctx, gR):
            (u,) = ctx.saved_tensors
            gu, gmu = ctx.asm.vjp(u, gR.contiguous(), rho=ctx.rho, mu=ctx.mu, dt=ctx.dt)
            return gu.to(u.dtype), gmu.reshape(()).to(torch.float64), None, None, None

    return _NsiResidual


class _LazyResidual:
    _fn = None

    def apply(self, *args):
        if _LazyResidual._fn is None:
            _LazyResidual._fn = _make_residual_function()
        return _LazyResidual._fn.apply(*args)


NsiResidual = _LazyResidual()
