"""FP64 CPU oracle for P1 tetrahedral incompressible-flow assembly (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and the
two share no code.  The arithmetic lives in ``nsi_oracle.c`` (plain C, IEEE
double); this module compiles it with gcc on first use and wraps it for numpy.

Array conventions (see ``nsi_oracle.c``): ``coord``, ``u``, ``un``, ``w`` are
node-major float64 [n, 3]; ``lnods`` int32 [E, 4] 0-based; CSR ``row_ptr``
int32 [n+1], ``col_idx`` int32 [nnz]; ``G`` float64 [3, nnz]; ``rhs`` float64
[3, n]; the stabilised velocity block ``Auu`` float64 [9, nnz], component
3 i + j the (i, j) entry of every entry's 3x3 block.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no fast-math; OpenMP for
    the multi-threaded assembly where the compiler has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_element_batch.restype = ctypes.c_int
            lib.oracle_element_batch.argtypes = [ctypes.c_int64, _d, _i32, _d, _d, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, _i64, ctypes.c_int64,
                                                 _d, _d, _d, _d, _d]
            lib.oracle_nodal.restype = ctypes.c_int
            lib.oracle_nodal.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, ctypes.c_double,
                                         ctypes.c_double, _d, _d, _d]
            lib.oracle_pattern.restype = ctypes.c_int64
            lib.oracle_pattern.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32, _i32, _i32]
            lib.oracle_assemble.restype = ctypes.c_int
            lib.oracle_assemble.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, _d, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, _i32, _i32, _d, _d, _d]
            lib.oracle_assemble_rows.restype = ctypes.c_int
            lib.oracle_assemble_rows.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, _d,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, _i64,
                                                 ctypes.c_int64, ctypes.c_int64, _i32, _i32, _d, _d, _d]
            lib.oracle_vjp.restype = ctypes.c_int
            lib.oracle_vjp.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _d, _d, _d]
            lib.oracle_assemble_threads.restype = ctypes.c_int
            lib.oracle_assemble_threads.argtypes = lib.oracle_assemble.argtypes + [ctypes.c_int]
            lib.oracle_assemble_stabilized.restype = ctypes.c_int
            lib.oracle_assemble_stabilized.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, _d,
                                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _i32, _i32,
                                                       _d, _d, _d]
            lib.oracle_stab_rows.restype = ctypes.c_int
            lib.oracle_stab_rows.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, ctypes.c_double,
                                             ctypes.c_double, _i64, ctypes.c_int64, ctypes.c_int64, _i32, _i32, _d]
            lib.oracle_stab_element.restype = None
            lib.oracle_stab_element.argtypes = [_d, _d, ctypes.c_double, ctypes.c_double, _d, _d]
            lib.oracle_tau.restype = ctypes.c_double
            lib.oracle_tau.argtypes = [_d, _d, ctypes.c_double, ctypes.c_double, _d]
            lib.oracle_vjp_mu_abs.restype = ctypes.c_int
            lib.oracle_vjp_mu_abs.argtypes = [ctypes.c_int64, ctypes.c_int64, _d, _i32, _d, _d, _d]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ln(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def element_matrices(coord, lnods, u, un=None, rho=1.0, mu=1e-3, dt=1e-2, elems=None):
    """Per-element (A_e [m,4,4], G_e [m,4,4,3], b_e [m,4,3], vol [m], detJ [m])."""
    lib = _load()
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    un = u if un is None else _f64(un)
    if elems is None:
        elems = np.arange(lnods.shape[0], dtype=np.int64)
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    m = elems.size
    A = np.empty((m, 4, 4)); G = np.empty((m, 4, 4, 3)); b = np.empty((m, 4, 3))
    vol = np.empty(m); det = np.empty(m)
    rc = lib.oracle_element_batch(coord.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), _p(un, _d),
                                  rho, mu, dt, _p(elems, _i64), m, _p(A, _d), _p(G, _d), _p(b, _d),
                                  _p(vol, _d), _p(det, _d))
    if rc != 0:
        raise ValueError(f"oracle_element_batch failed ({rc})")
    return A, G, b, vol, det


def pattern(n, lnods):
    """CSR pattern (row_ptr int32 [n+1], col_idx int32 [nnz]) of all (lnods[e,a], lnods[e,b])."""
    lib = _load()
    lnods = _ln(lnods)
    E = lnods.shape[0]
    nnz = lib.oracle_pattern(n, E, _p(lnods, _i32), None, None)
    if nnz < 0:
        raise ValueError(f"oracle_pattern failed ({nnz})")
    row_ptr = np.empty(n + 1, dtype=np.int32)
    col_idx = np.empty(max(nnz, 1), dtype=np.int32)
    nnz2 = lib.oracle_pattern(n, E, _p(lnods, _i32), _p(row_ptr, _i32), _p(col_idx, _i32))
    assert nnz2 == nnz
    return row_ptr, col_idx[:nnz]


def assemble(coord, lnods, u, un=None, rho=1.0, mu=1e-3, dt=1e-2, csr=None):
    """Global assembly -> (row_ptr, col_idx, A [nnz], G [3, nnz], rhs [3, n])."""
    lib = _load()
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    un = u if un is None else _f64(un)
    n = coord.shape[0]
    row_ptr, col_idx = pattern(n, lnods) if csr is None else csr
    nnz = int(row_ptr[-1])
    A = np.empty(nnz); G = np.empty((3, nnz)); rhs = np.empty((3, n))
    rc = lib.oracle_assemble(n, lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), _p(un, _d),
                             rho, mu, dt, _p(_ln(row_ptr), _i32), _p(_ln(col_idx), _i32),
                             _p(A, _d), _p(G, _d), _p(rhs, _d))
    if rc != 0:
        raise ValueError(f"oracle_assemble failed ({rc})")
    return row_ptr, col_idx, A, G, rhs


def tau(X, U, rho=1.0, mu=1e-3):
    """(tau1, tau2) of one element (X, U: [4, 3]); see ``oracle_tau``."""
    lib = _load()
    t2 = np.zeros(1)
    t1 = lib.oracle_tau(_p(_f64(X), _d), _p(_f64(U), _d), rho, mu, _p(t2, _d))
    return float(t1), float(t2[0])


def stab_element(X, U, rho=1.0, mu=1e-3):
    """(S [4, 4], K [4, 4, 3, 3]) of one element; see ``oracle_stab_element``."""
    lib = _load()
    S = np.empty((4, 4)); K = np.empty((4, 4, 3, 3))
    lib.oracle_stab_element(_p(_f64(X), _d), _p(_f64(U), _d), rho, mu, _p(S, _d), _p(K, _d))
    return S, K


def assemble_stabilized(coord, lnods, u, un=None, rho=1.0, mu=1e-3, dt=1e-2, csr=None):
    """Stabilised assembly -> (row_ptr, col_idx, Auu [9, nnz], G [3, nnz],
    rhs [3, n]); Auu[3 i + j] is the (i, j) entry of every 3x3 block (see
    ``oracle_assemble_stabilized``)."""
    lib = _load()
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    un = u if un is None else _f64(un)
    n = coord.shape[0]
    row_ptr, col_idx = pattern(n, lnods) if csr is None else csr
    nnz = int(row_ptr[-1])
    Auu = np.empty((9, nnz)); G = np.empty((3, nnz)); rhs = np.empty((3, n))
    rc = lib.oracle_assemble_stabilized(n, lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), _p(un, _d),
                                        rho, mu, dt, _p(_ln(row_ptr), _i32), _p(_ln(col_idx), _i32),
                                        _p(Auu, _d), _p(G, _d), _p(rhs, _d))
    if rc != 0:
        raise ValueError(f"oracle_assemble_stabilized failed ({rc})")
    return row_ptr, col_idx, Auu, G, rhs


def assemble_stabilized_rows(coord, lnods, u, rows, un=None, rho=1.0, mu=1e-3, dt=1e-2, maxc=64):
    """Stabilised rows for a list of row ids -> list of (cols, Auu [9, c],
    G [3, c], rhs [3]): the Galerkin rows of ``assemble_rows`` on the diagonal
    components plus the stabilisation of ``oracle_stab_rows``."""
    lib = _load()
    gal = assemble_rows(coord, lnods, u, rows, un=un, rho=rho, mu=mu, dt=dt, maxc=maxc)
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    m = rows.size
    cols = np.zeros((m, maxc), dtype=np.int32); count = np.zeros(m, dtype=np.int32)
    Auu = np.zeros((m, 9, maxc))
    rc = lib.oracle_stab_rows(coord.shape[0], lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), rho, mu,
                              _p(rows, _i64), m, maxc, _p(cols, _i32), _p(count, _i32), _p(Auu, _d))
    if rc != 0:
        raise ValueError(f"oracle_stab_rows failed ({rc})")
    out = []
    for t in range(m):
        c, A, G, rhs = gal[t]
        if not np.array_equal(c, cols[t, :count[t]]):
            raise ValueError("oracle_stab_rows: columns differ from the Galerkin row")
        blk = Auu[t, :, :count[t]].copy()
        for i in range(3):
            blk[4 * i] += A
        out.append((c, blk, G, rhs))
    return out


def assemble_threads(coord, lnods, u, un=None, rho=1.0, mu=1e-3, dt=1e-2, csr=None, threads=0):
    """``assemble`` on several host threads (0: all OpenMP threads); bitwise
    equal to ``assemble`` (see ``oracle_assemble_threads``)."""
    lib = _load()
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    un = u if un is None else _f64(un)
    n = coord.shape[0]
    row_ptr, col_idx = pattern(n, lnods) if csr is None else csr
    nnz = int(row_ptr[-1])
    A = np.empty(nnz); G = np.empty((3, nnz)); rhs = np.empty((3, n))
    rc = lib.oracle_assemble_threads(n, lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), _p(un, _d),
                                     rho, mu, dt, _p(_ln(row_ptr), _i32), _p(_ln(col_idx), _i32),
                                     _p(A, _d), _p(G, _d), _p(rhs, _d), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_assemble_threads failed ({rc})")
    return row_ptr, col_idx, A, G, rhs


def assemble_rows(coord, lnods, u, rows, un=None, rho=1.0, mu=1e-3, dt=1e-2, maxc=64):
    """Assembled rows for a list of row ids -> list of (cols, A, G [3, c], rhs [3])."""
    lib = _load()
    coord, lnods, u = _f64(coord), _ln(lnods), _f64(u)
    un = u if un is None else _f64(un)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    m = rows.size
    cols = np.zeros((m, maxc), dtype=np.int32); count = np.zeros(m, dtype=np.int32)
    A = np.zeros((m, maxc)); G = np.zeros((m, 3, maxc)); rhs = np.zeros((m, 3))
    rc = lib.oracle_assemble_rows(coord.shape[0], lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d),
                                  _p(un, _d), rho, mu, dt, _p(rows, _i64), m, maxc, _p(cols, _i32),
                                  _p(count, _i32), _p(A, _d), _p(G, _d), _p(rhs, _d))
    if rc != 0:
        raise ValueError(f"oracle_assemble_rows failed ({rc})")
    return [(cols[t, :count[t]].copy(), A[t, :count[t]].copy(), G[t, :, :count[t]].copy(), rhs[t].copy())
            for t in range(m)]


def nodal(coord, lnods, un, rho=1.0, dt=1e-2):
    """The paper's per-node outputs of the assembly (Section II-A): (rhsid
    [3, n], dt_rho [n], mass_rho [n]); see ``oracle_nodal``."""
    lib = _load()
    coord, lnods, un = _f64(coord), _ln(lnods), _f64(un)
    n = coord.shape[0]
    rhs = np.empty((3, n)); dtr = np.empty(n); mr = np.empty(n)
    rc = lib.oracle_nodal(n, lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(un, _d), rho, dt,
                          _p(rhs, _d), _p(dtr, _d), _p(mr, _d))
    if rc != 0:
        raise ValueError(f"oracle_nodal failed ({rc})")
    return rhs, dtr, mr


def vjp(coord, lnods, u, w, rho=1.0, mu=1e-3, dt=1e-2):
    """(grad_u [n, 3], grad_mu) of w . R(u, mu), R = A(u) u - b with b fixed."""
    lib = _load()
    coord, lnods, u, w = _f64(coord), _ln(lnods), _f64(u), _f64(w)
    n = coord.shape[0]
    gu = np.empty((n, 3)); gmu = np.zeros(1)
    rc = lib.oracle_vjp(n, lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d), rho, mu, dt,
                        _p(w, _d), _p(gu, _d), _p(gmu, _d))
    if rc != 0:
        raise ValueError(f"oracle_vjp failed ({rc})")
    return gu, float(gmu[0])


def vjp_mu_abs(coord, lnods, u, w, rho=1.0, mu=1e-3, dt=1e-2):
    """Sum of the magnitudes of the terms of grad_mu (the scale of its rounding
    error bound); see ``oracle_vjp_mu_abs``.  rho, mu and dt do not enter."""
    lib = _load()
    coord, lnods, u, w = _f64(coord), _ln(lnods), _f64(u), _f64(w)
    out = np.zeros(1)
    rc = lib.oracle_vjp_mu_abs(coord.shape[0], lnods.shape[0], _p(coord, _d), _p(lnods, _i32), _p(u, _d),
                               _p(w, _d), _p(out, _d))
    if rc != 0:
        raise ValueError(f"oracle_vjp_mu_abs failed ({rc})")
    return float(out[0])


def residual(csr_A, rhs, u):
    """R = A u - b for node-major u [n, 3] and an assembled (row_ptr, col_idx, A) triple."""
    import scipy.sparse as sp

    row_ptr, col_idx, A = csr_A
    n = row_ptr.size - 1
    M = sp.csr_matrix((A, col_idx, row_ptr), shape=(n, n))
    return M @ u - rhs.T
