"""Shared helpers for the tests: error metrics and oracle/GPU plumbing."""
import numpy as np

import meshgen


def row_scaled_err(row_ptr, got, ref):
    """max_i max_j |got_ij - ref_ij| / max_j |ref_ij| over the rows of a CSR value array.

    The per-entry relative error is ill-posed on entries that cancel to ~0
    (e.g. the interior diagonal of G); every row is instead scaled by its own
    largest reference entry.  Rows whose reference is all zero are scaled by 1.
    """
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    if ref.size == 0:
        return 0.0
    lens = np.diff(rp)
    rows = np.repeat(np.arange(lens.size), lens)
    scale = np.zeros(lens.size)
    np.maximum.at(scale, rows, np.abs(ref))
    scale[scale == 0] = 1.0
    err = np.zeros(lens.size)
    np.maximum.at(err, rows, np.abs(got - ref))
    return float(np.max(err / scale))


def vec_scaled_err(got, ref):
    """max |got - ref| / max |ref| for one nodal component."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    s = np.abs(ref).max()
    return float(np.abs(got - ref).max() / (s if s > 0 else 1.0))


def errors(row_ptr, A, G, rhs, A_ref, G_ref, rhs_ref):
    """dict of row-scaled errors for A, G_x, G_y, G_z and rhs components."""
    out = {"A": row_scaled_err(row_ptr, A, A_ref)}
    for d in range(3):
        out[f"G{d}"] = row_scaled_err(row_ptr, G[d], G_ref[d])
    for k in range(3):
        out[f"rhs{k}"] = vec_scaled_err(rhs[k], rhs_ref[k])
    return out


def mesh_case(name=None, **kw):
    mesh, u = meshgen.config_mesh(name, **kw) if name else meshgen.config_mesh(**kw)
    return mesh, u
