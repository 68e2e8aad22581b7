"""Seeded synthetic inputs for P1 tetrahedral assembly.

This module only *produces inputs*: meshes (coordinates + connectivity),
nodal velocity fields, adjoint weights and node renumberings.  It contains
none of the assembly arithmetic (no Jacobians, no quadrature, no CSR
pattern), so both the FP64 oracle and the CUDA library can be fed from it
without sharing any of the method's code.

The paper's benchmarks are Alya meshes (Sphere 100K/16M/32M, Elbow, ...;
Table II) which are not public.  They are stood in for by unit cubes of
N^3 hexahedra, each split into 6 linear tetrahedra (the paper's benchmarks
use 4-node elements, Section II-A), which reproduces the ~5.8
elements-per-node ratio of Table II's 3D meshes.

Conventions (all fixed here so that every consumer agrees):

* node id of grid point (i, j, k) = i + (N+1) * (j + (N+1) * k), coordinates
  (i, j, k) * h with h = 1/N;
* hexes are enumerated with i fastest, then j, then k; inside a hex the 6
  tets follow the permutations of the axes in ``itertools.permutations``
  order, tet = {v, v+e_s0, v+e_s0+e_s1, v+(1,1,1)} (Kuhn/Freudenthal split,
  conforming across hexes), with local nodes 2 and 3 swapped for odd
  permutations so that every tet is positively oriented;
* jitter moves each coordinate of each *interior* node by U[-f h, f h]
  (boundary nodes stay put, so the domain stays the unit cube); at f = 0.15
  every tet stays positively oriented (the smallest Kuhn altitude is h/sqrt 2);
* a renumbering maps old node id -> new node id; coordinates and velocities
  are reordered and connectivity is relabelled, the element order is kept.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "kuhn_cube", "jitter_interior", "renumber", "random_permutation",
    "rcm_permutation", "sinusoid_velocity", "add_noise", "gaussian_weights", "delaunay_hub",
    "config_mesh", "batch_meshes", "delaunay_cube", "CONFIGS",
]

# permutations of (x, y, z) in itertools order and their parities
_PERMS = list(itertools.permutations(range(3)))
_ODD = [((p[0] > p[1]) + (p[0] > p[2]) + (p[1] > p[2])) % 2 == 1 for p in _PERMS]


@dataclass
class Mesh:
    """A tetrahedral mesh: ``coord`` float64 [n, 3], ``lnods`` int32 [E, 4] (0-based)."""

    coord: np.ndarray
    lnods: np.ndarray
    N: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coord.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.lnods.shape[0])


def kuhn_cube(N: int) -> Mesh:
    """Unit cube of N^3 hexes, each split into 6 Kuhn tets (see module doc)."""
    if N < 1:
        raise ValueError("N must be >= 1")
    M = N + 1
    g = np.arange(M, dtype=np.float64) / N
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    coord = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).copy()

    hi, hj, hk = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    # enumerate hexes with i fastest: order by (k, j, i)
    hi = hi.transpose(2, 1, 0).ravel()
    hj = hj.transpose(2, 1, 0).ravel()
    hk = hk.transpose(2, 1, 0).ravel()
    base = (hi + M * (hj + M * hk)).astype(np.int64)
    step = np.array([1, M, M * M], dtype=np.int64)

    tets = np.empty((base.size, 6, 4), dtype=np.int64)
    for t, (p, odd) in enumerate(zip(_PERMS, _ODD)):
        n0 = base
        n1 = base + step[p[0]]
        n2 = n1 + step[p[1]]
        n3 = base + step.sum()
        if odd:
            n2, n3 = n3, n2
        tets[:, t, 0], tets[:, t, 1], tets[:, t, 2], tets[:, t, 3] = n0, n1, n2, n3
    lnods = tets.reshape(-1, 4).astype(np.int32)
    return Mesh(coord=coord, lnods=lnods, N=N, meta={"kind": "kuhn_cube", "N": N})


def jitter_interior(mesh: Mesh, frac: float, rng: np.random.Generator) -> Mesh:
    """Move every coordinate of every interior grid node by U[-frac*h, frac*h]."""
    N = mesh.N
    M = N + 1
    h = 1.0 / N
    ids = np.arange(M ** 3)
    i, j, k = ids % M, (ids // M) % M, ids // (M * M)
    interior = (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)
    delta = rng.uniform(-frac * h, frac * h, size=(M ** 3, 3))
    coord = mesh.coord.copy()
    coord[interior] += delta[interior]
    meta = dict(mesh.meta, jitter=frac)
    return Mesh(coord=coord, lnods=mesh.lnods, N=N, meta=meta)


def random_permutation(n: int, rng: np.random.Generator) -> np.ndarray:
    """old id -> new id, a seeded uniform random permutation."""
    return rng.permutation(n).astype(np.int64)


def rcm_permutation(mesh: Mesh) -> np.ndarray:
    """old id -> new id from reverse Cuthill-McKee on the node graph."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    n = mesh.n_nodes
    ln = mesh.lnods.astype(np.int64)
    r = np.repeat(ln, 4, axis=1).ravel()
    c = np.tile(ln, (1, 4)).ravel()
    g = sp.csr_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(n, n))
    order = reverse_cuthill_mckee(g, symmetric_mode=True)  # new position -> old id
    perm = np.empty(n, dtype=np.int64)
    perm[order] = np.arange(n)
    return perm


def renumber(mesh: Mesh, perm: np.ndarray, *fields: np.ndarray):
    """Apply node renumbering ``perm`` (old -> new) to a mesh and nodal fields [n, ...]."""
    n = mesh.n_nodes
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    coord = mesh.coord[inv]
    lnods = perm[mesh.lnods.astype(np.int64)].astype(np.int32)
    out = Mesh(coord=coord, lnods=lnods, N=mesh.N, meta=dict(mesh.meta, renumbered=True))
    if fields:
        return (out,) + tuple(f[inv] for f in fields)
    return out


def sinusoid_velocity(coord: np.ndarray, rng: np.random.Generator, n_terms: int = 3) -> np.ndarray:
    """u_k(x) = sum_m sin(2 pi kappa_{k,m} . x + phi_{k,m}), kappa in {1,2,3}^3, phi in [0, 2 pi)."""
    kappa = rng.integers(1, 4, size=(3, n_terms, 3)).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(3, n_terms))
    u = np.zeros((coord.shape[0], 3), dtype=np.float64)
    for k in range(3):
        for m in range(n_terms):
            u[:, k] += np.sin(2.0 * np.pi * (coord @ kappa[k, m]) + phi[k, m])
    return u


def add_noise(u: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return u + sigma * rng.standard_normal(u.shape)


def gaussian_weights(n: int, rng: np.random.Generator) -> np.ndarray:
    """Adjoint weights w ~ N(0, 1), shape [n, 3]."""
    return rng.standard_normal((n, 3))


# Physical parameters of the Galerkin P1 form used throughout.
RHO, MU, DT = 1.0, 1.0e-3, 1.0e-2

CONFIGS = {
    # name: (N, jitter, numbering, seed)
    "cube8": dict(N=8, jitter=0.0, numbering="natural", seed=0),
    "cube100": dict(N=100, jitter=0.15, numbering="random", seed=1),
    "cube70": dict(N=70, jitter=0.15, numbering="random", seed=1),  # the cube100 recipe, smaller (profiling)
    "cube200_rcm": dict(N=200, jitter=0.15, numbering="rcm", seed=2, noise=0.05),
    "cube200_random": dict(N=200, jitter=0.15, numbering="random", seed=2, noise=0.05),
    "cube50": dict(N=50, jitter=0.15, numbering="natural", seed=4),
}


def config_mesh(name: str = None, *, N: int = None, jitter: float = 0.0, numbering: str = "natural",
                seed: int = 0, noise: float = 0.0):
    """Build (mesh, u) for a named workload or explicit parameters.

    Seeds: the mesh jitter and the velocity draw from ``default_rng(seed)``;
    a random numbering draws from ``default_rng(10*seed + 1)``; noise from
    ``default_rng(10*seed)``.
    """
    if name is not None:
        p = dict(CONFIGS[name])
        N, jitter, numbering, seed = p["N"], p["jitter"], p["numbering"], p["seed"]
        noise = p.get("noise", 0.0)
    rng = np.random.default_rng(seed)
    mesh = kuhn_cube(N)
    if jitter > 0:
        mesh = jitter_interior(mesh, jitter, rng)
    u = sinusoid_velocity(mesh.coord, rng)
    if noise > 0:
        u = add_noise(u, noise, np.random.default_rng(10 * seed))
    if numbering == "random":
        perm = random_permutation(mesh.n_nodes, np.random.default_rng(10 * seed + 1))
        mesh, u = renumber(mesh, perm, u)
    elif numbering == "rcm":
        perm = rcm_permutation(mesh)
        mesh, u = renumber(mesh, perm, u)
    elif numbering != "natural":
        raise ValueError(numbering)
    mesh.meta.update(numbering=numbering, seed=seed, noise=noise)
    return mesh, np.ascontiguousarray(u)


def delaunay_cube(m: int = 8, jitter: float = 0.25, seed: int = 5):
    """(mesh, u): an unstructured mesh of the unit cube, the Delaunay
    tetrahedralization (scipy / Qhull) of the (m+1)^3 lattice with interior
    points moved by U[-jitter/m, jitter/m] per coordinate.  Irregular stars
    (rows of 5..24 entries), holes where flat tets (|volume| <= 1e-9 / m^3,
    on the unjittered faces) are dropped, and slivers.  Tets are listed with
    positive orientation (two nodes swapped where the triple product of the
    edge vectors is negative).  u: the seeded sinusoids, as config_mesh."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    g = np.arange(m + 1, dtype=np.float64) / m
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).copy()
    inner = np.all((P > 0) & (P < 1), axis=1)
    P[inner] += rng.uniform(-jitter / m, jitter / m, size=(int(inner.sum()), 3))
    T = Delaunay(P).simplices.astype(np.int64)
    X = P[T]
    vol6 = np.linalg.det(X[:, 1:] - X[:, :1])
    keep = np.abs(vol6) > 1e-9 / m ** 3
    T, vol6 = T[keep], vol6[keep]
    T[vol6 < 0] = T[vol6 < 0][:, [0, 1, 3, 2]]
    mesh = Mesh(coord=P, lnods=T.astype(np.int32), N=m, meta={"kind": "delaunay_cube", "m": m, "jitter": jitter,
                                                            "seed": seed})
    u = sinusoid_velocity(P, rng)
    return mesh, np.ascontiguousarray(u)


def delaunay_hub(m: int = 4, k: int = 48, radius: float = 0.3, seed: int = 6):
    """(mesh, u): an unstructured mesh of the unit cube with one node of very
    high valence -- the Delaunay tetrahedralization (scipy / Qhull) of the
    (m+1)^3 lattice, minus its points within `radius` of the centre, plus the
    centre itself and k points spread evenly over the sphere of that radius
    around it (a Fibonacci lattice, seeded rotation).  Every sphere point is a
    Delaunay neighbour of the centre, so the centre's row has about k + 1
    entries.  Flat tets are dropped and tets listed with positive orientation,
    as delaunay_cube.  u: the seeded sinusoids, as config_mesh."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    g = np.arange(m + 1, dtype=np.float64) / m
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    c = np.full(3, 0.5)
    P = P[np.linalg.norm(P - c, axis=1) > 1.2 * radius]
    i = np.arange(k) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / k)
    theta = np.pi * (1.0 + 5.0 ** 0.5) * i + rng.uniform(0.0, 2.0 * np.pi)
    S = c + radius * np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], 1)
    P = np.vstack([P, c[None, :], S])
    T = Delaunay(P).simplices.astype(np.int64)
    X = P[T]
    vol6 = np.linalg.det(X[:, 1:] - X[:, :1])
    keep = np.abs(vol6) > 1e-9 / m ** 3
    T, vol6 = T[keep], vol6[keep]
    T[vol6 < 0] = T[vol6 < 0][:, [0, 1, 3, 2]]
    mesh = Mesh(coord=np.ascontiguousarray(P), lnods=T.astype(np.int32), N=m,
                meta={"kind": "delaunay_hub", "m": m, "k": k, "radius": radius, "seed": seed})
    u = sinusoid_velocity(P, rng)
    return mesh, np.ascontiguousarray(u)


def batch_meshes(count: int = 64, lo: int = 10, hi: int = 60, seed: int = 3, jitter: float = 0.15):
    """Independent jittered cubes with side lengths ~ U{lo..hi}; mesh i uses seed 1000*seed + i."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=count)
    out = []
    for i, N in enumerate(sides):
        out.append(config_mesh(N=int(N), jitter=jitter, numbering="natural", seed=1000 * seed + i))
    return out
