"""The row-gather element walk (host logic, no GPU).

tests/walk_replay.cu compiles the library's create-time code with a small
driver: for every row of a mesh it builds the row's star, encodes the walk
with the library's encode_walk, and replays it the way the kernel runs it
(window registers with the newest node always in q, the first window loaded
directly, orientation bits, the carried cofactor and its sign,
the next node read before the leaving node is written back).  The replayed
row sums must equal direct sums over the star in double, every element must
be walked exactly once, and no step may read a node still held in registers.
Meshes: Kuhn cubes in natural, random and RCM numbering, and Delaunay meshes
of jittered lattices (irregular stars, holes, slivers).
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import meshgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def replay(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("walk") / "walk_replay"
    cmd = [nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "walk_replay.cu"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _write(path, mesh, u):
    with open(path, "wb") as f:
        np.array([mesh.n_nodes, mesh.n_elems], dtype=np.int64).tofile(f)
        np.ascontiguousarray(mesh.coord, dtype=np.float64).tofile(f)
        np.ascontiguousarray(mesh.lnods, dtype=np.int32).tofile(f)
        np.ascontiguousarray(u, dtype=np.float64).tofile(f)


def _small(coord, lnods, seed):
    coord = np.asarray(coord, dtype=np.float64)
    lnods = np.asarray(lnods, dtype=np.int32)
    for e in range(len(lnods)):  # positive orientation
        X = coord[lnods[e]]
        if np.linalg.det(np.c_[X[1] - X[0], X[2] - X[0], X[3] - X[0]]) < 0:
            lnods[e, [2, 3]] = lnods[e, [3, 2]]
    return meshgen.Mesh(coord=coord, lnods=lnods), np.random.default_rng(seed).standard_normal(coord.shape)


def _fan(m):
    ang = 2 * np.pi * np.arange(m) / m
    coord = np.vstack([[0, 0, 0], np.c_[np.cos(ang), np.sin(ang), np.zeros(m)], [0, 0, 1]])
    return _small(coord, [[0, 1 + k, 1 + (k + 1) % m, m + 1] for k in range(m)], 70 + m)


CASES = [
    # every row of one tet walks 1 element; two tets on a face; a ring of 30
    # tets around an edge (rows of 32 entries, the walk's limit)
    ("one_tet", lambda: _small([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], [[0, 1, 2, 3]], 71)),
    ("two_tets", lambda: _small([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]],
                                [[0, 1, 2, 3], [1, 2, 3, 4]], 72)),
    ("fan30", lambda: _fan(30)),
    ("kuhn6_natural", lambda: meshgen.config_mesh(N=6, jitter=0.0, numbering="natural", seed=0)),
    ("kuhn9_random", lambda: meshgen.config_mesh(N=9, jitter=0.15, numbering="random", seed=1)),
    ("kuhn8_rcm", lambda: meshgen.config_mesh(N=8, jitter=0.15, numbering="rcm", seed=2)),
    ("delaunay6", lambda: meshgen.delaunay_cube(6, 0.2, seed=5)),
    ("delaunay10", lambda: meshgen.delaunay_cube(10, 0.3, seed=6)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_walk_replays_the_star(replay, tmp_path, name, make):
    mesh, u = make()
    f = tmp_path / "mesh.bin"
    _write(f, mesh, u)
    r = subprocess.run([str(replay), str(f)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    stats = dict(re.findall(r"(\w+)=([0-9.eE+-]+)", r.stdout))
    assert int(stats["elements"]) == 4 * mesh.n_elems
    assert int(stats["skipped"]) == 0 and int(stats["stale_reads"]) == 0
    assert float(stats["worst"]) <= 1e-12
    # one path per row on the Kuhn cubes and the small meshes: two filling
    # steps per row, then one per element
    if not name.startswith("delaunay"):
        assert int(stats["multipath_rows"]) == 0
        assert int(stats["steps"]) == int(stats["elements"]) + 2 * mesh.n_nodes
    else:
        assert int(stats["multipath_rows"]) > 0  # holes and boundaries split some stars
