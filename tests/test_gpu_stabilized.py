"""GPU parity of the stabilised velocity block (nsi_assemble_stabilized).

The library's Auu [9, nnz] (3x3 block per CSR entry: the Galerkin operator on
the diagonal components plus the SUPG product, the transposed-gradient
viscous coupling and the grad-div term of Codina's algebraic subgrid scales),
G and rhs against the FP64 oracle, row-scaled per component.  Bars as the
Galerkin assembly: FP64 1e-12, mixed modes 1e-5 (against the oracle on the
float velocities the kernels receive, and on the original double ones).
Paths: the row kernel (one warp per row or pair of rows; Kuhn meshes, a
Delaunay mesh with rows of up to 32 entries), the per-row double kernel for
rows of more than 32 entries (a hub mesh) and, in the mixed modes, for the
rows of badly shaped elements (a sliver mesh), and the 100^3 cube at full
size on sampled rows.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests._common import row_scaled_err, vec_scaled_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


def vel_in(u, precision):
    return u if precision == "fp64" else u.astype(np.float32).astype(np.float64)


def run(mesh, u, precision, rho=RHO, mu=MU, dt=DT, debug=False, un=None):
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, debug_checks=debug)
    info = asm.info()
    unt = torch.as_tensor(un.T.copy()) if un is not None else None
    Auu, G, rhs = asm.assemble_stabilized(torch.as_tensor(u.T.copy()), u_n=unt, rho=rho, mu=mu, dt=dt)
    torch.cuda.synchronize()
    if debug:
        asm.device_status()
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    out = (info, rp, ci, Auu.double().cpu().numpy(), G.double().cpu().numpy(), rhs.double().cpu().numpy())
    asm.close()
    return out


def errors(rp, Auu, G, rhs, oAuu, oG, orhs):
    err = {f"Auu{c // 3}{c % 3}": row_scaled_err(rp, Auu[c], oAuu[c]) for c in range(9)}
    for d in range(3):
        err[f"G{d}"] = row_scaled_err(rp, G[d], oG[d])
        err[f"rhs{d}"] = vec_scaled_err(rhs[d], orhs[d])
    return err


def check(mesh, u, precision, rho=RHO, mu=MU, dt=DT, un=None, debug=False):
    info, rp, ci, Auu, G, rhs = run(mesh, u, precision, rho, mu, dt, debug=debug, un=un)
    refs = [vel_in(u, precision)] + ([u] if precision != "fp64" else [])
    for uu in refs:
        unn = None if un is None else vel_in(un, precision)
        orp, oci, oAuu, oG, orhs = oracle.assemble_stabilized(mesh.coord, mesh.lnods, uu, unn, rho, mu, dt)
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        err = errors(rp, Auu, G, rhs, oAuu, oG, orhs)
        assert max(err.values()) <= TOL[precision], err
    return info


CASES = [
    ("cube8", dict(name="cube8")),
    ("cube6_jit_random", dict(N=6, jitter=0.15, numbering="random", seed=31)),
    ("cube7_jit_rcm_noise", dict(N=7, jitter=0.15, numbering="rcm", seed=32, noise=0.05)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_stabilized_parity(case, precision):
    name, kw = case
    mesh, u = meshgen.config_mesh(kw["name"]) if "name" in kw else meshgen.config_mesh(**kw)
    info = check(mesh, u, precision)
    assert info.long_rows == 0 and info.max_row <= 16


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("rho,mu", [(1.0, 1e-2), (1.0, 1e-4), (3.0, 5e-3), (0.0, 1e-3)])
def test_stabilized_physical_constants(precision, rho, mu):
    """Viscous, convective and rho = 0 (no SUPG term, tau2 = mu) regimes."""
    mesh, u = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=33)
    check(mesh, u, precision, rho=rho, mu=mu, dt=2e-3)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_stabilized_separate_rhs_velocity(precision):
    mesh, u = meshgen.config_mesh(N=5, jitter=0.15, numbering="random", seed=34)
    un = np.random.default_rng(35).standard_normal(u.shape)
    check(mesh, u, precision, un=un)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_stabilized_unstructured_mesh(precision):
    """A Delaunay mesh: irregular stars, rows of 17..32 entries on whole-warp
    tasks, slivers."""
    mesh, u = meshgen.delaunay_cube(8, 0.25, seed=7)
    info = check(mesh, u, precision)
    assert info.max_row > 16 and info.long_rows == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_stabilized_long_rows(precision):
    """A hub node joined to 48 surrounding nodes: its row (and its
    neighbours' longer rows) exceed 32 entries and go to the per-row double
    kernel; the rest of the mesh stays on the row kernel."""
    mesh, u = meshgen.delaunay_hub()
    info = check(mesh, u, precision)
    assert info.long_rows > 0


@pytest.mark.parametrize("precision", ["mixed64", "mixed32"])
def test_stabilized_badly_shaped_elements(precision):
    """4^3 Kuhn cube with node (2,2,2) moved by 0.499 h along (1,-1,0): two
    slivers (|d1||d2||d3| / det about 1.1e3); their rows are recomputed in
    double after the row kernel."""
    mesh, u = meshgen.config_mesh(N=4, jitter=0.0, numbering="natural", seed=0)
    coord = mesh.coord.copy()
    coord[2 + 5 * (2 + 5 * 2)] += 0.499 * 0.25 * np.array([1.0, -1.0, 0.0])
    mesh = meshgen.Mesh(coord=coord, lnods=mesh.lnods, N=4)
    info = check(mesh, u, precision)
    assert info.exact_rows > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
def test_stabilized_debug_checks_and_determinism(precision):
    mesh, u = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=36)
    check(mesh, u, precision, debug=True)
    a = run(mesh, u, precision)
    b = run(mesh, u, precision)
    for x, y in zip(a[3:], b[3:]):
        assert np.array_equal(x, y)


def test_stabilized_single_tet_and_isolated_node():
    """One tetrahedron plus a node in no element (empty row, zero rhs)."""
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [5, 5, 5]], dtype=np.float64)
    lnods = np.array([[0, 1, 2, 3]], dtype=np.int32)
    u = np.random.default_rng(37).standard_normal((5, 3))
    mesh = meshgen.Mesh(coord=coord, lnods=lnods, N=0)
    for precision in ("fp64", "mixed64", "mixed32"):
        check(mesh, u, precision)


def test_stabilized_rejects_bad_constants():
    mesh, u = meshgen.config_mesh(N=2, jitter=0.0, numbering="natural", seed=0)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="fp64")
    ut = torch.as_tensor(u.T.copy())
    for kw in (dict(mu=0.0), dict(mu=-1e-3), dict(rho=-1.0), dict(dt=0.0), dict(mu=float("inf"))):
        with pytest.raises(nsi.NsiError) as e:
            asm.assemble_stabilized(ut, **kw)
        assert e.value.status == nsi.NSI_ERR_INVALID_ARG
    asm.close()


@pytest.fixture(scope="module")
def cube100():
    return meshgen.config_mesh("cube100")


@pytest.mark.parametrize("precision", ["mixed64", "mixed32", "fp64"])
def test_stabilized_cube100_sampled_rows(cube100, precision):
    """The 100^3 cube (6 M tets, random numbering) at full size: sampled rows
    (boundary, interior, first and last) against the oracle's row-restricted
    stabilised assembly, pattern of those rows bit-exact."""
    mesh, u = cube100
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    Auu, G, rhs = asm.assemble_stabilized(torch.as_tensor(u.T.copy()), rho=RHO, mu=MU, dt=DT)
    torch.cuda.synchronize()
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    Auu, G, rhs = (t.double().cpu().numpy() for t in (Auu, G, rhs))
    asm.close()
    rng = np.random.default_rng(8)
    n = mesh.n_nodes
    rows = np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.integers(0, n, 96)]))
    refs = [vel_in(u, precision)] + ([u] if precision != "fp64" else [])
    for uu in refs:
        ref = oracle.assemble_stabilized_rows(mesh.coord, mesh.lnods, uu, rows, None, RHO, MU, DT)
        worst = 0.0
        for r, (cols, blk, g, rh) in zip(rows, ref):
            s, e = rp[r], rp[r + 1]
            np.testing.assert_array_equal(ci[s:e], cols)
            for c in range(9):
                worst = max(worst, np.abs(Auu[c, s:e] - blk[c]).max() / np.abs(blk[c]).max())
            for d in range(3):
                worst = max(worst, np.abs(G[d, s:e] - g[d]).max() / np.abs(g[d]).max())
            worst = max(worst, np.abs(rhs[:, r] - rh).max() / np.abs(rhs).max())
        assert worst <= TOL[precision], worst


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_stabilized_repeated_elements(precision):
    """Two tetrahedra sharing a face, each listed 40 times: the stars hold 40
    or 80 copies of a few triangles, which the row-gather walk encoder cannot
    walk, so every row becomes a long row (the per-row double kernels of the
    assembly and of the stabilised block) while the handle stays valid.  The
    stabilised block and the Galerkin assembly against the oracle."""
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.6, 0.7, 0.8]], dtype=np.float64)
    t1, t2 = [0, 1, 2, 3], [1, 2, 3, 4]
    X = coord[t2]
    if np.linalg.det(np.c_[np.ones(4), X]) < 0:
        t2 = [1, 3, 2, 4]
    lnods = np.array([t1] * 40 + [t2] * 40, dtype=np.int32)
    u = np.random.default_rng(38).standard_normal((5, 3))
    mesh = meshgen.Mesh(coord=coord, lnods=lnods, N=0)
    check(mesh, u, precision)
    asm = nsi.Assembler(coord, lnods, precision=precision)
    A, G, rhs = asm.assemble(torch.as_tensor(u.T.copy()), rho=RHO, mu=MU, dt=DT)
    torch.cuda.synchronize()
    asm.close()
    _, _, oA, oG, orhs = oracle.assemble(coord, lnods, vel_in(u, precision), None, RHO, MU, DT)
    rp = oracle.pattern(5, lnods)[0]
    assert row_scaled_err(rp, A.double().cpu().numpy(), oA) <= TOL[precision]
    for d in range(3):
        assert row_scaled_err(rp, G[d].double().cpu().numpy(), oG[d]) <= TOL[precision]
        assert vec_scaled_err(rhs[d].double().cpu().numpy(), orhs[d]) <= TOL[precision]
