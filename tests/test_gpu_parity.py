"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars: CSR pattern bit-exact; FP64 mode within 1e-12 row-scaled error; mixed
modes within 1e-5 (the benchmark spec's tolerances), both against the oracle fed
the exact inputs the kernels see (mixed modes receive float32 velocities, so
the oracle is run on those values promoted to float64) and, for the mixed
modes, also against the oracle on the original float64 velocities.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests._common import errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


def _run(mesh, u, precision, scatter, un=None, rho=RHO, mu=MU, dt=DT, debug=False):
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter=scatter, debug_checks=debug)
    ut = torch.as_tensor(u.T.copy())
    unt = torch.as_tensor(un.T.copy()) if un is not None else None
    A, G, rhs = asm.assemble(ut, unt, rho=rho, mu=mu, dt=dt)
    torch.cuda.synchronize()
    if debug:
        asm.device_status()
    rp, ci = asm.pattern()
    res = (rp.cpu().numpy(), ci.cpu().numpy(), A.double().cpu().numpy(), G.double().cpu().numpy(),
           rhs.double().cpu().numpy())
    asm.close()
    return res


def _oracle(mesh, u, precision, un=None, rho=RHO, mu=MU, dt=DT):
    if precision != "fp64":
        u = u.astype(np.float32).astype(np.float64)
        un = None if un is None else un.astype(np.float32).astype(np.float64)
    return oracle.assemble(mesh.coord, mesh.lnods, u, un, rho, mu, dt)


CASES = [
    ("cube8", dict(name="cube8")),
    ("cube6_jit_random", dict(N=6, jitter=0.15, numbering="random", seed=31)),
    ("cube7_jit_rcm", dict(N=7, jitter=0.15, numbering="rcm", seed=32, noise=0.05)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("scatter", ["gather", "color", "atomic"])
def test_parity_vs_oracle(case, precision, scatter):
    name, kw = case
    mesh, u = meshgen.config_mesh(**kw) if "name" not in kw else meshgen.config_mesh(kw["name"])
    rp, ci, A, G, rhs = _run(mesh, u, precision, scatter)
    orp, oci, oA, oG, orhs = _oracle(mesh, u, precision)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], err
    if precision != "fp64":
        # also against the unrounded float64 velocities
        _, _, fA, fG, frhs = oracle.assemble(mesh.coord, mesh.lnods, u, None, RHO, MU, DT)
        err2 = errors(rp, A, G, rhs, fA, fG, frhs)
        assert max(err2.values()) <= TOL[precision], err2


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
@pytest.mark.parametrize("scatter", ["gather", "color", "atomic"])
def test_integer_valued_assembly_is_exact(precision, scatter):
    """Integer lattice (unit Kuhn tets, det = 1), integer velocities below 2^19,
    rho = 120 (rho/120 = 1), mu = 0 and dt = 5 / 2^20 (lumped mass rho|T|/(4 dt)
    = 2^20 per element): every element term of A and of the RHS is an integer
    exact in float (the convection terms below 2^22), while the diagonal
    entries, the lumped mass minus the row's other entries, need up to 26 bits
    (the off-diagonal sums stay below 2^24, exact in float).  FP64 and
    mixed64's compensated float-pair diagonal, lumped mass and RHS with their
    conversion to double must then give the exact integers: the oracle's values rounded to
    the nearest integer (its 4-point quadrature leaves them within 1e-3 of
    one).  The cached-geometry time step (A_static + C(u)) must give them too."""
    N = 7
    mesh, _ = meshgen.config_mesh(N=N, numbering="random", seed=86)
    coord = np.rint(mesh.coord * N)
    rng = np.random.default_rng(87)
    u = rng.integers(-2**19, 2**19, size=(mesh.n_nodes, 3)).astype(np.float64)
    un = rng.integers(-2**10, 2**10, size=(mesh.n_nodes, 3)).astype(np.float64)
    rho, mu, dt = 120.0, 0.0, 5.0 / 2**20
    _, _, oA, _, orhs = oracle.assemble(coord, mesh.lnods, u, un, rho, mu, dt)
    iA, irhs = np.rint(oA), np.rint(orhs)
    assert np.abs(oA - iA).max() < 1e-3 and np.abs(orhs - irhs).max() < 1e-3
    assert (iA.astype(np.float32).astype(np.float64) != iA).sum() >= 10  # entries past float's integers
    asm = nsi.Assembler(coord, mesh.lnods, precision=precision, scatter=scatter)
    ut, unt = torch.as_tensor(u.T.copy()), torch.as_tensor(un.T.copy())
    A, _, rhs = asm.assemble(ut, unt, rho=rho, mu=mu, dt=dt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(A.cpu().numpy(), iA)
    np.testing.assert_array_equal(rhs.cpu().numpy(), irhs)
    if scatter == "gather":
        A_static, _ = asm.static_part(rho=rho, mu=mu, dt=dt)
        A2, rhs2 = asm.assemble_convective(ut, A_static, u_n=unt, rho=rho, mu=mu, dt=dt)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(A2.cpu().numpy(), iA)
        np.testing.assert_array_equal(rhs2.cpu().numpy(), irhs)
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_warp_aggregated_atomics(precision):
    """The atomic scatter with warp aggregation (nsi_set_launch(ATOMIC, 1)):
    same results as the oracle within the precision's bar on a randomly
    numbered jittered mesh and a Delaunay mesh, and the exact integers of the
    integer lattice in FP64 and mixed64 (the lanes' partial sums are formed in
    the output type)."""
    for mesh, u in (meshgen.config_mesh(N=9, jitter=0.15, numbering="random", seed=91),
                    meshgen.delaunay_cube(m=7, jitter=0.3, seed=92)):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter="atomic")
        nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_ATOMIC, 1)
        A, G, rhs = (t.double().cpu().numpy() for t in asm.assemble(torch.as_tensor(u.T.copy())))
        rp = asm.pattern()[0].cpu().numpy()
        asm.close()
        orp, oci, oA, oG, orhs = _oracle(mesh, u, precision)
        np.testing.assert_array_equal(rp, orp)
        err = errors(rp, A, G, rhs, oA, oG, orhs)
        assert max(err.values()) <= TOL[precision], err
    if precision != "mixed32":
        N = 7
        mesh, _ = meshgen.config_mesh(N=N, numbering="random", seed=86)
        coord = np.rint(mesh.coord * N)
        rng = np.random.default_rng(87)
        u = rng.integers(-2**19, 2**19, size=(mesh.n_nodes, 3)).astype(np.float64)
        rho, mu, dt = 120.0, 0.0, 5.0 / 2**20
        _, _, oA, _, orhs = oracle.assemble(coord, mesh.lnods, u, None, rho, mu, dt)
        asm = nsi.Assembler(coord, mesh.lnods, precision=precision, scatter="atomic")
        nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_ATOMIC, 1)
        A, _, rhs = asm.assemble(torch.as_tensor(u.T.copy()), rho=rho, mu=mu, dt=dt)
        np.testing.assert_array_equal(A.cpu().numpy(), np.rint(oA))
        np.testing.assert_array_equal(rhs.cpu().numpy(), np.rint(orhs))
        asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("bad", [np.nan, np.inf], ids=["nan", "inf"])
def test_nonfinite_velocity_propagates(precision, bad):
    """A NaN or infinite velocity at one node makes the A entries and the RHS
    of that node's row non-finite, in the assembly and in the cached-geometry
    step; rows outside its neighbourhood and G (velocity-free) stay finite."""
    mesh, u = meshgen.config_mesh(N=6, jitter=0.1, numbering="random", seed=88)
    b = int(np.argmin(np.abs(mesh.coord - 0.5).sum(1)))  # an interior node
    u = u.copy()
    u[b, 1] = bad
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = (x.double().cpu().numpy() for x in asm.assemble(ut))
    A_static, _ = asm.static_part()
    A2, rhs2 = (x.double().cpu().numpy() for x in asm.assemble_convective(ut, A_static))
    rp, ci = (x.cpu().numpy() for x in asm.pattern())
    asm.close()
    near = np.zeros(mesh.n_nodes, dtype=bool)
    near[ci[rp[b]:rp[b + 1]]] = True  # b and its neighbours
    far = np.repeat(~near, np.diff(rp))
    for a, r in ((A, rhs), (A2, rhs2)):
        assert not np.isfinite(a[rp[b]:rp[b + 1]]).all()
        assert not np.isfinite(r[1, b])
        assert np.isfinite(a[far]).all()
        assert np.isfinite(r[:, ~near]).all()
    assert np.isfinite(G).all()


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
def test_separate_rhs_velocity(precision):
    mesh, u = meshgen.config_mesh(N=5, jitter=0.1, numbering="random", seed=40)
    un = np.random.default_rng(41).standard_normal(u.shape)
    rp, ci, A, G, rhs = _run(mesh, u, precision, "gather", un=un, rho=1.3, mu=0.02, dt=0.05)
    _, _, oA, oG, orhs = _oracle(mesh, u, precision, un=un, rho=1.3, mu=0.02, dt=0.05)
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], err


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("scatter", ["gather", "color"])
def test_deterministic_bitwise(precision, scatter):
    """Gather and colour scatter are run-to-run bit-reproducible."""
    mesh, u = meshgen.config_mesh(N=9, jitter=0.15, numbering="random", seed=42)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter=scatter)
    ut = torch.as_tensor(u.T.copy())
    r1 = [t.clone() for t in asm.assemble(ut)]
    r2 = asm.assemble(ut)
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)


def test_single_tet_and_isolated_node():
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [5, 5, 5]], dtype=float)
    lnods = np.array([[0, 1, 2, 3]], dtype=np.int32)
    u = np.random.default_rng(3).standard_normal((5, 3))
    mesh = meshgen.Mesh(coord=coord, lnods=lnods)
    for precision in ["fp64", "mixed64", "mixed32"]:
        for scatter in ["gather", "color", "atomic"]:
            rp, ci, A, G, rhs = _run(mesh, u, precision, scatter)
            orp, oci, oA, oG, orhs = _oracle(mesh, u, precision)
            np.testing.assert_array_equal(rp, orp)
            np.testing.assert_array_equal(ci, oci)
            assert rp[4] == rp[5]                  # isolated node: empty row
            assert np.all(rhs[:, 4] == 0)
            err = errors(rp, A, G, rhs, oA, oG, orhs)
            assert max(err.values()) <= TOL[precision], (precision, scatter, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("scatter", ["gather", "color", "atomic"])
def test_mesh_without_elements(precision, scatter):
    """Nodes and no elements: an empty pattern (nnz = 0, NULL A and G are
    accepted), a zero RHS, and the same from the time-step entry points."""
    coord = np.random.default_rng(91).standard_normal((7, 3))
    lnods = np.zeros((0, 4), dtype=np.int32)
    asm = nsi.Assembler(coord, lnods, precision=precision, scatter=scatter)
    assert asm.nnz == 0
    ut = torch.as_tensor(np.random.default_rng(92).standard_normal((3, 7)))
    A, G, rhs = asm.assemble(ut)
    torch.cuda.synchronize()
    assert A.numel() == 0 and G.numel() == 0
    assert torch.count_nonzero(rhs) == 0
    rp = asm.pattern()[0].cpu().numpy()
    assert np.all(rp == 0)
    if scatter == "gather":
        A_static, _ = asm.static_part()
        A2, rhs2 = asm.assemble_convective(ut, A_static)
        r3, dtr, mr = asm.nodal(ut)
        torch.cuda.synchronize()
        assert A2.numel() == 0 and torch.count_nonzero(rhs2) == 0
        assert torch.count_nonzero(r3) == 0 and torch.count_nonzero(dtr) == 0 and torch.count_nonzero(mr) == 0
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_edge_fan_kernel_matches_oracle(precision):
    """The edge-fan variant of the row gather (selected with nsi_set_launch(-1))."""
    for kw in (dict(N=7, jitter=0.15, numbering="random", seed=71), dict(name="cube8")):
        mesh, u = meshgen.config_mesh(**kw) if "name" not in kw else meshgen.config_mesh(kw["name"])
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter="gather")
        nsi.nsi_set_launch(asm.handle, nsi.NSI_SCATTER_GATHER, -1)
        assert asm.info().rows_per_block == -1
        A, G, rhs = asm.assemble(torch.as_tensor(u.T.copy()))
        rp, ci = asm.pattern()
        _, _, oA, oG, orhs = _oracle(mesh, u, precision)
        err = errors(rp.cpu().numpy(), A.double().cpu().numpy(), G.double().cpu().numpy(),
                     rhs.double().cpu().numpy(), oA, oG, orhs)
        assert max(err.values()) <= TOL[precision], err
        asm.close()


def test_ragged_row_blocks():
    """n not a multiple of the rows-per-block and rows of uneven length (boundary)."""
    mesh, u = meshgen.config_mesh(N=11, jitter=0.15, numbering="random", seed=43)
    assert mesh.n_nodes % 128 != 0
    rp, ci, A, G, rhs = _run(mesh, u, "mixed64", "gather")
    _, _, oA, oG, orhs = _oracle(mesh, u, "mixed64")
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= 1e-5, err


def test_debug_checks_clean():
    mesh, u = meshgen.config_mesh(N=5, jitter=0.1, numbering="random", seed=44)
    for precision in ["fp64", "mixed64"]:
        for scatter in ["gather", "color", "atomic"]:
            rp, ci, A, G, rhs = _run(mesh, u, precision, scatter, debug=True)
            _, _, oA, oG, orhs = _oracle(mesh, u, precision)
            err = errors(rp, A, G, rhs, oA, oG, orhs)
            assert max(err.values()) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_batched_equals_single(precision):
    meshes = [meshgen.config_mesh(N=n, jitter=0.15, numbering="natural", seed=50 + n) for n in (3, 7, 5)]
    asms = [nsi.Assembler(m.coord, m.lnods, precision=precision) for m, _ in meshes]
    us = [torch.as_tensor(u.T.copy()) for _, u in meshes]
    singles = [[t.clone() for t in a.assemble(u)] for a, u in zip(asms, us)]
    batched = nsi.assemble_batched(asms, us)
    torch.cuda.synchronize()
    for s, b in zip(singles, batched):
        for x, y in zip(s, b):
            assert torch.equal(x, y)


@pytest.mark.parametrize("pinned", ["all", "none", "inputs"])
@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_host_end_to_end_matches_device(precision, pinned):
    """nsi_assemble_host gives the device call's bits, with every buffer pinned
    (the kernels read and write host memory directly) and with pageable
    buffers or a mix (staged copies)."""
    mesh, u = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=45)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = asm.assemble(ut)

    def host(t, pin):
        return t.pin_memory() if pin else t

    uh = host(ut.to(asm.vel_dtype), pinned != "none")
    Ah = host(torch.empty(asm.nnz, dtype=asm.out_dtype), pinned == "all")
    Gh = host(torch.empty(3, asm.nnz, dtype=asm.out_dtype), pinned == "all")
    rh = host(torch.empty(3, asm.n, dtype=asm.out_dtype), pinned == "all")
    asm.assemble_host(uh, Ah, Gh, rh)
    assert torch.equal(A.cpu(), Ah)
    assert torch.equal(G.cpu(), Gh)
    assert torch.equal(rhs.cpu(), rh)
    asm.close()


def test_host_end_to_end_badly_shaped_elements():
    """The direct host path also runs the double-precision fix-up of the rows
    of badly shaped elements (on the host buffers)."""
    mesh, u = _sliver_mesh()
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    assert asm.info().exact_rows > 0
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = asm.assemble(ut)
    uh = ut.float().pin_memory()
    Ah = torch.empty(asm.nnz, dtype=torch.float64).pin_memory()
    Gh = torch.empty(3, asm.nnz, dtype=torch.float64).pin_memory()
    rh = torch.empty(3, asm.n, dtype=torch.float64).pin_memory()
    asm.assemble_host(uh, Ah, Gh, rh)
    assert torch.equal(A.cpu(), Ah) and torch.equal(G.cpu(), Gh) and torch.equal(rhs.cpu(), rh)
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
def test_residual_matches_oracle(precision):
    mesh, u = meshgen.config_mesh(N=5, jitter=0.15, numbering="random", seed=46)
    un = np.random.default_rng(2).standard_normal(u.shape)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    R = asm.residual(torch.as_tensor(u.T.copy()), u_n=torch.as_tensor(un.T.copy())).double().cpu().numpy()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    uno = un if precision == "fp64" else un.astype(np.float32).astype(np.float64)
    rp, ci, oA, oG, orhs = oracle.assemble(mesh.coord, mesh.lnods, uo, uno)
    Ro = oracle.residual((rp, ci, oA), orhs, uo)   # [n, 3]
    tol = 1e-12 if precision == "fp64" else 1e-5
    scale = np.abs(Ro).max()
    assert np.abs(R.T - Ro).max() <= tol * scale


@pytest.mark.parametrize("precision", ["fp64", "mixed64"])
def test_vjp_matches_oracle(precision):
    mesh, u = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=47)
    w = np.random.default_rng(40).standard_normal(u.shape)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    gu, gmu = asm.vjp(torch.as_tensor(u.T.copy()), torch.as_tensor(w.T.copy()))
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    wo = w if precision == "fp64" else w.astype(np.float32).astype(np.float64)
    ogu, ogmu = oracle.vjp(mesh.coord, mesh.lnods, uo, wo, RHO, MU, DT)
    tol = 1e-12 if precision == "fp64" else 1e-5
    gu = gu.double().cpu().numpy().T
    assert np.abs(gu - ogu).max() <= tol * np.abs(ogu).max()
    # grad_mu is one sum of terms of both signs over every element: its error
    # is bounded by the rounding unit times the sum of the terms' magnitudes
    # (the standard bound for a floating-point sum), so that sum is the scale
    gabs = oracle.vjp_mu_abs(mesh.coord, mesh.lnods, uo, wo, RHO, MU, DT)
    assert abs(float(gmu.item()) - ogmu) <= tol * gabs


def test_autograd_residual():
    mesh, u = meshgen.config_mesh(N=4, jitter=0.15, numbering="natural", seed=48)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="fp64")
    ut = torch.as_tensor(u.T.copy()).cuda().requires_grad_(True)
    mu = torch.tensor(0.01, dtype=torch.float64, requires_grad=True)
    w = torch.randn(3, mesh.n_nodes, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    R = nsi.NsiResidual.apply(ut, mu, asm, 1.0, 0.01)
    (R * w).sum().backward()
    ogu, ogmu = oracle.vjp(mesh.coord, mesh.lnods, u, w.cpu().numpy().T, 1.0, 0.01, 0.01)
    assert np.abs(ut.grad.cpu().numpy().T - ogu).max() <= 1e-12 * np.abs(ogu).max()
    assert mu.grad.item() == pytest.approx(ogmu, rel=1e-11)


def test_bad_meshes_rejected():
    coord = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    with pytest.raises(nsi.NsiError) as ex:
        nsi.Assembler(coord, np.array([[0, 1, 3, 2]], dtype=np.int32))     # inverted
    assert ex.value.status == nsi.NSI_ERR_BAD_MESH
    with pytest.raises(nsi.NsiError) as ex:
        nsi.Assembler(coord, np.array([[0, 1, 2, 4]], dtype=np.int32))     # out of range
    assert ex.value.status == nsi.NSI_ERR_BAD_MESH
    with pytest.raises(nsi.NsiError) as ex:
        nsi.Assembler(coord, np.array([[0, 1, 2, 2]], dtype=np.int32))     # degenerate
    assert ex.value.status == nsi.NSI_ERR_BAD_MESH


def _fan_mesh(m):
    """m tets around the vertical edge from node 0 (origin) to node m + 1 (top),
    with a ring of m nodes: rows 0 and m + 1 have m + 2 entries."""
    ang = 2 * np.pi * np.arange(m) / m
    coord = np.vstack([[0, 0, 0], np.c_[np.cos(ang), np.sin(ang), np.zeros(m)], [0, 0, 1]]).astype(float)
    lnods = []
    for k in range(m):
        t = [0, 1 + k, 1 + (k + 1) % m, m + 1]
        X = coord[t]
        if np.linalg.det(np.c_[X[1] - X[0], X[2] - X[0], X[3] - X[0]]) < 0:
            t[2], t[3] = t[3], t[2]
        lnods.append(t)
    u = np.random.default_rng(90 + m).standard_normal(coord.shape)
    return coord, np.array(lnods, dtype=np.int32), u


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_longest_rows_of_the_row_gather(precision):
    """Rows of 32 entries, the most the row-gather kernels take (five bits of
    row position per walk step), run on them and match the oracle, in the
    assembly and the cached-geometry step; with 33-entry rows the mesh stays
    on the row gather, the two long rows computed by the per-row kernel."""
    coord, lnods, u = _fan_mesh(30)
    asm = nsi.Assembler(coord, lnods, precision=precision)
    assert asm.max_row == 32 and asm.scatter == nsi.SCATTERS["gather"]
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = (x.double().cpu().numpy() for x in asm.assemble(ut))
    A_static, _ = asm.static_part()
    A2, rhs2 = (x.double().cpu().numpy() for x in asm.assemble_convective(ut, A_static))
    rp, ci = (x.cpu().numpy() for x in asm.pattern())
    asm.close()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    orp, oci, oA, oG, orhs = oracle.assemble(coord, lnods, uo, None, RHO, MU, DT)
    np.testing.assert_array_equal(ci, oci)
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], err
    err2 = errors(rp, A2, oG, rhs2, oA, oG, orhs)
    assert max(err2.values()) <= TOL[precision], err2
    coord, lnods, u = _fan_mesh(31)
    asm = nsi.Assembler(coord, lnods, precision=precision)
    assert asm.max_row == 33 and asm.scatter == nsi.SCATTERS["gather"] and asm.info().long_rows == 2
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = (x.double().cpu().numpy() for x in asm.assemble(ut))
    A_static, _ = asm.static_part()
    A2, rhs2 = (x.double().cpu().numpy() for x in asm.assemble_convective(ut, A_static))
    At, Gt, rhst = (x.double().cpu().numpy() for x in asm.assemble(ut, scatter="atomic"))
    rp = asm.pattern()[0].cpu().numpy()
    asm.close()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    _, _, oA, oG, orhs = oracle.assemble(coord, lnods, uo, None, RHO, MU, DT)
    for got in ((A, G, rhs), (A2, oG, rhs2), (At, Gt, rhst)):
        err = errors(rp, *got, oA, oG, orhs)
        assert max(err.values()) <= TOL[precision], err


def _sliver_mesh():
    """4^3 Kuhn cube with node (2,2,2) moved by 0.499 h along (1,-1,0): every
    tet stays positive, two become slivers whose |d1||d2||d3| / |det| is about
    1.1e3 (a float determinant would be off by about that many roundings)."""
    mesh, u = meshgen.config_mesh(N=4, jitter=0.0, numbering="natural", seed=0)
    coord = mesh.coord.copy()
    coord[2 + 5 * (2 + 5 * 2)] += 0.499 * 0.25 * np.array([1.0, -1.0, 0.0])
    return meshgen.Mesh(coord=coord, lnods=mesh.lnods, N=4), u


@pytest.mark.parametrize("precision", ["mixed64", "mixed32"])
def test_badly_shaped_elements_in_the_adjoint_and_residual(precision):
    """The sliver mesh through nsi_assemble_vjp and nsi_residual in a mixed
    precision: the badly shaped elements are taken in double (a float
    determinant would carry ~1e3 float roundings), so both match the oracle
    on the float velocities at the mixed bar (grad_mu relative to the sum of
    its terms' magnitudes)."""
    mesh, u = _sliver_mesh()
    w = np.random.default_rng(97).standard_normal(u.shape)
    un = np.random.default_rng(98).standard_normal(u.shape)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    assert asm.info().exact_rows > 0
    gu, gmu = asm.vjp(torch.as_tensor(u.T.copy()), torch.as_tensor(w.T.copy()))
    R = asm.residual(torch.as_tensor(u.T.copy()), u_n=torch.as_tensor(un.T.copy())).double().cpu().numpy()
    asm.close()
    uo, wo, uno = (x.astype(np.float32).astype(np.float64) for x in (u, w, un))
    ogu, ogmu = oracle.vjp(mesh.coord, mesh.lnods, uo, wo, RHO, MU, DT)
    gu = gu.double().cpu().numpy().T
    assert np.abs(gu - ogu).max() <= 1e-5 * np.abs(ogu).max()
    gabs = oracle.vjp_mu_abs(mesh.coord, mesh.lnods, uo, wo, RHO, MU, DT)
    assert abs(float(gmu.item()) - ogmu) <= 1e-5 * gabs
    rp, ci, oA, oG, orhs = oracle.assemble(mesh.coord, mesh.lnods, uo, uno)
    Ro = oracle.residual((rp, ci, oA), orhs, uo)
    assert np.abs(R.T - Ro).max() <= 1e-5 * np.abs(Ro).max()


@pytest.mark.parametrize("precision", ["mixed64", "mixed32"])
def test_badly_shaped_elements_use_double_determinants(precision):
    mesh, u = _sliver_mesh()
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter="gather")
    assert asm.info().exact_rows > 0
    ut = torch.as_tensor(u.T.copy())
    A, G, rhs = asm.assemble(ut)
    torch.cuda.synchronize()
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    _, _, oA, oG, orhs = _oracle(mesh, u, precision)
    err = errors(rp, A.double().cpu().numpy(), G.double().cpu().numpy(), rhs.double().cpu().numpy(), oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], err
    # the time-step kernels take the same path for the determinant sums
    A_static, _ = asm.static_part()
    A2, rhs2 = asm.assemble_convective(ut, A_static)
    r3, dtr, mr = asm.nodal(ut)
    torch.cuda.synchronize()
    from tests._common import row_scaled_err, vec_scaled_err
    assert row_scaled_err(rp, A2.double().cpu().numpy(), oA) <= TOL[precision]
    onr, ondt, onm = oracle.nodal(mesh.coord, mesh.lnods, u.astype(np.float32).astype(np.float64), RHO, DT)
    for k in range(3):
        assert vec_scaled_err(rhs2[k].double().cpu().numpy(), orhs[k]) <= TOL[precision]
        assert vec_scaled_err(r3[k].double().cpu().numpy(), onr[k]) <= TOL[precision]
    assert vec_scaled_err(mr.double().cpu().numpy(), onm) <= TOL[precision]
    asm.close()


def test_regular_meshes_flag_no_rows():
    mesh, u = meshgen.config_mesh(N=8, jitter=0.15, numbering="random", seed=91)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    assert asm.info().exact_rows == 0
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("scatter", ["gather", "color", "atomic"])
def test_delaunay_mesh_parity(precision, scatter):
    """An unstructured mesh (Delaunay tetrahedralization of a jittered lattice):
    irregular stars of 5..24 entries, holes (several walks per row), slivers."""
    mesh, u = meshgen.delaunay_cube(8, 0.25, seed=7)
    rp, ci, A, G, rhs = _run(mesh, u, precision, scatter)
    orp, oci, oA, oG, orhs = _oracle(mesh, u, precision)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    err = errors(rp, A, G, rhs, oA, oG, orhs)
    assert max(err.values()) <= TOL[precision], (precision, scatter, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_delaunay_mesh_steps(precision):
    from tests._common import row_scaled_err, vec_scaled_err

    mesh, u = meshgen.delaunay_cube(10, 0.3, seed=8)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    if precision != "fp64":
        assert asm.info().exact_rows > 0  # the slivers' rows
    ut = torch.as_tensor(u.T.copy())
    A_static, _ = asm.static_part()
    A, rhs = asm.assemble_convective(ut, A_static)
    r3, dtr, mr = asm.nodal(ut)
    torch.cuda.synchronize()
    rp = asm.pattern()[0].cpu().numpy()
    uo = u if precision == "fp64" else u.astype(np.float32).astype(np.float64)
    _, _, oA, _, orhs = oracle.assemble(mesh.coord, mesh.lnods, uo, None, RHO, MU, DT)
    onr, ondt, onm = oracle.nodal(mesh.coord, mesh.lnods, uo, RHO, DT)
    assert row_scaled_err(rp, A.double().cpu().numpy(), oA) <= TOL[precision]
    for k in range(3):
        assert vec_scaled_err(rhs[k].double().cpu().numpy(), orhs[k]) <= TOL[precision]
        assert vec_scaled_err(r3[k].double().cpu().numpy(), onr[k]) <= TOL[precision]
    assert vec_scaled_err(dtr.double().cpu().numpy(), ondt) <= TOL[precision]
    assert vec_scaled_err(mr.double().cpu().numpy(), onm) <= TOL[precision]
    asm.close()
