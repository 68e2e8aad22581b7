"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

The oracle cannot assemble 6-48 M tets in test time, so it computes sampled
rows one by one (every element touching a sampled row, in element order) and
the library's rows are compared to them; the CSR pattern is checked on the
same rows and through the closed-form Kuhn nnz.  Workloads: the 100^3 cube
(6 M tets, random numbering), the 200^3 cube (48 M tets) in RCM and random
numbering with 5% noise and mu in {1e-2, 1e-4} (with the stabilised block at
mu = 1e-4), 64 batched cubes of 10..60 hexes a side, and the 50^3 adjoint
case.
"""
import numpy as np
import pytest

import meshgen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nsi = pytest.importorskip("paper_2111_05651_gb300")

TOL = {"fp64": 1e-12, "mixed64": 1e-5, "mixed32": 1e-5}
RHO, MU, DT = meshgen.RHO, meshgen.MU, meshgen.DT


def kuhn_nnz(N):
    return (N + 1) ** 3 + 2 * (3 * N * (N + 1) ** 2 + 3 * N * N * (N + 1) + N ** 3)


def sample_rows(n, rng, k=48):
    return np.unique(np.concatenate([[0, 1, n // 2, n - 2, n - 1], rng.integers(0, n, k)]))


def check_rows(asm, out, mesh, u_in, rows, tol, mu=MU):
    """Row-scaled errors of sampled rows against the oracle; pattern of those rows bit-exact."""
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    A, G, rhs = (t.double().cpu().numpy() for t in out)
    ref = oracle.assemble_rows(mesh.coord, mesh.lnods, u_in, rows, None, RHO, mu, DT)
    worst = 0.0
    for r, (cols, a, g, rh) in zip(rows, ref):
        s, e = rp[r], rp[r + 1]
        np.testing.assert_array_equal(ci[s:e], cols)
        worst = max(worst, np.abs(A[s:e] - a).max() / np.abs(a).max())
        for d in range(3):
            worst = max(worst, np.abs(G[d, s:e] - g[d]).max() / np.abs(g[d]).max())
        worst = max(worst, np.abs(rhs[:, r] - rh).max() / max(np.abs(rhs).max(), 1e-300))
    assert worst <= tol, worst
    return worst


def vel_in(u, precision):
    return u if precision == "fp64" else u.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def cube100():
    return meshgen.config_mesh("cube100")


@pytest.mark.parametrize("precision,scatter", [("mixed64", "auto"), ("mixed32", "auto"), ("fp64", "auto"),
                                               ("mixed64", "color"), ("mixed64", "atomic")])
def test_cube100_sampled_rows(cube100, precision, scatter):
    mesh, u = cube100
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision, scatter=scatter)
    assert asm.nnz == kuhn_nnz(100) == 15210901
    assert asm.max_row == 15
    ut = torch.as_tensor(u.T.copy())
    out = asm.assemble(ut, rho=RHO, mu=MU, dt=DT)
    torch.cuda.synchronize()
    rows = sample_rows(mesh.n_nodes, np.random.default_rng(5))
    check_rows(asm, out, mesh, vel_in(u, precision), rows, TOL[precision])
    if precision != "fp64":
        check_rows(asm, out, mesh, u, rows, TOL[precision])
    rp = asm.pattern()[0].cpu().numpy()
    assert np.all(np.diff(rp) >= 1) and rp[-1] == asm.nnz
    asm.close()


@pytest.fixture(scope="module")
def cube100_oracle(cube100):
    """The oracle's full assembly of the 100^3 cube on its own CSR pattern: for
    the double velocities and for the same velocities rounded to float (what
    the mixed modes receive)."""
    mesh, u = cube100
    csr = oracle.pattern(mesh.n_nodes, mesh.lnods)
    full = {}
    for key, uu in (("f64", u), ("f32", vel_in(u, "mixed64"))):
        full[key] = oracle.assemble(mesh.coord, mesh.lnods, uu, None, RHO, MU, DT, csr=csr)
    return full


@pytest.mark.parametrize("precision", ["mixed64", "mixed32", "fp64"])
def test_cube100_every_row(cube100, cube100_oracle, precision):
    """Every row of A, G and rhs at the headline size (6 M tets), in the launch
    configuration bench.py times, element by element against the oracle:
    row-scaled error within the precision's bar, pattern bit-exact."""
    from tests._common import errors

    mesh, u = cube100
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    out = asm.assemble(torch.as_tensor(u.T.copy()), rho=RHO, mu=MU, dt=DT)
    torch.cuda.synchronize()
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    A, G, rhs = (t.double().cpu().numpy() for t in out)
    del out
    refs = ("f64",) if precision == "fp64" else ("f32", "f64")
    for key in refs:
        orp, oci, oA, oG, orhs = cube100_oracle[key]
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        err = errors(orp, A, G, rhs, oA, oG, orhs)
        assert max(err.values()) <= TOL[precision], (key, err)
    asm.close()


def test_cube100_colour_bit_reproducible(cube100):
    mesh, u = cube100
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64", scatter="color")
    ut = torch.as_tensor(u.T.copy())
    r1 = [t.clone() for t in asm.assemble(ut)]
    r2 = asm.assemble(ut)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(r1, r2))
    asm.close()


@pytest.mark.parametrize("name", ["cube200_rcm", "cube200_random"])
def test_cube200(name):
    mesh, u = meshgen.config_mesh(name)
    rows = sample_rows(mesh.n_nodes, np.random.default_rng(6), k=32)
    # mixed, float accumulation: gather, colour and atomic scatter at mu = 1e-2
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed32")
    assert asm.nnz == kuhn_nnz(200) == 120841801
    ut = torch.as_tensor(u.T.copy())
    for scatter in ("gather", "color", "atomic"):
        out = asm.assemble(ut, rho=RHO, mu=1e-2, dt=DT, scatter=scatter)
        torch.cuda.synchronize()
        check_rows(asm, out, mesh, vel_in(u, "mixed32"), rows, 1e-5, mu=1e-2)
        del out
    asm.close()
    # mixed64 (compensated sums where the row cancels; double outputs), mu = 1e-4
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    for scatter in ("gather", "atomic"):
        out = asm.assemble(ut, rho=RHO, mu=1e-4, dt=DT, scatter=scatter)
        torch.cuda.synchronize()
        check_rows(asm, out, mesh, vel_in(u, "mixed64"), rows, 1e-5, mu=1e-4)
        check_rows(asm, out, mesh, u, rows, 1e-5, mu=1e-4)
        del out
    # the stabilised velocity block at the same size (convective regime)
    Auu, G, rhs = (t.double().cpu().numpy() for t in asm.assemble_stabilized(ut, rho=RHO, mu=1e-4, dt=DT))
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    asm.close()
    ref = oracle.assemble_stabilized_rows(mesh.coord, mesh.lnods, vel_in(u, "mixed64"), rows, None, RHO, 1e-4, DT)
    worst = 0.0
    for r, (cols, blk, g, rh) in zip(rows, ref):
        s_, e_ = rp[r], rp[r + 1]
        np.testing.assert_array_equal(ci[s_:e_], cols)
        for c in range(9):
            worst = max(worst, np.abs(Auu[c, s_:e_] - blk[c]).max() / np.abs(blk[c]).max())
        for d in range(3):
            worst = max(worst, np.abs(G[d, s_:e_] - g[d]).max() / np.abs(g[d]).max())
        worst = max(worst, np.abs(rhs[:, r] - rh).max() / np.abs(rhs).max())
    assert worst <= 1e-5, worst


def test_batch64_batched_equals_single_and_oracle():
    meshes = meshgen.batch_meshes()
    assert len(meshes) == 64
    asms = [nsi.Assembler(m.coord, m.lnods, precision="mixed64") for m, _ in meshes]
    us = [torch.as_tensor(u.T.copy()) for _, u in meshes]
    batched = nsi.assemble_batched(asms, us, rho=RHO, mu=MU, dt=DT)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for k, (asm, (mesh, u)) in enumerate(zip(asms, meshes)):
        single = asm.assemble(us[k], rho=RHO, mu=MU, dt=DT)
        torch.cuda.synchronize()
        for a, b in zip(single, batched[k]):
            assert torch.equal(a, b)
        if k % 8 == 0:
            check_rows(asm, batched[k], mesh, vel_in(u, "mixed64"), sample_rows(mesh.n_nodes, rng, 6), 1e-5)
    for a in asms:
        a.close()


def test_batch64_graph_replay():
    """One CUDA graph (velocity update + batched assembly) replayed over steps
    gives the same result as direct calls."""
    meshes = meshgen.batch_meshes(count=8, lo=10, hi=20)
    asms = [nsi.Assembler(m.coord, m.lnods, precision="mixed32") for m, _ in meshes]
    base = [torch.as_tensor(u.T.copy()).cuda().float() for _, u in meshes]
    cur = [b.clone() for b in base]
    outs = [a.empty_outputs() for a in asms]
    step = torch.zeros(1, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        nsi.assemble_batched(asms, cur, outs=outs)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step.add_(1.0)
        for c, b in zip(cur, base):
            c.copy_(b * torch.cos(0.0628 * step))
        nsi.assemble_batched(asms, cur, outs=outs)
    for it in range(1, 4):
        g.replay()
        torch.cuda.synchronize()
        t_it = torch.full((1,), float(it), device="cuda")
        for a, b, o in zip(asms, base, outs):
            ref = a.assemble(b * torch.cos(0.0628 * t_it))  # the same float ops as in the graph
            torch.cuda.synchronize()
            for x, y in zip(o, ref):
                assert torch.equal(x, y)
    for a in asms:
        a.close()


def test_autotune_choice_and_cache(tmp_path):
    mesh, u = meshgen.config_mesh(N=20, jitter=0.15, numbering="random", seed=8)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    ut = torch.as_tensor(u.T.copy())
    ref = [t.clone() for t in asm.assemble(ut, scatter="gather")]
    cache = str(tmp_path / "tune.json")
    sc, rows = asm.autotune(ut, cache=cache, reps=3)
    assert sc in ("gather", "color", "atomic")
    if sc == "gather":
        assert rows in (-1, 32, 64, 96, 128)
    elif sc == "atomic":
        assert rows in (1, 2)  # warp-aggregated or one atomic per value
    out = asm.assemble(ut)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        torch.testing.assert_close(a, b, rtol=1e-6, atol=1e-9)
    asm2 = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    assert asm2.autotune(ut, cache=cache) == (sc, rows)  # from the cache, no timing
    assert asm2.scatter == asm.scatter
    asm.close()
    asm2.close()


def test_cube50_adjoint():
    mesh, u = meshgen.config_mesh("cube50")
    w = meshgen.gaussian_weights(mesh.n_nodes, np.random.default_rng(40))
    ogu, ogmu = oracle.vjp(mesh.coord, mesh.lnods, u, w, RHO, MU, DT)
    for precision, tol in (("fp64", 1e-12), ("mixed64", 1e-5)):
        asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
        gu, gmu = asm.vjp(torch.as_tensor(u.T.copy()), torch.as_tensor(w.T.copy()), rho=RHO, mu=MU, dt=DT)
        gu = gu.double().cpu().numpy().T
        ref_gu, ref_gmu = (ogu, ogmu) if precision == "fp64" else oracle.vjp(
            mesh.coord, mesh.lnods, vel_in(u, precision), vel_in(w, precision), RHO, MU, DT)
        assert np.abs(gu - ref_gu).max() <= tol * np.abs(ref_gu).max()
        # a sum of terms of both signs over every element: scaled by the sum
        # of the terms' magnitudes (the standard bound of a floating-point sum)
        ref_abs = oracle.vjp_mu_abs(mesh.coord, mesh.lnods, vel_in(u, precision), vel_in(w, precision),
                                    RHO, MU, DT)
        assert abs(gmu.item() - ref_gmu) <= tol * ref_abs
        if precision == "fp64":
            # central differences of the library's own residual (exact for a quadratic R)
            rng = np.random.default_rng(41)
            ut = torch.as_tensor(u.T.copy()).cuda()
            wt = torch.as_tensor(w.T.copy()).cuda()
            h = 1e-6
            for _ in range(2):
                v = torch.as_tensor(rng.standard_normal(ut.shape)).cuda()
                Rp = asm.residual(ut + h * v, rho=RHO, mu=MU, dt=DT, u_n=ut)
                Rm = asm.residual(ut - h * v, rho=RHO, mu=MU, dt=DT, u_n=ut)
                fd = float((wt * (Rp - Rm)).sum() / (2 * h))
                assert float((torch.as_tensor(gu.T).cuda() * v).sum()) == pytest.approx(fd, rel=1e-6)
        asm.close()
