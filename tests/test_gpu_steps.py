"""GPU parity of the time-step entry points, through the C ABI.

nsi_assemble_convective (cached geometry): A = A_static + C(u) with A_static
the full assembly at u = 0 must equal the oracle's A(u), and its rhs the
oracle's; G is left alone.  nsi_assemble_nodal: the paper's per-node
outputs (rhsid, dt_rho_nsi, mass_rho_nsi of Listing 2) against the oracle's
``nodal``.  Bars as in the other parity tests: FP64 1e-12, mixed 1e-5.
"""
import ctypes

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


CASES = [
    dict(name="cube8"),
    dict(N=9, jitter=0.15, numbering="random", seed=81),
    dict(N=7, jitter=0.15, numbering="rcm", seed=82, noise=0.05),
]


def _mesh(kw):
    return meshgen.config_mesh(kw["name"]) if "name" in kw else meshgen.config_mesh(**kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_convective_step_matches_oracle(precision, ci):
    mesh, u = _mesh(CASES[ci])
    rng = np.random.default_rng(83 + ci)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    A_static, G_static = asm.static_part(rho=RHO, mu=MU, dt=DT)
    rp = asm.pattern()[0].cpu().numpy()
    G_before = G_static.clone()
    for step in range(3):  # several steps on one cached A_static
        uu = meshgen.add_noise(u, 0.2 * step, rng)
        un = meshgen.add_noise(u, 0.1, rng)
        A, rhs = asm.assemble_convective(torch.as_tensor(uu.T.copy()), A_static,
                                         u_n=torch.as_tensor(un.T.copy()), rho=RHO, mu=MU, dt=DT)
        torch.cuda.synchronize()
        _, _, oA, oG, orhs = oracle.assemble(mesh.coord, mesh.lnods, vel_in(uu, precision), vel_in(un, precision),
                                             RHO, MU, DT)
        assert row_scaled_err(rp, A.double().cpu().numpy(), oA) <= TOL[precision]
        for k in range(3):
            assert vec_scaled_err(rhs[k].double().cpu().numpy(), orhs[k]) <= TOL[precision]
        # the full assembly of the same step agrees within the bar too
        fA, fG, frhs = asm.assemble(torch.as_tensor(uu.T.copy()), torch.as_tensor(un.T.copy()), rho=RHO, mu=MU,
                                    dt=DT)
        torch.cuda.synchronize()
        assert row_scaled_err(rp, A.double().cpu().numpy(), fA.double().cpu().numpy()) <= 2 * TOL[precision]
        # the velocity-independent part: G of the static call is the oracle's G
        for d in range(3):
            assert row_scaled_err(rp, G_static[d].double().cpu().numpy(), oG[d]) <= TOL[precision]
    assert torch.equal(G_static, G_before)  # the step does not touch G
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
def test_convective_step_in_place_and_deterministic(precision):
    """A_val may alias A_static; two identical calls give identical bits."""
    mesh, u = meshgen.config_mesh(N=10, jitter=0.15, numbering="random", seed=84)
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    A_static, _ = asm.static_part()
    ut = torch.as_tensor(u.T.copy())
    A1, r1 = asm.assemble_convective(ut, A_static)
    A2, r2 = asm.assemble_convective(ut, A_static)
    torch.cuda.synchronize()
    assert torch.equal(A1, A2) and torch.equal(r1, r2)
    work = A_static.clone()
    A3, _ = asm.assemble_convective(ut, work, out=(work, torch.empty_like(r1)))
    torch.cuda.synchronize()
    assert A3.data_ptr() == work.data_ptr()
    assert torch.equal(A3, A1)
    asm.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed64", "mixed32"])
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_nodal_outputs_match_oracle(precision, ci):
    mesh, u = _mesh(CASES[ci])
    rho, dt = 1.3, 0.02
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision=precision)
    rhs, dtr, mr = asm.nodal(torch.as_tensor(u.T.copy()), rho=rho, dt=dt)
    torch.cuda.synchronize()
    orhs, odtr, omr = oracle.nodal(mesh.coord, mesh.lnods, vel_in(u, precision), rho, dt)
    for k in range(3):
        assert vec_scaled_err(rhs[k].double().cpu().numpy(), orhs[k]) <= TOL[precision]
    assert vec_scaled_err(dtr.double().cpu().numpy(), odtr) <= TOL[precision]
    assert vec_scaled_err(mr.double().cpu().numpy(), omr) <= TOL[precision]
    assert float(mr.double().sum()) == pytest.approx(rho, rel=10 * TOL[precision])  # rho x unit-cube volume
    asm.close()


def test_steps_take_rows_beyond_the_walk():
    """Rows of more than 32 entries (a fan of 40 tets around an edge: rows of
    42 entries at its two ends) no longer make the time-step kernels refuse the
    mesh: those rows are computed by the per-row kernel.  Checked against the
    oracle's assembly at u = 0 (A_static) plus the convection."""
    m = 40
    ang = 2 * np.pi * np.arange(m) / m
    coord = np.vstack([[0, 0, 0], np.c_[np.cos(ang), np.sin(ang), np.zeros(m)], [0, 0, 1]]).astype(float)
    top = m + 1
    lnods = []
    for k in range(m):
        t = [0, 1 + k, 1 + (k + 1) % m, top]
        X = coord[t]
        if np.linalg.det(np.c_[X[1] - X[0], X[2] - X[0], X[3] - X[0]]) < 0:
            t[2], t[3] = t[3], t[2]
        lnods.append(t)
    lnods = np.array(lnods, dtype=np.int32)
    u = np.random.default_rng(94).standard_normal(coord.shape)
    asm = nsi.Assembler(coord, lnods, precision="mixed64")
    assert asm.max_row == 42 and asm.info().long_rows == 2
    ut = torch.as_tensor(u.T.copy())
    A_static, _ = asm.static_part(rho=RHO, mu=MU, dt=DT)
    A, rhs = (x.double().cpu().numpy() for x in asm.assemble_convective(ut, A_static, rho=RHO, mu=MU, dt=DT))
    rp = asm.pattern()[0].cpu().numpy()
    asm.close()
    _, _, oA, oG, orhs = oracle.assemble(coord, lnods, vel_in(u, "mixed64"), None, RHO, MU, DT)
    assert row_scaled_err(rp, A, oA) <= TOL["mixed64"]
    for k in range(3):
        assert vec_scaled_err(rhs[k], orhs[k]) <= TOL["mixed64"]
    with pytest.raises(nsi.NsiError):
        asm.nodal(u)
    asm.close()


def test_convective_cube100_sampled_rows():
    """The 100^3 cube (6 M tets), mixed64: sampled rows against the oracle."""
    mesh, u = meshgen.config_mesh("cube100")
    asm = nsi.Assembler(mesh.coord, mesh.lnods, precision="mixed64")
    A_static, _ = asm.static_part()
    A, rhs = asm.assemble_convective(torch.as_tensor(u.T.copy()), A_static)
    torch.cuda.synchronize()
    rp, ci = (t.cpu().numpy() for t in asm.pattern())
    rows = np.unique(np.concatenate([[0, 1, mesh.n_nodes - 1], np.random.default_rng(85).integers(0, mesh.n_nodes, 40)]))
    ref = oracle.assemble_rows(mesh.coord, mesh.lnods, vel_in(u, "mixed64"), rows, None, RHO, MU, DT)
    Ah, rh = A.cpu().numpy(), rhs.cpu().numpy()
    worst = 0.0
    for r, (cols, a, g, orh) in zip(rows, ref):
        s, e = rp[r], rp[r + 1]
        np.testing.assert_array_equal(ci[s:e], cols)
        worst = max(worst, np.abs(Ah[s:e] - a).max() / np.abs(a).max())
        worst = max(worst, np.abs(rh[:, r] - orh).max() / np.abs(rh).max())
    assert worst <= 1e-5, worst
    asm.close()
