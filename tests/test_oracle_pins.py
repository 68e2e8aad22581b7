"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: textbook
closed forms of P1 integrals, an independent construction of the shape
gradients with exact monomial integration, global invariants of the
assembled operators, and finite differences for the adjoint.  Between them a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one test (see the comment on each).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle

RTOL = 1e-13


# ----------------------------------------------------------------------------
# independent element reference: barycentric gradients by matrix inversion and
# exact integration of barycentric monomials over a tetrahedron:
#     int_T lam_0^k0 lam_1^k1 lam_2^k2 lam_3^k3 = 3! prod(k_i!) / (sum k_i + 3)! |T|
# ----------------------------------------------------------------------------
def monomial_integral(ks, vol):
    num = 6 * math.prod(math.factorial(k) for k in ks)
    return num / math.factorial(sum(ks) + 3) * vol


def independent_element(X, U, Un, rho, mu, dt):
    """A_e, G_e, b_e of the Galerkin P1 form, built without the Gauss rule."""
    M = np.hstack([np.ones((4, 1)), X])          # rows [1, x_a, y_a, z_a]
    Minv = np.linalg.inv(M)                       # lam = Minv^T [1, x, y, z]
    grad = Minv[1:, :].T                          # grad[a] = d lam_a / dx
    vol = abs(np.linalg.det(M)) / 6.0
    mass = np.empty((4, 4))                       # int lam_a lam_c
    for a in range(4):
        for c in range(4):
            ks = [0, 0, 0, 0]
            ks[a] += 1
            ks[c] += 1
            mass[a, c] = monomial_integral(ks, vol)
    lin = np.array([monomial_integral([1 if i == a else 0 for i in range(4)], vol) for a in range(4)])
    # convection: int rho lam_a (u_h . grad lam_b), u_h = sum_c lam_c U_c
    C = rho * np.einsum("ac,ck,bk->ab", mass, U, grad)
    K = mu * vol * grad @ grad.T
    A = C + K + np.diag(rho * lin / dt)
    # G[a, b, d] = - int d_d lam_a lam_b
    G = -np.einsum("ad,b->abd", grad, lin)
    b = rho * lin[:, None] * Un / dt
    return A, G, b, vol


def test_reference_tet_closed_forms():
    """Reference tet (0, e1, e2, e3): |T| = 1/6, grad N_0 = -(1,1,1), grad N_j = e_j.

    K/mu: K00 = 1/2, K0b = -1/6, Kaa = 1/6, Kab = 0 (a != b >= 1) (textbook);
    C[a, b] = rho sum_c |T| (1 + d_ac)/20 (u_c . grad N_b); G[a, b, d] = -d_d N_a |T|/4;
    b = rho |T| u / (4 dt).  A sign error in G, a transposed C or a missing
    mass/viscous term each change one of these.
    """
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    rng = np.random.default_rng(7)
    U = rng.standard_normal((4, 3))
    Un = rng.standard_normal((4, 3))
    rho, mu, dt = 1.3, 0.7, 0.25
    lnods = np.arange(4, dtype=np.int32)[None]
    A, G, b, vol, det = oracle.element_matrices(X, lnods, U, Un, rho, mu, dt)
    A, G, b = A[0], G[0], b[0]
    assert det[0] == pytest.approx(1.0, abs=0)
    assert vol[0] == pytest.approx(1.0 / 6.0, rel=1e-15)

    Kref = np.array([[Fraction(1, 2), -Fraction(1, 6), -Fraction(1, 6), -Fraction(1, 6)],
                     [-Fraction(1, 6), Fraction(1, 6), 0, 0],
                     [-Fraction(1, 6), 0, Fraction(1, 6), 0],
                     [-Fraction(1, 6), 0, 0, Fraction(1, 6)]], dtype=object).astype(float) * mu
    gradN = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    W = np.array([[(1 + (a == c)) / 120.0 for c in range(4)] for a in range(4)])   # |T|(1+d)/20
    Cref = rho * W @ U @ gradN.T
    Mref = np.eye(4) * rho / 6.0 / 4.0 / dt
    np.testing.assert_allclose(A, Cref + Kref + Mref, rtol=1e-14, atol=1e-15)
    Gref = -np.einsum("ad,b->abd", gradN, np.full(4, 1.0 / 24.0))
    np.testing.assert_allclose(G, Gref, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(b, rho / 24.0 * Un / dt, rtol=1e-14)


@pytest.mark.parametrize("ntets", [1, 2, 3, 6])
def test_random_tets_brute_force(ntets):
    """Oracle (4-point Gauss rule, cofactor inverse) == exact monomial integration
    with gradients from a 4x4 inverse, on random well-shaped tets."""
    rng = np.random.default_rng(100 + ntets)
    coords, lnods, U, Un = [], [], [], []
    for t in range(ntets):
        while True:
            X = rng.uniform(-1, 1, (4, 3))
            d = np.linalg.det(np.column_stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))
            if abs(d) > 0.05:
                break
        if d < 0:
            X[[2, 3]] = X[[3, 2]]
        coords.append(X)
        lnods.append(np.arange(4 * t, 4 * t + 4))
        U.append(rng.standard_normal((4, 3)))
        Un.append(rng.standard_normal((4, 3)))
    coord = np.concatenate(coords)
    u = np.concatenate(U)
    un = np.concatenate(Un)
    ln = np.array(lnods, dtype=np.int32)
    rho, mu, dt = 0.9, 0.05, 0.03
    A, G, b, vol, det = oracle.element_matrices(coord, ln, u, un, rho, mu, dt)
    for t in range(ntets):
        Ar, Gr, br, vr = independent_element(coords[t], U[t], Un[t], rho, mu, dt)
        scale = np.abs(Ar).max()
        np.testing.assert_allclose(A[t], Ar, rtol=0, atol=RTOL * scale * 10)
        np.testing.assert_allclose(G[t], Gr, rtol=0, atol=RTOL * np.abs(Gr).max() * 10)
        np.testing.assert_allclose(b[t], br, rtol=1e-13)
        assert vol[t] == pytest.approx(vr, rel=1e-13)
        assert det[t] == pytest.approx(6 * vr, rel=1e-13)


def test_gauss_rule_degree():
    """The 4-point rule reproduces int lam_a lam_c exactly (degree 2), which is
    what makes the oracle's quadrature equal the exact Galerkin integrals:
    checked through the convection block with u = e_x on a random tet."""
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (4, 3))
    if np.linalg.det(np.column_stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])) < 0:
        X[[2, 3]] = X[[3, 2]]
    U = np.zeros((4, 3))
    U[2, 0] = 1.0                       # u_h = lam_2 e_x: integrand lam_a lam_2 d_x lam_b
    A, G, b, vol, det = oracle.element_matrices(X, np.arange(4, dtype=np.int32)[None], U, U,
                                                rho=1.0, mu=0.0, dt=1e30)
    Ar, _, _, _ = independent_element(X, U, U, 1.0, 0.0, 1e30)
    np.testing.assert_allclose(A[0], Ar, rtol=0, atol=1e-15 * np.abs(Ar).max() * 10)


# ----------------------------------------------------------------------------
# mesh-level invariants
# ----------------------------------------------------------------------------
def _mesh(N, jitter, numbering, seed=0):
    return meshgen.config_mesh(N=N, jitter=jitter, numbering=numbering, seed=seed)


def _dense(row_ptr, col_idx, vals, n):
    import scipy.sparse as sp
    return sp.csr_matrix((vals, col_idx, row_ptr), shape=(n, n)).toarray()


def kuhn_nnz(N):
    n = (N + 1) ** 3
    edges = 3 * N * (N + 1) ** 2 + 3 * N * N * (N + 1) + N ** 3
    return n + 2 * edges


@pytest.mark.parametrize("N,jitter,numbering", [(3, 0.0, "natural"), (4, 0.15, "random"), (5, 0.15, "rcm")])
def test_pattern_brute_force(N, jitter, numbering):
    mesh, u = _mesh(N, jitter, numbering)
    row_ptr, col_idx = oracle.pattern(mesh.n_nodes, mesh.lnods)
    ln = mesh.lnods.astype(np.int64)
    pairs = np.unique((ln[:, :, None] * mesh.n_nodes + ln[:, None, :]).ravel())
    rows = np.repeat(np.arange(mesh.n_nodes), np.diff(row_ptr))
    got = rows.astype(np.int64) * mesh.n_nodes + col_idx
    np.testing.assert_array_equal(got, pairs)
    assert row_ptr[-1] == kuhn_nnz(N)
    if N == 8:
        assert row_ptr[-1] == 9097


def test_cube8_counts():
    mesh, u = meshgen.config_mesh("cube8")
    assert (mesh.n_elems, mesh.n_nodes) == (3072, 729)
    row_ptr, col_idx = oracle.pattern(mesh.n_nodes, mesh.lnods)
    assert row_ptr[-1] == 9097 == kuhn_nnz(8)


@pytest.mark.parametrize("N,jitter,numbering", [(4, 0.0, "natural"), (5, 0.15, "random")])
def test_volume_and_orientation(N, jitter, numbering):
    """Sum of element volumes = unit-cube volume; every tet positively oriented;
    unjittered tets have |T| = h^3/6 exactly."""
    mesh, u = _mesh(N, jitter, numbering)
    _, _, _, vol, det = oracle.element_matrices(mesh.coord, mesh.lnods, u)
    assert np.all(det > 0)
    assert vol.sum() == pytest.approx(1.0, rel=1e-13)
    if jitter == 0:
        np.testing.assert_allclose(vol, (1.0 / N) ** 3 / 6.0, rtol=1e-13)


@pytest.mark.parametrize("numbering", ["natural", "random"])
def test_viscous_rows_and_symmetry(numbering):
    """rho = 0 leaves A = K: every row sums to zero (sum_b grad N_b = 0) and K is symmetric."""
    mesh, u = _mesh(4, 0.15, numbering, seed=5)
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=0.0, mu=0.37, dt=1.0)
    K = _dense(rp, ci, A, mesh.n_nodes)
    scale = np.abs(K).max()
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-14 * scale)
    np.testing.assert_allclose(K, K.T, atol=1e-15 * scale)
    assert np.all(np.diag(K) > 0)


def test_kuhn_laplacian_is_seven_point():
    """Textbook special case: on an unjittered Kuhn (Freudenthal) mesh the P1
    stiffness of an interior node is the 7-point stencil times h:
    K_ii = 6 h, K_{i,i+-e_d} = -h, every other coupling 0."""
    N = 4
    mesh, u = _mesh(N, 0.0, "natural")
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=0.0, mu=1.0, dt=1.0)
    K = _dense(rp, ci, A, mesh.n_nodes)
    h = 1.0 / N
    M = N + 1
    for (i, j, k) in [(1, 1, 1), (2, 1, 3), (2, 2, 2)]:
        node = i + M * (j + M * k)
        expect = np.zeros(mesh.n_nodes)
        expect[node] = 6 * h
        for s in (1, M, M * M):
            expect[node + s] = -h
            expect[node - s] = -h
        np.testing.assert_allclose(K[node], expect, atol=1e-15)


def test_convection_constant_velocity():
    """mu = 0, constant u: C = A - M_L rho/dt satisfies C 1 = 0, C f = rho (u.grad f) M_L
    for affine f, and column sums vanish on interior nodes."""
    mesh, _ = _mesh(4, 0.15, "random", seed=9)
    n = mesh.n_nodes
    uc = np.array([0.3, -1.1, 0.7])
    u = np.tile(uc, (n, 1))
    rho, dt = 1.7, 0.05
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=rho, mu=0.0, dt=dt)
    _, _, Am, _, _ = oracle.assemble(mesh.coord, mesh.lnods, np.zeros_like(u), rho=rho, mu=0.0, dt=dt)
    Mdiag = _dense(rp, ci, Am, n)
    ML = np.diag(Mdiag) * dt / rho                      # lumped mass sum_e |T|/4
    C = _dense(rp, ci, A, n) - Mdiag
    scale = np.abs(C).max()
    np.testing.assert_allclose(C.sum(axis=1), 0.0, atol=1e-14 * scale)
    gradf = np.array([2.0, -0.5, 1.25])
    f = mesh.coord @ gradf + 0.4
    np.testing.assert_allclose(C @ f, rho * (uc @ gradf) * ML, atol=1e-14 * scale)
    interior = np.all((mesh.coord > 1e-12) & (mesh.coord < 1 - 1e-12), axis=1)
    np.testing.assert_allclose(C.sum(axis=0)[interior], 0.0, atol=1e-14 * scale)
    assert not np.allclose(C.sum(axis=0)[~interior], 0.0)


def test_mass_only():
    """mu = 0 and u = 0: A is diagonal with trace rho |Omega| / dt."""
    mesh, u = _mesh(4, 0.15, "natural", seed=4)
    rho, dt = 2.0, 0.1
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, np.zeros_like(u), rho=rho, mu=0.0, dt=dt)
    D = _dense(rp, ci, A, mesh.n_nodes)
    assert np.count_nonzero(D - np.diag(np.diag(D))) == 0
    assert np.trace(D) == pytest.approx(rho / dt, rel=1e-13)
    np.testing.assert_allclose(rhs, 0.0)


def test_pressure_gradient_identities():
    """sum_i G[i,j,d] = 0 and sum_i G[i,j,d] x_i[d'] = -delta_dd' M_L(j):
    G^T applied to a linear field is exact (a sign or transpose error fails)."""
    mesh, u = _mesh(4, 0.15, "random", seed=11)
    n = mesh.n_nodes
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=1.0, mu=0.0, dt=1.0)
    _, _, Am, _, _ = oracle.assemble(mesh.coord, mesh.lnods, np.zeros_like(u), rho=1.0, mu=0.0, dt=1.0)
    ML = np.diag(_dense(rp, ci, Am, n))
    for d in range(3):
        Gd = _dense(rp, ci, G[d], n)
        scale = np.abs(Gd).max()
        np.testing.assert_allclose(Gd.sum(axis=0), 0.0, atol=1e-14 * scale)
        for dp in range(3):
            expect = -ML if d == dp else np.zeros(n)
            np.testing.assert_allclose(Gd.T @ mesh.coord[:, dp], expect, atol=1e-14 * scale)


def test_rhs_totals():
    """sum_i rhs_{i,k} = rho/dt sum_e |T_e| mean_a u_{a,k}; = rho u vol/dt for constant u."""
    mesh, u = _mesh(4, 0.15, "natural", seed=2)
    rho, dt = 1.0, 0.01
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, rho=rho, mu=1e-3, dt=dt)
    _, _, _, vol, _ = oracle.element_matrices(mesh.coord, mesh.lnods, u)
    ubar = u[mesh.lnods].mean(axis=1)
    np.testing.assert_allclose(rhs.sum(axis=1), rho / dt * (vol[:, None] * ubar).sum(axis=0), rtol=1e-12)
    uc = np.tile([0.5, 1.5, -2.0], (mesh.n_nodes, 1))
    _, _, _, _, rhs_c = oracle.assemble(mesh.coord, mesh.lnods, uc, rho=rho, mu=1e-3, dt=dt)
    np.testing.assert_allclose(rhs_c.sum(axis=1), rho * np.array([0.5, 1.5, -2.0]) / dt, rtol=1e-12)


def test_nodal_outputs_closed_forms():
    """The paper's nodal outputs (rhsid, dt_rho, mass_rho of Section II-A).

    Unjittered Kuhn cube: every tet has volume h^3/6, so node i receives
    rho h^3/24 per incident tet (counted from the connectivity, no geometry);
    mass_rho sums to rho times the cube's volume on any mesh; dt_rho is
    mass_rho / dt; rhsid is the lumped dt_rho u^n and equals the RHS of the
    matrix assembly.  A wrong lumping factor, a missing rho or dt, or a
    transposed rhs layout fails one of these."""
    N, rho, dt = 4, 1.7, 0.02
    mesh, u = _mesh(N, 0.0, "random", seed=3)
    rhs, dtr, mr = oracle.nodal(mesh.coord, mesh.lnods, u, rho=rho, dt=dt)
    count = np.bincount(mesh.lnods.ravel(), minlength=mesh.n_nodes)
    np.testing.assert_allclose(mr, rho * count / (24.0 * N ** 3), rtol=1e-13)
    assert mr.sum() == pytest.approx(rho, rel=1e-13)
    np.testing.assert_allclose(dtr, mr / dt, rtol=1e-13)
    np.testing.assert_allclose(rhs, dtr[None, :] * u.T, rtol=1e-13, atol=1e-13 * np.abs(rhs).max())
    mesh, u = _mesh(5, 0.15, "rcm", seed=4)
    rhs, dtr, mr = oracle.nodal(mesh.coord, mesh.lnods, u, rho=rho, dt=dt)
    assert mr.sum() == pytest.approx(rho, rel=1e-13)  # jitter keeps the unit cube's volume
    _, _, _, _, rhs_a = oracle.assemble(mesh.coord, mesh.lnods, u, rho=rho, mu=1e-3, dt=dt)
    np.testing.assert_allclose(rhs, rhs_a, rtol=1e-13, atol=1e-13 * np.abs(rhs_a).max())


def test_separate_rhs_velocity():
    """u^n enters only the RHS; u only A."""
    mesh, u = _mesh(3, 0.1, "natural", seed=6)
    un = np.random.default_rng(1).standard_normal(u.shape)
    r1 = oracle.assemble(mesh.coord, mesh.lnods, u, un)
    r2 = oracle.assemble(mesh.coord, mesh.lnods, u)
    r3 = oracle.assemble(mesh.coord, mesh.lnods, un)
    np.testing.assert_array_equal(r1[2], r2[2])
    np.testing.assert_array_equal(r1[4], r3[4])


def test_rows_match_full_assembly():
    """Row-restricted assembly adds in the same (element) order -> bitwise equal."""
    mesh, u = _mesh(5, 0.15, "random", seed=8)
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u)
    rows = np.array([0, 7, 100, mesh.n_nodes - 1, 55])
    got = oracle.assemble_rows(mesh.coord, mesh.lnods, u, rows)
    for r, (cols, a, g, rh) in zip(rows, got):
        s, e = rp[r], rp[r + 1]
        np.testing.assert_array_equal(cols, ci[s:e])
        np.testing.assert_array_equal(a, A[s:e])
        np.testing.assert_array_equal(g, G[:, s:e])
        np.testing.assert_array_equal(rh, rhs[:, r])


@pytest.mark.parametrize("rho,mu,dt", [(1.0, 1e-3, 1e-2), (2.5, 0.3, 0.05)])
def test_residual_vanishes_for_constant_velocity(rho, mu, dt):
    """R = A(u) u - b is zero for a constant velocity c with u^n = u: the
    convection and viscous parts annihilate constants (the shape gradients of
    an element sum to zero) and the lumped mass on the diagonal of A is the
    same lumped mass that forms b.  Pins oracle.residual and the mass terms
    together."""
    mesh, _ = _mesh(5, 0.15, "random", seed=12)
    c = np.array([0.7, -1.3, 2.1])
    u = np.tile(c, (mesh.n_nodes, 1))
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, None, rho, mu, dt)
    R = oracle.residual((rp, ci, A), rhs, u)
    assert np.abs(R).max() <= 1e-12 * np.abs(rhs).max()
    # and a non-constant field does not give zero
    u2 = u + 0.1 * mesh.coord
    rp, ci, A2, G2, rhs2 = oracle.assemble(mesh.coord, mesh.lnods, u2, None, rho, mu, dt)
    assert np.abs(oracle.residual((rp, ci, A2), rhs2, u2)).max() > 1e-6 * np.abs(rhs2).max()


# ----------------------------------------------------------------------------
# adjoint
# ----------------------------------------------------------------------------
def _residual(mesh, u, un, rho, mu, dt, csr):
    rp, ci, A, G, rhs = oracle.assemble(mesh.coord, mesh.lnods, u, un, rho, mu, dt, csr=csr)
    return oracle.residual((rp, ci, A), rhs, u)


def test_vjp_full_finite_differences():
    """R = A(u) u - b is quadratic in u and linear in mu, so central differences
    have no truncation error: full FD gradient on a 48-tet mesh."""
    mesh, u = _mesh(2, 0.15, "natural", seed=12)
    n = mesh.n_nodes
    rho, mu, dt = 1.0, 0.05, 0.1
    w = np.random.default_rng(40).standard_normal((n, 3))
    csr = oracle.pattern(n, mesh.lnods)
    un = u.copy()                      # b held fixed
    gu, gmu = oracle.vjp(mesh.coord, mesh.lnods, u, w, rho, mu, dt)
    h = 1e-3
    fd = np.zeros_like(u)
    for m in range(n):
        for l in range(3):
            up = u.copy(); up[m, l] += h
            um = u.copy(); um[m, l] -= h
            Rp = _residual(mesh, up, un, rho, mu, dt, csr)
            Rm = _residual(mesh, um, un, rho, mu, dt, csr)
            fd[m, l] = np.sum(w * (Rp - Rm)) / (2 * h)
    np.testing.assert_allclose(gu, fd, rtol=0, atol=1e-10 * np.abs(fd).max())
    Rp = _residual(mesh, u, un, rho, mu + h, dt, csr)
    Rm = _residual(mesh, u, un, rho, mu - h, dt, csr)
    assert gmu == pytest.approx(np.sum(w * (Rp - Rm)) / (2 * h), rel=1e-10)


def test_vjp_directional_fd_h1e6():
    """Seeded random directions at h = 1e-6 on a jittered 6^3 mesh."""
    mesh, u = _mesh(6, 0.15, "random", seed=4)
    n = mesh.n_nodes
    rho, mu, dt = 1.0, 1e-3, 1e-2
    rng = np.random.default_rng(40)
    w = rng.standard_normal((n, 3))
    csr = oracle.pattern(n, mesh.lnods)
    gu, gmu = oracle.vjp(mesh.coord, mesh.lnods, u, w, rho, mu, dt)
    h = 1e-6
    for _ in range(3):
        v = rng.standard_normal((n, 3))
        Rp = _residual(mesh, u + h * v, u, rho, mu, dt, csr)
        Rm = _residual(mesh, u - h * v, u, rho, mu, dt, csr)
        fd = np.sum(w * (Rp - Rm)) / (2 * h)
        assert np.sum(gu * v) == pytest.approx(fd, rel=1e-7)


def test_vjp_closed_form():
    """(w^T dR/du)_{m,l} = sum_e [ sum_a w_{a,l} A_e[a,m] + rho sum_a W_am sum_k w_{a,k} (d_l u^k)_e ],
    W_am = |T|(1 + d_am)/20, with gradients from the independent 4x4 inverse."""
    mesh, u = _mesh(3, 0.15, "natural", seed=13)
    n = mesh.n_nodes
    rho, mu, dt = 1.2, 0.02, 0.05
    w = np.random.default_rng(41).standard_normal((n, 3))
    gu, gmu = oracle.vjp(mesh.coord, mesh.lnods, u, w, rho, mu, dt)
    ref = np.zeros((n, 3))
    ref_mu = 0.0
    for e in range(mesh.n_elems):
        ln = mesh.lnods[e]
        X, U, Wn = mesh.coord[ln], u[ln], w[ln]
        Ae, _, _, vol = independent_element(X, U, U, rho, mu, dt)
        M = np.hstack([np.ones((4, 1)), X])
        grad = np.linalg.inv(M)[1:, :].T
        gradu = U.T @ grad                         # [k, l] = d u^k / d x_l
        Wm = vol * (1 + np.eye(4)) / 20
        contrib = Ae.T @ Wn + rho * Wm.T @ (Wn @ gradu)
        ref[ln] += contrib
        ref_mu += vol * np.sum(Wn * (grad @ gradu.T))
    np.testing.assert_allclose(gu, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert gmu == pytest.approx(ref_mu, rel=1e-12)


def test_vjp_mu_abs_brute_force():
    """The grad_mu error scale: the sum over elements, the 4 Gauss points and
    (a, k) of |w_ak (|T|/4) grad N_a . grad u^k|, with the gradients from the
    independent 4x4 inversion; and |grad_mu| never exceeds it, with equality
    when no term is negative (one tet, u = x, w the signs of the gradients)."""
    mesh, u = meshgen.config_mesh(N=2, jitter=0.15, numbering="random", seed=71)
    w = np.random.default_rng(72).standard_normal(u.shape)
    s = 0.0
    for ln in mesh.lnods:
        X = mesh.coord[ln]
        M = np.hstack([np.ones((4, 1)), X])
        grad = np.linalg.inv(M)[1:, :].T
        vol = abs(np.linalg.det(M)) / 6.0
        gradu = u[ln].T @ grad                     # gradu[k] = grad u^k
        terms = w[ln] * (grad @ gradu.T) * vol / 4  # [a, k], one Gauss point
        s += 4 * np.abs(terms).sum()
    got = oracle.vjp_mu_abs(mesh.coord, mesh.lnods, u, w)
    assert got == pytest.approx(s, rel=RTOL)
    _, gmu = oracle.vjp(mesh.coord, mesh.lnods, u, w, 1.0, 1e-3, 1e-2)
    assert abs(gmu) <= got
    # one tet, u linear with grad u^k = e_k and w_ak = grad N_a[k] sign-matched:
    # every term w_ak grad N_a . e_k = w_ak dN_a/dx_k is |dN_a/dx_k| >= 0
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    ln1 = np.array([[0, 1, 2, 3]], dtype=np.int32)
    grad = np.linalg.inv(np.hstack([np.ones((4, 1)), X]))[1:, :].T
    u1 = X.copy()
    w1 = np.sign(grad)
    _, gmu1 = oracle.vjp(X, ln1, u1, w1, 1.0, 1e-3, 1e-2)
    assert gmu1 == pytest.approx(oracle.vjp_mu_abs(X, ln1, u1, w1), rel=RTOL)


@pytest.mark.parametrize("threads", [1, 3, 0])
def test_threaded_assembly_is_bitwise_the_serial_one(threads):
    """The multi-threaded oracle (element pass, then a row pass adding each
    row's contributions in increasing element order) returns exactly the
    serial oracle's arrays, on a randomly numbered, jittered mesh with a
    separate RHS velocity."""
    mesh, u = meshgen.config_mesh(N=6, jitter=0.15, numbering="random", seed=73)
    un = np.random.default_rng(74).standard_normal(u.shape)
    ref = oracle.assemble(mesh.coord, mesh.lnods, u, un, 1.0, 1e-3, 1e-2)
    got = oracle.assemble_threads(mesh.coord, mesh.lnods, u, un, 1.0, 1e-3, 1e-2, threads=threads)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)
