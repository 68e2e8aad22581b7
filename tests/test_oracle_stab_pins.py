"""Pins of the stabilised oracle (CPU only).

The stabilised velocity block adds to the Galerkin operator the implicit terms
of Codina's algebraic subgrid-scale method (Comput. Methods Appl. Mech. Engrg.
191 (2002) 4295-4321; linear elements, c1 = 4, c2 = 2):
  tau1 = (c1 mu / h^2 + c2 rho |ubar| / h)^{-1},  tau2 = h^2 / (c1 tau1),
  S[a][b] = tau1 rho^2 int (u . grad N_a)(u . grad N_b),
  K[a][b][i][j] = mu int d_j N_a d_i N_b + tau2 int d_i N_a d_j N_b,
with h = (6 |T|)^{1/3} and ubar the mean node velocity of the element.  The
element operator of the paper's 12x12 form is delta_ij (A + S) + K.

Each pin comes from outside the oracle: tau's closed forms at the limits the
publication states (diffusive h^2 / (c1 mu), convective h / (c2 rho |u|)); the
barycentric moment formula int lam_c lam_d = |T| (1 + delta_cd) / 20 for the
SUPG integral (not the oracle's Gauss rule); the viscous stress of an affine
velocity field (a rigid rotation exerts no force, a dilation exerts
(2 mu + 3 tau2) grad N_a |T| per unit rate); and global invariants of the
assembled block operator.  A dropped term, a transposed index pair or a wrong
constant fails at least one of them (see each test).
"""
import numpy as np
import pytest

import meshgen
import oracle

RTOL = 1e-13
REF = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def barycentric_gradients(X):
    """Gradients of the barycentric coordinates by inverting [1 x y z]."""
    M = np.hstack([np.ones((4, 1)), X])
    return np.linalg.inv(M)[1:, :].T, abs(np.linalg.det(M)) / 6.0


def random_tet(rng, scale=1.0):
    while True:
        X = rng.uniform(-1.0, 1.0, (4, 3)) * scale
        M = np.hstack([np.ones((4, 1)), X])
        d = np.linalg.det(M)
        if abs(d) > 0.05 * scale ** 3:
            if d < 0:
                X[[2, 3]] = X[[3, 2]]
            return X


def test_tau_closed_forms():
    """tau1 on the unit right tetrahedron (6|T| = 1, so h = 1) and its scaled
    copies: at rest tau1 = h^2 / (4 mu), tau2 = mu; with a uniform velocity c
    tau1 = 1 / (4 mu / h^2 + 2 rho |c| / h), tau2 = mu + rho |c| h / 2 (a wrong
    element size, constant or mean velocity changes these)."""
    for s in (1.0, 0.5, 3.0):
        X = REF * s
        h = s  # 6 |T| = s^3
        for mu in (1e-3, 1e-1):
            t1, t2 = oracle.tau(X, np.zeros((4, 3)), 1.0, mu)
            assert t1 == pytest.approx(h * h / (4 * mu), rel=RTOL)
            assert t2 == pytest.approx(mu, rel=RTOL)
            c = np.array([0.3, -1.2, 0.4])
            rho = 2.5
            t1, t2 = oracle.tau(X, np.tile(c, (4, 1)), rho, mu)
            speed = np.linalg.norm(c)
            assert t1 == pytest.approx(1.0 / (4 * mu / h ** 2 + 2 * rho * speed / h), rel=RTOL)
            assert t2 == pytest.approx(mu + rho * speed * h / 2, rel=RTOL)


def test_tau_limits_and_mean_velocity():
    """Convective limit tau1 -> h / (2 rho |ubar|) as mu -> 0, with ubar the
    mean of the four node velocities (not one node's, not the norm mean)."""
    rng = np.random.default_rng(11)
    X = random_tet(rng)
    U = rng.standard_normal((4, 3))
    h = np.cbrt(abs(np.linalg.det(np.hstack([np.ones((4, 1)), X]))))
    ub = np.linalg.norm(U.mean(axis=0))
    t1, _ = oracle.tau(X, U, 1.3, 1e-14)
    assert t1 == pytest.approx(h / (2 * 1.3 * ub), rel=1e-9)


def test_supg_by_barycentric_moments():
    """S[a][b] = tau1 rho^2 sum_{c,d} (U_c . g_a)(U_d . g_b) |T| (1 + d_cd) / 20,
    exact for the degree-2 integrand, independent of the Gauss rule (a dropped
    rho, a wrong weight or a swapped gradient fails)."""
    rng = np.random.default_rng(3)
    for _ in range(6):
        X = random_tet(rng, scale=rng.uniform(0.2, 2.0))
        U = rng.standard_normal((4, 3))
        rho, mu = rng.uniform(0.5, 2.0), 10 ** rng.uniform(-4, -1)
        g, vol = barycentric_gradients(X)
        t1, _ = oracle.tau(X, U, rho, mu)
        mom = vol * (np.ones((4, 4)) + np.eye(4)) / 20.0
        v = U @ g.T  # v[c, a] = U_c . g_a
        S_ref = t1 * rho * rho * (v.T @ mom @ v)
        S, _ = oracle.stab_element(X, U, rho, mu)
        assert np.allclose(S, S_ref, rtol=1e-12, atol=1e-14 * np.abs(S_ref).max())
        # symmetric, positive semi-definite, annihilates constants
        assert np.allclose(S, S.T, rtol=0, atol=1e-14 * np.abs(S).max())
        assert np.linalg.eigvalsh(S).min() > -1e-12 * np.abs(S).max()
        assert np.abs(S.sum(axis=1)).max() < 1e-13 * np.abs(S).max()


def test_supg_uniform_velocity():
    """Uniform velocity c: S = tau1 rho^2 |T| (c . g_a)(c . g_b)."""
    rng = np.random.default_rng(4)
    X = random_tet(rng)
    c = np.array([1.0, -0.5, 0.25])
    g, vol = barycentric_gradients(X)
    t1, _ = oracle.tau(X, np.tile(c, (4, 1)), 1.0, 1e-3)
    S, _ = oracle.stab_element(X, np.tile(c, (4, 1)), 1.0, 1e-3)
    a = g @ c
    assert np.allclose(S, t1 * vol * np.outer(a, a), rtol=1e-12, atol=1e-15)


def element_force(X, U_aff, rho, mu):
    """The Galerkin viscous part plus K applied to the nodal values of an
    affine field: f[a][i] = sum_{b,j} (delta_ij mu |T| g_a . g_b + K[a][b][i][j]) U[b][j]."""
    _, K = oracle.stab_element(X, np.zeros((4, 3)), rho, mu)
    g, vol = barycentric_gradients(X)
    lap = mu * vol * (g @ g.T)
    return lap @ U_aff + np.einsum("abij,bj->ai", K, U_aff)


def test_coupling_rigid_rotation_and_dilation():
    """With the fluid at rest (tau2 = mu): a rigid rotation u = W x (W
    antisymmetric) has zero symmetric gradient and zero divergence, so the
    stress mu (grad u + grad u^T) + tau2 div u exerts no force on any node; a
    dilation u = x has grad u = I, div u = 3: force (2 mu + 3 tau2) |T| g_a.
    A transposed viscous pair (i, j) or a dropped grad-div term fails one of
    the two."""
    rng = np.random.default_rng(5)
    for _ in range(4):
        X = random_tet(rng)
        mu = 10 ** rng.uniform(-3, 0)
        w = rng.standard_normal(3)
        W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
        U_rot = X @ W.T + rng.standard_normal(3)
        f = element_force(X, U_rot, 1.0, mu)
        assert np.abs(f).max() < 1e-12 * mu * np.abs(X).max()
        g, vol = barycentric_gradients(X)
        f = element_force(X, X.copy(), 1.0, mu)
        assert np.allclose(f, 5 * mu * vol * g, rtol=1e-12, atol=1e-15)


def test_coupling_general_affine_field():
    """Affine u = M x: f[a] = |T| ( mu (M + M^T) + tau2 tr(M) I ) g_a."""
    rng = np.random.default_rng(6)
    X = random_tet(rng)
    M = rng.standard_normal((3, 3))
    mu = 0.02
    f = element_force(X, X @ M.T, 1.0, mu)
    g, vol = barycentric_gradients(X)
    t2 = mu  # at rest
    ref = vol * (g @ (mu * (M + M.T)).T + t2 * np.trace(M) * g)
    assert np.allclose(f, ref, rtol=1e-11, atol=1e-15)


def test_grad_div_weight_follows_velocity():
    """tau2 = mu + rho |ubar| h / 2 enters K's grad-div term: with a uniform
    velocity the dilation force is (2 mu + 3 tau2) |T| g_a."""
    X = REF * 0.7
    c = np.array([0.0, 2.0, 0.0])
    _, K = oracle.stab_element(X, np.tile(c, (4, 1)), 1.5, 1e-2)
    g, vol = barycentric_gradients(X)
    t2 = 1e-2 + 1.5 * 2.0 * 0.7 / 2
    f = vol * 1e-2 * (g @ g.T) @ X + np.einsum("abij,bj->ai", K, X)
    assert np.allclose(f, (2 * 1e-2 + 3 * t2) * vol * g, rtol=1e-12)


def small_mesh(N=4, seed=0):
    rng = np.random.default_rng(seed)
    m = meshgen.jitter_interior(meshgen.kuhn_cube(N), 0.15, rng)
    u = meshgen.sinusoid_velocity(m.coord, rng)
    return m, u


def block_matrix(row_ptr, col_idx, Auu, n):
    """Dense 3n x 3n matrix, unknown (node, dim) at 3 node + dim."""
    D = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            j = col_idx[p]
            D[3 * i:3 * i + 3, 3 * j:3 * j + 3] = Auu[:, p].reshape(3, 3)
    return D


def test_assembled_block_invariants():
    """Assembled Auu: (1) a uniform velocity field meets only the lumped mass,
    Auu (1 (x) c) = rho M_L / dt (x) c, since convection, viscosity, S and K
    annihilate constants; (2) the operator minus the Galerkin convection is
    symmetric: Auu - Auu^T = (A - A^T) (x) I."""
    m, u = small_mesh()
    n = m.n_nodes
    rho, mu, dt = 1.0, 1e-2, 1e-2
    rp, ci, Auu, G, rhs = oracle.assemble_stabilized(m.coord, m.lnods, u, rho=rho, mu=mu, dt=dt)
    _, _, A, G0, rhs0 = oracle.assemble(m.coord, m.lnods, u, rho=rho, mu=mu, dt=dt, csr=(rp, ci))
    assert np.array_equal(G, G0) and np.array_equal(rhs, rhs0)
    D = block_matrix(rp, ci, Auu, n)
    c = np.array([0.7, -1.1, 0.2])
    got = (D @ np.tile(c, n)).reshape(n, 3)
    ref = np.outer(rhs_of_ones(m, rho, dt), c)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    Ad = np.zeros((n, n))
    for i in range(n):
        Ad[i, ci[rp[i]:rp[i + 1]]] = A[rp[i]:rp[i + 1]]
    asym = D - D.T
    ref_asym = np.kron(Ad - Ad.T, np.eye(3))
    assert np.abs(asym - ref_asym).max() < 1e-12 * np.abs(D).max()


def rhs_of_ones(m, rho, dt):
    """Lumped mass rho |Omega_i| / dt of every node, from the Galerkin rhs of u^n = 1."""
    n = m.n_nodes
    rp, ci = oracle.pattern(n, m.lnods)
    _, _, _, _, rhs = oracle.assemble(m.coord, m.lnods, np.zeros((n, 3)), un=np.ones((n, 3)), rho=rho, dt=dt,
                                      csr=(rp, ci))
    return rhs[0]


def test_assembled_block_by_closed_forms():
    """Every component of the assembled Auu minus delta_ij A equals the
    scatter of the element closed forms: S by barycentric moments on the
    diagonal components, mu |T| g_a[j] g_b[i] + tau2 |T| g_a[i] g_b[j] on all
    nine (gradients by matrix inversion, not the oracle's cofactors)."""
    m, u = small_mesh(N=3, seed=2)
    n = m.n_nodes
    rho, mu = 1.0, 1e-3
    rp, ci, Auu, _, _ = oracle.assemble_stabilized(m.coord, m.lnods, u, rho=rho, mu=mu)
    _, _, A, _, _ = oracle.assemble(m.coord, m.lnods, u, rho=rho, mu=mu, csr=(rp, ci))
    ref = np.zeros((3, 3, n, n))
    for e in range(m.n_elems):
        v = m.lnods[e]
        X, U = m.coord[v], u[v]
        g, vol = barycentric_gradients(X)
        t1, t2 = oracle.tau(X, U, rho, mu)
        mom = vol * (np.ones((4, 4)) + np.eye(4)) / 20.0
        w = U @ g.T
        S = t1 * rho * rho * (w.T @ mom @ w)
        for i in range(3):
            for j in range(3):
                blk = mu * vol * np.outer(g[:, j], g[:, i]) + t2 * vol * np.outer(g[:, i], g[:, j])
                if i == j:
                    blk = blk + S
                ref[i, j][np.ix_(v, v)] += blk
    scale = np.abs(ref).max()
    for i in range(3):
        for j in range(3):
            got = np.zeros((n, n))
            val = Auu[3 * i + j] - (A if i == j else 0.0)
            for r in range(n):
                got[r, ci[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
            assert np.abs(got - ref[i, j]).max() < 1e-12 * scale, (i, j)


def test_stabilised_rows_match_full_assembly():
    """The row-restricted oracle (used on meshes too large for the full
    assembly) agrees with the full stabilised assembly on every row."""
    m, u = small_mesh(N=3, seed=4)
    rp, ci, Auu, G, rhs = oracle.assemble_stabilized(m.coord, m.lnods, u)
    rows = np.array([0, 5, 17, m.n_nodes - 1])
    for r, (cols, blk, g, b) in zip(rows, oracle.assemble_stabilized_rows(m.coord, m.lnods, u, rows)):
        s, e = rp[r], rp[r + 1]
        assert np.array_equal(cols, ci[s:e])
        assert np.allclose(blk, Auu[:, s:e], rtol=1e-13, atol=1e-15 * np.abs(Auu).max())
        assert np.allclose(g, G[:, s:e], rtol=1e-13, atol=1e-18)
        assert np.allclose(b, rhs[:, r], rtol=1e-13, atol=0)
