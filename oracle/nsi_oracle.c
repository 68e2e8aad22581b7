/*
 * FP64 CPU oracle for incompressible-flow P1 tetrahedral matrix assembly.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library never does.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What is computed: the element matrix assembly of Section II-A of the paper
 * for linear tetrahedra (4 nodes, 3 dimensions), in the Galerkin P1 form
 * (the paper names the terms but prints no formulas).  For an element with
 * nodes a = 0..3, shape functions N_a and velocity u_h = sum_c N_c u_c:
 *
 *   A_e[a][b]    = int rho N_a (u_h . grad N_b) + mu grad N_a . grad N_b      (convection, viscosity)
 *                  + delta_ab rho/dt int N_a                                  (row-sum lumped mass)
 *   G_e[a][b][d] = - int d_d N_a N_b                                          (pressure gradient)
 *   b_e[a][k]    = rho/dt (int N_a) u^n_a[k]                                  (lumped right-hand side)
 *
 * The integrals are evaluated by the 4-point rule on the reference
 * tetrahedron (barycentric points (alpha, beta, beta, beta) and its
 * permutations, weights 1/24 of the reference volume 1/6 each, beta =
 * (5 - sqrt 5)/20, alpha = 1 - 3 beta: the printed 10-digit constants are
 * these rounded), exact for the degree-2 integrands above; the shape-function
 * gradients are J^{-T} times the reference gradients, with the Jacobian J of
 * the element map, its determinant and its inverse by cofactors.  The
 * element matrices are summed over elements, in increasing element order,
 * into a CSR matrix whose pattern is every node pair sharing an element.
 *
 * Layouts: coord/u/un/w are node-major [n][3] (the dimension fastest); lnods
 * is [E][4], 0-based; CSR row_ptr[n+1], col_idx[nnz] ascending per row,
 * diagonal included; G is component-major [3][nnz]; rhs is [3][n].
 *
 * All arithmetic is IEEE double (the paper: all calculations are double
 * precision, Section II-A).  Return codes: 0 ok, negative on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PNODE 4
#define PGAUS 4
#define NDIME 3

/* gradients of the reference shape functions N_0 = 1-xi-eta-zeta, N_j = xi_j */
static const double REF_GRAD[PNODE][NDIME] = {
    {-1.0, -1.0, -1.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};

/* the 4-point rule: N_c at point q (the barycentric coordinates of the point)
   and the reference weights */
static void quadrature_rule(double lam[PGAUS][PNODE], double wref[PGAUS]) {
    const double beta = (5.0 - sqrt(5.0)) / 20.0;
    const double alpha = 1.0 - 3.0 * beta;
    for (int q = 0; q < PGAUS; ++q) {
        for (int c = 0; c < PNODE; ++c) lam[q][c] = (c == q) ? alpha : beta;
        wref[q] = 1.0 / 24.0; /* reference tet volume 1/6 split over 4 points */
    }
}

/*
 * Shape-function gradients of a linear tetrahedron: the Jacobian
 * J[i][j] = dx_i/dxi_j of the element map, its determinant, its inverse by
 * cofactors, and grad[a][i] = dN_a/dx_i = sum_j Jinv[j][i] dN_a/dxi_j
 * (Section II-A: Jacobian, determinant, inverse and Cartesian derivatives).
 * Returns det J.
 */
static double shape_gradients(const double X[PNODE][NDIME], double grad[PNODE][NDIME]) {
    double J[NDIME][NDIME];
    for (int i = 0; i < NDIME; ++i)
        for (int j = 0; j < NDIME; ++j) {
            J[i][j] = 0.0;
            for (int a = 0; a < PNODE; ++a) J[i][j] += X[a][i] * REF_GRAD[a][j];
        }
    /* cofactor matrix C[i][j] = (-1)^{i+j} minor(i, j) */
    double C[NDIME][NDIME];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = -(J[1][0] * J[2][2] - J[1][2] * J[2][0]);
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = -(J[0][1] * J[2][2] - J[0][2] * J[2][1]);
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = -(J[0][0] * J[2][1] - J[0][1] * J[2][0]);
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = -(J[0][0] * J[1][2] - J[0][2] * J[1][0]);
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    /* J^{-1} = adj(J) / det with adj(J)[j][i] = C[i][j] */
    double Jinv[NDIME][NDIME];
    for (int i = 0; i < NDIME; ++i)
        for (int j = 0; j < NDIME; ++j) Jinv[i][j] = C[j][i] / det;
    for (int a = 0; a < PNODE; ++a)
        for (int i = 0; i < NDIME; ++i) {
            grad[a][i] = 0.0;
            for (int j = 0; j < NDIME; ++j) grad[a][i] += Jinv[j][i] * REF_GRAD[a][j];
        }
    return det;
}

/*
 * The element integrals of the form above for one tetrahedron, by the
 * 4-point rule.  X: node coordinates, U: advection velocity, Un: velocity of
 * the right-hand side.  Returns det J (negative or zero for an inverted or
 * degenerate element); *volume gets the element's volume.
 */
double oracle_element(const double X[PNODE][NDIME], const double U[PNODE][NDIME],
                      const double Un[PNODE][NDIME], double rho, double mu, double dt,
                      double A[PNODE][PNODE], double G[PNODE][PNODE][NDIME],
                      double b[PNODE][NDIME], double* volume) {
    double lam[PGAUS][PNODE], wref[PGAUS];
    quadrature_rule(lam, wref);

    /* gradients and integration weights w_q det J at every point (the
       gradients of a linear element are the same at every point) */
    double grad[PGAUS][PNODE][NDIME], wq[PGAUS], detjac = 0.0;
    for (int q = 0; q < PGAUS; ++q) {
        detjac = shape_gradients(X, grad[q]);
        wq[q] = wref[q] * detjac;
    }

    /* the advection velocity u_h at every point */
    double uq[PGAUS][NDIME];
    for (int q = 0; q < PGAUS; ++q)
        for (int k = 0; k < NDIME; ++k) {
            uq[q][k] = 0.0;
            for (int c = 0; c < PNODE; ++c) uq[q][k] += lam[q][c] * U[c][k];
        }

    memset(A, 0, sizeof(double) * PNODE * PNODE);
    memset(G, 0, sizeof(double) * PNODE * PNODE * NDIME);
    memset(b, 0, sizeof(double) * PNODE * NDIME);
    double vol = 0.0;
    for (int q = 0; q < PGAUS; ++q) {
        /* u_h . grad N_b and grad N_a . grad N_b at the point */
        double adv[PNODE], stiff[PNODE][PNODE];
        for (int bb = 0; bb < PNODE; ++bb) {
            adv[bb] = 0.0;
            for (int k = 0; k < NDIME; ++k) adv[bb] += uq[q][k] * grad[q][bb][k];
        }
        for (int a = 0; a < PNODE; ++a)
            for (int bb = 0; bb < PNODE; ++bb) {
                stiff[a][bb] = 0.0;
                for (int k = 0; k < NDIME; ++k) stiff[a][bb] += grad[q][a][k] * grad[q][bb][k];
            }
        /* convection rho N_a (u_h . grad N_b) and viscosity mu grad N_a . grad N_b */
        for (int a = 0; a < PNODE; ++a)
            for (int bb = 0; bb < PNODE; ++bb)
                A[a][bb] += wq[q] * (rho * lam[q][a] * adv[bb] + mu * stiff[a][bb]);
        /* pressure gradient -d_d N_a N_b */
        for (int a = 0; a < PNODE; ++a)
            for (int bb = 0; bb < PNODE; ++bb)
                for (int d = 0; d < NDIME; ++d) G[a][bb][d] -= wq[q] * grad[q][a][d] * lam[q][bb];
        vol += wq[q];
    }
    /* row-sum lumped mass int N_a on the diagonal and in the right-hand side */
    for (int a = 0; a < PNODE; ++a) {
        double lump = 0.0;
        for (int q = 0; q < PGAUS; ++q) lump += wq[q] * lam[q][a];
        A[a][a] += rho * lump / dt;
        for (int k = 0; k < NDIME; ++k) b[a][k] = rho * lump * Un[a][k] / dt;
    }
    if (volume) *volume = vol;
    return detjac;
}

/* the element's node coordinates and velocities, from the global arrays */
static void element_nodes(const double* coord, const double* u, const double* un, const int32_t* ln,
                          double X[PNODE][NDIME], double U[PNODE][NDIME], double Un[PNODE][NDIME]) {
    for (int a = 0; a < PNODE; ++a) {
        int64_t p = ln[a];
        for (int k = 0; k < NDIME; ++k) {
            X[a][k] = coord[3 * p + k];
            U[a][k] = u[3 * p + k];
            Un[a][k] = un[3 * p + k];
        }
    }
}

/* element matrices for a list of elements: A[m][4][4], G[m][4][4][3], b[m][4][3], vol[m], det[m] */
int oracle_element_batch(int64_t n, const double* coord, const int32_t* lnods, const double* u,
                         const double* un, double rho, double mu, double dt, const int64_t* elems,
                         int64_t m, double* A, double* G, double* b, double* vol, double* det) {
    for (int64_t t = 0; t < m; ++t) {
        const int32_t* ln = lnods + 4 * elems[t];
        for (int a = 0; a < PNODE; ++a)
            if (ln[a] < 0 || ln[a] >= n) return -1;
        double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME];
        element_nodes(coord, u, un, ln, X, U, Un);
        det[t] = oracle_element(X, U, Un, rho, mu, dt, (double(*)[PNODE])(A + 16 * t),
                                (double(*)[PNODE][NDIME])(G + 48 * t), (double(*)[NDIME])(b + 12 * t),
                                vol + t);
    }
    return 0;
}

/*
 * The paper's per-node outputs of the assembly (Section II-A: the
 * right-hand side rhsid and the nodal arrays dt_rho_nsi and mass_rho_nsi,
 * accumulated over the elements of each node), in increasing element order:
 *   rhsid[k][i]  += rho/dt (int_e N_a) un[a][k]
 *   dt_rho[i]    += rho/dt  int_e N_a
 *   mass_rho[i]  += rho     int_e N_a            for every element e and node a of it, i = lnods[e][a],
 * with int_e N_a by the 4-point rule.  The paper gives the accumulation, not
 * the element values: they are read as the row-sum lumped density mass over
 * dt and the lumped density mass (the lumping of the matrix diagonal and the
 * RHS).  rhs is [3][n]; dt_rho and mass_rho are [n].
 */
int oracle_nodal(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* un,
                 double rho, double dt, double* rhs, double* dt_rho, double* mass_rho) {
    double lam[PGAUS][PNODE], wref[PGAUS];
    quadrature_rule(lam, wref);
    memset(rhs, 0, sizeof(double) * 3 * n);
    memset(dt_rho, 0, sizeof(double) * n);
    memset(mass_rho, 0, sizeof(double) * n);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        for (int a = 0; a < PNODE; ++a)
            if (ln[a] < 0 || ln[a] >= n) return -1;
        double X[PNODE][NDIME], Un[PNODE][NDIME];
        element_nodes(coord, un, un, ln, X, Un, Un);
        double grad[PNODE][NDIME];
        const double detjac = shape_gradients(X, grad);
        if (!(detjac > 0.0)) return -2;
        for (int a = 0; a < PNODE; ++a) {
            double lump = 0.0;
            for (int g = 0; g < PGAUS; ++g) lump += wref[g] * detjac * lam[g][a];
            const double mdt = rho * lump / dt, mrho = rho * lump;
            for (int k = 0; k < NDIME; ++k) rhs[k * n + ln[a]] += rho * lump * Un[a][k] / dt;
            dt_rho[ln[a]] += mdt;
            mass_rho[ln[a]] += mrho;
        }
    }
    return 0;
}

static int cmp_i64(const void* x, const void* y) {
    int64_t a = *(const int64_t*)x, c = *(const int64_t*)y;
    return (a > c) - (a < c);
}

/*
 * CSR pattern of the assembled matrix: every pair (lnods[e][a], lnods[e][b]),
 * sorted by (row, col), duplicates removed.  Call with col_idx == NULL to get
 * nnz only; then call again with col_idx sized nnz.  Returns nnz or < 0.
 */
int64_t oracle_pattern(int64_t n, int64_t E, const int32_t* lnods, int32_t* row_ptr, int32_t* col_idx) {
    int64_t npairs = 16 * E;
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (npairs > 0 ? npairs : 1));
    if (!key) return -2;
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c) {
                int64_t r = lnods[4 * e + a], s = lnods[4 * e + c];
                if (r < 0 || r >= n || s < 0 || s >= n) { free(key); return -1; }
                key[16 * e + 4 * a + c] = r * n + s;
            }
    qsort(key, npairs, sizeof(int64_t), cmp_i64);
    int64_t nnz = 0;
    for (int64_t t = 0; t < npairs; ++t)
        if (t == 0 || key[t] != key[t - 1]) {
            if (col_idx) col_idx[nnz] = (int32_t)(key[t] % n);
            ++nnz;
        }
    if (col_idx && row_ptr) {
        for (int64_t i = 0; i <= n; ++i) row_ptr[i] = 0;
        int64_t q = 0;
        for (int64_t t = 0; t < npairs; ++t)
            if (t == 0 || key[t] != key[t - 1]) {
                row_ptr[key[t] / n + 1] += 1;
                ++q;
            }
        for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    }
    free(key);
    return nnz;
}

static int64_t find_pos(const int32_t* row_ptr, const int32_t* col_idx, int64_t r, int64_t c) {
    int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col_idx[mid] == c) return mid;
        if (col_idx[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Global assembly into the oracle's CSR pattern (outputs zeroed here). */
int oracle_assemble(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u,
                    const double* un, double rho, double mu, double dt, const int32_t* row_ptr,
                    const int32_t* col_idx, double* A, double* G, double* rhs) {
    int64_t nnz = row_ptr[n];
    memset(A, 0, sizeof(double) * nnz);
    memset(G, 0, sizeof(double) * 3 * nnz);
    memset(rhs, 0, sizeof(double) * 3 * n);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        for (int a = 0; a < PNODE; ++a)
            if (ln[a] < 0 || ln[a] >= n) return -1;
        double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME];
        double Ae[PNODE][PNODE], Ge[PNODE][PNODE][NDIME], be[PNODE][NDIME], vol;
        element_nodes(coord, u, un, ln, X, U, Un);
        oracle_element(X, U, Un, rho, mu, dt, Ae, Ge, be, &vol);
        /* the element's 16 entries added at their CSR positions */
        for (int a = 0; a < PNODE; ++a) {
            for (int c = 0; c < PNODE; ++c) {
                int64_t pos = find_pos(row_ptr, col_idx, ln[a], ln[c]);
                if (pos < 0) return -3;
                A[pos] += Ae[a][c];
                for (int d = 0; d < NDIME; ++d) G[d * nnz + pos] += Ge[a][c][d];
            }
            for (int k = 0; k < NDIME; ++k) rhs[k * n + ln[a]] += be[a][k];
        }
    }
    return 0;
}

/*
 * The same assembly restricted to a list of rows (for spot checks on meshes too
 * large for the full oracle).  For sampled row t (t < m), the row's columns
 * (ascending) go to cols[t*maxc ...], count[t] holds their number, A/G/rhs
 * hold the values: A[t*maxc + q], G[(t*3 + d)*maxc + q], rhs[t*3 + k].
 * Contributions are added in increasing element order.
 */
int oracle_assemble_rows(int64_t n, int64_t E, const double* coord, const int32_t* lnods,
                         const double* u, const double* un, double rho, double mu, double dt,
                         const int64_t* rows, int64_t m, int64_t maxc, int32_t* cols, int32_t* count,
                         double* A, double* G, double* rhs) {
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!slot) return -2;
    for (int64_t i = 0; i < n; ++i) slot[i] = -1;
    for (int64_t t = 0; t < m; ++t) {
        if (rows[t] < 0 || rows[t] >= n || slot[rows[t]] >= 0) { free(slot); return -1; }
        slot[rows[t]] = t;
        count[t] = 0;
    }
    memset(A, 0, sizeof(double) * m * maxc);
    memset(G, 0, sizeof(double) * m * 3 * maxc);
    memset(rhs, 0, sizeof(double) * m * 3);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        int hit = 0;
        for (int a = 0; a < PNODE; ++a) {
            if (ln[a] < 0 || ln[a] >= n) { free(slot); return -1; }
            hit |= slot[ln[a]] >= 0;
        }
        if (!hit) continue;
        double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME];
        double Ae[PNODE][PNODE], Ge[PNODE][PNODE][NDIME], be[PNODE][NDIME], vol;
        element_nodes(coord, u, un, ln, X, U, Un);
        oracle_element(X, U, Un, rho, mu, dt, Ae, Ge, be, &vol);
        for (int a = 0; a < PNODE; ++a) {
            int64_t t = slot[ln[a]];
            if (t < 0) continue;
            for (int c = 0; c < PNODE; ++c) {
                int64_t q = 0;
                while (q < count[t] && cols[t * maxc + q] != ln[c]) ++q;
                if (q == count[t]) {
                    if (q >= maxc) { free(slot); return -4; }
                    cols[t * maxc + q] = ln[c];
                    count[t] += 1;
                }
                A[t * maxc + q] += Ae[a][c];
                for (int d = 0; d < NDIME; ++d) G[(t * 3 + d) * maxc + q] += Ge[a][c][d];
            }
            for (int k = 0; k < NDIME; ++k) rhs[t * 3 + k] += be[a][k];
        }
    }
    /* sort each row by column (insertion sort; values move with their column) */
    for (int64_t t = 0; t < m; ++t) {
        for (int32_t q = 1; q < count[t]; ++q) {
            for (int32_t r = q; r > 0 && cols[t * maxc + r - 1] > cols[t * maxc + r]; --r) {
                int64_t i0 = t * maxc + r - 1, i1 = t * maxc + r;
                int32_t tc = cols[i0]; cols[i0] = cols[i1]; cols[i1] = tc;
                double ta = A[i0]; A[i0] = A[i1]; A[i1] = ta;
                for (int d = 0; d < NDIME; ++d) {
                    int64_t j0 = (t * 3 + d) * maxc + r - 1, j1 = j0 + 1;
                    double tg = G[j0]; G[j0] = G[j1]; G[j1] = tg;
                }
            }
        }
    }
    free(slot);
    return 0;
}

/*
 * Adjoint of the assembled residual R = A(u) u - b (b held fixed):
 *   grad_u[m][l] = sum_{i,k} w[i][k] dR[i][k]/du[m][l]
 *   grad_mu      = sum_{i,k} w[i][k] dR[i][k]/dmu
 * Per element, from the Gauss-point form of R_e[a][k] =
 *   sum_g wq_g ( rho N_a(g) uq_g . grad u^k + mu grad_a . grad u^k )
 *   + rho/dt lump_a u[a][k] - b_e[a][k],     grad u^k = sum_c u[c][k] grad_c,
 * differentiated term by term:
 *   dR_e[a][k]/du[m][l] = sum_g wq_g ( rho N_a(g) N_m(g) (grad u^k)_l
 *                          + delta_kl (rho N_a(g) uq_g . grad_m + mu grad_a . grad_m) )
 *                          + delta_kl delta_am rho/dt lump_a
 *   dR_e[a][k]/dmu      = sum_g wq_g grad_a . grad u^k
 * w, u, grad_u are node-major [n][3].  grad_u is overwritten.
 */
int oracle_vjp(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u,
               double rho, double mu, double dt, const double* w, double* grad_u, double* grad_mu) {
    double lam[PGAUS][PNODE], wref[PGAUS];
    quadrature_rule(lam, wref);
    memset(grad_u, 0, sizeof(double) * 3 * n);
    double gmu = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        for (int a = 0; a < PNODE; ++a)
            if (ln[a] < 0 || ln[a] >= n) return -1;
        double X[PNODE][NDIME], U[PNODE][NDIME], W[PNODE][NDIME];
        for (int a = 0; a < PNODE; ++a)
            for (int k = 0; k < NDIME; ++k) {
                X[a][k] = coord[3 * (int64_t)ln[a] + k];
                U[a][k] = u[3 * (int64_t)ln[a] + k];
                W[a][k] = w[3 * (int64_t)ln[a] + k];
            }
        double grad[PNODE][NDIME], wq[PGAUS];
        double det = shape_gradients(X, grad);
        for (int g = 0; g < PGAUS; ++g) wq[g] = wref[g] * det;
        /* velocity gradient grad u^k (constant on a P1 element) */
        double gradu[NDIME][NDIME]; /* gradu[k][l] = d u^k / d x_l */
        for (int k = 0; k < NDIME; ++k)
            for (int l = 0; l < NDIME; ++l) {
                gradu[k][l] = 0.0;
                for (int c = 0; c < PNODE; ++c) gradu[k][l] += U[c][k] * grad[c][l];
            }
        for (int g = 0; g < PGAUS; ++g) {
            double uq[NDIME];
            for (int k = 0; k < NDIME; ++k) {
                uq[k] = 0.0;
                for (int c = 0; c < PNODE; ++c) uq[k] += lam[g][c] * U[c][k];
            }
            for (int a = 0; a < PNODE; ++a)
                for (int mm = 0; mm < PNODE; ++mm) {
                    double adv_m = 0.0, visc_am = 0.0;
                    for (int i = 0; i < NDIME; ++i) {
                        adv_m += uq[i] * grad[mm][i];
                        visc_am += grad[a][i] * grad[mm][i];
                    }
                    for (int k = 0; k < NDIME; ++k)
                        for (int l = 0; l < NDIME; ++l) {
                            double d = rho * lam[g][a] * lam[g][mm] * gradu[k][l];
                            if (k == l) d += rho * lam[g][a] * adv_m + mu * visc_am;
                            grad_u[3 * (int64_t)ln[mm] + l] += W[a][k] * wq[g] * d;
                        }
                }
            for (int a = 0; a < PNODE; ++a)
                for (int k = 0; k < NDIME; ++k) {
                    double dmu = 0.0;
                    for (int i = 0; i < NDIME; ++i) dmu += grad[a][i] * gradu[k][i];
                    gmu += W[a][k] * wq[g] * dmu;
                }
        }
        /* lumped mass term */
        for (int a = 0; a < PNODE; ++a) {
            double lump = 0.0;
            for (int g = 0; g < PGAUS; ++g) lump += wq[g] * lam[g][a];
            for (int k = 0; k < NDIME; ++k) grad_u[3 * (int64_t)ln[a] + k] += W[a][k] * rho * lump / dt;
        }
    }
    *grad_mu = gmu;
    return 0;
}

/*
 * Condition scale of grad_mu: the sum, over elements e, Gauss points g and
 * node/component pairs (a, k), of the magnitudes of the terms whose sum is
 * grad_mu in oracle_vjp,
 *   sum |w[a][k] wq_g (grad_a . grad u^k)|.
 * A floating-point evaluation of grad_mu in any summation order differs from
 * the exact sum by at most (number of terms) x (rounding unit) x this scale
 * (the standard error bound of a floating-point sum), so comparisons of the
 * cancelling scalar grad_mu are made relative to it.
 */
int oracle_vjp_mu_abs(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u,
                      const double* w, double* out) {
    double lam[PGAUS][PNODE], wref[PGAUS];
    quadrature_rule(lam, wref);
    double s = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        for (int a = 0; a < PNODE; ++a)
            if (ln[a] < 0 || ln[a] >= n) return -1;
        double X[PNODE][NDIME], U[PNODE][NDIME], W[PNODE][NDIME];
        for (int a = 0; a < PNODE; ++a)
            for (int k = 0; k < NDIME; ++k) {
                X[a][k] = coord[3 * (int64_t)ln[a] + k];
                U[a][k] = u[3 * (int64_t)ln[a] + k];
                W[a][k] = w[3 * (int64_t)ln[a] + k];
            }
        double grad[PNODE][NDIME];
        const double det = shape_gradients(X, grad);
        double gradu[NDIME][NDIME];
        for (int k = 0; k < NDIME; ++k)
            for (int l = 0; l < NDIME; ++l) {
                gradu[k][l] = 0.0;
                for (int c = 0; c < PNODE; ++c) gradu[k][l] += U[c][k] * grad[c][l];
            }
        for (int g = 0; g < PGAUS; ++g)
            for (int a = 0; a < PNODE; ++a)
                for (int k = 0; k < NDIME; ++k) {
                    double dmu = 0.0;
                    for (int i = 0; i < NDIME; ++i) dmu += grad[a][i] * gradu[k][i];
                    s += fabs(W[a][k] * wref[g] * det * dmu);
                }
    }
    *out = s;
    return 0;
}

/*
 * oracle_assemble on several host threads (OpenMP), to time the oracle on all
 * of a host's cores.  Pass 1, over elements in parallel: every element's
 * matrices (oracle_element) and the 16 CSR positions of its node pairs.
 * Pass 2, over rows in parallel: each row's entries and right-hand side
 * receive the contributions of the row's elements in increasing element
 * order -- the order of oracle_assemble's single loop -- so the result is
 * bitwise that of oracle_assemble.  Working memory: 672 bytes per element.
 * nthreads <= 0 lets OpenMP choose.  Returns 0, < 0 on bad input (as
 * oracle_assemble) or -2 when memory runs out.
 */
int oracle_assemble_threads(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u,
                            const double* un, double rho, double mu, double dt, const int32_t* row_ptr,
                            const int32_t* col_idx, double* A, double* G, double* rhs, int nthreads) {
    for (int64_t t = 0; t < 4 * E; ++t)
        if (lnods[t] < 0 || lnods[t] >= n) return -1;
    const int64_t nnz = row_ptr[n];
    int64_t* first = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t)); /* node -> its (element, local) pairs */
    int64_t* inc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(4 * E > 0 ? 4 * E : 1));
    double* Ae = (double*)malloc(sizeof(double) * (size_t)(16 * E > 0 ? 16 * E : 1));
    double* Ge = (double*)malloc(sizeof(double) * (size_t)(48 * E > 0 ? 48 * E : 1));
    double* be = (double*)malloc(sizeof(double) * (size_t)(12 * E > 0 ? 12 * E : 1));
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(16 * E > 0 ? 16 * E : 1));
    int rc = 0;
    if (!first || !inc || !Ae || !Ge || !be || !pos) rc = -2;
    if (rc == 0) {
        for (int64_t t = 0; t < 4 * E; ++t) first[lnods[t] + 1] += 1;
        for (int64_t i = 0; i < n; ++i) first[i + 1] += first[i];
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        if (!fill) rc = -2;
        else {
            memcpy(fill, first, sizeof(int64_t) * (size_t)n);
            for (int64_t t = 0; t < 4 * E; ++t) inc[fill[lnods[t]]++] = t; /* t = 4 e + a, increasing e */
            free(fill);
        }
    }
    int nt = 1;
#ifdef _OPENMP
    nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
    int bad = 0;
    if (rc == 0) {
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
        for (int64_t e = 0; e < E; ++e) {
            const int32_t* ln = lnods + 4 * e;
            double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME], vol;
            element_nodes(coord, u, un, ln, X, U, Un);
            oracle_element(X, U, Un, rho, mu, dt, (double(*)[PNODE])(Ae + 16 * e),
                           (double(*)[PNODE][NDIME])(Ge + 48 * e), (double(*)[NDIME])(be + 12 * e), &vol);
            for (int a = 0; a < PNODE; ++a)
                for (int c = 0; c < PNODE; ++c) {
                    const int64_t p = find_pos(row_ptr, col_idx, ln[a], ln[c]);
                    pos[16 * e + 4 * a + c] = p;
                    bad |= p < 0;
                }
        }
        if (bad) rc = -3;
    }
    if (rc == 0) {
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nt)
        for (int64_t r = 0; r < n; ++r) {
            for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
                A[p] = 0.0;
                for (int d = 0; d < NDIME; ++d) G[d * nnz + p] = 0.0;
            }
            for (int k = 0; k < NDIME; ++k) rhs[k * n + r] = 0.0;
            for (int64_t s = first[r]; s < first[r + 1]; ++s) {
                const int64_t e = inc[s] >> 2;
                const int a = (int)(inc[s] & 3);
                for (int c = 0; c < PNODE; ++c) {
                    const int64_t p = pos[16 * e + 4 * a + c];
                    A[p] += Ae[16 * e + 4 * a + c];
                    for (int d = 0; d < NDIME; ++d) G[d * nnz + p] += Ge[48 * e + 12 * a + 3 * c + d];
                }
                for (int k = 0; k < NDIME; ++k) rhs[k * n + r] += be[12 * e + 3 * a + k];
            }
        }
    }
    free(first); free(inc); free(Ae); free(Ge); free(be); free(pos);
    return rc;
}

/*
 * The stabilised momentum operator: the block of the velocity unknowns,
 * (PNODE x NDIME)^2 per element, as the paper's 12x12 element matrix (Section
 * II-A, Listing 4: every pair of dimensions coupled, equal dimensions receiving
 * the scalar part).  For element e, nodes a, b and dimensions i, j
 *
 *   Auu[(a,i),(b,j)] = delta_ij ( A_e[a][b] + S_e[a][b] ) + K_e[a][b][i][j]
 *
 * with A_e the Galerkin element matrix (convection, viscosity, lumped mass)
 * and the terms of the algebraic subgrid-scale stabilisation of R. Codina,
 * Comput. Methods Appl. Mech. Engrg. 191 (2002) 4295-4321 (linear elements,
 * c1 = 4, c2 = 2), taken implicitly (the projection of that method's
 * orthogonal subscales belongs to the right-hand side and is not built here):
 *   tau1_e = ( c1 mu / h_e^2 + c2 rho |ubar_e| / h_e )^{-1}
 *   tau2_e = h_e^2 / (c1 tau1_e)
 *   S_e[a][b]        = tau1_e rho^2 int (u_h . grad N_a)(u_h . grad N_b)
 *   K_e[a][b][i][j]  = mu int d_j N_a d_i N_b      (the transposed-gradient
 *                      half of the viscous stress mu (grad u + grad u^T))
 *                    + tau2_e int d_i N_a d_j N_b  (the grad-div term of the
 *                      pressure subscale)
 * with h_e = (6 |T_e|)^{1/3} and ubar_e the mean of the element's node
 * velocities u.  S is integrated with the 4-point rule (its integrand has
 * degree 2); the integrands of K are constant.
 */
double oracle_tau(const double X[PNODE][NDIME], const double U[PNODE][NDIME], double rho, double mu, double* tau2) {
    double grad[PNODE][NDIME];
    const double det = shape_gradients(X, grad);
    const double h = cbrt(det); /* det = 6 |T| */
    double ub[NDIME] = {0.0, 0.0, 0.0};
    for (int c = 0; c < PNODE; ++c)
        for (int k = 0; k < NDIME; ++k) ub[k] += U[c][k] / PNODE;
    const double speed = sqrt(ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2]);
    const double c1 = 4.0, c2 = 2.0;
    const double tau1 = 1.0 / (c1 * mu / (h * h) + c2 * rho * speed / h);
    if (tau2) *tau2 = h * h / (c1 * tau1);
    return tau1;
}

void oracle_stab_element(const double X[PNODE][NDIME], const double U[PNODE][NDIME], double rho, double mu,
                         double S[PNODE][PNODE], double K[PNODE][PNODE][NDIME][NDIME]) {
    double lam[PGAUS][PNODE], wref[PGAUS];
    quadrature_rule(lam, wref);
    double grad[PNODE][NDIME];
    const double det = shape_gradients(X, grad);
    double tau2;
    const double tau1 = oracle_tau(X, U, rho, mu, &tau2);
    memset(S, 0, sizeof(double) * PNODE * PNODE);
    for (int q = 0; q < PGAUS; ++q) {
        double uq[NDIME] = {0.0, 0.0, 0.0};
        for (int k = 0; k < NDIME; ++k)
            for (int c = 0; c < PNODE; ++c) uq[k] += lam[q][c] * U[c][k];
        double adv[PNODE];
        for (int a = 0; a < PNODE; ++a) {
            adv[a] = 0.0;
            for (int k = 0; k < NDIME; ++k) adv[a] += uq[k] * grad[a][k];
        }
        for (int a = 0; a < PNODE; ++a)
            for (int b = 0; b < PNODE; ++b) S[a][b] += wref[q] * det * tau1 * rho * rho * adv[a] * adv[b];
    }
    const double vol = det / 6.0;
    for (int a = 0; a < PNODE; ++a)
        for (int b = 0; b < PNODE; ++b)
            for (int i = 0; i < NDIME; ++i)
                for (int j = 0; j < NDIME; ++j)
                    K[a][b][i][j] = mu * vol * grad[a][j] * grad[b][i] + tau2 * vol * grad[a][i] * grad[b][j];
}

/*
 * Stabilised assembly on the CSR pattern: Auu [9][nnz] with component 3 i + j
 * the (i, j) entry of the 3x3 block of (row node, column node), G [3][nnz] and
 * rhs [3][n] as oracle_assemble.  Elements in increasing order.
 */
int oracle_assemble_stabilized(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u,
                               const double* un, double rho, double mu, double dt, const int32_t* row_ptr,
                               const int32_t* col_idx, double* Auu, double* G, double* rhs) {
    const int64_t nnz = row_ptr[n];
    double* A = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    if (!A) return -4;
    int rc = oracle_assemble(n, E, coord, lnods, u, un, rho, mu, dt, row_ptr, col_idx, A, G, rhs);
    if (rc != 0) {
        free(A);
        return rc;
    }
    memset(Auu, 0, sizeof(double) * 9 * (size_t)nnz);
    for (int64_t p = 0; p < nnz; ++p)
        for (int i = 0; i < NDIME; ++i) Auu[(4 * i) * nnz + p] = A[p];
    free(A);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME];
        double Se[PNODE][PNODE], Ke[PNODE][PNODE][NDIME][NDIME];
        element_nodes(coord, u, un, ln, X, U, Un);
        oracle_stab_element(X, U, rho, mu, Se, Ke);
        for (int a = 0; a < PNODE; ++a)
            for (int c = 0; c < PNODE; ++c) {
                const int64_t pos = find_pos(row_ptr, col_idx, ln[a], ln[c]);
                if (pos < 0) return -3;
                for (int i = 0; i < NDIME; ++i)
                    for (int j = 0; j < NDIME; ++j)
                        Auu[(3 * i + j) * nnz + pos] += (i == j ? Se[a][c] : 0.0) + Ke[a][c][i][j];
            }
    }
    return 0;
}

/*
 * The stabilisation part alone (S on the diagonal components, K on all nine)
 * restricted to a list of rows, for spot checks on meshes too large for the
 * full oracle: for sampled row t, cols[t*maxc ...] its columns (ascending),
 * count[t] their number, Auu[(t*9 + 3 i + j)*maxc + q] the values.
 * Contributions are added in increasing element order.
 */
int oracle_stab_rows(int64_t n, int64_t E, const double* coord, const int32_t* lnods, const double* u, double rho,
                     double mu, const int64_t* rows, int64_t m, int64_t maxc, int32_t* cols, int32_t* count,
                     double* Auu) {
    int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!slot) return -2;
    for (int64_t i = 0; i < n; ++i) slot[i] = -1;
    for (int64_t t = 0; t < m; ++t) {
        if (rows[t] < 0 || rows[t] >= n || slot[rows[t]] >= 0) { free(slot); return -1; }
        slot[rows[t]] = t;
        count[t] = 0;
    }
    memset(Auu, 0, sizeof(double) * m * 9 * maxc);
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ln = lnods + 4 * e;
        int hit = 0;
        for (int a = 0; a < PNODE; ++a) {
            if (ln[a] < 0 || ln[a] >= n) { free(slot); return -1; }
            hit |= slot[ln[a]] >= 0;
        }
        if (!hit) continue;
        double X[PNODE][NDIME], U[PNODE][NDIME], Un[PNODE][NDIME];
        double Se[PNODE][PNODE], Ke[PNODE][PNODE][NDIME][NDIME];
        element_nodes(coord, u, u, ln, X, U, Un);
        oracle_stab_element(X, U, rho, mu, Se, Ke);
        for (int a = 0; a < PNODE; ++a) {
            const int64_t t = slot[ln[a]];
            if (t < 0) continue;
            for (int c = 0; c < PNODE; ++c) {
                int64_t q = 0;
                while (q < count[t] && cols[t * maxc + q] != ln[c]) ++q;
                if (q == count[t]) {
                    if (q >= maxc) { free(slot); return -4; }
                    cols[t * maxc + q] = ln[c];
                    count[t] += 1;
                }
                for (int i = 0; i < NDIME; ++i)
                    for (int j = 0; j < NDIME; ++j)
                        Auu[(t * 9 + 3 * i + j) * maxc + q] += (i == j ? Se[a][c] : 0.0) + Ke[a][c][i][j];
            }
        }
    }
    for (int64_t t = 0; t < m; ++t) {
        for (int32_t q = 1; q < count[t]; ++q) {
            for (int32_t r = q; r > 0 && cols[t * maxc + r - 1] > cols[t * maxc + r]; --r) {
                const int64_t i0 = t * maxc + r - 1, i1 = t * maxc + r;
                const int32_t tc = cols[i0]; cols[i0] = cols[i1]; cols[i1] = tc;
                for (int k = 0; k < 9; ++k) {
                    const int64_t j0 = (t * 9 + k) * maxc + r - 1, j1 = j0 + 1;
                    const double tv = Auu[j0]; Auu[j0] = Auu[j1]; Auu[j1] = tv;
                }
            }
        }
    }
    free(slot);
    return 0;
}
