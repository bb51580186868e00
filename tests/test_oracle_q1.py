"""Pins of the checker's Q1 discretisation.

* constant-coefficient operators equal their tensor-product construction from the 1D
  linear-element matrices (textbook closed forms), on grids with hx != hy;
* rigid-body motions give zero force for any damage field; the internal force equals
  the frozen-indicator tangent times u;
* a brute-force element-by-element evaluation with the shape functions evaluated at
  physical points agrees with the vectorised assembly on tiny meshes;
* the FE patch test: a linear displacement on the boundary is reproduced exactly.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import specimens as S


def _1d(n, h):
    """Linear-element stiffness, mass and convection matrices on n elements of size h."""
    K = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    C = np.zeros((n + 1, n + 1))          # C[a, b] = int phi_a' phi_b
    for e in range(n):
        idx = [e, e + 1]
        K[np.ix_(idx, idx)] += np.array([[1, -1], [-1, 1]]) / h
        M[np.ix_(idx, idx)] += np.array([[2, 1], [1, 2]]) * h / 6
        C[np.ix_(idx, idx)] += np.array([[-0.5, -0.5], [0.5, 0.5]])
    return K, M, C


def _grid(nx, ny, Lx, Ly, flags=None, active=None):
    return q1.Grid(nx, ny, Lx, Ly, flags, active)


def test_damage_operator_is_tensor_product():
    nx, ny, Lx, Ly = 5, 3, 1.3, 0.7
    g = _grid(nx, ny, Lx, Ly)
    c, kappa = 2.5, 0.37
    A = q1.assemble_damage(g, np.full((g.ne, 4), c), kappa).toarray()
    Kx, Mx, _ = _1d(nx, Lx / nx)
    Ky, My, _ = _1d(ny, Ly / ny)
    ref = c * np.kron(My, Mx) + kappa * (np.kron(My, Kx) + np.kron(Ky, Mx))
    assert np.allclose(A, ref, rtol=1e-13, atol=1e-15)
    # rhs with constant H is the mass matrix applied to 2H
    b = q1.damage_rhs(g, np.full((g.ne, 4), 0.8))
    assert np.allclose(b, np.kron(My, Mx) @ np.full(g.nn, 1.6), rtol=1e-13)


@pytest.mark.parametrize("tension", [True, False])
def test_elasticity_operator_is_tensor_product(tension):
    nx, ny, Lx, Ly = 4, 3, 1.1, 0.9
    g = _grid(nx, ny, Lx, Ly)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1e-3, 0.1, 1e-6)
    dval = 0.3
    gd = model.g(dval, m.eta)
    K = q1.assemble_elasticity(g, np.full((g.ne, 4), dval), np.full((g.ne, 4), tension), m).toarray()
    # effective Lame constants of the frozen tangent
    if tension:
        lam_e, mu_e = gd * (m.K - 2 * m.mu / 3), gd * m.mu
    else:
        lam_e, mu_e = m.K - gd * 2 * m.mu / 3, gd * m.mu
    Kx, Mx, Cx = _1d(nx, Lx / nx)
    Ky, My, Cy = _1d(ny, Ly / ny)
    nn = g.nn
    # N_a = phi_ia(x) psi_ja(y) and a = ja (nx+1) + ia, so 2D integrals are kron(Y, X)
    xx = np.kron(My, Kx)
    yy = np.kron(Ky, Mx)
    xy = np.kron(Cy.T, Cx)                 # [a, b] = int dNa/dx dNb/dy
    ref = np.zeros((2 * nn, 2 * nn))
    ref[0::2, 0::2] = (lam_e + 2 * mu_e) * xx + mu_e * yy
    ref[1::2, 1::2] = (lam_e + 2 * mu_e) * yy + mu_e * xx
    ref[0::2, 1::2] = lam_e * xy + mu_e * xy.T
    ref[1::2, 0::2] = lam_e * xy.T + mu_e * xy
    assert np.allclose(K, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _random_grid_and_fields(nx, ny, seed, masked=False):
    r = np.random.default_rng(seed)
    active = None
    if masked:
        active = r.random(nx * ny) > 0.3
    g = _grid(nx, ny, 0.8, 0.6, active=active)
    d = r.random(g.nn)
    u = r.standard_normal(2 * g.nn) * 1e-3
    return g, d, u


@pytest.mark.parametrize("masked", [False, True])
def test_rigid_body_modes(masked):
    g, d, u = _random_grid_and_fields(6, 5, 1, masked)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1e-3, 0.1, 1e-6)
    dq = q1.interp_qp(g, d)
    ip = np.random.default_rng(2).random((g.ne, 4)) > 0.5
    K = q1.assemble_elasticity(g, dq, ip, m)
    j, i = np.divmod(np.arange(g.nn), g.nx + 1)
    x, y = i * g.hx, j * g.hy
    modes = [np.stack([np.ones(g.nn), np.zeros(g.nn)], 1).ravel(),
             np.stack([np.zeros(g.nn), np.ones(g.nn)], 1).ravel(),
             np.stack([-y, x], 1).ravel()]
    scale = abs(K).max()
    for r_ in modes:
        assert np.max(np.abs(K @ r_)) < 1e-12 * scale
        assert np.max(np.abs(q1.internal_force(g, r_ * 1e-3, dq, m))) < 1e-15 * scale


def test_internal_force_equals_tangent_times_u():
    g, d, u = _random_grid_and_fields(7, 4, 3)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1e-3, 0.1, 1e-6)
    dq = q1.interp_qp(g, d)
    exx, eyy, _ = q1.strains_qp(g, u)
    K = q1.assemble_elasticity(g, dq, model.tension(exx, eyy), m)
    F = q1.internal_force(g, u, dq, m)
    assert np.allclose(F, K @ u, rtol=1e-12, atol=1e-14 * np.abs(F).max())


def test_interpolation_and_strain_exact_for_bilinear_fields():
    g = _grid(5, 4, 1.5, 0.8)
    j, i = np.divmod(np.arange(g.nn), g.nx + 1)
    x, y = i * g.hx, j * g.hy
    a, b, c, e = 0.3, -1.2, 0.7, 2.1
    f = a + b * x + c * y + e * x * y
    s, t = q1.gauss_points_unit()
    ej, ei = np.divmod(np.arange(g.ne), g.nx)
    xq = (ei[:, None] + s[None]) * g.hx
    yq = (ej[:, None] + t[None]) * g.hy
    assert np.allclose(q1.interp_qp(g, f), a + b * xq + c * yq + e * xq * yq, rtol=1e-13)
    u = np.stack([f, 2 * f], 1).ravel()
    exx, eyy, exy = q1.strains_qp(g, u)
    assert np.allclose(exx, b + e * yq, rtol=1e-12)
    assert np.allclose(eyy, 2 * (c + e * xq), rtol=1e-12)
    assert np.allclose(exy, 0.5 * ((c + e * xq) + 2 * (b + e * yq)), rtol=1e-12)


def _brute_force(g, d, ip, m, c_q, kappa):
    """Element-by-element Gauss quadrature with the basis evaluated at physical points."""
    s_ref = [-1 / np.sqrt(3), 1 / np.sqrt(3)]
    Ku = np.zeros((2 * g.nn, 2 * g.nn))
    Kd = np.zeros((g.nn, g.nn))
    for e in range(g.ne):
        if not g.elem_active[e]:
            continue
        ej, ei = divmod(e, g.nx)
        x0, y0 = ei * g.hx, ej * g.hy
        nodes = [(ei, ej), (ei + 1, ej), (ei, ej + 1), (ei + 1, ej + 1)]
        ids = [jj * (g.nx + 1) + ii for ii, jj in nodes]
        q = 0
        for et in s_ref:
            for xi in s_ref:
                x = x0 + (xi + 1) / 2 * g.hx
                y = y0 + (et + 1) / 2 * g.hy
                N, dx, dy = [], [], []
                for ii, jj in nodes:
                    xa, ya = ii * g.hx, jj * g.hy
                    fx = 1 - abs(x - xa) / g.hx
                    fy = 1 - abs(y - ya) / g.hy
                    # hat functions 1 - |x - x_a| / h, derivative -sign(x - x_a) / h
                    sx = (-1.0 if xa <= x else 1.0) / g.hx
                    sy = (-1.0 if ya <= y else 1.0) / g.hy
                    N.append(fx * fy)
                    dx.append(sx * fy)
                    dy.append(fx * sy)
                N, dx, dy = map(np.array, (N, dx, dy))
                w = g.hx * g.hy / 4
                dval = N @ d[ids]
                D = model.tangent_voigt(np.array(dval), np.array(ip[e, q]), m)
                B = np.zeros((3, 8))
                B[0, 0::2], B[1, 1::2], B[2, 0::2], B[2, 1::2] = dx, dy, dy, dx
                dofs = np.ravel([[2 * a, 2 * a + 1] for a in ids])
                Ku[np.ix_(dofs, dofs)] += w * B.T @ D @ B
                Kd[np.ix_(ids, ids)] += w * (c_q[e, q] * np.outer(N, N)
                                             + kappa * (np.outer(dx, dx) + np.outer(dy, dy)))
                q += 1
    return Ku, Kd


@pytest.mark.parametrize("shape,masked", [((1, 1), False), ((2, 1), False), ((3, 3), False),
                                          ((3, 3), True)])
def test_assembly_matches_brute_force(shape, masked):
    g, d, u = _random_grid_and_fields(*shape, seed=4, masked=masked)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1e-3, 0.1, 1e-6)
    r = np.random.default_rng(5)
    ip = r.random((g.ne, 4)) > 0.5
    c_q = r.random((g.ne, 4)) * 3 - 1.0   # indefinite coefficients allowed
    Ku_ref, Kd_ref = _brute_force(g, d, ip, m, c_q, 0.25)
    Ku = q1.assemble_elasticity(g, q1.interp_qp(g, d), ip, m).toarray()
    Kd = q1.assemble_damage(g, c_q, 0.25).toarray()
    assert np.allclose(Ku, Ku_ref, rtol=1e-12, atol=1e-13 * np.abs(Ku_ref).max())
    assert np.allclose(Kd, Kd_ref, rtol=1e-12, atol=1e-13 * np.abs(Kd_ref).max())
    assert np.allclose(Ku, Ku.T, atol=1e-13 * np.abs(Ku).max())
    assert np.allclose(Kd, Kd.T, atol=1e-14 * np.abs(Kd).max())


def test_operators_spd_with_constraints():
    sp_ = S.tensile(6, l=0.2)
    g = q1.Grid(sp_.nx, sp_.ny, sp_.Lx, sp_.Ly, sp_.node_flags, sp_.elem_active)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 2.7e-3, 0.2, 1e-9)
    r = np.random.default_rng(6)
    dq = q1.interp_qp(g, r.random(g.nn))
    ip = r.random((g.ne, 4)) > 0.5
    free = ~g.u_constrained()
    K = q1.assemble_elasticity(g, dq, ip, m).toarray()[np.ix_(free, free)]
    assert np.linalg.eigvalsh(K).min() > 0
    fd = ~g.d_constrained()
    Kd = q1.assemble_damage(g, m.Gc / m.l + 2 * r.random((g.ne, 4)), m.Gc * m.l).toarray()
    assert np.linalg.eigvalsh(Kd[np.ix_(fd, fd)]).min() > 0


@pytest.mark.parametrize("dval,sign", [(0.0, 1.0), (0.5, 1.0), (0.0, -1.0), (0.5, -1.0)])
def test_patch_test(dval, sign):
    """Linear displacement prescribed on the boundary; interior reproduced exactly."""
    nx, ny = 6, 5
    j, i = np.divmod(np.arange((nx + 1) * (ny + 1)), nx + 1)
    bnd = (i == 0) | (i == nx) | (j == 0) | (j == ny)
    flags = np.where(bnd, q1.FIX_X | q1.FIX_Y, 0).astype(np.uint8)
    g = _grid(nx, ny, 1.2, 0.9, flags)
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1e-3, 0.1, 1e-6)
    x, y = i * g.hx, j * g.hy
    ex, ey, gxy = 1e-3 * sign, 0.4e-3 * sign, 0.3e-3
    u_lin = np.stack([ex * x + 0.5 * gxy * y, ey * y + 0.5 * gxy * x], 1).ravel()
    u0 = np.where(g.u_constrained(), u_lin, 0.0)
    d = np.full(g.nn, dval)
    u, nn, ok = stg.solve_u(g, m, u0, d, stg.Options(tol_nr=1e-12))
    assert ok
    assert np.allclose(u, u_lin, rtol=0, atol=1e-13)
    F = q1.internal_force(g, u_lin, q1.interp_qp(g, d), m)
    inner = ~g.u_constrained()
    assert np.max(np.abs(F[inner])) < 1e-12 * np.max(np.abs(F))
