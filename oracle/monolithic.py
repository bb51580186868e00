"""Monolithic Newton for the coupled momentum balance and evolution equation (oracle;
test infrastructure only).

Sec. 3.2 writes one Newton iteration of the coupled problem as a linear system for the
increments of (u, d) with the full Jacobian [[K_uu, K_ud], [K_du, K_dd]], K_ab = dF_a/db,
and obtains the staggered d-u iteration from it by dropping K_du inside a pass.  This
module keeps K_du: it solves each load step with the full Jacobian (plain Newton, exact
sparse LU, no line search) and serves as a reference for the converged state of a load
step, i.e. the staggered fixed point as TOL_ST -> 0.  AT2 with the history field:

  R_u = F_u(u, d)                      (internal force, q1.internal_force)
  R_d = K_dd(G_c/l + 2H) d - int 2H N  (evolution equation, H = max(H_{n-1}, Psi+(u)))

  K_uu = dF_u/du                       (q1.assemble_elasticity_at: the semismooth VD
                                        tangent or the spectral consistent tangent)
  K_ud = sum_q w B^T g'(d_q) sigma+_q N^T                  (g' = -2(1-d))
  K_du = sum_q w N (-2 (1-d_q)) [Psi+_q > H_{n-1,q}] sigma+_q^T B
  K_dd = sum_q w (G_c/l + 2H_q) N N^T + G_c l grad N grad N^T

Start: the momentum balance solved at d_{n-1} (the first half-step of the staggered
schemes); from the previous converged u with only the new Dirichlet values the plain coupled
iteration diverges on the notched specimens.  Stop: the Newton test of R10 on R_u and the
staggered test of R9 on R_d, both at the returned state.  ``newton`` counts the linear
solves, predictor included.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import model, q1, staggered


def history(grid, m, u, H_prev):
    exx, eyy, exy = q1.strains_qp(grid, u)
    psi = model.psi_plus(exx, eyy, exy, m)
    return np.maximum(H_prev, psi), psi > H_prev


def residual(grid, m, u, d, H_prev):
    """(R_u over 2N DOFs, R_d over N DOFs, H at the points)."""
    d_q = q1.interp_qp(grid, d)
    R_u = q1.internal_force(grid, u, d_q, m)
    H, _ = history(grid, m, u, H_prev)
    R_d = q1.assemble_damage(grid, m.Gc / m.l + 2.0 * H, m.Gc * m.l) @ d \
        - q1.damage_rhs(grid, H)
    return R_u, R_d, H


def jacobian(grid, m, u, d, H_prev):
    """Full Jacobian of (R_u, R_d) with respect to (u, d), CSR of size 3N, unknowns
    ordered [u (2N, interleaved); d (N)]."""
    nn = grid.nn
    d_q = q1.interp_qp(grid, d)
    H, grow = history(grid, m, u, H_prev)
    K_uu = q1.assemble_elasticity_at(grid, u, d_q, m)
    K_dd = q1.assemble_damage(grid, m.Gc / m.l + 2.0 * H, m.Gc * m.l)
    exx, eyy, exy = q1.strains_qp(grid, u)
    sp_ = np.stack(model.stress_plus(exx, eyy, exy, m), axis=2)        # (ne, 4, 3)
    N, _, _ = q1.shape_tables(grid.hx, grid.hy)                         # (4 q, 4 a)
    B = q1._bmat(grid)                                                  # (4 q, 3, 8)
    w = q1.qp_weight(grid) * grid.elem_active[:, None]                  # (ne, 1)
    BtS = np.einsum('qia,eqi->eqa', B, sp_)                             # (ne, 4, 8)
    gp = model.dg(d_q)                                                  # g'(d) = -2(1-d)
    Ke_ud = np.einsum('eqa,eq,qb->eab', BtS, w * gp, N)                 # (ne, 8, 4)
    Ke_du = np.einsum('qa,eq,eqb->eab', N, w * gp * grow, BtS)          # (ne, 4, 8)
    udofs = q1._elem_dofs(grid)
    ddofs = grid.conn + 2 * nn
    rows = np.concatenate([np.repeat(udofs, 4, axis=1).ravel(),
                           np.repeat(ddofs, 8, axis=1).ravel()])
    cols = np.concatenate([np.tile(ddofs, (1, 8)).ravel(), np.tile(udofs, (1, 4)).ravel()])
    vals = np.concatenate([Ke_ud.ravel(), Ke_du.ravel()])
    off = sp.csr_matrix((vals, (rows, cols)), shape=(3 * nn, 3 * nn))
    return sp.block_diag([K_uu, K_dd], format='csr') + off


class Result:
    def __init__(self):
        self.converged = False
        self.newton = 0
        self.reaction = 0.0
        self.ubar = 0.0


def load_step(grid, m, state, dubar, tol_nr=1e-7, tol_st=1e-9, max_newton=50,
              reaction_dir=1):
    """Advance ``state`` (staggered.State) by one load increment with monolithic Newton
    from the previous converged state."""
    res = Result()
    state.ubar += dubar
    res.ubar = state.ubar
    nn = grid.nn
    cu = grid.u_constrained()
    cd = grid.d_constrained()
    u = state.u.copy()
    u[cu] = grid.u_dirichlet_values(state.ubar)[cu]
    d = state.d.copy()
    # start from the momentum balance solved at d_{n-1}, as the staggered schemes do
    u, res.newton, _ = staggered.solve_u(grid, m, u, d, staggered.Options(tol_nr=tol_nr))
    free = np.concatenate([~cu, ~cd])
    r0 = None
    for it in range(max_newton + 1):
        R_u, R_d, H = residual(grid, m, u, d, state.H)
        rn = np.linalg.norm(R_u[~cu])
        fref = np.linalg.norm(R_u[cu])
        if r0 is None:
            r0 = rn
        K_dd = q1.assemble_damage(grid, m.Gc / m.l + 2.0 * H, m.Gc * m.l)
        rd = np.max(np.abs(R_d[~cd] / K_dd.diagonal()[~cd])) if np.any(~cd) else 0.0
        if (rn == 0.0 or rn <= tol_nr * max(r0, fref)) and rd <= tol_st:
            res.converged = True
            break
        if it == max_newton:
            break
        J = jacobian(grid, m, u, d, state.H)
        R = np.concatenate([R_u, R_d])
        dz = np.zeros(3 * nn)
        dz[free] = spla.splu(J[free][:, free].tocsc()).solve(-R[free])
        u += dz[:2 * nn]
        d += dz[2 * nn:]
        res.newton += 1
    state.u, state.d = u, d
    state.H = history(grid, m, u, state.H)[0]
    state.step += 1
    F = q1.internal_force(grid, u, q1.interp_qp(grid, d), m)
    res.reaction = q1.reaction_force(grid, F, reaction_dir)
    return res
