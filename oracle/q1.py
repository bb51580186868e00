"""Bilinear (Q1) finite elements on a structured grid (oracle; test infrastructure only).

Discretisation of the weak forms F_u and F_d of Sec. 3.2 (shape functions N_u, N_d and
derivative operators B_u, B_d) on an nx-by-ny grid of rectangular elements of size
hx-by-hy, integrated with the 2x2 Gauss rule.

Numbering.  Node (i, j), 0 <= i <= nx, 0 <= j <= ny, has id j (nx+1) + i and sits at
(i hx, j hy).  Element (i, j) has id j nx + i and local nodes
a0 = (i, j), a1 = (i+1, j), a2 = (i, j+1), a3 = (i+1, j+1).  Displacement DOFs are
interleaved: 2 id + 0 is u_x, 2 id + 1 is u_y.  Quadrature points are stored
element-major, four per element, in the order (-,-), (+,-), (-,+), (+,+) of the
reference coordinates (+-1/sqrt 3); each carries the weight hx hy / 4.

Node flags (bit field, one byte per node):
    FIX_X=1, FIX_Y=2   u_x / u_y held at zero
    LOAD_X=4, LOAD_Y=8 u_x / u_y held at the prescribed load value
    D_FIX1=16          d held at 1 (the initial slit)
    D_FIX0=32          d held at 0 (protected region under a load patch)
A node with no active element (masked-out region of an L-shaped panel) has all of its
DOFs held at zero.
"""
import numpy as np
import scipy.sparse as sp

from . import model

FIX_X, FIX_Y, LOAD_X, LOAD_Y, D_FIX1, D_FIX0 = 1, 2, 4, 8, 16, 32


class Grid:
    def __init__(self, nx, ny, Lx, Ly, node_flags=None, elem_active=None):
        self.nx, self.ny = int(nx), int(ny)
        self.Lx, self.Ly = float(Lx), float(Ly)
        self.hx, self.hy = self.Lx / self.nx, self.Ly / self.ny
        self.nn = (self.nx + 1) * (self.ny + 1)
        self.ne = self.nx * self.ny
        self.node_flags = (np.zeros(self.nn, np.uint8) if node_flags is None
                           else np.asarray(node_flags, np.uint8).copy())
        self.elem_active = (np.ones(self.ne, bool) if elem_active is None
                            else np.asarray(elem_active).astype(bool).copy())
        assert self.node_flags.shape == (self.nn,)
        assert self.elem_active.shape == (self.ne,)
        ej, ei = np.divmod(np.arange(self.ne), self.nx)
        n0 = ej * (self.nx + 1) + ei
        self.conn = np.stack([n0, n0 + 1, n0 + self.nx + 1, n0 + self.nx + 2], axis=1)
        touched = np.zeros(self.nn, bool)
        touched[self.conn[self.elem_active].ravel()] = True
        self.orphan = ~touched

    # ---- constraints -----------------------------------------------------------------
    def u_constrained(self):
        """Boolean mask over the 2N displacement DOFs that carry a Dirichlet value."""
        f = self.node_flags
        cx = ((f & (FIX_X | LOAD_X)) != 0) | self.orphan
        cy = ((f & (FIX_Y | LOAD_Y)) != 0) | self.orphan
        return np.stack([cx, cy], axis=1).ravel()

    def u_dirichlet_values(self, ubar):
        """Prescribed displacement on constrained DOFs (zero elsewhere)."""
        f = self.node_flags
        vx = np.where(((f & LOAD_X) != 0) & ~self.orphan, ubar, 0.0)
        vy = np.where(((f & LOAD_Y) != 0) & ~self.orphan, ubar, 0.0)
        return np.stack([vx, vy], axis=1).ravel()

    def d_constrained(self):
        return ((self.node_flags & (D_FIX1 | D_FIX0)) != 0) | self.orphan

    def d_dirichlet_values(self):
        return np.where(((self.node_flags & D_FIX1) != 0) & ~self.orphan, 1.0, 0.0)


# ---- reference element ------------------------------------------------------------------
def gauss_points_unit():
    """Unit-square coordinates (s, t) of the 2x2 Gauss points in storage order."""
    a = 0.5 * (1.0 - 1.0 / np.sqrt(3.0))
    b = 0.5 * (1.0 + 1.0 / np.sqrt(3.0))
    s = np.array([a, b, a, b])
    t = np.array([a, a, b, b])
    return s, t


def shape_tables(hx, hy):
    """N[q, a], dN/dx[q, a], dN/dy[q, a] of the bilinear element at the Gauss points."""
    s, t = gauss_points_unit()
    N = np.stack([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t], axis=1)
    dNds = np.stack([-(1 - t), (1 - t), -t, t], axis=1)
    dNdt = np.stack([-(1 - s), -s, (1 - s), s], axis=1)
    return N, dNds / hx, dNdt / hy


def qp_weight(grid):
    """Gauss weight (1) times the Jacobian determinant hx hy / 4 of the reference map."""
    return grid.hx * grid.hy / 4.0


# ---- fields at quadrature points --------------------------------------------------------
def interp_qp(grid, f):
    """Nodal scalar field -> values at the quadrature points, shape (ne, 4)."""
    N, _, _ = shape_tables(grid.hx, grid.hy)
    return f[grid.conn] @ N.T


def strains_qp(grid, u):
    """Strain components (exx, eyy, exy) at the quadrature points, each (ne, 4)."""
    _, Bx, By = shape_tables(grid.hx, grid.hy)
    ux = u[0::2][grid.conn]
    uy = u[1::2][grid.conn]
    exx = ux @ Bx.T
    eyy = uy @ By.T
    exy = 0.5 * (ux @ By.T + uy @ Bx.T)
    return exx, eyy, exy


def _bmat(grid):
    """Strain-displacement matrices B[q] (3 x 8, Voigt xx, yy, engineering xy)."""
    _, Bx, By = shape_tables(grid.hx, grid.hy)
    B = np.zeros((4, 3, 8))
    B[:, 0, 0::2] = Bx
    B[:, 1, 1::2] = By
    B[:, 2, 0::2] = By
    B[:, 2, 1::2] = Bx
    return B


def _elem_dofs(grid):
    c = grid.conn
    return np.stack([2 * c[:, 0], 2 * c[:, 0] + 1, 2 * c[:, 1], 2 * c[:, 1] + 1,
                     2 * c[:, 2], 2 * c[:, 2] + 1, 2 * c[:, 3], 2 * c[:, 3] + 1], axis=1)


# ---- elasticity (momentum balance) ------------------------------------------------------
def assemble_elasticity(grid, d_q, ip, m, D=None):
    """Tangent K_uu = sum_e sum_q w B_q^T D_q B_q (CSR, 2N x 2N), all DOFs, no constraints.

    ``d_q`` (ne, 4) phase field at the points, ``ip`` (ne, 4) frozen tension indicator of
    the VD split; ``D`` (ne, 4, 3, 3) gives the point tangents directly instead.
    """
    B = _bmat(grid)
    if D is None:
        D = model.tangent_voigt(d_q, ip, m)                  # (ne, 4, 3, 3)
    Ke = np.einsum('qia,eqij,qjb->eab', B, D, B) * qp_weight(grid)
    Ke *= grid.elem_active[:, None, None]
    dofs = _elem_dofs(grid)
    rows = np.repeat(dofs, 8, axis=1).ravel()
    cols = np.tile(dofs, (1, 8)).ravel()
    n = 2 * grid.nn
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))


def assemble_elasticity_at(grid, u, d_q, m):
    """Newton tangent of the internal force at u for the material's split
    (model.tangent_at at every point)."""
    exx, eyy, exy = strains_qp(grid, u)
    return assemble_elasticity(grid, d_q, None, m, D=model.tangent_at(exx, eyy, exy, d_q, m))


def internal_force(grid, u, d_q, m):
    """F_u^int = sum_e sum_q w B_q^T sigma(eps(u), d) over all 2N DOFs (Sec. 3.2)."""
    exx, eyy, exy = strains_qp(grid, u)
    sxx, syy, sxy = model.stress(exx, eyy, exy, d_q, m)
    S = np.stack([sxx, syy, sxy], axis=2) * grid.elem_active[:, None, None]
    B = _bmat(grid)
    fe = np.einsum('qia,eqi->ea', B, S) * qp_weight(grid)
    F = np.zeros(2 * grid.nn)
    np.add.at(F, _elem_dofs(grid).ravel(), fe.ravel())
    return F


# ---- phase field (evolution equation) ---------------------------------------------------
def assemble_damage(grid, c_q, kappa):
    """K_dd = sum_e sum_q w [c_q N N^T + kappa (dN/dx dN/dx^T + dN/dy dN/dy^T)] (CSR, N x N).

    For AT2 with a history field, c_q = G_c/l + 2 H_q and kappa = G_c l (Sec. 2 and 3.2,
    c_w = 2).  The fixed-stress schemes add K~ to c_q (Sec. 3.4).
    """
    N, Bx, By = shape_tables(grid.hx, grid.hy)
    w = qp_weight(grid)
    mass = np.einsum('eq,qa,qb->eab', c_q, N, N)
    lap = np.einsum('qa,qb->ab', Bx, Bx) + np.einsum('qa,qb->ab', By, By)
    Ke = (mass + kappa * lap[None]) * w
    Ke *= grid.elem_active[:, None, None]
    c = grid.conn
    rows = np.repeat(c, 4, axis=1).ravel()
    cols = np.tile(c, (1, 4)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(grid.nn, grid.nn))


def damage_rhs(grid, H_q):
    """b = sum_e sum_q w 2 H_q N_q (the AT2 driving term, Sec. 3.2 with Psi+ -> H)."""
    N, _, _ = shape_tables(grid.hx, grid.hy)
    be = 2.0 * (H_q * grid.elem_active[:, None]) @ N * qp_weight(grid)
    b = np.zeros(grid.nn)
    np.add.at(b, grid.conn.ravel(), be.ravel())
    return b


# ---- post-processing ----------------------------------------------------------------------
def reaction_force(grid, F_int, direction):
    """Sum of the internal-force component ``direction`` over the loaded nodes.

    The loaded nodes are those with LOAD_X (direction 0) or LOAD_Y (direction 1); the
    reaction there balances the internal force (units: force per unit thickness).
    """
    bit = LOAD_X if direction == 0 else LOAD_Y
    sel = ((grid.node_flags & bit) != 0) & ~grid.orphan
    return float(np.sum(F_int[2 * np.nonzero(sel)[0] + direction]))
