"""Standard and fixed-stress staggered schemes (oracle; test infrastructure only).

Follows Sec. 3 of the paper step by step, for the AT2 model with a history field
(Sec. 2: the history variable replacing Psi+; Sec. 3.1 and 3.3: with AT2 and a history
field the evolution equation is linear, so one NR iteration solves it).  Every linear
system is solved exactly with SciPy's sparse LU (SuperLU); the augmented fixed-stress
system is SPD under the reading of model.augmented_coefficient (LU also solves the
unlimited, indefinite form when that reading is switched off).

Per load step n (Sec. 3.1, Fig. 1, d-u order):
  1. ubar_n = ubar_{n-1} + dubar; the Dirichlet values are applied to u.
  2. k = 0: the evolution equation is skipped, the momentum balance is solved with
     d_{n-1} (semismooth Newton, frozen tension indicator per iteration).
  3. staggered loop: d-step, u-step, then the residual of the evolution equation at
     (d^{k+1}, u^{k+1}) is checked against TOL_ST.
  4. commit H_n = max(H_{n-1}, Psi+(u_n)), report the reaction force.

The d-step of the S1/S2/S3 schemes (Sec. 3.3-3.5): the extra stiffness K~^S is added
where the softening test holds; the first NR iteration of the evolution equation with
the augmented tangent gives Delta d; the active energy is predicted from Delta d
(Sec. 3.3, Delta d > 0 rule of Sec. 3.5); the energy is then frozen (footnote of
Sec. 3.3) and the now linear evolution equation is solved once more, exactly.

Both energy splits of Sec. 2 are supported (model.VD, model.SPECTRAL); the spectral split
uses the consistent tangent of its stress in the Newton iteration (model.tangent_spectral).

Readings where the paper is silent (the same readings are used by the CUDA path):
  * Newton stop: ||R_free||_2 <= TOL_NR * max(||R_free^0||_2, ||F_int on constrained||_2)
  * staggered residual: max over free d-DOFs of |R_d_i / (K_dd)_ii| with H from u^{k+1}
  * Psi_max of the activation test = committed history H_{n-1} at the point
  * at least one d-u pass per load step
  * the augmented per-point coefficient G_c/l + 2H + K~ is kept >= G_c/l (convexity
    of the d-subproblem, footnote of Sec. 3.3); see model.augmented_coefficient
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import model, q1


class Options:
    def __init__(self, tol_nr=1e-7, tol_st=1e-6, max_newton=50, max_stag=1000,
                 psi_crit=None, project=False, kt_floor=True, model=0, tol_ir=0.01,
                 tol_d=1e-10):
        self.tol_nr = tol_nr          # TOL_NR (Sec. 4 intro: 1e-7)
        self.tol_st = tol_st          # TOL_ST (Sec. 4 intro: 1e-6)
        self.max_newton = max_newton
        self.max_stag = max_stag
        self.psi_crit = psi_crit      # override of Psi_crit (None: G_c/(c_w l))
        self.project = project        # clamp d into [d_{n-1}, 1] after each d-solve
        self.kt_floor = kt_floor      # augmented coefficient >= G_c/l (model.augmented_coefficient)
        self.model = model            # model.AT2 (history field) or model.AT1 (penalty)
        self.tol_ir = tol_ir          # AT1 irreversibility tolerance (Sec. 2: 0.01)
        self.tol_d = tol_d            # AT1 d-Newton stop (relative; the equation is piecewise
                                      # linear, so Newton is exact once the penalty set settles)


class State:
    """Committed state between load steps: u (2N), d (N), H (ne, 4), ubar, step."""

    def __init__(self, grid):
        self.u = np.zeros(2 * grid.nn)
        self.d = grid.d_dirichlet_values().astype(float)
        self.H = np.zeros((grid.ne, 4))
        self.ubar = 0.0
        self.step = 0

    def copy(self):
        s = State.__new__(State)
        s.u, s.d, s.H = self.u.copy(), self.d.copy(), self.H.copy()
        s.ubar, s.step = self.ubar, self.step
        return s


class StepResult:
    def __init__(self):
        self.reaction = 0.0
        self.stag_residual = np.inf
        self.stag_iters = 0
        self.newton_u = 0
        self.d_solves = 0
        self.converged = False
        self.ubar = 0.0


def _lu_solve(A, b):
    return spla.splu(A.tocsc()).solve(b)


def psi_plus_qp(grid, u, m):
    exx, eyy, exy = q1.strains_qp(grid, u)
    return model.psi_plus(exx, eyy, exy, m)


def solve_u(grid, m, u, d, opts):
    """Semismooth Newton for F_u(u; d) = 0; u carries its Dirichlet values on entry.

    Returns (u, number of linear solves, converged).
    """
    u = u.copy()
    d_q = q1.interp_qp(grid, d)
    cu = grid.u_constrained()
    free = ~cu
    r0 = None
    for it in range(opts.max_newton + 1):
        F = q1.internal_force(grid, u, d_q, m)
        rn = np.linalg.norm(F[free])
        fref = np.linalg.norm(F[cu])
        if r0 is None:
            r0 = rn
        if rn == 0.0 or rn <= opts.tol_nr * max(r0, fref):
            return u, it, True
        if it == opts.max_newton:
            break
        if m.split == model.SPECTRAL:
            K = q1.assemble_elasticity_at(grid, u, d_q, m)
        else:
            exx, eyy, _ = q1.strains_qp(grid, u)
            ip = model.tension(exx, eyy)
            K = q1.assemble_elasticity(grid, d_q, ip, m)
        Kff = K[free][:, free]
        u[free] += _lu_solve(Kff, -F[free])
    return u, opts.max_newton, False


def _solve_damage_dirichlet(grid, c_q, kappa, rhs):
    """Solve K_dd(c_q) d = rhs with the Dirichlet values of the phase field."""
    K = q1.assemble_damage(grid, c_q, kappa)
    cd = grid.d_constrained()
    free = ~cd
    d = grid.d_dirichlet_values().astype(float)
    r = rhs[free] - K[free][:, cd] @ d[cd]
    d[free] = _lu_solve(K[free][:, free], r)
    return d


def d_step_standard(grid, m, H_k):
    """ST d-step: [int (G_c/l + 2H) N N^T + G_c l int grad N grad N^T] d = int 2H N."""
    c_q = m.Gc / m.l + 2.0 * H_k
    return _solve_damage_dirichlet(grid, c_q, m.Gc * m.l, q1.damage_rhs(grid, H_k))


class _FixedStressTerms:
    """K~ and the prediction at the points of u^k: the VD forms on (tr, e.e) for the VD
    split, the forms on the energy parts for the spectral split (model module docstring)."""

    def __init__(self, grid, m, u_k):
        exx, eyy, exy = q1.strains_qp(grid, u_k)
        self.m = m
        self.psi = model.psi_plus(exx, eyy, exy, m)
        if m.split == model.SPECTRAL:
            self.pa, self.pb = model.psi_parts(exx, eyy, exy, m)
        else:
            self.tr, self.ee = model.invariants(exx, eyy, exy, m.cdim)

    def extra(self, d_q, scheme):
        if self.m.split == model.SPECTRAL:
            return model.extra_stiffness_parts(self.pa, self.pb, d_q, scheme, self.m)
        return model.extra_stiffness(self.tr, self.ee, d_q, scheme, self.m)

    def predict(self, d_q, dd_q, scheme):
        if self.m.split == model.SPECTRAL:
            return model.predict_psi_parts(self.pa, self.pb, d_q, dd_q, scheme, self.m)
        return model.predict_psi(self.tr, self.ee, d_q, dd_q, scheme, self.m)


def d_step_fixed_stress(grid, m, u_k, d_k, H_prev, scheme, opts, info=None):
    """S1/S2/S3 d-step (Sec. 3.3-3.5): augmented NR iteration, prediction, frozen solve."""
    fs = _FixedStressTerms(grid, m, u_k)
    psi = fs.psi
    H_k = np.maximum(H_prev, psi)
    d_q = q1.interp_qp(grid, d_k)
    act = model.activation(psi, H_prev, d_q, m, opts.psi_crit) & grid.elem_active[:, None]
    k_extra = np.where(act, fs.extra(d_q, scheme), 0.0)
    c_std = m.Gc / m.l + 2.0 * H_k
    kappa = m.Gc * m.l
    # residual of the evolution equation at (d^k, H^k)
    R = q1.assemble_damage(grid, c_std, kappa) @ d_k - q1.damage_rhs(grid, H_k)
    # first NR iteration with the augmented tangent K_dd + K~^S
    K_aug = q1.assemble_damage(grid, model.augmented_coefficient(H_k, k_extra, m, opts.kt_floor),
                               kappa)
    cd = grid.d_constrained()
    free = ~cd
    dd = np.zeros(grid.nn)
    dd[free] = _lu_solve(K_aug[free][:, free], -R[free])
    # predicted active energy, then the frozen (linear) solve
    dd_q = q1.interp_qp(grid, dd)
    psi_hat = np.where(act, fs.predict(d_q, dd_q, scheme), psi)
    H_half = np.maximum(H_prev, psi_hat)
    if info is not None:
        info['active'] = act
        info['delta_d'] = dd
        info['H_half'] = H_half
    return d_step_standard(grid, m, H_half)


def stag_residual(grid, m, u, d, H_prev):
    """max_i |R_d,i / (K_dd)_ii| over free d-DOFs, with H = max(H_{n-1}, Psi+(u))."""
    H = np.maximum(H_prev, psi_plus_qp(grid, u, m))
    K = q1.assemble_damage(grid, m.Gc / m.l + 2.0 * H, m.Gc * m.l)
    R = K @ d - q1.damage_rhs(grid, H)
    free = ~grid.d_constrained()
    if not np.any(free):
        return 0.0
    return float(np.max(np.abs(R[free] / K.diagonal()[free])))


# ---- AT1 with penalty irreversibility --------------------------------------------------
def at1_residual(grid, m, psi, d, d_prev, opts):
    """R_d(d) = int [-2(1-d) Psi + a + gamma <d - d_{n-1}>_-] N + kappa int grad N . grad d
    (Sec. 2) at per-point energy ``psi``; also returns the Jacobian coefficient and kappa."""
    a, kappa, gamma = model.at1_constants(m, opts.tol_ir)
    d_q = q1.interp_qp(grid, d)
    dp_q = q1.interp_qp(grid, d_prev)
    K = q1.assemble_damage(grid, 2.0 * psi, kappa)        # 2 Psi d N + kappa grad grad
    src = -2.0 * psi + a + gamma * np.minimum(d_q - dp_q, 0.0)
    R = K @ d + q1.damage_rhs(grid, 0.5 * src)            # damage_rhs integrates 2 (.) N
    return R, model.at1_mass_coefficient(psi, d_q, dp_q, gamma), kappa


def at1_newton(grid, m, psi, d, d_prev, opts, c_first=None):
    """Semismooth Newton for the AT1 evolution equation at fixed energy ``psi``.

    c_first: per-point mass coefficient of the first iteration's matrix (the fixed-stress
    augmented tangent), None for the exact Jacobian.  Stop: ||R_free|| <= tol_d *
    max(||R^0_free||, ||int a N||).  The equation is piecewise linear (the penalty), so once
    the penalised set stops changing the next iterate is exact; tol_d (1e-10) is therefore
    tighter than TOL_NR, which would leave a d-residual above the staggered test's
    tolerance.  Returns (d, first increment, iterations).
    """
    a, kappa, _ = model.at1_constants(m, opts.tol_ir)
    cd = grid.d_constrained()
    free = ~cd
    d = d.copy()
    fscale = np.linalg.norm(q1.damage_rhs(grid, np.full((grid.ne, 4), 0.5 * a))[free])
    r0 = None
    first = np.zeros(grid.nn)
    for it in range(opts.max_newton + 1):
        R, cJ, _ = at1_residual(grid, m, psi, d, d_prev, opts)
        rn = np.linalg.norm(R[free])
        if r0 is None:
            r0 = rn
        if rn == 0.0 or rn <= opts.tol_d * max(r0, fscale):
            return d, first, it
        if it == opts.max_newton:
            break
        c = c_first if (it == 0 and c_first is not None) else cJ
        J = q1.assemble_damage(grid, c, kappa)
        dd = np.zeros(grid.nn)
        dd[free] = _lu_solve(J[free][:, free], -R[free])
        if it == 0:
            first = dd
        d = d + dd
    return d, first, opts.max_newton


def at1_d_step(grid, m, u_k, d_k, d_prev, H_prev, scheme, opts):
    """AT1 d-step.  ST: Newton with Psi+(u^k).  S1/S2/S3 (Sec. 3.3-3.5): the first NR
    iteration with the augmented tangent gives Delta d; the active energy is predicted from
    it where the softening test holds and frozen; the NR iterations continue with it."""
    fs = _FixedStressTerms(grid, m, u_k)
    psi = fs.psi
    if scheme == model.ST:
        return at1_newton(grid, m, psi, d_k, d_prev, opts)[0]
    a, kappa, gamma = model.at1_constants(m, opts.tol_ir)
    d_q = q1.interp_qp(grid, d_k)
    pc = a if opts.psi_crit is None else opts.psi_crit
    act = model.activation(psi, H_prev, d_q, m, pc) & grid.elem_active[:, None]
    k_extra = np.where(act, fs.extra(d_q, scheme), 0.0)
    cJ = model.at1_mass_coefficient(psi, d_q, q1.interp_qp(grid, d_prev), gamma)
    c_aug = model.at1_augmented_coefficient(cJ, k_extra, m, opts.kt_floor)
    opts1 = Options(tol_nr=opts.tol_nr, max_newton=1, model=opts.model, tol_ir=opts.tol_ir,
                    tol_d=opts.tol_d)
    d_half, dd, _ = at1_newton(grid, m, psi, d_k, d_prev, opts1, c_first=c_aug)
    dd_q = q1.interp_qp(grid, dd)
    psi_hat = np.where(act, fs.predict(d_q, dd_q, scheme), psi)
    return at1_newton(grid, m, psi_hat, d_k + dd, d_prev, opts)[0]


def at1_stag_residual(grid, m, u, d, d_prev, opts):
    """max_i |R_d,i / J_ii| over free d-DOFs with Psi+(u^{k+1}) and the penalty at d."""
    psi = psi_plus_qp(grid, u, m)
    R, cJ, kappa = at1_residual(grid, m, psi, d, d_prev, opts)
    J = q1.assemble_damage(grid, cJ, kappa)
    free = ~grid.d_constrained()
    if not np.any(free):
        return 0.0
    return float(np.max(np.abs(R[free] / J.diagonal()[free])))


def load_step(grid, m, state, dubar, scheme, opts, reaction_dir=1, trace=None):
    """Advance ``state`` by one load increment ``dubar`` with the given scheme.

    Returns a StepResult; ``state`` is updated in place (also when not converged).
    """
    res = StepResult()
    state.ubar += dubar
    res.ubar = state.ubar
    cu = grid.u_constrained()
    u = state.u.copy()
    u[cu] = grid.u_dirichlet_values(state.ubar)[cu]
    d = state.d.copy()
    d_prev = state.d.copy()
    H_prev = state.H
    u, nn, ok = solve_u(grid, m, u, d, opts)
    res.newton_u += nn
    for k in range(opts.max_stag):
        if opts.model == model.AT1:
            d = at1_d_step(grid, m, u, d, d_prev, H_prev, scheme, opts)
            res.d_solves += 1 if scheme == model.ST else 2
        elif scheme == model.ST:
            H_k = np.maximum(H_prev, psi_plus_qp(grid, u, m))
            d = d_step_standard(grid, m, H_k)
            res.d_solves += 1
        else:
            d = d_step_fixed_stress(grid, m, u, d, H_prev, scheme, opts)
            res.d_solves += 2
        if opts.project:
            d = np.clip(d, d_prev, 1.0)
        u, nn, ok = solve_u(grid, m, u, d, opts)
        res.newton_u += nn
        if opts.model == model.AT1:
            r = at1_stag_residual(grid, m, u, d, d_prev, opts)
        else:
            r = stag_residual(grid, m, u, d, H_prev)
        res.stag_iters = k + 1
        res.stag_residual = r
        if trace is not None:
            trace.append((k + 1, r, d.copy()))
        if r <= opts.tol_st:
            res.converged = True
            break
    state.u, state.d = u, d
    state.H = np.maximum(H_prev, psi_plus_qp(grid, u, m))
    state.step += 1
    F = q1.internal_force(grid, u, q1.interp_qp(grid, d), m)
    res.reaction = q1.reaction_force(grid, F, reaction_dir)
    return res


def load_path(grid, m, increments, scheme, opts, reaction_dir=1, state=None):
    """Run a sequence of load increments; returns (results, final state)."""
    st = State(grid) if state is None else state
    out = []
    for du in increments:
        out.append(load_step(grid, m, st, du, scheme, opts, reaction_dir))
    return out, st
