"""Pins of the checker's AT1 model with penalty irreversibility (Sec. 2, Table 1).

AT1: g(d) = (1-d)^2 + eta, w(d) = d, c_w = 8/3; the evolution equation

    -2 (1-d) Psi+ + G_c/(c_w l) + gamma <d - d_{n-1}>_- - (2 G_c l / c_w) lap d = 0,

gamma = 27 G_c / (64 l tol_ir^2), is nonlinear through the penalty term and is solved by
semismooth Newton.  Pinned against closed forms:
- the homogeneous uniaxial-strain bar, where the strain is prescribed by the boundary and
  d solves the scalar stationarity equation at every load step (also across unloading,
  where the penalty keeps d_n >= d_{n-1} - (8/9) tol_ir^2);
- the 1D profile (1 - x/(2l))^2 of a crack at x = 0 with no elastic energy (second-order
  convergence with h);
- S1/S2/S3 equal ST bit for bit when the softening test never holds.
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import specimens as S


def _grid(sp):
    return q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)


def _mat(sp):
    return model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane)


def _scalar_d(psi, d_prev, a, gamma):
    """Solution of -2(1-d) psi + a + gamma <d - d_prev>_- = 0 (homogeneous state)."""
    d_free = 1.0 - a / (2.0 * psi) if psi > 0 else -np.inf
    if d_free >= d_prev:
        return d_free
    return (2.0 * psi - a + gamma * d_prev) / (2.0 * psi + gamma)


@pytest.mark.parametrize("scheme", [model.ST, model.S1, model.S3])
def test_at1_homogeneous_bar(scheme):
    lam, mu, Gc, l, eta = 121.15, 80.77, 2.7e-3, 0.03, 1e-9
    M = lam + 2 * mu
    tol_ir = 0.01
    opts = stg.Options(tol_st=1e-10, tol_nr=1e-11, max_stag=300, model=model.AT1,
                       tol_ir=tol_ir)
    sp = S.uniaxial_bar(3, 4, Lx=0.5, Ly=1.0, lam=lam, mu=mu, Gc=Gc, l=l, eta=eta)
    g, m = _grid(sp), _mat(sp)
    a, kappa, gamma = model.at1_constants(m, tol_ir)
    eps_c = np.sqrt(2 * a / M)                    # Psi+ reaches a / 2 = 3 G_c / (16 l)
    # load past the elastic limit, unload, reload below the previous maximum
    ubars = np.concatenate([np.linspace(0.2, 2.0, 7), [1.5, 1.0, 1.8]]) * eps_c * sp.Ly
    st = stg.State(g)
    d_ref = 0.0
    for ub in ubars:
        r = stg.load_step(g, m, st, ub - st.ubar, scheme, opts, reaction_dir=1)
        assert r.converged
        eps = st.ubar / sp.Ly
        psi = 0.5 * M * eps ** 2
        d_new = _scalar_d(psi, d_ref, a, gamma)
        assert d_new >= d_ref - (8.0 / 9.0) * tol_ir ** 2 * (1 + 1e-12)
        d_ref = d_new
        assert np.allclose(st.d, d_ref, rtol=1e-8, atol=1e-11)
        F = ((1 - d_ref) ** 2 + eta) * M * eps * sp.Lx
        assert r.reaction == pytest.approx(F, rel=1e-8)
    # the softening branch was reached (d well above the penalty's O(tol_ir^2) range)
    assert d_ref > 0.3


def test_at1_profile_second_order():
    L, l = 1.0, 0.1
    errs = []
    for nx in (40, 80, 160):
        sp = S.strip_1d(nx, ny=2, L=L, l=l)
        g, m = _grid(sp), _mat(sp)
        # a tight irreversibility tolerance makes the penalised solution the d >= 0 one;
        # from the Dirichlet start the free boundary x = 2l advances a node per iteration
        opts = stg.Options(tol_d=1e-10, max_newton=400, model=model.AT1, tol_ir=1e-4)
        d0 = g.d_dirichlet_values().astype(float)
        d, _, it = stg.at1_newton(g, m, np.zeros((g.ne, 4)), d0, np.zeros(g.nn), opts)
        assert it < opts.max_newton
        s, _ = q1.gauss_points_unit()
        ej, ei = np.divmod(np.arange(g.ne), g.nx)
        xq = (ei[:, None] + s[None]) * g.hx
        exact = np.where(xq < 2 * l, (1.0 - xq / (2 * l)) ** 2, 0.0)
        err = q1.interp_qp(g, d) - exact
        errs.append(np.sqrt(np.sum(err ** 2) * q1.qp_weight(g) / (g.Lx * g.Ly)))
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert errs[-1] < 1e-4
    assert np.all(orders > 1.8), orders


@pytest.mark.parametrize("scheme", [model.S1, model.S2, model.S3])
def test_at1_fixed_stress_equals_standard_without_softening(scheme):
    sp = S.tensile(12, l=0.2, steps=3, u_max=6e-3)
    g, m = _grid(sp), _mat(sp)
    out = []
    for sch in (model.ST, scheme):
        opts = stg.Options(tol_st=1e-8, model=model.AT1, psi_crit=np.inf)
        res, st = stg.load_path(g, m, sp.increments, sch, opts, reaction_dir=1)
        out.append(([r.reaction for r in res], [r.stag_iters for r in res], st.d))
    (Fa, ka, da), (Fb, kb, db) = out
    assert Fa == Fb and ka == kb and np.array_equal(da, db)


@pytest.mark.parametrize("split", [model.VD, model.SPECTRAL])
@pytest.mark.parametrize("scheme", [model.ST, model.S1])
def test_at1_free_sided_bar_both_splits(split, scheme):
    # Free sides: the lateral strain follows from sigma_xx = 0 and, for the spectral split,
    # depends on d; the homogeneous state solves the scalar stationarity equation
    # -2 (1-d) Psi+(d) + a + gamma <d - d_{n-1}>_- = 0 at every step (below the elastic
    # limit Psi+ = a/2 the penalty holds d slightly below d_{n-1} = 0).  Past the limit the
    # AT1 bar softens at once and the homogeneous state is unstable under displacement
    # control: with the spectral split the checker localizes in the first damaging step
    # (a band with d = 1, also a solution), with VD it stays homogeneous for a few steps.
    # The path therefore stops below the limit for the spectral split and four steps past
    # it for VD.
    lam, mu, Gc, l, eta = 121.15, 80.77, 2.7e-3, 0.03, 1e-9
    from scipy.optimize import brentq
    u_max, steps = (1.8e-2, 12) if split == model.VD else (1.2e-2, 8)
    sp = S.uniaxial_stress_bar(3, 4, Lx=0.5, Ly=1.0, lam=lam, mu=mu, Gc=Gc, l=l, eta=eta,
                               steps=steps, u_max=u_max)
    g = _grid(sp)
    m = model.material_from_E_nu(sp.E, sp.nu, Gc, l, eta, sp.plane, split)
    a, _, gamma = model.at1_constants(m, 0.01)

    def psi_syy(d, eyy):
        gd = (1 - d) ** 2 + eta
        if split == model.SPECTRAL:
            exx = -gd * lam * eyy / (gd * lam + 2 * mu)
            tr = exx + eyy
            return 0.5 * lam * tr ** 2 + mu * eyy ** 2, gd * (lam * tr + 2 * mu * eyy)
        exx = -lam * eyy / (lam + 2 * mu)
        tr = exx + eyy
        K = lam + 2 * mu / 3
        return (mu * (exx ** 2 + eyy ** 2 - tr ** 2 / 3) + 0.5 * K * tr ** 2,
                gd * (lam * tr + 2 * mu * eyy))

    opts = stg.Options(tol_st=1e-11, tol_nr=1e-11, max_stag=400, model=model.AT1, tol_ir=0.01)
    st = stg.State(g)
    d_prev = 0.0
    for du in sp.increments:
        r = stg.load_step(g, m, st, du, scheme, opts, reaction_dir=1)
        assert r.converged
        eyy = st.ubar / sp.Ly
        f = lambda d: (-2 * (1 - d) * psi_syy(d, eyy)[0] + a
                       + gamma * min(d - d_prev, 0.0))
        d_ex = brentq(f, -0.5, 1 - 1e-12, xtol=1e-15, rtol=1e-15)
        assert np.allclose(st.d, d_ex, rtol=1e-8, atol=1e-10)
        assert r.reaction == pytest.approx(psi_syy(d_ex, eyy)[1] * sp.Lx, rel=1e-7)
        d_prev = d_ex
    if split == model.VD:
        assert d_prev > 0.4                    # four damaging steps
    else:
        assert -1e-3 < d_prev < 0.0            # penalty branch just below the limit


def test_at1_stag_residual_on_one_element_by_hand():
    # AT1 staggered residual (Sec. 2 evolution equation, penalty irreversibility) on the
    # unit square, one element, mu = 1, lambda = 2, G_c = l = 1 (plane strain) and
    # u_x = x / 2: Psi+ = 1/2 at every point.  Then a = G_c/(c_w l) = 3/8,
    # kappa = 2 G_c l / c_w = 3/4, gamma = 27 G_c / (64 l tol_ir^2) = 4218.75 (tol_ir 0.01).
    # R_d = (M + kappa G) d + int (-2 Psi + a + gamma <d - d_{n-1}>_-) N with the Q1 mass
    # M = m1 (x) m1 and gradient matrix G = k1 (x) m1 + m1 (x) k1 of the unit square, so
    # M + 3/4 G has rows [11/18, -5/72, -5/72, -2/9] (and permutations); the Jacobian adds
    # gamma M where the penalty is active.
    g = q1.Grid(1, 1, 1.0, 1.0)
    m = model.Material(1.0, 2.0 + 2.0 / 3.0, 1.0, 1.0, 1e-9, 1.0 / 3.0)
    u = np.zeros(8)
    u[0::2] = 0.5 * np.array([0.0, 1.0, 0.0, 1.0])
    d = np.array([0.0, 0.2, 0.4, 0.6])
    opts = stg.Options(model=model.AT1, tol_ir=0.01)
    K = np.array([[11 / 18, -5 / 72, -5 / 72, -2 / 9],
                  [-5 / 72, 11 / 18, -2 / 9, -5 / 72],
                  [-5 / 72, -2 / 9, 11 / 18, -5 / 72],
                  [-2 / 9, -5 / 72, -5 / 72, 11 / 18]])
    # no penalty (d = d_{n-1}): source -1 + 3/8 = -5/8, integral -5/32 per node
    R = K @ d - 5.0 / 32.0
    assert stg.at1_stag_residual(g, m, u, d, d.copy(), opts) == pytest.approx(
        np.max(np.abs(R / (11 / 18))), rel=1e-12)
    assert np.max(np.abs(R / (11 / 18))) == pytest.approx(0.33125 * 18 / 11, rel=1e-12)
    # penalty everywhere (d_{n-1} = d + 0.1): source -5/8 - 0.1 gamma, Jacobian diagonal
    # (1 + gamma) 4/36 + 3/4 * 4/6
    gamma = 27.0 / (64.0 * 1e-4)
    R = K @ d + (-5.0 / 8.0 - 0.1 * gamma) / 4.0
    Jd = (1.0 + gamma) * 4.0 / 36.0 + 0.5
    assert stg.at1_stag_residual(g, m, u, d, d + 0.1, opts) == pytest.approx(
        np.max(np.abs(R / Jd)), rel=1e-12)
