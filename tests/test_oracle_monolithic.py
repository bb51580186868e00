"""Pins of the checker's monolithic Newton (the coupled system of Sec. 3.2).

The full Jacobian is checked against central differences of the residual (both energy
splits, with points where the history grows and where it does not); the monolithic solution
of the homogeneous bar against its closed form across the peak; and on the notched square
the monolithic solution against the staggered fixed point (TOL_ST -> 0), for both splits.
"""
import numpy as np
import pytest

from oracle import model, monolithic as mono, q1, staggered as stg
from paper_2209_07969_gb300 import specimens as S

SPLITS = [model.VD, model.SPECTRAL]


def _setup(sp, split, eta=None):
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta if eta is None else eta,
                                 sp.plane, split)
    return g, m


@pytest.mark.parametrize("split", SPLITS)
def test_stress_plus_is_energy_derivative(split):
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 2.7e-3, 0.03, 0.0, model.PLANE_STRAIN, split)
    exx, eyy, exy = np.random.default_rng(2).standard_normal((3, 300)) * 1e-3
    h = 1e-9
    P = lambda a, b, c: model.psi_plus(a, b, c, m)
    fd = ((P(exx + h, eyy, exy) - P(exx - h, eyy, exy)) / (2 * h),
          (P(exx, eyy + h, exy) - P(exx, eyy - h, exy)) / (2 * h),
          (P(exx, eyy, exy + h) - P(exx, eyy, exy - h)) / (4 * h))
    got = model.stress_plus(exx, eyy, exy, m)
    scale = np.max(np.abs(got[0]))
    for a, b in zip(got, fd):
        assert np.max(np.abs(a - b)) < 1e-6 * scale


@pytest.mark.parametrize("split", SPLITS)
def test_jacobian_is_residual_derivative(split):
    sp = S.tensile(6, l=0.2)
    g, m = _setup(sp, split, eta=1e-3)
    u, d, _ = S.random_state(sp, 4)
    exx, eyy, exy = q1.strains_qp(g, u)
    psi = model.psi_plus(exx, eyy, exy, m)
    pick = np.random.default_rng(5).random(psi.shape) < 0.5
    H_prev = np.where(pick, 0.5 * psi, 2.0 * psi)        # history grows at about half the points
    J = mono.jacobian(g, m, u, d, H_prev)
    r = np.random.default_rng(6)
    for _ in range(3):
        vu = r.standard_normal(2 * g.nn) * 1e-3 * np.abs(u).max()
        vd = r.standard_normal(g.nn) * 1e-3
        h = 1e-4
        Rp = np.concatenate(mono.residual(g, m, u + h * vu, d + h * vd, H_prev)[:2])
        Rm = np.concatenate(mono.residual(g, m, u - h * vu, d - h * vd, H_prev)[:2])
        fd = (Rp - Rm) / (2 * h)
        Jv = J @ np.concatenate([vu, vd])
        assert np.linalg.norm(Jv - fd) <= 1e-6 * np.linalg.norm(Jv)
        # both coupling blocks take part
        nu_ = 2 * g.nn
        assert np.linalg.norm(J[:nu_, nu_:] @ vd) > 1e-3 * np.linalg.norm(Jv[:nu_])
        assert np.linalg.norm(J[nu_:, :nu_] @ vu) > 1e-3 * np.linalg.norm(Jv[nu_:])


def test_uniaxial_bar_closed_form_before_the_peak():
    # Past the peak plain Newton on the coupled system cycles at the kink of
    # max(H_{n-1}, Psi+) and through the non-convex energy (the reason the paper's schemes
    # are staggered); the comparator is a reference for converged states, used pre-peak.
    lam, mu, Gc, l, eta = 121.15, 80.77, 2.7e-3, 0.03, 1e-9
    M = lam + 2 * mu
    eps_c = np.sqrt(Gc / (3 * M * l))
    sp = S.uniaxial_bar(3, 4, Lx=0.5, Ly=1.0, lam=lam, mu=mu, Gc=Gc, l=l, eta=eta, steps=5,
                        u_max=0.95 * eps_c)
    g, m = _setup(sp, model.VD)
    st = stg.State(g)
    H = 0.0
    for du in sp.increments:
        r = mono.load_step(g, m, st, du, tol_nr=1e-10, tol_st=1e-12, reaction_dir=1)
        assert r.converged and r.newton <= 8
        eps = st.ubar / sp.Ly
        H = max(H, 0.5 * M * eps ** 2)
        dex = 2 * H / (Gc / l + 2 * H)
        assert np.allclose(st.d, dex, rtol=1e-9, atol=1e-12)
        assert r.reaction == pytest.approx(((1 - dex) ** 2 + eta) * M * eps * sp.Lx, rel=1e-9)
    assert st.d.min() > 0.1


@pytest.mark.parametrize("split", SPLITS)
def test_equals_the_staggered_fixed_point(split):
    sp = S.tensile(16, l=0.1, steps=6, u_max=6e-3)
    g, m = _setup(sp, split)
    a, b = stg.State(g), stg.State(g)
    for du in sp.increments[:3]:
        rm = mono.load_step(g, m, a, du, tol_nr=1e-11, tol_st=1e-12)
        rs = stg.load_step(g, m, b, du, 1, stg.Options(tol_nr=1e-11, tol_st=1e-12), 1)
        assert rm.converged and rs.converged
        assert rm.newton < rs.newton_u      # coupled Newton needs fewer linear solves
        assert np.max(np.abs(a.d - b.d)) < 1e-9
        assert rm.reaction == pytest.approx(rs.reaction, rel=1e-9)
