"""Pins of the checker's spectral energy split (the alternative split named in Sec. 2).

Independent of how the oracle writes its formulas: energies against the Hooke energy and
closed forms for strains of known principal values, invariance under rotation of the
strain, stresses as numerical derivatives of the energy, the tangent as the numerical
derivative of the stress, the fixed-stress rules against the paper's VD forms (for the VD
parts) and against the stress law in fully tensile states, and the staggered solution of
a homogeneous bar with free sides against its scalar closed form.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import specimens as S

LAM, MU = 121.15, 80.77
SCHEMES = (model.S1, model.S2, model.S3)


def _mat(plane=model.PLANE_STRAIN, eta=0.0, split=model.SPECTRAL):
    E, nu = model.E_nu_from_lame(LAM, MU)
    return model.material_from_E_nu(E, nu, 2.7e-3, 0.03, eta, plane, split)


def _strains(n, seed):
    return np.random.default_rng(seed).standard_normal((3, n)) * 1e-3


def _rotate(exx, eyy, exy, t):
    exx, eyy, exy, t = np.broadcast_arrays(exx, eyy, exy, t)
    c, s = np.cos(t), np.sin(t)
    R = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)
    e = np.stack([np.stack([exx, exy], -1), np.stack([exy, eyy], -1)], -2)
    r = np.einsum('...ij,...jk,...lk->...il', R, e, R)
    return r[..., 0, 0], r[..., 1, 1], r[..., 0, 1]


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
def test_split_sums_to_hooke_energy(plane):
    m = _mat(plane)
    exx, eyy, exy = _strains(400, 1)
    E, nu = model.E_nu_from_lame(LAM, MU)
    lam = LAM if plane == model.PLANE_STRAIN else E * nu / (1 - nu ** 2)
    W = 0.5 * lam * (exx + eyy) ** 2 + MU * (exx ** 2 + eyy ** 2 + 2 * exy ** 2)
    got = model.psi_plus(exx, eyy, exy, m) + model.psi_minus(exx, eyy, exy, m)
    assert np.allclose(got, W, rtol=1e-12, atol=0)


def test_closed_forms():
    m = _mat()
    t = np.linspace(0.0, np.pi, 7)
    for e in (1e-3, -1e-3):
        # uniaxial strain e along n = (cos t, sin t): Psi+ = (lam/2 + mu) e^2 or 0
        exx, eyy, exy = e * np.cos(t) ** 2, e * np.sin(t) ** 2, e * np.sin(t) * np.cos(t)
        want = (0.5 * LAM + MU) * e * e if e > 0 else 0.0
        assert np.allclose(model.psi_plus(exx, eyy, exy, m), want, rtol=1e-12, atol=1e-20)
    # pure shear: principal strains +-gamma/2, tr = 0: Psi+ = Psi- = mu gamma^2 / 4
    gam = 2e-3
    assert model.psi_plus(0.0, 0.0, gam / 2, m) == pytest.approx(MU * gam ** 2 / 4, rel=1e-12)
    assert model.psi_minus(0.0, 0.0, gam / 2, m) == pytest.approx(MU * gam ** 2 / 4, rel=1e-12)
    # equibiaxial: all of the energy is active in tension, none in compression
    assert model.psi_plus(1e-3, 1e-3, 0.0, m) == pytest.approx((2 * LAM + 2 * MU) * 1e-6,
                                                               rel=1e-12)
    assert model.psi_plus(-1e-3, -1e-3, 0.0, m) == 0.0
    # the VD split keeps the whole deviatoric energy of a pure shear active
    vd = _mat(split=model.VD)
    assert model.psi_plus(0.0, 0.0, gam / 2, vd) == pytest.approx(MU * gam ** 2 / 2, rel=1e-12)


def test_rotation_invariance():
    m = _mat()
    exx, eyy, exy = _strains(300, 2)
    for t in (0.3, 1.1, 2.5):
        a = _rotate(exx, eyy, exy, t)
        assert np.allclose(model.psi_plus(*a, m), model.psi_plus(exx, eyy, exy, m),
                           rtol=1e-11, atol=1e-22)
        assert np.allclose(model.psi_minus(*a, m), model.psi_minus(exx, eyy, exy, m),
                           rtol=1e-11, atol=1e-22)


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
def test_stress_is_energy_derivative(plane):
    m = _mat(plane, eta=1e-3)
    r = np.random.default_rng(3)
    exx, eyy, exy = _strains(300, 4)
    d = r.random(300) * 0.9

    def W(a, b, c):
        return model.g(d, m.eta) * model.psi_plus(a, b, c, m) + model.psi_minus(a, b, c, m)

    h = 1e-9
    dxx = (W(exx + h, eyy, exy) - W(exx - h, eyy, exy)) / (2 * h)
    dyy = (W(exx, eyy + h, exy) - W(exx, eyy - h, exy)) / (2 * h)
    dxy = (W(exx, eyy, exy + h) - W(exx, eyy, exy - h)) / (2 * h)
    sxx, syy, sxy = model.stress(exx, eyy, exy, d, m)
    scale = np.max(np.abs(sxx))
    assert np.max(np.abs(dxx - sxx)) < 1e-6 * scale
    assert np.max(np.abs(dyy - syy)) < 1e-6 * scale
    assert np.max(np.abs(dxy - 2 * sxy)) < 1e-6 * scale


def test_tangent_is_stress_derivative():
    m = _mat(eta=1e-4)
    r = np.random.default_rng(5)
    exx, eyy, exy = _strains(400, 6)
    d = r.random(400) * 0.9
    e1, e2, _, _ = model.principal(exx, eyy, exy)
    keep = (np.abs(e1) > 2e-5) & (np.abs(e2) > 2e-5) & (np.abs(exx + eyy) > 2e-5)
    exx, eyy, exy, d = exx[keep], eyy[keep], exy[keep], d[keep]
    D = model.tangent_spectral(exx, eyy, exy, d, m)
    assert np.allclose(D, np.swapaxes(D, -1, -2), rtol=1e-12, atol=1e-12)
    h = 1e-10
    for k, (a, b, c) in enumerate([(h, 0, 0), (0, h, 0), (0, 0, h / 2)]):
        plus = np.stack(model.stress(exx + a, eyy + b, exy + c, d, m), axis=1)
        minus = np.stack(model.stress(exx - a, eyy - b, exy - c, d, m), axis=1)
        col = (plus - minus) / (2 * h)
        assert np.allclose(col, D[:, :, k], rtol=1e-5, atol=1e-6 * np.abs(D).max())


def test_tangent_equal_principal_strains():
    # e1 = e2: the tangent is g C in tension and C in compression (no direction needed)
    m = _mat(eta=1e-4)
    d = np.array([0.4])
    gd = model.g(d, m.eta)[0]
    C = np.array([[LAM + 2 * MU, LAM, 0], [LAM, LAM + 2 * MU, 0], [0, 0, MU]])
    assert np.allclose(model.tangent_spectral(1e-3, 1e-3, 0.0, d, m)[0], gd * C, rtol=1e-12)
    assert np.allclose(model.tangent_spectral(-1e-3, -1e-3, 0.0, d, m)[0], C, rtol=1e-12)


def test_vd_parts_give_the_paper_forms():
    # the parts rule reproduces the VD forms printed after Table 2 and the VD prediction
    m = _mat(eta=1e-6, split=model.VD)
    r = np.random.default_rng(7)
    exx, eyy, exy = _strains(300, 8)
    d = r.random(300) * 0.9
    dd = r.standard_normal(300) * 0.1
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    pa, pb = model.psi_parts(exx, eyy, exy, m)
    assert np.allclose(pa + pb, model.psi_plus(exx, eyy, exy, m), rtol=1e-14)
    for s in SCHEMES:
        assert np.allclose(model.extra_stiffness_parts(pa, pb, d, s, m),
                           model.extra_stiffness(tr, ee, d, s, m), rtol=1e-14, atol=0)
        assert np.allclose(model.predict_psi_parts(pa, pb, d, dd, s, m),
                           model.predict_psi(tr, ee, d, dd, s, m), rtol=1e-12, atol=0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_extra_stiffness_is_tangent_of_prediction(scheme):
    m = _mat(eta=1e-6)
    r = np.random.default_rng(9)
    exx, eyy, exy = _strains(128, 10)
    d = r.random(128) * 0.9
    pa, pb = model.psi_parts(exx, eyy, exy, m)
    h = 1e-7
    p = [model.predict_psi_parts(pa, pb, d, np.full_like(d, k * h), scheme, m) for k in range(3)]
    slope = (-3 * p[0] + 4 * p[1] - p[2]) / (2 * h)
    kt = model.extra_stiffness_parts(pa, pb, d, scheme, m)
    assert np.allclose(kt, -2 * (1 - d) * slope, rtol=1e-6, atol=1e-9 * np.abs(kt).max())
    assert np.allclose(p[0], model.psi_plus(exx, eyy, exy, m), rtol=1e-14)
    # negative increments leave the energy unchanged (Delta d > 0 rule of Sec. 3.5)
    assert np.allclose(model.predict_psi_parts(pa, pb, d, -np.ones_like(d), scheme, m), p[0],
                       rtol=1e-14)


def test_s3_prediction_holds_the_stress_in_tension():
    # all principal strains positive: sigma = g (lam tr I + 2 mu eps) is g times a linear
    # map, so the strain that keeps sigma fixed as d -> d + Dd is eps g(d)/g(d + Dd); the
    # S3 prediction is its energy to first order in Dd (error ratio 4 on halving Dd)
    m = _mat(eta=1e-6)
    r = np.random.default_rng(11)
    a = np.abs(r.standard_normal((2, 50))) * 1e-3 + 1e-4
    t = r.random(50) * np.pi
    exx, eyy, exy = _rotate(a[0], a[1], 0.0 * a[0], t)
    d = r.random(50) * 0.8
    pa, pb = model.psi_parts(exx, eyy, exy, m)
    errs = []
    for dd in (1e-3, 5e-4):
        k = model.g(d, m.eta) / model.g(d + dd, m.eta)
        exact = model.psi_plus(k * exx, k * eyy, k * exy, m)
        pred = model.predict_psi_parts(pa, pb, d, np.full_like(d, dd), model.S3, m)
        errs.append(np.abs(pred - exact) / exact)
    ratio = errs[0] / errs[1]
    assert np.all((ratio > 3.5) & (ratio < 4.5)), ratio


def _bar_closed_form(split, eyy, Gc, l, eta, plane=model.PLANE_STRAIN):
    """Homogeneous bar with free sides at axial strain eyy (AT2, monotone): (d, sigma_yy)
    from sigma_xx = 0 and d = 2 Psi+ / (G_c/l + 2 Psi+).  Plane strain: Lame constant
    LAM, 3D bulk modulus; plane stress: lam* = E nu / (1 - nu^2), K2 = E / (2 (1 - nu))
    (2D invariants)."""
    E, nu = model.E_nu_from_lame(LAM, MU)
    if plane == model.PLANE_STRAIN:
        lam, K, c = LAM, LAM + 2 * MU / 3, 1.0 / 3.0
    else:
        lam, K, c = E * nu / (1 - nu ** 2), E / (2 * (1 - nu)), 0.5

    def state(d):
        gd = (1 - d) ** 2 + eta
        if split == model.SPECTRAL:
            exx = -gd * lam * eyy / (gd * lam + 2 * MU)
            tr = exx + eyy
            psi = 0.5 * lam * tr ** 2 + MU * eyy ** 2
            syy = gd * (lam * tr + 2 * MU * eyy)
        else:
            # sigma_xx = g [2 mu (e_xx - c tr) + K tr] = 0
            exx = -(K - 2 * MU * c) * eyy / (2 * MU * (1 - c) + K)
            tr = exx + eyy
            psi = MU * (exx ** 2 + eyy ** 2 - c * tr ** 2) + 0.5 * K * tr ** 2
            syy = gd * (2 * MU * (eyy - c * tr) + K * tr)
        return psi, syy

    f = lambda d: d * (Gc / l + 2 * state(d)[0]) - 2 * state(d)[0]
    d = brentq(f, 0.0, 1.0 - 1e-12, xtol=1e-15, rtol=1e-15)
    return d, state(d)[1]


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
@pytest.mark.parametrize("split", [model.VD, model.SPECTRAL])
@pytest.mark.parametrize("scheme", [model.ST, model.S1, model.S2, model.S3])
def test_free_sided_bar_closed_form(split, scheme, plane):
    Gc, l, eta = 2.7e-3, 0.03, 1e-9
    sp = S.uniaxial_stress_bar(3, 4, Lx=0.5, Ly=1.0, Gc=Gc, l=l, eta=eta, steps=5,
                               u_max=1.1e-2)
    sp.plane = plane
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, Gc, l, eta, sp.plane, split)
    st = stg.State(g)
    opts = stg.Options(tol_st=1e-11, tol_nr=1e-11, max_stag=400)
    for du in sp.increments:
        r = stg.load_step(g, m, st, du, scheme, opts, reaction_dir=1)
        assert r.converged
        d_ex, syy = _bar_closed_form(split, st.ubar / sp.Ly, Gc, l, eta, plane)
        assert np.allclose(st.d, d_ex, rtol=1e-8, atol=1e-10)
        assert r.reaction == pytest.approx(syy * sp.Lx, rel=1e-7)
    # the path ends just before the peak of the homogeneous response (past it, under
    # displacement control, the staggered iteration may find a localized solution)
    assert st.d.min() > 0.2
