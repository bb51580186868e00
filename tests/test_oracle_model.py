"""Pins of the checker's pointwise constitutive law against closed forms and calculus.

Each check is independent of how the oracle writes its formulas: energies against the
undamaged Hooke energy, stresses as numerical derivatives of the energy, the fixed-stress
relations against the stress law to first order in Delta d, and the scheme map against
Table 2 (tests/golden/table2_schemes.txt).
"""
import os

import numpy as np
import pytest

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHEMES = {"ST": model.ST, "S1": model.S1, "S2": model.S2, "S3": model.S3}


def _mat(plane=model.PLANE_STRAIN, eta=0.0):
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    return model.material_from_E_nu(E, nu, 2.7e-3, 0.03, eta, plane)


def _strains(n, seed, sign=None):
    r = np.random.default_rng(seed)
    e = r.standard_normal((3, n)) * 1e-3
    if sign is not None:
        tr = e[0] + e[1]
        flip = np.sign(tr) != sign
        e[0][flip] *= -1
        e[1][flip] *= -1
    return e


def test_table1_at2_constants():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_at_models.txt"))
            if l.strip() and not l.startswith("#")]
    at2 = [r for r in rows if r[0] == "AT2"][0]
    assert float(eval(at2[3])) == model.C_W_AT2
    m = _mat()
    assert m.psi_crit == pytest.approx(m.Gc / (2.0 * m.l), rel=1e-15)
    d = np.linspace(0, 1, 11)
    assert np.allclose(model.g(d, 1e-6), (1 - d) ** 2 + 1e-6, rtol=0, atol=0)


def test_lame_roundtrip_and_plane_strain_bulk():
    E, nu = model.E_nu_from_lame(121.15, 80.77)
    m = model.material_from_E_nu(E, nu, 1, 1, 0)
    assert m.mu == pytest.approx(80.77, rel=1e-14)
    assert m.K == pytest.approx(121.15 + 2 * 80.77 / 3, rel=1e-14)


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
def test_split_sums_to_hooke_energy(plane):
    """Psi+ + Psi- equals the undamaged elastic energy 1/2 sigma0 : eps."""
    m = _mat(plane)
    exx, eyy, exy = _strains(500, 1)
    if plane == model.PLANE_STRAIN:
        lam = m.K - 2 * m.mu / 3
        W = 0.5 * lam * (exx + eyy) ** 2 + m.mu * (exx ** 2 + eyy ** 2 + 2 * exy ** 2)
    else:
        E = 4 * m.mu * m.K / (m.mu + m.K)
        nu = (m.K - m.mu) / (m.K + m.mu)
        c = E / (1 - nu ** 2)
        sxx = c * (exx + nu * eyy)
        syy = c * (eyy + nu * exx)
        sxy = c * (1 - nu) * exy
        W = 0.5 * (sxx * exx + syy * eyy + 2 * sxy * exy)
    got = model.psi_plus(exx, eyy, exy, m) + model.psi_minus(exx, eyy, exy, m)
    assert np.allclose(got, W, rtol=1e-12, atol=0)


def test_plane_stress_reproduces_hooke_stress():
    m = _mat(model.PLANE_STRESS)
    E = 4 * m.mu * m.K / (m.mu + m.K)
    nu = (m.K - m.mu) / (m.K + m.mu)
    exx, eyy, exy = _strains(200, 2)
    sxx, syy, sxy = model.stress(exx, eyy, exy, np.zeros_like(exx), m)
    c = E / (1 - nu ** 2)
    assert np.allclose(sxx, c * (exx + nu * eyy), rtol=1e-12, atol=1e-18)
    assert np.allclose(syy, c * (eyy + nu * exx), rtol=1e-12, atol=1e-18)
    assert np.allclose(sxy, c * (1 - nu) * exy, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
def test_stress_is_energy_derivative(plane):
    """sigma = d/d eps [g Psi+ + Psi-] by central differences (exy counted twice)."""
    m = _mat(plane, eta=1e-3)
    r = np.random.default_rng(3)
    exx, eyy, exy = _strains(300, 4)
    d = r.random(300) * 0.9
    keep = np.abs(exx + eyy) > 1e-5
    exx, eyy, exy, d = exx[keep], eyy[keep], exy[keep], d[keep]

    def W(a, b, c):
        return model.g(d, m.eta) * model.psi_plus(a, b, c, m) + model.psi_minus(a, b, c, m)

    h = 1e-8
    dxx = (W(exx + h, eyy, exy) - W(exx - h, eyy, exy)) / (2 * h)
    dyy = (W(exx, eyy + h, exy) - W(exx, eyy - h, exy)) / (2 * h)
    dxy = (W(exx, eyy, exy + h) - W(exx, eyy, exy - h)) / (2 * h)
    sxx, syy, sxy = model.stress(exx, eyy, exy, d, m)
    scale = np.max(np.abs(sxx))
    assert np.max(np.abs(dxx - sxx)) < 1e-6 * scale
    assert np.max(np.abs(dyy - syy)) < 1e-6 * scale
    assert np.max(np.abs(dxy - 2 * sxy)) < 1e-6 * scale


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_tangent_is_stress_derivative(sign):
    m = _mat(eta=1e-4)
    r = np.random.default_rng(5)
    exx, eyy, exy = _strains(100, 6, sign=sign)
    d = r.random(100) * 0.9
    ip = model.tension(exx, eyy)
    assert np.all(ip == (sign > 0))
    D = model.tangent_voigt(d, ip, m)
    h = 1e-9
    base = np.stack(model.stress(exx, eyy, exy, d, m), axis=1)
    for k, (a, b, c) in enumerate([(h, 0, 0), (0, h, 0), (0, 0, h / 2)]):
        pert = np.stack(model.stress(exx + a, eyy + b, exy + c, d, m), axis=1)
        col = (pert - base) / h
        assert np.allclose(col, D[:, :, k], rtol=1e-5, atol=1e-6 * np.abs(D).max())


def test_tension_indicator_is_strict():
    assert not model.tension(np.array([1.0]), np.array([-1.0]))[0]
    assert model.tension(np.array([1.0]), np.array([-0.5]))[0]


def test_activation_strict_inequalities():
    m = _mat()
    pc = m.psi_crit
    psi = np.array([pc, 2 * pc, 2 * pc, 2 * pc, 2 * pc])
    H = np.array([0.0, 2 * pc, 0.0, 0.0, 0.0])
    dq = np.array([0.0, 0.0, 0.95, 0.9499, 0.0])
    act = model.activation(psi, H, dq, m)
    assert act.tolist() == [False, False, False, True, True]


def _table2():
    out = {}
    for line in open(os.path.join(GOLDEN, "table2_schemes.txt")):
        if line.strip() and not line.startswith("#"):
            name, i1, dev = line.split()
            out[SCHEMES[name]] = (bool(int(i1)), bool(int(dev)))
    return out


def _increment_for(scheme, exx, eyy, exy, d, dd, m):
    """A strain increment satisfying the scalar relations the scheme uses.

    Only the contractions tr(Delta eps) and eps_dev . Delta eps are prescribed by the
    relations; the increment is built in-plane from two directions (I and the in-plane
    part of eps_dev) to hit the prescribed values.
    """
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    want_tr = model.trace_increment(tr, d, dd, m) if scheme in (model.S1, model.S3) else None
    want_dev = model.dev_increment(ee, d, dd, m) if scheme in (model.S2, model.S3) else None
    # basis A = in-plane identity, B = in-plane part of eps_dev
    Bxx, Byy, Bxy = exx - m.cdim * tr, eyy - m.cdim * tr, exy
    # contractions: tr(A)=2, tr(B)=Bxx+Byy; dev.A = Bxx+Byy; dev.B = Bxx^2+Byy^2+2Bxy^2
    trA, trB = 2.0, Bxx + Byy
    dA, dB = Bxx + Byy, Bxx ** 2 + Byy ** 2 + 2 * Bxy ** 2
    if want_tr is not None and want_dev is not None:
        det = trA * dB - trB * dA
        a = (want_tr * dB - trB * want_dev) / det
        b = (trA * want_dev - dA * want_tr) / det
    elif want_tr is not None:
        a, b = want_tr / trA, 0.0 * want_tr
    else:
        a, b = 0.0 * want_dev, want_dev / dB
    return a + b * Bxx, a + b * Byy, b * Bxy


def _I1_and_dev(exx, eyy, exy, d, ref, m):
    sxx, syy, sxy = model.stress(exx, eyy, exy, d, m)
    szz = model.stress_zz(exx, eyy, d, m) if m.cdim < 0.4 else 0.0
    rxx, ryy, rxy = ref
    tr0 = rxx + ryy
    dev = sxx * (rxx - m.cdim * tr0) + syy * (ryy - m.cdim * tr0) + 2 * sxy * rxy
    if m.cdim < 0.4:
        dev = dev + szz * (-m.cdim * tr0)
    return sxx + syy + szz, dev


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
@pytest.mark.parametrize("name", ["S1", "S2", "S3"])
def test_fixed_stress_relations_first_order(plane, name):
    """Table 2: the scheme's relations keep the named stress quantities fixed to O(Dd^2).

    The stress increment is evaluated with the full nonlinear stress law at
    (d + Dd, eps + Deps) against (d, eps); quantities the scheme holds must change by
    O(Dd^2) (ratio / Dd -> 0 linearly); quantities it does not hold change at O(Dd).
    """
    scheme = SCHEMES[name]
    fix_i1, fix_dev = _table2()[scheme]
    m = _mat(plane, eta=1e-6)
    r = np.random.default_rng(7)
    exx, eyy, exy = _strains(64, 8, sign=1.0)
    d = r.random(64) * 0.8
    ref = (exx, eyy, exy)
    I0, D0 = _I1_and_dev(exx, eyy, exy, d, ref, m)
    errs = []
    for dd in (1e-3, 5e-4, 2.5e-4):
        ddv = np.full_like(d, dd)
        a, b, c = _increment_for(scheme, exx, eyy, exy, d, ddv, m)
        I1, D1 = _I1_and_dev(exx + a, eyy + b, exy + c, d + ddv, ref, m)
        errs.append((np.max(np.abs(I1 - I0) / np.abs(I0)), np.max(np.abs(D1 - D0) / np.abs(D0))))
    errs = np.array(errs)
    for col, fixed in ((0, fix_i1), (1, fix_dev)):
        e = errs[:, col]
        if fixed:
            # second order: halving Dd quarters the change
            assert e[0] < 1e-2
            assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5
        else:
            assert e[0] > 1e-4
            assert 1.8 < e[0] / e[1] < 2.2


@pytest.mark.parametrize("plane", [model.PLANE_STRAIN, model.PLANE_STRESS])
@pytest.mark.parametrize("name", ["S1", "S2", "S3"])
def test_extra_stiffness_is_tangent_of_prediction(plane, name):
    """K~_q = -2 (1-d) dPsi^{k+1/2}/dDd at Dd = 0+ (the coupling term of Sec. 3.3)."""
    scheme = SCHEMES[name]
    m = _mat(plane, eta=1e-6)
    r = np.random.default_rng(9)
    exx, eyy, exy = _strains(128, 10)
    d = r.random(128) * 0.9
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    h = 1e-7
    p0 = model.predict_psi(tr, ee, d, np.zeros_like(d), scheme, m)
    p1 = model.predict_psi(tr, ee, d, np.full_like(d, h), scheme, m)
    p2 = model.predict_psi(tr, ee, d, np.full_like(d, 2 * h), scheme, m)
    slope = (-3 * p0 + 4 * p1 - p2) / (2 * h)
    kt = model.extra_stiffness(tr, ee, d, scheme, m)
    assert np.allclose(kt, -2 * (1 - d) * slope, rtol=1e-6, atol=1e-9 * np.abs(kt).max())
    assert np.allclose(p0, model.psi_plus(exx, eyy, exy, m), rtol=1e-14)


@pytest.mark.parametrize("name", ["S1", "S2", "S3"])
def test_prediction_is_energy_of_updated_strain(name):
    """With 2D invariants the updated invariants belong to an explicit strain: scale the
    volumetric part (S1), the deviatoric part (S2) or all of it (S3) by s = 1 + a Dd.
    The prediction equals Psi+ of that strain, also for large Dd."""
    scheme = SCHEMES[name]
    m = _mat(model.PLANE_STRESS, eta=1e-6)
    r = np.random.default_rng(11)
    exx, eyy, exy = _strains(200, 12, sign=1.0)
    d = r.random(200) * 0.9
    dd = r.random(200) * 0.3
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    s = 1 + 2 * (1 - d) / ((1 - d) ** 2 + m.eta) * dd
    vol, dxx, dyy = tr / 2, exx - tr / 2, eyy - tr / 2
    sv = s if scheme in (model.S1, model.S3) else 1.0
    sd = s if scheme in (model.S2, model.S3) else 1.0
    hat = model.psi_plus(sv * vol + sd * dxx, sv * vol + sd * dyy, sd * exy, m)
    got = model.predict_psi(tr, ee, d, dd, scheme, m)
    assert np.allclose(got, hat, rtol=1e-12)
    # negative increments leave the energy unchanged (Delta d > 0 rule)
    same = model.predict_psi(tr, ee, d, -dd, scheme, m)
    assert np.allclose(same, model.psi_plus(exx, eyy, exy, m), rtol=1e-14)


def test_s3_prediction_scales_plane_strain_energy():
    m = _mat(model.PLANE_STRAIN, eta=1e-6)
    r = np.random.default_rng(13)
    exx, eyy, exy = _strains(100, 14, sign=1.0)
    d = r.random(100) * 0.9
    dd = r.random(100) * 0.2
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    s = 1 + 2 * (1 - d) / ((1 - d) ** 2 + m.eta) * dd
    got = model.predict_psi(tr, ee, d, dd, model.S3, m)
    assert np.allclose(got, model.psi_plus(s * exx, s * eyy, s * exy, m), rtol=1e-12)


def test_augmented_coefficient_floor():
    """Reading of the footnote of Sec. 3.3: K~ cancels at most the 2H part of the tangent."""
    m = _mat(eta=1e-9)
    r = np.random.default_rng(15)
    exx, eyy, exy = _strains(400, 16, sign=1.0)
    exx, eyy, exy = exx * 30, eyy * 30, exy * 30
    d = r.random(400) * 0.9
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    H = model.psi_plus(exx, eyy, exy, m)
    for s in (model.S1, model.S2, model.S3):
        kt = model.extra_stiffness(tr, ee, d, s, m)
        lit = model.augmented_coefficient(H, kt, m, floor=False)
        c = model.augmented_coefficient(H, kt, m)
        assert np.all(c >= m.Gc / m.l)
        assert np.any(lit < 0)                      # the unlimited form goes indefinite
        keep = lit >= m.Gc / m.l
        assert np.array_equal(c[keep], lit[keep])
