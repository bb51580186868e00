"""Pointwise constitutive law of the phase-field model (oracle; test infrastructure only).

All functions are vectorised over numpy arrays and work in float64.  Strains are given
by their in-plane tensor components (exx, eyy, exy) -- exy is the tensor shear, half
the engineering shear.  The out-of-plane strain is zero (plane strain, Sec. 4 intro:
one element thick, thickness-direction motion suppressed).

Invariants.  With ``cdim`` the deviatoric factor (1/3 for plane strain, where the 3D
deviator of a tensor with ezz = 0 is used; 1/2 for the 2D-invariant plane-stress
variant) and ``tr = exx + eyy``::

    e.e = exx^2 + eyy^2 + 2 exy^2 - cdim * tr^2      (eps_dev : eps_dev)

Energy split (Sec. 2, volumetric/deviatoric split; the paper prints the symbol Psi^+
twice, the second one is the inactive part Psi^-)::

    Psi+ = mu e.e + (K/2) <tr>_+^2 ,   Psi- = (K/2) <tr>_-^2

Degraded stress (Sec. 2, constitutive equation for sigma)::

    sigma = g(d) [2 mu eps_dev + K <tr>_+ I] + K <tr>_- I

AT2 model (Table 1): g(d) = (1-d)^2 + eta, w(d) = d^2, c_w = 2 (history field).
AT1 model (Table 1): same g, w(d) = d, c_w = 8/3, irreversibility by the penalty term of
the evolution equation (Sec. 2, penalty parameter gamma = 27 G_c / (64 l tol_ir^2)).

Spectral split (the alternative split that Sec. 2 names; the paper runs the VD split).
With lam = K - 2 mu cdim (the Lame constant of the plane mode: lambda in plane strain,
E nu / (1 - nu^2) in plane stress) and e1 >= e2 the in-plane principal strains (the
out-of-plane principal strain of plane strain is 0 and adds nothing)::

    Psi+ = (lam/2) <tr>_+^2 + mu (<e1>_+^2 + <e2>_+^2)
    Psi- = (lam/2) <tr>_-^2 + mu (<e1>_-^2 + <e2>_-^2)
    sigma = g(d) [lam <tr>_+ I + 2 mu eps+] + lam <tr>_- I + 2 mu eps-,
    eps+- = sum_i <e_i>_+- n_i (x) n_i

Both splits write Psi+ = Psi_a + Psi_b with a trace part Psi_a (VD: K/2 <tr>_+^2; spectral:
lam/2 <tr>_+^2) and a second part Psi_b (VD: mu e.e; spectral: mu sum <e_i>_+^2).  The
fixed-stress schemes act on these parts (``psi_parts``, ``extra_stiffness_parts``,
``predict_psi_parts``).
"""
import numpy as np

PLANE_STRAIN = 0
PLANE_STRESS = 1

C_W_AT2 = 2.0  # Table 1, AT2 row
VD, SPECTRAL = 0, 1  # energy splits (Sec. 2)


class Material:
    """Material constants in the paper's notation.

    ``mu`` shear modulus, ``K`` bulk modulus (the paper's k, Sec. 2), ``Gc`` critical
    energy release rate, ``l`` length scale, ``eta`` residual stiffness in g(d)
    (Table 1), ``cdim`` deviatoric factor (see module docstring).
    """

    def __init__(self, mu, K, Gc, l, eta, cdim, split=VD):
        self.mu = float(mu)
        self.K = float(K)
        self.Gc = float(Gc)
        self.l = float(l)
        self.eta = float(eta)
        self.cdim = float(cdim)
        self.split = int(split)

    @property
    def lam(self):
        """Lame constant of the plane mode, K - 2 mu cdim."""
        return self.K - 2.0 * self.mu * self.cdim

    @property
    def psi_crit(self):
        """Psi_crit = G_c / (c_w l), Sec. 3.5 (activation condition), AT2 c_w = 2."""
        return self.Gc / (C_W_AT2 * self.l)


def material_from_E_nu(E, nu, Gc, l, eta, plane=PLANE_STRAIN, split=VD):
    """Lame constants from (E, nu); bulk modulus K per plane mode.

    Plane strain keeps the 3D bulk modulus K = lambda + 2 mu / 3.  Plane stress uses
    2D invariants with K = E / (2 (1 - nu)), which reproduces the plane-stress Hooke
    law for an undamaged solid (2 mu eps + (K - mu) tr I).
    """
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    if plane == PLANE_STRAIN:
        return Material(mu, lam + 2.0 * mu / 3.0, Gc, l, eta, 1.0 / 3.0, split)
    return Material(mu, E / (2.0 * (1.0 - nu)), Gc, l, eta, 0.5, split)


def E_nu_from_lame(lam, mu):
    """Inverse of the Lame relations: E = mu (3 lam + 2 mu)/(lam + mu), nu = lam/(2(lam+mu))."""
    return mu * (3.0 * lam + 2.0 * mu) / (lam + mu), lam / (2.0 * (lam + mu))


def g(d, eta):
    """Degradation function g(d) = (1-d)^2 + eta (Table 1)."""
    return (1.0 - d) ** 2 + eta


def dg(d):
    """dg/dd = -2 (1-d)."""
    return -2.0 * (1.0 - d)


def pos(x):
    """<x>_+ = (x + |x|)/2 (Sec. 2)."""
    return 0.5 * (x + np.abs(x))


def neg(x):
    """<x>_- = (x - |x|)/2 (Sec. 2)."""
    return 0.5 * (x - np.abs(x))


def invariants(exx, eyy, exy, cdim):
    """Return (tr eps, eps_dev : eps_dev)."""
    tr = exx + eyy
    ee = exx * exx + eyy * eyy + 2.0 * exy * exy - cdim * tr * tr
    return tr, ee


def principal(exx, eyy, exy):
    """In-plane principal strains e1 >= e2 and (cos 2t, sin 2t) of the direction n1 =
    (cos t, sin t) of e1, from the eigenvalue problem of the symmetric 2 x 2 strain.
    Where e1 = e2 the direction is arbitrary and (1, 0) is returned."""
    exx, eyy, exy = np.broadcast_arrays(*(np.asarray(a, dtype=float) for a in (exx, eyy, exy)))
    mean = 0.5 * (exx + eyy)
    half = 0.5 * (exx - eyy)
    R = np.hypot(half, exy)
    safe = np.where(R > 0.0, R, 1.0)
    c2 = np.where(R > 0.0, half / safe, 1.0)
    s2 = np.where(R > 0.0, exy / safe, 0.0)
    return mean + R, mean - R, c2, s2


def psi_parts(exx, eyy, exy, m):
    """(Psi_a, Psi_b): trace part and second part of Psi+ for the material's split."""
    tr = exx + eyy
    if m.split == SPECTRAL:
        e1, e2, _, _ = principal(exx, eyy, exy)
        return 0.5 * m.lam * pos(tr) ** 2, m.mu * (pos(e1) ** 2 + pos(e2) ** 2)
    _, ee = invariants(exx, eyy, exy, m.cdim)
    return 0.5 * m.K * pos(tr) ** 2, m.mu * ee


def psi_plus(exx, eyy, exy, m):
    """Active strain energy (Sec. 2): VD Psi+ = mu e.e + K/2 <tr>_+^2; spectral split as in
    the module docstring."""
    if m.split == SPECTRAL:
        a, b = psi_parts(exx, eyy, exy, m)
        return a + b
    tr, ee = invariants(exx, eyy, exy, m.cdim)
    return m.mu * ee + 0.5 * m.K * pos(tr) ** 2


def psi_minus(exx, eyy, exy, m):
    """Inactive strain energy: VD Psi- = K/2 <tr>_-^2 (Sec. 2); spectral split as in the
    module docstring."""
    tr, _ = invariants(exx, eyy, exy, m.cdim)
    if m.split == SPECTRAL:
        e1, e2, _, _ = principal(exx, eyy, exy)
        return 0.5 * m.lam * neg(tr) ** 2 + m.mu * (neg(e1) ** 2 + neg(e2) ** 2)
    return 0.5 * m.K * neg(tr) ** 2


def _spectral_stress(exx, eyy, exy, d, m):
    tr = exx + eyy
    gd = g(d, m.eta)
    e1, e2, c2, s2 = principal(exx, eyy, exy)
    # n1 (x) n1 = [(1 + c2)/2, s2/2; s2/2, (1 - c2)/2], n2 (x) n2 = I - n1 (x) n1
    m1 = (0.5 * (1 + c2), 0.5 * (1 - c2), 0.5 * s2)
    m2 = (0.5 * (1 - c2), 0.5 * (1 + c2), -0.5 * s2)
    vol = m.lam * (gd * pos(tr) + neg(tr))
    w1 = 2.0 * m.mu * (gd * pos(e1) + neg(e1))
    w2 = 2.0 * m.mu * (gd * pos(e2) + neg(e2))
    sxx = vol + w1 * m1[0] + w2 * m2[0]
    syy = vol + w1 * m1[1] + w2 * m2[1]
    sxy = w1 * m1[2] + w2 * m2[2]
    return sxx, syy, sxy


def stress_plus(exx, eyy, exy, m):
    """Undegraded active stress sigma+ = d Psi+ / d eps (in-plane components): VD
    2 mu eps_dev + K <tr>_+ I; spectral lam <tr>_+ I + 2 mu eps+."""
    if m.split == SPECTRAL:
        tr = exx + eyy
        e1, e2, c2, s2 = principal(exx, eyy, exy)
        vol = m.lam * pos(tr)
        w1, w2 = 2.0 * m.mu * pos(e1), 2.0 * m.mu * pos(e2)
        return (vol + 0.5 * (w1 * (1 + c2) + w2 * (1 - c2)),
                vol + 0.5 * (w1 * (1 - c2) + w2 * (1 + c2)), 0.5 * s2 * (w1 - w2))
    tr = exx + eyy
    vol = m.K * pos(tr)
    return (2.0 * m.mu * (exx - m.cdim * tr) + vol, 2.0 * m.mu * (eyy - m.cdim * tr) + vol,
            2.0 * m.mu * exy)


def stress(exx, eyy, exy, d, m):
    """In-plane components (sxx, syy, sxy) of the degraded stress (Sec. 2)."""
    if m.split == SPECTRAL:
        return _spectral_stress(exx, eyy, exy, d, m)
    tr = exx + eyy
    gd = g(d, m.eta)
    vol = gd * m.K * pos(tr) + m.K * neg(tr)
    sxx = gd * 2.0 * m.mu * (exx - m.cdim * tr) + vol
    syy = gd * 2.0 * m.mu * (eyy - m.cdim * tr) + vol
    sxy = gd * 2.0 * m.mu * exy
    return sxx, syy, sxy


def stress_zz(exx, eyy, d, m):
    """Out-of-plane normal stress of the plane-strain state (ezz = 0), same law (Sec. 2).

    Only meaningful for the 3D-invariant (plane strain) mode; the weak form does not
    need it, the invariant checks of the fixed-stress relations do.
    """
    tr = exx + eyy
    gd = g(d, m.eta)
    if m.split == SPECTRAL:       # principal strain 0 along z: only the trace term
        return m.lam * (gd * pos(tr) + neg(tr))
    return gd * 2.0 * m.mu * (-m.cdim * tr) + gd * m.K * pos(tr) + m.K * neg(tr)


def tension(exx, eyy):
    """Sign indicator I_+ of Sec. 3.3: 1 where tr eps > 0 strictly, else 0."""
    return (exx + eyy) > 0.0


def tangent_voigt(d, ip, m):
    """Consistent tangent of the stress in Voigt form (xx, yy, engineering xy).

    For a frozen sign indicator ``ip`` the stress is linear in the strain; this is the
    bracket of the stress-increment equation in Sec. 3.3 (the part multiplying
    Delta eps).  Returns an array of shape d.shape + (3, 3).
    """
    gd = g(d, m.eta)
    kv = np.where(ip, gd * m.K, m.K)
    D = np.zeros(np.shape(d) + (3, 3))
    c = m.cdim
    two_mu_g = 2.0 * m.mu * gd
    D[..., 0, 0] = two_mu_g * (1.0 - c) + kv
    D[..., 1, 1] = two_mu_g * (1.0 - c) + kv
    D[..., 0, 1] = -two_mu_g * c + kv
    D[..., 1, 0] = -two_mu_g * c + kv
    D[..., 2, 2] = m.mu * gd  # sxy = g 2 mu exy = g mu gamma
    return D


def tangent_spectral(exx, eyy, exy, d, m):
    """Consistent tangent of the spectral-split stress in Voigt form (xx, yy, engineering
    xy) at the strain (exx, eyy, exy).

    d sigma = lam [g H(tr) + 1 - H(tr)] tr(d eps) I + 2 mu [g P+ + (I - P+)] d eps with
    H(x) = 1 for x > 0 (strict, as the VD indicator), and P+ = d eps+ / d eps, which in
    the principal frame keeps the normal components with weights H(e1), H(e2) and the
    shear component with the divided difference c12 = (<e1>_+ - <e2>_+)/(e1 - e2)
    (H(e1) where e1 = e2): the derivative of an isotropic tensor function of a
    symmetric 2 x 2 tensor.  Returns shape d.shape + (3, 3).
    """
    exx, eyy, exy, d = np.broadcast_arrays(*(np.asarray(a, dtype=float)
                                             for a in (exx, eyy, exy, d)))
    gd = g(d, m.eta)
    tr = exx + eyy
    e1, e2, c2, s2 = principal(exx, eyy, exy)
    h1 = (e1 > 0.0).astype(float)
    h2 = (e2 > 0.0).astype(float)
    gap = e1 - e2
    c12 = np.where(gap > 0.0, (pos(e1) - pos(e2)) / np.where(gap > 0.0, gap, 1.0), h1)
    # unit strain tensors of the three Voigt components (engineering shear)
    basis = [np.array([[1.0, 0.0], [0.0, 0.0]]), np.array([[0.0, 0.0], [0.0, 1.0]]),
             np.array([[0.0, 0.5], [0.5, 0.0]])]
    t = 0.5 * np.arctan2(s2, c2)                          # direction of e1
    n1 = np.stack([np.cos(t), np.sin(t)], axis=-1)
    n2 = np.stack([-np.sin(t), np.cos(t)], axis=-1)
    M1 = n1[..., :, None] * n1[..., None, :]
    M2 = n2[..., :, None] * n2[..., None, :]
    N12 = n1[..., :, None] * n2[..., None, :] + n2[..., :, None] * n1[..., None, :]
    kv = m.lam * np.where(tr > 0.0, gd, 1.0)
    D = np.zeros(np.shape(d) + (3, 3))
    for c, E in enumerate(basis):
        a1 = np.einsum('...ij,ij->...', M1, E)
        a2 = np.einsum('...ij,ij->...', M2, E)
        a12 = np.einsum('...i,ij,...j->...', n1, E, n2)
        Pp = (h1 * a1)[..., None, None] * M1 + (h2 * a2)[..., None, None] * M2 \
            + (c12 * a12)[..., None, None] * N12
        dsig = 2.0 * m.mu * ((gd - 1.0)[..., None, None] * Pp + E) \
            + (kv * np.trace(E))[..., None, None] * np.eye(2)
        D[..., 0, c] = dsig[..., 0, 0]
        D[..., 1, c] = dsig[..., 1, 1]
        D[..., 2, c] = dsig[..., 0, 1]
    return D


def tangent_at(exx, eyy, exy, d, m):
    """Newton tangent of the stress at the strain (exx, eyy, exy) for the material's split
    (VD: the frozen-indicator form ``tangent_voigt``)."""
    if m.split == SPECTRAL:
        return tangent_spectral(exx, eyy, exy, d, m)
    return tangent_voigt(d, tension(exx, eyy), m)


# --------------------------------------------------------------------------------------
# Fixed-stress schemes (Sec. 3.3-3.5)
# --------------------------------------------------------------------------------------
ST, S1, S2, S3 = 0, 1, 2, 3


def fixed_stress_Q(tr, ee, scheme, m):
    """Bracket of the extra stiffness K~^S (Sec. 3.4, three forms after Table 2).

    S1: K <tr>_+^2 ;  S2: 2 mu e.e ;  S3: 2 mu e.e + K <tr>_+^2 ;  ST: 0.
    """
    tp2 = m.K * pos(tr) ** 2
    dev = 2.0 * m.mu * ee
    if scheme == S1:
        return tp2
    if scheme == S2:
        return dev
    if scheme == S3:
        return dev + tp2
    return np.zeros_like(tr)


# ---- AT1 with penalty (Sec. 2, Table 1) -------------------------------------------------
AT2, AT1 = 0, 1
CW_AT1 = 8.0 / 3.0


def at1_constants(m, tol_ir):
    """(a, kappa, gamma) of the AT1 evolution equation (Sec. 2)

        -2 (1-d) Psi+ + a + gamma <d - d_{n-1}>_- - kappa lap d = 0,

    a = G_c / (c_w l) (the w'(d) = 1 term), kappa = 2 G_c l / c_w, gamma = 27 G_c /
    (64 l tol_ir^2).  a is also Psi_crit of the softening test for AT1 (Sec. 3.5)."""
    a = m.Gc / (CW_AT1 * m.l)
    kappa = 2.0 * m.Gc * m.l / CW_AT1
    gamma = 27.0 * m.Gc / (64.0 * m.l * tol_ir ** 2)
    return a, kappa, gamma


def at1_mass_coefficient(psi, d_q, dprev_q, gamma):
    """Per-point mass coefficient of the AT1 Jacobian: g''/2-term 2 Psi+ plus gamma where
    the penalty is active (d < d_{n-1}, strict)."""
    return 2.0 * psi + np.where(d_q < dprev_q, gamma, 0.0)


def at1_augmented_coefficient(c_J, k_extra, m, floor=True):
    """AT1 counterpart of ``augmented_coefficient``.  At activated points (K~ < 0) the
    augmented mass coefficient is limited below by 2 G_c / (c_w l), the expression that
    gives the AT2 limit G_c / l.  AT1 has no w'' term in its tangent (w = d), so without a
    positive limit K~ can remove the whole mass term and leave the pure gradient term,
    singular wherever no phase-field Dirichlet value anchors it (the homogeneous bar).
    Inactive points keep the Jacobian coefficient."""
    c = c_J + k_extra
    if not floor:
        return c
    lim = np.minimum(c_J, 2.0 * m.Gc / (CW_AT1 * m.l))
    return np.where(k_extra < 0.0, np.maximum(c, lim), c_J)


def activation(psi, H_prev, d_q, m, psi_crit=None):
    """Softening-region test of Sec. 3.5.

    Active where Psi+ > Psi_crit, Psi+ > Psi_max and phi < 0.95, all strict.  Psi_max
    is read as the quadrature point's history maximum from the last converged load
    step, and phi as the phase field interpolated to the point.
    """
    pc = m.psi_crit if psi_crit is None else psi_crit
    return (psi > pc) & (psi > H_prev) & (d_q < 0.95)


def extra_stiffness(tr, ee, d_q, scheme, m):
    """Per-point value of K~^S without the shape functions (Sec. 3.4).

    K~ = -4 (1-d)^2 / g(d) * Q_S, Q_S from ``fixed_stress_Q``.
    """
    return -4.0 * (1.0 - d_q) ** 2 / g(d_q, m.eta) * fixed_stress_Q(tr, ee, scheme, m)


def augmented_coefficient(H_k, k_extra, m, floor=True):
    """Per-point mass coefficient of the augmented d-tangent K_dd + K~^S (Sec. 3.4).

    The standard AT2 coefficient is G_c/l + 2H.  Adding K~ can make it negative: at an
    activated point the material is past its peak, the fixed-stress linearisation has
    no equilibrium and the augmented system turns indefinite and near-singular, so
    the exact first NR iterate explodes and the staggered iteration stagnates.  The
    footnote of Sec. 3.3 requires the d-subproblem to stay convex; the reading used
    here lets K~ cancel at most the history part 2H of the tangent, i.e. the
    coefficient never drops below the crack-surface term G_c/l.  ``floor=False``
    gives the unlimited form.
    """
    c = m.Gc / m.l + 2.0 * H_k + k_extra
    if floor:
        c = np.maximum(c, m.Gc / m.l)
    return c


def trace_increment(tr, d_q, dd_q, m):
    """tr Delta eps = 2(1-d)/g(d) <tr>_+ Delta d for Delta d > 0, else 0.

    First fixed-invariant relation (Sec. 3.3, from Delta sigma . I = 0) with the
    Delta d > 0 rule of Sec. 3.5.
    """
    a = 2.0 * (1.0 - d_q) / g(d_q, m.eta)
    return np.where(dd_q > 0.0, a * pos(tr) * dd_q, 0.0)


def dev_increment(ee, d_q, dd_q, m):
    """eps_dev . Delta eps = 2(1-d)/g(d) (eps_dev . eps_dev) Delta d for Delta d > 0, else 0.

    Second fixed-invariant relation (Sec. 3.3, from Delta sigma . eps_dev = 0) with the
    Delta d > 0 rule of Sec. 3.5.
    """
    a = 2.0 * (1.0 - d_q) / g(d_q, m.eta)
    return np.where(dd_q > 0.0, a * ee * dd_q, 0.0)


def predict_psi(tr, ee, d_q, dd_q, scheme, m):
    """Predicted active energy Psi+^{k+1/2} (Sec. 3.3) with the Delta d > 0 rule (Sec. 3.5).

    The increments from the fixed-invariant relations are
        tr Delta eps        = a <tr>_+ Delta d        (first relation, used by S1, S3)
        eps_dev . Delta eps = a (e.e) Delta d        (second relation, used by S2, S3)
    with a = 2(1-d)/g(d), both set to zero unless Delta d > 0.  The updated invariants
    are  <tr>_+^{k+1/2} = <tr>_+ (1 + a Delta d)  and
        e.e^{k+1/2} = e.e + 4 e.e [ (1-d)/g Delta d + (1-d)^2/g^2 Delta d^2 ],
    i.e. e.e times (1 + a Delta d)^2.  The scheme picks which invariant is updated.
    """
    tp = pos(tr)
    if scheme in (S1, S3):
        tp_new = tp + trace_increment(tr, d_q, dd_q, m)
    else:
        tp_new = tp
    if scheme in (S2, S3):
        r = (1.0 - d_q) / g(d_q, m.eta)
        ddp = np.where(dd_q > 0.0, dd_q, 0.0)
        ee_new = ee + 4.0 * ee * (r * ddp + r * r * ddp * ddp)
    else:
        ee_new = ee
    return m.mu * ee_new + 0.5 * m.K * tp_new ** 2


# ---- fixed-stress forms on the energy parts (both splits) ----------------------------------
def fixed_stress_Q_parts(pa, pb, scheme):
    """Q_S on the energy parts: S1 2 Psi_a, S2 2 Psi_b, S3 2 (Psi_a + Psi_b), ST 0.  With
    the VD parts these are the three forms after Table 2 (K <tr>_+^2, 2 mu e.e, sum); the
    spectral split takes the same rule (the paper derives the schemes for VD only)."""
    if scheme == S1:
        return 2.0 * pa
    if scheme == S2:
        return 2.0 * pb
    if scheme == S3:
        return 2.0 * (pa + pb)
    return np.zeros_like(pa)


def extra_stiffness_parts(pa, pb, d_q, scheme, m):
    """K~ = -4 (1-d)^2 / g(d) Q_S with Q_S from ``fixed_stress_Q_parts``."""
    return -4.0 * (1.0 - d_q) ** 2 / g(d_q, m.eta) * fixed_stress_Q_parts(pa, pb, scheme)


def predict_psi_parts(pa, pb, d_q, dd_q, scheme, m):
    """Predicted active energy on the parts: the part(s) the scheme fixes are scaled by
    s^2, s = 1 + 2(1-d)/g(d) max(Delta d, 0) -- the VD update of ``predict_psi``
    (<tr>_+ and e.e^(1/2) scaled by s), written for any split with trace and second part."""
    s = 1.0 + 2.0 * (1.0 - d_q) / g(d_q, m.eta) * np.where(dd_q > 0.0, dd_q, 0.0)
    sa = s if scheme in (S1, S3) else 1.0
    sb = s if scheme in (S2, S3) else 1.0
    return pa * sa * sa + pb * sb * sb
