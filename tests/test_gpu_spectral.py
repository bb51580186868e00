"""The spectral energy split on the GPU path against the FP64 checker.

Operator level (1e-10 relative in FP64): the internal force, the per-point Newton tangent
and the assembled-stencil tangent product of the spectral split on seeded crack-like states
of a ragged grid and of a masked one; for the VD split the per-point tangent equals the
frozen-indicator form and the stencil product equals the matrix-free operator.  Point
kernels: Psi+, the fixed-stress coefficient and the prediction on the spectral parts.
Paths: the free-sided bar against its closed form (every precision and preconditioner,
ST/S1/S3), and the notched tensile square through the crack against the checker.
"""
import numpy as np
import pytest
import torch
from scipy.optimize import brentq

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S
from tests.gpu_util import dev, host, masked_matrix, rel_err, setup, stream
from tests.test_gpu_solver import _d_rms

pytestmark = pytest.mark.gpu


def _cases():
    return [("tensile38", S.tensile(38, l=0.05)), ("lshape40", S.l_shape(40, l=30.0))]


@pytest.fixture(scope="module", params=["tensile38", "lshape40"])
def case(request, gpu):
    spec = dict(_cases())[request.param]
    g, m_vd, gm, gfull, mat, keep = setup(spec)
    mat.split = binding.SPLIT_SPECTRAL
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane,
                                 model.SPECTRAL)
    u, d, H = S.random_state(spec, seed=5)
    cd = g.d_constrained()
    d[cd] = g.d_dirichlet_values()[cd]
    return dict(spec=spec, g=g, m=m, m_vd=m_vd, gm=gm, gfull=gfull, mat=mat, keep=keep,
                u=u, d=d, H=H)


def _Dq_matrix(Dq, nq):
    D = Dq.reshape(6, nq)
    out = np.empty((nq, 3, 3))
    idx = [(0, 0, 0), (1, 0, 1), (2, 0, 2), (3, 1, 1), (4, 1, 2), (5, 2, 2)]
    for k, i, j in idx:
        out[:, i, j] = D[k]
        out[:, j, i] = D[k]
    return out


def test_force_tangent_and_stencil_product(case):
    L = binding.lib()
    g, m = case["g"], case["m"]
    u, d = case["u"], case["d"]
    u_d, d_d = dev(u), dev(d)
    F = torch.empty(2 * g.nn, dtype=torch.float64, device="cuda")
    binding.check(L.pf_op_elas_residual(case["gfull"], case["mat"], u_d.data_ptr(),
                                        d_d.data_ptr(), F.data_ptr(), None, stream()))
    dq = q1.interp_qp(g, d)
    assert rel_err(host(F), q1.internal_force(g, u, dq, m)) < 1e-10
    nq = 4 * g.ne
    Dq = torch.empty(6 * nq, dtype=torch.float64, device="cuda")
    binding.check(L.pf_op_elas_tangent_qp(case["gfull"], case["mat"], u_d.data_ptr(),
                                          d_d.data_ptr(), Dq.data_ptr(), stream()))
    exx, eyy, exy = q1.strains_qp(g, u)
    Dref = model.tangent_at(exx, eyy, exy, dq, m) * g.elem_active[:, None, None, None]
    got = _Dq_matrix(host(Dq), nq).reshape(g.ne, 4, 3, 3)
    assert np.max(np.abs(got - Dref)) <= 1e-10 * np.max(np.abs(Dref))
    K = masked_matrix(q1.assemble_elasticity_at(g, u, dq, m), g.u_constrained())
    x = np.random.default_rng(7).standard_normal(2 * g.nn) * (~g.u_constrained())
    ref = K @ x
    for dtype, tdt, tol in ((binding.F64, torch.float64, 1e-10), (binding.F32, torch.float32, 2e-5)):
        xd = dev(x, tdt)
        y = torch.empty(2 * g.nn, dtype=tdt, device="cuda")
        binding.check(L.pf_op_elas_apply_qp(case["gm"], dtype, Dq.data_ptr(), xd.data_ptr(),
                                            y.data_ptr(), stream()))
        assert rel_err(host(y), ref) < tol


def test_vd_tangent_qp_equals_the_matrix_free_operator(case):
    # the assembled path with the VD law reproduces the frozen-indicator operator
    L = binding.lib()
    g, m = case["g"], case["m_vd"]
    u, d = case["u"], case["d"]
    spec = case["spec"]
    mat = binding.material(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    u_d, d_d = dev(u), dev(d)
    nq = 4 * g.ne
    Dq = torch.empty(6 * nq, dtype=torch.float64, device="cuda")
    binding.check(L.pf_op_elas_tangent_qp(case["gfull"], mat, u_d.data_ptr(), d_d.data_ptr(),
                                          Dq.data_ptr(), stream()))
    exx, eyy, _ = q1.strains_qp(g, u)
    ip = model.tension(exx, eyy)
    Dref = model.tangent_voigt(q1.interp_qp(g, d), ip, m) * g.elem_active[:, None, None, None]
    got = _Dq_matrix(host(Dq), nq).reshape(g.ne, 4, 3, 3)
    assert np.max(np.abs(got - Dref)) <= 1e-12 * np.max(np.abs(Dref))
    tb = torch.tensor((ip * (1 << np.arange(4))).sum(axis=1).astype(np.uint8), device="cuda")
    x = dev(np.random.default_rng(8).standard_normal(2 * g.nn))
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    binding.check(L.pf_op_elas_apply(case["gm"], mat, binding.F64, d_d.data_ptr(),
                                     tb.data_ptr(), x.data_ptr(), y1.data_ptr(), stream()))
    binding.check(L.pf_op_elas_apply_qp(case["gm"], binding.F64, Dq.data_ptr(), x.data_ptr(),
                                        y2.data_ptr(), stream()))
    assert rel_err(host(y2), host(y1)) < 1e-12


def test_point_kernels(case):
    L = binding.lib()
    g, m = case["g"], case["m"]
    u, d, H = case["u"], case["d"], case["H"]
    spec = case["spec"]
    Hp = 0.05 * H
    u_d, d_d, H_d = dev(u), dev(d), dev(Hp.ravel())
    nq = 4 * g.ne
    psi = torch.empty(nq, dtype=torch.float64, device="cuda")
    Hout = torch.empty(nq, dtype=torch.float64, device="cuda")
    binding.check(L.pf_op_qp_energy(case["gfull"], case["mat"], u_d.data_ptr(), H_d.data_ptr(),
                                    psi.data_ptr(), Hout.data_ptr(), stream()))
    exx, eyy, exy = q1.strains_qp(g, u)
    live = g.elem_active[:, None].astype(bool)
    pref = np.where(live, model.psi_plus(exx, eyy, exy, m), 0.0)
    assert rel_err(host(psi), pref) < 1e-12
    assert rel_err(host(Hout), np.maximum(Hp, pref)) < 1e-12
    pa, pb = model.psi_parts(exx, eyy, exy, m)
    dq = q1.interp_qp(g, d)
    dd = np.random.default_rng(3).standard_normal(g.nn) * 0.05
    ddq = q1.interp_qp(g, dd)
    # threshold between two well-separated energies near the median (no point at a tie)
    v = np.sort(pref[np.broadcast_to(live, pref.shape)])
    k = len(v) // 2
    while v[k + 1] - v[k] < 1e-9 * v[k + 1]:
        k += 1
    pc = 0.5 * (v[k] + v[k + 1])
    for scheme in (1, 2, 3):
        c = torch.empty(nq, dtype=torch.float64, device="cuda")
        a = torch.empty(nq, dtype=torch.uint8, device="cuda")
        binding.check(L.pf_op_fs_coeff(case["gfull"], case["mat"], scheme, pc, u_d.data_ptr(),
                                       d_d.data_ptr(), H_d.data_ptr(), c.data_ptr(),
                                       a.data_ptr(), stream()))
        act = model.activation(pref, Hp, dq, m, pc) & live
        assert np.array_equal(host(a).reshape(-1, 4).astype(bool), act)
        assert act.sum() > 0
        Hk = np.maximum(Hp, pref)
        kx = model.extra_stiffness_parts(pa, pb, dq, scheme, m)
        cref = np.where(act, model.augmented_coefficient(Hk, kx, m), m.Gc / m.l + 2 * Hk)
        assert rel_err(host(c), cref) < 1e-12
        Hh = torch.empty(nq, dtype=torch.float64, device="cuda")
        binding.check(L.pf_op_fs_predict(case["gfull"], case["mat"], scheme, u_d.data_ptr(),
                                         d_d.data_ptr(), dev(dd).data_ptr(), H_d.data_ptr(),
                                         a.data_ptr(), Hh.data_ptr(), stream()))
        ph = np.where(act, model.predict_psi_parts(pa, pb, dq, ddq, scheme, m), pref)
        href = np.where(live, np.maximum(Hp, ph), Hp)
        assert rel_err(host(Hh), href) < 1e-12


LAM, MU = S.MIEHE_LAMBDA, S.MIEHE_MU


def _bar_closed_form(eyy, Gc, l, eta):
    """Homogeneous free-sided bar, spectral split: sigma_xx = 0 gives
    e_xx = -g lam e_yy / (g lam + 2 mu); d = 2 Psi+ / (G_c/l + 2 Psi+)."""
    def state(d):
        gd = (1 - d) ** 2 + eta
        exx = -gd * LAM * eyy / (gd * LAM + 2 * MU)
        tr = exx + eyy
        return 0.5 * LAM * tr ** 2 + MU * eyy ** 2, gd * (LAM * tr + 2 * MU * eyy)

    d = brentq(lambda d: d * (Gc / l + 2 * state(d)[0]) - 2 * state(d)[0], 0.0, 1.0 - 1e-12,
               xtol=1e-15, rtol=1e-15)
    return d, state(d)[1]


MODES = [(binding.FP64, binding.PRECOND_JACOBI), (binding.FP64, binding.PRECOND_GMG),
         (binding.FP32_IR, binding.PRECOND_GMG)]


@pytest.mark.parametrize("mode", MODES, ids=["fp64-jacobi", "fp64-gmg", "fp32ir-gmg"])
@pytest.mark.parametrize("scheme", [0, 1, 3])
def test_free_sided_bar_closed_form(gpu, scheme, mode):
    precision, precond = mode
    Gc, l, eta = 2.7e-3, 0.03, 1e-9
    spec = S.uniaxial_stress_bar(9, 12, Lx=0.5, Ly=1.0, Gc=Gc, l=l, eta=eta, steps=5,
                                 u_max=1.1e-2)
    sim = binding.Simulation(spec, precision=precision, precond=precond,
                             split=binding.SPLIT_SPECTRAL)
    sim.set_options(tol_lin=1e-12, max_stag=400)
    for du in spec.increments:
        r = sim.load_step(du, scheme, 1e-10)
        assert r["converged"] == 1
        d_ex, syy = _bar_closed_form(r["ubar"] / spec.Ly, Gc, l, eta)
        _, d, _ = sim.fields()
        assert np.allclose(d, d_ex, rtol=1e-7, atol=1e-9)
        assert r["reaction"] == pytest.approx(syy * spec.Lx, rel=1e-7)
    assert d.min() > 0.2
    sim.close()


@pytest.mark.parametrize("mode", MODES, ids=["fp64-jacobi", "fp64-gmg", "fp32ir-gmg"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_tensile_path_matches_checker(gpu, scheme, mode):
    precision, precond = mode
    if precision == binding.FP32_IR and scheme == 0:
        pytest.skip("one FP32 case suffices")
    spec = S.tensile(24, l=0.08, steps=6, u_max=8e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane,
                                 model.SPECTRAL)
    fp64 = precision == binding.FP64
    tol = 1e-8 if fp64 else 1e-7
    st = stg.State(g)
    sim = binding.Simulation(spec, precision=precision, precond=precond,
                             split=binding.SPLIT_SPECTRAL)
    sim.set_options(tol_lin=1e-12 if fp64 else 1e-10)
    out = []
    for du in spec.increments:
        r_ref = stg.load_step(g, m, st, du, scheme, stg.Options(tol_st=tol), spec.reaction_dir)
        r = sim.load_step(du, scheme, tol)
        out.append((r_ref, r, st.d.copy(), sim.fields()[1]))
    sim.close()
    peak = max(abs(o[0].reaction) for o in out)
    mirror = lambda f: f.reshape(g.ny + 1, g.nx + 1)[::-1].ravel()
    cracked = False
    for r_ref, r, d_ref, d in out:
        assert r["converged"] == 1 and r_ref.converged
        if fp64:
            assert abs(r["reaction"] - r_ref.reaction) <= 1e-6 * peak
            assert min(np.max(np.abs(d - d_ref)), np.max(np.abs(d - mirror(d_ref)))) < 1e-5
        else:
            assert abs(r["reaction"] - r_ref.reaction) <= 1e-4 * peak
            assert _d_rms(g, d, d_ref) <= 1e-3
        cracked |= r_ref.stag_iters > 20
    assert cracked


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_IR])
def test_multilevel_hierarchy_path(gpu, precision):
    # 48 x 48: the hierarchy has a grid-wide level above the single-CTA coarse cycle, so
    # the V-cycle runs its stencil fine level and the separate coarse-level kernels
    spec = S.tensile(48, l=0.04, steps=8, u_max=4.8e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane,
                                 model.SPECTRAL)
    fp64 = precision == binding.FP64
    st = stg.State(g)
    sim = binding.Simulation(spec, precision=precision, precond=binding.PRECOND_GMG,
                             split=binding.SPLIT_SPECTRAL)
    sim.set_options(tol_lin=1e-12 if fp64 else 1e-10)
    for du in spec.increments[:3]:
        r_ref = stg.load_step(g, m, st, du, 1, stg.Options(tol_st=1e-8), spec.reaction_dir)
        r = sim.load_step(du, 1, 1e-8)
        assert r["converged"] == 1
        assert abs(r["reaction"] - r_ref.reaction) <= (1e-6 if fp64 else 1e-4) * abs(r_ref.reaction)
        assert np.max(np.abs(sim.fields()[1] - st.d)) < (1e-6 if fp64 else 1e-4)
    sim.close()
