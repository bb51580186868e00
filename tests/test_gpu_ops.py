"""Operator-level parity of the CUDA kernels against the FP64 checker (1e-10 relative).

Every kernel is called through the C ABI on seeded inputs of crack-like structure, at
sizes that span several 32 x 8 node tiles with ragged edges (37 x 23, 130 x 70 with an
element mask) and at the 512 x 512 size of the tensile benchmark.  FP32 variants are
compared at single-precision tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S
from tests.gpu_util import dev, host, masked_matrix, rel_err, setup, stream

pytestmark = pytest.mark.gpu
L = None


def _custom(nx, ny, Lx, Ly, slit_row, slit_len, active=None):
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    j, i = np.divmod(np.arange(flags.size), nx + 1)
    flags[j == 0] |= S.FIX_X | S.FIX_Y
    flags[j == ny] |= S.FIX_X | S.LOAD_Y
    flags[(j == slit_row) & (i < slit_len)] |= S.D_FIX1
    E, nu = S.lame_to_E_nu(S.MIEHE_LAMBDA, S.MIEHE_MU)
    if active is None:
        active = np.ones(nx * ny, np.uint8)
    return S.Specimen("custom", nx, ny, Lx, Ly, flags, active.astype(np.uint8), 1,
                      S.PLANE_STRAIN, E, nu, S.MIEHE_GC, 0.03, 1e-9)


def _spec(case):
    if case == "ragged":
        return _custom(37, 23, 1.3, 0.9, 11, 9)
    if case == "masked":
        nx, ny = 130, 70
        r = np.random.default_rng(3)
        ej, ei = np.divmod(np.arange(nx * ny), nx)
        active = ~((ei >= 90) & (ej >= 40)) & (r.random(nx * ny) > 0.02)
        return _custom(nx, ny, 1.3, 0.7, 35, 40, active)
    if case == "full":
        return S.tensile(512, l=0.0075)
    return S.tensile(64)


CASES = ["ragged", "tensile64", "masked", "full"]


@pytest.fixture(scope="module", params=CASES)
def case(request, gpu):
    global L
    L = binding.lib()
    spec = _spec(request.param)
    g, m, gm, gfull, mat, keep = setup(spec)
    u, d, H = S.random_state(spec, seed=11)
    cd = g.d_constrained()
    d[cd] = g.d_dirichlet_values()[cd]
    return dict(name=request.param, spec=spec, g=g, m=m, gm=gm, gfull=gfull, mat=mat,
                keep=keep, u=u, d=d, H=H)


def _tension(c):
    exx, eyy, _ = q1.strains_qp(c["g"], c["u"])
    ip = model.tension(exx, eyy)
    return (ip * (1 << np.arange(4))).sum(axis=1).astype(np.uint8), ip


def test_residual_and_tension_bits(case):
    g, m = case["g"], case["m"]
    u_d, d_d = dev(case["u"]), dev(case["d"])
    F = torch.empty(2 * g.nn, dtype=torch.float64, device="cuda")
    tb = torch.empty(g.ne, dtype=torch.uint8, device="cuda")
    binding.check(L.pf_op_elas_residual(case["gfull"], case["mat"], u_d.data_ptr(), d_d.data_ptr(),
                                        F.data_ptr(), tb.data_ptr(), stream()))
    ref = q1.internal_force(g, case["u"], q1.interp_qp(g, case["d"]), m)
    assert rel_err(host(F), ref) < 1e-10
    bits, _ = _tension(case)
    got = host(tb)
    live = g.elem_active
    assert np.array_equal(got[live], bits[live])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_elasticity_apply_and_diag(case, dtype):
    g, m = case["g"], case["m"]
    bits, ip = _tension(case)
    K = q1.assemble_elasticity(g, q1.interp_qp(g, case["d"]), ip, m)
    Km = masked_matrix(K, g.u_constrained())
    x = np.random.default_rng(5).standard_normal(2 * g.nn)
    tdt, code, tol = ((torch.float64, binding.F64, 1e-10) if dtype == "f64"
                      else (torch.float32, binding.F32, 2e-5))
    y = torch.empty(2 * g.nn, dtype=tdt, device="cuda")
    dg = torch.empty(2 * g.nn, dtype=tdt, device="cuda")
    d_d, x_d, t_d = dev(case["d"], tdt), dev(x, tdt), dev(bits)
    binding.check(L.pf_op_elas_apply(case["gm"], case["mat"], code, d_d.data_ptr(), t_d.data_ptr(),
                                     x_d.data_ptr(), y.data_ptr(), stream()))
    binding.check(L.pf_op_elas_diag(case["gm"], case["mat"], code, d_d.data_ptr(), t_d.data_ptr(),
                                    dg.data_ptr(), stream()))
    xin = host(x_d).astype(np.float64)
    assert rel_err(host(y), Km @ xin) < tol
    assert rel_err(host(dg), Km.diagonal()) < tol
    # unmasked operator = plain K x
    binding.check(L.pf_op_elas_apply(case["gfull"], case["mat"], code, d_d.data_ptr(), t_d.data_ptr(),
                                     x_d.data_ptr(), y.data_ptr(), stream()))
    assert rel_err(host(y), K @ xin) < tol


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_damage_apply_diag_rhs(case, dtype):
    g, m = case["g"], case["m"]
    c = m.Gc / m.l + 2.0 * case["H"]
    kappa = m.Gc * m.l
    K = q1.assemble_damage(g, c, kappa)
    Km = masked_matrix(K, g.d_constrained())
    x = np.random.default_rng(6).standard_normal(g.nn)
    tdt, code, tol = ((torch.float64, binding.F64, 1e-10) if dtype == "f64"
                      else (torch.float32, binding.F32, 2e-5))
    c_d, x_d = dev(c.ravel(), tdt), dev(x, tdt)
    y = torch.empty(g.nn, dtype=tdt, device="cuda")
    dg = torch.empty(g.nn, dtype=tdt, device="cuda")
    binding.check(L.pf_op_damage_apply(case["gm"], code, c_d.data_ptr(), kappa, x_d.data_ptr(),
                                       y.data_ptr(), stream()))
    binding.check(L.pf_op_damage_diag(case["gm"], code, c_d.data_ptr(), kappa, dg.data_ptr(), stream()))
    xin = host(x_d).astype(np.float64)
    assert rel_err(host(y), Km @ xin) < tol
    assert rel_err(host(dg), Km.diagonal()) < tol
    if dtype == "f64":
        b = torch.empty(g.nn, dtype=torch.float64, device="cuda")
        H_d = dev(case["H"].ravel())
        binding.check(L.pf_op_damage_rhs(case["gm"], H_d.data_ptr(), b.data_ptr(), stream()))
        assert rel_err(host(b), q1.damage_rhs(g, case["H"])) < 1e-12


def test_qp_energy_history(case):
    g, m = case["g"], case["m"]
    u_d, Hp = dev(case["u"]), dev(case["H"].ravel())
    psi = torch.empty(g.ne * 4, dtype=torch.float64, device="cuda")
    Hn = torch.empty_like(psi)
    binding.check(L.pf_op_qp_energy(case["gm"], case["mat"], u_d.data_ptr(), Hp.data_ptr(),
                                    psi.data_ptr(), Hn.data_ptr(), stream()))
    ref = stg.psi_plus_qp(g, case["u"], m)
    live = g.elem_active
    assert rel_err(host(psi).reshape(-1, 4)[live], ref[live]) < 1e-12
    Hg = host(Hn).reshape(-1, 4)
    assert rel_err(Hg[live], np.maximum(case["H"], ref)[live]) < 1e-12
    assert np.all(Hg >= case["H"])            # monotone history, exactly


@pytest.mark.parametrize("scheme", [1, 2, 3])
def test_fixed_stress_coeff_and_predict(case, scheme):
    g, m = case["g"], case["m"]
    u, d, Hp = case["u"] * 12.0, case["d"], case["H"]      # push points into softening
    u_d, d_d, Hp_d = dev(u), dev(d), dev(Hp.ravel())
    c = torch.empty(g.ne * 4, dtype=torch.float64, device="cuda")
    act = torch.empty(g.ne * 4, dtype=torch.uint8, device="cuda")
    binding.check(L.pf_op_fs_coeff(case["gm"], case["mat"], scheme, m.psi_crit, u_d.data_ptr(),
                                   d_d.data_ptr(), Hp_d.data_ptr(), c.data_ptr(), act.data_ptr(), stream()))
    exx, eyy, exy = q1.strains_qp(g, u)
    tr, ee = model.invariants(exx, eyy, exy, m.cdim)
    psi = model.psi_plus(exx, eyy, exy, m)
    Hk = np.maximum(Hp, psi)
    dq = q1.interp_qp(g, d)
    ref_act = model.activation(psi, Hp, dq, m) & g.elem_active[:, None]
    live = g.elem_active
    got_act = host(act).reshape(-1, 4).astype(bool)
    assert np.array_equal(got_act[live], ref_act[live])
    assert ref_act.sum() > 10
    kt = np.where(ref_act, model.extra_stiffness(tr, ee, dq, scheme, m), 0.0)
    ref_c = model.augmented_coefficient(Hk, kt, m)
    assert rel_err(host(c).reshape(-1, 4)[live], ref_c[live]) < 1e-12
    # prediction with a seeded Delta d of both signs
    dd = np.random.default_rng(8).standard_normal(g.nn) * 0.05
    dd_d = dev(dd)
    Hh = torch.empty_like(c)
    binding.check(L.pf_op_fs_predict(case["gm"], case["mat"], scheme, u_d.data_ptr(), d_d.data_ptr(),
                                     dd_d.data_ptr(), Hp_d.data_ptr(), act.data_ptr(), Hh.data_ptr(), stream()))
    ddq = q1.interp_qp(g, dd)
    ps_hat = np.where(ref_act, model.predict_psi(tr, ee, dq, ddq, scheme, m), psi)
    ref_H = np.maximum(Hp, ps_hat)
    assert rel_err(host(Hh).reshape(-1, 4)[live], ref_H[live]) < 1e-12


def test_reaction_and_staggered_residual(case):
    g, m, spec = case["g"], case["m"], case["spec"]
    u_d, d_d, Hp_d = dev(case["u"]), dev(case["d"]), dev(case["H"].ravel())
    F = torch.empty(2 * g.nn, dtype=torch.float64, device="cuda")
    binding.check(L.pf_op_elas_residual(case["gfull"], case["mat"], u_d.data_ptr(), d_d.data_ptr(),
                                        F.data_ptr(), None, stream()))
    out = binding.D()
    flags_d = case["keep"][0]
    binding.check(L.pf_op_reaction(case["gm"], flags_d.data_ptr(), F.data_ptr(), spec.reaction_dir,
                                   binding.C.byref(out), stream()))
    Fi = q1.internal_force(g, case["u"], q1.interp_qp(g, case["d"]), m)
    ref = q1.reaction_force(g, Fi, spec.reaction_dir)
    assert out.value == pytest.approx(ref, rel=1e-10, abs=1e-14 * np.abs(Fi).max())
    binding.check(L.pf_op_stag_residual(case["gm"], case["mat"], u_d.data_ptr(), d_d.data_ptr(),
                                        Hp_d.data_ptr(), binding.C.byref(out), stream()))
    assert out.value == pytest.approx(stg.stag_residual(g, m, case["u"], case["d"], case["H"]), rel=1e-10)
