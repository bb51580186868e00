"""AT1 with penalty irreversibility (Sec. 2, Table 1) on the GPU path against the checker.

- Homogeneous uniaxial-strain bar: the strain is prescribed by the boundary, so at every
  load step the phase field solves the scalar stationarity equation
  -2 (1-d) Psi+ + G_c/(c_w l) + gamma <d - d_{n-1}>_- = 0 (loading past the elastic limit,
  unloading and reloading), for the standard and a fixed-stress scheme, both precisions and
  both preconditioners.
- The notched-square path in FP64 against the checker's AT1 path (same specimen,
  increments, scheme and tolerances): reaction within 1e-6 of the peak force at every step,
  phase field within 1e-6 (or its mirror image, see test_gpu_solver).
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu

TOL_IR = 0.01


def _scalar_d(psi, d_prev, a, gamma):
    d_free = 1.0 - a / (2.0 * psi) if psi > 0 else -np.inf
    if d_free >= d_prev:
        return d_free
    return (2.0 * psi - a + gamma * d_prev) / (2.0 * psi + gamma)


@pytest.mark.parametrize("precond", [binding.PRECOND_JACOBI, binding.PRECOND_GMG])
@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_IR])
@pytest.mark.parametrize("scheme", [binding.ST, binding.S1])
def test_at1_bar_closed_form(gpu, scheme, precision, precond):
    lam, mu, Gc, l, eta = 121.15, 80.77, 2.7e-3, 0.03, 1e-9
    M = lam + 2 * mu
    sp = S.uniaxial_bar(9, 12, Lx=0.5, Ly=1.0, lam=lam, mu=mu, Gc=Gc, l=l, eta=eta)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane)
    a, kappa, gamma = model.at1_constants(m, TOL_IR)
    eps_c = np.sqrt(2 * a / M)
    ubars = np.concatenate([np.linspace(0.2, 2.0, 7), [1.5, 1.0, 1.8]]) * eps_c * sp.Ly
    sim = binding.Simulation(sp, precision=precision, precond=precond,
                             model=binding.AT1_PENALTY, tol_ir=TOL_IR)
    sim.set_options(tol_lin=1e-12, max_stag=300)
    ubar, d_ref = 0.0, 0.0
    for ub in ubars:
        r = sim.load_step(ub - ubar, scheme, 1e-9)
        ubar = ub
        assert r["converged"] == 1
        eps = ubar / sp.Ly
        d_ref = _scalar_d(0.5 * M * eps ** 2, d_ref, a, gamma)
        _, d, _ = sim.fields()
        assert np.allclose(d, d_ref, rtol=1e-7, atol=1e-9)
        F = ((1 - d_ref) ** 2 + eta) * M * eps * sp.Lx
        assert r["reaction"] == pytest.approx(F, rel=1e-7)
    assert d_ref > 0.3
    sim.close()
    # (reloading past the previous maximum re-enters the softening branch, where the
    # homogeneous state is unstable under displacement control: a rounding difference can
    # seed a localized solution of the same discrete equations -- a damaging band with the
    # rest unloading elastically -- so the closed form stops below the maximum)


def _mirror_nodes(g, f):
    return f.reshape(g.ny + 1, g.nx + 1)[::-1].ravel()


@pytest.mark.parametrize("precond", [binding.PRECOND_JACOBI, binding.PRECOND_GMG])
@pytest.mark.parametrize("scheme", [binding.ST, binding.S1])
def test_at1_tensile_path_matches_checker(gpu, scheme, precond):
    spec = S.tensile(24, l=0.08, steps=6, u_max=8e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    opts = stg.Options(tol_st=1e-8, model=model.AT1, tol_ir=TOL_IR)
    st = stg.State(g)
    sim = binding.Simulation(spec, precision=binding.FP64, precond=precond,
                             model=binding.AT1_PENALTY, tol_ir=TOL_IR)
    sim.set_options(tol_lin=1e-12)
    out = []
    for du in spec.increments:
        r_ref = stg.load_step(g, m, st, du, scheme, opts, spec.reaction_dir)
        r = sim.load_step(du, scheme, 1e-8)
        u, d, H = sim.fields()
        out.append((r_ref, r, st.d.copy(), d))
    sim.close()
    peak = max(abs(o[0].reaction) for o in out)
    damaged = False
    for r_ref, r, d_ref, d in out:
        assert r["converged"] == 1 and r_ref.converged
        assert abs(r["reaction"] - r_ref.reaction) <= 1e-6 * peak
        dd = min(np.abs(d - d_ref).max(), np.abs(d - _mirror_nodes(g, d_ref)).max())
        assert dd < 1e-6
        damaged |= d_ref[~g.d_constrained()].max() > 0.5
    assert damaged, "the path must develop damage away from the slit"
