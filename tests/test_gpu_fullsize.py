"""Parity at the full sizes of the benchmark workloads, checked by the FP64 checker.

The checker cannot run these paths itself (a direct solve of the 2048 x 2048 L-shape is
out of reach), but it can evaluate the discrete equations at the state the GPU path
returns.  After load steps run exactly as the benchmark runs them (FP32 CG with FP64
refinement, multigrid, scheme S1), the checker verifies, from (u, d, H) alone:

- momentum balance: the free-DOF residual of its own internal force satisfies the Newton
  test of Sec. 4 (relative to the constrained-DOF force, TOL_NR = 1e-7);
- the staggered test of Sec. 3.1: max |R_d / K_dd,ii| with H = max(H_{n-1}, Psi+(u)) is
  below the step tolerance;
- the committed history H_n = max(H_{n-1}, Psi+(u_n)) and the reaction force;
- Dirichlet values (slit d = 1, d = 0 under the L-shape's load patch, prescribed u) and
  0 <= d <= 1.
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu

TOL_ST = 1e-5


def _check_state(spec, steps, scheme=binding.S1, split=binding.SPLIT_VD, max_stag=1000):
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane,
                                 split)
    sim = binding.Simulation(spec, precision=binding.FP32_IR, precond=binding.PRECOND_GMG,
                             split=split)
    sim.set_options(max_stag=max_stag)
    ubar = 0.0
    H_prev = np.zeros((g.ne, 4))
    for k in range(steps):
        if k == steps - 1:
            H_prev = sim.fields()[2]
        r = sim.load_step(spec.increments[k], scheme, TOL_ST)
        ubar += spec.increments[k]
        assert r["converged"] == 1
    u, d, H = sim.fields()
    sim.close()

    # momentum balance at the returned state (checker's internal force)
    F = q1.internal_force(g, u, q1.interp_qp(g, d), m)
    cu = g.u_constrained()
    f_free = np.linalg.norm(F[~cu])
    f_con = np.linalg.norm(F[cu])
    assert f_free <= 5e-7 * f_con, (f_free, f_con)
    # staggered residual with the true H of u (Sec. 3.1 test)
    assert stg.stag_residual(g, m, u, d, H_prev) <= 1.05 * TOL_ST
    # committed history and reaction
    # (strains are differences of nodal values: where a part moves almost rigidly, as the
    # L-shape's arm does, both codes carry relative rounding |u| / |du| ~ 1e4 times eps)
    # Masked elements enter no equation; the GPU path keeps their H, the checker does not.
    act = g.elem_active.astype(bool)
    H_ref = np.maximum(H_prev, stg.psi_plus_qp(g, u, m))
    assert np.allclose(H[act], H_ref[act], rtol=1e-8, atol=1e-12 * H_ref[act].max())
    R_ref = q1.reaction_force(g, F, spec.reaction_dir)
    assert r["reaction"] == pytest.approx(R_ref, rel=1e-9)
    # Dirichlet data and bounds
    cd = g.d_constrained()
    assert np.array_equal(d[cd], g.d_dirichlet_values()[cd])
    assert d.min() >= -1e-8 and d.max() <= 1.0 + 1e-8
    uc = g.u_dirichlet_values(ubar)
    assert np.allclose(u[cu], uc[cu], rtol=0, atol=1e-15)
    return r


def test_tensile_512_bench_workload():
    r = _check_state(S.tensile(512, l=0.0075, steps=100, u_max=6e-3), 3)
    assert r["reaction"] > 0


def test_shear_1024():
    r = _check_state(S.shear(1024, l=0.0075, steps=150, u_max=1.5e-2), 2)
    assert r["reaction"] != 0


def test_lshape_2048_plane_stress():
    r = _check_state(S.l_shape(2048), 2)
    assert r["reaction"] != 0


def test_tensile_512_spectral_split():
    # the spectral split's stencil u-solves on the full-size multigrid hierarchy
    r = _check_state(S.tensile(512, l=0.0075, steps=100, u_max=6e-3), 3,
                     split=binding.SPLIT_SPECTRAL)
    assert r["reaction"] > 0


def test_tensile_256_inside_the_running_crack():
    # 256 x 256 at the l/h of the 512 x 512 workload, through the first crack jump (step 44)
    # into the running crack (steps 84-85: thousands of staggered passes); the checker
    # verifies the state the GPU path returns at step 85
    r = _check_state(S.tensile(256, l=0.015, steps=100, u_max=6e-3), 85, max_stag=20000)
    assert r["stag_iters"] > 100
