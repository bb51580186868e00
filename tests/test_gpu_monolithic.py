"""The GPU path's converged load steps against the checker's monolithic Newton.

At a tight staggered tolerance the staggered iteration's fixed point is the solution of the
coupled system of Sec. 3.2, which the checker solves directly with the full Jacobian
(oracle/monolithic.py).  Pre-crack steps of the notched tensile square, both energy
splits, ST and S3 (the comparator is a reference for converged states; past the peak plain
coupled Newton does not converge reliably).
"""
import numpy as np
import pytest

from oracle import model, monolithic as mono, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("split", [binding.SPLIT_VD, binding.SPLIT_SPECTRAL])
@pytest.mark.parametrize("scheme", [0, 3])
def test_staggered_fixed_point_is_the_monolithic_solution(gpu, split, scheme):
    spec = S.tensile(24, l=0.08, steps=6, u_max=8e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane,
                                 split)
    st = stg.State(g)
    sim = binding.Simulation(spec, precision=binding.FP64, precond=binding.PRECOND_GMG,
                             split=split)
    sim.set_options(tol_lin=1e-12, tol_nr=1e-10)
    for du in spec.increments[:3]:
        rm = mono.load_step(g, m, st, du, tol_nr=1e-11, tol_st=1e-12)
        r = sim.load_step(du, scheme, 1e-10)
        assert rm.converged and r["converged"] == 1
        _, d, H = sim.fields()
        assert np.max(np.abs(d - st.d)) < 1e-7
        assert np.max(np.abs(H - st.H)) <= 1e-7 * np.max(st.H)
        assert r["reaction"] == pytest.approx(rm.reaction, rel=1e-7)
    sim.close()
