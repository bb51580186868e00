"""The launch-shape autotuner (pf_autotune) on the GPU.

It times strip heights of the FP32 tangent kernel and single-CTA coarse-cycle limits on
the context's own grid, records the fastest, and the tuned context still follows the
FP64 checker within the mixed-precision tolerances.
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu


def test_autotune_records_a_valid_choice_and_keeps_parity(gpu):
    spec = S.tensile(80, l=0.05, steps=5, u_max=3e-3)      # damage grows, no crack jump
    sim = binding.Simulation(spec, precision=binding.FP32_IR, precond=binding.PRECOND_GMG)
    sim.set_options(tol_lin=1e-12)
    t = sim.autotune()
    assert t["strip_rows"] in (2, 4, 8) and t["coarse_nodes"] in (300, 1100, 4300)
    assert all(x > 0 for x in t["apply_us"])
    k = (2, 4, 8).index(t["strip_rows"])
    assert t["apply_us"][k] == min(t["apply_us"])
    assert sim.tuning() == t
    with pytest.raises(binding.PfError) as e:      # only before the first load step
        sim.load_step(spec.increments[0], 1, 1e-9)
        sim.autotune()
    assert e.value.status == binding.PF_EBUSY
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    st = stg.State(g)
    Fr, Fg = [], []
    stg.load_step(g, m, st, spec.increments[0], 1, stg.Options(tol_st=1e-9), spec.reaction_dir)
    for du in spec.increments[1:]:
        Fr.append(stg.load_step(g, m, st, du, 1, stg.Options(tol_st=1e-9),
                                spec.reaction_dir).reaction)
        r = sim.load_step(du, 1, 1e-9)
        assert r["converged"] == 1
        Fg.append(r["reaction"])
    sim.close()
    assert np.max(np.abs(np.array(Fg) - np.array(Fr))) <= 1e-4 * max(Fr)


def test_autotune_rejects_other_forms(gpu):
    sim = binding.Simulation(S.tensile(40, l=0.1), precision=binding.FP64,
                             precond=binding.PRECOND_GMG)
    with pytest.raises(binding.PfError) as e:
        sim.autotune()
    assert e.value.status == binding.PF_EINVAL
    sim.close()
