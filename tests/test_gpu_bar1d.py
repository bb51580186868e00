"""The paper's one-dimensional example (appendix "A one-dimensional example") on the GPU
path against the checker.

A bar of length 1 (E = 1, G_c = 0.1, l = 0.01, AT1 with penalty, tol_ir = 0.01), fixed at one
end and extended by 0.01 per step at the other, as one row of 200 plane-strain elements with
nu = 0 and u_y = 0 (the volumetric-deviatoric split then is the 1D law).  The bar stays
elastic up to the AT1 limit, damages homogeneously, and the crack nucleates within one load
step, which takes many staggered passes.  The paper reports the nucleation at t = 201 with 25
passes for the standard scheme and 17 for the fixed-stress one on an unstated mesh.

Localization out of the homogeneous state is an instability seeded by rounding, so the step
at which the crack nucleates is not a unique result (the checker and the GPU path may differ
by a few steps).  Checked: the homogeneous path (reaction at every step before either code
localizes, within 1e-6 of the peak), nucleation by a multi-pass step inside the same window,
and a formed crack (d close to 1 at one place) after it.
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu


def _oracle(sp, scheme, nsteps):
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane)
    opts = stg.Options(tol_st=1e-6, model=model.AT1, tol_ir=0.01, max_stag=500)
    st = stg.State(g)
    out = [stg.load_step(g, m, st, du, scheme, opts, reaction_dir=0)
           for du in sp.increments[:nsteps]]
    return out, st.d


@pytest.mark.parametrize("scheme", [binding.ST, binding.S3])
def test_bar_1d_nucleation_matches_checker(gpu, scheme):
    sp = S.bar_1d(200)
    nsteps = 212
    ref, d_ref = _oracle(sp, scheme, nsteps)
    sim = binding.Simulation(sp, precision=binding.FP64, precond=binding.PRECOND_GMG,
                             model=binding.AT1_PENALTY, tol_ir=0.01)
    sim.set_options(tol_lin=1e-12, max_stag=500)
    got = [sim.load_step(du, scheme, 1e-6) for du in sp.increments[:nsteps]]
    d = sim.fields()[1]
    sim.close()
    passes_ref = [r.stag_iters for r in ref]
    passes = [r["stag_iters"] for r in got]
    k_ref, k = int(np.argmax(passes_ref)), int(np.argmax(passes))
    print(f"scheme {scheme}: nucleation at step {k + 1} with {passes[k]} passes "
          f"(checker: step {k_ref + 1}, {passes_ref[k_ref]} passes)")
    for kk, n in ((k, passes[k]), (k_ref, passes_ref[k_ref])):
        assert 190 <= kk + 1 < nsteps and n >= 10
    peak = max(r.reaction for r in ref)
    for r_ref, r in zip(ref[:min(k, k_ref)], got[:min(k, k_ref)]):
        assert r["converged"] == 1
        assert abs(r["reaction"] - r_ref.reaction) <= 1e-6 * peak
    assert all(r["converged"] == 1 for r in got)
    assert d.max() > 0.99 and d_ref.max() > 0.99
