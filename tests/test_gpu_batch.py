"""Batched solves (pf_batch_*) give every simulation the results it gives alone (GPU).

Simulations of different grids, specimens and schemes advance together; their FP32
multigrid solves run as shared launches, each simulation keeping its own block
decomposition and reduction order.  So a simulation's reactions, pass counts and fields
must be bit-identical in a batch of several, in a batch of one, and without a batch, and
the batched path must still match the FP64 checker within the mixed-precision
tolerances.
"""
import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu

FP32, GMG = binding.FP32_IR, binding.PRECOND_GMG


def _specs():
    # grids above the single-CTA coarse cycle (more than 1,100 nodes), so the fused
    # multigrid solve (the batched one) is taken
    return [
        (S.tensile(48, l=0.08, steps=5, u_max=8e-3), 1),
        (S.tensile(64, l=0.06, steps=5, u_max=8e-3), 0),
        (S.shear(40, l=0.1, steps=5, u_max=1.2e-2), 3),
        (S.tensile(72, l=0.05, steps=5, u_max=8e-3), 2),
    ]


def _run(specs, mode):
    """mode: 'batch' (all together), 'one' (each in a batch of one), 'plain' (no batch)."""
    sims = [binding.Simulation(sp, precision=FP32, precond=GMG) for sp, _ in specs]
    for s in sims:
        s.set_options(tol_lin=1e-12)
    out = [[] for _ in sims]
    nsteps = len(specs[0][0].increments)
    if mode == "batch":
        b = binding.Batch(sims)
        for k in range(nsteps):
            res = b.step([sp.increments[k] for sp, _ in specs], [sc for _, sc in specs], 1e-8)
            for i, r in enumerate(res):
                out[i].append(r)
        stats = b.stats()
        b.close()
    else:
        stats = None
        for i, (sp, sc) in enumerate(specs):
            b = binding.Batch([sims[i]]) if mode == "one" else None
            for k in range(nsteps):
                if b is not None:
                    out[i].append(b.step([sp.increments[k]], [sc], 1e-8)[0])
                else:
                    out[i].append(sims[i].load_step(sp.increments[k], sc, 1e-8))
            if b is not None:
                b.close()
    fields = [s.fields() for s in sims]
    for s in sims:
        s.close()
    return out, fields, stats


def _same(a, b):
    (ra, fa), (rb, fb) = a, b
    for sa, sb in zip(ra, rb):
        for x, y in zip(sa, sb):
            assert x["reaction"] == y["reaction"]
            assert x["stag_iters"] == y["stag_iters"]
            assert x["lin_u"] == y["lin_u"] and x["lin_d"] == y["lin_d"]
    for (ua, da, Ha), (ub, db, Hb) in zip(fa, fb):
        assert np.array_equal(ua, ub) and np.array_equal(da, db) and np.array_equal(Ha, Hb)


def test_batched_equals_batch_of_one_bitwise(gpu):
    specs = _specs()
    rb, fb, stats = _run(specs, "batch")
    ro, fo, _ = _run(specs, "one")
    _same((rb, fb), (ro, fo))
    # the solves did run together
    assert stats["max_group"] >= 2 and stats["solves"] > stats["groups"]
    for steps in rb:
        assert all(r["converged"] == 1 for r in steps)


def test_batched_equals_unbatched_bitwise(gpu):
    specs = _specs()[:2]
    rb, fb, _ = _run(specs, "batch")
    rp, fp, _ = _run(specs, "plain")
    _same((rb, fb), (rp, fp))


def test_ineligible_member_runs_alone_in_a_batch(gpu):
    # an FP64 context attached to a batch solves per context; results unchanged
    sp64, sp32 = S.tensile(48, l=0.08, steps=3, u_max=6e-3), S.tensile(56, l=0.08, steps=3,
                                                                        u_max=6e-3)
    a = binding.Simulation(sp64, precision=binding.FP64, precond=GMG)
    c = binding.Simulation(sp32, precision=FP32, precond=GMG)
    ref = binding.Simulation(sp64, precision=binding.FP64, precond=GMG)
    b = binding.Batch([a, c])
    for k in range(3):
        r = b.step([sp64.increments[k], sp32.increments[k]], [1, 1], 1e-8)
        r0 = ref.load_step(sp64.increments[k], 1, 1e-8)
        assert r[0]["reaction"] == r0["reaction"] and r[0]["stag_iters"] == r0["stag_iters"]
        assert r[1]["converged"] == 1
    b.close()
    for s in (a, c, ref):
        s.close()


def test_batched_path_matches_checker(gpu):
    spec = S.tensile(48, l=0.08, steps=6, u_max=8e-3)
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    other = S.shear(64, l=0.06, steps=6, u_max=1.2e-2)
    sims = [binding.Simulation(sp, precision=FP32, precond=GMG) for sp in (spec, other)]
    for s in sims:
        s.set_options(tol_lin=1e-12)
    b = binding.Batch(sims)
    st = stg.State(g)
    Fr, Fg = [], []
    for k in range(6):
        ref = stg.load_step(g, m, st, spec.increments[k], 1, stg.Options(tol_st=1e-9),
                            spec.reaction_dir)
        r = b.step([spec.increments[k], other.increments[k]], [1, 0], 1e-9)
        assert r[0]["converged"] == 1 and ref.converged
        Fr.append(ref.reaction)
        Fg.append(r[0]["reaction"])
    _, d, _ = sims[0].fields()
    b.close()
    for s in sims:
        s.close()
    Fr, Fg = np.array(Fr), np.array(Fg)
    assert abs(Fg.max() - Fr.max()) <= 1e-4 * Fr.max()
    # the notched square is mirror-symmetric: the crack may branch up or down
    mirror = st.d.reshape(g.ny + 1, g.nx + 1)[::-1].ravel()
    rms = []
    for ref in (st.d, mirror):
        diff = q1.interp_qp(g, d - ref)
        rms.append(np.sqrt(np.sum(diff ** 2) * q1.qp_weight(g) / (g.Lx * g.Ly)))
    assert min(rms) <= 1e-3
