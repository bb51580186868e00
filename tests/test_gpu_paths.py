"""Whole load paths of the tensile notched square against the stored checker paths (GPU).

The checker paths are written by tests/golden/make_oracle_paths.py (FP64 checker only):

* 64 x 64, l = 0.03 mm, 20 steps to 6e-3 mm, ST, TOL_ST 1e-9 -- the plain standard-scheme
  benchmark in FP64.  Reaction within 1e-6 of the peak at every step and the phase field
  within 1e-5 (up to the mirror image of the notched square: the crack may branch up or
  down) at every step, through crack initiation, propagation and the broken state.
* 128 x 128, l = 0.03 mm (l/h = 3.84, the l/h of the 512 x 512 workload), 100 steps to
  6e-3 mm, TOL_ST 1e-5, ST/S1/S2/S3, each in FP64 and in FP32 CG with FP64 refinement,
  multigrid preconditioning with grid levels above the single-CTA coarse cycle.  The path
  has a first, partial crack jump near step 50 and the running crack of steps 83-91.  The
  step of the first jump is not a unique result: at TOL_ST 1e-5 the iteration may stop on
  the un-cracked plateau for one or two more steps (reading R25), and which step it
  leaves it on is decided by rounding.  Compared: every step converged; reactions before
  the step preceding the first jump of either code within 1e-6 (FP64) / 1e-4 (mixed) of
  the peak; the jump
  within two steps; the peak reaction within 1e-4; the phase field (RMS over the domain,
  mirror-aware) within 1e-3 at steps 40, 60, 80 and 100; the broken state at step 100.
"""
import os

import numpy as np
import pytest

from oracle import q1
from paper_2209_07969_gb300 import binding, specimens as S

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _grid(spec):
    return q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)


def _mirror(g, f):
    return f.reshape(g.ny + 1, g.nx + 1)[::-1].ravel()


def _rms(g, a, b):
    def one(bb):
        diff = q1.interp_qp(g, a - bb)
        return np.sqrt(np.sum(diff ** 2) * q1.qp_weight(g) / (g.Lx * g.Ly))
    return min(one(b), one(_mirror(g, b)))


def _maxdiff(g, a, b):
    return min(np.max(np.abs(a - b)), np.max(np.abs(a - _mirror(g, b))))


def _first_jump(F):
    """First step whose reaction falls by more than 5% (the first crack jump)."""
    for k in range(1, len(F)):
        if F[k] < 0.95 * F[k - 1]:
            return k
    return len(F)


def test_config0_full_path_fp64(gpu):
    z = np.load(os.path.join(GOLD, "oracle_tensile64.npz"))
    spec = S.tensile(64)
    g = _grid(spec)
    Fr, dref = z["s0_reaction"], z["s0_d"]
    peak = np.max(np.abs(Fr))
    sim = binding.Simulation(spec, precision=binding.FP64)
    sim.set_options(tol_lin=1e-12, max_stag=20000)
    for k, du in enumerate(spec.increments):
        r = sim.load_step(du, binding.ST, float(z["tol"]))
        assert r["converged"] == 1
        assert abs(r["reaction"] - Fr[k]) <= 1e-6 * peak, k
        _, d, _ = sim.fields()
        assert _maxdiff(g, d, dref[k]) < 1e-5, k
    sim.close()
    assert Fr[-1] < 0.05 * peak        # the path ends broken


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_IR])
@pytest.mark.parametrize("scheme", [0, 1, 2, 3])
def test_tensile128_same_l_over_h_path(gpu, scheme, precision):
    z = np.load(os.path.join(GOLD, "oracle_tensile128.npz"))
    assert f"s{scheme}_reaction" in z, "checker path not written (make_oracle_paths.py)"
    spec = S.tensile(128, l=0.03, steps=100, u_max=6e-3)
    g = _grid(spec)
    Fr, dref, keep = z[f"s{scheme}_reaction"], z[f"s{scheme}_d"], list(z["keep"])
    peak = np.max(Fr)
    sim = binding.Simulation(spec, precision=precision, precond=binding.PRECOND_GMG)
    sim.set_options(max_stag=20000)
    Fg, dg = [], {}
    for k, du in enumerate(spec.increments):
        r = sim.load_step(du, scheme, float(z["tol"]))
        assert r["converged"] == 1, k
        Fg.append(r["reaction"])
        if k + 1 in keep:
            dg[k + 1] = sim.fields()[1]
    sim.close()
    Fg = np.array(Fg)
    jr, jg = _first_jump(Fr), _first_jump(Fg)
    assert jr < 90 and abs(jr - jg) <= 2
    tol = 1e-6 if precision == binding.FP64 else 1e-4
    # the step before the jump stops near the unstable equilibrium (reading R25): at
    # TOL_ST 1e-5 its stopping point is not unique, so the comparison ends one step earlier
    before = min(jr, jg) - 1
    assert np.max(np.abs(Fg[:before] - Fr[:before])) <= tol * peak
    assert abs(Fg.max() - peak) <= 1e-4 * peak
    for i, step in enumerate(keep):
        assert _rms(g, dg[step], dref[i]) <= 1e-3, step
    assert Fg[-1] < 0.05 * peak and Fr[-1] < 0.05 * peak
