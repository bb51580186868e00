"""The paper's two-rate loading schedules (Sec. 4.1-4.3) and the checker on the large
first step of the tensile schedule.

Sec. 4.1: 3e-5 mm/s, one step of 170 s, then 1 s steps up to 220 s.  Sec. 4.2: the same
rate, one step of 250 s, then 1 s steps up to 380 s.  Sec. 4.3: 1e-3 mm/s, 0.01 s steps
up to 0.2 s, then 0.001 s steps up to 0.6 s.
"""
import os

import numpy as np
import pytest

from oracle import model, q1, staggered as stg
from paper_2209_07969_gb300 import specimens as S


@pytest.mark.parametrize("kind,n1,inc1,n2,inc2,t_end", [
    ("tensile", 1, 170 * 3e-5, 50, 3e-5, 220.0),
    ("shear", 1, 250 * 3e-5, 130, 3e-5, 380.0),
    ("l_shape", 20, 1e-5, 400, 1e-6, 0.6),
])
def test_paper_schedules(kind, n1, inc1, n2, inc2, t_end):
    t, inc = S.paper_schedule(kind)
    assert len(inc) == n1 + n2
    assert np.allclose(inc[:n1], inc1, rtol=1e-12)
    assert np.allclose(inc[n1:], inc2, rtol=1e-12)
    assert t[-1] == pytest.approx(t_end, rel=1e-12)
    assert np.all(np.diff(t) > 0)
    # displacement = rate x time at every step
    rate = S.PAPER_SCHEDULES[kind]["rate"]
    assert np.allclose(np.cumsum(inc), rate * t, rtol=1e-12)


def test_schedule_table_matches_the_printed_values():
    path = os.path.join(os.path.dirname(__file__), "golden", "loading_schedules.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert {r[0] for r in rows} == set(S.PAPER_SCHEDULES)
    for kind, *vals in rows:
        want = dict(zip(("rate", "dt1", "t1", "dt2", "t2"), map(float, vals)))
        assert S.PAPER_SCHEDULES[kind] == pytest.approx(want, rel=1e-15)


def test_specimens_take_the_schedule():
    assert np.array_equal(S.tensile(8, schedule="paper").increments, S.paper_schedule("tensile")[1])
    assert np.array_equal(S.shear(8, schedule="paper").increments, S.paper_schedule("shear")[1])
    assert np.array_equal(S.l_shape(8, schedule="paper").increments,
                          S.paper_schedule("l_shape")[1])
    # the default stays the uniform schedule of the benchmark configurations
    assert np.allclose(S.tensile(8, steps=20, u_max=6e-3).increments, 3e-4)
    with pytest.raises(ValueError):
        S.tensile(8, schedule="bogus")


def test_checker_first_paper_step_tensile():
    # One 5.1e-3 mm step from the unloaded state (Sec. 4.1), ST and S1: both converge to
    # the same state, the phase field and the history stay irreversible and bounded.
    sp = S.tensile(16, l=0.1, schedule="paper")
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane)
    opts = stg.Options(tol_st=1e-9)
    out = []
    for scheme in (model.ST, model.S1):
        st = stg.State(g)
        r = stg.load_step(g, m, st, sp.increments[0], scheme, opts, sp.reaction_dir)
        assert r.converged
        assert st.d.min() >= 0.0 and st.d.max() <= 1.0 + 1e-12
        out.append((r, st))
    (ra, sa), (rb, sb) = out
    assert rb.reaction == pytest.approx(ra.reaction, rel=1e-6)
    assert np.max(np.abs(sa.d - sb.d)) < 1e-6
