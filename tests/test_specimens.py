"""The synthetic specimens follow the readings of the paper's benchmark set-ups (Sec. 4.1-4.3):
slit d = 1 on the left half of the mid row (R13), tensile and shear boundary conditions
(R14), the masked L-shaped panel with its clamp, load patch and protected strip (R15), and
the material data of the configurations (lambda = 121.15, mu = 80.77 kN/mm^2, G_c =
2.7e-3 kN/mm; E = 25.85 GPa, nu = 0.18, G_c = 8.9e-5 kN/mm, plane stress)."""
import numpy as np
import pytest

from oracle import model
from paper_2209_07969_gb300 import specimens as S

F = S   # flag bits live in the specimen module


def _ij(sp):
    j, i = np.divmod(np.arange((sp.nx + 1) * (sp.ny + 1)), sp.nx + 1)
    return i, j


def test_tensile_set_up():
    sp = S.tensile(16, steps=20, u_max=6e-3)
    i, j = _ij(sp)
    f = sp.node_flags
    slit = (f & F.D_FIX1) != 0
    assert np.array_equal(slit, (j == 8) & (i <= 8))
    assert np.all((f[j == 0] & (F.FIX_X | F.FIX_Y)) == (F.FIX_X | F.FIX_Y))
    assert np.all((f[j == 16] & (F.FIX_X | F.LOAD_Y)) == (F.FIX_X | F.LOAD_Y))
    assert not np.any(f[(j > 0) & (j < 16)] & (F.FIX_X | F.FIX_Y | F.LOAD_X | F.LOAD_Y))
    assert sp.reaction_dir == 1 and sp.plane == model.PLANE_STRAIN
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane)
    assert m.lam == pytest.approx(121.15, rel=1e-12) and m.mu == pytest.approx(80.77, rel=1e-12)
    assert sp.Gc == 2.7e-3 and sp.l == 0.03 and sp.eta == 1e-9
    assert np.allclose(sp.increments, 3e-4) and sp.increments.sum() == pytest.approx(6e-3)


def test_shear_set_up():
    sp = S.shear(16, steps=150, u_max=1.5e-2)
    i, j = _ij(sp)
    f = sp.node_flags
    assert np.all((f[j == 16] & (F.LOAD_X | F.FIX_Y)) == (F.LOAD_X | F.FIX_Y))
    assert not np.any(f[j == 16] & (F.LOAD_Y | F.FIX_X))
    sides = ((i == 0) | (i == 16)) & (j > 0) & (j < 16)
    assert np.all(f[sides] & F.FIX_Y) and not np.any(f[sides] & F.FIX_X)   # rollers
    assert sp.reaction_dir == 0
    assert sp.increments.sum() == pytest.approx(1.5e-2) and len(sp.increments) == 150


def test_l_shape_set_up():
    n = 64
    sp = S.l_shape(n)
    assert sp.Lx == sp.Ly == 500.0 and sp.plane == model.PLANE_STRESS
    assert (sp.E, sp.nu, sp.Gc, sp.l) == (25.85, 0.18, 8.9e-5, 2.5)
    ej, ei = np.divmod(np.arange(n * n), n)
    act = sp.elem_active.astype(bool)
    assert np.array_equal(~act, (ei >= n // 2) & (ej >= n // 2))     # top-right quadrant
    assert act.sum() == 3 * n * n // 4
    i, j = _ij(sp)
    x = i * 500.0 / n
    f = sp.node_flags
    clamp = (f & (F.FIX_X | F.FIX_Y)) == (F.FIX_X | F.FIX_Y)
    assert np.array_equal(clamp, (j == 0) & (x <= 250.0 + 1e-9))
    load = (f & F.LOAD_Y) != 0
    assert np.array_equal(load, (j == 0) & (x >= 470.0 - 1e-9))       # 30 mm patch
    protected = (f & F.D_FIX0) != 0
    assert np.all(protected[load]) and not np.any(protected[clamp])
    assert sp.increments.sum() == pytest.approx(1.0) and len(sp.increments) == 200
