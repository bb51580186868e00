"""Synthetic specimens and seeded inputs (input generation only, no method arithmetic).

Builds the structured-grid specimens of the paper's benchmark family -- tensile and
shear notched squares (Sec. 4.1-4.2), an L-shaped panel (Sec. 4.3) -- plus small
analytic specimens used for checks, and seeded random fields.  Everything here is data:
node flag bytes, element masks, load schedules and material constants.  The solver
(CUDA library) and the independent checker both take these arrays as inputs.

Node flag bits (one byte per node): FIX_X=1, FIX_Y=2, LOAD_X=4, LOAD_Y=8, D_FIX1=16
(phase field held at 1), D_FIX0=32 (phase field held at 0).  Node (i, j) has id
j (nx+1) + i; element (i, j) has id j nx + i.
"""
from dataclasses import dataclass, field

import numpy as np

FIX_X, FIX_Y, LOAD_X, LOAD_Y, D_FIX1, D_FIX0 = 1, 2, 4, 8, 16, 32
PLANE_STRAIN, PLANE_STRESS = 0, 1

# Tensile/shear material of the notched-square benchmarks in kN and mm
# (lambda = 121.15 kN/mm^2, mu = 80.77 kN/mm^2, G_c = 2.7e-3 kN/mm).
MIEHE_LAMBDA = 121.15
MIEHE_MU = 80.77
MIEHE_GC = 2.7e-3


def lame_to_E_nu(lam, mu):
    """(lambda, mu) -> (E, nu); the library's create call takes E and nu."""
    return mu * (3.0 * lam + 2.0 * mu) / (lam + mu), lam / (2.0 * (lam + mu))


@dataclass
class Specimen:
    name: str
    nx: int
    ny: int
    Lx: float
    Ly: float
    node_flags: np.ndarray
    elem_active: np.ndarray
    reaction_dir: int
    plane: int
    E: float
    nu: float
    Gc: float
    l: float
    eta: float
    increments: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def nn(self):
        return (self.nx + 1) * (self.ny + 1)

    @property
    def ne(self):
        return self.nx * self.ny


# Two-rate loading schedules of the paper's benchmarks: the load point moves at a constant
# rate, in steps of dt1 up to time t1 and of dt2 from there up to t2 (Sec. 4.1 tensile,
# Sec. 4.2 shear, Sec. 4.3 L-shape; rate in mm/s, times in s).
PAPER_SCHEDULES = {
    "tensile": dict(rate=3e-5, dt1=170.0, t1=170.0, dt2=1.0, t2=220.0),
    "shear": dict(rate=3e-5, dt1=250.0, t1=250.0, dt2=1.0, t2=380.0),
    "l_shape": dict(rate=1e-3, dt1=0.01, t1=0.2, dt2=0.001, t2=0.6),
}


def two_rate_schedule(rate, dt1, t1, dt2, t2):
    """(times, increments) of a two-rate schedule: t_n after each step and the prescribed
    displacement increment rate * dt_n of each step."""
    n1 = int(round(t1 / dt1))
    n2 = int(round((t2 - t1) / dt2))
    dt = np.concatenate([np.full(n1, dt1), np.full(n2, dt2)])
    return np.cumsum(dt), rate * dt


def paper_schedule(kind):
    """(times, increments) of the paper's schedule for ``kind`` in PAPER_SCHEDULES."""
    return two_rate_schedule(**PAPER_SCHEDULES[kind])


def _increments(kind, schedule, steps, u_max):
    if schedule == "paper":
        return paper_schedule(kind)[1]
    if schedule not in (None, "uniform"):
        raise ValueError(f"unknown schedule {schedule!r}")
    return np.full(steps, u_max / steps)


def _node_ij(nx, ny):
    j, i = np.divmod(np.arange((nx + 1) * (ny + 1)), nx + 1)
    return i, j


def _slit(flags, nx, ny):
    """Horizontal slit from the left edge to the centre: d = 1 on nodes y = Ly/2, x <= Lx/2."""
    if ny % 2 or nx % 2:
        raise ValueError("slit specimens need even nx and ny")
    i, j = _node_ij(nx, ny)
    flags[(j == ny // 2) & (i <= nx // 2)] |= D_FIX1


def tensile(n, l=None, steps=20, u_max=6e-3, eta=1e-9, schedule=None):
    """Tensile notched unit square: bottom fixed, top pulled up (u_x = 0 on top).

    ``schedule``: None or "uniform" gives ``steps`` equal increments to ``u_max``;
    "paper" gives the two-rate schedule of Sec. 4.1 (steps and u_max ignored)."""
    nx = ny = int(n)
    i, j = _node_ij(nx, ny)
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    flags[j == 0] |= FIX_X | FIX_Y
    flags[j == ny] |= FIX_X | LOAD_Y
    _slit(flags, nx, ny)
    E, nu = lame_to_E_nu(MIEHE_LAMBDA, MIEHE_MU)
    return Specimen("tensile", nx, ny, 1.0, 1.0, flags, np.ones(nx * ny, np.uint8), 1,
                    PLANE_STRAIN, E, nu, MIEHE_GC, 0.03 if l is None else l, eta,
                    _increments("tensile", schedule, steps, u_max))


def shear(n, l=None, steps=150, u_max=1.5e-2, eta=1e-9, schedule=None):
    """Shear notched unit square: bottom fixed, top moved in x (u_y = 0), rollers on sides.
    ``schedule="paper"``: the two-rate schedule of Sec. 4.2."""
    nx = ny = int(n)
    i, j = _node_ij(nx, ny)
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    side = ((i == 0) | (i == nx)) & (j > 0) & (j < ny)
    flags[side] |= FIX_Y
    flags[j == 0] |= FIX_X | FIX_Y
    flags[j == ny] |= LOAD_X | FIX_Y
    _slit(flags, nx, ny)
    E, nu = lame_to_E_nu(MIEHE_LAMBDA, MIEHE_MU)
    return Specimen("shear", nx, ny, 1.0, 1.0, flags, np.ones(nx * ny, np.uint8), 0,
                    PLANE_STRAIN, E, nu, MIEHE_GC, 0.03 if l is None else l, eta,
                    _increments("shear", schedule, steps, u_max))


def l_shape(n, steps=200, u_max=1.0, l=2.5, eta=1e-9, patch=30.0, schedule=None):
    """L-shaped panel: 500 x 500 mm with the top-right quadrant masked out, plane stress.

    The bottom edge under the upright part (x <= 250 mm) is clamped; the lower arm
    (x > 250 mm) is a cantilever lifted on a ``patch``-wide strip of its bottom edge at
    the free end, where the phase field is held at zero.
    """
    nx = ny = int(n)
    if n % 2:
        raise ValueError("l_shape needs an even grid")
    L = 500.0
    h = L / n
    ej, ei = np.divmod(np.arange(nx * ny), nx)
    active = ~((ei >= nx // 2) & (ej >= ny // 2))
    i, j = _node_ij(nx, ny)
    x = i * h
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    flags[(j == 0) & (x <= 0.5 * L + 1e-9)] |= FIX_X | FIX_Y
    load = (j == 0) & (x >= L - patch - 1e-9)
    flags[load] |= LOAD_Y
    flags[(j <= max(1, int(round(patch / h)))) & (x >= L - patch - 1e-9)] |= D_FIX0
    return Specimen("l_shape", nx, ny, L, L, flags, active.astype(np.uint8), 1,
                    PLANE_STRESS, 25.85, 0.18, 8.9e-5, l, eta,
                    _increments("l_shape", schedule, steps, u_max))


def uniaxial_bar(nx, ny, Lx=1.0, Ly=1.0, lam=MIEHE_LAMBDA, mu=MIEHE_MU, Gc=MIEHE_GC,
                 l=0.03, eta=1e-9, steps=10, u_max=1e-2):
    """Homogeneous uniaxial strain: u_x = 0 everywhere on the boundary sides, bottom
    u_y = 0, top u_y = ubar, no slit.  The exact state is uniform (closed form)."""
    i, j = _node_ij(nx, ny)
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    flags[(i == 0) | (i == nx)] |= FIX_X
    flags[j == 0] |= FIX_X | FIX_Y
    flags[j == ny] |= FIX_X | LOAD_Y
    E, nu = lame_to_E_nu(lam, mu)
    return Specimen("uniaxial", nx, ny, Lx, Ly, flags, np.ones(nx * ny, np.uint8), 1,
                    PLANE_STRAIN, E, nu, Gc, l, eta, np.full(steps, u_max / steps))


def uniaxial_stress_bar(nx, ny, Lx=0.5, Ly=1.0, lam=MIEHE_LAMBDA, mu=MIEHE_MU, Gc=MIEHE_GC,
                        l=0.03, eta=1e-9, steps=10, u_max=1e-2):
    """Plane-strain bar pulled along y with free sides: bottom u_y = 0, u_x = 0 at the
    bottom-left node only, top u_y = ubar, no slit.  The exact state is uniform, with the
    lateral strain set by sigma_xx = 0 (closed form per energy split)."""
    i, j = _node_ij(nx, ny)
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    flags[j == 0] |= FIX_Y
    flags[(j == 0) & (i == 0)] |= FIX_X
    flags[j == ny] |= LOAD_Y
    E, nu = lame_to_E_nu(lam, mu)
    return Specimen("uniaxial_stress", nx, ny, Lx, Ly, flags, np.ones(nx * ny, np.uint8), 1,
                    PLANE_STRAIN, E, nu, Gc, l, eta, np.full(steps, u_max / steps))


def strip_1d(nx, ny=4, L=1.0, l=0.05):
    """Phase-field strip [0, L] x [0, L ny / nx] with d = 1 held on x = 0 and no load."""
    i, j = _node_ij(nx, ny)
    flags = np.zeros((nx + 1) * (ny + 1), np.uint8)
    flags[i == 0] |= D_FIX1
    flags[:] |= 0
    E, nu = lame_to_E_nu(MIEHE_LAMBDA, MIEHE_MU)
    return Specimen("strip", nx, ny, L, L * ny / nx, flags, np.ones(nx * ny, np.uint8), 1,
                    PLANE_STRAIN, E, nu, MIEHE_GC, l, 1e-9)


def bar_1d(nx, steps=260, du=0.01, E=1.0, Gc=0.1, l=0.01, eta=1e-9):
    """The paper's one-dimensional example: a bar of length 1 fixed at x = 0 and extended at
    x = 1 by du per step (E = 1, G_c = 0.1, l = 0.01).  Modelled as one row of nx square
    plane-strain elements with nu = 0 and u_y = 0 everywhere, where the volumetric-deviatoric
    split reduces exactly to the 1D law (Psi+ = E eps^2 / 2, sigma = g(d) E eps in tension).
    Reaction: x-force at x = 1."""
    ny = 1
    i, j = _node_ij(nx, ny)
    flags = np.full((nx + 1) * (ny + 1), FIX_Y, np.uint8)
    flags[i == 0] |= FIX_X
    flags[i == nx] |= LOAD_X
    return Specimen("bar_1d", nx, ny, 1.0, 1.0 / nx, flags, np.ones(nx * ny, np.uint8), 0,
                    PLANE_STRAIN, E, 0.0, Gc, l, eta, np.full(steps, du))


# ---- seeded random inputs ------------------------------------------------------------------
def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_state(spec, seed, u_scale=1e-3, h_scale=None):
    """Seeded (u, d, H) of crack-like structure for operator checks.

    u: smooth field plus noise (strain of order u_scale), d in [0, 1) with a damaged
    band and values up to 1, H >= 0 per quadrature point of the order of Psi_crit.
    """
    r = rng(seed)
    i, j = _node_ij(spec.nx, spec.ny)
    x = i / spec.nx
    y = j / spec.ny
    ux = u_scale * (np.sin(3.1 * x + 0.3) * y + 0.2 * r.standard_normal(spec.nn))
    uy = u_scale * (np.cos(2.3 * y) * x + y + 0.2 * r.standard_normal(spec.nn))
    u = np.stack([ux, uy], axis=1).ravel() * spec.Lx
    band = np.exp(-((y - 0.5) / 0.08) ** 2)
    d = np.clip(band * (0.7 + 0.3 * r.random(spec.nn)) + 0.05 * r.random(spec.nn), 0.0, 1.0)
    d[r.random(spec.nn) < 0.02] = 1.0
    if h_scale is None:
        h_scale = spec.Gc / spec.l
    H = h_scale * r.random((spec.ne, 4)) * (1.0 + 3.0 * r.random((spec.ne, 1)))
    return u, d, H


def served_batch(n_requests=256, seed=0, rate_per_s=1.0, grids=(128, 256, 512, 1024)):
    """Seeded request mix of the served-batch workload.

    Each request: tensile or shear notched square (50/50) on a grid drawn from ``grids``,
    E ~ U[20, 210] GPa, nu ~ U[0.15, 0.35], G_c ~ U[1e-4, 3e-3] kN/mm, l ~ U[2h, 4h], scheme
    from {ST, S1, S2}; 100 (tensile) or 150 (shear) load steps to a final displacement
    scaled from the benchmark's by the homogeneous critical strain
    sqrt(G_c / (3 M l)) (M = lambda + 2 mu).  Arrivals are a Poisson process of the given
    rate.  Returns a list of (arrival_time_s, Specimen, scheme).
    """
    r = rng(seed)
    M0 = MIEHE_LAMBDA + 2 * MIEHE_MU
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += r.exponential(1.0 / rate_per_s)
        n = int(r.choice(grids))
        h = 1.0 / n
        E = r.uniform(20.0, 210.0)
        nu = r.uniform(0.15, 0.35)
        Gc = r.uniform(1e-4, 3e-3)
        l = r.uniform(2 * h, 4 * h)
        scheme = int(r.integers(0, 3))
        tensile_kind = r.random() < 0.5
        mu = E / (2 * (1 + nu))
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        scale = np.sqrt((Gc / MIEHE_GC) * (M0 / (lam + 2 * mu)) * (0.0075 / l))
        if tensile_kind:
            sp = tensile(n, l=l, steps=100, u_max=6e-3 * scale)
        else:
            sp = shear(n, l=l, steps=150, u_max=1.5e-2 * scale)
        sp.E, sp.nu, sp.Gc = E, nu, Gc
        out.append((t, sp, scheme))
    return out
