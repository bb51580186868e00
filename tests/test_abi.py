"""The C-ABI library builds, loads and exports every entry point declared in include/pf.h.

No GPU needed: only host-side entry points (defaults, material conversion, status
strings) are called.
"""
import ctypes
import os
import re

import pytest

from paper_2209_07969_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(L, n), n
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)
    # the binding declares prototypes for exactly the declared set
    assert set(binding._PROTOS) == names


def test_host_only_entry_points(L):
    o = binding.default_options()
    assert o.tol_nr == 1e-7 and o.max_stag == 1000 and o.check_every == 8
    assert o.newton_forcing == 1e-3 and o.device_loop == 1
    m = binding.material(210.0, 0.3, 2.7e-3, 0.03, 1e-9, 0)
    assert m.mu == pytest.approx(210.0 / 2.6, rel=1e-15)
    lam = 210.0 * 0.3 / (1.3 * 0.4)
    assert m.K == pytest.approx(lam + 2 * m.mu / 3, rel=1e-15)
    assert m.cdim == pytest.approx(1 / 3)
    ms = binding.material(25.85, 0.18, 8.9e-5, 2.5, 1e-9, 1)
    assert ms.K == pytest.approx(25.85 / (2 * 0.82), rel=1e-15) and ms.cdim == 0.5
    assert L.pf_status_string(3) == b"PF_ENOTCONV"


@pytest.mark.parametrize("args", [(0.0, 0.3), (210.0, 0.5), (210.0, -1.0)])
def test_material_rejects_bad_input(L, args):
    m = binding.Material()
    assert L.pf_material_make(args[0], args[1], 1e-3, 0.1, 0.0, 0, ctypes.byref(m)) == binding.PF_EINVAL


def test_create_rejects_bad_mesh_without_touching_the_gpu(L):
    out = ctypes.c_void_p()
    mesh = binding.Mesh(0, 4, 1.0, 1.0, None, None, 0, 0, 1, 0)
    assert L.pf_create(ctypes.byref(mesh), 210.0, 0.3, 1e-3, 0.1, 0.0, ctypes.byref(out)) == binding.PF_EINVAL
    assert not out.value


def test_create_rejects_bad_model_and_split(L):
    out = ctypes.c_void_p()
    flags = (ctypes.c_uint8 * 25)()
    for model, split in ((5, 0), (0, 2), (0, -1)):
        mesh = binding.Mesh(4, 4, 1.0, 1.0, None, ctypes.addressof(flags), 0, 0, 1, 0, model,
                            0.0, split)
        assert L.pf_create(ctypes.byref(mesh), 210.0, 0.3, 1e-3, 0.1, 0.0,
                           ctypes.byref(out)) == binding.PF_EINVAL
        assert not out.value


def test_footprint_of_the_spectral_split(L):
    # the spectral split adds per-point stress and tangent (3 + 6 doubles per point) and the
    # nodal stencil of the tangent (36 values per node, FP64 and, in FP32-IR, FP32); every
    # array of the context's slab starts on a 256-byte boundary
    nx, ny = 30, 20
    nn, nq = (nx + 1) * (ny + 1), 4 * nx * ny

    def al(b):
        return (b + 255) // 256 * 256
    for prec, extra in ((binding.FP64, 0), (binding.FP32_IR, al(36 * nn * 4))):
        vals = []
        for split in (binding.SPLIT_VD, binding.SPLIT_SPECTRAL):
            mesh = binding.Mesh(nx, ny, 1.0, 1.0, None, 1, 0, prec, 1, binding.PRECOND_GMG, 0,
                                0.0, split)
            vals.append(L.pf_footprint_bytes(ctypes.byref(mesh)))
        assert vals[1] - vals[0] == al(3 * nq * 8) + al(6 * nq * 8) + al(36 * nn * 8) + extra


def test_operator_calls_reject_an_unknown_split(L):
    g = binding.grid(4, 4, 0.25, 0.25)
    m = binding.material(210.0, 0.3, 2.7e-3, 0.03, 1e-9, 0)
    m.split = 3
    fake = ctypes.c_void_p(16)                  # never dereferenced: validation comes first
    assert L.pf_op_qp_energy(ctypes.byref(g), ctypes.byref(m), fake, fake, None, fake,
                             None) == binding.PF_EINVAL
    assert L.pf_op_elas_tangent_qp(ctypes.byref(g), ctypes.byref(m), fake, fake, fake,
                                   None) == binding.PF_EINVAL


def test_batch_entry_points_reject_bad_arguments(L):
    # no device work: argument checks come first
    assert L.pf_batch_create(None) == binding.PF_EINVAL
    assert L.pf_batch_attach(None, None) == binding.PF_EINVAL
    assert L.pf_batch_detach(None, None) == binding.PF_EINVAL
    assert L.pf_batch_load_step(None, 1, None, None, None, None, None, None) == binding.PF_EINVAL
    assert L.pf_batch_stats(None, None, None, None, None) == binding.PF_EINVAL
    L.pf_batch_destroy(None)
