"""The allocation-free staggered residual against the allocating one (GPU).

pf_op_stag_residual_noalloc exists for callers that cannot allocate device memory per
call: code whose device memory belongs to another allocator with a fixed budget, and
code that must not stall the device (cudaMalloc/cudaFree can synchronise it).  It keeps
its scratch in a static device array shared by all calls.  This file is collected last
so that a run stopping at the first failure has run every other test before it; it also
passes alone in a fresh process (the first call on the device resolves the scratch).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2209_07969_gb300 import binding, specimens as S
from tests.gpu_util import dev, setup, stream

pytestmark = pytest.mark.gpu


def _residuals(L, case, fn):
    out = binding.D()
    binding.check(fn(case["gm"], case["mat"], case["u"].data_ptr(), case["d"].data_ptr(),
                     case["H"].data_ptr(), ctypes.byref(out), stream()))
    return out.value


def _case(spec, seed, scale):
    g, m, gm, gfull, mat, keep = setup(spec)
    u, d, H = S.random_state(spec, seed=seed)
    cd = g.d_constrained()
    d[cd] = g.d_dirichlet_values()[cd]
    return dict(gm=gm, mat=mat, keep=keep, u=dev(u * scale), d=dev(d), H=dev(H.ravel()))


def test_noalloc_matches_allocating_twice_in_a_row(gpu):
    L = binding.lib()
    # two different inputs (sizes, states) one after the other: the shared scratch keeps
    # the first call's contents, which must not leak into the second result
    cases = [_case(S.tensile(64), 3, 1.0), _case(S.tensile(200, l=0.01), 4, 3.0)]
    for c in cases:
        ref = _residuals(L, c, L.pf_op_stag_residual)
        got = _residuals(L, c, L.pf_op_stag_residual_noalloc)
        assert np.isfinite(ref) and ref > 0
        assert got == pytest.approx(ref, rel=1e-12)


def test_noalloc_rejects_grids_beyond_the_static_scratch(gpu):
    L = binding.lib()
    n = 400                                    # 2*Q + 3*N > PF_NOALLOC_MAX_DOUBLES
    assert 8 * n * n + 3 * (n + 1) ** 2 > binding.NOALLOC_MAX_DOUBLES
    g = binding.grid(n, n, 1.0 / n, 1.0 / n, None, None)
    mat = binding.material(210.0, 0.3, 2.7e-3, 0.01, 1e-9, 0)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = binding.D()
    st = L.pf_op_stag_residual_noalloc(g, mat, dummy.data_ptr(), dummy.data_ptr(),
                                       dummy.data_ptr(), ctypes.byref(out), stream())
    assert st == binding.PF_EINVAL
