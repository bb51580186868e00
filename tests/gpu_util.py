"""Helpers shared by the GPU tests: device arrays through torch, descriptors, checker setup."""
import numpy as np
import torch

from oracle import model, q1
from paper_2209_07969_gb300 import binding


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def stream():
    return torch.cuda.current_stream().cuda_stream


def setup(spec):
    """Checker grid/material and device-side descriptors for a specimen."""
    g = q1.Grid(spec.nx, spec.ny, spec.Lx, spec.Ly, spec.node_flags, spec.elem_active)
    m = model.material_from_E_nu(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    flags_d = dev(spec.node_flags.astype(np.uint8))
    active_d = dev(spec.elem_active.astype(np.uint8)) if not np.all(spec.elem_active) else None
    mask_d = torch.empty(g.nn, dtype=torch.uint8, device="cuda")
    binding.check(binding.lib().pf_op_dof_mask(
        spec.nx, spec.ny, flags_d.data_ptr(), active_d.data_ptr() if active_d is not None else None,
        mask_d.data_ptr(), stream()), "pf_op_dof_mask")
    gm = binding.grid(spec.nx, spec.ny, g.hx, g.hy,
                      active_d.data_ptr() if active_d is not None else None, mask_d.data_ptr())
    gfull = binding.grid(spec.nx, spec.ny, g.hx, g.hy,
                         active_d.data_ptr() if active_d is not None else None, None)
    mat = binding.material(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    keep = (flags_d, active_d, mask_d)
    return g, m, gm, gfull, mat, keep


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def masked_matrix(K, constrained):
    """K with constrained rows and columns zeroed (operator form of the free block)."""
    free = (~constrained).astype(float)
    import scipy.sparse as sp
    P = sp.diags(free)
    return P @ K @ P
