"""ctypes binding of libpf (C ABI in include/pf.h): argument marshalling only.

Every computation runs in the CUDA library.  ``lib()`` raises ``LibraryMissing`` when
libpf.so has not been built; nothing here falls back to another implementation.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpf.so")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ENOTCONV, PF_ECUDA, PF_ETIMEOUT, PF_EBUSY = range(7)
ST, S1, S2, S3 = 0, 1, 2, 3
SCHEMES = {"ST": ST, "standard": ST, "S1": S1, "S2": S2, "S3": S3}
FP64, FP32_IR = 0, 1
PRECOND_JACOBI, PRECOND_GMG = 0, 1
AT2_HISTORY, AT1_PENALTY = 0, 1
SPLIT_VD, SPLIT_SPECTRAL = 0, 1
F64, F32 = 0, 1


class LibraryMissing(RuntimeError):
    pass


class PfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("Lx", C.c_double), ("Ly", C.c_double),
                ("elem_active", C.c_void_p), ("node_flags", C.c_void_p), ("plane", C.c_int),
                ("precision", C.c_int), ("reaction_dir", C.c_int), ("precond", C.c_int),
                ("model", C.c_int), ("tol_ir", C.c_double), ("split", C.c_int)]


class Options(C.Structure):
    _fields_ = [("tol_nr", C.c_double), ("tol_lin", C.c_double), ("tol_inner", C.c_double),
                ("max_newton", C.c_int), ("max_stag", C.c_int), ("max_lin", C.c_int),
                ("max_refine", C.c_int), ("psi_crit", C.c_double), ("project", C.c_int),
                ("check_every", C.c_int), ("newton_forcing", C.c_double),
                ("device_loop", C.c_int)]


class StepResult(C.Structure):
    _fields_ = [("ubar", C.c_double), ("reaction", C.c_double), ("stag_residual", C.c_double),
                ("stag_iters", C.c_int), ("newton_u", C.c_int), ("lin_u", C.c_int),
                ("lin_d", C.c_int), ("d_solves", C.c_int), ("refine_steps", C.c_int),
                ("converged", C.c_int), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("strip_rows", C.c_int), ("coarse_nodes", C.c_int),
                ("apply_us", C.c_double * 3), ("vcycle_us", C.c_double * 3)]

    def as_dict(self):
        return {"strip_rows": self.strip_rows, "coarse_nodes": self.coarse_nodes,
                "apply_us": list(self.apply_us), "vcycle_us": list(self.vcycle_us)}


class Request(C.Structure):
    _fields_ = [("mesh", Mesh), ("E", C.c_double), ("nu", C.c_double), ("Gc", C.c_double),
                ("l", C.c_double), ("k_res", C.c_double), ("increments", C.c_void_p),
                ("n_steps", C.c_int), ("scheme", C.c_int), ("tol", C.c_double),
                ("options", C.c_void_p)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("steps_done", C.c_int),
                ("steps_converged", C.c_int), ("admit_seq", C.c_int64),
                ("footprint", C.c_size_t), ("queue_ms", C.c_double), ("path_ms", C.c_double),
                ("step_ms_p50", C.c_double), ("step_ms_p99", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("hx", C.c_double), ("hy", C.c_double),
                ("elem_active", C.c_void_p), ("dof_mask", C.c_void_p)]


class Material(C.Structure):
    _fields_ = [("mu", C.c_double), ("K", C.c_double), ("cdim", C.c_double),
                ("eta", C.c_double), ("Gc", C.c_double), ("l", C.c_double), ("split", C.c_int)]


_LIB = None
P = C.c_void_p
I = C.c_int
D = C.c_double
S = C.c_int  # pf_status

_PROTOS = {
    "pf_default_options": (None, [C.POINTER(Options)]),
    "pf_status_string": (C.c_char_p, [I]),
    "pf_material_make": (S, [D, D, D, D, D, I, C.POINTER(Material)]),
    "pf_create": (S, [C.POINTER(Mesh), D, D, D, D, D, C.POINTER(P)]),
    "pf_footprint_bytes": (C.c_size_t, [C.POINTER(Mesh)]),
    "pf_set_options": (S, [P, C.POINTER(Options)]),
    "pf_get_options": (S, [P, C.POINTER(Options)]),
    "pf_load_step": (S, [P, D, I, D, C.POINTER(StepResult)]),
    "pf_get_fields": (S, [P, P, P, P]),
    "pf_set_fields": (S, [P, P, P, P, D]),
    "pf_state_size": (C.c_size_t, [P]),
    "pf_get_state": (S, [P, P, C.c_size_t]),
    "pf_set_state": (S, [P, P, C.c_size_t]),
    "pf_sizes": (S, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pf_launch_count": (C.c_int64, [P]),
    "pf_profile": (S, [P, P, I, I]),
    "pf_last_error": (C.c_char_p, [P]),
    "pf_destroy": (None, [P]),
    "pf_autotune": (S, [P, C.POINTER(Tuning)]),
    "pf_get_tuning": (S, [P, C.POINTER(Tuning)]),
    "pf_batch_create": (S, [C.POINTER(P)]),
    "pf_batch_attach": (S, [P, P]),
    "pf_batch_detach": (S, [P, P]),
    "pf_batch_load_step": (S, [P, I, P, P, P, P, P, P]),
    "pf_batch_stats": (S, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                           C.POINTER(C.c_int64), C.POINTER(I)]),
    "pf_batch_destroy": (None, [P]),
    "pf_server_create": (S, [C.c_size_t, I, C.POINTER(P)]),
    "pf_server_submit": (S, [P, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "pf_server_poll": (S, [P, C.c_int64, C.POINTER(RequestInfo), P, P]),
    "pf_server_drain": (S, [P, D]),
    "pf_server_stats": (S, [P, C.POINTER(C.c_size_t), C.POINTER(I)]),
    "pf_server_cancel": (S, [P, C.c_int64]),
    "pf_server_pause": (S, [P, I]),
    "pf_server_release": (S, [P, C.c_int64]),
    "pf_server_destroy": (None, [P]),
    "pf_op_dof_mask": (S, [I, I, P, P, P, P]),
    "pf_op_elas_residual": (S, [C.POINTER(Grid), C.POINTER(Material), P, P, P, P, P]),
    "pf_op_elas_apply": (S, [C.POINTER(Grid), C.POINTER(Material), I, P, P, P, P, P]),
    "pf_op_elas_diag": (S, [C.POINTER(Grid), C.POINTER(Material), I, P, P, P, P]),
    "pf_op_elas_tangent_qp": (S, [C.POINTER(Grid), C.POINTER(Material), P, P, P, P]),
    "pf_op_elas_apply_qp": (S, [C.POINTER(Grid), I, P, P, P, P]),
    "pf_op_damage_apply": (S, [C.POINTER(Grid), I, P, D, P, P, P]),
    "pf_op_damage_diag": (S, [C.POINTER(Grid), I, P, D, P, P]),
    "pf_op_damage_rhs": (S, [C.POINTER(Grid), P, P, P]),
    "pf_op_qp_energy": (S, [C.POINTER(Grid), C.POINTER(Material), P, P, P, P, P]),
    "pf_op_fs_coeff": (S, [C.POINTER(Grid), C.POINTER(Material), I, D, P, P, P, P, P, P]),
    "pf_op_fs_predict": (S, [C.POINTER(Grid), C.POINTER(Material), I, P, P, P, P, P, P, P]),
    "pf_op_reaction": (S, [C.POINTER(Grid), P, P, I, C.POINTER(D), P]),
    "pf_op_stag_residual": (S, [C.POINTER(Grid), C.POINTER(Material), P, P, P, C.POINTER(D), P]),
    "pf_op_stag_residual_noalloc": (S, [C.POINTER(Grid), C.POINTER(Material), P, P, P,
                                        C.POINTER(D), P]),
}
NOALLOC_MAX_DOUBLES = 1500000


def lib():
    """Load libpf.so (built by paper_2209_07969_gb300.build); raise if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing(f"{LIB_PATH} not built; run python -m paper_2209_07969_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status, what="libpf call", ctx=None):
    if status != PF_OK:
        msg = what
        if ctx:
            msg += ": " + lib().pf_last_error(ctx).decode()
        raise PfError(status, msg)


def default_options():
    o = Options()
    lib().pf_default_options(C.byref(o))
    return o


def material(E, nu, Gc, l, k_res, plane=0, split=SPLIT_VD):
    m = Material()
    check(lib().pf_material_make(E, nu, Gc, l, k_res, plane, C.byref(m)), "pf_material_make")
    m.split = split
    return m


def grid(nx, ny, hx, hy, elem_active_ptr=None, dof_mask_ptr=None):
    return Grid(nx, ny, hx, hy, elem_active_ptr, dof_mask_ptr)


def footprint_bytes(spec, precision=FP64, precond=PRECOND_JACOBI, model=AT2_HISTORY,
                    split=SPLIT_VD):
    """Device bytes pf_create would allocate for the specimen (admission control)."""
    active = None if spec.elem_active is None or np.all(spec.elem_active) else 1
    mesh = Mesh(spec.nx, spec.ny, spec.Lx, spec.Ly, active, 1, spec.plane, precision,
                spec.reaction_dir, precond, model, 0.0, split)
    return int(lib().pf_footprint_bytes(C.byref(mesh)))


class Simulation:
    """One fracture simulation resident on the current CUDA device (pf_create)."""

    def __init__(self, spec, precision=FP64, precond=PRECOND_JACOBI, options=None,
                 model=AT2_HISTORY, tol_ir=0.01, split=SPLIT_VD):
        self.spec = spec
        self._flags = np.ascontiguousarray(spec.node_flags, dtype=np.uint8)
        self._active = None
        if spec.elem_active is not None and not np.all(spec.elem_active):
            self._active = np.ascontiguousarray(spec.elem_active, dtype=np.uint8)
        mesh = Mesh(spec.nx, spec.ny, spec.Lx, spec.Ly,
                    self._active.ctypes.data if self._active is not None else None,
                    self._flags.ctypes.data, spec.plane, precision, spec.reaction_dir, precond,
                    model, tol_ir, split)
        ctx = P()
        check(lib().pf_create(C.byref(mesh), spec.E, spec.nu, spec.Gc, spec.l, spec.eta,
                              C.byref(ctx)), "pf_create")
        self.ctx = ctx
        self.nn = (spec.nx + 1) * (spec.ny + 1)
        self.nq = 4 * spec.nx * spec.ny
        if options is not None:
            self.set_options(**options)

    def set_options(self, **kw):
        o = Options()
        check(lib().pf_get_options(self.ctx, C.byref(o)), "pf_get_options", self.ctx)
        for k, v in kw.items():
            setattr(o, k, v)
        check(lib().pf_set_options(self.ctx, C.byref(o)), "pf_set_options", self.ctx)

    def load_step(self, d_ubar, scheme=ST, tol=1e-6, raise_on_notconv=False):
        r = StepResult()
        s = lib().pf_load_step(self.ctx, float(d_ubar), int(scheme), float(tol), C.byref(r))
        if s not in (PF_OK, PF_ENOTCONV) or (raise_on_notconv and s != PF_OK):
            check(s, "pf_load_step", self.ctx)
        out = r.as_dict()
        out["status"] = s
        return out

    def fields(self):
        u = np.empty(2 * self.nn)
        d = np.empty(self.nn)
        H = np.empty(self.nq)
        check(lib().pf_get_fields(self.ctx, u.ctypes.data, d.ctypes.data, H.ctypes.data),
              "pf_get_fields", self.ctx)
        return u, d, H.reshape(-1, 4)

    def fields_into(self, u=None, d=None, H=None):
        """Copy the committed fields into caller-owned float64 arrays (any may be None);
        pinned host arrays make the copy asynchronous-capable."""
        ptr = lambda a: None if a is None else a.ctypes.data
        for a, n in ((u, 2 * self.nn), (d, self.nn), (H, self.nq)):
            if a is not None and (a.dtype != np.float64 or a.size != n or not a.flags.c_contiguous):
                raise ValueError("field buffer has the wrong size or type")
        check(lib().pf_get_fields(self.ctx, ptr(u), ptr(d), ptr(H)), "pf_get_fields", self.ctx)

    def set_fields(self, u, d, H, ubar):
        u = np.ascontiguousarray(u, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        H = np.ascontiguousarray(H, dtype=np.float64)
        check(lib().pf_set_fields(self.ctx, u.ctypes.data, d.ctypes.data, H.ctypes.data,
                                  float(ubar)), "pf_set_fields", self.ctx)

    def get_state(self):
        n = lib().pf_state_size(self.ctx)
        buf = np.empty(n, dtype=np.uint8)
        check(lib().pf_get_state(self.ctx, buf.ctypes.data, n), "pf_get_state", self.ctx)
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        check(lib().pf_set_state(self.ctx, buf.ctypes.data, buf.size), "pf_set_state", self.ctx)

    PHASES = ("u_setup", "u_solve", "u_resid", "d_setup", "d_solve", "stag", "total")

    def profile(self, reset=False):
        ms = np.zeros(8)
        check(lib().pf_profile(self.ctx, ms.ctypes.data, 8, int(reset)), "pf_profile", self.ctx)
        return dict(zip(self.PHASES, ms[:7].tolist()))

    def autotune(self):
        """Time the launch-shape candidates on this grid and keep the fastest
        (pf_autotune); returns the choice and the timings."""
        t = Tuning()
        check(lib().pf_autotune(self.ctx, C.byref(t)), "pf_autotune", self.ctx)
        return t.as_dict()

    def tuning(self):
        t = Tuning()
        check(lib().pf_get_tuning(self.ctx, C.byref(t)), "pf_get_tuning", self.ctx)
        return t.as_dict()

    def launches(self):
        return int(lib().pf_launch_count(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            lib().pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Simulations advanced together with batched Krylov solves (pf_batch_*, include/pf.h).

    ``step(increments, schemes, tols)`` runs one load step of every member on its own host
    thread inside the library; their FP32 multigrid solves share kernel launches."""

    def __init__(self, sims=()):
        p = P()
        check(lib().pf_batch_create(C.byref(p)), "pf_batch_create")
        self.b = p
        self.sims = []
        for sim in sims:
            self.attach(sim)

    def attach(self, sim):
        check(lib().pf_batch_attach(self.b, sim.ctx), "pf_batch_attach", sim.ctx)
        self.sims.append(sim)

    def detach(self, sim):
        check(lib().pf_batch_detach(self.b, sim.ctx), "pf_batch_detach", sim.ctx)
        self.sims.remove(sim)

    def step(self, increments, schemes, tols, sims=None):
        """One load step of each simulation (default: all members); returns the per-
        simulation result dicts with their 'status'."""
        sims = self.sims if sims is None else list(sims)
        n = len(sims)
        ctxs = (P * n)(*[s.ctx for s in sims])
        du = np.ascontiguousarray(np.broadcast_to(increments, (n,)), dtype=np.float64)
        sc = np.ascontiguousarray(np.broadcast_to(schemes, (n,)), dtype=np.int32)
        tl = np.ascontiguousarray(np.broadcast_to(tols, (n,)), dtype=np.float64)
        res = (StepResult * n)()
        st = np.zeros(n, dtype=np.int32)
        s = lib().pf_batch_load_step(self.b, n, ctxs, du.ctypes.data, sc.ctypes.data,
                                     tl.ctypes.data, C.addressof(res), st.ctypes.data)
        if s not in (PF_OK, PF_ENOTCONV):
            bad = [i for i in range(n) if st[i] not in (PF_OK, PF_ENOTCONV)]
            check(s, "pf_batch_load_step", sims[bad[0]].ctx if bad else None)
        out = []
        for i in range(n):
            d = res[i].as_dict()
            d["status"] = int(st[i])
            out.append(d)
        return out

    def stats(self):
        la, so, gr, mg = C.c_int64(), C.c_int64(), C.c_int64(), I()
        check(lib().pf_batch_stats(self.b, C.byref(la), C.byref(so), C.byref(gr), C.byref(mg)),
              "pf_batch_stats")
        return {"launches": la.value, "solves": so.value, "groups": gr.value,
                "max_group": mg.value}

    def close(self):
        if self.b:
            lib().pf_batch_destroy(self.b)
            self.b = None
            self.sims = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NativeServer:
    """The library's request server (pf_server_*, include/pf.h): FIFO admission by device
    footprint, one host worker thread per slot, each simulation on its own stream."""

    def __init__(self, hbm_budget, slots):
        p = P()
        check(lib().pf_server_create(int(hbm_budget), int(slots), C.byref(p)),
              "pf_server_create")
        self.s = p
        self._steps = {}

    def submit(self, spec, scheme=ST, tol=1e-5, precision=FP64, precond=PRECOND_JACOBI,
               model=AT2_HISTORY, tol_ir=0.01, split=SPLIT_VD, options=None):
        flags = np.ascontiguousarray(spec.node_flags, dtype=np.uint8)
        active = None
        if spec.elem_active is not None and not np.all(spec.elem_active):
            active = np.ascontiguousarray(spec.elem_active, dtype=np.uint8)
        inc = np.ascontiguousarray(spec.increments, dtype=np.float64)
        mesh = Mesh(spec.nx, spec.ny, spec.Lx, spec.Ly,
                    active.ctypes.data if active is not None else None, flags.ctypes.data,
                    spec.plane, precision, spec.reaction_dir, precond, model, tol_ir, split)
        opt = None
        if options:
            opt = default_options()
            for k, v in options.items():
                setattr(opt, k, v)
        req = Request(mesh, spec.E, spec.nu, spec.Gc, spec.l, spec.eta, inc.ctypes.data,
                      len(inc), int(scheme), float(tol),
                      C.addressof(opt) if opt is not None else None)
        rid = C.c_int64()
        check(lib().pf_server_submit(self.s, C.byref(req), C.byref(rid)), "pf_server_submit")
        self._steps[rid.value] = len(inc)
        return rid.value

    def poll(self, rid):
        if rid not in self._steps:
            check(PF_EINVAL, f"pf_server_poll: unknown request {rid}")
        n = self._steps[rid]
        info = RequestInfo()
        reactions = np.zeros(n)
        iters = np.zeros(n, dtype=np.int32)
        check(lib().pf_server_poll(self.s, rid, C.byref(info), reactions.ctypes.data,
                                   iters.ctypes.data), "pf_server_poll")
        out = info.as_dict()
        out["reactions"] = reactions[:info.steps_done]
        out["stag_iters"] = iters[:info.steps_done]
        return out

    def drain(self, timeout=-1.0):
        """True when every submitted request has finished within ``timeout`` seconds."""
        s = lib().pf_server_drain(self.s, float(timeout))
        if s not in (PF_OK, PF_ETIMEOUT):
            check(s, "pf_server_drain")
        return s == PF_OK

    def stats(self):
        b = C.c_size_t()
        r = I()
        check(lib().pf_server_stats(self.s, C.byref(b), C.byref(r)), "pf_server_stats")
        return {"peak_bytes": b.value, "peak_running": r.value}

    def cancel(self, rid):
        check(lib().pf_server_cancel(self.s, rid), "pf_server_cancel")

    def release(self, rid):
        """Free a finished request's record (its id becomes unknown)."""
        check(lib().pf_server_release(self.s, rid), "pf_server_release")
        self._steps.pop(rid, None)

    def pause(self, paused=True):
        check(lib().pf_server_pause(self.s, 1 if paused else 0), "pf_server_pause")

    def close(self):
        if self.s:
            lib().pf_server_destroy(self.s)
            self.s = None
