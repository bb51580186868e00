#!/usr/bin/env python3
"""Benchmark of the staggered phase-field solver on the 512 x 512 tensile notched square.

Workload (tensile notched square, 512 x 512 Q1 elements, l = 0.0075 mm, 100 load steps to
6e-3 mm, staggered tolerance 1e-5 with up to 20,000 passes per load step; S1 fixed-stress
scheme, FP32 CG with FP64 refinement, geometric multigrid): a batch of B simulations of
that specimen (default 2), each on its own stream and host thread, or with --executor
batched through the batched executor (pf_batch_*: their FP32 multigrid solves share
kernel launches).

The timed region is one WHOLE load path of every simulation: the K bench steps split the
100 load steps into K consecutive chunks (one bench step = 100/K load steps of every
simulation, each load step one pass of every part of the method).  W warm-up steps run
the first W chunks on the same simulations, which are then reset to their initial state.
Reported metric: load paths/s = B whole paths / time.  The crack phase (steps ~81-87 at
this size, thousands of staggered passes) dominates the path.  Also reported: DOF.CG-
iterations/s, per-load-step latency percentiles, the end-to-end rate (a second whole path
through the public API with the increment read from pinned host memory and the phase
field copied back to pinned host memory every load step), the FP64 per-simulation form
against the mixed-precision form on whole paths of the same specimen at 128 x 128 with
the same l/h (same run), the roofline of the FP32 tangent apply, and the FP64 CPU checker
on a bounded sample scaled by this run's pass and Newton counts.

--impl reference times the FP64 CPU checker (oracle/) on a bounded sample of the same
workload: each step is one exact phase-field solve (assembly + sparse LU) of load step 1
on the 512 x 512 grid; a load path needs PASSES_PER_PATH staggered passes of at least one
such solve each (and displacement solves, several times more expensive), so
1 / (PASSES_PER_PATH x sample time) is an upper bound of the checker's load paths/s.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STEPS_PER_PATH = 100
PASSES_PER_PATH = 8511   # staggered passes of the S1 FP32-IR path at 512 x 512 (measured)
METRIC = "load paths/s"
UNIT = "load paths/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=2)
    p.add_argument("--executor", default="streams", choices=["batched", "streams"],
                   help="batched: pf_batch (shared launches); streams: one stream per simulation")
    p.add_argument("--max-stag", type=int, default=20000)
    p.add_argument("--no-tune", action="store_true", help="skip pf_autotune")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end whole path")
    p.add_argument("--no-fp64", action="store_true",
                   help="skip the FP64-form comparison on the 128 x 128 path")
    p.add_argument("--grid", type=int, default=512)
    p.add_argument("--scheme", default="S1")
    p.add_argument("--full-path", action="store_true",
                   help="whole paths of the workload in FP32-IR and in FP64, one simulation "
                        "per --scheme (comma list): the full-size FP64-form comparison")
    p.add_argument("--kernel", default=None, choices=["elas"],
                   help="time one operator kernel on the --grid tensile mesh and exit")
    p.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--serve", action="store_true",
                   help="served-batch mode: a seeded mix of full load paths through the "
                        "continuous-batching server; prints served paths/s and p50/p99 latencies")
    p.add_argument("--requests", type=int, default=24)
    p.add_argument("--grids", default="64,128")
    p.add_argument("--rate", type=float, default=4.0, help="Poisson arrival rate, requests/s")
    p.add_argument("--slots", type=int, default=8)
    p.add_argument("--split", default="vd", choices=["vd", "spectral"],
                   help="energy split (Sec. 2): vd (the workload's) or spectral")
    p.add_argument("--host-loop", action="store_true",
                   help="host-checked Krylov batches instead of device-side loops (same "
                        "kernels; for profilers that cannot see inside conditional graph nodes)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload_name(args, l):
    """The workload as both arms name it in `config`."""
    return (f"tensile notched square {args.grid}x{args.grid} Q1, l={l:g} mm, 100 load steps to "
            f"6e-3 mm, TOL_ST 1e-5 (up to {args.max_stag} passes per step), scheme "
            f"{args.scheme}; whole load paths")


def workload(grid):
    from paper_2209_07969_gb300 import specimens as S
    return S.tensile(grid, l=0.0075 if grid == 512 else 0.0075 * 512 / grid,
                     steps=STEPS_PER_PATH, u_max=6e-3)


# ---- clocks ------------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- checker sample (CPU) ---------------------------------------------------------------
def oracle_sample(grid, split=0):
    """One exact phase-field solve of load step 1 (assembly + LU); returns seconds."""
    import numpy as np
    from oracle import model, q1, staggered as stg
    sp = workload(grid)
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane, split)
    j = np.arange(g.nn) // (g.nx + 1)
    u = np.stack([np.zeros(g.nn), sp.increments[0] * j / g.ny], 1).ravel()
    t0 = time.perf_counter()
    H = stg.psi_plus_qp(g, u, m)
    stg.d_step_standard(g, m, H)
    return time.perf_counter() - t0


def oracle_u_sample(grid, split=0):
    """One exact Newton linear solve for u of load step 1 (residual, assembly, SuperLU);
    returns seconds."""
    import numpy as np
    from oracle import model, q1, staggered as stg
    sp = workload(grid)
    g = q1.Grid(sp.nx, sp.ny, sp.Lx, sp.Ly, sp.node_flags, sp.elem_active)
    m = model.material_from_E_nu(sp.E, sp.nu, sp.Gc, sp.l, sp.eta, sp.plane, split)
    u = g.u_dirichlet_values(sp.increments[0])
    d = g.d_dirichlet_values()
    t0 = time.perf_counter()
    stg.solve_u(g, m, u, d, stg.Options(max_newton=1))
    return time.perf_counter() - t0


def cpu_baseline(grid, split=0, newton_per_path=None, dsolves_per_path=None):
    """The checker on a bounded sample of the workload: one exact u Newton solve and one
    exact phase-field solve of load step 1, scaled to a whole path by the Newton
    corrections and phase-field solves the path took in this run (the checker runs the
    same iteration: its pass counts equal the GPU path's, checked at 128 x 128)."""
    t_u = oracle_u_sample(grid, split)
    t_d = oracle_sample(grid, split)
    if newton_per_path is None:
        newton_per_path, dsolves_per_path = 2 * STEPS_PER_PATH, 2 * STEPS_PER_PATH
    path = newton_per_path * t_u + dsolves_per_path * t_d
    return {"value": 1.0 / path, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"one exact Newton solve for u ({t_u:.1f} s) and one exact phase-field "
                       f"solve ({t_d:.1f} s) of load step 1 on the {grid}x{grid} grid (assembly + "
                       f"SuperLU, single-threaded); a whole path takes {newton_per_path:.0f} u "
                       f"Newton corrections and {dsolves_per_path:.0f} phase-field solves "
                       f"(this run's counts): {path:.3g} s"),
            "host_cpus": os.cpu_count()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(args.grid)
    ts = [oracle_sample(args.grid) for _ in range(args.steps)]
    total = sum(ts)
    value = args.steps / (PASSES_PER_PATH * total)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, workload(args.grid).l),
                       "form": "FP64 CPU checker (sparse LU), sampled"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step one exact phase-field solve (assembly + "
                                       "SuperLU) of load step 1, the least work of one "
                                       f"staggered pass; a path takes {PASSES_PER_PATH} passes; "
                                       f"value = steps/({PASSES_PER_PATH} x time), an upper "
                                       "bound"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU arm --------------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def profiled_traffic(grid=512):
    """DRAM bytes per launch of the roofline kernel from the committed ncu summary (taken
    on the 512 x 512 grid), or None for another grid or when the operator source changed
    since the counters were taken."""
    if grid != 512:
        return None
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_elas_strip_f32_512_traffic.md")
    src = os.path.join(ROOT, "paper_2209_07969_gb300", "csrc", "pf_ops.cu")
    try:
        fields = dict(l.split(":", 1) for l in open(prof) if l.startswith(("traffic_bytes_per_launch:", "pf_ops_sha256_16:")))
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None
    if fields.get("pf_ops_sha256_16", "").strip() != digest:
        return None
    return float(fields["traffic_bytes_per_launch"])


def kernel_roofline(spec, sims, peak_gbs, reps=30):
    """Time the FP32 matrix-free elasticity tangent apply (the operator inside every fused
    fine-level stage of the multigrid PCG) on the workload grid with CUDA events on the
    launching stream, flushing L2 before each launch.  Algorithmic bytes per node: x (8) +
    y (8) + d (4) + DOF mask (1) + tension byte (1 per element, ~1 per node) = 22.  By
    launch-list share the single-CTA coarse cycle is the largest single kernel; every
    kernel of the iteration is latency-bound at this size."""
    import numpy as np
    import torch
    from paper_2209_07969_gb300 import binding
    L = binding.lib()
    nn = (spec.nx + 1) * (spec.ny + 1)
    ne = spec.nx * spec.ny
    dev = torch.device("cuda")
    flags = torch.from_numpy(spec.node_flags.astype(np.uint8)).to(dev)
    mask = torch.empty(nn, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    binding.check(L.pf_op_dof_mask(spec.nx, spec.ny, flags.data_ptr(), None, mask.data_ptr(),
                                   st.cuda_stream))
    g = binding.grid(spec.nx, spec.ny, spec.Lx / spec.nx, spec.Ly / spec.ny, None, mask.data_ptr())
    mat = binding.material(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    gen = torch.Generator(device="cpu").manual_seed(0)
    d = (torch.rand(nn, generator=gen) * 0.5).to(dev, torch.float32)
    x = torch.randn(2 * nn, generator=gen).to(dev, torch.float32)
    y = torch.empty_like(x)
    tens = torch.randint(0, 16, (ne,), generator=gen, dtype=torch.uint8).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    times = []
    for k in range(reps + 3):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        binding.check(L.pf_op_elas_apply(g, mat, binding.F32, d.data_ptr(), tens.data_ptr(),
                                         x.data_ptr(), y.data_ptr(), st.cuda_stream))
        e1.record(st)
        e1.synchronize()
        if k >= 3:
            times.append(e0.elapsed_time(e1) * 1e-3)
    t = statistics.mean(times)
    bytes_ = 22.0 * nn
    ach = bytes_ / t / 1e9
    return {"kernel": "k_elas_strip<float,2> (matrix-free Q1 elasticity tangent, FP32)",
            "bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
            "frac": ach / peak_gbs, "traffic": profiled_traffic(spec.nx),
            "traffic_source": "carried over from the committed ncu capture "
                              "(profiles/k_elas_strip_f32_512_traffic.md); null when the "
                              "operator source differs from the captured one",
            "algorithmic_bytes": bytes_,
            "launch_us": t * 1e6, "l2": "flushed before each launch",
            "share_note": "launch-list shares of the whole-path bench command "
                          "(profiles/bench_tensile128_launch_list.md): single-CTA coarse "
                          "cycle 27%, fused fine-level stages 35%, grid-level stencil "
                          "kernels 30%; all latency-bound"}


def chunks(K):
    """Load-step bounds of the K bench steps that make up one whole path."""
    K = max(1, min(K, STEPS_PER_PATH))
    return [round(k * STEPS_PER_PATH / K) for k in range(K + 1)]


class Runner:
    """B simulations of one specimen and the executor that advances them."""

    def __init__(self, spec, B, executor, split, max_stag, host_loop=False, scheme=1,
                 precision=None, tune=False):
        from paper_2209_07969_gb300 import binding
        self.binding = binding
        self.spec, self.B, self.scheme = spec, B, scheme
        prec = binding.FP32_IR if precision is None else precision
        self.sims = [binding.Simulation(spec, precision=prec, precond=binding.PRECOND_GMG,
                                        split=split) for _ in range(B)]
        for s in self.sims:
            s.set_options(max_stag=max_stag, device_loop=0 if host_loop else 1)
        # launch shapes timed on this grid (pf_autotune) before the first load step
        self.tuning = [s.autotune() for s in self.sims] if tune else None
        self.batch = binding.Batch(self.sims) if executor == "batched" else None
        self.init = [s.get_state() for s in self.sims]
        self.results = [[] for _ in range(B)]

    def reset(self):
        for i, s in enumerate(self.sims):
            s.set_state(self.init[i])
        self.results = [[] for _ in range(self.B)]

    def run(self, k0, k1, inc_host=None, d_host=None):
        """Load steps k0..k1-1 of every simulation.  With host buffers (end-to-end form)
        the increment is read from pinned host memory and d copied back every step."""
        incs = self.spec.increments
        sc = self.scheme

        def inc(i, k):
            if inc_host is None:
                return float(incs[k])
            inc_host[i][0] = incs[k]
            return float(inc_host[i][0])

        if self.batch is not None:
            for k in range(k0, k1):
                res = self.batch.step([inc(i, k) for i in range(self.B)], sc, 1e-5)
                for i, r in enumerate(res):
                    self.results[i].append(r)
                    if d_host is not None:
                        self.sims[i].fields_into(d=d_host[i])
            return

        def adv(i):
            for k in range(k0, k1):
                r = self.sims[i].load_step(inc(i, k), sc, 1e-5)
                self.results[i].append(r)
                if d_host is not None:
                    self.sims[i].fields_into(d=d_host[i])
        th = [threading.Thread(target=adv, args=(i,)) for i in range(self.B)]
        for t in th:
            t.start()
        for t in th:
            t.join()

    def launches(self):
        n = sum(s.launches() for s in self.sims)
        return n + (self.batch.stats()["launches"] if self.batch is not None else 0)

    def close(self):
        if self.batch is not None:
            self.batch.close()
        for s in self.sims:
            s.close()


def fp64_form_comparison(split):
    """Whole paths of the same specimen at 128 x 128 (l = 0.03 mm, the l/h of the 512 x 512
    workload): the mixed-precision form against the plain per-simulation FP64 form, both
    to TOL_ST 1e-5 on every load step, timed in this run."""
    import numpy as np
    import torch
    from paper_2209_07969_gb300 import binding
    spec = workload(128)
    out = {}
    for name, prec in (("fp32_ir", binding.FP32_IR), ("fp64", binding.FP64)):
        r = Runner(spec, 1, "streams", split, 20000, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r.run(0, STEPS_PER_PATH)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        F = np.array([x["reaction"] for x in r.results[0]])
        out[name] = {"path_s": dt, "load_paths_per_s": 1.0 / dt, "peak_reaction": float(F.max()),
                     "passes": int(sum(x["stag_iters"] for x in r.results[0])),
                     "converged_steps": int(sum(x["converged"] for x in r.results[0]))}
        d = r.sims[0].fields()[1]
        out[name]["_d"] = d
        r.close()
    dd = out["fp32_ir"].pop("_d") - out["fp64"].pop("_d")
    pk = out["fp64"]["peak_reaction"]
    out["speedup"] = out["fp32_ir"]["load_paths_per_s"] / out["fp64"]["load_paths_per_s"]
    out["peak_rel_diff"] = abs(out["fp32_ir"]["peak_reaction"] - pk) / pk
    out["final_d_rms_diff"] = float(np.sqrt(np.mean(dd ** 2)))
    out["workload"] = ("tensile notched square 128x128, l=0.03 mm, 100 load steps to 6e-3 mm, "
                       "TOL_ST 1e-5, S1, GMG, one simulation per form, whole paths")
    return out


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2209_07969_gb300 import binding, build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    binding.lib()
    spec = workload(args.grid)
    split = binding.SPLIT_SPECTRAL if args.split == "spectral" else binding.SPLIT_VD
    B = args.batch
    R = Runner(spec, B, args.executor, split, args.max_stag, args.host_loop,
               binding.SCHEMES[args.scheme], tune=not args.no_tune and split == binding.SPLIT_VD)
    bounds = chunks(args.steps)
    K = len(bounds) - 1
    nn = (spec.nx + 1) * (spec.ny + 1)
    # warm-up: the first W chunks of the path, then back to the initial state
    R.run(0, bounds[min(args.warmup, K)])
    R.reset()
    launches0 = R.launches()
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    t0 = time.perf_counter()
    for k in range(K):
        R.run(bounds[k], bounds[k + 1])
    torch.cuda.synchronize()
    e1.record()
    e1.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    T = max(e0.elapsed_time(e1) * 1e-3, wall)
    if world > 1:
        tt = torch.tensor([T], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        T = float(tt.item())
    launches = R.launches() - launches0
    results = R.results
    work = sum(r["lin_u"] * 2 * nn + r["lin_d"] * nn for rs in results for r in rs)
    lat = sorted(r["ms"] for rs in results for r in rs)
    value = B * world / T
    conv = sum(r["converged"] for rs in results for r in rs)
    passes = sum(r["stag_iters"] for rs in results for r in rs)
    newton = sum(r["newton_u"] for rs in results for r in rs)
    dsolves = sum(r["d_solves"] for rs in results for r in rs)
    F0 = np.array([r["reaction"] for r in results[0]])
    # end to end: a second whole path through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        R.reset()
        inc_host = [torch.empty(1, dtype=torch.float64, pin_memory=True).numpy() for _ in range(B)]
        d_host = [torch.empty(nn, dtype=torch.float64, pin_memory=True).numpy() for _ in range(B)]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for k in range(K):
            R.run(bounds[k], bounds[k + 1], inc_host, d_host)
        torch.cuda.synchronize()
        T_e2e = time.perf_counter() - t1
        e2e = {"value": B * world / T_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 8 * B * (bounds[1] - bounds[0]),
               "d2h_bytes_per_step": (nn * 8 + 88) * B * (bounds[1] - bounds[0])}
    out = None
    if rank == 0:
        pk, which = peaks()
        if split == binding.SPLIT_VD:
            roof = kernel_roofline(spec, R.sims, pk.get("hbm_gbs", 6800.0))
            roof["peak_source"] = which
        else:   # the matrix-free VD kernel is not on this path
            roof = {"bound": "hbm", "achieved": None, "peak": pk.get("hbm_gbs", 6800.0),
                    "unit": "GB/s", "frac": None, "traffic": None,
                    "note": "spectral split: u-solves apply the assembled stencil "
                            "(k_sp_apply, 161 B/node in FP32); not timed by this leg"}
        R.close()
        base = cpu_baseline(args.grid, split, newton / B, dsolves / B)
        fp64 = None if args.no_fp64 or split != binding.SPLIT_VD else fp64_form_comparison(split)
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": K, "warmup": args.warmup, "ms_per_step": 1e3 * T / K,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64", "data": "synthetic",
               "config": {"workload": workload_name(args, spec.l)
                                      + ("; spectral energy split" if split else ""),
                          "form": "FP32 CG + FP64 refinement, geometric multigrid",
                          "batch": B, "executor": args.executor,
                          "autotune": (R.tuning[0] if R.tuning else None),
                          "load_steps_per_bench_step": bounds[1] - bounds[0],
                          "l2": "working set per simulation ~0.2 GB; every load step reads "
                                "the operator data anew"},
               "whole_paths": B * world, "path_s": T,
               "converged_load_steps": conv, "load_steps": sum(len(rs) for rs in results),
               "staggered_passes": passes, "peak_reaction": float(F0.max()),
               "dof_cg_iters_per_s": work * world / T,
               "load_steps_per_s": B * world * STEPS_PER_PATH / T,
               "step_latency_ms": {"p50": lat[len(lat) // 2],
                                   "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
               "clocks": clk, "gpu_launches": launches,
               "roofline": roof, "cpu_baseline": base, "fp64_form": fp64}
        if e2e is not None:
            out["e2e"] = e2e
        print(json.dumps(out), flush=True)
    else:
        R.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_kernel(args):
    """Standalone timing of the matrix-free elasticity tangent apply (pf_op_elas_apply)
    on the --grid tensile mesh: 2 untimed launches, then --reps launches back to back
    between CUDA events on the launching stream (inputs resident, L2 not flushed)."""
    import numpy as np
    import torch
    from paper_2209_07969_gb300 import binding, build
    build.build()
    L = binding.lib()
    spec = workload(args.grid)
    nn, ne = (spec.nx + 1) * (spec.ny + 1), spec.nx * spec.ny
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    flags = torch.from_numpy(spec.node_flags.astype(np.uint8)).to(dev)
    mask = torch.empty(nn, dtype=torch.uint8, device=dev)
    binding.check(L.pf_op_dof_mask(spec.nx, spec.ny, flags.data_ptr(), None, mask.data_ptr(),
                                   st.cuda_stream))
    g = binding.grid(spec.nx, spec.ny, spec.Lx / spec.nx, spec.Ly / spec.ny, None, mask.data_ptr())
    mat = binding.material(spec.E, spec.nu, spec.Gc, spec.l, spec.eta, spec.plane)
    T, code = (torch.float32, binding.F32) if args.dtype == "f32" else (torch.float64, binding.F64)
    gen = torch.Generator(device="cpu").manual_seed(0)
    d = (torch.rand(nn, generator=gen) * 0.5).to(dev, T)
    x = torch.randn(2 * nn, generator=gen).to(dev, T)
    y = torch.empty_like(x)
    tens = torch.randint(0, 16, (ne,), generator=gen, dtype=torch.uint8).to(dev)

    def launch():
        binding.check(L.pf_op_elas_apply(g, mat, code, d.data_ptr(), tens.data_ptr(),
                                         x.data_ptr(), y.data_ptr(), st.cuda_stream))
    for _ in range(2):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.reps):
        launch()
    e1.record(st)
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / args.reps
    bpn = 22.0 if args.dtype == "f32" else 42.0
    print(json.dumps({"kernel": "pf_op_elas_apply", "grid": args.grid, "dtype": args.dtype,
                      "launch_us": t * 1e6, "algorithmic_GBps": bpn * nn / t / 1e9}), flush=True)


def run_full_path(args):
    """Complete load paths (all 100 steps) of the workload, one simulation per scheme."""
    from paper_2209_07969_gb300 import binding, build
    build.build()
    spec = workload(args.grid)
    for name in args.scheme.split(","):
        for prec in (binding.FP32_IR, binding.FP64):
            s = binding.Simulation(spec, precision=prec, precond=binding.PRECOND_GMG)
            s.set_options(max_stag=args.max_stag)
            t0 = time.perf_counter()
            passes = 0
            for du in spec.increments:
                r = s.load_step(du, binding.SCHEMES[name], 1e-5)
                passes += r["stag_iters"]
            dt = time.perf_counter() - t0
            print(json.dumps({"scheme": name, "precision": "fp32_ir" if prec else "fp64",
                              "path_s": dt, "load_paths_per_s": 1.0 / dt, "passes": passes}), flush=True)
            s.close()


def run_serve(args):
    """The served-batch workload at reduced grid sizes: requests (tensile or shear notched
    square, random material, scheme ST/S1/S2, full 100/150-step paths) arrive as a Poisson
    process and are admitted by the server by slot and HBM footprint; FP32 CG + FP64
    refinement, multigrid.  Reports completed load paths per second of wall time and
    p50/p99 latency per load step (device time) and per path (arrival to completion)."""
    import torch
    from paper_2209_07969_gb300 import binding, build, server, specimens as S
    build.build()
    torch.cuda.set_device(0)
    grids = tuple(int(g) for g in args.grids.split(","))
    mix = S.served_batch(args.requests, seed=0, rate_per_s=args.rate, grids=grids)
    reqs = [server.Request(sp, scheme=sch, precision=binding.FP32_IR,
                           precond=binding.PRECOND_GMG, tol=1e-5,
                           options={"max_stag": args.max_stag}) for _, sp, sch in mix]
    free, _ = torch.cuda.mem_get_info()
    srv = server.Server(hbm_budget=int(0.8 * free), slots=args.slots, device=0)
    t0 = time.perf_counter()
    for (t, _, _), r in zip(mix, reqs):
        wait = t0 + t - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        srv.submit(r)
    srv.drain()
    wall = time.perf_counter() - t0
    srv.close()
    res = srv.results
    done = [r for r in res.values() if r.ok]
    steps, paths = server.latency_percentiles(res)
    conv = sum(sum(r.converged) for r in done) / max(1, sum(len(r.converged) for r in done))
    line = {"mode": "serve", "metric": METRIC, "value": len(done) / wall, "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "served batch: tensile/shear notched squares, random "
                                   "E, nu, G_c, l in [2h, 4h], scheme ST/S1/S2, full paths "
                                   "(100/150 steps)",
                       "requests": args.requests, "grids": list(grids), "rate_per_s": args.rate,
                       "slots": args.slots, "seed": 0},
            "wall_s": wall, "completed": len(done), "failed": len(res) - len(done),
            "steps_converged_fraction": conv,
            "step_latency_ms": steps, "path_latency_s": paths,
            "queue_s_p50": float(statistics.median(r.queue_s for r in done)) if done else None,
            "peak_running": srv.peak_running, "peak_hbm_bytes": srv.peak_in_use}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.kernel:
        run_kernel(a)
    elif a.full_path:
        run_full_path(a)
    elif a.serve:
        run_serve(a)
    else:
        run_ours(a)
