"""A served mix of simulations gives, for every request, the result it gives alone (GPU).

Requests of different grids, materials, specimens and schemes arrive while others run;
the server admits them by slot and HBM footprint and their kernels overlap on the GPU.
The kernels are deterministic (no atomics, fixed reduction order), so every request's
reaction forces and final phase field match its stand-alone run bit for bit.
"""
import numpy as np
import pytest

from paper_2209_07969_gb300 import binding, server, specimens as S

pytestmark = pytest.mark.gpu


def _requests():
    mix = S.served_batch(8, seed=3, rate_per_s=50.0, grids=(16, 24, 32))
    reqs = []
    for k, (t, sp, scheme) in enumerate(mix):
        sp.increments = sp.increments[:5] * (len(sp.increments) / 5.0)  # 5 coarse steps
        prec = binding.FP32_IR if k % 2 == 0 else binding.FP64
        pc = binding.PRECOND_GMG if k % 3 else binding.PRECOND_JACOBI
        reqs.append((t, server.Request(sp, scheme=scheme, precision=prec, precond=pc,
                                       tol=1e-6, keep_fields=True)))
    return reqs


def test_results_alone_and_in_the_mix_agree(gpu):
    reqs = _requests()
    fps = [binding.footprint_bytes(r.spec, r.precision, r.precond) for _, r in reqs]
    srv = server.Server(hbm_budget=2 * max(fps), slots=3, device=0)
    import time
    t0 = time.perf_counter()
    for t, r in reqs:                       # Poisson arrivals, compressed in time
        wait = t0 + 0.01 * t - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        srv.submit(r)
    assert srv.drain(timeout=600)
    srv.close()
    assert srv.peak_in_use <= 2 * max(fps)
    assert len(srv.results) == len(reqs)
    for _, r in reqs:
        mixed = srv.results[r.rid]
        assert mixed.ok, mixed.error
        alone = server.run_path(server.Request(r.spec, r.scheme, r.precision, r.precond,
                                               r.tol, keep_fields=True))
        assert mixed.reactions == alone.reactions
        assert mixed.stag_iters == alone.stag_iters
        assert np.array_equal(mixed.d, alone.d)
    steps, paths = server.latency_percentiles(srv.results)
    assert steps["p50"] > 0 and paths["p99"] >= paths["p50"] > 0


def test_native_server_results_alone_and_in_the_mix_agree(gpu):
    # the library's own request loop (pf_server_*): same mix, same bitwise agreement
    reqs = _requests()
    fps = [binding.footprint_bytes(r.spec, r.precision, r.precond) for _, r in reqs]
    srv = binding.NativeServer(2 * max(fps), 3)
    ids = [srv.submit(r.spec, scheme=r.scheme, tol=r.tol, precision=r.precision,
                      precond=r.precond) for _, r in reqs]
    assert srv.drain(600.0)
    st = srv.stats()
    assert 1 <= st["peak_running"] <= 3 and st["peak_bytes"] <= 2 * max(fps)
    infos = [srv.poll(i) for i in ids]
    srv.close()
    assert sorted(x["admit_seq"] for x in infos) == list(range(len(reqs)))
    for (_, r), x in zip(reqs, infos):
        assert x["state"] == binding.REQ_DONE and x["status"] == binding.PF_OK
        assert x["steps_done"] == len(r.spec.increments) >= x["steps_converged"]
        assert x["step_ms_p99"] >= x["step_ms_p50"] > 0 and x["path_ms"] > 0
        alone = server.run_path(server.Request(r.spec, r.scheme, r.precision, r.precond, r.tol))
        assert list(x["reactions"]) == alone.reactions
        assert list(x["stag_iters"]) == alone.stag_iters


def test_native_server_cancels_a_running_request_between_steps(gpu):
    sp = S.tensile(32, l=0.06, steps=400, u_max=6e-3)
    srv = binding.NativeServer(1 << 36, 1)
    rid = srv.submit(sp, scheme=binding.S1, tol=1e-6)
    import time
    for _ in range(600):                        # wait until it has run a few steps
        if srv.poll(rid)["steps_done"] >= 3:
            break
        time.sleep(0.01)
    srv.cancel(rid)
    assert srv.drain(120.0)
    x = srv.poll(rid)
    srv.close()
    assert x["state"] == binding.REQ_CANCELLED and x["status"] == binding.PF_OK
    assert 3 <= x["steps_done"] < 400
    assert len(x["reactions"]) == x["steps_done"]


@pytest.mark.parametrize("n,precision,precond,split", [
    (512, binding.FP32_IR, binding.PRECOND_GMG, binding.SPLIT_VD),
    (512, binding.FP64, binding.PRECOND_GMG, binding.SPLIT_VD),
    (1024, binding.FP32_IR, binding.PRECOND_GMG, binding.SPLIT_VD),
    (512, binding.FP64, binding.PRECOND_JACOBI, binding.SPLIT_VD),
    (256, binding.FP32_IR, binding.PRECOND_GMG, binding.SPLIT_SPECTRAL),
])
def test_footprint_bounds_the_device_allocation(gpu, n, precision, precond, split):
    # The server admits requests by pf_footprint_bytes, so the formula must not undercount
    # what pf_create takes from the device (nor overcount it grossly).  cudaMemGetInfo
    # moves in 2 MiB pages; the slack covers that rounding.  The first context of a process
    # also loads the library's kernels (code, static scratch, the local-memory reserve):
    # a small context created first takes that one-time cost out of the measurement.
    import torch
    spec = S.tensile(n, l=4.0 / n)
    fp = binding.footprint_bytes(spec, precision, precond, split=split)
    warm = binding.Simulation(S.tensile(8, l=0.5), precision=precision, precond=precond,
                              split=split)
    warm.load_step(1e-4, 1, 1e-6)
    warm.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sim = binding.Simulation(spec, precision=precision, precond=precond, split=split)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    sim.close()
    used = free0 - free1
    # one slab per context: the footprint is the allocation, up to the 2 MiB page
    assert used <= fp + (4 << 20), (used, fp)
    assert used >= fp - (4 << 20), (used, fp)
