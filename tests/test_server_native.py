"""Host logic of the library's request server (pf_server_*), without a GPU.

On a machine without a CUDA device every admitted request fails at pf_create and is
reported as failed; admission order, footprint limits, draining and shutdown are the same
as on a GPU (the GPU suite checks the results of served requests).
"""
import numpy as np
import pytest

from paper_2209_07969_gb300 import binding, specimens as S


def _spec(n=8):
    return S.tensile(n, l=0.1, steps=3, u_max=3e-3)


def test_create_rejects_bad_arguments():
    p = binding.P()
    assert binding.lib().pf_server_create(0, 2, binding.C.byref(p)) == binding.PF_EINVAL
    assert binding.lib().pf_server_create(1 << 30, 0, binding.C.byref(p)) == binding.PF_EINVAL


def test_submit_validation_and_unknown_ids():
    srv = binding.NativeServer(1 << 40, 2)
    try:
        big = _spec(64)
        fp = binding.footprint_bytes(big)
        small_srv = binding.NativeServer(fp - 1, 1)
        with pytest.raises(binding.PfError) as e:
            small_srv.submit(big)            # footprint above the whole budget
        assert e.value.status == binding.PF_EINVAL
        small_srv.close()
        with pytest.raises(binding.PfError):
            srv.submit(_spec(), scheme=7)
        with pytest.raises(binding.PfError):
            srv.submit(_spec(), tol=0.0)
        sp = _spec()
        sp.increments = np.zeros(0)
        with pytest.raises(binding.PfError):
            srv.submit(sp)
        info = binding.RequestInfo()
        assert binding.lib().pf_server_poll(srv.s, 12345, binding.C.byref(info), None,
                                            None) == binding.PF_EINVAL
    finally:
        srv.close()


def test_fifo_admission_within_the_budget():
    sp = _spec()
    fp = binding.footprint_bytes(sp)
    # room for one simulation at a time although three slots are free
    srv = binding.NativeServer(fp + fp // 2, 3)
    try:
        ids = [srv.submit(sp, scheme=s) for s in (0, 1, 3, 1)]
        assert srv.drain(60.0)
        infos = [srv.poll(i) for i in ids]
        assert [x["admit_seq"] for x in infos] == [0, 1, 2, 3]
        for x in infos:
            assert x["state"] in (binding.REQ_DONE, binding.REQ_FAILED)
            assert x["footprint"] == fp
            if x["state"] == binding.REQ_FAILED:
                assert x["status"] != binding.PF_OK
        st = srv.stats()
        assert st["peak_running"] == 1 and st["peak_bytes"] == fp
    finally:
        srv.close()


def test_destroy_with_queued_requests_returns():
    sp = _spec()
    fp = binding.footprint_bytes(sp)
    srv = binding.NativeServer(fp, 1)
    for _ in range(5):
        srv.submit(sp)
    srv.close()          # queued requests are dropped, the running one finishes


def test_pause_and_cancel_of_queued_requests():
    sp = _spec()
    srv = binding.NativeServer(1 << 40, 2)
    try:
        srv.pause()
        ids = [srv.submit(sp) for _ in range(4)]
        srv.cancel(ids[1])
        srv.cancel(ids[3])
        info = srv.poll(ids[0])
        assert info["state"] == binding.REQ_QUEUED and info["admit_seq"] == -1
        assert srv.poll(ids[1])["state"] == binding.REQ_CANCELLED
        assert not srv.drain(0.2)               # paused with requests queued
        srv.pause(False)
        assert srv.drain(60.0)
        seq = [srv.poll(i)["admit_seq"] for i in ids]
        assert seq[0] == 0 and seq[2] == 1 and seq[1] == seq[3] == -1
        assert srv.poll(ids[3])["state"] == binding.REQ_CANCELLED
        assert srv.poll(ids[3])["path_ms"] >= 0.0
        with pytest.raises(binding.PfError):
            srv.cancel(999)
        srv.cancel(ids[0])                      # finished: left as it is
        assert srv.poll(ids[0])["state"] in (binding.REQ_DONE, binding.REQ_FAILED)
    finally:
        srv.close()


def test_release_of_finished_requests():
    sp = _spec()
    srv = binding.NativeServer(1 << 40, 1)
    try:
        srv.pause()
        a, b = srv.submit(sp), srv.submit(sp)
        with pytest.raises(binding.PfError) as e:
            srv.release(a)                      # still queued
        assert e.value.status == binding.PF_EBUSY
        srv.cancel(b)
        srv.release(b)                          # cancelled counts as finished
        with pytest.raises(binding.PfError):
            srv.poll(b)
        srv.pause(False)
        assert srv.drain(60.0)
        srv.release(a)
        with pytest.raises(binding.PfError):
            srv.release(a)
    finally:
        srv.close()


def test_release_right_after_completion_keeps_admission_accounting():
    # A client that releases a request the moment it sees it finished must not race the
    # worker that ran it: the final state is published together with the return of the
    # request's footprint, so the budget stays exact and later requests are still admitted.
    import time
    sp = _spec()
    fp = binding.footprint_bytes(sp)
    srv = binding.NativeServer(fp, 2)           # one simulation at a time, two workers
    try:
        for _ in range(60):
            rid = srv.submit(sp)
            t0 = time.time()
            while srv.poll(rid)["state"] < binding.REQ_DONE:
                assert time.time() - t0 < 30.0
            srv.release(rid)
        last = srv.submit(sp)
        assert srv.drain(30.0)
        assert srv.poll(last)["admit_seq"] == 60
        assert srv.stats()["peak_bytes"] == fp
    finally:
        srv.close()
