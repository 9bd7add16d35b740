"""Failure detection of the serving runtime, with faults made on the host.

No device fault is involved: the test hook sfh_serve_inject_fault makes an
allocation of the server's creation fail, keeps one tile of a request from
ever being published (the request can never complete), or stalls the host
admission thread.  The server must report each case with a status, keep every
wait bounded, stay usable for other requests, and shut down cleanly.  Also
checked: the device-start timestamp of a served request lies between its
admission and its completion.
"""
import time

import numpy as np
import pytest
import torch

from paper_2306_11665_gb300 import _abi as A
from paper_2306_11665_gb300 import api
from paper_2306_11665_gb300 import inputs as I
from tests._helpers import rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11665_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _fp64_request(p=4, n_elem=300, seed=3):
    N = int(np.ceil(n_elem ** (1.0 / 3.0) - 1e-9))
    u, Ja = I.workload(3, p, 0, N, n_elem=n_elem, seed0=seed)
    tu, tJ = torch.from_numpy(u).cuda(), torch.from_numpy(Ja).cuda()
    out = torch.empty_like(tu)
    req = A.Request(A.SFH_REQ_RESIDUAL, p, 0, A.SFH_FP64, n_elem, tu.data_ptr(), tJ.data_ptr(), None, out.data_ptr())
    return req, (tu, tJ, out)


def _standalone(p, tu, tJ):
    ctx = api.Context(3, p, 0, "euler")
    return ctx.volume_residual(tu, tJ, "fp64").cpu().numpy()


def _same(out, ref):
    # the standalone FP64 call may pick another kernel (another summation
    # order) than the server's tiles: equal to round-off
    return rel_err_per_var(out.cpu().numpy(), ref) <= 1e-13


def _poll_until(srv, ticket, limit_s):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = A.sfh_serve_poll(srv, ticket)
        if r is not None:
            return r
        time.sleep(0.001)
    return None


def test_timestamps_are_ordered_with_device_start():
    srv = A.sfh_server_create(8 << 30, 8, 20000)
    try:
        torch.cuda.synchronize()
        keep = []
        tickets = []
        for k in range(4):
            req, arrs = _fp64_request(p=3 + k, n_elem=200 + 50 * k, seed=5 + k)
            keep.append(arrs)
            tickets.append(A.sfh_serve_submit(srv, req))
        for t in tickets:
            r = _poll_until(srv, t, 30.0)
            assert r is not None and r.status == A.SFH_OK
            slack = 200_000   # ns: the calibrated device-to-host clock mapping
            assert r.t_submit_ns <= r.t_admit_ns <= r.t_done_ns
            assert r.t_start_ns > 0
            assert r.t_admit_ns - slack <= r.t_start_ns <= r.t_done_ns + slack
    finally:
        A.sfh_server_destroy(srv)


@pytest.mark.parametrize("step", [1, 2, 3, 4])
def test_allocation_failure_at_creation_then_usable(step):
    A.sfh_serve_inject_fault(None, A.SFH_FAULT_CREATE_ALLOC, step)
    with pytest.raises(A.SfhError) as e:
        A.sfh_server_create(8 << 30, 8, 20000)
    assert e.value.status == A.SFH_ENOMEM
    # the failure released what it had allocated; the next creation works and serves
    srv = A.sfh_server_create(8 << 30, 8, 20000)
    try:
        req, (tu, tJ, out) = _fp64_request()
        torch.cuda.synchronize()
        r = _poll_until(srv, A.sfh_serve_submit(srv, req), 30.0)
        assert r is not None and r.status == A.SFH_OK
        assert _same(out, _standalone(4, tu, tJ))
    finally:
        A.sfh_server_destroy(srv)


def test_request_with_a_dropped_tile_times_out_and_server_stays_usable():
    timeout_ms = 400
    srv = A.sfh_server_create(8 << 30, 4, timeout_ms)
    destroyed = False
    try:
        req_a, keep_a = _fp64_request(n_elem=400, seed=11)   # several tiles; its last is never published
        req_b, (tu, tJ, out_b) = _fp64_request(n_elem=250, seed=12)
        torch.cuda.synchronize()
        A.sfh_serve_inject_fault(srv, A.SFH_FAULT_DROP_TILE, 1)
        t0 = time.time()
        ta = A.sfh_serve_submit(srv, req_a)
        ra = _poll_until(srv, ta, 10.0)
        waited = time.time() - t0
        assert ra is not None and ra.status == A.SFH_ETIMEOUT
        assert waited < timeout_ms * 1e-3 + 2.0            # the watchdog's bound
        # drain is bounded while the abandoned request holds its slot
        t1 = time.time()
        with pytest.raises(A.SfhError) as e:
            A.sfh_serve_drain(srv, 200)
        assert e.value.status == A.SFH_ETIMEOUT and time.time() - t1 < 2.0
        # another request still runs and is right
        rb = _poll_until(srv, A.sfh_serve_submit(srv, req_b), 30.0)
        assert rb is not None and rb.status == A.SFH_OK
        assert _same(out_b, _standalone(4, tu, tJ))
        # shutdown: bounded, frees the server, reports that a request never finished
        t2 = time.time()
        with pytest.raises(A.SfhError) as e:
            A.sfh_server_destroy(srv)
        destroyed = True
        assert e.value.status == A.SFH_ETIMEOUT and time.time() - t2 < 3 * timeout_ms * 1e-3 + 2.0
        del keep_a
    finally:
        if not destroyed:
            try:
                A.sfh_server_destroy(srv)
            except A.SfhError:
                pass
    # the device is fine afterwards: a plain residual runs and checks clean
    req, (tu, tJ, out) = _fp64_request(n_elem=64, seed=13)
    ctx = api.Context(3, 4, 0, "euler")
    ctx.volume_residual(tu, tJ, "fp64")
    assert ctx.check() == A.SFH_OK


def test_stalled_admission_thread_keeps_waits_bounded():
    srv = A.sfh_server_create(8 << 30, 8, 20000)
    try:
        req, (tu, tJ, out) = _fp64_request(seed=21)
        torch.cuda.synchronize()
        A.sfh_serve_inject_fault(srv, A.SFH_FAULT_STALL_ADMISSION, 800)
        time.sleep(0.01)   # the admission thread is now asleep
        t = A.sfh_serve_submit(srv, req)
        t0 = time.time()
        with pytest.raises(A.SfhError) as e:
            A.sfh_serve_drain(srv, 100)
        assert e.value.status == A.SFH_ETIMEOUT and time.time() - t0 < 1.0
        assert A.sfh_serve_poll(srv, t) is None                 # not done while the thread sleeps
        A.sfh_serve_drain(srv, 20000)                           # it wakes up and finishes the work
        r = A.sfh_serve_poll(srv, t)
        assert r is not None and r.status == A.SFH_OK
        assert _same(out, _standalone(4, tu, tJ))
    finally:
        A.sfh_server_destroy(srv)


def test_serial_fifo_replay_matches_standalone_and_orders_timestamps():
    reqs, keep = [], []
    for k in range(6):
        req, arrs = _fp64_request(p=2 + k, n_elem=120, seed=30 + k)
        reqs.append(req)
        keep.append(arrs)
    torch.cuda.synchronize()
    arr = [0.0, 0.0, 0.001, 0.002, 0.002, 0.010]
    res = A.sfh_serial_replay(reqs, arr, 30000)
    prev = 0
    for k, r in enumerate(res):
        assert r.status == A.SFH_OK
        assert r.t_admit_ns <= r.t_start_ns <= r.t_done_ns
        assert r.t_done_ns >= prev            # FIFO: completions in order
        prev = r.t_done_ns
        tu, tJ, out = keep[k]
        assert _same(out, _standalone(2 + k, tu, tJ))
