"""Continuous batching (libqtraj's server; paper_2107_06147_gb300.serving is its binding).

A request's results must be the same when it is served alone and when it shares launches with other
requests of the same and of another grid size that arrive while it runs, and the same as a direct
evolve of its trajectories.  Argument checks that run before any CUDA call are tested on the CPU.
"""
import ctypes as C

import numpy as np
import pytest


def _cfg(qtraj, Ns, specs, **kw):
    p = qtraj.Config().params()
    ns = (C.c_int * len(Ns))(*Ns)
    sp = (qtraj.InitSpec * len(specs))(*specs)
    c = qtraj.ServerConfig(ns, len(Ns), kw.get("dr", 5.0 / 512), kw.get("dt", 0.001), 4.65, C.pointer(p), sp,
                           kw.get("n_specs", len(specs)), kw.get("slots", 1), kw.get("waves", 1), kw.get("budget", 100),
                           kw.get("order", 0))
    return c, (p, ns, sp)


def test_server_arguments_checked_on_host():
    from paper_2107_06147_gb300 import build, qtraj, serving
    build.build()
    lib = qtraj.load()
    nb = C.c_size_t()
    for Ns, kw, msg in (((100,), {}, b"power of two"), ((64, 64), {}, b"twice"), ((64,), {"n_specs": 0}, b"n_specs"),
                        ((64,), {"budget": 0}, b"positive"), ((64,), {"dt": 0.0}, b"positive"),
                        ((64,), {"order": 2}, b"order")):
        c, keep = _cfg(qtraj, Ns, serving.INIT_SPECS, **kw)
        assert lib.qtraj_server_workspace_bytes(C.byref(c), C.byref(nb)) == 1
        assert msg in lib.qtraj_last_error(None)
    n = C.c_int()
    assert lib.qtraj_poll(None, None, 0, C.byref(n)) == 1
    assert lib.qtraj_submit(None, None, 1, 0) == 1
    # a request's descriptors: one record per trajectory, seeds seed0 + i
    r = serving.Request(rid=3, N=512, init=2, T0=0.4, kappa_hat=4.0, gamma_hat=-1.0, ntraj=5, seed0=100, Tf=0.3)
    d = r.descriptors()
    assert d.dtype.itemsize == C.sizeof(qtraj.TrajDesc) and list(d["seed"]) == [100, 101, 102, 103, 104]
    assert (d["N"] == 512).all() and (d["spec"] == 2).all() and (d["kind"] == 0).all() and (d["Tf"] == 0.3).all()


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import build
    build.build()


def _direct(qtraj, N, prec, specs, desc, dr=5.0 / 512, dt=0.001):
    """The same trajectories through a plain context (fused form, rMin shortcut off)."""
    import torch
    e = qtraj.Engine(qtraj.Config(N=N, L=N * dr, dt=dt, precision=prec, use_rmin=0))
    e.init(list(specs), len(desc), np.ascontiguousarray(desc["spec"], dtype=np.int32))
    media = [qtraj.medium(float(x["T0"]), float(x["tau0"]), float(x["Tf"]), float(x["kappa_hat"]),
                          float(x["gamma_hat"])) for x in desc]
    e.evolve(media, np.ascontiguousarray(desc["seed"]), np.arange(len(desc), dtype=np.int32))
    o = e.observables(check_finite=False)
    torch.cuda.synchronize()
    e.close()
    return o


@pytest.mark.gpu
def test_request_same_alone_and_in_mix():
    _gpu()
    from paper_2107_06147_gb300 import qtraj, serving

    def req(rid, N, init, ntraj, seed0, T0=0.3, kap=4.0, gam=-1.0):
        return serving.Request(rid=rid, N=N, init=init, T0=T0, kappa_hat=kap, gamma_hat=gam, ntraj=ntraj,
                               seed0=seed0, Tf=0.27)

    for prec in (qtraj.FP64, qtraj.FP32):
        srv = serving.Server(Ns=(256, 512), slots_per_n=2, precision=prec, wave_mult=1)
        alone = req(0, 512, 1, 50, 77)
        srv.run_stream([alone], [0.0])
        mix = [req(1, 512, 0, 700, 5, T0=0.33), req(2, 256, 2, 300, 9), req(3, 512, 1, 50, 77), req(4, 512, 2, 90, 3)]
        srv.run_stream(mix, [0.0, 0.001, 0.002, 0.004])
        srv.close()
        a, b = alone.obs, mix[2].obs
        for f in qtraj.OBS_DTYPE.names:
            assert np.array_equal(a[f], b[f]), f
        assert all(r.done_time >= r.arrival for r in mix)
        ref = _direct(qtraj, 512, prec, serving.INIT_SPECS, alone.descriptors())
        for f in qtraj.OBS_DTYPE.names:
            assert np.array_equal(a[f], ref[f]), f


@pytest.mark.gpu
def test_budget_fifo_and_mixed_grid_request():
    """Admission within the budget in arrival order; a request whose trajectories use two grid sizes
    comes back in submission order, equal to direct evolves of each part."""
    _gpu()
    from paper_2107_06147_gb300 import qtraj, serving
    srv = serving.Server(Ns=(64, 128), slots_per_n=1, precision=qtraj.FP64, wave_mult=1, max_inflight_traj=100)
    reqs = [serving.Request(rid=10 + i, N=64, init=i % 3, T0=0.35, kappa_hat=5.0, gamma_hat=-0.5, ntraj=n,
                            seed0=1000 * i, Tf=0.3) for i, n in enumerate((20, 30, 70))]
    for r in reqs:
        srv.submit(r)
    srv.poll()
    assert srv.counts()[:2] == (1, 2)        # 20 + 30 admitted; 70 would exceed the budget of 100
    while not srv.idle():
        srv.poll()
    for r in reqs:
        ref = _direct(qtraj, 64, qtraj.FP64, serving.INIT_SPECS, r.descriptors())
        for f in qtraj.OBS_DTYPE.names:
            assert np.array_equal(r.obs[f], ref[f]), (r.rid, f)
    # one request, trajectories alternating between N = 64 and N = 128
    d = np.concatenate([reqs[0].descriptors(), reqs[1].descriptors()])
    d["N"][1::2] = 128
    lib = srv.lib
    assert lib.qtraj_submit(srv.h, C.c_void_p(d.ctypes.data), len(d), 99) == 0
    ids, n = (C.c_uint64 * 4)(), C.c_int()
    got = []
    while not got:
        assert lib.qtraj_poll(srv.h, ids, 4, C.byref(n)) == 0
        got = [int(ids[i]) for i in range(n.value)]
    assert got == [99]
    out = np.zeros(len(d), dtype=qtraj.OBS_DTYPE)
    assert lib.qtraj_request_result(srv.h, 99, C.c_void_p(out.ctypes.data), len(d)) == 0
    for N in (64, 128):
        sel = d["N"] == N
        ref = _direct(qtraj, N, qtraj.FP64, serving.INIT_SPECS, d[sel])
        for f in qtraj.OBS_DTYPE.names:
            assert np.array_equal(out[f][sel], ref[f]), (N, f)
    srv.close()


@pytest.mark.gpu
def test_server_errors():
    _gpu()
    from paper_2107_06147_gb300 import qtraj, serving
    srv = serving.Server(Ns=(64,), slots_per_n=1, precision=qtraj.FP32)
    lib = srv.lib
    r = serving.Request(rid=1, N=64, init=0, T0=0.4, kappa_hat=4.0, gamma_hat=-1.0, ntraj=8, seed0=0, Tf=0.38)
    d = r.descriptors()
    bad = d.copy()
    bad["N"][3] = 128
    assert lib.qtraj_submit(srv.h, C.c_void_p(bad.ctypes.data), len(bad), 5) == 1          # N not served
    bad = d.copy()
    bad["spec"][0] = 3
    assert lib.qtraj_submit(srv.h, C.c_void_p(bad.ctypes.data), len(bad), 5) == 1          # spec outside catalogue
    bad = d.copy()
    bad["kappa_hat"][1] = -0.5
    assert lib.qtraj_submit(srv.h, C.c_void_p(bad.ctypes.data), len(bad), 5) == 1          # invalid medium
    bad = d.copy()
    bad["kind"][2], bad["table_offset"][2], bad["table_len"][2] = 1, 0, 4
    assert lib.qtraj_submit(srv.h, C.c_void_p(bad.ctypes.data), len(bad), 5) == 1          # tabulated medium
    assert b"profile store" in lib.qtraj_last_error(None)
    assert lib.qtraj_submit(srv.h, C.c_void_p(d.ctypes.data), len(d), 5) == 0
    assert lib.qtraj_submit(srv.h, C.c_void_p(d.ctypes.data), len(d), 5) == 1              # id already queued
    out = np.zeros(len(d), dtype=qtraj.OBS_DTYPE)
    assert lib.qtraj_request_result(srv.h, 5, C.c_void_p(out.ctypes.data), len(d)) == 6    # EBUSY: not finished
    ids, n = (C.c_uint64 * 1)(), C.c_int()
    while n.value == 0:
        assert lib.qtraj_poll(srv.h, ids, 1, C.byref(n)) == 0
    assert lib.qtraj_request_result(srv.h, 5, C.c_void_p(out.ctypes.data), len(d)) == 0
    assert lib.qtraj_request_result(srv.h, 5, C.c_void_p(out.ctypes.data), len(d)) == 1    # forgotten
    srv.close()


@pytest.mark.gpu
def test_requests_overlap_on_the_device():
    """Continuous batching, not a queue: two requests of different grid sizes submitted together run
    on their slots' streams at the same time -- the device intervals of their launches (events around
    each evolve, qtraj_server_launch_log) overlap -- and each result is the same as alone."""
    _gpu()
    from paper_2107_06147_gb300 import qtraj, serving
    srv = serving.Server(Ns=(256, 512), slots_per_n=1, precision=qtraj.FP32, wave_mult=1)
    a = serving.Request(rid=1, N=256, init=0, T0=0.45, kappa_hat=4.0, gamma_hat=-1.0, ntraj=3000, seed0=0, Tf=0.3)
    b = serving.Request(rid=2, N=512, init=2, T0=0.45, kappa_hat=4.0, gamma_hat=-1.0, ntraj=1500, seed0=10 ** 6, Tf=0.3)
    srv.run_stream([a, b], [0.0, 0.0])
    log = srv.launch_log()
    srv.close()
    assert set(log["N"]) == {256, 512} and (log["end_ms"] > log["start_ms"]).all()
    la, lb = log[log["N"] == 256], log[log["N"] == 512]
    overlap = min(la["end_ms"].max(), lb["end_ms"].max()) - max(la["start_ms"].min(), lb["start_ms"].min())
    span = max(la["end_ms"].max(), lb["end_ms"].max()) - min(la["start_ms"].min(), lb["start_ms"].min())
    assert overlap > 0.5 * min(la["end_ms"].max() - la["start_ms"].min(), lb["end_ms"].max() - lb["start_ms"].min()), log
    assert span > 0
    for r in (a, b):
        ref = _direct(qtraj, r.N, qtraj.FP32, serving.INIT_SPECS, r.descriptors())
        for f in qtraj.OBS_DTYPE.names:
            assert np.array_equal(r.obs[f], ref[f]), (r.rid, f)


@pytest.mark.gpu
def test_shortest_work_first_order():
    """QTRAJ_ORDER_SHORTEST: of the requests admitted for one grid size, the launch takes those of
    least work first.  Three requests of one N arrive together, the long one first; with a launch of
    one wave the short ones finish before it (in arrival order the long one would hold the slot)."""
    _gpu()
    from paper_2107_06147_gb300 import qtraj, serving
    done = {}
    for order in (qtraj.ORDER_ARRIVAL, qtraj.ORDER_SHORTEST):
        srv = serving.Server(Ns=(256,), slots_per_n=1, precision=qtraj.FP32, wave_mult=1, order=order)
        cap = srv.launch_log  # noqa: F841  (the log is read below)
        reqs = [serving.Request(rid=1, N=256, init=0, T0=0.5, kappa_hat=4.0, gamma_hat=-1.0, ntraj=6000, seed0=0,
                                Tf=0.25),
                serving.Request(rid=2, N=256, init=1, T0=0.35, kappa_hat=4.0, gamma_hat=-1.0, ntraj=64, seed0=10 ** 6,
                                Tf=0.3),
                serving.Request(rid=3, N=256, init=2, T0=0.35, kappa_hat=4.0, gamma_hat=-1.0, ntraj=64, seed0=2 * 10 ** 6,
                                Tf=0.3)]
        srv.run_stream(reqs, [0.0, 0.0, 0.0])
        srv.close()
        done[order] = {r.rid: r.done_time for r in reqs}
        for r in reqs[1:]:
            ref = _direct(qtraj, 256, qtraj.FP32, serving.INIT_SPECS, r.descriptors())
            for f in qtraj.OBS_DTYPE.names:
                assert np.array_equal(r.obs[f], ref[f]), (order, r.rid, f)
    s = done[qtraj.ORDER_SHORTEST]
    assert s[2] < s[1] and s[3] < s[1]
    a = done[qtraj.ORDER_ARRIVAL]
    assert a[1] <= a[2] and a[1] <= a[3]
