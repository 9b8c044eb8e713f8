"""Continuous-batching request loop (paper_2107_06147_gb300.serving).

A request's results must be the same when it is served alone and when it shares launches with
other requests of the same and of another grid size that arrive while it runs.  Host-side
scheduling logic (FIFO split of requests into launches, admission budget) is checked on the CPU with
a fake engine.
"""
import numpy as np
import pytest


class _FakeEngine:
    def __init__(self, *a, **k):
        self.log = []

    def set_spec_idx(self, idx):
        self.idx = np.array(idx)

    def evolve(self, media, seeds, midx, stream=None):
        self.log.append((list(seeds), list(midx)))
        self.seeds = np.array(seeds)

    def observables(self, stream=None, check_finite=True):
        from paper_2107_06147_gb300 import qtraj
        o = np.zeros(len(self.seeds), dtype=qtraj.OBS_DTYPE)
        o["r0"] = self.seeds.astype(np.float64)
        return o


class _FakeEvent:
    def record(self, s):
        pass

    def query(self):
        return True


def test_scheduler_splits_requests_fifo_and_respects_budget():
    from paper_2107_06147_gb300 import serving
    srv = serving.Server.__new__(serving.Server)
    srv.pending, srv.slots, srv.waiting, srv.completed = {}, {}, serving.deque(), []
    srv.max_inflight, srv.inflight = 100, 0
    slot = serving._Slot.__new__(serving._Slot)
    slot.eng, slot.cap, slot.stream, slot.event, slot.busy, slot.parts = _FakeEngine(), 32, None, _FakeEvent(), False, []
    srv.slots[64] = [slot]
    srv.pending[64] = serving.deque()
    reqs = [serving.Request(rid=i, N=64, init=i % 3, T0=0.4, kappa_hat=4, gamma_hat=-1, ntraj=n, seed0=1000 * i)
            for i, n in enumerate((20, 30, 70))]
    for r in reqs:
        srv.submit(r, now=0.0)
    srv.poll()                       # admits 20 + 30 (70 would exceed 100), launches 32 of them
    assert srv.inflight == 50 and len(srv.waiting) == 1
    seeds, midx = slot.eng.log[-1]
    assert seeds[:20] == list(range(0, 20)) and seeds[20:] == list(range(1000, 1012))
    assert midx == [0] * 20 + [1] * 12
    while not srv.idle():
        srv.poll()
    assert [r.n_done for r in reqs] == [20, 30, 70]
    for r in reqs:                   # every trajectory came back to its own request and slot
        assert np.array_equal(r.obs["r0"], r.seed0 + np.arange(r.ntraj))


@pytest.mark.gpu
def test_request_same_alone_and_in_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import build, qtraj, serving
    build.build()

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
        for f in ("surv", "ov_re", "ov_im", "norm2", "r0"):
            assert np.array_equal(a[f], b[f]), f
        for f in ("n_jumps", "first_jump_step", "l", "color", "n_steps_exec", "flags"):
            assert np.array_equal(a[f], b[f]), f
        assert all(r.done_time >= r.arrival for r in mix)
