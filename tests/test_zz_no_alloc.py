"""qtraj_evolve_static -- the entry point for callers that cannot allocate -- against qtraj_evolve.

Some callers cannot call cudaMalloc when they evolve trajectories (a service whose device memory is
all handed to its own pool at start-up, or a latency-bound loop where an allocation could stall the
device).  qtraj_evolve_static keeps its intermediates in a fixed array inside the library instead of
a caller workspace.  This test calls it through the C ABI twice in a row, with different batches,
and checks each result against the workspace-based entry point on the same inputs, within the
parity tolerance of the FP64 tests (1e-10 relative).  The file is named so that pytest collects it
last; it creates its own contexts, so it passes alone and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import build, qtraj
    build.build()
    qtraj.load()
    return qtraj


def _workspace_run(q, w, precision, basis):
    e = q.Engine(q.Config(N=w.grid.N, L=w.grid.L, dt=w.grid.dt, precision=precision, basis=basis))
    e.init([q.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits], w.n_traj, w.init_idx)
    e.evolve([q.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media], w.seeds, w.medium_idx)
    out = e.observables()
    e.close()
    return out


def _static_run(q, ctx, w):
    import torch
    lib = q.load()
    specs = (q.InitSpec * len(w.inits))(*[q.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits])
    media = (q.Medium * len(w.media))(*[q.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media])
    si = np.ascontiguousarray(w.init_idx, dtype=np.int32)
    mi = np.ascontiguousarray(w.medium_idx, dtype=np.int32)
    sd = np.ascontiguousarray(w.seeds, dtype=np.uint64)
    n = w.n_traj
    d_out = torch.zeros(n * q.OBS_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.qtraj_evolve_static(ctx, n, specs, len(w.inits), si.ctypes.data_as(C.POINTER(C.c_int)), media,
                                 len(w.media), mi.ctypes.data_as(C.POINTER(C.c_int)),
                                 sd.ctypes.data_as(C.POINTER(C.c_uint64)), C.c_void_p(d_out.data_ptr()),
                                 C.c_void_p(stream))
    assert st == 0, lib.qtraj_last_error(None)
    torch.cuda.synchronize()
    return np.frombuffer(d_out.cpu().numpy().tobytes(), dtype=q.OBS_DTYPE)


def _same(a, b):
    # the rMin shortcut is taken once a group's no-jump record is published inside the launch, so
    # whether a trajectory took it can differ between two launches; its record is the same either way
    sc = 1   # QTRAJ_F_NOJUMP_SHORTCUT
    both = (a["flags"] & sc) == (b["flags"] & sc)
    for f in ("n_jumps", "first_jump_step", "l", "color"):
        assert np.array_equal(a[f], b[f]), f
    assert np.array_equal(a["n_steps_exec"][both], b["n_steps_exec"][both])
    assert np.array_equal(a["flags"] & ~sc, b["flags"] & ~sc)
    assert np.array_equal(a["r0"], b["r0"])
    for f in ("surv", "ov_re", "ov_im", "norm2"):
        np.testing.assert_allclose(a[f], b[f], rtol=TOL, atol=1e-300)


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_static_entry_matches_workspace_entry_twice(q, precision, basis):
    """Both overlap bases: with basis = 1 (numerical vacuum eigenstates) the initial overlaps and
    their structural zeros must follow the context's basis, as qtraj_init takes them."""
    from paper_2107_06147_gb300 import inputs
    first = inputs.small_parity(N=512, n_traj=40, seed=21)
    second = inputs.small_parity(N=512, n_traj=17, seed=22)   # other states, media, seeds and size
    h = C.c_void_p()
    p = q.Config(N=512, L=first.grid.L, dt=first.grid.dt, precision=precision, basis=basis).params()
    lib = q.load()
    assert lib.qtraj_create(512, first.grid.L, first.grid.dt, first.grid.M, C.byref(p), C.byref(h)) == 0
    try:
        for w in (first, second):
            _same(_static_run(q, h, w), _workspace_run(q, w, precision, basis))
        # requests beyond the fixed capacity are refused with a message, before any GPU work
        too_many = inputs.small_parity(N=512, n_traj=1, seed=23)
        specs = (q.InitSpec * 1)(q.init_spec())
        media = (q.Medium * 1)(q.medium())
        sd = np.zeros(5000, dtype=np.uint64)
        st = lib.qtraj_evolve_static(h, 5000, specs, 1, None, media, 1, None,
                                     sd.ctypes.data_as(C.POINTER(C.c_uint64)), C.c_void_p(256), None)
        assert st == 1 and b"QTRAJ_STATIC_MAX_TRAJ" in lib.qtraj_last_error(None)
        del too_many
        # an initial state that is not finite on the host (2 w^2 underflows) is refused, no GPU work
        bad = (q.InitSpec * 1)(q.init_spec("gauss", 1e-200, 1, 0, 0))
        sd1 = np.zeros(1, dtype=np.uint64)
        st = lib.qtraj_evolve_static(h, 1, bad, 1, None, media, 1, None,
                                     sd1.ctypes.data_as(C.POINTER(C.c_uint64)), C.c_void_p(256), None)
        assert st == 1 and b"not finite" in lib.qtraj_last_error(None)
    finally:
        lib.qtraj_destroy(h)
