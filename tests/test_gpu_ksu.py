"""GPU parity of the isotropic KSU potential (App. E, "Isotropic KSU potential"; potential = 1)
against the oracle, through the C ABI.

The KSU evolution is deterministic (singlet, H_eff, no jumps), so every record is compared
trajectory by trajectory: FP64 within 1e-10 relative (final states, norms and survival ratios),
FP32 within the FP32 error model of the Munich tests (the sine transform's running-sum noise,
FP32_MODEL sqrt(N n_steps)).  The overlap basis is the numerical Cornell vacuum eigenstates: the
library's eigensolver against the oracle's dense diagonalisation first.
"""
import numpy as np
import pytest

from test_gpu_parity import FP32_MODEL, fp32_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import build, qtraj
    build.build()
    qtraj.load()
    return qtraj


# initial states: Gaussian S and P waves, the numerical 1S, 2S, 1P of the Cornell vacuum (kind 2)
INITS = [("gauss", 0.3, 1, 0), ("gauss", 0.5, 2, 1), ("numerical", 0.0, 1, 0), ("numerical", 0.0, 2, 0),
         ("numerical", 0.0, 2, 1)]


def _media(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(3):
        T0 = float(rng.uniform(0.3, 0.5))
        out.append((T0, 0.6, T0 * float(rng.uniform(0.85, 0.95))))
    return out


def _oracle(N, L, dt, fmd, media, idx, mi):
    import oracle as o
    from oracle import eigen
    g = o.Grid(N=N, L=L, dt=dt, potential=1, ksu_fmd=fmd, use_rmin=0)
    g.basis = eigen.numerical_basis(g)
    inits = []
    for kind, w, n, l in INITS:
        if kind == "numerical":
            _, v = eigen.vacuum_eigenstates(g, l, n - l)
            inits.append(o.given_state(v[-1], n, l, 0))
        else:
            inits.append(o.init_spec(kind, w, n, l, 0))
    om = [o.medium(T0, tau0, Tf, 0.0, 0.0) for (T0, tau0, Tf) in media]
    ref, _, u = o.run_batch(g, inits, idx, om, mi, np.arange(len(idx), dtype=np.uint64), want_states=True)
    return g, ref, u


def _gpu(q, N, L, dt, fmd, precision, media, idx, mi):
    import torch
    e = q.Engine(q.Config(N=N, L=L, dt=dt, precision=precision, potential=1, ksu_mD_factor=fmd, save_states=1))
    e.init([q.init_spec(kind, w, n, l, 0) for kind, w, n, l in INITS], len(idx), idx)
    e.evolve([q.medium(T0, tau0, Tf, 0.0, 0.0) for (T0, tau0, Tf) in media], np.arange(len(idx), dtype=np.uint64), mi)
    obs = e.observables()
    u = e.states()
    basis = e.basis()
    torch.cuda.synchronize()
    e.close()
    return obs, u, basis


@pytest.mark.parametrize("N,precision,fmd", [(64, 0, 1.0), (256, 0, 1.0), (1024, 0, 1.0), (256, 0, 0.4),
                                             (64, 1, 1.0), (256, 1, 1.0), (1024, 1, 1.0), (4096, 1, 1.0)])
def test_ksu_against_oracle(q, N, precision, fmd):
    """Gaussian and Cornell-eigenstate initial states in three Bjorken media (T0 0.3-0.5 GeV, a few
    hundred to two thousand steps); fmd = 0.4 weakens the screening so that the real part reaches the
    string-breaking cap inside the box."""
    L, dt = 12.0, 0.001
    media = _media(N + int(10 * fmd))
    n = 15
    idx = (np.arange(n) % len(INITS)).astype(np.int32)
    mi = ((np.arange(n) // len(INITS)) % len(media)).astype(np.int32)
    g, ref, uref = _oracle(N, L, dt, fmd, media, idx, mi)
    obs, u, basis = _gpu(q, N, L, dt, fmd, precision, media, idx, mi)
    assert np.abs(basis - g.basis).max() < 1e-9 * np.abs(g.basis).max()
    assert (ref["n_jumps"] == 0).all() and (obs["n_jumps"] == 0).all() and (obs["r0"] == 0).all()
    assert np.array_equal(obs["n_steps_exec"], ref["n_steps_exec"]) and (ref["n_steps_exec"] > 100).all()
    assert np.array_equal(obs["flags"], ref["flags"]) and np.array_equal(obs["jump_digest"], ref["jump_digest"])
    assert (ref["norm2"] < 0.999).all()                       # V_I acted
    du = np.linalg.norm(u - uref, axis=1) / np.linalg.norm(uref, axis=1)
    dn = np.abs(obs["norm2"] / ref["norm2"] - 1)
    ds = np.abs(obs["surv"] - ref["surv"]).max(axis=1) / np.maximum(1.0, np.abs(ref["surv"]).max(axis=1))
    tol = 1e-10 if precision == 0 else fp32_bound(N, ref["n_steps_exec"])
    assert (du <= tol).all(), (du / tol).max()
    assert (dn <= tol).all(), (dn / tol).max()
    assert (ds <= tol).all(), (ds / tol).max()


def test_ksu_argument_checks(q):
    import ctypes as C
    lib = q.load()
    h = C.c_void_p()
    for cfg in (dict(form=q.PLAIN), dict(t_vacuum=0.1), dict(ksu_mD_factor=0.0)):
        p = q.Config(N=64, L=12.0, potential=1, **cfg).params()
        assert lib.qtraj_create(64, 12.0, 0.001, 4.65, C.byref(p), C.byref(h)) == 1
    e = q.Engine(q.Config(N=64, L=12.0, potential=1))
    with pytest.raises(q.QtrajError):
        e.init([q.init_spec("gauss", 0.3, 1, 0, 1)], 2)       # octet
    e.init([q.init_spec("gauss", 0.3, 1, 0, 0)], 2)
    with pytest.raises(q.QtrajError):
        e.evolve([q.medium(0.3, 0.6, 0.05, 0.0, 0.0)], np.arange(2, dtype=np.uint64))   # Tf below 0.1 GeV
    with pytest.raises(q.QtrajError):
        e.set_trace(every=10, n_traced=1, max_records=4)
    e.close()
