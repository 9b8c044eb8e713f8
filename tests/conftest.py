import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")


def oracle_inputs(w):
    """Maps a paper_2107_06147_gb300.inputs.Workload onto the oracle's records."""
    import oracle as o
    g = o.Grid(N=w.grid.N, L=w.grid.L, dt=w.grid.dt, M=w.grid.M, alpha_s=w.grid.alpha_s, Nc=w.grid.Nc)
    inits = [o.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits]
    media = [o.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media]
    return g, inits, media


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle as o
    o.build()
    return o
