"""Demag extrapolation at RK4 sub-steps on the GPU (gbd_llg_step_ex with GBD_STEP_EXTRAP).

Sec. III's one-evaluation-per-step scheme, in the reading of oracle/extrap.py: the GPU run
must track the oracle's FP64 run of the same scheme from the same FP32-rounded start; the
start-up steps are plain RK4 (bit-identical to gbd_llg_step); GBD_STEP_CONTINUE splits a run
across calls without changing it.
"""
import numpy as np
import pytest

from gpu_util import lib, to_dev, to_host
from oracle import extrap as X
from oracle import tensor as T
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    return lib()


@pytest.mark.parametrize("n,cell,Hext", [((32, 24, 2), (3e-9, 3e-9, 3e-9), (0.0, 0.0, 5e4)),
                                         ((64, 48, 1), (2e-9, 2e-9, 3e-9), (0.0, 0.0, 0.0)),
                                         ((20, 16, 5), (4e-9, 3e-9, 2e-9), (1e4, 0.0, 0.0))])
def test_extrapolated_run_tracks_oracle(g, n, cell, Hext):
    Ms, A, alpha, dt, steps = 8e5, 1.3e-11, 0.1, 1e-13, 14
    m = W.random_unit(n, 41)
    mesh = g.Mesh(n, cell, Ms, A_ex=A, alpha=alpha, Hext=Hext)
    md = to_dev(m)
    mesh.llg_step(md, steps, dt, extrap=True)
    got = to_host(md)
    mesh.close()
    Nf = T.tensor_all_offsets(n, cell)
    want, nev = X.llg_run_extrap(m.astype(np.float64), steps, dt, Nf, cell, Ms, A, alpha, Hext=Hext)
    assert nev == 16 + (steps - 4)
    assert np.abs(got - want).max() < 2e-5


def test_startup_steps_are_plain_rk4(g):
    n, cell = (48, 40, 1), (2e-9, 2e-9, 3e-9)
    m = W.random_unit(n, 42)
    mesh = g.Mesh(n, cell, 8.6e5, A_ex=1.3e-11, alpha=0.02)
    a, b = to_dev(m), to_dev(m)
    mesh.llg_step(a, 4, 1e-13, extrap=True)
    mesh.llg_step(b, 4, 1e-13)
    assert np.array_equal(to_host(a), to_host(b))
    mesh.close()


def test_continue_splits_a_run(g):
    n, cell = (48, 40, 1), (2e-9, 2e-9, 3e-9)
    m = W.random_unit(n, 43)
    mesh = g.Mesh(n, cell, 8.6e5, A_ex=1.3e-11, alpha=0.02)
    a, b, c = to_dev(m), to_dev(m), to_dev(m)
    mesh.llg_step(a, 12, 1e-13, extrap=True)
    mesh.llg_step(b, 5, 1e-13, extrap=True)
    mesh.llg_step(b, 7, 1e-13, extrap=True, cont=True)
    assert np.array_equal(to_host(a), to_host(b))
    # without GBD_STEP_CONTINUE the second call starts a new history (four exact steps)
    mesh.llg_step(c, 5, 1e-13, extrap=True)
    mesh.llg_step(c, 7, 1e-13, extrap=True)
    assert not np.array_equal(to_host(a), to_host(c))
    mesh.close()


def test_unknown_flags_refused(g):
    mesh = g.Mesh((16, 16, 1), (2e-9, 2e-9, 3e-9), 8e5)
    m = to_dev(W.random_unit((16, 16, 1), 44))
    with pytest.raises(g.GbdError) as ei:
        g.gbd_llg_step_ex(mesh.handle, m, 2, 1e-13, 4, mesh.shape)
    assert ei.value.status == g.GBD_EINVAL
    mesh.close()
