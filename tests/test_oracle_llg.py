"""Pins of the oracle's exchange field (Eq. 4), LLG right-hand side (Eq. 5) and RK4 step (Sec. III).

* Exchange: a uniform m gives 0; the cosine modes cos(pi p (i + 1/2) / n) are
  eigenvectors of the free-boundary Laplacian with eigenvalue
  -(2 - 2 cos(pi p / n)) / d^2 (the DCT-II diagonalisation of the Neumann
  second difference).
* LLG: dm/dt is orthogonal to m and vanishes for H parallel to m.
* A single cubic cell in a field H0 z has the closed-form solution
  tan(theta/2) = tan(theta0/2) exp(-alpha gamma H0 t / (1 + alpha^2)),
  phi = phi0 + gamma H0 t / (1 + alpha^2) (its demag field -M/3 exerts no torque).
* RK4's error at fixed end time falls as dt^4 (the Fig. 2 time-step study).
* |m| = 1 after each step; with damping and no applied field the
  demag + exchange energy does not increase.
"""
import math

import numpy as np
import pytest

from oracle import GAMMA, MU0
from oracle import conv as C
from oracle import llg as L
from oracle import tensor as T


def test_exchange_uniform_is_zero():
    m = np.zeros((3, 3, 4, 5))
    m[0] = 0.6
    m[2] = 0.8
    assert np.abs(L.exchange_field(m, (1e-9, 2e-9, 3e-9), 8e5, 1.3e-11)).max() == 0.0


@pytest.mark.parametrize("axis,p", [(3, 1), (3, 4), (2, 2), (1, 1)])
def test_exchange_cosine_modes(axis, p):
    shape = (3, 3, 4, 7)
    cell = (1e-9, 2e-9, 3e-9)
    n = shape[axis]
    d = {3: cell[0], 2: cell[1], 1: cell[2]}[axis]
    i = np.arange(n)
    mode = np.cos(math.pi * p * (i + 0.5) / n)
    bshape = [1, 1, 1, 1]
    bshape[axis] = n
    m = np.broadcast_to(mode.reshape(bshape), shape) * np.array([1.0, -2.0, 0.5])[:, None, None, None]
    lap = L.laplacian_neumann(np.ascontiguousarray(m), cell)
    lam = -(2.0 - 2.0 * math.cos(math.pi * p / n)) / (d * d)
    np.testing.assert_allclose(lap, lam * m, rtol=0, atol=1e-9 * abs(lam))


def test_llg_rhs_orthogonal_and_zero_for_parallel_field():
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, 2, 3, 4))
    m /= np.linalg.norm(m, axis=0)
    H = 1e5 * rng.standard_normal((3, 2, 3, 4))
    f = L.llg_rhs(m, H, 0.1)
    assert np.abs((f * m).sum(axis=0)).max() < 1e-9 * np.abs(f).max()
    assert np.abs(L.llg_rhs(m, 3e4 * m, 0.1)).max() < 1e-6


def _macrospin(theta0, phi0, H0, alpha, t):
    th = 2 * math.atan(math.tan(theta0 / 2) * math.exp(-alpha * GAMMA * H0 * t / (1 + alpha ** 2)))
    ph = phi0 + GAMMA * H0 * t / (1 + alpha ** 2)
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def _macrospin_run(dt, T_end, theta0=2.5, phi0=0.3, H0=1e5, alpha=0.1):
    cell = (3e-9, 3e-9, 3e-9)
    Nf = T.tensor_all_offsets((1, 1, 1), cell)
    m = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0),
                  math.cos(theta0)]).reshape(3, 1, 1, 1)
    steps = int(round(T_end / dt))
    m = L.llg_run(m, steps, dt, Nf, cell, 8e5, 1.3e-11, alpha, Hext=(0.0, 0.0, H0))
    return m[:, 0, 0, 0], _macrospin(theta0, phi0, H0, alpha, steps * dt)


def test_macrospin_closed_form():
    got, want = _macrospin_run(1e-13, 2e-10)
    assert np.linalg.norm(got - want) < 1e-9


def test_rk4_fourth_order():
    errs = []
    for dt in (4e-12, 2e-12, 1e-12):
        got, want = _macrospin_run(dt, 1.6e-10)
        errs.append(np.linalg.norm(got - want))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


def _energy(m, Nf, cell, Ms, A):
    Hd = C.fft_conv(Ms * m, Nf)
    Hx = L.exchange_field(m, cell, Ms, A)
    return -0.5 * MU0 * Ms * (m * (Hd + Hx)).sum() * cell[0] * cell[1] * cell[2]


def test_unit_norm_and_energy_decrease():
    n, cell, Ms, A = (8, 6, 2), (3e-9, 3e-9, 3e-9), 8e5, 1.3e-11
    rng = np.random.default_rng(11)
    m = rng.standard_normal((3, n[2], n[1], n[0]))
    m /= np.linalg.norm(m, axis=0)
    Nf = T.tensor_all_offsets(n, cell)
    f = lambda v: L.rhs(v, Nf, cell, Ms, A, 0.5)
    E = [_energy(m, Nf, cell, Ms, A)]
    for _ in range(20):
        m = L.rk4_step(m, 2e-14, f)
        assert np.abs(np.linalg.norm(m, axis=0) - 1.0).max() < 1e-14
        E.append(_energy(m, Nf, cell, Ms, A))
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(E, E[1:]))
    assert E[-1] < E[0]


def test_trajectory_error_hand_value():
    """eps = sum_i |M(t_i) - M_ref(t_i)| / (n Ms) (Sec. II, Fig. 2 discussion) on a two-sample
    trajectory worked out by hand: the differences (3, 4, 0) and (0, 5, 12) have Euclidean norms
    5 and 13, so with Ms = 2 A/m eps = (5 + 13) / (2 * 2) = 4.5. Summing squared norms (97),
    taking the norm of the whole difference (13.9 / 4), dropping Ms (9), dividing by n only, or
    the largest sample instead of the mean (6.5) all give another number."""
    ref = np.array([[1.0, 1.0, 1.0], [-2.0, 0.5, 3.0]])
    traj = ref + np.array([[3.0, 4.0, 0.0], [0.0, 5.0, 12.0]])
    assert L.trajectory_error(traj, ref, 2.0) == pytest.approx(4.5, rel=1e-15)
    # symmetric in its two trajectories, zero for identical ones
    assert L.trajectory_error(ref, traj, 2.0) == pytest.approx(4.5, rel=1e-15)
    assert L.trajectory_error(ref, ref, 2.0) == 0.0


def test_trajectory_error_unit_and_scaled_forms_agree():
    """For trajectories of the normalised magnetization m = M / Ms the same measure is the mean
    |m - m_ref|: scaling both trajectories by Ms and passing Ms changes nothing, and a constant
    offset of length r along the whole trajectory gives r exactly."""
    rng = np.random.default_rng(3)
    ref = rng.standard_normal((40, 3))
    off = np.array([0.0, 0.6, 0.8]) * 1e-3          # |off| = 1e-3
    Ms = 8e5
    assert L.trajectory_error(ref + off, ref, 1.0) == pytest.approx(1e-3, rel=1e-12)
    assert L.trajectory_error(Ms * (ref + off), Ms * ref, Ms) == pytest.approx(1e-3, rel=1e-12)
