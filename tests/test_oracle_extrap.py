"""Pins of the oracle's demag extrapolation at RK4 sub-steps (Sec. III; reading in oracle/extrap.py).

Checked against facts outside the module: the fifth backward difference of a quartic
vanishes (the weights at c = 1 are binomial), numpy's least-squares polynomial through five
points is the interpolant, the interpolation remainder of a monic quintic is the node product,
the start-up steps are plain RK4, and the macrospin closed form keeps fourth-order convergence.
"""
import math

import numpy as np

from oracle import extrap as X
from oracle import llg as L
from oracle import tensor as T
from test_oracle_llg import _macrospin


def test_weights_at_full_step_are_binomial():
    assert np.array_equal(X.lagrange_weights(1.0), np.array([5.0, -10.0, 10.0, -5.0, 1.0]))


def test_weights_match_numpy_interpolant():
    rng = np.random.default_rng(3)
    nodes = np.array(X.NODES)
    for c in (0.5, 1.0, 0.25, 2.0):
        for _ in range(5):
            y = rng.standard_normal(5)
            want = np.polyval(np.polyfit(nodes, y, 4), c)
            assert abs(X.lagrange_weights(c) @ y - want) <= 1e-9 * max(1.0, abs(want))


def test_quartic_exact_quintic_remainder():
    rng = np.random.default_rng(4)
    coef = rng.standard_normal((5, 3, 2, 4))              # a quartic field in t
    quartic = lambda t: sum(coef[p] * t ** p for p in range(5))
    hist = [quartic(s) for s in X.NODES]
    for c in (0.5, 1.0):
        assert np.abs(X.extrapolate(hist, c) - quartic(c)).max() <= 1e-12 * np.abs(quartic(c)).max()
        # t^5: the remainder is f^(5)/5! prod(c - s_k) = c (c+1) (c+2) (c+3) (c+4)
        got = X.extrapolate([np.array([s ** 5]) for s in X.NODES], c)[0]
        assert abs((c ** 5 - got) - c * (c + 1) * (c + 2) * (c + 3) * (c + 4)) <= 1e-12


def test_first_four_steps_are_plain_rk4():
    n, cell, Ms, A, alpha, dt = (6, 5, 2), (3e-9, 3e-9, 3e-9), 8e5, 1.3e-11, 0.1, 1e-13
    rng = np.random.default_rng(5)
    m = L.normalize(rng.standard_normal((3, n[2], n[1], n[0])))
    Nf = T.tensor_all_offsets(n, cell)
    got, nev = X.llg_run_extrap(m, 4, dt, Nf, cell, Ms, A, alpha, Hext=(0.0, 0.0, 2e4))
    want = L.llg_run(m, 4, dt, Nf, cell, Ms, A, alpha, Hext=(0.0, 0.0, 2e4))
    assert np.array_equal(got, want) and nev == 16
    hist = []
    X.llg_run_extrap(m, 4, dt, Nf, cell, Ms, A, alpha, history=hist)
    _, nev = X.llg_run_extrap(m, 6, dt, Nf, cell, Ms, A, alpha, history=hist)
    assert nev == 6 and len(hist) == 5                   # one evaluation per step once warm


def _macrospin_extrap(dt, T_end, theta0=2.5, phi0=0.3, H0=1e5, alpha=0.1):
    cell = (3e-9, 3e-9, 3e-9)
    Nf = T.tensor_all_offsets((1, 1, 1), cell)
    m = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0),
                  math.cos(theta0)]).reshape(3, 1, 1, 1)
    steps = int(round(T_end / dt))
    m, _ = X.llg_run_extrap(m, steps, dt, Nf, cell, 8e5, 1.3e-11, alpha, Hext=(0.0, 0.0, H0))
    return m[:, 0, 0, 0], _macrospin(theta0, phi0, H0, alpha, steps * dt)


def test_extrapolated_rk4_keeps_fourth_order():
    # a single cube: H_d = -Ms m / 3 is parallel to m on the exact path, so the closed form of
    # the Zeeman precession holds; the extrapolated field must not spoil the dt^4 convergence
    errs = []
    for dt in (4e-12, 2e-12, 1e-12):
        got, want = _macrospin_extrap(dt, 1.6e-10)
        errs.append(np.linalg.norm(got - want))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs
