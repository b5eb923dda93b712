"""Pins of the oracle's adaptive RKF5(6) stepping (reading in oracle/rkf.py; Sec. III).

From outside the module: Butcher's order conditions (one per rooted tree, elementary weight
sum_i b_i Phi_i(t) = 1/gamma(t)) hold exactly for b5 up to order 5 (17 trees) and for b6 up to
order 6 (37 trees); with a fixed step the method converges at fifth order on the macrospin
closed form, the error estimate shrinks at sixth order, and an adaptive run meets its
tolerance.
"""
import math
from fractions import Fraction as Fr

import numpy as np

from oracle import conv as C_
from oracle import llg as L
from oracle import rkf as R
from oracle import tensor as T
from test_oracle_llg import _macrospin


def _trees(order, memo={}):
    """Rooted trees with `order` vertices, each a sorted tuple of child trees."""
    if order in memo:
        return memo[order]
    if order == 1:
        memo[1] = [()]
        return memo[1]
    out = set()

    def forests(n, lo):
        if n == 0:
            yield ()
            return
        for k in range(1, n + 1):
            for t in _trees(k):
                key = (k, repr(t))
                if key < lo:
                    continue
                for rest in forests(n - k, key):
                    yield (t,) + rest

    for f in forests(order - 1, (0, "")):
        out.add(tuple(sorted(f, key=repr)))
    memo[order] = sorted(out, key=repr)
    return memo[order]


def _size(t):
    return 1 + sum(_size(u) for u in t)


def _gamma(t):
    g = _size(t)
    for u in t:
        g *= _gamma(u)
    return g


def _phi(t, a):
    s = len(a)
    v = [Fr(1)] * s
    for u in t:
        pu = _phi(u, a)
        w = [sum(a[i][j] * pu[j] for j in range(s)) for i in range(s)]
        v = [v[i] * w[i] for i in range(s)]
    return v


def test_butcher_order_conditions():
    s = 8
    a = [[R.A[i][j] if j < len(R.A[i]) else Fr(0) for j in range(s)] for i in range(s)]
    for i in range(s):
        assert sum(a[i]) == R.C[i]
    for b, order, count in ((R.B5, 5, 17), (R.B6, 6, 37)):
        trees = [t for p in range(1, order + 1) for t in _trees(p)]
        assert len(trees) == count
        for t in trees:
            assert sum(b[i] * _phi(t, a)[i] for i in range(s)) == Fr(1, _gamma(t))
    # b5 is not sixth order: some order-6 condition fails
    assert any(sum(R.B5[i] * _phi(t, a)[i] for i in range(s)) != Fr(1, _gamma(t)) for t in _trees(6))


def _macro(theta0=2.5, phi0=0.3, H0=1e5, alpha=0.1):
    cell = (3e-9, 3e-9, 3e-9)
    Nf = T.tensor_all_offsets((1, 1, 1), cell)
    m = np.array([math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0),
                  math.cos(theta0)]).reshape(3, 1, 1, 1)
    f = lambda v: L.rhs(v, Nf, cell, 8e5, 1.3e-11, alpha, Hext=(0.0, 0.0, H0))
    return m, f, lambda t: _macrospin(theta0, phi0, H0, alpha, t)


def test_fixed_step_fifth_order():
    m0, f, exact = _macro()
    errs = []
    for dt in (8e-12, 4e-12, 2e-12):
        m = m0
        steps = int(round(1.6e-10 / dt))
        for _ in range(steps):
            m, _ = R.rkf56_step(m, dt, f)
        errs.append(np.linalg.norm(m[:, 0, 0, 0] - exact(steps * dt)))
    for a, b in zip(errs, errs[1:]):
        assert 24.0 < a / b < 44.0, errs


def test_error_estimate_sixth_order():
    m0, f, _ = _macro()
    est = [R.rkf56_step(m0, dt, f)[1] for dt in (1.6e-11, 8e-12, 4e-12)]
    for a, b in zip(est, est[1:]):
        assert 48.0 < a / b < 80.0, est


def test_adaptive_run_meets_tolerance():
    m0, f, exact = _macro()
    m, acc, rej, _ = R.run_adaptive(m0, 2e-10, 1e-13, 1e-9, f)
    assert acc > 0 and np.linalg.norm(m[:, 0, 0, 0] - exact(2e-10)) < 1e-7
    # a looser tolerance takes fewer, larger steps
    _, acc2, _, _ = R.run_adaptive(m0, 2e-10, 1e-13, 1e-6, f)
    assert acc2 < acc


def test_extrapolated_rkf_keeps_fifth_order_and_one_evaluation_per_step():
    # quintic extrapolation at stages 2-8 (Sec. III): the demag field along the exact path is
    # reproduced to O(dt^6), so fixed-step runs still converge at fifth order on the macrospin
    from oracle import extrap as X
    cell = (3e-9, 3e-9, 3e-9)
    Nf = T.tensor_all_offsets((1, 1, 1), cell)
    m0, _, exact = _macro()
    demag = lambda v: C_.fft_conv(8e5 * v, Nf)
    rest = lambda v, hd: L.llg_rhs(v, hd + L.exchange_field(v, cell, 8e5, 1.3e-11) + np.array([0.0, 0.0, 1e5])[:, None, None, None], 0.1)
    # (steps of 2 ps and below: the five earlier steps the quintic spans then cover < 0.25 rad of
    # the 2.2e10 rad/s precession; at 8 ps they cover ~1 rad and the extrapolation dominates)
    errs = []
    for dt in (2e-12, 1e-12, 5e-13):
        steps = int(round(1.6e-10 / dt))
        m, hist = m0, []
        for n in range(steps):
            m, _, hd1 = R.rkf56_step_extrap(m, dt, demag, rest, [(-(i + 1) * dt, h) for i, h in enumerate(hist)])
            hist = [hd1] + hist[:4]
        errs.append(np.linalg.norm(m[:, 0, 0, 0] - exact(steps * dt)))
    for a, b in zip(errs, errs[1:]):
        assert 20.0 < a / b < 48.0, errs
    # the adaptive driver evaluates the field once per step after five accepted steps
    _, acc, rej, _, nev = R.run_adaptive_extrap(m0, 2e-10, 1e-12, 1e-9, demag, rest)
    assert acc > 5 and nev <= 8 * 5 + 8 * rej + (acc - 5)
    # the weights at unequal nodes reproduce quintics exactly (the interpolation it relies on)
    nodes = [0.0, -1.3, -2.1, -3.7, -4.2, -5.9]
    for c in (0.25, 0.8, 1.0):
        vals = [s ** 5 - 2 * s ** 3 + s for s in nodes]
        assert abs(X.lagrange_weights(c, nodes) @ np.array(vals) - (c ** 5 - 2 * c ** 3 + c)) <= 1e-10
