"""Adaptive RKF5(6) time stepping of the LLG equation in FP64 (oracle; test infrastructure).

Sec. III names the Runge-Kutta-Fehlberg 5th-order method with 6th-order error estimation
(RKF56) for adaptive time stepping; its tableau (Ref. [29]) is not in the paper. Reading: the
eight-stage RK5(6) pair of Fehlberg (NASA TR R-287, 1968) below, whose weights satisfy every
Butcher order condition up to order 5 (b5) and 6 (b6) in exact arithmetic (pinned in the tests).

* A step from m with size dt evaluates k_i = f(m + dt sum_j a_ij k_j), i = 1..8; the step's
  result is the fifth-order m5 = m + dt sum_i b5_i k_i, renormalized per cell (as for RK4); the
  error estimate is err = dt max_cells |sum_i (b6_i - b5_i) k_i|.
* A step is accepted when err <= tol; either way the next size is
  dt * min(FAC_MAX, max(FAC_MIN, SAFETY (tol / err)^(1/6))), and a rejected step is retried
  from the same m with that size. The last step is shortened to end exactly at t_end.
"""
from fractions import Fraction as Fr

import numpy as np

from .llg import normalize

# Fehlberg RK5(6): nodes c, matrix a (rows 2..8), fifth-order b5, sixth-order b6
C = [Fr(0), Fr(1, 6), Fr(4, 15), Fr(2, 3), Fr(4, 5), Fr(1), Fr(0), Fr(1)]
A = [[],
     [Fr(1, 6)],
     [Fr(4, 75), Fr(16, 75)],
     [Fr(5, 6), Fr(-8, 3), Fr(5, 2)],
     [Fr(-8, 5), Fr(144, 25), Fr(-4), Fr(16, 25)],
     [Fr(361, 320), Fr(-18, 5), Fr(407, 128), Fr(-11, 80), Fr(55, 128)],
     [Fr(-11, 640), Fr(0), Fr(11, 256), Fr(-11, 160), Fr(11, 256), Fr(0)],
     [Fr(93, 640), Fr(-18, 5), Fr(803, 256), Fr(-11, 160), Fr(99, 256), Fr(0), Fr(1)]]
B5 = [Fr(31, 384), Fr(0), Fr(1125, 2816), Fr(9, 32), Fr(125, 768), Fr(5, 66), Fr(0), Fr(0)]
B6 = [Fr(7, 1408), Fr(0), Fr(1125, 2816), Fr(9, 32), Fr(125, 768), Fr(0), Fr(5, 66), Fr(5, 66)]

SAFETY, FAC_MIN, FAC_MAX = 0.9, 0.2, 5.0


def rkf56_step(m, dt, f):
    """One RKF5(6) step: (normalized fifth-order result, error estimate)."""
    k = []
    for i in range(8):
        mi = m.copy()
        for j, aij in enumerate(A[i]):
            if aij != 0:
                mi = mi + dt * float(aij) * k[j]
        k.append(f(mi))
    m5 = m.copy()
    d = np.zeros_like(m)
    for i in range(8):
        if B5[i] != 0:
            m5 = m5 + dt * float(B5[i]) * k[i]
        if B6[i] != B5[i]:
            d = d + float(B6[i] - B5[i]) * k[i]
    err = dt * float(np.sqrt((d * d).sum(axis=0)).max())
    return normalize(m5), err


def next_dt(dt, err, tol):
    """The controller's next step size (see the module docstring)."""
    fac = FAC_MAX if err == 0 else min(FAC_MAX, max(FAC_MIN, SAFETY * (tol / err) ** (1.0 / 6.0)))
    return dt * fac


def rkf56_step_extrap(m, dt, demag, rest, history):
    """One RKF5(6) step with the demag field extrapolated at stages 2-8 (Sec. III: a quintic
    for RKF56). history: earlier accepted step starts as (t - t_n, H_d) pairs, newest first.
    The field is evaluated at stage 1; with five earlier step starts, stages i >= 2 take the
    quintic Lagrange polynomial through (0, H_d(t_n)) and those five, at time c_i dt.
    Returns (m5, err, H_d(t_n))."""
    from .extrap import lagrange_weights
    hd1 = demag(m)
    warm = len(history) >= 5
    nodes = [0.0] + [t for t, _ in history[:5]]
    fields = [hd1] + [h for _, h in history[:5]]
    k = []
    for i in range(8):
        mi = m.copy()
        for j, aij in enumerate(A[i]):
            if aij != 0:
                mi = mi + dt * float(aij) * k[j]
        if i == 0:
            hd = hd1
        elif warm:
            w = lagrange_weights(float(C[i]) * dt, nodes)
            hd = sum(wk * fk for wk, fk in zip(w, fields))
        else:
            hd = demag(mi)
        k.append(rest(mi, hd))
    m5 = m.copy()
    d = np.zeros_like(m)
    for i in range(8):
        if B5[i] != 0:
            m5 = m5 + dt * float(B5[i]) * k[i]
        if B6[i] != B5[i]:
            d = d + float(B6[i] - B5[i]) * k[i]
    err = dt * float(np.sqrt((d * d).sum(axis=0)).max())
    return normalize(m5), err, hd1


def run_adaptive_extrap(m, t_end, dt, tol, demag, rest, max_steps=100000):
    """run_adaptive with the demag field extrapolated at stages 2-8 once five accepted step
    starts are recorded; rest(m, H_d) gives dm/dt from the stage state and its demag field.
    Returns (m, accepted, rejected, last dt proposal, demag evaluations)."""
    t, acc, rej, nev = 0.0, 0, 0, 0
    history = []                                 # (t_k, H_d(t_k)) of accepted step starts, newest first
    while t < t_end and acc + rej < max_steps:
        h = min(dt, t_end - t)
        rel = [(tk - t, hk) for tk, hk in history]
        m_new, err, hd1 = rkf56_step_extrap(m, h, demag, rest, rel)
        nev += 1 if len(history) >= 5 else 8
        dt = next_dt(h, err, tol)
        if err <= tol:
            history.insert(0, (t, hd1))
            del history[5:]
            m, t, acc = m_new, t + h, acc + 1
        else:
            rej += 1
    return m, acc, rej, dt, nev


def run_adaptive(m, t_end, dt, tol, f, max_steps=100000):
    """Adaptive RKF5(6) from t = 0 to t_end; returns (m, accepted, rejected, last dt proposal)."""
    t, acc, rej = 0.0, 0, 0
    while t < t_end and acc + rej < max_steps:
        h = min(dt, t_end - t)
        m_new, err = rkf56_step(m, h, f)
        dt = next_dt(h, err, tol)
        if err <= tol:
            m, t, acc = m_new, t + h, acc + 1
        else:
            rej += 1
    return m, acc, rej, dt
