"""Demag-field extrapolation at RK4 sub-steps in FP64 (oracle; test infrastructure).

Sec. III: the demag field at the sub-steps of a higher-order evaluation method can be
extrapolated from values computed earlier instead of evaluated, RK4 needing a quartic
polynomial; one demag evaluation per step remains (the paper's r_D = 1/4). The formula is in
a reference the paper does not reproduce, so this module takes a reading:

* the demag field is evaluated at the first stage of every step, at the step's start state
  m_n (time t_n);
* the last five such values H_d(t_n), H_d(t_n - dt), ..., H_d(t_n - 4 dt), on equally spaced
  step starts, define the quartic Lagrange polynomial in t;
* stages 2 and 3 (time t_n + dt/2) and stage 4 (time t_n + dt) take that polynomial's value
  instead of an evaluation; the exchange and Zeeman fields are still evaluated at the stage
  state;
* until five values exist (the first four steps of a run) every stage evaluates the field.

Along the exact trajectory the extrapolated field is H_d(t) + O(dt^5), so the scheme is RK4
applied to dm/dt = F(m, t) with the demag part as a forcing in time, and keeps fourth order.
"""
import numpy as np

from . import GAMMA
from .conv import fft_conv
from .llg import exchange_field, llg_rhs, normalize

NODES = (0.0, -1.0, -2.0, -3.0, -4.0)   # step starts t_n, t_n - dt, ..., in units of dt


def lagrange_weights(c, nodes=NODES):
    """w_k such that p(c) = sum_k w_k p(s_k) for every polynomial p of degree < len(nodes)."""
    w = []
    for k, sk in enumerate(nodes):
        num, den = 1.0, 1.0
        for j, sj in enumerate(nodes):
            if j != k:
                num *= c - sj
                den *= sk - sj
        w.append(num / den)
    return np.array(w)


def extrapolate(history, c):
    """Value at t_n + c dt of the polynomial through history = [H(t_n), H(t_n - dt), ...]."""
    w = lagrange_weights(c, NODES[:len(history)])
    out = np.zeros_like(history[0])
    for wk, hk in zip(w, history):
        out += wk * hk
    return out


def llg_run_extrap(m, nsteps, dt, Nfull, cell, Ms, A, alpha, Hext=(0.0, 0.0, 0.0), gamma=GAMMA, history=None):
    """nsteps RK4 steps with the demag field extrapolated at stages 2-4 (reading above).

    history: list of earlier step-start demag fields, newest first (continued in place), or
    None to start a new run. Returns (m, number of demag evaluations)."""
    hist = [] if history is None else history
    nev = 0

    def heff(v, hd):
        H = hd + exchange_field(v, cell, Ms, A)
        for c in range(3):
            H[c] += Hext[c]
        return H

    def exact(v):
        nonlocal nev
        nev += 1
        return fft_conv(Ms * v, Nfull)

    for _ in range(nsteps):
        hd1 = exact(m)
        hist.insert(0, hd1)
        del hist[len(NODES):]
        k1 = llg_rhs(m, heff(m, hd1), alpha, gamma)
        if len(hist) == len(NODES):
            h_half, h_one = extrapolate(hist, 0.5), extrapolate(hist, 1.0)
            hd2 = lambda v: h_half
            hd4 = lambda v: h_one
        else:
            hd2 = hd4 = exact
        m2 = m + 0.5 * dt * k1
        k2 = llg_rhs(m2, heff(m2, hd2(m2)), alpha, gamma)
        m3 = m + 0.5 * dt * k2
        k3 = llg_rhs(m3, heff(m3, hd2(m3)), alpha, gamma)
        m4 = m + dt * k3
        k4 = llg_rhs(m4, heff(m4, hd4(m4)), alpha, gamma)
        m = normalize(m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))
    return m, nev
