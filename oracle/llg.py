"""Exchange field, LLG right-hand side and RK4 step in FP64 (oracle; test infrastructure).

Sec. III: H_ex = 2A/(mu0 Ms) lap(m) (Eq. 4); the LLG equation
dm/dt = -gamma m x H_eff + alpha m x dm/dt (Eq. 5); H_eff = H_Zee + H_ex + H_d
(anisotropy is outside this path); RK4 as the evaluation method. Arrays are
[component, z, y, x].

Readings where the paper is silent:
* Laplacian: 7-point finite difference with free (Neumann) boundaries -- a
  missing neighbour is replaced by the cell itself, so a dimension of size 1
  contributes nothing.
* Eq. 5 solved for dm/dt with |m| = 1:
  dm/dt = -gamma/(1+alpha^2) [m x H + alpha m x (m x H)].
* RK4: the classic four-stage scheme; stage inputs are not renormalized, and m
  is renormalized once at the end of each step.
"""
import numpy as np

from . import MU0, GAMMA
from .conv import fft_conv


def laplacian_neumann(m, cell):
    """sum_d (m_{i+e_d} - 2 m_i + m_{i-e_d}) / d_d^2, missing neighbours replaced by m_i."""
    dx, dy, dz = cell
    out = np.zeros_like(m)
    for axis, d in ((3, dx), (2, dy), (1, dz)):
        n = m.shape[axis]
        if n == 1:
            continue
        up = np.concatenate([np.take(m, range(1, n), axis=axis), np.take(m, [n - 1], axis=axis)], axis=axis)
        dn = np.concatenate([np.take(m, [0], axis=axis), np.take(m, range(0, n - 1), axis=axis)], axis=axis)
        out += (up - 2.0 * m + dn) / (d * d)
    return out


def exchange_field(m, cell, Ms, A):
    """Eq. 4: H_ex = 2A / (mu0 Ms) lap(m), in A/m."""
    return (2.0 * A / (MU0 * Ms)) * laplacian_neumann(m, cell)


def llg_rhs(m, H, alpha, gamma=GAMMA):
    """dm/dt = -gamma/(1+alpha^2) [m x H + alpha m x (m x H)] (Eq. 5 solved for dm/dt)."""
    mxH = np.cross(m, H, axis=0)
    mxmxH = np.cross(m, mxH, axis=0)
    return -gamma / (1.0 + alpha * alpha) * (mxH + alpha * mxmxH)


def effective_field(m, Nfull, cell, Ms, A, Hext=(0.0, 0.0, 0.0)):
    """H_eff = H_d(Ms m) + H_ex(m) + H_ext."""
    Hd = fft_conv(Ms * m, Nfull)
    H = Hd + exchange_field(m, cell, Ms, A)
    for c in range(3):
        H[c] += Hext[c]
    return H


def rhs(m, Nfull, cell, Ms, A, alpha, Hext=(0.0, 0.0, 0.0), gamma=GAMMA):
    """f(m) = dm/dt with the demag field recomputed from m."""
    return llg_rhs(m, effective_field(m, Nfull, cell, Ms, A, Hext), alpha, gamma)


def normalize(m):
    return m / np.sqrt((m * m).sum(axis=0, keepdims=True))


def rk4_step(m, dt, f):
    """Classic RK4: k1 = f(m), k2 = f(m + dt k1/2), k3 = f(m + dt k2/2), k4 = f(m + dt k3),
    m+ = normalize(m + dt (k1 + 2 k2 + 2 k3 + k4) / 6)."""
    k1 = f(m)
    k2 = f(m + 0.5 * dt * k1)
    k3 = f(m + 0.5 * dt * k2)
    k4 = f(m + dt * k3)
    return normalize(m + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))


def llg_run(m, nsteps, dt, Nfull, cell, Ms, A, alpha, Hext=(0.0, 0.0, 0.0), gamma=GAMMA):
    """nsteps RK4 steps of the LLG equation with demag, exchange and Zeeman fields."""
    f = lambda v: rhs(v, Nfull, cell, Ms, A, alpha, Hext, gamma)
    for _ in range(nsteps):
        m = rk4_step(m, dt, f)
    return m


def trajectory_error(Ms_traj, ref_traj, Ms):
    """epsilon = sum_i |M(t_i) - M~(t_i)| / (n Ms) (Sec. II, discussion of Fig. 2)."""
    d = np.asarray(Ms_traj) - np.asarray(ref_traj)
    return np.linalg.norm(d, axis=-1).sum() / (len(d) * Ms)
