"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds only input generation (random numbers, mesh descriptions);
it contains none of the demag / exchange / LLG arithmetic. Each generator draws
from numpy's PCG64 with an explicit seed and returns FP32 arrays laid out as
[component, z, y, x] (x fastest), the layout the library takes.

Workloads (the paper measures on synthetic micromagnetic problems only):
* ``random_unit``: M = Ms * u with u uniform on the sphere (normalised
  Gaussian triples) -- the 32x32x8 parity mesh and the 512x512x64 3D mesh.
* ``vortex_noise``: an in-plane vortex with a 10 nm out-of-plane core plus
  0.3 x (sum of 16 random-phase plane waves with |k| <= 2 pi / 64 cells),
  normalised -- the 1024x1024x1 thin film (2x2x3 nm cells).
* ``batch_meshes`` / ``served_requests``: seeded mesh-size and material
  mixes for the batched and served patterns.
* ``switching``: the switching problem of the paper's time-step study (Fig. 2),
  a deterministic start (``uniform``) and a stated relax protocol.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class MeshSpec:
    n: tuple                 # (nx, ny, nz) cells
    cell: tuple              # (dx, dy, dz) metres
    Ms: float = 8.0e5        # A/m
    A_ex: float = 1.3e-11    # J/m
    alpha: float = 0.02
    dt: float = 1.0e-13      # s
    Hext: tuple = (0.0, 0.0, 0.0)
    steps: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def cells(self):
        return self.n[0] * self.n[1] * self.n[2]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_unit(n, seed):
    """(3, nz, ny, nx) float32 unit vectors, uniform on the sphere."""
    nx, ny, nz = n
    g = _rng(seed).standard_normal((3, nz, ny, nx))
    g /= np.sqrt((g * g).sum(axis=0, keepdims=True))
    return g.astype(np.float32)


def vortex_noise(n, cell, seed, core=10e-9, amp=0.3, waves=16, kmax_cells=64):
    """(3, nz, ny, nx) float32 unit vectors: vortex + core + random-phase plane-wave noise."""
    nx, ny, nz = n
    dx, dy, _ = cell
    rng = _rng(seed)
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dy
    Y, X = np.meshgrid(y, x, indexing="ij")
    phi = np.arctan2(Y, X)
    r2 = X * X + Y * Y
    m = np.stack([-np.sin(phi), np.cos(phi), np.exp(-r2 / (2.0 * core * core))])
    kmax = 2.0 * np.pi / (kmax_cells * max(dx, dy))
    for _ in range(waves):
        kabs = kmax * np.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * np.pi)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        dirv = rng.standard_normal(3)
        dirv /= np.linalg.norm(dirv)
        wave = np.cos(kabs * (np.cos(th) * X + np.sin(th) * Y)[None] + ph[:, None, None])
        m = m + (amp / np.sqrt(waves)) * dirv[:, None, None] * wave
    m = m / np.sqrt((m * m).sum(axis=0, keepdims=True))
    return np.repeat(m[:, None, :, :], nz, axis=1).astype(np.float32)


# The five workloads, by size and material. Parameters the configs leave open
# are fixed here: Ms = 8e5 A/m, A = 1.3e-11 J/m, alpha = 0.02, dt = 1e-13 s for
# the 3D mesh; dt = min(1e-13, 1.5 / omega_ex) for the batched and served mixes.
def parity_cube():
    return MeshSpec(n=(32, 32, 8), cell=(4e-9, 4e-9, 4e-9), Ms=8.0e5, seed=1)


def thin_film():
    return MeshSpec(n=(1024, 1024, 1), cell=(2e-9, 2e-9, 3e-9), Ms=8.6e5, A_ex=1.3e-11,
                    alpha=0.02, dt=1e-13, steps=1000, seed=2)


def large_3d():
    return MeshSpec(n=(512, 512, 64), cell=(4e-9, 4e-9, 4e-9), Ms=8.0e5, A_ex=1.3e-11,
                    alpha=0.02, dt=1e-13, steps=100, seed=3)


def switching(scale=1):
    """The switching problem of Fig. 2 (Sec. II): a 2.4 um x 1.2 um x 10 nm film in 5 nm cells
    (480 x 240 x 2), Ms = 800 kA/m, switched by H = (-20, 1, 0) kA/m for 1 ns from an S state.

    Readings where the paper is silent: A = 1.3e-11 J/m and alpha = 0.02 during switching;
    the S state is prepared from m = [1, 1, 1]/sqrt(3) in a field along [1, 1, 1] stepped from
    1 MA/m down to 0 in eleven holds (1.0, 0.9, ..., 0.0 MA/m) of 50 ps each at alpha = 0.5.
    scale > 1 shrinks the film by that factor in x and y (same cells), for parity tests."""
    nx, ny = 480 // scale, 240 // scale
    u = 1.0 / np.sqrt(3.0)
    return MeshSpec(n=(nx, ny, 2), cell=(5e-9, 5e-9, 5e-9), Ms=8.0e5, A_ex=1.3e-11, alpha=0.02, dt=1e-13,
                    Hext=(-2.0e4, 1.0e3, 0.0), seed=0,
                    meta={"m_init": (u, u, u), "relax_fields": [1e6 * (1.0 - 0.1 * k) for k in range(11)],
                          "relax_dir": (u, u, u), "relax_alpha": 0.5, "relax_hold": 50e-12, "t_switch": 1e-9})


def uniform(n, direction):
    """(3, nz, ny, nx) float32: every cell along the unit vector `direction`."""
    nx, ny, nz = n
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    return np.broadcast_to(d[:, None, None, None], (3, nz, ny, nx)).astype(np.float32).copy()


def stable_dt(cell, Ms, A_ex, gamma=2.212761569e5, mu0=4e-7 * np.pi, cap=1e-13):
    """min(cap, 1.5 / omega_ex), omega_ex = gamma (2A/(mu0 Ms)) sum_d 4/d_d^2 (RK4 stability margin)."""
    w = gamma * (2.0 * A_ex / (mu0 * Ms)) * sum(4.0 / (d * d) for d in cell)
    return min(cap, 1.5 / w)


def batch_meshes(count=64, seed=4, steps=100):
    """Uneven meshes: nx, ny in {64, 96, ..., 512}, nz in {1, 2, 4, 8, 16}, cubic cell U[2, 5] nm."""
    out = []
    for i in range(count):
        r = _rng(seed + i)
        nx = int(r.choice(np.arange(64, 513, 32)))
        ny = int(r.choice(np.arange(64, 513, 32)))
        nz = int(r.choice([1, 2, 4, 8, 16]))
        d = float(r.uniform(2e-9, 5e-9))
        Ms = float(r.uniform(4e5, 1.4e6))
        cell = (d, d, d)
        out.append(MeshSpec(n=(nx, ny, nz), cell=cell, Ms=Ms, A_ex=1.3e-11, alpha=0.02,
                            dt=stable_dt(cell, Ms, 1.3e-11), steps=steps, seed=seed + i))
    return out


def served_requests(count=2000, rate=200.0, seed=5, max_side=1024, max_nz=16):
    """Poisson arrivals (mean `rate`/s) of relaxation jobs: steps U{200..2000},
    nx, ny = 32 * round(2^U[6,10] / 32), nz = 2^round(U[0, log2 max_nz]), cubic 2-5 nm, alpha = 0.5."""
    r = _rng(seed)
    t = np.cumsum(r.exponential(1.0 / rate, size=count))
    out = []
    lo, hi = 6.0, np.log2(max_side)
    for i in range(count):
        nx = int(max(64, 32 * round(2 ** r.uniform(lo, hi) / 32)))
        ny = int(max(64, 32 * round(2 ** r.uniform(lo, hi) / 32)))
        nz = int(2 ** round(r.uniform(0, np.log2(max_nz))))
        d = float(r.uniform(2e-9, 5e-9))
        Ms = float(r.uniform(4e5, 1.4e6))
        steps = int(r.integers(200, 2001))
        cell = (d, d, d)
        out.append(MeshSpec(n=(nx, ny, nz), cell=cell, Ms=Ms, A_ex=1.3e-11, alpha=0.5,
                            dt=stable_dt(cell, Ms, 1.3e-11), steps=steps, seed=10_000 + i,
                            meta={"arrival": float(t[i])}))
    return out
