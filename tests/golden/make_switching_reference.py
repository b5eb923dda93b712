"""Writes the FP64 reference of the time-step study on the reduced switching film.

The paper's time-step study (Sec. II, Fig. 2) measures the mean relative error eps of a run at
time step dt against a double-precision run at a small time step, on the switching problem
(a 2.4 um x 1.2 um x 10 nm film in 5 nm cells, switched by H = (-20, 1, 0) kA/m for 1 ns from
an S state). The reduced film here keeps the cells and the protocol and shrinks the film five
times in x and y (96 x 48 x 2 cells), so that the FP64 oracle can integrate it. Everything
below calls only ``oracle/`` (FP64 numpy) and ``paper_2308_08447_gb300.workloads`` (inputs):

1. S state: m = [1, 1, 1]/sqrt(3), relaxed by the stated protocol (field along [1, 1, 1]
   stepped 1.0, 0.9, ..., 0.0 MA/m, 50 ps each, alpha = 0.5, RK4 at 100 fs), rounded to
   float32 -- the input both the oracle and the GPU runs start from.
   -> switching_96x48x2_S_state.npy  (float32, [3][nz][ny][nx])
2. Switching: 1 ns at alpha = 0.02 under the switching field from that state, RK4 in FP64 at
   dt_ref = 50 fs, <m> recorded every 10 ps (100 samples); the same at 100 fs gives the
   reference's own error estimate (RK4: about 1/16 of the 100 fs run's difference).
   -> switching_96x48x2_fp64_traj.txt

Run from the repository root (about half an hour on one core per run; the two switching runs
go in parallel):

    python tests/golden/make_switching_reference.py
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
from oracle import llg as L  # noqa: E402
from oracle import tensor as T  # noqa: E402
from paper_2308_08447_gb300 import workloads as W  # noqa: E402

SCALE = 5
DT_RELAX = 100e-15
DT_REF = 50e-15
DT_CHECK = 100e-15
INTERVAL = 10e-12
STATE = os.path.join(HERE, "switching_96x48x2_S_state.npy")
TRAJ = os.path.join(HERE, "switching_96x48x2_fp64_traj.txt")


def relax(spec, Nf):
    meta = spec.meta
    m = W.uniform(spec.n, meta["m_init"]).astype(np.float64)
    steps = int(round(meta["relax_hold"] / DT_RELAX))
    for h in meta["relax_fields"]:
        Hext = tuple(h * c for c in meta["relax_dir"])
        f = lambda v: L.rhs(v, Nf, spec.cell, spec.Ms, spec.A_ex, meta["relax_alpha"], Hext)
        for _ in range(steps):
            m = L.rk4_step(m, DT_RELAX, f)
    return m.astype(np.float32)


def switch(dt):
    spec = W.switching(scale=SCALE)
    Nf = T.tensor_all_offsets(spec.n, spec.cell)
    m = np.load(STATE).astype(np.float64)
    f = lambda v: L.rhs(v, Nf, spec.cell, spec.Ms, spec.A_ex, spec.alpha, spec.Hext)
    per = int(round(INTERVAL / dt))
    n_rec = int(round(spec.meta["t_switch"] / INTERVAL))
    rec = []
    for _ in range(n_rec):
        for _ in range(per):
            m = L.rk4_step(m, dt, f)
        rec.append(m.mean(axis=(1, 2, 3)))
    return np.array(rec)


def main():
    spec = W.switching(scale=SCALE)
    t0 = time.time()
    if not os.path.exists(STATE):
        Nf = T.tensor_all_offsets(spec.n, spec.cell)
        np.save(STATE, relax(spec, Nf))
        print("S state: %.0f s" % (time.time() - t0), flush=True)
    with mp.get_context("spawn").Pool(2) as pool:
        ref, chk = pool.map(switch, [DT_REF, DT_CHECK])
    est = L.trajectory_error(chk, ref, 1.0)
    with open(TRAJ, "w") as fh:
        fh.write("# Mean unit magnetization <m>(t_i), t_i = 10 ps * i (i = 1..100), of the reduced switching film\n")
        fh.write("# (96 x 48 x 2 cells of 5 nm, Ms 800 kA/m, A 1.3e-11 J/m, alpha 0.02, H = (-20, 1, 0) kA/m; Sec. II,\n")
        fh.write("# Fig. 2) from switching_96x48x2_S_state.npy, FP64 oracle RK4 at dt = 50 fs.\n")
        fh.write("# eps (Sec. II) of the FP64 100 fs run against this one: %.6e\n" % est)
        fh.write("# written by tests/golden/make_switching_reference.py\n")
        for row in ref:
            fh.write("%.17e %.17e %.17e\n" % tuple(row))
    print("done: %.0f s, eps(100 fs vs 50 fs, FP64) = %.3e" % (time.time() - t0, est), flush=True)


if __name__ == "__main__":
    main()
