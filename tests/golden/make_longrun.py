"""Writes the long-run parity goldens ``tests/golden/longrun_<case>.npz``.

Every number stored here comes from the FP64 oracle (``oracle.gp``) run over
the workload's stated step count from the workload's own seeded input
(``synth``); nothing is read from the CUDA path.  The GPU tests in
``tests/test_gpu_longrun.py`` rebuild the same inputs, run the CUDA path over
the same steps and compare element by element at the stored sites, plus the
full-grid sums stored beside them.

Cases (RK4 of Eqs. rk4_K1-rk4_final on Eqs. PULSE_psi / PULSE_res):

* ``res1024_f64``  -- scalar reservoir workload, 1024^2, 100 um, ring pump
  1.5 P_thr, 10^4 steps, from the FP64 inputs.
* ``res1024_f32``  -- the same from the inputs rounded to FP32 (psi0, P), the
  values an FP32 run starts from.
* ``ens128`` / ``ens512`` / ``ens1024`` -- members 0, 128 and 192 of the
  256-member uneven-grid ensemble (128^2, 512^2, 1024^2; pump peak
  U[0.8, 3] P_thr), 5000 steps each, FP32-rounded inputs.
* ``spin256``      -- the two-component TE-TM + reservoir physics of the
  2048^2 spinor workload (dx = 200/2048 um, its dt, Delta_LT = 0.025, Philox
  noise of variance 1e-3 per step, Gaussian pump of waist 10 um at
  1.5 P_thr) on a 256^2 grid (25 um, periodic), 2 x 10^4 steps,
  FP32-rounded inputs.

Stored per case: the sampled sites (j, i), psi and n at them (FP64), and the
full-grid sums S_pp = sum |psi|^2 and S_n = sum n.

Run from the repository root (each case is independent; they may run in
parallel):  python tests/golden/make_longrun.py <case> [<case> ...]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gp  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def to_prec(a, prec):
    """Input values an FP32 (or FP64) run starts from, held in FP64."""
    if a is None or prec == 64:
        return a
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return a.astype(np.complex64).astype(np.complex128)
    return a.astype(np.float32).astype(np.float64)


def spin256_config():
    """Two-component workload physics at the 2048^2 grid's cell size and
    time step, on 256^2 cells."""
    c = synth.load_constants()
    n = 256
    L = n * 200.0 / 2048
    d = synth.base_params(n, n, L, L, spinor=True, delta_lt=0.025, noise_var=1e-3,
                          seed=3, dt=c["spinor_2048_L200"]["dt"],
                          **synth.reservoir_physics())
    P = synth.gaussian(n, n, L, L, 1.5 * c["pump_threshold"], 10.0)[None]
    psi0 = synth.complex_normal((2, n, n), 1e-2, 3)
    return dict(name="spin256", params=d, psi0=psi0, n0=np.zeros((2, n, n)), P=P,
                V=None, steps=20000)


def case_input(case):
    """(workload dict, precision of the inputs) of a golden case."""
    if case == "res1024_f64":
        return synth.reservoir_1024(), 64
    if case == "res1024_f32":
        return synth.reservoir_1024(), 32
    if case in ("ens128", "ens512", "ens1024"):
        idx = {"ens128": 0, "ens512": 128, "ens1024": 192}[case]
        return synth.ensemble()[idx], 32
    if case == "spin256":
        return spin256_config(), 32
    raise ValueError(case)


def golden_sites(nx, ny):
    """Sites compared: a strided sublattice (offset 3, so that it does not
    line up with tile borders) covering about 16k sites, the four 8 x 8
    domain corners (periodic wrap) and one 64 x 64 window around the grid
    centre's row at 0.7 of the width (it crosses the ring pump of the
    1024^2 workloads)."""
    stride = max(1, int(np.sqrt(nx * ny / 16384.0)))
    jj, ii = np.meshgrid(np.arange(3 % stride, ny, stride), np.arange(3 % stride, nx, stride),
                         indexing="ij")
    pts = set(zip(jj.ravel().tolist(), ii.ravel().tolist()))
    for j0 in (0, ny - 8):
        for i0 in (0, nx - 8):
            for dj in range(8):
                for di in range(8):
                    pts.add((j0 + dj, i0 + di))
    w = min(64, nx, ny)
    jc, ic = ny // 2 - w // 2, min(int(0.7 * nx), nx - w)
    for dj in range(w):
        for di in range(w):
            pts.add((jc + dj, ic + di))
    pts = sorted(p for p in pts if 0 <= p[0] < ny and 0 <= p[1] < nx)
    return np.array([p[0] for p in pts]), np.array([p[1] for p in pts])


def make(case):
    cfg, prec = case_input(case)
    d = cfg["params"]
    p = gp.Params(**d)
    psi0 = to_prec(cfg["psi0"], prec)
    P = to_prec(cfg["P"], prec)
    n0 = cfg["n0"]
    t0 = time.time()
    psi, n = gp.run(psi0, n0, P, None, p, cfg["steps"])
    jj, ii = golden_sites(p.nx, p.ny)
    out = os.path.join(HERE, "longrun_%s.npz" % case)
    np.savez_compressed(
        out, j=jj.astype(np.int32), i=ii.astype(np.int32),
        psi=psi[:, jj, ii], n=n[:, jj, ii], steps=np.int64(cfg["steps"]),
        S_pp=np.float64(np.sum(np.abs(psi) ** 2)), S_n=np.float64(np.sum(n)),
        input_precision=np.int32(prec))
    print("%s: %d steps, %d sites, %.0f s -> %s" % (case, cfg["steps"], len(jj),
                                                  time.time() - t0, out), flush=True)


if __name__ == "__main__":
    for c in sys.argv[1:]:
        make(c)
