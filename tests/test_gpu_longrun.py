"""Parity at the stated step counts on the workloads' own seeded inputs.

The expected values are the FP64 oracle's, written by
``tests/golden/make_longrun.py`` (which calls only ``oracle/``) into
``tests/golden/longrun_<case>.npz``: psi and n after the full step count at
sampled sites (a strided sublattice, the four domain corners and one 64 x 64
window), plus the full-grid sums S_pp = sum |psi|^2 and S_n = sum n.  Here the
CUDA path runs the same inputs over the same steps in the launch
configuration the benchmark times (single handles with the autotuned step
kernel; the whole 256-member ensemble as one batch) and is compared element
by element: relative L2 <= 1e-11 (FP64) and <= 1e-4 (FP32).

* reservoir workload, 1024^2, 10^4 RK4 steps: FP64 from the FP64 inputs and
  FP32 from the inputs rounded to FP32;
* the uneven-grid ensemble, 5000 steps: members 0 (128^2), 128 (512^2) and
  192 (1024^2);
* the two-component TE-TM workload's physics with Philox noise on 256^2
  cells of the 2048^2 grid's size, 2 x 10^4 steps."""
import os
import sys

import numpy as np
import pytest

import synth
from gpu_util import phx, make_handle, get_state, rel_l2, TOL

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
import make_longrun  # noqa: E402


def golden(case):
    path = os.path.join(GOLDEN, "longrun_%s.npz" % case)
    if not os.path.exists(path):
        pytest.fail("missing golden %s (run tests/golden/make_longrun.py %s)" % (path, case))
    return dict(np.load(path))


def compare(g, psi, n, prec, what):
    jj, ii = g["j"], g["i"]
    e_psi = rel_l2(psi[:, jj, ii].astype(np.complex128), g["psi"])
    e_n = rel_l2(n[:, jj, ii].astype(np.float64), g["n"])
    e_spp = abs(float(np.sum(np.abs(psi.astype(np.complex128)) ** 2)) - float(g["S_pp"])) / float(g["S_pp"])
    e_sn = abs(float(np.sum(n.astype(np.float64))) - float(g["S_n"])) / float(g["S_n"])
    print("%s: rel L2 psi %.3e n %.3e, S_pp %.3e, S_n %.3e" % (what, e_psi, e_n, e_spp, e_sn))
    assert e_psi <= TOL[prec], (what, e_psi)
    assert e_n <= TOL[prec], (what, e_n)
    assert e_spp <= TOL[prec], (what, e_spp)
    assert e_sn <= TOL[prec], (what, e_sn)


@pytest.mark.parametrize("case,prec", [("res1024_f64", 64), ("res1024_f32", 32),
                                       ("spin256", 32)])
def test_single_handle_full_step_count(case, prec):
    g = golden(case)
    cfg, in_prec = make_longrun.case_input(case)
    assert in_prec == (64 if case.endswith("f64") else 32)
    steps = int(g["steps"])
    assert steps == cfg["steps"]
    h = make_handle(cfg["params"], prec, cfg["psi0"], cfg["n0"], cfg["P"])
    phx().phx_step_n(h, steps)
    psi, n = get_state(h, prec)
    compare(g, psi, n, prec, "%s (tile %d)" % (case, phx().phx_tile(h)))
    step, _ = phx().phx_time(h)
    assert step == steps


def test_ensemble_members_full_step_count():
    """The whole 256-member ensemble (64 each at 128^2 ... 1024^2) advanced
    as one batch for 5000 steps, as the benchmark runs it; three members
    compared with their oracle runs.  Members have their own time steps;
    every member takes 5000 steps."""
    m = phx()
    members = synth.ensemble()
    b = m.phx_batch_create([m.params_from_dict(x["params"], precision=32) for x in members])
    for i, x in enumerate(members):
        m.phx_batch_set_pump(b, i, np.ascontiguousarray(x["P"][0], np.float32))
        m.phx_batch_set_state(b, i, np.ascontiguousarray(x["psi0"][0], np.complex64),
                              np.ascontiguousarray(x["n0"][0], np.float32))
    m.phx_batch_step_n(b, 5000)
    for case, idx in (("ens128", 0), ("ens512", 128), ("ens1024", 192)):
        g = golden(case)
        d = members[idx]["params"]
        psi = np.empty((1, d["ny"], d["nx"]), np.complex64)
        n = np.empty((1, d["ny"], d["nx"]), np.float32)
        m.phx_batch_get_state(b, idx, psi, n)
        compare(g, psi, n, 32, "%s (member %d, batch tile %d)" % (case, idx, m.phx_batch_tile(b)))
    m.phx_batch_destroy(b)
