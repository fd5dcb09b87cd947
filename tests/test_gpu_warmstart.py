"""What the learned warm start gains over the plain method.

A reduced run of the whole loop on the steady-state workload (256 x 256,
128 um, random sums of 1-4 Gaussian pumps at 1-3 P_thr): training pairs
generated by the batched solver, the network trained on the GPU by this
package's kernels, then held-out pumps relaxed to r_psi < 1e-6 from noise
(cold) and from the network's prediction (warm) under the same protocol.
Every kernel is deterministic, so the outcome is reproducible."""
import numpy as np
import pytest

from gpu_util import phx

pytestmark = pytest.mark.gpu


def test_warm_start_beats_cold_start():
    phx()
    from paper_2411_18341_gb300 import warmstart
    rep, net = warmstart.run_experiment(n_train=192, n_test=96, gen_steps=30000, epochs=12,
                                        cap=60000, log=lambda s: None)
    # the network learned something it did not know at initialisation
    assert rep["heldout_loss"] < 0.5 * rep["train_loss"][0]
    s = rep.get("summary")
    assert s is not None and s["pairs"] >= 3, rep["screen"]
    # warm and cold relax to the same stationary state (densities agree); a
    # pump with two stationary states may, rarely, pick different ones
    assert s["same_state_fraction"] >= 0.75, s
    # the warm start gets there in fewer steps and less GPU time, per pump
    # (medians over the pairs) and on most pumps
    assert s["warm_steps_q"][1] < s["cold_steps_q"][1], s
    assert s["speedup_median_ms"] > 1.0, s
    assert s["warm_faster_fraction"] >= 0.5, s
    # every converged relaxation really reached the tolerance
    pairs = [r for r in rep["relax"] if r["cold_converged"] and r["warm_converged"]]
    assert all(r["cold_r"] < 1e-6 and r["warm_r"] < 1e-6 for r in pairs)
