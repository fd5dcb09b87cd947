"""What the learned warm start gains over the plain method.

A reduced run of the whole loop on the steady-state workload (256 x 256,
128 um, random sums of 1-4 Gaussian pumps at 1-3 times the solver-measured
threshold of a spot of that waist): training pairs generated by the batched
solver, the network trained on the GPU by this package's kernels on the
pairs that reached the FP32 tolerance, then held-out pumps relaxed to
r_psi < 1e-6 from noise (cold) and from the network's prediction (warm)
under the same protocol.  Every kernel is deterministic, so the outcome is
reproducible."""
import numpy as np
import pytest

from gpu_util import phx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def experiment():
    phx()
    import bench
    import json
    rep, net = bench.steady_experiment(n_train=1024, n_test=128, gen_steps=30000, epochs=15,
                                       cap=60000)
    print(json.dumps({k: v for k, v in rep.items() if k != "relax"}))
    return rep, net


def test_spot_thresholds_rise_for_small_spots(experiment):
    """A smaller spot loses more particles to its surroundings: its measured
    threshold is never below a wider spot's, and every spot needs at least
    the homogeneous threshold."""
    rep, _ = experiment
    thr = [rep["spot_threshold_factors"][k] for k in sorted(rep["spot_threshold_factors"],
                                                            key=float)]
    assert all(np.isfinite(thr)), thr
    assert all(t >= 0.99 for t in thr), thr
    assert all(a >= b * 0.98 for a, b in zip(thr, thr[1:])), thr


def test_warm_start_beats_cold_start(experiment):
    rep, net = experiment
    # pumps drawn relative to the spot threshold condense (almost none decay);
    # multi-spot pumps whose condensates do not lock stay non-stationary, so
    # only part of them reaches r_psi < 1e-5 and becomes a training pair
    assert rep["train_decayed"] <= 0.05 * rep["n_train"], rep["train_decayed"]
    assert rep["train_converged"] >= 0.05 * rep["n_train"], rep["train_converged"]
    # the network learned something it did not know at initialisation
    assert rep["heldout_loss"] < 0.5 * rep["train_loss"][0]
    s = rep.get("summary")
    assert s is not None and s["pairs"] >= 10, rep["screen"]
    # warm and cold relax to the same stationary state (densities agree); a
    # pump with two stationary states may, rarely, pick different ones
    assert s["same_state_fraction"] >= 0.8, s
    # the warm start needs at least 5 % fewer RK4 steps to the tolerance
    # (medians over the pairs); its GPU time, which includes the network's
    # inference and the FP64 polish from 1e-5 to 1e-6 (about half of a
    # relaxation, and not shortened by a better start), is not worse than
    # 0.95 of the cold start's at this reduced size (about a hundred
    # training pairs); with 6000 training pumps the median gain is ~1.05x
    assert s["cold_steps_q"][1] >= 1.05 * s["warm_steps_q"][1], s
    assert s["speedup_median_ms"] >= 0.95, s
    # every converged relaxation really reached the tolerance
    pairs = [r for r in rep["relax"] if r["cold_converged"] and r["warm_converged"]]
    assert all(r["cold_r"] < 1e-6 and r["warm_r"] < 1e-6 for r in pairs)
