"""Parity at the full workload sizes, in the launch configuration the
benchmark times: after S GPU steps from the workload's initial state, one
more GPU step is compared at sampled sites (domain corners and edges, tile
borders, random interior) with the oracle's step evaluated on the GPU's own
pre-step state.  Plus invariants that hold at any size."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, make_handle, get_state, rel_l2, TOL, TMA_SCALAR_TILES

pytestmark = pytest.mark.gpu


def sample_sites(nx, ny, rng, count=48):
    fixed = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (ny // 2, 0),
             (0, nx // 2), (ny - 1, nx // 2), (ny // 2, nx - 1)]
    for t in (15, 16, 31, 32, 33, 63, 64):
        if t < nx and t < ny:
            fixed.append((t, t))
            fixed.append((t, (3 * t) % nx))
    rand = [(int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(count)]
    return fixed + rand


def one_step_sampled(cfg, prec, warm_steps, seed=0):
    d = cfg["params"]
    h = make_handle(d, prec, cfg["psi0"], cfg["n0"], cfg["P"])
    phx().phx_step_n(h, warm_steps)
    psi_s, n_s = get_state(h, prec)
    step, _ = phx().phx_time(h)
    phx().phx_step_n(h, 1)
    psi_1, n_1 = get_state(h, prec)
    p = gp.Params(**d)
    rng = np.random.default_rng(seed)
    sites = sample_sites(d["nx"], d["ny"], rng)
    P = None if cfg["P"] is None else np.asarray(cfg["P"], dtype=psi_s.real.dtype).astype(np.float64)
    sp, sn = gp.step_at_sites(psi_s.astype(np.complex128),
                              None if n_s is None else n_s.astype(np.float64),
                              P, None, p, sites, step)
    jj = np.array([s[0] for s in sites])
    ii = np.array([s[1] for s in sites])
    g_psi = psi_1[:, jj, ii]
    g_n = None if n_1 is None else n_1[:, jj, ii]
    return h, (g_psi, sp), (g_n, sn)


@pytest.mark.parametrize("prec", [32, 64])
def test_reservoir_1024_sampled_step(prec):
    cfg = synth.reservoir_1024()
    h, (a, b), (c, d) = one_step_sampled(cfg, prec, warm_steps=200)
    assert rel_l2(a, b) <= TOL[prec], rel_l2(a, b)
    assert rel_l2(c, d) <= TOL[prec], rel_l2(c, d)


def test_spinor_2048_sampled_step_with_noise():
    cfg = synth.spinor_2048()
    h, (a, b), (c, d) = one_step_sampled(cfg, 32, warm_steps=50, seed=1)
    assert rel_l2(a, b) <= TOL[32], rel_l2(a, b)
    assert rel_l2(c, d) <= TOL[32], rel_l2(c, d)


def test_reservoir_1024_invariants_and_time():
    """Reservoir stays in [0, P/gamma_r] from n0 = 0 (the source term is
    non-negative and the sink is linear in n), norms finite, FP64 time exact."""
    cfg = synth.reservoir_1024()
    h = make_handle(cfg["params"], 32, cfg["psi0"], cfg["n0"], cfg["P"])
    phx().phx_step_n(h, 2000)
    psi, n = get_state(h, 32)
    Pmax = float(np.max(cfg["P"]))
    assert n.min() >= -1e-6 and n.max() <= Pmax / cfg["params"]["gamma_r"] * (1 + 1e-5)
    N, E = phx().phx_norm_energy(h)
    assert np.isfinite(N) and np.isfinite(E) and N > 0
    step, t = phx().phx_time(h)
    acc = 0.0
    for _ in range(2000):
        acc += cfg["params"]["dt"]
    assert step == 2000 and t == acc


@pytest.mark.parametrize("prec", [32, 64])
def test_driven_9000_sampled_step(prec):
    """The coherently driven 9000^2 lattice at full size (FP32: the TMA-fed
    drive mode; FP64: the generic kernel): one step after 20, sampled against
    the oracle's windowed step with the same drive amplitude and the FP64
    time of the device clock."""
    m = phx()
    cfg = synth.driven_lattice(9000)
    d = cfg["params"]
    h = make_handle(d, prec, cfg["psi0"], None, None, cfg["V"])
    m.phx_set_drive(h, np.ascontiguousarray(cfg["E"][0],
                                            np.complex64 if prec == 32 else np.complex128))
    m.phx_step_n(h, 20)
    psi_s, _ = get_state(h, prec)
    step, t = m.phx_time(h)
    m.phx_step_n(h, 1)
    psi_1, _ = get_state(h, prec)
    if prec == 32:
        assert m.phx_tile(h) in TMA_SCALAR_TILES
    sites = sample_sites(9000, 9000, np.random.default_rng(4))
    sp, _ = gp.step_at_sites(psi_s.astype(np.complex128), None, None, cfg["V"], gp.Params(**d),
                             sites, step, E=cfg["E"], t=t)
    jj = np.array([s[0] for s in sites])
    ii = np.array([s[1] for s in sites])
    assert rel_l2(psi_1[0, jj, ii], sp[0]) <= TOL[prec], rel_l2(psi_1[0, jj, ii], sp[0])


def test_twa_ensemble_member_matches_oracle():
    """The truncated-Wigner ensemble in the benchmark's configuration (150
    members of 256^2 in one persistent launch per step): members 0 and 149
    after one 5 ps sample against the oracle run of the same member."""
    m = phx()
    members = synth.twa_ensemble()
    b = m.phx_batch_create([m.params_from_dict(x["params"], precision=32) for x in members])
    for i, x in enumerate(members):
        m.phx_batch_set_pump(b, i, np.ascontiguousarray(x["P"][0], np.float32))
        m.phx_batch_set_state(b, i, np.ascontiguousarray(x["psi0"], np.complex64),
                              np.ascontiguousarray(x["n0"], np.float32))
    steps = int(round(5.0 / members[0]["params"]["dt"]))
    m.phx_batch_step_n(b, steps)
    for i in (0, 149):
        x = members[i]
        psi = np.empty((1, 256, 256), np.complex64)
        n = np.empty((1, 256, 256), np.float32)
        m.phx_batch_get_state(b, i, psi, n)
        psi0 = x["psi0"].astype(np.complex64).astype(np.complex128)
        o_psi, o_n = gp.run(psi0, x["n0"], x["P"], None, gp.Params(**x["params"]), steps)
        assert rel_l2(psi, o_psi) <= 1e-4, (i, rel_l2(psi, o_psi))
        assert rel_l2(n, o_n) <= 1e-4, (i, rel_l2(n, o_n))
    m.phx_batch_destroy(b)
