"""Several RK4 steps per launch (step-kernel configuration 8).

Configuration 8 runs the tiles of configuration 7 over many steps in one
persistent launch, each tile's load waiting for its neighbours' previous
step.  The arithmetic per site is that of configuration 7, so every result
must equal, bit for bit, configuration 7 stepped one launch at a time: state,
reservoir, step counter and FP64 time, noise included."""
import numpy as np
import pytest

import synth
from oracle import gp
from gpu_util import phx, make_handle, get_state, rel_l2, rounded
from test_gpu_parity import model

pytestmark = pytest.mark.gpu


def handles(d, tiles, seed=3, with_V=False, prec=32):
    psi0, n0, P, V = synth.random_state(1, d["ny"], d["nx"], seed, amp=0.7,
                                        reservoir=d["reservoir"], smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    out = []
    for t in tiles:
        m = phx()
        h = m.phx_create(m.params_from_dict(d, precision=prec, tile=t))
        if d["reservoir"]:
            m.phx_set_pump(h, np.ascontiguousarray(P[0], np.float32))
        if with_V:
            m.phx_set_potential(h, np.ascontiguousarray(V, np.float32))
        m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64),
                        None if n0 is None else np.ascontiguousarray(n0, np.float32))
        out.append(h)
    return out, (psi0, n0, P, V if with_V else None)


def assert_same(h7, h8):
    m = phx()
    a_psi, a_n = get_state(h7, 32)
    b_psi, b_n = get_state(h8, 32)
    assert np.array_equal(a_psi.view(np.uint32), b_psi.view(np.uint32))
    if a_n is not None:
        assert np.array_equal(a_n.view(np.uint32), b_n.view(np.uint32))
    assert m.phx_time(h7) == m.phx_time(h8)


@pytest.mark.parametrize("kind", ["reservoir", "conservative", "loss"])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("size", [(301, 157), (128, 512)])
def test_multistep_equals_single_steps(kind, bc, size):
    d = model(kind, size[0], size[1], bc=bc)
    (h7, h8), _ = handles(d, (7, 8), with_V=(kind == "loss"))
    m = phx()
    for _ in range(37):  # odd count: the state ends in the other buffer
        m.phx_step_n(h7, 1)
    m.phx_step_n(h8, 37)
    assert m.phx_tile(h8) == 8
    assert_same(h7, h8)


@pytest.mark.parametrize("steps", [2, 129, 300])
def test_multistep_chunks_and_noise(steps):
    """Chunk boundaries (128 steps per launch) and Philox noise keyed by the
    step index of each item."""
    d = model("reservoir", 520, 260, noise_var=1e-4)
    (h7, h8), _ = handles(d, (7, 8))
    m = phx()
    for _ in range(steps):
        m.phx_step_n(h7, 1)
    m.phx_step_n(h8, steps)
    assert_same(h7, h8)


def test_multistep_against_oracle():
    d = model("reservoir", 190, 133, bc=(0, 1))
    (h8,), (psi0, n0, P, V) = handles(d, (8,), seed=5)
    m = phx()
    m.phx_step_n(h8, 60)
    g_psi, g_n = get_state(h8, 32)
    o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 60)
    assert rel_l2(g_psi, o_psi) <= 1e-4
    assert rel_l2(g_n, o_n) <= 1e-4


def test_multistep_with_kfilter():
    """Launches end where the k-space filter applies (every 5 steps)."""
    d = model("reservoir", 256, 256)
    (h7, h8), _ = handles(d, (7, 8))
    m = phx()
    for h in (h7, h8):
        m.phx_set_kfilter(h, 3.0, 8, 5)
    for _ in range(23):
        m.phx_step_n(h7, 1)
    m.phx_step_n(h8, 23)
    assert_same(h7, h8)


def test_multistep_fallback_grid():
    """A grid whose tile count is within three tile rows of the persistent
    grid (2 CTAs per SM) steps one launch at a time: same results."""
    m = phx()
    # configuration 7: tiles of 58 x 26 outputs, tiles_x = (nx + 1 + 57) // 58
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    G = 2 * nsm
    nx = 8 * 58 - 1
    ty = G // 8
    d = model("reservoir", nx, ty * 26)
    (h7, h8), _ = handles(d, (7, 8))
    for _ in range(9):
        m.phx_step_n(h7, 1)
    m.phx_step_n(h8, 9)
    assert_same(h7, h8)


def test_multistep_reductions_and_time():
    d = model("reservoir", 333, 222)
    (h7, h8), _ = handles(d, (7, 8))
    m = phx()
    m.phx_step_n(h7, 50)
    m.phx_step_n(h8, 50)
    assert m.phx_time(h8)[0] == 50
    acc = 0.0
    for _ in range(50):
        acc += d["dt"]
    assert m.phx_time(h8)[1] == acc
    assert m.phx_norm_energy(h7) == m.phx_norm_energy(h8)
    assert m.phx_residual(h7) == m.phx_residual(h8)


def test_multistep_bounded_wait_timeout_recoverable():
    """A load that never completes (test hook) ends the launch through the
    bounded waits: the error is reported and the handle computes again."""
    m = phx()
    d = model("reservoir", 400, 300)
    (h8,), (psi0, n0, P, V) = handles(d, (8,), seed=2)
    m.phx_debug_inject(m.INJECT_TIMEOUT)
    m.phx_step_n(h8, 20)
    with pytest.raises(m.PhxError) as e:
        m.phx_norm_energy(h8)
    assert e.value.status == 5
    m.phx_set_state(h8, np.ascontiguousarray(psi0, np.complex64),
                    np.ascontiguousarray(n0, np.float32))
    m.phx_set_time(h8, 0, 0.0)
    m.phx_step_n(h8, 12)
    g_psi, g_n = get_state(h8, 32)
    o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 12)
    assert rel_l2(g_psi, o_psi) <= 1e-4
    assert rel_l2(g_n, o_n) <= 1e-4


def test_multistep_full_size_workload():
    """The 2048^2 reservoir workload (ring pump, noise-free), 40 steps."""
    m = phx()
    cfg = synth.reservoir_2048()
    hs = []
    for t in (7, 8):
        h = m.phx_create(m.params_from_dict(cfg["params"], precision=32, tile=t))
        m.phx_set_pump(h, np.ascontiguousarray(cfg["P"][0], np.float32))
        m.phx_set_state(h, np.ascontiguousarray(cfg["psi0"], np.complex64),
                        np.ascontiguousarray(cfg["n0"], np.float32))
        hs.append(h)
    for _ in range(40):
        m.phx_step_n(hs[0], 1)
    m.phx_step_n(hs[1], 40)
    assert_same(hs[0], hs[1])
