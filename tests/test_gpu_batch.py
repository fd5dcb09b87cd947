"""Batches: many independent FP32 scalar instances on uneven grids advanced
by one persistent launch per step (CUDA-graph replay).  Members are checked
against the oracle and against single handles, including graph and non-graph
step counts, per-member reductions and FP64 times."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, make_handle, get_state, rel_l2, rounded

pytestmark = pytest.mark.gpu


def members(sizes, reservoir=True, seed0=40, bc=(0, 0)):
    out = []
    for k, (nx, ny) in enumerate(sizes):
        d = synth.base_params(nx, ny, 0.3 * nx, 0.3 * ny, bc_x=bc[0], bc_y=bc[1],
                              g=0.2 + 0.01 * k, seed=seed0 + k, instance=k)
        if reservoir:
            d.update({kk: v for kk, v in synth.reservoir_physics().items() if kk != "g"})
            d.update(g_r=0.4, R=0.2 + 0.02 * k, gamma_r=0.3)
        else:
            d.update(gamma_c=0.1)
        d["dt"] = min((0.3 + 0.02 * k) * gp.stability_dt_max(gp.Params(**d)), 0.05)
        psi0, n0, P, V = synth.random_state(1, ny, nx, seed0 + k, amp=0.6,
                                            reservoir=reservoir, smooth=True)
        out.append((d, rounded(psi0, 32), rounded(n0, 32), rounded(P, 32)))
    return out


def make_batch(ms, tile=0):
    m = phx()
    b = m.phx_batch_create([m.params_from_dict(d, precision=32, tile=tile) for d, *_ in ms])
    for i, (d, psi0, n0, P) in enumerate(ms):
        if P is not None:
            m.phx_batch_set_pump(b, i, np.ascontiguousarray(P[0], np.float32))
        m.phx_batch_set_state(b, i, np.ascontiguousarray(psi0, np.complex64),
                              None if n0 is None else np.ascontiguousarray(n0, np.float32))
    return b


def member_state(b, i, d):
    m = phx()
    psi = np.empty((1, d["ny"], d["nx"]), np.complex64)
    n = np.empty((1, d["ny"], d["nx"]), np.float32) if b.reservoir else None
    m.phx_batch_get_state(b, i, psi, n)
    return psi, n


SIZES = [(40, 33), (96, 70), (130, 57), (64, 200), (17, 150), (256, 96)]


@pytest.mark.parametrize("steps", [7, 20, 45])
@pytest.mark.parametrize("reservoir", [True, False])
def test_batch_members_match_oracle(steps, reservoir):
    ms = members(SIZES, reservoir)
    b = make_batch(ms)
    phx().phx_batch_step_n(b, steps)
    for i, (d, psi0, n0, P) in enumerate(ms):
        g_psi, g_n = member_state(b, i, d)
        o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), steps)
        assert rel_l2(g_psi, o_psi) <= 1e-4, (i, rel_l2(g_psi, o_psi))
        if reservoir:
            assert rel_l2(g_n, o_n) <= 1e-4


@pytest.mark.parametrize("tile", [1, 3, 4, 6, 7])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0)])
def test_batch_fixed_tile_configs(tile, bc):
    """Every member against the oracle with the step kernel configuration
    fixed (the per-tile instance table of the persistent kernel), uneven
    grids, graph and non-graph step counts."""
    ms = members(SIZES, True, bc=bc)
    b = make_batch(ms, tile=tile)
    phx().phx_batch_step_n(b, 27)
    assert phx().phx_batch_tile(b) == tile
    for i, (d, psi0, n0, P) in enumerate(ms):
        g_psi, g_n = member_state(b, i, d)
        o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 27)
        assert rel_l2(g_psi, o_psi) <= 1e-4, (i, rel_l2(g_psi, o_psi))
        assert rel_l2(g_n, o_n) <= 1e-4


def test_batch_equals_single_handles_and_zero_bc():
    ms = members(SIZES[:4], True, bc=(1, 0))
    b = make_batch(ms)
    phx().phx_batch_step_n(b, 33)
    for i, (d, psi0, n0, P) in enumerate(ms):
        h = make_handle(d, 32, psi0, n0, P)
        phx().phx_step_n(h, 33)
        s_psi, s_n = get_state(h, 32)
        g_psi, g_n = member_state(b, i, d)
        assert rel_l2(g_psi, s_psi) <= 1e-6
        assert rel_l2(g_n, s_n) <= 1e-6


def test_batch_reductions_and_times():
    m = phx()
    ms = members(SIZES[:5], True)
    b = make_batch(ms)
    m.phx_batch_step_n(b, 24)
    N, E = m.phx_batch_norm_energy(b)
    r, rn, om = m.phx_batch_residual(b)
    step, t = m.phx_batch_time(b)
    assert step == 24
    for i, (d, psi0, n0, P) in enumerate(ms):
        g_psi, g_n = member_state(b, i, d)
        p = gp.Params(**d)
        gpsi = g_psi.astype(np.complex128)
        gn = g_n.astype(np.float64)
        assert abs(N[i] - gp.norm(gpsi, p)) <= 1e-12 * N[i]
        Eo = gp.energy(gpsi, gn, None, p)
        assert abs(E[i] - Eo) <= 1e-11 * max(abs(Eo), 1.0)
        ro, rno, omo = gp.residual(gpsi, gn, P, None, p)
        assert abs(r[i] - ro) <= 1e-10 * ro and abs(rn[i] - rno) <= 1e-10 * rno
        acc = 0.0
        for _ in range(24):
            acc += d["dt"]
        assert t[i] == acc


def test_batch_validation():
    m = phx()
    d = synth.base_params(32, 32, 10.0, 10.0, dt=1e-3)
    with pytest.raises(m.PhxError) as e:
        m.phx_batch_create([m.params_from_dict(d, precision=64)])
    assert e.value.status == 1
    d2 = dict(d, reservoir=True)
    with pytest.raises(m.PhxError) as e:
        m.phx_batch_create([m.params_from_dict(d), m.params_from_dict(d2)])
    assert e.value.status == 1
    with pytest.raises(m.PhxError) as e:
        m.phx_batch_create([m.params_from_dict(dict(d, nx=4))])
    assert e.value.status == 1


def drive_plane(nx, ny, seed, amp=0.4):
    rng = np.random.default_rng(seed)
    y = np.arange(ny)[:, None] / ny
    x = np.arange(nx)[None, :] / nx
    a, b2, ph = rng.uniform(1, 3, 3)
    return (amp * (np.cos(2 * np.pi * a * x + ph) + 0.5j * np.sin(2 * np.pi * b2 * y))
            ).astype(np.complex64)


def driven_members(reservoir, sizes=SIZES, bc=(0, 0)):
    """Members with their own drive frequencies; member 2 has no drive."""
    ms = members(sizes, reservoir, bc=bc)
    E = {}
    for k, (d, *_) in enumerate(ms):
        d["drive_omega"] = 0.5 + 0.3 * k
        if k != 2:
            E[k] = drive_plane(d["nx"], d["ny"], 70 + k)
    return ms, E


@pytest.mark.parametrize("tile", [0, 3, 4])
@pytest.mark.parametrize("reservoir", [True, False])
def test_batch_drive_members_match_oracle(tile, reservoir):
    """Coherent drive E_i(r) exp(-i omega_i t_i) per member (Eq. PULSE_psi)
    in the batched persistent kernel: each member's own frequency and FP64
    time, a member without drive among driven ones, graph and single-launch
    steps (23 = one replay of 20 + 3)."""
    m = phx()
    ms, E = driven_members(reservoir)
    b = make_batch(ms, tile=tile)
    for i, Ei in E.items():
        m.phx_batch_set_drive(b, i, Ei)
    m.phx_batch_step_n(b, 23)
    if reservoir:
        assert m.phx_batch_tile(b) in (2, 3, 4)
    for i, (d, psi0, n0, P) in enumerate(ms):
        g_psi, g_n = member_state(b, i, d)
        o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 23,
                            E=E[i].astype(np.complex128) if i in E else None)
        assert rel_l2(g_psi, o_psi) <= 1e-4, (i, rel_l2(g_psi, o_psi))
        if reservoir:
            assert rel_l2(g_n, o_n) <= 1e-4, (i, rel_l2(g_n, o_n))


def test_batch_drive_equals_single_handles():
    """Batch members with a drive against driven single handles (zero x
    boundary, reservoir), and a member whose drive is set and then removed
    against an undriven handle."""
    m = phx()
    ms, E = driven_members(True, SIZES[:4], bc=(1, 0))
    b = make_batch(ms)
    for i, Ei in E.items():
        m.phx_batch_set_drive(b, i, Ei)
    m.phx_batch_set_drive(b, 3, None)
    m.phx_batch_step_n(b, 31)
    for i, (d, psi0, n0, P) in enumerate(ms):
        h = make_handle(d, 32, psi0, n0, P)
        if i in E and i != 3:
            m.phx_set_drive(h, E[i])
        m.phx_step_n(h, 31)
        s_psi, s_n = get_state(h, 32)
        g_psi, g_n = member_state(b, i, d)
        assert rel_l2(g_psi, s_psi) <= 1e-6, (i, rel_l2(g_psi, s_psi))
        assert rel_l2(g_n, s_n) <= 1e-6


def test_batch_drive_fixed_tile_without_variant():
    m = phx()
    ms, E = driven_members(True, SIZES[:2])
    b = make_batch(ms, tile=7)
    m.phx_batch_set_drive(b, 0, E[0])
    with pytest.raises(m.PhxError) as e:
        m.phx_batch_step_n(b, 2)
    assert e.value.status == 1
