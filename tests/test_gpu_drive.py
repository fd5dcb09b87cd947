"""Coherent drive E_c(r) exp(-i omega t) (Eq. PULSE_psi, Sec. V) through the
C ABI against the oracle: every model, FP64 (1e-11) and FP32 (1e-4), ragged
grids, periodic and zero boundaries, a time origin other than zero, separate
and shared drive planes, together with truncated-Wigner noise."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, get_state, rel_l2, rounded, TOL, TMA_SCALAR_TILES

pytestmark = pytest.mark.gpu


def drive_model(kind, nx, ny, bc=(0, 0), omega=2.3):
    d = synth.base_params(nx, ny, 0.3 * nx, 0.3 * ny, bc_x=bc[0], bc_y=bc[1])
    if kind == "loss":
        d.update(g=0.3, gamma_c=0.2)
    elif kind == "reservoir":
        d.update(synth.reservoir_physics())
        d.update(g=0.3, g_r=0.5, R=0.3, gamma_r=0.4)
    elif kind == "spinor_tetm":
        d.update(spinor=True, g=0.3, g_x=0.1, delta_lt=0.2, gamma_c=0.05)
    elif kind == "spinor_res_tetm":
        d.update(synth.reservoir_physics())
        d.update(spinor=True, g=0.3, g_x=0.1, g_r=0.4, R=0.3, delta_lt=0.2)
    d.update(drive_omega=omega, seed=29)
    d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    return d


def smooth_field(nc, ny, nx, seed, amp):
    rng = np.random.default_rng(seed)
    y = np.arange(ny)[:, None] / ny
    x = np.arange(nx)[None, :] / nx
    out = np.empty((nc, ny, nx), complex)
    for c in range(nc):
        a, b, ph = rng.uniform(1, 3, 3)
        out[c] = amp * (np.cos(2 * np.pi * a * x + ph) + 0.5j * np.sin(2 * np.pi * b * y)) \
            + 0.05 * amp * (rng.normal(size=(ny, nx)) + 1j * rng.normal(size=(ny, nx)))
    return out


def run_driven(d, prec, E, shared, steps, tile=0, t0=3.7, step0=50):
    m = phx()
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    nc = 2 if d["spinor"] else 1
    psi0, n0, P, V = synth.random_state(nc, d["ny"], d["nx"], 12, amp=0.6,
                                        reservoir=d["reservoir"], smooth=True)
    if not d["reservoir"]:
        n0 = P = None
    E = rounded(E, prec)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=prec, tile=tile))
    if d["reservoir"]:
        m.phx_set_pump(h, *[np.ascontiguousarray(P[c], real) for c in range(nc)])
    m.phx_set_potential(h, np.ascontiguousarray(V, real))
    if shared or nc == 1:
        m.phx_set_drive(h, np.ascontiguousarray(E[0], cplx))
        E_or = np.broadcast_to(E[0], (nc,) + E.shape[1:])
    else:
        m.phx_set_drive(h, np.ascontiguousarray(E[0], cplx), np.ascontiguousarray(E[1], cplx))
        E_or = E
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx),
                    None if n0 is None else np.ascontiguousarray(n0, real))
    m.phx_set_time(h, step0, t0)
    m.phx_step_n(h, steps)
    g_psi, g_n = get_state(h, prec)
    o_psi, o_n = gp.run(psi0, n0, P, V, gp.Params(**d), steps, step0=step0, E=E_or, t0=t0)
    return h, (g_psi, g_n), (o_psi, o_n)


KINDS = ["loss", "reservoir", "spinor_tetm", "spinor_res_tetm"]
# tile configurations of the TMA-fed kernel with the reservoir-and-drive variant
DRIVE_RES_TILES = (2, 3, 4)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("shared", [False, True])
def test_drive_parity(prec, kind, bc, shared):
    d = drive_model(kind, 131, 77, bc=bc)
    nc = 2 if d["spinor"] else 1
    if nc == 1 and shared:
        pytest.skip("one component")
    E = smooth_field(nc, 77, 131, 3, 0.4)
    h, (g_psi, g_n), (o_psi, o_n) = run_driven(d, prec, E, shared, steps=11)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    if d["reservoir"]:
        assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)


@pytest.mark.parametrize("prec", [64, 32])
def test_drive_changes_the_state_and_can_be_removed(prec):
    """The drive's contribution is far above the tolerance; removing it
    (E_plus = NULL) gives the undriven trajectory, and the FP32 step returns
    to the TMA-fed kernel."""
    m = phx()
    d = drive_model("reservoir", 97, 66)
    E = smooth_field(1, 66, 97, 4, 0.5)
    h, (g_psi, _), (o_psi, _) = run_driven(d, prec, E, False, steps=9)
    assert rel_l2(g_psi, o_psi) <= TOL[prec]
    psi0, n0, P, V = synth.random_state(1, 66, 97, 12, amp=0.6, smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    u_psi, _ = gp.run(psi0, n0, P, V, gp.Params(**d), 9)
    assert rel_l2(u_psi, o_psi) > 100 * TOL[prec]
    if prec == 32:
        assert m.phx_tile(h) in DRIVE_RES_TILES
    m.phx_set_drive(h, None)
    real, cplx = (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx), np.ascontiguousarray(n0, real))
    m.phx_set_time(h, 0, 0.0)
    m.phx_step_n(h, 9)
    g2, _ = get_state(h, prec)
    assert rel_l2(g2, u_psi) <= TOL[prec]
    if prec == 32:
        assert m.phx_tile(h) in TMA_SCALAR_TILES


@pytest.mark.parametrize("prec", [64, 32])
def test_drive_with_truncated_wigner_noise(prec):
    d = drive_model("reservoir", 83, 58)
    d.update(wigner_nu=0.7, gamma_r=4.0)
    E = smooth_field(1, 58, 83, 5, 0.3)
    h, (g_psi, g_n), (o_psi, o_n) = run_driven(d, prec, E, False, steps=8)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)


@pytest.mark.parametrize("tile", [9, 10, 11, 12])
def test_drive_fp32_spinor_generic_shapes(tile):
    d = drive_model("spinor_res_tetm", 70, 45)
    E = smooth_field(2, 45, 70, 6, 0.4)
    h, (g_psi, g_n), (o_psi, o_n) = run_driven(d, 32, E, False, steps=7, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4
    assert rel_l2(g_n, o_n) <= 1e-4


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (0, 1)])
def test_drive_tma_scalar_kernel(tile, bc):
    """FP32 scalar field without reservoir: the drive runs in the TMA-fed
    persistent kernel (Re / Im planes staged like the reservoir's) in every
    tile configuration, ragged grid, with a potential."""
    m = phx()
    d = drive_model("loss", 131, 77, bc=bc)
    E = smooth_field(1, 77, 131, 8, 0.4)
    h, (g_psi, _), (o_psi, _) = run_driven(d, 32, E, False, steps=11, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert m.phx_tile(h) in TMA_SCALAR_TILES
    if tile:
        assert m.phx_tile(h) == tile


@pytest.mark.parametrize("tile", [0, 6])
def test_drive_tma_with_truncated_wigner_noise(tile):
    d = drive_model("loss", 97, 66)
    d.update(wigner_nu=1.2, noise_var=1e-5)
    E = smooth_field(1, 66, 97, 9, 0.3)
    h, (g_psi, _), (o_psi, _) = run_driven(d, 32, E, False, steps=9, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert phx().phx_tile(h) in TMA_SCALAR_TILES


@pytest.mark.parametrize("tile", [0, 2, 3, 4])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (0, 1)])
def test_drive_reservoir_tma_kernel(tile, bc):
    """FP32 scalar field with reservoir and drive: the TMA-fed kernel stages
    n, P, Re E, Im E and V per tile (configurations 2, 3, 4), ragged grid."""
    m = phx()
    d = drive_model("reservoir", 131, 77, bc=bc)
    E = smooth_field(1, 77, 131, 10, 0.4)
    h, (g_psi, g_n), (o_psi, o_n) = run_driven(d, 32, E, False, steps=11, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= 1e-4, rel_l2(g_n, o_n)
    assert m.phx_tile(h) in DRIVE_RES_TILES
    if tile:
        assert m.phx_tile(h) == tile


@pytest.mark.parametrize("tile", [1, 5, 6, 7])
def test_drive_reservoir_fixed_tile_without_variant(tile):
    """A fixed tile configuration without the reservoir-and-drive variant
    steps on the generic kernel: same results, reported as tile 9."""
    m = phx()
    d = drive_model("reservoir", 97, 66, bc=(1, 1))
    E = smooth_field(1, 66, 97, 11, 0.4)
    h, (g_psi, g_n), (o_psi, o_n) = run_driven(d, 32, E, False, steps=7, tile=tile)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= 1e-4, rel_l2(g_n, o_n)
    assert m.phx_tile(h) == 9


def test_drive_set_after_tuning_retunes():
    """A reservoir handle tuned without a drive (any configuration) is tuned
    again when a drive is set, among the configurations with that variant;
    the trajectory (undriven steps, then driven ones) matches the oracle."""
    m = phx()
    d = drive_model("reservoir", 301, 157, bc=(1, 1))
    psi0, n0, P, V = synth.random_state(1, 157, 301, 13, amp=0.6, smooth=True)
    psi0, n0, P = (rounded(x, 32) for x in (psi0, n0, P))
    E = rounded(smooth_field(1, 157, 301, 12, 0.4), 32)
    h = m.phx_create(m.params_from_dict(d, precision=32))
    m.phx_set_pump(h, np.ascontiguousarray(P[0], np.float32))
    m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64),
                    np.ascontiguousarray(n0, np.float32))
    m.phx_step_n(h, 5)
    assert m.phx_tile(h) in TMA_SCALAR_TILES + [8]
    m.phx_set_drive(h, np.ascontiguousarray(E[0], np.complex64))
    m.phx_step_n(h, 6)
    assert m.phx_tile(h) in DRIVE_RES_TILES
    g_psi, g_n = get_state(h, 32)
    p = gp.Params(**d)
    o_psi, o_n = gp.run(psi0, n0, P, None, p, 5)
    t5 = 0.0
    for _ in range(5):
        t5 += d["dt"]
    o_psi, o_n = gp.run(o_psi, o_n, P, None, p, 6, step0=5, E=E, t0=t5)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= 1e-4, rel_l2(g_n, o_n)
