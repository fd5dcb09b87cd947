"""GPU (C-ABI, sm_103a kernels) vs the FP64 oracle on the same seeded inputs.

Tolerances: relative L2 <= 1e-11 for FP64 and <= 1e-4 for FP32 stencils;
noise bit-exact.  Sizes span several tiles plus ragged tails; edge cases
cover tiny grids, zero / mixed boundaries, potentials and every model."""
import numpy as np
import pytest

from oracle import gp, noise
import synth
from gpu_util import phx, make_handle, get_state, rel_l2, rounded, TOL, types

pytestmark = pytest.mark.gpu


def model(kind, nx, ny, bc=(0, 0), noise_var=0.0, L=None):
    L = L or (0.3 * nx, 0.3 * ny)
    d = synth.base_params(nx, ny, L[0], L[1], bc_x=bc[0], bc_y=bc[1])
    if kind == "conservative":
        d.update(g=0.3)
    elif kind == "loss":
        d.update(g=0.3, gamma_c=0.2)
    elif kind == "reservoir":
        d.update(synth.reservoir_physics())
        d.update(g=0.3, g_r=0.5, R=0.3, gamma_r=0.4)
    elif kind == "spinor":
        d.update(spinor=True, g=0.3, g_x=0.1, gamma_c=0.05)
    elif kind == "spinor_tetm":
        d.update(spinor=True, g=0.3, g_x=0.1, delta_lt=0.2, gamma_c=0.05)
    elif kind == "spinor_res_tetm":
        d.update(synth.reservoir_physics())
        d.update(spinor=True, g=0.3, g_x=0.1, g_r=0.4, R=0.3, delta_lt=0.2)
    d["noise_var"] = noise_var
    d["seed"] = 17
    p = gp.Params(**d)
    d["dt"] = min(0.45 * gp.stability_dt_max(p), 0.05)
    return d


def run_both(d, prec, steps, seed=1, with_V=True, amp=0.7):
    nc = 2 if d["spinor"] else 1
    psi0, n0, P, V = synth.random_state(nc, d["ny"], d["nx"], seed, amp=amp,
                                        reservoir=d["reservoir"], smooth=True)
    if not with_V:
        V = None
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = make_handle(d, prec, psi0, n0, P, V)
    phx().phx_step_n(h, steps)
    g_psi, g_n = get_state(h, prec)
    o_psi, o_n = gp.run(psi0, n0, P, V, gp.Params(**d), steps)
    return h, (g_psi, g_n), (o_psi, o_n)


KINDS = ["conservative", "loss", "reservoir", "spinor", "spinor_tetm", "spinor_res_tetm"]
SIZES = [(37, 29), (70, 45), (16, 16), (33, 64)]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("size", SIZES)
def test_parity_models(prec, kind, size):
    d = model(kind, *size)
    h, (gp_, gn), (op, on) = run_both(d, prec, steps=12)
    assert rel_l2(gp_, op) <= TOL[prec], rel_l2(gp_, op)
    if d["reservoir"]:
        assert rel_l2(gn, on) <= TOL[prec], rel_l2(gn, on)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("bc", [(1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("kind", ["reservoir", "spinor_res_tetm"])
def test_parity_zero_and_mixed_boundaries(prec, bc, kind):
    d = model(kind, 45, 38, bc=bc)
    h, (gp_, gn), (op, on) = run_both(d, prec, steps=10)
    assert rel_l2(gp_, op) <= TOL[prec]
    if d["reservoir"]:
        assert rel_l2(gn, on) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("size", [(1, 1), (2, 3), (4, 4), (5, 3), (3, 7), (9, 1)])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1)])
def test_tiny_grids(prec, size, bc):
    d = model("spinor_res_tetm", *size, bc=bc, L=(0.5 * size[0], 0.5 * size[1]))
    h, (gp_, gn), (op, on) = run_both(d, prec, steps=7)
    assert rel_l2(gp_, op) <= TOL[prec]
    assert rel_l2(gn, on) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_noise_run_parity(prec):
    d = model("spinor_res_tetm", 40, 36, noise_var=1e-3)
    h, (gp_, gn), (op, on) = run_both(d, prec, steps=9)
    assert rel_l2(gp_, op) <= TOL[prec]
    assert rel_l2(gn, on) <= TOL[prec]


def test_noise_sample_bit_exact():
    import torch
    for (seed, step, inst, nc, nx, ny, var) in [(3, 0, 0, 2, 64, 33, 1e-3),
                                                (2 ** 40 + 7, 2 ** 33 + 5, 9, 1, 17, 5, 0.5),
                                                (0, 12345, 3, 2, 300, 2, 2.0)]:
        out = torch.empty(nc * ny * nx * 2, dtype=torch.float32, device="cuda")
        phx().phx_noise_sample(seed, step, inst, nc, nx, ny, var, out)
        torch.cuda.synchronize()
        g = out.cpu().numpy().reshape(nc, ny, nx, 2)
        re, im = noise.noise_field(seed, step, inst, nc, ny, nx, var)
        assert np.array_equal(g[..., 0].view(np.uint32), re.view(np.uint32))
        assert np.array_equal(g[..., 1].view(np.uint32), im.view(np.uint32))


@pytest.mark.parametrize("prec", [32, 64])
def test_noise_enters_step_bit_exact(prec):
    """kappa = 0 and no other term: one step from psi = 0 gives exactly xi."""
    d = synth.base_params(50, 21, 5.0, 2.1, kappa=0.0, spinor=True, noise_var=3e-3,
                          seed=99, dt=0.01)
    h = make_handle(d, prec, np.zeros((2, 21, 50)))
    phx().phx_set_time(h, 41, 0.0)
    phx().phx_step_n(h, 1)
    g, _ = get_state(h, prec)
    re, im = noise.noise_field(99, 41, 0, 2, 21, 50, 3e-3)
    assert np.array_equal(g.real.astype(np.float32), re)
    assert np.array_equal(g.imag.astype(np.float32), im)
    if prec == 64:
        assert np.array_equal(g.real, re.astype(np.float64))


def test_conservative_64_full_run_fp64():
    """64x64 conservative GP, 1000 FP64 steps at half the stability limit."""
    cfg = synth.conservative_64()
    d = cfg["params"]
    h = make_handle(d, 64, cfg["psi0"])
    phx().phx_step_n(h, cfg["steps"])
    g, _ = get_state(h, 64)
    p = gp.Params(**d)
    o, _ = gp.run(cfg["psi0"], None, None, None, p, cfg["steps"])
    assert rel_l2(g, o) <= 1e-11
    N, E = phx().phx_norm_energy(h)
    assert abs(N - gp.norm(o, p)) <= 1e-12 * abs(N)
    assert abs(E - gp.energy(o, None, None, p)) <= 1e-11 * abs(E)
    step, t = phx().phx_time(h)
    acc = 0.0
    for _ in range(cfg["steps"]):
        acc += d["dt"]
    assert step == cfg["steps"] and t == acc


@pytest.fixture(scope="module")
def reservoir_long_reference():
    """Reservoir GP at the 1024^2 workload's dx (100/1024 um) and dt
    (half the RK4 limit), on a 64x64 window with a ring pump of radius 2 um
    and width 0.5 um at 1.5 P_thr, noise 1e-2 initial state, 10^4 steps."""
    c = synth.load_constants()
    n, L = 64, 64 * 100.0 / 1024
    d = synth.base_params(n, n, L, L, dt=c["reservoir_1024_L100"]["dt"],
                          **synth.reservoir_physics())
    P = synth.ring(n, n, L, L, 1.5 * c["pump_threshold"], 2.0, 0.5)[None]
    psi0 = synth.complex_normal((1, n, n), 1e-2, 2)
    n0 = np.zeros((1, n, n))
    p = gp.Params(**d)
    out = {}
    for prec in (64, 32):
        psi0r, Pr = rounded(psi0, prec), rounded(P, prec)
        out[prec] = (psi0r, Pr, gp.run(psi0r, n0, Pr, None, p, 10000))
    return d, n0, out


@pytest.mark.parametrize("prec", [64, 32])
def test_reservoir_long_run(reservoir_long_reference, prec):
    d, n0, ref = reservoir_long_reference
    psi0, P, (o_psi, o_n) = ref[prec]
    h = make_handle(d, prec, psi0, n0, P)
    phx().phx_step_n(h, 10000)
    g_psi, g_n = get_state(h, prec)
    assert rel_l2(g_psi, o_psi) <= TOL[prec], rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= TOL[prec], rel_l2(g_n, o_n)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["reservoir", "spinor_res_tetm", "conservative"])
@pytest.mark.parametrize("bc", [(0, 0), (1, 0)])
def test_reductions_match_oracle(prec, kind, bc):
    d = model(kind, 41, 27, bc=bc)
    nc = 2 if d["spinor"] else 1
    psi0, n0, P, V = synth.random_state(nc, 27, 41, 4, amp=0.8,
                                        reservoir=d["reservoir"], smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    h = make_handle(d, prec, psi0, n0, P, V)
    p = gp.Params(**d)
    N, E = phx().phx_norm_energy(h)
    assert abs(N - gp.norm(psi0, p)) <= 1e-12 * abs(N)
    Eo = gp.energy(psi0, n0, V, p)
    assert abs(E - Eo) <= 1e-11 * max(abs(Eo), 1.0)
    r, rn, om = phx().phx_residual(h)
    Pn = None if P is None else np.broadcast_to(P, (nc, 27, 41))
    ro, rno, omo = gp.residual(psi0, n0, Pn, V, p)
    assert abs(r - ro) <= 1e-10 * ro
    assert abs(om - omo) <= 1e-10 * max(abs(omo), 1.0)
    if d["reservoir"]:
        assert abs(rn - rno) <= 1e-10 * rno


@pytest.mark.parametrize("prec", [32, 64])
def test_checkpoint_resume_bit_exact(prec):
    d = model("spinor_res_tetm", 48, 40, noise_var=1e-4)
    psi0, n0, P, V = synth.random_state(2, 40, 48, 8, amp=0.5, smooth=True)
    h = make_handle(d, prec, psi0, n0, P, V)
    phx().phx_step_n(h, 14)
    full_psi, full_n = get_state(h, prec)
    h2 = make_handle(d, prec, psi0, n0, P, V)
    phx().phx_step_n(h2, 7)
    mid_psi, mid_n = get_state(h2, prec)
    step, t = phx().phx_time(h2)
    phx().phx_destroy(h2)
    h3 = make_handle(d, prec, mid_psi, mid_n, P, V)
    phx().phx_set_time(h3, step, t)
    phx().phx_step_n(h3, 7)
    res_psi, res_n = get_state(h3, prec)
    assert np.array_equal(full_psi.view(np.uint8), res_psi.view(np.uint8))
    assert np.array_equal(full_n.view(np.uint8), res_n.view(np.uint8))
    assert phx().phx_time(h3)[0] == 14


def test_zero_steps_and_errors():
    m = phx()
    d = model("reservoir", 20, 20)
    psi0, n0, P, V = synth.random_state(1, 20, 20, 1)
    h = make_handle(d, 32, psi0, n0, P)
    before, _ = get_state(h, 32)
    m.phx_step_n(h, 0)
    after, _ = get_state(h, 32)
    assert np.array_equal(before, after)
    with pytest.raises(m.PhxError) as e:
        m.phx_step_n(h, -1)
    assert e.value.status == 1
    h2 = make_handle(model("conservative", 8, 8), 32, np.zeros((1, 8, 8)))
    with pytest.raises(m.PhxError) as e:
        m.phx_set_pump(h2, np.zeros(64, np.float32))
    assert e.value.status == 6
    with pytest.raises(m.PhxError) as e:
        m.phx_create(m.params_from_dict(dict(d, dt=10.0)))
    assert e.value.status == 1


def test_nonfinite_state_reported():
    m = phx()
    d = model("conservative", 16, 16)
    psi = np.zeros((1, 16, 16), complex)
    psi[0, 3, 4] = np.nan
    h = make_handle(d, 64, psi)
    with pytest.raises(m.PhxError) as e:
        m.phx_norm_energy(h)
    assert e.value.status == 4


def test_device_pointers_and_torch_stream():
    import torch
    m = phx()
    d = model("spinor_res_tetm", 30, 22)
    psi0, n0, P, V = synth.random_state(2, 22, 30, 2, amp=0.4, smooth=True)
    s = torch.cuda.Stream()
    h = m.phx_create(m.params_from_dict(d, precision=32, stream=s.cuda_stream))
    tp = torch.tensor(psi0.astype(np.complex64), device="cuda")
    tn = torch.tensor(n0.astype(np.float32), device="cuda")
    tP = torch.tensor(P.astype(np.float32), device="cuda")
    torch.cuda.synchronize()
    m.phx_set_pump(h, tP[0].contiguous(), tP[1].contiguous())
    m.phx_set_state(h, tp, tn)
    m.phx_step_n(h, 5)
    outp = torch.empty_like(tp)
    outn = torch.empty_like(tn)
    m.phx_get_state(h, outp, outn)
    o_psi, o_n = gp.run(rounded(psi0, 32), rounded(n0, 32), rounded(P, 32), None,
                        gp.Params(**d), 5)
    assert rel_l2(outp.cpu().numpy(), o_psi) <= 1e-4
    assert rel_l2(outn.cpu().numpy(), o_n) <= 1e-4


TILES = [0, 1, 2, 3, 4, 5, 6, 7, 9]  # auto, TMA-fed persistent configurations 1..7, generic


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("kind", ["reservoir", "loss"])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (0, 1)])
@pytest.mark.parametrize("size", [(131, 77), (58, 58), (59, 116), (200, 3)])
def test_fp32_scalar_tile_configs(tile, kind, bc, size):
    """Every tile configuration of the FP32 scalar kernel against the oracle,
    with a potential, on grids that are exact tile multiples and ragged."""
    m = phx()
    d = model(kind, *size, bc=bc)
    nc = 1
    psi0, n0, P, V = synth.random_state(nc, size[1], size[0], 5, amp=0.7,
                                        reservoir=d["reservoir"], smooth=True)
    psi0, n0, P, V = (rounded(x, 32) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=32, tile=tile))
    if d["reservoir"]:
        m.phx_set_pump(h, np.ascontiguousarray(P[0], np.float32))
    m.phx_set_potential(h, np.ascontiguousarray(V, np.float32))
    m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64),
                    None if n0 is None else np.ascontiguousarray(n0, np.float32))
    m.phx_step_n(h, 9)
    g_psi, g_n = get_state(h, 32)
    o_psi, o_n = gp.run(psi0, n0, P, V, gp.Params(**d), 9)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    if d["reservoir"]:
        assert rel_l2(g_n, o_n) <= 1e-4


@pytest.mark.parametrize("size", [(1, 1), (2, 3), (4, 4), (5, 3), (3, 7), (9, 1), (1, 9)])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (1, 0)])
def test_fp32_scalar_tiny_grids(size, bc):
    d = model("reservoir", *size, bc=bc, L=(0.5 * size[0], 0.5 * size[1]))
    h, (gp_, gn), (op, on) = run_both(d, 32, steps=7)
    assert rel_l2(gp_, op) <= 1e-4
    assert rel_l2(gn, on) <= 1e-4


def test_fp32_scalar_noise_bit_path():
    """Scalar FP32 with noise through the TMA kernel: kappa = 0 and no other
    term, so one step from psi = 0 yields exactly xi_+."""
    d = synth.base_params(70, 61, 7.0, 6.1, kappa=0.0, noise_var=2e-3, seed=5, dt=0.01)
    h = make_handle(d, 32, np.zeros((1, 61, 70)))
    phx().phx_set_time(h, 7, 0.0)
    phx().phx_step_n(h, 1)
    g, _ = get_state(h, 32)
    re, im = noise.noise_field(5, 7, 0, 1, 61, 70, 2e-3)
    assert np.array_equal(g.real.astype(np.float32), re)
    assert np.array_equal(g.imag.astype(np.float32), im)


SPINOR_TILES = [0, 21, 22, 23, 9, 10, 11, 12]  # auto, TMA-fed 21..23, generic shapes 9..12


@pytest.mark.parametrize("tile", SPINOR_TILES)
@pytest.mark.parametrize("tetm", [True, False])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("size", [(131, 77), (58, 58), (70, 45), (5, 3)])
def test_fp32_spinor_tile_configs(tile, tetm, bc, size):
    """Every configuration of the FP32 two-component reservoir kernels (with
    and without TE-TM, separate pump planes, a potential) against the oracle."""
    m = phx()
    d = model("spinor_res_tetm", *size, bc=bc)
    if not tetm:
        d["delta_lt"] = 0.0
        d["dt"] = min(0.45 * gp.stability_dt_max(gp.Params(**d)), 0.05)
    psi0, n0, P, V = synth.random_state(2, size[1], size[0], 6, amp=0.7, smooth=True)
    psi0, n0, P, V = (rounded(x, 32) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=32, tile=tile))
    m.phx_set_pump(h, np.ascontiguousarray(P[0], np.float32), np.ascontiguousarray(P[1], np.float32))
    m.phx_set_potential(h, np.ascontiguousarray(V, np.float32))
    m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64), np.ascontiguousarray(n0, np.float32))
    m.phx_step_n(h, 9)
    g_psi, g_n = get_state(h, 32)
    o_psi, o_n = gp.run(psi0, n0, P, V, gp.Params(**d), 9)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= 1e-4, rel_l2(g_n, o_n)
    if tile in (21, 22, 23) or (tile == 0 and size[0] >= 8):
        assert m.phx_tile(h) in (21, 22, 23)


@pytest.mark.parametrize("tile", [21, 22, 23])
def test_fp32_spinor_shared_pump_and_noise(tile):
    """TMA-fed two-component kernel with one pump plane for both components
    and per-step noise: against the oracle (which adds the same Philox bits)."""
    m = phx()
    d = model("spinor_res_tetm", 97, 66, noise_var=1e-4)
    psi0, n0, P, V = synth.random_state(2, 66, 97, 8, amp=0.7, smooth=True)
    psi0, n0, P, V = (rounded(x, 32) for x in (psi0, n0, P, V))
    h = m.phx_create(m.params_from_dict(d, precision=32, tile=tile))
    m.phx_set_pump(h, np.ascontiguousarray(P[0], np.float32))
    m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64), np.ascontiguousarray(n0, np.float32))
    m.phx_step_n(h, 6)
    g_psi, g_n = get_state(h, 32)
    Pboth = np.stack([P[0], P[0]])
    o_psi, o_n = gp.run(psi0, n0, Pboth, None, gp.Params(**d), 6)
    assert rel_l2(g_psi, o_psi) <= 1e-4, rel_l2(g_psi, o_psi)
    assert rel_l2(g_n, o_n) <= 1e-4


@pytest.mark.parametrize("prec", [32, 64])
def test_caller_owned_state_buffers(prec):
    """phx_create_with_buffers on torch device tensors gives bit-identical
    steps to a handle that allocates its own state; bad buffers are refused."""
    import torch
    m = phx()
    d = model("reservoir", 97, 66)
    psi0, n0, P, V = synth.random_state(1, 66, 97, 3, amp=0.7, smooth=True)
    psi0, n0, P, V = (rounded(x, prec) for x in (psi0, n0, P, V))
    p = m.params_from_dict(d, precision=prec)
    sizes = m.phx_buffer_sizes(p)
    bufs = [torch.empty(s, dtype=torch.uint8, device="cuda") if s else None for s in sizes]
    real, cplx = types(prec)
    hs = []
    for h in (m.phx_create_with_buffers(p, bufs), m.phx_create(p)):
        m.phx_set_pump(h, np.ascontiguousarray(P[0], real))
        m.phx_set_potential(h, np.ascontiguousarray(V, real))
        m.phx_set_state(h, np.ascontiguousarray(psi0, cplx), np.ascontiguousarray(n0, real))
        m.phx_step_n(h, 13)
        hs.append(get_state(h, prec))
    assert np.array_equal(hs[0][0], hs[1][0]) and np.array_equal(hs[0][1], hs[1][1])
    o_psi, _ = gp.run(psi0, n0, P, V, gp.Params(**d), 13)
    assert rel_l2(hs[0][0], o_psi) <= TOL[prec]
    # misaligned and host buffers are refused
    bad = list(bufs)
    bad[0] = bufs[0][1:]
    with pytest.raises(m.PhxError) as e:
        m.phx_create_with_buffers(p, bad)
    assert e.value.status == 1
    bad = list(bufs)
    bad[2] = torch.empty(sizes[2], dtype=torch.uint8).pin_memory()
    with pytest.raises(m.PhxError) as e:
        m.phx_create_with_buffers(p, bad)
    assert e.value.status == 1
