"""FNO warm-start network on the GPU (BF16 tensor-core GEMMs, FP32
accumulation) against the FP64 oracle: forward output, full parameter
gradient, one Adam step, determinism and argument errors.

Tolerance: every contraction rounds its two operands to BF16 (relative
error <= 2^-9 each), so one GEMM output carries a relative error of a few
1e-3; through the lift, four spectral layers (five chained GEMMs each) and
the projection the forward output is expected within ~1e-2 relative L2 and
the gradient blocks (one more chain in reverse) within a few 1e-2.  The
bounds below are 3e-2 (forward) and 6e-2 (gradient blocks)."""
import numpy as np
import pytest
import torch

from oracle import fno as ofno
import synth
from gpu_util import phx, rel_l2

pytestmark = pytest.mark.gpu

FWD_TOL = 3e-2
GRAD_TOL = 6e-2

TINY = dict(height=12, width=10, channels=5, layers=2, modes_x=3, modes_y=4,
            in_channels=3, out_channels=3, proj_hidden=7)
MID = dict(height=72, width=80, channels=16, layers=3, modes_x=9, modes_y=12,
           in_channels=3, out_channels=3, proj_hidden=24)
FULL = dict(height=256, width=256, channels=32, layers=4, modes_x=16, modes_y=32,
            in_channels=3, out_channels=3, proj_hidden=64)


def weights(cfg, seed, spectral_scale=1.0):
    """Seeded weights; spectral blocks rescaled to U[-s, s)/C so the spectral
    branch carries a share of the signal comparable to the local one."""
    shapes = ofno.param_shapes(cfg)
    w = synth.fno_init_weights(shapes, seed, cfg.channels).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    o = 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        if name.startswith("R"):
            w[o:o + n] = rng.uniform(-spectral_scale, spectral_scale, n) / cfg.channels
        elif len(shape) == 1:
            w[o:o + n] = rng.uniform(-0.1, 0.1, n)
        o += n
    return w.astype(np.float32)


def inputs(cfg, batch, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(batch, cfg.height, cfg.width, cfg.in_channels)).astype(np.float32)
    t = rng.normal(size=(batch, cfg.height, cfg.width, cfg.out_channels)).astype(np.float32)
    return a, t


def make(cfg_dict, batch, seed=0, scale=1.0):
    m = phx()
    cfg = ofno.FnoConfig(**cfg_dict)
    f = m.phx_fno_create(max_batch=batch, **cfg_dict)
    assert f.num_params == ofno.num_params(cfg)
    w = weights(cfg, seed, scale)
    m.phx_fno_set_params(f, w)
    return m, cfg, f, w


def blocks(cfg, v):
    return ofno.unflatten(np.asarray(v), cfg)


@pytest.mark.parametrize("name,cfg_dict,batch", [("tiny", TINY, 3), ("mid", MID, 2)])
def test_forward_matches_oracle(name, cfg_dict, batch):
    m, cfg, f, w = make(cfg_dict, batch, seed=11)
    a, _ = inputs(cfg, batch, 12)
    x = torch.from_numpy(a).cuda()
    out = torch.empty(batch, cfg.height, cfg.width, cfg.out_channels, device="cuda")
    m.phx_fno_forward(f, x, out)
    torch.cuda.synchronize()
    ref = ofno.predict(w, a, cfg)
    err = rel_l2(out.cpu().numpy().astype(np.float64), ref)
    assert err < FWD_TOL, err


@pytest.mark.parametrize("name,cfg_dict,batch", [("tiny", TINY, 3), ("mid", MID, 2)])
def test_gradient_matches_oracle(name, cfg_dict, batch):
    m, cfg, f, w = make(cfg_dict, batch, seed=21)
    a, t = inputs(cfg, batch, 22)
    g = torch.empty(f.num_params, device="cuda")
    loss = m.phx_fno_loss_grad(f, torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda(), g)
    L, gref = ofno.loss_and_grad(w, a, t, cfg)
    assert abs(loss - L) / L < FWD_TOL
    gg = g.cpu().numpy().astype(np.float64)
    got, ref = blocks(cfg, gg), blocks(cfg, gref)
    for k in ref:
        assert rel_l2(got[k], ref[k]) < GRAD_TOL, (k, rel_l2(got[k], ref[k]))
    # the whole vector, and its direction
    assert rel_l2(gg, gref) < GRAD_TOL
    cos = float(gg @ gref / (np.linalg.norm(gg) * np.linalg.norm(gref)))
    assert cos > 0.998


def test_full_size_forward_and_gradient():
    """The warm-start configuration itself: 256^2, C = 32, 4 layers,
    16 x 32 modes, on realistic pump features and steady-state-like targets."""
    batch = 2
    m, cfg, f, w = make(FULL, batch, seed=31, scale=0.5)
    pumps = synth.random_gaussian_pumps(256, 128.0, batch, seed=7000)
    pthr = synth.load_constants()["pump_threshold"]
    a = synth.fno_features(pumps, 128.0, pthr)
    rng = np.random.default_rng(32)
    t = (0.3 * rng.normal(size=(batch, 256, 256, 3))).astype(np.float32)
    x = torch.from_numpy(a).cuda()
    out = torch.empty(batch, 256, 256, 3, device="cuda")
    m.phx_fno_forward(f, x, out)
    g = torch.empty(f.num_params, device="cuda")
    loss = m.phx_fno_loss_grad(f, x, torch.from_numpy(t).cuda(), g)
    torch.cuda.synchronize()
    ref = ofno.predict(w, a, cfg)
    assert rel_l2(out.cpu().numpy().astype(np.float64), ref) < FWD_TOL
    L, gref = ofno.loss_and_grad(w, a, t, cfg)
    assert abs(loss - L) / L < FWD_TOL
    got, refb = blocks(cfg, g.cpu().numpy().astype(np.float64)), blocks(cfg, gref)
    for k in refb:
        assert rel_l2(got[k], refb[k]) < GRAD_TOL, (k, rel_l2(got[k], refb[k]))


def test_deterministic_and_batch_prefix():
    """Same inputs give bit-identical gradients; a batch of one uses the first
    sample only (buffers sized for max_batch are not read beyond batch)."""
    m, cfg, f, w = make(TINY, 4, seed=41)
    a, t = inputs(cfg, 4, 42)
    x, y = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
    g1 = torch.empty(f.num_params, device="cuda")
    g2 = torch.empty_like(g1)
    l1 = m.phx_fno_loss_grad(f, x, y, g1)
    l2 = m.phx_fno_loss_grad(f, x, y, g2)
    assert l1 == l2 and torch.equal(g1, g2)
    g3 = torch.empty_like(g1)
    l3 = m.phx_fno_loss_grad(f, x[:1].contiguous(), y[:1].contiguous(), g3)
    L, gref = ofno.loss_and_grad(w, a[:1], t[:1], cfg)
    assert abs(l3 - L) / L < FWD_TOL
    assert rel_l2(g3.cpu().numpy().astype(np.float64), gref) < GRAD_TOL


def test_adam_step_matches_oracle():
    m, cfg, f, w = make(TINY, 2, seed=51)
    a, t = inputs(cfg, 2, 52)
    x, y = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
    mom = np.zeros(f.num_params)
    vel = np.zeros(f.num_params)
    lr = 1e-3
    wg = w.astype(np.float64)
    for step in (1, 2, 3):
        g = torch.empty(f.num_params, device="cuda")
        m.phx_fno_loss_grad(f, x, y, g)           # gradient at the current weights
        m.phx_fno_train_step(f, x, y, lr)         # recomputes the same gradient, then Adam
        wref, mom, vel = ofno.adam_step(wg, g.cpu().numpy().astype(np.float64), mom, vel,
                                        step, lr)
        wg = m.phx_fno_get_params(f).astype(np.float64)
        # FP32 storage of w (|w| < 1) plus the FP32 update arithmetic
        assert np.max(np.abs(wg - wref)) < 1e-7 + 1e-4 * lr, step


def test_training_reduces_loss():
    """A few hundred Adam steps on a fixed mini-batch cut the loss by > 10x."""
    m, cfg, f, w = make(TINY, 4, seed=61, scale=0.3)
    a, _ = inputs(cfg, 4, 62)
    t = np.ascontiguousarray(np.tanh(0.5 * a), np.float32)   # a learnable pointwise map
    x, y = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
    first = m.phx_fno_train_step(f, x, y, 3e-3)
    for _ in range(400):
        last = m.phx_fno_train_step(f, x, y, 3e-3)
    assert last < first / 10, (first, last)


def test_errors():
    m = phx()
    with pytest.raises(m.PhxError):
        m.phx_fno_create(modes_x=200, height=64, width=64)
    with pytest.raises(m.PhxError):
        m.phx_fno_create(modes_y=3)
    f = m.phx_fno_create(max_batch=2, **TINY)
    x = torch.zeros(3, 12, 10, 3, device="cuda")
    out = torch.zeros(3, 12, 10, 3, device="cuda")
    with pytest.raises(m.PhxError):
        m.phx_fno_forward(f, x, out)       # batch 3 > max_batch 2
    with pytest.raises(TypeError):
        m.phx_fno_forward(f, x.double(), out)


def test_feature_target_state_maps():
    """Device input/output maps against the host definitions used for the
    oracle's inputs (synth.fno_features / fno_targets / fno_state_from_output)."""
    m = phx()
    pthr = synth.load_constants()["pump_threshold"]
    P = synth.random_gaussian_pumps(64, 128.0, 3, seed=900).astype(np.float32)
    feat = torch.empty(3, 64, 64, 3, device="cuda")
    m.phx_fno_features(torch.from_numpy(P).cuda(), 128.0, 128.0, pthr, feat)
    ref = synth.fno_features(P.astype(np.float64), 128.0, pthr)
    torch.cuda.synchronize()
    assert np.max(np.abs(feat.cpu().numpy() - ref)) < 1e-6 * max(1.0, np.abs(ref).max())
    rng = np.random.default_rng(901)
    psi = (rng.normal(size=(3, 64, 64)) + 1j * rng.normal(size=(3, 64, 64)) + 0.5j).astype(np.complex64)
    n = rng.uniform(0, 20, size=(3, 64, 64)).astype(np.float32)
    tgt = torch.empty(3, 64, 64, 3, device="cuda")
    m.phx_fno_targets(torch.from_numpy(psi).cuda(), torch.from_numpy(n).cuda(),
                      synth.FNO_SCALE_PSI, synth.FNO_SCALE_N, tgt)
    ref = synth.fno_targets(psi.astype(np.complex128), n.astype(np.float64))
    torch.cuda.synchronize()
    assert np.max(np.abs(tgt.cpu().numpy() - ref)) < 2e-6
    # round trip back to a state: psi up to the removed global phase, n exact
    ps = torch.empty(3, 64, 64, dtype=torch.complex64, device="cuda")
    nn = torch.empty(3, 64, 64, device="cuda")
    m.phx_fno_to_state(tgt, synth.FNO_SCALE_PSI, synth.FNO_SCALE_N, ps, nn)
    torch.cuda.synchronize()
    for b in range(3):
        rp, rn = synth.fno_state_from_output(ref[b])
        assert np.max(np.abs(ps[b].cpu().numpy() - rp)) < 1e-5
        assert np.max(np.abs(nn[b].cpu().numpy() - rn)) < 1e-5
        assert abs(abs(ps[b].cpu().numpy().astype(np.complex128).sum())
                   - abs(psi[b].astype(np.complex128).sum())) < 1e-3 * abs(psi[b].sum())
