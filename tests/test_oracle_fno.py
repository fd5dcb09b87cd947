"""Pins of the FNO oracle (oracle/fno.py): gradients against central finite
differences, the spectral layer against its closed form on single Fourier
modes, GELU against erf, one Adam step against its closed form."""
import math

import numpy as np
import pytest
import torch

from oracle import fno
import synth

TINY = fno.FnoConfig(height=16, width=12, channels=4, layers=2, modes_x=3, modes_y=4,
                     in_channels=3, out_channels=3, proj_hidden=5)


def test_default_parameter_count():
    assert fno.num_params(fno.FnoConfig()) == (3 * 32 + 32 + 4 * (2 * 32 * 16 * 32 * 32 + 32 * 32 + 32)
                                              + 32 * 64 + 64 + 64 * 3 + 3)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = synth.fno_init_weights(fno.param_shapes(TINY), seed=1, channels=TINY.channels).astype(np.float64)
    w += 0.05 * rng.normal(size=w.size)
    a = rng.normal(size=(2, 16, 12, 3))
    t = rng.normal(size=(2, 16, 12, 3))
    L, g = fno.loss_and_grad(w, a, t, TINY)
    offs = {}
    o = 0
    for name, shape in fno.param_shapes(TINY):
        offs[name] = (o, int(np.prod(shape)))
        o += int(np.prod(shape))
    h = 1e-6
    checked = 0
    for name, (o, n) in offs.items():
        for idx in rng.choice(n, size=min(n, 3), replace=False):
            k = o + idx
            wp = w.copy(); wp[k] += h
            wm = w.copy(); wm[k] -= h
            Lp = float(fno.loss(torch.tensor(wp), torch.tensor(a), torch.tensor(t), TINY))
            Lm = float(fno.loss(torch.tensor(wm), torch.tensor(a), torch.tensor(t), TINY))
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, idx, fd, g[k])
            checked += 1
    assert checked > 20


# TINY keeps kx in {0, 1, 2} and ky in {0, 1, -2, -1}
@pytest.mark.parametrize("kx,ky,inside", [(1, 1, True), (2, -2, True), (0, 1, True),
                                          (3, 1, False), (1, 2, False), (2, 5, False)])
def test_spectral_layer_single_mode(kx, ky, inside):
    """A real mode cos(2 pi (kx x/W + ky y/H)) in channel 0 with R = I gives the
    same mode if (kx, ky) is kept, else 0; with R = iI it gives -sin(...)."""
    cfg = TINY
    H, W, C = cfg.height, cfg.width, cfg.channels
    y = np.arange(H)[:, None]
    x = np.arange(W)[None, :]
    ph = 2 * np.pi * (kx * x / W + ky * y / H)
    v = np.zeros((1, H, W, C))
    v[0, :, :, 0] = np.cos(ph)
    eye = np.zeros((cfg.modes_y, cfg.modes_x, C, C))
    eye[:, :, np.arange(C), np.arange(C)] = 1.0
    zero = np.zeros_like(eye)
    out = fno.spectral_conv(torch.tensor(v), torch.tensor(eye), torch.tensor(zero), cfg).numpy()
    expect = np.cos(ph) if inside else np.zeros_like(ph)
    assert np.allclose(out[0, :, :, 0], expect, atol=1e-12)
    assert np.allclose(out[0, :, :, 1:], 0.0, atol=1e-12)
    out = fno.spectral_conv(torch.tensor(v), torch.tensor(zero), torch.tensor(eye), cfg).numpy()
    expect = -np.sin(ph) if inside else np.zeros_like(ph)
    if kx == 0 and inside:
        # the kx = 0 column keeps only the real part under the inverse real
        # transform: +ky and -ky rotate opposite ways and cancel in sum
        expect = np.zeros_like(ph) if ky != 0 else expect
    assert np.allclose(out[0, :, :, 0], expect, atol=1e-12)


def test_gelu_erf_form():
    z = torch.tensor([-3.0, -1.0, -0.1, 0.0, 0.5, 2.0], dtype=torch.float64)
    g = fno.gelu(z).numpy()
    ref = [0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z.tolist()]
    assert np.allclose(g, ref, atol=1e-15)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    w, m, v = fno.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(w, -0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
