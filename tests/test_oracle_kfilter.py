"""Pins of the oracle's k-space smoothing (Sec. III.B): FFT, product with the
super-Gaussian low-pass mask exp(-((k_x^2 + k_y^2)/k_c^2)^p), inverse FFT."""
import numpy as np

from oracle import gp


def params(**kw):
    d = dict(nx=24, ny=15, lx=12.0, ly=4.5, kfilter_kc=2.0, kfilter_order=2)
    d.update(kw)
    return gp.Params(**d)


def test_plane_wave_is_scaled_by_the_mask_value():
    """exp(i(k_x x + k_y y)) with k on the grid is an eigenfunction: the
    smoothing multiplies it by exp(-((k_x^2 + k_y^2)/k_c^2)^p) written out
    here (non-square grid, distinct lengths, negative wavenumbers, p = 2)."""
    p = params()
    x = np.arange(p.nx) * p.dx
    y = np.arange(p.ny) * p.dy
    for mx, my in [(0, 0), (3, -2), (-5, 1), (12, 7), (1, -7)]:
        kx, ky = 2 * np.pi * mx / p.lx, 2 * np.pi * my / p.ly
        w = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))[None]
        want = np.exp(-(((kx ** 2 + ky ** 2) / 2.0 ** 2) ** 2))
        out = gp.kfilter(w, p)
        assert np.allclose(out, want * w, rtol=0, atol=1e-13), (mx, my)


def test_first_order_mask_is_a_gaussian_blur_kernel():
    """p = 1: the mask exp(-k^2/k_c^2) is the Fourier transform of a Gaussian
    of variance 2/k_c^2 per axis, so a narrow Gaussian in the middle of a
    large periodic box comes out with its variance increased by 2/k_c^2."""
    p = gp.Params(nx=256, ny=256, lx=64.0, ly=64.0, kfilter_kc=1.5, kfilter_order=1)
    x = (np.arange(256) - 128) * p.dx
    s2 = 1.3
    g = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / (2 * s2))[None] + 0j
    out = gp.kfilter(g, p).real[0]
    s2_new = s2 + 2.0 / 1.5 ** 2
    want = s2 / s2_new * np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / (2 * s2_new))
    assert np.abs(out - want).max() < 1e-10


def test_large_cutoff_is_identity_and_smoothing_never_adds_norm():
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(2, 15, 24)) + 1j * rng.normal(size=(2, 15, 24))
    assert np.allclose(gp.kfilter(psi, params(kfilter_kc=1e6)), psi, rtol=0, atol=1e-12)
    out = gp.kfilter(psi, params())
    for c in range(2):
        assert np.linalg.norm(out[c]) < np.linalg.norm(psi[c])
    # components are filtered independently
    one = gp.kfilter(psi[1:], params())
    assert np.array_equal(one[0], out[1])


def test_run_applies_smoothing_after_every_kth_step():
    p = gp.Params(nx=10, ny=8, lx=5.0, ly=4.0, g=0.2, gamma_c=0.1, dt=0.02,
                  kfilter_kc=3.0, kfilter_order=3, kfilter_every=3)
    rng = np.random.default_rng(4)
    psi0 = rng.normal(size=(1, 8, 10)) + 1j * rng.normal(size=(1, 8, 10))
    q = p.with_(kfilter_every=0)
    a, _ = gp.run(psi0, None, None, None, p, 7, step0=1)
    # steps 1..7: smoothing after steps 2 and 5 ((k + 1) % 3 == 0)
    b, _ = gp.run(psi0, None, None, None, q, 2, step0=1)
    b = gp.kfilter(b, p)
    b, _ = gp.run(b, None, None, None, q, 3, step0=3)
    b = gp.kfilter(b, p)
    b, _ = gp.run(b, None, None, None, q, 2, step0=6)
    assert np.array_equal(a, b)
