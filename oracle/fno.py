"""FP64 oracle of the Fourier neural operator (FNO) used as a learned warm
start for the steady-state solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The network follows Li et al., "Fourier Neural Operator for Parametric
Partial Differential Equations" (2020), in the 2D form with real FFTs:

    v0 = a W_lift + b_lift                                  (pointwise)
    v_{l+1} = sigma( K_l(v_l) + v_l W_l + b_l ),  l = 0..L-1 (no sigma on the last)
    u = sigma(v_L Q1 + q1) Q2 + q2                          (pointwise)
    K(v) = irfft2( R . rfft2(v) ) keeping kx in [0, MX) and
           ky in [0, MY/2) U [H - MY/2, H); R is a complex C x C matrix per
           kept mode; every other mode is zero.
    sigma = GELU (exact, erf form).

Tensors are channels-last [B, H, W, C] (H = y rows, W = x columns).  The flat
FP32 parameter vector is laid out, in this order:
    W_lift [Cin, C], b_lift [C],
    per layer: Rr [MY, MX, C, C], Ri [MY, MX, C, C], W [C, C], b [C]
               (mode index my: 0..MY/2-1 are ky = my, MY/2..MY-1 are
                ky = H - MY + my),
    Q1 [C, P], q1 [P], Q2 [P, Cout], q2 [Cout].
Loss: mean squared error over all output elements.
The forward uses torch.fft (a library primitive); gradients come from
torch.autograd and are pinned by central finite differences in the tests.
"""
from dataclasses import dataclass

import numpy as np
import torch


@dataclass(frozen=True)
class FnoConfig:
    height: int = 256
    width: int = 256
    channels: int = 32
    layers: int = 4
    modes_x: int = 16
    modes_y: int = 32
    in_channels: int = 3
    out_channels: int = 3
    proj_hidden: int = 64


def param_shapes(cfg):
    C, MX, MY = cfg.channels, cfg.modes_x, cfg.modes_y
    shapes = [("W_lift", (cfg.in_channels, C)), ("b_lift", (C,))]
    for l in range(cfg.layers):
        shapes += [("Rr%d" % l, (MY, MX, C, C)), ("Ri%d" % l, (MY, MX, C, C)),
                   ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
    shapes += [("Q1", (C, cfg.proj_hidden)), ("q1", (cfg.proj_hidden,)),
               ("Q2", (cfg.proj_hidden, cfg.out_channels)), ("q2", (cfg.out_channels,))]
    return shapes


def num_params(cfg):
    return int(sum(np.prod(s) for _, s in param_shapes(cfg)))


def unflatten(w, cfg):
    out = {}
    o = 0
    for name, shape in param_shapes(cfg):
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def spectral_conv(v, Rr, Ri, cfg):
    """K(v) for v [B, H, W, C] (float64 tensor)."""
    B, H, W, C = v.shape
    MX, MY = cfg.modes_x, cfg.modes_y
    vh = torch.fft.rfft2(v, dim=(1, 2))                 # [B, H, W//2+1, C]
    R = torch.complex(Rr, Ri)                            # [MY, MX, C, C]
    out = torch.zeros(B, H, W // 2 + 1, C, dtype=vh.dtype)
    lo = vh[:, :MY // 2, :MX, :]                         # ky = 0 .. MY/2-1
    hi = vh[:, H - MY // 2:, :MX, :]                     # ky = H-MY/2 .. H-1
    out[:, :MY // 2, :MX, :] = torch.einsum("byxc,yxco->byxo", lo, R[:MY // 2])
    out[:, H - MY // 2:, :MX, :] = torch.einsum("byxc,yxco->byxo", hi, R[MY // 2:])
    return torch.fft.irfft2(out, s=(H, W), dim=(1, 2))


def gelu(z):
    return 0.5 * z * (1.0 + torch.erf(z / np.sqrt(2.0)))


def forward(w, a, cfg):
    """w: flat parameters (torch float64), a: [B, H, W, Cin] -> [B, H, W, Cout]."""
    p = unflatten(w, cfg)
    v = a @ p["W_lift"] + p["b_lift"]
    for l in range(cfg.layers):
        z = spectral_conv(v, p["Rr%d" % l], p["Ri%d" % l], cfg) + v @ p["W%d" % l] + p["b%d" % l]
        v = gelu(z) if l < cfg.layers - 1 else z
    h = gelu(v @ p["Q1"] + p["q1"])
    return h @ p["Q2"] + p["q2"]


def loss(w, a, target, cfg):
    u = forward(w, a, cfg)
    return torch.mean((u - target) ** 2)


def loss_and_grad(w_np, a_np, t_np, cfg):
    """Loss (float) and its gradient (float64 numpy, flat) at w."""
    w = torch.tensor(np.asarray(w_np, np.float64), requires_grad=True)
    a = torch.tensor(np.asarray(a_np, np.float64))
    t = torch.tensor(np.asarray(t_np, np.float64))
    L = loss(w, a, t, cfg)
    L.backward()
    return float(L.detach()), w.grad.detach().numpy().copy()


def predict(w_np, a_np, cfg):
    with torch.no_grad():
        return forward(torch.tensor(np.asarray(w_np, np.float64)),
                       torch.tensor(np.asarray(a_np, np.float64)), cfg).numpy()


def adam_step(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Kingma & Ba (2015) Adam with bias correction; returns (w, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
