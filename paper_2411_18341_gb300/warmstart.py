"""Learned warm start for steady-state solves.

A Fourier neural operator (the ``phx_fno_*`` calls) maps a pump image to an
approximate stationary state (psi, n) of Eqs. (PULSE_psi)/(PULSE_res); the
RK4 relaxation then starts from that state instead of from noise.  This
module drives the loop on the GPU through the C ABI:

* ``spot_thresholds`` -- the condensation threshold of a single Gaussian pump
  spot per waist, measured with the batched solver (a finite spot loses
  particles to its surroundings, so it needs more than the homogeneous
  threshold gamma_c gamma_r / R).
* ``generate`` -- solver-generated training pairs: batches of instances (one
  persistent launch per RK4 step) relaxed from a caller-given initial state;
  features and gauge-fixed targets are formed on the device.
* ``train``    -- mini-batch Adam on the GPU (forward, backward and update in
  this package's kernels).
* ``screen``   -- a batch relaxed from cold or warm starts, recording for each
  member the first check at which r_psi < tol32.
* ``relax``    -- one instance relaxed to r_psi < tol, timed with CUDA events
  (network inference included for warm starts).

Relaxation protocol (identical for cold and warm starts): FP32 steps until
r_psi < tol32, then the FP32 state continues in FP64 until r_psi < tol.  The
FP32 stencil has a residual floor of a few 1e-6 at dx = 0.5 um (rounding of
the Laplacian's cancellation), so the last decade needs FP64.  r_psi is
||K + i omega psi|| / ||psi|| with K = dpsi/dt and omega the best-fit
rotation frequency (a stationary condensate rotates with a global phase).
A member whose mean |psi|^2 falls below ``tiny`` has no condensate (the pump
is below the threshold of its finite spot) and is reported as decayed.

Only torch device memory, dtype casts and events come from PyTorch; every
arithmetic step of the method runs in the package's CUDA kernels.
"""
import time

import numpy as np
import torch

from . import (phx_batch_create, phx_batch_get_state, phx_batch_norm_energy,
               phx_batch_residual, phx_batch_set_pump, phx_batch_set_state, phx_batch_step_n,
               phx_create, phx_fno_create, phx_fno_features, phx_fno_forward,
               phx_fno_loss_grad, phx_fno_set_params, phx_fno_targets,
               phx_fno_to_state, phx_fno_train_step, phx_get_state,
               phx_residual, phx_set_pump, phx_set_state, phx_stability_dt, phx_step_n,
               params_from_dict)

SCALE_PSI = 5.0     # |psi| ~ 5 at 1-3 P_thr: output normalisation of Re/Im psi
SCALE_N = 15.0      # n ~ gamma_c / R = 15 in a condensate: normalisation of n


class Problem:
    """Parameters of the steady-state workload (one square grid) and its
    pump threshold."""

    def __init__(self, params, pump_threshold):
        self.params = dict(params)
        self.pump_threshold = float(pump_threshold)
        self.n = int(params["nx"])
        self.length = float(params["lx"])
        self.cell = (self.length / self.n) ** 2
        if params["nx"] != params["ny"] or params["lx"] != params["ly"]:
            raise ValueError("square grids only")


def pump_threshold(params):
    """Homogeneous condensation threshold P_thr = gamma_c gamma_r / R: with
    psi = 0 the reservoir settles at n = P / gamma_r (Eq. PULSE_res), and the
    gain R n of Eq. PULSE_psi balances the loss gamma_c at P = P_thr."""
    return params["gamma_c"] * params["gamma_r"] / params["R"]


def stable_dt(params, fraction):
    """`fraction` of the RK4 stability limit of the grid (phx_stability_dt)."""
    return fraction * phx_stability_dt(params_from_dict(dict(params, dt=0.0)))


def _stream():
    return torch.cuda.current_stream()


def _grid_r2(problem, cx=0.0, cy=0.0):
    """|r - c|^2 on the cell positions -L/2 + i L/n (origin at the centre)."""
    x = -0.5 * problem.length + np.arange(problem.n) * (problem.length / problem.n)
    return (x[None, :] - cx) ** 2 + (x[:, None] - cy) ** 2


def spot_thresholds(problem, waists, factors=(1.0, 1.25, 1.5, 2.0, 2.5, 3.0, 4.0, 5.0, 6.5,
                                              8.0, 10.0, 13.0, 17.0, 22.0, 28.0, 36.0),
                    chunks=120, chunk_steps=25, seed=0):
    """Condensation threshold of one Gaussian spot P0 exp(-r^2/w^2) per waist
    w, in units of the homogeneous threshold, measured with the solver.

    Every (w, f) pair is one member of a batch: pump f P_thr exp(-r^2/w^2),
    reservoir started at its below-threshold value n = P / gamma_r, psi at
    weak seeded noise.  The batch runs `chunks` chunks of `chunk_steps` RK4
    steps; after each chunk every member's psi is scaled back to the start
    norm (|psi|^2 ~ 1e-10 per site, so the Kerr term and the reservoir
    depletion stay negligible: the linearised dynamics around psi = 0).  Over
    the second half, when the decaying modes have died out, the mean of
    ln(N_after / N_before) per chunk is the growth rate of the leading mode's
    |psi|^2; it is positive above threshold.  The threshold is the factor at
    which that rate crosses zero (linear in log f between the bracketing
    factors); inf if no factor in the list condenses.
    Returns (thresholds [len(waists)], rates [len(waists), len(factors)],
    rates in 1/ps)."""
    pthr = pump_threshold(problem.params)
    n = problem.n
    members, pumps = [], []
    for w in waists:
        shape = np.exp(-_grid_r2(problem) / w ** 2)
        for f in factors:
            members.append(_member_params(problem, len(members)))
            pumps.append((f * pthr * shape).astype(np.float32))
    b = phx_batch_create(members)
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    amp = 1e-5
    for k, P in enumerate(pumps):
        Pd = torch.as_tensor(P).cuda()
        phx_batch_set_pump(b, k, Pd)
        z = torch.complex(torch.randn(n, n, generator=g, device="cuda"),
                          torch.randn(n, n, generator=g, device="cuda")) * amp
        phx_batch_set_state(b, k, z.to(torch.complex64).contiguous(),
                            (Pd / problem.params["gamma_r"]).contiguous())
    N0, _ = phx_batch_norm_energy(b)
    psi = torch.empty(n, n, dtype=torch.complex64, device="cuda")
    nres = torch.empty(n, n, device="cuda")
    logs = []
    for c in range(chunks):
        phx_batch_step_n(b, chunk_steps)
        N1, _ = phx_batch_norm_energy(b)
        logs.append(np.log(np.maximum(N1, 1e-300) / N0))
        for k in range(len(members)):  # back to the start norm
            phx_batch_get_state(b, k, psi, nres)
            psi *= float(np.sqrt(N0[k] / max(N1[k], 1e-300)))
            phx_batch_set_state(b, k, psi, nres)
    del b
    half = np.asarray(logs[chunks // 2:])
    rate = half.mean(axis=0) / (chunk_steps * problem.params["dt"])
    rate = rate.reshape(len(waists), len(factors))
    lf = np.log(np.asarray(factors, np.float64))
    thr = np.full(len(waists), np.inf)
    for a in range(len(waists)):
        up = np.where(rate[a] > 0)[0]
        if len(up) == 0:
            continue
        k = int(up[0])
        if k == 0:
            thr[a] = factors[0]
            continue
        r0, r1 = rate[a, k - 1], rate[a, k]
        thr[a] = float(np.exp(lf[k - 1] + (lf[k] - lf[k - 1]) * (-r0) / (r1 - r0)))
    return thr, rate


def features(problem, pumps):
    """Network inputs [B, H, W, 3] on the device from pump images [B, H, W]."""
    P = torch.as_tensor(np.asarray(pumps, np.float32)).cuda().contiguous()
    out = torch.empty(tuple(P.shape) + (3,), device="cuda")
    phx_fno_features(P, problem.length, problem.length, problem.pump_threshold, out, _stream())
    return out


def predict_states(net, problem, feats, batch=8):
    """Network prediction as solver states: psi [B, H, W] complex64, n [B, H, W]."""
    B = feats.shape[0]
    n = problem.n
    u = torch.empty(B, n, n, 3, device="cuda")
    for k in range(0, B, batch):
        m = min(batch, B - k)
        phx_fno_forward(net, feats[k:k + m], u[k:k + m])
    psi = torch.empty(B, n, n, dtype=torch.complex64, device="cuda")
    nn = torch.empty(B, n, n, device="cuda")
    phx_fno_to_state(u, SCALE_PSI, SCALE_N, psi, nn, _stream())
    return psi, nn


def _member_params(problem, i, precision=32, stream=None):
    d = dict(problem.params)
    d["instance"] = int(i)
    return params_from_dict(d, precision=precision, stream=stream)


def screen(problem, pumps, init, tol32=1e-5, check_every=100, cap=200000, tiny=1e-10,
           chunk=512, collect=False, log=None):
    """Relax every pump in batches of `chunk` (one persistent launch per RK4
    step).  init(i0, i1) -> (psi [m,H,W] complex64, n [m,H,W] float32) device
    tensors for members i0..i1-1.  Returns a dict of host arrays: steps (first
    check with r < tol32, or -1), r (at that check, else final), decayed,
    diverged (the state became non-finite: a strongly pumped spot whose
    transient density left the time step's stability region), and with
    collect=True the final states as device tensors."""
    N = len(pumps)
    n = problem.n
    steps = np.full(N, -1, np.int64)
    r_at = np.zeros(N)
    decayed = np.zeros(N, bool)
    diverged = np.zeros(N, bool)
    psi_all = torch.empty(N, n, n, dtype=torch.complex64, device="cuda") if collect else None
    n_all = torch.empty(N, n, n, device="cuda") if collect else None
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        m = c1 - c0
        b = phx_batch_create([_member_params(problem, i) for i in range(c0, c1)])
        psi0, n0 = init(c0, c1)
        for k in range(m):
            phx_batch_set_pump(b, k, np.ascontiguousarray(pumps[c0 + k], np.float32))
            phx_batch_set_state(b, k, psi0[k], n0[k])
        done = np.zeros(m, bool)
        s = 0
        t0 = time.time()
        while s < cap and not done.all():
            phx_batch_step_n(b, check_every)
            s += check_every
            norms, _ = phx_batch_norm_energy(b, allow_nonfinite=True)
            bad = ~np.isfinite(norms)
            dec = (norms / (problem.cell * n * n) < tiny) & ~bad
            r, _, _ = _safe_residual(b, dec | bad)
            newly = (~done) & (r < tol32) & (~dec) & (~bad)
            steps[c0:c1][newly] = s
            r_at[c0:c1][newly] = r[newly]
            decayed[c0:c1] |= (~done) & dec
            diverged[c0:c1] |= (~done) & bad
            done |= newly | dec | bad
        if not done.all():
            r, _, _ = _safe_residual(b, decayed[c0:c1] | diverged[c0:c1])
            r_at[c0:c1][~done] = r[~done]
        if collect:
            for k in range(m):
                phx_batch_get_state(b, k, psi_all[c0 + k], n_all[c0 + k])
        if log:
            log("screen %d..%d: %d steps, %.1f s, converged %d, decayed %d"
                % (c0, c1 - 1, s, time.time() - t0, int((steps[c0:c1] >= 0).sum()),
                   int(decayed[c0:c1].sum())))
        del b
    out = dict(steps=steps, r=r_at, decayed=decayed, diverged=diverged)
    if collect:
        out["psi"], out["nres"] = psi_all, n_all
    return out


def _safe_residual(b, skip):
    """Per-member residuals; members whose psi has decayed to (near) zero or
    become non-finite report r = 1 (their ratio is meaningless)."""
    r, rn, om = phx_batch_residual(b, allow_nonfinite=True)
    r = np.where(skip | ~np.isfinite(r), 1.0, r)
    return r, rn, om


def generate(problem, pumps, init, steps=40000, tol32=1e-5, chunk=512, log=None):
    """Training pairs: each pump relaxed from init(i0, i1) (see ``screen``)
    until r_psi < tol32 or `steps`; the final state, gauge-fixed and scaled,
    is the target.  Returns (features, targets, screen dict); the screen
    dict's ``steps`` is >= 0 exactly for the pairs that reached tol32."""
    n = problem.n
    res = screen(problem, pumps, init, tol32=tol32, cap=steps, chunk=chunk, collect=True,
                 log=log)
    feats = features(problem, pumps)
    targs = torch.empty(len(pumps), n, n, 3, device="cuda")
    phx_fno_targets(res.pop("psi"), res.pop("nres"), SCALE_PSI, SCALE_N, targs, _stream())
    torch.cuda.synchronize()
    return feats, targs, res


def train(net, feats, targs, epochs, batch=8, lr=1e-3, lr_final=1e-5, seed=0, log=None):
    """Mini-batch Adam with a cosine learning-rate decay; returns the mean
    training loss of each epoch."""
    N = feats.shape[0]
    rng = np.random.default_rng(seed)
    nb = N // batch
    total = max(epochs * nb - 1, 1)
    hist = []
    it = 0
    xb = torch.empty((batch,) + tuple(feats.shape[1:]), device="cuda")
    yb = torch.empty((batch,) + tuple(targs.shape[1:]), device="cuda")
    for ep in range(epochs):
        perm = torch.as_tensor(rng.permutation(N), device="cuda")
        acc = 0.0
        t0 = time.time()
        for k in range(nb):
            sel = perm[k * batch:(k + 1) * batch]
            torch.index_select(feats, 0, sel, out=xb)
            torch.index_select(targs, 0, sel, out=yb)
            a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * it / total))
            acc += phx_fno_train_step(net, xb, yb, a)
            it += 1
        hist.append(acc / max(nb, 1))
        if log:
            log("epoch %d loss %.3e (%.1f s)" % (ep, hist[-1], time.time() - t0))
    return hist


def eval_loss(net, feats, targs, batch=8):
    """Mean squared error of the network over a data set."""
    N = feats.shape[0]
    tot = 0.0
    cnt = 0
    for k in range(0, N, batch):
        m = min(batch, N - k)
        tot += phx_fno_loss_grad(net, feats[k:k + m], targs[k:k + m]) * m
        cnt += m
    return tot / max(cnt, 1)


def relax(problem, pump, init=None, net=None, tol=1e-6, tol32=1e-5, check_every=100,
          cap=200000, instance=0):
    """Relax one instance to r_psi < tol (FP32 to tol32, then FP64).

    init: (psi0, n0) device tensors for a cold start; or net for a warm
    start, whose inference is inside the timed region.  Returns
    dict(steps, steps32, ms, r, converged)."""
    n = problem.n
    stream = _stream()
    h = phx_create(_member_params(problem, instance, 32, stream.cuda_stream))
    P = torch.as_tensor(np.ascontiguousarray(pump, np.float32)).cuda()
    phx_set_pump(h, P)
    h64 = phx_create(_member_params(problem, instance, 64, stream.cuda_stream))
    phx_set_pump(h64, P.double())
    if net is not None:
        x = features(problem, pump[None])
        u = torch.empty(1, n, n, 3, device="cuda")
        psi = torch.empty(1, n, n, dtype=torch.complex64, device="cuda")
        nn = torch.empty(1, n, n, device="cuda")
    psi32 = torch.empty(n, n, dtype=torch.complex64, device="cuda")
    n32 = torch.empty(n, n, device="cuda")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if net is not None:
        phx_fno_forward(net, x, u)
        phx_fno_to_state(u, SCALE_PSI, SCALE_N, psi, nn, stream)
        phx_set_state(h, psi[0], nn[0])
    else:
        phx_set_state(h, init[0], init[1])
    s = 0
    r = float("inf")
    while s < cap:
        phx_step_n(h, check_every)
        s += check_every
        r, _, _ = phx_residual(h)
        if r < tol32:
            break
    s32 = s
    if r < tol32 and r >= tol:
        phx_get_state(h, psi32, n32)
        phx_set_state(h64, psi32.to(torch.complex128), n32.double())
        while s < cap:
            phx_step_n(h64, check_every)
            s += check_every
            r, _, _ = phx_residual(h64)
            if r < tol:
                break
    e1.record(stream)
    torch.cuda.synchronize()
    return dict(steps=s, steps32=s32, ms=e0.elapsed_time(e1), r=float(r), converged=bool(r < tol),
                state=_last_state(h64 if s > s32 else h, n))


def _state_buffers(n, h):
    if h.real == np.float64:
        return (torch.empty(n, n, dtype=torch.complex128, device="cuda"),
                torch.empty(n, n, dtype=torch.float64, device="cuda"))
    return (torch.empty(n, n, dtype=torch.complex64, device="cuda"),
            torch.empty(n, n, device="cuda"))


def _last_state(h, n):
    psi, nn = _state_buffers(n, h)
    phx_get_state(h, psi, nn)
    return psi, nn


def new_network(problem, max_batch=8, channels=32, layers=4, modes_x=16, modes_y=32,
                proj_hidden=64, weights=None):
    """The warm-start network on this grid, with `weights` (flat FP32 in the
    layout of include/phx.h) loaded when given."""
    net = phx_fno_create(height=problem.n, width=problem.n, channels=channels, layers=layers,
                         modes_x=modes_x, modes_y=modes_y, in_channels=3, out_channels=3,
                         proj_hidden=proj_hidden, max_batch=max_batch,
                         stream=_stream().cuda_stream)
    if weights is not None:
        phx_fno_set_params(net, np.ascontiguousarray(weights, np.float32))
    return net


def initial_weights(net, seed):
    """Seeded initial weights in the flat layout (spectral ~ U[0, 1/C^2)
    (Li et al.), dense ~ U[-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0)."""
    c = net.cfg
    C, MX, MY, Pp = c["channels"], c["modes_x"], c["modes_y"], c["proj_hidden"]
    shapes = [("W_lift", (c["in_channels"], C)), ("b_lift", (C,))]
    for l in range(c["layers"]):
        shapes += [("Rr%d" % l, (MY, MX, C, C)), ("Ri%d" % l, (MY, MX, C, C)),
                   ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
    shapes += [("Q1", (C, Pp)), ("q1", (Pp,)), ("Q2", (Pp, c["out_channels"])),
               ("q2", (c["out_channels"],))]
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in shapes:
        size = int(np.prod(shape))
        if name.startswith("R"):
            parts.append(rng.uniform(0.0, 1.0 / (C * C), size))
        elif len(shape) == 2:
            bound = 1.0 / np.sqrt(shape[0])
            parts.append(rng.uniform(-bound, bound, size))
        else:
            parts.append(np.zeros(size))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == net.num_params
    return w


def density_match(psi_a, psi_b):
    """Relative L2 difference of the densities |psi|^2 of two states."""
    a = psi_a.abs().double() ** 2
    b = psi_b.abs().double() ** 2
    return float(torch.linalg.vector_norm(a - b) / max(float(torch.linalg.vector_norm(b)), 1e-300))
