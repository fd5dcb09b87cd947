"""Learned warm start for steady-state solves.

A Fourier neural operator (the ``phx_fno_*`` calls) maps a pump image to an
approximate stationary state (psi, n) of Eqs. (PULSE_psi)/(PULSE_res); the
RK4 relaxation then starts from that state instead of from noise.  This
module drives the loop on the GPU through the C ABI:

* ``generate`` -- solver-generated training pairs: batches of instances (one
  persistent launch per RK4 step) relaxed from noise; features and
  gauge-fixed targets are formed on the device.
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
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

from . import (phx_batch_create, phx_batch_get_state, phx_batch_norm_energy,
               phx_batch_residual, phx_batch_set_pump, phx_batch_set_state, phx_batch_step_n,
               phx_create, phx_fno_create, phx_fno_features, phx_fno_forward,
               phx_fno_get_params, phx_fno_loss_grad, phx_fno_set_params, phx_fno_targets,
               phx_fno_to_state, phx_fno_train_step, phx_get_state, phx_norm_energy,
               phx_residual, phx_set_pump, phx_set_state, phx_step_n, params_from_dict)

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


def _stream():
    return torch.cuda.current_stream()


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
    and with collect=True the final states as device tensors."""
    N = len(pumps)
    n = problem.n
    steps = np.full(N, -1, np.int64)
    r_at = np.zeros(N)
    decayed = np.zeros(N, bool)
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
            norms, _ = phx_batch_norm_energy(b)
            dec = norms / (problem.cell * n * n) < tiny
            r, _, _ = _safe_residual(b, dec)
            newly = (~done) & (r < tol32) & (~dec)
            steps[c0:c1][newly] = s
            r_at[c0:c1][newly] = r[newly]
            decayed[c0:c1] |= (~done) & dec
            done |= newly | dec
        if not done.all():
            r, _, _ = _safe_residual(b, decayed[c0:c1])
            r_at[c0:c1][~done] = r[~done]
        if collect:
            for k in range(m):
                phx_batch_get_state(b, k, psi_all[c0 + k], n_all[c0 + k])
        if log:
            log("screen %d..%d: %d steps, %.1f s, converged %d, decayed %d"
                % (c0, c1 - 1, s, time.time() - t0, int((steps[c0:c1] >= 0).sum()),
                   int(decayed[c0:c1].sum())))
        del b
    out = dict(steps=steps, r=r_at, decayed=decayed)
    if collect:
        out["psi"], out["nres"] = psi_all, n_all
    return out


def _safe_residual(b, decayed):
    """Per-member residuals; members whose psi has decayed to (near) zero
    report r = 1 (their ratio of two vanishing norms is meaningless)."""
    r, rn, om = phx_batch_residual(b)
    r = np.where(decayed, 1.0, r)
    return r, rn, om


def generate(problem, pumps, noise_seed0, steps=40000, tol32=1e-5, chunk=512, log=None):
    """Training pairs: each pump relaxed from seeded noise (std 1e-2 per
    quadrature) until r_psi < tol32 or `steps`; the final state, gauge-fixed
    and scaled, is the target.  Returns (features, targets, screen dict)."""
    import synth
    n = problem.n

    def cold(i0, i1):
        z = np.stack([synth.complex_normal((n, n), 1e-2, noise_seed0 + i) for i in range(i0, i1)])
        return (torch.as_tensor(z.astype(np.complex64)).cuda(),
                torch.zeros(i1 - i0, n, n, device="cuda"))

    res = screen(problem, pumps, cold, tol32=tol32, cap=steps, chunk=chunk, collect=True, log=log)
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
    """Seeded initial weights in the flat layout (spectral ~ U[0, 1/C^2),
    dense ~ U[-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0)."""
    import synth
    c = net.cfg
    C, MX, MY, Pp = c["channels"], c["modes_x"], c["modes_y"], c["proj_hidden"]
    shapes = [("W_lift", (c["in_channels"], C)), ("b_lift", (C,))]
    for l in range(c["layers"]):
        shapes += [("Rr%d" % l, (MY, MX, C, C)), ("Ri%d" % l, (MY, MX, C, C)),
                   ("W%d" % l, (C, C)), ("b%d" % l, (C,))]
    shapes += [("Q1", (C, Pp)), ("q1", (Pp,)), ("Q2", (Pp, c["out_channels"])),
               ("q2", (c["out_channels"],))]
    w = synth.fno_init_weights(shapes, seed, C)
    assert w.size == net.num_params
    return w


def density_match(psi_a, psi_b):
    """Relative L2 difference of the densities |psi|^2 of two states."""
    a = psi_a.abs().double() ** 2
    b = psi_b.abs().double() ** 2
    return float(torch.linalg.vector_norm(a - b) / max(float(torch.linalg.vector_norm(b)), 1e-300))


def run_experiment(n_train=2000, n_test=200, gen_steps=40000, epochs=40, cap=200000,
                   tol=1e-6, tol32=1e-5, check_every=100, seed=0, time_limit=None, log=print):
    """Generate, train, and compare warm and cold relaxations on held-out
    pumps.  Returns a JSON-able report."""
    import synth
    c = synth.load_constants()["steady_256_L128"]
    pthr = synth.load_constants()["pump_threshold"]
    d = synth.base_params(256, 256, 128.0, 128.0, dt=c["dt"], **synth.reservoir_physics())
    prob = Problem(d, pthr)
    n = prob.n
    rep = {"workload": "steady_256: 256x256, 128 um periodic, config-2 physics, dt %.6g ps "
                       "(0.85 of the RK4 limit); pumps: sums of 1-4 Gaussians, waist 3-15 um, "
                       "peak 1-3 P_thr" % c["dt"],
           "n_train": n_train, "n_test": n_test, "gen_steps": gen_steps, "epochs": epochs,
           "tol": tol, "tol32": tol32, "check_every": check_every, "cap": cap}
    t_all = time.time()
    train_pumps = synth.random_gaussian_pumps(256, 128.0, n_train, seed=5000)
    test_pumps = synth.random_gaussian_pumps(256, 128.0, n_test, seed=5000 + n_train)
    t0 = time.time()
    feats, targs, gen = generate(prob, train_pumps, 105000, steps=gen_steps, tol32=tol32, log=log)
    rep["generate_s"] = time.time() - t0
    rep["train_converged_fraction"] = float((gen["steps"] >= 0).mean())
    rep["train_decayed_fraction"] = float(gen["decayed"].mean())
    # held-out targets from the same protocol (for the held-out loss)
    tf, tt, tgen = generate(prob, test_pumps, 105000 + n_train, steps=gen_steps, tol32=tol32,
                            log=log)
    net = new_network(prob)
    phx_fno_set_params(net, initial_weights(net, seed))
    t0 = time.time()
    hist = train(net, feats, targs, epochs, log=log)
    torch.cuda.synchronize()
    rep["train_s"] = time.time() - t0
    rep["train_loss"] = hist
    rep["heldout_loss"] = eval_loss(net, tf, tt)
    del feats, targs
    # screening of held-out pumps: cold (fresh noise) and warm (prediction)
    cold_seed = 205000

    def cold(i0, i1):
        z = np.stack([synth.complex_normal((n, n), 1e-2, cold_seed + i) for i in range(i0, i1)])
        return (torch.as_tensor(z.astype(np.complex64)).cuda(),
                torch.zeros(i1 - i0, n, n, device="cuda"))

    wpsi, wn = predict_states(net, prob, tf)

    def warm(i0, i1):
        return wpsi[i0:i1].contiguous(), wn[i0:i1].contiguous()

    t0 = time.time()
    sc = screen(prob, test_pumps, cold, tol32=tol32, cap=cap, check_every=check_every, log=log)
    sw = screen(prob, test_pumps, warm, tol32=tol32, cap=cap, check_every=check_every, log=log)
    rep["screen_s"] = time.time() - t0
    both = np.where((sc["steps"] >= 0) & (sw["steps"] >= 0))[0]
    rep["screen"] = {
        "cold_converged": int((sc["steps"] >= 0).sum()), "warm_converged": int((sw["steps"] >= 0).sum()),
        "cold_decayed": int(sc["decayed"].sum()), "warm_decayed": int(sw["decayed"].sum()),
        "both_converged": int(len(both)),
        "cold_steps32_median": float(np.median(sc["steps"][both])) if len(both) else None,
        "warm_steps32_median": float(np.median(sw["steps"][both])) if len(both) else None}
    # timed single-instance relaxations to tol for members converged in both
    rows = []
    for i in both:
        if time_limit and time.time() - t_all > time_limit:
            break
        z = cold(int(i), int(i) + 1)
        rc = relax(prob, test_pumps[i], init=(z[0][0], z[1][0]), tol=tol, tol32=tol32,
                   check_every=check_every, cap=cap, instance=int(i))
        rw = relax(prob, test_pumps[i], net=net, tol=tol, tol32=tol32, check_every=check_every,
                   cap=cap, instance=int(i))
        row = {"i": int(i), "cold_steps": rc["steps"], "warm_steps": rw["steps"],
               "cold_ms": rc["ms"], "warm_ms": rw["ms"], "cold_r": rc["r"], "warm_r": rw["r"],
               "cold_converged": rc["converged"], "warm_converged": rw["converged"]}
        if rc["converged"] and rw["converged"]:
            row["density_rel_diff"] = density_match(rw["state"][0], rc["state"][0])
        rows.append(row)
    rep["relax"] = rows
    ok = [r for r in rows if r["cold_converged"] and r["warm_converged"]]
    if ok:
        cs = np.array([r["cold_steps"] for r in ok])
        ws = np.array([r["warm_steps"] for r in ok])
        cm = np.array([r["cold_ms"] for r in ok])
        wm = np.array([r["warm_ms"] for r in ok])
        dm = np.array([r.get("density_rel_diff", np.nan) for r in ok])
        q = lambda a: [float(np.percentile(a, 25)), float(np.median(a)), float(np.percentile(a, 75))]
        rep["summary"] = {"pairs": len(ok), "cold_steps_q": q(cs), "warm_steps_q": q(ws),
                          "cold_ms_q": q(cm), "warm_ms_q": q(wm),
                          "warm_faster_fraction": float((wm < cm).mean()),
                          "speedup_median_ms": float(np.median(cm / wm)),
                          "same_state_fraction": float((dm < 1e-3).mean()),
                          "density_rel_diff_median": float(np.nanmedian(dm))}
    rep["total_s"] = time.time() - t_all
    return rep, net


def main(argv=None):
    ap = argparse.ArgumentParser(description="FNO warm start: generate, train, compare")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--gen-steps", type=int, default=40000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--cap", type=int, default=200000)
    ap.add_argument("--time-limit", type=float, default=None)
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-weights", default=None)
    a = ap.parse_args(argv)
    from . import _build
    _build.build()
    rep, net = run_experiment(a.train, a.test, a.gen_steps, a.epochs, a.cap,
                              time_limit=a.time_limit,
                              log=lambda s: print(s, file=sys.stderr, flush=True))
    if a.save_weights:
        np.save(a.save_weights, phx_fno_get_params(net))
    js = json.dumps(rep, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(js)
    print(js)


if __name__ == "__main__":
    main()
