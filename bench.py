"""Benchmark of the fused RK4 dNLSE step on GB300.

One bench step = one full run of the driven-dissipative reservoir workload
(default: 2048x2048 grid over a 200 um periodic box -- the 1024^2 workload's
cell size and time step --, ring pump of radius 20 um / width 3 um at
1.5 P_thr, initial noise 1e-2, 10^4 RK4 steps at half the stability limit)
plus the FP64 norm/energy and steady-state-residual reductions, through the
C ABI.

Prints ONE JSON line (rank 0).  Metric: RK4 site-updates/s (whole job).
  value      device-timed (CUDA events on the solver's stream), inputs resident
  e2e        same metric through the C ABI with pinned host buffers, H2D/D2H
             copies inside the timed region (host wall clock)
  roofline   dominant kernel (the fused RK4 step): algorithmic bytes / average
             launch time against the measured HBM copy bandwidth
  cpu_baseline  the FP64 numpy oracle timed on a bounded sample (rank 0, N=1)
  precision_error  FP32 runs: relative L2 error of the final state against
             the FP64 path run on the same inputs over the same steps

--impl reference times the oracle itself on the same workload.
Under torchrun (N > 1) every rank runs an independent replica (different
seeds); value = all ranks' site-updates / max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RK4_STEPS = 10000
# Algorithmic FP64 flops per site per RK4 step (FMA = 2): per stage the
# complex 5-point stencil 14, |psi|^2 3, local potential 4 (2 without the
# reservoir), H 4, gain G 2, K 4, Kn 4, accumulators 6, stage values 6; four
# stages plus the final combination.  The coherent drive adds the complex
# product E exp(-i omega t)/hbar into H, 4 FMA per stage.
FLOPS_PER_SITE = {"reservoir": 194, "conservative": 144, "driven": 176}
# FP64 pipe of GB300 from unit counts: 2 DFMA per SM per cycle (152 SMs,
# 2.07 GHz max clock) -- context only; the roofline uses the measured peak
# (phx_alu_peak_probe).
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
BYTES_PER_SITE = {  # algorithmic bytes per site per RK4 step (read + write once)
    (32, "reservoir"): 28, (64, "reservoir"): 56,
    (32, "conservative"): 16, (64, "conservative"): 32,
    (32, "spinor"): 52, (64, "spinor"): 104,
    (32, "driven"): 28, (64, "driven"): 56,   # psi in/out, V, E
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="phx", choices=["phx", "reference"])
    ap.add_argument("--workload", default="reservoir_2048",
                    choices=["reservoir_2048", "reservoir_1024", "reservoir", "spinor_2048",
                             "conservative_64", "ensemble", "twa_ensemble", "driven_9000",
                             "drive_sweep", "steady_256", "fno_train"])
    ap.add_argument("--grid", type=int, default=1024,
                    help="grid size of the 'reservoir' workload (100 um box, config-2 physics)")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--rk4-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--integrator", default="rk4", choices=["rk4", "ssf"],
                    help="time stepper of the single-handle workloads: fused RK4 or split-step Fourier")
    ap.add_argument("--dt-factor", type=float, default=1.0,
                    help="split-step only: time step = this x the workload's (half the RK4 "
                         "limit); above 2 the handle is created with the split-step integrator")
    ap.add_argument("--tile", type=int, default=0,
                    help="step-kernel configuration (0 = autotune, 1..7 TMA-fed, 9 generic)")
    ap.add_argument("--no-precision-error", action="store_true",
                    help="skip the FP64 run that measures the FP32 error (profiling runs)")
    ap.add_argument("--no-steady", action="store_true",
                    help="skip the reduced warm-vs-cold steady-state measurement")
    # steady_256 (warm-start experiment) sizes
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--gen-steps", type=int, default=40000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--cap", type=int, default=200000)
    ap.add_argument("--time-limit", type=float, default=None)
    ap.add_argument("--out", default=None)
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate(pg, world, units_per_rank, ms_local):
    """Whole-job throughput of `world` weak-scaled replicas: every rank did
    `units_per_rank` units; the job took the slowest rank's time."""
    ms = max_over_ranks(pg, ms_local)
    return ms, world * units_per_rank / (ms * 1e-3)


def workload_name(args):
    if args.workload == "reservoir":
        return "reservoir_%d" % args.grid
    return args.workload


def workload(name, seed_offset=0, grid=1024):
    import synth
    if name == "reservoir_2048":
        cfg = synth.reservoir_2048(seed=2 + seed_offset)
        kind = "reservoir"
        desc = ("driven-dissipative GP + reservoir, 2048x2048, 200 um periodic (cell 100/1024 um), "
                "ring pump r=20 um w=3 um at 1.5 P_thr, psi0 noise 1e-2, dt = half RK4 limit")
    elif name == "reservoir_1024" or (name == "reservoir" and grid == 1024):
        cfg = synth.reservoir_1024(seed=2 + seed_offset)
        kind = "reservoir"
        desc = ("driven-dissipative GP + reservoir, 1024x1024, 100 um periodic, ring "
                "pump r=20 um w=3 um at 1.5 P_thr, psi0 noise 1e-2, dt = half RK4 limit")
    elif name == "reservoir":
        cfg = synth.reservoir_grid(grid, seed=2 + seed_offset)
        kind = "reservoir"
        desc = ("driven-dissipative GP + reservoir, %dx%d, 100 um periodic, ring pump r=20 um "
                "w=3 um at 1.5 P_thr, psi0 noise 1e-2, dt = half RK4 limit" % (grid, grid))
    elif name == "driven_9000":
        cfg = synth.driven_lattice(9000, seed=11 + seed_offset)
        kind = "driven"
        desc = ("coherently driven potential lattice, 9000x9000, 900 um periodic, 272^2 SSH "
                "super-Gaussian wells with AAH depth modulation, drive E0 = 5.6856 ueV at "
                "omega = -5.6883 /ps on the corner well, loss 0.15 /ps, dt = half RK4 limit")
    elif name == "spinor_2048":
        cfg = synth.spinor_grid(2048, seed=3 + seed_offset, const_key="spinor_2048_L200")
        kind = "spinor"
        desc = ("TE-TM spinor GP + reservoir, 2048x2048, 200 um periodic, Gaussian pump "
                "w=10 um at 1.5 P_thr, Philox noise var 1e-3 per step")
    else:
        cfg = synth.conservative_64(seed=1 + seed_offset)
        kind = "conservative"
        desc = "conservative GP 64x64, 20 um periodic, Gaussian amp 5 w 3 um + noise"
    return cfg, kind, desc


STEP_KERNEL_SOURCES = ("phx_internal.h", "phx_noise.cuh", "rk4_generic.cuh", "rk4_tma.h",
                       "rk4_tma_kernel.cuh", "rk4_tma.cu", "rk4_tma_cfg1.cu", "rk4_tma_cfg2.cu",
                       "rk4_tma_cfg3.cu", "rk4_tma_cfg4.cu", "rk4_tma_cfg5.cu", "rk4_tma_cfg6.cu",
                       "rk4_tma_cfg7.cu")


def step_kernel_name(tile):
    if 1 <= tile <= 7:
        return "rk4_f32_tma (fused, one launch per RK4 step)"
    return "rk4_step_generic (fused, one launch per RK4 step)"


def kernel_hash():
    """Hash of the sources the TMA-fed scalar step kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2411_18341_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name, precision, tile=None):
    """DRAM bytes per launch of the fused step kernel from the committed ncu
    summary, if it was captured from the current kernel sources (and, when
    given, with the tile configuration in use)."""
    path = os.path.join(ROOT, "profiles", "rk4_step_traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    key = "%s_fp%d" % (workload_name, precision)
    e = rec.get(key)
    if not e or e.get("kernel_sources") != kernel_hash():
        return None
    tiles = e.get("tiles", {})
    if tile is not None:
        e = tiles.get(str(tile))
    return e.get("dram_bytes_per_launch") if e else None


class Clocks:
    """Samples nvidia-smi clocks during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.path = os.path.join("/tmp", "phx_clocks_%d.csv" % os.getpid())
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            try:
                pw.append(float(parts[3]))
            except ValueError:
                pass
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
               "reasons": sorted(reasons), "samples": len(sm)}
        if pw:
            out["power_w_median"] = float(np.median(pw))
        return out


def energy(clk, seconds, updates):
    """Board energy per site-update (the paper's energy per grid point and
    step) from the median power sampled during the timed region."""
    if not clk or "power_w_median" not in clk or updates <= 0:
        return None
    return {"nJ_per_site_update": clk["power_w_median"] * seconds / updates * 1e9,
            "power_w_median": clk["power_w_median"], "source": "nvidia-smi power.draw"}


def _oracle_steps(path, warmup, nsteps, per, budget_s):
    """One worker process: the FP64 oracle as it stands (numpy, one thread)
    on its own copy of the workload: `warmup` untimed steps, then either
    nsteps x per steps or, with nsteps None, steps until budget_s (at most
    50).  Returns (timed steps, seconds)."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import pickle
    from oracle import gp
    with open(path, "rb") as f:
        cfg = pickle.load(f)
    p = gp.Params(**cfg["params"])
    psi, n = np.array(cfg["psi0"], complex), cfg["n0"]
    P = None if cfg["P"] is None else np.broadcast_to(cfg["P"], (p.ncomp, p.ny, p.nx))
    V, E = cfg.get("V"), cfg.get("E")
    for _ in range(warmup):
        gp.run(psi, n, P, V, p, 1, E=E)
    t0 = time.perf_counter()
    steps = 0
    while True:
        k = per if nsteps is not None else 1
        psi, n = gp.run(psi, n, P, V, p, k, step0=steps, E=E, t0=steps * p.dt)
        steps += k
        if nsteps is not None:
            if steps >= nsteps * per:
                break
        elif time.perf_counter() - t0 > budget_s or steps >= 50:
            break
    return steps, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_on_cores(cfg, warmup=0, nsteps=None, per=1, budget_s=15.0, cores=None):
    """The oracle timed on every host core at once: one process per core
    (spawned, so no GPU context is inherited), each running its own copy of
    the workload.  Returns (site-updates/s of all processes together, the
    processes used, per-process site-updates/s)."""
    import multiprocessing as mp
    import pickle
    import tempfile
    cores = cores or host_cores()
    fd, path = tempfile.mkstemp(suffix=".pkl")
    with os.fdopen(fd, "wb") as f:
        pickle.dump(cfg, f, protocol=pickle.HIGHEST_PROTOCOL)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_steps, [(path, warmup, nsteps, per, budget_s)] * cores)
    finally:
        os.unlink(path)
    sites = cfg["params"]["nx"] * cfg["params"]["ny"]
    total = sites * sum(s for s, _ in res) / max(e for _, e in res)
    per_proc = [sites * s / e for s, e in res]
    return total, cores, per_proc, res


def cpu_baseline(name, cfg, budget_s=15.0):
    """Time the FP64 oracle (as it stands) on a bounded sample of the
    workload, on all host cores (one process per core)."""
    total, cores, per_proc, res = oracle_on_cores(cfg, budget_s=budget_s)
    p = cfg["params"]
    return {"value": total, "unit": "site-updates/s", "cores": cores, "kind": "oracle",
            "per_core_value": float(np.median(per_proc)),
            "sample": "%d processes x %d-%d RK4 steps of the %dx%d %s workload (numpy FP64, one "
                      "thread each, all at once), %.1f s" % (
                          cores, min(s for s, _ in res), max(s for s, _ in res), p["nx"], p["ny"],
                          name, max(e for _, e in res))}


def _rel_l2(a, b):
    import torch
    a, b = a.reshape(-1), b.reshape(-1)
    den = float(torch.linalg.vector_norm(b))
    return float(torch.linalg.vector_norm(a - b)) / den if den > 0 else None


def fresh_run(phx, d, cfg, nsteps, stream, dev, step_fn_name="phx_step_n", prec=64):
    """The workload run from step 0 and time 0 on a new handle in `prec`
    (inputs rounded to it): with prec 64 the FP64 path, pinned to the oracle
    at 1e-11, the yardstick of the FP32 error; with prec 32 the FP32 result
    it is compared with (same noise counters and drive phases)."""
    import torch
    h = phx.phx_create(phx.params_from_dict(d, precision=prec, stream=stream.cuda_stream))
    f64, c128 = (torch.float64, torch.complex128) if prec == 64 else (torch.float32,
                                                                      torch.complex64)
    dt = lambda a, t: None if a is None else torch.tensor(np.asarray(a), dtype=t, device=dev)  # noqa: E731
    P = None if cfg.get("P") is None else dt(np.asarray(cfg["P"])[0], f64)
    V = dt(cfg.get("V"), f64)
    E = None if cfg.get("E") is None else dt(np.asarray(cfg["E"])[0], c128)
    psi0 = dt(np.ascontiguousarray(cfg["psi0"]), c128)
    n0 = dt(cfg.get("n0"), f64)
    # the copies above run on torch's stream; the handle reads them on its own
    torch.cuda.synchronize()
    if P is not None:
        phx.phx_set_pump(h, P)
    if V is not None:
        phx.phx_set_potential(h, V)
    if E is not None:
        phx.phx_set_drive(h, E)
    phx.phx_set_state(h, psi0, n0)
    getattr(phx, step_fn_name)(h, nsteps)
    psi = torch.empty_like(psi0)
    n = None if n0 is None else torch.empty_like(n0)
    phx.phx_get_state(h, psi, n)
    torch.cuda.synchronize()
    phx.phx_destroy(h)
    return psi, n


def fp64_run(phx, d, cfg, nsteps, stream, dev, step_fn_name="phx_step_n"):
    return fresh_run(phx, d, cfg, nsteps, stream, dev, step_fn_name, 64)


def precision_error(psi32, n32, psi64, n64, what):
    """Relative L2 error of an FP32 result against the FP64 result of the
    same inputs and steps (the FP32 run starts from the inputs rounded to
    FP32; that rounding is part of its error)."""
    dev = psi64.device
    out = {"psi_rel_l2": _rel_l2(psi32.to(dev).to(psi64.dtype), psi64),
           "against": "FP64 GPU path (pinned to the oracle at rel. L2 1e-11) on the same "
                      "inputs and steps", "what": what}
    if n32 is not None and n64 is not None:
        out["n_rel_l2"] = _rel_l2(n32.to(dev).to(n64.dtype), n64)
    return out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "ensemble":
        cfg, kind, desc = workload("reservoir", grid=128)
        desc = "one 128x128 member of the ensemble workload"
    elif args.workload == "twa_ensemble":
        import synth
        cfg = synth.twa_ensemble(count=1)[0]
        desc = "one 256x256 realisation of the truncated-Wigner ensemble"
    elif args.workload == "driven_9000":
        import synth
        cfg = synth.crop(workload("driven_9000")[0], 512)
        desc = "512x512 corner window of the driven 9000x9000 lattice"
    elif args.workload == "drive_sweep":
        import synth
        cfg = synth.drive_sweep(count=1)[0]
        desc = "one 512x512 member of the drive-frequency sweep"
    else:
        cfg, kind, desc = workload(args.workload, grid=args.grid)
    d = cfg["params"]
    per = 1 if d["nx"] * d["ny"] >= 1 << 20 else 20
    # every host core runs its own copy (one process each), all at once
    val, cores, per_proc, res = oracle_on_cores(cfg, warmup=args.warmup, nsteps=args.steps,
                                                per=per)
    el = max(e for _, e in res)
    line = {"metric": "RK4 site-updates/s", "impl": "reference", "value": val,
            "unit": "site-updates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc,
                       "grid": "%dx%d" % (d["nx"], d["ny"]), "sample_rk4_steps_per_step": per},
            "cpu_baseline": {"value": val, "unit": "site-updates/s", "cores": cores,
                             "kind": "oracle", "per_core_value": float(np.median(per_proc)),
                             "sample": "%d processes, each %d RK4 steps per bench step of the "
                                       "%s workload (numpy FP64, one thread each)"
                                       % (cores, per, args.workload)},
            "e2e": {"value": val, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


TWA_SAMPLE_PS = 5.0   # sampling interval of the truncated-Wigner ensemble
TWA_SAMPLES = 10      # samples per bench step


def run_ensemble(args, world, rank, local, pg):
    """Batched workloads, one persistent launch per RK4 step for all members,
    replayed from a CUDA graph.

    ensemble: 256 independent reservoir instances on uneven grids (64 each
    at 128^2, 256^2, 512^2, 1024^2; pumps U[0.8, 3] P_thr, distinct seeds);
    per step 500 RK4 steps, then per-member FP64 norm/energy and residual.
    twa_ensemble: 150 truncated-Wigner realisations (256^2, 200 um,
    super-Gaussian pump w = 65 um at 2 P_thr, nu = 1, Wigner vacuum start);
    per step 10 samples, each 5 ps of RK4 steps followed by the per-member
    FP64 norm/energy read back to the host (the sampled observable).
    drive_sweep: 64 coherently driven scalar fields (512^2, 100 um, loss and
    Kerr, no reservoir), one drive spot at 64 frequencies; per step 500 RK4
    steps, then per-member FP64 norm/energy and residual."""
    import torch
    import synth
    import paper_2411_18341_gb300 as phx
    from paper_2411_18341_gb300 import _build
    _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    twa = args.workload == "twa_ensemble"
    sweep = args.workload == "drive_sweep"
    res = not sweep  # members with a reservoir
    if twa:
        members = synth.twa_ensemble(seed=7 + rank)
        dt = members[0]["params"]["dt"]
        per_sample = args.rk4_steps or int(round(TWA_SAMPLE_PS / dt))
        samples = TWA_SAMPLES
    elif sweep:
        members = synth.drive_sweep(seed0=3000 + 10000 * rank)
        per_sample = args.rk4_steps or 500
        samples = 1
    else:
        members = synth.ensemble(seed0=1000 + 10000 * rank)
        per_sample = args.rk4_steps or 500
        samples = 1
    rk4_steps = per_sample * samples
    stream = torch.cuda.Stream(device=dev)
    b = phx.phx_batch_create([phx.params_from_dict(m["params"], precision=32,
                                                   stream=stream.cuda_stream) for m in members])
    psi_d, n_d = [], []
    P_d = [torch.tensor(m["P"][0], dtype=torch.float32, device=dev) for m in members] if res else []
    E_d = [torch.tensor(m["E"][0], dtype=torch.complex64, device=dev) for m in members] \
        if sweep else []
    # the copies run on torch's stream; the batch reads them on its own
    torch.cuda.synchronize()
    for i, m in enumerate(members):
        if res:
            phx.phx_batch_set_pump(b, i, P_d[i])
        if sweep:
            phx.phx_batch_set_drive(b, i, E_d[i])
        psi_d.append(torch.tensor(m["psi0"][0], dtype=torch.complex64, device=dev))
        n_d.append(torch.tensor(m["n0"][0], dtype=torch.float32, device=dev) if res else None)
    del P_d, E_d
    sites = sum(m["params"]["nx"] * m["params"]["ny"] for m in members)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(k0=None, k1=None):
        for i in range(len(members)):
            phx.phx_batch_set_state(b, i, psi_d[i], n_d[i])
        if twa:
            # kernel time = the first sample's RK4 steps (no host sync inside)
            for k in range(samples):
                if k == 0 and k0 is not None:
                    k0.record(stream)
                phx.phx_batch_step_n(b, per_sample)
                if k == 0 and k1 is not None:
                    k1.record(stream)
                phx.phx_batch_norm_energy(b)
            return
        if k0 is not None:
            k0.record(stream)
        phx.phx_batch_step_n(b, rk4_steps)
        if k1 is not None:
            k1.record(stream)
        phx.phx_batch_norm_energy(b)
        phx.phx_batch_residual(b)

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    launches0 = phx.phx_launch_count()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        a, e, k0, k1 = ev[k]
        a.record(stream)
        one_step(k0, k1)
        e.record(stream)
    torch.cuda.synchronize()
    launches = phx.phx_launch_count() - launches0
    barrier(pg)
    clk = clocks.stop() if clocks else None
    ms, value = aggregate(pg, world, sites * rk4_steps,
                          float(np.mean([x[0].elapsed_time(x[1]) for x in ev])))
    kern_steps = per_sample if twa else rk4_steps
    kern_s = float(np.mean([x[2].elapsed_time(x[3]) for x in ev])) * 1e-3 / kern_steps

    # end to end: pinned host inputs in, every member's state out
    psi_h = [t.cpu().pin_memory() for t in psi_d]
    n_h = [t.cpu().pin_memory() if t is not None else None for t in n_d]
    P_h = [torch.tensor(m["P"][0], dtype=torch.float32).pin_memory() for m in members] \
        if res else []
    E_h = [torch.tensor(m["E"][0], dtype=torch.complex64).pin_memory() for m in members] \
        if sweep else []
    out_psi = [torch.empty_like(t).pin_memory() for t in psi_h]
    out_n = [torch.empty_like(t).pin_memory() if t is not None else None for t in n_h]
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    for i in range(len(members)):
        if res:
            phx.phx_batch_set_pump(b, i, P_h[i])
        if sweep:
            phx.phx_batch_set_drive(b, i, E_h[i])
        phx.phx_batch_set_state(b, i, psi_h[i], n_h[i])
    if twa:
        for k in range(samples):
            phx.phx_batch_step_n(b, per_sample)
            phx.phx_batch_norm_energy(b)
    else:
        phx.phx_batch_step_n(b, rk4_steps)
        phx.phx_batch_norm_energy(b)
        phx.phx_batch_residual(b)
    for i in range(len(members)):
        phx.phx_batch_get_state(b, i, out_psi[i], out_n[i])
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, time.perf_counter() - t0)
    # FP32 error per result: two members (the smallest and the largest grid
    # of the ensemble; member 0 of the truncated-Wigner ensemble) against
    # the FP64 path over the same steps (noise bits identical in both)
    picks = [] if args.no_precision_error else ([0] if twa else [0, len(members) - 1])
    prec_err = []
    for i in picks:
        m = members[i]
        psi32, n32 = fresh_run(phx, m["params"], m, rk4_steps, stream, dev, prec=32)
        psi64, n64 = fresh_run(phx, m["params"], m, rk4_steps, stream, dev, prec=64)
        e = precision_error(psi32, n32, psi64, n64,
                            "member %d (%dx%d) run on its own handle, %d steps from step 0, "
                            "both precisions" % (i, m["params"]["nx"], m["params"]["ny"],
                                                 rk4_steps))
        prec_err.append(e)
        del psi32, n32, psi64, n64
    pk, pk_kind = peaks()
    bps = 24 if sweep else 28  # psi in/out + (n in/out, P) or (Re E, Im E)
    achieved = bps * sites / kern_s / 1e9
    if sweep:
        desc = ("64 coherently driven scalar fields, 512^2, 100 um periodic, loss 0.15 /ps, "
                "g = 6e-3 meV um^2, one Gaussian drive spot (0.05 meV, w = 20 um) at 64 "
                "frequencies in [-1, 2] /ps, each member its own frequency and FP64 time")
        per_step = ("set_state x64 + %d batched RK4 steps + per-member FP64 norm/energy + "
                    "residual" % rk4_steps)
    elif twa:
        desc = ("150 truncated-Wigner realisations (nu = 1), 256^2, 200 um periodic, "
                "super-Gaussian pump w = 65 um at 2 P_thr, Wigner vacuum start")
        per_step = ("set_state x150 + %d samples, each %d batched RK4 steps (%.2f ps) + "
                    "per-member FP64 norm/energy to the host" % (samples, per_sample,
                                                                 per_sample * dt))
    else:
        desc = ("256 reservoir instances, 64 each at 128^2/256^2/512^2/1024^2, "
                "100 um, ring pumps U[0.8,3] P_thr, distinct seeds")
        per_step = ("set_state x256 + %d batched RK4 steps + per-member FP64 "
                    "norm/energy + residual" % rk4_steps)
    line = {
        "metric": "RK4 site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc,
                   "sites": sites, "rk4_steps_per_step": rk4_steps, "tile": phx.phx_batch_tile(b),
                   "per_step": per_step,
                   "l2": "inputs (%.2f GB) larger than L2" % (bps * sites / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": world * sites * rk4_steps / e2e_s, "unit": "site-updates/s",
                "h2d_bytes_per_step": sites * 16,
                "d2h_bytes_per_step": sites * (8 if sweep else 12)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"],
                     "traffic": recorded_traffic(args.workload, 32, phx.phx_batch_tile(b)),
                     "kernel": step_kernel_name(phx.phx_batch_tile(b)) + ", all members per launch",
                     "algorithmic_bytes_per_site": bps, "avg_launch_us": kern_s * 1e6,
                     "peak_source": pk_kind,
                     **({"note": "per-site Philox + Box-Muller noise every step: the kernel is "
                                 "bound by instruction issue, not by HBM"} if twa else {})},
        "clocks": clk,
        "energy": energy(clk, ms * 1e-3, sites * rk4_steps),
        "precision_error": prec_err,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if twa:
            line["cpu_baseline"] = cpu_baseline("twa_ensemble (one 256x256 member)",
                                                members[0])
        else:
            cfg, _, _ = workload("reservoir", grid=128)
            line["cpu_baseline"] = cpu_baseline("ensemble (one 128x128 member)", cfg)
    phx.phx_batch_destroy(b)
    if rank == 0:
        print(json.dumps(line), flush=True)


WAISTS = (3.0, 4.5, 6.0, 9.0, 12.0, 15.0)   # um, spot waists whose threshold is measured


def steady_experiment(n_train=2000, n_test=200, gen_steps=40000, epochs=40, cap=200000,
                      tol=1e-6, tol32=1e-5, check_every=100, seed=0, time_limit=None,
                      log=None):
    """Learned warm start against cold start on the steady-state workload
    (256x256, 128 um periodic, the reservoir workload's physics, dt at 0.7 of
    the RK4 limit of the linear part: the strongest pumps' reservoir
    blueshift g_r n of several meV shifts the spectrum, which 0.85 of the
    limit leaves unstable, while RK4 still damps the zero-group-velocity
    lattice modes of the 5-point stencil that a smaller dt would let grow
    inside the spot): the finite-spot thresholds are measured with the
    solver, pumps (sums of 1-4 Gaussians, waist 3-15 um, peak 1-3 times the
    threshold of a spot of that waist) are drawn, the training pairs are
    relaxed from noise by the batched solver, the network is trained only on
    the pairs that reached r_psi < tol32, and held-out pumps are relaxed to
    r_psi < tol from noise (cold) and from the prediction (warm) under the
    same protocol.  Returns (report dict, network)."""
    import torch
    import synth
    from paper_2411_18341_gb300 import warmstart as ws
    log = log or (lambda s: None)
    d = synth.base_params(256, 256, 128.0, 128.0, dt=0.0, **synth.reservoir_physics())
    d["dt"] = ws.stable_dt(d, 0.7)
    pthr = ws.pump_threshold(d)
    prob = ws.Problem(d, pthr)
    n = prob.n
    t_all = time.time()
    thr, _ = ws.spot_thresholds(prob, WAISTS)
    fin = np.isfinite(thr)
    top = float(np.max(thr[fin])) if fin.any() else 1.0
    thr_used = np.where(fin, thr, top)
    lw, lt = np.log(np.asarray(WAISTS)), np.log(thr_used)
    spot = lambda w: pthr * float(np.exp(np.interp(np.log(w), lw, lt)))  # noqa: E731
    rep = {"workload": "steady_256: 256x256, 128 um periodic, config-2 physics, dt %.6g ps "
                       "(0.7 of the RK4 limit); pumps: sums of 1-4 Gaussians, waist 3-15 um, "
                       "peak 1-3 x the solver-measured threshold of a spot of that waist"
                       % d["dt"],
           "spot_threshold_factors": {"%g" % w: float(t) for w, t in zip(WAISTS, thr)},
           "n_train": n_train, "n_test": n_test, "gen_steps": gen_steps, "epochs": epochs,
           "tol": tol, "tol32": tol32, "check_every": check_every, "cap": cap}
    train_pumps = synth.random_gaussian_pumps(256, 128.0, n_train, seed=5000, threshold=spot)
    test_pumps = synth.random_gaussian_pumps(256, 128.0, n_test, seed=5000 + n_train,
                                             threshold=spot)

    def noise_init(seed0):
        def init(i0, i1):
            z = np.stack([synth.complex_normal((n, n), 1e-2, seed0 + i) for i in range(i0, i1)])
            return (torch.as_tensor(z.astype(np.complex64)).cuda(),
                    torch.zeros(i1 - i0, n, n, device="cuda"))
        return init

    t0 = time.time()
    feats, targs, gen = ws.generate(prob, train_pumps, noise_init(105000), steps=gen_steps,
                                    tol32=tol32, log=log)
    rep["generate_s"] = time.time() - t0
    keep = np.where(gen["steps"] >= 0)[0]
    rep["train_converged"] = int(len(keep))
    rep["train_decayed"] = int(gen["decayed"].sum())
    rep["train_diverged"] = int(gen["diverged"].sum())
    sel = torch.as_tensor(keep, device="cuda")
    feats, targs = feats.index_select(0, sel), targs.index_select(0, sel)
    tf, tt, tgen = ws.generate(prob, test_pumps, noise_init(105000 + n_train), steps=gen_steps,
                               tol32=tol32, log=log)
    tkeep = torch.as_tensor(np.where(tgen["steps"] >= 0)[0], device="cuda")
    rep["heldout_converged"] = int(len(tkeep))
    net = ws.new_network(prob)
    ws.phx_fno_set_params(net, ws.initial_weights(net, seed))
    t0 = time.time()
    hist = ws.train(net, feats, targs, epochs, log=log) if len(keep) >= 8 else []
    torch.cuda.synchronize()
    rep["train_s"] = time.time() - t0
    rep["train_loss"] = hist
    if len(tkeep):
        rep["heldout_loss"] = ws.eval_loss(net, tf.index_select(0, tkeep),
                                           tt.index_select(0, tkeep))
    del feats, targs, tt
    cold = noise_init(205000)
    wpsi, wn = ws.predict_states(net, prob, tf)

    def warm(i0, i1):
        return wpsi[i0:i1].contiguous(), wn[i0:i1].contiguous()

    t0 = time.time()
    sc = ws.screen(prob, test_pumps, cold, tol32=tol32, cap=cap, check_every=check_every, log=log)
    sw = ws.screen(prob, test_pumps, warm, tol32=tol32, cap=cap, check_every=check_every, log=log)
    rep["screen_s"] = time.time() - t0
    both = np.where((sc["steps"] >= 0) & (sw["steps"] >= 0))[0]
    rep["screen"] = {
        "cold_converged": int((sc["steps"] >= 0).sum()),
        "warm_converged": int((sw["steps"] >= 0).sum()),
        "cold_decayed": int(sc["decayed"].sum()), "warm_decayed": int(sw["decayed"].sum()),
        "cold_diverged": int(sc["diverged"].sum()), "warm_diverged": int(sw["diverged"].sum()),
        "both_converged": int(len(both)),
        "cold_steps32_median": float(np.median(sc["steps"][both])) if len(both) else None,
        "warm_steps32_median": float(np.median(sw["steps"][both])) if len(both) else None}
    rows = []
    for i in both:
        if time_limit and time.time() - t_all > time_limit:
            break
        z = cold(int(i), int(i) + 1)
        rc = ws.relax(prob, test_pumps[i], init=(z[0][0], z[1][0]), tol=tol, tol32=tol32,
                      check_every=check_every, cap=cap, instance=int(i))
        rw = ws.relax(prob, test_pumps[i], net=net, tol=tol, tol32=tol32,
                      check_every=check_every, cap=cap, instance=int(i))
        row = {"i": int(i), "cold_steps": rc["steps"], "warm_steps": rw["steps"],
               "cold_ms": rc["ms"], "warm_ms": rw["ms"], "cold_r": rc["r"], "warm_r": rw["r"],
               "cold_converged": rc["converged"], "warm_converged": rw["converged"]}
        if rc["converged"] and rw["converged"]:
            row["density_rel_diff"] = ws.density_match(rw["state"][0], rc["state"][0])
        rows.append(row)
    rep["relax"] = rows
    ok = [r for r in rows if r["cold_converged"] and r["warm_converged"]]
    if ok:
        cs = np.array([r["cold_steps"] for r in ok])
        wsp = np.array([r["warm_steps"] for r in ok])
        cm = np.array([r["cold_ms"] for r in ok])
        wm = np.array([r["warm_ms"] for r in ok])
        dm = np.array([r.get("density_rel_diff", np.nan) for r in ok])
        q = lambda a: [float(np.percentile(a, 25)), float(np.median(a)),  # noqa: E731
                       float(np.percentile(a, 75))]
        rep["summary"] = {"pairs": len(ok), "cold_steps_q": q(cs), "warm_steps_q": q(wsp),
                          "cold_ms_q": q(cm), "warm_ms_q": q(wm),
                          "warm_faster_fraction": float((wm < cm).mean()),
                          "speedup_median_ms": float(np.median(cm / wm)),
                          "same_state_fraction": float((dm < 1e-3).mean()),
                          "density_rel_diff_median": float(np.nanmedian(dm))}
    rep["total_s"] = time.time() - t_all
    return rep, net


def quick_rate(phx, torch, name, steps=500, warmup=50, drive=None):
    """Site-updates/s of one workload's step kernel (CUDA events around
    `steps` steps after `warmup`), for an extra key of the default line.
    drive: (E plane, omega) added to the workload (a coherent drive on top
    of its own terms)."""
    cfg, kind, desc = workload(name)
    d = dict(cfg["params"])
    if drive is not None:
        d["drive_omega"] = drive[1]
    stream = torch.cuda.Stream()
    h = phx.phx_create(phx.params_from_dict(d, precision=32, stream=stream.cuda_stream))
    real, cplx = torch.float32, torch.complex64
    P = None if cfg.get("P") is None else torch.tensor(np.asarray(cfg["P"])[0], dtype=real,
                                                           device="cuda")
    psi0 = torch.tensor(np.ascontiguousarray(cfg["psi0"]), dtype=cplx, device="cuda")
    n0 = None if cfg.get("n0") is None else torch.tensor(cfg["n0"], dtype=real, device="cuda")
    torch.cuda.synchronize()  # the handle reads the copies on its own stream
    if P is not None:
        phx.phx_set_pump(h, P)
    if drive is not None:
        phx.phx_set_drive(h, np.ascontiguousarray(drive[0], np.complex64))
    phx.phx_set_state(h, psi0, n0)
    phx.phx_step_n(h, warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    phx.phx_step_n(h, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / steps
    sites = d["nx"] * d["ny"]
    pk, _ = peaks()
    bps = BYTES_PER_SITE[(32, kind)] + (8 if drive is not None else 0)
    if drive is not None:
        desc += "; plus a coherent drive (plane wave, 0.05 meV, omega = %g /ps)" % drive[1]
    out = {"workload": name, "description": desc, "site_updates_per_s": sites / (us * 1e-6),
           "us_per_step": us, "tile": phx.phx_tile(h),
           "roofline_frac": bps * sites / (us * 1e-6) / 1e9 / pk["hbm_gbs"],
           "algorithmic_bytes_per_site": bps, "steps_timed": steps}
    phx.phx_destroy(h)
    return out


def steady_key(rep):
    """The warm-vs-cold summary carried in a bench line."""
    s = rep.get("summary") or {}
    return {"workload": rep["workload"], "n_train": rep["n_train"],
            "train_converged": rep["train_converged"], "n_test": rep["n_test"],
            "heldout_converged": rep["heldout_converged"], "epochs": rep["epochs"],
            "pairs": s.get("pairs", 0),
            "cold_ms_median": s.get("cold_ms_q", [None] * 3)[1],
            "warm_ms_median": s.get("warm_ms_q", [None] * 3)[1],
            "cold_steps_median": s.get("cold_steps_q", [None] * 3)[1],
            "warm_steps_median": s.get("warm_steps_q", [None] * 3)[1],
            "speedup_median_ms": s.get("speedup_median_ms"),
            "warm_faster_fraction": s.get("warm_faster_fraction"),
            "same_state_fraction": s.get("same_state_fraction"),
            "tol": rep["tol"], "timing": "CUDA events, FNO inference inside the warm runs",
            "seconds": rep["total_s"]}


def run_fno_train(args, world, rank, local):
    """--workload fno_train: Adam training steps of the warm-start network
    (256x256 grid, 4 layers, width 32, 16 x 32 kept modes, batch 8) on seeded
    synthetic features and targets, through the C ABI.  value = training
    samples/s; roofline = the algorithmic GEMM flops the steps issue (BF16
    operands, FP32 accumulation) against the measured BF16 tensor peak."""
    import torch
    import synth
    import paper_2411_18341_gb300 as phx
    from paper_2411_18341_gb300 import warmstart as ws
    torch.cuda.set_device(local)
    d = synth.base_params(256, 256, 128.0, 128.0, dt=0.0, **synth.reservoir_physics())
    d["dt"] = ws.stable_dt(d, 0.7)
    prob = ws.Problem(d, ws.pump_threshold(d))
    net = ws.new_network(prob, max_batch=8)
    phx.phx_fno_set_params(net, ws.initial_weights(net, 0))
    pumps = synth.random_gaussian_pumps(256, 128.0, 64, seed=9000)
    feats = ws.features(prob, pumps)
    rng = np.random.default_rng(9)
    targs = torch.tensor(rng.normal(0.0, 0.3, size=(64, 256, 256, 3)).astype(np.float32),
                         device="cuda")
    per_step = 16   # Adam steps per bench step (128 samples)
    stream = torch.cuda.current_stream()

    def one_step():
        for k in range(per_step):
            b = (k * 8) % 64
            phx.phx_fno_train_step(net, feats[b:b + 8], targs[b:b + 8], 1e-4)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    f0 = phx.phx_fno_gemm_flops(net)
    launches0 = phx.phx_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(torch.cuda.current_device())
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    flops = (phx.phx_fno_gemm_flops(net) - f0) / args.steps
    pk, pk_kind = peaks()
    tf = flops / (ms * 1e-3) / 1e12
    line = {"metric": "FNO training samples/s", "value": per_step * 8 / (ms * 1e-3),
            "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands, f32 accumulate", "data": "synthetic",
            "config": {"workload": "fno_train", "network": "4 layers, width 32, 16 x 32 modes, "
                       "projection 64, 256 x 256 grid", "batch": 8,
                       "per_step": "%d Adam steps (forward, backward, update)" % per_step,
                       "ms_per_adam_step": ms / per_step},
            "gpu_launches": int(phx.phx_launch_count() - launches0),
            "roofline": {"bound": "tensor", "achieved": tf, "peak": pk["bf16_tflops"],
                         "unit": "TFLOP/s", "frac": tf / pk["bf16_tflops"], "traffic": None,
                         "kernel": "all GEMMs of the step (tcgen05 and mma.sync)",
                         "algorithmic_gflops_per_adam_step": flops / per_step / 1e9,
                         "peak_source": pk_kind + " (bf16 burst)"},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_steady(args, world, rank):
    """--workload steady_256: the warm-start experiment as one JSON line."""
    if rank != 0:
        return
    rep, _ = steady_experiment(args.train, args.test, args.gen_steps, args.epochs, args.cap,
                               time_limit=args.time_limit,
                               log=lambda s: print(s, file=sys.stderr, flush=True))
    s = rep.get("summary") or {}
    line = {"metric": "time to steady state r_psi < 1e-6 (GPU ms, median over held-out pumps)",
            "value": s.get("warm_ms_q", [None] * 3)[1], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": 1, "warmup": 0,
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "steady_256"}, "steady_state": steady_key(rep),
            "report": rep}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        if pg is not None:
            pg.destroy_process_group()
        return

    import torch
    import paper_2411_18341_gb300 as phx
    from paper_2411_18341_gb300 import _build
    _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    if args.workload == "fno_train":
        if rank == 0:
            run_fno_train(args, world, rank, local)
        if pg is not None:
            pg.destroy_process_group()
        return
    if args.workload == "steady_256":
        run_steady(args, world, rank)
        if pg is not None:
            pg.destroy_process_group()
        return
    if args.workload in ("ensemble", "twa_ensemble", "drive_sweep"):
        run_ensemble(args, world, rank, local, pg)
        if pg is not None:
            pg.destroy_process_group()
        return
    wname = workload_name(args)
    cfg, kind, desc = workload(args.workload, seed_offset=rank, grid=args.grid)
    rk4_steps = args.rk4_steps or (RK4_STEPS if args.workload != "conservative_64" else 1000)
    if args.workload == "spinor_2048" and args.rk4_steps is None:
        rk4_steps = 2000
    if args.workload == "driven_9000" and args.rk4_steps is None:
        rk4_steps = 200
    prec = args.precision
    real = torch.float32 if prec == 32 else torch.float64
    cplx = torch.complex64 if prec == 32 else torch.complex128
    d = cfg["params"]
    if args.dt_factor != 1.0:
        if args.integrator != "ssf":
            raise SystemExit("--dt-factor applies to --integrator ssf only")
        d = dict(d, dt=d["dt"] * args.dt_factor, integrator=1)
        cfg = dict(cfg, params=d)
    nx, ny = d["nx"], d["ny"]
    nc = 2 if d["spinor"] else 1
    sites = nx * ny
    stream = torch.cuda.Stream(device=dev)
    h = phx.phx_create(phx.params_from_dict(d, precision=prec, stream=stream.cuda_stream,
                                            tile=args.tile))

    # resident inputs on the device
    psi0_d = torch.tensor(np.ascontiguousarray(cfg["psi0"]), dtype=cplx, device=dev)
    n0_d = None if cfg["n0"] is None else torch.tensor(cfg["n0"], dtype=real, device=dev)
    P_d = None if cfg["P"] is None else torch.tensor(cfg["P"][0], dtype=real, device=dev)
    V_d = None if cfg.get("V") is None else torch.tensor(cfg["V"], dtype=real, device=dev)
    E_d = None if cfg.get("E") is None else torch.tensor(cfg["E"][0], dtype=cplx, device=dev)
    # the copies above run on torch's stream; the handle reads them on its own
    torch.cuda.synchronize()
    if P_d is not None:
        phx.phx_set_pump(h, P_d)
    if V_d is not None:
        phx.phx_set_potential(h, V_d)
    if E_d is not None:
        phx.phx_set_drive(h, E_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    step_fn = phx.phx_step_ssf if args.integrator == "ssf" else phx.phx_step_n

    def one_step(ev_k0=None, ev_k1=None):
        phx.phx_set_state(h, psi0_d, n0_d)
        if ev_k0 is not None:
            ev_k0.record(stream)
        step_fn(h, rk4_steps)
        if ev_k1 is not None:
            ev_k1.record(stream)
        phx.phx_norm_energy(h)
        phx.phx_residual(h)

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(pg)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    launches0 = phx.phx_launch_count()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps (not timed)
        a, b, k0, k1 = ev[k]
        a.record(stream)
        one_step(k0, k1)
        b.record(stream)
    torch.cuda.synchronize()
    launches = phx.phx_launch_count() - launches0
    barrier(pg)
    clk = clocks.stop() if clocks else None
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    kern_ms = [e[2].elapsed_time(e[3]) for e in ev]
    ms, value = aggregate(pg, world, sites * rk4_steps, float(np.mean(step_ms)))

    # end to end through the C ABI with pinned host buffers
    psi_h = torch.tensor(np.ascontiguousarray(cfg["psi0"]), dtype=cplx).pin_memory()
    n_h = None if cfg["n0"] is None else torch.tensor(cfg["n0"], dtype=real).pin_memory()
    P_h = None if cfg["P"] is None else torch.tensor(cfg["P"][0], dtype=real).pin_memory()
    V_h = None if V_d is None else V_d.cpu().pin_memory()
    E_h = None if E_d is None else E_d.cpu().pin_memory()
    del V_d, E_d
    out_psi = torch.empty_like(psi_h).pin_memory()
    out_n = None if n_h is None else torch.empty_like(n_h).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        if P_h is not None:
            phx.phx_set_pump(h, P_h)
        if V_h is not None:
            phx.phx_set_potential(h, V_h)
        if E_h is not None:
            phx.phx_set_drive(h, E_h)
        phx.phx_set_state(h, psi_h, n_h)
        step_fn(h, rk4_steps)
        phx.phx_norm_energy(h)
        phx.phx_residual(h)
        phx.phx_get_state(h, out_psi, out_n)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(pg, (time.perf_counter() - t0) / e2e_steps)
    if prec == 32 and args.no_precision_error:
        prec_err = None
    elif prec == 32:
        fn = "phx_step_ssf" if args.integrator == "ssf" else "phx_step_n"
        psi32, n32 = fresh_run(phx, d, cfg, rk4_steps, stream, dev, fn, 32)
        psi64, n64 = fresh_run(phx, d, cfg, rk4_steps, stream, dev, fn, 64)
        prec_err = precision_error(psi32, n32, psi64, n64,
                                   "final state after %d steps from step 0, both precisions"
                                   % rk4_steps)
        del psi32, n32, psi64, n64
    else:
        prec_err = {"note": "FP64 run: the FP64 path is the yardstick of the FP32 error"}
    esz = 4 if prec == 32 else 8
    h2d = sites * nc * 2 * esz + (0 if n_h is None else sites * nc * esz) + \
        (0 if P_h is None else sites * esz) + (0 if V_h is None else sites * esz) + \
        (0 if E_h is None else sites * 2 * esz)
    d2h = sites * nc * 2 * esz + (0 if n_h is None else sites * nc * esz) + 2 * 8 + 8 * 8

    state_mb = (2 * sites * nc * 2 * esz + (2 * sites * nc * esz if n_h is not None else 0)
                + (sites * esz if P_h is not None else 0) + (sites * esz if V_h is not None else 0)
                + (sites * 2 * esz if E_h is not None else 0)) / 2 ** 20
    if state_mb > 129:
        l2_note = "256 MB buffer written between timed steps; the %.0f MB state is larger than L2" % state_mb
    else:
        l2_note = ("256 MB buffer written between timed steps; the %.0f MB state stays L2-resident "
                   "within a step" % state_mb)
    pk, pk_kind = peaks()
    bps = BYTES_PER_SITE[(prec, kind)]
    kern_s = float(np.mean(kern_ms)) * 1e-3 / rk4_steps
    achieved = bps * sites / kern_s / 1e9
    traffic = recorded_traffic(wname, prec, phx.phx_tile(h))
    if prec == 64 and kind in FLOPS_PER_SITE and args.integrator == "rk4":
        # the FP64 stencil is bound by the FP64 pipe, not by HBM
        tf = FLOPS_PER_SITE[kind] * sites / kern_s / 1e12
        fp64_peak = phx.phx_alu_peak_probe(64)
        roof = {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": tf / fp64_peak, "traffic": traffic,
                "kernel": "rk4_step_generic (FP64)", "algorithmic_flops_per_site": FLOPS_PER_SITE[kind],
                "hbm_gbs_algorithmic": achieved, "avg_launch_us": kern_s * 1e6,
                "peak_source": "measured: phx_alu_peak_probe(64), independent DFMA chains "
                               "timed with CUDA events in this run (nominal from unit counts "
                               "%.2f TFLOP/s)" % FP64_NOMINAL_TFLOPS}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                "traffic": traffic,
                "kernel": ("split-step (local kernels + cuFFT round trip per step)"
                           if args.integrator == "ssf" else step_kernel_name(phx.phx_tile(h))),
                "algorithmic_bytes_per_site": bps,
                "avg_launch_us": kern_s * 1e6,
                "peak_source": pk_kind}
        if args.integrator == "ssf":
            roof["note"] = ("split-step: the FFT round trip re-reads the state several times per "
                            "step; traffic is not the fused kernel's")
            roof["traffic"] = None
        elif d.get("noise_var", 0) > 0 or d.get("wigner_nu", 0) > 0:
            roof["note"] = ("per-site Philox + Box-Muller noise every step: the kernel is bound by "
                            "instruction issue, not by HBM")
        elif sites * bps < 129e6:
            roof["note"] = "state smaller than L2: bound by instruction issue and latency, not by HBM"
    line = {
        "metric": "RK4 site-updates/s",
        "value": value, "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == 32 else "f64", "data": "synthetic",
        "config": {"workload": wname, "description": desc,
                   "grid": "%dx%d" % (nx, ny), "rk4_steps_per_step": rk4_steps,
                   "per_step": "set_state + %d %s + FP64 norm/energy + FP64 residual" % (
                       rk4_steps, "split-step Fourier steps" if args.integrator == "ssf"
                       else "fused RK4 steps"),
                   "l2": l2_note,
                   "tile": phx.phx_tile(h), "integrator": args.integrator,
                   "dt_ps": d["dt"],
                   "simulated_ps_per_s": d["dt"] * rk4_steps / (ms * 1e-3),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": world * sites * rk4_steps / e2e_s, "unit": "site-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk,
        "energy": energy(clk, ms * 1e-3, sites * rk4_steps),
        "precision_error": prec_err,
    }
    if rank == 0 and world == 1 and args.workload == "reservoir_2048":
        # the two-component TE-TM workload's step (noise every step), timed briefly
        line["spinor_2048"] = quick_rate(phx, torch, "spinor_2048")
        # the same workload with a coherent drive on top (reservoir + drive
        # variant of the TMA-fed kernel)
        n = d["nx"]
        xx = np.arange(n)[None, :] / n
        yy = np.arange(n)[:, None] / n
        E = (0.05 * np.exp(2j * np.pi * (3 * xx + 2 * yy))).astype(np.complex64)
        line["drive_reservoir_2048"] = quick_rate(phx, torch, "reservoir_2048", drive=(E, -0.3))
    if rank == 0 and world == 1 and not args.no_steady and args.workload == "reservoir_2048":
        # reduced warm-vs-cold time to steady state (the metric's second part)
        rep, _ = steady_experiment(n_train=1024, n_test=128, gen_steps=30000, epochs=12,
                                   cap=60000, time_limit=120)
        line["steady_state"] = dict(steady_key(rep), reduced=(
            "1024 training / 128 held-out pumps, 12 epochs, cap 6e4 steps; the full "
            "experiment is --workload steady_256"))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if sites > 1 << 24:
            import synth
            line["cpu_baseline"] = cpu_baseline(wname + " (512x512 corner window)",
                                                synth.crop(cfg, 512))
        else:
            line["cpu_baseline"] = cpu_baseline(wname, cfg)
    phx.phx_destroy(h)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
