"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle-driven
checks.  It holds none of the method's arithmetic: only grids, pump and
initial-state profiles, random draws and parameter tables.  Two derived
numbers per workload (the time step at half the RK4 stability limit and the
pump threshold) are read from ``constants.json``, which
``synth/derive_constants.py`` writes by calling the oracle.

Workloads (sizes and physics as stated for each; the paper's own parameter
files are not available, so these stand in for them):

* ``conservative_64``  -- scalar Eq. (1) without loss, 64x64, 20 um, periodic,
  psi0 = 5 exp(-r^2/3^2) + complex normal noise (std 1e-2 per quadrature).
* ``reservoir_1024``   -- scalar + reservoir, 1024x1024, 100 um, periodic, ring
  pump of radius 20 um and width 3 um at 1.5 P_thr, psi0 = noise, n0 = 0.
* ``reservoir_2048``   -- the same physics, cell size and time step on
  2048x2048 over 200 um.
* ``spinor_2048``      -- TE-TM spinor + reservoir, 2048x2048, 200 um, Gaussian
  pump of waist 10 um at 1.5 P_thr on both components, per-step noise.
* ``ensemble``         -- 256 reservoir instances, 64 each at 128^2 .. 1024^2,
  100 um, ring pumps at U[0.8, 3] P_thr.
* ``steady_256``       -- 256x256, 128 um, sums of 1-4 Gaussian pumps.
* ``drive_sweep``      -- 64 coherently driven scalar fields, 512x512, 100 um,
  the same drive spot at 64 frequencies (one batch).
"""
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))

PERIODIC = 0
ZERO = 1

# Shared physical parameters of the driven-dissipative workloads
# (meV um^2 for kappa, g, g_r, delta_lt; ps^-1 um^2 for R; ps^-1 for rates).
KAPPA = 0.67
G_C = 6e-3
G_R = 2 * G_C
R_GAIN = 0.01
GAMMA_C = 0.15
GAMMA_R = 1.5 * GAMMA_C


def load_constants():
    with open(os.path.join(_HERE, "constants.json")) as f:
        return json.load(f)


def coords(n, length):
    """Cell positions -L/2 + i*L/n (origin at the grid centre)."""
    return -0.5 * length + np.arange(n) * (length / n)


def mesh(nx, ny, lx, ly):
    x = coords(nx, lx)
    y = coords(ny, ly)
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]


def gaussian(nx, ny, lx, ly, amp, w, cx=0.0, cy=0.0):
    X, Y = mesh(nx, ny, lx, ly)
    return amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / w ** 2)


def ring(nx, ny, lx, ly, amp, radius, width):
    X, Y = mesh(nx, ny, lx, ly)
    r = np.sqrt(X ** 2 + Y ** 2)
    return amp * np.exp(-((r - radius) ** 2) / width ** 2)


def complex_normal(shape, std, seed):
    """Complex normal field, std per quadrature, numpy PCG64 stream `seed`."""
    rng = np.random.default_rng(seed)
    re = rng.normal(0.0, std, shape)
    im = rng.normal(0.0, std, shape)
    return re + 1j * im


def base_params(nx, ny, lx, ly, **kw):
    p = dict(nx=nx, ny=ny, lx=lx, ly=ly, bc_x=PERIODIC, bc_y=PERIODIC,
             spinor=False, reservoir=False, kappa=KAPPA, g=0.0, g_x=0.0,
             g_r=0.0, R=0.0, gamma_c=0.0, gamma_r=0.0, delta_lt=0.0, dt=0.0,
             noise_var=0.0, seed=0)
    p.update(kw)
    return p


def reservoir_physics():
    return dict(reservoir=True, g=G_C, g_r=G_R, R=R_GAIN, gamma_c=GAMMA_C,
                gamma_r=GAMMA_R)


def conservative_64(seed=1):
    c = load_constants()["conservative_64"]
    p = base_params(64, 64, 20.0, 20.0, g=6e-3, dt=c["dt"])
    psi0 = (gaussian(64, 64, 20.0, 20.0, 5.0, 3.0)
            + complex_normal((64, 64), 1e-2, seed))[None]
    return dict(name="conservative_64", params=p, psi0=psi0, n0=None, P=None,
                V=None, steps=1000)


def reservoir_grid(n, length=100.0, pump_factor=1.5, seed=2, dt=None,
                   const_key=None):
    """Scalar driven-dissipative GP + reservoir with the ring pump."""
    c = load_constants()
    key = const_key or ("reservoir_%d_L%g" % (n, length))
    if dt is None:
        dt = c[key]["dt"]
    pthr = c["pump_threshold"]
    p = base_params(n, n, length, length, dt=dt, **reservoir_physics())
    P = ring(n, n, length, length, pump_factor * pthr, 20.0, 3.0)[None]
    psi0 = complex_normal((1, n, n), 1e-2, seed)
    n0 = np.zeros((1, n, n))
    return dict(name="reservoir_%d" % n, params=p, psi0=psi0, n0=n0, P=P,
                V=None, steps=10000)


def reservoir_1024(seed=2):
    return reservoir_grid(1024, seed=seed, const_key="reservoir_1024_L100")


def reservoir_2048(seed=2):
    """The reservoir workload's physics, cell size (100/1024 um) and time step
    on a 2048^2 grid over 200 um (ring pump radius 20 um, width 3 um)."""
    cfg = reservoir_grid(2048, length=200.0, seed=seed, const_key="reservoir_2048_L200")
    cfg["name"] = "reservoir_2048"
    return cfg


def spinor_grid(n, length=200.0, seed=3, const_key=None):
    """TE-TM spinor + reservoir, Gaussian pump waist 10 um at 1.5 P_thr."""
    c = load_constants()
    key = const_key or ("spinor_%d_L%g" % (n, length))
    pthr = c["pump_threshold"]
    p = base_params(n, n, length, length, spinor=True, delta_lt=0.025,
                    noise_var=1e-3, seed=seed, dt=c[key]["dt"],
                    **reservoir_physics())
    P = gaussian(n, n, length, length, 1.5 * pthr, 10.0)[None]
    psi0 = complex_normal((2, n, n), 1e-2, seed)
    n0 = np.zeros((2, n, n))
    return dict(name="spinor_%d" % n, params=p, psi0=psi0, n0=n0, P=P, V=None,
                steps=20000)


def spinor_2048(seed=3):
    return spinor_grid(2048, const_key="spinor_2048_L200")


def ensemble(count_per_size=64, sizes=(128, 256, 512, 1024), seed0=1000):
    """Uneven-grid ensemble: pump peaks ~ U[0.8, 3] P_thr, seeds seed0+i."""
    c = load_constants()
    pthr = c["pump_threshold"]
    rng = np.random.default_rng(seed0 - 1)
    out = []
    i = 0
    for n in sizes:
        for _ in range(count_per_size):
            factor = float(rng.uniform(0.8, 3.0))
            p = base_params(n, n, 100.0, 100.0,
                            dt=c["reservoir_%d_L100" % n]["dt"],
                            **reservoir_physics())
            P = ring(n, n, 100.0, 100.0, factor * pthr, 20.0, 3.0)[None]
            psi0 = complex_normal((1, n, n), 1e-2, seed0 + i)
            out.append(dict(name="ens_%d" % i, params=p, psi0=psi0,
                            n0=np.zeros((1, n, n)), P=P, V=None, steps=5000,
                            pump_factor=factor))
            i += 1
    return out


def super_gaussian(nx, ny, lx, ly, amp, w):
    """amp * exp(-(r/w)^4): the flat-top pump of the truncated-Wigner example,
    with the printed exponent r^4/w_p^2 read as (r^2/w_p^2)^2 so that w_p is
    the width in um."""
    X, Y = mesh(nx, ny, lx, ly)
    r2 = (X ** 2 + Y ** 2) / w ** 2
    return amp * np.exp(-r2 * r2)


def twa_ensemble(count=150, n=256, length=200.0, pump_factor=2.0, nu=1.0, seed=7,
                 width=65.0):
    """Truncated-Wigner Monte-Carlo ensemble: `count` realisations of one
    scalar reservoir problem (super-Gaussian pump of width 65 um at
    pump_factor P_thr, noise intensity nu), one Philox seed, member i drawing
    counter word `instance` = i.  Each starts from the Wigner vacuum:
    complex normal psi with E|psi|^2 = 1/(2 dV) per site, n = 0."""
    c = load_constants()
    pthr = c["pump_threshold"]
    dt = c["twa_%d_L%g" % (n, length)]["dt"]
    P = super_gaussian(n, n, length, length, pump_factor * pthr, width)[None]
    dv = (length / n) ** 2
    out = []
    for i in range(count):
        p = base_params(n, n, length, length, dt=dt, wigner_nu=nu, seed=seed,
                        instance=i, **reservoir_physics())
        psi0 = complex_normal((1, n, n), 0.5 / np.sqrt(dv), seed * 100003 + i)
        out.append(dict(name="twa_%d" % i, params=p, psi0=psi0,
                        n0=np.zeros((1, n, n)), P=P, V=None, steps=None))
    return out


def driven_lattice(n=9000, dx=0.1, seed=11, wells=272, a1=2.8, a2=3.8, depth=4.0,
                   width=1.2, aah=0.2, e0=5.6856e-3, omega=-5.6883, spot=10.0):
    """Coherently driven potential lattice with the shapes of the paper's
    topological corner-state example (9000^2 grid, 272^2 wells, resonant
    drive omega = -5.6883 ps^-1, E0 = 5.6856 ueV); its own parameters are not
    available, so these stand in: an SSH lattice (alternating spacings a1, a2
    um) of super-Gaussian wells -depth exp(-(r/width)^4) meV whose depths
    carry an Aubry-Andre-Harper modulation 1 + aah cos(2 pi beta (i + j)),
    beta the golden ratio's fractional part, and a Gaussian drive spot of
    waist `spot` um on the corner well.  Scalar, no reservoir, loss
    gamma_c = 0.15 ps^-1, g = 6e-3 meV um^2, periodic."""
    c = load_constants()
    length = n * dx
    p = base_params(n, n, length, length, g=G_C, gamma_c=GAMMA_C,
                    dt=c["driven_%d_L%g" % (n, length)]["dt"], drive_omega=omega)
    gaps = np.where(np.arange(wells - 1) % 2 == 0, a1, a2)
    pos = np.concatenate([[0.0], np.cumsum(gaps)])
    pos = pos - 0.5 * pos[-1]                  # lattice centred in the box
    x = coords(n, length)
    k = np.clip(np.searchsorted(pos, x), 1, wells - 1)
    near = np.where(np.abs(x - pos[k - 1]) < np.abs(x - pos[k]), k - 1, k)
    d = x - pos[near]                          # distance to the nearest well per axis
    beta = 0.5 * (np.sqrt(5.0) - 1.0)
    amp = depth * (1.0 + aah * np.cos(2 * np.pi * beta * (near[:, None] + near[None, :])))
    r2 = (d[:, None] ** 2 + d[None, :] ** 2) / width ** 2
    V = (-amp * np.exp(-r2 * r2)).astype(np.float32)
    del r2, amp
    E = gaussian(n, n, length, length, e0, spot, pos[0], pos[0]).astype(np.complex64)[None]
    psi0 = complex_normal((1, n, n), 1e-3, seed).astype(np.complex64)
    return dict(name="driven_%d" % n, params=p, psi0=psi0, n0=None, P=None, V=V, E=E,
                steps=None)


def drive_sweep(count=64, n=512, length=100.0, seed0=3000, omega_lo=-1.0, omega_hi=2.0,
                e0=0.05, spot=20.0):
    """Drive-frequency sweep of a coherently driven scalar field (the scan
    that maps a driven condensate's response against detuning): `count`
    members on n x n grids over `length` um, periodic, Kerr g = 6e-3 meV um^2,
    loss gamma_c = 0.15 ps^-1, no reservoir; member i is driven by the same
    Gaussian spot (amplitude e0 meV, waist `spot` um, centred) at frequency
    omega_i, evenly spaced over [omega_lo, omega_hi] ps^-1; psi0 = complex
    normal noise of std 1e-3, seed seed0 + i."""
    c = load_constants()
    E = gaussian(n, n, length, length, e0, spot).astype(np.complex64)[None]
    out = []
    for i, om in enumerate(np.linspace(omega_lo, omega_hi, count)):
        p = base_params(n, n, length, length, g=G_C, gamma_c=GAMMA_C,
                        dt=c["drive_%d_L%g" % (n, length)]["dt"], drive_omega=float(om),
                        seed=seed0 + i, instance=i)
        psi0 = complex_normal((1, n, n), 1e-3, seed0 + i).astype(np.complex64)
        out.append(dict(name="sweep_%d" % i, params=p, psi0=psi0, n0=None, P=None, V=None,
                        E=E, steps=None))
    return out


def crop(cfg, m):
    """The m x m corner window of a workload (same cell size and physics,
    periodic over the window): a bounded sample for CPU timing."""
    d = dict(cfg["params"])
    dx, dy = d["lx"] / d["nx"], d["ly"] / d["ny"]
    d.update(nx=m, ny=m, lx=m * dx, ly=m * dy)
    win = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a)[..., :m, :m])
    return dict(cfg, params=d, psi0=win(cfg["psi0"]), n0=win(cfg["n0"]), P=win(cfg["P"]),
                V=win(cfg.get("V")), E=win(cfg.get("E")))


def random_gaussian_pumps(n=256, length=128.0, count=1, seed=5000, threshold=None):
    """count pump images, each a sum of 1-4 Gaussians exp(-|r-c|^2/w^2) with
    w ~ U[3, 15] um, peak ~ U[1, 3] x threshold(w), centres within L/2 - 2w.
    threshold: callable waist -> threshold pump peak of a spot of that waist
    (supplied by the caller, e.g. measured with the solver); default the
    homogeneous P_thr for every waist."""
    pthr = load_constants()["pump_threshold"]
    if threshold is None:
        threshold = lambda w: pthr  # noqa: E731
    imgs = np.empty((count, n, n))
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        m = int(rng.integers(1, 5))
        img = np.zeros((n, n))
        for _ in range(m):
            w = float(rng.uniform(3.0, 15.0))
            amp = float(rng.uniform(1.0, 3.0)) * float(threshold(w))
            lim = 0.5 * length - 2.0 * w
            cx, cy = rng.uniform(-lim, lim, size=2)
            img += gaussian(n, n, length, length, amp, w, cx, cy)
        imgs[k] = img
    return imgs


def steady_256(seed=5000):
    c = load_constants()["steady_256_L128"]
    p = base_params(256, 256, 128.0, 128.0, dt=c["dt"], **reservoir_physics())
    P = random_gaussian_pumps(256, 128.0, 1, seed)[:, None][0]
    psi0 = complex_normal((1, 256, 256), 1e-2, seed)
    return dict(name="steady_256", params=p, psi0=psi0,
                n0=np.zeros((1, 256, 256)), P=P, V=None, steps=200000)


def random_state(ncomp, ny, nx, seed, amp=1.0, reservoir=True, smooth=False):
    """Generic random test state: psi (complex), n >= 0, P >= 0, V."""
    rng = np.random.default_rng(seed)
    psi = amp * (rng.normal(size=(ncomp, ny, nx)) + 1j * rng.normal(size=(ncomp, ny, nx)))
    if smooth:
        # smooth by repeated neighbour averaging (periodic) -- a pure input
        # shaping step, not part of the method
        for _ in range(6):
            psi = 0.2 * (psi + np.roll(psi, 1, -1) + np.roll(psi, -1, -1)
                         + np.roll(psi, 1, -2) + np.roll(psi, -1, -2))
    n = rng.uniform(0.0, 2.0, size=(ncomp, ny, nx)) if reservoir else None
    P = rng.uniform(0.0, 5.0, size=(ncomp, ny, nx)) if reservoir else None
    V = rng.uniform(-1.0, 1.0, size=(ny, nx))
    return psi, n, P, V


# ------------------------------------------------------------ FNO inputs

FNO_SCALE_PSI = 5.0    # output normalisation of Re/Im psi (|psi| ~ 5 at 1-3 P_thr)
FNO_SCALE_N = 15.0     # output normalisation of n (n ~ gamma_c / R = 15)


def fno_init_weights(shapes, seed=0, channels=32):
    """Seeded initial parameters for the flat layout given by `shapes`
    [(name, shape), ...]: spectral weights ~ U[0, 1/(C*C)) (Li et al.),
    dense weights ~ U[-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in shapes:
        n = int(np.prod(shape))
        if name.startswith("R"):
            parts.append(rng.uniform(0.0, 1.0 / (channels * channels), n))
        elif len(shape) == 2:
            bound = 1.0 / np.sqrt(shape[0])
            parts.append(rng.uniform(-bound, bound, n))
        else:
            parts.append(np.zeros(n))
    return np.concatenate(parts).astype(np.float32)


def fno_features(P, length, pump_threshold):
    """Network input [B, H, W, 3]: (P / P_thr, x / (L/2), y / (L/2))."""
    P = np.asarray(P, np.float64)
    if P.ndim == 2:
        P = P[None]
    B, H, W = P.shape
    X, Y = mesh(W, H, length, length)
    a = np.empty((B, H, W, 3), np.float32)
    a[..., 0] = P / pump_threshold
    a[..., 1] = X / (0.5 * length)
    a[..., 2] = Y / (0.5 * length)
    return a


def fno_targets(psi, n):
    """Target [B, H, W, 3] = (Re psi, Im psi, n) scaled, with the global phase
    removed (psi multiplied by exp(-i arg sum psi))."""
    psi = np.asarray(psi)
    if psi.ndim == 2:
        psi = psi[None]
        n = np.asarray(n)[None]
    out = np.empty(psi.shape + (3,), np.float32)
    for b in range(psi.shape[0]):
        s = psi[b].sum()
        ph = np.exp(-1j * np.angle(s)) if abs(s) > 0 else 1.0
        q = psi[b] * ph
        out[b, ..., 0] = q.real / FNO_SCALE_PSI
        out[b, ..., 1] = q.imag / FNO_SCALE_PSI
        out[b, ..., 2] = np.asarray(n[b]) / FNO_SCALE_N
    return out


def fno_state_from_output(u):
    """Inverse of fno_targets for one sample [H, W, 3] -> (psi, n)."""
    u = np.asarray(u, np.float64)
    return (u[..., 0] + 1j * u[..., 1]) * FNO_SCALE_PSI, u[..., 2] * FNO_SCALE_N
