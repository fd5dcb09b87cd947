"""Writes synth/constants.json: time steps at half the RK4 stability limit
and the pump threshold, computed by the oracle only (oracle.gp).

Run from the repository root:  python synth/derive_constants.py
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import gp  # noqa: E402

KAPPA = 0.67


def half_limit(**kw):
    p = gp.Params(**kw)
    return 0.5 * gp.stability_dt_max(p)


def main():
    out = {"note": "written by synth/derive_constants.py from oracle.gp; "
                   "dt = 0.5 * 2 sqrt(2) hbar / lambda_max (0.85 for steady_256)"}
    res = dict(reservoir=True, g=6e-3, g_r=1.2e-2, R=0.01, gamma_c=0.15,
               gamma_r=0.225, kappa=KAPPA)
    out["pump_threshold"] = gp.pump_threshold(gp.Params(nx=1, ny=1, lx=1, ly=1, **res))
    out["conservative_64"] = {"dt": half_limit(nx=64, ny=64, lx=20.0, ly=20.0,
                                               kappa=KAPPA, g=6e-3)}
    for n in (16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192):
        out["reservoir_%d_L100" % n] = {"dt": half_limit(nx=n, ny=n, lx=100.0,
                                                         ly=100.0, **res)}
    # config-2 physics at 2048^2 with config 2's cell size (200 um box)
    out["reservoir_2048_L200"] = {"dt": half_limit(nx=2048, ny=2048, lx=200.0, ly=200.0, **res)}
    for n, L in ((2048, 200.0), (512, 50.0), (64, 6.25), (96, 9.375)):
        out["spinor_%d_L%g" % (n, L)] = {"dt": half_limit(
            nx=n, ny=n, lx=L, ly=L, spinor=True, delta_lt=0.025, **res)}
    # Steady-state workload: dt at 0.85 of the limit.  RK4 damps the band
    # |lambda| dt ~ 1 (|R(i y)|^2 = 1 - y^6/72 + y^8/576); at 0.85 that damping
    # exceeds the reservoir gain for the zero-group-velocity lattice modes at
    # the (pi/dx, 0) saddles of the 5-point dispersion, which at 0.5 out-grow
    # the k ~ 0 condensate.  The stationary state does not depend on dt.
    dmax = 2 * half_limit(nx=256, ny=256, lx=128.0, ly=128.0, **res)
    out["steady_256_L128"] = {"dt": 0.85 * dmax, "dt_max": dmax}
    # truncated-Wigner ensemble: 256^2 over 200 um, half the limit
    out["twa_256_L200"] = {"dt": half_limit(nx=256, ny=256, lx=200.0, ly=200.0, **res)}
    # driven lattice: 9000^2 cells of 0.1 um, scalar with loss and g
    out["driven_9000_L900"] = {"dt": half_limit(nx=9000, ny=9000, lx=900.0, ly=900.0,
                                                kappa=KAPPA, g=6e-3, gamma_c=0.15)}
    # drive-frequency sweep: 512^2 over 100 um, scalar with loss and g
    out["drive_512_L100"] = {"dt": half_limit(nx=512, ny=512, lx=100.0, ly=100.0,
                                              kappa=KAPPA, g=6e-3, gamma_c=0.15)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "constants.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
