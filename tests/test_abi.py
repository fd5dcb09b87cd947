"""C-ABI library: loads, exports every symbol include/phx.h declares, and its
host-only logic (parameter validation, stability limit) agrees with the
oracle.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from oracle import gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def phx():
    __graft_entry__.build()
    import paper_2411_18341_gb300 as m
    return m


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        names += re.findall(r"\b(phx_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_boundary(phx):
    names = declared_functions()
    for must in ("phx_create", "phx_set_pump", "phx_step_n", "phx_norm_energy",
                 "phx_destroy", "phx_residual", "phx_set_state", "phx_get_state"):
        assert must in names


def test_library_exports_every_declared_symbol(phx):
    L = ctypes.CDLL(phx.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_params_struct_layout_matches_c(phx):
    p = phx.phx_params_init()
    assert p.struct_size == ctypes.sizeof(phx.phx_params)
    assert p.nx == 64 and p.precision == 32 and p.hbar2_over_2m == 0.67


CASES = [
    dict(nx=64, ny=64, lx=20.0, ly=20.0),
    dict(nx=37, ny=29, lx=11.1, ly=8.7, bc_x=1),
    dict(nx=10, ny=12, lx=3.0, ly=3.3, bc_x=1, bc_y=1),
    dict(nx=33, ny=16, lx=5.0, ly=4.0, spinor=True, delta_lt=0.4),
    dict(nx=24, ny=24, lx=6.0, ly=6.0, spinor=True, delta_lt=0.025, bc_y=1),
    dict(nx=2048, ny=2048, lx=200.0, ly=200.0, spinor=True, delta_lt=0.025),
]


@pytest.mark.parametrize("case", CASES)
def test_stability_dt_matches_oracle(phx, case):
    p = gp.Params(**case)
    kw = dict(case)
    kw["spinor"] = int(kw.get("spinor", False))
    got = phx.phx_stability_dt(phx.phx_params_init(**kw))
    assert abs(got - gp.stability_dt_max(p)) <= 1e-12 * got


def test_invalid_params_rejected_before_device(phx):
    bad = [dict(nx=0), dict(ny=-3), dict(lx=0.0), dict(bc_x=2), dict(precision=16),
           dict(g_x=0.1), dict(delta_lt=0.1), dict(noise_var=-1.0),
           dict(wigner_nu=-0.5), dict(wigner_nu=float("inf")),
           dict(dt=0.0), dict(dt=1.0), dict(g=float("nan")), dict(spinor=2)]
    for kw in bad:
        base = dict(nx=16, ny=16, lx=4.0, ly=4.0, dt=1e-3)
        base.update(kw)
        with pytest.raises(phx.PhxError) as e:
            phx.phx_create(phx.phx_params_init(**base))
        assert e.value.status == 1, (kw, e.value)


def test_integrator_limits_checked_before_device(phx):
    """dt above the RK4 limit: rejected (EINVAL) for the RK4 integrator,
    accepted by validation for the split-step integrator (then ENODEV on a
    machine without a GB300, PHX_OK with one); the split-step integrator
    refuses zero boundaries, truncated-Wigner noise, a reservoir time step
    beyond its local RK4 half step, and unknown integrator codes."""
    base = dict(nx=16, ny=16, lx=4.0, ly=4.0)
    lim = phx.phx_stability_dt(phx.phx_params_init(**base, dt=1e-3))
    with pytest.raises(phx.PhxError) as e:
        phx.phx_create(phx.phx_params_init(**base, dt=5 * lim))
    assert e.value.status == 1
    try:
        h = phx.phx_create(phx.phx_params_init(**base, dt=5 * lim, integrator=1))
        phx.phx_destroy(h)
    except phx.PhxError as err:
        assert err.status == 7, err  # ENODEV: validation passed
    for kw in (dict(bc_x=1), dict(wigner_nu=1.0),
               dict(reservoir=1, gamma_r=1.0, dt=6.0), dict(integrator=2)):
        q = dict(base, dt=5 * lim, integrator=1)
        q.update(kw)
        with pytest.raises(phx.PhxError) as e:
            phx.phx_create(phx.phx_params_init(**q))
        assert e.value.status == 1, kw


def test_struct_size_checked(phx):
    p = phx.phx_params_init(dt=1e-3)
    p.struct_size = 8
    with pytest.raises(phx.PhxError) as e:
        phx.phx_create(p)
    assert e.value.status == 1


def test_status_strings(phx):
    L = phx.lib()
    assert L.phx_status_string(0) == b"PHX_OK"
    assert L.phx_status_string(5) == b"PHX_ETIMEOUT"
    assert L.phx_last_error(None)


def test_fno_config_struct_layout_matches_c(phx):
    """phx_fno_config_init fills the binding's struct: size and defaults agree
    (256 x 256, C = 32, 4 layers, 16 x 32 modes, P = 64)."""
    c = phx.phx_fno_config()
    assert phx.lib().phx_fno_config_init(ctypes.byref(c)) == 0
    assert c.struct_size == ctypes.sizeof(phx.phx_fno_config)
    assert (c.height, c.width, c.channels, c.layers, c.modes_x, c.modes_y) == (256, 256, 32, 4, 16, 32)
    assert (c.in_channels, c.out_channels, c.proj_hidden, c.max_batch) == (3, 3, 64, 8)


def test_fno_invalid_config_rejected_before_device(phx):
    c = phx.phx_fno_config()
    phx.lib().phx_fno_config_init(ctypes.byref(c))
    c.modes_y = 3  # must be even
    out = ctypes.c_void_p()
    assert phx.lib().phx_fno_create(ctypes.byref(c), ctypes.byref(out)) == 1  # PHX_EINVAL
    assert not out.value


def test_buffer_sizes_are_the_padded_layout(phx):
    """Caller-owned state buffers: psi is ncomp planes of (ny + 8) rows x
    pitch complex elements, pitch = nx + 8 rounded up to 32; n and P are
    real planes, absent without reservoir (host-only call)."""
    for kw, es, nc, res in [(dict(nx=100, ny=37, lx=10.0, ly=3.7), 4, 1, False),
                            (dict(nx=64, ny=64, lx=5.0, ly=5.0, precision=64, reservoir=1), 8, 1, True),
                            (dict(nx=33, ny=9, lx=3.3, ly=0.9, spinor=1, reservoir=1), 4, 2, True)]:
        kw = dict(kw, dt=1e-4)
        sizes = phx.phx_buffer_sizes(phx.phx_params_init(**kw))
        pitch = -(-(kw["nx"] + 8) // 32) * 32
        plane = pitch * (kw["ny"] + 8)
        assert sizes[0] == sizes[1] == nc * plane * 2 * es
        assert sizes[2] == sizes[3] == sizes[4] == (nc * plane * es if res else 0)
    with pytest.raises(phx.PhxError) as e:
        phx.phx_buffer_sizes(phx.phx_params_init(nx=0))
    assert e.value.status == 1


C_CLIENT = r"""
#include <stdio.h>
#include "phx.h"
int main(void) {
  phx_params p;
  double dt = 0.0;
  size_t sizes[5];
  if (phx_params_init(&p) != PHX_OK) return 1;
  p.nx = 128; p.ny = 96; p.lx = 40.0; p.ly = 30.0;
  if (phx_stability_dt(&p, &dt) != PHX_OK) return 2;
  p.dt = 0.5 * dt;
  if (phx_buffer_sizes(&p, sizes) != PHX_OK) return 3;
  p.nx = 0;
  if (phx_stability_dt(&p, &dt) != PHX_EINVAL) return 4;
  printf("%.17g %lu\n", 2.0 * p.dt, (unsigned long)sizes[0]);
  return 0;
}
"""


def test_plain_c_client_compiles_links_and_runs(phx, tmp_path):
    """The boundary is a C ABI: a strict C99 program (-pedantic -Werror)
    includes the header, links the shared library and calls its host-only
    entry points, which agree with the oracle."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    lib_dir = os.path.dirname(phx.LIB_PATH)
    exe = tmp_path / "client"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), str(src), "-L", lib_dir, "-lphx",
                        "-Wl,-rpath," + lib_dir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.returncode
    dt, size0 = out.stdout.split()
    want = gp.stability_dt_max(gp.Params(nx=128, ny=96, lx=40.0, ly=30.0))
    assert abs(float(dt) - want) <= 1e-12 * want
    pitch = -(-(128 + 8) // 32) * 32
    assert int(size0) == pitch * (96 + 8) * 8
