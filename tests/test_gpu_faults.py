"""Failure detection without faulting the GPU: host-side injected allocation
and launch failures, and a device-side bounded wait that is made to run out
(an mbarrier nothing arms).  The handle must stay usable afterwards."""
import numpy as np
import pytest

from oracle import gp
import synth
from gpu_util import phx, make_handle, get_state, rel_l2, rounded

pytestmark = pytest.mark.gpu


def small_case():
    d = synth.base_params(150, 90, 15.0, 9.0, g=0.3, dt=0.0, **{
        k: v for k, v in synth.reservoir_physics().items() if k != "g"})
    d["dt"] = 0.4 * gp.stability_dt_max(gp.Params(**d))
    psi0, n0, P, V = synth.random_state(1, 90, 150, 3, amp=0.5, smooth=True)
    return d, rounded(psi0, 32), rounded(n0, 32), rounded(P, 32)


def test_injected_alloc_failure():
    m = phx()
    d, psi0, n0, P = small_case()
    m.phx_debug_inject(m.INJECT_ALLOC)
    with pytest.raises(m.PhxError) as e:
        m.phx_create(m.params_from_dict(d, precision=32))
    assert e.value.status == 2
    h = make_handle(d, 32, psi0, n0, P)  # next create succeeds
    m.phx_step_n(h, 2)


def test_injected_launch_failure_keeps_state():
    m = phx()
    d, psi0, n0, P = small_case()
    h = make_handle(d, 32, psi0, n0, P)
    m.phx_debug_inject(m.INJECT_LAUNCH)
    with pytest.raises(m.PhxError) as e:
        m.phx_step_n(h, 3)
    assert e.value.status == 3
    assert m.phx_time(h)[0] == 0
    m.phx_step_n(h, 4)
    g_psi, g_n = get_state(h, 32)
    o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 4)
    assert rel_l2(g_psi, o_psi) <= 1e-4


def test_bounded_wait_timeout_reported_and_recoverable():
    m = phx()
    d, psi0, n0, P = small_case()
    h = make_handle(d, 32, psi0, n0, P)
    m.phx_debug_inject(m.INJECT_TIMEOUT)
    m.phx_step_n(h, 1)
    with pytest.raises(m.PhxError) as e:
        m.phx_norm_energy(h)
    assert e.value.status == 5
    # the context is intact: reset the state and the handle computes again
    m.phx_set_state(h, np.ascontiguousarray(psi0, np.complex64),
                    np.ascontiguousarray(n0, np.float32))
    m.phx_set_time(h, 0, 0.0)
    m.phx_step_n(h, 5)
    g_psi, g_n = get_state(h, 32)
    o_psi, o_n = gp.run(psi0, n0, P, None, gp.Params(**d), 5)
    assert rel_l2(g_psi, o_psi) <= 1e-4
    assert rel_l2(g_n, o_n) <= 1e-4
