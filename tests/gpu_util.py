"""Helpers for the GPU parity tests: run the C-ABI path on numpy inputs."""
import numpy as np

import __graft_entry__

_built = False


def phx():
    global _built
    if not _built:
        __graft_entry__.build()
        _built = True
    import paper_2411_18341_gb300 as m
    return m


def types(prec):
    return (np.float64, np.complex128) if prec == 64 else (np.float32, np.complex64)


def rounded(a, prec):
    """Inputs as the GPU sees them (rounded to the stencil precision), in FP64."""
    if a is None:
        return None
    real, cplx = types(prec)
    return np.asarray(a).astype(cplx if np.iscomplexobj(a) else real).astype(
        np.complex128 if np.iscomplexobj(a) else np.float64)


def make_handle(d, prec, psi0, n0=None, P=None, V=None, stream=None):
    m = phx()
    real, cplx = types(prec)
    h = m.phx_create(m.params_from_dict(d, precision=prec, stream=stream))
    if d.get("reservoir") and P is not None:
        P = np.asarray(P)
        if P.shape[0] == 2:
            m.phx_set_pump(h, np.ascontiguousarray(P[0], real), np.ascontiguousarray(P[1], real))
        else:
            m.phx_set_pump(h, np.ascontiguousarray(P[0], real))
    if V is not None:
        m.phx_set_potential(h, np.ascontiguousarray(V, real))
    m.phx_set_state(h, np.ascontiguousarray(psi0, cplx),
                    None if n0 is None else np.ascontiguousarray(n0, real))
    return h


def get_state(h, prec):
    m = phx()
    real, cplx = types(prec)
    psi = np.empty((h.ncomp, h.ny, h.nx), cplx)
    n = np.empty((h.ncomp, h.ny, h.nx), real) if h.reservoir else None
    m.phx_get_state(h, psi, n)
    return psi, n


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


TOL = {64: 1e-11, 32: 1e-4}


# FP32 scalar step configurations of the TMA-fed persistent kernel
TMA_SCALAR_TILES = [1, 2, 3, 4, 5, 6, 7]


def tma_scalar(tile):
    return tile in TMA_SCALAR_TILES
