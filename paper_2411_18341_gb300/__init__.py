"""GB300 RK4 solver for the 2D driven-dissipative Gross-Pitaevskii / dNLSE
(PHOENIX, arXiv 2411.18341): Python binding of the C ABI in include/phx.h.

The binding only marshals arguments: every step of the computation runs in
the CUDA kernels of ``_build/libphx.so``.  Importing works without a GPU (the
library loads; nothing is computed); any compute call on a machine without
an sm_103a device returns PHX_ENODEV, and a missing library raises at load.

Functions carry the C names (``phx_create``, ``phx_set_pump``, ``phx_step_n``,
``phx_norm_energy``, ``phx_destroy``, ...).  Arrays may be numpy arrays (host)
or torch tensors (host or CUDA); complex arrays are interleaved (re, im).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libphx.so")

PHX_OK = 0
PHX_ENONFINITE = 4
INTEGRATOR_RK4, INTEGRATOR_SPLIT = 0, 1
STATUS = {0: "PHX_OK", 1: "PHX_EINVAL", 2: "PHX_ENOMEM", 3: "PHX_ECUDA",
          4: "PHX_ENONFINITE", 5: "PHX_ETIMEOUT", 6: "PHX_ESTATE",
          7: "PHX_ENODEV"}
BC_PERIODIC = 0
BC_ZERO = 1


class PhxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.message = message


class phx_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("spinor", ctypes.c_int32),
        ("reservoir", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("hbar2_over_2m", ctypes.c_double),
        ("g", ctypes.c_double), ("g_x", ctypes.c_double), ("g_r", ctypes.c_double),
        ("R", ctypes.c_double),
        ("gamma_c", ctypes.c_double), ("gamma_r", ctypes.c_double),
        ("delta_lt", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("noise_var", ctypes.c_double),
        ("wigner_nu", ctypes.c_double),
        ("drive_omega", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("instance", ctypes.c_uint32), ("integrator", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
    ]


class phx_fno_config(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("height", ctypes.c_int32), ("width", ctypes.c_int32),
        ("channels", ctypes.c_int32), ("layers", ctypes.c_int32),
        ("modes_x", ctypes.c_int32), ("modes_y", ctypes.c_int32),
        ("in_channels", ctypes.c_int32), ("out_channels", ctypes.c_int32),
        ("proj_hidden", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


_lib = None

_SIGS = {
    "phx_params_init": (ctypes.c_int, [ctypes.POINTER(phx_params)]),
    "phx_stability_dt": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.POINTER(ctypes.c_double)]),
    "phx_create": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.POINTER(ctypes.c_void_p)]),
    "phx_buffer_sizes": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.POINTER(ctypes.c_size_t)]),
    "phx_create_with_buffers": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.POINTER(ctypes.c_void_p),
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "phx_set_pump": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_set_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_set_drive": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_set_kfilter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64]),
    "phx_step_ssf": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "phx_step_imag": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "phx_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_step_n": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "phx_norm_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "phx_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "phx_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "phx_set_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double]),
    "phx_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "phx_tile": (ctypes.c_int32, [ctypes.c_void_p]),
    "phx_launch_count": (ctypes.c_uint64, []),
    "phx_alu_peak_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "phx_debug_inject": (ctypes.c_int, [ctypes.c_uint32]),
    "phx_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "phx_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "phx_destroy": (None, [ctypes.c_void_p]),
    "phx_noise_sample": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "phx_batch_create": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "phx_batch_set_pump": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int]),
    "phx_batch_set_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int]),
    "phx_batch_set_drive": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int]),
    "phx_batch_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int]),
    "phx_batch_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int]),
    "phx_batch_step_n": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "phx_batch_norm_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "phx_batch_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "phx_batch_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "phx_batch_tile": (ctypes.c_int32, [ctypes.c_void_p]),
    "phx_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "phx_batch_destroy": (None, [ctypes.c_void_p]),
    "phx_norm_energy_static": (ctypes.c_int, [ctypes.POINTER(phx_params), ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "phx_fno_config_init": (ctypes.c_int, [ctypes.POINTER(phx_fno_config)]),
    "phx_fno_create": (ctypes.c_int, [ctypes.POINTER(phx_fno_config), ctypes.POINTER(ctypes.c_void_p)]),
    "phx_fno_num_params": (ctypes.c_int64, [ctypes.c_void_p]),
    "phx_fno_gemm_flops": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "phx_fno_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_fno_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "phx_fno_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "phx_fno_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "phx_fno_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "phx_fno_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "phx_fno_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "phx_fno_targets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "phx_fno_to_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "phx_fno_destroy": (None, [ctypes.c_void_p]),
}


def lib():
    """Load libphx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libphx.so is not built (%s); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, h=None):
    if st != PHX_OK:
        msg = lib().phx_last_error(h).decode(errors="replace")
        raise PhxError(st, msg)


def _ptr(a, dtype_real, expect_complex, expect_elems):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    try:
        import torch
        is_t = isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {(np.float32, False): torch.float32, (np.float64, False): torch.float64,
                (np.float32, True): torch.complex64, (np.float64, True): torch.complex128}
        if a.dtype != want[(dtype_real, expect_complex)]:
            raise TypeError("tensor dtype %s, expected %s" % (a.dtype, want[(dtype_real, expect_complex)]))
        if a.numel() != expect_elems:
            raise ValueError("tensor has %d elements, expected %d" % (a.numel(), expect_elems))
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.asarray(a)
    want = {(np.float32, False): np.float32, (np.float64, False): np.float64,
            (np.float32, True): np.complex64, (np.float64, True): np.complex128}[(dtype_real, expect_complex)]
    if arr.dtype != want or not arr.flags.c_contiguous:
        raise TypeError("array must be C-contiguous %s (got %s)" % (np.dtype(want), arr.dtype))
    if arr.size != expect_elems:
        raise ValueError("array has %d elements, expected %d" % (arr.size, expect_elems))
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


# ---------------------------------------------------------------- C-ABI calls

def phx_params_init(**kw):
    p = phx_params()
    _check(lib().phx_params_init(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "kappa":
            k = "hbar2_over_2m"
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v)
        setattr(p, k, v)
    return p


def phx_stability_dt(p):
    out = ctypes.c_double()
    _check(lib().phx_stability_dt(ctypes.byref(p), ctypes.byref(out)))
    return out.value


class Handle:
    """Owns a phx_handle*; remembers sizes for argument checks."""

    def __init__(self, ptr, p):
        self.ptr = ptr
        self.nx, self.ny = p.nx, p.ny
        self.ncomp = 2 if p.spinor else 1
        self.reservoir = bool(p.reservoir)
        self.real = np.float32 if p.precision == 32 else np.float64

    @property
    def as_parameter(self):
        return self.ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().phx_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def phx_create(p):
    out = ctypes.c_void_p()
    _check(lib().phx_create(ctypes.byref(p), ctypes.byref(out)))
    return Handle(out, p)


def phx_buffer_sizes(p):
    """Bytes of the five state buffers (psi 0/1, n 0/1, P) for params p."""
    out = (ctypes.c_size_t * 5)()
    _check(lib().phx_buffer_sizes(ctypes.byref(p), out))
    return [int(v) for v in out]


def phx_create_with_buffers(p, buffers):
    """Handle on caller-owned device buffers (five CUDA tensors or None for
    the zero-size entries); the tensors must outlive the handle."""
    ptrs = (ctypes.c_void_p * 5)(*[None if b is None else b.data_ptr() for b in buffers])
    out = ctypes.c_void_p()
    _check(lib().phx_create_with_buffers(ctypes.byref(p), ptrs, ctypes.byref(out)))
    h = Handle(out, p)
    h.buffers = list(buffers)  # keep the tensors alive with the handle
    return h


def phx_set_pump(h, P_plus, P_minus=None):
    n = h.nx * h.ny
    a, dev_a, ka = _ptr(P_plus, h.real, False, n)
    b, dev_b, kb = _ptr(P_minus, h.real, False, n)
    if b is not None and dev_a != dev_b:
        raise ValueError("P_plus and P_minus must both be host or both device")
    _check(lib().phx_set_pump(h.ptr, a, b, dev_a), h.ptr)


def phx_set_potential(h, V):
    a, dev, k = _ptr(V, h.real, False, h.nx * h.ny)
    _check(lib().phx_set_potential(h.ptr, a, dev), h.ptr)


def phx_set_drive(h, E_plus, E_minus=None):
    """E_plus None removes the drive; E_minus None drives both components
    with E_plus."""
    n = h.nx * h.ny
    a, dev_a, ka = _ptr(E_plus, h.real, True, n)
    b, dev_b, kb = _ptr(E_minus, h.real, True, n)
    if a is not None and b is not None and dev_a != dev_b:
        raise ValueError("E_plus and E_minus must both be host or both device")
    _check(lib().phx_set_drive(h.ptr, a, b, dev_a if a is not None else 0), h.ptr)


def phx_step_ssf(h, nsteps):
    _check(lib().phx_step_ssf(h.ptr, int(nsteps)), h.ptr)


def phx_step_imag(h, nsteps):
    _check(lib().phx_step_imag(h.ptr, int(nsteps)), h.ptr)


def phx_set_kfilter(h, k_cut, order=1, every=1):
    _check(lib().phx_set_kfilter(h.ptr, float(k_cut), int(order), int(every)), h.ptr)


def phx_set_state(h, psi, n=None):
    m = h.ncomp * h.nx * h.ny
    a, dev_a, ka = _ptr(psi, h.real, True, m)
    b, dev_b, kb = _ptr(n, h.real, False, m)
    if a is not None and b is not None and dev_a != dev_b:
        raise ValueError("psi and n must both be host or both device")
    dev = dev_a if a is not None else dev_b
    _check(lib().phx_set_state(h.ptr, a, b, dev), h.ptr)


def phx_get_state(h, psi_out=None, n_out=None):
    """Fill psi_out / n_out (numpy or torch, preallocated)."""
    m = h.ncomp * h.nx * h.ny
    a, dev_a, ka = _ptr(psi_out, h.real, True, m)
    b, dev_b, kb = _ptr(n_out, h.real, False, m)
    if a is not None and b is not None and dev_a != dev_b:
        raise ValueError("outputs must both be host or both device")
    dev = dev_a if a is not None else dev_b
    _check(lib().phx_get_state(h.ptr, a, b, dev), h.ptr)


def phx_step_n(h, nsteps):
    _check(lib().phx_step_n(h.ptr, int(nsteps)), h.ptr)


def phx_norm_energy(h):
    N, E = ctypes.c_double(), ctypes.c_double()
    _check(lib().phx_norm_energy(h.ptr, ctypes.byref(N), ctypes.byref(E)), h.ptr)
    return N.value, E.value


def phx_residual(h):
    r, rn, om = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().phx_residual(h.ptr, ctypes.byref(r), ctypes.byref(rn), ctypes.byref(om)), h.ptr)
    return r.value, rn.value, om.value


def phx_time(h):
    s, t = ctypes.c_int64(), ctypes.c_double()
    _check(lib().phx_time(h.ptr, ctypes.byref(s), ctypes.byref(t)), h.ptr)
    return s.value, t.value


def phx_set_time(h, step, t):
    _check(lib().phx_set_time(h.ptr, int(step), float(t)), h.ptr)


def phx_set_stream(h, stream):
    _check(lib().phx_set_stream(h.ptr, ctypes.c_void_p(int(stream) if stream else 0)), h.ptr)


def phx_tile(h):
    return int(lib().phx_tile(h.ptr))


def phx_launch_count():
    return int(lib().phx_launch_count())


def phx_alu_peak_probe(precision):
    """Measured FMA throughput (TFLOP/s) of the current device in FP32 or FP64."""
    out = ctypes.c_double()
    _check(lib().phx_alu_peak_probe(int(precision), ctypes.byref(out)))
    return out.value


INJECT_ALLOC, INJECT_LAUNCH, INJECT_TIMEOUT = 1, 2, 4


def phx_debug_inject(mask):
    _check(lib().phx_debug_inject(int(mask)))


def phx_last_error(h=None):
    return lib().phx_last_error(h.ptr if h is not None else None).decode(errors="replace")


def phx_destroy(h):
    if h.ptr:
        lib().phx_destroy(h.ptr)
        h.ptr = None


def phx_noise_sample(seed, step, instance, ncomp, nx, ny, noise_var, out, stream=0):
    """out: float32 CUDA tensor with ncomp*ny*nx*2 elements."""
    if out.numel() != ncomp * nx * ny * 2 or not out.is_cuda:
        raise ValueError("out must be a CUDA float32 tensor of ncomp*ny*nx*2 elements")
    _check(lib().phx_noise_sample(int(seed), int(step), int(instance), int(ncomp), int(nx),
                                  int(ny), float(noise_var), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(int(stream) if stream else 0)))


def phx_norm_energy_static(p, psi, n=None, V=None):
    """Allocation-free norm/energy of caller-owned CUDA tensors (plain layout).
    Raises PhxError with the status code on failure (this call records no
    message)."""
    import torch
    for t in (psi, n, V):
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("inputs must be contiguous CUDA tensors")
    # The C entry point cannot see buffer sizes: check every array against
    # the grid and the precision here, before any kernel reads it.
    ncomp = 2 if p.spinor else 1
    sites = int(p.nx) * int(p.ny)
    cplx = torch.complex64 if p.precision == 32 else torch.complex128
    real = torch.float32 if p.precision == 32 else torch.float64
    if psi.dtype != cplx or psi.numel() != ncomp * sites:
        raise ValueError("psi must be a %s tensor of ncomp*ny*nx = %d elements"
                         % (cplx, ncomp * sites))
    if p.reservoir:
        if n is None or n.dtype != real or n.numel() != ncomp * sites:
            raise ValueError("n must be a %s tensor of ncomp*ny*nx = %d elements"
                             % (real, ncomp * sites))
    else:
        n = None
    if V is not None and (V.dtype != real or V.numel() != sites):
        raise ValueError("V must be a %s tensor of ny*nx = %d elements" % (real, sites))
    N, E = ctypes.c_double(), ctypes.c_double()
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    st = lib().phx_norm_energy_static(ctypes.byref(p), ptr(psi), ptr(n), ptr(V),
                                      ctypes.byref(N), ctypes.byref(E))
    if st != PHX_OK:
        raise PhxError(st, "phx_norm_energy_static failed")
    return N.value, E.value


# ------------------------------------------------------------------ batches

class Batch:
    """Owns a phx_batch*; remembers member sizes for argument checks."""

    def __init__(self, ptr, plist):
        self.ptr = ptr
        self.sizes = [(p.nx, p.ny) for p in plist]
        self.count = len(plist)
        self.reservoir = bool(plist[0].reservoir)

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().phx_batch_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _bcheck(st, b):
    if st != PHX_OK:
        raise PhxError(st, lib().phx_batch_last_error(b.ptr if b is not None else None)
                       .decode(errors="replace"))


def phx_batch_create(params):
    arr = (phx_params * len(params))(*params)
    out = ctypes.c_void_p()
    st = lib().phx_batch_create(arr, len(params), ctypes.byref(out))
    if st != PHX_OK:
        raise PhxError(st, lib().phx_batch_last_error(None).decode(errors="replace"))
    return Batch(out, list(params))


def phx_batch_set_pump(b, i, P):
    nx, ny = b.sizes[i]
    a, dev, k = _ptr(P, np.float32, False, nx * ny)
    _bcheck(lib().phx_batch_set_pump(b.ptr, i, a, dev), b)


def phx_batch_set_potential(b, i, V):
    nx, ny = b.sizes[i]
    a, dev, k = _ptr(V, np.float32, False, nx * ny)
    _bcheck(lib().phx_batch_set_potential(b.ptr, i, a, dev), b)


def phx_batch_set_drive(b, i, E):
    """E None sets member i's drive to zero."""
    nx, ny = b.sizes[i]
    a, dev, k = _ptr(E, np.float32, True, nx * ny)
    _bcheck(lib().phx_batch_set_drive(b.ptr, i, a, dev if a is not None else 0), b)


def phx_batch_set_state(b, i, psi, n=None):
    nx, ny = b.sizes[i]
    a, da, ka = _ptr(psi, np.float32, True, nx * ny)
    c, dc, kc = _ptr(n, np.float32, False, nx * ny)
    dev = da if a is not None else dc
    _bcheck(lib().phx_batch_set_state(b.ptr, i, a, c, dev), b)


def phx_batch_get_state(b, i, psi_out=None, n_out=None):
    nx, ny = b.sizes[i]
    a, da, ka = _ptr(psi_out, np.float32, True, nx * ny)
    c, dc, kc = _ptr(n_out, np.float32, False, nx * ny)
    dev = da if a is not None else dc
    _bcheck(lib().phx_batch_get_state(b.ptr, i, a, c, dev), b)


def phx_batch_step_n(b, nsteps):
    _bcheck(lib().phx_batch_step_n(b.ptr, int(nsteps)), b)


def phx_batch_norm_energy(b, allow_nonfinite=False):
    """Per-member (norms, energies).  allow_nonfinite: a member whose state
    holds NaN or Inf reports non-finite values instead of raising (the C call
    fills every member's values before it returns PHX_ENONFINITE)."""
    N = np.zeros(b.count)
    E = np.zeros(b.count)
    st = lib().phx_batch_norm_energy(b.ptr, N.ctypes.data, E.ctypes.data)
    if not (allow_nonfinite and st == PHX_ENONFINITE):
        _bcheck(st, b)
    return N, E


def phx_batch_residual(b, allow_nonfinite=False):
    """Per-member (r_psi, r_n, omega); allow_nonfinite as for
    phx_batch_norm_energy."""
    r = np.zeros(b.count)
    rn = np.zeros(b.count)
    om = np.zeros(b.count)
    st = lib().phx_batch_residual(b.ptr, r.ctypes.data, rn.ctypes.data, om.ctypes.data)
    if not (allow_nonfinite and st == PHX_ENONFINITE):
        _bcheck(st, b)
    return r, rn, om


def phx_batch_time(b):
    s = ctypes.c_int64()
    t = np.zeros(b.count)
    _bcheck(lib().phx_batch_time(b.ptr, ctypes.byref(s), t.ctypes.data), b)
    return s.value, t


def phx_batch_tile(b):
    return int(lib().phx_batch_tile(b.ptr))


def phx_batch_destroy(b):
    if b.ptr:
        lib().phx_batch_destroy(b.ptr)
        b.ptr = None


# ------------------------------------------------------------- conveniences

PARAM_KEYS = ("nx", "ny", "lx", "ly", "bc_x", "bc_y", "spinor", "reservoir",
              "kappa", "g", "g_x", "g_r", "R", "gamma_c", "gamma_r", "delta_lt",
              "dt", "noise_var", "wigner_nu", "drive_omega", "seed", "instance",
              "integrator")


def params_from_dict(d, precision=32, stream=None, tile=0):
    kw = {k: d[k] for k in PARAM_KEYS if k in d}
    kw["spinor"] = int(bool(kw.get("spinor", 0)))
    kw["reservoir"] = int(bool(kw.get("reservoir", 0)))
    return phx_params_init(precision=precision, stream=stream or 0, tile=tile, **kw)


# -------------------------------------------------------- FNO warm start

FNO_CONFIG_KEYS = ("height", "width", "channels", "layers", "modes_x", "modes_y",
                   "in_channels", "out_channels", "proj_hidden", "max_batch")


class Fno:
    """Owns a phx_fno*; remembers the configuration for argument checks."""

    def __init__(self, ptr, cfg):
        self.ptr = ptr
        self.cfg = {k: int(getattr(cfg, k)) for k in FNO_CONFIG_KEYS}
        self.num_params = int(lib().phx_fno_num_params(ptr))

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                lib().phx_fno_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


def _fcheck(st, f):
    if st != PHX_OK:
        raise PhxError(st, lib().phx_fno_last_error(f.ptr if f is not None else None)
                       .decode(errors="replace"))


def _dev_f32(t, numel, what):
    """Pointer of a contiguous float32 CUDA tensor of `numel` elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % what)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (what, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def phx_fno_create(stream=None, **kw):
    c = phx_fno_config()
    _fcheck(lib().phx_fno_config_init(ctypes.byref(c)), None)
    for k, v in kw.items():
        if k not in FNO_CONFIG_KEYS:
            raise KeyError(k)
        setattr(c, k, int(v))
    c.stream = stream or 0
    out = ctypes.c_void_p()
    _fcheck(lib().phx_fno_create(ctypes.byref(c), ctypes.byref(out)), None)
    return Fno(out, c)


def _fno_io(f, x, batch, channels, what):
    c = f.cfg
    return _dev_f32(x, batch * c["height"] * c["width"] * channels, what)


def phx_fno_set_params(f, w):
    a, dev, keep = _ptr(w, np.float32, False, f.num_params)
    _fcheck(lib().phx_fno_set_params(f.ptr, a, dev), f)


def phx_fno_get_params(f, out=None):
    if out is None:
        out = np.empty(f.num_params, np.float32)
    a, dev, keep = _ptr(out, np.float32, False, f.num_params)
    _fcheck(lib().phx_fno_get_params(f.ptr, a, dev), f)
    return out


def phx_fno_forward(f, x, out):
    """out[B,H,W,Cout] = FNO(x[B,H,W,Cin]); both float32 CUDA tensors."""
    B = x.shape[0]
    _fcheck(lib().phx_fno_forward(f.ptr, _fno_io(f, x, B, f.cfg["in_channels"], "input"),
                                  _fno_io(f, out, B, f.cfg["out_channels"], "output"), B), f)
    return out


def phx_fno_loss_grad(f, x, target, grad=None):
    """Loss (float) and, into `grad` (float32 CUDA tensor), the gradient."""
    B = x.shape[0]
    loss = ctypes.c_double()
    g = _dev_f32(grad, f.num_params, "grad") if grad is not None else None
    _fcheck(lib().phx_fno_loss_grad(f.ptr, _fno_io(f, x, B, f.cfg["in_channels"], "input"),
                                    _fno_io(f, target, B, f.cfg["out_channels"], "target"), B,
                                    ctypes.byref(loss), g), f)
    return loss.value


def phx_fno_train_step(f, x, target, lr):
    B = x.shape[0]
    loss = ctypes.c_double()
    _fcheck(lib().phx_fno_train_step(f.ptr, _fno_io(f, x, B, f.cfg["in_channels"], "input"),
                                     _fno_io(f, target, B, f.cfg["out_channels"], "target"), B,
                                     float(lr), ctypes.byref(loss)), f)
    return loss.value


def phx_fno_gemm_flops(f):
    """Algorithmic GEMM flops (2 M N K per product) issued on f so far."""
    out = ctypes.c_double()
    _fcheck(lib().phx_fno_gemm_flops(f.ptr, ctypes.byref(out)), f)
    return out.value


def phx_fno_destroy(f):
    if f.ptr:
        lib().phx_fno_destroy(f.ptr)
        f.ptr = None


def _cdev(t, dtype, numel, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError("%s must be a contiguous %s CUDA tensor" % (what, dtype))
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (what, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def phx_fno_features(P, lx, ly, p_thr, out, stream=None):
    """P [B,H,W] float32 CUDA -> out [B,H,W,3] float32 CUDA."""
    import torch
    B, H, W = P.shape
    _fcheck(lib().phx_fno_features(_cdev(P, torch.float32, B * H * W, "P"), B, H, W, float(lx),
                                   float(ly), float(p_thr), _cdev(out, torch.float32, 3 * B * H * W, "out"),
                                   _stream_ptr(stream)), None)
    return out


def phx_fno_targets(psi, n, scale_psi, scale_n, out, stream=None):
    """psi [B,H,W] complex64, n [B,H,W] float32 -> out [B,H,W,3] float32."""
    import torch
    B, H, W = psi.shape
    _fcheck(lib().phx_fno_targets(_cdev(psi, torch.complex64, B * H * W, "psi"),
                                  _cdev(n, torch.float32, B * H * W, "n"), B, H, W,
                                  float(scale_psi), float(scale_n),
                                  _cdev(out, torch.float32, 3 * B * H * W, "out"), _stream_ptr(stream)),
            None)
    return out


def phx_fno_to_state(u, scale_psi, scale_n, psi, n=None, stream=None):
    """u [B,H,W,3] float32 -> psi [B,H,W] complex64, n [B,H,W] float32."""
    import torch
    B, H, W, _ = u.shape
    _fcheck(lib().phx_fno_to_state(_cdev(u, torch.float32, 3 * B * H * W, "u"), B, H, W,
                                   float(scale_psi), float(scale_n),
                                   _cdev(psi, torch.complex64, B * H * W, "psi"),
                                   None if n is None else _cdev(n, torch.float32, B * H * W, "n"),
                                   _stream_ptr(stream)), None)
    return psi, n
