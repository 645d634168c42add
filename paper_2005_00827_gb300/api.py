"""Thin ctypes binding of the qpfrg C ABI (include/qpfrg.h), same call names.

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Device buffers are passed as raw pointers (``tensor.data_ptr()``)
and the CUDA stream as ``torch.cuda.current_stream().cuda_stream``; PyTorch
is used for device memory and streams, nothing else.  Loading fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

QPFRG_OK, QPFRG_ERR_INVALID, QPFRG_ERR_CUDA, QPFRG_ERR_OOM = 0, -1, -2, -3
QPFRG_ERR_UNSUPPORTED, QPFRG_ERR_TIMEOUT, QPFRG_ERR_NONFINITE = -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "ERR_INVALID", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_UNSUPPORTED",
                -5: "ERR_TIMEOUT", -6: "ERR_NONFINITE"}
QPFRG_REG_TEMPERATURE, QPFRG_REG_INTERACTION = 0, 1
QPFRG_FP64, QPFRG_MIXED, QPFRG_MIXED_TC = 0, 1, 2
QPFRG_PROP_PAPER, QPFRG_PROP_QP = 0, 1
QPFRG_CH_PP, QPFRG_CH_CR, QPFRG_CH_D, QPFRG_CH_ALL = 1, 2, 4, 7
QPFRG_GRID_WEDGE, QPFRG_GRID_LATTICE, QPFRG_GRID_SHELL = 0, 1, 2
FLOW_STATUS = {0: "RUNNING", 1: "REACHED_END", 2: "DIVERGED", 3: "NONFINITE", 4: "Z_OUT_OF_RANGE",
               5: "MAX_STEPS", 6: "TIMEOUT"}

# Every entry point declared in include/qpfrg.h.
EXPORTS = (
    "qpfrg_default_options", "qpfrg_create", "qpfrg_rhs", "qpfrg_selfenergy", "qpfrg_step",
    "qpfrg_flow", "qpfrg_state_size", "qpfrg_get_state", "qpfrg_set_state", "qpfrg_read_state",
    "qpfrg_geometry", "qpfrg_set_profiling", "qpfrg_profile_reset", "qpfrg_profile_count",
    "qpfrg_profile_name", "qpfrg_profile_get", "qpfrg_last_error", "qpfrg_version", "qpfrg_destroy",
    "qpfrg_zfactor_static", "qpfrg_flow_batch", "qpfrg_autotune", "qpfrg_set_tuning", "qpfrg_rhs_work",
    "qpfrg_spectral", "qpfrg_read_sigma_flow", "qpfrg_sigma_table", "qpfrg_alu_rates",
)


class QpfrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class qpfrg_lattice(C.Structure):
    _fields_ = [("t", C.c_double), ("tp", C.c_double), ("mu", C.c_double)]


class qpfrg_fine_grid(C.Structure):
    _fields_ = [("n_theta", C.c_int), ("n_r", C.c_int), ("mode", C.c_int), ("n_shell", C.c_int),
                ("shell_width", C.c_double)]


class qpfrg_options(C.Structure):
    _fields_ = [("channel_mask", C.c_uint), ("z_feedback", C.c_int), ("propagator", C.c_int),
                ("precision", C.c_int), ("eta", C.c_double), ("n_omega", C.c_int),
                ("omega_min", C.c_double), ("omega_max", C.c_double), ("stop_abs_v", C.c_double),
                ("step", C.c_double), ("lambda_end", C.c_double), ("z_max", C.c_double),
                ("max_steps", C.c_int), ("T_fixed", C.c_double), ("timeout_s", C.c_double),
                ("autotune", C.c_int), ("no_loop_symmetry", C.c_int), ("sigma_ode", C.c_int),
                ("katanin", C.c_int), ("a_mode", C.c_int), ("sigma_table", C.c_int)]


class qpfrg_tuning(C.Structure):
    _fields_ = [("bubble_qchunk", C.c_int), ("sigma_qblocks", C.c_int), ("tc_splits", C.c_int * 3),
                ("ms_bubble", C.c_double), ("ms_sigma", C.c_double), ("ms_contract", C.c_double),
                ("bubble_transfers", C.c_int)]

    def as_dict(self):
        return dict(bubble_qchunk=self.bubble_qchunk, sigma_qblocks=self.sigma_qblocks,
                    tc_splits=list(self.tc_splits), ms_bubble=self.ms_bubble, ms_sigma=self.ms_sigma,
                    ms_contract=self.ms_contract, bubble_transfers=self.bubble_transfers)


class qpfrg_flow_result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps", C.c_int), ("lambda_", C.c_double),
                ("lambda_c", C.c_double), ("max_abs_v", C.c_double)]

    def as_dict(self):
        return dict(status=FLOW_STATUS.get(self.status, self.status), steps=self.steps, lam=self.lambda_,
                    lambda_c=self.lambda_c, max_abs_v=self.max_abs_v)


class qpfrg_flow_spec(C.Structure):
    _fields_ = [("n_p", C.c_int), ("U", C.c_double), ("lambda0", C.c_double), ("lambda_end", C.c_double)]


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libqpfrg.so (building it in-tree when missing); raise when absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"qpfrg CUDA library not built: {path}")
        _build.build()
    L = C.CDLL(path)
    L.qpfrg_default_options.argtypes = [C.POINTER(qpfrg_options)]
    L.qpfrg_default_options.restype = None
    L.qpfrg_create.argtypes = [C.POINTER(qpfrg_lattice), C.c_int, C.POINTER(qpfrg_fine_grid), C.c_double,
                               C.c_double, C.c_int, C.POINTER(qpfrg_options), _P, C.POINTER(_P)]
    L.qpfrg_rhs.argtypes = [_P, C.c_double, _P, _P, _P]
    L.qpfrg_selfenergy.argtypes = [_P, C.c_double, _P, _P, _P, _P, _P]
    L.qpfrg_step.argtypes = [_P, C.c_int, C.POINTER(qpfrg_flow_result)]
    L.qpfrg_flow.argtypes = [_P, C.POINTER(qpfrg_flow_result)]
    L.qpfrg_state_size.argtypes = [_P, C.POINTER(C.c_size_t)]
    L.qpfrg_get_state.argtypes = [_P, _P, C.c_size_t]
    L.qpfrg_set_state.argtypes = [_P, _P, C.c_size_t]
    L.qpfrg_read_state.argtypes = [_P, _P, _P]
    L.qpfrg_geometry.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _D, _D]
    L.qpfrg_set_profiling.argtypes = [_P, C.c_int]
    L.qpfrg_profile_reset.argtypes = [_P]
    L.qpfrg_profile_count.argtypes = []
    L.qpfrg_profile_name.argtypes = [C.c_int]
    L.qpfrg_profile_name.restype = C.c_char_p
    L.qpfrg_profile_get.argtypes = [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
    L.qpfrg_autotune.argtypes = [_P, C.c_double, C.POINTER(qpfrg_tuning)]
    L.qpfrg_set_tuning.argtypes = [_P, C.POINTER(qpfrg_tuning)]
    L.qpfrg_last_error.argtypes = [_P]
    L.qpfrg_last_error.restype = C.c_char_p
    L.qpfrg_version.restype = C.c_char_p
    L.qpfrg_alu_rates.argtypes = [C.POINTER(C.c_double)] * 3
    L.qpfrg_alu_rates.restype = C.c_int
    L.qpfrg_zfactor_static.argtypes = [C.POINTER(qpfrg_lattice), C.c_int, C.c_int, C.c_int, C.c_int, _P, _P,
                                       _P, _P, C.c_double, C.c_double, _P, _P]
    L.qpfrg_zfactor_static.restype = C.c_int
    L.qpfrg_flow_batch.argtypes = [C.POINTER(qpfrg_lattice), C.POINTER(qpfrg_fine_grid), C.c_int,
                                   C.POINTER(qpfrg_options), C.c_int, C.POINTER(qpfrg_flow_spec), _P,
                                   C.POINTER(qpfrg_flow_result)]
    L.qpfrg_flow_batch.restype = C.c_int
    L.qpfrg_read_sigma_flow.argtypes = [_P, _P, _P, _P]
    L.qpfrg_read_sigma_flow.restype = C.c_int
    L.qpfrg_spectral.argtypes = [_P, _P, _P, _P, _P, _P]
    L.qpfrg_spectral.restype = C.c_int
    L.qpfrg_rhs_work.argtypes = [_P] + [C.POINTER(C.c_longlong)] * 4
    L.qpfrg_sigma_table.argtypes = [_P, C.POINTER(C.c_size_t), C.c_longlong, C.c_longlong, _P]
    L.qpfrg_sigma_table.restype = C.c_int
    L.qpfrg_rhs_work.restype = C.c_int
    L.qpfrg_destroy.argtypes = [_P]
    L.qpfrg_destroy.restype = None
    for name in ("qpfrg_create", "qpfrg_rhs", "qpfrg_selfenergy", "qpfrg_step", "qpfrg_flow",
                 "qpfrg_state_size", "qpfrg_get_state", "qpfrg_set_state", "qpfrg_read_state",
                 "qpfrg_geometry", "qpfrg_set_profiling", "qpfrg_profile_reset", "qpfrg_profile_get",
                 "qpfrg_autotune", "qpfrg_set_tuning"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(ctx, status):
    if status != QPFRG_OK:
        msg = load().qpfrg_last_error(ctx).decode(errors="replace") if ctx else ""
        raise QpfrgError(status, msg)


def _ptr(x):
    """Raw pointer of a torch tensor (or an int address, or None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


# --- same-name wrappers ------------------------------------------------------
def qpfrg_default_options() -> qpfrg_options:
    o = qpfrg_options()
    load().qpfrg_default_options(C.byref(o))
    return o


def qpfrg_create(lattice, n_p, grid, U, lambda0, regulator, options, cuda_stream):
    h = _P()
    st = load().qpfrg_create(C.byref(lattice), int(n_p), C.byref(grid), float(U), float(lambda0),
                             int(regulator), C.byref(options) if options is not None else None,
                             _P(cuda_stream) if cuda_stream else None, C.byref(h))
    if st != QPFRG_OK:
        raise QpfrgError(st, "qpfrg_create failed (details on stderr)")
    return h


def qpfrg_rhs(ctx, lam, V, Z, dV):
    _check(ctx, load().qpfrg_rhs(ctx, float(lam), _ptr(V), _ptr(Z), _ptr(dV)))


def qpfrg_selfenergy(ctx, lam, V, Z, sigma_re, sigma_im, Z_out):
    _check(ctx, load().qpfrg_selfenergy(ctx, float(lam), _ptr(V), _ptr(Z), _ptr(sigma_re), _ptr(sigma_im),
                                        _ptr(Z_out)))


def qpfrg_step(ctx, n_steps):
    r = qpfrg_flow_result()
    _check(ctx, load().qpfrg_step(ctx, int(n_steps), C.byref(r)))
    return r


def qpfrg_flow(ctx):
    r = qpfrg_flow_result()
    _check(ctx, load().qpfrg_flow(ctx, C.byref(r)))
    return r


def qpfrg_flow_batch(lattice, grid, regulator, options, specs, cuda_stream):
    """Run the flows of `specs` (sequence of (n_p, U, lambda0, lambda_end)) in one call."""
    n = len(specs)
    arr = (qpfrg_flow_spec * n)(*[qpfrg_flow_spec(int(a), float(b), float(c), float(d)) for a, b, c, d in specs])
    res = (qpfrg_flow_result * n)()
    st = load().qpfrg_flow_batch(C.byref(lattice), C.byref(grid), int(regulator),
                                 C.byref(options) if options is not None else None, n, arr,
                                 _P(cuda_stream) if cuda_stream else None, res)
    if st != QPFRG_OK:
        raise QpfrgError(st, "qpfrg_flow_batch failed")
    return [r.as_dict() for r in res]


def qpfrg_state_size(ctx) -> int:
    n = C.c_size_t()
    _check(ctx, load().qpfrg_state_size(ctx, C.byref(n)))
    return n.value


def qpfrg_get_state(ctx) -> bytes:
    n = qpfrg_state_size(ctx)
    buf = C.create_string_buffer(n)
    _check(ctx, load().qpfrg_get_state(ctx, buf, n))
    return buf.raw


def qpfrg_set_state(ctx, image: bytes):
    buf = C.create_string_buffer(bytes(image), len(image))
    _check(ctx, load().qpfrg_set_state(ctx, buf, len(image)))


def qpfrg_get_state_into(ctx, buf):
    """qpfrg_get_state into a caller-owned host buffer (e.g. a pinned uint8
    tensor of qpfrg_state_size bytes): no allocation or copy on the Python side."""
    _check(ctx, load().qpfrg_get_state(ctx, C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()))


def qpfrg_set_state_from(ctx, buf):
    """qpfrg_set_state from a caller-owned host buffer (e.g. a pinned uint8 tensor)."""
    _check(ctx, load().qpfrg_set_state(ctx, C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size()))


def qpfrg_read_state(ctx, V, Z):
    _check(ctx, load().qpfrg_read_state(ctx, _ptr(V), _ptr(Z)))


def qpfrg_geometry(ctx):
    import numpy as np
    n, m = C.c_int(), C.c_int()
    _check(ctx, load().qpfrg_geometry(ctx, C.byref(n), C.byref(m), None, None))
    kf = np.zeros((n.value, 2))
    fine = np.zeros((m.value, 4))
    _check(ctx, load().qpfrg_geometry(ctx, None, None, kf.ctypes.data_as(_D), fine.ctypes.data_as(_D)))
    return kf, fine


def qpfrg_set_profiling(ctx, on: bool):
    _check(ctx, load().qpfrg_set_profiling(ctx, int(bool(on))))


def qpfrg_profile_reset(ctx):
    _check(ctx, load().qpfrg_profile_reset(ctx))


def qpfrg_autotune(ctx, lam: float) -> dict:
    """Measure and keep the fastest launch shapes at Lambda = lam."""
    t = qpfrg_tuning()
    _check(ctx, load().qpfrg_autotune(ctx, float(lam), C.byref(t)))
    return t.as_dict()


def qpfrg_set_tuning(ctx, bubble_qchunk=0, sigma_qblocks=0, tc_splits=(0, 0, 0), bubble_transfers=0):
    t = qpfrg_tuning()
    t.bubble_qchunk, t.sigma_qblocks = int(bubble_qchunk), int(sigma_qblocks)
    t.bubble_transfers = int(bubble_transfers)
    for i in range(3):
        t.tc_splits[i] = int(tc_splits[i])
    _check(ctx, load().qpfrg_set_tuning(ctx, C.byref(t)))


def qpfrg_profile(ctx) -> dict:
    """{kernel name: (total ms, launches)} from the library's CUDA events."""
    L = load()
    out = {}
    for i in range(L.qpfrg_profile_count()):
        ms, n = C.c_double(), C.c_longlong()
        _check(ctx, L.qpfrg_profile_get(ctx, i, C.byref(ms), C.byref(n)))
        out[L.qpfrg_profile_name(i).decode()] = (ms.value, n.value)
    return out


def qpfrg_zfactor_static(lattice, n_p, n_fine, grid_mode, propagator, fine, kf, V, Z, T, eta, cuda_stream,
                         Z_out):
    """Z_j without any device allocation (static scratch); see include/qpfrg.h."""
    st = load().qpfrg_zfactor_static(C.byref(lattice), int(n_p), int(n_fine), int(grid_mode), int(propagator),
                                     _ptr(fine), _ptr(kf), _ptr(V), _ptr(Z), float(T), float(eta),
                                     _P(cuda_stream) if cuda_stream else None, _ptr(Z_out))
    if st != QPFRG_OK:
        raise QpfrgError(st, "qpfrg_zfactor_static failed")


def qpfrg_spectral(ctx, sigma_re, sigma_im, Z, A, A_fl):
    _check(ctx, load().qpfrg_spectral(ctx, _ptr(sigma_re), _ptr(sigma_im), _ptr(Z), _ptr(A), _ptr(A_fl)))


def qpfrg_read_sigma_flow(ctx, slopes, sigma, zka):
    _check(ctx, load().qpfrg_read_sigma_flow(ctx, _ptr(slopes), _ptr(sigma), _ptr(zka)))


def qpfrg_rhs_work(ctx) -> dict:
    """Loop-kernel evaluations of the last RHS (C4v-reduced) and of the full
    one, the rows evaluated by themselves because their partner maps broke
    covariance, and the rows of each channel GEMM (N^2, or the row orbits)."""
    a, b, r, m = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check(ctx, load().qpfrg_rhs_work(ctx, C.byref(a), C.byref(b), C.byref(r), C.byref(m)))
    return dict(loop_evals=a.value, loop_evals_full=b.value, rows_unreduced=r.value, contraction_rows=m.value)


def qpfrg_sigma_table(ctx, offset=0, count=0):
    """Size of the self-energy's patch-of-r table (0 while not built) and, for
    count > 0, the bytes [offset, offset + count) as a numpy uint8 array."""
    import numpy as np
    n = C.c_size_t()
    _check(ctx, load().qpfrg_sigma_table(ctx, C.byref(n), 0, 0, None))
    if count <= 0:
        return n.value, None
    out = np.zeros(count, dtype=np.uint8)
    _check(ctx, load().qpfrg_sigma_table(ctx, None, int(offset), int(count), out.ctypes.data_as(_P)))
    return n.value, out


def qpfrg_last_error(ctx) -> str:
    return load().qpfrg_last_error(ctx).decode(errors="replace")


def qpfrg_version() -> str:
    return load().qpfrg_version().decode()


def qpfrg_alu_rates() -> dict:
    """Measured ex2.approx, rcp.approx and FP32 FMA results per SM per clock
    of the current device."""
    e, r, f = C.c_double(), C.c_double(), C.c_double()
    st = load().qpfrg_alu_rates(C.byref(e), C.byref(r), C.byref(f))
    if st != 0:
        raise QpfrgError(st, "qpfrg_alu_rates failed")
    return dict(ex2=e.value, rcp=r.value, ffma=f.value)


def qpfrg_destroy(ctx):
    if ctx:
        load().qpfrg_destroy(ctx)


class Context:
    """Convenience owner of a qpfrg context (destroys it on close)."""

    def __init__(self, N, n_theta=8, n_r=8, U=2.0, lambda0=1.0, mode=QPFRG_GRID_WEDGE, t=1.0, tp=0.0,
                 mu=0.0, regulator=QPFRG_REG_TEMPERATURE, stream=None, n_shell=1, shell_width=0.0, **opts):
        o = qpfrg_default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.N = N
        self.options = o
        grid = qpfrg_fine_grid(n_theta, n_r, mode, n_shell, shell_width)
        self.h = qpfrg_create(qpfrg_lattice(t, tp, mu), N, grid, U, lambda0, regulator, o, stream)

    def close(self):
        if self.h:
            qpfrg_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
