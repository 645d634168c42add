"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline leg and its reference arm) may import this module.  The product
library under ``paper_2005_00827_gb300`` never loads it, and the oracle shares
no code with that library.

The C source (``qpfrg_oracle.c``) restates the method of Rohe & Honerkamp,
arXiv:2005.00827 (Sec. 2.1 dispersion; App. A.1-A.3 flow equations and
propagators; Sec. 3.1.1 and Eq. (definition_Z) for Z).  This module only
marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qpfrg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

MODE_WEDGE, MODE_LATTICE, MODE_SHELL = 0, 1, 2
REG_TEMPERATURE, REG_INTERACTION = 0, 1
PROP_PAPER, PROP_QP = 0, 1
CH_PP, CH_CR, CH_D = 1, 2, 4
CH_ALL = 7
STATUS = {0: "REACHED_END", 1: "DIVERGED", 2: "NONFINITE", 3: "Z_OUT_OF_RANGE", 4: "MAX_STEPS"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "qpfrg_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-D_GNU_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("t", C.c_double), ("tp", C.c_double), ("mu", C.c_double),
                ("mode", C.c_int), ("N", C.c_int), ("n_theta", C.c_int), ("n_r", C.c_int),
                ("regulator", C.c_int), ("prop_mode", C.c_int), ("channels", C.c_uint),
                ("T_fixed", C.c_double), ("eta", C.c_double), ("n_shell", C.c_int),
                ("shell_width", C.c_double)]


class FlowOpts(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("lambda_end", C.c_double), ("step", C.c_double),
                ("stop_abs_v", C.c_double), ("z_max", C.c_double), ("z_feedback", C.c_int),
                ("max_steps", C.c_int)]


class FlowResult(C.Structure):
    _fields_ = [("status", C.c_int), ("steps", C.c_int), ("lambda_", C.c_double),
                ("lambda_c", C.c_double), ("max_abs_v", C.c_double)]


class GFlowOpts(C.Structure):
    _fields_ = [("g0", C.c_double), ("g_end", C.c_double), ("dg", C.c_double), ("stop_abs_v", C.c_double),
                ("z_feedback", C.c_int), ("katanin", C.c_int), ("a_mode", C.c_int), ("freeze_vertex", C.c_int),
                ("max_steps", C.c_int), ("n_omega", C.c_int), ("omega", C.POINTER(C.c_double))]


A_AVG, A_MIN, A_MAX, A_DROP = 0, 1, 2, 3

_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_geom_create.argtypes = [C.POINTER(Params), C.POINTER(C.c_void_p)]
        L.orc_geom_free.argtypes = [C.c_void_p]
        L.orc_geom_M.argtypes = [C.c_void_p]
        L.orc_geom_export.argtypes = [C.c_void_p, _D, _D, _D, _I]
        L.orc_proj.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_xi.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
        L.orc_xi.restype = C.c_double
        L.orc_shell_width.argtypes = [C.POINTER(Params)]
        L.orc_shell_width.restype = C.c_double
        for name in ("orc_fermi", "orc_dfermi_dT"):
            getattr(L, name).argtypes = [C.c_double, C.c_double]
            getattr(L, name).restype = C.c_double
        for name in ("orc_D", "orc_dD_dT", "orc_Lph", "orc_Lpp", "orc_dLph_dT", "orc_dLpp_dT"):
            getattr(L, name).argtypes = [C.c_double, C.c_double, C.c_double]
            getattr(L, name).restype = C.c_double
        L.orc_rhs_triple.argtypes = [C.c_void_p, C.c_double, _D, _D, C.c_int, C.c_int, C.c_int, _D]
        L.orc_rhs.argtypes = [C.c_void_p, C.c_double, _D, _D, _D, C.c_int]
        L.orc_sigma.argtypes = [C.c_void_p, C.c_double, _D, _D, C.c_int, C.c_int, _D, _D, _D, C.c_int]
        L.orc_zfactor.argtypes = [C.c_void_p, C.c_double, _D, _D, _D, C.c_int]
        L.orc_zfactor_targets.argtypes = [C.c_void_p, C.c_double, _D, _D, C.c_int, _I, _D, C.c_int]
        L.orc_sigma_gflow.argtypes = [C.c_void_p, C.c_double, _D, _D, _D, C.c_int, C.c_int, _D, _D, _D, C.c_int]
        L.orc_gflow_zka.argtypes = [C.c_void_p, C.POINTER(GFlowOpts), C.c_double, _D, _D, _D, _D, _D, _D]
        L.orc_gflow_rhs.argtypes = [C.c_void_p, C.POINTER(GFlowOpts), C.c_double, _D, _D, _D, _D, _D, _D, _D,
                                    _D, _D, _D, C.c_int]
        L.orc_gflow.argtypes = [C.c_void_p, C.POINTER(GFlowOpts), _D, _D, _D, _D, _D, C.POINTER(FlowResult),
                                C.c_int]
        L.orc_spectral.argtypes = [C.c_void_p, C.c_int, C.c_int, _D, _D, _D, C.c_double, _D, _D]
        L.orc_rk4_step.argtypes = [C.c_void_p, C.c_double, C.c_double, _D, _D, C.c_int]
        L.orc_flow.argtypes = [C.c_void_p, C.POINTER(FlowOpts), _D, _D, C.POINTER(FlowResult), C.c_int]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Oracle:
    """One problem: lattice, patching, regulator, channels, propagator mode."""

    def __init__(self, N, n_theta=8, n_r=8, mode=MODE_WEDGE, t=1.0, tp=0.0, mu=0.0,
                 regulator=REG_TEMPERATURE, prop_mode=PROP_PAPER, channels=CH_ALL,
                 T_fixed=0.1, eta=0.02, nthreads=0, n_shell=1, shell_width=0.0):
        self.P = Params(t, tp, mu, mode, N, n_theta, n_r, regulator, prop_mode, channels,
                        T_fixed, eta, n_shell, shell_width)
        self.N = N
        self.nthreads = nthreads
        h = C.c_void_p()
        rc = lib().orc_geom_create(C.byref(self.P), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle geometry rejected the parameters (rc={rc})")
        self._h = h
        self.M = lib().orc_geom_M(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_geom_free(h)
            self._h = None

    # geometry -------------------------------------------------------------
    def geometry(self):
        kf = np.zeros((self.N, 2)); fk = np.zeros((self.M, 2)); fw = np.zeros(self.M)
        fp = np.zeros(self.M, dtype=np.int32)
        lib().orc_geom_export(self._h, _dp(kf), _dp(fk), _dp(fw), fp.ctypes.data_as(_I))
        return kf, fk, fw, fp

    def proj(self, kx, ky):
        return lib().orc_proj(self._h, float(kx), float(ky))

    def xi(self, kx, ky):
        return lib().orc_xi(C.byref(self.P), float(kx), float(ky))

    def shell_width(self):
        return lib().orc_shell_width(C.byref(self.P))

    # right-hand side --------------------------------------------------------
    def rhs_triple(self, lam, V, Z, i, j, l):
        V = np.ascontiguousarray(V, dtype=np.float64); Z = np.ascontiguousarray(Z, dtype=np.float64)
        out = np.zeros(3)
        lib().orc_rhs_triple(self._h, float(lam), _dp(V), _dp(Z), int(i), int(j), int(l), _dp(out))
        return out

    def rhs(self, lam, V, Z):
        V = np.ascontiguousarray(V, dtype=np.float64); Z = np.ascontiguousarray(Z, dtype=np.float64)
        dV = np.zeros_like(V)
        lib().orc_rhs(self._h, float(lam), _dp(V), _dp(Z), _dp(dV), self.nthreads)
        return dV

    # self-energy --------------------------------------------------------------
    def sigma(self, T, V, Z, j, omega):
        V = np.ascontiguousarray(V, dtype=np.float64); Z = np.ascontiguousarray(Z, dtype=np.float64)
        w = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        re = np.zeros_like(w); im = np.zeros_like(w)
        lib().orc_sigma(self._h, float(T), _dp(V), _dp(Z), int(j), len(w), _dp(w), _dp(re), _dp(im),
                        self.nthreads)
        return re + 1j * im

    def zfactor(self, T, V, Z):
        V = np.ascontiguousarray(V, dtype=np.float64); Z = np.ascontiguousarray(Z, dtype=np.float64)
        Zo = np.zeros(self.N)
        lib().orc_zfactor(self._h, float(T), _dp(V), _dp(Z), _dp(Zo), self.nthreads)
        return Zo

    def zfactor_targets(self, T, V, Z, targets):
        """Z of the listed patches only (same arithmetic as zfactor)."""
        V = np.ascontiguousarray(V, dtype=np.float64); Z = np.ascontiguousarray(Z, dtype=np.float64)
        js = np.ascontiguousarray(targets, dtype=np.int32)
        Zo = np.zeros(len(js))
        lib().orc_zfactor_targets(self._h, float(T), _dp(V), _dp(Z), len(js), js.ctypes.data_as(_I), _dp(Zo),
                                  self.nthreads)
        return Zo

    def spectral(self, j, omega, sigma, Zj):
        """A(k_j, w) and its Fermi-liquid Gaussian approximation from Sigma on the grid."""
        w = np.ascontiguousarray(omega, dtype=np.float64)
        re = np.ascontiguousarray(np.real(sigma), dtype=np.float64)
        im = np.ascontiguousarray(np.imag(sigma), dtype=np.float64)
        A = np.zeros_like(w); Afl = np.zeros_like(w)
        lib().orc_spectral(self._h, int(j), len(w), _dp(w), _dp(re), _dp(im), float(Zj), _dp(A), _dp(Afl))
        return A, Afl

    # interaction flow with the self-energy ODE ----------------------------------
    def _gopts(self, g0=0.0, g_end=1.0, dg=0.05, omega=(), z_feedback=True, katanin=False, a_mode=A_AVG,
               freeze_vertex=False, stop_abs_v=20.0, max_steps=100000):
        w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
        self._gw = w                     # keep the grid alive for the call
        return GFlowOpts(g0, g_end, dg, stop_abs_v, int(z_feedback), int(katanin), int(a_mode),
                         int(freeze_vertex), max_steps, len(w), _dp(w) if len(w) else None)

    def sigma_gflow(self, T, V, Z, K, j, omega):
        V = np.ascontiguousarray(V, dtype=np.float64)
        Z = np.ascontiguousarray(Z, dtype=np.float64); K = np.ascontiguousarray(K, dtype=np.float64)
        w = np.ascontiguousarray(np.atleast_1d(omega), dtype=np.float64)
        re = np.zeros_like(w); im = np.zeros_like(w)
        lib().orc_sigma_gflow(self._h, float(T), _dp(V), _dp(Z), _dp(K), int(j), len(w), _dp(w), _dp(re), _dp(im),
                              self.nthreads)
        return re + 1j * im

    def gflow_zka(self, gv, S, D, **kw):
        """Z, K, A per patch and the A that enters the flow, from the state's
        Sigma and Sigma' (arrays N x (2 + n_omega), chord points first)."""
        o = self._gopts(**kw)
        Sre = np.ascontiguousarray(np.real(S), dtype=np.float64); Dre = np.ascontiguousarray(np.real(D), dtype=np.float64)
        Z, K, A = np.zeros(self.N), np.zeros(self.N), np.zeros(self.N)
        Ab = C.c_double()
        lib().orc_gflow_zka(self._h, C.byref(o), float(gv), _dp(Sre), _dp(Dre), _dp(Z), _dp(K), _dp(A), C.byref(Ab))
        return Z, K, A, Ab.value

    def gflow(self, U, **kw):
        """Interaction flow from g0 with V = U, Sigma = Sigma' = 0: returns the
        final V, Sigma and Sigma' (N x (2 + n_omega), frequencies xi_j + 2T,
        xi_j - 2T, then the grid) and the flow outcome."""
        o = self._gopts(**kw)
        N, nw = self.N, 2 + o.n_omega
        V = np.full((N, N, N), float(U))
        Sre, Sim, Dre, Dim = (np.zeros((N, nw)) for _ in range(4))
        r = FlowResult()
        lib().orc_gflow(self._h, C.byref(o), _dp(V), _dp(Sre), _dp(Sim), _dp(Dre), _dp(Dim), C.byref(r), self.nthreads)
        return dict(status=STATUS[r.status], steps=r.steps, g=r.lambda_, g_c=r.lambda_c, max_abs_v=r.max_abs_v,
                    V=V, S=Sre + 1j * Sim, D=Dre + 1j * Dim)

    # ODE -----------------------------------------------------------------------
    def rk4_step(self, x, h, V, Z):
        V = np.array(V, dtype=np.float64, order="C"); Z = np.ascontiguousarray(Z, dtype=np.float64)
        lib().orc_rk4_step(self._h, float(x), float(h), _dp(V), _dp(Z), self.nthreads)
        return V

    def flow(self, V, Z, lambda0, lambda_end, step, stop_abs_v=20.0, z_feedback=False,
             z_max=2.0, max_steps=100000):
        V = np.array(V, dtype=np.float64, order="C"); Z = np.array(Z, dtype=np.float64, order="C")
        o = FlowOpts(lambda0, lambda_end, step, stop_abs_v, z_max, int(z_feedback), max_steps)
        r = FlowResult()
        lib().orc_flow(self._h, C.byref(o), _dp(V), _dp(Z), C.byref(r), self.nthreads)
        return dict(status=STATUS[r.status], steps=r.steps, lam=r.lambda_, lambda_c=r.lambda_c,
                    max_abs_v=r.max_abs_v, V=V, Z=Z)


def fermi(x, T):
    return lib().orc_fermi(float(x), float(T))


def dfermi_dT(x, T):
    return lib().orc_dfermi_dT(float(x), float(T))


def D(a, b, T):
    return lib().orc_D(float(a), float(b), float(T))


def dD_dT(a, b, T):
    return lib().orc_dD_dT(float(a), float(b), float(T))


def Lph(a, b, T):
    return lib().orc_Lph(float(a), float(b), float(T))


def Lpp(a, b, T):
    return lib().orc_Lpp(float(a), float(b), float(T))


def dLph_dT(a, b, T):
    return lib().orc_dLph_dT(float(a), float(b), float(T))


def dLpp_dT(a, b, T):
    return lib().orc_dLpp_dT(float(a), float(b), float(T))
