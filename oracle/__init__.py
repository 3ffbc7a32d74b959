"""FP64 CPU oracle for the FoE despeckling model solved by iPiano.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package.  It never imports the
CUDA library or its binding, and the CUDA path never imports it.

The arithmetic lives in ``fe_oracle.c`` (plain C, double precision, OpenMP
over image rows); this module compiles it with gcc into ``_build/`` and wraps
it with ctypes.  Every function takes NumPy arrays and promotes them to
float64.  Citations are to the paper's sections and equations:

* ``K``, ``KT``         - K_i u <=> k_i * u and its exact transpose (Sec. II-C),
                          symmetric boundary extension (a stated reading)
* ``F``, ``gradF``      - E_FoE (Eq. FOEmodel) and sum_i theta_i K_i^T rho'(K_i u)
* ``G``                 - (lambda/2) <u^2 - 2 f^2 log u, 1> (Eq. dataterm2)
* ``prox``              - closed-form proximal map (Sec. II-C, variant model)
* ``ipiano``/``ipiano_step`` - the inertial forward-backward iteration
                          (Sec. II-C) with Lipschitz backtracking
* ``Fw``, ``gradFw``, ``Gc``, ``proxc`` - the combined model (Eq. newmodel,
                          Sec. III-A) in w = log u: F(e^w), e^w (.) grad F(e^w),
                          its data term, and the prox by Newton's method;
                          lambda2 = 0 is Eq. original (Sec. II-C)

Parity: every function here is pinned by the ``-m "not gpu"`` tests
(tests/test_oracle_*.py) against closed forms, library routines, dense brute
force and the mathematical identities the paper's definitions imply.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fe_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_REC = 9
REC_FIELDS = ("L", "alpha", "F", "G", "H", "backtracks", "gd", "dd", "dp")


def build(force: bool = False) -> str:
    """Compile fe_oracle.c with gcc (portable flags, no -march) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", "-fvisibility=hidden",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


MODEL_VARIANT, MODEL_COMBINED = 0, 1


class OrcParams(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("beta", C.c_double), ("L0", C.c_double),
                ("eta", C.c_double), ("c2", C.c_double), ("max_backtrack", C.c_int),
                ("max_iter", C.c_int), ("tol", C.c_double), ("model", C.c_int),
                ("lambda1", C.c_double)]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.orc_mirror.restype = C.c_long
            L.orc_mirror.argtypes = [C.c_long, C.c_long]
            L.orc_pad.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D]
            L.orc_pad_adjoint.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D]
            L.orc_conv_valid.argtypes = [_D, C.c_int, C.c_int, _D, C.c_int, _D]
            L.orc_conv_valid_adjoint.argtypes = [_D, C.c_int, C.c_int, _D, C.c_int, _D]
            L.orc_K.argtypes = [_D, C.c_int, C.c_int, _D, C.c_int, _D]
            L.orc_KT.argtypes = [_D, C.c_int, C.c_int, _D, C.c_int, _D]
            L.orc_rho.restype = C.c_double
            L.orc_rho.argtypes = [C.c_double]
            L.orc_drho.restype = C.c_double
            L.orc_drho.argtypes = [C.c_double]
            L.orc_F.restype = C.c_double
            L.orc_F.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int]
            L.orc_G.restype = C.c_double
            L.orc_G.argtypes = [_D, _D, C.c_long, C.c_double]
            L.orc_gradF.restype = C.c_double
            L.orc_gradF.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int, _D]
            L.orc_gradF_at.restype = C.c_double
            L.orc_gradF_at.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int,
                                       C.c_int, C.c_int]
            for n in ("orc_prox", "orc_prox_literal"):
                getattr(L, n).restype = C.c_double
                getattr(L, n).argtypes = [C.c_double] * 4
            L.orc_Fw.restype = C.c_double
            L.orc_Fw.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int]
            L.orc_gradFw.restype = C.c_double
            L.orc_gradFw.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int, _D]
            L.orc_Gc.restype = C.c_double
            L.orc_Gc.argtypes = [_D, _D, C.c_long, C.c_double, C.c_double]
            L.orc_proxc.restype = C.c_double
            L.orc_proxc.argtypes = [C.c_double] * 5
            L.orc_proxc_iters.restype = C.c_double
            L.orc_proxc_iters.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_int)]
            L.orc_ipiano.restype = C.c_int
            L.orc_ipiano.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int,
                                     C.POINTER(OrcParams), _D, _D, _D,
                                     C.POINTER(C.c_int), _D, _D, C.POINTER(C.c_int)]
            L.orc_ipiano_step.restype = C.c_int
            L.orc_ipiano_step.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int,
                                          C.POINTER(OrcParams), _D, _D, C.c_double,
                                          _D, _D, _D]
            L.orc_ipiano_fixed.restype = C.c_int
            L.orc_ipiano_fixed.argtypes = [_D, C.c_int, C.c_int, _D, _D, C.c_int, C.c_int,
                                           C.POINTER(OrcParams), _D, C.c_int, _D, _D, _D]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _d(a):
    """float64 C-contiguous copy/view of a."""
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(_D)


def _bank(filters, theta):
    k = _d(filters)
    if k.ndim == 2:
        k = k[None]
    nf, ks, ks2 = k.shape
    assert ks == ks2 and ks % 2 == 1
    th = _d(theta).reshape(nf)
    return k, th, nf, ks


def mirror(j: int, n: int) -> int:
    return int(lib().orc_mirror(int(j), int(n)))


def pad(u, p: int):
    u = _d(u)
    H, W = u.shape
    out = np.empty((H + 2 * p, W + 2 * p))
    lib().orc_pad(_p(u), H, W, p, _p(out))
    return out


def pad_adjoint(up, H: int, W: int, p: int):
    up = _d(up)
    out = np.empty((H, W))
    lib().orc_pad_adjoint(_p(up), H, W, p, _p(out))
    return out


def conv_valid(up, k):
    up, k = _d(up), _d(k)
    Hp, Wp = up.shape
    ks = k.shape[0]
    out = np.empty((Hp - ks + 1, Wp - ks + 1))
    lib().orc_conv_valid(_p(up), Hp, Wp, _p(k), ks, _p(out))
    return out


def conv_valid_adjoint(r, k):
    r, k = _d(r), _d(k)
    Ho, Wo = r.shape
    ks = k.shape[0]
    out = np.empty((Ho + ks - 1, Wo + ks - 1))
    lib().orc_conv_valid_adjoint(_p(r), Ho, Wo, _p(k), ks, _p(out))
    return out


def K(u, k):
    """K u = k * u with symmetric boundary (one filter k[ks, ks])."""
    u, k = _d(u), _d(k)
    H, W = u.shape
    out = np.empty((H, W))
    lib().orc_K(_p(u), H, W, _p(k), k.shape[0], _p(out))
    return out


def KT(r, k):
    """Exact transpose K^T r."""
    r, k = _d(r), _d(k)
    H, W = r.shape
    out = np.empty((H, W))
    lib().orc_KT(_p(r), H, W, _p(k), k.shape[0], _p(out))
    return out


def rho(x):
    return lib().orc_rho(float(x))


def drho(x):
    return lib().orc_drho(float(x))


def F(u, filters, theta):
    u = _d(u)
    k, th, nf, ks = _bank(filters, theta)
    H, W = u.shape
    return lib().orc_F(_p(u), H, W, _p(k), _p(th), nf, ks)


def G(u, f, lam: float):
    u, f = _d(u), _d(f)
    return lib().orc_G(_p(u), _p(f), u.size, float(lam))


def gradF(u, filters, theta):
    """Returns (grad F(u), F(u))."""
    u = _d(u)
    k, th, nf, ks = _bank(filters, theta)
    H, W = u.shape
    g = np.empty((H, W))
    Fv = lib().orc_gradF(_p(u), H, W, _p(k), _p(th), nf, ks, _p(g))
    return g, Fv


def gradF_at(u, filters, theta, points):
    """grad F(u) evaluated only at the given (y, x) pixels."""
    u = _d(u)
    k, th, nf, ks = _bank(filters, theta)
    H, W = u.shape
    L = lib()
    return np.array([L.orc_gradF_at(_p(u), H, W, _p(k), _p(th), nf, ks, int(y), int(x))
                     for (y, x) in points])


def prox(uhat, f, tau, lam, literal: bool = False):
    fn = lib().orc_prox_literal if literal else lib().orc_prox
    return fn(float(uhat), float(f), float(tau), float(lam))


def prox_array(uhat, f, tau, lam):
    uhat, f = _d(uhat), _d(f)
    fn = lib().orc_prox
    return np.array([fn(a, b, float(tau), float(lam))
                     for a, b in zip(uhat.ravel(), f.ravel())]).reshape(uhat.shape)


def Fw(w, filters, theta):
    """F(e^w) of the combined model."""
    w = _d(w)
    k, th, nf, ks = _bank(filters, theta)
    H, W = w.shape
    return lib().orc_Fw(_p(w), H, W, _p(k), _p(th), nf, ks)


def gradFw(w, filters, theta):
    """Returns (grad_w F(e^w) = e^w (.) grad F(e^w), F(e^w))."""
    w = _d(w)
    k, th, nf, ks = _bank(filters, theta)
    H, W = w.shape
    g = np.empty((H, W))
    Fv = lib().orc_gradFw(_p(w), H, W, _p(k), _p(th), nf, ks, _p(g))
    return g, Fv


def Gc(w, f, lam1: float, lam2: float):
    """sum_p lam1/2 (2w + f^2 e^{-2w}) + lam2/2 (e^{2w} - 2 f^2 w)."""
    w, f = _d(w), _d(f)
    return lib().orc_Gc(_p(w), _p(f), w.size, float(lam1), float(lam2))


def proxc(what, f, tau, lam1, lam2):
    """Prox of tau*G of the combined model at one pixel (Newton's method)."""
    return lib().orc_proxc(float(what), float(f), float(tau), float(lam1), float(lam2))


def proxc_iters(what, f, tau, lam1, lam2):
    """proxc and the number of Newton (or bisection) steps it took."""
    n = C.c_int(0)
    w = lib().orc_proxc_iters(float(what), float(f), float(tau), float(lam1), float(lam2), C.byref(n))
    return w, n.value


def params(lam=5.0, beta=0.8, L0=1.0, eta=2.0, c2=1e-6, max_backtrack=30,
           max_iter=100, tol=0.0, model=MODEL_VARIANT, lam1=0.0) -> OrcParams:
    """iPiano parameters.  model = MODEL_COMBINED: the iterate is w = log u,
    lam weights the variant term (lambda_2) and lam1 the log-domain term
    (lambda_1) of Eq. newmodel."""
    return OrcParams(float(lam), float(beta), float(L0), float(eta), float(c2),
                     int(max_backtrack), int(max_iter), float(tol), int(model), float(lam1))


def ipiano(f, filters, theta, prm: OrcParams, u0=None, L_start=None):
    """Full iPiano solve.  Returns dict with u, u_prev, rec (n x 9),
    n, L, status, F0, G0, converged.  For the combined model the iterate
    (u, u_prev, u0) is w = log u and the default start is log f."""
    f = _d(f)
    k, th, nf, ks = _bank(filters, theta)
    H, W = f.shape
    if u0 is None:
        u0 = np.log(f) if prm.model == MODEL_COMBINED else f
    u = _d(u0).copy()
    up = np.empty_like(u)
    rec = np.zeros((max(prm.max_iter, 1), ORC_REC))
    n = C.c_int(0)
    conv = C.c_int(0)
    Lio = np.array([float(L_start) if L_start else 0.0])
    h0 = np.zeros(2)
    st = lib().orc_ipiano(_p(f), H, W, _p(k), _p(th), nf, ks, C.byref(prm), _p(u), _p(up),
                          _p(rec), C.byref(n), _p(Lio), _p(h0), C.byref(conv))
    return dict(u=u, u_prev=up, rec=rec[:n.value], n=n.value, L=float(Lio[0]),
                status=int(st), F0=float(h0[0]), G0=float(h0[1]),
                converged=bool(conv.value))


def ipiano_step(f, filters, theta, prm: OrcParams, u, u_prev, L_in):
    """One iteration from (u^n, u^{n-1}) with starting estimate L_in.
    Returns dict with u1, rec (9,), L, status."""
    f = _d(f)
    k, th, nf, ks = _bank(filters, theta)
    H, W = f.shape
    u, up = _d(u), _d(u_prev)
    u1 = np.empty_like(u)
    rec = np.zeros(ORC_REC)
    Lout = np.zeros(1)
    st = lib().orc_ipiano_step(_p(f), H, W, _p(k), _p(th), nf, ks, C.byref(prm),
                               _p(u), _p(up), float(L_in), _p(u1), _p(rec), _p(Lout))
    return dict(u1=u1, rec=rec, L=float(Lout[0]), status=int(st))


def ipiano_fixed(f, filters, theta, prm: OrcParams, Lseq, u, u_prev=None):
    """Iterations with the prescribed L_k (no backtracking test).  Returns
    dict with u, u_prev, rec (n x 9, rec[:, 5] = descent-test margin), status."""
    f = _d(f)
    k, th, nf, ks = _bank(filters, theta)
    H, W = f.shape
    Ls = _d(np.atleast_1d(Lseq))
    n = Ls.size
    u = _d(u).copy()
    up = _d(u if u_prev is None else u_prev).copy()
    rec = np.zeros((max(n, 1), ORC_REC))
    st = lib().orc_ipiano_fixed(_p(f), H, W, _p(k), _p(th), nf, ks, C.byref(prm), _p(Ls), n,
                                _p(u), _p(up), _p(rec))
    return dict(u=u, u_prev=up, rec=rec[:n], status=int(st))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))
